// common.cuh -- device-side types and helpers of the sm_103a gradient-SAT path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "turbosat.h"

namespace tsat {

constexpr int kBlock = 256;              // threads per block of the step kernels
constexpr int kWarps = kBlock / 32;
constexpr uint32_t kTagInit = 0x494E4954u;  // Philox counter word 3 for the init draw
constexpr uint32_t kTagBin = 0x42494E41u;   // Philox counter word 3 for sampled binarisation
// 16-bit half h (0..3) of two Philox output words (w0, w1): low half first
__device__ __forceinline__ uint32_t half16(uint32_t w0, uint32_t w1, int h) {
  const uint32_t x = (h & 2) ? w1 : w0;
  return (h & 1) ? (x >> 16) : (x & 0xFFFFu);
}

struct InstInfo {
  int32_t v_off, n_vars, c_off, n_clauses;
  int32_t lmax, item_off, n_items;
  int32_t gid;   // the instance's id for its random streams (default: its index in the loaded batch)
};

// Problem view passed by value to kernels.
struct ProbDev {
  int32_t n_inst, V, C, lmax;
  int64_t nnz;
  int32_t n_items;
  int32_t rec_stride;      // 4: {hdr, lit, lit, 0} per occurrence (lmax <= 3); 8: {hdr, lit x 6, 0} (lmax <= 7);
                           // 0: variable length; fixed records sit at xptr[v] = stride * vptr[v]
  const int32_t *cptr;     // [C+1] clause offsets into clit
  const int32_t *clit;     // [nnz] (global var << 1) | negated
  const int64_t *xptr;     // [V+1] offsets (int32 words) into xrec, multiples of 4
  const int32_t *xrec;     // variable-major occurrence records
  const int32_t *vptr;     // [V+1] occurrence offsets (variable-major)
  const int32_t *vocc;     // [nnz] (clause << 1) | negated, same order as the records
  const int32_t *var_inst; // [V]
  const int4 *items;       // [n_items] {inst, clause begin, clause end, 0}
  const InstInfo *inst;    // [n_inst]
  const int4 *crec;        // [C] clause records {var0, var1, var2, flags} when every clause has <= 3
                           // literals, else NULL; flags byte u = 0xFF if literal u is negated, byte 3 =
                           // clause length; a missing literal repeats var0 (the kernels mask it)
  int32_t full3;           // every clause has exactly 3 literals
  int32_t pad_;
};

// Device header of a state buffer.
struct StateHdr {
  int64_t t;          // next step index
  int32_t all_done;   // every instance frozen and stop requested
  int32_t err;
  int32_t n_active;   // instances still being optimised
  int32_t blocks_done;   // persistent solver: blocks finished in the current launch (the last resets it)
  int32_t pad[10];
};

struct InstState {
  int32_t found, found_sample, min_unsat, best_sample;
  int64_t found_step;
  float loss, pad;
};

// Per-step scalars written by the gamma kernel for the update kernel.
struct StepParams {
  int64_t t;          // step being executed
  int32_t src;        // bits buffer read this step (t & 1)
  int32_t mix_now;    // this step mixes assignments instead of the gradient update
  float lr, step_size, inv_sqrt_bc2, decay;
};

struct StateDev {
  int32_t N, W, lm1, layer;    // samples, words per row, histogram width, layer
  int32_t sample_base;         // global index of this state's first sample (sample-sharded states; else 0)
  int32_t n_total;             // samples of the whole problem over all shards (= N when not sharded)
  StateHdr *hdr;
  InstState *inst;
  StepParams *sp;
  float *z, *m, *v;            // [V][N]
  uint32_t *bits;              // [2][V][W]
  float *nu;                   // [V]
  int32_t *hist;               // [n_inst][lm1][N]
  float *gamma;                // [n_inst][lm1][N]
  float *gdelta;               // [n_inst][4][N] gamma0, g1-g0, g2-g0, g3-g2-g1+g0 (lmax <= 3)
  float *S;                    // [n_inst][N]
  int32_t *unsat;              // [n_inst][N]
  float *zy;                   // relaxed: [n_items][2][N] partial (Z, Y) sums
  float *zs;                   // relaxed: [n_inst][2][N] (Z, S)
  float *rbuf;                 // relaxed: [C][N] clause sums R
  uint32_t *dr16;              // relaxed, BF16 storage: [C][N] dL/dR as bf16 (pairs of samples per word), else NULL
  void *lit;                   // relaxed: [V][N] literal values (f32 or bf16)
  int32_t lit_bf16, pad;
  int64_t V;
};

// Hyper-parameters in the form the kernels use.
struct Hyper {
  float tau, beta1, beta2, eps;
  float omb1, omb2;            // 1 - beta1, 1 - beta2 formed in double on the host
  float bin_c;                 // 0.25 / T
  int32_t norm, binarize;
  uint32_t key0, key1;
  int32_t stop_on_sat;
};

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: ten rounds of two 32x32->64 products with a Weyl key
// schedule; implemented here from the published description.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint32_t lo0 = 0xD2511F53u * c.x;
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    uint32_t lo1 = 0xCD9E8D57u * c.z;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Philox stream of one variable row: the counter's row word is the
// instance-local variable index and the key's low word is offset by the
// instance's id, so an instance's random draws (init and sampled
// binarisation) are the same whichever batch it is loaded in and wherever its
// rows sit.  A single instance (id 0, first row 0) keeps the plain layout:
// row word = variable index, key = the seed.
struct RowStream {
  uint32_t row, k0;
};
__device__ __forceinline__ RowStream row_stream(const ProbDev &pd, uint32_t key0, int inst, int64_t v) {
  const int32_t voff = __ldg(&pd.inst[inst].v_off), gid = __ldg(&pd.inst[inst].gid);
  return RowStream{(uint32_t)(v - voff), key0 + (uint32_t)gid};
}

// ---------------------------------------------------------------- bit tricks
// 32x32 bit transpose across a warp: afterwards bit l of lane j equals bit j
// of lane l's input (recursive swap of off-diagonal blocks).
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int s = 16 >> k;
    const uint32_t m = masks[k];
    uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, s);
    x = (lane & s) ? ((x & ~m) | ((y >> s) & m)) : ((x & m) | ((y << s) & ~m));
  }
  return x;
}

// Add a 1-bit-per-lane value into a P-plane bit-sliced counter.
template <int P>
__device__ __forceinline__ void bitslice_add(uint32_t (&pl)[P], uint32_t a) {
#pragma unroll
  for (int p = 0; p < P; ++p) {
    uint32_t t = pl[p] & a;
    pl[p] ^= a;
    a = t;
  }
}

// Mask of lanes whose bit-sliced value equals r.
template <int P>
__device__ __forceinline__ uint32_t bitslice_eq(const uint32_t (&t)[P], int r) {
  uint32_t m = 0xFFFFFFFFu;
#pragma unroll
  for (int p = 0; p < P; ++p) m &= ((r >> p) & 1) ? t[p] : ~t[p];
  return m;
}

// AdamW's 1 / (sqrt(v / bc2) + eps), given 1 / sqrt(bc2): the hardware
// approximations sqrt.approx and rcp.approx (about 1 ulp each) with denormal
// inputs flushed to zero.  v >= 0 and the denominator is >= eps, so only a
// denormal v is affected (its square root is far below eps either way);
// skipping the denormal range fix-ups of sqrtf and of the division saves
// about 2 % of the fused update's time.
__device__ __forceinline__ float adam_inv_denom(float v, float inv_sqrt_bc2, float eps) {
  float s, r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(v));
  const float d = fmaf(s, inv_sqrt_bc2, eps);
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return r;
}

// 0/1 bytes from the 4 bits of n (bit b -> byte b)
__device__ __forceinline__ uint32_t spread4(uint32_t n) { return (n * 0x00204081u) & 0x01010101u; }
// (byte q of x) - 128 as an exact float: 2^23 + byte assembled in the mantissa
__device__ __forceinline__ float biased_byte(uint32_t x, uint32_t q) {
  return __int_as_float((int)__byte_perm(x, 0x4B000000u, 0x7440u | q)) - 8388736.0f;
}

// Byte-wise sum of two words of biased byte counts: bytes 128 + a and 128 + b
// give 128 + a + b, with no carry between bytes (valid while |a + b| <= 127):
// the low 7 bits add without leaving the byte and bit 7 takes the carry-less
// sum of the two top bits and the bias
__device__ __forceinline__ uint32_t add_biased_bytes(uint32_t x, uint32_t y) {
  const uint32_t s = (x & 0x7F7F7F7Fu) + (y & 0x7F7F7F7Fu);
  return s ^ (~(x ^ y) & 0x80808080u);
}

// Sum over the W consecutive lanes of a row group (W a power of two dividing
// 32); every lane of the warp takes part.
__device__ __forceinline__ float seg_sum(float x, int W) {
  for (int o = 1; o < W; o <<= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
  return x;
}

__device__ __forceinline__ float guard_nu(float mu) {
  const float g = 1e-12f;
  if (fabsf(mu) < g) return (mu < 0.0f) ? -g : g;
  return mu;
}

// Streaming (evict-first) 16-byte load and store of the state arrays.
__device__ __forceinline__ float4 ld_cs(const float *p) { return __ldcs(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ void st_cs(float *p, float4 v) { __stcs(reinterpret_cast<float4 *>(p), v); }

// Bits of step t: the ping-pong half t & 1.
__device__ __forceinline__ const uint32_t *cur_bits(const StateDev &sd, int64_t t) {
  return sd.bits + (size_t)(t & 1) * (size_t)sd.V * sd.W;
}

// Eq. 2 / Philox rule on one value, decided in FP32 without contraction.
// half: the sample's 16-bit Philox output (counter (i / 8, v, t, kTagBin),
// half i mod 8 of the four output words, low half first); u = half 2^-16.
__device__ __forceinline__ uint32_t binarize_one(float zt, int mode, float c, uint32_t half) {
  if (mode == TSAT_BIN_DET) return zt > 0.0f ? 1u : 0u;
  float u = __uint2float_rn(half) * (1.0f / 65536.0f);
  float p = __fadd_rn(0.5f, __fmul_rn(c, zt));
  p = fminf(fmaxf(p, 0.0f), 1.0f);
  return u < p ? 1u : 0u;
}

__device__ __forceinline__ int32_t load_nc(const int32_t *p) { return __ldg(p); }

// ---------------------------------------------------------------- L2 prefetch
// Bulk prefetch of `bytes` (multiple of 16, 16-byte aligned) into L2; a hint
// only: no shared memory, no barrier, nothing waits on it.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// The cache line holding p into L2 (a hint).
__device__ __forceinline__ void prefetch_l2_line(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

}  // namespace tsat
