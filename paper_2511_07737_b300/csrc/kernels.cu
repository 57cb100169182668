// kernels.cu -- sm_103a kernels of one optimisation step (Sec. III-B, IV-A).
//
// Data layout (row = global variable v, N samples, W = N/32 words):
//   z, m, v  float [V][N]        bits  uint32 [2][V][W] (ping-pong by step parity)
//   nu float [V]                 hist  int32 [n_inst][lm1][N]   gamma float [n_inst][lm1][N]
//
// k_fwd_hist   clause-major Eq. 1 + histogram of R per sample (integer exact)
// k_gamma      Eq. 4 / Eq. 3 from the histogram, dL/dR table per (sample, r),
//              exact SAT detection (a zero-unsat sample), lr schedule scalars
// k_update     variable-major: STE backward (P^T) from the occurrence records,
//              Eq. 5 chain rule, AdamW, new normaliser, Eq. 2 / Philox binarise
// k_check      bit-packed exact satisfaction check (OR of literal words)
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace tsat {

// ------------------------------------------------------------------ group sync / reductions
// A "row group" is N/4 consecutive threads of a block; it owns one variable row.
// Groups narrower than a warp share it with other groups that may take other
// paths, so every warp-level primitive uses the group's own lane mask.
struct Group {
  int GT, grp, gl, lane;
  __device__ __forceinline__ unsigned mask() const {
    return (GT >= 32) ? 0xFFFFFFFFu : (((1u << GT) - 1u) << (lane & ~(GT - 1)));
  }
  __device__ __forceinline__ void sync() const {
    if (GT <= 32) {
      __syncwarp(mask());
    } else if (GT == kBlock) {
      __syncthreads();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(GT) : "memory");
    }
  }
  // sum over the group, identical result in every thread (fixed order)
  __device__ __forceinline__ float sum(float x, float *red) const {
    const int span = GT < 32 ? GT : 32;
    const unsigned m = mask();
    for (int o = 1; o < span; o <<= 1) x += __shfl_xor_sync(m, x, o);
    if (GT <= 32) return x;
    const int nw = GT >> 5;
    const int wg = gl >> 5;
    sync();
    if ((gl & 31) == 0) red[wg] = x;
    sync();
    float s = 0.0f;
    for (int k = 0; k < nw; ++k) s += red[k];
    return s;
  }
};


// ------------------------------------------------------------------ init (Sec. IV-A)
// z ~ Irwin-Hall(12) from Philox, m = v = 0, nu, bits at t = 0.
__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

__device__ __forceinline__ void store_lits(const StateDev &sd, size_t off, const float a[4]) {
  if (sd.lit_bf16) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(a[0], a[1]), hi = __floats2bfloat162_rn(a[2], a[3]);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t *>(&lo);
    u.y = *reinterpret_cast<uint32_t *>(&hi);
    *reinterpret_cast<uint2 *>(reinterpret_cast<__nv_bfloat16 *>(sd.lit) + off) = u;
  } else {
    *reinterpret_cast<float4 *>(reinterpret_cast<float *>(sd.lit) + off) = make_float4(a[0], a[1], a[2], a[3]);
  }
}

// New normaliser (Eq. 5), Eq. 2 / Philox bits for step t, and (relaxed layer)
// the literal values sigmoid(z / nu).
__device__ __forceinline__ void row_binarize_store(const ProbDev &pd, const StateDev &sd, const Hyper &hy,
                                                   const Group &g, float *red, int inst, int64_t v,
                                                   const float zq[4], int64_t t, uint32_t *dst_bits,
                                                   bool want_lits = false) {
  const int N = sd.N;
  float nu = 1.0f;
  if (hy.norm != TSAT_NORM_NONE) {
    float part = (hy.norm == TSAT_NORM_ABSMEAN)
                     ? (fabsf(zq[0]) + fabsf(zq[1])) + (fabsf(zq[2]) + fabsf(zq[3]))
                     : (zq[0] + zq[1]) + (zq[2] + zq[3]);
    nu = guard_nu(g.sum(part, red) / (float)N);
  }
  const int s0 = g.gl * 4;
  // samples s0 .. s0+3 are halves 0..3 or 4..7 of the block s0 / 8
  uint4 rnd = make_uint4(0, 0, 0, 0);
  if (hy.binarize == TSAT_BIN_PHILOX) {
    const RowStream rs = row_stream(pd, hy.key0, inst, v);
    rnd = philox4x32_10(make_uint4((uint32_t)(g.gl >> 1), rs.row, (uint32_t)t, kTagBin), rs.k0, hy.key1);
  }
  const uint32_t w0 = (g.gl & 1) ? rnd.z : rnd.x, w1 = (g.gl & 1) ? rnd.w : rnd.y;
  uint32_t nib = 0;
  float a[4];
  const float rnu = __frcp_rn(nu);  // zt = z * (1/nu), both correctly rounded (FP32 decision)
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    float zt = __fmul_rn(zq[s], rnu);
    nib |= binarize_one(zt, hy.binarize, hy.bin_c, half16(w0, w1, s)) << s;
    a[s] = sigmoidf_(zt);
  }
  if (want_lits) store_lits(sd, (size_t)v * N + s0, a);
  uint32_t val = nib << (s0 & 31);
  const unsigned gm = g.mask();
  val |= __shfl_xor_sync(gm, val, 1);
  val |= __shfl_xor_sync(gm, val, 2);
  val |= __shfl_xor_sync(gm, val, 4);
  if ((g.gl & 7) == 0) dst_bits[v * sd.W + (s0 >> 5)] = val;
  if (g.gl == 0) sd.nu[v] = nu;
}

__global__ void __launch_bounds__(kBlock) k_init(ProbDev pd, StateDev sd, Hyper hy, const float *logits,
                                                 float scale) {
  __shared__ float red[64];
  const int GT = sd.N >> 2, RPB = kBlock / GT;
  Group g{GT, (int)threadIdx.x / GT, (int)threadIdx.x % GT, (int)(threadIdx.x & 31)};
  const int64_t NG = (int64_t)gridDim.x * RPB;
  const int64_t rows_round = ((int64_t)pd.V + NG - 1) / NG * NG;
  for (int64_t v = (int64_t)blockIdx.x * RPB + g.grp; v < rows_round; v += NG) {
    if (v >= pd.V) continue;  // whole group skips together (group-uniform v)
    const int s0 = g.gl * 4;
    const int inst = __ldg(pd.var_inst + v);
    const RowStream rs = row_stream(pd, hy.key0, inst, v);
    float zq[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int32_t acc = 0;
      for (uint32_t j = 0; j < 3; ++j) {
        // counter: the sample's global index (sample-sharded states start at sample_base)
        uint4 o = philox4x32_10(make_uint4((uint32_t)(sd.sample_base + s0 + s), rs.row, j, kTagInit), rs.k0,
                                hy.key1);
        acc += (int32_t)(o.x >> 8) + (int32_t)(o.y >> 8) + (int32_t)(o.z >> 8) + (int32_t)(o.w >> 8);
      }
      float noise = __int2float_rn(acc - 6 * (1 << 24)) * (1.0f / 16777216.0f);
      zq[s] = logits ? __fadd_rn(__fmul_rn(logits[v], scale), noise) : noise;
    }
    const size_t off = (size_t)v * sd.N + s0;
    st_cs(sd.z + off, make_float4(zq[0], zq[1], zq[2], zq[3]));
    st_cs(sd.m + off, make_float4(0.f, 0.f, 0.f, 0.f));
    st_cs(sd.v + off, make_float4(0.f, 0.f, 0.f, 0.f));
    row_binarize_store(pd, sd, hy, g, red + (GT > 32 ? g.grp * 8 : 0), inst, v, zq, 0, sd.bits);
  }
}

// Assignment mixing at an lr restart (the step's sp.mix_now): per instance the
// sample i* with the fewest unsatisfied clauses (gamma's best_sample) is kept,
// every other sample's z becomes (z + z_i*) / 2, m = v = 0, and the new
// normaliser and bits of step t + 1 follow from the mixed z (the update
// kernels skip this step).  Frozen instances keep their bits.
__global__ void __launch_bounds__(kBlock) k_mix(ProbDev pd, StateDev sd, Hyper hy) {
  __shared__ float red[64];
  const StepParams sp = *sd.sp;
  if (!sp.mix_now || sd.hdr->all_done) return;
  const int GT = sd.N >> 2, RPB = kBlock / GT;
  Group g{GT, (int)threadIdx.x / GT, (int)threadIdx.x % GT, (int)(threadIdx.x & 31)};
  const int64_t NG = (int64_t)gridDim.x * RPB;
  const int64_t rows_round = ((int64_t)pd.V + NG - 1) / NG * NG;
  const uint32_t *bsrc = cur_bits(sd, sp.t);
  uint32_t *bdst = const_cast<uint32_t *>(cur_bits(sd, sp.t + 1));
  for (int64_t v = (int64_t)blockIdx.x * RPB + g.grp; v < rows_round; v += NG) {
    if (v >= pd.V) continue;  // whole group skips together (group-uniform v)
    const int inst = __ldg(pd.var_inst + v);
    const int s0 = g.gl * 4;
    if (sd.inst[inst].found) {
      if ((g.gl & 7) == 0) bdst[v * sd.W + (s0 >> 5)] = bsrc[v * sd.W + (s0 >> 5)];
      continue;
    }
    const int best = sd.inst[inst].best_sample;
    const size_t off = (size_t)v * sd.N + s0;
    const float zb = sd.z[(size_t)v * sd.N + best];
    const float4 z4 = *reinterpret_cast<const float4 *>(sd.z + off);
    float zq[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (s0 + e != best) zq[e] = 0.5f * (zq[e] + zb);
    g.sync();   // every thread of the row has read z_i* before it is stored (unchanged, but ordered)
    *reinterpret_cast<float4 *>(sd.z + off) = make_float4(zq[0], zq[1], zq[2], zq[3]);
    *reinterpret_cast<float4 *>(sd.m + off) = make_float4(0.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float4 *>(sd.v + off) = make_float4(0.f, 0.f, 0.f, 0.f);
    row_binarize_store(pd, sd, hy, g, red + (GT > 32 ? g.grp * 8 : 0), inst, v, zq, sp.t + 1, bdst,
                       sd.layer == TSAT_LAYER_RELAXED);
  }
}

// Binarise an external z (autograd forward) into the current bits buffer.
__global__ void __launch_bounds__(kBlock) k_binarize(ProbDev pd, StateDev sd, Hyper hy, const float *zin,
                                                     int64_t t_bin, int want_lits) {
  __shared__ float red[64];
  const int GT = sd.N >> 2, RPB = kBlock / GT;
  Group g{GT, (int)threadIdx.x / GT, (int)threadIdx.x % GT, (int)(threadIdx.x & 31)};
  const int64_t NG = (int64_t)gridDim.x * RPB;
  const int64_t rows_round = ((int64_t)pd.V + NG - 1) / NG * NG;
  uint32_t *dst = const_cast<uint32_t *>(cur_bits(sd, sd.hdr->t));
  if (t_bin < 0) t_bin = sd.hdr->t;
  for (int64_t v = (int64_t)blockIdx.x * RPB + g.grp; v < rows_round; v += NG) {
    if (v >= pd.V) continue;
    const int s0 = g.gl * 4;
    const float *zsrc = zin ? zin : sd.z;
    float4 z4 = *reinterpret_cast<const float4 *>(zsrc + (size_t)v * sd.N + s0);
    float zq[4] = {z4.x, z4.y, z4.z, z4.w};
    row_binarize_store(pd, sd, hy, g, red + (GT > 32 ? g.grp * 8 : 0), __ldg(pd.var_inst + v), v, zq, t_bin, dst,
                       want_lits != 0);
  }
}

// ------------------------------------------------------------------ forward histogram (Eq. 1)
// Warp = 32 clauses x WB words.  Each lane forms the bit-sliced R of its
// clause for 32*WB samples (P planes); a 32x32 warp transpose turns the
// planes so that lane j holds, for sample j, one bit per clause; popcounts
// of the plane-match masks give the histogram h[r] of that sample.
template <int P, int WB>
__global__ void __launch_bounds__(kBlock) k_fwd_hist(ProbDev pd, StateDev sd, int32_t *hist, int skip_frozen) {
  const StateHdr *hdr = sd.hdr;
  if (skip_frozen && hdr->all_done) return;
  const int4 it = pd.items[blockIdx.x];
  const int inst = it.x;
  if (skip_frozen && sd.inst[inst].found) return;
  const int W = sd.W, N = sd.N, lm1 = sd.lm1;
  const int lmax = pd.inst[inst].lmax;
  const uint32_t *bits = cur_bits(sd, hdr->t);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nWB = W / WB;
  const bool many = nWB >= kWarps;
  const int nsub = many ? 1 : kWarps / nWB;
  const int sub = many ? 0 : warp / nWB;
  const int wb0 = many ? warp : warp % nWB;
  const int wbs = many ? kWarps : nWB;
  for (int wb = wb0; wb < nWB; wb += wbs) {
    int32_t cnt[WB][1 << P];
#pragma unroll
    for (int q = 0; q < WB; ++q)
#pragma unroll
      for (int r = 0; r < (1 << P); ++r) cnt[q][r] = 0;
    for (int g0 = it.y + sub * 32; g0 < it.z; g0 += nsub * 32) {
      const int c = g0 + lane;
      const bool active = c < it.z;
      uint32_t pl[WB][P];
#pragma unroll
      for (int q = 0; q < WB; ++q)
#pragma unroll
        for (int p = 0; p < P; ++p) pl[q][p] = 0;
      if (active) {
        // literals in chunks of 4: the chunk's literal loads, then its gathers,
        // are issued together (one dependent-load round each per chunk)
        const int32_t b = __ldg(pd.cptr + c), e = __ldg(pd.cptr + c + 1);
        for (int32_t j0 = b; j0 < e; j0 += 4) {
          int32_t lit[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) lit[u] = (j0 + u < e) ? __ldg(pd.clit + j0 + u) : -1;
          uint32_t x[4][WB];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const uint32_t negm = 0u - (uint32_t)(lit[u] & 1);
            const uint32_t *row = bits + (size_t)(lit[u] >> 1) * W + wb * WB;
            if (lit[u] < 0) {
#pragma unroll
              for (int q = 0; q < WB; ++q) x[u][q] = 0u;
            } else if constexpr (WB == 4) {
              const uint4 y = __ldg(reinterpret_cast<const uint4 *>(row));
              x[u][0] = y.x ^ negm; x[u][1] = y.y ^ negm; x[u][2] = y.z ^ negm; x[u][3] = y.w ^ negm;
            } else if constexpr (WB == 2) {
              const uint2 y = __ldg(reinterpret_cast<const uint2 *>(row));
              x[u][0] = y.x ^ negm; x[u][1] = y.y ^ negm;
            } else {
              x[u][0] = __ldg(row) ^ negm;
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (lit[u] >= 0) {
#pragma unroll
              for (int q = 0; q < WB; ++q) bitslice_add<P>(pl[q], x[u][q]);
            }
        }
      }
      const uint32_t valid = __ballot_sync(0xFFFFFFFFu, active);
#pragma unroll
      for (int q = 0; q < WB; ++q) {
        uint32_t tp[P];
#pragma unroll
        for (int p = 0; p < P; ++p) tp[p] = warp_transpose32(pl[q][p], lane);
#pragma unroll
        for (int r = 0; r < (1 << P); ++r) cnt[q][r] += __popc(valid & bitslice_eq<P>(tp, r));
      }
    }
#pragma unroll
    for (int q = 0; q < WB; ++q) {
      const int sample = (wb * WB + q) * 32 + lane;
#pragma unroll
      for (int r = 0; r < (1 << P); ++r)
        if (r <= lmax && cnt[q][r]) atomicAdd(hist + ((size_t)inst * lm1 + r) * N + sample, cnt[q][r]);
    }
  }
}

// ------------------------------------------------------------------ forward histogram, word per lane
// Clause length <= 3 and N >= 512 (W >= 16 words per row).  A row group of W
// lanes takes one clause at a time: lane w gathers word w of the clause's three
// literal rows (W consecutive words, one 128-byte line per literal when W = 32)
// and forms R's bit planes for its 32 samples, p0 = [R odd], p1 = [R >= 2].
// The masks p0, p1 and p0 & p1 are added into vertical (bit-sliced) counters
// with carry-save adders (Harley-Seal: seven CSAs per mask per 8 clauses, the
// eights rippled into a 5-plane counter).  Their sums are C0 = h1 + h3,
// C1 = h2 + h3 and C01 = h3, so over n clauses
//   h3 = C01, h2 = C1 - C01, h1 = C0 - C01, h0 = (n - C0) - h2.
// Every <= 248 clauses a lane turns its counters into per-sample byte counts
// and adds them to the block's histogram in shared memory; at the end the
// block adds its histogram to the global one.  Compared with k_fwd_hist (lane
// = clause, 32x32 warp transposes) this issues about a third of the
// instructions per clause and gathers whole lines instead of 16-byte pieces.
constexpr int kFwdUnitsPerFlush = 31;   // 8-clause units between flushes: counts <= 248 fit a byte

// lo + b + c = 2 hi + lo' (one carry-save adder, two 3-input logic ops)
__device__ __forceinline__ void csa(uint32_t &hi, uint32_t &lo, uint32_t b, uint32_t c) {
  const uint32_t u = lo ^ b;
  hi = (lo & b) | (u & c);
  lo = u ^ c;
}

// Column j of a vertical counter (planes pl[0..7], weights 1..128) as strided
// byte counts: byte q = the count of sample 8 q + j of the word.
__device__ __forceinline__ uint32_t vertical_column(const uint32_t (&pl)[8], int j) {
  uint32_t a = 0;
#pragma unroll
  for (int b = 0; b < 8; ++b) a += ((pl[b] >> j) & 0x01010101u) << b;
  return a;
}

// The three masks of one clause for this lane's 32 samples.  MASKED: the clause
// may lie past the item's end (valid = 0) or be shorter than 3 literals.
template <bool MASKED>
__device__ __forceinline__ void clause_masks(const ProbDev &pd, const uint32_t *bw, int W, int c, bool valid,
                                             uint32_t &m0, uint32_t &m1, uint32_t &m2) {
  const int4 cr = __ldg(pd.crec + c);
  uint32_t a = __ldg(bw + (size_t)cr.x * W) ^ __byte_perm((uint32_t)cr.w, 0u, 0x0000u);
  uint32_t b = __ldg(bw + (size_t)cr.y * W) ^ __byte_perm((uint32_t)cr.w, 0u, 0x1111u);
  uint32_t d = __ldg(bw + (size_t)cr.z * W) ^ __byte_perm((uint32_t)cr.w, 0u, 0x2222u);
  if constexpr (MASKED) {
    const uint32_t len = valid ? ((uint32_t)cr.w >> 24) : 0u;
    a = len > 0 ? a : 0u;
    b = len > 1 ? b : 0u;
    d = len > 2 ? d : 0u;
  }
  m0 = a ^ b ^ d;
  m1 = (a & b) | (d & (a ^ b));
  m2 = m0 & m1;
}

// One unit: 8 clauses of this row group (c, c + RW, ..., c + 7 RW), their
// masks added into the vertical counters pl[mask][plane].
template <bool MASKED>
__device__ __forceinline__ void fwd_unit(const ProbDev &pd, const uint32_t *bw, int W, int RW, int c, int cend,
                                         uint32_t (&pl)[3][8]) {
  uint32_t fA[3];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t m[3][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int ck = c + (4 * h + k) * RW;
      const bool ok = !MASKED || ck < cend;
      clause_masks<MASKED>(pd, bw, W, ok ? ck : cend - 1, ok, m[0][k], m[1][k], m[2][k]);
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      uint32_t tA, tB, fX;
      csa(tA, pl[s][0], m[s][0], m[s][1]);
      csa(tB, pl[s][0], m[s][2], m[s][3]);
      csa(fX, pl[s][1], tA, tB);
      if (h == 0) {
        fA[s] = fX;
      } else {
        uint32_t e;
        csa(e, pl[s][2], fA[s], fX);
#pragma unroll
        for (int q = 3; q < 8; ++q) {
          const uint32_t cy = pl[s][q] & e;
          pl[s][q] ^= e;
          e = cy;
        }
      }
    }
  }
}

// W: words per row as a compile-time constant (16 or 32, i.e. N = 512 or 1024,
// the sizes this kernel runs at); the row-group arithmetic then folds into
// immediates (0.433 -> 0.331 ms at n = 1e6, N = 1024).
template <int WC>
__global__ void __launch_bounds__(kBlock, 4) k_fwd_w3(ProbDev pd, StateDev sd, int32_t *hist, int skip_frozen) {
  extern __shared__ int32_t shh[];   // [nr][N] block histogram; sample 32 w + i at 32 w + ((i + w) & 31)
  const StateHdr *hdr = sd.hdr;
  if (skip_frozen && hdr->all_done) return;
  const int4 it = pd.items[blockIdx.x];
  const int inst = it.x;
  if (skip_frozen && sd.inst[inst].found) return;
  constexpr int W = WC, RW = 32 / W, N = 32 * W;
  const int lm1 = sd.lm1;
  const int nr = min(pd.inst[inst].lmax, 3) + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rsub = lane / W, w = lane % W;
  for (int i = threadIdx.x; i < nr * N; i += kBlock) shh[i] = 0;
  __syncthreads();
  const uint32_t *bw = cur_bits(sd, hdr->t) + w;
  const int U = 8 * RW;
  const int nunits = (it.z - it.y + U - 1) / U;
  uint32_t pl[3][8];
#pragma unroll
  for (int s = 0; s < 3; ++s)
#pragma unroll
    for (int q = 0; q < 8; ++q) pl[s][q] = 0u;
  int n = 0, since = 0;
  for (int u = warp; u < nunits; u += kWarps) {
    const int c = it.y + u * U + rsub;
    if (pd.full3 && it.y + (u + 1) * U <= it.z) {   // a whole unit of 3-literal clauses
      fwd_unit<false>(pd, bw, W, RW, c, it.z, pl);
      n += 8;
    } else {
      fwd_unit<true>(pd, bw, W, RW, c, it.z, pl);
      n += max(0, min(8, (it.z - c + RW - 1) / RW));
    }
    ++since;
    const bool last = u + kWarps >= nunits;
    if (since == kFwdUnitsPerFlush || last) {
      // per-sample byte counts of the three masks, then h0..h3 (no byte borrows: all are >= 0)
      const uint32_t nrep = (uint32_t)n * 0x01010101u;
#pragma unroll 1
      for (int j = 0; j < 8; ++j) {
        const uint32_t c0 = vertical_column(pl[0], j), c1 = vertical_column(pl[1], j);
        const uint32_t c01 = vertical_column(pl[2], j);
        const uint32_t h3 = c01, h2 = c1 - c01, h1 = c0 - c01, h0 = (nrep - c0) - h2;
        const uint32_t hv[4] = {h0, h1, h2, h3};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int idx = 32 * w + ((8 * q + j + w) & 31);
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (r < nr) atomicAdd(shh + r * N + idx, (int32_t)((hv[r] >> (8 * q)) & 0xFFu));
        }
      }
#pragma unroll
      for (int s = 0; s < 3; ++s)
#pragma unroll
        for (int q = 0; q < 8; ++q) pl[s][q] = 0u;
      n = 0;
      since = 0;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nr * N; i += kBlock) {
    const int val = shh[i];
    if (!val) continue;
    const int r = i / N, k = i - r * N, wd = k >> 5;
    const int sample = 32 * wd + (((k & 31) - wd) & 31);
    atomicAdd(hist + ((size_t)inst * lm1 + r) * N + sample, val);
  }
}

// Per-instance loss / best sample / exact-SAT freeze, then (step mode) the
// step scalars: lr(t) of Sec. IV-A, AdamW bias corrections, t <- t + 1.
// pows: the three parts of step t's scalars (step_part) formed earlier in the
// kernel and published by the barrier below, or NULL: all formed here, by
// thread 0.
__device__ void gamma_tail(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const LrSched &ls,
                           int step_mode, float *loss_out, const float *Sb, int64_t t,
                           const double *pows = nullptr) {
  StateHdr *hdr = sd.hdr;
  const int N = sd.N;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int inst = warp; inst < pd.n_inst; inst += nw) {
    InstState *is = sd.inst + inst;
    if (step_mode && is->found) continue;
    float ls_ = 0.f;
    int32_t mu = 0x7FFFFFFF, mi = 0;
    for (int i = lane; i < N; i += 32) {
      ls_ += Sb[(size_t)inst * N + i];
      int32_t u = sd.unsat[(size_t)inst * N + i];
      if (u < mu) { mu = u; mi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      ls_ += __shfl_xor_sync(0xFFFFFFFFu, ls_, o);
      int32_t u2 = __shfl_xor_sync(0xFFFFFFFFu, mu, o);
      int32_t i2 = __shfl_xor_sync(0xFFFFFFFFu, mi, o);
      if (u2 < mu || (u2 == mu && i2 < mi)) { mu = u2; mi = i2; }
    }
    if (lane == 0) {
      if (loss_out) loss_out[inst] = -ls_;
      if (step_mode) {
        is->loss = -ls_;
        is->min_unsat = mu;
        is->best_sample = mi;
        if (mu == 0) {
          is->found = 1;
          is->found_sample = mi;
          is->found_step = t;
        }
      }
    }
  }
  if (!step_mode) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    int active = 0;
    for (int j = 0; j < pd.n_inst; ++j) active += sd.inst[j].found ? 0 : 1;
    hdr->n_active = active;
    if (active == 0 && hy.stop_on_sat) {
      hdr->all_done = 1;
      return;
    }
    *sd.sp = pows ? step_finish(ls, t, pows[0], pows[1], pows[2]) : step_params(ls, t);
    hdr->t = t + 1;
  }
}

// ------------------------------------------------------------------ gamma (Eq. 3, Eq. 4)
// One block.  For each (instance, sample) with histogram h[r]:
//   Z = sum_r h_r e^{-tau r},  S = sum_r r h_r e^{-tau r} / Z,
//   gamma[r] = dL/dR for a clause with R = r = -(e^{-tau r}/Z)(1 - tau (r - S)).
// step_mode 1 also freezes instances that reached a zero-unsat sample, writes
// the step scalars (lr schedule, AdamW bias corrections) and advances t.
__global__ void __launch_bounds__(1024) k_gamma(ProbDev pd, StateDev sd, Hyper hy, LrSched ls, const int32_t *hist_in,
                                                int step_mode, int write_gamma, float *loss_out, float *S_out) {
  __shared__ float etab[32];
  __shared__ double sh_pow[3];
  StateHdr *hdr = sd.hdr;
  if (step_mode && hdr->all_done) return;
  const int64_t t = hdr->t;
  if (threadIdx.x < 32) etab[threadIdx.x] = expf(-hy.tau * (float)threadIdx.x);
  __syncthreads();
  // the three double-precision parts of the step scalars (each a serial chain
  // of a few microseconds) by the last three threads, side by side and under
  // the other threads' histogram work; gamma_tail's barrier publishes them and
  // thread 0 combines them
  if (step_mode && threadIdx.x >= blockDim.x - 3) {
    const int j = (int)(threadIdx.x - (blockDim.x - 3));
    sh_pow[j] = step_part(ls, t, j);
  }
  const int N = sd.N, lm1 = sd.lm1;
  int32_t *hist = const_cast<int32_t *>(hist_in);
  float *Sb = S_out ? S_out : sd.S;
  const int64_t total = (int64_t)pd.n_inst * N;
  for (int64_t p = threadIdx.x; p < total; p += blockDim.x) {
    const int inst = (int)(p / N), i = (int)(p - (int64_t)inst * N);
    if (step_mode && sd.inst[inst].found) continue;
    const int lmax = pd.inst[inst].lmax;
    int32_t *h = hist + (size_t)inst * lm1 * N + i;
    float Z = 0.f, Y = 0.f;
    for (int r = 0; r <= lmax; ++r) {
      float hv = (float)h[(size_t)r * N];
      Z += hv * etab[r];
      Y += (float)r * hv * etab[r];
    }
    const float S = Y / Z;
    const float invZ = 1.0f / Z;
    const int32_t h0 = h[0];
    if (write_gamma) {
      float *gm = sd.gamma + (size_t)inst * lm1 * N + i;
      float gr[4] = {0.f, 0.f, 0.f, 0.f};
      for (int r = 0; r <= lmax; ++r) {
        const float gv = -(etab[r] * invZ) * (1.0f - hy.tau * ((float)r - S));
        gm[(size_t)r * N] = gv;
        if (r < 4) gr[r] = gv;
      }
      if (lm1 <= 4) {
        float *gd = sd.gdelta + (size_t)inst * 4 * N + i;
        gd[0] = gr[0];
        gd[N] = gr[1] - gr[0];
        gd[2 * N] = gr[2] - gr[0];
        gd[3 * N] = (gr[3] - gr[2]) - (gr[1] - gr[0]);
      }
    }
    if (step_mode)
      for (int r = 0; r <= lmax; ++r) h[(size_t)r * N] = 0;
    Sb[(size_t)inst * N + i] = S;
    sd.unsat[(size_t)inst * N + i] = h0;
  }
  gamma_tail(pd, sd, hy, ls, step_mode, loss_out, Sb, t, step_mode ? sh_pow : nullptr);
}

// ------------------------------------------------------------------ fused update
// Row group = N/4 threads, thread owns samples s0..s0+3 (one nibble of word w).
// mode 0: backward (STE, P^T through the occurrence records), Eq. 5 chain
//         rule, AdamW, new normaliser, binarise into the other bits buffer.
// mode 1: backward + Eq. 5 chain rule only; grad = dL * g (autograd).
constexpr int kRecInts = 2048;  // record staging per block (int32 words)

__device__ __forceinline__ float sel4(int r, float g0, float g1, float g2, float g3) {
  float a = (r & 1) ? g1 : g0;
  float b = (r & 1) ? g3 : g2;
  return (r & 2) ? b : a;
}

// 2^x by the PTX base-2 exponential (flushes subnormal results to zero)
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int P, bool GREG, bool RELAX, bool DR16 = false>
__global__ void __launch_bounds__(kBlock, 3) k_update(ProbDev pd, StateDev sd, Hyper hy, int mode,
                                                      const float *zin, float *grad, float dL,
                                                      int rows_per_item) {
  extern __shared__ int32_t smem[];
  const StateHdr *hdr = sd.hdr;
  if (mode == 0 && hdr->all_done) return;
  const int N = sd.N, W = sd.W, lm1 = sd.lm1;
  const int GT = N >> 2, RPB = kBlock / GT;
  Group g{GT, (int)threadIdx.x / GT, (int)threadIdx.x % GT, (int)(threadIdx.x & 31)};
  const int cap = kRecInts / RPB;
  int32_t *rec = smem + g.grp * cap;
  float *red = reinterpret_cast<float *>(smem + kRecInts) + g.grp * 8;
  float *gtab = reinterpret_cast<float *>(smem + kRecInts + 8 * RPB) + (size_t)g.grp * lm1 * N;
  const int s0 = g.gl * 4, w = s0 >> 5, sh = s0 & 31;
  StepParams sp;
  if (mode == 0) sp = *sd.sp;
  if (mode == 0 && sp.mix_now) return;   // this step mixes assignments (k_mix)
  const int64_t tcur = (mode == 0) ? sp.t : hdr->t;
  const uint32_t *bsrc = cur_bits(sd, tcur);
  uint32_t *bdst = const_cast<uint32_t *>(cur_bits(sd, tcur + 1));
  const float b1 = hy.beta1, b2 = hy.beta2;
  float gam[4][4];
  // relaxed layer, FP32 storage: dL/dR_ci = e^{-tau R} (ra R + rb) per sample,
  // ra = tau / Z_i, rb = -(1 + tau S_i) / Z_i (Eq. 4 differentiated), formed
  // from the gathered R of each occurrence
  float ra[4] = {0.f, 0.f, 0.f, 0.f}, rb[4] = {0.f, 0.f, 0.f, 0.f};
  int cur_inst = -1;
  const int64_t NG = (int64_t)gridDim.x * RPB;
  const int64_t n_items = ((int64_t)pd.V + rows_per_item - 1) / rows_per_item;
  for (int64_t item = (int64_t)blockIdx.x * RPB + g.grp; item < n_items; item += NG) {
    const int64_t v_end = min((int64_t)pd.V, (item + 1) * rows_per_item);
    for (int64_t v = item * rows_per_item; v < v_end; ++v) {
      const int inst = __ldg(pd.var_inst + v);
      if (mode == 0 && sd.inst[inst].found) {  // frozen instance: keep its model
        if ((g.gl & 7) == 0) bdst[v * W + w] = bsrc[v * W + w];
        continue;
      }
      if (inst != cur_inst) {
        cur_inst = inst;
        const float *gsrc = sd.gamma + (size_t)inst * lm1 * N;
        if constexpr (RELAX) {
          if constexpr (!DR16) {
            const float4 zz = *reinterpret_cast<const float4 *>(sd.zs + (size_t)inst * 2 * N + s0);
            const float4 ss = *reinterpret_cast<const float4 *>(sd.zs + ((size_t)inst * 2 + 1) * N + s0);
            const float Zq[4] = {zz.x, zz.y, zz.z, zz.w}, Sq[4] = {ss.x, ss.y, ss.z, ss.w};
#pragma unroll
            for (int s = 0; s < 4; ++s) {
              const float iz = 1.0f / Zq[s];
              ra[s] = hy.tau * iz;
              rb[s] = -(1.0f + hy.tau * Sq[s]) * iz;
            }
          }
        } else if constexpr (GREG) {
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            float4 x = (r < lm1) ? *reinterpret_cast<const float4 *>(gsrc + (size_t)r * N + s0)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
            gam[0][r] = x.x; gam[1][r] = x.y; gam[2][r] = x.z; gam[3][r] = x.w;
          }
        } else {
          g.sync();
          for (int k = g.gl; k < lm1 * N; k += GT) gtab[k] = gsrc[k];
          g.sync();
        }
      }
      const size_t off = (size_t)v * N + s0;
      const float4 z4 = (mode == 0) ? ld_cs(sd.z + off) : *reinterpret_cast<const float4 *>(zin + off);
      float4 m4 = make_float4(0.f, 0.f, 0.f, 0.f), v4 = m4;
      if (mode == 0) { m4 = ld_cs(sd.m + off); v4 = ld_cs(sd.v + off); }
      const uint32_t ownw = __ldg(bsrc + v * W + w);
      const float nu = sd.nu[v];
      float G[4] = {0.f, 0.f, 0.f, 0.f};
      if constexpr (RELAX) {
        // ---- relaxed backward: sum of +-dL/dR_ci over the row's occurrences, 8
        // occurrences' loads in flight.  BF16 storage: the buffer holds dL/dR
        // (k_relaxed_dr); FP32: the buffer holds R, and dL/dR is formed here
        // (one exponential per occurrence and sample instead of a pass that
        // writes and re-reads the whole [C][N] buffer)
        const int32_t ob = __ldg(pd.vptr + v), oe = __ldg(pd.vptr + v + 1);
        int32_t o = ob;
        // the stored value of clause c for this thread's 4 samples
        auto dR = [&](int32_t c) -> float4 {
          if constexpr (DR16) {
            const uint2 u = __ldg(reinterpret_cast<const uint2 *>(sd.dr16 + ((size_t)c * N + s0) / 2));
            const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
            const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
            return make_float4(lo.x, lo.y, hi.x, hi.y);
          } else {
            return __ldg(reinterpret_cast<const float4 *>(sd.rbuf + (size_t)c * N + s0));
          }
        };
        // dL/dR from the stored value: e^{-tau R} as 2^{c R}, c = -tau log2(e),
        // one multiply and the hardware base-2 exponential (relative error
        // about 2^-22, plus c R's rounding)
        const float c2 = -hy.tau * 1.4426950408889634f;
        auto toD = [&](float4 x) -> float4 {
          if constexpr (DR16) {
            return x;
          } else {
            return make_float4(ex2_approx(c2 * x.x) * fmaf(ra[0], x.x, rb[0]), ex2_approx(c2 * x.y) * fmaf(ra[1], x.y, rb[1]),
                               ex2_approx(c2 * x.z) * fmaf(ra[2], x.z, rb[2]), ex2_approx(c2 * x.w) * fmaf(ra[3], x.w, rb[3]));
          }
        };
        for (; o + 8 <= oe; o += 8) {
          int32_t e[8];
          float4 D[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) e[q] = __ldg(pd.vocc + o + q);
#pragma unroll
          for (int q = 0; q < 8; ++q) D[q] = dR(e[q] >> 1);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float sg = (e[q] & 1) ? -1.0f : 1.0f;
            const float4 Dq = toD(D[q]);
            G[0] = fmaf(sg, Dq.x, G[0]);
            G[1] = fmaf(sg, Dq.y, G[1]);
            G[2] = fmaf(sg, Dq.z, G[2]);
            G[3] = fmaf(sg, Dq.w, G[3]);
          }
        }
        for (; o < oe; ++o) {
          const int32_t e = __ldg(pd.vocc + o);
          const float4 D = toD(dR(e >> 1));
          const float sg = (e & 1) ? -1.0f : 1.0f;
          G[0] = fmaf(sg, D.x, G[0]);
          G[1] = fmaf(sg, D.y, G[1]);
          G[2] = fmaf(sg, D.z, G[2]);
          G[3] = fmaf(sg, D.w, G[3]);
        }
        const float zq_[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const float a = sigmoidf_(__fmul_rn(zq_[s], __frcp_rn(nu)));
          G[s] *= a * (1.0f - a);
        }
      } else {
      // ---- STE backward: G_vi = sum_{c owns x_v} gamma_i[R_ci] - sum_{c owns x_v'} gamma_i[R_ci]
      int64_t pos0 = pd.xptr[v];
      const int64_t pend = pd.xptr[v + 1];
      while (pos0 < pend) {
        const int n = (int)min((int64_t)cap, pend - pos0);
        g.sync();
        for (int k = g.gl; k < n; k += GT) rec[k] = __ldg(pd.xrec + pos0 + k);
        g.sync();
        int pos = 0;
        bool end = false;
        while (pos < n) {
          const int32_t h = rec[pos];
          if (h == 0) { end = true; break; }          // padding: end of this row
          const int len = h >> 1;
          if (pos + len > n) break;                    // record continues in the next chunk
          const uint32_t ownneg = (uint32_t)(h & 1);
          uint32_t pl[P];
          pl[0] = ownw ^ (0u - ownneg);
#pragma unroll
          for (int p = 1; p < P; ++p) pl[p] = 0;
          for (int q = 1; q < len; ++q) {
            const int32_t lit = rec[pos + q];
            const uint32_t x = __ldg(bsrc + (size_t)(lit >> 1) * W + w) ^ (0u - (uint32_t)(lit & 1));
            bitslice_add<P>(pl, x);
          }
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            int r = 0;
#pragma unroll
            for (int p = 0; p < P; ++p) r |= (int)((pl[p] >> (sh + s)) & 1u) << p;
            float gv;
            if constexpr (GREG) gv = sel4(r, gam[s][0], gam[s][1], gam[s][2], gam[s][3]);
            else gv = gtab[r * N + s0 + s];
            G[s] += ownneg ? -gv : gv;
          }
          pos += len;
        }
        pos0 = end ? pend : pos0 + pos;
      }
      }
      // ---- chain rule through Eq. 5
      const float zq[4] = {z4.x, z4.y, z4.z, z4.w};
      float gq[4];
      if (hy.norm == TSAT_NORM_NONE) {
#pragma unroll
        for (int s = 0; s < 4; ++s) gq[s] = G[s];
      } else {
        const float dot = g.sum((G[0] * zq[0] + G[1] * zq[1]) + (G[2] * zq[2] + G[3] * zq[3]), red);
        const float c2 = dot / ((float)N * nu * nu);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const float dmu = (hy.norm == TSAT_NORM_ABSMEAN) ? (float)((zq[s] > 0.f) - (zq[s] < 0.f)) : 1.0f;
          gq[s] = G[s] / nu - c2 * dmu;
        }
      }
      if (mode == 1) {
        *reinterpret_cast<float4 *>(grad + off) = make_float4(dL * gq[0], dL * gq[1], dL * gq[2], dL * gq[3]);
        continue;
      }
      // ---- AdamW (decoupled weight decay, bias-corrected moments)
      float mq[4] = {m4.x, m4.y, m4.z, m4.w}, vq[4] = {v4.x, v4.y, v4.z, v4.w}, zn[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const float gs = gq[s];
        mq[s] = b1 * mq[s] + hy.omb1 * gs;
        vq[s] = b2 * vq[s] + hy.omb2 * (gs * gs);
        zn[s] = zq[s] * sp.decay - sp.step_size * (mq[s] * adam_inv_denom(vq[s], sp.inv_sqrt_bc2, hy.eps));
      }
      st_cs(sd.z + off, make_float4(zn[0], zn[1], zn[2], zn[3]));
      st_cs(sd.m + off, make_float4(mq[0], mq[1], mq[2], mq[3]));
      st_cs(sd.v + off, make_float4(vq[0], vq[1], vq[2], vq[3]));
      // ---- new normaliser and Eq. 2 for step t+1
      row_binarize_store(pd, sd, hy, g, red, inst, v, zn, tcur + 1, bdst, RELAX);
    }
  }
}


// ------------------------------------------------------------------ fused update, word per lane
// Clause length <= 3 (R in 0..3, two bit planes).  Counting phase: a lane owns
// one 32-sample word of one variable row (W = N/32 lanes per row, 32/W rows
// per warp), so
//   * the occurrence records of a row are loaded by its W lanes in parallel
//     and broadcast by shuffles; the other literals' words are gathered
//     coalesced (W consecutive lanes read W consecutive words) and the R bit
//     planes stay in registers;
//   * the lane counts, byte-packed with bias 128 for its 32 samples, the
//     signed occurrences whose R has plane-0 bit, plane-1 bit, both bits set;
//     gamma[R] = g0 + b0 d1 + b1 d2 + b0 b1 d3 turns the STE sum into
//     G = (n+ - n-) g0 + C0 d1 + C1 d2 + C01 d3 (exact rewrite).
// The counters are strided (byte b of counter j counts sample 8b + j, so a
// bit plane is added with one shift and one mask per register); a 4x4 byte
// transpose per row turns them into words of 4 consecutive samples, stored in
// shared memory by sample/4.  Sample phase: each lane reads back the words of
// its own 4 consecutive samples per pass (8 passes), with coalesced 16-byte
// accesses to z, m, v (z is read in both passes; the second read hits L2).
// Row reductions (Eq. 5 dot product, new normaliser) are shuffles across the
// row's lanes; each lane binarises its 4 samples into a nibble and lane w
// assembles bits word w from the eight nibbles of its samples.  The row's z,
// m, v and the next row's gathered bits rows are prefetched into L2 as late
// as still pays (see the prefetches below), to keep the bits array resident.
// The counting loop and the two sample passes are unrolled by 2 (two passes'
// z, m, v loads in flight: 6.24 -> 6.01 ms at n = 1e6); full unrolling loses:
// with 28 warps per SM in different phases, instruction-cache misses cost
// more than the loop overhead.
constexpr int kCntChunk = 127;   // occurrences per byte-counter chunk (|count| <= 127)
// Blocks of 4 warps at <= 73 registers: 7 blocks (28 warps) per SM.  Measured
// at n = 1e6, N = 1024: 5.97 ms, against 6.02 ms for 8-warp blocks at 80
// registers (24 warps per SM) and 6.42 ms at 64 registers (spills).
constexpr int kUpd3Block = 128, kUpd3Warps = 4, kUpd3MinB = 7;


// Word i (0..255) of a per-warp word array lives at cswz(i): i XOR g(i / 32),
// g = {0, 29, 26, 7, 20, 9, 14, 19}.  Both access patterns of the kernel,
// word 8 * lane + c (counting layout) and word 8 W r + W k + w (sample layout),
// then hit 32 distinct banks for every W in {1, 2, ..., 32}.
__device__ __forceinline__ int cswz(int i) {
  const int u = (i >> 5) & 7;
  return i ^ (((9 * u) ^ (20 * u)) & 31);
}

// C0 d1 + C1 d2 + C01 d3 for 4 samples from their count words (biased bytes)
__device__ __forceinline__ float4 fold_counts(uint32_t w0, uint32_t w1, uint32_t w2, float4 d1, float4 d2, float4 d3) {
  float4 r;
  r.x = fmaf(biased_byte(w0, 0), d1.x, fmaf(biased_byte(w1, 0), d2.x, biased_byte(w2, 0) * d3.x));
  r.y = fmaf(biased_byte(w0, 1), d1.y, fmaf(biased_byte(w1, 1), d2.y, biased_byte(w2, 1) * d3.y));
  r.z = fmaf(biased_byte(w0, 2), d1.z, fmaf(biased_byte(w1, 2), d2.z, biased_byte(w2, 2) * d3.z));
  r.w = fmaf(biased_byte(w0, 3), d1.w, fmaf(biased_byte(w1, 3), d2.w, biased_byte(w2, 3) * d3.w));
  return r;
}

__device__ __forceinline__ float4 f4_add(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// MODE 0: optimisation step; MODE 1: autograd backward (gradient out, no
// update).  BIN and NORM are the binarisation and Eq. 5 modes: one kernel per
// combination keeps each kernel's code small and free of mode branches.  WC:
// the words per row as a compile-time constant (32: N = 1024; the swizzled
// shared-memory indices, shuffle sources and row offsets then fold into
// immediates, 5.85 -> 5.58 ms at n = 1e6), or 0 for the runtime value.
template <int MODE, int BIN, int NORM, int WC>
__global__ void __launch_bounds__(kUpd3Block, kUpd3MinB) k_update3(ProbDev pd, StateDev sd, Hyper hy, const float *zin, float *grad,
                                                       float dL) {
  extern __shared__ __align__(16) float sm3[];
  const StateHdr *hdr = sd.hdr;
  if (MODE == 0 && hdr->all_done) return;
  const int W = WC ? WC : sd.W, N = 32 * W, RW = 32 / W;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rsub = lane / W, w = lane % W, rbase = rsub * W;   // row group: lanes rbase .. rbase + W - 1
  float4 *gbuf = reinterpret_cast<float4 *>(sm3) + warp * 448;                     // [8 passes][32 lanes]: G, then z(t+1)
  uint32_t *cbuf = reinterpret_cast<uint32_t *>(gbuf + 256);                         // [3 counts][256 words]
  uint32_t *nbuf = cbuf;                                                             // [256 nibbles] after the counts
  StepParams sp;
  if (MODE == 0) sp = *sd.sp;
  if (MODE == 0 && sp.mix_now) return;   // this step mixes assignments (k_mix)
  const int64_t tcur = (MODE == 0) ? sp.t : hdr->t;
  const uint32_t *bsrc = cur_bits(sd, tcur);
  uint32_t *bdst = const_cast<uint32_t *>(cur_bits(sd, tcur + 1));
  const float *zsrc = (MODE == 0) ? sd.z : zin;
  const int4 *xrec4 = reinterpret_cast<const int4 *>(pd.xrec);
  const int64_t nwarps = (int64_t)gridDim.x * kUpd3Warps;
  const int ist = 8 * lane;          // count words this lane stores: its 32 samples
  const int isam = rsub * 8 * W + w; // + W k: the word of this lane's samples in pass k
  // first record round of the row group's current row, loaded during the previous row
  int4 crec = make_int4(0, 0, 0, 0);
  bool have_crec = false;
  for (int64_t base = ((int64_t)blockIdx.x * kUpd3Warps + warp) * RW; base < pd.V; base += nwarps * RW) {
    __syncwarp();   // the previous row's readers of gbuf / zbuf are done
    const int64_t v = base + rsub;
    const bool valid = v < pd.V;
    int inst = 0;
    bool frozen = false;
    if (valid) {
      inst = __ldg(pd.var_inst + v);
      frozen = (MODE == 0) && sd.inst[inst].found;
    }
    const bool act = valid && !frozen;
    const float4 *gd4 = reinterpret_cast<const float4 *>(sd.gdelta + (size_t)inst * 4 * N);   // [4][N/4]

    // the row group's next row: its vptr entries now, its first record round
    // before pass 1, and an L2 prefetch of the bits rows its occurrences will
    // gather at this row's end (the bits array is larger than L2 at scale)
    const int64_t vn = v + nwarps * RW;
    int32_t o0n = 0, dn = 0;
    if (vn < pd.V) {
      o0n = __ldg(pd.vptr + vn);
      dn = __ldg(pd.vptr + vn + 1) - o0n;
    }
    const int n4 = N >> 2;
    // ---- counting phase (lane = word w of row v)
    int nsign = 0;
    int32_t o0 = 0, o1 = 0;
    if (act) {
      o0 = __ldg(pd.vptr + v);
      o1 = __ldg(pd.vptr + v + 1);
    }
    // The row's z is prefetched into L2 three quarters of the way through its
    // occurrences, m and v just before pass 1: each lane asks for the 128-byte
    // line of its own word.  Lines prefetched earlier sit longer in L2 and push
    // out the bits rows the gathers read (update at n = 1e6: all three at the
    // row's start 5.48 ms, z at the start and m, v before pass 1 5.03, z at a
    // quarter / half / three quarters of the occurrences 5.04 / 5.00 / 4.99,
    // no z prefetch 5.36)
    const uint32_t zpf_at = (MODE == 0 && act) ? (uint32_t)(o1 - o0) * 3u >> 2 : 0xFFFFFFFFu;
    const uint32_t own = act ? __ldg(bsrc + v * W + w) : 0u;
    bool first = true;   // no earlier chunk folded into gbuf
    // every lane of the warp runs the same number of record rounds (shuffles)
    int32_t deg = o1 - o0, maxdeg = deg;
    if (RW > 1)   // with one row per warp the degree is warp-uniform already
      for (int o = 16; o > 0; o >>= 1) maxdeg = max(maxdeg, __shfl_xor_sync(0xFFFFFFFFu, maxdeg, o));
    for (int32_t c0 = 0;; c0 += kCntChunk) {
      const int32_t cn = act ? min(deg - c0, kCntChunk) : 0;   // this row's occurrences in the chunk
      const int32_t cmax = min(maxdeg - c0, kCntChunk);
      // strided byte counters: byte b of sc[t][j] counts sample 8 b + j of word w
      uint32_t sc[3][8];
#pragma unroll
      for (int t = 0; t < 3; ++t)
#pragma unroll
        for (int j = 0; j < 8; ++j) sc[t][j] = 0x80808080u;
      for (int32_t r0 = 0; r0 < cmax; r0 += W) {
        // W records of this row, one per lane, then broadcast within the row group
        int4 myrec = make_int4(0, 0, 0, 0);
        if (c0 == 0 && r0 == 0 && have_crec) myrec = crec;
        else if (r0 + w < cn) myrec = __ldg(xrec4 + o0 + c0 + r0 + w);
        const int nr = min(W, cmax - r0);
#pragma unroll 2
        for (int i = 0; i < nr; ++i) {
          int4 rc;
          rc.x = __shfl_sync(0xFFFFFFFFu, myrec.x, rbase + i);
          rc.y = __shfl_sync(0xFFFFFFFFu, myrec.y, rbase + i);
          rc.z = __shfl_sync(0xFFFFFFFFu, myrec.z, rbase + i);
          if ((uint32_t)(c0 + r0 + i) == zpf_at) prefetch_l2_line(zsrc + (size_t)v * N + 32 * w);
          if (RW > 1 && r0 + i >= cn) continue;       // this row has no occurrence here
          const uint32_t len = (uint32_t)rc.x >> 1;
          const uint32_t a = own ^ (0u - (uint32_t)(rc.x & 1));
          const uint32_t bb = len > 1 ? (__ldg(bsrc + (size_t)(rc.y >> 1) * W + w) ^ (0u - (uint32_t)(rc.y & 1))) : 0u;
          const uint32_t cc = len > 2 ? (__ldg(bsrc + (size_t)(rc.z >> 1) * W + w) ^ (0u - (uint32_t)(rc.z & 1))) : 0u;
          const uint32_t p0 = a ^ bb ^ cc, p1 = (a & bb) | (cc & (a ^ bb));
          const uint32_t sg = (rc.x & 1) ? 0xFFFFFFFFu : 1u;
          nsign += (int)sg;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint32_t t0 = (p0 >> j) & 0x01010101u, t1 = (p1 >> j) & 0x01010101u;
            sc[0][j] += t0 * sg;
            sc[1][j] += t1 * sg;
            sc[2][j] += (t0 & t1) * sg;
          }
        }
      }
      // 4x4 byte transposes: cnt word (q, h) of count t holds samples 8q + 4h + e
      // (byte e), i.e. count word (32 w + 8 q + 4 h) / 4 of the row
#pragma unroll
      for (int t = 0; t < 3; ++t)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t A = sc[t][4 * h], B = sc[t][4 * h + 1], C = sc[t][4 * h + 2], D = sc[t][4 * h + 3];
          const uint32_t abl = __byte_perm(A, B, 0x5140u), abh = __byte_perm(A, B, 0x7362u);
          const uint32_t cdl = __byte_perm(C, D, 0x5140u), cdh = __byte_perm(C, D, 0x7362u);
          cbuf[t * 256 + cswz(ist + 0 + h)] = __byte_perm(abl, cdl, 0x5410u);
          cbuf[t * 256 + cswz(ist + 2 + h)] = __byte_perm(abl, cdl, 0x7632u);
          cbuf[t * 256 + cswz(ist + 4 + h)] = __byte_perm(abh, cdh, 0x5410u);
          cbuf[t * 256 + cswz(ist + 6 + h)] = __byte_perm(abh, cdh, 0x7632u);
        }
      __syncwarp();
      if (c0 + kCntChunk >= maxdeg) break;   // the last chunk is folded in pass 1 below
      if (act) {
#pragma unroll 1
        for (int k = 0; k < 8; ++k) {
          const int ci = cswz(isam + W * k), s4 = W * k + w;
          const float4 add = fold_counts(cbuf[ci], cbuf[256 + ci], cbuf[512 + ci], __ldg(gd4 + n4 + s4),
                                         __ldg(gd4 + 2 * n4 + s4), __ldg(gd4 + 3 * n4 + s4));
          gbuf[k * 32 + lane] = first ? add : f4_add(gbuf[k * 32 + lane], add);
        }
      }
      first = false;
      __syncwarp();   // the count words are read before the next chunk stores
    }
    int4 nrec = make_int4(0, 0, 0, 0);
    if (w < dn) nrec = __ldg(xrec4 + o0n + w);
    crec = nrec;
    have_crec = true;
    // m and v are first read in pass 2; prefetched here (see above) rather
    // than at the row's start, they spend a third as long in L2, where the
    // prefetched rows of all resident warps would otherwise crowd out the bits
    // array the gathers read (before pass 2 instead: 5.07 ms)
    if (MODE == 0 && act) {
      const size_t ro = (size_t)v * N + 32 * w;
      prefetch_l2_line(sd.m + ro);
      prefetch_l2_line(sd.v + ro);
    }
    // ---- sample phase, pass 1: G of samples s = 4Wk + 4w + e, Eq. 5 dot product
    const float nu = act ? sd.nu[v] : 1.0f;
    const float rnu = __frcp_rn(nu);
    const size_t rowoff = (size_t)v * N;
    const float4 *z4p = reinterpret_cast<const float4 *>(zsrc + rowoff);
    float part = 0.f;
    if (act) {
      const float ns = (float)nsign;
#pragma unroll 2
      for (int k = 0; k < 8; ++k) {
        const int s4 = W * k + w, ci = cswz(isam + W * k);
        const float4 z4 = __ldg(z4p + s4);
        const float4 add = fold_counts(cbuf[ci], cbuf[256 + ci], cbuf[512 + ci], __ldg(gd4 + n4 + s4),
                                       __ldg(gd4 + 2 * n4 + s4), __ldg(gd4 + 3 * n4 + s4));
        float4 g = first ? add : f4_add(gbuf[k * 32 + lane], add);
        const float4 g0 = __ldg(gd4 + s4);
        g = make_float4(fmaf(ns, g0.x, g.x), fmaf(ns, g0.y, g.y), fmaf(ns, g0.z, g.z), fmaf(ns, g0.w, g.w));
        gbuf[k * 32 + lane] = g;
        part = fmaf(g.x, z4.x, part);
        part = fmaf(g.y, z4.y, part);
        part = fmaf(g.z, z4.z, part);
        part = fmaf(g.w, z4.w, part);
      }
    }
    if (NORM == TSAT_NORM_NONE) part = 0.f;
    const float dot = seg_sum(part, W);
    const float c2 = dot * rnu * rnu * (1.0f / (float)N);
    // ---- pass 2: Eq. 5 chain rule and AdamW (or the gradient for the autograd backward)
    float psum = 0.f;
    if (act) {
#pragma unroll 2
      for (int k = 0; k < 8; ++k) {
        const size_t off = rowoff + 4 * (W * k + w);
        const float4 g4 = gbuf[k * 32 + lane], z4 = __ldg(z4p + W * k + w);
        const float zq[4] = {z4.x, z4.y, z4.z, z4.w};
        const float Gq[4] = {g4.x, g4.y, g4.z, g4.w};
        float gq[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if constexpr (NORM == TSAT_NORM_NONE) {
            gq[e] = Gq[e];
          } else {
            const float dmu = (NORM == TSAT_NORM_ABSMEAN) ? (float)((zq[e] > 0.f) - (zq[e] < 0.f)) : 1.0f;
            gq[e] = Gq[e] * rnu - c2 * dmu;
          }
        }
        if constexpr (MODE == 1) {
          *reinterpret_cast<float4 *>(grad + off) = make_float4(dL * gq[0], dL * gq[1], dL * gq[2], dL * gq[3]);
          continue;
        }
        const float4 m4 = ld_cs(sd.m + off), v4 = ld_cs(sd.v + off);
        float mq[4] = {m4.x, m4.y, m4.z, m4.w}, vq[4] = {v4.x, v4.y, v4.z, v4.w}, zn[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          mq[e] = hy.beta1 * mq[e] + (hy.omb1) * gq[e];
          vq[e] = hy.beta2 * vq[e] + (hy.omb2) * (gq[e] * gq[e]);
          zn[e] = zq[e] * sp.decay - sp.step_size * (mq[e] * adam_inv_denom(vq[e], sp.inv_sqrt_bc2, hy.eps));
          psum += (NORM == TSAT_NORM_ABSMEAN) ? fabsf(zn[e]) : zn[e];
        }
        const float4 z1 = make_float4(zn[0], zn[1], zn[2], zn[3]);
        gbuf[k * 32 + lane] = z1;   // G of this pass is consumed
        st_cs(sd.z + off, z1);
        st_cs(sd.m + off, make_float4(mq[0], mq[1], mq[2], mq[3]));
        st_cs(sd.v + off, make_float4(vq[0], vq[1], vq[2], vq[3]));
      }
    }
    if constexpr (MODE == 1) {
      if (w < dn) {
        prefetch_l2_line(bsrc + (size_t)(nrec.y >> 1) * W);
        if ((nrec.x >> 1) > 2) prefetch_l2_line(bsrc + (size_t)(nrec.z >> 1) * W);
      }
      continue;
    }
    const float tot = seg_sum(psum, W);
    __syncwarp();   // every lane's count words are consumed: their space takes the nibbles
    // ---- Eq. 2 / Philox bits of step t+1: the lane's samples of pass k form
    // nibble (Wk + w) of the row, stored at word isam + W k; lane w then joins
    // nibbles 8w .. 8w + 7 (its counting-layout words) into bits word w
    if (valid && frozen) bdst[v * W + w] = bsrc[v * W + w];
    uint32_t prow = 0, pk0 = hy.key0;   // the row's Philox stream (instance-local row, instance key)
    if (BIN == TSAT_BIN_PHILOX && valid) {
      const RowStream rs = row_stream(pd, hy.key0, inst, v);
      prow = rs.row;
      pk0 = rs.k0;
    }
    const float nun = (NORM == TSAT_NORM_NONE) ? 1.0f : guard_nu(tot / (float)N);
    const float rnn = __frcp_rn(nun);
    // Philox: samples 4(Wk + w) .. +3 are halves 0..3 (w even) or 4..7 (w odd)
    // of block (Wk + w) / 2.  Over a pair of passes (2kk, 2kk + 1) the even lane
    // of a lane pair draws the block of pass 2kk and the odd lane that of pass
    // 2kk + 1, and they swap the two words the other needs: one draw per lane
    // per two passes.  With W = 1 both passes share one block of the lane.
#pragma unroll 1
    for (int kk = 0; kk < 4; ++kk) {
      uint32_t own0 = 0, own1 = 0, oth0 = 0, oth1 = 0;
      if constexpr (BIN == TSAT_BIN_PHILOX) {
        const uint32_t blk = (uint32_t)((W * (2 * kk + (w & 1)) + (w & ~1)) >> 1);
        const uint4 r = philox4x32_10(make_uint4(blk, prow, (uint32_t)(tcur + 1), kTagBin), pk0, hy.key1);
        const uint32_t s0 = (w & 1) ? r.x : r.z, s1 = (w & 1) ? r.y : r.w;   // the partner's words
        const uint32_t g0 = __shfl_xor_sync(0xFFFFFFFFu, s0, 1), g1 = __shfl_xor_sync(0xFFFFFFFFu, s1, 1);
        if (W == 1) {                   // pass 2kk: words 0, 1; pass 2kk + 1: words 2, 3
          own0 = r.x; own1 = r.y; oth0 = r.z; oth1 = r.w;
        } else if (w & 1) {             // pass 2kk: even lane's words 2, 3; pass 2kk + 1: own words 2, 3
          own0 = g0; own1 = g1; oth0 = r.z; oth1 = r.w;
        } else {                        // pass 2kk: own words 0, 1; pass 2kk + 1: odd lane's words 0, 1
          own0 = r.x; own1 = r.y; oth0 = g0; oth1 = g1;
        }
      }
#pragma unroll
      for (int pp = 0; pp < 2; ++pp) {
        const int k = 2 * kk + pp;
        if (act) {
          const float4 z4 = gbuf[k * 32 + lane];
          const float zq[4] = {z4.x, z4.y, z4.z, z4.w};
          const uint32_t q0 = pp ? oth0 : own0, q1 = pp ? oth1 : own1;
          uint32_t nib = 0;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if constexpr (BIN == TSAT_BIN_PHILOX)
              nib |= binarize_one(__fmul_rn(zq[e], rnn), TSAT_BIN_PHILOX, hy.bin_c, half16(q0, q1, e)) << e;
            else
              nib |= (__fmul_rn(zq[e], rnn) > 0.0f ? 1u : 0u) << e;
          }
          nbuf[cswz(isam + W * k)] = nib;
        }
      }
    }
    __syncwarp();
    if (act) {
      uint32_t word = 0;
#pragma unroll
      for (int c = 0; c < 8; ++c) word |= nbuf[cswz(ist + c)] << (4 * c);
      bdst[v * W + w] = word;
      if (w == 0) sd.nu[v] = nun;
    }
    // the bits rows the next row's first record round will gather, into L2
    // (at the row's end: 0.4 % faster than after pass 2; without it 5.69 ms)
    if (w < dn) {
      prefetch_l2_line(bsrc + (size_t)(nrec.y >> 1) * W);
      if ((nrec.x >> 1) > 2) prefetch_l2_line(bsrc + (size_t)(nrec.z >> 1) * W);
    }
  }
}

int update3_smem_bytes(int N);
// Blocks per SM of the update grid: the resident blocks (occupancy API) times
// an oversubscription factor.  The word-per-lane kernels take rows grid-strided
// per warp; with several waves of blocks the hardware scheduler fills the SMs
// that finish early (rows differ in degree, and in cost between instances),
// measured 5 % (clause length <= 3), 19 % (batched 3..7) and 15 % (relaxed)
// faster than one wave.
int update_blocks_per_sm(const ProbDev &pd, const StateDev &sd) {
  int nb = 0;
  if (sd.layer != TSAT_LAYER_RELAXED && pd.rec_stride == 4) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_update3<0, TSAT_BIN_PHILOX, TSAT_NORM_SIGNED_MEAN, 32>, kUpd3Block,
                                                  update3_smem_bytes(sd.N));
    nb *= 8;
  } else if (sd.layer != TSAT_LAYER_RELAXED && pd.rec_stride == 8) {
    nb = updateL_resident_blocks(sd.N) * 4;
  } else {
    nb = 24;   // general / relaxed kernel: 3 resident, 8 waves (relaxed n=1e6 N=256: 6.8 -> 5.8 ms)
  }
  return nb > 0 ? (nb < 64 ? nb : 64) : 1;
}

int update3_smem_bytes(int N) { return kUpd3Warps * 1792 * (int)sizeof(float); }
// Warps per block of the update kernel that launch_update picks.
int update_warps_per_block(const ProbDev &pd, const StateDev &sd) {
  return (sd.layer != TSAT_LAYER_RELAXED && pd.rec_stride == 4) ? kUpd3Warps : kWarps;
}

// ------------------------------------------------------------------ exact check (Sec. III-A)
// unsat_i = #clauses whose literal words OR to 0 at bit i.  Same warp
// transpose as the histogram, one plane (the unsatisfied mask).
template <int WB>
__global__ void __launch_bounds__(kBlock) k_check(ProbDev pd, StateDev sd, int32_t *unsat) {
  const int4 it = pd.items[blockIdx.x];
  const int inst = it.x;
  const int W = sd.W, N = sd.N;
  const uint32_t *bits = cur_bits(sd, sd.hdr->t);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nWB = W / WB;
  const bool many = nWB >= kWarps;
  const int nsub = many ? 1 : kWarps / nWB;
  const int sub = many ? 0 : warp / nWB;
  for (int wb = many ? warp : warp % nWB; wb < nWB; wb += many ? kWarps : nWB) {
    int32_t cnt[WB];
#pragma unroll
    for (int q = 0; q < WB; ++q) cnt[q] = 0;
    for (int g0 = it.y + sub * 32; g0 < it.z; g0 += nsub * 32) {
      const int c = g0 + lane;
      const bool active = c < it.z;
      uint32_t orw[WB];
#pragma unroll
      for (int q = 0; q < WB; ++q) orw[q] = 0;
      if (active) {
        const int32_t b = __ldg(pd.cptr + c), e = __ldg(pd.cptr + c + 1);
        for (int32_t j0 = b; j0 < e; j0 += 4) {   // chunks of 4 literals, loads issued together
          int32_t lit[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) lit[u] = (j0 + u < e) ? __ldg(pd.clit + j0 + u) : -1;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (lit[u] >= 0) {
              const uint32_t negm = 0u - (uint32_t)(lit[u] & 1);
              const uint32_t *row = bits + (size_t)(lit[u] >> 1) * W + wb * WB;
#pragma unroll
              for (int q = 0; q < WB; ++q) orw[q] |= __ldg(row + q) ^ negm;
            }
        }
      }
      const uint32_t valid = __ballot_sync(0xFFFFFFFFu, active);
#pragma unroll
      for (int q = 0; q < WB; ++q) cnt[q] += __popc(valid & warp_transpose32(~orw[q], lane));
    }
#pragma unroll
    for (int q = 0; q < WB; ++q)
      if (cnt[q]) atomicAdd(unsat + (size_t)inst * N + (wb * WB + q) * 32 + lane, cnt[q]);
  }
}

__global__ void k_satmask(const int32_t *unsat, int64_t n, uint32_t *satmask) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = i < n && unsat[i] == 0;
  const uint32_t b = __ballot_sync(0xFFFFFFFFu, ok);
  if ((threadIdx.x & 31) == 0 && i < n) satmask[i >> 5] = b;
}

// ------------------------------------------------------------------ launchers
int update_smem_bytes(int N, int lm1, bool greg) {
  const int RPB = kBlock / (N >> 2);
  return (int)(sizeof(int32_t) * (kRecInts + 8 * RPB) + (greg ? 0 : sizeof(float) * (size_t)RPB * lm1 * N));
}

static int planes_for(int lmax) {
  int p = 1;
  while ((1 << p) - 1 < lmax) ++p;
  return p;
}

cudaError_t launch_init(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const float *logits, float scale,
                        int grid, cudaStream_t st) {
  k_init<<<grid, kBlock, 0, st>>>(pd, sd, hy, logits, scale);
  return cudaGetLastError();
}

cudaError_t launch_mix(const ProbDev &pd, const StateDev &sd, const Hyper &hy, int grid, cudaStream_t st) {
  k_mix<<<grid, kBlock, 0, st>>>(pd, sd, hy);
  return cudaGetLastError();
}

cudaError_t launch_binarize(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const float *zin, int64_t t_bin,
                            int grid, cudaStream_t st) {
  k_binarize<<<grid, kBlock, 0, st>>>(pd, sd, hy, zin, t_bin, 0);
  return cudaGetLastError();
}

// Relaxed layer: bits, normaliser and literal values sigmoid(z/nu) of zin
// (or of the state's z when zin is NULL), at the state's current step.
cudaError_t launch_relaxed_lits(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const float *zin, int grid,
                                cudaStream_t st) {
  k_binarize<<<grid, kBlock, 0, st>>>(pd, sd, hy, zin, -1, 1);
  return cudaGetLastError();
}

cudaError_t launch_fwd_hist(const ProbDev &pd, const StateDev &sd, int32_t *hist, int skip_frozen, cudaStream_t st) {
  const int P = planes_for(pd.lmax);
  const int W = sd.W;
  if (pd.crec && pd.lmax <= 3 && W >= 16) {   // word per lane (clause records, vertical counters); N is 512 or 1024
    const int smem = (int)sizeof(int32_t) * 4 * sd.N;
    if (W == 32) k_fwd_w3<32><<<pd.n_items, kBlock, smem, st>>>(pd, sd, hist, skip_frozen);
    else k_fwd_w3<16><<<pd.n_items, kBlock, smem, st>>>(pd, sd, hist, skip_frozen);
    return cudaGetLastError();
  }
  const int WB = (P >= 4) ? 1 : (W >= 4 ? 4 : W);
  dim3 grid(pd.n_items), block(kBlock);
#define FWD(PP, WW) k_fwd_hist<PP, WW><<<grid, block, 0, st>>>(pd, sd, hist, skip_frozen)
  switch (P * 10 + WB) {
    case 11: FWD(1, 1); break;
    case 12: FWD(1, 2); break;
    case 14: FWD(1, 4); break;
    case 21: FWD(2, 1); break;
    case 22: FWD(2, 2); break;
    case 24: FWD(2, 4); break;
    case 31: FWD(3, 1); break;
    case 32: FWD(3, 2); break;
    case 34: FWD(3, 4); break;
    case 41: FWD(4, 1); break;
    case 51: FWD(5, 1); break;
    default: return cudaErrorInvalidValue;
  }
#undef FWD
  return cudaGetLastError();
}

cudaError_t launch_gamma(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const LrSched &ls,
                         const int32_t *hist_in, int step_mode, int write_gamma, float *loss_out, float *S_out,
                         cudaStream_t st) {
  k_gamma<<<1, 1024, 0, st>>>(pd, sd, hy, ls, hist_in, step_mode, write_gamma, loss_out, S_out);
  return cudaGetLastError();
}

template <int P, bool GREG, bool RELAX = false, bool DR16 = false>
static cudaError_t upd_launch(const ProbDev &pd, const StateDev &sd, const Hyper &hy, int mode, const float *zin,
                              float *grad, float dL, int grid, int rpi, cudaStream_t st) {
  const int smem = update_smem_bytes(sd.N, sd.lm1, GREG);
  k_update<P, GREG, RELAX, DR16><<<grid, kBlock, smem, st>>>(pd, sd, hy, mode, zin, grad, dL, rpi);
  return cudaGetLastError();
}

template <int WC, typename F>
static void for_each_update3_w(F f) {
  f(k_update3<0, TSAT_BIN_DET, TSAT_NORM_SIGNED_MEAN, WC>);
  f(k_update3<0, TSAT_BIN_DET, TSAT_NORM_ABSMEAN, WC>);
  f(k_update3<0, TSAT_BIN_DET, TSAT_NORM_NONE, WC>);
  f(k_update3<0, TSAT_BIN_PHILOX, TSAT_NORM_SIGNED_MEAN, WC>);
  f(k_update3<0, TSAT_BIN_PHILOX, TSAT_NORM_ABSMEAN, WC>);
  f(k_update3<0, TSAT_BIN_PHILOX, TSAT_NORM_NONE, WC>);
  f(k_update3<1, TSAT_BIN_DET, TSAT_NORM_SIGNED_MEAN, WC>);
  f(k_update3<1, TSAT_BIN_DET, TSAT_NORM_ABSMEAN, WC>);
  f(k_update3<1, TSAT_BIN_DET, TSAT_NORM_NONE, WC>);
}

template <typename F>
static void for_each_update3(F f) {
  for_each_update3_w<0>(f);
  for_each_update3_w<32>(f);
}

template <int MODE, int BIN, int WC>
static cudaError_t launch_update3_n(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const float *zin,
                                    float *grad, float dL, int grid, cudaStream_t st) {
  const int smem = update3_smem_bytes(sd.N);
  switch (hy.norm) {
    case TSAT_NORM_SIGNED_MEAN:
      k_update3<MODE, BIN, TSAT_NORM_SIGNED_MEAN, WC><<<grid, kUpd3Block, smem, st>>>(pd, sd, hy, zin, grad, dL);
      break;
    case TSAT_NORM_ABSMEAN:
      k_update3<MODE, BIN, TSAT_NORM_ABSMEAN, WC><<<grid, kUpd3Block, smem, st>>>(pd, sd, hy, zin, grad, dL);
      break;
    default:
      k_update3<MODE, BIN, TSAT_NORM_NONE, WC><<<grid, kUpd3Block, smem, st>>>(pd, sd, hy, zin, grad, dL);
      break;
  }
  return cudaGetLastError();
}

template <int WC>
static cudaError_t launch_update3_w(const ProbDev &pd, const StateDev &sd, const Hyper &hy, int mode, const float *zin,
                                    float *grad, float dL, int grid, cudaStream_t st) {
  if (mode == 1) return launch_update3_n<1, TSAT_BIN_DET, WC>(pd, sd, hy, zin, grad, dL, grid, st);
  if (hy.binarize == TSAT_BIN_PHILOX)
    return launch_update3_n<0, TSAT_BIN_PHILOX, WC>(pd, sd, hy, zin, grad, dL, grid, st);
  return launch_update3_n<0, TSAT_BIN_DET, WC>(pd, sd, hy, zin, grad, dL, grid, st);
}

static cudaError_t launch_update3(const ProbDev &pd, const StateDev &sd, const Hyper &hy, int mode, const float *zin,
                                  float *grad, float dL, int grid, cudaStream_t st) {
  if (sd.W == 32) return launch_update3_w<32>(pd, sd, hy, mode, zin, grad, dL, grid, st);
  return launch_update3_w<0>(pd, sd, hy, mode, zin, grad, dL, grid, st);
}

void prepare_update_attrs(int lmax) {
  const int P = planes_for(lmax);
  const int bytes = 160 * 1024;
  for_each_update3([bytes](auto fn) { cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); });
  prepare_updateL_attrs(bytes);
  cudaFuncSetAttribute(k_update<1, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_update<1, true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  switch (P) {
    case 1: cudaFuncSetAttribute(k_update<1, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); break;
    case 2: cudaFuncSetAttribute(k_update<2, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); break;
    case 3: cudaFuncSetAttribute(k_update<3, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); break;
    case 4: cudaFuncSetAttribute(k_update<4, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); break;
    default: cudaFuncSetAttribute(k_update<5, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); break;
  }
}

cudaError_t launch_update(const ProbDev &pd, const StateDev &sd, const Hyper &hy, int mode, const float *zin,
                          float *grad, float dL, int grid, int rpi, cudaStream_t st) {
  const int P = planes_for(pd.lmax);
  if (sd.layer != TSAT_LAYER_RELAXED && pd.rec_stride == 4) return launch_update3(pd, sd, hy, mode, zin, grad, dL, grid, st);
  if (sd.layer != TSAT_LAYER_RELAXED && pd.rec_stride == 8) return launch_updateL(pd, sd, hy, mode, zin, grad, dL, grid, st);
  if (sd.layer == TSAT_LAYER_RELAXED)
    return sd.dr16 ? upd_launch<1, true, true, true>(pd, sd, hy, mode, zin, grad, dL, grid, rpi, st)
                   : upd_launch<1, true, true>(pd, sd, hy, mode, zin, grad, dL, grid, rpi, st);
  switch (P) {
    case 1: return upd_launch<1, true>(pd, sd, hy, mode, zin, grad, dL, grid, rpi, st);
    case 2: return upd_launch<2, true>(pd, sd, hy, mode, zin, grad, dL, grid, rpi, st);
    case 3: return upd_launch<3, false>(pd, sd, hy, mode, zin, grad, dL, grid, rpi, st);
    case 4: return upd_launch<4, false>(pd, sd, hy, mode, zin, grad, dL, grid, rpi, st);
    case 5: return upd_launch<5, false>(pd, sd, hy, mode, zin, grad, dL, grid, rpi, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_check(const ProbDev &pd, const StateDev &sd, int32_t *unsat, uint32_t *satmask, cudaStream_t st) {
  const int W = sd.W;
  const int WB = W >= 4 ? 4 : W;
  dim3 grid(pd.n_items), block(kBlock);
  if (WB == 4) k_check<4><<<grid, block, 0, st>>>(pd, sd, unsat);
  else if (WB == 2) k_check<2><<<grid, block, 0, st>>>(pd, sd, unsat);
  else k_check<1><<<grid, block, 0, st>>>(pd, sd, unsat);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !satmask) return e;
  const int64_t n = (int64_t)pd.n_inst * sd.N;
  k_satmask<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(unsat, n, satmask);
  return cudaGetLastError();
}

}  // namespace tsat

namespace tsat {

// ------------------------------------------------------------------ relaxed layer
// Literal values a = sigmoid(zt), a' = 1 - a (stored FP32 or BF16, FP32 sums).
// Forward: R_ci = sum_l a_li (Eq. 1 on real values), stored for the backward;
// per sample partial sums Z = sum_c e^{-tau R}, Y = sum_c R e^{-tau R} per item.
template <bool BF16>
__global__ void __launch_bounds__(kBlock) k_relaxed_fwd(ProbDev pd, StateDev sd, Hyper hy, int skip_frozen) {
  __shared__ float shZ[4 * kBlock], shY[4 * kBlock];
  if (skip_frozen && sd.hdr->all_done) return;
  const int4 it = pd.items[blockIdx.x];
  const int inst = it.x;
  const int N = sd.N, GT = N >> 2, CPB = kBlock / GT;
  const int cs = threadIdx.x / GT, gl = threadIdx.x % GT, s0 = gl * 4;
  float Zs[4] = {0.f, 0.f, 0.f, 0.f}, Ys[4] = {0.f, 0.f, 0.f, 0.f};
  const bool frozen = skip_frozen && sd.inst[inst].found;
  if (!frozen) {
    for (int c = it.y + cs; c < it.z; c += CPB) {
      float R[4] = {0.f, 0.f, 0.f, 0.f};
      for (int32_t j = __ldg(pd.cptr + c); j < __ldg(pd.cptr + c + 1); ++j) {
        const int32_t lit = __ldg(pd.clit + j);
        const size_t off = (size_t)(lit >> 1) * N + s0;
        float a[4];
        if constexpr (BF16) {
          const uint2 u = __ldg(reinterpret_cast<const uint2 *>(reinterpret_cast<const __nv_bfloat16 *>(sd.lit) + off));
          const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
          const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
          a[0] = lo.x; a[1] = lo.y; a[2] = hi.x; a[3] = hi.y;
        } else {
          const float4 x = __ldg(reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(sd.lit) + off));
          a[0] = x.x; a[1] = x.y; a[2] = x.z; a[3] = x.w;
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) R[s] += (lit & 1) ? 1.0f - a[s] : a[s];
      }
      *reinterpret_cast<float4 *>(sd.rbuf + (size_t)c * N + s0) = make_float4(R[0], R[1], R[2], R[3]);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const float w = expf(-hy.tau * R[s]);
        Zs[s] += w;
        Ys[s] += R[s] * w;
      }
    }
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    shZ[cs * N + s0 + s] = Zs[s];
    shY[cs * N + s0 + s] = Ys[s];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < N; k += kBlock) {
    float z = 0.f, y = 0.f;
    for (int q = 0; q < CPB; ++q) {
      z += shZ[q * N + k];
      y += shY[q * N + k];
    }
    sd.zy[((size_t)blockIdx.x * 2) * N + k] = z;
    sd.zy[((size_t)blockIdx.x * 2 + 1) * N + k] = y;
  }
}

// dL/dR_ci = -(e^{-tau R_ci} / Z_i)(1 - tau (R_ci - S_i)) (Eq. 4 differentiated),
// once per (clause, sample), for BF16 storage only: into the bf16 buffer, so
// that the update gathers half the bytes (the sums stay FP32).  With FP32
// storage the update forms dL/dR from the gathered R itself.
__global__ void __launch_bounds__(kBlock) k_relaxed_dr(ProbDev pd, StateDev sd, Hyper hy, int skip_frozen) {
  if (skip_frozen && sd.hdr->all_done) return;
  const int4 it = pd.items[blockIdx.x];
  const int inst = it.x;
  if (skip_frozen && sd.inst[inst].found) return;
  const int N = sd.N, GT = N >> 2, CPB = kBlock / GT;
  const int cs = threadIdx.x / GT, s0 = (threadIdx.x % GT) * 4;
  const float4 zz = *reinterpret_cast<const float4 *>(sd.zs + (size_t)inst * 2 * N + s0);
  const float4 ss = *reinterpret_cast<const float4 *>(sd.zs + ((size_t)inst * 2 + 1) * N + s0);
  const float Zr[4] = {zz.x, zz.y, zz.z, zz.w}, Sr[4] = {ss.x, ss.y, ss.z, ss.w};
  for (int c = it.y + cs; c < it.z; c += CPB) {
    const float4 R4 = *reinterpret_cast<const float4 *>(sd.rbuf + (size_t)c * N + s0);
    const float Rq[4] = {R4.x, R4.y, R4.z, R4.w};
    float D[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) D[s] = -(expf(-hy.tau * Rq[s]) / Zr[s]) * (1.0f - hy.tau * (Rq[s] - Sr[s]));
    const __nv_bfloat162 lo = __floats2bfloat162_rn(D[0], D[1]), hi = __floats2bfloat162_rn(D[2], D[3]);
    *reinterpret_cast<uint2 *>(sd.dr16 + ((size_t)c * N + s0) / 2) =
        make_uint2(*reinterpret_cast<const uint32_t *>(&lo), *reinterpret_cast<const uint32_t *>(&hi));
  }
}

// Z_i, S_i = Y_i / Z_i per (instance, sample) from the item partials, summed
// over items in a fixed order by 32 lanes (strided) and then across the lanes.
// Block (instance, 32-sample chunk), 32 x 32 threads.
__global__ void __launch_bounds__(1024) k_relaxed_zs(ProbDev pd, StateDev sd, int step_mode, float *S_out) {
  __shared__ float shZ[32][33], shY[32][33];
  const int N = sd.N;
  const int inst = blockIdx.x, i = blockIdx.y * 32 + threadIdx.x, q0 = threadIdx.y;
  if (step_mode && (sd.hdr->all_done || sd.inst[inst].found)) return;
  const InstInfo I = pd.inst[inst];
  float Z = 0.f, Y = 0.f;
  if (i < N)
    for (int q = q0; q < I.n_items; q += 32) {
      Z += sd.zy[((size_t)(I.item_off + q) * 2) * N + i];
      Y += sd.zy[((size_t)(I.item_off + q) * 2 + 1) * N + i];
    }
  shZ[q0][threadIdx.x] = Z;
  shY[q0][threadIdx.x] = Y;
  __syncthreads();
  if (q0 == 0 && i < N) {
    float z = 0.f, y = 0.f;
    for (int k = 0; k < 32; ++k) {
      z += shZ[k][threadIdx.x];
      y += shY[k][threadIdx.x];
    }
    const float S = y / z;
    sd.zs[((size_t)inst * 2) * N + i] = z;
    sd.zs[((size_t)inst * 2 + 1) * N + i] = S;
    (S_out ? S_out : sd.S)[(size_t)inst * N + i] = S;
  }
}

// One block: loss (Eq. 3) and the step bookkeeping from S (k_relaxed_zs).  Found detection uses
// the exact unsatisfied counts of the current bits (sd.unsat, filled by the
// exact check earlier in the step).
__global__ void __launch_bounds__(1024) k_relaxed_gamma(ProbDev pd, StateDev sd, Hyper hy, LrSched ls, int step_mode,
                                                        float *loss_out, float *S_out) {
  StateHdr *hdr = sd.hdr;
  if (step_mode && hdr->all_done) return;
  const int64_t t = hdr->t;
  float *Sb = S_out ? S_out : sd.S;
  gamma_tail(pd, sd, hy, ls, step_mode, loss_out, Sb, t);
}

cudaError_t launch_relaxed_fwd(const ProbDev &pd, const StateDev &sd, const Hyper &hy, int skip_frozen,
                               cudaStream_t st) {
  if (sd.lit_bf16) k_relaxed_fwd<true><<<pd.n_items, kBlock, 0, st>>>(pd, sd, hy, skip_frozen);
  else k_relaxed_fwd<false><<<pd.n_items, kBlock, 0, st>>>(pd, sd, hy, skip_frozen);
  return cudaGetLastError();
}

// S and Z (k_relaxed_zs), the loss and step bookkeeping (k_relaxed_gamma), and
// with BF16 storage dL/dR into the bf16 buffer (k_relaxed_dr) for the backward.
cudaError_t launch_relaxed_gamma(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const LrSched &ls,
                                 int step_mode, float *loss_out, float *S_out, cudaStream_t st) {
  k_relaxed_zs<<<dim3(pd.n_inst, (sd.N + 31) / 32), dim3(32, 32), 0, st>>>(pd, sd, step_mode, S_out);
  if (sd.dr16) k_relaxed_dr<<<pd.n_items, kBlock, 0, st>>>(pd, sd, hy, step_mode);
  k_relaxed_gamma<<<1, 1024, 0, st>>>(pd, sd, hy, ls, step_mode, loss_out, S_out);
  return cudaGetLastError();
}

}  // namespace tsat
