// mpnn_tc.cu -- the proposer's dense layers on the 5th-generation tensor cores
// (tcgen05.mma, BF16 operands, FP32 accumulation in tensor memory).
//
// Layer forms (64 outputs; W is BF16, row-major [64][Ktot]):
//   dense       Y[r]  = relu(W x[r] + b)                          x: K = 3 or 64
//   literal     Y[r]  = relu(W0 h[r] + W1 a[r] + W2 h[r^1] + b)   W = [W0 W1 W2], 64 x 192
//   dx          dX[r] = s[r] W^T dZ[r]                            W: 64 x 64
//   literal dx  dh[r] = W0^T dZ[r] + W2^T dZ[r^1],  da[r] = s[r] W1^T dZ[r]
// (s: a per-row scale, the 1 / count of the mean that the next backward
// gather transposes)
//   weight grad part[b][o][k] = sum over block b's rows r of dZ[r][o] X[r][k],
//               with a column of ones after the last k for the bias gradient.
// Rows r and r^1 are the two literals of a variable.  Tiles start at
// multiples of 128 rows, so both sit in one tile, in adjacent tensor-memory
// lanes of the same warp: the r^1 terms are computed into a second
// accumulator and exchanged between lane pairs (shfl_xor 1) in the epilogue,
// and h and dZ are staged once.
//
// The weights are BF16 (the network's declared precision), so B is exact in
// BF16.  The activations are FP32: each is split into three BF16 parts,
// x = hi + mid + lo with hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi -
// mid), exact to about 2^-24 relative, and the three products are
// accumulated into the same FP32 tile -- the layer keeps FP32 accuracy with
// BF16 tensor-core inputs.
//
// Shared-memory operands use the no-swizzle K-major core-matrix layout (8 x
// 16-byte core matrices; K-adjacent ones 128 bytes apart, 8-row groups K/8 x
// 128 bytes apart).  Forward / dx blocks stage the weights once, then loop
// over 128-row tiles: the tile's FP32 rows arrive by one bulk copy per tile
// (64-wide dense, dx) or by 16-byte vector loads all issued before the first
// conversion, each warp's stores of the BF16 parts cover contiguous shared
// memory, one thread issues the MMAs (M 128, N 64, K 16), and tcgen05.commit
// signals an mbarrier.  Every wait on an mbarrier is bounded, and the outcome
// is decided for the whole block: on time-out the block records an error in the
// caller's flag and leaves after freeing its tensor memory.  The epilogue reads
// the accumulators with tcgen05.ld (warp q: rows 32q .. 32q + 31, one row per
// thread) into an output tile in shared memory, written out whole rows at a time.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.h"
#include "kernels.cuh"

namespace tsat {

constexpr int kTcRows = 128;      // rows per tile (MMA M)
constexpr int kTcN = 64;          // outputs (MMA N)
constexpr int kTcParts = 3;       // BF16 parts of an FP32 activation
constexpr uint32_t kTcSpinLimit = 1u << 24;

// forward / dx shared memory: B [3 blocks][64 x 64] bf16, A [3 parts][128 x 64] bf16, mbarrier, tmem address
constexpr int kTcBBlock = kTcN * 64 * 2;
constexpr int kTcAPart = kTcRows * 64 * 2;
constexpr int kTcSmem = 3 * kTcBBlock + kTcParts * kTcAPart + 64;
// the literal input gradient holds 256 tensor-memory columns, so at most two
// of its blocks may share an SM: its shared memory is padded past a third
constexpr int kTcSmemTwoPerSm = 80 * 1024;

enum TcForm { kDense = 0, kLiteral = 1, kDx = 2, kLiteralDx = 3 };

// Byte offset of element (row, k) in the K-major no-swizzle layout with
// kw = K (row width in elements, a multiple of 8).
__device__ __forceinline__ uint32_t tc_off(int row, int k, int kw) {
  return (uint32_t)((row >> 3) * (kw >> 3) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading byte
// offset (K-adjacent core matrices), stride byte offset (8-row groups), all
// >> 4; bits 46..47 = 1 (this descriptor format); no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor for kind::f16: FP32 accumulator (bits 4..5 = 1),
// A and B BF16 (bits 7..9, 10..12 = 1), both K-major, N >> 3 at bit 17,
// M >> 4 at bit 24.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar) : "memory");
}

// Bounded wait for mbarrier phase `parity`; false on time-out.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t it = 0; it < kTcSpinLimit; ++it) {
    uint32_t done = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 16 consecutive accumulator columns of this thread's row.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16 &hi, __nv_bfloat16 &mid, __nv_bfloat16 &lo) {
  hi = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(hi);
  mid = __float2bfloat16_rn(r1);
  lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// The three parts of two values as packed pairs (first value in the low half).
__device__ __forceinline__ void split3x2(float x, float y, uint32_t &hi, uint32_t &mid, uint32_t &lo) {
  __nv_bfloat16 h0, m0, l0, h1, m1, l1;
  split3(x, h0, m0, l0);
  split3(y, h1, m1, l1);
  hi = pack2(h0, h1);
  mid = pack2(m0, m1);
  lo = pack2(l0, l1);
}

// Rows [r0, r0 + 128) of a 64-wide FP32 matrix (rows at or past M are zero)
// as three BF16 parts, part p at sA + p * kTcAPart.  Warp q covers k in
// [16q, 16q + 16): in load i, lanes 4a .. 4a + 3 read 64 bytes of row 8i + a,
// so every load instruction reads eight 64-byte segments; all 16 loads are
// issued before the first conversion; each warp's 8-byte stores fill 256
// contiguous bytes (two K-adjacent core matrices).
__device__ __forceinline__ void stage_a64(unsigned char *sA, const float *__restrict__ x, int64_t r0, int64_t M,
                                          int tid) {
  const int warp = tid >> 5, lane = tid & 31;
  const int k = 16 * warp + 4 * (lane & 3);
  float4 v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {   // rows past M load row M - 1 and are zeroed, so no load is conditional
    const int64_t r = r0 + 8 * i + (lane >> 2);
    const float4 t = __ldg(reinterpret_cast<const float4 *>(x + (size_t)min(r, M - 1) * 64 + k));
    v[i] = r < M ? t : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const uint32_t o = tc_off(8 * i + (lane >> 2), k, 64);
    uint2 h, m, l;
    split3x2(v[i].x, v[i].y, h.x, m.x, l.x);
    split3x2(v[i].z, v[i].w, h.y, m.y, l.y);
    *reinterpret_cast<uint2 *>(sA + o) = h;
    *reinterpret_cast<uint2 *>(sA + kTcAPart + o) = m;
    *reinterpret_cast<uint2 *>(sA + 2 * kTcAPart + o) = l;
  }
}

// The 3-wide input features: one row per thread, columns 3..15 zero (K 16).
__device__ __forceinline__ void stage_a3(unsigned char *sA, const float *__restrict__ x, int64_t r0, int64_t M,
                                         int tid) {
  const int64_t r = r0 + tid, rc = min(r, M - 1);
  const bool in = r < M;
  const float f0 = in ? __ldg(x + 3 * rc) : 0.f, f1 = in ? __ldg(x + 3 * rc + 1) : 0.f,
              f2 = in ? __ldg(x + 3 * rc + 2) : 0.f;
  uint32_t h01, m01, l01, h2, m2, l2;
  split3x2(f0, f1, h01, m01, l01);
  split3x2(f2, 0.f, h2, m2, l2);
  const uint32_t o = tc_off(tid, 0, 16);
  const uint4 z = make_uint4(0u, 0u, 0u, 0u);
  *reinterpret_cast<uint4 *>(sA + o) = make_uint4(h01, h2, 0u, 0u);
  *reinterpret_cast<uint4 *>(sA + o + 128) = z;
  *reinterpret_cast<uint4 *>(sA + kTcAPart + o) = make_uint4(m01, m2, 0u, 0u);
  *reinterpret_cast<uint4 *>(sA + kTcAPart + o + 128) = z;
  *reinterpret_cast<uint4 *>(sA + 2 * kTcAPart + o) = make_uint4(l01, l2, 0u, 0u);
  *reinterpret_cast<uint4 *>(sA + 2 * kTcAPart + o + 128) = z;
}

// Weight block j as the MMA's B operand [64 n][64 k] at sB + j * kTcBBlock:
//   TRANS = false: B[n][k] = W[n][64 j + k]   (forward)
//   TRANS = true : B[n][k] = W[k][64 j + n]   (input gradient)
// Forward: 16-byte chunk e holds k 8c .. 8c + 7 of row n with n = 8(e >> 6) +
// (e & 7), c = (e >> 3) & 7, which is byte offset 16 e of the layout.
template <bool TRANS>
__device__ __forceinline__ void stage_b64(unsigned char *sB, const __nv_bfloat16 *__restrict__ W, int Ktot, int j,
                                          int tid) {
  unsigned char *dst = sB + j * kTcBBlock;
  uint4 t[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = i * kTcRows + tid;
    if (!TRANS) {
      const int n = ((e >> 6) << 3) | (e & 7), c = (e >> 3) & 7;
      t[i] = __ldg(reinterpret_cast<const uint4 *>(W + (size_t)n * Ktot + 64 * j + 8 * c));
    } else {
      const int k = e & 63, c = e >> 6;
      t[i] = __ldg(reinterpret_cast<const uint4 *>(W + (size_t)k * Ktot + 64 * j + 8 * c));
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = i * kTcRows + tid;
    if (!TRANS) {
      *reinterpret_cast<uint4 *>(dst + 16 * e) = t[i];
    } else {   // the eight n of the chunk go to eight rows of the layout
      const int k = e & 63, c = e >> 6;
      unsigned char *d = dst + tc_off(8 * c, k, 64);
      *reinterpret_cast<unsigned short *>(d + 0 * 16) = (unsigned short)(t[i].x & 0xFFFFu);
      *reinterpret_cast<unsigned short *>(d + 1 * 16) = (unsigned short)(t[i].x >> 16);
      *reinterpret_cast<unsigned short *>(d + 2 * 16) = (unsigned short)(t[i].y & 0xFFFFu);
      *reinterpret_cast<unsigned short *>(d + 3 * 16) = (unsigned short)(t[i].y >> 16);
      *reinterpret_cast<unsigned short *>(d + 4 * 16) = (unsigned short)(t[i].z & 0xFFFFu);
      *reinterpret_cast<unsigned short *>(d + 5 * 16) = (unsigned short)(t[i].z >> 16);
      *reinterpret_cast<unsigned short *>(d + 6 * 16) = (unsigned short)(t[i].w & 0xFFFFu);
      *reinterpret_cast<unsigned short *>(d + 7 * 16) = (unsigned short)(t[i].w >> 16);
    }
  }
}

// The 3-wide input layer's weights: B[n][k] = W[n][k] for k < 3, zero to k 16.
__device__ __forceinline__ void stage_b3(unsigned char *sB, const __nv_bfloat16 *__restrict__ W, int tid) {
  if (tid < kTcN) {
    const __nv_bfloat16 zb = __float2bfloat16_rn(0.f);
    const uint32_t o = tc_off(tid, 0, 16);
    *reinterpret_cast<uint4 *>(sB + o) =
        make_uint4(pack2(W[3 * tid], W[3 * tid + 1]), pack2(W[3 * tid + 2], zb), 0u, 0u);
    *reinterpret_cast<uint4 *>(sB + o + 128) = make_uint4(0u, 0u, 0u, 0u);
  }
}

struct TcArgs {
  const float *x0, *x1;          // A sources: dense / dx: x0; literal: h = x0, a = x1; literal dx: dZ = x0
  int K;                         // dense: width of x0 (3 or 64)
  int64_t M;                     // rows
  const __nv_bfloat16 *W, *bias;
  const float *rscale;           // dx: per-row scale of dX; literal dx: per-row scale of da
  float *y0, *y1;                // outputs: y0 (Y, dX, dh), y1 (literal dx: da)
  int *err;
};

// Output tiles pass through shared memory, rows kOtStride floats apart (the
// row-per-thread writes then spread over the banks): tile_out writes the
// tile's rows below M with 16 lanes per 256-byte row, two rows per warp store.
constexpr int kOtStride = 68;

__device__ __forceinline__ void tile_out(const float *otile, float *y, int64_t r0, int64_t M, int tid) {
#pragma unroll 4
  for (int i = 0; i < kTcRows / 8; ++i) {
    const int rr = 8 * i + (tid >> 4), c4 = 4 * (tid & 15);
    if (r0 + rr < M)
      *reinterpret_cast<float4 *>(y + (size_t)(r0 + rr) * kTcN + c4) =
          *reinterpret_cast<const float4 *>(otile + rr * kOtStride + c4);
  }
}

// MMAs of one staged A tile (3 parts, kA wide) against weight block j into
// the accumulator at tensor-memory column `col`.
__device__ __forceinline__ void tc_mma_tile(uint32_t tmem, uint32_t col, uint32_t sa, uint32_t sb, int j, int kA,
                                            bool first) {
  for (int part = 0; part < kTcParts; ++part)
    for (int ks = 0; ks < kA / 16; ++ks) {
      const uint64_t ad = tc_desc(sa + part * kTcAPart + ks * 256, 128, (uint32_t)(kA / 8) * 128);
      const uint64_t bd = tc_desc(sb + j * kTcBBlock + ks * 256, 128, (uint32_t)(kA / 8) * 128);
      tc_mma(tmem + col, ad, bd, (first && part == 0 && ks == 0) ? 0u : 1u);
    }
}

// The dense layer on the 3-wide input features, the literal layer and the
// literal input gradient: tiles staged by per-thread vector loads (the
// 64-wide dense layer and dx use the bulk-staged k_mp_tcb below).
template <int FORM>
__global__ void __launch_bounds__(kTcRows) k_mp_tc(TcArgs g) {
  constexpr int NB = (FORM == kLiteral || FORM == kLiteralDx) ? 3 : 1;   // weight blocks
  constexpr uint32_t NCOL = FORM == kLiteralDx ? 256 : (FORM == kLiteral ? 128 : 64);   // tensor-memory columns
  extern __shared__ __align__(1024) unsigned char smt[];
  unsigned char *sB = smt;
  unsigned char *sA = smt + 3 * kTcBBlock;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sA + kTcParts * kTcAPart);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sA + kTcParts * kTcAPart + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool k3 = FORM == kDense && g.K == 3;
  const int kA = k3 ? 16 : 64;
  if (k3) {
    stage_b3(sB, g.W, tid);
  } else {
#pragma unroll
    for (int j = 0; j < NB; ++j) stage_b64<FORM == kDx || FORM == kLiteralDx>(sB, g.W, NB * 64, j, tid);
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)) : "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(NCOL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t mb = smem_u32(mbar), sa = smem_u32(sA), sb = smem_u32(sB);
  uint32_t phase = 0;
  bool ok = true;
  const int64_t M = g.M, ntiles = (M + kTcRows - 1) / kTcRows;
  for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int64_t r0 = tile * kTcRows;
    // stage 0: x (dense), dZ (dx, literal dx) or h (literal)
    if (k3)
      stage_a3(sA, g.x0, r0, M, tid);
    else
      stage_a64(sA, g.x0, r0, M, tid);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      if (FORM == kLiteral) {
        tc_mma_tile(tmem, 0, sa, sb, 0, 64, true);     // W0 h[r]
        tc_mma_tile(tmem, 64, sa, sb, 2, 64, true);    // W2 h[r]  (moved to row r^1 in the epilogue)
      } else if (FORM == kLiteralDx) {
        tc_mma_tile(tmem, 0, sa, sb, 0, 64, true);     // W0^T dZ[r]
        tc_mma_tile(tmem, 64, sa, sb, 1, 64, true);    // W1^T dZ[r]
        tc_mma_tile(tmem, 128, sa, sb, 2, 64, true);   // W2^T dZ[r]  (moved to row r^1)
      } else {
        tc_mma_tile(tmem, 0, sa, sb, 0, kA, true);
      }
      tc_commit(mb);
    }
    // the MMAs are done (the A tile may be overwritten); the decision is the
    // whole block's, so no thread leaves the loop while others wait at a barrier
    ok = __syncthreads_and(tc_wait(mb, phase)) != 0;
    phase ^= 1u;
    if (!ok) break;
    if (FORM == kLiteral) {   // stage 1: a
      stage_a64(sA, g.x1, r0, M, tid);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        tc_mma_tile(tmem, 0, sa, sb, 1, 64, false);   // + W1 a[r]
        tc_commit(mb);
      }
      ok = __syncthreads_and(tc_wait(mb, phase)) != 0;
      phase ^= 1u;
      if (!ok) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // epilogue: warp q reads rows 32 q .. 32 q + 31 (tensor memory lanes) into
    // the output tile in shared memory (the A parts are free once the MMAs
    // are done), then the tile goes out two whole rows per warp store; the
    // literal input gradient writes its two outputs one after the other
    float *otile = reinterpret_cast<float *>(sA);
    const int row = 32 * warp + (tid & 31);
    const uint32_t lrow = (uint32_t)(32 * warp) << 16;
#pragma unroll
    for (int c = 0; c < kTcN; c += 16) {
      float v[16];
      tc_ld16(tmem + lrow + (uint32_t)c, v);
      if (FORM == kLiteral || FORM == kLiteralDx) {
        float s[16];
        tc_ld16(tmem + lrow + (uint32_t)(FORM == kLiteral ? 64 : 128) + (uint32_t)c, s);
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] += __shfl_xor_sync(0xFFFFFFFFu, s[q], 1);
      }
#pragma unroll
      for (int q = 0; q < 16; q += 4) {
        float4 o = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
        if (FORM == kDense || FORM == kLiteral) {
          o.x = fmaxf(o.x + __bfloat162float(g.bias[c + q]), 0.f);
          o.y = fmaxf(o.y + __bfloat162float(g.bias[c + q + 1]), 0.f);
          o.z = fmaxf(o.z + __bfloat162float(g.bias[c + q + 2]), 0.f);
          o.w = fmaxf(o.w + __bfloat162float(g.bias[c + q + 3]), 0.f);
        }
        *reinterpret_cast<float4 *>(otile + row * kOtStride + c + q) = o;
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    tile_out(otile, g.y0, r0, M, tid);
    if (FORM == kLiteralDx) {   // da = s W1^T dZ, scaled for the gather that follows
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const float sc = __ldg(g.rscale + min(r0 + row, M - 1));
#pragma unroll
      for (int c = 0; c < kTcN; c += 16) {
        float u[16];
        tc_ld16(tmem + lrow + 64u + (uint32_t)c, u);
#pragma unroll
        for (int q = 0; q < 16; q += 4)
          *reinterpret_cast<float4 *>(otile + row * kOtStride + c + q) =
              make_float4(u[q] * sc, u[q + 1] * sc, u[q + 2] * sc, u[q + 3] * sc);
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncthreads();
      tile_out(otile, g.y1, r0, M, tid);
    }
    __syncthreads();   // the output tile is read before the next tile's parts overwrite it
  }
  if (!ok && g.err && (tid & 31) == 0) atomicExch(g.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NCOL) : "memory");
}

// ---------------------------------------------------------------- bulk-staged forms
// The dense layer with 64-wide input (the clause layer) and the dx form read
// one contiguous FP32 tile per 128 rows (32 KB).  One thread fetches it with a
// 1-D bulk copy (cp.async.bulk, global -> shared, completing on an mbarrier)
// into a staging buffer; as soon as the block has turned the staged rows into
// the three BF16 parts, that thread issues the copy of the block's next tile,
// which then runs under this tile's MMAs and epilogue.  Shared memory: B
// [64 x 64] bf16 | A [3 parts][128 x 64] bf16 | FP32 tile [128][64] | two
// mbarriers (tile copy, MMAs) | tensor-memory address: 88 KB, two blocks per SM.
constexpr int kTbStage = kTcRows * 64 * 4;
constexpr int kTbSmem = kTcBBlock + kTcParts * kTcAPart + kTbStage + 64;

// Copy `bytes` (a multiple of 16) from global `src` to shared `dst`, completing
// on the mbarrier `bar` (one arrival with the byte count).
__device__ __forceinline__ void tb_fetch(uint32_t dst, const float *src, uint32_t bytes, uint32_t bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// The staged rows (row-major [128][64] FP32) as three BF16 parts, with the
// thread mapping of stage_a64 (each warp's stores fill contiguous shared memory).
__device__ __forceinline__ void convert_a64(unsigned char *sA, const float *stg, int tid) {
  const int warp = tid >> 5, lane = tid & 31;
  const int k = 16 * warp + 4 * (lane & 3);
  float4 v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = *reinterpret_cast<const float4 *>(stg + (8 * i + (lane >> 2)) * 64 + k);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const uint32_t o = tc_off(8 * i + (lane >> 2), k, 64);
    uint2 h, m, l;
    split3x2(v[i].x, v[i].y, h.x, m.x, l.x);
    split3x2(v[i].z, v[i].w, h.y, m.y, l.y);
    *reinterpret_cast<uint2 *>(sA + o) = h;
    *reinterpret_cast<uint2 *>(sA + kTcAPart + o) = m;
    *reinterpret_cast<uint2 *>(sA + 2 * kTcAPart + o) = l;
  }
}

// FORM: kDense (64-wide input) or kDx.
template <int FORM>
__global__ void __launch_bounds__(kTcRows) k_mp_tcb(TcArgs g) {
  extern __shared__ __align__(1024) unsigned char smb[];
  unsigned char *sB = smb;
  unsigned char *sA = smb + kTcBBlock;
  float *stg = reinterpret_cast<float *>(sA + kTcParts * kTcAPart);
  uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(stg) + kTbStage);   // copy, MMAs
  uint32_t *tslot = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(stg) + kTbStage + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  stage_b64<FORM == kDx>(sB, g.W, 64, 0, tid);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bars)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bars + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(kTcN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t lb = smem_u32(bars), mb = smem_u32(bars + 1), sa = smem_u32(sA), sb = smem_u32(sB),
                 ss = smem_u32(stg);
  const int64_t M = g.M, ntiles = (M + kTcRows - 1) / kTcRows;
  auto tile_bytes = [&](int64_t t) { return (uint32_t)(min((int64_t)kTcRows, M - t * kTcRows) * 64 * 4); };
  uint32_t lph = 0, mph = 0;
  bool ok = true, pending = false;   // pending: a copy issued and not yet waited for (thread 0)
  int64_t tile = blockIdx.x;
  if (tid == 0 && tile < ntiles) {
    tb_fetch(ss, g.x0 + (size_t)tile * kTcRows * 64, tile_bytes(tile), lb);
    pending = true;
  }
  for (; tile < ntiles && ok; tile += gridDim.x) {
    const int64_t r0 = tile * kTcRows;
    const bool got = tc_wait(lb, lph);
    ok = __syncthreads_and(got) != 0;   // the tile's rows are in shared memory
    if (got) {                          // else the copy may still be in flight: waited for below
      lph ^= 1u;
      pending = false;
    }
    if (!ok) break;
    convert_a64(sA, stg, tid);   // rows past M hold stale values; their outputs are not stored
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();             // the parts are written and the staged rows consumed
    if (tid == 0) {
      const int64_t nt = tile + gridDim.x;
      if (nt < ntiles) {         // the next tile's copy runs under this tile's MMAs and epilogue
        tb_fetch(ss, g.x0 + (size_t)nt * kTcRows * 64, tile_bytes(nt), lb);
        pending = true;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      tc_mma_tile(tmem, 0, sa, sb, 0, 64, true);
      tc_commit(mb);
    }
    ok = __syncthreads_and(tc_wait(mb, mph)) != 0;
    mph ^= 1u;
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // epilogue: the accumulator rows (thread = row) into the output tile in
    // shared memory (the A parts are free once the MMAs are done), then out
    // with each warp writing two whole rows per store
    float *otile = reinterpret_cast<float *>(sA);
    const int row = 32 * warp + (tid & 31);
    const float sc = FORM == kDx ? __ldg(g.rscale + min(r0 + row, M - 1)) : 1.0f;
#pragma unroll
    for (int c = 0; c < kTcN; c += 16) {
      float v[16];
      tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
#pragma unroll
      for (int q = 0; q < 16; q += 4) {
        float4 o;
        if (FORM == kDense)
          o = make_float4(fmaxf(v[q] + __bfloat162float(g.bias[c + q]), 0.f),
                          fmaxf(v[q + 1] + __bfloat162float(g.bias[c + q + 1]), 0.f),
                          fmaxf(v[q + 2] + __bfloat162float(g.bias[c + q + 2]), 0.f),
                          fmaxf(v[q + 3] + __bfloat162float(g.bias[c + q + 3]), 0.f));
        else
          o = make_float4(v[q] * sc, v[q + 1] * sc, v[q + 2] * sc, v[q + 3] * sc);
        *reinterpret_cast<float4 *>(otile + row * kOtStride + c + q) = o;
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();   // the tile is in shared memory; every warp has read the accumulator
    tile_out(otile, g.y0, r0, M, tid);
    __syncthreads();   // the output tile is read before the next tile's parts overwrite it
  }
  if (!ok) {
    if (g.err && (tid & 31) == 0) atomicExch(g.err, 1);
    if (tid == 0 && pending) tc_wait(lb, lph);   // a copy still in flight lands before the block leaves
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcN) : "memory");
}

// ---------------------------------------------------------------- weight gradient
// part[b][o][k] = sum over block b's rows r of dZ[r][o] X[r][k], k < Kt,
// and part[b][o][Kt] = sum of dZ[r][o] (the bias gradient: a column of ones).
// As MMAs: D[k][o] = sum_r X[r][k] dZ[r][o], the rows as the reduction
// dimension (32 per tile, 2 MMAs of K = 16), k in M-tiles of 128 (at most two:
// Kt + 1 <= 193), o as N = 64.  Both operands are FP32 and split into three
// BF16 parts; the six products hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid
// keep the sum at about FP32 accuracy.
// Both tiles are stored transposed (rows contiguous, K-major for the MMA).  A
// warp reads an 8-row x 32-column block as four 8 x 8 pieces in the register
// layout of an 8 x 8 matrix fragment (lane t: row t / 4, columns 2 (t % 4)
// and 2 (t % 4) + 1, one 8-byte load per piece) and writes each piece
// transposed with one stmatrix .trans: row j of piece i (16 bytes: the eight
// rows' values of column 8 i + j) is one row of a core matrix.
constexpr int kWgRows = 32;                                   // rows per tile (MMA reduction)
constexpr int kWgAPart = kTcRows * kWgRows * 2;               // one part of one k M-tile
constexpr int kWgBPart = kTcN * kWgRows * 2;                  // one part of the dZ tile
constexpr int kWgSmem = 2 * kTcParts * kWgAPart + kTcParts * kWgBPart + 64;

__device__ __forceinline__ void stmatrix_t4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "r"(a), "r"(b),
               "r"(c), "r"(d)
               : "memory");
}

// One 8-row x 32-column block of a 64-wide FP32 matrix: rows rt + 8 rg .. +7
// (row r read from row r ^ xr, rows at or past r1 zero), columns cb .. cb + 31.
__device__ __forceinline__ void wg_load(const float *__restrict__ x, int xr, int64_t rt, int64_t r1, int rg, int cb,
                                        int lane, float2 (&v)[4]) {
  // rows past r1 load row r1 - 1 (a row of the block, rt < r1) and are zeroed: no load is conditional
  const int64_t r = rt + 8 * rg + (lane >> 2);
  const float *p = x + (size_t)(min(r, r1 - 1) ^ xr) * 64 + cb + 2 * (lane & 3);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 t = __ldg(reinterpret_cast<const float2 *>(p + 8 * i));
    v[i] = r < r1 ? t : make_float2(0.f, 0.f);
  }
}

// Store the block transposed: column c of the block becomes row m0 + c of a
// K-major operand with 32-wide rows (part p at base + p * pstride).
__device__ __forceinline__ void wg_store(uint32_t base, uint32_t pstride, int m0, int rg, int lane,
                                         const float2 (&v)[4]) {
  uint32_t h[4], m[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) split3x2(v[i].x, v[i].y, h[i], m[i], l[i]);
  const uint32_t a = base + tc_off(m0 + 8 * (lane >> 3) + (lane & 7), 8 * rg, kWgRows);
  stmatrix_t4(a, h[0], h[1], h[2], h[3]);
  stmatrix_t4(a + pstride, m[0], m[1], m[2], m[3]);
  stmatrix_t4(a + 2 * pstride, l[0], l[1], l[2], l[3]);
}

// NIN 64-wide inputs (KIN = 64) or the 3-wide input features (NIN = 1, KIN = 3).
template <int NIN, int KIN>
__global__ void __launch_bounds__(kTcRows) k_mp_tc_wgrad(const float *dZ, int64_t M, const float *x0, int xr0,
                                                         const float *x1, int xr1, const float *x2, int xr2,
                                                         float *part, int *err) {
  constexpr int Kt = NIN * KIN, ncol = Kt + 1, nmt = (ncol + kTcRows - 1) / kTcRows;
  constexpr uint32_t NCOL = nmt * kTcN;
  // X blocks of 8 rows x 32 columns per warp per tile: warp w takes row group
  // w and every 32-column group of the concatenated input
  constexpr int XT = KIN == 64 ? 2 * NIN : 0;
  extern __shared__ __align__(1024) unsigned char smw[];
  unsigned char *sA = smw;                                   // [nmt][3 parts][128 k][32 rows]
  unsigned char *sB = smw + 2 * kTcParts * kWgAPart;         // [3 parts][64 o][32 rows]
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sB + kTcParts * kWgBPart);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sB + kTcParts * kWgBPart + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the X^T operand's rows past the ones column stay zero
  for (int e = tid; e < nmt * kTcParts * kWgAPart / 16; e += kTcRows)
    reinterpret_cast<uint4 *>(sA)[e] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)) : "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(NCOL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t mb = smem_u32(mbar), sa = smem_u32(sA), sb = smem_u32(sB);
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  uint32_t phase = 0;
  bool ok = true, first = true;
  // this warp's X blocks and two dZ blocks of the tile at rt, into registers:
  // the next tile's loads are issued before the wait for this tile's MMAs
  float2 xv[XT > 0 ? XT : 1][4], zv[2][4];
  auto load_tile = [&](int64_t rt) {
#pragma unroll
    for (int i = 0; i < XT; ++i) {   // column group i: input i / 2, columns 32 (i % 2) ..
      const float *xi = i < 2 ? x0 : (i < 4 ? x1 : x2);
      const int xri = i < 2 ? xr0 : (i < 4 ? xr1 : xr2);
      wg_load(xi, xri, rt, r1, warp, 32 * (i & 1), lane, xv[i]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) wg_load(dZ, 0, rt, r1, warp, 32 * i, lane, zv[i]);
  };
  if (r0 < r1) load_tile(r0);
  for (int64_t rt = r0; rt < r1 && ok; rt += kWgRows) {
    if (KIN == 3 && tid < 3 * kWgRows) {   // the 3-wide features, one value per thread
      const int row = tid & (kWgRows - 1), f = tid >> 5;
      const int64_t r = rt + row;
      __nv_bfloat16 h, m, l;
      split3(r < r1 ? __ldg(x0 + 3 * (r ^ xr0) + f) : 0.f, h, m, l);
      const uint32_t o = tc_off(f, row, kWgRows);
      *reinterpret_cast<__nv_bfloat16 *>(sA + o) = h;
      *reinterpret_cast<__nv_bfloat16 *>(sA + kWgAPart + o) = m;
      *reinterpret_cast<__nv_bfloat16 *>(sA + 2 * kWgAPart + o) = l;
    }
    if (tid < kWgRows) {   // the ones column (zero past r1); its mid and lo parts stay zero
      constexpr int mt = Kt / kTcRows;
      const uint32_t o = (uint32_t)(mt * kTcParts * kWgAPart) + tc_off(Kt - mt * kTcRows, tid, kWgRows);
      *reinterpret_cast<__nv_bfloat16 *>(sA + o) = __float2bfloat16_rn(rt + tid < r1 ? 1.f : 0.f);
    }
#pragma unroll
    for (int i = 0; i < XT; ++i) {
      const int k = 32 * i, mt = k / kTcRows;
      wg_store(sa + (uint32_t)(mt * kTcParts * kWgAPart), kWgAPart, k - mt * kTcRows, warp, lane, xv[i]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) wg_store(sb, kWgBPart, 32 * i, warp, lane, zv[i]);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      // (A part, B part) products kept: hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid
      const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
#pragma unroll
      for (int mt = 0; mt < nmt; ++mt)
#pragma unroll
        for (int q = 0; q < 6; ++q)
#pragma unroll
          for (int ks = 0; ks < kWgRows / 16; ++ks) {
            const uint64_t ad = tc_desc(sa + mt * kTcParts * kWgAPart + pa[q] * kWgAPart + ks * 256, 128,
                                        (uint32_t)(kWgRows / 8) * 128);
            const uint64_t bd = tc_desc(sb + pb[q] * kWgBPart + ks * 256, 128, (uint32_t)(kWgRows / 8) * 128);
            tc_mma(tmem + (uint32_t)(mt * kTcN), ad, bd, (first && q == 0 && ks == 0) ? 0u : 1u);
          }
      tc_commit(mb);
    }
    first = false;
    if (rt + kWgRows < r1) load_tile(rt + kWgRows);   // in flight during this tile's MMAs
    ok = __syncthreads_and(tc_wait(mb, phase)) != 0;   // the MMAs are done (block-wide decision)
    phase ^= 1u;
  }
  if (ok) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    float *out = part + (size_t)blockIdx.x * kTcN * ncol;
#pragma unroll
    for (int mt = 0; mt < nmt; ++mt) {
      const int k = mt * kTcRows + 32 * warp + lane;
#pragma unroll
      for (int c = 0; c < kTcN; c += 16) {
        float v[16];
        tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(mt * kTcN + c), v);
        if (k < ncol)
#pragma unroll
          for (int q = 0; q < 16; ++q) out[(size_t)(c + q) * ncol + k] = first ? 0.f : v[q];
      }
    }
  } else if (err && lane == 0) {
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NCOL) : "memory");
}

// ---------------------------------------------------------------- small layers
// A forward layer of at most kFmaRows rows runs on the CUDA cores instead: at
// a few hundred rows the tensor-core kernel's fixed work per block (weights
// staged, tensor memory allocated, one or two staging + MMA + wait rounds)
// takes longer than the layer's whole arithmetic.  A block of 256 threads owns
// 4 rows (their inputs staged in shared memory) and thread (q, o) forms output
// o of row q as an FP32 sum over k of W[o][k] x[k] in k order, reading its
// BF16 weight row through L1 (the layer's weights stay cached there).
// The literal layer's form, x = [h[r], a[r], h[r^1]] with W = [W0 W1 W2], is
// k_mp_fma_literal below (rows r and r^1 share a block: its first row is a
// multiple of 4).
constexpr int kFmaRows = 2048;

// The dot product of the CUDA-core layers: output o of staged row q, over K
// inputs, plus the bias, through the ReLU.
template <int KT>
__device__ __forceinline__ float fma_row(const float (&xs)[4][KT], int q, int o, const __nv_bfloat16 *W, int K,
                                         const __nv_bfloat16 *bias) {
  const __nv_bfloat16 *wr = W + (size_t)o * K;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += 8) {
    const uint4 u = __ldg(reinterpret_cast<const uint4 *>(wr + k0));
    const __nv_bfloat162 *w2 = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 w = __bfloat1622float2(w2[j]);
      acc = fmaf(w.x, xs[q][k0 + 2 * j], acc);
      acc = fmaf(w.y, xs[q][k0 + 2 * j + 1], acc);
    }
  }
  return fmaxf(acc + __bfloat162float(bias[o]), 0.f);
}

// Dense form (the input layer, K = 3, and a 64-wide layer given its inputs);
// the message-passing layers of a small graph use the fused kernels below.
template <int FORM>
__global__ void __launch_bounds__(256) k_mp_fma(TcArgs g) {
  static_assert(FORM == kDense, "CUDA-core form of the dense layer only");
  constexpr int KT = 64;   // inputs per row (K of 3 or 64)
  __shared__ __align__(16) float xs[4][KT];
  const int tid = threadIdx.x, q = tid >> 6, o = tid & 63;
  const int K = g.K;
  for (int64_t r0 = 4 * (int64_t)blockIdx.x; r0 < g.M; r0 += 4 * (int64_t)gridDim.x) {
    __syncthreads();   // the previous rows' readers are done
    for (int e = tid; e < 4 * K; e += 256) {
      const int rq = e / K, k = e - rq * K;
      const int64_t r = r0 + rq;
      float v = 0.f;
      if (r < g.M) v = g.x0[r * (int64_t)K + k];
      xs[rq][k] = v;
    }
    __syncthreads();
    const int64_t r = r0 + q;
    if (r >= g.M) continue;   // the next round's barrier is reached by every thread
    if (K % 8 == 0) {
      g.y0[r * 64 + o] = fma_row<KT>(xs, q, o, g.W, K, g.bias);
    } else {   // the 3-wide input features
      const __nv_bfloat16 *wr = g.W + (size_t)o * K;
      float acc = 0.f;
      for (int k = 0; k < K; ++k) acc = fmaf(__bfloat162float(wr[k]), xs[q][k], acc);
      g.y0[r * 64 + o] = fmaxf(acc + __bfloat162float(g.bias[o]), 0.f);
    }
  }
}

// A small graph's clause layer with its gather in one kernel: the clause
// mean x[c] = cinv[c] sum over the literals l of c of h[l] (summed in the
// clause's literal order, as the separate gather does) is staged, stored to m
// for the backward, and Y[c] = relu(W x[c] + b).
__global__ void __launch_bounds__(256) k_mp_fma_clause(ProbDev pd, const float *h, const float *cinv, float *m,
                                                       const __nv_bfloat16 *W, const __nv_bfloat16 *bias, float *Y) {
  __shared__ __align__(16) float xs[4][64];
  const int tid = threadIdx.x, q = tid >> 6, o = tid & 63;
  const int64_t C = pd.C;
  for (int64_t r0 = 4 * (int64_t)blockIdx.x; r0 < C; r0 += 4 * (int64_t)gridDim.x) {
    __syncthreads();
    {
      const int64_t c = r0 + q;   // element (q, o): clause r0 + q, input o
      float v = 0.f;
      if (c < C) {
        // literal ids, then rows, 8 at a time (loads in flight together)
        const int32_t jb = __ldg(pd.cptr + c), je = __ldg(pd.cptr + c + 1);
        for (int32_t j0 = jb; j0 < je; j0 += 8) {
          int32_t l[8];
          float x[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) l[u] = j0 + u < je ? __ldg(pd.clit + j0 + u) : -1;
#pragma unroll
          for (int u = 0; u < 8; ++u) x[u] = l[u] >= 0 ? __ldg(h + (int64_t)l[u] * 64 + o) : 0.f;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (l[u] >= 0) v += x[u];
        }
        v *= __ldg(cinv + c);
        m[c * 64 + o] = v;
      }
      xs[q][o] = v;
    }
    __syncthreads();
    const int64_t c = r0 + q;
    if (c < C) Y[c * 64 + o] = fma_row<64>(xs, q, o, W, 64, bias);
  }
}

// A small graph's literal layer with its gather: a[r] = linv[r] sum over the
// clauses c holding literal r of e[c] (in occurrence order, as the separate
// gather does) is staged with h[r] and h[r^1], stored to a for the backward,
// and Y[r] = relu(W0 h[r] + W1 a[r] + W2 h[r^1] + b).
__global__ void __launch_bounds__(256) k_mp_fma_literal(ProbDev pd, const float *h, const float *e,
                                                        const float *linv, float *a, const __nv_bfloat16 *W,
                                                        const __nv_bfloat16 *bias, float *Y) {
  __shared__ __align__(16) float xs[4][192];
  const int tid = threadIdx.x, q = tid >> 6, o = tid & 63;
  const int64_t L = 2 * (int64_t)pd.V;
  for (int64_t r0 = 4 * (int64_t)blockIdx.x; r0 < L; r0 += 4 * (int64_t)gridDim.x) {
    __syncthreads();
    {
      const int64_t r = r0 + q;   // element (q, o) of each of the three inputs
      float hv = 0.f, av = 0.f, hp = 0.f;
      if (r < L) {
        hv = __ldg(h + r * 64 + o);
        hp = __ldg(h + (r ^ 1) * 64 + o);
        const int64_t v = r >> 1;
        const int32_t sgn = (int32_t)(r & 1);
        // occurrence records, then the matching clauses' rows, 8 at a time
        const int32_t jb = __ldg(pd.vptr + v), je = __ldg(pd.vptr + v + 1);
        for (int32_t j0 = jb; j0 < je; j0 += 8) {
          int32_t oc[8];
          float x[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) oc[u] = j0 + u < je ? __ldg(pd.vocc + j0 + u) : -1;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            x[u] = (oc[u] >= 0 && (oc[u] & 1) == sgn) ? __ldg(e + (int64_t)(oc[u] >> 1) * 64 + o) : 0.f;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (oc[u] >= 0 && (oc[u] & 1) == sgn) av += x[u];
        }
        av *= __ldg(linv + r);
        a[r * 64 + o] = av;
      }
      xs[q][o] = hv;
      xs[q][64 + o] = av;
      xs[q][128 + o] = hp;
    }
    __syncthreads();
    const int64_t r = r0 + q;
    if (r < L) Y[r * 64 + o] = fma_row<192>(xs, q, o, W, 192, bias);
  }
}

cudaError_t mp_clause_small(const ProbDev &pd, const float *h, const float *cinv, float *m, const __nv_bfloat16 *W,
                            const __nv_bfloat16 *bias, float *Y, cudaStream_t st) {
  k_mp_fma_clause<<<(int)std::max<int64_t>(1, ((int64_t)pd.C + 3) / 4), 256, 0, st>>>(pd, h, cinv, m, W, bias, Y);
  return cudaGetLastError();
}

cudaError_t mp_literal_small(const ProbDev &pd, const float *h, const float *e, const float *linv, float *a,
                             const __nv_bfloat16 *W, const __nv_bfloat16 *bias, float *Y, cudaStream_t st) {
  k_mp_fma_literal<<<(int)std::max<int64_t>(1, (2 * (int64_t)pd.V + 3) / 4), 256, 0, st>>>(pd, h, e, linv, a, W,
                                                                                           bias, Y);
  return cudaGetLastError();
}

// Rows up to which a message-passing layer takes the fused CUDA-core kernel:
// 2,048 for the clause layer, 1,536 for the literal layer, whose per-row work
// (the literal mean walks the variable's occurrences, and 192 inputs) is
// larger (forward back to back: one n = 1,000 instance, 2,000 literal rows,
// 86.2 us with the literal layer on the CUDA cores, 76.7 us on the tensor
// cores; n = 600, 1,200 rows, 76.0 against 77.9 us; n = 300, 600 literal and
// 1,278 clause rows, 55.5 us against 77.0 us with both on the tensor cores).
int mp_small_rows(bool literal) { return literal ? 1536 : kFmaRows; }

template <int FORM>
static cudaError_t fma_go(const TcArgs &g, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, (g.M + 3) / 4);
  k_mp_fma<FORM><<<grid, 256, 0, st>>>(g);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- host side
static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

template <int FORM>
static cudaError_t tc_go(const TcArgs &g, cudaStream_t st) {
  const int smem = FORM == kLiteralDx ? kTcSmemTwoPerSm : kTcSmem;
  cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(k_mp_tc<FORM>), smem);
  if (e != cudaSuccess) return e;
  const int per_sm = FORM == kLiteralDx ? 2 : 3;   // as many as shared and tensor memory allow
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(148 * per_sm, (g.M + kTcRows - 1) / kTcRows));
  k_mp_tc<FORM><<<grid, kTcRows, smem, st>>>(g);
  return cudaGetLastError();
}

template <int FORM>
static cudaError_t tb_go(const TcArgs &g, cudaStream_t st) {
  cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(k_mp_tcb<FORM>), kTbSmem);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(148 * 2, (g.M + kTcRows - 1) / kTcRows));
  k_mp_tcb<FORM><<<grid, kTcRows, kTbSmem, st>>>(g);
  return cudaGetLastError();
}

// The shared-memory limits of the forward's tensor-core kernels, set ahead of
// a graph capture of the forward.
cudaError_t mp_prepare_forward() {
  cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(k_mp_tc<kDense>), kTcSmem);
  if (e == cudaSuccess) e = ensure_dyn_smem(reinterpret_cast<const void *>(k_mp_tc<kLiteral>), kTcSmem);
  if (e == cudaSuccess) e = ensure_dyn_smem(reinterpret_cast<const void *>(k_mp_tcb<kDense>), kTbSmem);
  return e;
}

// Y[r] = relu(W x[r] + b), x FP32 [M][K] with K = 3 or 64, W bf16 [64][K]
cudaError_t mp_dense_tc(const float *x, int K, int64_t M, const __nv_bfloat16 *W, const __nv_bfloat16 *bias, float *Y,
                        int *err, cudaStream_t st) {
  if ((K != 3 && K != 64) || !aligned16(x) || !aligned16(W) || !aligned16(Y)) return cudaErrorInvalidValue;
  const TcArgs g{x, nullptr, K, M, W, bias, nullptr, Y, nullptr, err};
  if (M <= kFmaRows) return fma_go<kDense>(g, st);
  return K == 64 ? tb_go<kDense>(g, st) : tc_go<kDense>(g, st);
}

// Y[r] = relu(W0 h[r] + W1 a[r] + W2 h[r^1] + b), W bf16 [64][192], M even
cudaError_t mp_literal_tc(const float *h, const float *a, int64_t M, const __nv_bfloat16 *W, const __nv_bfloat16 *bias,
                          float *Y, int *err, cudaStream_t st) {
  if ((M & 1) || !aligned16(h) || !aligned16(a) || !aligned16(W) || !aligned16(Y)) return cudaErrorInvalidValue;
  return tc_go<kLiteral>(TcArgs{h, a, 64, M, W, bias, nullptr, Y, nullptr, err}, st);
}

// dX[r] = rscale[r] W^T dZ[r], W bf16 [64][64]
cudaError_t mp_dx_tc(const float *dZ, int64_t M, const __nv_bfloat16 *W, const float *rscale, float *dX, int *err,
                     cudaStream_t st) {
  if (!rscale || !aligned16(dZ) || !aligned16(W) || !aligned16(dX)) return cudaErrorInvalidValue;
  return tb_go<kDx>(TcArgs{dZ, nullptr, 64, M, W, nullptr, rscale, dX, nullptr, err}, st);
}

// dh[r] = W0^T dZ[r] + W2^T dZ[r^1], da[r] = rscale[r] W1^T dZ[r], W bf16 [64][192], M even
cudaError_t mp_literal_dx_tc(const float *dZ, int64_t M, const __nv_bfloat16 *W, const float *rscale, float *dh,
                             float *da, int *err, cudaStream_t st) {
  if ((M & 1) || !rscale || !aligned16(dZ) || !aligned16(W) || !aligned16(dh) || !aligned16(da))
    return cudaErrorInvalidValue;
  return tc_go<kLiteralDx>(TcArgs{dZ, nullptr, 64, M, W, nullptr, rscale, dh, da, err}, st);
}

template <int NIN, int KIN>
static cudaError_t wg_go(const float *dZ, int64_t M, const float *const *x, const int *xr, float *part, int nb,
                         int *err, cudaStream_t st) {
  cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(k_mp_tc_wgrad<NIN, KIN>), kWgSmem);
  if (e != cudaSuccess) return e;
  k_mp_tc_wgrad<NIN, KIN><<<nb, kTcRows, kWgSmem, st>>>(dZ, M, x[0], xr[0], x[1], xr[1], x[2], xr[2], part, err);
  return cudaGetLastError();
}

// Partial weight gradients of one layer into part[nb][64][K nin + 1] (nin
// 64-wide inputs, or nin = 1 with the 3-wide features); returns nb.
int mp_wgrad_tc(const float *dZ, int64_t M, int nin, int K, const float *const *x, const int *xr, float *part,
                int max_blocks, int *err, cudaStream_t st, cudaError_t *e) {
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(max_blocks, (M + 16 * kWgRows - 1) / (16 * kWgRows)));
  bool al = aligned16(dZ);
  for (int i = 0; i < nin; ++i) al = al && aligned16(x[i]);
  const float *xx[3] = {x[0], nin > 1 ? x[1] : nullptr, nin > 2 ? x[2] : nullptr};
  const int rr[3] = {xr[0], nin > 1 ? xr[1] : 0, nin > 2 ? xr[2] : 0};
  if (!al)
    *e = cudaErrorInvalidValue;
  else if (nin == 1 && K == 3)
    *e = wg_go<1, 3>(dZ, M, xx, rr, part, nb, err, st);
  else if (nin == 1 && K == 64)
    *e = wg_go<1, 64>(dZ, M, xx, rr, part, nb, err, st);
  else if (nin == 3 && K == 64)
    *e = wg_go<3, 64>(dZ, M, xx, rr, part, nb, err, st);
  else
    *e = cudaErrorInvalidValue;
  return nb;
}

}  // namespace tsat
