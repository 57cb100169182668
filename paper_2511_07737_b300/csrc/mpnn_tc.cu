// mpnn_tc.cu -- the proposer's dense layers on the 5th-generation tensor cores
// (tcgen05.mma, BF16 operands, FP32 accumulation in tensor memory).
//
// Y[r][0:64] = act( sum_j X_j[r ^ xr_j][0:K_j] . B_j^T + bias )
//   forward layers: B_j = the weight slice W[:, koff_j : koff_j + K_j] (64 x K_j)
//   input gradient: one slice, B = W[:, koff : koff + 64]^T (the 64 outputs are
//                   the slice's inputs, the reduction runs over W's 64 rows)
//
// The weights are BF16 (the network's declared precision), so B is exact in
// BF16.  The activations are FP32: each is split into three BF16 parts,
// x = hi + mid + lo with hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi -
// mid), exact to about 2^-24 relative, and the three products are
// accumulated into the same FP32 tile -- the layer keeps FP32 accuracy with
// BF16 tensor-core inputs.
//
// A block of 128 threads owns a tile of 128 rows.  Per input slice it stages
// the three BF16 parts of its rows and (once per block) the BF16 weight slices
// into shared memory in the no-swizzle K-major core-matrix layout (8 x 16-byte
// core matrices; K-adjacent ones 128 bytes apart, 8-row groups K/8 x 128 bytes
// apart), makes the writes visible to the tensor core's async proxy, and one
// thread issues 3 x (K/16) MMAs of shape 128 x 64 x 16 into a 64-column tensor
// memory tile; tcgen05.commit signals an mbarrier when they are done.  Every
// wait on the mbarrier is bounded: on time-out the block records an error in
// the caller's flag and leaves after freeing its tensor memory.  The epilogue
// reads the accumulator with tcgen05.ld (warp q: rows 32q .. 32q + 31, one row
// per thread), adds the bias and applies the ReLU.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.h"
#include "kernels.cuh"

namespace tsat {

constexpr int kTcRows = 128;      // rows per tile (MMA M)
constexpr int kTcN = 64;          // outputs (MMA N)
constexpr int kTcMaxK = 192;      // widest input (three 64-wide slices)
constexpr int kTcParts = 3;       // BF16 parts of an FP32 activation
constexpr uint32_t kTcSpinLimit = 1u << 24;

// shared memory: B [64 x kTcMaxK] bf16, A [3 parts][128 x 64] bf16, mbarrier, tmem address
constexpr int kTcBBytes = kTcN * kTcMaxK * 2;
constexpr int kTcABytes = kTcParts * kTcRows * 64 * 2;
constexpr int kTcSmem = kTcBBytes + kTcABytes + 64;

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

struct TcIn {
  const float *x;   // [rows][K]
  int K, xr;        // row r reads x[r ^ xr]
  int koff;         // first column of the slice in W (forward) / of the inputs (input gradient)
};

// TRANSB = false: forward, B_j = W[:, koff_j : koff_j + K_j], Y = act(sum + bias)
// TRANSB = true : input gradient, one slice, B = W[:, koff : koff + 64]^T,
//                 Y[r ^ yxr] = (accumulate ? Y : 0) + sum
template <int NIN, bool TRANSB>
__global__ void __launch_bounds__(kTcRows) k_mp_tc(TcIn i0, TcIn i1, TcIn i2, int64_t M, const __nv_bfloat16 *W,
                                                   int Ktot, const __nv_bfloat16 *bias, int relu, float *Y, int yxr,
                                                   int accumulate, int *err) {
  extern __shared__ __align__(1024) unsigned char smt[];
  unsigned char *sB = smt;                          // [64][Kb] K-major
  unsigned char *sA = smt + kTcBBytes;               // [3][128][64] K-major
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smt + kTcBBytes + kTcABytes);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smt + kTcBBytes + kTcABytes + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  const TcIn in[3] = {i0, i1, i2};
  // B in shared memory: width Kb (the padded widths of the slices)
  int Kp[3], kb0[3], Kb = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    Kp[j] = j < NIN ? (in[j].K + 15) / 16 * 16 : 0;
    kb0[j] = Kb;
    Kb += Kp[j];
  }
  for (int e = tid; e < kTcN * Kb; e += kTcRows) {
    const int n = e / Kb, kk = e - n * Kb;
    int j = 0;
    while (j + 1 < NIN && kk >= kb0[j + 1]) ++j;
    const int k = kk - kb0[j];
    __nv_bfloat16 val = __float2bfloat16_rn(0.f);
    if (k < in[j].K) val = TRANSB ? W[(size_t)k * Ktot + in[j].koff + n] : W[(size_t)n * Ktot + in[j].koff + k];
    *reinterpret_cast<__nv_bfloat16 *>(sB + tc_off(n, kk, Kb)) = val;
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)) : "memory");
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
  const uint32_t mb = smem_u32(mbar), sa = smem_u32(sA), sb = smem_u32(sB);
  uint32_t phase = 0;
  bool ok = true;
  const int64_t ntiles = (M + kTcRows - 1) / kTcRows;
  for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int64_t r0 = tile * kTcRows;
#pragma unroll
    for (int j = 0; j < NIN; ++j) {
      // the three BF16 parts of the slice's activations (rows past M are zero)
      const int K = in[j].K, K16 = Kp[j];
      for (int e = tid; e < kTcRows * K16; e += kTcRows) {
        const int row = e / K16, k = e - row * K16;
        const int64_t r = r0 + row;
        float x = 0.f;
        if (r < M && k < K) x = in[j].x[(size_t)(r ^ in[j].xr) * K + k];
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(hi);
        const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
        const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
        const uint32_t o = tc_off(row, k, K16);
        *reinterpret_cast<__nv_bfloat16 *>(sA + o) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(sA + kTcRows * 64 * 2 + o) = mid;
        *reinterpret_cast<__nv_bfloat16 *>(sA + 2 * kTcRows * 64 * 2 + o) = lo;
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        for (int part = 0; part < kTcParts; ++part)
          for (int ks = 0; ks < K16 / 16; ++ks) {
            const uint64_t ad = tc_desc(sa + part * kTcRows * 64 * 2 + ks * 256, 128, (uint32_t)(K16 / 8) * 128);
            const uint64_t bd = tc_desc(sb + (uint32_t)(kb0[j] / 8) * 128 + ks * 256, 128, (uint32_t)(Kb / 8) * 128);
            tc_mma(tmem, ad, bd, (j > 0 || part > 0 || ks > 0) ? 1u : 0u);
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mb)
                     : "memory");
      }
      ok = tc_wait(mb, phase);   // the slice's MMAs are done: its A tile may be overwritten
      phase ^= 1u;
      if (!ok) break;
    }
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // epilogue: warp q reads rows 32 q .. 32 q + 31 (tensor memory lanes), 64 columns
    const int row = 32 * warp + (tid & 31);
    const int64_t r = r0 + row;
#pragma unroll
    for (int c = 0; c < kTcN; c += 16) {
      float v[16];
      tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
      if (r < M) {
        float *dst = TRANSB ? Y + (size_t)(r ^ yxr) * kTcN + c : Y + (size_t)r * kTcN + c;
#pragma unroll
        for (int q = 0; q < 16; q += 4) {
          float4 o = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
          if (!TRANSB) {
            o.x += __bfloat162float(bias[c + q]);
            o.y += __bfloat162float(bias[c + q + 1]);
            o.z += __bfloat162float(bias[c + q + 2]);
            o.w += __bfloat162float(bias[c + q + 3]);
            if (relu) {
              o.x = fmaxf(o.x, 0.f);
              o.y = fmaxf(o.y, 0.f);
              o.z = fmaxf(o.z, 0.f);
              o.w = fmaxf(o.w, 0.f);
            }
          } else if (accumulate) {
            const float4 p = *reinterpret_cast<const float4 *>(dst + q);
            o.x += p.x;
            o.y += p.y;
            o.z += p.z;
            o.w += p.w;
          }
          *reinterpret_cast<float4 *>(dst + q) = o;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();   // every warp has read the accumulator before the next tile's MMAs
  }
  if (!ok && err && (tid & 31) == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcN) : "memory");
}

// ---------------------------------------------------------------- weight gradient
// part[b][o][k] = sum over block b's rows r of dZ[r][o] X[r ^ xr][k], k < Kt,
// and part[b][o][Kt] = sum of dZ[r][o] (the bias gradient: a column of ones).
// As MMAs: D[k][o] = sum_r X[r][k] dZ[r][o], the rows as the reduction
// dimension (64 per tile, 4 MMAs of K = 16), k in M-tiles of 128 (at most two:
// Kt + 1 <= 193), o as N = 64.  Both operands are FP32 and split into three
// BF16 parts; the six products hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid
// keep the sum at about FP32 accuracy.  The tiles are staged transposed
// (rows contiguous, K-major for the MMA).
constexpr int kWgRows = 64;                                       // rows per tile (MMA reduction)
constexpr int kWgAPart = kTcRows * kWgRows * 2;                   // one part of one k M-tile
constexpr int kWgBPart = kTcN * kWgRows * 2;                      // one part of the dZ tile
constexpr int kWgSmem = 2 * kTcParts * kWgAPart + kTcParts * kWgBPart + 64;

__device__ __forceinline__ void split3(float x, __nv_bfloat16 &hi, __nv_bfloat16 &mid, __nv_bfloat16 &lo) {
  hi = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(hi);
  mid = __float2bfloat16_rn(r1);
  lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
}

__global__ void __launch_bounds__(kTcRows) k_mp_tc_wgrad(const float *dZ, int64_t M, TcIn i0, TcIn i1, TcIn i2,
                                                         int nin, float *part, int *err) {
  extern __shared__ __align__(1024) unsigned char smw[];
  unsigned char *sA = smw;                                   // [2 m-tiles][3 parts][128 k][64 rows]
  unsigned char *sB = smw + 2 * kTcParts * kWgAPart;         // [3 parts][64 o][64 rows]
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sB + kTcParts * kWgBPart);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sB + kTcParts * kWgBPart + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  const TcIn in[3] = {i0, i1, i2};
  const int Kt = i0.K + (nin > 1 ? i1.K : 0) + (nin > 2 ? i2.K : 0);
  const int ncol = Kt + 1, nmt = (ncol + kTcRows - 1) / kTcRows;
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)) : "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(2 * kTcN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t mb = smem_u32(mbar), sa = smem_u32(sA), sb = smem_u32(sB);
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  uint32_t phase = 0;
  bool ok = true, first = true;
  for (int64_t rt = r0; rt < r1 && ok; rt += kWgRows) {
    // X^T tile parts: A[mt][p][k][row]; k = Kt is the ones column, rows past r1 are zero
    for (int e = tid; e < nmt * kTcRows * kWgRows; e += kTcRows) {
      const int kk = e / kWgRows, row = e - kk * kWgRows;
      const int64_t r = rt + row;
      float x = 0.f;
      if (r < r1) {
        if (kk == Kt) {
          x = 1.f;
        } else if (kk < Kt) {
          const int j = kk < in[0].K ? 0 : (kk < in[0].K + in[1].K ? 1 : 2);
          const int k = kk - (j == 0 ? 0 : (j == 1 ? in[0].K : in[0].K + in[1].K));
          x = in[j].x[(size_t)(r ^ in[j].xr) * in[j].K + k];
        }
      }
      __nv_bfloat16 h, m, l;
      split3(x, h, m, l);
      const int mt = kk / kTcRows;
      const uint32_t o = (uint32_t)(mt * kTcParts * kWgAPart) + tc_off(kk - mt * kTcRows, row, kWgRows);
      *reinterpret_cast<__nv_bfloat16 *>(sA + o) = h;
      *reinterpret_cast<__nv_bfloat16 *>(sA + kWgAPart + o) = m;
      *reinterpret_cast<__nv_bfloat16 *>(sA + 2 * kWgAPart + o) = l;
    }
    // dZ^T tile parts: B[p][o][row]
    for (int e = tid; e < kTcN * kWgRows; e += kTcRows) {
      const int row = e / kTcN, oo = e - row * kTcN;
      const int64_t r = rt + row;
      const float z = r < r1 ? dZ[(size_t)r * kTcN + oo] : 0.f;
      __nv_bfloat16 h, m, l;
      split3(z, h, m, l);
      const uint32_t o = tc_off(oo, row, kWgRows);
      *reinterpret_cast<__nv_bfloat16 *>(sB + o) = h;
      *reinterpret_cast<__nv_bfloat16 *>(sB + kWgBPart + o) = m;
      *reinterpret_cast<__nv_bfloat16 *>(sB + 2 * kWgBPart + o) = l;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      // (A part, B part) products kept: hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid
      const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
      for (int mt = 0; mt < nmt; ++mt)
        for (int q = 0; q < 6; ++q)
          for (int ks = 0; ks < kWgRows / 16; ++ks) {
            const uint64_t ad = tc_desc(sa + mt * kTcParts * kWgAPart + pa[q] * kWgAPart + ks * 256, 128,
                                        (uint32_t)(kWgRows / 8) * 128);
            const uint64_t bd = tc_desc(sb + pb[q] * kWgBPart + ks * 256, 128, (uint32_t)(kWgRows / 8) * 128);
            tc_mma(tmem + (uint32_t)(mt * kTcN), ad, bd, (first && q == 0 && ks == 0) ? 0u : 1u);
          }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mb)
                   : "memory");
    }
    first = false;
    ok = tc_wait(mb, phase);
    phase ^= 1u;
  }
  if (ok) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    float *out = part + (size_t)blockIdx.x * kTcN * ncol;
    for (int mt = 0; mt < nmt; ++mt) {
      const int k = mt * kTcRows + 32 * warp + (tid & 31);
#pragma unroll
      for (int c = 0; c < kTcN; c += 16) {
        float v[16];
        tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(mt * kTcN + c), v);
        if (k < ncol)
#pragma unroll
          for (int q = 0; q < 16; ++q) out[(size_t)(c + q) * ncol + k] = first ? 0.f : v[q];
      }
    }
  } else if (err && (tid & 31) == 0) {
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * kTcN) : "memory");
}

// Partial weight gradients of one layer into part[nb][64][Kt + 1]; returns nb.
int mp_wgrad_tc(const float *dZ, int64_t M, int nin, const float *x0, int k0, int xr0, const float *x1, int k1,
                int xr1, const float *x2, int k2, int xr2, float *part, int max_blocks, int *err, cudaStream_t st,
                cudaError_t *e) {
  static bool attr = false;
  if (!attr) {
    *e = cudaFuncSetAttribute(k_mp_tc_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem);
    if (*e != cudaSuccess) return 0;
    attr = true;
  }
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(max_blocks, (M + 4 * kWgRows - 1) / (4 * kWgRows)));
  const TcIn a{x0, k0, xr0, 0}, b{x1, k1, xr1, 0}, c{x2, k2, xr2, 0};
  k_mp_tc_wgrad<<<nb, kTcRows, kWgSmem, st>>>(dZ, M, a, b, c, nin, part, err);
  *e = cudaGetLastError();
  return nb;
}

static int tc_grid(int64_t M) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(148 * 3, (M + kTcRows - 1) / kTcRows));
}

template <int NIN, bool TRANSB>
static cudaError_t tc_go(TcIn a, TcIn b, TcIn c, int64_t M, const __nv_bfloat16 *W, int Ktot,
                         const __nv_bfloat16 *bias, int relu, float *Y, int yxr, int accumulate, int *err,
                         cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_mp_tc<NIN, TRANSB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_mp_tc<NIN, TRANSB><<<tc_grid(M), kTcRows, kTcSmem, st>>>(a, b, c, M, W, Ktot, bias, relu, Y, yxr, accumulate,
                                                              err);
  return cudaGetLastError();
}

// Y[r] = act(sum_j x_j[r ^ xr_j] . W[:, koff_j : koff_j + K_j]^T + bias), W bf16 [64][Ktot]
cudaError_t mp_dense_tc(int nin, const float *x0, int k0, int xr0, const float *x1, int k1, int xr1, const float *x2,
                        int k2, int xr2, int64_t M, const __nv_bfloat16 *W, const __nv_bfloat16 *bias, int relu,
                        float *Y, int *err, cudaStream_t st) {
  const int Ktot = k0 + (nin > 1 ? k1 : 0) + (nin > 2 ? k2 : 0);
  const TcIn a{x0, k0, xr0, 0}, b{x1, k1, xr1, k0}, c{x2, k2, xr2, k0 + k1};
  if (nin == 1) return tc_go<1, false>(a, b, c, M, W, Ktot, bias, relu, Y, 0, 0, err, st);
  if (nin == 2) return tc_go<2, false>(a, b, c, M, W, Ktot, bias, relu, Y, 0, 0, err, st);
  return tc_go<3, false>(a, b, c, M, W, Ktot, bias, relu, Y, 0, 0, err, st);
}

// dX[r ^ xr] (+)= dZ[r] . W[:, koff : koff + 64]   (dZ [M][64], W bf16 [64][Ktot])
cudaError_t mp_dx_tc(const float *dZ, int64_t M, const __nv_bfloat16 *W, int Ktot, int koff, float *dX, int accumulate,
                     int xr, int *err, cudaStream_t st) {
  const TcIn a{dZ, kTcN, 0, koff}, none{nullptr, 0, 0, 0};
  return tc_go<1, true>(a, none, none, M, W, Ktot, nullptr, 0, dX, xr, accumulate, err, st);
}

}  // namespace tsat
