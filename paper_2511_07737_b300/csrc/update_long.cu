// update_long.cu -- the fused update for clause length 4..7 (Sec. III-B
// straight-through backward through P^T, Eq. 5 chain rule, AdamW with the
// Sec. IV-A schedule, Eq. 2 / Philox re-binarisation), word per lane.
#include "kernels.cuh"

namespace tsat {

// ------------------------------------------------------------------ fused update, clause length 4..7
// Word per lane like k_update3, with fixed 8-int records {hdr, lit x 6, 0}.
// Counting phase: for every occurrence the lane gathers the other literals'
// words, forms the bit-sliced R planes (3 planes, R <= 7) and adds
// sign * gamma_i[R_i] to one FP32 accumulator per sample, looking gamma up in
// a per-warp shared-memory table laid out [sample][8] with an 8-float skew per
// word so that the 32 lanes of one lookup (same bit position, any words, any
// R) hit distinct banks or the same address when W <= 4 (N <= 128); larger N
// reads the table through L1.  The accumulators go to shared memory
// bit-major ([32][33]) and the sample phase (Eq. 5, AdamW, bits) reads them
// back with each lane owning 4 consecutive samples per pass.  A row group
// whose rows span several instances is processed once per instance.
constexpr int kGS = 33;   // padded row of the [32 bits][32 lanes] buffer

__device__ __forceinline__ int ltab_off(int s) { return 8 * s + 8 * ((s >> 5) & 3); }
__host__ __device__ __forceinline__ int updateL_tab_floats(int N) { return N <= 128 ? 8 * N + 32 : 0; }
// Per-warp shared memory in floats: the table first, rounded up to 256 bytes,
// then the [32][33] G buffer; every warp's region starts on a 256-byte
// boundary (relative to the dynamic shared memory), which the byte-permute
// addressing of the lookups needs.
__host__ __device__ __forceinline__ int updateL_tab_span(int N) { return (updateL_tab_floats(N) + 63) / 64 * 64; }
__host__ __device__ __forceinline__ int updateL_warp_floats(int N) {
  return (updateL_tab_span(N) + 32 * kGS + 63) / 64 * 64;
}

// gamma_i[R] of the 4 samples 8b + j (b = 0..3) of one lane's word, with
// R as bytes of q: byte b of q = 4 R + the lane's skew (0, 32, 64 or 96:
// 8 floats per word, the bank skew of the table).  The byte and the lane's
// word base (a multiple of 256 bytes) make the address in one byte permute,
// and the sample's offset 32 (8b + j) bytes is an immediate of the load.
template <int J>
__device__ __forceinline__ void ltab_lookup4(const char *smb, uint32_t tbase, uint32_t q, float sg, float (&acc)[32]) {
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const uint32_t off = __byte_perm(q, tbase, 0x7650u | (uint32_t)b);
    const float gv = *reinterpret_cast<const float *>(smb + off + 32 * (8 * b + J));
    acc[8 * b + J] = fmaf(sg, gv, acc[8 * b + J]);
  }
}

// Byte b of the result: 4 R + skew for the sample at bit 8b + J, from R's
// three bit planes (R bit p of sample s is bit s of plane p).
template <int J>
__device__ __forceinline__ uint32_t ltab_rbytes(uint32_t p0, uint32_t p1, uint32_t p2, uint32_t skew) {
  const uint32_t x0 = (J >= 2 ? (p0 >> (J - 2)) : (p0 << (2 - J))) & 0x04040404u;
  const uint32_t x1 = (J >= 3 ? (p1 >> (J - 3)) : (p1 << (3 - J))) & 0x08080808u;
  const uint32_t x2 = (J >= 4 ? (p2 >> (J - 4)) : (p2 << (4 - J))) & 0x10101010u;
  return x0 | x1 | x2 | skew;
}

template <int MODE, int BIN, int NORM, bool STAB>
__global__ void __launch_bounds__(kBlock, 3) k_updateL(ProbDev pd, StateDev sd, Hyper hy, const float *zin, float *grad,
                                                       float dL) {
  extern __shared__ __align__(16) float smL[];
  const StateHdr *hdr = sd.hdr;
  if (MODE == 0 && hdr->all_done) return;
  const int N = sd.N, W = sd.W, RW = 32 / W, lm1 = sd.lm1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rsub = lane / W, w = lane % W, rbase = rsub * W;
  float *tab = smL + warp * updateL_warp_floats(N);   // [N][8] + skew: gamma of the warp's current instance
  float *gbuf = tab + updateL_tab_span(N);            // [32 bits][33]: G, then z(t+1)
  // the lane's word of the table as a byte offset from the start of dynamic
  // shared memory (a multiple of 256: the warp's region plus 1024 bytes per
  // word), and its bank skew replicated in every byte
  const char *smb = reinterpret_cast<const char *>(smL);
  const uint32_t tbase = (uint32_t)(warp * updateL_warp_floats(N) * 4 + 1024 * w);
  const uint32_t tskew = 0x01010101u * (32u * (uint32_t)(w & 3));
  int tinst = -1;
  StepParams sp;
  if (MODE == 0) sp = *sd.sp;
  if (MODE == 0 && sp.mix_now) return;   // this step mixes assignments (k_mix)
  const int64_t tcur = (MODE == 0) ? sp.t : hdr->t;
  const uint32_t *bsrc = cur_bits(sd, tcur);
  uint32_t *bdst = const_cast<uint32_t *>(cur_bits(sd, tcur + 1));
  const float *zsrc = (MODE == 0) ? sd.z : zin;
  const int4 *xrec8 = reinterpret_cast<const int4 *>(pd.xrec);   // two int4 per occurrence
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  for (int64_t base = ((int64_t)blockIdx.x * kWarps + warp) * RW; base < pd.V; base += nwarps * RW) {
    const int64_t v = base + rsub;
    const bool valid = v < pd.V;
    const int inst = valid ? __ldg(pd.var_inst + v) : INT_MAX;
    bool todo = valid;
    while (__any_sync(0xFFFFFFFFu, todo)) {
      // the lowest instance among the rows not yet done
      int cur = todo ? inst : INT_MAX;
      for (int o = 16; o > 0; o >>= 1) cur = min(cur, __shfl_xor_sync(0xFFFFFFFFu, cur, o));
      const bool mine = todo && inst == cur;
      todo = todo && !mine;
      __syncwarp();   // readers of the previous table / gbuf are done
      const bool frozen = mine && MODE == 0 && sd.inst[cur].found;
      const bool act = mine && !frozen;
      if (STAB && cur != tinst) {
        const float *gsrc = sd.gamma + (size_t)cur * lm1 * N;
        for (int k = lane; k < 8 * N; k += 32) {
          const int ss = k >> 3, r = k & 7;
          tab[ltab_off(ss) + r] = r < lm1 ? gsrc[(size_t)r * N + ss] : 0.f;
        }
        tinst = cur;
        __syncwarp();
      }
      const float *gglob = sd.gamma + (size_t)cur * lm1 * N + 32 * w;
      if (MODE == 0 && act && w == 0) {
        const size_t ro = (size_t)v * N;
        prefetch_l2(zsrc + ro, N * 4);
        prefetch_l2(sd.m + ro, N * 4);
        prefetch_l2(sd.v + ro, N * 4);
      }
      // ---- counting phase: G of the lane's 32 samples, bit position 8b + j in acc[8b + j]
      float acc[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[i] = 0.f;
      int32_t o0 = 0, deg = 0;
      if (act) {
        o0 = __ldg(pd.vptr + v);
        deg = __ldg(pd.vptr + v + 1) - o0;
      }
      const uint32_t own = act ? __ldg(bsrc + v * W + w) : 0u;
      int4 ra_n = make_int4(0, 0, 0, 0), rb_n = ra_n;
      if (deg > 0) {
        ra_n = __ldg(xrec8 + 2 * (int64_t)o0);
        rb_n = __ldg(xrec8 + 2 * (int64_t)o0 + 1);
      }
#pragma unroll 1
      for (int32_t i = 0; i < deg; ++i) {
        const int4 ra = ra_n, rb = rb_n;
        if (i + 1 < deg) {
          ra_n = __ldg(xrec8 + 2 * (int64_t)(o0 + i + 1));
          rb_n = __ldg(xrec8 + 2 * (int64_t)(o0 + i + 1) + 1);
        }
        if (i + 8 < deg) prefetch_l2_line(xrec8 + 2 * (int64_t)(o0 + i + 8));
        const int len = ra.x >> 1;
        const int lits[6] = {ra.y, ra.z, ra.w, rb.x, rb.y, rb.z};
        uint32_t pl[3] = {own ^ (0u - (uint32_t)(ra.x & 1)), 0u, 0u};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          if (q + 1 < len) {
            const uint32_t x = __ldg(bsrc + (size_t)(lits[q] >> 1) * W + w) ^ (0u - (uint32_t)(lits[q] & 1));
            bitslice_add<3>(pl, x);
          }
        }
        const float sg = (ra.x & 1) ? -1.0f : 1.0f;
        if constexpr (STAB) {
          ltab_lookup4<0>(smb, tbase, ltab_rbytes<0>(pl[0], pl[1], pl[2], tskew), sg, acc);
          ltab_lookup4<1>(smb, tbase, ltab_rbytes<1>(pl[0], pl[1], pl[2], tskew), sg, acc);
          ltab_lookup4<2>(smb, tbase, ltab_rbytes<2>(pl[0], pl[1], pl[2], tskew), sg, acc);
          ltab_lookup4<3>(smb, tbase, ltab_rbytes<3>(pl[0], pl[1], pl[2], tskew), sg, acc);
          ltab_lookup4<4>(smb, tbase, ltab_rbytes<4>(pl[0], pl[1], pl[2], tskew), sg, acc);
          ltab_lookup4<5>(smb, tbase, ltab_rbytes<5>(pl[0], pl[1], pl[2], tskew), sg, acc);
          ltab_lookup4<6>(smb, tbase, ltab_rbytes<6>(pl[0], pl[1], pl[2], tskew), sg, acc);
          ltab_lookup4<7>(smb, tbase, ltab_rbytes<7>(pl[0], pl[1], pl[2], tskew), sg, acc);
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            // R of the samples at bit positions j, 8 + j, 16 + j, 24 + j, one per byte
            const uint32_t r4 = ((pl[0] >> j) & 0x01010101u) + 2u * ((pl[1] >> j) & 0x01010101u) +
                                4u * ((pl[2] >> j) & 0x01010101u);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const int r = (int)((r4 >> (8 * b)) & 0xFFu);
              acc[8 * b + j] = fmaf(sg, __ldg(gglob + (size_t)r * N + 8 * b + j), acc[8 * b + j]);
            }
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 32; ++i) gbuf[i * kGS + lane] = acc[i];
      __syncwarp();
      // ---- sample phase: lane w holds samples s = 4Wk + 4w + e; G of sample s
      // lives at gbuf[(s % 32) * 33 + rbase + s / 32]
      const float nu = act ? sd.nu[v] : 1.0f;
      const float rnu = __frcp_rn(nu);
      const size_t rowoff = (size_t)v * N;
      float part = 0.f;
      if (NORM != TSAT_NORM_NONE && act) {
#pragma unroll 1
        for (int k = 0; k < 8; ++k) {
          const int s = 4 * W * k + 4 * w;
          const float4 z4 = __ldg(reinterpret_cast<const float4 *>(zsrc + rowoff + s));
          const float *gp = gbuf + (s & 31) * kGS + rbase + (s >> 5);
          part = fmaf(gp[0], z4.x, part);
          part = fmaf(gp[kGS], z4.y, part);
          part = fmaf(gp[2 * kGS], z4.z, part);
          part = fmaf(gp[3 * kGS], z4.w, part);
        }
      }
      const float dot = seg_sum(part, W);
      const float c2 = dot * rnu * rnu * (1.0f / (float)N);
      float psum = 0.f;
      if (act) {
#pragma unroll 1
        for (int k = 0; k < 8; ++k) {
          const int s = 4 * W * k + 4 * w;
          const size_t off = rowoff + s;
          float *gp = gbuf + (s & 31) * kGS + rbase + (s >> 5);
          const float4 z4 = __ldg(reinterpret_cast<const float4 *>(zsrc + off));
          const float zq[4] = {z4.x, z4.y, z4.z, z4.w};
          float gq[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float G = gp[e * kGS];
            if constexpr (NORM == TSAT_NORM_NONE) {
              gq[e] = G;
            } else {
              const float dmu = (NORM == TSAT_NORM_ABSMEAN) ? (float)((zq[e] > 0.f) - (zq[e] < 0.f)) : 1.0f;
              gq[e] = G * rnu - c2 * dmu;
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
            gp[e * kGS] = zn[e];
            psum += (NORM == TSAT_NORM_ABSMEAN) ? fabsf(zn[e]) : zn[e];
          }
          st_cs(sd.z + off, make_float4(zn[0], zn[1], zn[2], zn[3]));
          st_cs(sd.m + off, make_float4(mq[0], mq[1], mq[2], mq[3]));
          st_cs(sd.v + off, make_float4(vq[0], vq[1], vq[2], vq[3]));
        }
      }
      if constexpr (MODE == 1) continue;
      const float tot = seg_sum(psum, W);
      __syncwarp();
      // ---- Eq. 2 / Philox bits of step t+1: lane w assembles word w (bits b of gbuf)
      if (frozen) bdst[v * W + w] = bsrc[v * W + w];
      if (act) {
        const float nun = (NORM == TSAT_NORM_NONE) ? 1.0f : guard_nu(tot / (float)N);
        const float rnn = __frcp_rn(nun);
        uint32_t word = 0;
        if constexpr (BIN == TSAT_BIN_PHILOX) {
          const RowStream rs = row_stream(pd, hy.key0, cur, v);
#pragma unroll 1
          for (int h = 0; h < 4; ++h) {   // samples 32 w + 8 h + e: block 4 w + h, half e
            const uint4 r = philox4x32_10(make_uint4((uint32_t)(4 * w + h), rs.row, (uint32_t)(tcur + 1), kTagBin),
                                          rs.k0, hy.key1);
#pragma unroll
            for (int e = 0; e < 8; ++e)
              word |= binarize_one(__fmul_rn(gbuf[(8 * h + e) * kGS + lane], rnn), TSAT_BIN_PHILOX, hy.bin_c,
                                   half16(e < 4 ? r.x : r.z, e < 4 ? r.y : r.w, e & 3))
                      << (8 * h + e);
          }
        } else {
#pragma unroll 8
          for (int b = 0; b < 32; ++b) word |= (__fmul_rn(gbuf[b * kGS + lane], rnn) > 0.0f ? 1u : 0u) << b;
        }
        bdst[v * W + w] = word;
        if (w == 0) sd.nu[v] = nun;
      }
    }
  }
}

int updateL_smem_bytes(int N) { return kWarps * updateL_warp_floats(N) * (int)sizeof(float); }

template <typename F>
static void for_each_updateL(F f) {
  f(k_updateL<0, TSAT_BIN_DET, TSAT_NORM_SIGNED_MEAN, true>);
  f(k_updateL<0, TSAT_BIN_DET, TSAT_NORM_ABSMEAN, true>);
  f(k_updateL<0, TSAT_BIN_DET, TSAT_NORM_NONE, true>);
  f(k_updateL<0, TSAT_BIN_PHILOX, TSAT_NORM_SIGNED_MEAN, true>);
  f(k_updateL<0, TSAT_BIN_PHILOX, TSAT_NORM_ABSMEAN, true>);
  f(k_updateL<0, TSAT_BIN_PHILOX, TSAT_NORM_NONE, true>);
  f(k_updateL<1, TSAT_BIN_DET, TSAT_NORM_SIGNED_MEAN, true>);
  f(k_updateL<1, TSAT_BIN_DET, TSAT_NORM_ABSMEAN, true>);
  f(k_updateL<1, TSAT_BIN_DET, TSAT_NORM_NONE, true>);
  f(k_updateL<0, TSAT_BIN_DET, TSAT_NORM_SIGNED_MEAN, false>);
  f(k_updateL<0, TSAT_BIN_DET, TSAT_NORM_ABSMEAN, false>);
  f(k_updateL<0, TSAT_BIN_DET, TSAT_NORM_NONE, false>);
  f(k_updateL<0, TSAT_BIN_PHILOX, TSAT_NORM_SIGNED_MEAN, false>);
  f(k_updateL<0, TSAT_BIN_PHILOX, TSAT_NORM_ABSMEAN, false>);
  f(k_updateL<0, TSAT_BIN_PHILOX, TSAT_NORM_NONE, false>);
  f(k_updateL<1, TSAT_BIN_DET, TSAT_NORM_SIGNED_MEAN, false>);
  f(k_updateL<1, TSAT_BIN_DET, TSAT_NORM_ABSMEAN, false>);
  f(k_updateL<1, TSAT_BIN_DET, TSAT_NORM_NONE, false>);
}

template <int MODE, int BIN, bool STAB>
static cudaError_t launch_updateL_n(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const float *zin,
                                    float *grad, float dL, int grid, cudaStream_t st) {
  const int smem = updateL_smem_bytes(sd.N);
  switch (hy.norm) {
    case TSAT_NORM_SIGNED_MEAN:
      k_updateL<MODE, BIN, TSAT_NORM_SIGNED_MEAN, STAB><<<grid, kBlock, smem, st>>>(pd, sd, hy, zin, grad, dL);
      break;
    case TSAT_NORM_ABSMEAN:
      k_updateL<MODE, BIN, TSAT_NORM_ABSMEAN, STAB><<<grid, kBlock, smem, st>>>(pd, sd, hy, zin, grad, dL);
      break;
    default:
      k_updateL<MODE, BIN, TSAT_NORM_NONE, STAB><<<grid, kBlock, smem, st>>>(pd, sd, hy, zin, grad, dL);
      break;
  }
  return cudaGetLastError();
}

template <bool STAB>
static cudaError_t launch_updateL_s(const ProbDev &pd, const StateDev &sd, const Hyper &hy, int mode,
                                    const float *zin, float *grad, float dL, int grid, cudaStream_t st) {
  if (mode == 1) return launch_updateL_n<1, TSAT_BIN_DET, STAB>(pd, sd, hy, zin, grad, dL, grid, st);
  if (hy.binarize == TSAT_BIN_PHILOX)
    return launch_updateL_n<0, TSAT_BIN_PHILOX, STAB>(pd, sd, hy, zin, grad, dL, grid, st);
  return launch_updateL_n<0, TSAT_BIN_DET, STAB>(pd, sd, hy, zin, grad, dL, grid, st);
}

cudaError_t launch_updateL(const ProbDev &pd, const StateDev &sd, const Hyper &hy, int mode, const float *zin,
                                  float *grad, float dL, int grid, cudaStream_t st) {
  if (updateL_tab_floats(sd.N) > 0) return launch_updateL_s<true>(pd, sd, hy, mode, zin, grad, dL, grid, st);
  return launch_updateL_s<false>(pd, sd, hy, mode, zin, grad, dL, grid, st);
}


void prepare_updateL_attrs(int bytes) {
  for_each_updateL([bytes](auto fn) { cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); });
}

int updateL_resident_blocks(int N) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_updateL<0, TSAT_BIN_PHILOX, TSAT_NORM_SIGNED_MEAN, true>, kBlock,
                                                updateL_smem_bytes(N));
  return nb;
}

}  // namespace tsat
