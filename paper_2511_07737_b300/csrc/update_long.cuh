// update_long.cuh -- the row-group body of the fused update for clause
// length 4..7 (word per lane), shared by the multi-kernel update and the
// cluster-persistent solver.
#pragma once
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

// One row group's rows of instance `cur`, word per lane: lane (rsub, w) of the
// warp owns word w of row v (act: the row takes this step's update; frozen:
// its instance is frozen, so its bits are copied).  The warp's gamma table of
// `cur` is ready in shared memory (STAB: at byte offset tbase from smb, bank
// skew tskew) or gglob points at its gamma in global memory (+ 32 w).
// Counting phase (the straight-through sum over the row's occurrences, Sec.
// III-B), then Eq. 5's chain rule, AdamW (Sec. IV-A), the new normaliser and
// the bits of step tcur + 1 (Eq. 2 or the Philox rule); MODE 1 writes
// dL * dL/dz to grad instead and stops after the chain rule.  COH: the bits
// and z were written earlier in the same launch (after a barrier with acquire
// semantics), so they are read with ordinary cached loads (ld.global.ca),
// which that barrier makes see those writes, instead of the read-only path.
template <int MODE, int BIN, int NORM, bool STAB, bool COH = false>
__device__ __forceinline__ void updateL_rows(const ProbDev &pd, const StateDev &sd, const Hyper &hy,
                                             const StepParams &sp, int64_t tcur, const uint32_t *bsrc, uint32_t *bdst,
                                             const float *zsrc, float *grad, float dL, const char *smb,
                                             uint32_t tbase, uint32_t tskew, float *gbuf, const float *gglob, int cur,
                                             int64_t v, bool act, bool frozen, int lane, int w, int rbase) {
  const int N = sd.N, W = sd.W;
  const int4 *xrec8 = reinterpret_cast<const int4 *>(pd.xrec);   // two int4 per occurrence
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
  auto bits_at = [&](size_t k) -> uint32_t { return COH ? __ldca(bsrc + k) : __ldg(bsrc + k); };
  auto ld_z4 = [&](const float *p) -> float4 {
    return COH ? __ldca(reinterpret_cast<const float4 *>(p)) : __ldg(reinterpret_cast<const float4 *>(p));
  };
  const uint32_t own = act ? bits_at((size_t)v * W + w) : 0u;
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
        const uint32_t x = bits_at((size_t)(lits[q] >> 1) * W + w) ^ (0u - (uint32_t)(lits[q] & 1));
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
      const float4 z4 = ld_z4(zsrc + rowoff + s);
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
      const float4 z4 = ld_z4(zsrc + off);
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
  if constexpr (MODE == 1) return;
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

}  // namespace tsat
