// persist.cu -- persistent solver for batches of small instances: one block per
// instance runs many optimisation steps (Sec. III-B, IV-A) in a single launch.
//
// A step of one instance touches only that instance's rows and clauses, so the
// instances of a batch are independent and each block owns one.  The phases of
// a step -- forward histogram of R = P A (Eq. 1), Eq. 4 with its dL/dR table,
// fused STE backward + Eq. 5 + AdamW + re-binarisation (Eq. 2 or Philox) --
// are separated by block barriers only; no block ever waits on another.  On
// the multi-kernel path every step pays three kernel boundaries, which is what
// bounds a step of an instance with a few thousand clauses; here a launch pays
// one.  State layout, per-instance records and every result follow the
// multi-kernel path: G is formed from exact integer counts (per sample, the
// signed counts of the products of R's bit planes, folded with the Moebius
// coefficients of the dL/dR table), so only FP32 rounding order differs from
// it, and an instance freezes at the step whose forward finds a sample with no
// unsatisfied clause.
//
// Split instances (SPLIT): when the batch leaves most SMs idle (one instance,
// or a few), each instance gets a thread-block cluster of CS blocks instead of
// one block.  Every block keeps a copy of the instance's bits; block q of the
// cluster runs every CS-th forward task into its own histogram (one per step
// parity), and after a cluster barrier every block sums the CS histograms over
// distributed shared memory (integers: every block gets the same table and
// takes the same found / stop decisions).  Block q updates the rows
// [V q / CS, V (q + 1) / CS) (their z, m, v and normaliser resident in its
// shared memory) and writes each new bits word into every block's copy; a
// second cluster barrier ends the step.  The rows' arithmetic is the one-block
// kernel's: with the same samples per thread (the same placement of z, m, v)
// the results are the same bit for bit.

#include <cooperative_groups.h>

#include "internal.h"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace tsat {

constexpr int kPsSched = 256;   // steps whose scalars are formed at once (one per thread)

// dL/dR table of one sample: 8 floats (r = 0..7); every 16 samples are
// followed by 8 floats of padding (272 floats per 32-sample word), so that the
// lanes of one lookup (same bit, threads at different words or at the two
// halves of a word) start on different banks
__device__ __forceinline__ int ps_tab(int s) { return 8 * s + 8 * (s >> 4); }
// offset of sample s0 + j from ps_tab(s0), s0 a multiple of 16 or j + s0 % 16 < 16
__device__ __forceinline__ int ps_tab_rel(int j) { return 8 * j + 8 * (j >> 4); }

// In place: c[m] = sum over m' subset of m of (-1)^{|m| - |m'|} g[m'] (R's three
// bit planes b0, b1, b2 as the bits of m), so that g[R] = sum over the
// subsets m of the bits set in R of c[m]
__device__ __forceinline__ void ps_moebius(float (&c)[8]) {
#pragma unroll
  for (int bit = 1; bit < 8; bit <<= 1)
#pragma unroll
    for (int m = 0; m < 8; ++m)
      if (m & bit) c[m] -= c[m ^ bit];
}

constexpr int kPsChunk = 127;   // occurrences per byte-counter chunk (|count| <= 127)

__device__ __forceinline__ uint32_t *ps_bits(const StateDev &sd, int64_t t) {
  return sd.bits + (size_t)(t & 1) * (size_t)sd.V * sd.W;
}

// RES: the instance's z, m, v and normaliser stay in shared memory for the
// whole launch (layout [row][word][33]: the samples of one lane start on
// their own bank) and are written back once at the end; otherwise they are
// read and written in global memory at every step.
// SPT: samples per thread in the update's sample phase; Q = 32 / SPT threads
// share a 32-sample word, and a block has 1024 (SPT 8), 512 (16) or 256 (32)
// threads.  With clause length <= 3 the Q threads of a word also
// share its occurrences in the counting phase.
template <int SPT>
constexpr int ps_block() { return SPT == 8 ? 1024 : (SPT == 16 ? 512 : 256); }

// SPLIT: the launch has clusters of CS blocks per instance (see the top of
// the file); vmax bounds the instances' variables, vown the rows of one block.
template <int BIN, int NORM, bool RES, int SPT, bool SPLIT>
__global__ void __launch_bounds__(ps_block<SPT>(), SPT == 32 ? 2 : 1)
    k_persist(ProbDev pd, StateDev sd, Hyper hy, LrSched ls, int32_t K, int32_t vmax, int32_t vown) {
  constexpr int BS = ps_block<SPT>(), NW = BS / 32, Q = 32 / SPT;
  constexpr int HP = SPLIT ? 2 : 1;   // histograms: one per step parity when other blocks read them
  extern __shared__ __align__(16) float smP[];
  __shared__ int64_t sh_t0;
  __shared__ int sh_skip, sh_found, sh_mu0, sh_mi0, sh_fs;
  __shared__ float sh_L;
  __shared__ int64_t sh_ft;
  __shared__ float sh_ls[NW], etab[8];
  __shared__ int sh_mu[NW], sh_mi[NW];
  __shared__ StepParams sh_sps[kPsSched];   // step scalars of the next kPsSched steps
  StateHdr *hdr = sd.hdr;
  const int CS = SPLIT ? (int)cg::this_cluster().num_blocks() : 1;
  const int rank = SPLIT ? (int)cg::this_cluster().block_rank() : 0;
  const int inst = blockIdx.x / CS;
  // the barrier between the phases of a step: the block's, or the cluster's
  // (release / acquire: the histograms and bits written before it are seen
  // by every block after it)
  auto phase_barrier = [] {
    if constexpr (SPLIT) cg::this_cluster().sync();
    else __syncthreads();
  };
  const int N = sd.N, W = sd.W;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    sh_t0 = hdr->t;
    sh_skip = hdr->all_done;
    sh_found = sd.inst[inst].found;
  }
  if (tid < 8) etab[tid] = expf(-hy.tau * (float)tid);
  __syncthreads();
  if (sh_skip) return;   // every instance was frozen and stopped before this launch (all blocks see it)
  const int64_t t0 = sh_t0;
  const InstInfo I = pd.inst[inst];
  const int lmax = I.lmax;
  // the rows this block updates (all of them unless SPLIT)
  const int r_lo = (int)((int64_t)I.n_vars * rank / CS), r_hi = (int)((int64_t)I.n_vars * (rank + 1) / CS);
  int32_t *hist = reinterpret_cast<int32_t *>(smP);   // [HP][8][N]: [lmax + 1][N] used
  float *tab = smP + HP * 8 * N;                        // [N][8] with 8 floats of padding per 16 samples (ps_tab)
  // S and the unsatisfied count of every sample, and the instance's status
  // fields, are kept in shared memory and written to the state once at the end
  // of the launch: only the last step's values are visible outside
  float *sS = tab + 272 * W;                                     // [N]
  int32_t *sU = reinterpret_cast<int32_t *>(sS + N);             // [N]
  // the instance's bits, both step parities, rows numbered from the instance's
  // first variable: every gather of the forward and the backward reads them here
  uint32_t *sbits = reinterpret_cast<uint32_t *>(sU + N);        // [2][vmax][W]
  const size_t vw = (size_t)vmax * W;
  for (int64_t i = tid; i < (int64_t)I.n_vars * W; i += BS)
    sbits[(t0 & 1) * vw + i] = ps_bits(sd, t0)[(size_t)I.v_off * W + i];
  // RES: z, m, v of the block's rows [vown][W][33], then their normaliser [vown]
  const size_t ow = (size_t)vown * W;
  float *smz = reinterpret_cast<float *>(sbits + 2 * vw);
  float *smm = smz + ow * 33, *smv = smm + ow * 33, *snu = smv + ow * 33;
  const int nown = r_hi - r_lo;
  const size_t g0 = ((size_t)I.v_off + r_lo) * N;   // the block's first row in the state arrays
  if (RES && !sh_found) {
    for (int64_t i = tid; i < (int64_t)nown * N; i += BS) {
      const size_t si = (size_t)(i / 32) * 33 + (i & 31);   // [row][word][33]: word index i / 32 of the row-major array
      smz[si] = sd.z[g0 + i];
      smm[si] = sd.m[g0 + i];
      smv[si] = sd.v[g0 + i];
    }
    for (int i = tid; i < nown; i += BS) snu[i] = sd.nu[I.v_off + r_lo + i];
  }
  // the histograms start at zero; each step's update phase clears the one the
  // next step's forward fills (the barrier ending the step orders the two;
  // with SPLIT that is the other parity, whose last readers in other blocks
  // passed the barrier that ended the previous step)
  for (int i = tid; i < HP * 8 * N; i += BS) hist[i] = 0;
  __syncthreads();
  int found = sh_found;
  const bool ran = !found;   // the instance is live at the start of the launch
  int64_t t = t0;
  for (int32_t k = 0; k < K && !found; ++k, ++t) {
    if (k % kPsSched == 0) {   // the double-precision schedule of the next kPsSched steps, in parallel
      if (tid < kPsSched) sh_sps[tid] = step_params(ls, t + tid);
      __syncthreads();
    }
    // ---- forward (Eq. 1): lane = clause, 32 samples of word w; bit-sliced R,
    // warp transpose, popcounts of the R = r masks into the block histogram
    const uint32_t *bsrc = sbits + (t & 1) * vw;
    int32_t *hcur = hist + (SPLIT ? (int)(t & 1) * 8 * N : 0);
    // A task is a group of 32 clauses (lane = clause) and WT words of the
    // samples (WT = 2 when N >= 64): the clause is decoded once for both words
    // and a small instance needs half the task rounds (n = 100, N = 64: 14
    // tasks for 16 warps instead of 28).  The 1024-thread kernel (SPT 8, 64
    // registers) keeps one word per task, which spills less under its register
    // cap (264 against 292 bytes) at the same speed.
    constexpr int WTM = SPT == 8 ? 1 : 2;
    const int ngroups = (I.n_clauses + 31) >> 5;
    const int WT = W >= WTM ? WTM : 1, wtasks = W / WT;
    for (int task = warp + NW * rank; task < ngroups * wtasks; task += NW * CS) {
      const int g = task / wtasks, w0 = (task - g * wtasks) * WT;
      const bool active = 32 * g + lane < I.n_clauses;
      uint32_t pl[WTM][3] = {};
      if (active) {
        const int c = I.c_off + 32 * g + lane;
        if (pd.crec) {
          // clause length <= 3: one record {v0, v1, v2, negation bytes | length << 24}
          // instead of the clause pointers and literals (a missing literal repeats v0)
          const int4 cr = __ldg(pd.crec + c);
          const uint32_t len = (uint32_t)cr.w >> 24;
          const uint32_t na = __byte_perm((uint32_t)cr.w, 0u, 0x0000u), nb = __byte_perm((uint32_t)cr.w, 0u, 0x1111u),
                         nd = __byte_perm((uint32_t)cr.w, 0u, 0x2222u);
          const uint32_t *ra = bsrc + (size_t)(cr.x - I.v_off) * W + w0, *rb = bsrc + (size_t)(cr.y - I.v_off) * W + w0,
                         *rd = bsrc + (size_t)(cr.z - I.v_off) * W + w0;
#pragma unroll
          for (int ww = 0; ww < WTM; ++ww) {
            if (ww < WT) {
              const uint32_t a = ra[ww] ^ na;
              const uint32_t b = len > 1 ? (rb[ww] ^ nb) : 0u;
              const uint32_t d = len > 2 ? (rd[ww] ^ nd) : 0u;
              pl[ww][0] = a ^ b ^ d;
              pl[ww][1] = (a & b) | (d & (a ^ b));
            }
          }
        } else {
          const int32_t b = __ldg(pd.cptr + c), e = __ldg(pd.cptr + c + 1);
          for (int32_t j = b; j < e; ++j) {
            const int32_t lit = __ldg(pd.clit + j);
            const uint32_t *row = bsrc + (size_t)((lit >> 1) - I.v_off) * W + w0, neg = 0u - (uint32_t)(lit & 1);
#pragma unroll
            for (int ww = 0; ww < WTM; ++ww)
              if (ww < WT) bitslice_add<3>(pl[ww], row[ww] ^ neg);
          }
        }
      }
      const uint32_t valid = __ballot_sync(0xFFFFFFFFu, active);
#pragma unroll
      for (int ww = 0; ww < WTM; ++ww) {
        if (ww < WT) {
          uint32_t tp[3];
          tp[0] = warp_transpose32(pl[ww][0], lane);
          tp[1] = warp_transpose32(pl[ww][1], lane);
          tp[2] = pd.crec ? 0u : warp_transpose32(pl[ww][2], lane);   // R <= 3 with clause records
          for (int r = 0; r <= lmax; ++r) {
            const int cnt = __popc(valid & bitslice_eq<3>(tp, r));
            if (cnt) atomicAdd(hcur + r * N + 32 * (w0 + ww) + lane, cnt);
          }
        }
      }
    }
    phase_barrier();
    // ---- Eq. 4 per sample, the dL/dR table, loss, fewest-unsatisfied sample
    float lsum = 0.f;
    int mu = 0x7FFFFFFF, mi = 0x7FFFFFFF;
    for (int i = tid; i < N; i += BS) {
      // the sample's histogram (SPLIT: summed over the cluster's blocks, in
      // integers, so every block gets the same values)
      int hv[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) hv[r] = 0;
      for (int q = 0; q < CS; ++q) {
        const int32_t *hq = hcur;
        if constexpr (SPLIT) hq = cg::this_cluster().map_shared_rank(hcur, q);
#pragma unroll
        for (int r = 0; r < 8; ++r)
          if (r <= lmax) hv[r] += hq[r * N + i];
      }
      float Z = 0.f, Y = 0.f;
      for (int r = 0; r <= lmax; ++r) {
        const float h = (float)hv[r];
        Z += h * etab[r];
        Y += (float)r * h * etab[r];
      }
      const float S = Y / Z;
      const float invZ = 1.0f / Z;
      float c[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) c[r] = r <= lmax ? -(etab[r] * invZ) * (1.0f - hy.tau * ((float)r - S)) : 0.f;
      ps_moebius(c);   // the update counts product masks of R's bit planes
#pragma unroll
      for (int r = 0; r < 8; ++r) tab[ps_tab(i) + r] = c[r];
      const int h0 = hv[0];
      lsum += S;
      if (h0 < mu || (h0 == mu && i < mi)) { mu = h0; mi = i; }
      sS[i] = S;
      sU[i] = h0;
    }
    for (int o = 16; o > 0; o >>= 1) {
      lsum += __shfl_xor_sync(0xFFFFFFFFu, lsum, o);
      const int u2 = __shfl_xor_sync(0xFFFFFFFFu, mu, o), i2 = __shfl_xor_sync(0xFFFFFFFFu, mi, o);
      if (u2 < mu || (u2 == mu && i2 < mi)) { mu = u2; mi = i2; }
    }
    if (lane == 0) { sh_ls[warp] = lsum; sh_mu[warp] = mu; sh_mi[warp] = mi; }
    __syncthreads();
    {
      // every warp reduces the warps' partials (one per lane) itself: the
      // inputs and the butterfly order are the same, so all warps reach the same
      // loss and fewest-unsatisfied sample and know without another barrier
      // whether the instance is found (the partials are rewritten only after
      // the barrier that ends the step)
      float L = lane < NW ? sh_ls[lane] : 0.f;
      mu = lane < NW ? sh_mu[lane] : 0x7FFFFFFF;
      mi = lane < NW ? sh_mi[lane] : 0x7FFFFFFF;
      for (int o = 16; o > 0; o >>= 1) {
        L += __shfl_xor_sync(0xFFFFFFFFu, L, o);
        const int u2 = __shfl_xor_sync(0xFFFFFFFFu, mu, o), i2 = __shfl_xor_sync(0xFFFFFFFFu, mi, o);
        if (u2 < mu || (u2 == mu && i2 < mi)) { mu = u2; mi = i2; }
      }
      if (tid == 0) {
        sh_L = -L;
        sh_mu0 = mu;
        sh_mi0 = mi;
        if (mu == 0) {
          sh_found = 1;
          sh_fs = mi;
          sh_ft = t;
        }
      }
      found = mu == 0;
    }
    if (found) break;   // the bits of step t are the model; z, m, v stay
    {   // the histogram the next forward fills (without SPLIT: this one, read for the last time above)
      int32_t *hnext = hist + (SPLIT ? (int)((t + 1) & 1) * 8 * N : 0);
      for (int i = tid; i < (lmax + 1) * N; i += BS) hnext[i] = 0;
    }
    // ---- fused update: thread = (row, word w); G of its 32 samples summed over
    // the row's occurrences in record order, then Eq. 5, AdamW, the new
    // normaliser and the bits of step t + 1
    const StepParams sp = sh_sps[k % kPsSched];
    uint32_t *bdst = ps_bits(sd, t + 1), *sdst = sbits + ((t + 1) & 1) * vw;
    const int WQ = W * Q;                 // threads of one row: W words x Q parts
    const int rpp = BS / WQ;              // rows per pass
    const int rl = tid % WQ, w = rl / Q, sb = SPT * (rl % Q);   // word, first bit of this thread's samples
    for (int vb = r_lo; vb < r_hi; vb += rpp) {
      const int vl = vb + tid / WQ;
      const bool act = vl < r_hi;
      const int64_t v = (int64_t)I.v_off + vl;
      // G of this thread's samples: signed byte counts of the product masks of
      // R's bit planes (mask m of the subset m of {b0, b1, b2}), folded with
      // the Moebius coefficients of the dL/dR table (an exact rewrite of the
      // per-sample sum over the occurrences).  Word u of a mask holds samples
      // sb + 4u .. sb + 4u + 3, one byte each with bias 128.
      constexpr int NWD = SPT / 4;
      float acc[SPT];
#pragma unroll
      for (int j = 0; j < SPT; ++j) acc[j] = 0.f;
      const bool two = pd.rec_stride == 4;   // clause length <= 3: R <= 3, masks b0, b1, b0 b1
      if (two) {
        // Clause length <= 3: the word's occurrences are dealt round-robin to
        // its Q threads, each counting all 32 samples of the word in strided
        // byte counters (byte b of sc[m][j] counts sample 8b + j); the Q
        // partial counts are summed byte-wise across the threads and thread q
        // folds its own samples SPT q + j.  An occurrence is decoded and
        // gathered once per word instead of once per thread.  The chunk rounds
        // are warp-uniform (shuffles).
        const int q = rl % Q;
        uint32_t own = 0;
        int32_t o0 = 0, deg = 0;
        if (act) {
          own = bsrc[(size_t)vl * W + w];
          o0 = __ldg(pd.vptr + v);
          deg = __ldg(pd.vptr + v + 1) - o0;
        }
        int maxdeg = deg;
        for (int o = 16; o > 0; o >>= 1) maxdeg = max(maxdeg, __shfl_xor_sync(0xFFFFFFFFu, maxdeg, o));
        const int tb = ps_tab(32 * w + sb);
        const int4 *xr4 = reinterpret_cast<const int4 *>(pd.xrec) + o0;   // {hdr, lit, lit, 0} per occurrence
        for (int32_t c0 = 0; c0 < maxdeg; c0 += kPsChunk) {
          const int32_t ce = min(deg, c0 + kPsChunk);
          int nsign = 0;   // signed occurrences of the chunk
          uint32_t sc[3][8];
#pragma unroll
          for (int mk = 0; mk < 3; ++mk)
#pragma unroll
            for (int j = 0; j < 8; ++j) sc[mk][j] = 0x80808080u;
#pragma unroll 2
          for (int32_t o = c0 + q; o < ce; o += Q) {
            const int4 ra = __ldg(xr4 + o);
            const int h = ra.x, len = h >> 1;
            const uint32_t a = own ^ (0u - (uint32_t)(h & 1));
            const uint32_t bb =
                len > 1 ? (bsrc[(size_t)((ra.y >> 1) - I.v_off) * W + w] ^ (0u - (uint32_t)(ra.y & 1))) : 0u;
            const uint32_t cc =
                len > 2 ? (bsrc[(size_t)((ra.z >> 1) - I.v_off) * W + w] ^ (0u - (uint32_t)(ra.z & 1))) : 0u;
            const uint32_t p0 = a ^ bb ^ cc, p1 = (a & bb) | (cc & (a ^ bb));   // R = p0 + 2 p1
            const uint32_t sg = (h & 1) ? 0xFFFFFFFFu : 1u;
            nsign += (int)sg;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const uint32_t t0 = (p0 >> j) & 0x01010101u, t1 = (p1 >> j) & 0x01010101u;
              sc[0][j] += t0 * sg;
              sc[1][j] += t1 * sg;
              sc[2][j] += (t0 & t1) * sg;
            }
          }
#pragma unroll
          for (int o = 1; o < Q; o <<= 1)
#pragma unroll
            for (int mk = 0; mk < 3; ++mk)
#pragma unroll
              for (int j = 0; j < 8; ++j)
                sc[mk][j] = add_biased_bytes(sc[mk][j], __shfl_xor_sync(0xFFFFFFFFu, sc[mk][j], o));
#pragma unroll
          for (int o = 1; o < Q; o <<= 1) nsign += __shfl_xor_sync(0xFFFFFFFFu, nsign, o);
          // sample SPT q + j: byte (SPT q + j) / 8 of counter (j mod 8); its
          // coefficients c0..c3 are one aligned 16-byte load
#pragma unroll
          for (int j = 0; j < SPT; ++j) {
            const float4 cf = *reinterpret_cast<const float4 *>(tab + tb + ps_tab_rel(j));
            const uint32_t bq = (uint32_t)((SPT / 8) * q + (j >> 3));
            float g = fmaf((float)nsign, cf.x, acc[j]);
            g = fmaf(biased_byte(sc[0][j & 7], bq), cf.y, g);
            g = fmaf(biased_byte(sc[1][j & 7], bq), cf.z, g);
            g = fmaf(biased_byte(sc[2][j & 7], bq), cf.w, g);
            acc[j] = g;
          }
        }
      } else if (act) {
        const uint32_t own = bsrc[(size_t)vl * W + w];
        const int32_t o0 = __ldg(pd.vptr + v), o1 = __ldg(pd.vptr + v + 1);
        const int tb = ps_tab(32 * w + sb);
        int nsign = 0;
        for (int32_t c0 = o0; c0 < o1; c0 += kPsChunk) {
          const int32_t c1 = min(o1, c0 + kPsChunk);
          uint32_t sc[7][NWD];
#pragma unroll
          for (int mk = 0; mk < 7; ++mk)
#pragma unroll
            for (int u = 0; u < NWD; ++u) sc[mk][u] = 0x80808080u;
#pragma unroll 2
          for (int32_t o = c0; o < c1; ++o) {
            // the fixed record {hdr, lit x 2, 0} (clause length <= 3) or {hdr, lit x 6, 0}, in one or two loads
            const int4 *rp = reinterpret_cast<const int4 *>(pd.xrec) + (two ? o : 2 * (int64_t)o);
            const int4 ra = __ldg(rp), rb = two ? make_int4(0, 0, 0, 0) : __ldg(rp + 1);
            const int h = ra.x, len = h >> 1;
            const int lits[6] = {ra.y, ra.z, ra.w, rb.x, rb.y, rb.z};
            uint32_t pl[3] = {own ^ (0u - (uint32_t)(h & 1)), 0u, 0u};
#pragma unroll
            for (int q = 0; q < 6; ++q) {
              if (q + 1 < len)
                bitslice_add<3>(pl, bsrc[(size_t)((lits[q] >> 1) - I.v_off) * W + w] ^ (0u - (uint32_t)(lits[q] & 1)));
            }
            const uint32_t sg = (h & 1) ? 0xFFFFFFFFu : 1u;
            nsign += (int)sg;
            const uint32_t b0 = pl[0] >> sb, b1 = pl[1] >> sb, b01 = b0 & b1;
#pragma unroll
            for (int u = 0; u < NWD; ++u) {
              sc[0][u] += spread4((b0 >> (4 * u)) & 15u) * sg;
              sc[1][u] += spread4((b1 >> (4 * u)) & 15u) * sg;
              sc[2][u] += spread4((b01 >> (4 * u)) & 15u) * sg;
            }
            if (!two) {
              const uint32_t b2 = pl[2] >> sb;
#pragma unroll
              for (int u = 0; u < NWD; ++u) {
                sc[3][u] += spread4((b2 >> (4 * u)) & 15u) * sg;
                sc[4][u] += spread4(((b0 & b2) >> (4 * u)) & 15u) * sg;
                sc[5][u] += spread4(((b1 & b2) >> (4 * u)) & 15u) * sg;
                sc[6][u] += spread4(((b01 & b2) >> (4 * u)) & 15u) * sg;
              }
            }
          }
          // fold the chunk: acc[j] += sum over masks of count * coefficient
#pragma unroll
          for (int u = 0; u < NWD; ++u)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float *cf = tab + tb + ps_tab_rel(4 * u + e);
              float g = acc[4 * u + e];
              g = fmaf(biased_byte(sc[0][u], e), cf[1], g);
              g = fmaf(biased_byte(sc[1][u], e), cf[2], g);
              g = fmaf(biased_byte(sc[2][u], e), cf[3], g);
              if (!two) {
#pragma unroll
                for (int mk = 3; mk < 7; ++mk) g = fmaf(biased_byte(sc[mk][u], e), cf[mk + 1], g);
              }
              acc[4 * u + e] = g;
            }
        }
#pragma unroll
        for (int j = 0; j < SPT; ++j) acc[j] = fmaf((float)nsign, tab[tb + ps_tab_rel(j)], acc[j]);
      }
      const size_t off = RES ? ((size_t)(vl - r_lo) * W + w) * 33 + sb : (size_t)v * N + 32 * w + sb;
      float *zp = RES ? smz : sd.z, *mp = RES ? smm : sd.m, *vp = RES ? smv : sd.v;
      const float nu = act ? (RES ? snu[vl - r_lo] : sd.nu[v]) : 1.0f;
      const float rnu = __frcp_rn(nu);
      float part = 0.f;
      if (act && NORM != TSAT_NORM_NONE) {
#pragma unroll
        for (int j = 0; j < SPT; ++j) part = fmaf(acc[j], zp[off + j], part);
      }
      const float dot = seg_sum(part, WQ);
      const float c2 = dot * rnu * rnu * (1.0f / (float)N);
      float psum = 0.f;
      if (act) {
#pragma unroll
        for (int j = 0; j < SPT; ++j) {
          const float z = zp[off + j];
          float g;
          if constexpr (NORM == TSAT_NORM_NONE) {
            g = acc[j];
          } else {
            const float dmu = (NORM == TSAT_NORM_ABSMEAN) ? (float)((z > 0.f) - (z < 0.f)) : 1.0f;
            g = acc[j] * rnu - c2 * dmu;
          }
          float m = mp[off + j], vv = vp[off + j];
          m = hy.beta1 * m + (hy.omb1) * g;
          vv = hy.beta2 * vv + (hy.omb2) * (g * g);
          const float zn = z * sp.decay - sp.step_size * (m * adam_inv_denom(vv, sp.inv_sqrt_bc2, hy.eps));
          zp[off + j] = zn;
          mp[off + j] = m;
          vp[off + j] = vv;
          acc[j] = zn;
          psum += (NORM == TSAT_NORM_ABSMEAN) ? fabsf(zn) : zn;
        }
      }
      const float tot = seg_sum(psum, WQ);
      const float nun = (NORM == TSAT_NORM_NONE) ? 1.0f : guard_nu(tot / (float)N);
      uint32_t part_bits = 0;
      if (act) {
        const float rnn = __frcp_rn(nun);
        if constexpr (BIN == TSAT_BIN_PHILOX) {
#pragma unroll
          for (int hb = 0; hb < SPT / 8; ++hb) {   // samples 32 w + sb + 8 hb + e: block 4 w + sb / 8 + hb, half e
            // the row's Philox stream: instance-local row, key offset by the instance's id
            const uint4 r = philox4x32_10(
                make_uint4((uint32_t)(4 * w + (sb >> 3) + hb), (uint32_t)vl, (uint32_t)(t + 1), kTagBin),
                hy.key0 + (uint32_t)I.gid, hy.key1);
#pragma unroll
            for (int e = 0; e < 8; ++e)
              part_bits |= binarize_one(__fmul_rn(acc[8 * hb + e], rnn), TSAT_BIN_PHILOX, hy.bin_c,
                                        half16(e < 4 ? r.x : r.z, e < 4 ? r.y : r.w, e & 3))
                           << (8 * hb + e);
          }
        } else {
#pragma unroll
          for (int j = 0; j < SPT; ++j) part_bits |= (__fmul_rn(acc[j], rnn) > 0.0f ? 1u : 0u) << j;
        }
      }
      // the Q parts of word w are consecutive lanes: join their bits
      uint32_t word = (SPT == 32) ? part_bits : (part_bits << sb);
#pragma unroll
      for (int o = 1; o < Q; o <<= 1) word |= __shfl_xor_sync(0xFFFFFFFFu, word, o);
      if (act && sb == 0) {
        if (!RES) bdst[v * W + w] = word;
        sdst[(size_t)vl * W + w] = word;
        if constexpr (SPLIT) {   // every block's copy of the bits
          for (int q = 0; q < CS; ++q)
            if (q != rank) cg::this_cluster().map_shared_rank(sdst, q)[(size_t)vl * W + w] = word;
        }
        if (w == 0) {
          if (RES) snu[vl - r_lo] = nun;
          else sd.nu[v] = nun;
        }
      }
    }
    phase_barrier();   // the bits, z and normaliser of step t + 1 are written before its forward
  }
  // SPLIT: no block goes on (and leaves) while another may still read its
  // histogram: all blocks leave the loop at the same step
  phase_barrier();
  // the last forward's S, unsatisfied counts and status (and the model's
  // sample and step); every block of a cluster holds the same values
  if (ran && K > 0 && rank == 0) {
    for (int i = tid; i < N; i += BS) {
      sd.S[(size_t)inst * N + i] = sS[i];
      sd.unsat[(size_t)inst * N + i] = sU[i];
    }
    if (tid == 0) {
      InstState *is = sd.inst + inst;
      is->loss = sh_L;
      is->min_unsat = sh_mu0;
      is->best_sample = sh_mi0;
      if (found) {
        is->found = 1;
        is->found_sample = sh_fs;
        is->found_step = sh_ft;
      }
    }
  }
  // an instance found in this launch keeps its model in both bit buffers (the
  // multi-kernel path copies a frozen instance's bits at every step)
  if (found && ran) {   // the block's rows
    const int64_t tf = sh_ft;
    for (int64_t i = (int64_t)r_lo * W + tid; i < (int64_t)r_hi * W; i += BS) {
      if (RES) sbits[((tf + 1) & 1) * vw + i] = sbits[(tf & 1) * vw + i];
      else ps_bits(sd, tf + 1)[(size_t)I.v_off * W + i] = ps_bits(sd, tf)[(size_t)I.v_off * W + i];
    }
  }
  if (RES && ran) {   // write the resident state back
    __syncthreads();
    for (int64_t i = tid; i < (int64_t)nown * N; i += BS) {
      const size_t si = (size_t)(i / 32) * 33 + (i & 31);
      sd.z[g0 + i] = smz[si];
      sd.m[g0 + i] = smm[si];
      sd.v[g0 + i] = smv[si];
    }
    for (int i = tid; i < nown; i += BS) sd.nu[I.v_off + r_lo + i] = snu[i];
    for (int64_t i = (int64_t)r_lo * W + tid; i < (int64_t)r_hi * W; i += BS) {
      ps_bits(sd, 0)[(size_t)I.v_off * W + i] = sbits[i];
      ps_bits(sd, 1)[(size_t)I.v_off * W + i] = sbits[vw + i];
    }
  }
  // the last block to finish advances the step counter for the whole batch
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const int prev = atomicAdd(&hdr->blocks_done, 1);
    if (prev == (int)gridDim.x - 1) {
      __threadfence();
      int active = 0;
      int64_t tlast = t0;
      for (int j = 0; j < pd.n_inst; ++j) {
        const volatile InstState *js = sd.inst + j;
        if (js->found) {
          const int64_t fs = js->found_step;
          if (fs > tlast) tlast = fs;
        } else {
          ++active;
        }
      }
      hdr->n_active = active;
      if (active == 0 && hy.stop_on_sat) {
        hdr->all_done = 1;
        hdr->t = tlast;        // the step that froze the last instance, as the multi-kernel path leaves it
      } else {
        hdr->t = t0 + K;
      }
      hdr->blocks_done = 0;
    }
  }
}

// histograms [HP][8][N] int32 (HP = 2 step parities with clusters), the table
// (272 floats per 32-sample word), S and the unsatisfied counts [N] each, the
// bits [2][vmax][N/32]; resident: z, m, v of one block's rows
// [vown][N/32][33] and their normaliser [vown], vown = ceil(vmax / cs)
int64_t persist_smem_bytes(int N, int32_t vmax, bool resident, int cs) {
  const int64_t vw = (int64_t)vmax * (N / 32), vown = (vmax + cs - 1) / cs, ow = vown * (N / 32);
  const int64_t hp = cs > 1 ? 2 : 1;
  return 4 * (hp * 8LL * N + 272LL * (N / 32) + 2LL * N + 2 * vw + (resident ? 3 * 33 * ow + vown : 0));
}

cudaError_t launch_persist(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const LrSched &ls, int32_t K,
                           int32_t vmax, bool resident, int cs, cudaStream_t st) {
  const int smem = (int)persist_smem_bytes(sd.N, vmax, resident, cs);
  const int32_t vown = (vmax + cs - 1) / cs;
  auto go = [&](auto kern, int block) -> cudaError_t {
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(kern), smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(pd.n_inst * cs));
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = cs > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, pd, sd, hy, ls, K, vmax, vown);
  };
  const bool ph = hy.binarize == TSAT_BIN_PHILOX;
  // samples per thread: resident instances run at 512 threads (16), the
  // others hide their global z, m, v latency with 1024 (8); measured at
  // N = 32..256, n = 100..1000 (16 is 16-31 % faster when resident, 8 is
  // 8-20 % faster when not)
  const int spt = sd.N > 256 ? 32 : (resident ? 16 : 8);
  if (cs > 1 && spt == 32) return cudaErrorInvalidValue;
  const bool split = cs > 1;
  // (clusters only with N <= 256: SPT 8 or 16)
#define PS_GO2(B, M, R, S) (split ? go(k_persist<B, M, R, S, true>, ps_block<S>()) : go(k_persist<B, M, R, S, false>, ps_block<S>()))
#define PS_GO1(B, M, S) (resident ? PS_GO2(B, M, true, S) : PS_GO2(B, M, false, S))
#define PS_GO32(B, M) (resident ? go(k_persist<B, M, true, 32, false>, 256) : go(k_persist<B, M, false, 32, false>, 256))
#define PS_GO(B, M) (spt == 8 ? PS_GO1(B, M, 8) : (spt == 16 ? PS_GO1(B, M, 16) : PS_GO32(B, M)))
  switch (hy.norm) {
    case TSAT_NORM_SIGNED_MEAN:
      return ph ? PS_GO(TSAT_BIN_PHILOX, TSAT_NORM_SIGNED_MEAN) : PS_GO(TSAT_BIN_DET, TSAT_NORM_SIGNED_MEAN);
    case TSAT_NORM_ABSMEAN:
      return ph ? PS_GO(TSAT_BIN_PHILOX, TSAT_NORM_ABSMEAN) : PS_GO(TSAT_BIN_DET, TSAT_NORM_ABSMEAN);
    default:
      return ph ? PS_GO(TSAT_BIN_PHILOX, TSAT_NORM_NONE) : PS_GO(TSAT_BIN_DET, TSAT_NORM_NONE);
  }
#undef PS_GO
#undef PS_GO32
#undef PS_GO1
#undef PS_GO2
}

}  // namespace tsat
