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
// multi-kernel path: G is summed per sample in occurrence order exactly as the
// clause-length 4..7 update kernel does, and an instance freezes at the step
// whose forward finds a sample with no unsatisfied clause.
#include "internal.h"
#include "kernels.cuh"

namespace tsat {

constexpr int kPsBlock = 256, kPsWarps = kPsBlock / 32;

// dL/dR table of one sample: 8 floats (r = 0..7); each word's 32 samples are
// followed by 8 floats of padding (264 floats per word), so that the lanes of
// one lookup (same bit, rows at different words) start on different banks
__device__ __forceinline__ int ps_tab(int s) { return 8 * s + 8 * (s >> 5); }

__device__ __forceinline__ uint32_t *ps_bits(const StateDev &sd, int64_t t) {
  return sd.bits + (size_t)(t & 1) * (size_t)sd.V * sd.W;
}

// RES: the instance's z, m, v and normaliser stay in shared memory for the
// whole launch (layout [row][word][33]: a lane's 32 samples start on their
// own bank) and are written back once at the end; otherwise they are read and
// written in global memory at every step.
template <int BIN, int NORM, bool RES>
__global__ void __launch_bounds__(kPsBlock, 2) k_persist(ProbDev pd, StateDev sd, Hyper hy, LrSched ls, int32_t K,
                                                         int32_t vmax) {
  extern __shared__ __align__(16) float smP[];
  __shared__ int64_t sh_t0;
  __shared__ int sh_skip, sh_found;
  __shared__ float sh_ls[kPsWarps], etab[8];
  __shared__ int sh_mu[kPsWarps], sh_mi[kPsWarps];
  __shared__ StepParams sh_sps[kPsBlock];   // step scalars of the next kPsBlock steps, one per thread
  StateHdr *hdr = sd.hdr;
  const int inst = blockIdx.x;
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
  int32_t *hist = reinterpret_cast<int32_t *>(smP);   // [lmax + 1][N]
  float *tab = smP + 8 * N;                             // [N][8] with 8 floats of padding per word (ps_tab)
  // the instance's bits, both step parities, rows numbered from the instance's
  // first variable: every gather of the forward and the backward reads them here
  uint32_t *sbits = reinterpret_cast<uint32_t *>(tab + 264 * W);   // [2][vmax][W]
  const size_t vw = (size_t)vmax * W;
  for (int64_t i = tid; i < (int64_t)I.n_vars * W; i += kPsBlock)
    sbits[(t0 & 1) * vw + i] = ps_bits(sd, t0)[(size_t)I.v_off * W + i];
  float *smz = reinterpret_cast<float *>(sbits + 2 * vw);   // RES: z, m, v [vmax][W][33], then nu [vmax]
  float *smm = smz + vw * 33, *smv = smm + vw * 33, *snu = smv + vw * 33;
  const size_t g0 = (size_t)I.v_off * N;
  if (RES && !sh_found) {
    for (int64_t i = tid; i < (int64_t)I.n_vars * N; i += kPsBlock) {
      const size_t si = (size_t)(i / 32) * 33 + (i & 31);   // [row][word][33]: word index i / 32 of the row-major array
      smz[si] = sd.z[g0 + i];
      smm[si] = sd.m[g0 + i];
      smv[si] = sd.v[g0 + i];
    }
    for (int i = tid; i < I.n_vars; i += kPsBlock) snu[i] = sd.nu[I.v_off + i];
  }
  __syncthreads();
  int found = sh_found;
  const bool ran = !found;   // the instance is live at the start of the launch
  int64_t t = t0;
  for (int32_t k = 0; k < K && !found; ++k, ++t) {
    if (k % kPsBlock == 0) {   // the double-precision schedule of the next kPsBlock steps, in parallel
      sh_sps[tid] = step_params(ls, t + tid);
      __syncthreads();
    }
    // ---- forward (Eq. 1): lane = clause, 32 samples of word w; bit-sliced R,
    // warp transpose, popcounts of the R = r masks into the block histogram
    for (int i = tid; i < (lmax + 1) * N; i += kPsBlock) hist[i] = 0;
    __syncthreads();
    const uint32_t *bsrc = sbits + (t & 1) * vw;
    const int ngroups = (I.n_clauses + 31) >> 5;
    for (int task = warp; task < ngroups * W; task += kPsWarps) {
      const int g = task / W, w = task - g * W;
      const bool active = 32 * g + lane < I.n_clauses;
      uint32_t pl[3] = {0u, 0u, 0u};
      if (active) {
        const int c = I.c_off + 32 * g + lane;
        const int32_t b = __ldg(pd.cptr + c), e = __ldg(pd.cptr + c + 1);
        for (int32_t j = b; j < e; ++j) {
          const int32_t lit = __ldg(pd.clit + j);
          bitslice_add<3>(pl, bsrc[(size_t)((lit >> 1) - I.v_off) * W + w] ^ (0u - (uint32_t)(lit & 1)));
        }
      }
      const uint32_t valid = __ballot_sync(0xFFFFFFFFu, active);
      uint32_t tp[3];
#pragma unroll
      for (int p = 0; p < 3; ++p) tp[p] = warp_transpose32(pl[p], lane);
      for (int r = 0; r <= lmax; ++r) {
        const int cnt = __popc(valid & bitslice_eq<3>(tp, r));
        if (cnt) atomicAdd(hist + r * N + 32 * w + lane, cnt);
      }
    }
    __syncthreads();
    // ---- Eq. 4 per sample, the dL/dR table, loss, fewest-unsatisfied sample
    float lsum = 0.f;
    int mu = 0x7FFFFFFF, mi = 0x7FFFFFFF;
    for (int i = tid; i < N; i += kPsBlock) {
      float Z = 0.f, Y = 0.f;
      for (int r = 0; r <= lmax; ++r) {
        const float hv = (float)hist[r * N + i];
        Z += hv * etab[r];
        Y += (float)r * hv * etab[r];
      }
      const float S = Y / Z;
      const float invZ = 1.0f / Z;
#pragma unroll
      for (int r = 0; r < 8; ++r)
        tab[ps_tab(i) + r] = r <= lmax ? -(etab[r] * invZ) * (1.0f - hy.tau * ((float)r - S)) : 0.f;
      const int h0 = hist[i];
      lsum += S;
      if (h0 < mu || (h0 == mu && i < mi)) { mu = h0; mi = i; }
      sd.S[(size_t)inst * N + i] = S;
      sd.unsat[(size_t)inst * N + i] = h0;
    }
    for (int o = 16; o > 0; o >>= 1) {
      lsum += __shfl_xor_sync(0xFFFFFFFFu, lsum, o);
      const int u2 = __shfl_xor_sync(0xFFFFFFFFu, mu, o), i2 = __shfl_xor_sync(0xFFFFFFFFu, mi, o);
      if (u2 < mu || (u2 == mu && i2 < mi)) { mu = u2; mi = i2; }
    }
    if (lane == 0) { sh_ls[warp] = lsum; sh_mu[warp] = mu; sh_mi[warp] = mi; }
    __syncthreads();
    if (tid == 0) {
      float L = 0.f;
      for (int q = 0; q < kPsWarps; ++q) {
        L += sh_ls[q];
        if (sh_mu[q] < mu || (sh_mu[q] == mu && sh_mi[q] < mi)) { mu = sh_mu[q]; mi = sh_mi[q]; }
      }
      InstState *is = sd.inst + inst;
      is->loss = -L;
      is->min_unsat = mu;
      is->best_sample = mi;
      if (mu == 0) {
        is->found = 1;
        is->found_sample = mi;
        is->found_step = t;
        sh_found = 1;
      }
    }
    __syncthreads();
    found = sh_found;
    if (found) break;   // the bits of step t are the model; z, m, v stay
    // ---- fused update: thread = (row, word w); G of its 32 samples summed over
    // the row's occurrences in record order, then Eq. 5, AdamW, the new
    // normaliser and the bits of step t + 1
    const StepParams sp = sh_sps[k % kPsBlock];
    uint32_t *bdst = ps_bits(sd, t + 1), *sdst = sbits + ((t + 1) & 1) * vw;
    const int rpp = kPsBlock / W;
    for (int vb = 0; vb < I.n_vars; vb += rpp) {
      const int vl = vb + tid / W, w = tid % W;
      const bool act = vl < I.n_vars;
      const int64_t v = (int64_t)I.v_off + vl;
      float acc[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = 0.f;
      if (act) {
        const uint32_t own = bsrc[(size_t)vl * W + w];
        const int32_t o0 = __ldg(pd.vptr + v), o1 = __ldg(pd.vptr + v + 1);
        const int tb = ps_tab(32 * w);
        for (int32_t o = o0; o < o1; ++o) {
          const int32_t *rec = pd.xrec + (size_t)pd.rec_stride * o;
          const int32_t h = __ldg(rec);
          const int len = h >> 1;
          uint32_t pl[3] = {own ^ (0u - (uint32_t)(h & 1)), 0u, 0u};
          for (int q = 1; q < len; ++q) {
            const int32_t lit = __ldg(rec + q);
            bitslice_add<3>(pl, bsrc[(size_t)((lit >> 1) - I.v_off) * W + w] ^ (0u - (uint32_t)(lit & 1)));
          }
          const float sg = (h & 1) ? -1.0f : 1.0f;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int r = (int)(((pl[0] >> j) & 1u) | (((pl[1] >> j) & 1u) << 1) | (((pl[2] >> j) & 1u) << 2));
            acc[j] = fmaf(sg, tab[tb + 8 * j + r], acc[j]);
          }
        }
      }
      const size_t off = RES ? ((size_t)vl * W + w) * 33 : (size_t)v * N + 32 * w;
      float *zp = RES ? smz : sd.z, *mp = RES ? smm : sd.m, *vp = RES ? smv : sd.v;
      const float nu = act ? (RES ? snu[vl] : sd.nu[v]) : 1.0f;
      const float rnu = __frcp_rn(nu);
      float part = 0.f;
      if (act && NORM != TSAT_NORM_NONE) {
#pragma unroll
        for (int j = 0; j < 32; ++j) part = fmaf(acc[j], zp[off + j], part);
      }
      const float dot = seg_sum(part, W);
      const float c2 = dot * rnu * rnu * (1.0f / (float)N);
      float psum = 0.f;
      if (act) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
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
      const float tot = seg_sum(psum, W);
      if (act) {
        const float nun = (NORM == TSAT_NORM_NONE) ? 1.0f : guard_nu(tot / (float)N);
        const float rnn = __frcp_rn(nun);
        uint32_t word = 0;
        if constexpr (BIN == TSAT_BIN_PHILOX) {
#pragma unroll
          for (int h = 0; h < 4; ++h) {   // samples 32 w + 8 h + e: block 4 w + h, half e
            const uint4 r = philox4x32_10(make_uint4((uint32_t)(4 * w + h), (uint32_t)v, (uint32_t)(t + 1), kTagBin),
                                          hy.key0, hy.key1);
#pragma unroll
            for (int e = 0; e < 8; ++e)
              word |= binarize_one(__fmul_rn(acc[8 * h + e], rnn), TSAT_BIN_PHILOX, hy.bin_c,
                                   half16(e < 4 ? r.x : r.z, e < 4 ? r.y : r.w, e & 3))
                      << (8 * h + e);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) word |= (__fmul_rn(acc[j], rnn) > 0.0f ? 1u : 0u) << j;
        }
        if (!RES) bdst[v * W + w] = word;
        sdst[(size_t)vl * W + w] = word;
        if (w == 0) {
          if (RES) snu[vl] = nun;
          else sd.nu[v] = nun;
        }
      }
    }
    __syncthreads();   // the bits, z and normaliser of step t + 1 are written before its forward
  }
  // an instance found in this launch keeps its model in both bit buffers (the
  // multi-kernel path copies a frozen instance's bits at every step)
  __syncthreads();
  if (found && ran) {
    const int64_t tf = sd.inst[inst].found_step;
    for (int64_t i = tid; i < (int64_t)I.n_vars * W; i += kPsBlock) {
      if (RES) sbits[((tf + 1) & 1) * vw + i] = sbits[(tf & 1) * vw + i];
      else ps_bits(sd, tf + 1)[(size_t)I.v_off * W + i] = ps_bits(sd, tf)[(size_t)I.v_off * W + i];
    }
  }
  if (RES && ran) {   // write the resident state back
    __syncthreads();
    for (int64_t i = tid; i < (int64_t)I.n_vars * N; i += kPsBlock) {
      const size_t si = (size_t)(i / 32) * 33 + (i & 31);
      sd.z[g0 + i] = smz[si];
      sd.m[g0 + i] = smm[si];
      sd.v[g0 + i] = smv[si];
    }
    for (int i = tid; i < I.n_vars; i += kPsBlock) sd.nu[I.v_off + i] = snu[i];
    for (int64_t i = tid; i < (int64_t)I.n_vars * W; i += kPsBlock) {
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

// histogram [8][N] int32, then the table: 264 floats per 32-sample word
// histogram [8][N] int32, the table (264 floats per 32-sample word), the bits
// [2][vmax][N/32]; resident: z, m, v [vmax][N/32][33] and the normaliser [vmax]
int64_t persist_smem_bytes(int N, int32_t vmax, bool resident) {
  const int64_t vw = (int64_t)vmax * (N / 32);
  return 4 * (8LL * N + 264LL * (N / 32) + 2 * vw + (resident ? 3 * 33 * vw + vmax : 0));
}

cudaError_t launch_persist(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const LrSched &ls, int32_t K,
                           int32_t vmax, bool resident, cudaStream_t st) {
  const int smem = (int)persist_smem_bytes(sd.N, vmax, resident);
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<pd.n_inst, kPsBlock, smem, st>>>(pd, sd, hy, ls, K, vmax);
    return cudaGetLastError();
  };
  const bool ph = hy.binarize == TSAT_BIN_PHILOX;
#define PS_GO(B, M) (resident ? go(k_persist<B, M, true>) : go(k_persist<B, M, false>))
  switch (hy.norm) {
    case TSAT_NORM_SIGNED_MEAN:
      return ph ? PS_GO(TSAT_BIN_PHILOX, TSAT_NORM_SIGNED_MEAN) : PS_GO(TSAT_BIN_DET, TSAT_NORM_SIGNED_MEAN);
    case TSAT_NORM_ABSMEAN:
      return ph ? PS_GO(TSAT_BIN_PHILOX, TSAT_NORM_ABSMEAN) : PS_GO(TSAT_BIN_DET, TSAT_NORM_ABSMEAN);
    default:
      return ph ? PS_GO(TSAT_BIN_PHILOX, TSAT_NORM_NONE) : PS_GO(TSAT_BIN_DET, TSAT_NORM_NONE);
  }
#undef PS_GO
}

}  // namespace tsat
