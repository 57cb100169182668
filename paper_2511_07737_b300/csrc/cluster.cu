// cluster.cu -- persistent solver for batches whose instances are too large
// for one thread block: many optimisation steps (Sec. III-B, IV-A) of a whole
// batch in one launch of thread-block clusters.
//
// A cluster (kClSize blocks of kClBlock threads, one block per SM) owns a bin
// of instances, dealt by the host so that the bins hold about the same number
// of literal occurrences (largest first).  The cluster works through its bin
// one instance at a time with every warp of its blocks on that instance, and
// runs the instance's steps back to back:
//   forward (Eq. 1): 32 clauses x one or two sample words per warp task, into
//     the block's histogram of R (one per step parity);
//   cluster barrier; each block sums the blocks' histograms over distributed
//     shared memory and forms Eq. 4, the loss and the dL/dR table of every
//     sample (every block gets the same integers, so every block takes the
//     same decisions -- found, stop -- without further communication);
//   the fused update of the instance's rows (the row-group body of the
//     multi-kernel update for clause length 4..7: straight-through sum over
//     the occurrences, Eq. 5, AdamW, the bits of the next step);
//   cluster barrier (the next forward reads those bits).
// Barriers are the hardware cluster barrier; no block ever spins on memory.
// Data written in the launch by other blocks (the bits, z) is read with
// ordinary cached loads after a barrier (release / acquire at cluster scope),
// never through the read-only path.
// Every block of a cluster runs the same sequence of barriers, and a block
// leaves only after a last cluster barrier, so no block reads the shared
// memory of a block that has exited.  Results follow tsat_step: freezing at
// the first sample with no unsatisfied clause (both bit buffers keep the
// model), the status records, S and unsatisfied counts of the last forward,
// the step counter (advanced by the last block to finish).
#include <cooperative_groups.h>

#include <algorithm>

#include "internal.h"
#include "update_long.cuh"

namespace cg = cooperative_groups;

namespace tsat {

constexpr int kClBlock = 768;                // threads per block: 24 warps, one block per SM
constexpr int kClWarps = kClBlock / 32;
constexpr int kClSize = 4;                   // blocks per cluster (C3: 51.6 ms per step at 4, 61.8 at 8, 97.8 at 2)
constexpr int kClSched = 256;                // steps whose scalars are formed at once

// dynamic shared memory: the gamma table (256-byte aligned, first), the warps'
// [32][33] buffers, two step-parity histograms [8][N], S and unsat [N]
__host__ __device__ inline int cl_gbuf_off(int N) { return updateL_tab_span(N); }
__host__ __device__ inline int cl_hist_off(int N) { return cl_gbuf_off(N) + kClWarps * 32 * kGS; }
__host__ __device__ inline int cl_s_off(int N) { return cl_hist_off(N) + 2 * 8 * N; }
__host__ __device__ inline int cl_smem_floats(int N) { return cl_s_off(N) + 2 * N; }

template <int BIN, int NORM>
__global__ void __launch_bounds__(kClBlock, 1)
    k_cluster(ProbDev pd, StateDev sd, Hyper hy, LrSched ls, int32_t K, const int32_t *bin_ptr,
              const int32_t *bin_inst) {
  extern __shared__ __align__(256) float smC[];
  __shared__ StepParams sh_sps[kClSched];
  __shared__ float etab[8];
  __shared__ int64_t sh_t0;
  __shared__ int sh_skip;
  __shared__ float sh_L;
  __shared__ int sh_mu, sh_mi;
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int cid = (int)(blockIdx.x / CS);
  const int N = sd.N, W = sd.W, RW = 32 / W;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rsub = lane / W, w = lane % W, rbase = rsub * W;
  StateHdr *hdr = sd.hdr;
  if (tid == 0) {
    sh_t0 = hdr->t;
    sh_skip = hdr->all_done;
  }
  if (tid < 8) etab[tid] = expf(-hy.tau * (float)tid);
  __syncthreads();
  if (sh_skip) return;   // stopped before this launch: every block of every cluster leaves here
  const int64_t t0 = sh_t0;
  float *tab = smC;                                          // [N][8] + skew (update_long.cuh layout)
  float *gbuf = smC + cl_gbuf_off(N) + warp * 32 * kGS;      // this warp's [32][33]
  int32_t *hist = reinterpret_cast<int32_t *>(smC + cl_hist_off(N));   // [2 parities][8][N] partial
  float *sS = smC + cl_s_off(N);
  int32_t *sU = reinterpret_cast<int32_t *>(sS + N);
  const char *smb = reinterpret_cast<const char *>(smC);
  const uint32_t tbase = (uint32_t)(1024 * w);               // the table sits at offset 0
  const uint32_t tskew = 0x01010101u * (32u * (uint32_t)(w & 3));
  const int gw = rank * kClWarps + warp, nw = CS * kClWarps;   // warp within the cluster
  for (int bi = bin_ptr[cid]; bi < bin_ptr[cid + 1]; ++bi) {
    const int inst = bin_inst[bi];
    const InstInfo I = pd.inst[inst];
    if (sd.inst[inst].found) continue;   // frozen before this launch (read by every block before any write)
    const int lmax = I.lmax;
    for (int i = tid; i < 2 * 8 * N; i += kClBlock) hist[i] = 0;
    __syncthreads();
    int found = 0, fsample = -1;
    int64_t fstep = -1, t = t0;
    for (int32_t k = 0; k < K; ++k, ++t) {
      if (k % kClSched == 0) {
        if (tid < kClSched) sh_sps[tid] = step_params(ls, t + tid);
        __syncthreads();
      }
      // ---- forward (Eq. 1) of step t into this block's histogram of parity t & 1
      const uint32_t *bsrc = cur_bits(sd, t);
      int32_t *hcur = hist + (t & 1) * 8 * N;
      const int WT = W >= 2 ? 2 : 1, wtasks = W / WT;
      const int ngc = (I.n_clauses + 31) >> 5;
      for (int task = gw; task < ngc * wtasks; task += nw) {
        const int g = task / wtasks, w0 = (task - g * wtasks) * WT;
        const bool active = 32 * g + lane < I.n_clauses;
        uint32_t pl[2][3] = {};
        if (active) {
          const int c = I.c_off + 32 * g + lane;
          const int32_t b = __ldg(pd.cptr + c), e = __ldg(pd.cptr + c + 1);
          for (int32_t j = b; j < e; ++j) {
            const int32_t lit = __ldg(pd.clit + j);
            const uint32_t *row = bsrc + (size_t)(lit >> 1) * W + w0, neg = 0u - (uint32_t)(lit & 1);
            bitslice_add<3>(pl[0], __ldca(row) ^ neg);
            if (WT == 2) bitslice_add<3>(pl[1], __ldca(row + 1) ^ neg);
          }
        }
        const uint32_t valid = __ballot_sync(0xFFFFFFFFu, active);
#pragma unroll
        for (int ww = 0; ww < 2; ++ww) {
          if (ww >= WT) break;
          uint32_t tp[3];
          tp[0] = warp_transpose32(pl[ww][0], lane);
          tp[1] = warp_transpose32(pl[ww][1], lane);
          tp[2] = warp_transpose32(pl[ww][2], lane);
          for (int r = 0; r <= lmax; ++r) {
            const int cnt = __popc(valid & bitslice_eq<3>(tp, r));
            if (cnt) atomicAdd(hcur + r * N + 32 * (w0 + ww) + lane, cnt);
          }
        }
      }
      cl.sync();   // every block's histogram of step t is complete
      // ---- the instance's histogram (sum over the cluster's blocks), Eq. 4,
      // the loss, the dL/dR table and the fewest-unsatisfied sample
      // the blocks' partial histograms summed entry by entry over all threads
      // (into this block's histogram of the other parity, cleared below for
      // the next step), then Eq. 4 per sample
      int32_t *hsum = hist + ((t + 1) & 1) * 8 * N;
      for (int e = tid; e < (lmax + 1) * N; e += kClBlock) {
        int32_t hs = 0;
        for (int q = 0; q < CS; ++q) hs += cl.map_shared_rank(hcur, q)[e];
        hsum[e] = hs;
      }
      __syncthreads();
      for (int i = tid; i < N; i += kClBlock) {
        float Z = 0.f, Y = 0.f;
        const int32_t h0 = hsum[i];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          if (r <= lmax) {
            const float hv = (float)hsum[r * N + i];
            Z += hv * etab[r];
            Y += (float)r * hv * etab[r];
          }
        }
        const float S = Y / Z;
        const float invZ = 1.0f / Z;
#pragma unroll
        for (int r = 0; r < 8; ++r)
          tab[ltab_off(i) + r] = r <= lmax ? -(etab[r] * invZ) * (1.0f - hy.tau * ((float)r - S)) : 0.f;
        sS[i] = S;
        sU[i] = h0;
      }
      __syncthreads();
      if (warp == 0) {
        float L = 0.f;
        int mu = 0x7FFFFFFF, mi = 0x7FFFFFFF;
        for (int i = lane; i < N; i += 32) {
          L += sS[i];
          if (sU[i] < mu) { mu = sU[i]; mi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          L += __shfl_xor_sync(0xFFFFFFFFu, L, o);
          const int u2 = __shfl_xor_sync(0xFFFFFFFFu, mu, o), i2 = __shfl_xor_sync(0xFFFFFFFFu, mi, o);
          if (u2 < mu || (u2 == mu && i2 < mi)) { mu = u2; mi = i2; }
        }
        if (lane == 0) {
          sh_L = -L;
          sh_mu = mu;
          sh_mi = mi;
        }
      }
      __syncthreads();
      if (sh_mu == 0) {   // the same integers in every block: every block stops here
        found = 1;
        fsample = sh_mi;
        fstep = t;
        cl.sync();        // every block has read every histogram of this step
        break;
      }
      // the other parity's histogram: its readers finished before the last barrier
      for (int i = tid; i < 8 * N; i += kClBlock) hist[((t + 1) & 1) * 8 * N + i] = 0;
      // ---- fused update of the instance's rows (row groups over the cluster's warps)
      const StepParams sp = sh_sps[k % kClSched];
      uint32_t *bdst = const_cast<uint32_t *>(cur_bits(sd, t + 1));
      const int ngr = (I.n_vars + RW - 1) / RW;
      for (int g = gw; g < ngr; g += nw) {
        const int vl = g * RW + rsub;
        __syncwarp();   // the previous group's readers of gbuf are done
        updateL_rows<0, BIN, NORM, true, true>(pd, sd, hy, sp, t, bsrc, bdst, sd.z, nullptr, 0.f, smb, tbase, tskew,
                                               gbuf, nullptr, inst, (int64_t)I.v_off + vl, vl < I.n_vars, false,
                                               lane, w, rbase);
      }
      cl.sync();   // the bits, z and normaliser of step t + 1 are written
    }
    // the instance's status, S and unsatisfied counts of its last forward (every
    // block holds the same values; block 0 writes them)
    if (rank == 0 && K > 0) {
      for (int i = tid; i < N; i += kClBlock) {
        sd.S[(size_t)inst * N + i] = sS[i];
        sd.unsat[(size_t)inst * N + i] = sU[i];
      }
      if (tid == 0) {
        InstState *is = sd.inst + inst;
        is->loss = sh_L;
        is->min_unsat = sh_mu;
        is->best_sample = sh_mi;
        if (found) {
          is->found = 1;
          is->found_sample = fsample;
          is->found_step = fstep;
        }
      }
    }
    // a model found in this launch is kept in both bit buffers
    if (found) {
      const uint32_t *src = cur_bits(sd, fstep);
      uint32_t *dst = const_cast<uint32_t *>(cur_bits(sd, fstep + 1));
      for (int64_t i = (int64_t)rank * kClBlock + tid; i < (int64_t)I.n_vars * W; i += (int64_t)CS * kClBlock)
        dst[(size_t)I.v_off * W + i] = __ldca(src + (size_t)I.v_off * W + i);
    }
    __syncthreads();
  }
  cl.sync();   // no block leaves while another may still read its shared memory
  // the last block to finish advances the step counter for the whole batch
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
        hdr->t = tlast;
      } else {
        hdr->t = t0 + K;
      }
      hdr->blocks_done = 0;
    }
  }
}

int cluster_smem_bytes(int N) { return cl_smem_floats(N) * (int)sizeof(float); }

// Clusters that fit on the device at once (the launch's grid).
static int cluster_count(const void *kern, int smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClSize);
  cfg.blockDim = dim3(kClBlock);
  cfg.dynamicSmemBytes = (size_t)smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kClSize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) return 0;
  return n;
}

int cluster_grid_clusters(int N) {
  const int smem = cluster_smem_bytes(N);
  const void *k = reinterpret_cast<const void *>(k_cluster<TSAT_BIN_DET, TSAT_NORM_ABSMEAN>);
  if (ensure_dyn_smem(k, smem) != cudaSuccess) return 0;
  return cluster_count(k, smem);
}

// Instances to clusters, largest first onto the bin with the fewest occurrences
// so far (a per-instance constant stands for the fixed cost of its steps).
void cluster_bins(const tsat_problem *p, int ncl, std::vector<int32_t> &ptr, std::vector<int32_t> &list) {
  std::vector<int64_t> cost(p->n_inst);
  std::vector<int32_t> order(p->n_inst);
  for (int j = 0; j < p->n_inst; ++j) {
    cost[j] = p->inst_nnz[j] + (1 << 15);
    order[j] = j;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<int64_t> load(ncl, 0);
  std::vector<std::vector<int32_t>> bins(ncl);
  for (int j : order) {
    int best = 0;
    for (int c = 1; c < ncl; ++c)
      if (load[c] < load[best]) best = c;
    bins[best].push_back(j);
    load[best] += cost[j];
  }
  ptr.assign(ncl + 1, 0);
  list.clear();
  for (int c = 0; c < ncl; ++c) {
    list.insert(list.end(), bins[c].begin(), bins[c].end());
    ptr[c + 1] = (int32_t)list.size();
  }
}

cudaError_t launch_cluster(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const LrSched &ls, int32_t K,
                           int ncl, const int32_t *bin_ptr, const int32_t *bin_inst, cudaStream_t st) {
  const int smem = cluster_smem_bytes(sd.N);
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(kern), smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ncl * kClSize);
    cfg.blockDim = dim3(kClBlock);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kClSize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, pd, sd, hy, ls, K, bin_ptr, bin_inst);
  };
  const bool ph = hy.binarize == TSAT_BIN_PHILOX;
  switch (hy.norm) {
    case TSAT_NORM_SIGNED_MEAN:
      return ph ? go(k_cluster<TSAT_BIN_PHILOX, TSAT_NORM_SIGNED_MEAN>) : go(k_cluster<TSAT_BIN_DET, TSAT_NORM_SIGNED_MEAN>);
    case TSAT_NORM_ABSMEAN:
      return ph ? go(k_cluster<TSAT_BIN_PHILOX, TSAT_NORM_ABSMEAN>) : go(k_cluster<TSAT_BIN_DET, TSAT_NORM_ABSMEAN>);
    default:
      return ph ? go(k_cluster<TSAT_BIN_PHILOX, TSAT_NORM_NONE>) : go(k_cluster<TSAT_BIN_DET, TSAT_NORM_NONE>);
  }
}

}  // namespace tsat
