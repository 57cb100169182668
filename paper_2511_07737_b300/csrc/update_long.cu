// update_long.cu -- the fused update for clause length 4..7 (Sec. III-B
// straight-through backward through P^T, Eq. 5 chain rule, AdamW with the
// Sec. IV-A schedule, Eq. 2 / Philox re-binarisation), word per lane.
#include "update_long.cuh"

namespace tsat {

// ------------------------------------------------------------------ fused update, clause length 4..7
// The warp-level row-group body (updateL_rows) and the table layout live in
// update_long.cuh.
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
      updateL_rows<MODE, BIN, NORM, STAB>(pd, sd, hy, sp, tcur, bsrc, bdst, zsrc, grad, dL, smb, tbase, tskew, gbuf,
                                          sd.gamma + (size_t)cur * lm1 * N + 32 * w, cur, v, act, frozen, lane, w,
                                          rbase);
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
