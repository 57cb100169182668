// kernels.cuh -- declarations of the step kernels (definitions in kernels.cu).
#pragma once
#include "common.cuh"

namespace tsat {

struct LrSched {
  float lr0, factor, floor, wd;
  int32_t period, restart;
  double beta1, beta2;
  int32_t mix;   // assignment mixing at each restart
};

// launch helpers (return cudaGetLastError of the launch)
cudaError_t launch_init(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const float *logits,
                        float scale, int grid, cudaStream_t st);
cudaError_t launch_mix(const ProbDev &pd, const StateDev &sd, const Hyper &hy, int grid, cudaStream_t st);
cudaError_t launch_binarize(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const float *zin,
                            int64_t t_bin, int grid, cudaStream_t st);
cudaError_t launch_fwd_hist(const ProbDev &pd, const StateDev &sd, int32_t *hist, int skip_frozen,
                            cudaStream_t st);
cudaError_t launch_gamma(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const LrSched &ls,
                         const int32_t *hist_in, int step_mode, int write_gamma, float *loss_out, float *S_out,
                         cudaStream_t st);
cudaError_t launch_update(const ProbDev &pd, const StateDev &sd, const Hyper &hy, int mode,
                          const float *zin, float *grad, float dL, int grid, int rows_per_item,
                          cudaStream_t st);
cudaError_t launch_check(const ProbDev &pd, const StateDev &sd, int32_t *unsat, uint32_t *satmask,
                         cudaStream_t st);
cudaError_t launch_relaxed_lits(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const float *zin,
                                int grid, cudaStream_t st);
cudaError_t launch_relaxed_fwd(const ProbDev &pd, const StateDev &sd, const Hyper &hy, int skip_frozen,
                               cudaStream_t st);
cudaError_t launch_relaxed_gamma(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const LrSched &ls,
                                 int step_mode, float *loss_out, float *S_out, cudaStream_t st);

// tsat_best helpers (best.cu)
cudaError_t best_pick(const int32_t *unsat, int N, int32_t *small, cudaStream_t st);
cudaError_t best_gcol(const ProbDev &pd, const StateDev &sd, const Hyper &hy, int inst, int n_vars,
                      int n_clauses, const int32_t *small, int32_t *hist1, float *gcol, cudaStream_t st);
cudaError_t best_select(const ProbDev &pd, const StateDev &sd, int inst, int n_vars, int k,
                        const float *gcol, unsigned long long *sel, int32_t *digits, int64_t *selstate,
                        int32_t *small, int32_t *part_var, uint8_t *part_val, uint32_t *outbits,
                        cudaStream_t st);
void prepare_update_attrs(int lmax);
int update_blocks_per_sm(const ProbDev &pd, const StateDev &sd);
int update_warps_per_block(const ProbDev &pd, const StateDev &sd);

int update_smem_bytes(int N, int lm1, bool greg);

}  // namespace tsat
