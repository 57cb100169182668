// kernels.cuh -- declarations of the step kernels (definitions in kernels.cu).
#pragma once
#include "common.cuh"

namespace tsat {

constexpr int kLrTab = 16;
struct LrSched {
  float lr0, factor, floor, wd;
  int32_t period, restart;
  double beta1, beta2;
  int32_t mix;   // assignment mixing at each restart
  // formed on the host in double: lr of decay step k (max(lr0 factor^k, floor)
  // for k < n_lr, when restarts bound k; n_lr = 0: the device forms it) and
  // log2 of the two moment decays
  int32_t n_lr;
  double lr_tab[kLrTab];
  double l2b1, l2b2;
};

// Scalars of step t (Sec. IV-A): lr(t) = max(lr0 factor^floor((t mod restart) / period), floor),
// AdamW bias corrections with the 1-based step count (counted from the last
// restart when assignments are mixed), decoupled weight decay.  Formed in
// double, stored as float.  Each double-precision part is a serial chain of a
// few microseconds, so step_part(ls, t, j) forms part j alone (0: lr, 1:
// 1 / (1 - beta1^cnt), 2: 1 / sqrt(1 - beta2^cnt)) for three threads to form
// side by side, and step_finish combines them.
__device__ __forceinline__ double step_part(const LrSched &ls, int64_t t, int j) {
  if (j == 0) {
    const int64_t tt = ls.restart > 0 ? t % ls.restart : t;
    const int64_t kdec = ls.period > 0 ? tt / ls.period : 0;
    if (kdec < ls.n_lr) return ls.lr_tab[kdec];
    const double lr = (double)ls.lr0 * pow((double)ls.factor, (double)kdec);
    return lr < (double)ls.floor ? (double)ls.floor : lr;
  }
  // beta^cnt as 2^(cnt log2 beta): one double exponential instead of a power
  const int64_t cnt = (ls.mix && ls.restart > 0 && t >= ls.restart) ? t % ls.restart : t + 1;
  const double bc = 1.0 - exp2((double)cnt * (j == 1 ? ls.l2b1 : ls.l2b2));
  return j == 1 ? 1.0 / bc : 1.0 / sqrt(bc);
}

__device__ __forceinline__ StepParams step_finish(const LrSched &ls, int64_t t, double lr, double rbc1,
                                                  double rsbc2) {
  StepParams sp;
  sp.t = t;
  sp.src = (int32_t)(t & 1);
  sp.mix_now = (ls.mix && ls.restart > 0 && t > 0 && t % ls.restart == 0) ? 1 : 0;
  sp.lr = (float)lr;
  sp.step_size = (float)(lr * rbc1);
  sp.inv_sqrt_bc2 = (float)rsbc2;
  sp.decay = (float)(1.0 - lr * (double)ls.wd);
  return sp;
}

__device__ __forceinline__ StepParams step_params(const LrSched &ls, int64_t t) {
  return step_finish(ls, t, step_part(ls, t, 0), step_part(ls, t, 1), step_part(ls, t, 2));
}

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
// fused update for clause length 4..7 (update_long.cu)
cudaError_t launch_updateL(const ProbDev &pd, const StateDev &sd, const Hyper &hy, int mode, const float *zin,
                           float *grad, float dL, int grid, cudaStream_t st);
void prepare_updateL_attrs(int bytes);
int updateL_resident_blocks(int N);
int update_blocks_per_sm(const ProbDev &pd, const StateDev &sd);
int update_warps_per_block(const ProbDev &pd, const StateDev &sd);

int update_smem_bytes(int N, int lm1, bool greg);

// persistent solver (persist.cu): one block per instance, n_steps steps per launch
constexpr int64_t kPersistMaxWork = 1LL << 26;   // clauses x longest clause x samples of one instance
constexpr int64_t kPersistMaxSmem = 200 * 1024;   // shared memory of one block (bits of both parities included)
// cs: blocks per instance (1, or a cluster of 2, 4 or 8 with N <= 256)
int64_t persist_smem_bytes(int N, int32_t vmax, bool resident, int cs);
cudaError_t launch_persist(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const LrSched &ls, int32_t K,
                           int32_t vmax, bool resident, int cs, cudaStream_t st);

}  // namespace tsat
