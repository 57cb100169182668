// internal.h -- host-side structures shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "turbosat.h"

namespace tsat {

void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
// Raise kernel `kern`'s dynamic shared-memory limit on the current device to at
// least `bytes`: one attribute call per kernel, device and larger size,
// thread-safe (api.cu).
cudaError_t ensure_dyn_smem(const void *kern, int bytes);

#define TSAT_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return ::tsat::cuda_fail(e_, #call); \
  } while (0)

#define TSAT_LAUNCH_CHECK(what)                                        \
  do {                                                                 \
    cudaError_t e_ = cudaGetLastError();                               \
    if (e_ != cudaSuccess) return ::tsat::cuda_fail(e_, what);         \
  } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Forward work items hold a multiple of this many clauses (the smallest item;
// the default and the autotuned sizes are larger on large problems).
constexpr int kItemMin = 64;

struct Layout {  // byte offsets inside the problem workspace
  size_t cptr, clit, xptr, xrec, vptr, vocc, var_inst, items, inst, err, crec;
  size_t raw_cptr, raw_lits, tmp, clen, deg, recsz, fill, occ_j, occ_c, occ_s, scan_tmp;
  size_t total;
  int64_t xrec_cap, items_cap, scan_blocks;
};

}  // namespace tsat

struct tsat_problem {
  int32_t n_inst = 0, V = 0, C = 0, lmax = 0;
  int64_t nnz = 0, nnz_raw = 0, xrec_words = 0;
  int32_t device = 0;
  int32_t item_clauses = 2048;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  tsat::Layout lay{};
  tsat::ProbDev dev{};
  std::vector<tsat::InstInfo> inst;  // host copy (lmax filled after the build)
  std::vector<int64_t> inst_nnz;     // literal occurrences of each instance as loaded (before de-duplication)
  std::vector<int32_t> cperm;        // clause order of a locality load: loaded clause -> caller's index (else empty)
  // tsat_mpnn_forward's launch sequence captured as a CUDA graph, for the
  // parameter, workspace and output pointers it was captured with
  struct MpForwardGraph {
    const void *params = nullptr, *ws = nullptr, *logits = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture = nullptr;   // private stream the capture runs on
  };
  mutable MpForwardGraph mp_fwd;
  mutable std::mutex mp_mu;
  int set_items(int32_t item_clauses, cudaStream_t stream);
  tsat_problem() = default;
  tsat_problem(const tsat_problem &) = delete;
  tsat_problem &operator=(const tsat_problem &) = delete;
  ~tsat_problem() {
    if (mp_fwd.exec) cudaGraphExecDestroy(mp_fwd.exec);
    if (mp_fwd.capture) cudaStreamDestroy(mp_fwd.capture);
  }
};

struct GraphKey {
  int32_t n_steps, stop;
  std::vector<uint8_t> hp;
  bool operator<(const GraphKey &o) const {
    if (n_steps != o.n_steps) return n_steps < o.n_steps;
    if (stop != o.stop) return stop < o.stop;
    return hp < o.hp;
  }
};

namespace tsat {
// Host helpers shared by the entry points (api.cu).
Hyper make_hyper(const tsat_hparams &hp, int stop);
LrSched make_sched(const tsat_hparams &hp);
int state_enter(tsat_state *s, cudaStream_t user);   // the state's stream waits for the caller's
int state_leave(tsat_state *s, cudaStream_t user);   // the caller's stream waits for the state's
int update_grid(const tsat_state *s);                // blocks of the fused update
int reset_state(tsat_state *s, cudaStream_t st);     // step counter and status records to their start
// cluster-persistent solver (cluster.cu)
constexpr int kMaxClusters = 256;
int cluster_grid_clusters(int N);
int cluster_smem_bytes(int N);
void cluster_bins(const tsat_problem *p, int ncl, std::vector<int32_t> &ptr, std::vector<int32_t> &list);
cudaError_t launch_cluster(const ProbDev &pd, const StateDev &sd, const Hyper &hy, const LrSched &ls, int32_t K,
                           int ncl, const int32_t *bin_ptr, const int32_t *bin_inst, cudaStream_t st);
}  // namespace tsat

struct tsat_state {
  tsat_problem *prob = nullptr;
  void *base = nullptr;
  size_t bytes = 0;
  int32_t N = 0, layer = 0, lit_dtype = 0;
  bool initialised = false;
  tsat::StateDev dev{};
  // scratch for tsat_best / tsat_evaluate (inside the state buffer)
  int32_t *eval_hist = nullptr;     // [n_inst][lm1][N]
  int32_t *eval_unsat = nullptr;    // [n_inst][N]
  int32_t *part_var = nullptr;      // [TSAT_MAX_PARTIAL_K]
  uint8_t *part_val = nullptr;      // [TSAT_MAX_PARTIAL_K]
  int32_t *hist1 = nullptr;         // [32]
  float *gcol = nullptr;            // [max instance V]
  unsigned long long *sel = nullptr;  // [TSAT_MAX_PARTIAL_K] selected keys
  int32_t *digits = nullptr;        // [65536] radix-select histogram
  int64_t *selstate = nullptr;      // [8] radix-select bookkeeping
  uint32_t *outbits = nullptr;      // [ceil(max V/32)]
  int32_t *small = nullptr;         // [64] misc ints
  float *fwd_scratch = nullptr;     // tsat_forward outputs staging
  // regions a step changes (tsat_autotune saves and restores them)
  size_t core_bytes = 0;            // [0, core_bytes): header .. nu
  size_t lit_off = 0, lit_bytes = 0;  // relaxed literal values
  // schedules
  int32_t upd_blocks_per_sm = 0;   // 0: resident blocks per SM from the occupancy API
  mutable int32_t occ_bps = -1;     // that occupancy figure, queried once per state
  int32_t upd_rows_per_item = 1;
  int32_t persist_cs = 0;           // persistent solver: blocks per instance (0: automatic)
  int32_t sm_count = 148;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  void *h_stat = nullptr;           // pinned host copy of the header and status records (tsat_status)
  size_t h_stat_bytes = 0;
  std::map<GraphKey, cudaGraphExec_t> graphs;
  // cluster-persistent solver: clusters of the launch and the instance bins
  // (device arrays in the state buffer: bin offsets [ncl + 1], instances [n_inst])
  int32_t cl_ncl = 0;
  int32_t *cl_bins = nullptr;
  int32_t launches_per_step = 3;
};
