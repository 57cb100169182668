// api.cu -- C ABI: state buffers, init, graph-replayed steps, exact
// evaluation, hand-off selection, autograd hooks and launch-shape tuning.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>

#include "internal.h"
#include "kernels.cuh"

namespace tsat {

struct StatePlan {
  size_t hdr, inst, sp, z, m, v, bits, nu, hist, gamma, gdelta, S, unsat;
  size_t ehist, eunsat, gcol, sel, digits, selstate, outbits, small, part_var, part_val, fwdS, hist1;
  size_t lit, rbuf, dr16, zy, zs;
  size_t cbins;
  size_t total;
};

static StatePlan plan_state(const tsat_problem *p, int32_t N, int32_t layer, int32_t dt) {
  StatePlan S{};
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
  const size_t V = (size_t)p->V, W = (size_t)N / 32, I = (size_t)p->n_inst, lm1 = (size_t)p->lmax + 1;
  int32_t maxv = 0;
  for (auto &x : p->inst) maxv = std::max(maxv, x.n_vars);
  S.hdr = take(sizeof(StateHdr));
  S.inst = take(sizeof(InstState) * I);
  S.sp = take(sizeof(StepParams));
  S.z = take(sizeof(float) * V * N);
  S.m = take(sizeof(float) * V * N);
  S.v = take(sizeof(float) * V * N);
  S.bits = take(sizeof(uint32_t) * 2 * V * W);
  S.nu = take(sizeof(float) * V);
  S.hist = take(sizeof(int32_t) * I * lm1 * N);
  S.gamma = take(sizeof(float) * I * lm1 * N);
  S.gdelta = take(sizeof(float) * I * 4 * N);
  S.S = take(sizeof(float) * I * N);
  S.unsat = take(sizeof(int32_t) * I * N);
  S.ehist = take(sizeof(int32_t) * I * lm1 * N);
  S.eunsat = take(sizeof(int32_t) * I * N);
  S.gcol = take(sizeof(float) * (size_t)maxv);
  S.sel = take(sizeof(unsigned long long) * TSAT_MAX_PARTIAL_K);
  S.digits = take(sizeof(int32_t) * 65536);
  S.selstate = take(sizeof(int64_t) * 8);
  S.outbits = take(sizeof(uint32_t) * ((size_t)maxv + 31) / 32);
  S.small = take(sizeof(int32_t) * 64);
  S.part_var = take(sizeof(int32_t) * TSAT_MAX_PARTIAL_K);
  S.part_val = take(TSAT_MAX_PARTIAL_K);
  S.fwdS = take(sizeof(float) * I * N);
  S.hist1 = take(sizeof(int32_t) * 32);
  S.cbins = take(sizeof(int32_t) * (I + kMaxClusters + 1));
  if (layer == TSAT_LAYER_RELAXED) {
    S.lit = take((dt == TSAT_DTYPE_BF16 ? 2 : 4) * V * N);
    S.rbuf = take(sizeof(float) * (size_t)p->C * N);
    if (dt == TSAT_DTYPE_BF16) S.dr16 = take(sizeof(uint16_t) * (size_t)p->C * N);
    S.zy = take(sizeof(float) * 2 * (size_t)p->lay.items_cap * N);
    S.zs = take(sizeof(float) * 2 * I * N);
  }
  S.total = o;
  return S;
}

Hyper make_hyper(const tsat_hparams &hp, int stop) {
  Hyper h{};
  h.tau = hp.tau;
  h.beta1 = (float)hp.beta1;
  h.beta2 = (float)hp.beta2;
  h.omb1 = (float)(1.0 - hp.beta1);
  h.omb2 = (float)(1.0 - hp.beta2);
  h.eps = hp.eps;
  h.bin_c = 0.25f / hp.bin_temp;
  h.norm = hp.norm;
  h.binarize = hp.binarize;
  h.key0 = (uint32_t)hp.seed;
  h.key1 = (uint32_t)(hp.seed >> 32);
  h.stop_on_sat = stop;
  return h;
}

LrSched make_sched(const tsat_hparams &hp) {
  LrSched l{};
  l.lr0 = hp.lr0;
  l.factor = hp.lr_factor;
  l.floor = hp.lr_floor;
  l.wd = hp.weight_decay;
  l.period = hp.decay_period;
  l.restart = hp.restart_period;
  l.beta1 = hp.beta1;
  l.beta2 = hp.beta2;
  l.mix = hp.mix_restart;
  l.l2b1 = std::log2(hp.beta1);
  l.l2b2 = std::log2(hp.beta2);
  // the decay steps a restart period holds, when they fit the table
  l.n_lr = 0;
  if (hp.restart_period > 0 && hp.decay_period > 0) {
    const int64_t kmax = ((int64_t)hp.restart_period - 1) / hp.decay_period;
    if (kmax < kLrTab) {
      l.n_lr = (int32_t)kmax + 1;
      for (int k = 0; k < l.n_lr; ++k) {
        const double lr = (double)hp.lr0 * std::pow((double)hp.lr_factor, (double)k);
        l.lr_tab[k] = lr < (double)hp.lr_floor ? (double)hp.lr_floor : lr;
      }
    }
  }
  return l;
}

static int check_hp(const tsat_hparams *hp) {
  if (!hp) { set_error("hparams is NULL"); return TSAT_EINVAL; }
  if (!(hp->tau > 0.f) || hp->norm < 0 || hp->norm > 2 || hp->binarize < 0 || hp->binarize > 1 ||
      !(hp->bin_temp > 0.f) || !(hp->beta1 >= 0.0 && hp->beta1 < 1.0) || !(hp->beta2 >= 0.0 && hp->beta2 < 1.0) ||
      hp->mix_restart < 0 || hp->mix_restart > 1 || hp->reserved != 0) {
    set_error("hparams out of range");
    return TSAT_EINVAL;
  }
  return TSAT_OK;
}

// caller stream -> internal stream ordering
int state_enter(tsat_state *s, cudaStream_t user) {
  TSAT_CUDA(cudaEventRecord(s->ev_in, user));
  TSAT_CUDA(cudaStreamWaitEvent(s->stream, s->ev_in, 0));
  return TSAT_OK;
}
int state_leave(tsat_state *s, cudaStream_t user) {
  TSAT_CUDA(cudaEventRecord(s->ev_out, s->stream));
  TSAT_CUDA(cudaStreamWaitEvent(user, s->ev_out, 0));
  return TSAT_OK;
}
static int enter(tsat_state *s, cudaStream_t user) { return state_enter(s, user); }
static int leave(tsat_state *s, cudaStream_t user) { return state_leave(s, user); }

// Update grid: resident blocks per SM (occupancy API) unless tuned explicitly.
int update_grid(const tsat_state *s) {
  if (s->upd_blocks_per_sm <= 0 && s->occ_bps < 0) s->occ_bps = update_blocks_per_sm(s->prob->dev, s->dev);
  const int bps = s->upd_blocks_per_sm > 0 ? s->upd_blocks_per_sm : s->occ_bps;
  // no more blocks than needed to give every warp a row group (32/W rows)
  const int64_t rows_per_block = (int64_t)update_warps_per_block(s->prob->dev, s->dev) * (32 / s->dev.W);
  const int64_t need = (s->prob->dev.V + rows_per_block - 1) / rows_per_block;
  return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)s->sm_count * bps, need));
}

// The part of a step before the fused update: forward histogram (relaxed:
// exact check, relaxed forward) and the gamma kernel, which also writes the
// step scalars and advances the step counter.
static int issue_pre_update(tsat_state *s, const Hyper &hy, const LrSched &ls, cudaStream_t st) {
  const ProbDev &pd = s->prob->dev;
  cudaError_t e;
  if (s->layer == TSAT_LAYER_RELAXED) {
    const size_t n = (size_t)pd.n_inst * s->N;
    TSAT_CUDA(cudaMemsetAsync(s->dev.unsat, 0, sizeof(int32_t) * n, st));
    if ((e = launch_check(pd, s->dev, s->dev.unsat, nullptr, st)) != cudaSuccess) return cuda_fail(e, "check");
    if ((e = launch_relaxed_fwd(pd, s->dev, hy, 1, st)) != cudaSuccess) return cuda_fail(e, "relaxed forward");
    if ((e = launch_relaxed_gamma(pd, s->dev, hy, ls, 1, nullptr, nullptr, st)) != cudaSuccess)
      return cuda_fail(e, "relaxed gamma");
  } else {
    if ((e = launch_fwd_hist(pd, s->dev, s->dev.hist, 1, st)) != cudaSuccess) return cuda_fail(e, "forward");
    if ((e = launch_gamma(pd, s->dev, hy, ls, s->dev.hist, 1, 1, nullptr, nullptr, st)) != cudaSuccess)
      return cuda_fail(e, "gamma");
  }
  return TSAT_OK;
}

// The fused update of a step (with assignment mixing first when enabled):
// STE backward, Eq. 5, AdamW and the next step's bits, in the launch shape
// the state is tuned to.
static int issue_update(tsat_state *s, const Hyper &hy, const LrSched &ls, cudaStream_t st) {
  const ProbDev &pd = s->prob->dev;
  cudaError_t e;
  if (ls.mix && (e = launch_mix(pd, s->dev, hy, update_grid(s), st)) != cudaSuccess) return cuda_fail(e, "mix");
  if ((e = launch_update(pd, s->dev, hy, 0, nullptr, nullptr, 0.f, update_grid(s), s->upd_rows_per_item, st)) !=
      cudaSuccess)
    return cuda_fail(e, "update");
  return TSAT_OK;
}

// One optimisation step: forward histogram, gamma, fused update.
static int issue_step(tsat_state *s, const Hyper &hy, const LrSched &ls, cudaStream_t st) {
  int rc = issue_pre_update(s, hy, ls, st);
  return rc ? rc : issue_update(s, hy, ls, st);
}

__global__ void k_reset(StateDev sd, int n_inst) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j == 0) {
    sd.hdr->t = 0;
    sd.hdr->all_done = 0;
    sd.hdr->err = 0;
    sd.hdr->n_active = n_inst;
    sd.hdr->blocks_done = 0;
  }
  if (j < n_inst) {
    InstState is{};
    is.found = 0;
    is.found_sample = -1;
    is.found_step = -1;
    is.min_unsat = -1;
    is.best_sample = -1;
    is.loss = 0.f;
    sd.inst[j] = is;
  }
}

int reset_state(tsat_state *s, cudaStream_t st) {
  const int n = s->prob->dev.n_inst;
  k_reset<<<(n + 255) / 256, 256, 0, st>>>(s->dev, n);
  TSAT_LAUNCH_CHECK("reset");
  return TSAT_OK;
}

// A sample shard (tsat_state_set_shard) holds part of each row's samples: the
// calls that form Eq. 5's means over the state's own samples would take them
// over the shard only, so they refuse it.
static int check_not_shard(const tsat_state *s) {
  if (s->dev.n_total != s->N) {
    set_error("the state holds samples [%d, %d) of %d: run it with the tsat_shard_* calls", s->dev.sample_base,
              s->dev.sample_base + s->N, s->dev.n_total);
    return TSAT_ESTATE;
  }
  return TSAT_OK;
}

}  // namespace tsat

namespace tsat {

cudaError_t ensure_dyn_smem(const void *kern, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, int> have;   // (device, kernel) -> limit set
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  int &h = have[{dev, kern}];
  if (bytes <= h) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) h = bytes;
  return e;
}

}  // namespace tsat

using namespace tsat;

extern "C" {

void tsat_hparams_default(tsat_hparams *hp) {
  if (!hp) return;
  hp->tau = 1.0f;
  hp->lr0 = 0.1f;
  hp->lr_factor = 0.1f;
  hp->lr_floor = 1e-15f;
  hp->decay_period = 30;
  hp->restart_period = 360;
  hp->beta1 = 0.9;
  hp->beta2 = 0.999;
  hp->eps = 1e-8f;
  hp->weight_decay = 0.01f;
  hp->norm = TSAT_NORM_SIGNED_MEAN;
  hp->binarize = TSAT_BIN_DET;
  hp->bin_temp = 1.0f;
  hp->layer = TSAT_LAYER_STE;
  hp->seed = 0;
  hp->mix_restart = 0;
  hp->reserved = 0;
}

int tsat_state_bytes(const tsat_problem *p, int32_t N, int32_t layer, int32_t dt, size_t *bytes) {
  if (!p || !bytes) { set_error("NULL argument"); return TSAT_EINVAL; }
  if (N < TSAT_MIN_SAMPLES || N > TSAT_MAX_SAMPLES || (N & (N - 1))) {
    set_error("n_samples must be a power of two in [32, 1024], got %d", N);
    return TSAT_EINVAL;
  }
  if (layer != TSAT_LAYER_STE && layer != TSAT_LAYER_RELAXED) { set_error("bad layer"); return TSAT_EINVAL; }
  if (dt != TSAT_DTYPE_F32 && dt != TSAT_DTYPE_BF16) { set_error("bad dtype"); return TSAT_EINVAL; }
  *bytes = plan_state(p, N, layer, dt).total;
  return TSAT_OK;
}

int tsat_state_create(tsat_problem *p, void *d_state, size_t state_bytes, int32_t N, int32_t layer, int32_t dt,
                      tsat_state **out) {
  if (!out) return TSAT_EINVAL;
  *out = nullptr;
  size_t need = 0;
  int rc = tsat_state_bytes(p, N, layer, dt, &need);
  if (rc) return rc;
  if (!d_state) { set_error("state buffer is NULL"); return TSAT_EINVAL; }
  if (state_bytes < need) { set_error("state buffer %zu < %zu bytes", state_bytes, need); return TSAT_EWS; }
  if (((uintptr_t)d_state) % 256) { set_error("state buffer must be 256-byte aligned"); return TSAT_EINVAL; }
  tsat_state *s = new (std::nothrow) tsat_state();
  if (!s) return TSAT_ENOMEM;
  StatePlan P = plan_state(p, N, layer, dt);
  char *b = (char *)d_state;
  s->prob = p;
  s->base = d_state;
  s->bytes = state_bytes;
  s->N = N;
  s->layer = layer;
  s->lit_dtype = dt;
  StateDev &D = s->dev;
  D.N = N;
  D.W = N / 32;
  D.sample_base = 0;
  D.n_total = N;
  D.lm1 = p->lmax + 1;
  D.layer = layer;
  D.hdr = (StateHdr *)(b + P.hdr);
  D.inst = (InstState *)(b + P.inst);
  D.sp = (StepParams *)(b + P.sp);
  D.z = (float *)(b + P.z);
  D.m = (float *)(b + P.m);
  D.v = (float *)(b + P.v);
  D.bits = (uint32_t *)(b + P.bits);
  D.nu = (float *)(b + P.nu);
  D.hist = (int32_t *)(b + P.hist);
  D.gamma = (float *)(b + P.gamma);
  D.gdelta = (float *)(b + P.gdelta);
  D.S = (float *)(b + P.S);
  D.unsat = (int32_t *)(b + P.unsat);
  D.V = p->V;
  if (layer == TSAT_LAYER_RELAXED) {
    D.lit = b + P.lit;
    D.rbuf = (float *)(b + P.rbuf);
    D.dr16 = dt == TSAT_DTYPE_BF16 ? (uint32_t *)(b + P.dr16) : nullptr;
    D.zy = (float *)(b + P.zy);
    D.zs = (float *)(b + P.zs);
    D.lit_bf16 = dt == TSAT_DTYPE_BF16;
  }
  s->eval_hist = (int32_t *)(b + P.ehist);
  s->eval_unsat = (int32_t *)(b + P.eunsat);
  s->gcol = (float *)(b + P.gcol);
  s->sel = (unsigned long long *)(b + P.sel);
  s->digits = (int32_t *)(b + P.digits);
  s->selstate = (int64_t *)(b + P.selstate);
  s->outbits = (uint32_t *)(b + P.outbits);
  s->small = (int32_t *)(b + P.small);
  s->part_var = (int32_t *)(b + P.part_var);
  s->part_val = (uint8_t *)(b + P.part_val);
  s->fwd_scratch = (float *)(b + P.fwdS);
  s->hist1 = (int32_t *)(b + P.hist1);
  s->cl_bins = (int32_t *)(b + P.cbins);
  // what a step changes: the header, status records, step scalars, z, m, v,
  // both bit parities and nu (adjacent, from the start of the buffer), plus the
  // relaxed layer's literal values
  s->core_bytes = P.hist;
  s->lit_off = layer == TSAT_LAYER_RELAXED ? P.lit : 0;
  s->lit_bytes = layer == TSAT_LAYER_RELAXED ? (size_t)(dt == TSAT_DTYPE_BF16 ? 2 : 4) * p->V * N : 0;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev);
  auto fail = [&](cudaError_t e, const char *w) { tsat_state_free(s); return cuda_fail(e, w); };   // releases what was created
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess) return fail(e, "stream");
  if ((e = cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
  if ((e = cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
  // pinned copy of the header and the status records for tsat_status, made
  // here so that no status read pays for the allocation
  s->h_stat_bytes = (P.inst - P.hdr) + sizeof(InstState) * (size_t)p->n_inst;
  if ((e = cudaMallocHost(&s->h_stat, s->h_stat_bytes)) != cudaSuccess) {
    s->h_stat = nullptr;
    s->h_stat_bytes = 0;
    return fail(e, "pinned status buffer");
  }
  if ((e = cudaMemsetAsync(b + P.digits, 0, sizeof(int32_t) * 65536, s->stream)) != cudaSuccess) return fail(e, "memset");
  if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return fail(e, "sync");
  prepare_update_attrs(p->lmax);
  *out = s;
  return TSAT_OK;
}

void tsat_state_free(tsat_state *s) {
  if (!s) return;
  for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->ev_in) cudaEventDestroy(s->ev_in);
  if (s->ev_out) cudaEventDestroy(s->ev_out);
  if (s->h_stat) cudaFreeHost(s->h_stat);
  delete s;
}


int tsat_init(tsat_state *s, const tsat_hparams *hp, const float *d_logits, float scale, cudaStream_t stream) {
  if (!s) return TSAT_EINVAL;
  int rc = check_hp(hp);
  if (rc) return rc;
  if ((rc = check_not_shard(s))) return rc;
  if (hp->layer != s->layer) { set_error("hp->layer differs from the state's layer"); return TSAT_ESTATE; }
  if ((rc = enter(s, stream))) return rc;
  const Hyper hy = make_hyper(*hp, 0);
  const ProbDev &pd = s->prob->dev;
  const size_t histb = sizeof(int32_t) * (size_t)pd.n_inst * s->dev.lm1 * s->N;
  TSAT_CUDA(cudaMemsetAsync(s->dev.hist, 0, histb, s->stream));
  k_reset<<<(pd.n_inst + 255) / 256, 256, 0, s->stream>>>(s->dev, pd.n_inst);
  TSAT_LAUNCH_CHECK("reset");
  cudaError_t e = launch_init(pd, s->dev, hy, d_logits, scale, update_grid(s), s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "init");
  if (s->layer == TSAT_LAYER_RELAXED) {
    e = launch_relaxed_lits(pd, s->dev, hy, nullptr, update_grid(s), s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "relaxed literals");
  }
  s->initialised = true;
  return leave(s, stream);
}

static int get_graph(tsat_state *s, const tsat_hparams *hp, int32_t n_steps, int32_t stop_on_sat,
                     cudaGraphExec_t *out) {
  GraphKey key;
  key.n_steps = n_steps;
  key.stop = stop_on_sat ? 1 : 0;
  key.hp.assign((const uint8_t *)hp, (const uint8_t *)hp + sizeof(tsat_hparams));
  // the launch shapes baked into the graph (every byte: no two shapes share a key)
  for (int32_t x : {s->upd_blocks_per_sm, s->upd_rows_per_item, s->prob->item_clauses})
    for (int b = 0; b < 4; ++b) key.hp.push_back((uint8_t)((uint32_t)x >> (8 * b)));
  auto it = s->graphs.find(key);
  if (it != s->graphs.end()) {
    *out = it->second;
    return TSAT_OK;
  }
  const Hyper hy = make_hyper(*hp, key.stop);
  const LrSched ls = make_sched(*hp);
  cudaGraph_t graph = nullptr;
  TSAT_CUDA(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  int irc = TSAT_OK;
  for (int32_t k = 0; k < n_steps && irc == TSAT_OK; ++k) irc = issue_step(s, hy, ls, s->stream);
  cudaError_t ec = cudaStreamEndCapture(s->stream, &graph);
  if (irc) {
    if (graph) cudaGraphDestroy(graph);
    return irc;
  }
  if (ec != cudaSuccess) return cuda_fail(ec, "end capture");
  cudaGraphExec_t exec = nullptr;
  cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return cuda_fail(ei, "graph instantiate");
  if (s->graphs.size() >= 16) {
    for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second);
    s->graphs.clear();
  }
  s->graphs[key] = exec;
  *out = exec;
  return TSAT_OK;
}

static int check_step_args(tsat_state *s, const tsat_hparams *hp, int32_t n_steps) {
  if (!s) return TSAT_EINVAL;
  int rc = check_hp(hp);
  if (rc) return rc;
  if ((rc = check_not_shard(s))) return rc;
  if (!s->initialised) { set_error("state not initialised"); return TSAT_ESTATE; }
  if (hp->layer != s->layer) { set_error("hp->layer differs from the state's layer"); return TSAT_ESTATE; }
  if (n_steps <= 0) { set_error("n_steps must be positive"); return TSAT_EINVAL; }
  return TSAT_OK;
}

int tsat_step_prepare(tsat_state *s, const tsat_hparams *hp, int32_t n_steps, int32_t stop_on_sat) {
  int rc = check_step_args(s, hp, n_steps);
  if (rc) return rc;
  cudaGraphExec_t exec = nullptr;
  return get_graph(s, hp, n_steps, stop_on_sat, &exec);
}

int tsat_step(tsat_state *s, const tsat_hparams *hp, int32_t n_steps, int32_t stop_on_sat, cudaStream_t stream) {
  int rc = check_step_args(s, hp, n_steps);
  if (rc) return rc;
  if ((rc = enter(s, stream))) return rc;
  cudaGraphExec_t exec = nullptr;
  if ((rc = get_graph(s, hp, n_steps, stop_on_sat, &exec))) return rc;
  TSAT_CUDA(cudaGraphLaunch(exec, s->stream));
  return leave(s, stream);
}

// Blocks per instance of the persistent solver: the state's setting, or, when
// it is 0 (N <= 256 only): one block when that block keeps its instance's z,
// m, v in shared memory, else the largest power of two up to 8 such that the
// batch's clusters all fit on the device at once (or a larger one, below).  Measured per step at
// N = 64 (planted 3-SAT, 1 / 2 / 4 / 8 blocks): n = 100 (resident in one
// block) 8.4 / 9.2 / 8.5 / 9.4 us, the step being a chain of dependent phases
// that more blocks do not shorten; n = 1,000 152.8 / 89.0 / 49.7 / 12.9 us
// (resident from 8 blocks); n = 3,000 436 / 232 / 127 / 73 us; 5-SAT n = 300
// 235 / 121 / 68 / 59 us.
static int persist_blocks(const tsat_state *s, int32_t vmax) {
  const tsat_problem *p = s->prob;
  if (s->N > 256) return 1;
  if (s->persist_cs > 0) return s->persist_cs;
  auto resident = [&](int c) { return persist_smem_bytes(s->N, vmax, true, c) <= kPersistMaxSmem; };
  if (resident(1)) return 1;
  int cs = 1;
  while (cs < 8 && (int64_t)p->n_inst * cs * 2 <= s->sm_count) cs *= 2;
  // a larger cluster that keeps the instances resident beats one that fits the
  // device at once but does not, up to two waves of clusters (32 instances of
  // n = 1,000: 4 blocks, all at once, 52.2 us per step; 8 blocks, two waves,
  // 34.1 us)
  if (!resident(cs))
    for (int c2 = cs * 2; c2 <= 8; c2 *= 2)
      if (resident(c2) && ((int64_t)p->n_inst * c2 + s->sm_count - 1) / s->sm_count <= 2) {
        cs = c2;
        break;
      }
  return cs;
}

int tsat_persist_blocks(const tsat_state *s, int32_t *blocks, int32_t *resident) {
  if (!s || !blocks) {
    set_error("NULL argument");
    return TSAT_EINVAL;
  }
  int32_t vmax = 0;
  for (const InstInfo &I : s->prob->inst) vmax = std::max(vmax, I.n_vars);
  *blocks = persist_blocks(s, vmax);
  if (resident) *resident = persist_smem_bytes(s->N, vmax, true, *blocks) <= kPersistMaxSmem ? 1 : 0;
  return TSAT_OK;
}

int tsat_set_persist_blocks(tsat_state *s, int32_t blocks) {
  if (!s) {
    set_error("NULL state");
    return TSAT_EINVAL;
  }
  if (blocks != 0 && blocks != 1 && blocks != 2 && blocks != 4 && blocks != 8) {
    set_error("blocks per instance must be 0 (automatic), 1, 2, 4 or 8, got %d", blocks);
    return TSAT_EINVAL;
  }
  if (blocks > 1 && s->N > 256) {
    set_error("several blocks per instance need at most 256 samples (N %d)", s->N);
    return TSAT_EINVAL;
  }
  s->persist_cs = blocks;
  return TSAT_OK;
}

// Checks and launch of the persistent solver on the state's stream (the
// caller has entered it).  *to_clustered: the instances suit the cluster
// solver instead (nothing launched).
static int persist_launch(tsat_state *s, const tsat_hparams *hp, int32_t n_steps, int32_t stop_on_sat,
                          bool *to_clustered) {
  *to_clustered = false;
  const tsat_problem *p = s->prob;
  if (s->layer != TSAT_LAYER_STE || hp->mix_restart) {
    set_error("the persistent solver runs the STE layer without assignment mixing");
    return TSAT_EINVAL;
  }
  if (p->lmax > 7 || (p->dev.rec_stride != 4 && p->dev.rec_stride != 8)) {
    set_error("the persistent solver needs clauses of at most 7 literals (longest: %d)", p->lmax);
    return TSAT_EINVAL;
  }
  int32_t vmax = 0;
  for (const InstInfo &I : p->inst) vmax = std::max(vmax, I.n_vars);
  const int cs = persist_blocks(s, vmax);
  bool too_big = false;
  for (const InstInfo &I : p->inst) too_big = too_big || (int64_t)I.n_clauses * I.lmax * s->N > cs * kPersistMaxWork;
  too_big = too_big || persist_smem_bytes(s->N, vmax, false, cs) > kPersistMaxSmem;
  // instances too large for one block: clusters of blocks, when the batch suits them
  if (too_big && s->persist_cs == 0 && p->dev.rec_stride == 8 && s->N <= 128) {
    *to_clustered = true;
    return TSAT_OK;
  }
  for (const InstInfo &I : p->inst) {
    if ((int64_t)I.n_clauses * I.lmax * s->N > cs * kPersistMaxWork) {
      set_error("instance too large for %d block(s): %d clauses x %d literals x %d samples > %lld", cs,
                I.n_clauses, I.lmax, s->N, (long long)(cs * kPersistMaxWork));
      return TSAT_ERANGE;
    }
  }
  if (persist_smem_bytes(s->N, vmax, false, cs) > kPersistMaxSmem) {
    set_error("instance too large for one block: %d variables x %d samples need %lld bytes of shared memory",
              vmax, s->N, (long long)persist_smem_bytes(s->N, vmax, false, cs));
    return TSAT_ERANGE;
  }
  const bool resident = persist_smem_bytes(s->N, vmax, true, cs) <= kPersistMaxSmem;
  const Hyper hy = make_hyper(*hp, stop_on_sat ? 1 : 0);
  const LrSched ls = make_sched(*hp);
  cudaError_t e = launch_persist(p->dev, s->dev, hy, ls, n_steps, vmax, resident, cs, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "persistent solver");
  return TSAT_OK;
}

int tsat_step_persistent(tsat_state *s, const tsat_hparams *hp, int32_t n_steps, int32_t stop_on_sat,
                         cudaStream_t stream) {
  int rc = check_step_args(s, hp, n_steps);
  if (rc) return rc;
  if ((rc = enter(s, stream))) return rc;
  bool to_clustered = false;
  if ((rc = persist_launch(s, hp, n_steps, stop_on_sat, &to_clustered))) {
    leave(s, stream);
    return rc;
  }
  if ((rc = leave(s, stream))) return rc;
  if (to_clustered) return tsat_step_clustered(s, hp, n_steps, stop_on_sat, stream);
  return TSAT_OK;
}

int tsat_step_clustered(tsat_state *s, const tsat_hparams *hp, int32_t n_steps, int32_t stop_on_sat,
                        cudaStream_t stream) {
  int rc = check_step_args(s, hp, n_steps);
  if (rc) return rc;
  const tsat_problem *p = s->prob;
  if (s->layer != TSAT_LAYER_STE || hp->mix_restart) {
    set_error("the cluster solver runs the STE layer without assignment mixing");
    return TSAT_EINVAL;
  }
  if (p->dev.rec_stride != 8 || s->N > 128) {
    set_error("the cluster solver needs a longest clause of 4..7 literals and at most 128 samples (longest %d, N %d)",
              p->lmax, s->N);
    return TSAT_EINVAL;
  }
  if (s->cl_ncl == 0) {   // the launch's clusters and the instance bins, once per state
    int ncl = std::min(cluster_grid_clusters(s->N), kMaxClusters);
    if (ncl <= 0) {
      set_error("no cluster of the solver fits on this device");
      return TSAT_ECUDA;
    }
    std::vector<int32_t> ptr, list;
    cluster_bins(p, ncl, ptr, list);
    TSAT_CUDA(cudaMemcpy(s->cl_bins, ptr.data(), sizeof(int32_t) * ptr.size(), cudaMemcpyHostToDevice));
    TSAT_CUDA(cudaMemcpy(s->cl_bins + ptr.size(), list.data(), sizeof(int32_t) * list.size(),
                         cudaMemcpyHostToDevice));
    s->cl_ncl = ncl;
  }
  if ((rc = enter(s, stream))) return rc;
  const Hyper hy = make_hyper(*hp, stop_on_sat ? 1 : 0);
  const LrSched ls = make_sched(*hp);
  cudaError_t e = launch_cluster(p->dev, s->dev, hy, ls, n_steps, s->cl_ncl, s->cl_bins,
                                 s->cl_bins + s->cl_ncl + 1, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cluster solver");
  return leave(s, stream);
}

int tsat_profile_step(tsat_state *s, const tsat_hparams *hp, int32_t n_steps, float h_ms[4]) {
  int rc = check_step_args(s, hp, n_steps);
  if (rc) return rc;
  if (!h_ms) return TSAT_EINVAL;
  const ProbDev &pd = s->prob->dev;
  const Hyper hy = make_hyper(*hp, 0);
  const LrSched ls = make_sched(*hp);
  cudaStream_t st = s->stream;
  TSAT_CUDA(cudaStreamSynchronize(st));
  cudaEvent_t ev[5];
  for (auto &e : ev) TSAT_CUDA(cudaEventCreate(&e));
  double acc[4] = {0, 0, 0, 0};
  cudaError_t e = cudaSuccess;
  for (int32_t k = 0; k < n_steps && e == cudaSuccess; ++k) {
    TSAT_CUDA(cudaEventRecord(ev[0], st));
    if (s->layer == TSAT_LAYER_RELAXED) {
      TSAT_CUDA(cudaMemsetAsync(s->dev.unsat, 0, sizeof(int32_t) * (size_t)pd.n_inst * s->N, st));
      e = launch_check(pd, s->dev, s->dev.unsat, nullptr, st);
      TSAT_CUDA(cudaEventRecord(ev[4], st));
      if (e == cudaSuccess) e = launch_relaxed_fwd(pd, s->dev, hy, 1, st);
      TSAT_CUDA(cudaEventRecord(ev[1], st));
      if (e == cudaSuccess) e = launch_relaxed_gamma(pd, s->dev, hy, ls, 1, nullptr, nullptr, st);
    } else {
      e = launch_fwd_hist(pd, s->dev, s->dev.hist, 1, st);
      TSAT_CUDA(cudaEventRecord(ev[1], st));
      if (e == cudaSuccess) e = launch_gamma(pd, s->dev, hy, ls, s->dev.hist, 1, 1, nullptr, nullptr, st);
    }
    TSAT_CUDA(cudaEventRecord(ev[2], st));
    if (e == cudaSuccess && ls.mix) e = launch_mix(pd, s->dev, hy, update_grid(s), st);
    if (e == cudaSuccess)
      e = launch_update(pd, s->dev, hy, 0, nullptr, nullptr, 0.f, update_grid(s), s->upd_rows_per_item, st);
    TSAT_CUDA(cudaEventRecord(ev[3], st));
    TSAT_CUDA(cudaEventSynchronize(ev[3]));
    float a = 0, b = 0, c = 0, d = 0;
    if (s->layer == TSAT_LAYER_RELAXED) {
      TSAT_CUDA(cudaEventElapsedTime(&d, ev[0], ev[4]));
      TSAT_CUDA(cudaEventElapsedTime(&a, ev[4], ev[1]));
    } else {
      TSAT_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]));
    }
    TSAT_CUDA(cudaEventElapsedTime(&b, ev[1], ev[2]));
    TSAT_CUDA(cudaEventElapsedTime(&c, ev[2], ev[3]));
    acc[0] += a; acc[1] += b; acc[2] += c; acc[3] += d;
  }
  for (auto &x : ev) cudaEventDestroy(x);
  if (e != cudaSuccess) return cuda_fail(e, "profile step");
  for (int j = 0; j < 4; ++j) h_ms[j] = (float)(acc[j] / n_steps);
  return TSAT_OK;
}

int tsat_evaluate(tsat_state *s, const tsat_hparams *hp, int32_t *d_unsat, uint32_t *d_satmask, float *d_loss,
                  cudaStream_t stream) {
  if (!s || !d_unsat || !d_satmask) { set_error("NULL argument"); return TSAT_EINVAL; }
  if (!s->initialised) { set_error("state not initialised"); return TSAT_ESTATE; }
  int rc = check_hp(hp);
  if (rc) return rc;
  if ((rc = enter(s, stream))) return rc;
  const ProbDev &pd = s->prob->dev;
  const size_t n = (size_t)pd.n_inst * s->N;
  TSAT_CUDA(cudaMemsetAsync(d_unsat, 0, sizeof(int32_t) * n, s->stream));
  cudaError_t e = launch_check(pd, s->dev, d_unsat, d_satmask, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "check");
  if (d_loss) {
    const Hyper hy = make_hyper(*hp, 0);
    const LrSched ls = make_sched(*hp);
    TSAT_CUDA(cudaMemsetAsync(s->eval_hist, 0, sizeof(int32_t) * n * s->dev.lm1, s->stream));
    StateDev sd = s->dev;
    sd.unsat = s->eval_unsat;
    if ((e = launch_fwd_hist(pd, sd, s->eval_hist, 0, s->stream)) != cudaSuccess) return cuda_fail(e, "forward");
    if ((e = launch_gamma(pd, sd, hy, ls, s->eval_hist, 0, 0, d_loss, s->fwd_scratch, s->stream)) != cudaSuccess)
      return cuda_fail(e, "loss");
  }
  return leave(s, stream);
}

int tsat_histogram(tsat_state *s, int32_t *d_hist, cudaStream_t stream) {
  if (!s || !d_hist) { set_error("NULL argument"); return TSAT_EINVAL; }
  if (!s->initialised) { set_error("state not initialised"); return TSAT_ESTATE; }
  int rc;
  if ((rc = enter(s, stream))) return rc;
  const ProbDev &pd = s->prob->dev;
  TSAT_CUDA(cudaMemsetAsync(d_hist, 0, sizeof(int32_t) * (size_t)pd.n_inst * s->dev.lm1 * s->N, s->stream));
  cudaError_t e = launch_fwd_hist(pd, s->dev, d_hist, 0, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "forward");
  return leave(s, stream);
}

int tsat_best(tsat_state *s, const tsat_hparams *hp, int32_t inst, int32_t k, uint32_t *h_bits, int32_t *h_unsat,
              int32_t *h_sample, int32_t *h_part_var, uint8_t *h_part_val, int32_t *h_ready, cudaStream_t stream) {
  if (!s || !h_bits || !h_unsat || !h_sample || !h_part_var || !h_part_val) {
    set_error("NULL argument");
    return TSAT_EINVAL;
  }
  if (!s->initialised) { set_error("state not initialised"); return TSAT_ESTATE; }
  int rc = check_hp(hp);
  if (rc) return rc;
  const tsat_problem *p = s->prob;
  if (inst < 0 || inst >= p->n_inst) { set_error("instance %d out of range", inst); return TSAT_ERANGE; }
  const InstInfo &I = p->inst[inst];
  if (k < 1 || k > std::min<int32_t>(TSAT_MAX_PARTIAL_K, I.n_vars)) { set_error("k=%d out of range", k); return TSAT_ERANGE; }
  if ((rc = enter(s, stream))) return rc;
  const ProbDev &pd = p->dev;
  const Hyper hy = make_hyper(*hp, 0);
  const size_t n = (size_t)pd.n_inst * s->N;
  cudaStream_t st = s->stream;
  TSAT_CUDA(cudaMemsetAsync(s->eval_unsat, 0, sizeof(int32_t) * n, st));
  cudaError_t e = launch_check(pd, s->dev, s->eval_unsat, nullptr, st);
  if (e != cudaSuccess) return cuda_fail(e, "check");
  if ((e = best_pick(s->eval_unsat + (size_t)inst * s->N, s->N, s->small, st)) != cudaSuccess) return cuda_fail(e, "pick");
  TSAT_CUDA(cudaMemsetAsync(s->hist1, 0, sizeof(int32_t) * 32, st));
  if ((e = best_gcol(pd, s->dev, hy, inst, I.n_vars, I.n_clauses, s->small, s->hist1, s->gcol, st)) != cudaSuccess)
    return cuda_fail(e, "gradient column");
  int64_t ss[2] = {0, (int64_t)k};
  TSAT_CUDA(cudaMemcpyAsync(s->selstate, ss, sizeof(ss), cudaMemcpyHostToDevice, st));
  if ((e = best_select(pd, s->dev, inst, I.n_vars, k, s->gcol, s->sel, s->digits, s->selstate, s->small, s->part_var,
                       s->part_val, s->outbits, st)) != cudaSuccess)
    return cuda_fail(e, "select");
  int32_t small[4] = {0, 0, 0, 0};
  TSAT_CUDA(cudaMemcpyAsync(small, s->small, sizeof(small), cudaMemcpyDeviceToHost, st));
  TSAT_CUDA(cudaMemcpyAsync(h_bits, s->outbits, sizeof(uint32_t) * ((I.n_vars + 31) / 32), cudaMemcpyDeviceToHost, st));
  TSAT_CUDA(cudaMemcpyAsync(h_part_var, s->part_var, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, st));
  TSAT_CUDA(cudaMemcpyAsync(h_part_val, s->part_val, k, cudaMemcpyDeviceToHost, st));
  TSAT_CUDA(cudaStreamSynchronize(st));
  if ((rc = leave(s, stream))) return rc;
  if (small[2] != k) { set_error("selection returned %d of %d keys", small[2], k); return TSAT_ECUDA; }
  *h_sample = small[0];
  *h_unsat = small[1];
  if (h_ready) *h_ready = (double)(I.n_clauses - small[1]) / (double)I.n_clauses > 0.99 ? 1 : 0;
  return small[1] == 0 ? 1 : 0;
}

int tsat_status(tsat_state *s, int64_t *h_step, int32_t *h_all_done, tsat_inst_status *h_inst, cudaStream_t stream) {
  if (!s) return TSAT_EINVAL;
  int rc = enter(s, stream);
  if (rc) return rc;
  // the header and the status records are adjacent at the start of the state
  // buffer: one copy into a pinned host buffer kept with the state (two
  // pageable copies took about 30 us of a 0.5 ms time to SAT)
  const size_t off = (size_t)((const char *)s->dev.inst - (const char *)s->dev.hdr);
  const size_t bytes = off + sizeof(InstState) * (size_t)s->prob->n_inst;
  if (s->h_stat_bytes < bytes) {
    if (s->h_stat) cudaFreeHost(s->h_stat);
    s->h_stat = nullptr;
    s->h_stat_bytes = 0;
    TSAT_CUDA(cudaMallocHost(&s->h_stat, bytes));
    s->h_stat_bytes = bytes;
  }
  TSAT_CUDA(cudaMemcpyAsync(s->h_stat, s->dev.hdr, bytes, cudaMemcpyDeviceToHost, s->stream));
  TSAT_CUDA(cudaStreamSynchronize(s->stream));
  const StateHdr &h = *static_cast<const StateHdr *>(s->h_stat);
  const InstState *is = reinterpret_cast<const InstState *>(static_cast<const char *>(s->h_stat) + off);
  if (h_step) *h_step = h.t;
  if (h_all_done) *h_all_done = h.all_done;
  if (h_inst)
    for (size_t j = 0; j < (size_t)s->prob->n_inst; ++j) {
      h_inst[j].found = is[j].found;
      h_inst[j].found_sample = is[j].found_sample;
      h_inst[j].found_step = is[j].found_step;
      h_inst[j].min_unsat = is[j].min_unsat;
      h_inst[j].best_sample = is[j].best_sample;
      h_inst[j].loss = is[j].loss;
      h_inst[j].pad = 0.f;
    }
  return TSAT_OK;   // the library stream is idle: the caller's stream has nothing to wait for
}

int tsat_state_views(tsat_state *s, float **z, float **m, float **v, uint32_t **bits_cur, float **nu, float **gamma,
                     int32_t **hist) {
  if (!s) return TSAT_EINVAL;
  StateHdr h{};
  TSAT_CUDA(cudaMemcpy(&h, s->dev.hdr, sizeof(h), cudaMemcpyDeviceToHost));
  if (z) *z = s->dev.z;
  if (m) *m = s->dev.m;
  if (v) *v = s->dev.v;
  if (bits_cur) *bits_cur = s->dev.bits + (size_t)(h.t & 1) * (size_t)s->prob->V * (s->N / 32);
  if (nu) *nu = s->dev.nu;
  if (gamma) *gamma = s->dev.gamma;
  if (hist) *hist = s->dev.hist;
  return TSAT_OK;
}

int tsat_forward(tsat_state *s, const tsat_hparams *hp, const float *d_z, int64_t t_bin, float *d_S, float *d_loss,
                 cudaStream_t stream) {
  if (!s || !d_z || !d_S || !d_loss) { set_error("NULL argument"); return TSAT_EINVAL; }
  int rc = check_hp(hp);
  if (rc) return rc;
  if ((rc = check_not_shard(s))) return rc;
  if (hp->layer != s->layer) { set_error("hp->layer differs from the state's layer"); return TSAT_ESTATE; }
  if ((rc = enter(s, stream))) return rc;
  const ProbDev &pd = s->prob->dev;
  const Hyper hy = make_hyper(*hp, 0);
  const LrSched ls = make_sched(*hp);
  if (!s->initialised) {
    k_reset<<<(pd.n_inst + 255) / 256, 256, 0, s->stream>>>(s->dev, pd.n_inst);
    TSAT_LAUNCH_CHECK("reset");
  }
  cudaError_t e;
  if (s->layer == TSAT_LAYER_RELAXED) {
    if ((e = launch_relaxed_lits(pd, s->dev, hy, d_z, update_grid(s), s->stream)) != cudaSuccess)
      return cuda_fail(e, "relaxed literals");
    if ((e = launch_relaxed_fwd(pd, s->dev, hy, 0, s->stream)) != cudaSuccess) return cuda_fail(e, "relaxed forward");
    if ((e = launch_relaxed_gamma(pd, s->dev, hy, ls, 0, d_loss, d_S, s->stream)) != cudaSuccess)
      return cuda_fail(e, "relaxed gamma");
  } else {
    const size_t n = (size_t)pd.n_inst * s->N;
    if ((e = launch_binarize(pd, s->dev, hy, d_z, t_bin, update_grid(s), s->stream)) != cudaSuccess)
      return cuda_fail(e, "binarize");
    TSAT_CUDA(cudaMemsetAsync(s->eval_hist, 0, sizeof(int32_t) * n * s->dev.lm1, s->stream));
    if ((e = launch_fwd_hist(pd, s->dev, s->eval_hist, 0, s->stream)) != cudaSuccess) return cuda_fail(e, "forward");
    if ((e = launch_gamma(pd, s->dev, hy, ls, s->eval_hist, 0, 1, d_loss, d_S, s->stream)) != cudaSuccess)
      return cuda_fail(e, "gamma");
  }
  return leave(s, stream);
}

int tsat_backward(tsat_state *s, const tsat_hparams *hp, const float *d_z, float dL, float *d_grad,
                  cudaStream_t stream) {
  if (!s || !d_z || !d_grad) { set_error("NULL argument"); return TSAT_EINVAL; }
  int rc = check_hp(hp);
  if (rc) return rc;
  if ((rc = check_not_shard(s))) return rc;
  if ((rc = enter(s, stream))) return rc;
  const Hyper hy = make_hyper(*hp, 0);
  cudaError_t e = launch_update(s->prob->dev, s->dev, hy, 1, d_z, d_grad, dL, update_grid(s), s->upd_rows_per_item,
                                s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "backward");
  return leave(s, stream);
}

int tsat_get_tuning(const tsat_state *s, int32_t h_tuning[4]) {
  if (!s || !h_tuning) return TSAT_EINVAL;
  h_tuning[0] = s->prob->item_clauses;
  h_tuning[1] = kBlock;
  h_tuning[2] = s->upd_blocks_per_sm;
  h_tuning[3] = s->upd_rows_per_item;
  return TSAT_OK;
}

int tsat_set_tuning(tsat_state *s, const int32_t h_tuning[4]) {
  if (!s || !h_tuning) return TSAT_EINVAL;
  if (h_tuning[0] < kItemMin || h_tuning[1] != kBlock || h_tuning[2] < 0 || h_tuning[2] > 128 || h_tuning[3] < 1 ||
      h_tuning[3] > 4096) {
    set_error("tuning values out of range");
    return TSAT_EINVAL;
  }
  int rc = s->prob->set_items(h_tuning[0], s->stream);
  if (rc) return rc;
  s->upd_blocks_per_sm = h_tuning[2];
  s->upd_rows_per_item = h_tuning[3];
  return TSAT_OK;
}

namespace {
// Candidate launch shapes of tsat_autotune: forward work-item sizes, update
// blocks per SM around the default d (resident blocks x waves): d/8, d/4, d/2,
// d and 5d/4, and update rows per work item.
constexpr int kTuneItems[4] = {512, 1024, 2048, 4096};
constexpr int kTuneRpi[3] = {1, 8, 64};
void tune_bps(const tsat_state *s, int out[5]) {
  const int d = update_blocks_per_sm(s->prob->dev, s->dev);
  out[0] = std::max(1, d / 8);
  out[1] = std::max(1, d / 4);
  out[2] = std::max(1, d / 2);
  out[3] = d;
  out[4] = d * 5 / 4;
}

// Events of one tuning run, destroyed on every return path.
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};
}  // namespace

int tsat_tuning_space(const tsat_state *s, int32_t h_fwd_items[4], int32_t h_upd_bps[5], int32_t h_upd_rpi[3]) {
  if (!s || !h_fwd_items || !h_upd_bps || !h_upd_rpi) { set_error("NULL argument"); return TSAT_EINVAL; }
  int b[5];
  tune_bps(s, b);
  for (int j = 0; j < 4; ++j) h_fwd_items[j] = kTuneItems[j];
  for (int j = 0; j < 5; ++j) h_upd_bps[j] = b[j];
  for (int j = 0; j < 3; ++j) h_upd_rpi[j] = kTuneRpi[j];
  return TSAT_OK;
}

int tsat_autotune_persistent(tsat_state *s, const tsat_hparams *hp, void *d_snapshot, size_t snapshot_bytes,
                             int32_t n_steps, cudaStream_t stream, int32_t *h_blocks) {
  if (!s || !h_blocks || !d_snapshot) { set_error("NULL argument"); return TSAT_EINVAL; }
  int rc = check_step_args(s, hp, n_steps);
  if (rc) return rc;
  const size_t need = s->core_bytes + s->lit_bytes;
  if (snapshot_bytes < need) { set_error("snapshot buffer %zu < %zu bytes", snapshot_bytes, need); return TSAT_EWS; }
  if ((rc = enter(s, stream))) return rc;
  cudaStream_t st = s->stream;
  char *base = static_cast<char *>(s->base);
  char *snap = static_cast<char *>(d_snapshot);
  const int32_t keep = s->persist_cs;
  int32_t best_cs = 1;
  float best = 1e30f;
  EventPair ev;
  bool saved = false;
  // candidates: one block, and (N <= 256) clusters of 2, 4, 8 blocks while
  // the batch's clusters fit the device at most twice over; every trial
  // starts from the caller's state
  auto trials = [&]() -> int {
    TSAT_CUDA(cudaMemcpyAsync(snap, base, s->core_bytes, cudaMemcpyDeviceToDevice, st));
    saved = true;
    TSAT_CUDA(cudaEventCreate(&ev.a));
    TSAT_CUDA(cudaEventCreate(&ev.b));
    for (int cs : {1, 2, 4, 8}) {
      if (cs > 1 && (s->N > 256 || (int64_t)s->prob->n_inst * cs > 2LL * s->sm_count)) continue;
      s->persist_cs = cs;
      float ms = 1e30f;
      int r = TSAT_OK;
      for (int rep = 0; rep < 2; ++rep) {
        TSAT_CUDA(cudaMemcpyAsync(base, snap, s->core_bytes, cudaMemcpyDeviceToDevice, st));
        TSAT_CUDA(cudaEventRecord(ev.a, st));
        bool to_clustered = false;
        r = persist_launch(s, hp, n_steps, 0, &to_clustered);
        if (r == TSAT_OK && to_clustered) {
          set_error("the instances suit the cluster solver, not the persistent one");
          r = TSAT_EINVAL;
        }
        if (r != TSAT_OK) break;
        TSAT_CUDA(cudaEventRecord(ev.b, st));
        TSAT_CUDA(cudaEventSynchronize(ev.b));
        float x = 0;
        TSAT_CUDA(cudaEventElapsedTime(&x, ev.a, ev.b));
        ms = std::min(ms, x);
      }
      if (r == TSAT_ERANGE && cs == 1) continue;   // one block cannot take the instances: try the clusters
      if (r != TSAT_OK) return r;
      if (ms < best) { best = ms; best_cs = cs; }
    }
    TSAT_CUDA(cudaMemcpyAsync(base, snap, s->core_bytes, cudaMemcpyDeviceToDevice, st));
    return TSAT_OK;
  };
  rc = trials();
  if (rc == TSAT_OK && best >= 1e30f) { set_error("no persistent launch shape runs these instances"); rc = TSAT_ERANGE; }
  // a failed call keeps the previous setting and, as far as the device allows,
  // the caller's state
  if (rc != TSAT_OK && saved) (void)cudaMemcpyAsync(base, snap, s->core_bytes, cudaMemcpyDeviceToDevice, st);
  s->persist_cs = rc == TSAT_OK ? best_cs : keep;
  const int rl = leave(s, stream);
  if (rc != TSAT_OK) return rc;
  *h_blocks = best_cs;
  return rl;
}

int tsat_autotune_bytes(const tsat_state *s, size_t *bytes) {
  if (!s || !bytes) { set_error("NULL argument"); return TSAT_EINVAL; }
  *bytes = s->core_bytes + s->lit_bytes;
  return TSAT_OK;
}


int tsat_autotune(tsat_state *s, const tsat_hparams *hp, void *d_snapshot, size_t snapshot_bytes,
                  cudaStream_t stream, int32_t h_tuning[4]) {
  if (!s || !h_tuning || !d_snapshot) { set_error("NULL argument"); return TSAT_EINVAL; }
  int rc = check_hp(hp);
  if (rc) return rc;
  if ((rc = check_not_shard(s))) return rc;
  if (!s->initialised) { set_error("state not initialised"); return TSAT_ESTATE; }
  if (hp->layer != s->layer) { set_error("hp->layer differs from the state's layer"); return TSAT_ESTATE; }
  const size_t need = s->core_bytes + s->lit_bytes;
  if (snapshot_bytes < need) { set_error("snapshot buffer %zu < %zu bytes", snapshot_bytes, need); return TSAT_EWS; }
  if ((rc = enter(s, stream))) return rc;
  cudaStream_t st = s->stream;
  char *base = static_cast<char *>(s->base);
  char *snap = static_cast<char *>(d_snapshot);
  // the state as the caller left it; every trial starts from it, and it is
  // put back at the end
  auto save = [&]() -> int {
    TSAT_CUDA(cudaMemcpyAsync(snap, base, s->core_bytes, cudaMemcpyDeviceToDevice, st));
    if (s->lit_bytes)
      TSAT_CUDA(cudaMemcpyAsync(snap + s->core_bytes, base + s->lit_off, s->lit_bytes, cudaMemcpyDeviceToDevice, st));
    return TSAT_OK;
  };
  auto restore = [&]() -> int {
    TSAT_CUDA(cudaMemcpyAsync(base, snap, s->core_bytes, cudaMemcpyDeviceToDevice, st));
    if (s->lit_bytes)
      TSAT_CUDA(cudaMemcpyAsync(base + s->lit_off, snap + s->core_bytes, s->lit_bytes, cudaMemcpyDeviceToDevice, st));
    return TSAT_OK;
  };
  EventPair ev;
  const Hyper hy = make_hyper(*hp, 0);
  const LrSched ls = make_sched(*hp);
  const ProbDev &pd = s->prob->dev;
  // forward work-item size: the forward reads the bits and writes a scratch histogram
  const int keep_items = s->prob->item_clauses;
  int best_items = keep_items;
  float best = 1e30f;
  auto tune_items = [&]() -> int {
    for (int ic : kTuneItems) {
      int r;
      if ((r = s->prob->set_items(ic, st))) return r;
      float ms = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        TSAT_CUDA(cudaMemsetAsync(s->eval_hist, 0, sizeof(int32_t) * pd.n_inst * s->dev.lm1 * s->N, st));
        TSAT_CUDA(cudaEventRecord(ev.a, st));
        cudaError_t e = s->layer == TSAT_LAYER_RELAXED ? launch_relaxed_fwd(pd, s->dev, hy, 1, st)
                                                      : launch_fwd_hist(pd, s->dev, s->eval_hist, 0, st);
        if (e != cudaSuccess) return cuda_fail(e, "forward");
        TSAT_CUDA(cudaEventRecord(ev.b, st));
        TSAT_CUDA(cudaEventSynchronize(ev.b));
        float x = 0;
        TSAT_CUDA(cudaEventElapsedTime(&x, ev.a, ev.b));
        ms = std::min(ms, x);
      }
      if (ms < best) { best = ms; best_items = ic; }
    }
    return TSAT_OK;
  };
  // update launch shape: the step's own update (mode 0, hp's binarisation and
  // Eq. 5 mode), timed after the step's forward and gamma from the saved state;
  // blocks per SM around the default (resident blocks x 8 waves): 1, 2, 4, 8 and 10 waves
  int bps[5];
  tune_bps(s, bps);
  const int keep_b = s->upd_blocks_per_sm, keep_r = s->upd_rows_per_item;
  int best_b = keep_b, best_r = keep_r;
  auto sweep = [&]() -> int {
    best = 1e30f;
    for (int bb : bps)
      for (int rr : kTuneRpi) {
        s->upd_blocks_per_sm = bb;
        s->upd_rows_per_item = rr;
        float ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
          int r;
          if ((r = restore())) return r;
          if ((r = issue_pre_update(s, hy, ls, st))) return r;
          TSAT_CUDA(cudaEventRecord(ev.a, st));
          if ((r = issue_update(s, hy, ls, st))) return r;
          TSAT_CUDA(cudaEventRecord(ev.b, st));
          TSAT_CUDA(cudaEventSynchronize(ev.b));
          float x = 0;
          TSAT_CUDA(cudaEventElapsedTime(&x, ev.a, ev.b));
          ms = std::min(ms, x);
        }
        if (ms < best) { best = ms; best_b = bb; best_r = rr; }
      }
    return TSAT_OK;
  };
  bool saved = false;
  auto run = [&]() -> int {
    int r;
    if ((r = save())) return r;
    saved = true;
    TSAT_CUDA(cudaEventCreate(&ev.a));
    TSAT_CUDA(cudaEventCreate(&ev.b));
    if ((r = tune_items())) return r;
    if ((r = s->prob->set_items(best_items, st))) return r;
    if ((r = sweep())) return r;
    return restore();
  };
  rc = run();
  if (rc) {
    // a failed trial leaves the launch shapes as they were before the call
    // and, as far as the device allows, the caller's state
    if (saved) (void)restore();
    (void)s->prob->set_items(keep_items, st);
    s->upd_blocks_per_sm = keep_b;
    s->upd_rows_per_item = keep_r;
    (void)leave(s, stream);
    return rc;
  }
  s->upd_blocks_per_sm = best_b;
  s->upd_rows_per_item = best_r;
  if ((rc = leave(s, stream))) return rc;
  return tsat_get_tuning(s, h_tuning);
}

int32_t tsat_launches_per_step(const tsat_state *s) { return s ? s->launches_per_step : 0; }

}  // extern "C"
