// shard.cu -- one problem's N samples split over several processes, one GPU
// each (the paper ran on up to two GPUs, Sec. V; it gives no split).
//
// Every per-sample part of a step stays on its shard: the forward product
// R = P A (Eq. 1), SmoothMin and the loss (Eqs. 3-4) and the straight-through
// backward (Sec. III-B) of sample i read only column i.  Eq. 5 is what couples
// the samples of a row: the normaliser nu_v is a mean over all N samples, and
// its chain rule needs sum_i G_vi z_vi over all N samples.  So a sharded step
// is three calls with two all-reduces of V floats between them, which the
// caller makes (NCCL on GPUs):
//
//   tsat_shard_grad    forward, gamma, G = dL/dzt of the shard's samples, and
//                      the shard's row sums sum_i G_vi z_vi        -> all-reduce
//   tsat_shard_update  Eq. 5 chain rule with the summed dot, AdamW, and the
//                      shard's row sums of the new z (or |z|)      -> all-reduce
//   tsat_shard_finish  the new normaliser from the summed row sums and the
//                      bits of the next step (Eq. 2 or Philox, counters at the
//                      samples' global indices)
//
// tsat_shard_init is the init (Sec. IV-A) with global sample indices,
// followed by the same row-sum / finish pair.  Random draws use each sample's
// global index, so the shards together draw what one process with all N
// samples would.
#include <algorithm>

#include "internal.h"
#include "kernels.cuh"

namespace tsat {

// Row sums over this shard's samples, one warp per row: sum z (signed mean)
// or sum |z| (mean |z|); 0 for no normalisation.
__global__ void __launch_bounds__(kBlock) k_shard_rowsum(StateDev sd, int norm, float *out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  for (int64_t v = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); v < sd.V; v += nw) {
    float s = 0.f;
    if (norm != TSAT_NORM_NONE) {
      const float *z = sd.z + (size_t)v * sd.N;
      for (int i = lane; i < sd.N; i += 32) s += norm == TSAT_NORM_ABSMEAN ? fabsf(z[i]) : z[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) out[v] = s;
  }
}

// sum_i G_vi z_vi over this shard's samples (0 for rows of frozen instances
// and without normalisation).
__global__ void __launch_bounds__(kBlock) k_shard_dot(ProbDev pd, StateDev sd, int norm, const float *G, float *out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  for (int64_t v = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); v < sd.V; v += nw) {
    float s = 0.f;
    if (norm != TSAT_NORM_NONE && !sd.inst[__ldg(pd.var_inst + v)].found) {
      const float *z = sd.z + (size_t)v * sd.N, *g = G + (size_t)v * sd.N;
      for (int i = lane; i < sd.N; i += 32) s = fmaf(g[i], z[i], s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) out[v] = s;
  }
}

// Eq. 5 chain rule with the all-reduced dot, AdamW with the step scalars the
// gamma kernel wrote, and this shard's row sums of the new z.  Rows of frozen
// instances keep z, m, v (their row sums still cover the current z).
template <int NORM>
__global__ void __launch_bounds__(kBlock) k_shard_adamw(ProbDev pd, StateDev sd, Hyper hy, const float *G,
                                                       const float *dot_total, float *rowsum) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  const StepParams sp = *sd.sp;
  for (int64_t v = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); v < sd.V; v += nw) {
    const bool frozen = sd.inst[__ldg(pd.var_inst + v)].found;
    const size_t row = (size_t)v * sd.N;
    float psum = 0.f;
    if (frozen) {
      for (int i = lane; i < sd.N; i += 32) psum += NORM == TSAT_NORM_ABSMEAN ? fabsf(sd.z[row + i]) : sd.z[row + i];
    } else {
      const float rnu = __frcp_rn(sd.nu[v]);
      const float c2 = NORM == TSAT_NORM_NONE ? 0.f : dot_total[v] * rnu * rnu * (1.0f / (float)sd.n_total);
      for (int i = lane; i < sd.N; i += 32) {
        const size_t k = row + i;
        const float z = sd.z[k], Gv = G[k];
        float g;
        if (NORM == TSAT_NORM_NONE) {
          g = Gv;
        } else {
          const float dmu = (NORM == TSAT_NORM_ABSMEAN) ? (float)((z > 0.f) - (z < 0.f)) : 1.0f;
          g = Gv * rnu - c2 * dmu;
        }
        const float m = hy.beta1 * sd.m[k] + hy.omb1 * g;
        const float vv = hy.beta2 * sd.v[k] + hy.omb2 * (g * g);
        const float zn = z * sp.decay - sp.step_size * (m * adam_inv_denom(vv, sp.inv_sqrt_bc2, hy.eps));
        sd.z[k] = zn;
        sd.m[k] = m;
        sd.v[k] = vv;
        psum += NORM == TSAT_NORM_ABSMEAN ? fabsf(zn) : zn;
      }
    }
    for (int o = 16; o > 0; o >>= 1) psum += __shfl_xor_sync(0xFFFFFFFFu, psum, o);
    if (lane == 0) rowsum[v] = psum;
  }
}

// New normaliser nu_v = guard(total_v / N_total) (Eq. 5; 1 without
// normalisation) and the bits of step t = hdr->t from the current z: lane l
// decides samples 32 k + l (Eq. 2, or the Philox rule with the counter of
// the sample's global index), a ballot forms word k.  Rows of frozen
// instances keep their normaliser and copy the previous step's bits.
template <int NORM, int BIN>
__global__ void __launch_bounds__(kBlock) k_shard_bits(ProbDev pd, StateDev sd, Hyper hy, const float *total) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  const int64_t t = sd.hdr->t;
  uint32_t *dst = sd.bits + (size_t)(t & 1) * (size_t)sd.V * sd.W;
  const uint32_t *prev = sd.bits + (size_t)((t + 1) & 1) * (size_t)sd.V * sd.W;
  for (int64_t v = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); v < sd.V; v += nw) {
    const int inst = __ldg(pd.var_inst + v);
    if (t > 0 && sd.inst[inst].found) {
      for (int k = lane; k < sd.W; k += 32) dst[(size_t)v * sd.W + k] = prev[(size_t)v * sd.W + k];
      continue;
    }
    const float nun = NORM == TSAT_NORM_NONE ? 1.0f : guard_nu(total[v] / (float)sd.n_total);
    const float rnn = __frcp_rn(nun);
    const RowStream rs = row_stream(pd, hy.key0, inst, v);
    for (int k = 0; k < sd.W; ++k) {
      const int i = 32 * k + lane;
      const float zt = __fmul_rn(sd.z[(size_t)v * sd.N + i], rnn);
      uint32_t half = 0;
      if (BIN == TSAT_BIN_PHILOX) {
        const uint32_t ig = (uint32_t)(sd.sample_base + i);   // global sample index
        const uint4 r = philox4x32_10(make_uint4(ig >> 3, rs.row, (uint32_t)t, kTagBin), rs.k0, hy.key1);
        const uint32_t e = ig & 7;   // half e of the block: word e / 2, low half first
        half = half16(e < 4 ? r.x : r.z, e < 4 ? r.y : r.w, (int)(e & 3));
      }
      const uint32_t word = __ballot_sync(0xFFFFFFFFu, binarize_one(zt, BIN, hy.bin_c, half) != 0u);
      if (lane == 0) dst[(size_t)v * sd.W + k] = word;
    }
    if (lane == 0) sd.nu[v] = nun;
  }
}

static int shard_grid(const tsat_state *s) {
  const int64_t need = (s->prob->dev.V + kWarps - 1) / kWarps;
  return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)s->sm_count * 16, need));
}

static int check_shard(tsat_state *s, const tsat_hparams *hp) {
  if (!s || !hp) { set_error("NULL argument"); return TSAT_EINVAL; }
  if (hp->layer != TSAT_LAYER_STE || s->layer != TSAT_LAYER_STE) {
    set_error("sample sharding runs the STE layer");
    return TSAT_EINVAL;
  }
  if (hp->mix_restart) { set_error("sample sharding does not mix assignments"); return TSAT_EINVAL; }
  if (hp->norm < 0 || hp->norm > 2 || hp->binarize < 0 || hp->binarize > 1 || !(hp->tau > 0.f) ||
      !(hp->bin_temp > 0.f) || hp->reserved != 0) {
    set_error("hparams out of range");
    return TSAT_EINVAL;
  }
  return TSAT_OK;
}

template <int NORM>
static cudaError_t launch_shard_bits_n(const tsat_state *s, const Hyper &hy, const float *total, cudaStream_t st) {
  if (hy.binarize == TSAT_BIN_PHILOX)
    k_shard_bits<NORM, TSAT_BIN_PHILOX><<<shard_grid(s), kBlock, 0, st>>>(s->prob->dev, s->dev, hy, total);
  else
    k_shard_bits<NORM, TSAT_BIN_DET><<<shard_grid(s), kBlock, 0, st>>>(s->prob->dev, s->dev, hy, total);
  return cudaGetLastError();
}

static cudaError_t launch_shard_bits(const tsat_state *s, const Hyper &hy, const float *total, cudaStream_t st) {
  switch (hy.norm) {
    case TSAT_NORM_SIGNED_MEAN: return launch_shard_bits_n<TSAT_NORM_SIGNED_MEAN>(s, hy, total, st);
    case TSAT_NORM_ABSMEAN: return launch_shard_bits_n<TSAT_NORM_ABSMEAN>(s, hy, total, st);
    default: return launch_shard_bits_n<TSAT_NORM_NONE>(s, hy, total, st);
  }
}

}  // namespace tsat

using namespace tsat;

extern "C" {

int tsat_state_set_shard(tsat_state *s, int32_t sample_base, int32_t n_total) {
  if (!s) { set_error("NULL argument"); return TSAT_EINVAL; }
  if (n_total < s->N || n_total % s->N || sample_base < 0 || sample_base % s->N || sample_base + s->N > n_total) {
    set_error("shard [%d, %d) does not tile %d samples in blocks of %d", sample_base, sample_base + s->N, n_total,
              s->N);
    return TSAT_EINVAL;
  }
  s->dev.sample_base = sample_base;
  s->dev.n_total = n_total;
  for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second);
  s->graphs.clear();
  return TSAT_OK;
}

int tsat_shard_init(tsat_state *s, const tsat_hparams *hp, float *d_rowsum, cudaStream_t stream) {
  int rc = check_shard(s, hp);
  if (rc) return rc;
  if (!d_rowsum) { set_error("NULL argument"); return TSAT_EINVAL; }
  if ((rc = state_enter(s, stream))) return rc;
  const ProbDev &pd = s->prob->dev;
  const Hyper hy = make_hyper(*hp, 0);
  TSAT_CUDA(cudaMemsetAsync(s->dev.hist, 0, sizeof(int32_t) * (size_t)pd.n_inst * s->dev.lm1 * s->N, s->stream));
  if ((rc = reset_state(s, s->stream))) return rc;
  cudaError_t e = launch_init(pd, s->dev, hy, nullptr, 1.0f, shard_grid(s), s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "init");
  k_shard_rowsum<<<shard_grid(s), kBlock, 0, s->stream>>>(s->dev, hp->norm, d_rowsum);
  TSAT_LAUNCH_CHECK("row sums");
  s->initialised = true;
  return state_leave(s, stream);
}

int tsat_shard_grad(tsat_state *s, const tsat_hparams *hp, float *d_G, float *d_rowdot, cudaStream_t stream) {
  int rc = check_shard(s, hp);
  if (rc) return rc;
  if (!d_G || !d_rowdot) { set_error("NULL argument"); return TSAT_EINVAL; }
  if (!s->initialised) { set_error("state not initialised (tsat_shard_init)"); return TSAT_ESTATE; }
  if ((rc = state_enter(s, stream))) return rc;
  const ProbDev &pd = s->prob->dev;
  const Hyper hy = make_hyper(*hp, 0);
  const LrSched ls = make_sched(*hp);
  Hyper hg = hy;
  hg.norm = TSAT_NORM_NONE;   // the update kernels' gradient mode then returns G itself
  cudaStream_t st = s->stream;
  cudaError_t e;
  // Eq. 1 forward and the dL/dR table of this step (the step counter stays)
  if ((e = launch_fwd_hist(pd, s->dev, s->dev.hist, 1, st)) != cudaSuccess) return cuda_fail(e, "forward");
  if ((e = launch_gamma(pd, s->dev, hy, ls, s->dev.hist, 0, 1, nullptr, nullptr, st)) != cudaSuccess)
    return cuda_fail(e, "gamma");
  // G = dL/dzt of this shard's samples at the current bits (straight-through)
  if ((e = launch_update(pd, s->dev, hg, 1, s->dev.z, d_G, 1.0f, update_grid(s), s->upd_rows_per_item, st)) !=
      cudaSuccess)
    return cuda_fail(e, "gradient");
  // status records, freezing, step scalars, and the step counter advances
  if ((e = launch_gamma(pd, s->dev, hy, ls, s->dev.hist, 1, 1, nullptr, nullptr, st)) != cudaSuccess)
    return cuda_fail(e, "gamma");
  k_shard_dot<<<shard_grid(s), kBlock, 0, st>>>(pd, s->dev, hp->norm, d_G, d_rowdot);
  TSAT_LAUNCH_CHECK("row dot");
  return state_leave(s, stream);
}

int tsat_shard_update(tsat_state *s, const tsat_hparams *hp, const float *d_G, const float *d_rowdot_total,
                      float *d_rowsum, cudaStream_t stream) {
  int rc = check_shard(s, hp);
  if (rc) return rc;
  if (!d_G || !d_rowdot_total || !d_rowsum) { set_error("NULL argument"); return TSAT_EINVAL; }
  if (!s->initialised) { set_error("state not initialised (tsat_shard_init)"); return TSAT_ESTATE; }
  if ((rc = state_enter(s, stream))) return rc;
  const Hyper hy = make_hyper(*hp, 0);
  const ProbDev &pd = s->prob->dev;
  switch (hp->norm) {
    case TSAT_NORM_SIGNED_MEAN:
      k_shard_adamw<TSAT_NORM_SIGNED_MEAN><<<shard_grid(s), kBlock, 0, s->stream>>>(pd, s->dev, hy, d_G,
                                                                                     d_rowdot_total, d_rowsum);
      break;
    case TSAT_NORM_ABSMEAN:
      k_shard_adamw<TSAT_NORM_ABSMEAN><<<shard_grid(s), kBlock, 0, s->stream>>>(pd, s->dev, hy, d_G, d_rowdot_total,
                                                                                 d_rowsum);
      break;
    default:
      k_shard_adamw<TSAT_NORM_NONE><<<shard_grid(s), kBlock, 0, s->stream>>>(pd, s->dev, hy, d_G, d_rowdot_total,
                                                                              d_rowsum);
      break;
  }
  TSAT_LAUNCH_CHECK("shard update");
  return state_leave(s, stream);
}

int tsat_shard_finish(tsat_state *s, const tsat_hparams *hp, const float *d_rowsum_total, cudaStream_t stream) {
  int rc = check_shard(s, hp);
  if (rc) return rc;
  if (!d_rowsum_total) { set_error("NULL argument"); return TSAT_EINVAL; }
  if (!s->initialised) { set_error("state not initialised (tsat_shard_init)"); return TSAT_ESTATE; }
  if ((rc = state_enter(s, stream))) return rc;
  cudaError_t e = launch_shard_bits(s, make_hyper(*hp, 0), d_rowsum_total, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "shard bits");
  return state_leave(s, stream);
}

}  // extern "C"
