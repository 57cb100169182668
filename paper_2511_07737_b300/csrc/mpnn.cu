// mpnn.cu -- learned proposer of initial variable logits: a 3-layer message-
// passing network on the literal-clause bipartite graph of a loaded problem
// (the problem's clause-major CSR and variable-major occurrence index), with
// BF16 weights and FP32 accumulation, forward and hand-written backward.
//
// Network (hidden H = 64, literal l, its negation l^1, clause c):
//   f_l   = [1, log(1 + deg l), log(1 + deg l^1)]
//   h0_l  = relu(W0 f_l + b0)
//   for t = 1..3:
//     m_c  = mean_{l in c} h_l                    (clause-major gather)
//     e_c  = relu(Wc_t m_c + bc_t)
//     a_l  = mean_{c owns l} e_c                  (variable-major gather)
//     h_l  = relu(Wl_t [h_l ; a_l ; h_{l^1}] + bl_t)
//   logit_v = wo [h_{2v} ; h_{2v+1}] + bo
// Every gradient of a gather is the opposite gather (no atomics); weight
// gradients reduce per-block partials in a fixed order.  The dense layers,
// their input gradients and their weight gradients run on the tensor cores
// (tcgen05.mma, mpnn_tc.cu).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "kernels.cuh"

namespace tsat {

constexpr int kH = 64;
constexpr int kLayers = 3;
constexpr int kFeat = 3;
// parameter layout (floats)
constexpr int kOffW0 = 0;
constexpr int kOffB0 = kOffW0 + kH * kFeat;
constexpr int kOffLayer = kOffB0 + kH;
constexpr int kLayerSize = kH * kH + kH + kH * 3 * kH + kH;   // Wc, bc, Wl, bl
constexpr int kOffOut = kOffLayer + kLayers * kLayerSize;
constexpr int kNParams = kOffOut + 2 * kH + 1;
__host__ __device__ constexpr int off_wc(int t) { return kOffLayer + t * kLayerSize; }
__host__ __device__ constexpr int off_bc(int t) { return off_wc(t) + kH * kH; }
__host__ __device__ constexpr int off_wl(int t) { return off_bc(t) + kH; }
__host__ __device__ constexpr int off_bl(int t) { return off_wl(t) + kH * 3 * kH; }

struct MpWs {  // activations kept for the backward pass
  float *feat;                     // [2V][3]
  float *h[kLayers + 1];           // [2V][H]
  float *m[kLayers], *e[kLayers];  // [C][H]
  float *a[kLayers];               // [2V][H]
  float *dh, *dh2, *da, *de, *dm;  // gradient buffers
  float *part;                     // weight-gradient partials [kPartBlocks][64][193]
  __nv_bfloat16 *wb;               // BF16 copy of the parameters
  float *linv;                     // [2V] 1 / max(literal degree, 1)
  float *cinv;                     // [C] 1 / clause length
  float *dlog, *lossv;             // [V] dL/dlogit and per-variable loss terms
  int *err;                        // set by a tensor-core layer whose completion wait timed out
};
constexpr int kPartBlocks = 148 * 3;   // weight-gradient blocks: three per SM

static size_t mp_ws_bytes(int64_t V, int64_t C) {
  const int64_t L = 2 * V;
  size_t b = 0;
  auto add = [&](size_t x) { b += align_up(x, 256); };
  add(sizeof(float) * L * kFeat);
  for (int t = 0; t <= kLayers; ++t) add(sizeof(float) * L * kH);
  for (int t = 0; t < kLayers; ++t) {
    add(sizeof(float) * C * kH);
    add(sizeof(float) * C * kH);
    add(sizeof(float) * L * kH);
  }
  add(sizeof(float) * L * kH * 3);   // dh, dh2, da
  add(sizeof(float) * C * kH * 2);   // de, dm
  add(sizeof(float) * kPartBlocks * kH * (3 * kH + 1));
  add(sizeof(__nv_bfloat16) * kNParams);
  add(sizeof(float) * L);
  add(sizeof(float) * C);
  add(sizeof(float) * V);
  add(sizeof(float) * V);
  add(sizeof(int) * 4);
  return b;
}

static MpWs mp_ws_plan(void *base, int64_t V, int64_t C) {
  const int64_t L = 2 * V;
  MpWs w{};
  char *p = (char *)base;
  auto take = [&](size_t x) { char *r = p; p += align_up(x, 256); return r; };
  w.feat = (float *)take(sizeof(float) * L * kFeat);
  for (int t = 0; t <= kLayers; ++t) w.h[t] = (float *)take(sizeof(float) * L * kH);
  for (int t = 0; t < kLayers; ++t) {
    w.m[t] = (float *)take(sizeof(float) * C * kH);
    w.e[t] = (float *)take(sizeof(float) * C * kH);
    w.a[t] = (float *)take(sizeof(float) * L * kH);
  }
  w.dh = (float *)take(sizeof(float) * L * kH);
  w.dh2 = (float *)take(sizeof(float) * L * kH);
  w.da = (float *)take(sizeof(float) * L * kH);
  w.de = (float *)take(sizeof(float) * C * kH);
  w.dm = (float *)take(sizeof(float) * C * kH);
  w.part = (float *)take(sizeof(float) * kPartBlocks * kH * (3 * kH + 1));
  w.wb = (__nv_bfloat16 *)take(sizeof(__nv_bfloat16) * kNParams);
  w.linv = (float *)take(sizeof(float) * L);
  w.cinv = (float *)take(sizeof(float) * C);
  w.dlog = (float *)take(sizeof(float) * V);
  w.lossv = (float *)take(sizeof(float) * V);
  w.err = (int *)take(sizeof(int) * 4);
  return w;
}

// ------------------------------------------------------------------ kernels
// The forward's preparation in one launch (a small graph's forward is a chain
// of short kernels, each paying its launch): the error flag cleared, the BF16
// copy of the parameters (items [0, n)), the input features and inverse
// literal degrees 1 / max(deg, 1), the variable-major mean's scale (items
// [n, n + V), one variable each), and the inverse clause lengths, the
// clause-major mean's scale (items [n + V, n + V + C)).
__global__ void k_mp_prep(const float *p, __nv_bfloat16 *b, int n, ProbDev pd, float *linv, float *feat,
                          float *cinv, int *err) {
  const int64_t total = (int64_t)n + pd.V + pd.C;
  if (blockIdx.x == 0 && threadIdx.x == 0) *err = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      b[i] = __float2bfloat16_rn(p[i]);
    } else if (i < n + pd.V) {
      const int64_t v = i - n;
      int dp = 0, dn = 0;
      for (int32_t o = pd.vptr[v]; o < pd.vptr[v + 1]; ++o) (pd.vocc[o] & 1) ? ++dn : ++dp;
      linv[2 * v] = 1.0f / fmaxf((float)dp, 1.f);
      linv[2 * v + 1] = 1.0f / fmaxf((float)dn, 1.f);
      const float lp = logf(1.0f + (float)dp), ln = logf(1.0f + (float)dn);
      float *f0 = feat + (2 * v) * kFeat, *f1 = feat + (2 * v + 1) * kFeat;
      f0[0] = 1.f; f0[1] = lp; f0[2] = ln;
      f1[0] = 1.f; f1[1] = ln; f1[2] = lp;
    } else {
      const int64_t c = i - n - pd.V;
      cinv[c] = 1.0f / (float)(pd.cptr[c + 1] - pd.cptr[c]);
    }
  }
}

struct DIn {
  const float *x;
  int K, xr;
};

// tensor-core dense layers (mpnn_tc.cu)
cudaError_t mp_dense_tc(const float *x, int K, int64_t M, const __nv_bfloat16 *W, const __nv_bfloat16 *bias, float *Y,
                        int *err, cudaStream_t st);
cudaError_t mp_literal_tc(const float *h, const float *a, int64_t M, const __nv_bfloat16 *W, const __nv_bfloat16 *bias,
                          float *Y, int *err, cudaStream_t st);
cudaError_t mp_dx_tc(const float *dZ, int64_t M, const __nv_bfloat16 *W, const float *rscale, float *dX, int *err,
                     cudaStream_t st);
cudaError_t mp_literal_dx_tc(const float *dZ, int64_t M, const __nv_bfloat16 *W, const float *rscale, float *dh,
                             float *da, int *err, cudaStream_t st);
int mp_wgrad_tc(const float *dZ, int64_t M, int nin, int K, const float *const *x, const int *xr, float *part,
                int max_blocks, int *err, cudaStream_t st, cudaError_t *e);
cudaError_t mp_prepare_forward();
// small graphs (a layer of at most mp_small_rows(literal) rows): each
// message-passing layer's gather fused into its CUDA-core dense layer
cudaError_t mp_clause_small(const ProbDev &pd, const float *h, const float *cinv, float *m, const __nv_bfloat16 *W,
                            const __nv_bfloat16 *bias, float *Y, cudaStream_t st);
cudaError_t mp_literal_small(const ProbDev &pd, const float *h, const float *e, const float *linv, float *a,
                             const __nv_bfloat16 *W, const __nv_bfloat16 *bias, float *Y, cudaStream_t st);
int mp_small_rows(bool literal);

__device__ __forceinline__ int warp_max(int x) {
  for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xFFFFFFFFu, x, o));
  return x;
}

__device__ __forceinline__ void add4(float4 &a, const float4 &b) {
  a.x += b.x;
  a.y += b.y;
  a.z += b.z;
  a.w += b.w;
}

__device__ __forceinline__ float4 scale4(const float4 &a, float s) { return make_float4(a.x * s, a.y * s, a.z * s, a.w * s); }

// y = x where m > 0, else 0 (the ReLU's backward, mask from its output)
__device__ __forceinline__ float4 relu_mask4(const float4 &x, const float4 &m) {
  return make_float4(m.x > 0.f ? x.x : 0.f, m.y > 0.f ? x.y : 0.f, m.z > 0.f ? x.z : 0.f, m.w > 0.f ? x.w : 0.f);
}

// Clause-major gather: out[c] = sum over the literals l of clause c of
// src[l] (64 floats).  A warp takes 4 gpw consecutive clauses (gpw = 1..8
// groups; 8 for large graphs, fewer when the graph is too small to give every
// SM enough warps, so that a small graph's warps do not walk eight groups one
// after another): their offsets come in two coalesced loads (lane l:
// cptr[c0 + l], cptr[c0 + l + 1]) and are handed out by shuffles; it then
// works through them in gpw groups of 4 clauses (8 lanes per clause, 8 floats
// per lane as two float4).  A group's
// literal ids are loaded 8 at a time by its lanes and broadcast, and the next
// group's ids are loaded while this group's rows are summed, so only the row
// loads wait.  The row loads of the four clauses are issued together, four
// rows per round (the round count follows the group's longest clause; a
// shorter clause's loads past its end are predicated off).
//   MODE 0 (forward, clause mean): out[c] = sum * cinv[c]
//   MODE 1 (backward of the variable-major mean, src pre-scaled by 1 / deg):
//          out[c] = sum where e[c] > 0 (the clause layer's ReLU), else 0
template <int MODE>
__global__ void __launch_bounds__(256) k_mp_clause_gather(ProbDev pd, const float *__restrict__ src,
                                                          const float *__restrict__ cinv, const float *__restrict__ e,
                                                          float *__restrict__ out, int gpw) {
  const int lane = threadIdx.x & 31, gl = lane & 7, gbase = lane & ~7;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5, C = pd.C;
  const int cpw = 4 * gpw;   // clauses per warp
  for (int64_t c0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * cpw; c0 < C; c0 += nw * cpw) {
    const int32_t pb = __ldg(pd.cptr + min(c0 + lane, C)), pe = __ldg(pd.cptr + min(c0 + lane + 1, C));
    // group g: clauses c0 + 4 g + lane / 8; returns the lane's first literal id (clauses past C are empty)
    auto ids = [&](int g, int32_t &b, int32_t &n) -> int32_t {
      const int q = 4 * g + (lane >> 3);
      b = __shfl_sync(0xFFFFFFFFu, pb, q);
      n = __shfl_sync(0xFFFFFFFFu, pe, q) - b;
      return gl < min(n, 8) ? __ldg(pd.clit + b + gl) : 0;
    };
    int32_t b, n;
    int32_t myl = ids(0, b, n);
    for (int g = 0; g < gpw; ++g) {
      int32_t bn = 0, nn = 0, myln = 0;
      if (g + 1 < gpw) myln = ids(g + 1, bn, nn);
      const int64_t c = c0 + 4 * g + (lane >> 3);
      const int nmax = warp_max(n);
      float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;
      for (int o = 0; o < nmax; o += 8) {
        const int cnt = min(max(n - o, 0), 8);
        const int32_t ml = o == 0 ? myl : (gl < cnt ? __ldg(pd.clit + b + o + gl) : 0);
        const int rounds = min(nmax - o, 8);
        for (int j = 0; j < rounds; j += 4) {
          float4 x[4][2];
#pragma unroll
          for (int q = 0; q < 4; ++q) {   // predicated loads: a clause past its end loads nothing
            const int32_t l = __shfl_sync(0xFFFFFFFFu, ml, gbase + ((j + q) & 7));
            const float4 *p = reinterpret_cast<const float4 *>(src + (int64_t)l * kH) + 2 * gl;
            const bool in = j + q < cnt;
            x[q][0] = in ? __ldg(p) : make_float4(0.f, 0.f, 0.f, 0.f);
            x[q][1] = in ? __ldg(p + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            add4(s0, x[q][0]);
            add4(s1, x[q][1]);
          }
        }
      }
      if (c < C) {
        float4 *dst = reinterpret_cast<float4 *>(out + c * kH) + 2 * gl;
        if (MODE == 0) {
          const float sc = __ldg(cinv + c);
          dst[0] = scale4(s0, sc);
          dst[1] = scale4(s1, sc);
        } else {
          const float4 *ep = reinterpret_cast<const float4 *>(e + c * kH) + 2 * gl;
          dst[0] = relu_mask4(s0, __ldg(ep));
          dst[1] = relu_mask4(s1, __ldg(ep + 1));
        }
      }
      b = bn;
      n = nn;
      myl = myln;
    }
  }
}

// Variable-major gather: for both literals of variable v, the sum over the
// clauses c owning the literal of src[c] (64 floats), warp per variable (two
// floats per lane).  The occurrence records are loaded 32 at a time by the
// lanes and broadcast; 8 row loads are issued per round (predicated off past
// the last occurrence).
//   MODE 0 (forward, literal mean): out[l] = sum * linv[l]
//   MODE 1 (backward of the clause-major mean, src pre-scaled by 1 / |c|):
//          out[l] = (out[l] + sum) where h[l] > 0, else 0 (the ReLU of the
//          layer that produced h, whose backward comes next)
template <int MODE>
__global__ void __launch_bounds__(256) k_mp_var_gather(ProbDev pd, const float *__restrict__ src,
                                                       const float *__restrict__ linv, const float *__restrict__ h,
                                                       float *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < pd.V; v += nw) {
    const int32_t ob = __ldg(pd.vptr + v), oe = __ldg(pd.vptr + v + 1);
    float2 ap = make_float2(0.f, 0.f), an = ap;
    for (int32_t base = ob; base < oe; base += 32) {
      const int cnt = min(32, oe - base);
      const int32_t myoc = lane < cnt ? __ldg(pd.vocc + base + lane) : 0;
      for (int j = 0; j < cnt; j += 8) {
        float2 x[8];
        int32_t oc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {   // predicated loads past the last occurrence
          oc[q] = __shfl_sync(0xFFFFFFFFu, myoc, (j + q) & 31);
          x[q] = j + q < cnt ? __ldg(reinterpret_cast<const float2 *>(src + (int64_t)(oc[q] >> 1) * kH) + lane)
                             : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (oc[q] & 1) {
            an.x += x[q].x;
            an.y += x[q].y;
          } else {
            ap.x += x[q].x;
            ap.y += x[q].y;
          }
        }
      }
    }
    float2 *p0 = reinterpret_cast<float2 *>(out + (2 * v) * kH) + lane;
    float2 *p1 = reinterpret_cast<float2 *>(out + (2 * v + 1) * kH) + lane;
    if (MODE == 0) {
      const float sp = __ldg(linv + 2 * v), sn = __ldg(linv + 2 * v + 1);
      *p0 = make_float2(ap.x * sp, ap.y * sp);
      *p1 = make_float2(an.x * sn, an.y * sn);
    } else {
      const float2 m0 = __ldg(reinterpret_cast<const float2 *>(h + (2 * v) * kH) + lane);
      const float2 m1 = __ldg(reinterpret_cast<const float2 *>(h + (2 * v + 1) * kH) + lane);
      const float2 d0 = *p0, d1 = *p1;
      *p0 = make_float2(m0.x > 0.f ? d0.x + ap.x : 0.f, m0.y > 0.f ? d0.y + ap.y : 0.f);
      *p1 = make_float2(m1.x > 0.f ? d1.x + an.x : 0.f, m1.y > 0.f ? d1.y + an.y : 0.f);
    }
  }
}

__global__ void k_mp_out(ProbDev pd, const float *h, const __nv_bfloat16 *wb, float *logits) {
  const int lane = threadIdx.x & 31;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < pd.V;
       v += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    float s = 0.f;
    for (int k = lane; k < 2 * kH; k += 32) s += h[(2 * v) * kH + k] * __bfloat162float(wb[kOffOut + k]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) logits[v] = s + __bfloat162float(wb[kOffOut + 2 * kH]);
  }
}

// binary cross-entropy per variable, mean over the variables of each instance
__global__ void k_mp_bce(ProbDev pd, const float *logits, const uint8_t *y, float *loss_v, float *dlog) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < pd.V; v += (int64_t)gridDim.x * blockDim.x) {
    const float x = logits[v], t = (float)y[v];
    const int inst = pd.var_inst[v];
    const float inv = 1.0f / (float)pd.inst[inst].n_vars;
    loss_v[v] = (fmaxf(x, 0.f) - x * t + log1pf(expf(-fabsf(x)))) * inv;
    dlog[v] = (1.0f / (1.0f + expf(-x)) - t) * inv;
  }
}

// output layer backward: dh3[2v .. 2v+1] = dlogit_v * wo
// dh[l] = dlogit[v] wo[k] where h[l] > 0 (the last literal layer's ReLU), else 0
__global__ void k_mp_out_bwd(ProbDev pd, const float *dlog, const __nv_bfloat16 *wb, const float *h, float *dh) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)pd.V * 2 * kH;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / (2 * kH);
    const int k = (int)(i % (2 * kH));
    dh[i] = h[i] > 0.f ? dlog[v] * __bfloat162float(wb[kOffOut + k]) : 0.f;
  }
}

// grad[W(o,k)] (+)= sum_b part[b][o][k], bias into gbias[o]
__global__ void k_mp_wgrad_reduce(const float *part, int nb, int Kt, float *gW, float *gb) {
  const int ncol = Kt + 1;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < kH * ncol; idx += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part[(size_t)b * kH * ncol + idx];
    const int o = idx / ncol, k = idx % ncol;
    if (k == Kt) gb[o] = s; else gW[o * Kt + k] = s;
  }
}

// output-layer weight gradient: gwo[k] = sum_v dlog_v h[2v*H + k], gbo = sum_v dlog_v
__global__ void k_mp_out_wgrad(ProbDev pd, const float *h, const float *dlog, float *part) {
  const int64_t r0 = (int64_t)pd.V * blockIdx.x / gridDim.x, r1 = (int64_t)pd.V * (blockIdx.x + 1) / gridDim.x;
  for (int k = threadIdx.x; k <= 2 * kH; k += blockDim.x) {
    float acc = 0.f;
    for (int64_t v = r0; v < r1; ++v) acc = fmaf(dlog[v], k < 2 * kH ? h[2 * v * kH + k] : 1.f, acc);
    part[(size_t)blockIdx.x * (2 * kH + 1) + k] = acc;
  }
}
__global__ void k_mp_out_reduce(const float *part, int nb, float *g) {
  for (int k = threadIdx.x; k <= 2 * kH; k += blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part[(size_t)b * (2 * kH + 1) + k];
    g[kOffOut + k] = s;
  }
}

// parameter init: Xavier-uniform from Philox, zero biases
__global__ void k_mp_init(float *p, uint32_t k0, uint32_t k1) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParams; i += gridDim.x * blockDim.x) {
    float fan_in = 0.f, fan_out = kH;
    bool bias = false;
    if (i < kOffB0) fan_in = kFeat;
    else if (i < kOffLayer) bias = true;
    else if (i < kOffOut) {
      const int j = (i - kOffLayer) % kLayerSize;
      if (j < kH * kH) fan_in = kH;
      else if (j < kH * kH + kH) bias = true;
      else if (j < kH * kH + kH + 3 * kH * kH) fan_in = 3 * kH;
      else bias = true;
    } else if (i < kOffOut + 2 * kH) { fan_in = 2 * kH; fan_out = 1; }
    else bias = true;
    if (bias) { p[i] = 0.f; continue; }
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, 0, 0, 0x4D504E4Eu), k0, k1);
    const float u = ((float)(r.x >> 8) + 0.5f) * (1.0f / 16777216.0f);
    const float lim = sqrtf(6.0f / (fan_in + fan_out));
    p[i] = (2.f * u - 1.f) * lim;
  }
}

__global__ void k_mp_adam(float *p, const float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                          float bc1, float bc2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    m[i] = b1 * m[i] + (1.f - b1) * gi;
    v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
    p[i] -= lr * (m[i] / bc1) / (sqrtf(v[i] / bc2) + eps);
  }
}

__global__ void k_mp_sum(const float *x, int64_t n, float *out) {  // one block, fixed order
  __shared__ float sh[1024];
  float s = 0.f;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// ------------------------------------------------------------------ host orchestration
static int grid_for(int64_t work, int per_block) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(148 * 16, (work + per_block - 1) / per_block));
}

// Groups of 4 clauses per warp of the clause-major gather, and its grid: 8
// groups when the graph gives at least 16 warps per SM that way, else fewer
// (down to one group per warp).
static int mp_cgather_gpw(int64_t C) {
  const int64_t target = 148 * 16;
  int gpw = 8;
  while (gpw > 1 && (C + 4 * gpw - 1) / (4 * gpw) < target) gpw >>= 1;
  return gpw;
}
static int mp_cgather_grid(int64_t C, int gpw) { return grid_for((C + 4 * gpw - 1) / (4 * gpw) * 32, 256); }

static int mp_forward(const tsat_problem *p, const float *params, MpWs &w, float *logits, cudaStream_t st) {
  const ProbDev &pd = p->dev;
  const int64_t L = 2 * (int64_t)p->V, C = p->C;
  k_mp_prep<<<grid_for(kNParams + p->V + C, 256), 256, 0, st>>>(params, w.wb, kNParams, pd, w.linv, w.feat, w.cinv,
                                                                  w.err);
  TSAT_LAUNCH_CHECK("mpnn features");
  cudaError_t e = mp_dense_tc(w.feat, kFeat, L, w.wb + kOffW0, w.wb + kOffB0, w.h[0], w.err, st);
  if (e != cudaSuccess) return cuda_fail(e, "mpnn input layer");
  for (int t = 0; t < kLayers; ++t) {
    if (C <= mp_small_rows(false)) {
      e = mp_clause_small(pd, w.h[t], w.cinv, w.m[t], w.wb + off_wc(t), w.wb + off_bc(t), w.e[t], st);
    } else {
      const int gpw = mp_cgather_gpw(C);
      k_mp_clause_gather<0><<<mp_cgather_grid(C, gpw), 256, 0, st>>>(pd, w.h[t], w.cinv, nullptr, w.m[t], gpw);
      e = mp_dense_tc(w.m[t], kH, C, w.wb + off_wc(t), w.wb + off_bc(t), w.e[t], w.err, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "mpnn clause layer");
    if (L <= mp_small_rows(true)) {
      e = mp_literal_small(pd, w.h[t], w.e[t], w.linv, w.a[t], w.wb + off_wl(t), w.wb + off_bl(t), w.h[t + 1], st);
    } else {
      k_mp_var_gather<0><<<grid_for((int64_t)p->V * 32, 256), 256, 0, st>>>(pd, w.e[t], w.linv, nullptr, w.a[t]);
      e = mp_literal_tc(w.h[t], w.a[t], L, w.wb + off_wl(t), w.wb + off_bl(t), w.h[t + 1], w.err, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "mpnn literal layer");
  }
  if (logits) k_mp_out<<<grid_for((int64_t)p->V * 32, 256), 256, 0, st>>>(pd, w.h[kLayers], w.wb, logits);
  TSAT_LAUNCH_CHECK("mpnn forward");
  return TSAT_OK;
}

static int wgrad(int nin, DIn a, DIn b, DIn c, const float *dZ, int64_t M, float *part, float *gW, float *gb,
                 int *err, cudaStream_t st) {
  const int Kt = a.K + (nin > 1 ? b.K : 0) + (nin > 2 ? c.K : 0);
  const float *x[3] = {a.x, b.x, c.x};
  const int xr[3] = {a.xr, b.xr, c.xr};
  cudaError_t e = cudaSuccess;
  const int nb = mp_wgrad_tc(dZ, M, nin, a.K, x, xr, part, kPartBlocks, err, st, &e);
  if (e != cudaSuccess) return cuda_fail(e, "mpnn weight gradient");
  k_mp_wgrad_reduce<<<(kH * (Kt + 1) + 255) / 256, 256, 0, st>>>(part, nb, Kt, gW, gb);
  TSAT_LAUNCH_CHECK("mpnn weight gradient");
  return TSAT_OK;
}

static int mp_backward(const tsat_problem *p, MpWs &w, const float *dlog, float *grad, cudaStream_t st) {
  const ProbDev &pd = p->dev;
  const int64_t L = 2 * (int64_t)p->V, C = p->C;
  DIn none{nullptr, 0, 0};
  int rc;
  // output layer; dh leaves masked by the last literal layer's ReLU
  {
    const int nb = (int)std::min<int64_t>(kPartBlocks, std::max<int64_t>(1, p->V / 64));
    k_mp_out_wgrad<<<nb, 256, 0, st>>>(pd, w.h[kLayers], dlog, w.part);
    k_mp_out_reduce<<<1, 256, 0, st>>>(w.part, nb, grad);
    k_mp_out_bwd<<<grid_for(p->V * 2 * kH, 256), 256, 0, st>>>(pd, dlog, w.wb, w.h[kLayers], w.dh);
    TSAT_LAUNCH_CHECK("mpnn output backward");
  }
  for (int t = kLayers - 1; t >= 0; --t) {
    // literal layer: h[t+1] = relu(Wl [h[t]; a[t]; h[t]^1] + bl), dh = dL/d(pre-activation)
    if ((rc = wgrad(3, DIn{w.h[t], kH, 0}, DIn{w.a[t], kH, 0}, DIn{w.h[t], kH, 1}, w.dh, L, w.part,
                    grad + off_wl(t), grad + off_bl(t), w.err, st)))
      return rc;
    // dh2 from h_l and h_{l^1}; da from a_l, scaled by 1 / deg_l (the transpose of the variable-major mean)
    cudaError_t e = mp_literal_dx_tc(w.dh, L, w.wb + off_wl(t), w.linv, w.dh2, w.da, w.err, st);
    if (e != cudaSuccess) return cuda_fail(e, "mpnn literal-layer input gradient");
    // a = mean over owning clauses of e  ->  de, masked by the clause layer's ReLU (e = relu(Wc m + bc))
    const int gpw = mp_cgather_gpw(C);
    k_mp_clause_gather<1><<<mp_cgather_grid(C, gpw), 256, 0, st>>>(pd, w.da, nullptr, w.e[t], w.de, gpw);
    if ((rc = wgrad(1, DIn{w.m[t], kH, 0}, none, none, w.de, C, w.part, grad + off_wc(t), grad + off_bc(t), w.err,
                    st)))
      return rc;
    // dm scaled by 1 / |c| (the transpose of the clause-major mean)
    if ((e = mp_dx_tc(w.de, C, w.wb + off_wc(t), w.cinv, w.dm, w.err, st)) != cudaSuccess)
      return cuda_fail(e, "mpnn clause-layer input gradient");
    // m = mean of h over the clause's literals -> dh2 += ..., then masked by the ReLU that produced h[t]
    k_mp_var_gather<1><<<grid_for((int64_t)p->V * 32, 256), 256, 0, st>>>(pd, w.dm, nullptr, w.h[t], w.dh2);
    TSAT_LAUNCH_CHECK("mpnn layer backward");
    std::swap(w.dh, w.dh2);
  }
  // input layer (dh is masked by its ReLU already)
  if ((rc = wgrad(1, DIn{w.feat, kFeat, 0}, none, none, w.dh, L, w.part, grad + kOffW0, grad + kOffB0, w.err, st)))
    return rc;
  return TSAT_OK;
}

}  // namespace tsat

using namespace tsat;

extern "C" {

int32_t tsat_mpnn_param_count(void) { return kNParams; }

int tsat_mpnn_workspace_bytes(const tsat_problem *p, size_t *bytes) {
  if (!p || !bytes) return TSAT_EINVAL;
  *bytes = mp_ws_bytes(p->V, p->C);
  return TSAT_OK;
}

int tsat_mpnn_init(float *d_params, uint64_t seed, cudaStream_t stream) {
  if (!d_params) return TSAT_EINVAL;
  k_mp_init<<<(kNParams + 255) / 256, 256, 0, stream>>>(d_params, (uint32_t)seed, (uint32_t)(seed >> 32));
  TSAT_LAUNCH_CHECK("mpnn init");
  return TSAT_OK;
}

// The forward's launch sequence (about 18 launches) captured into a CUDA
// graph on the problem's private stream, for these pointers; the values behind
// them (the parameters, the workspace) are read when the graph runs.
static int mp_capture_forward(const tsat_problem *p, const float *params, MpWs &w, void *ws, float *logits) {
  tsat_problem::MpForwardGraph &gc = p->mp_fwd;
  TSAT_CUDA(mp_prepare_forward());
  if (!gc.capture) TSAT_CUDA(cudaStreamCreateWithFlags(&gc.capture, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  TSAT_CUDA(cudaStreamBeginCapture(gc.capture, cudaStreamCaptureModeThreadLocal));
  const int rc = mp_forward(p, params, w, logits, gc.capture);
  const cudaError_t ec = cudaStreamEndCapture(gc.capture, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (ec != cudaSuccess) return cuda_fail(ec, "mpnn forward capture");
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return cuda_fail(ei, "mpnn forward graph");
  if (gc.exec) cudaGraphExecDestroy(gc.exec);
  gc.exec = exec;
  gc.params = params;
  gc.ws = ws;
  gc.logits = logits;
  return TSAT_OK;
}

int tsat_mpnn_forward(const tsat_problem *p, const float *d_params, void *d_ws, size_t ws_bytes, float *d_logits,
                      cudaStream_t stream) {
  if (!p || !d_params || !d_ws || !d_logits) return TSAT_EINVAL;
  if (ws_bytes < mp_ws_bytes(p->V, p->C)) { set_error("mpnn workspace too small"); return TSAT_EWS; }
  if ((uintptr_t)d_ws & 255u) { set_error("mpnn workspace not 256-byte aligned"); return TSAT_EINVAL; }
  MpWs w = mp_ws_plan(d_ws, p->V, p->C);
  // A small graph's forward is bound by its launches: the second call with
  // the same pointers captures the sequence as a CUDA graph and later ones
  // replay it in one launch; a call with new pointers runs directly (so a
  // caller whose buffers move pays no capture).
  std::lock_guard<std::mutex> lock(p->mp_mu);
  tsat_problem::MpForwardGraph &gc = p->mp_fwd;
  const bool same = gc.params == d_params && gc.ws == d_ws && gc.logits == d_logits;
  if (!same) {
    if (gc.exec) cudaGraphExecDestroy(gc.exec);
    gc.exec = nullptr;
    gc.params = d_params;
    gc.ws = d_ws;
    gc.logits = d_logits;
    return mp_forward(p, d_params, w, d_logits, stream);
  }
  if (!gc.exec) {
    const int rc = mp_capture_forward(p, d_params, w, d_ws, d_logits);
    if (rc) {
      gc.params = gc.ws = gc.logits = nullptr;
      return rc;
    }
  }
  TSAT_CUDA(cudaGraphLaunch(gc.exec, stream));
  return TSAT_OK;
}

int tsat_mpnn_loss_grad(const tsat_problem *p, const float *d_params, void *d_ws, size_t ws_bytes,
                        const uint8_t *d_targets, float *d_logits, float *d_loss, float *d_grad, cudaStream_t stream) {
  if (!p || !d_params || !d_ws || !d_targets || !d_logits || !d_loss || !d_grad) return TSAT_EINVAL;
  if (ws_bytes < mp_ws_bytes(p->V, p->C)) { set_error("mpnn workspace too small"); return TSAT_EWS; }
  if ((uintptr_t)d_ws & 255u) { set_error("mpnn workspace not 256-byte aligned"); return TSAT_EINVAL; }
  MpWs w = mp_ws_plan(d_ws, p->V, p->C);
  int rc = mp_forward(p, d_params, w, d_logits, stream);
  if (rc) return rc;
  k_mp_bce<<<grid_for(p->V, 256), 256, 0, stream>>>(p->dev, d_logits, d_targets, w.lossv, w.dlog);
  k_mp_sum<<<1, 1024, 0, stream>>>(w.lossv, p->V, d_loss);
  TSAT_LAUNCH_CHECK("mpnn loss");
  return mp_backward(p, w, w.dlog, d_grad, stream);
}

int tsat_mpnn_status(const tsat_problem *p, const void *d_ws, size_t ws_bytes, cudaStream_t stream) {
  if (!p || !d_ws) return TSAT_EINVAL;
  if (ws_bytes < mp_ws_bytes(p->V, p->C)) { set_error("mpnn workspace too small"); return TSAT_EWS; }
  if ((uintptr_t)d_ws & 255u) { set_error("mpnn workspace not 256-byte aligned"); return TSAT_EINVAL; }
  const MpWs w = mp_ws_plan(const_cast<void *>(d_ws), p->V, p->C);
  int flag = 0;
  TSAT_CUDA(cudaMemcpyAsync(&flag, w.err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  TSAT_CUDA(cudaStreamSynchronize(stream));
  if (flag) {
    set_error("a tensor-core layer of the proposer gave up waiting for its MMAs; its outputs are not valid");
    return TSAT_ETIMEOUT;
  }
  return TSAT_OK;
}
int tsat_mpnn_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int64_t step, float lr,
                   cudaStream_t stream) {
  if (!d_params || !d_grad || !d_m || !d_v || step < 1) return TSAT_EINVAL;
  const float bc1 = (float)(1.0 - std::pow(0.9, (double)step)), bc2 = (float)(1.0 - std::pow(0.999, (double)step));
  k_mp_adam<<<(kNParams + 255) / 256, 256, 0, stream>>>(d_params, d_grad, d_m, d_v, kNParams, lr, 0.9f, 0.999f,
                                                       1e-8f, bc1, bc2);
  TSAT_LAUNCH_CHECK("mpnn adam");
  return TSAT_OK;
}

}  // extern "C"
