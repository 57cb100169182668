/*
 * oracle.c -- plain FP64 CPU oracle for the gradient-guided SAT method
 * (TurboSAT, arXiv 2511.07737, Sections III and IV-A).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * Every function follows the paper's definitions in the paper's order:
 *   Eq. 1   R = P A                       (Sec. III-A, "Result Matrix")
 *   Eq. 2   A = B(A_real) = clip(sign,0,1) (Sec. III-B)
 *   Eq. 3   L = -sum_i S_i                (Sec. III-B)
 *   Eq. 4   S_i = SmoothMin(R_i)          (Sec. III-B)
 *   STE     identity gradient through B   (Sec. III-B, Fig. 3)
 *   Eq. 5   per-variable normalisation    (Sec. IV-A)
 *   AdamW + step-decay / restart schedule (Sec. IV-A)
 *   top-k confidence extraction           (Sec. IV-B)
 *
 * Readings of points the paper leaves open (all are parameters here):
 *   - one trainable row per variable; the negated literal row is the
 *     complement (Sec. III-A: assignments are complete, x' = not x);
 *   - normalisation modes: 0 = divide by the signed row mean (Eq. 5 as
 *     printed), 1 = divide by the mean absolute value, 2 = none; a mean
 *     with magnitude below 1e-12 is replaced by +-1e-12 (0 -> +1e-12);
 *   - B(0) = 0 (Eq. 2: non-positive values map to 0);
 *   - AdamW uses PyTorch semantics (decoupled decay, bias correction with
 *     the 1-based step count); a restart resets only the learning rate;
 *   - lr(t) = max(lr0 * f^floor((t mod restart)/period), floor), t 0-based;
 *   - the stochastic binarisation draws u from Philox4x32-10 (Salmon et al.,
 *     SC'11) and sets x = [u < clamp(1/2 + c*zt, 0, 1)], decided in FP32;
 *   - the random-normal init is an Irwin-Hall sum of twelve 24-bit Philox
 *     uniforms, built from integers so both sides get identical FP32 values.
 *
 * Parity pins (tests/): brute force over all assignments of tiny formulas,
 * a dense integer matmul for R, the Fig. 2 fragments, closed forms and
 * limits of SmoothMin, central finite differences of the gradient,
 * torch.optim.AdamW in FP64, and published Philox4x32-10 answer vectors.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no fast-math;
 * FP32 decisions below rely on IEEE single rounding without contraction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_EVAR -2
#define ORC_EEMPTY -3
#define ORC_ENOMEM -7

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* CNF -> problem matrix P (Sec. III-A, "Problem Matrix").             */
/* P is 0/1, so a literal repeated inside a clause is kept once.       */
/* A clause holding both x and x' is kept (it is always satisfied).    */
/* An empty clause cannot be satisfied and is rejected.                */
/* Output: per clause the list of (variable, negated) pairs, order of  */
/* first appearance.                                                   */
/* ------------------------------------------------------------------ */
int orc_parse(int32_t V, int32_t C, const int64_t *cptr, const int32_t *lits,
              int64_t *ocptr, int32_t *ovar, uint8_t *oneg) {
  if (V <= 0 || C <= 0 || !cptr || !lits) return ORC_EINVAL;
  int64_t out = 0;
  ocptr[0] = 0;
  for (int32_t c = 0; c < C; ++c) {
    int64_t b = cptr[c], e = cptr[c + 1];
    if (e < b) return ORC_EINVAL;
    if (e == b) return ORC_EEMPTY;
    int64_t start = out;
    for (int64_t j = b; j < e; ++j) {
      int32_t L = lits[j];
      if (L == 0 || L > V || L < -V) return ORC_EVAR;
      int32_t v = (L > 0 ? L : -L) - 1;
      uint8_t n = (L < 0);
      int dup = 0;
      for (int64_t q = start; q < out; ++q)
        if (ovar[q] == v && oneg[q] == n) { dup = 1; break; }
      if (!dup) { ovar[out] = v; oneg[out] = n; ++out; }
    }
    ocptr[c + 1] = out;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Exact satisfaction check (Sec. III-A, "Satisfiability Matrix"):     */
/* a clause is satisfied by an assignment iff one of its literals is   */
/* true; sample i satisfies the formula iff every clause is satisfied. */
/* X is V x N (row = variable), values 0/1.                            */
/* unsat[i] = number of clauses sample i leaves unsatisfied.           */
/* satmask bit i of word i/32 = sample i satisfies every clause.       */
/* ------------------------------------------------------------------ */
void orc_check(int32_t V, int32_t C, const int64_t *cptr, const int32_t *var,
               const uint8_t *neg, int32_t N, const uint8_t *X, int32_t *unsat,
               uint32_t *satmask) {
  (void)V;
#pragma omp parallel for schedule(static)
  for (int32_t i = 0; i < N; ++i) {
    int32_t cnt = 0;
    for (int32_t c = 0; c < C; ++c) {
      int sat = 0;
      for (int64_t j = cptr[c]; j < cptr[c + 1]; ++j) {
        uint8_t x = X[(int64_t)var[j] * N + i];
        if ((neg[j] ? !x : x)) { sat = 1; break; }
      }
      if (!sat) ++cnt;
    }
    unsat[i] = cnt;
  }
  if (satmask) {
    for (int32_t w = 0; w < (N + 31) / 32; ++w) satmask[w] = 0;
    for (int32_t i = 0; i < N; ++i)
      if (unsat[i] == 0) satmask[i / 32] |= (1u << (i % 32));
  }
}

/* Eq. 1: R = P A.  A has one row per literal; the row of x_v is X_v and
 * the row of x_v' is 1 - X_v (complete assignments, Sec. III-A).        */
void orc_result_matrix(int32_t V, int32_t C, const int64_t *cptr,
                       const int32_t *var, const uint8_t *neg, int32_t N,
                       const uint8_t *X, int32_t *R) {
  (void)V;
#pragma omp parallel for schedule(static)
  for (int32_t c = 0; c < C; ++c) {
    for (int32_t i = 0; i < N; ++i) {
      int32_t r = 0;
      for (int64_t j = cptr[c]; j < cptr[c + 1]; ++j) {
        int32_t a = X[(int64_t)var[j] * N + i];
        r += neg[j] ? 1 - a : a;
      }
      R[(int64_t)c * N + i] = r;
    }
  }
}

/* Eq. 4 on one column r[0..C) and its derivative dS/dR_j.
 * S = sum_j r_j w_j / sum_j w_j with w_j = exp(-tau r_j).
 * dS/dr_j = (w_j / Z) (1 - tau (r_j - S)).                              */
static double smoothmin_col(int32_t C, const double *r, double tau,
                            double *dSdr) {
  double Z = 0.0, Y = 0.0;
  for (int32_t j = 0; j < C; ++j) {
    double w = exp(-tau * r[j]);
    Z += w;
    Y += r[j] * w;
  }
  double S = Y / Z;
  if (dSdr)
    for (int32_t j = 0; j < C; ++j) {
      double w = exp(-tau * r[j]);
      dSdr[j] = (w / Z) * (1.0 - tau * (r[j] - S));
    }
  return S;
}

/* SmoothMin over the columns of a C x N real matrix (Eq. 4).  dSdR may be
 * NULL.  Used directly by the tests for closed forms and limits.          */
void orc_smoothmin(int32_t C, int32_t N, const double *R, double tau,
                   double *S, double *dSdR) {
#pragma omp parallel
  {
    double *col = (double *)malloc(sizeof(double) * (size_t)C);
    double *dcol = dSdR ? (double *)malloc(sizeof(double) * (size_t)C) : NULL;
#pragma omp for schedule(static)
    for (int32_t i = 0; i < N; ++i) {
      for (int32_t j = 0; j < C; ++j) col[j] = R[(int64_t)j * N + i];
      S[i] = smoothmin_col(C, col, tau, dcol);
      if (dSdR)
        for (int32_t j = 0; j < C; ++j) dSdR[(int64_t)j * N + i] = dcol[j];
    }
    free(col);
    free(dcol);
  }
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* ------------------------------------------------------------------ */
/* Objective and its gradient with respect to the normalised assignment */
/* zt (one row per variable).                                          */
/*                                                                     */
/* relaxed == 0 (the paper's layer, Fig. 3): literal values are the     */
/*   binary X (already binarised, Eq. 2); the backward pass uses the    */
/*   straight-through estimator, so dA_x/dzt = +1 and dA_x'/dzt = -1.   */
/* relaxed == 1: literal values are a = sigmoid(zt) and 1 - a, so R is  */
/*   real and the chain rule carries sigmoid' = a (1 - a).              */
/*                                                                     */
/* Per sample i: R_ci (Eq. 1), S_i (Eq. 4), L = -sum S_i (Eq. 3),       */
/* dL/dR_ci = -dS_i/dR_ci, then G = D P^T dL/dR (D = +1 / -1 on the     */
/* positive / negated literal of each variable).                       */
/* Outputs: S[N], *L, G[V*N] (nullable), unsat[N] (STE only, nullable). */
/* ------------------------------------------------------------------ */
int orc_objective(int32_t V, int32_t C, const int64_t *cptr,
                  const int32_t *var, const uint8_t *neg, int32_t N,
                  int32_t relaxed, const uint8_t *X, const double *zt,
                  double tau, double *S, double *L, double *G,
                  int32_t *unsat) {
  if (relaxed ? !zt : !X) return ORC_EINVAL;
  if (G) memset(G, 0, sizeof(double) * (size_t)V * (size_t)N);
  int fail = 0;
#pragma omp parallel
  {
    double *r = (double *)malloc(sizeof(double) * (size_t)C);
    double *d = (double *)malloc(sizeof(double) * (size_t)C);
    if (!r || !d) {
#pragma omp atomic write
      fail = 1;
    }
#pragma omp for schedule(static)
    for (int32_t i = 0; i < N; ++i) {
      if (!r || !d) continue;
      int32_t nz = 0;
      /* Eq. 1, column i */
      for (int32_t c = 0; c < C; ++c) {
        double s = 0.0;
        for (int64_t j = cptr[c]; j < cptr[c + 1]; ++j) {
          int64_t vi = (int64_t)var[j] * N + i;
          double a = relaxed ? sigmoid(zt[vi]) : (double)X[vi];
          s += neg[j] ? 1.0 - a : a;
        }
        r[c] = s;
        if (s == 0.0) ++nz;
      }
      /* Eq. 4 and its derivative */
      S[i] = smoothmin_col(C, r, tau, d);
      if (unsat && !relaxed) unsat[i] = nz;
      if (!G) continue;
      /* dL/dR = -dS/dR (Eq. 3); P^T scatter with the literal sign */
      for (int32_t c = 0; c < C; ++c) {
        double gR = -d[c];
        for (int64_t j = cptr[c]; j < cptr[c + 1]; ++j) {
          int64_t vi = (int64_t)var[j] * N + i;
          double dadz = 1.0; /* straight-through estimator */
          if (relaxed) {
            double a = sigmoid(zt[vi]);
            dadz = a * (1.0 - a);
          }
          G[vi] += (neg[j] ? -1.0 : 1.0) * dadz * gR;
        }
      }
    }
    free(r);
    free(d);
  }
  if (fail) return ORC_ENOMEM;
  double sum = 0.0;
  for (int32_t i = 0; i < N; ++i) sum += S[i];
  *L = -sum; /* Eq. 3 */
  return ORC_OK;
}

/* Guard for the normaliser: magnitudes below 1e-12 become +-1e-12. */
static double guard_nu(double mu) {
  const double g = 1e-12;
  if (fabs(mu) < g) return (mu < 0.0) ? -g : g;
  return mu;
}

/* Eq. 5: nu_v = (1/N) sum_i z_vi (mode 0), or (1/N) sum_i |z_vi| (mode 1),
 * or 1 (mode 2); zt = z / nu.  zt may be NULL.                          */
void orc_normalize(int32_t V, int32_t N, const double *z, int32_t mode,
                   double *nu, double *zt) {
#pragma omp parallel for schedule(static)
  for (int32_t v = 0; v < V; ++v) {
    const double *row = z + (int64_t)v * N;
    double s = 0.0;
    if (mode == 2) {
      s = 1.0;
    } else {
      for (int32_t i = 0; i < N; ++i) s += (mode == 1) ? fabs(row[i]) : row[i];
      s = guard_nu(s / (double)N);
    }
    nu[v] = s;
    if (zt)
      for (int32_t i = 0; i < N; ++i) zt[(int64_t)v * N + i] = row[i] / s;
  }
}

/* Chain rule through Eq. 5.  G = dL/dzt, output g = dL/dz.
 * mode 0: zt_k = z_k / mu, mu = mean(z):
 *         g_i = G_i / mu - (sum_k G_k z_k) / (N mu^2)
 * mode 1: zt_k = z_k / a, a = mean|z|:
 *         g_i = G_i / a - (sum_k G_k z_k) sign(z_i) / (N a^2)
 * mode 2: g = G.
 * nu is the (guarded) normaliser used in the forward pass.             */
void orc_normalize_backward(int32_t V, int32_t N, const double *z,
                            const double *nu, const double *G, int32_t mode,
                            double *g) {
#pragma omp parallel for schedule(static)
  for (int32_t v = 0; v < V; ++v) {
    const double *zr = z + (int64_t)v * N;
    const double *Gr = G + (int64_t)v * N;
    double *gr = g + (int64_t)v * N;
    if (mode == 2) {
      for (int32_t i = 0; i < N; ++i) gr[i] = Gr[i];
      continue;
    }
    double s = nu[v];
    double dot = 0.0;
    for (int32_t k = 0; k < N; ++k) dot += Gr[k] * zr[k];
    for (int32_t i = 0; i < N; ++i) {
      double dmu = (mode == 1) ? ((zr[i] > 0.0) - (zr[i] < 0.0)) : 1.0;
      gr[i] = Gr[i] / s - dot * dmu / ((double)N * s * s);
    }
  }
}

/* Learning-rate schedule (Sec. IV-A): start at lr0, divide by 1/f every
 * `period` iterations, go back to lr0 every `restart` iterations, never
 * below lr_floor.  t is the 0-based iteration.                          */
double orc_lr(int64_t t, double lr0, double f, int32_t period,
              int32_t restart, double lr_floor) {
  int64_t tt = (restart > 0) ? (t % restart) : t;
  int64_t k = (period > 0) ? (tt / period) : 0;
  double lr = lr0 * pow(f, (double)k);
  return lr > lr_floor ? lr : lr_floor;
}

/* AdamW (Loshchilov & Hutter) with PyTorch's formulation:
 *   z <- z (1 - lr wd)
 *   m <- b1 m + (1 - b1) g ;  v <- b2 v + (1 - b2) g^2
 *   z <- z - lr/(1 - b1^s) * m / (sqrt(v)/sqrt(1 - b2^s) + eps)
 * s is the 1-based step count.                                           */
void orc_adamw(int64_t n, double *z, double *m, double *v, const double *g,
               int64_t s, double lr, double b1, double b2, double eps,
               double wd) {
  double bc1 = 1.0 - pow(b1, (double)s);
  double bc2 = 1.0 - pow(b2, (double)s);
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    z[j] *= 1.0 - lr * wd;
    m[j] = b1 * m[j] + (1.0 - b1) * g[j];
    v[j] = b2 * v[j] + (1.0 - b2) * g[j] * g[j];
    double denom = sqrt(v[j]) / sqrt(bc2) + eps;
    z[j] -= (lr / bc1) * m[j] / denom;
  }
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,   */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of */
/* two 32x32->64 multiplies and a Weyl-sequence key schedule.           */
/* ------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
  uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n1 = lo1;
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  uint32_t n3 = lo0;
  c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
    philox_round(c, k);
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Counter layout (both sides use this definition):
 *   key     = (seed low 32 bits, seed high 32 bits)
 *   init    : counter = (i, v, j, 0x494E4954) for j = 0,1,2  -> 12 words
 *   binarize: counter = (i / 8, v, t, 0x42494E41); sample i takes the
 *             16-bit half i mod 8 (word (i mod 8) / 2, low half first)  */
#define ORC_TAG_INIT 0x494E4954u
#define ORC_TAG_BIN 0x42494E41u

/* Random-normal init (Sec. IV-A): Irwin-Hall sum of twelve 24-bit
 * uniforms, sum - 6*2^24 converted to float and scaled by 2^-24.  Mean 0,
 * variance 1, support (-6, 6).  With logits != NULL the row is shifted:
 * z = logit_v * scale + noise, in FP32 without contraction.             */
void orc_init_normal(int32_t V, int32_t N, uint64_t seed, const float *logits,
                     float scale, float *z) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
  for (int32_t v = 0; v < V; ++v) {
    for (int32_t i = 0; i < N; ++i) {
      int32_t acc = 0;
      for (uint32_t j = 0; j < 3; ++j) {
        uint32_t ctr[4] = {(uint32_t)i, (uint32_t)v, j, ORC_TAG_INIT}, o[4];
        orc_philox4x32_10(ctr, key, o);
        for (int q = 0; q < 4; ++q) acc += (int32_t)(o[q] >> 8);
      }
      int32_t centred = acc - 6 * (1 << 24);
      float noise = (float)centred * (1.0f / 16777216.0f);
      float val = noise;
      if (logits) {
        float sh = logits[v] * scale;
        val = sh + noise;
      }
      z[(int64_t)v * N + i] = val;
    }
  }
}

/* FP32 normaliser of FP32 rows, summed in FP64 and rounded once; used to
 * state what the GPU's FP32 statistic approximates.                      */
void orc_nu_f32(int32_t V, int32_t N, const float *z, int32_t mode,
                double *nu) {
#pragma omp parallel for schedule(static)
  for (int32_t v = 0; v < V; ++v) {
    double s = 0.0;
    if (mode == 2) { nu[v] = 1.0; continue; }
    for (int32_t i = 0; i < N; ++i) {
      double x = (double)z[(int64_t)v * N + i];
      s += (mode == 1) ? fabs(x) : x;
    }
    nu[v] = guard_nu(s / (double)N);
  }
}

/* Eq. 2 decided in FP32 from FP32 inputs z and nu (the GPU's precision).
 * The normalised value zt of Eq. 5 is evaluated as z * (1/nu): an FP32
 * reciprocal and an FP32 product, each correctly rounded.
 * mode 0 (deterministic): x = [zt > 0].
 * mode 1 (Philox): p = clamp(0.5 + c * (z/nu), 0, 1) with one FP32
 * multiply and one FP32 add (no fused multiply-add), u = half 2^-16 with
 * half the 16-bit Philox output of the sample (counter layout above),
 * x = [u < p].  t is the step the bits belong to.                         */
void orc_binarize_f32(int32_t V, int32_t N, const float *z, const float *nu,
                      int32_t mode, float c, uint64_t seed, int64_t t,
                      uint8_t *X) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
  for (int32_t v = 0; v < V; ++v) {
    volatile float rnu = 1.0f / nu[v];
    for (int32_t i = 0; i < N; ++i) {
      volatile float zt = z[(int64_t)v * N + i] * rnu;
      uint8_t x;
      if (mode == 0) {
        x = (zt > 0.0f);
      } else {
        uint32_t ctr[4] = {(uint32_t)(i / 8), (uint32_t)v, (uint32_t)t,
                           ORC_TAG_BIN},
                 o[4];
        orc_philox4x32_10(ctr, key, o);
        uint32_t half = (o[(i % 8) / 2] >> (16 * (i % 2))) & 0xFFFFu;
        float u = (float)half * (1.0f / 65536.0f);
        volatile float prod = c * zt;
        volatile float p = 0.5f + prod;
        if (p < 0.0f) p = 0.0f;
        if (p > 1.0f) p = 1.0f;
        x = (u < p);
      }
      X[(int64_t)v * N + i] = x;
    }
  }
}

/* ------------------------------------------------------------------ */
/* One optimisation step (Sec. IV-A), in FP64:                          */
/*   nu_t from z (or taken from nu_in), zt = z/nu_t                     */
/*   objective and gradient at the given assignments (X for the STE     */
/*   layer, sigmoid(zt) for the relaxed layer)                          */
/*   chain rule through Eq. 5, AdamW with lr(t), step count s = t + 1   */
/*   (with mix: at t = k R, k >= 1, assignment mixing instead, and the  */
/*   step count restarts: s = t mod R after the first restart)          */
/*   nu_{t+1} from the updated z.                                       */
/* z, m, v are updated in place.  Outputs: S[N], *L, G[V*N] (nullable), */
/* g[V*N] (nullable), nu_next[V] (nullable), unsat[N] (nullable).       */
/* ------------------------------------------------------------------ */
typedef struct {
  double tau, lr0, lr_factor, lr_floor;
  int32_t decay_period, restart_period;
  double beta1, beta2, eps, weight_decay;
  int32_t norm;
  int32_t relaxed;
  int32_t mix;      /* assignment mixing at each lr restart (see orc_step) */
  int32_t pad;
} orc_hparams;

int orc_step(int32_t V, int32_t C, const int64_t *cptr, const int32_t *var,
             const uint8_t *neg, int32_t N, const orc_hparams *hp, int64_t t,
             double *z, double *m, double *v, const uint8_t *X,
             const double *nu_in, double *S, double *L, double *G_out,
             double *g_out, double *nu_next, int32_t *unsat) {
  size_t n = (size_t)V * (size_t)N;
  double *nu = (double *)malloc(sizeof(double) * (size_t)V);
  double *zt = (double *)malloc(sizeof(double) * n);
  double *G = G_out ? G_out : (double *)malloc(sizeof(double) * n);
  double *g = g_out ? g_out : (double *)malloc(sizeof(double) * n);
  if (!nu || !zt || !G || !g) return ORC_ENOMEM;
  orc_normalize(V, N, z, hp->norm, nu, zt);
  if (nu_in) {
    for (int32_t r = 0; r < V; ++r) nu[r] = nu_in[r];
    for (int32_t r = 0; r < V; ++r)
      for (int32_t i = 0; i < N; ++i)
        zt[(int64_t)r * N + i] = z[(int64_t)r * N + i] / nu[r];
  }
  int32_t *us = unsat ? unsat : (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  if (!us) return ORC_ENOMEM;
  int rc = orc_objective(V, C, cptr, var, neg, N, hp->relaxed, X, zt, hp->tau,
                         S, L, G, us);
  const int32_t R = hp->restart_period;
  if (rc == ORC_OK && hp->mix && R > 0 && t > 0 && t % R == 0) {
    /* assignment mixing at an lr restart (the paper's commented-out variant):
     * the sample with the most satisfied clauses, i*, is kept; every other
     * sample becomes the mean of itself and i*; the optimizer is reset.  No
     * gradient step is taken at this step. */
    int32_t best = 0;
    for (int32_t i = 1; i < N; ++i)
      if (us[i] < us[best]) best = i;
    for (int32_t r = 0; r < V; ++r)
      for (int32_t i = 0; i < N; ++i) {
        int64_t k = (int64_t)r * N + i;
        if (i != best) z[k] = 0.5 * (z[k] + z[(int64_t)r * N + best]);
        m[k] = 0.0;
        v[k] = 0.0;
      }
    for (size_t k = 0; k < n; ++k) g[k] = 0.0;
    if (nu_next) orc_normalize(V, N, z, hp->norm, nu_next, NULL);
  } else if (rc == ORC_OK) {
    orc_normalize_backward(V, N, z, nu, G, hp->norm, g);
    double lr = orc_lr(t, hp->lr0, hp->lr_factor, hp->decay_period,
                       hp->restart_period, hp->lr_floor);
    /* AdamW step count: global, or counted from the last mixing restart */
    int64_t cnt = (hp->mix && R > 0 && t >= R) ? t % R : t + 1;
    orc_adamw((int64_t)n, z, m, v, g, cnt, lr, hp->beta1, hp->beta2,
              hp->eps, hp->weight_decay);
    if (nu_next) orc_normalize(V, N, z, hp->norm, nu_next, NULL);
  }
  if (!unsat) free(us);
  free(nu);
  free(zt);
  if (!G_out) free(G);
  if (!g_out) free(g);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Hand-off selection (Sec. IV-B).                                     */
/* Sample ranking: fewer unsatisfied clauses first, ties to the lower   */
/* index.  A complete satisfying sample is one with unsat = 0.          */
/* Confidence: smaller |G_vi| means more confident; the k most          */
/* confident variables of the chosen sample, ties to the lower index,   */
/* k = max(20, ceil(1e-4 V)) capped at V (0.01 % of V, at least 20).    */
/* ------------------------------------------------------------------ */
int32_t orc_best_sample(int32_t N, const int32_t *unsat) {
  int32_t b = 0;
  for (int32_t i = 1; i < N; ++i)
    if (unsat[i] < unsat[b]) b = i;
  return b;
}

int32_t orc_partial_k(int32_t V) {
  int64_t k = ((int64_t)V + 9999) / 10000;
  if (k < 20) k = 20;
  if (k > V) k = V;
  return (int32_t)k;
}

/* Selection by repeated minimum: plain and slow on purpose. */
void orc_topk_confident(int32_t V, const double *absG, int32_t k,
                        int32_t *out_var) {
  uint8_t *taken = (uint8_t *)calloc((size_t)V, 1);
  for (int32_t s = 0; s < k; ++s) {
    int32_t b = -1;
    for (int32_t v = 0; v < V; ++v) {
      if (taken[v]) continue;
      if (b < 0 || absG[v] < absG[b]) b = v;
    }
    taken[b] = 1;
    out_var[s] = b;
  }
  free(taken);
}
