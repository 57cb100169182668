// layout.cu -- device build of the problem matrix P (Sec. III-A) in the two
// compressed sparse forms the step uses (Sec. IV-A: "compressed sparse format"
// in both passes):
//   * clause-major CSR (cptr, clit), literal = (global var << 1) | negated,
//     duplicate literals removed because P is 0/1;
//   * variable-major occurrence records (xptr, xrec): for every occurrence of
//     variable v, in clause order, a header (own negation | len << 1)
//     followed by the other literals of that clause.  The backward pass
//     (P^T, Fig. 3) re-forms each R_ci from these without global atomics.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace tsat {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return TSAT_ECUDA;
}

constexpr int kMaxRawLen = 64;
constexpr int kScanTile = 2048;  // elements per scan block (256 threads x 8)

// ------------------------------------------------------------------ scans
__global__ void k_scan_reduce(const int32_t *in, int64_t n, int32_t round4, int64_t *bsum) {
  __shared__ int64_t sh[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t s = 0;
  for (int k = 0; k < 8; ++k) {
    int64_t i = base + threadIdx.x * 8 + k;
    if (i < n) {
      int64_t x = in[i];
      s += round4 ? ((x + 3) & ~int64_t(3)) : x;
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    bsum[blockIdx.x] = t;
  }
}

// single block: exclusive scan of the block sums, in place
__global__ void k_scan_blocks(int64_t *bsum, int64_t nb) {
  __shared__ int64_t sh[1024];
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
    int64_t i = b0 + threadIdx.x;
    int64_t x = i < nb ? bsum[i] : 0;
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int64_t y = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += y;
      __syncthreads();
    }
    int64_t incl = sh[threadIdx.x];
    if (i < nb) bsum[i] = carry + incl - x;
    __syncthreads();
    carry += sh[1023];
    __syncthreads();
  }
}

// out[i] = exclusive prefix (int64), out[n] = total; out32 optional int32 copy
__global__ void k_scan_final(const int32_t *in, int64_t n, int32_t round4, const int64_t *boff,
                             int64_t *out64, int32_t *out32) {
  __shared__ int64_t sh[256];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t v[8];
  int64_t s = 0;
  for (int k = 0; k < 8; ++k) {
    int64_t i = base + threadIdx.x * 8 + k;
    int64_t x = 0;
    if (i < n) {
      x = in[i];
      if (round4) x = (x + 3) & ~int64_t(3);
    }
    v[k] = x;
    s += x;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    int64_t y = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += y;
    __syncthreads();
  }
  int64_t run = boff[blockIdx.x] + sh[threadIdx.x] - s;
  for (int k = 0; k < 8; ++k) {
    int64_t i = base + threadIdx.x * 8 + k;
    if (i < n) {
      if (out64) out64[i] = run;
      if (out32) out32[i] = (int32_t)run;
    }
    run += v[k];
    if (i == n - 1) {
      if (out64) out64[n] = run;
      if (out32) out32[n] = (int32_t)run;
    }
  }
}

static int exclusive_scan(const int32_t *in, int64_t n, bool round4, int64_t *bsum, int64_t *out64,
                          int32_t *out32, cudaStream_t st) {
  if (n <= 0) return TSAT_OK;
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  k_scan_reduce<<<(unsigned)nb, 256, 0, st>>>(in, n, round4, bsum);
  k_scan_blocks<<<1, 1024, 0, st>>>(bsum, nb);
  k_scan_final<<<(unsigned)nb, 256, 0, st>>>(in, n, round4, bsum, out64, out32);
  TSAT_LAUNCH_CHECK("exclusive_scan");
  return TSAT_OK;
}

// ------------------------------------------------------------------ build kernels
__device__ __forceinline__ int find_inst_by_clause(const InstInfo *inst, int n_inst, int64_t c) {
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (inst[mid].c_off <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int find_inst_by_var(const InstInfo *inst, int n_inst, int64_t v) {
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (inst[mid].v_off <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// error word: smallest (clause << 8 | code); codes 1 EVAR, 2 EEMPTY, 3 ELEN
__device__ __forceinline__ void report(unsigned long long *err, int64_t c, int code) {
  atomicMin(err, ((unsigned long long)c << 8) | (unsigned long long)code);
}

__global__ void k_dedup(const int64_t *raw_cptr, const int32_t *raw_lits, int32_t C,
                        InstInfo *inst, int32_t n_inst, int32_t *tmp, int32_t *clen,
                        unsigned long long *err) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  int ii = find_inst_by_clause(inst, n_inst, c);
  const int32_t v_off = inst[ii].v_off, nv = inst[ii].n_vars;
  int64_t b = raw_cptr[c], e = raw_cptr[c + 1];
  int64_t len = e - b;
  if (len == 0) { report(err, c, 2); clen[c] = 0; return; }
  if (len > kMaxRawLen) { report(err, c, 3); clen[c] = 0; return; }
  int32_t buf[kMaxRawLen];
  int n = 0;
  for (int64_t j = b; j < e; ++j) {
    int32_t L = raw_lits[j];
    if (L == 0 || L > nv || L < -nv) { report(err, c, 1); clen[c] = 0; return; }
    int32_t code = ((v_off + (L > 0 ? L : -L) - 1) << 1) | (L < 0 ? 1 : 0);
    // insertion into the sorted buffer, skipping duplicates
    int p = n;
    bool dup = false;
    while (p > 0 && buf[p - 1] >= code) {
      if (buf[p - 1] == code) { dup = true; break; }
      --p;
    }
    if (dup) continue;
    for (int q = n; q > p; --q) buf[q] = buf[q - 1];
    buf[p] = code;
    ++n;
  }
  if (n > TSAT_MAX_CLAUSE_LEN) { report(err, c, 3); clen[c] = 0; return; }
  for (int q = 0; q < n; ++q) tmp[b + q] = buf[q];
  clen[c] = n;
  atomicMax(&inst[ii].lmax, n);
}

__global__ void k_compact_count(const int64_t *raw_cptr, const int32_t *tmp, const int32_t *clen,
                                const int32_t *cptr, int32_t C, int32_t *clit, int32_t *deg,
                                int32_t *recsz) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  int64_t b = raw_cptr[c];
  int32_t o = cptr[c], n = clen[c];
  for (int q = 0; q < n; ++q) {
    int32_t lit = tmp[b + q];
    clit[o + q] = lit;
    atomicAdd(&deg[lit >> 1], 1);
    atomicAdd(&recsz[lit >> 1], n);
  }
}

// Fixed clause records for clause length <= 3: {var0, var1, var2, flags},
// flags byte u = 0xFF when literal u is negated, byte 3 = the clause length; a
// missing literal repeats var0 with flag byte 0 (the kernels mask it by length).
__global__ void k_crec(const int32_t *cptr, const int32_t *clit, int32_t C, int4 *crec) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const int32_t b = cptr[c], n = cptr[c + 1] - b;
  int32_t v[3];
  uint32_t fl = (uint32_t)n << 24;
  for (int u = 0; u < 3; ++u) {
    const int32_t lit = clit[b + (u < n ? u : 0)];
    v[u] = lit >> 1;
    if (u < n && (lit & 1)) fl |= 0xFFu << (8 * u);
  }
  crec[c] = make_int4(v[0], v[1], v[2], (int32_t)fl);
}

__global__ void k_fill(const int32_t *cptr, const int32_t *clit, int32_t C, const int32_t *vptr,
                       int32_t *fill, int32_t *occ_j, int32_t *occ_c) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  for (int32_t j = cptr[c]; j < cptr[c + 1]; ++j) {
    int32_t v = clit[j] >> 1;
    int32_t slot = atomicAdd(&fill[v], 1);
    occ_j[vptr[v] + slot] = j;
    occ_c[vptr[v] + slot] = (int32_t)c;
  }
}

// Block per variable: order its occurrences by position (deterministic, clause
// order) with rank counting, then write the occurrence records.
__global__ void k_records(const int32_t *cptr, const int32_t *clit, int32_t V, const int32_t *vptr,
                          const int32_t *occ_j, const int32_t *occ_c, int32_t *occ_s,
                          const int64_t *xptr, int32_t *xrec, int32_t *vocc, int stride) {
  __shared__ int32_t sh[128];
  __shared__ int32_t carry;
  const int32_t v = blockIdx.x;
  if (v >= V) return;
  const int32_t b = vptr[v], e = vptr[v + 1], d = e - b;
  for (int32_t a = threadIdx.x; a < d; a += blockDim.x) {
    int32_t key = occ_j[b + a];
    int32_t rank = 0;
    for (int32_t f = 0; f < d; ++f) rank += (occ_j[b + f] < key);
    occ_s[b + rank] = a;  // index into the unordered list
  }
  __syncthreads();
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int64_t base = xptr[v];
  for (int32_t a0 = 0; a0 < d; a0 += blockDim.x) {
    int32_t a = a0 + threadIdx.x;
    int32_t len = 0, j = 0, c = 0;
    if (a < d) {
      int32_t u = occ_s[b + a];
      j = occ_j[b + u];
      c = occ_c[b + u];
      len = cptr[c + 1] - cptr[c];
    }
    sh[threadIdx.x] = len;
    __syncthreads();
    for (int o = 1; o < 128; o <<= 1) {
      int32_t y = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += y;
      __syncthreads();
    }
    int32_t off = carry + sh[threadIdx.x] - len;
    if (a < d) {
      int32_t own = clit[j];
      vocc[b + a] = (c << 1) | (own & 1);
      int32_t *r = xrec + base + (stride ? stride * a : off);
      r[0] = (own & 1) | (len << 1);  // nonzero: padding words are 0
      int q = 1;
      for (int32_t k = cptr[c]; k < cptr[c + 1]; ++k)
        if (k != j) r[q++] = clit[k];
      if (stride)
        for (; q < stride; ++q) r[q] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 127) carry += sh[127];
    __syncthreads();
  }
  // zero the padding
  int64_t used = stride ? xptr[v + 1] : base + carry;
  for (int64_t p = used + threadIdx.x; p < xptr[v + 1]; p += blockDim.x) xrec[p] = 0;
}

__global__ void k_xptr_fixed(const int32_t *vptr, int32_t V, int64_t *xptr, int stride) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v <= V) xptr[v] = stride * (int64_t)vptr[v];
}

__global__ void k_var_inst(const InstInfo *inst, int32_t n_inst, int32_t V, int32_t *var_inst) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < V) var_inst[v] = find_inst_by_var(inst, n_inst, v);
}

// Clause offsets of a batch: each instance's clause pointers were copied as
// given (from 0), and the instance's first literal position in the batch is
// added here, up to kRawChunk instances per launch (their first clauses and
// literal offsets by value).
constexpr int kRawChunk = 64;
struct RawOffChunk {
  int32_t n;              // instances in this chunk
  int64_t coff[kRawChunk + 1];   // first clause of each instance, then the end of the last
  int64_t loff[kRawChunk];
};

__global__ void k_raw_offsets(int64_t *raw_cptr, RawOffChunk ch) {
  const int64_t c = ch.coff[0] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ch.coff[ch.n]) return;
  int lo = 0, hi = ch.n - 1;   // the instance whose clauses hold c
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ch.coff[mid] <= c) lo = mid;
    else hi = mid - 1;
  }
  raw_cptr[c] += ch.loff[lo];
}

// ------------------------------------------------------------------ host side
struct Sizes {
  int32_t n_inst;
  int64_t V, C, nnz_raw, xrec_cap, items_cap, lraw;
};

static int measure(int32_t n_inst, const tsat_cnf_desc *d, Sizes *s) {
  if (n_inst <= 0 || !d) { set_error("n_inst must be positive and descs non-NULL"); return TSAT_EINVAL; }
  s->n_inst = n_inst;
  s->V = s->C = s->nnz_raw = s->xrec_cap = s->items_cap = s->lraw = 0;
  for (int32_t j = 0; j < n_inst; ++j) {
    if (d[j].n_vars <= 0 || d[j].n_clauses <= 0 || !d[j].h_clause_ptr || !d[j].h_lits) {
      set_error("instance %d: empty or NULL arrays", j);
      return TSAT_EINVAL;
    }
    const int64_t *p = d[j].h_clause_ptr;
    if (p[0] != 0) { set_error("instance %d: clause_ptr[0] != 0", j); return TSAT_EINVAL; }
    for (int32_t c = 0; c < d[j].n_clauses; ++c) {
      int64_t len = p[c + 1] - p[c];
      if (len < 0) { set_error("instance %d: clause_ptr decreases at %d", j, c); return TSAT_EINVAL; }
      int64_t eff = std::min<int64_t>(len, TSAT_MAX_CLAUSE_LEN);
      s->xrec_cap += eff * eff;
      s->lraw = std::max<int64_t>(s->lraw, len);
    }
    s->V += d[j].n_vars;
    s->C += d[j].n_clauses;
    s->nnz_raw += p[d[j].n_clauses];
    s->items_cap += (d[j].n_clauses + kItemMin - 1) / kItemMin;
  }
  // fixed records: 4 ints per occurrence up to length 3, 8 up to length 7
  s->xrec_cap = std::max<int64_t>(s->xrec_cap, (s->lraw <= 7 ? 8 : 4) * s->nnz_raw) + 3 * s->V + 8;
  if (s->V >= (1LL << 30) || s->C >= (1LL << 31) - 1 || s->nnz_raw >= (1LL << 31) - 1) {
    set_error("problem too large: V=%lld C=%lld nnz=%lld", (long long)s->V, (long long)s->C,
              (long long)s->nnz_raw);
    return TSAT_EINVAL;
  }
  return TSAT_OK;
}

static Layout plan(const Sizes &s) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
  const int64_t nb = std::max<int64_t>(1, (std::max(s.nnz_raw, std::max(s.V, s.C)) + 1 + kScanTile - 1) / kScanTile);
  L.xrec_cap = s.xrec_cap;
  L.items_cap = s.items_cap;
  L.scan_blocks = nb;
  L.cptr = take(sizeof(int32_t) * (s.C + 1));
  L.clit = take(sizeof(int32_t) * (s.nnz_raw + 1));
  L.xptr = take(sizeof(int64_t) * (s.V + 1));
  L.xrec = take(sizeof(int32_t) * s.xrec_cap);
  L.vptr = take(sizeof(int32_t) * (s.V + 1));
  L.vocc = take(sizeof(int32_t) * (s.nnz_raw + 1));
  L.var_inst = take(sizeof(int32_t) * s.V);
  L.items = take(sizeof(int4) * s.items_cap);
  L.inst = take(sizeof(InstInfo) * s.n_inst);
  L.err = take(64);
  L.crec = s.lraw <= 3 ? take(sizeof(int4) * s.C) : 0;   // fixed clause records (clause length <= 3)
  L.raw_cptr = take(sizeof(int64_t) * (s.C + 1));
  L.raw_lits = take(sizeof(int32_t) * (s.nnz_raw + 1));
  L.tmp = take(sizeof(int32_t) * (s.nnz_raw + 1));
  L.clen = take(sizeof(int32_t) * (s.C + 1));
  L.deg = take(sizeof(int32_t) * (s.V + 1));
  L.recsz = take(sizeof(int32_t) * (s.V + 1));
  L.fill = take(sizeof(int32_t) * (s.V + 1));
  L.occ_j = take(sizeof(int32_t) * (s.nnz_raw + 1));
  L.occ_c = take(sizeof(int32_t) * (s.nnz_raw + 1));
  L.occ_s = take(sizeof(int32_t) * (s.nnz_raw + 1));
  L.scan_tmp = take(sizeof(int64_t) * (nb + 1));
  L.total = o;
  return L;
}

}  // namespace tsat

using namespace tsat;

int tsat_problem::set_items(int32_t ic, cudaStream_t stream) {
  if (ic < kItemMin) ic = kItemMin;
  ic = (ic / kItemMin) * kItemMin;
  std::vector<int4> items;
  for (int32_t j = 0; j < n_inst; ++j) {
    inst[j].item_off = (int32_t)items.size();
    for (int32_t c = 0; c < inst[j].n_clauses; c += ic)
      items.push_back(make_int4(j, inst[j].c_off + c, inst[j].c_off + std::min(c + ic, inst[j].n_clauses), 0));
    inst[j].n_items = (int32_t)items.size() - inst[j].item_off;
  }
  if ((int64_t)items.size() > lay.items_cap) { set_error("work list overflow"); return TSAT_EINVAL; }
  char *w = (char *)ws;
  TSAT_CUDA(cudaMemcpyAsync(w + lay.items, items.data(), sizeof(int4) * items.size(),
                            cudaMemcpyHostToDevice, stream));
  TSAT_CUDA(cudaMemcpyAsync(w + lay.inst, inst.data(), sizeof(InstInfo) * n_inst,
                            cudaMemcpyHostToDevice, stream));
  TSAT_CUDA(cudaStreamSynchronize(stream));
  item_clauses = ic;
  dev.n_items = (int32_t)items.size();
  return TSAT_OK;
}

extern "C" {

const char *tsat_strerror(int s) {
  switch (s) {
    case TSAT_OK: return "ok";
    case TSAT_EINVAL: return "invalid argument";
    case TSAT_EVAR: return "literal is 0 or out of range";
    case TSAT_EEMPTY: return "empty clause (formula unsatisfiable)";
    case TSAT_EWS: return "workspace or state buffer too small";
    case TSAT_ECUDA: return "CUDA error";
    case TSAT_ETIMEOUT: return "device wait timed out";
    case TSAT_ENOMEM: return "host allocation failed";
    case TSAT_ELEN: return "clause longer than TSAT_MAX_CLAUSE_LEN";
    case TSAT_ESTATE: return "state/handle mismatch or not initialised";
    case TSAT_ERANGE: return "index or count out of range";
    default: return "unknown status";
  }
}

const char *tsat_last_error(void) { return g_err; }

int tsat_problem_bytes(int32_t n_inst, const tsat_cnf_desc *descs, size_t *ws_bytes) {
  if (!ws_bytes) { set_error("ws_bytes is NULL"); return TSAT_EINVAL; }
  Sizes s;
  int rc = measure(n_inst, descs, &s);
  if (rc) return rc;
  *ws_bytes = plan(s).total;
  return TSAT_OK;
}

int tsat_load_batch(int32_t n_inst, const tsat_cnf_desc *descs, void *d_ws, size_t ws_bytes,
                    cudaStream_t stream, tsat_problem **out) {
  return tsat_load_batch_ex(n_inst, descs, 0u, d_ws, ws_bytes, stream, out);
}

int tsat_load_batch_ex(int32_t n_inst, const tsat_cnf_desc *descs, uint32_t flags, void *d_ws, size_t ws_bytes,
                       cudaStream_t stream, tsat_problem **out) {
  if (!out || !d_ws) { set_error("NULL output or workspace"); return TSAT_EINVAL; }
  if (flags & ~(uint32_t)TSAT_LOAD_CLAUSE_LOCALITY) { set_error("unknown load flags %#x", flags); return TSAT_EINVAL; }
  const bool locality = (flags & TSAT_LOAD_CLAUSE_LOCALITY) != 0;
  *out = nullptr;
  Sizes s;
  int rc = measure(n_inst, descs, &s);
  if (rc) return rc;
  Layout L = plan(s);
  if (ws_bytes < L.total) {
    set_error("workspace %zu bytes < required %zu", ws_bytes, L.total);
    return TSAT_EWS;
  }
  if (((uintptr_t)d_ws) % 256) { set_error("workspace must be 256-byte aligned"); return TSAT_EINVAL; }
  tsat_problem *p = new (std::nothrow) tsat_problem();
  if (!p) return TSAT_ENOMEM;
  p->n_inst = n_inst;
  p->V = (int32_t)s.V;
  p->C = (int32_t)s.C;
  p->nnz_raw = s.nnz_raw;
  p->ws = d_ws;
  p->ws_bytes = ws_bytes;
  p->lay = L;
  cudaGetDevice(&p->device);
  char *w = (char *)d_ws;
  // host: instance table and global raw clause offsets
  p->inst.resize(n_inst);
  p->inst_nnz.resize(n_inst);
  std::vector<int64_t> raw_cptr(locality ? (size_t)s.C + 1 : 0);
  // clause order: as given, or (locality) each instance's clauses ordered by
  // their smallest variable, ties in the given order (a counting sort);
  // cperm maps a loaded clause to its index in the caller's batch
  std::vector<std::vector<int32_t>> plits(locality ? n_inst : 0);
  if (locality) p->cperm.resize((size_t)s.C);
  int64_t voff = 0, coff = 0, loff = 0;
  for (int32_t j = 0; j < n_inst; ++j) {
    InstInfo &I = p->inst[j];
    I.v_off = (int32_t)voff;
    I.n_vars = descs[j].n_vars;
    I.c_off = (int32_t)coff;
    I.n_clauses = descs[j].n_clauses;
    I.lmax = 0;
    I.gid = j;
    const int64_t *cp = descs[j].h_clause_ptr;
    p->inst_nnz[j] = cp[descs[j].n_clauses];
    if (!locality) {
      // copied as given below, the literal offset added on the device
    } else {
      const int32_t nc = descs[j].n_clauses, nv = descs[j].n_vars;
      const int32_t *lits = descs[j].h_lits;
      std::vector<int32_t> key((size_t)nc), start((size_t)nv + 2, 0);
      for (int32_t c = 0; c < nc; ++c) {
        int32_t mn = nv;   // empty or invalid clauses last (the build reports them)
        for (int64_t k = cp[c]; k < cp[c + 1]; ++k) {
          const int32_t a = lits[k] < 0 ? -lits[k] : lits[k];
          if (a >= 1 && a <= nv) mn = std::min(mn, a - 1);
        }
        key[c] = mn;
        ++start[mn + 1];
      }
      for (int32_t v = 0; v <= nv; ++v) start[v + 1] += start[v];
      std::vector<int32_t> order((size_t)nc);
      for (int32_t c = 0; c < nc; ++c) order[start[key[c]]++] = c;
      std::vector<int32_t> &pl = plits[j];
      pl.reserve((size_t)cp[nc]);
      for (int32_t q = 0; q < nc; ++q) {
        const int32_t c = order[q];
        raw_cptr[coff + q] = loff + (int64_t)pl.size();
        pl.insert(pl.end(), lits + cp[c], lits + cp[c + 1]);
        p->cperm[coff + q] = (int32_t)(coff + c);
      }
    }
    voff += descs[j].n_vars;
    coff += descs[j].n_clauses;
    loff += cp[descs[j].n_clauses];
  }
  const int64_t total_lits = loff;
  auto fail = [&](int code) { delete p; return code; };
#define CK(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return fail(cuda_fail(e_, #call)); } while (0)
  if (locality) {
    raw_cptr[s.C] = total_lits;
    CK(cudaMemcpyAsync(w + L.raw_cptr, raw_cptr.data(), sizeof(int64_t) * raw_cptr.size(),
                       cudaMemcpyHostToDevice, stream));
  } else {
    // the caller's clause pointers straight to the device (no host pass over
    // the clauses), then each instance's literal offset added there
    int64_t *dcp = (int64_t *)(w + L.raw_cptr);
    RawOffChunk ch{};
    int64_t lo2 = 0;
    for (int32_t j = 0; j < n_inst; ++j) {
      const int32_t nc = descs[j].n_clauses;
      const int64_t c0 = p->inst[j].c_off;
      CK(cudaMemcpyAsync(dcp + c0, descs[j].h_clause_ptr, sizeof(int64_t) * nc, cudaMemcpyHostToDevice, stream));
      ch.coff[ch.n] = c0;
      ch.loff[ch.n] = lo2;
      ++ch.n;
      ch.coff[ch.n] = c0 + nc;
      lo2 += descs[j].h_clause_ptr[nc];
      if (ch.n == kRawChunk || j == n_inst - 1) {
        const int64_t span = ch.coff[ch.n] - ch.coff[0];
        if (ch.n > 1 || ch.loff[0] != 0)   // the first instance alone needs no offset
          k_raw_offsets<<<(unsigned)((span + 255) / 256), 256, 0, stream>>>(dcp, ch);
        CK(cudaGetLastError());
        ch = RawOffChunk{};
      }
    }
    // the end of the last clause: a host scalar that lives until the
    // synchronisation after the dedup below
    static_assert(sizeof(total_lits) == sizeof(int64_t), "offset width");
    CK(cudaMemcpyAsync(dcp + s.C, &total_lits, sizeof(int64_t), cudaMemcpyHostToDevice, stream));
  }
  int64_t lo = 0;
  for (int32_t j = 0; j < n_inst; ++j) {
    int64_t n = descs[j].h_clause_ptr[descs[j].n_clauses];
    if (n) CK(cudaMemcpyAsync(w + L.raw_lits + sizeof(int32_t) * lo, locality ? plits[j].data() : descs[j].h_lits,
                              sizeof(int32_t) * n, cudaMemcpyHostToDevice, stream));
    lo += n;
  }
  CK(cudaMemcpyAsync(w + L.inst, p->inst.data(), sizeof(InstInfo) * n_inst, cudaMemcpyHostToDevice, stream));
  CK(cudaMemsetAsync(w + L.err, 0xFF, 64, stream));
  CK(cudaMemsetAsync(w + L.deg, 0, sizeof(int32_t) * (s.V + 1), stream));
  CK(cudaMemsetAsync(w + L.recsz, 0, sizeof(int32_t) * (s.V + 1), stream));
  CK(cudaMemsetAsync(w + L.fill, 0, sizeof(int32_t) * (s.V + 1), stream));
  auto P32 = [&](size_t off) { return (int32_t *)(w + off); };
  auto P64 = [&](size_t off) { return (int64_t *)(w + off); };
  const int T = 256;
  const unsigned gc = (unsigned)((s.C + T - 1) / T), gv = (unsigned)((s.V + T - 1) / T);
  InstInfo *dinst = (InstInfo *)(w + L.inst);
  unsigned long long *derr = (unsigned long long *)(w + L.err);
  k_dedup<<<gc, T, 0, stream>>>(P64(L.raw_cptr), P32(L.raw_lits), p->C, dinst, n_inst, P32(L.tmp),
                                P32(L.clen), derr);
  CK(cudaGetLastError());
  unsigned long long herr = ~0ull;
  CK(cudaMemcpyAsync(&herr, derr, sizeof(herr), cudaMemcpyDeviceToHost, stream));
  CK(cudaMemcpyAsync(p->inst.data(), dinst, sizeof(InstInfo) * n_inst, cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  int32_t lmax_all = 0;
  for (auto &I : p->inst) lmax_all = std::max(lmax_all, I.lmax);
  const int stride = lmax_all <= 3 ? 4 : (lmax_all <= 7 && 8 * s.nnz_raw <= L.xrec_cap) ? 8 : 0;
  if (herr != ~0ull) {
    int code = (int)(herr & 0xFF);
    long long c = (long long)(herr >> 8);
    if (!p->cperm.empty() && c >= 0 && c < (long long)p->cperm.size()) c = p->cperm[(size_t)c];
    set_error("clause %lld (global index) is invalid", c);
    return fail(code == 1 ? TSAT_EVAR : code == 2 ? TSAT_EEMPTY : TSAT_ELEN);
  }
  int rc2 = exclusive_scan(P32(L.clen), s.C, false, P64(L.scan_tmp), nullptr, P32(L.cptr), stream);
  if (rc2) return fail(rc2);
  k_compact_count<<<gc, T, 0, stream>>>(P64(L.raw_cptr), P32(L.tmp), P32(L.clen), P32(L.cptr), p->C,
                                        P32(L.clit), P32(L.deg), P32(L.recsz));
  CK(cudaGetLastError());
  rc2 = exclusive_scan(P32(L.deg), s.V, false, P64(L.scan_tmp), nullptr, P32(L.vptr), stream);
  if (rc2) return fail(rc2);
  if (stride) {
    k_xptr_fixed<<<(unsigned)((s.V + 1 + T - 1) / T), T, 0, stream>>>(P32(L.vptr), p->V, P64(L.xptr), stride);
    CK(cudaGetLastError());
  } else {
    rc2 = exclusive_scan(P32(L.recsz), s.V, true, P64(L.scan_tmp), P64(L.xptr), nullptr, stream);
    if (rc2) return fail(rc2);
  }
  k_fill<<<gc, T, 0, stream>>>(P32(L.cptr), P32(L.clit), p->C, P32(L.vptr), P32(L.fill), P32(L.occ_j),
                               P32(L.occ_c));
  CK(cudaGetLastError());
  k_records<<<(unsigned)s.V, 128, 0, stream>>>(P32(L.cptr), P32(L.clit), p->V, P32(L.vptr), P32(L.occ_j),
                                               P32(L.occ_c), P32(L.occ_s), P64(L.xptr), P32(L.xrec), P32(L.vocc), stride);
  CK(cudaGetLastError());
  k_var_inst<<<gv, T, 0, stream>>>(dinst, n_inst, p->V, P32(L.var_inst));
  CK(cudaGetLastError());
  if (L.crec) {
    k_crec<<<gc, T, 0, stream>>>(P32(L.cptr), P32(L.clit), p->C, (int4 *)(w + L.crec));
    CK(cudaGetLastError());
  }
  int32_t nnz32 = 0;
  int64_t xlen = 0;
  CK(cudaMemcpyAsync(&nnz32, P32(L.cptr) + s.C, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
  CK(cudaMemcpyAsync(&xlen, P64(L.xptr) + s.V, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
  CK(cudaMemcpyAsync(p->inst.data(), dinst, sizeof(InstInfo) * n_inst, cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
#undef CK
  if (xlen > L.xrec_cap) { set_error("record overflow %lld > %lld", (long long)xlen, (long long)L.xrec_cap); return fail(TSAT_EINVAL); }
  p->nnz = nnz32;
  p->xrec_words = xlen;
  p->lmax = 0;
  for (auto &I : p->inst) p->lmax = std::max(p->lmax, I.lmax);
  ProbDev &D = p->dev;
  D.n_inst = n_inst;
  D.V = p->V;
  D.C = p->C;
  D.lmax = p->lmax;
  D.nnz = p->nnz;
  D.cptr = P32(L.cptr);
  D.clit = P32(L.clit);
  D.xptr = P64(L.xptr);
  D.xrec = P32(L.xrec);
  D.vptr = P32(L.vptr);
  D.vocc = P32(L.vocc);
  D.rec_stride = stride;
  D.var_inst = P32(L.var_inst);
  D.items = (const int4 *)(w + L.items);
  D.inst = dinst;
  D.crec = L.crec ? (const int4 *)(w + L.crec) : nullptr;
  D.full3 = (L.crec && p->nnz == 3LL * p->C) ? 1 : 0;
  // forward work items of 1024 clauses (measured 512..4096: near the best on
  // large problems); on small problems fewer clauses per item, down to
  // kItemMin, so that the forward has a couple of items per SM (one planted
  // 3-SAT instance of n = 100 would otherwise be one block)
  int32_t ic = 1024;
  while (ic > kItemMin && ((int64_t)p->C + ic - 1) / ic < 2 * 148) ic >>= 1;
  int rc3 = p->set_items(ic, stream);
  if (rc3) return fail(rc3);
  *out = p;
  return TSAT_OK;
}

int tsat_load(int32_t n_vars, int32_t n_clauses, const int64_t *h_clause_ptr, const int32_t *h_lits,
              void *d_ws, size_t ws_bytes, cudaStream_t stream, tsat_problem **out) {
  tsat_cnf_desc d{n_vars, n_clauses, h_clause_ptr, h_lits};
  return tsat_load_batch(1, &d, d_ws, ws_bytes, stream, out);
}

void tsat_problem_free(tsat_problem *p) { delete p; }

int tsat_problem_info(const tsat_problem *p, int64_t h_info[8]) {
  if (!p || !h_info) return TSAT_EINVAL;
  h_info[6] = p->xrec_words;
  h_info[7] = (int64_t)p->lay.total;
  h_info[0] = p->n_inst;
  h_info[1] = p->V;
  h_info[2] = p->C;
  h_info[3] = p->nnz;
  h_info[4] = p->lmax;
  h_info[5] = p->dev.n_items;
  return TSAT_OK;
}

int tsat_problem_set_instance_ids(tsat_problem *p, const int32_t *h_ids, cudaStream_t stream) {
  if (!p || !h_ids) { set_error("NULL argument"); return TSAT_EINVAL; }
  for (int32_t j = 0; j < p->n_inst; ++j) {
    if (h_ids[j] < 0) { set_error("instance id %d of instance %d is negative", h_ids[j], j); return TSAT_EINVAL; }
    p->inst[j].gid = h_ids[j];
  }
  TSAT_CUDA(cudaMemcpyAsync(const_cast<InstInfo *>(p->dev.inst), p->inst.data(), sizeof(InstInfo) * p->n_inst,
                            cudaMemcpyHostToDevice, stream));
  TSAT_CUDA(cudaStreamSynchronize(stream));
  return TSAT_OK;
}

int tsat_problem_csr(const tsat_problem *p, int32_t *h_cptr, int32_t *h_clit) {
  if (!p || !h_cptr || !h_clit) return TSAT_EINVAL;
  TSAT_CUDA(cudaMemcpy(h_cptr, p->dev.cptr, sizeof(int32_t) * (p->C + 1), cudaMemcpyDeviceToHost));
  TSAT_CUDA(cudaMemcpy(h_clit, p->dev.clit, sizeof(int32_t) * p->nnz, cudaMemcpyDeviceToHost));
  if (!p->cperm.empty()) {   // back to the caller's clause order
    std::vector<int32_t> cp(h_cptr, h_cptr + p->C + 1), cl(h_clit, h_clit + p->nnz), len((size_t)p->C);
    for (int32_t q = 0; q < p->C; ++q) len[(size_t)p->cperm[q]] = cp[q + 1] - cp[q];
    h_cptr[0] = 0;
    for (int32_t c = 0; c < p->C; ++c) h_cptr[c + 1] = h_cptr[c] + len[c];
    for (int32_t q = 0; q < p->C; ++q)
      std::copy(cl.begin() + cp[q], cl.begin() + cp[q + 1], h_clit + h_cptr[p->cperm[q]]);
  }
  return TSAT_OK;
}

int32_t tsat_partial_k(int32_t n_vars) {
  if (n_vars <= 0) return 0;
  int64_t k = ((int64_t)n_vars + 9999) / 10000;
  if (k < 20) k = 20;
  if (k > n_vars) k = n_vars;
  return (int32_t)k;
}

}  // extern "C"
