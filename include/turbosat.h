/*
 * turbosat.h -- C ABI of the B300 (sm_103a) gradient-guided SAT hot path.
 *
 * Method: TurboSAT, arXiv 2511.07737.  A CNF with V variables and C clauses
 * becomes the binarised product R = P A (Sec. III-A, Eq. 1) of the 0/1
 * clause-literal matrix P (C x 2V) and N candidate assignments A (2V x N).
 * Each step evaluates SmoothMin over every column of R (Eq. 4), the loss
 * L = -sum_i S_i (Eq. 3), back-propagates through the straight-through
 * estimator (Sec. III-B, Fig. 3) and the per-variable normalisation (Eq. 5),
 * applies AdamW with the step-decay / restart schedule (Sec. IV-A) and
 * re-binarises (Eq. 2, optionally Philox-sampled).  Exact satisfaction is
 * decided with bit-packed clause checks (Sec. III-A, Satisfiability Matrix);
 * the hand-off to CDCL takes the best sample and the k most confident
 * variables, ranked by the smallest |gradient| (Sec. IV-B).
 *
 * Conventions for every call:
 *   - Return value: TSAT_OK (0) or a negative TSAT_E* status; no call aborts.
 *     tsat_strerror() names a status, tsat_last_error() gives the detail of
 *     the most recent failure in this thread.
 *   - Pointers named h_* are host memory, d_* are device memory on the
 *     current device.  All device memory is owned by the caller (typically a
 *     torch tensor); the library never frees it and keeps the pointer for the
 *     life of the handle that was built on it.
 *   - Calls that take a cudaStream_t are asynchronous on that stream unless
 *     stated otherwise.  The state keeps an internal stream; calls order
 *     themselves after the work already queued on the caller's stream and
 *     make the caller's stream wait for their own work.
 *   - Sample count N is a power of two in [32, 1024].  Clause length after
 *     de-duplication is at most TSAT_MAX_CLAUSE_LEN.  The total number of
 *     literal occurrences of a problem is below 2^31.
 */
#ifndef TURBOSAT_H
#define TURBOSAT_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TSAT_OK 0
#define TSAT_EINVAL -1    /* bad argument (NULL, size out of range, N not a power of two) */
#define TSAT_EVAR -2      /* a literal is 0 or names a variable outside 1..n_vars */
#define TSAT_EEMPTY -3    /* an empty clause: the formula is unsatisfiable by definition */
#define TSAT_EWS -4       /* workspace / state buffer smaller than the queried size */
#define TSAT_ECUDA -5     /* a CUDA runtime call failed; see tsat_last_error() */
#define TSAT_ETIMEOUT -6  /* a device-side wait gave up (the proposer's tensor-core layers: tsat_mpnn_status) */
#define TSAT_ENOMEM -7    /* host allocation failed */
#define TSAT_ELEN -8      /* a clause is longer than TSAT_MAX_CLAUSE_LEN after de-duplication */
#define TSAT_ESTATE -9    /* handle used with a state it was not built for, or not initialised */
#define TSAT_ERANGE -10   /* instance index, k or another count outside its range */

#define TSAT_MAX_CLAUSE_LEN 31
#define TSAT_MIN_SAMPLES 32
#define TSAT_MAX_SAMPLES 1024
#define TSAT_MAX_PARTIAL_K 16384

/* Normalisation before binarisation (Eq. 5 and the readings of it). */
#define TSAT_NORM_SIGNED_MEAN 0 /* Eq. 5 as printed: z / mean_i z            */
#define TSAT_NORM_ABSMEAN 1     /* sign-keeping: z / mean_i |z|              */
#define TSAT_NORM_NONE 2        /* z itself                                  */

/* Binarisation (Eq. 2 and the stochastic exploration of the abstract). */
#define TSAT_BIN_DET 0    /* x = [zt > 0]                                       */
#define TSAT_BIN_PHILOX 1 /* x = [u < clamp(1/2 + c zt, 0, 1)], u from Philox4x32-10 */

/* Literal values in the forward pass. */
#define TSAT_LAYER_STE 0     /* binary literals, straight-through gradient (Fig. 3) */
#define TSAT_LAYER_RELAXED 1 /* sigmoid(zt) literals, exact gradient              */

/* Storage type of the relaxed literal values. */
#define TSAT_DTYPE_F32 0
#define TSAT_DTYPE_BF16 1

/* Hyper-parameters (Sec. IV-A where stated; readings where the paper is silent). */
typedef struct tsat_hparams {
  float tau;              /* SmoothMin temperature of Eq. 4 (not given in the paper; default 1) */
  float lr0;              /* initial learning rate, 1e-1 (Sec. IV-A) */
  float lr_factor;        /* multiplier per decay period, 0.1 (Sec. IV-A) */
  float lr_floor;         /* lower bound, 1e-15 (Sec. IV-A "final learning rate") */
  int32_t decay_period;   /* iterations per decay, 30 (Sec. IV-A) */
  int32_t restart_period; /* iterations per restart, 360 (Sec. IV-A) */
  double beta1, beta2;    /* AdamW moment decays (PyTorch defaults 0.9, 0.999); 1 - beta and the bias
                             corrections are formed in double, as PyTorch does */
  float eps, weight_decay; /* AdamW; PyTorch defaults 1e-8, 0.01 */
  int32_t norm;           /* TSAT_NORM_* (default TSAT_NORM_SIGNED_MEAN) */
  int32_t binarize;       /* TSAT_BIN_* (default TSAT_BIN_DET) */
  float bin_temp;         /* T of the Philox rule, c = 0.25 / T (default 1) */
  int32_t layer;          /* TSAT_LAYER_* (default TSAT_LAYER_STE) */
  uint64_t seed;          /* Philox key (init and sampled binarisation) */
  int32_t mix_restart;    /* 1: assignment mixing at each lr restart (t = k * restart_period, k >= 1):
                             the instance's sample with the fewest unsatisfied clauses, i*, is kept,
                             every other sample's z becomes (z + z_i*) / 2, m = v = 0, and the AdamW
                             step count restarts; that step takes no gradient step.  A variant the
                             paper describes and leaves disabled (Sec. IV-A); default 0 */
  int32_t reserved;       /* must be 0 */
} tsat_hparams;

/* One CNF in DIMACS form: clause c holds h_lits[h_clause_ptr[c] .. h_clause_ptr[c+1]),
 * literals are +-(1..n_vars), no zeros.  Host memory, read during the call only. */
typedef struct tsat_cnf_desc {
  int32_t n_vars;
  int32_t n_clauses;
  const int64_t *h_clause_ptr; /* n_clauses + 1 entries, non-decreasing, [0] = 0 */
  const int32_t *h_lits;
} tsat_cnf_desc;

typedef struct tsat_problem tsat_problem; /* host handle; device arrays live in the caller's workspace */
typedef struct tsat_state tsat_state;     /* host handle over a caller-owned device state buffer */

/* Per-instance progress (host copy). */
typedef struct tsat_inst_status {
  int32_t found;        /* 1 once a sample satisfied every clause (max S > 0, Sec. III-A) */
  int32_t found_sample; /* that sample, else -1 */
  int64_t found_step;   /* step at which it was found, else -1 */
  int32_t min_unsat;    /* fewest unsatisfied clauses over the samples at the last step */
  int32_t best_sample;  /* sample with min_unsat (lowest index on ties) */
  float loss;           /* L = -sum_i S_i of the last step (Eq. 3) */
  float pad;
} tsat_inst_status;

const char *tsat_strerror(int status);
const char *tsat_last_error(void);
void tsat_hparams_default(tsat_hparams *hp);

/* ---- problem (Sec. III-A "Problem Matrix", Sec. IV-A compressed sparse P) ----
 * tsat_problem_bytes: pure host computation of the device workspace size for a
 * batch of n_inst CNFs (a single CNF is a batch of one).
 * tsat_load_batch: copies the CNFs to the device and builds, on the device,
 *   - the clause-major CSR of P (duplicate literals removed, Sec. III-A: P is 0/1),
 *   - the variable-major occurrence records used by the backward pass (P^T),
 *   - the forward work list of (instance, clause range) items.
 * Errors: TSAT_EINVAL, TSAT_EVAR, TSAT_EEMPTY, TSAT_ELEN, TSAT_EWS, TSAT_ECUDA,
 * TSAT_ENOMEM.  Synchronous (waits for the build to finish, to report input
 * errors).  d_ws must stay allocated until tsat_problem_free. */
int tsat_problem_bytes(int32_t n_inst, const tsat_cnf_desc *descs, size_t *ws_bytes);
int tsat_load_batch(int32_t n_inst, const tsat_cnf_desc *descs, void *d_ws, size_t ws_bytes,
                    cudaStream_t stream, tsat_problem **out);
/* tsat_load_batch with flags.  TSAT_LOAD_CLAUSE_LOCALITY: the library stores
 * each instance's clauses ordered by their smallest variable (ties in the
 * caller's order; a counting sort on the host, O(clauses + literals)).  The
 * clause-major forward then visits the literal rows of nearby variables
 * together (the relaxed forward and the exact check of the structured mixed
 * workload take 15 % less time; loading takes about 0.5 s more at 8 M
 * clauses).  Every output
 * stays in the caller's numbering (variables are not renumbered; clause-indexed
 * exports such as tsat_problem_csr and error messages are mapped back); FP32
 * sums over clauses take the new order.  Other flag bits: TSAT_EINVAL. */
#define TSAT_LOAD_CLAUSE_LOCALITY 1u
int tsat_load_batch_ex(int32_t n_inst, const tsat_cnf_desc *descs, uint32_t flags, void *d_ws, size_t ws_bytes,
                       cudaStream_t stream, tsat_problem **out);
int tsat_load(int32_t n_vars, int32_t n_clauses, const int64_t *h_clause_ptr,
              const int32_t *h_lits, void *d_ws, size_t ws_bytes, cudaStream_t stream,
              tsat_problem **out);
void tsat_problem_free(tsat_problem *p);
/* Sizes after de-duplication: h_info = {n_inst, n_vars, n_clauses, nnz, lmax, n_items,
 * occurrence-record words, workspace bytes in use}. */
int tsat_problem_info(const tsat_problem *p, int64_t h_info[8]);
/* Random streams per instance.  Every random draw of an instance (the init of
 * Sec. IV-A and the Philox-sampled binarisation) uses a Philox4x32-10 key
 * whose low word is seed_low + the instance's id, and counters that carry the
 * instance-local variable index, so an instance gets the same draws whichever
 * batch it is loaded in.  Ids default to the position in the loaded batch
 * (0 .. n_inst-1; a single instance: id 0, i.e. the plain seed); a caller
 * that splits a batch over several processes sets each instance's position in
 * the whole batch here, before tsat_init.  h_ids: int32 [n_inst], >= 0.
 * Synchronous (waits for `stream`). */
int tsat_problem_set_instance_ids(tsat_problem *p, const int32_t *h_ids, cudaStream_t stream);
/* Device CSR views for inspection (clause-major, lit = (global var << 1) | negated):
 * copies cptr (n_clauses+1 int32) and clit (nnz int32) to host buffers. */
int tsat_problem_csr(const tsat_problem *p, int32_t *h_cptr, int32_t *h_clit);

/* ---- state: N assignment samples per instance (Sec. III-A "Assignment Matrix") ----
 * Layout inside d_state (all row-major, row = global variable):
 *   z, m, v   float [V][N]     trainable A_real (one row per variable) and AdamW moments
 *   bits      uint32 [2][V][N/32]  binarised A, bit (i mod 32) of word i/32 = x_vi
 *   nu        float [V]        normaliser of the current z (Eq. 5)
 * plus per-instance histograms, gamma tables, S and status records.
 * d_state stays caller-owned.  tsat_state_create also makes the state's own
 * stream, two events and a pinned host buffer for tsat_status (the header plus
 * 32 bytes per instance); tsat_state_free releases them, and so does a failed
 * tsat_state_create. */
int tsat_state_bytes(const tsat_problem *p, int32_t n_samples, int32_t layer,
                     int32_t relaxed_dtype, size_t *state_bytes);
int tsat_state_create(tsat_problem *p, void *d_state, size_t state_bytes, int32_t n_samples,
                      int32_t layer, int32_t relaxed_dtype, tsat_state **out);
void tsat_state_free(tsat_state *s);

/* Random init of A_real (Sec. IV-A: standard normal, balanced 0/1 after B).
 * d_logits (nullable, float [V]) shifts row v by d_logits[v] * logit_scale (a
 * learned proposal); the random part stays as the fallback.  Sets step t = 0
 * and binarises with hp->norm / hp->binarize.  Async. */
int tsat_init(tsat_state *s, const tsat_hparams *hp, const float *d_logits, float logit_scale,
              cudaStream_t stream);

/* n_steps optimisation steps (Sec. III-B and IV-A), replayed from a cached
 * CUDA graph.  An instance whose sample satisfies every clause is frozen at
 * that step (its bits keep the model).  With stop_on_sat, the remaining steps
 * become no-ops once every instance is frozen.  Async; hp is copied. */
int tsat_step(tsat_state *s, const tsat_hparams *hp, int32_t n_steps, int32_t stop_on_sat,
              cudaStream_t stream);

/* The same n_steps steps as tsat_step for a batch of small instances, in one
 * launch: each instance is owned by one thread block, which runs its steps
 * (Eq. 1 forward, Eq. 4, the STE backward, Eq. 5, AdamW, re-binarisation;
 * Sec. III-B, IV-A) with block barriers between the phases and no wait on any
 * other block.  Results follow tsat_step: per-instance freezing at the first
 * zero-unsat sample, the status records, the step counter and, with
 * stop_on_sat, the stop once every instance is frozen; FP32 sums may differ
 * from tsat_step in rounding order, integers and bits agree given the same
 * FP32 state.  Each block keeps its instance's bits (both step parities) in
 * shared memory.  When the batch leaves SMs idle (N <= 256), an instance may
 * instead get a thread-block cluster of 2, 4 or 8 blocks (see
 * tsat_set_persist_blocks): the blocks split its clauses in the forward and
 * its rows in the update, each keeps a copy of the bits, and the histograms
 * are summed over distributed shared memory between two cluster barriers per
 * step; where one block and the cluster keep z, m, v in the same place, the
 * results are those of one block per instance, bit for bit.
 * Requirements: the STE layer, hp->mix_restart = 0, clauses of at most 7
 * literals, clauses x longest clause x samples <= 2^26 per block of the
 * instance, and 4 (18.5 N + 2 n_vars N / 32) bytes of shared memory <= 200
 * KiB for the largest instance (26.5 N with a cluster; about 25,000 variables
 * at N = 32, 12,500 at N = 64, 500 at N = 1024); else TSAT_EINVAL /
 * TSAT_ERANGE.  Async on `stream`. */
int tsat_step_persistent(tsat_state *s, const tsat_hparams *hp, int32_t n_steps, int32_t stop_on_sat,
                         cudaStream_t stream);

/* Blocks per instance of tsat_step_persistent: 0 = automatic (the default:
 * 1 when one block keeps the largest instance's z, m, v in shared memory or
 * N > 256, else the largest of 2, 4, 8 with which every instance's cluster
 * fits on the device at once, or, when that does not keep the instances in
 * shared memory, the smallest larger one that does within two waves of
 * clusters), or 1, 2, 4, 8 (2..8 need N <= 256).  The
 * blocks keep their rows' z, m, v in shared memory when those fit (else in
 * global memory, with 8 instead of 16 samples per thread); two settings with
 * the same placement give the same results bit for bit, otherwise the FP32
 * row sums of Eq. 5 differ in rounding order.  tsat_persist_blocks: the
 * blocks per instance the next tsat_step_persistent call will use and, if
 * `resident` is not NULL, 1 when they keep z, m, v in shared memory.  Host
 * only; TSAT_EINVAL on other values. */
int tsat_set_persist_blocks(tsat_state *s, int32_t blocks_per_instance);
int tsat_persist_blocks(const tsat_state *s, int32_t *blocks_per_instance, int32_t *resident);

/* Times n_steps persistent steps (no early stop) from the state's current
 * contents with each candidate number of blocks per instance (1, and with
 * N <= 256 clusters of 2, 4 and 8 while the batch's clusters fit the device at
 * most twice over), keeps the fastest (tsat_set_persist_blocks) and returns it
 * in *h_blocks.  d_snapshot: caller-owned device scratch of
 * tsat_autotune_bytes; every trial starts from the saved state and the state
 * is put back at the end, so no result changes.  Synchronises with the
 * trials; TSAT_EINVAL / TSAT_ERANGE as tsat_step_persistent, TSAT_ERANGE when
 * no candidate runs the batch.  On any error the previous blocks-per-instance
 * setting is kept and the saved state is copied back. */
int tsat_autotune_persistent(tsat_state *s, const tsat_hparams *hp, void *d_snapshot, size_t snapshot_bytes,
                             int32_t n_steps, cudaStream_t stream, int32_t *h_blocks);

/* The same n_steps steps for a batch whose instances are too large for one
 * block, in one launch of thread-block clusters (4 blocks of 768 threads, one
 * per SM, as many clusters as fit on the device).  The host deals the
 * instances to the clusters so that each holds about the same number of
 * literal occurrences (largest first, once per state); a cluster runs its
 * instances one after another, every warp of its blocks on the same
 * instance: the forward (Eq. 1) into per-block histograms, a cluster barrier,
 * every block sums the histograms over distributed shared memory and forms
 * Eq. 4 and the dL/dR table, the fused update of the instance's rows
 * (straight-through backward, Eq. 5, AdamW, re-binarisation), a cluster
 * barrier.  Results follow tsat_step (freezing, status records, step counter,
 * stop_on_sat); FP32 sums may differ from it in rounding order.
 * tsat_step_persistent takes this path by itself when an instance does not
 * fit one block.  Requirements: the STE layer, hp->mix_restart = 0, a longest
 * clause of 4..7 literals, N <= 128; else TSAT_EINVAL.  Async on `stream`. */
int tsat_step_clustered(tsat_state *s, const tsat_hparams *hp, int32_t n_steps, int32_t stop_on_sat,
                        cudaStream_t stream);

/* Capture and instantiate the graph tsat_step(hp, n_steps, stop_on_sat) would
 * replay, without running it (keeps graph building out of timed regions). */
int tsat_step_prepare(tsat_state *s, const tsat_hparams *hp, int32_t n_steps, int32_t stop_on_sat);

/* ---- sample sharding (one problem's samples over several processes) ----
 * The paper ran on up to two GPUs (Sec. V) without saying how.  Every part of
 * a step except Eq. 5 reads one sample column only (Eq. 1 forward, Eqs. 3-4,
 * the straight-through backward of Sec. III-B), so the N samples split into
 * shards of equal power-of-two size, one state (n_samples = the shard's size)
 * per process.  Eq. 5 couples a row's samples through two sums over all N:
 * sum_i G_vi z_vi (its chain rule) and sum_i z_vi or sum_i |z_vi| (the new
 * normaliser).  A sharded step is therefore
 *     tsat_shard_grad -> all-reduce d_rowdot -> tsat_shard_update ->
 *     all-reduce d_rowsum -> tsat_shard_finish
 * and the init is tsat_shard_init -> all-reduce d_rowsum -> tsat_shard_finish;
 * the caller makes the all-reduces (sums of float [V], NCCL between GPUs).
 * Random draws use the samples' global indices, so the shards draw what one
 * state of all N samples would; FP32 sums differ from it in order only.
 * tsat_state_set_shard: this state holds samples [sample_base, sample_base +
 *   n_samples) of n_total (sample_base a multiple of n_samples); call before
 *   tsat_shard_init.  A shard refuses tsat_init, tsat_step(_persistent),
 *   tsat_forward / tsat_backward, tsat_autotune and tsat_profile_step
 *   (TSAT_ESTATE).
 * tsat_shard_init: Irwin-Hall init of z (Sec. IV-A), m = v = 0, step 0;
 *   d_rowsum float [V] receives this shard's row sums of z (|z| for mean |z|).
 * tsat_shard_grad: the step's forward and gamma (status records of this
 *   shard's samples, freezing of an instance when one of them satisfies it,
 *   step scalars; the step counter advances), d_G float [V][n_samples] = the
 *   straight-through gradient of L with respect to the normalised assignment
 *   of this shard's samples, d_rowdot float [V] = sum over them of G z (0 for
 *   frozen instances and without normalisation).
 * tsat_shard_update: with d_rowdot_total (the all-reduced d_rowdot), the Eq. 5
 *   chain rule, AdamW and the new z, m, v of live rows; d_rowsum float [V] =
 *   this shard's row sums of the new z (|z|).
 * tsat_shard_finish: with d_rowsum_total, nu_v = total / n_total (guarded as
 *   in Eq. 5's reading; 1 without normalisation) and the bits of the current
 *   step (Eq. 2 or the Philox rule); frozen instances keep theirs.
 * Requirements: the STE layer, hp->mix_restart = 0, and the same hp on every
 * shard.  found_sample in tsat_status is an index within the shard.  All
 * async on `stream`. */
int tsat_state_set_shard(tsat_state *s, int32_t sample_base, int32_t n_total);
int tsat_shard_init(tsat_state *s, const tsat_hparams *hp, float *d_rowsum, cudaStream_t stream);
int tsat_shard_grad(tsat_state *s, const tsat_hparams *hp, float *d_G, float *d_rowdot, cudaStream_t stream);
int tsat_shard_update(tsat_state *s, const tsat_hparams *hp, const float *d_G, const float *d_rowdot_total,
                      float *d_rowsum, cudaStream_t stream);
int tsat_shard_finish(tsat_state *s, const tsat_hparams *hp, const float *d_rowsum_total, cudaStream_t stream);

/* Runs n_steps steps as individual launches on the state's stream with CUDA
 * events around each kernel and returns the average device time per launch
 * in milliseconds: h_ms[0] forward, h_ms[1] gamma, h_ms[2] update (relaxed
 * layer: h_ms[3] exact check).  Synchronous.  The steps are real steps (the
 * state advances). */
int tsat_profile_step(tsat_state *s, const tsat_hparams *hp, int32_t n_steps, float h_ms[4]);

/* Exact check of the current bits (Sec. III-A): d_unsat int32 [n_inst][N]
 * unsatisfied-clause counts, d_satmask uint32 [n_inst][N/32] bit set = sample
 * satisfies every clause.  d_loss (nullable, float [n_inst]) receives
 * L = -sum_i S_i (Eq. 3, Eq. 4 with hp->tau) of the current bits.  Async. */
int tsat_evaluate(tsat_state *s, const tsat_hparams *hp, int32_t *d_unsat, uint32_t *d_satmask,
                  float *d_loss, cudaStream_t stream);

/* The forward product of the current bits as per-sample histograms (Sec.
 * III-A, Eq. 1): d_hist int32 [n_inst][lmax+1][N] (lmax = the longest clause
 * of the batch, tsat_problem_info), d_hist[j][r][i] = number of clauses of
 * instance j whose R_ci = r, the count of true literals of clause c in sample
 * i (r = 0: unsatisfied).  Integer exact.  The caller owns d_hist; it is
 * overwritten.  Async on `stream`. */
int tsat_histogram(tsat_state *s, int32_t *d_hist, cudaStream_t stream);

/* Evaluation without any device allocation.  The paper has no counterpart:
 * this exists for callers that cannot call cudaMalloc (code running inside a
 * memory pool it does not own, or a process whose device memory another
 * runtime reserved up front, where a late allocation could fail or stall).
 * Same results as tsat_evaluate, but for a caller-supplied bit matrix d_bits
 * (uint32 [n_vars][n_samples/32], bit i%32 of word i/32 = sample i's value)
 * instead of a state: d_unsat int32 [n_inst][N] unsatisfied-clause counts,
 * d_satmask uint32 [n_inst][N/32], d_loss (nullable) float [n_inst], the
 * same loss value tsat_evaluate writes, with SmoothMin temperature tau.  The
 * temporaries live in one fixed 4 MiB array inside the library's device
 * image (each GPU that loads the library holds it until the process exits);
 * a problem needs n_inst * N * (lmax + 3) + 64 ints of it, and larger
 * requests fail with TSAT_ERANGE.  The problem's device must be the current
 * device (else TSAT_EINVAL).  The array's device address is looked up once
 * per device and CUDA context, by the first call made with that context
 * current (make that first call before any stream capture; a context made
 * again after cudaDeviceReset gets a fresh lookup).  Every call shares the
 * array and it keeps the last call's contents (the call clears what must
 * start at zero), so calls that overlap on the GPU (different streams, or
 * different problems at once) race; serialise them.  Async on `stream`. */
int tsat_evaluate_bits_noalloc(const tsat_problem *p, const uint32_t *d_bits, int32_t n_samples, float tau,
                               int32_t *d_unsat, uint32_t *d_satmask, float *d_loss, cudaStream_t stream);

/* Hand-off of instance `inst` (Sec. IV-B).  Chooses the sample with unsat = 0
 * (lowest index) or else the fewest unsatisfied clauses (lowest index on
 * ties), computes the STE gradient of its current bits, and returns the k
 * variables with the smallest |gradient| (ties to the lower index), k in
 * [1, min(TSAT_MAX_PARTIAL_K, n_vars)], in increasing |gradient| order.
 * Host outputs: h_bits uint32 [ceil(n_vars/32)] the chosen sample's full
 * assignment (bit v%32 of word v/32, instance-local variable numbering),
 * h_unsat, h_sample, h_part_var int32 [k] (1-based DIMACS variables),
 * h_part_val uint8 [k], h_ready (nullable) = 1 when more than 99 % of clauses
 * are satisfied (Sec. IV-B hand-off trigger).  Synchronous.  Returns 1 if the
 * chosen sample satisfies every clause, 0 if not, < 0 on error. */
int tsat_best(tsat_state *s, const tsat_hparams *hp, int32_t inst, int32_t k, uint32_t *h_bits,
              int32_t *h_unsat, int32_t *h_sample, int32_t *h_part_var, uint8_t *h_part_val,
              int32_t *h_ready, cudaStream_t stream);
/* k = max(20, ceil(1e-4 * n_vars)) capped at n_vars (Sec. IV-B: 0.01 %, at least 20). */
int32_t tsat_partial_k(int32_t n_vars);

/* Step counter and per-instance progress; synchronous copy to the host. */
int tsat_status(tsat_state *s, int64_t *h_step, int32_t *h_all_done,
                tsat_inst_status *h_inst /* n_inst entries, nullable */, cudaStream_t stream);

/* Raw views of the state for tests and checkpoints (device pointers into d_state). */
int tsat_state_views(tsat_state *s, float **z, float **m, float **v, uint32_t **bits_cur,
                     float **nu, float **gamma, int32_t **hist);

/* ---- differentiation (Fig. 3 as a layer; torch.autograd.Function hooks) ----
 * tsat_forward: from d_z (float [V][N], caller-owned, not the state's z)
 * computes the normaliser, binarises (hp->norm, hp->binarize at step t_bin),
 * evaluates R and SmoothMin, and writes d_S float [n_inst][N] and d_loss
 * float [n_inst].  Keeps bits / gamma in the state for tsat_backward.
 * tsat_backward: gradient of sum_inst dL * L_inst with respect to d_z
 * (straight-through or relaxed chain rule, then Eq. 5), written to d_grad
 * float [V][N].  Must follow tsat_forward on the same d_z.  Async. */
int tsat_forward(tsat_state *s, const tsat_hparams *hp, const float *d_z, int64_t t_bin,
                 float *d_S, float *d_loss, cudaStream_t stream);
int tsat_backward(tsat_state *s, const tsat_hparams *hp, const float *d_z, float dL,
                  float *d_grad, cudaStream_t stream);

/* ---- schedules ----
 * Launch shapes of the forward and update kernels (tile and
 * warps-per-clause schedules reduce to these knobs here).
 * tsat_autotune times candidate shapes on this state and keeps the fastest:
 * the forward's work-item size (clauses per item) on the forward, then the
 * update's blocks per SM and rows per work item on the step's own fused
 * update (hp's binarisation and Eq. 5 mode), each trial run after the step's
 * forward and gamma kernels from the state as the caller left it.  That state
 * (header, status records, z, m, v, bits, nu and, for the relaxed layer, the
 * literal values) is saved into the caller's device buffer d_snapshot of at
 * least tsat_autotune_bytes bytes before the first trial, restored before
 * every trial and restored again at the end, so the call leaves the state
 * unchanged.  A failed trial leaves the previous launch shapes (forward work
 * items and update grid) and copies the saved state back.  Synchronous
 * (returns after the last trial).  tsat_get_tuning / tsat_set_tuning read or
 * force the shapes.
 * h_tuning = {fwd_chunk_clauses, fwd_block_threads, upd_blocks_per_sm, upd_rows_per_item};
 * upd_blocks_per_sm in [0, 128], 0 = the default (resident blocks x 8 waves). */
int tsat_autotune_bytes(const tsat_state *s, size_t *bytes);
/* The candidates tsat_autotune tries on this state: forward work-item sizes
 * (4), update blocks per SM (5: d/8, d/4, d/2, d, 5d/4 around the default d
 * of resident blocks x waves), update rows per work item (3).  Host only. */
int tsat_tuning_space(const tsat_state *s, int32_t h_fwd_items[4], int32_t h_upd_bps[5], int32_t h_upd_rpi[3]);
int tsat_autotune(tsat_state *s, const tsat_hparams *hp, void *d_snapshot, size_t snapshot_bytes,
                  cudaStream_t stream, int32_t h_tuning[4]);
int tsat_get_tuning(const tsat_state *s, int32_t h_tuning[4]);
int tsat_set_tuning(tsat_state *s, const int32_t h_tuning[4]);

/* ---- learned proposer (a message-passing network proposing initial logits) ----
 * The paper cites learned SAT models only as related work (Sec. II); this is
 * an addition.  A 3-layer message-passing network (hidden 64, BF16 weights,
 * FP32 accumulation) on the literal-clause bipartite graph of a loaded
 * problem maps every variable to a logit; tsat_init(d_logits, scale) turns
 * the logits into initial z (random init stays the fallback) and the exact
 * check judges every proposal.  Parameters are a flat float array of
 * tsat_mpnn_param_count() entries (FP32 master copy, owned by the caller).
 * Workspace: tsat_mpnn_workspace_bytes (activations for the backward pass),
 * 256-byte aligned (as cudaMalloc returns it; TSAT_EINVAL otherwise).
 * tsat_mpnn_forward: from the second call with the same parameter, workspace
 * and logits pointers on the same problem, the forward's launches replay as
 * one captured CUDA graph (the values behind the pointers are read when it
 * runs); a call with other pointers runs directly.
 * tsat_mpnn_loss_grad: logits (float [V]), mean binary cross-entropy of the
 * logits against d_targets (uint8 [V], a satisfying assignment per instance)
 * summed over instances into d_loss[0], and its gradient d_grad (float
 * [param_count]).  tsat_mpnn_adam: one Adam step (0.9, 0.999, 1e-8) with the
 * 1-based step count.  All async on `stream`. */
int32_t tsat_mpnn_param_count(void);
int tsat_mpnn_workspace_bytes(const tsat_problem *p, size_t *bytes);
int tsat_mpnn_init(float *d_params, uint64_t seed, cudaStream_t stream);
int tsat_mpnn_forward(const tsat_problem *p, const float *d_params, void *d_ws, size_t ws_bytes, float *d_logits,
                      cudaStream_t stream);
int tsat_mpnn_loss_grad(const tsat_problem *p, const float *d_params, void *d_ws, size_t ws_bytes,
                        const uint8_t *d_targets, float *d_logits, float *d_loss, float *d_grad, cudaStream_t stream);
int tsat_mpnn_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int64_t step, float lr,
                   cudaStream_t stream);
/* Whether the last tsat_mpnn_forward / tsat_mpnn_loss_grad on this workspace
 * completed every tensor-core layer.  Each layer's wait for its MMAs is
 * bounded; one that gives up sets a flag in the workspace (the forward clears
 * it when it starts) and leaves its outputs invalid.  Synchronises `stream`,
 * reads the flag: TSAT_OK, or TSAT_ETIMEOUT when a wait gave up. */
int tsat_mpnn_status(const tsat_problem *p, const void *d_ws, size_t ws_bytes, cudaStream_t stream);

/* Number of kernel launches one step issues (for launch accounting). */
int32_t tsat_launches_per_step(const tsat_state *s);

#ifdef __cplusplus
}
#endif
#endif /* TURBOSAT_H */
