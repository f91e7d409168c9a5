/*
 * bo_suggest.h -- C ABI of the GB300 Bayesian-optimization suggest library.
 *
 * The library implements the per-iteration step of the GPU-kernel tuner of
 * Willemsen, van Nieuwpoort and van Werkhoven, "Bayesian Optimization for
 * auto-tuning GPU kernels":
 *   - a discrete, normalized, constrained search space (Sec. III-D);
 *   - a zero-mean Gaussian-process surrogate with a fixed-lengthscale Matern
 *     covariance (Sec. III-B), updated one observation at a time;
 *   - exhaustive prediction of every valid, non-evaluated configuration and
 *     the acquisition functions EI, PI and LCB (Sec. III-C, III-G) with the
 *     contextual-variance exploration factor (Sec. III-F);
 *   - the masked argmax, and the 'multi' / 'advanced multi' selection of
 *     acquisition functions (Sec. III-G).
 *
 * Conventions for every entry point:
 *   - Return value: BO_OK (0) or one of the BO_ERR_* codes below; on error a
 *     message is available from bo_last_error() on the calling thread, and
 *     no output argument has been written unless stated otherwise.
 *   - Indices are positions in the *valid list*: the valid configurations of
 *     the Cartesian product of the parameter lists, enumerated row-major with
 *     the last parameter fastest, restricted configurations removed.
 *   - Host pointers are plain host memory owned by the caller unless the
 *     argument says "device".  Arrays passed to bo_space_create are copied.
 *   - All device work of a space is ordered on the stream given at creation.
 *     A space may be used by one host thread at a time.
 *   - Environment, read when a space / batch is created: BO_NO_COOP (set:
 *     a space's observation update runs as four phase launches instead of one
 *     cooperative launch), BO_FUSED_ACQ (set: a reduced-precision space's
 *     prediction pass carries the acquisition as its tail, one cooperative
 *     launch instead of two; the same results), BO_NO_PDL (read once per
 *     process; set: the kernels of a pass are launched without programmatic
 *     dependent launch; the same results) and BO_NO_GRAPH (set: a batch
 *     launches its kernels one by one instead of replaying a captured CUDA
 *     graph).  Results are the same up to the reduction order of the
 *     update's pivot.
 */
#ifndef BO_SUGGEST_H
#define BO_SUGGEST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum {
  BO_OK = 0,
  BO_ERR_ARG = 1,          /* invalid argument or descriptor field            */
  BO_ERR_INDEX = 2,        /* valid-list index out of range                   */
  BO_ERR_DUPLICATE = 3,    /* configuration already observed (Sec. III-D)     */
  BO_ERR_EXHAUSTED = 4,    /* no valid, non-evaluated configuration left      */
  BO_ERR_NUMERIC = 5,      /* non-positive Cholesky pivot / non-finite value  */
  BO_ERR_NOMEM = 6,        /* device or host allocation failed                */
  BO_ERR_CUDA = 7,         /* a CUDA call failed                              */
  BO_ERR_TIMEOUT = 8,      /* a bounded device wait ran out                   */
  BO_ERR_NOT_POSITIVE = 9, /* contextual variance needs f+ > 0 and mu_s > 0   */
  BO_ERR_STATE = 10,       /* call not allowed in the current state           */
  BO_ERR_CAPACITY = 11     /* more valid observations than n_max              */
};

/* acquisition function / selection mode (Sec. III-C, III-G) */
enum { BO_AF_EI = 0, BO_AF_PI = 1, BO_AF_LCB = 2, BO_AF_MULTI = 3, BO_AF_ADV_MULTI = 4 };
/* exploration factor: contextual variance (Sec. III-F) or a constant */
enum { BO_EXPLORE_CV = 0, BO_EXPLORE_CONST = 1 };
/* observation normalization before fitting */
enum { BO_YNORM_STANDARDIZE = 0, BO_YNORM_NONE = 1 };
/* arithmetic of the K* . L^-T contraction (Cholesky, L^-1, beta are FP64 always) */
enum {
  BO_PREC_FP64 = 0,    /* FP64 on CUDA cores                                       */
  BO_PREC_FP16X3 = 1,  /* tcgen05 f16 hi/lo split, 3 products, FP32 accumulate     */
  BO_PREC_BF16X3 = 2,  /* tcgen05 bf16 hi/lo split, 3 products, FP32 accumulate    */
  BO_PREC_TF32 = 3,    /* tcgen05 tf32, 1 product, FP32 accumulate                 */
  BO_PREC_TF32X3 = 4   /* tcgen05 tf32 hi/lo split, 3 products, FP32 accumulate    */
};

/* initial sample (Sec. III-E; Table I selects maximin):
 *   RANDOM   uniform random valid configurations
 *   LHS      a Latin hypercube over the parameters' value lists: parameter p
 *            of sample i takes value floor(u m_p) of its m_p values, with
 *            u = (pi_p(i) + U) / n_init, pi_p a random permutation of the
 *            n_init strata and U uniform in [0, 1); restricted or repeated
 *            configurations are replaced by random valid ones
 *   MAXIMIN  as LHS, keeping of init_designs Latin hypercubes the one whose
 *            smallest pairwise distance between normalized points is largest
 * The exact draw order is given at bo_initial_design. */
enum { BO_INIT_RANDOM = 0, BO_INIT_LHS = 1, BO_INIT_MAXIMIN = 2 };

#define BO_MAX_PARAMS 16   /* parameters per space                             */
#define BO_MAX_VALUES 256  /* values per parameter (codes are uint8)          */
#define BO_MAX_OBS 512     /* largest n_max (valid observations fitted)        */

/* Device memory provider.  alloc returns device memory of at least `bytes`
 * bytes usable on `stream` (NULL on failure); free releases it.  With
 * alloc == NULL the library uses cudaMallocAsync/cudaFreeAsync on the
 * space's stream. */
typedef void* (*bo_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*bo_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

typedef struct bo_space_desc {
  int32_t d;                      /* number of parameters, 1..BO_MAX_PARAMS          */
  const int32_t* n_values;        /* [d] list length per parameter, 1..BO_MAX_VALUES */
  const double* const* values;    /* [d][n_values[p]] normalized values in [0, 1]    */
  const uint8_t* invalid_mask;    /* [prod n_values] 1 = restricted, or NULL         */
  double nu;                      /* Matern smoothness: 1.5 or 2.5                   */
  double lengthscale;             /* fixed lengthscale l > 0                         */
  double jitter;                  /* added to the diagonal of K, >= 0                */
  int32_t af;                     /* BO_AF_*                                         */
  int32_t explore;                /* BO_EXPLORE_*                                    */
  double lambda_const;            /* exploration factor when explore == CONST        */
  int32_t skip_threshold;         /* multi / advanced multi skip threshold           */
  double rif;                     /* advanced multi required improvement factor      */
  double discount;                /* dos discount; <= 0 selects the Table I default  */
  int32_t y_norm;                 /* BO_YNORM_*                                      */
  int32_t precision;              /* BO_PREC_*                                       */
  int32_t n_max;                  /* capacity in valid observations, 1..BO_MAX_OBS   */
  int32_t n_init;                 /* initial-sample suggests are made while fewer
                                     valid (finite) observations than this exist     */
  uint64_t seed;                  /* splitmix64 seed of every random draw            */
  int32_t init_mode;              /* BO_INIT_*: how the initial sample is drawn      */
  int32_t init_designs;           /* BO_INIT_MAXIMIN: Latin hypercube designs compared */
  bo_alloc_fn alloc;              /* device memory provider, or NULL                 */
  bo_free_fn free;
  void* alloc_ctx;
  void* stream;                   /* cudaStream_t for all device work (NULL = legacy) */
} bo_space_desc;

/* Fill `desc` with the defaults of Table I: nu = 3/2, l = 1.5 with the
 * contextual-variance factor, jitter 1e-10, EI, skip threshold 5,
 * rif 0.1, Table I discounts, standardized y, FP64, n_max = 512, maximin
 * initial sampling over 100 designs (n_init = 0: the caller supplies it). */
void bo_space_desc_init(bo_space_desc* desc);

/* The initial sample a space built from `desc` draws (Sec. III-E), computed
 * on the host from desc->d, n_values, values, invalid_mask, init_mode,
 * init_designs and seed alone (no device, no space needed).  idx_out[count]
 * receives distinct valid-list indices; count must be in [1, number of valid
 * configurations].  Draws come from one splitmix64 stream seeded with
 * desc->seed, in this order:
 *   RANDOM: per sample, r = next() mod N_valid, redrawn while already taken.
 *   LHS / MAXIMIN, per design (one design for LHS, init_designs for MAXIMIN),
 *     per parameter p in order: a Fisher-Yates shuffle of the strata
 *     0..count-1 (for i = count-1 down to 1: swap i with next() mod (i+1)),
 *     then per sample i the jitter U = (next() >> 11) / 2^53; the value index
 *     floor((pi_p(i) + U) m_p / count) is computed exactly in integers.
 *     MAXIMIN keeps the first design with the largest minimum over pairs of
 *     sum_p (x_ip - x_jp)^2 (FP64, p in order, no fused multiply-add).
 *     The kept design's samples map to configurations in order; a restricted
 *     one, or a repeat of an earlier sample, is replaced (again in order) by
 *     r = next() mod N_valid, redrawn while already taken.
 * A space with n_init > 0 and init_mode LHS / MAXIMIN suggests exactly this
 * design (count = min(n_init, N_valid)) first, skipping configurations
 * already observed, then random unobserved ones until n_init valid
 * observations exist.  Errors: BO_ERR_ARG. */
int bo_initial_design(const bo_space_desc* desc, int32_t count, int64_t* idx_out);

typedef struct bo_space bo_space;   /* opaque, owned by the library */

/* Build the valid list, upload codes and value tables, and allocate the
 * resident state (observations, L^-1, beta, per-candidate buffers) for
 * n_max observations.  Synchronous.  BO_ERR_ARG for a bad descriptor, a
 * Cartesian product above 2^40 configurations, or (reduced precision) 2^32 - 1
 * or more valid configurations. */
int bo_space_create(const bo_space_desc* desc, bo_space** out);
/* Release every resource of the space (synchronizes its stream). */
int bo_space_destroy(bo_space* space);

int bo_valid_count(const bo_space* space, int64_t* out);
/* value_idx_out[p] = index into values[p] of configuration idx. */
int bo_decode(const bo_space* space, int64_t idx, int32_t* value_idx_out);

/* Record f(idx) = value.  A finite value is fitted: the FP64 L^-1 and beta
 * are extended on the device (asynchronous; a numeric failure of the update
 * is reported by the next bo_suggest / bo_sync).  A non-finite value marks
 * a runtime-invalid configuration: visited, never fitted (Sec. III-D).
 * BO_ERR_DUPLICATE if idx was observed before, BO_ERR_CAPACITY beyond n_max. */
int bo_observe(bo_space* space, int64_t idx, double value);

typedef struct bo_suggest_info {
  int64_t idx;        /* the suggested valid-list index                          */
  int32_t af;         /* BO_AF_EI / PI / LCB that picked it, -1 if random        */
  int32_t predicted;  /* 1 if it comes from a prediction pass                    */
  double mu;          /* posterior mean there (standardized units)               */
  double sigma;       /* posterior standard deviation there                      */
  double score;       /* acquisition value (larger is better)                    */
  double lambda;      /* exploration factor of the pass                          */
  double mean_var;    /* mean posterior variance over the scored candidates      */
  int64_t n_scored;   /* candidates scored by the pass                           */
} bo_suggest_info;

/* Next configuration to evaluate.  Runs a prediction pass (K* tiles,
 * contraction, row reduction, lambda, acquisition, masked top-k) unless the
 * current multi round still holds picks.  Synchronous; info may be NULL. */
int bo_suggest(bo_space* space, int64_t* idx_out, bo_suggest_info* info);

/* Posterior at valid-list indices [begin, begin + count) with the current
 * observations, copied to host arrays mu_out / var_out (standardized units,
 * var clamped at 0).  Synchronous.  For inspection and tests. */
int bo_predict(bo_space* space, int64_t begin, int64_t count, double* mu_out, double* var_out);

/* Host copy of the posterior the most recent prediction pass of this space
 * left on the device (bo_suggest, bo_predict, bo_batch_suggest, replay):
 * valid-list indices [begin, begin + count), no recomputation.  Synchronous. */
int bo_last_posterior(bo_space* space, int64_t begin, int64_t count, double* mu_out, double* var_out);

/* Enqueue the prediction kernels for the current observations on the
 * space's stream without waiting: the posterior of every candidate lands in
 * library-owned device memory.  For overlapping and for timing the
 * prediction kernels alone. */
int bo_predict_enqueue(bo_space* space);

/* Host copy of the FP64 L^-1 (n x n, row-major, lower triangular) and beta
 * (n); *n_out receives n.  Either array may be NULL.  Synchronous. */
int bo_get_factor(bo_space* space, double* linv_out, double* beta_out, int32_t* n_out);

/* Wait for the space's device work; returns a deferred update error, if any. */
int bo_sync(bo_space* space);

/* ---- device-resident replay (measurement) ----------------------------- */
typedef struct bo_pass_result {
  int32_t status;        /* BO_OK or a BO_ERR_* code of this pass              */
  int32_t n_fit;         /* valid observations fitted                         */
  int64_t n_scored;      /* candidates scored                                 */
  double sum_var;        /* sum of posterior variances over them              */
  double mean_var;
  double lambda;
  double mean_var_s;     /* contextual-variance baseline in use               */
  int64_t top_idx[3][3]; /* [af][rank] best valid-list indices (-1 if none)   */
  double top_score[3][3];
  double top_mu[3][3];
  double top_sigma[3][3];
} bo_pass_result;

/* Enqueue `steps` observe + predict + acquire passes on the space's stream
 * without host synchronization: step s observes (idx_host[s], y_host[s]) and
 * then scores every non-evaluated candidate with all three AFs (top-3 each).
 * The per-step results land in a library-owned device array; fetch them with
 * bo_replay_fetch.  Host arrays are read before return.  Selection state
 * (multi / advanced multi) is not touched. */
int bo_replay_enqueue(bo_space* space, const int64_t* idx_host, const double* y_host,
                      int32_t steps);
/* Synchronize and copy the results of the last bo_replay_enqueue. */
int bo_replay_fetch(bo_space* space, bo_pass_result* results_host, int32_t steps);

/* ---- batches of spaces --------------------------------------------------- */
/* Many sessions served together (paper Sec. III-G's suggest step, batched):
 * bo_batch_observe updates every space's surrogate in five kernel launches,
 * bo_batch_suggest runs the prediction passes of all spaces that need one in
 * a single persistent tensor-core launch (tiles of all spaces balanced over
 * the SMs) and one acquisition launch, replayed from a captured CUDA graph
 * once a batch shape repeats.  Per space the results equal bo_observe /
 * bo_suggest.  The spaces must share device, stream, precision and nu, and
 * stay alive while the batch exists; FP64 spaces are served one pass at a
 * time.  status_out[i] (optional) receives each space's BO_* code; the
 * return value is the first error or BO_OK. */
typedef struct bo_batch bo_batch;
int bo_batch_create(bo_space* const* spaces, int32_t count, bo_batch** out);
int bo_batch_destroy(bo_batch* batch);
/* idx[i] < 0 leaves space i unchanged; asynchronous on the spaces' stream. */
int bo_batch_observe(bo_batch* batch, const int64_t* idx, const double* values, int32_t* status_out);
/* idx_out[count]; info_out (optional) [count]. Synchronous. */
int bo_batch_suggest(bo_batch* batch, int64_t* idx_out, int32_t* status_out, bo_suggest_info* info_out);
/* As bo_batch_suggest for the spaces with want[i] != 0 only (others untouched, idx_out -1). */
int bo_batch_suggest_some(bo_batch* batch, const uint8_t* want, int64_t* idx_out, int32_t* status_out,
                          bo_suggest_info* info_out);
int bo_batch_launch_count(const bo_batch* batch, int64_t* out);

/* ---- autotuning of the tensor-core launch --------------------------------- */
/* Time candidate pipeline shapes of the prediction launch (depth of the K*
 * ring, slots of the L^-1 ring, resident L^-1 pieces or not) on the space's
 * or batch's current state, `reps` launches each with CUDA events, and keep
 * the fastest for every later launch of the same precision, Matern nu (3/2
 * or 5/2, Sec. III-B: separate kernel instantiations), dimension bucket and
 * padded observation count (per process).  The launches recompute the
 * current posterior (same values).  bo_batch_autotune times the batch's last
 * bo_batch_suggest pass (BO_ERR_STATE before one).  Reduced precision only. */
typedef struct bo_tune_result {
  int32_t stages_a;          /* chosen K* ring depth (0 = planner default)         */
  int32_t b_slots;           /* chosen L^-1 ring slots                             */
  int32_t b_resident;        /* 0 = resident pieces allowed, -1 = never            */
  int32_t tried;             /* shapes timed                                       */
  double best_ms;            /* median launch time of the chosen shape             */
  double default_ms;         /* median launch time of the planner's default        */
} bo_tune_result;
int bo_autotune(bo_space* space, int32_t reps, bo_tune_result* out);
int bo_batch_autotune(bo_batch* batch, int32_t reps, bo_tune_result* out);
/* The shape stored for the key of the space's next prediction launch (its
 * precision, nu, dimension bucket and padded observation count) in
 * stages_a / b_slots / b_resident (tried, best_ms, default_ms zero), or
 * BO_ERR_STATE when the autotuner has stored none for that key (or before the
 * first valid observation).  Host only, no device work. */
int bo_tuned_shape(const bo_space* space, bo_tune_result* out);

/* ---- serving: continuous batching of many sessions ----------------------- */
/* A request loop for many concurrent tuning sessions.  A worker thread takes,
 * in each iteration, at most one pending request of every admitted session
 * (requests that arrived while the previous iteration ran on the GPU join
 * this one), runs their observations as one batched update and their
 * suggestions as one batched prediction pass, and posts completions.
 * Sessions are admitted in arrival order while their device memory fits the
 * budget and a slot is free, and wait in a queue otherwise (closing a
 * session frees its memory and slot).  Each result equals what the session
 * would get alone. */
typedef struct bo_server bo_server;
typedef struct bo_server_config {
  size_t budget_bytes;       /* device memory the admitted sessions may hold       */
  int32_t max_sessions;      /* admitted sessions at most                          */
  int32_t pad;
  void* stream;              /* cudaStream_t of all device work                    */
  bo_alloc_fn alloc;         /* device memory provider of the sessions, or NULL    */
  bo_free_fn free;
  void* alloc_ctx;
} bo_server_config;

typedef struct bo_completion {
  uint64_t tag;              /* the request's tag                                  */
  int64_t session;
  int32_t status;            /* BO_* code of the request                           */
  int32_t observed;          /* 1 if the request's observation was applied         */
  int64_t idx;               /* suggested valid-list index (-1 if none asked)      */
  bo_suggest_info info;
  double t_submit, t_start, t_done;  /* seconds, server clock                     */
} bo_completion;

typedef struct bo_server_stats {
  int64_t admitted, queued, rejected, closed;
  int64_t requests, completed, iterations;
  int64_t candidates_scored;
  int64_t bytes_in_use;
} bo_server_stats;

int bo_server_create(const bo_server_config* config, bo_server** out);
/* Register a session (the descriptor's arrays are copied); *session_out
 * receives its id.  The descriptor is checked at once as bo_space_create
 * checks it (BO_ERR_ARG, nothing registered); BO_ERR_NOMEM if the session
 * could never fit the budget.  A session that later fails to be created on
 * the device completes its queued requests with that call's code.  The
 * descriptor's alloc / free / stream fields are ignored (the server's apply). */
int bo_server_open(bo_server* server, const bo_space_desc* desc, int64_t* session_out);
/* Queue a request: observe (idx, value) first if observe_idx >= 0, then
 * suggest unless suggest == 0 (an observe-only request, e.g. to warm-start). */
int bo_server_submit(bo_server* server, int64_t session, int64_t observe_idx, double observe_value,
                     int32_t suggest, uint64_t tag);
/* Up to max completions; waits up to wait_ms for the first one (0 = no wait). */
int bo_server_poll(bo_server* server, bo_completion* out, int32_t max, int32_t* n_out, int32_t wait_ms);
int bo_server_close(bo_server* server, int64_t session);
int bo_server_stats_get(bo_server* server, bo_server_stats* out);
/* Seconds on the server clock (the clock of bo_completion's times). */
double bo_server_now(const bo_server* server);
int bo_server_destroy(bo_server* server);

/* ---- acquisition without any allocation -------------------------------- */
/* No counterpart in the paper.  Some callers cannot allocate device memory
 * where they need a suggestion: code running inside a memory pool or arena
 * that must not grow, a process whose device memory is reserved up front by
 * another framework, or a real-time loop where an allocation (and the
 * synchronization it may bring) is not allowed.  For them this entry point
 * runs the acquisition and masked top-k (the same kernel bo_suggest uses) on
 * posterior arrays the caller already owns, and allocates nothing: its
 * per-block scratch is one fixed array of 147,520 bytes inside this library,
 * present on every device that loads it until the process exits.
 *
 * mu, var     device arrays [n_cand] of float (f64 = 0) or double (f64 = 1):
 *             posterior mean and variance, standardized units
 * visited     device array [ceil(n_cand / 32)] of uint32, bit i = candidate i
 *             evaluated (skipped)
 * params      host struct below, read before return
 * result      device bo_pass_result written by the kernel (status, lambda,
 *             mean variance, top-3 per acquisition function)
 * stream      cudaStream_t (NULL = legacy default stream)
 *
 * Returns BO_ERR_CAPACITY for n_cand > BO_NOALLOC_MAX_CAND, BO_ERR_ARG for
 * bad arguments (including an explore mode other than CV or CONST),
 * BO_ERR_NOT_POSITIVE when CV lacks positive f+ and mu_s, BO_ERR_CUDA if a
 * launch fails.  The scratch holds the partial top-k lists of the at most
 * 1,024 blocks one call launches; the blocks stride over the candidates, and
 * the cap bounds the work of one call (16 candidates per thread at the cap).
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress, no allocation) with that device current; make that
 * first call before any stream capture.  Every call shares the one array and
 * its last-block counter, which each call resets to zero first: calls whose
 * work overlaps on the GPU (other streams, other host threads) race. */
#define BO_NOALLOC_MAX_CAND 4194304

typedef struct bo_acq_params {
  int64_t n_cand;         /* candidates in mu / var / visited                     */
  int64_t n_unvisited;    /* valid, non-evaluated candidates (mean-variance count) */
  double sum_var;         /* sum of their variances                               */
  int32_t n_af;           /* active acquisition functions, 1..3                   */
  int32_t af[3];          /* BO_AF_EI / BO_AF_PI / BO_AF_LCB                      */
  int32_t explore;        /* BO_EXPLORE_CV or BO_EXPLORE_CONST                    */
  int32_t n_fit;          /* copied into the result                               */
  double lambda_const;    /* exploration factor when explore == CONST             */
  double fplus;           /* best observation, standardized units                 */
  double fplus_raw;       /* best observation, raw units (> 0 for CV)             */
  double mu_s_raw;        /* mean of the initial sample, raw units (> 0 for CV)    */
  double mean_var_s;      /* contextual-variance baseline; <= 0: this pass's mean */
} bo_acq_params;

int bo_acquire_noalloc(const void* mu, const void* var, const uint32_t* visited, int32_t f64,
                       const bo_acq_params* params, bo_pass_result* result, void* stream);

/* ---- self-test of the bounded device waits ------------------------------ */
/* Every wait inside this library's kernels (mbarrier phases of the prediction
 * kernel, grid barriers of the fused observation update) gives up after 2 s,
 * records BO_ERR_TIMEOUT and lets the kernel return, so that a stuck pipeline
 * surfaces as an error and the CUDA context stays usable.  This entry point
 * makes one wait of each kind run out on purpose (a barrier phase that nothing
 * completes; a grid barrier that one of two blocks never reaches) on the
 * current device and reports what each recorded: BO_ERR_TIMEOUT when the
 * mechanism works.  Takes about 4 s; allocates and frees 64 bytes of device
 * memory; synchronous.  Returns BO_ERR_ARG for null outputs, BO_ERR_CUDA if a
 * launch or copy fails. */
int bo_selftest_waits(int32_t* mbar_status, int32_t* grid_status);

/* Self-test of the exponential of the FP64 prediction pass (no counterpart in
 * the paper: the pass evaluates e^-t of the Matern covariance, Sec. III-B, with
 * its own table-driven reduction instead of a general exp).  For the n host
 * arguments t[i], writes that function's e^-t[i] to out[i] and CUDA's
 * exp(-t[i]) to ref[i] (both host arrays of n doubles), computed on the current
 * device.  Synchronous; allocates and frees 24 n bytes of device memory.
 * Returns BO_ERR_ARG for null arrays or n outside [1, 2^24], BO_ERR_CUDA if
 * a launch or copy fails. */
int bo_selftest_exp(const double* t, double* out, double* ref, int32_t n);

/* ---- arithmetic peaks of the current device (measurement) ----------------- */
/* Issue-rate probes of the units the prediction passes run on, for their
 * roofline denominators (no counterpart in the paper): register-resident
 * loops of 8 independent chains per thread, 64 warps per SM on every SM, best
 * of 5 launches timed with CUDA events on the legacy default stream.
 *   fp64_fma_tflops    DFMA (the FP64 pass), 2 flops each
 *   fp32_fma_tflops    scalar FFMA, 2 flops each
 *   fp32x2_fma_tflops  packed fma.rn.f32x2 (the K* producers), 4 flops each
 *   mufu_gops          ex2.approx + rsqrt.approx (the Matern evaluation), 1 op each
 * Synchronous, about 0.2 s; allocates and frees 256 bytes of device memory;
 * changes no clock or other device setting.  Returns BO_ERR_ARG for a null
 * output, BO_ERR_CUDA without a device or if a launch fails. */
typedef struct bo_alu_peaks {
  double fp64_fma_tflops;
  double fp32_fma_tflops;
  double fp32x2_fma_tflops;
  double mufu_gops;
  int32_t sms;
  int32_t pad;
} bo_alu_peaks;
int bo_measure_alu_peaks(bo_alu_peaks* out);

/* Number of kernel launches this library has issued on the space so far. */
int bo_launch_count(const bo_space* space, int64_t* out);

/* Thread-local message of the last error ("" if none). */
const char* bo_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BO_SUGGEST_H */
