/*
 * cox.h -- C ABI of the GB300 (sm_103a) library for regularized stratified and
 * time-varying Cox proportional-hazards fits by cyclic coordinate descent.
 *
 * Method: Yang, Schuemie & Suchard, "Massive parallelization of the stratified and
 * time-varying Cox models" (arXiv 2310.16238).
 *   - model: stratified partial likelihood, §2.1 eq. (strat_l); time-varying covariates as
 *     counting-process rows, §2.2 eq. (time_cov_l); time-varying coefficients reduce to
 *     time-varying covariates, §2.3;
 *   - optimizer: cyclic coordinate descent with the 1-D Newton step eq. (newton), the
 *     trust region and the L1 directional-derivative rule, §2.4;
 *   - per-coordinate gradient/Hessian eqs. (strat_g), (strat_h) as stratum-segmented
 *     reverse scans of exp(X beta) and X_j exp(X beta), §2.6-§2.7 eqs. (parallel_g)-(parallel_xb).
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: COX_OK (0), a warning (> 0) or an error (< 0).
 *     No exception or longjmp crosses the ABI. cox_last_error() gives the message of the
 *     last failing call on a handle (or, with NULL, of the last failing call on this thread).
 *   - Pointers to arrays may be host or device memory; the library detects which with
 *     cudaPointerGetAttributes. Output arrays are written in their own memory space.
 *   - cox_create copies everything it needs; the caller may free its inputs afterwards.
 *     The handle owns its device memory until cox_destroy.
 *   - All device work runs on the stream given in cox_options.stream (NULL: the legacy
 *     default stream). Calls return after their work on that stream has completed.
 *   - One handle must not be used from two threads at once. Distinct handles are independent.
 */
#ifndef COX_H
#define COX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define COX_OK 0
#define COX_W_NOT_CONVERGED 1   /* max_sweeps reached before the tolerance */
#define COX_E_INVALID (-1)      /* bad argument or malformed data */
#define COX_E_UNSORTED (-2)     /* rows not sorted by (stratum, stop) */
#define COX_E_OOM (-3)          /* device allocation failed */
#define COX_E_CUDA (-4)         /* a CUDA runtime call failed */
#define COX_E_TIMEOUT (-5)      /* a bounded device-side wait gave up */
#define COX_E_ADMISSION (-6)    /* serving: request can never fit the memory budget */
#define COX_E_RANGE (-7)        /* FP32 path: |eta - shift| left the exp range of float */
#define COX_E_NOT_FOUND (-8)    /* serving: unknown request id */
#define COX_E_BUSY (-9)         /* serving: result not ready yet (poll again) */

enum { COX_PEN_NONE = 0, COX_PEN_L1 = 1, COX_PEN_L2 = 2 };
enum {
  COX_FP64 = 0,   /* FP64 exp, scans, ratios, step and log-likelihood */
  COX_FP32C = 1   /* FP32 exp and compensated (two-sum) FP32 tile scans; FP64 tile carries,
                     gradient/Hessian accumulation, Newton step and log-likelihood */
};

/* ---------------------------------------------------------------- data
 * Rows are observations (right-censored) or counting-process intervals (start, stop].
 * They MUST be sorted by (stratum ascending, stop ascending); ties in any order.
 *   stop     int32[n_rows]  event or censoring time, integer days (paper §2.2: discrete time)
 *   start    int32[n_rows]  NULL for right-censored data; otherwise the interval start,
 *                           start < stop. A row is at risk at time t iff start < t <= stop.
 *   event    uint8[n_rows]  1 if the row ends with an event at `stop`, else 0
 *   stratum  int32[n_rows]  NULL: one stratum. Strata ids only need to be sorted.
 *   col_ptr  int64[p+1]     CSC column pointers into row_idx / val, col_ptr[0] = 0
 *   row_idx  int32[nnz]     row of each nonzero, strictly ascending within a column
 *   val      double[nnz]    NULL: binary X (every stored entry is 1)
 * Limits: n_rows < 2^30 (counting-process data use two sequence positions per row). */
typedef struct {
  int64_t n_rows;
  int32_t p;
  int32_t reserved;
  const int32_t *stop;
  const int32_t *start;
  const uint8_t *event;
  const int32_t *stratum;
  const int64_t *col_ptr;
  const int32_t *row_idx;
  const double *val;
} cox_data;

/* ---------------------------------------------------------------- options
 *   penalty    COX_PEN_NONE | COX_PEN_L1 (gamma * sum |beta_j|, §2.1) | COX_PEN_L2
 *              (sum beta_j^2 / (2 l2_var), Gaussian prior)
 *   lambda     L1 weight gamma
 *   l2_var     L2 prior variance
 *   penalize   uint8[p] (host or device), NULL: every coordinate penalized. 0 exempts a
 *              coordinate (e.g. a treatment covariate, §3.2)
 *   tol        convergence: |obj_s - obj_{s-1}| <= tol * |obj_s| after sweep s, on the
 *              penalized objective obj = -loglik + penalty
 *   max_sweeps sweep limit (COX_W_NOT_CONVERGED when reached)
 *   precision  COX_FP64 | COX_FP32C
 *   stream     cudaStream_t (NULL = default stream)
 *   tile       positions per tile of the streaming kernel, 0 = library default; a multiple
 *              of 32 in [1024, 4096 (FP64) or 8192 (FP32C)] otherwise
 *   engine     COX_ENGINE_AUTO: the incremental kernel when the data qualify (binary X and,
 *              per co-resident CTA, at most 1024 tie groups, 65,536 risk positions and 1024
 *              entries of any column, or 4096 groups, 32,768 positions and 512 entries; a
 *              few columns too dense for those lists are stepped by the resident kernel),
 *              else the resident kernel when the data qualify (binary X and the whole risk
 *              sequence fits the GPU's shared memory), else streaming. COX_ENGINE_STREAM /
 *              _RESIDENT / _INCR force one; RESIDENT and INCR fail with COX_E_INVALID when
 *              the data do not qualify. The incremental kernel keeps each tie group's
 *              risk-set sum S0 resident and updates it from the changed positions (cost per
 *              coordinate O(groups + nnz_j), not O(n)), rebuilding it from a full scan at the
 *              start of every sweep; its sums and ratios are double-word FP32 (about 48
 *              significant bits), eta, beta and the step FP64, for either precision. */
typedef struct {
  int32_t penalty;
  int32_t precision;
  double lambda;
  double l2_var;
  const uint8_t *penalize;
  double tol;
  int32_t max_sweeps;
  int32_t tile;
  void *stream;
  int32_t engine;
  int32_t reserved;
} cox_options;

enum { COX_ENGINE_AUTO = 0, COX_ENGINE_STREAM = 1, COX_ENGINE_RESIDENT = 2, COX_ENGINE_INCR = 3 };

typedef struct {
  int32_t sweeps;          /* full sweeps over the p coordinates */
  int32_t converged;       /* 1 when the tolerance was met */
  int64_t coord_updates;   /* coordinate evaluations (sweeps * p) */
  double loglik;           /* unpenalized log partial likelihood at beta_out */
  double objective;        /* -loglik + penalty at beta_out */
  int32_t status;          /* same as the return code */
  int32_t engine;          /* the kernel that ran the sweeps: COX_ENGINE_STREAM / _RESIDENT / _INCR
                              (0 when no sweep ran) */
  int64_t step_launches;   /* coordinate-step kernel launches issued by the sweep loop */
  double sweep_ms;         /* CUDA-event time of the sweep loop on the fit's stream */
  double wait_ms;          /* serving only: submission to admission (device memory granted) */
  double total_ms;         /* serving only: submission to result ready */
} cox_fit_info;

typedef struct cox_handle cox_handle;

/* Device memory allocator used for every buffer the library owns (NULL: cudaMalloc /
 * cudaFree). `alloc` returns a device pointer (or NULL on failure) and must be callable
 * from any thread. Set it before creating handles; it applies process-wide. */
typedef void *(*cox_alloc_fn)(size_t bytes, void *ctx);
typedef void (*cox_free_fn)(void *ptr, size_t bytes, void *ctx);
int cox_set_allocator(cox_alloc_fn alloc, cox_free_fn release, void *ctx);

/* Validate and prepare `data` on the device (sort check, strata, tie groups, delta'X,
 * tile plan; §2.7) and allocate the per-fit state. On success *out owns everything.
 * Errors: COX_E_INVALID, COX_E_UNSORTED, COX_E_OOM, COX_E_CUDA. */
int cox_create(const cox_data *data, const cox_options *opts, cox_handle **out);

/* Replace the options of an existing handle (penalty, tolerances, precision, stream).
 * Keeps the prepared data; the next cox_fit starts from its beta0. */
int cox_set_options(cox_handle *h, const cox_options *opts);

/* Cyclic coordinate descent (§2.4) from beta0 (p doubles, NULL = zeros) until the
 * tolerance or max_sweeps; writes beta_out (p doubles) and *info (may be NULL).
 * Returns COX_OK, COX_W_NOT_CONVERGED or an error. */
int cox_fit(cox_handle *h, const double *beta0, double *beta_out, cox_fit_info *info);

/* Unpenalized log partial likelihood (eq. strat_l / time_cov_l) at beta (p doubles). */
int cox_loglik(cox_handle *h, const double *beta, double *loglik_out);

/* Unpenalized gradient and Hessian diagonal of -loglik at beta (eqs. strat_g, strat_h):
 * grad[p] and, unless NULL, hess_diag[p]. */
int cox_gradient(cox_handle *h, const double *beta, double *grad, double *hess_diag);

/* Risk-set sums at every tie group g (sorted by stratum, then time) for column j at beta:
 * S0[g] = sum_{r in R(t_g)} exp(x_r'beta), S1[g] = sum x_rj exp(x_r'beta) (j < 0: S1 = 0).
 * *n_groups receives G; S0 / S1 may be NULL to query G. Diagnostic entry point. */
int cox_risk_sums(cox_handle *h, const double *beta, int32_t j, double *S0, double *S1, int64_t *n_groups);

/* Integer metadata built by cox_create (for verification): every output may be NULL.
 *   n_groups, n_strata   G and K
 *   group_stratum[G], group_time[G], group_events[G], group_at_risk[G] (rows at risk)
 *   strata_start[K+1]   first row of each stratum, strata_start[K] = n_rows */
int cox_metadata(cox_handle *h, int64_t *n_groups, int64_t *n_strata, int32_t *group_stratum,
                 int32_t *group_time, int32_t *group_events, int64_t *group_at_risk, int64_t *strata_start);

/* delta'X_j for every column (p doubles): the first term of eq. (parallel_g). */
int cox_dx(cox_handle *h, double *dx);

/* Release everything the handle owns. NULL is ignored. */
void cox_destroy(cox_handle *h);

/* Message of the last error on `h` (NULL: the calling thread's last error). Never NULL. */
const char *cox_last_error(const cox_handle *h);

/* ---------------------------------------------------------------- batching
 * Run the fits of n handles together: one persistent launch per coordinate step advances
 * every unfinished fit by one coordinate (each fit on its own coordinate and sweep),
 * replayed from a captured CUDA graph. The handles must share one precision; their
 * options' streams are ignored in favour of the first handle's. beta0[i] may be NULL
 * (or beta0 itself NULL); beta_out[i] receives p_i doubles; info[i] may be NULL.
 * Returns the worst status over the fits. */
int cox_batch_fit(cox_handle *const *h, int32_t n, const double *const *beta0, double *const *beta_out,
                  cox_fit_info *info);

/* New handle on the same prepared data as `src` (shared, reference counted) with its own
 * fit state and options: many fits of one data set (penalty grids) without re-preparing. */
int cox_clone(const cox_handle *src, const cox_options *opts, cox_handle **out);

/* ---------------------------------------------------------------- time-split view
 * §2.2 (time-varying covariates on discrete intervals) and §2.3 (time-varying
 * coefficients): cut days t_1 < ... < t_C split follow-up time into the C + 1 intervals
 * I_0 = (-inf, t_1), I_k = [t_k, t_{k+1}), I_C = [t_C, +inf) (integer days). A Cox model whose
 * covariates or coefficients are constant on each interval has the partial likelihood of a
 * model stratified on the intervals (§2.2), and a coefficient that steps at the cuts is a
 * covariate split into one copy per interval (§2.3). The view is that stratified model:
 *
 *   rows     stratum (s, k) holds every input row of stratum s that can be at risk at a time
 *            in I_k: stop >= t_k and, for counting-process rows, start + 1 < t_{k+1}. Such a
 *            row enters with stop' = min(stop, t_{k+1}) (stop when k = C), start' = start,
 *            event' = event when stop lies in I_k, else 0. The paper's augmented copy also
 *            keeps the rows that cannot be at risk in I_k; they add nothing to the likelihood
 *            and are left out. Stratum ids: s_index * (C + 1) + k (s_index = 0-based rank of s).
 *   columns  the input columns in order, each column listed in tvc_cols replaced by C + 1
 *            consecutive columns (the column on I_0, ..., on I_C); the others unchanged. The
 *            handle has p_view = p + n_tvc * C columns (cox_split_columns): options.penalize,
 *            beta0 and beta_out are in view columns.
 *
 * The view is built by device kernels straight from the caller's arrays (host or device);
 * no augmented copy is formed on the host or asked of the caller. Errors: COX_E_INVALID
 * (cuts not strictly ascending, tvc_cols not strictly ascending in [0, p), sizes beyond the
 * limits: view rows < 2^30, view nonzeros < 2^32), plus those of cox_create. */
typedef struct {
  int32_t n_cuts;           /* C >= 1 */
  int32_t n_tvc;            /* columns with one coefficient per interval, 0..p */
  const int32_t *cuts;      /* host, C strictly ascending days */
  const int32_t *tvc_cols;  /* host, n_tvc strictly ascending column indices (NULL when 0) */
} cox_split;

/* p_view of a split of a p-column data set. */
int cox_split_columns(int32_t p, const cox_split *split, int32_t *p_view);

/* cox_create on the time-split view of `data`. The view's arrays live only during the call. */
int cox_create_split(const cox_data *data, const cox_split *split, const cox_options *opts, cox_handle **out);

/* ---------------------------------------------------------------- cross-validated penalty path
 * K-fold cross-validation along a penalty path, the way the paper picks its L1 weight
 * (10-fold CV, §3.2 and §3.3). Training set k = the rows whose fold id is not k (built on the
 * device); the rows of one subject (counting-process rows) must share a fold id. The path is
 * walked in the given order: at each value every training fit and the full-data fit start from
 * their own fit at the previous value (warm start; zeros at the first), and the K + 1 fits of a
 * value run together as one batch (cox_batch_fit). For L1 the path values are the weight gamma
 * (opts.lambda), for L2 the prior variance sigma^2 (opts.l2_var); the other options apply to
 * every fit. Score: the cross-validated partial log-likelihood (P. Verweij and H. van
 * Houwelingen, Stat. Med. 12, 1993),
 *     cvl = sum_k [ l(beta_-k) - l_-k(beta_-k) ],
 * l the full data's log partial likelihood, l_-k training set k's, beta_-k the fit on training
 * set k: the held-out rows' contribution with their risk sets formed on all the data.
 *
 *   cvl        n_path doubles (host)
 *   beta_path  n_path x p doubles (host, row-major; NULL to skip): the full-data fits
 *   info       n_path x (K + 1) (host; NULL to skip): per value, the K training fits then the
 *              full-data fit
 *   best       index of the largest cvl (NULL to skip)
 * Returns the worst status over the fits. Errors: COX_E_INVALID (K < 2, n_path < 1, penalty
 * NONE, fold ids outside [0, K), a path value that is negative (L1) or not positive (L2)), plus
 * those of cox_create and cox_batch_fit. */
typedef struct {
  int32_t n_folds;          /* K >= 2 */
  int32_t n_path;           /* >= 1 */
  const int32_t *fold;      /* host or device, n_rows fold ids in [0, K) */
  const double *path;       /* host, n_path penalty values */
  const cox_split *split;   /* NULL, or every fit (training sets and full data) on its time-split
                               view (cox_create_split); fold ids stay per input row, so a row's
                               interval copies share its fold. beta_path has p_view columns. */
} cox_cv;

int cox_cv_path(const cox_data *data, const cox_options *opts, const cox_cv *cv, double *cvl, double *beta_path,
                cox_fit_info *info, int32_t *best);

/* Bytes of device memory a handle for `data` would hold (for admission control). */
int cox_footprint(const cox_data *data, const cox_options *opts, size_t *bytes);

/* Number of CUDA kernels this library has launched in this process (graph replays count
 * every kernel node). For measurement; never decreases. */
int64_t cox_launch_count(void);

/* ---------------------------------------------------------------- one fit sharded by stratum
 * The stratified partial likelihood is a sum over strata (§2.1 eq. strat_l) and every risk-set sum
 * a suffix sum within its stratum (§2.6-§2.7), so one fit's rows, sorted by (stratum, stop), can be
 * cut into contiguous shards, one per rank (GPU). A cut never splits a tie group (equal stratum and
 * stop with an event); a stratum may be split (right-censored data). Each rank makes a handle on its
 * own rows with cox_create (COX_FP64; options as for the whole fit) and, with the collectives done by
 * the caller, every rank runs per coordinate j = 0 .. p-1 of every sweep, in lock step:
 *   cox_shard_head     applies the previous step's update at the shard's entries of that column,
 *                      then head[0..2] = the sums of exp(eta), x_j exp(eta), x_j^2 exp(eta) from the
 *                      shard's first row to its first stratum end (head[3] = 0);
 *   (all-gather of the head sums; the carry of a rank whose last stratum continues is the sum of the
 *    next ranks' head sums that continue that stratum, up to the first rank where it ends)
 *   cox_shard_partial  out = (G1, G2, sum d log S0, beta'dX) of column j over the shard's tie groups,
 *                      the last stratum completed by `carry` (3 doubles; ignored unless set up with
 *                      last_continues); the last two only when need_ll (the first coordinate of a
 *                      sweep), else 0;
 *   (all-reduce of the four sums)
 *   cox_shard_step     from the summed `tot`: when need_ll the log-likelihood beta'dX - sum d log S0
 *                      and the convergence test of the penalized objective (sweep = completed sweeps,
 *                      stop when |obj_s - obj_{s-1}| <= tol |obj_s| or sweep >= max_sweeps), else /
 *                      then the coordinate step (§2.4) with g' = -dX_j + G1 (dX the whole fit's) and
 *                      g'' = G2, the same on every rank. *state: 0 running, 1 converged, 2 sweep
 *                      limit; *loglik when need_ll.
 * cox_shard_setup, once before the first coordinate: dx_global = delta'X of the whole fit (p
 * doubles, the sum of the ranks' cox_dx), last_continues = 1 when the shard's last stratum continues
 * on the next rank; it resets the fit state to beta = 0. cox_shard_beta copies the coefficients
 * (identical on every rank). A handle set up for sharding serves only these calls. */
int cox_shard_setup(cox_handle *h, const double *dx_global, int32_t last_continues);
int cox_shard_head(cox_handle *h, int32_t j, double *head);
int cox_shard_partial(cox_handle *h, int32_t j, const double *carry, int32_t need_ll, double *out);
int cox_shard_step(cox_handle *h, int32_t j, const double *tot, int32_t need_ll, int32_t sweep, int32_t max_sweeps,
                   int32_t *state, double *loglik);
int cox_shard_beta(cox_handle *h, double *beta);

/* Failure handling. Every device-side wait in the kernels (a tile waiting for the sums of the
 * tiles to its right, the CTAs of one fit exchanging their step records, the stages of the
 * streaming pipeline) gives up after a bounded number of SM clocks; the call then returns
 * COX_E_TIMEOUT and the kernel exits, so no wait can hang the GPU. This sets that bound for every
 * kernel launched afterwards, process-wide (clocks <= 0: the default, 4e9 clocks, about 2 s);
 * graphs already captured keep the bound they were captured with. A bound too short for a
 * kernel's exchanges exercises the failure path without any fault: the calls fail with
 * COX_E_TIMEOUT and later calls with the default bound succeed. Returns COX_OK. */
int cox_debug_set_wait_limit(long long clocks);

/* Chunk length of the FP32C streaming kernel. The kernel streams each fit's risk sequence as
 * chunks of consecutive tiles (4,096 positions per tile), one chunk per CTA, with one look-back
 * between chunks; by default the library picks the smallest chunk length for which every resident
 * CTA gets at most one chunk. This forces `tiles` tiles per chunk (1..64; 0 restores the automatic
 * choice) for every work list built afterwards, process-wide; it changes the summation order only,
 * not the method. Meant for tests of multi-tile chunks on small data. Returns COX_OK, or
 * COX_E_INVALID for a value outside 0..64. */
int cox_debug_set_chunk_tiles(int32_t tiles);

/* Chunks per resident CTA in the FP32C streaming kernel's plans (1..8; 0 restores the library's
 * default). With more than one, a CTA that finishes its chunk takes the next one of the work list,
 * so that cheap chunks (fits whose step reads the tie groups' cached S0) free their CTAs for the
 * others. A schedule parameter of the plan (chosen by the autotuner for batches): it changes the
 * summation order only, not the method. Applies to work lists built afterwards, process-wide.
 * Returns COX_OK, or COX_E_INVALID for a value outside 0..8. */
int cox_set_chunk_plan(int32_t chunks_per_cta);

/* The FP32C streaming kernel's cached-S0 path. A coordinate step of a fit whose eta has not changed
 * since its previous step (that step's update was 0, as for every coefficient an L1 penalty keeps
 * at 0) needs no new risk-set sums S0 at its tie groups (eq. parallel_d: the sums of exp(eta) are
 * those of the previous step); the kernel keeps them from one step to the next and then computes
 * only column j's S1 (S2) from the column's entries; cox_gradient's evaluation launches (every
 * column at one eta) read them too. On by default; `enable` = 0 turns it off for
 * work lists built afterwards, process-wide (for tests that compare the two paths). Returns COX_OK. */
int cox_debug_set_cached_s0(int32_t enable);

/* ---------------------------------------------------------------- primitives
 * Segmented inclusive scan with the flag-value operator of §2.6 ("Efficient parallel
 * segmented-scan on GPUs"): out[i] = sum of a[k] for k from the last index h <= i with
 * head_flags[h] != 0 (or from 0) up to i. a, head_flags, out: device arrays of n elements
 * (out may alias a). Runs on `stream` (cudaStream_t, NULL = default) and returns after it
 * completed. Scratch for the single-pass look-back (32 bytes per 4096 elements) is
 * taken from the library allocator for the duration of the call.
 * Errors: COX_E_INVALID (null/host pointers, n < 0), COX_E_OOM, COX_E_CUDA, COX_E_TIMEOUT. */
int cox_segscan(const double *a, const uint8_t *head_flags, int64_t n, double *out, void *stream);

/* Same result as cox_segscan, but the call allocates no device memory. No counterpart in the
 * paper: it exists for callers that cannot allocate device memory while they run -- a host
 * program whose own memory pool must own every device byte, a real-time loop that cannot risk
 * an allocator call blocking or failing mid-run, a process held to a fixed memory budget.
 * Its scratch is one static device array of 131,088 bytes that every GPU loading this library
 * holds until the process exits; n is therefore limited to 16,777,216 values (COX_E_INVALID
 * beyond that). The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, and looks it up again if the device's
 * context has been recreated since (cudaDeviceReset); make that first call before any stream
 * capture. All calls share the array and clear the parts that must start at zero, so calls
 * whose work overlaps on the GPU race with each other: issue them one at a time (same stream,
 * or synchronized). Other arguments, errors and stream behaviour as cox_segscan. */
int cox_segscan_noalloc(const double *a, const uint8_t *head_flags, int64_t n, double *out, void *stream);

/* ---------------------------------------------------------------- serving
 * Continuous batching of fit requests. Requests of any size and layout are submitted from any
 * thread; a preparation thread admits them in arrival order while their device footprint
 * (cox_footprint) fits the memory budget and the in-flight limit, prepares them on its own
 * stream (overlapping the fits in flight), and a run thread advances every in-flight fit by one
 * coordinate step per persistent launch (each fit on its own coordinate and sweep), replayed
 * from a CUDA graph; between replays finished fits are retired (their memory returned) and newly
 * prepared ones join. Each fit's state (eta, exp(eta), beta, scan state) stays on the device
 * from admission to retirement. */
typedef struct cox_server cox_server;
typedef struct {
  size_t memory_budget;    /* bytes of device memory for admitted requests; 0 = 80 % of free memory */
  int32_t max_active;      /* fits prepared or in flight at once; 0 = 256 */
  int32_t precision;       /* COX_FP64 | COX_FP32C for every request */
  int32_t steps_per_replay;/* coordinate steps per graph replay; 0 = 64 */
  int32_t reserved;
} cox_server_options;
typedef struct {
  int64_t submitted, completed, failed;
  int32_t queued, preparing, running, done_unpolled;
  size_t bytes_in_use, memory_budget;
  int64_t replays, step_launches;
} cox_server_stats;

int cox_server_create(const cox_server_options *opts, cox_server **out);
/* Queue one fit; `data` arrays may be host or device memory and are copied before return.
 * opts->stream and opts->precision are ignored (the server's apply). *request_id identifies it.
 * Errors: COX_E_INVALID (bad arguments), COX_E_ADMISSION (footprint above the whole budget). */
int cox_server_submit(cox_server *s, const cox_data *data, const cox_options *opts, uint64_t *request_id);
/* Result of a finished request: beta_out (p doubles, host or device) and *info (may be NULL);
 * returns the fit's status and forgets the request. COX_E_BUSY while it is queued or running,
 * COX_E_NOT_FOUND for an unknown or already collected id. */
int cox_server_poll(cox_server *s, uint64_t request_id, double *beta_out, cox_fit_info *info);
/* As cox_server_poll, but blocks up to timeout_s seconds (< 0: forever) for the result. */
int cox_server_wait(cox_server *s, uint64_t request_id, double timeout_s, double *beta_out, cox_fit_info *info);
/* Cancel a queued or running request (its memory is returned at the next replay boundary). */
int cox_server_cancel(cox_server *s, uint64_t request_id);
int cox_server_stats_get(cox_server *s, cox_server_stats *out);
/* Stops both threads (requests still in flight are abandoned) and releases everything. */
void cox_server_destroy(cox_server *s);

#ifdef __cplusplus
}
#endif
#endif /* COX_H */
