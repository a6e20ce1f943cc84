// Internal layout of the Cox CCD library (not part of the ABI).
//
// The method (arXiv 2310.16238 §2.6-§2.7) turns every risk-set sum into a stratum-segmented
// reverse scan. All model forms are mapped onto one "risk sequence" of M positions:
//   * right-censored rows: position = row (rows sorted by stratum, then time), M = n_rows;
//   * counting-process rows (start, stop]: every row appears twice in its stratum's
//     sequence, ordered by time -- an entry at `stop` holding +exp(eta) and an exit at
//     `start` holding -exp(eta) -- so the suffix sum from the first position with time >= t
//     is exactly the at-risk sum at t (rows with stop >= t minus rows with start >= t),
//     M = 2 n_rows.
// A tie group g (a (stratum, time) with events) reads the suffix sum at its read position
// head_pos[g]; strata are segments (a scan never crosses a stratum's last position).
#pragma once
#include <cstdint>

// Phase tracing of the resident and incremental kernels (timestamps per step, printed to stderr
// when COXGB_PHASE_TRACE=<steps> is set at run time) exists only in builds compiled with
// -DCOXGB_TRACE; the library's default build has none of it.
#ifdef COXGB_TRACE
#define COX_TRACE_ON 1
#else
#define COX_TRACE_ON 0
#endif

namespace coxgb {

constexpr int kThreads = 256;        // CTA size of the scan kernel
constexpr int kHeadCap = 1024;       // max tie-group read positions per tile
constexpr uint32_t kExitBit = 0x80000000u;
constexpr uint32_t kPosMask = 0x7fffffffu;

// Prepared, read-only data of one data set (shared by every fit on it).
struct DevData {
  int64_t M;              // risk-sequence length
  int64_t n_rows;
  int32_t p, T, G, K;     // columns, tiles, tie groups, strata
  int32_t tile;           // nominal positions per tile
  int32_t binary;         // 1: every stored x is 1
  int32_t counting;       // 1: counting-process sequence (exit positions carry -exp)
  double sum_d;           // total number of events (for the exp shift in the log-likelihood)
  const int64_t *col_ptr; // [p+1] position-space CSC
  const uint32_t *idx;    // [nnz_pos] position | kExitBit for exit positions
  const double *val;      // [nnz_pos] or nullptr
  const int32_t *col_tile;// [p*(T+1)] offset from col_ptr[j] of column j's first entry in tile t
  const int32_t *tile_lo; // [T+1] first position of each tile, tile_lo[T] = M
  const int32_t *head_pos;// [G] read positions, ascending
  const int32_t *head_d;  // [G] events per tie group
  const int32_t *tile_g;  // [T+1] first tie group of each tile
  const int32_t *cut_pos; // [K] last position of each stratum, ascending
  const int32_t *tile_k;  // [T+1] first stratum whose last position is in tile t
  const double *dX;       // [p] delta' X_j
  const uint32_t *exit_bits; // [ceil(M/32)] exit positions (counting process) or nullptr
  const uint32_t *head_bits; // [ceil(M/32) + 128] bitmap of the tie-group read positions
  const uint32_t *cut_bits;  // [ceil(M/32) + 128] bitmap of the stratum ends
};

// Mutable control block of one fit (written by the last CTA of each launch).
struct FitCtl {
  int32_t j;              // coordinate evaluated by the next launch
  int32_t sweep;          // completed sweeps
  int32_t state;          // kRunning / kConverged / kMaxed / kError
  int32_t need_ll;        // next launch also evaluates the log-likelihood
  int32_t pend_j;         // column of the update the next launch applies first (-1: none)
  int32_t error;          // COX_E_* raised on the device (0: none)
  double pend_db;         // its step
  double obj_prev, obj, loglik;
  uint32_t epoch;         // launch counter (tags look-back statuses)
  uint32_t done_tiles;    // tiles finished in the current launch
  uint32_t s0c_tag;       // FP32C chunked kernel: equals epoch when the tie groups' cached S0 holds for
                          // this launch's eta and the launch may take the cached-S0 path (0: never)
  uint32_t fast_no;       // chunks of the current launch that rule that path out for the next one
  int64_t coord_updates;
  double out_g1, out_g2;  // EVAL mode result
  double out_ll;          // LL mode result (shard mode: the tie groups' sum d log S0)
  double out_bdx;         // shard mode: beta'dX over the shard's rows (when the log-likelihood is due)
};

enum : int32_t { kRunning = 0, kConverged = 1, kMaxed = 2, kError = 3 };

// One fit: pointers into its data and state (read-only during a launch).
struct DevFit {
  const DevData *d;       // device copy of the data descriptor
  FitCtl *ctl;
  double *eta;            // [M] linear predictor per position
  void *v;                // [M_pad] +-exp(eta - shift), double or float
  double *beta;           // [p]
  double *trust;          // [p]
  const uint8_t *penalize;// [p] or nullptr
  uint32_t *tstat;        // [T] look-back status words
  double *tval;           // [T*6] published tile values: aggregate (0..2), inclusive (3..5)
  double *part;           // [T*3] tile partials (G1, G2, LL)
  double *out_S0, *out_S1;// [G] optional per-group sums (diagnostics)
  double *gout;           // [2p] EVAL mode: g'(beta_j), g''(beta_j) per column
  float *hscr;            // [6G] FP32C chunked kernel: compensated local sums (S0, S1[, S2]) of tie
                          // groups whose risk set reaches past their chunk, kept until its carry arrives;
                          // after a fit's launch each group's S0 slot holds its final S0 (the cached-S0 path)
  const void *vmap;       // FP32C: device copy of the tensor map (CUtensorMap, 128 bytes) that views v
                          // as rows of 32 floats, for the chunked kernel's tile copies
  // copies of data pointers the chunked kernel reads first (one dependent load fewer than via d)
  const int32_t *tile_lo, *tile_g, *col_tile, *head_d;
  const int64_t *col_ptr;
  const uint32_t *idx, *cut_bits, *head_bits;
  const double *val;
  int32_t T, p;
  int32_t penalty, max_sweeps;
  double lambda, l2_var, tol, shift;
};

// Persistent-launch control: ticket counter, work-list size, and (for the device-driven
// sweep loop) the number of fits still running and a hard bound on further launches.
struct LaunchCtl {
  uint32_t ticket;
  uint32_t exited;
  int32_t n_items;
  int32_t active;         // running fits in the work list; 0 ends a conditional sweep loop
  int64_t budget;         // launches left before a conditional sweep loop is ended regardless
  int32_t error;          // COX_E_TIMEOUT when a CTA's internal pipeline wait gave up (0: none)
  int32_t pad_;
  const double *ext;      // shard mode: sums (NV) of the last stratum beyond the data's end (null: none)
};

// Limit, in SM clocks, of every bounded device-side wait (look-backs, exchanges, pipeline
// barriers): the process-wide value set with cox_debug_set_wait_limit, else kSpinBudget.
long long wait_limit();

// kModeShard: one rank's part of a sharded fit -- column j's (G1, G2) and, when ctl->need_ll, the
// log-likelihood terms over the shard's rows, the last stratum completed by lc->ext; no step.
enum : int32_t { kModeFit = 0, kModeEval = 1, kModeLL = 2, kModeShard = 3 };

// One work item of the streaming kernel: tile t of fit f, covering risk positions [lo, hi) and
// tie groups [ga, gb).
struct WorkItem {
  int32_t f, t, lo, hi, ga, gb, pad_[2];
};

// One work item of the FP32C chunked kernel (ccd_chunk.cu), the same size as a WorkItem: chunk c
// (tiles [ta, tb)) of fit f, whose work list holds its nc chunks in descending order.
struct ChunkItem {
  int32_t f, c, ta, tb, nc;
  int32_t lo_last;        // first position of the chunk's last tile (tile tb - 1)
  int32_t fast_ok;        // the fit's chunks are within the cached-S0 path's limits (strata, tie groups)
  int32_t pad_;
};
static_assert(sizeof(ChunkItem) == sizeof(WorkItem), "chunk items share the work-list buffer");

// Arguments of the resident kernel (ccd_resident.cu), passed by value.
struct ResParams {
  DevFit F;               // the fit (its d pointer is not used)
  DevData D;              // the data descriptor
  const int32_t *tile_lo, *tile_g, *tile_k, *col_tile;   // resident tile plan: one tile per CTA
  uint64_t *tagg;         // [6T] epoch-tagged tile aggregates (2 values + stratum-end flag)
  uint64_t *tpart;        // [2][6T] epoch-tagged tile partials, double-buffered by step parity
  int64_t max_steps;      // coordinate steps this launch may take
  uint64_t *trace;        // optional [2][trace_steps][8] phase timestamps (ns) of the first and last CTA
  int64_t trace_steps;
  long long spin;         // limit of each device-side wait, SM clocks (wait_limit())
};

struct dw;   // double-word float (dw.cuh)

// Words of one step record of the incremental kernel: 6 tagged 8-byte payloads (G1, G2, H1, R, I
// as double-words, LL in FP64), two 8-byte words each.
constexpr int kIncRecWords = 12;

// One fit of the incremental kernel (ccd_incr.cu): passed by value for a single fit, or as a
// device array with a map from each CTA to (fit, tile of that fit) when one launch runs several.
struct IncParams {
  DevFit F;               // the fit (its d pointer is not used)
  DevData D;              // the data descriptor
  int32_t T, pad_;        // tiles (CTAs) of this fit
  const int32_t *tile_lo, *tile_g, *tile_k, *col_tile;   // incremental tile plan: one tile per CTA
  uint64_t *trec;         // [2][C readers][C writers][kIncRecWords] epoch-tagged step records (each
                          // CTA writes its record into every CTA's inbox), double-buffered by parity
  uint64_t *tref;         // [C][4] epoch-tagged head sums of the dense refresh
  double *bcopy;          // [C][2p] each CTA's copy of beta and the trust half-widths
  dw *vdw;                // [M] v per position as a double-word (the kernel's working copy)
  int64_t max_steps;      // coordinate steps this launch may take
  const uint8_t *halt;    // [p] columns too dense for the lists: the launch stops before them (null: none)
  uint64_t *trace;        // optional [trace_steps][C][24] phase timestamps (ns) and counters
  int64_t trace_steps;
  long long spin;         // limit of each device-side wait, SM clocks (wait_limit())
};

// One rank's part of a sharded fit (shard.cu).
int launch_shard_head(const DevFit *fit, int32_t j, double *out, void *stream);
int launch_shard_step(const DevFit *fit, const double *dxg, int32_t j, const double *tot, int32_t need_ll, int32_t sweep,
                      int32_t max_sweeps, double *out, void *stream);
int launch_shard_open_end(DevData *d, int32_t *tile_k, void *stream);

// Count of kernels launched by the library (every launcher adds to it).
void count_launches(int64_t n);

// Host-visible launchers (ccd.cu). The streaming kernel assigns work items to CTAs statically, so
// `grid` must not exceed ccd_max_grid(precision, valued) (every CTA resident at once).
// `cond`: handle of the enclosing conditional WHILE graph node (0 = none). The kernel sets it
// to 0 once no fit in the work list is running or the launch budget is spent.
int launch_ccd(int precision, const DevFit *fits, const WorkItem *items, LaunchCtl *lc, int grid, int mode,
               int j_eval, int valued, void *stream, unsigned long long cond = 0);
int ccd_max_grid(int precision, int valued);
int ccd_tile(int precision);
// The FP32C launches above run the chunked kernel (ccd_chunk.cu); its work items are ChunkItems.
int launch_chunk(const DevFit *fits, const ChunkItem *items, LaunchCtl *lc, int grid, int mode, int j_eval, int valued,
                 void *stream, unsigned long long cond);
int chunk_max_grid(int valued);
// Encodes (on the host) the tensor map of a fit's v for the chunked kernel's tile copies: n_floats
// floats from v (16-byte aligned) as rows of 32, one copy = 128 rows, 128-byte swizzle. out: 128
// bytes, 64-byte aligned. Returns COX_OK or COX_E_CUDA.
int chunk_encode_vmap(void *v, int64_t n_floats, void *out);
constexpr int kChunkTile = 4096;     // positions per tile of the chunked kernel
constexpr int kChunkMaxTiles = 64;   // tiles per chunk
// Limits per chunk of the chunked kernel's cached-S0 path (shared memory): column entries, stratum
// ends, tie groups.
constexpr int kChunksPerCtaDefault = 1;   // chunks per resident CTA of a plan (cox_set_chunk_plan)
constexpr int kChunkFastE = 1536;
constexpr int kChunkFastCuts = 256;
constexpr int kChunkFastH = 4096;
int launch_column_update(int precision, const DevFit *fit_dev, int32_t j, double db, int64_t nnz_j, void *stream);
int launch_fill_v(int precision, const DevFit *fit_dev, int64_t M, const uint32_t *exit_bits, void *stream);

// Resident kernel (ccd_resident.cu): positions per CTA, head capacity per CTA, largest
// cooperative grid (0 when unsupported), launch.
int res_tile(int precision);
int res_head_cap();
int res_max_grid(int precision);
int launch_resident(int precision, const ResParams &prm, int grid, void *stream);

// Incremental kernel (ccd_incr.cu): tie groups, column entries and positions one CTA holds,
// largest cooperative grid (0 when unsupported), launch.
// Incremental kernel configurations: 0 = one tie group per thread (1,024 per CTA), lists of
// 1,024 entries, 65,536 positions; 1 = group-dense data (4,096 groups, 512 entries, 32,768
// positions per CTA).
int inc_group_cap(int variant);
int inc_list_cap(int variant);
int inc_pos_cap(int variant);
int inc_max_grid(int precision, int variant);
int launch_incr(int precision, const IncParams &prm, int grid, void *stream, int variant);
int launch_incr_multi(int precision, const IncParams *prms, const int2 *cta_map, int grid, void *stream);

}  // namespace coxgb
