// C ABI of the Cox CCD library: handles, fit state, the CUDA-graph sweep loop, evaluations
// and batched fits. The arithmetic lives in ccd.cu (coordinate steps) and prep.cu (data
// preparation); this file only orchestrates launches and copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "cox.h"
#include "cox_internal.h"
#include "prep.h"

using namespace coxgb;

namespace {

thread_local std::string t_last_error = "no error";

struct SharedData {
  Prepared prep;
  DevData *d_desc = nullptr;   // device copy of prep.desc
  int precision = COX_FP64;
  std::atomic<int> refs{1};
};

void release_shared(SharedData *s) {
  if (s && s->refs.fetch_sub(1) == 1) {
    if (s->d_desc) dev_free(s->d_desc, sizeof(DevData));
    delete s;
  }
}

}  // namespace

int coxgb::set_last_error(int code, const char *msg) {
  t_last_error = msg ? msg : "error";
  return code;
}

struct cox_handle {
  SharedData *sd = nullptr;
  cox_options opts{};
  BufferSet bufs;
  DevFit hfit{};
  DevFit *dfit = nullptr;
  FitCtl *ctl = nullptr;
  LaunchCtl *lc = nullptr;
  WorkItem *items = nullptr;
  int n_items = 0;
  int nck = 0;                 // FP32C: chunks of this fit in its own work list
  int grid = 0;
  int valued = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_len = 0;
  long long graph_spin = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  FitCtl *h_ctl = nullptr;     // pinned readback
  LaunchCtl *h_lc = nullptr;   // pinned readback of the launch control (same allocation)
  uint8_t *penalize = nullptr; // device copy of the penalty mask
  double *gout = nullptr;
  double *S0 = nullptr, *S1 = nullptr;
  // resident-kernel scratch (allocated when the data qualify)
  uint64_t *r_tagg = nullptr, *r_tpart = nullptr;
  // incremental-kernel scratch (allocated when the data qualify)
  uint64_t *i_trec = nullptr, *i_tref = nullptr;
  double *i_bcopy = nullptr;
  dw *i_vdw = nullptr;
  // one rank's part of a sharded fit (cox_shard_*): the global delta'X, small result buffers, the
  // carry of a last stratum that continues on the next rank
  double *sh_dx = nullptr, *sh_buf = nullptr, *sh_ext = nullptr;
  int sh_open = 0;
  std::string err = "no error";
};

namespace {

constexpr int kSweepBody = 64;   // coordinate-step launches per iteration of the device-driven loop

int fail(cox_handle *h, int code, const std::string &msg) {
  t_last_error = msg;
  if (h) h->err = msg;
  return code;
}

int cuda_fail(cox_handle *h, const char *what) {
  cudaError_t e = cudaGetLastError();
  return fail(h, COX_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

const DevData &D(const cox_handle *h) { return h->sd->prep.desc; }

int resolve_stream(cox_handle *h) {
  if (h->opts.stream) {
    h->stream = static_cast<cudaStream_t>(h->opts.stream);
    return COX_OK;
  }
  if (!h->own_stream && cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess)
    return cuda_fail(h, "stream create");
  h->stream = h->own_stream;
  return COX_OK;
}

int check_options(const cox_options *o) {
  if (!o) return COX_OK;
  if (o->engine < COX_ENGINE_AUTO || o->engine > COX_ENGINE_INCR) return COX_E_INVALID;
  if (o->penalty < COX_PEN_NONE || o->penalty > COX_PEN_L2) return COX_E_INVALID;
  if (o->precision != COX_FP64 && o->precision != COX_FP32C) return COX_E_INVALID;
  if (o->penalty == COX_PEN_L1 && !(o->lambda >= 0.0)) return COX_E_INVALID;
  if (o->penalty == COX_PEN_L2 && !(o->l2_var > 0.0)) return COX_E_INVALID;
  if (!(o->tol >= 0.0) || o->max_sweeps < 0) return COX_E_INVALID;
  return COX_OK;
}

cox_options default_options() {
  cox_options o{};
  o.penalty = COX_PEN_NONE;
  o.precision = COX_FP64;
  o.l2_var = 1.0;
  o.tol = 1e-8;
  o.max_sweeps = 1000;
  return o;
}

// Work item of the streaming kernel: tile t of the handle's data as fit f of a work list.
WorkItem work_item(const cox_handle *h, int f, int t) {
  const std::vector<int32_t> &lo = h->sd->prep.h_tile_lo, &g = h->sd->prep.h_tile_g;
  return WorkItem{f, t, lo[size_t(t)], lo[size_t(t) + 1], g[size_t(t)], g[size_t(t) + 1], {0, 0}};
}

// Tiles per chunk forced for every plan (0: automatic), set by cox_debug_set_chunk_tiles.
std::atomic<int> g_chunk_tiles{0};
// Chunks per resident CTA of the chunked kernel's plans (cox_set_chunk_plan): the kernel hands out
// chunks past the first one per CTA in work-list order.
std::atomic<int> g_chunks_per_cta{kChunksPerCtaDefault};
// The chunked kernel's cached-S0 path admitted in plans built afterwards (cox_debug_set_cached_s0).
std::atomic<int> g_cached_s0{1};

// Chunk plan of the FP32C chunked kernel for fits of T[i] tiles sharing `slots` resident CTAs: the
// smallest chunk length C (tiles, at most kChunkMaxTiles) for which the fits' chunk counts
// ceil(T[i] / C) add up to at most `slots`, so one launch gives every CTA at most one chunk (the
// kernel assigns chunks to CTAs statically). Returns each fit's chunk count.
std::vector<int> plan_chunks(const std::vector<int64_t> &T, int slots) {
  slots *= std::max(1, g_chunks_per_cta.load());
  auto total = [&](int64_t C) {
    int64_t s = 0;
    for (int64_t t : T) s += (t + C - 1) / C;
    return s;
  };
  int64_t C = g_chunk_tiles.load();
  if (C <= 0) {
    int64_t lo = 1, hi = kChunkMaxTiles;
    if (total(hi) <= slots) {
      while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (total(mid) <= int64_t(slots)) hi = mid;
        else lo = mid + 1;
      }
    }
    C = hi;
  }
  C = std::max<int64_t>(1, std::min<int64_t>(C, kChunkMaxTiles));
  std::vector<int> n(T.size());
  for (size_t i = 0; i < T.size(); ++i) n[i] = int(T[i] > 0 ? (T[i] + C - 1) / C : 0);
  return n;
}

// Work items of fit f of a work list in the order the look-back needs (later positions first):
// the tiles of the FP64 kernel, or `nck` chunks of nearly equal tile counts for the FP32C kernel.
std::vector<WorkItem> fit_items(const cox_handle *h, int f, int nck) {
  std::vector<WorkItem> out;
  const int64_t T = D(h).T;
  if (h->sd->precision == COX_FP32C) {
    const std::vector<int32_t> &lo = h->sd->prep.h_tile_lo, &tg = h->sd->prep.h_tile_g;
    // the cached-S0 path's limits hold for every chunk of this plan (strata, tie groups per chunk)
    int fast_ok = g_cached_s0.load() != 0 && D(h).K <= kChunkFastCuts;
    for (int c = 0; c < nck && fast_ok; ++c) {
      const int ta = int(int64_t(c) * T / nck), tb = int(int64_t(c + 1) * T / nck);
      fast_ok = tg[size_t(tb)] - tg[size_t(ta)] <= kChunkFastH;
    }
    for (int c = nck - 1; c >= 0; --c) {
      const int ta = int(int64_t(c) * T / nck), tb = int(int64_t(c + 1) * T / nck);
      const ChunkItem ci{f, c, ta, tb, nck, lo[size_t(tb - 1)], fast_ok, 0};
      WorkItem w;
      std::memcpy(&w, &ci, sizeof(w));
      out.push_back(w);
    }
  } else {
    for (int64_t t = T - 1; t >= 0; --t) out.push_back(work_item(h, f, int(t)));
  }
  return out;
}

// Several fits' lists interleaved item by item (each fit's own order kept).
std::vector<WorkItem> interleave(const std::vector<std::vector<WorkItem>> &lists) {
  std::vector<WorkItem> out;
  size_t most = 0;
  for (const auto &l : lists) most = std::max(most, l.size());
  for (size_t k = 0; k < most; ++k)
    for (const auto &l : lists)
      if (k < l.size()) out.push_back(l[k]);
  return out;
}

// Clear a fit's published look-back words (the chunked kernel's tags are 4 bits: a word left from
// an earlier chunk layout must never read as current).
int clear_lookback(cox_handle *h, cudaStream_t s) {
  const int64_t T = D(h).T;
  if (T > 0 && cudaMemsetAsync(h->hfit.tval, 0, T * 6 * sizeof(double), s) != cudaSuccess) return COX_E_CUDA;
  return COX_OK;
}

// Allocate the per-fit state of a handle on its (shared) data.
int alloc_fit_state(cox_handle *h) {
  const DevData &d = D(h);
  const int64_t M = d.M, T = d.T, p = d.p, G = d.G;
  const int tile_k = ccd_tile(h->sd->precision);
  const size_t sv = h->sd->precision == COX_FP32C ? sizeof(float) : sizeof(double);
  BufferSet &B = h->bufs;
  h->hfit = DevFit{};
  h->hfit.d = h->sd->d_desc;
  {
    const DevData &hd = h->sd->prep.desc;
    h->hfit.tile_lo = hd.tile_lo;
    h->hfit.tile_g = hd.tile_g;
    h->hfit.col_tile = hd.col_tile;
    h->hfit.head_d = hd.head_d;
    h->hfit.col_ptr = hd.col_ptr;
    h->hfit.idx = hd.idx;
    h->hfit.cut_bits = hd.cut_bits;
    h->hfit.head_bits = hd.head_bits;
    h->hfit.val = hd.val;
    h->hfit.T = hd.T;
    h->hfit.p = hd.p;
  }
  h->ctl = static_cast<FitCtl *>(B.get(sizeof(FitCtl)));
  h->lc = static_cast<LaunchCtl *>(B.get(sizeof(LaunchCtl)));
  h->dfit = static_cast<DevFit *>(B.get(sizeof(DevFit)));
  h->items = static_cast<WorkItem *>(B.get(std::max<int64_t>(T, 1) * sizeof(WorkItem)));
  h->hfit.eta = static_cast<double *>(B.get(std::max<int64_t>(M, 1) * sizeof(double)));
  h->hfit.v = B.get((M + tile_k + 64) * sv);
  h->hfit.beta = static_cast<double *>(B.get(std::max<int64_t>(p, 1) * sizeof(double)));
  h->hfit.trust = static_cast<double *>(B.get(std::max<int64_t>(p, 1) * sizeof(double)));
  h->hfit.tstat = static_cast<uint32_t *>(B.get(std::max<int64_t>(T, 1) * sizeof(uint32_t)));
  h->hfit.tval = static_cast<double *>(B.get(std::max<int64_t>(T, 1) * 6 * sizeof(double)));
  h->hfit.part = static_cast<double *>(B.get(std::max<int64_t>(T, 1) * 3 * sizeof(double)));
  h->gout = static_cast<double *>(B.get(std::max<int64_t>(p, 1) * 2 * sizeof(double)));
  h->S0 = static_cast<double *>(B.get(std::max<int64_t>(G, 1) * sizeof(double)));
  h->S1 = static_cast<double *>(B.get(std::max<int64_t>(G, 1) * sizeof(double)));
  h->penalize = static_cast<uint8_t *>(B.get(std::max<int64_t>(p, 1)));
  if (h->sd->precision == COX_FP32C) h->hfit.hscr = static_cast<float *>(B.get(std::max<int64_t>(G, 1) * 6 * sizeof(float)));
  if (!h->ctl || !h->lc || !h->dfit || !h->items || !h->hfit.eta || !h->hfit.v || !h->hfit.beta || !h->hfit.trust ||
      !h->hfit.tstat || !h->hfit.tval || !h->hfit.part || !h->gout || !h->S0 || !h->S1 || !h->penalize ||
      (h->sd->precision == COX_FP32C && !h->hfit.hscr))
    return fail(h, COX_E_OOM, "device allocation failed for the fit state");
  h->hfit.ctl = h->ctl;
  if (h->sd->precision == COX_FP32C) {   // the tensor map of v for the chunked kernel's tile copies
    alignas(64) unsigned char map[128];
    void *dmap = B.get(sizeof(map));
    if (!dmap) return fail(h, COX_E_OOM, "device allocation failed for the fit state");
    if (chunk_encode_vmap(h->hfit.v, M + tile_k + 64, map)) return fail(h, COX_E_CUDA, "tensor map of v");
    if (cudaMemcpy(dmap, map, sizeof(map), cudaMemcpyHostToDevice) != cudaSuccess) return cuda_fail(h, "tensor map copy");
    h->hfit.vmap = dmap;
  }
  if (const int RT = h->sd->prep.res_T) {
    h->r_tagg = static_cast<uint64_t *>(B.get(6 * RT * sizeof(uint64_t)));
    h->r_tpart = static_cast<uint64_t *>(B.get(12 * RT * sizeof(uint64_t)));
    if (!h->r_tagg || !h->r_tpart)
      return fail(h, COX_E_OOM, "device allocation failed for the resident state");
  }
  if (const int IT = h->sd->prep.inc_T) {
    h->i_trec = static_cast<uint64_t *>(B.get(2 * kIncRecWords * int64_t(IT) * IT * sizeof(uint64_t)));
    h->i_tref = static_cast<uint64_t *>(B.get(4 * int64_t(IT) * sizeof(uint64_t)));
    h->i_bcopy = static_cast<double *>(B.get(std::max<int64_t>(2 * p * IT, 1) * sizeof(double)));
    h->i_vdw = static_cast<dw *>(B.get(std::max<int64_t>(M, 1) * 2 * sizeof(float)));
    if (!h->i_trec || !h->i_tref || !h->i_bcopy || !h->i_vdw)
      return fail(h, COX_E_OOM, "device allocation failed for the incremental state");
  }
  void *pin = nullptr;
  if (cudaMallocHost(&pin, sizeof(FitCtl) + sizeof(LaunchCtl)) != cudaSuccess) return cuda_fail(h, "pinned alloc");
  h->h_ctl = static_cast<FitCtl *>(pin);
  h->h_lc = reinterpret_cast<LaunchCtl *>(static_cast<unsigned char *>(pin) + sizeof(FitCtl));
  *h->h_lc = LaunchCtl{};
  // zero the padded tail of v once (positions >= M are read as whole 16-byte chunks)
  if (cudaMemsetAsync(h->hfit.v, 0, (M + tile_k + 64) * sv, h->stream) != cudaSuccess) return cuda_fail(h, "memset");
  h->valued = d.val != nullptr;
  const int mg = ccd_max_grid(h->sd->precision, h->valued);
  if (mg <= 0) return cuda_fail(h, "kernel attributes");
  h->nck = plan_chunks({T}, mg)[0];   // a fit alone: at most one chunk per resident CTA
  std::vector<WorkItem> it = fit_items(h, 0, h->nck);
  h->n_items = int(it.size());
  if (!it.empty() &&
      cudaMemcpyAsync(h->items, it.data(), it.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return cuda_fail(h, "items copy");
  LaunchCtl lc{0u, 0u, int32_t(h->n_items), 1, 0};
  if (cudaMemcpyAsync(h->lc, &lc, sizeof(lc), cudaMemcpyHostToDevice, h->stream) != cudaSuccess) return cuda_fail(h, "lc copy");
  h->grid = int(std::max<int64_t>(1, std::min<int64_t>(h->n_items, mg)));
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, "state init");
  return COX_OK;
}

int apply_options(cox_handle *h, const cox_options *o) {
  h->opts = o ? *o : default_options();
  h->hfit.penalty = h->opts.penalty;
  h->hfit.lambda = h->opts.lambda;
  h->hfit.l2_var = h->opts.l2_var;
  h->hfit.tol = h->opts.tol;
  h->hfit.max_sweeps = h->opts.max_sweeps;
  h->hfit.shift = 0.0;
  h->hfit.penalize = nullptr;
  int rc = resolve_stream(h);
  if (rc) return rc;
  const int64_t p = D(h).p;
  if (h->opts.penalize && p > 0) {
    if (cudaMemcpyAsync(h->penalize, h->opts.penalize, p, cudaMemcpyDefault, h->stream) != cudaSuccess)
      return cuda_fail(h, "penalize copy");
    h->hfit.penalize = h->penalize;
    h->opts.penalize = h->penalize;   // the caller's array may go away; clones copy from here
  }
  if (cudaMemcpyAsync(h->dfit, &h->hfit, sizeof(DevFit), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return cuda_fail(h, "fit descriptor copy");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, "options");
  return COX_OK;
}

int push_desc(cox_handle *h) {
  if (cudaMemcpyAsync(h->dfit, &h->hfit, sizeof(DevFit), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return cuda_fail(h, "fit descriptor copy");
  return COX_OK;
}

// Reset the fit to coefficients beta0 (host or device, NULL = 0): eta = X beta0 accumulated
// column by column, v = +-exp(eta - shift), trust half-widths 1, control block at sweep 0.
int init_state(cox_handle *h, const double *beta0) {
  const DevData &d = D(h);
  const int64_t p = d.p;
  cudaStream_t s = h->stream;
  std::vector<double> hb(static_cast<size_t>(std::max<int64_t>(p, 1)), 0.0);
  if (beta0 && p > 0 && cudaMemcpy(hb.data(), beta0, p * sizeof(double), cudaMemcpyDefault) != cudaSuccess)
    return cuda_fail(h, "beta0 read");
  for (int64_t j = 0; j < p; ++j)
    if (!std::isfinite(hb[j])) return fail(h, COX_E_INVALID, "beta0 must be finite");
  if (p > 0 && cudaMemcpyAsync(h->hfit.beta, hb.data(), p * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return cuda_fail(h, "beta copy");
  std::vector<double> ones(static_cast<size_t>(std::max<int64_t>(p, 1)), 1.0);
  if (p > 0 && cudaMemcpyAsync(h->hfit.trust, ones.data(), p * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return cuda_fail(h, "trust copy");
  if (d.T > 0 && cudaMemsetAsync(h->hfit.tstat, 0, d.T * sizeof(uint32_t), s) != cudaSuccess) return cuda_fail(h, "memset");
  if (clear_lookback(h, s)) return cuda_fail(h, "memset");
  if (cudaMemsetAsync(&h->lc->error, 0, sizeof(int32_t), s) != cudaSuccess) return cuda_fail(h, "memset");
  FitCtl c{};
  c.j = 0;
  c.state = kRunning;
  c.need_ll = 1;
  c.pend_j = -1;
  c.epoch = 1u;
  if (cudaMemcpyAsync(h->ctl, &c, sizeof(c), cudaMemcpyHostToDevice, s) != cudaSuccess) return cuda_fail(h, "ctl copy");
  int rc = push_desc(h);
  if (rc) return rc;
  if ((rc = launch_fill_v(h->sd->precision, h->dfit, d.M, d.exit_bits, s))) return cuda_fail(h, "fill");
  const auto &cp = h->sd->prep.h_col_ptr;
  for (int64_t j = 0; j < p; ++j)
    if (hb[j] != 0.0)
      if ((rc = launch_column_update(h->sd->precision, h->dfit, int32_t(j), hb[j], cp[j + 1] - cp[j], s)))
        return cuda_fail(h, "warm start");
  // *beta0 must stay valid until the copies above completed
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail(h, "state init");
  return COX_OK;
}

int read_ctl(cox_handle *h) {
  if (cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(FitCtl), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(h->h_lc, h->lc, sizeof(LaunchCtl), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return cuda_fail(h, "ctl read");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, "kernel execution");
  return COX_OK;
}

int launch_mode(cox_handle *h, int mode, int j) {
  if (D(h).T == 0) return COX_OK;
  int rc = launch_ccd(h->sd->precision, h->dfit, h->items, h->lc, h->grid, mode, j, h->valued, h->stream);
  return rc ? cuda_fail(h, "ccd launch") : COX_OK;
}

int device_error(cox_handle *h) {
  const int e = h->h_ctl->error ? h->h_ctl->error : h->h_lc->error;
  if (e == COX_E_TIMEOUT) return fail(h, COX_E_TIMEOUT, "a device-side wait exceeded its bound");
  if (e == COX_E_RANGE) return fail(h, COX_E_RANGE, "|eta - shift| left the float exp range (use COX_FP64)");
  if (e) return fail(h, e, "device error");
  return COX_OK;
}

// The sweep loop as one graph: a conditional WHILE node whose body is `len` coordinate-step
// launches. The kernel ends the loop (sets the condition to 0) when the fit has stopped or the
// launch budget in LaunchCtl is spent, so a whole fit is one cudaGraphLaunch.
int build_graph(cox_handle *h, int len) {
  if (h->graph && h->graph_len == len && h->graph_spin == wait_limit()) return COX_OK;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return cuda_fail(h, "graph create");
  cudaGraphConditionalHandle cond;
  if (cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault) != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(h, "conditional handle");
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(h, "conditional node");
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(h, "capture");
  }
  int rc = COX_OK;
  for (int i = 0; i < len && !rc; ++i)
    rc = launch_ccd(h->sd->precision, h->dfit, h->items, h->lc, h->grid, kModeFit, 0, h->valued, h->stream, cond);
  cudaGraph_t captured = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(h->stream, &captured);
  if (rc || ec != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(h, "capture launch");
  }
  const cudaError_t e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(h, "graph instantiate");
  h->graph_len = len;
  h->graph_spin = wait_limit();   // the wait bound is captured into the graph's launches
  return COX_OK;
}

int copy_out(cox_handle *h, double *dst, const double *src, int64_t count) {
  if (count <= 0) return COX_OK;
  if (cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDefault, h->stream) != cudaSuccess)
    return cuda_fail(h, "result copy");
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, "result copy");
  return COX_OK;
}

// The whole fit in one cooperative launch of the resident kernel (state already initialized).
ResParams res_params(cox_handle *h) {
  const Prepared &P = h->sd->prep;
  ResParams prm{};
  prm.F = h->hfit;
  prm.D = D(h);
  prm.tile_lo = P.res_tile_lo;
  prm.tile_g = P.res_tile_g;
  prm.tile_k = P.res_tile_k;
  prm.col_tile = P.res_col_tile;
  prm.tagg = h->r_tagg;
  prm.tpart = h->r_tpart;
  prm.max_steps = (int64_t(h->opts.max_sweeps) + 2) * D(h).p + 2;
  prm.spin = wait_limit();
  return prm;
}

int fit_resident(cox_handle *h, double *beta_out, cox_fit_info *info) {
  const DevData &d = D(h);
  const Prepared &P = h->sd->prep;
  const int RT = P.res_T;
  cudaStream_t s = h->stream;
  // tag 0 never matches: records start at epoch 1
  if (cudaMemsetAsync(h->r_tagg, 0, 6 * RT * sizeof(uint64_t), s) != cudaSuccess ||
      cudaMemsetAsync(h->r_tpart, 0, 12 * RT * sizeof(uint64_t), s) != cudaSuccess)
    return cuda_fail(h, "memset");
  ResParams prm = res_params(h);
#if COX_TRACE_ON
  // phase trace of the first steps (COXGB_PHASE_TRACE=<steps>), printed to stderr
  const char *tr_env = std::getenv("COXGB_PHASE_TRACE");
  const int64_t tr_steps = tr_env ? std::max<int64_t>(0, std::atoll(tr_env)) : 0;
  BufferSet trbuf;
  if (tr_steps > 0) {
    prm.trace = static_cast<uint64_t *>(trbuf.get(tr_steps * RT * 8 * sizeof(uint64_t)));
    prm.trace_steps = prm.trace ? tr_steps : 0;
    if (prm.trace) cudaMemsetAsync(prm.trace, 0, tr_steps * RT * 8 * sizeof(uint64_t), s);
  }
#endif
  if (!h->ev0 && (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess))
    return cuda_fail(h, "event create");
  cudaEventRecord(h->ev0, s);
  if (launch_resident(h->sd->precision, prm, RT, s)) return cuda_fail(h, "resident launch");
  cudaEventRecord(h->ev1, s);
  int rc;
  if ((rc = read_ctl(h))) return rc;
#if COX_TRACE_ON
  if (prm.trace_steps > 0) {
    // per CTA: mean phase times and the time from the earliest step start to its partial publish
    std::vector<uint64_t> tr(size_t(prm.trace_steps * RT * 8));
    cudaMemcpy(tr.data(), prm.trace, tr.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost);
    std::vector<int32_t> rlo(RT + 1), rg(RT + 1);
    cudaMemcpy(rlo.data(), P.res_tile_lo, (RT + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost);
    cudaMemcpy(rg.data(), P.res_tile_g, (RT + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost);
    std::vector<double> pub(RT, 0.0), ph(5 * RT, 0.0), stepm(RT, 0.0);
    int64_t n = 0;
    for (int64_t k = 1; k < prm.trace_steps; ++k) {
      uint64_t t0 = ~0ull;
      bool ok = true;
      for (int c = 0; c < RT; ++c) {
        const uint64_t *r = &tr[size_t((k * RT + c) * 8)];
        if (!r[0] || !r[5]) ok = false;
        t0 = std::min(t0, r[0]);
      }
      if (!ok) continue;
      for (int c = 0; c < RT; ++c) {
        const uint64_t *r = &tr[size_t((k * RT + c) * 8)];
        pub[c] += double(r[3] - t0);
        stepm[c] += double(r[5] - r[0]);
        for (int q = 0; q < 5; ++q) ph[5 * c + q] += double(r[q + 1] - r[q]);
      }
      ++n;
    }
    std::vector<int> order(RT);
    for (int c = 0; c < RT; ++c) order[c] = c;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return pub[a] > pub[b]; });
    std::fprintf(stderr, "[phase trace] %lld steps x %d CTAs; slowest to publish (ns after the first start):\n",
                 (long long)n, RT);
    for (int q = 0; q < std::min(RT, 6) && n; ++q) {
      const int c = order[q];
      std::fprintf(stderr, "  CTA %d positions %d groups %d: publish %.0f | scan %.0f carry %.0f ratios %.0f gather %.0f step %.0f\n",
                   c, rlo[c + 1] - rlo[c], rg[c + 1] - rg[c], pub[c] / n, ph[5 * c] / n, ph[5 * c + 1] / n,
                   ph[5 * c + 2] / n, ph[5 * c + 3] / n, ph[5 * c + 4] / n);
    }
    const int c = order[RT - 1];
    if (n) std::fprintf(stderr, "  fastest CTA %d positions %d groups %d: publish %.0f, step %.0f\n", c, rlo[c + 1] - rlo[c],
                        rg[c + 1] - rg[c], pub[c] / n, stepm[c] / n);
  }
#endif
  if ((rc = device_error(h))) return rc;
  const FitCtl &c = *h->h_ctl;
  if (c.state == kRunning) return fail(h, COX_E_INVALID, "cox_fit: the resident kernel stopped before the fit did");
  rc = c.state == kConverged ? COX_OK : COX_W_NOT_CONVERGED;
  if (info) {
    info->sweeps = c.sweep;
    info->converged = c.state == kConverged;
    info->coord_updates = c.coord_updates;
    info->loglik = c.loglik;
    info->objective = c.obj;
    info->status = rc;
    info->engine = COX_ENGINE_RESIDENT;
    info->step_launches = 1;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    info->sweep_ms = ms;
  }
  const int rc2 = copy_out(h, beta_out, h->hfit.beta, d.p);
  return rc2 ? rc2 : rc;
}

// Kernel arguments of a fit on the incremental kernel: the full plan (one fit over the whole GPU)
// or the compact plan (the fewest tiles; a batch runs several fits per launch).
IncParams incr_params(cox_handle *h, bool compact) {
  const Prepared &P = h->sd->prep;
  IncParams prm{};
  prm.F = h->hfit;
  prm.D = D(h);
  prm.T = compact ? P.cinc_T : P.inc_T;
  prm.tile_lo = compact ? P.cinc_tile_lo : P.inc_tile_lo;
  prm.tile_g = compact ? P.cinc_tile_g : P.inc_tile_g;
  prm.tile_k = compact ? P.cinc_tile_k : P.inc_tile_k;
  prm.col_tile = compact ? P.cinc_col_tile : P.inc_col_tile;
  prm.trec = h->i_trec;
  prm.tref = h->i_tref;
  prm.bcopy = h->i_bcopy;
  prm.vdw = h->i_vdw;
  prm.max_steps = (int64_t(h->opts.max_sweeps) + 2) * D(h).p + 2;
  prm.spin = wait_limit();
  return prm;
}

// The fit's result from its control block (already read into h_ctl).
int incr_result(cox_handle *h, double *beta_out, cox_fit_info *info, float ms, int64_t launches) {
  int rc;
  if ((rc = device_error(h))) return rc;
  const FitCtl &c = *h->h_ctl;
  if (c.state == kRunning) return fail(h, COX_E_INVALID, "cox_fit: the incremental kernel stopped before the fit did");
  rc = c.state == kConverged ? COX_OK : COX_W_NOT_CONVERGED;
  if (info) {
    info->sweeps = c.sweep;
    info->converged = c.state == kConverged;
    info->coord_updates = c.coord_updates;
    info->loglik = c.loglik;
    info->objective = c.obj;
    info->status = rc;
    info->engine = COX_ENGINE_INCR;
    info->step_launches = launches;
    info->sweep_ms = ms;
  }
  const int rc2 = copy_out(h, beta_out, h->hfit.beta, D(h).p);
  return rc2 ? rc2 : rc;
}

// Many fits on the incremental kernel: each fit runs on its compact plan's CTAs, fits packed
// largest first into waves of at most one CTA per SM, one cooperative launch per wave (the CTAs
// of a fit exchange records only among themselves).
int batch_incr(cox_handle *const *hs, int32_t n, const double *const *beta0, double *const *beta_out, cox_fit_info *info) {
  const int precision = hs[0]->sd->precision;
  cudaStream_t s = hs[0]->stream;
  const int grid = inc_max_grid(precision, 0);
  std::vector<cudaStream_t> saved(n);
  for (int i = 0; i < n; ++i) {
    saved[i] = hs[i]->stream;
    hs[i]->stream = s;
  }
  int rc = COX_OK;
  for (int i = 0; i < n && !rc; ++i) rc = init_state(hs[i], beta0 ? beta0[i] : nullptr);
  auto tiles = [&](int i) { return hs[i]->sd->prep.cinc_T; };
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return tiles(a) > tiles(b); });
  std::vector<std::vector<int>> waves;
  std::vector<int> used;
  for (int i : order) {
    size_t w = 0;
    while (w < waves.size() && used[w] + tiles(i) > grid) ++w;
    if (w == waves.size()) {
      waves.emplace_back();
      used.push_back(0);
    }
    waves[w].push_back(i);
    used[w] += tiles(i);
  }
  BufferSet B;
  IncParams *dprm = static_cast<IncParams *>(B.get(size_t(n) * sizeof(IncParams)));
  int2 *dmap = static_cast<int2 *>(B.get(size_t(waves.size()) * grid * sizeof(int2)));
  if (!rc && (!dprm || !dmap)) rc = fail(nullptr, COX_E_OOM, "cox_batch_fit: allocation");
  std::vector<IncParams> hp(n);
  std::vector<int2> hm(waves.size() * size_t(grid));
  std::vector<cudaEvent_t> ev(waves.size() + 1, nullptr);
  for (auto &e : ev)
    if (!rc && cudaEventCreate(&e) != cudaSuccess) rc = cuda_fail(nullptr, "event create");
  int off = 0;
  if (!rc) cudaEventRecord(ev[0], s);
  for (size_t w = 0; w < waves.size() && !rc; ++w) {
    int cta = 0;
    for (size_t k = 0; k < waves[w].size() && !rc; ++k) {
      cox_handle *h = hs[waves[w][k]];
      const int T = tiles(waves[w][k]);
      hp[off + k] = incr_params(h, true);
      for (int t = 0; t < T; ++t) hm[w * grid + cta++] = make_int2(int(k), t);
      // tag 0 never matches: records start at epoch 1
      if (cudaMemsetAsync(h->i_trec, 0, 2 * kIncRecWords * int64_t(T) * T * sizeof(uint64_t), s) != cudaSuccess ||
          cudaMemsetAsync(h->i_tref, 0, 4 * int64_t(T) * sizeof(uint64_t), s) != cudaSuccess)
        rc = cuda_fail(nullptr, "memset");
    }
    if (!rc && (cudaMemcpyAsync(dprm + off, hp.data() + off, waves[w].size() * sizeof(IncParams), cudaMemcpyHostToDevice, s) !=
                    cudaSuccess ||
                cudaMemcpyAsync(dmap + w * grid, hm.data() + w * grid, cta * sizeof(int2), cudaMemcpyHostToDevice, s) !=
                    cudaSuccess))
      rc = cuda_fail(nullptr, "params copy");
    if (!rc && launch_incr_multi(precision, dprm + off, dmap + w * grid, cta, s))
      rc = cuda_fail(nullptr, "incremental launch");
    if (!rc) cudaEventRecord(ev[w + 1], s);
    off += int(waves[w].size());
  }
  int worst = rc;
  if (!rc && cudaStreamSynchronize(s) != cudaSuccess) worst = rc = cuda_fail(nullptr, "batch execution");
  if (!rc) {
    // each fit's time is the time of its wave
    std::vector<float> wms(waves.size(), 0.0f);
    for (size_t w = 0; w < waves.size(); ++w) cudaEventElapsedTime(&wms[w], ev[w], ev[w + 1]);
#if COX_TRACE_ON
    if (std::getenv("COXGB_BATCH_TRACE")) {   // opt-in: the waves' composition and times
      for (size_t w = 0; w < waves.size(); ++w) {
        int64_t maxsteps = 0, sumsteps = 0;
        for (int i : waves[w]) {
          read_ctl(hs[i]);
          maxsteps = std::max<int64_t>(maxsteps, hs[i]->h_ctl->coord_updates + hs[i]->h_ctl->sweep);
          sumsteps += hs[i]->h_ctl->coord_updates;
        }
        std::fprintf(stderr, "[batch trace] wave %zu: %zu fits on %d CTAs, %.2f ms, longest fit %lld steps (%.2f us/step), "
                     "%lld coordinate steps in all\n", w, waves[w].size(), used[w], wms[w], (long long)maxsteps,
                     maxsteps ? 1e3 * wms[w] / double(maxsteps) : 0.0, (long long)sumsteps);
      }
    }
#endif
    for (size_t w = 0; w < waves.size(); ++w)
      for (int i : waves[w]) {
        cox_handle *h = hs[i];
        int r = read_ctl(h);
        if (!r) r = incr_result(h, beta_out[i], info ? info + i : nullptr, wms[w], 1);
        if (r == COX_E_RANGE && h->opts.engine == COX_ENGINE_AUTO) {
          // beyond the double-word range: this fit again on an FP64 engine
          h->stream = saved[i];
          r = cox_fit(h, beta0 ? beta0[i] : nullptr, beta_out[i], info ? info + i : nullptr);
          h->stream = s;
        }
        if (info) info[i].status = r;
        if (r < 0 || (worst >= 0 && r > worst)) worst = r;
      }
  }
  for (auto &e : ev)
    if (e) cudaEventDestroy(e);
  for (int i = 0; i < n; ++i) hs[i]->stream = saved[i];
  cudaStreamSynchronize(s);
  return worst;
}

// The whole fit in one cooperative launch of the incremental kernel (state already initialized).
int fit_incr(cox_handle *h, double *beta_out, cox_fit_info *info) {
  const DevData &d = D(h);
  const Prepared &P = h->sd->prep;
  const int IT = P.inc_T;
  cudaStream_t s = h->stream;
  // tag 0 never matches: records start at epoch 1
  if (cudaMemsetAsync(h->i_trec, 0, 2 * kIncRecWords * int64_t(IT) * IT * sizeof(uint64_t), s) != cudaSuccess ||
      cudaMemsetAsync(h->i_tref, 0, 4 * int64_t(IT) * sizeof(uint64_t), s) != cudaSuccess)
    return cuda_fail(h, "memset");
  IncParams prm = incr_params(h, false);
#if COX_TRACE_ON
  // phase trace of the first steps (COXGB_PHASE_TRACE=<steps>), printed to stderr
  const char *tr_env = std::getenv("COXGB_PHASE_TRACE");
  const int64_t tr_steps = tr_env ? std::max<int64_t>(0, std::atoll(tr_env)) : 0;
  BufferSet trbuf;
  if (tr_steps > 0) {
    prm.trace = static_cast<uint64_t *>(trbuf.get(tr_steps * IT * 24 * sizeof(uint64_t)));
    prm.trace_steps = prm.trace ? tr_steps : 0;
    if (prm.trace) cudaMemsetAsync(prm.trace, 0, tr_steps * IT * 24 * sizeof(uint64_t), s);
  }
#endif
  if (!h->ev0 && (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess))
    return cuda_fail(h, "event create");
  cudaEventRecord(h->ev0, s);
  int rc;
  int64_t launches = 1;
  if (P.inc_n_halt == 0) {
    if (launch_incr(h->sd->precision, prm, IT, s, P.inc_variant)) return cuda_fail(h, "incremental launch");
    cudaEventRecord(h->ev1, s);
    if ((rc = read_ctl(h))) return rc;
  } else {
    // columns too dense for the lists are stepped by the resident kernel: the incremental launch
    // halts before such a column; one resident launch then steps the run of them and the column
    // after it (whose step applies the last dense update), and the incremental kernel resumes
    // from the shared state (eta, v, beta, trust and the control block)
    if (P.res_T <= 0 || !h->r_tagg) return fail(h, COX_E_INVALID, "cox_fit: dense columns need the resident kernel");
    if (cudaMemsetAsync(h->r_tagg, 0, 6 * P.res_T * sizeof(uint64_t), s) != cudaSuccess ||
        cudaMemsetAsync(h->r_tpart, 0, 12 * P.res_T * sizeof(uint64_t), s) != cudaSuccess)
      return cuda_fail(h, "memset");
    prm.halt = P.inc_halt;
    ResParams rprm = res_params(h);
    const std::vector<uint8_t> &halt = P.h_inc_halt;
    const int32_t p = d.p;
    int64_t left = prm.max_steps;
    launches = 0;
    if ((rc = read_ctl(h))) return rc;
    while (h->h_ctl->state == kRunning && !h->h_ctl->error && left > 0) {
      const int64_t before = h->h_ctl->coord_updates;
      const int32_t j = h->h_ctl->j;
      if (!halt[size_t(j)]) {
        prm.max_steps = left;
        if (launch_incr(h->sd->precision, prm, IT, s, P.inc_variant)) return cuda_fail(h, "incremental launch");
      } else {
        int64_t k = 0;
        for (int32_t jj = j; k < p && halt[size_t(jj)]; jj = jj + 1 >= p ? 0 : jj + 1) ++k;
        rprm.max_steps = std::min<int64_t>(k + 1, left);
        if (launch_resident(h->sd->precision, rprm, P.res_T, s)) return cuda_fail(h, "resident launch");
      }
      ++launches;
      if ((rc = read_ctl(h))) return rc;
      left -= std::max<int64_t>(1, h->h_ctl->coord_updates - before);
    }
    cudaEventRecord(h->ev1, s);
    if (cudaEventSynchronize(h->ev1) != cudaSuccess) return cuda_fail(h, "event");
  }
#if COX_TRACE_ON
  if (prm.trace_steps > 0) {
    // per CTA, mean SM clocks between consecutive phase points of thread 0 (update | patch | scan
    // | barrier | S0 | ratios | group sums | barrier | CTA sums | barrier | push | inbox | barrier
    // | record sums | step) and the global time of its push after the earliest step start, for the
    // three CTAs that push last and the one that pushes first
    constexpr int kSl = 24, kPh = 15;
    std::vector<uint64_t> tr(size_t(prm.trace_steps * IT * kSl));
    cudaMemcpy(tr.data(), prm.trace, tr.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost);
    std::vector<double> pub(IT, 0.0), ph(kPh * IT, 0.0), tot(IT, 0.0), ex(4 * IT, 0.0);
    int64_t n = 0;
    for (int64_t k = 1; k < prm.trace_steps; ++k) {
      uint64_t t0 = ~0ull;
      bool ok = true;
      for (int c = 0; c < IT; ++c) {
        const uint64_t *r = &tr[size_t((k * IT + c) * kSl)];
        for (int q = 0; q < 16; ++q) ok = ok && r[q] != 0;
        ok = ok && r[19] != 0 && r[21] != 0;
        t0 = std::min(t0, r[21]);
      }
      if (!ok) continue;
      for (int c = 0; c < IT; ++c) {
        const uint64_t *r = &tr[size_t((k * IT + c) * kSl)];
        pub[c] += double(r[19] - t0);
        tot[c] += double(r[15] - r[0]);
        for (int q = 0; q < kPh; ++q) ph[kPh * c + q] += double(r[q + 1] - r[q]);
        ex[4 * c + 0] += double(r[16] - r[13]);   // warp 0's share of the record sums
        ex[4 * c + 1] += double(r[18] - r[17]);   // the step rule
        ex[4 * c + 2] += double(r[15] - r[18]);   // exp and bookkeeping after the rule
        ex[4 * c + 3] += double(r[20]);           // polls of thread 0's inbox wait
      }
      ++n;
    }
    std::vector<int> order(IT);
    for (int c = 0; c < IT; ++c) order[c] = c;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return pub[a] > pub[b]; });
    std::fprintf(stderr, "[phase trace] incremental kernel, %lld steps x %d CTAs: push time after the earliest step start "
                 "(ns) | SM clocks: upd patch scan bar S0 ratio gsum bar csum bar push inbox bar rsum step | total\n",
                 (long long)n, IT);
    auto row = [&](const char *tag, int c) {
      std::fprintf(stderr, "  %s CTA %3d: %6.0f |", tag, c, pub[c] / n);
      for (int q = 0; q < kPh; ++q) std::fprintf(stderr, " %5.0f", ph[kPh * c + q] / n);
      std::fprintf(stderr, " | %6.0f | rsum-own %5.0f rule %5.0f exp+ %5.0f polls %4.1f\n", tot[c] / n, ex[4 * c] / n,
                   ex[4 * c + 1] / n, ex[4 * c + 2] / n, ex[4 * c + 3] / n);
    };
    for (int q = 0; q < std::min(IT, 3) && n; ++q) row("last ", order[q]);
    if (n) row("first", order[IT - 1]);
  }
#endif
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  return incr_result(h, beta_out, info, ms, launches);
}

}  // namespace

// =================================================================== ABI
extern "C" {

int cox_set_allocator(cox_alloc_fn alloc, cox_free_fn release, void *ctx) {
  if ((alloc == nullptr) != (release == nullptr)) return fail(nullptr, COX_E_INVALID, "allocator: give both or neither");
  set_allocator(alloc, release, ctx);
  return COX_OK;
}

const char *cox_last_error(const cox_handle *h) { return h ? h->err.c_str() : t_last_error.c_str(); }

int cox_create(const cox_data *data, const cox_options *opts, cox_handle **out) {
  if (!data || !out) return fail(nullptr, COX_E_INVALID, "cox_create: null argument");
  *out = nullptr;
  if (check_options(opts)) return fail(nullptr, COX_E_INVALID, "cox_create: invalid options");
  std::unique_ptr<cox_handle> h(new cox_handle());
  h->opts = opts ? *opts : default_options();
  int rc = resolve_stream(h.get());
  if (rc) return rc;
  auto *sd = new SharedData();
  h->sd = sd;
  sd->precision = h->opts.precision;
  std::string err;
  rc = prepare_data(data, sd->precision, h->opts.tile, h->stream, &sd->prep, &err);
  if (rc) {
    cudaGetLastError();
    release_shared(sd);
    h->sd = nullptr;
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    return fail(nullptr, rc, err.empty() ? "cox_create: preparation failed" : err);
  }
  sd->d_desc = static_cast<DevData *>(dev_alloc(sizeof(DevData)));
  if (!sd->d_desc || cudaMemcpy(sd->d_desc, &sd->prep.desc, sizeof(DevData), cudaMemcpyHostToDevice) != cudaSuccess) {
    cox_destroy(h.release());
    return fail(nullptr, COX_E_OOM, "cox_create: descriptor");
  }
  if ((rc = alloc_fit_state(h.get())) || (rc = apply_options(h.get(), &h->opts))) {
    t_last_error = h->err;
    cox_destroy(h.release());
    return rc;
  }
  *out = h.release();
  return COX_OK;
}

int cox_split_columns(int32_t p, const cox_split *split, int32_t *p_view) {
  if (!p_view || p < 0) return fail(nullptr, COX_E_INVALID, "cox_split_columns: bad arguments");
  std::string err;
  const int rc = split_columns(p, split, p_view, &err);
  return rc ? fail(nullptr, rc, err) : COX_OK;
}

int cox_create_split(const cox_data *data, const cox_split *split, const cox_options *opts, cox_handle **out) {
  if (!data || !split || !out) return fail(nullptr, COX_E_INVALID, "cox_create_split: null argument");
  *out = nullptr;
  if (check_options(opts)) return fail(nullptr, COX_E_INVALID, "cox_create_split: invalid options");
  cudaStream_t s = opts && opts->stream ? static_cast<cudaStream_t>(opts->stream) : nullptr;
  cudaStream_t own = nullptr;
  if (!s) {
    if (cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess)
      return fail(nullptr, COX_E_CUDA, "cox_create_split: stream create");
    s = own;
  }
  int rc;
  {
    BufferSet vb;   // the view's arrays, released once cox_create has copied what it needs
    cox_data view{};
    std::string err;
    rc = build_split_view(data, split, s, vb, &view, &err);
    if (rc) {
      cudaGetLastError();
      if (own) cudaStreamDestroy(own);
      return fail(nullptr, rc, err.empty() ? "cox_create_split: view construction failed" : err);
    }
    rc = cox_create(&view, opts, out);
  }
  if (own) cudaStreamDestroy(own);
  return rc;
}

int cox_cv_path(const cox_data *data, const cox_options *opts, const cox_cv *cv, double *cvl, double *beta_path,
                cox_fit_info *info, int32_t *best) {
  if (!data || !opts || !cv || !cvl) return fail(nullptr, COX_E_INVALID, "cox_cv_path: null argument");
  const int32_t K = cv->n_folds, L = cv->n_path;
  if (K < 2 || L < 1 || !cv->fold || !cv->path) return fail(nullptr, COX_E_INVALID, "cox_cv_path: need n_folds >= 2, n_path >= 1, fold ids and the path");
  if (opts->penalty != COX_PEN_L1 && opts->penalty != COX_PEN_L2)
    return fail(nullptr, COX_E_INVALID, "cox_cv_path: the path needs an L1 or L2 penalty");
  for (int32_t i = 0; i < L; ++i)
    if (opts->penalty == COX_PEN_L1 ? !(cv->path[i] >= 0.0) : !(cv->path[i] > 0.0))
      return fail(nullptr, COX_E_INVALID, "cox_cv_path: path values must be >= 0 (L1 weights) or > 0 (L2 variances)");
  if (check_options(opts)) return fail(nullptr, COX_E_INVALID, "cox_cv_path: invalid options");
  cox_options o = *opts;
  auto set_value = [&](int32_t i) {
    if (o.penalty == COX_PEN_L1) o.lambda = cv->path[i];
    else o.l2_var = cv->path[i];
  };
  set_value(0);
  int32_t p = data->p;
  if (cv->split) {
    std::string err;
    const int rc = split_columns(data->p, cv->split, &p, &err);
    if (rc) return fail(nullptr, rc, err);
  }
  std::vector<cox_handle *> hs(size_t(K) + 1, nullptr);
  auto release = [&]() {
    for (cox_handle *h : hs) cox_destroy(h);
  };
  // training sets on the device, then the full data set (last)
  {
    cudaStream_t s = o.stream ? static_cast<cudaStream_t>(o.stream) : nullptr;
    cudaStream_t own = nullptr;
    if (!s) {
      if (cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess)
        return fail(nullptr, COX_E_CUDA, "cox_cv_path: stream create");
      s = own;
    }
    int rc = COX_OK;
    for (int32_t k = 0; k < K && !rc; ++k) {
      BufferSet vb;
      cox_data view{};
      std::string err;
      rc = build_fold_view(data, cv->fold, k, K, s, vb, &view, &err);
      if (rc) {
        cudaGetLastError();
        rc = fail(nullptr, rc, err.empty() ? "cox_cv_path: training set construction failed" : err);
        break;
      }
      if (cv->split) {   // the training set's time-split view
        BufferSet vb2;
        cox_data view2{};
        rc = build_split_view(&view, cv->split, s, vb2, &view2, &err);
        if (rc) {
          cudaGetLastError();
          rc = fail(nullptr, rc, err.empty() ? "cox_cv_path: split view construction failed" : err);
          break;
        }
        rc = cox_create(&view2, &o, &hs[size_t(k)]);
      } else {
        rc = cox_create(&view, &o, &hs[size_t(k)]);
      }
    }
    if (own) cudaStreamDestroy(own);
    if (!rc) rc = cv->split ? cox_create_split(data, cv->split, &o, &hs[size_t(K)]) : cox_create(data, &o, &hs[size_t(K)]);
    if (rc) {
      release();
      return rc;
    }
  }
  const size_t n = size_t(K) + 1;
  // the fits of one value run as one batch, unless every fit qualifies for the single-fit
  // incremental kernel but not for its batched form (dense columns, the group-dense
  // configuration): then one after the other, which is faster for fits of this size
  bool sequential = o.precision == COX_FP64 && (o.engine == COX_ENGINE_AUTO || o.engine == COX_ENGINE_INCR);
  bool batchable = sequential;
  for (size_t m = 0; m < n && sequential; ++m) {
    Prepared &P = hs[m]->sd->prep;
    sequential = P.inc_T > 0 && D(hs[m]).p > 0;
    std::string err;
    if (batchable && (P.inc_n_halt > 0 || P.inc_variant != 0 || prepare_compact_incr(&P, o.precision, hs[m]->stream, &err) ||
                      P.cinc_T <= 0))
      batchable = false;
  }
  sequential = sequential && !batchable;
  std::vector<std::vector<double>> prev(n, std::vector<double>(size_t(std::max(p, 1)))), cur = prev;
  std::vector<const double *> b0(n);
  std::vector<double *> bo(n);
  std::vector<cox_fit_info> fi(n);
  int worst = COX_OK;
  int rc = COX_OK;
  for (int32_t i = 0; i < L && rc >= 0; ++i) {
    set_value(i);
    for (size_t m = 0; m < n && rc >= 0; ++m) rc = cox_set_options(hs[m], &o);
    if (rc < 0) break;
    for (size_t m = 0; m < n; ++m) {
      b0[m] = prev[m].data();
      bo[m] = cur[m].data();
    }
    if (sequential) {
      for (size_t m = 0; m < n && rc >= 0; ++m) {
        const int r = cox_fit(hs[m], i == 0 ? nullptr : b0[m], bo[m], &fi[m]);
        rc = r < 0 ? r : std::max(rc, r);
      }
    } else {
      rc = cox_batch_fit(hs.data(), int32_t(n), i == 0 ? nullptr : b0.data(), bo.data(), fi.data());
    }
    if (rc < 0) break;
    if (rc > worst) worst = rc;
    double score = 0.0;
    for (int32_t k = 0; k < K && rc >= 0; ++k) {
      double l_full = 0.0, l_train = 0.0;
      if ((rc = cox_loglik(hs[size_t(K)], cur[size_t(k)].data(), &l_full)) < 0) break;
      if ((rc = cox_loglik(hs[size_t(k)], cur[size_t(k)].data(), &l_train)) < 0) break;
      score += l_full - l_train;
    }
    if (rc < 0) break;
    cvl[i] = score;
    if (beta_path && p > 0) std::memcpy(beta_path + size_t(i) * p, cur[size_t(K)].data(), size_t(p) * sizeof(double));
    if (info)
      for (size_t m = 0; m < n; ++m) info[size_t(i) * n + m] = fi[m];
    std::swap(prev, cur);
    rc = COX_OK;
  }
  if (rc >= 0 && best) {
    int32_t bi = 0;
    for (int32_t i = 1; i < L; ++i)
      if (cvl[i] > cvl[bi]) bi = i;
    *best = bi;
  }
  std::string msg = rc < 0 ? std::string(cox_last_error(nullptr)) : std::string();
  release();
  if (rc < 0) return fail(nullptr, rc, msg);
  return worst;
}

int cox_clone(const cox_handle *src, const cox_options *opts, cox_handle **out) {
  if (!src || !out) return fail(nullptr, COX_E_INVALID, "cox_clone: null argument");
  *out = nullptr;
  if (check_options(opts)) return fail(nullptr, COX_E_INVALID, "cox_clone: invalid options");
  if (opts && opts->precision != src->sd->precision)
    return fail(nullptr, COX_E_INVALID, "cox_clone: a clone shares the tile plan and must keep the precision");
  std::unique_ptr<cox_handle> h(new cox_handle());
  h->opts = opts ? *opts : src->opts;
  h->sd = src->sd;
  src->sd->refs.fetch_add(1);
  int rc = resolve_stream(h.get());
  if (!rc) rc = alloc_fit_state(h.get());
  if (!rc) rc = apply_options(h.get(), &h->opts);
  if (rc) {
    t_last_error = h->err;
    cox_destroy(h.release());
    return rc;
  }
  *out = h.release();
  return COX_OK;
}

int cox_set_options(cox_handle *h, const cox_options *opts) {
  if (!h || !opts) return fail(h, COX_E_INVALID, "cox_set_options: null argument");
  if (check_options(opts)) return fail(h, COX_E_INVALID, "cox_set_options: invalid options");
  if (opts->precision != h->sd->precision)
    return fail(h, COX_E_INVALID, "cox_set_options: precision is fixed when the data are prepared");
  if (h->graph && opts->stream != h->opts.stream) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return apply_options(h, opts);
}

void cox_destroy(cox_handle *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->h_ctl) cudaFreeHost(h->h_ctl);
  h->bufs.release();
  release_shared(h->sd);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
}

int cox_fit(cox_handle *h, const double *beta0, double *beta_out, cox_fit_info *info) {
  if (!h || !beta_out) return fail(h, COX_E_INVALID, "cox_fit: null argument");
  const DevData &d = D(h);
  int rc = init_state(h, beta0);
  if (rc) return rc;
  if (d.p == 0 || d.T == 0) {
    // nothing to update: the objective at beta0 is final
    if ((rc = launch_mode(h, kModeLL, -1)) || (rc = read_ctl(h))) return rc;
    if ((rc = device_error(h))) return rc;
    if (info) {
      *info = cox_fit_info{};
      info->converged = 1;
      info->loglik = d.T == 0 ? 0.0 : h->h_ctl->out_ll;
      info->objective = -info->loglik;
    }
    return copy_out(h, beta_out, h->hfit.beta, d.p);
  }
  const int eng = h->opts.engine;
  const bool incr = (eng == COX_ENGINE_AUTO || eng == COX_ENGINE_INCR) && h->sd->prep.inc_T > 0;
  if (eng == COX_ENGINE_INCR && !incr)
    return fail(h, COX_E_INVALID,
                "cox_fit: the data do not qualify for the incremental kernel (binary X; per CTA at most 1024 tie groups, "
                "65536 positions and 1024 entries of a column, or 4096 groups, 32768 positions and 512 entries)");
  if (incr) {
    rc = fit_incr(h, beta_out, info);
    // its double-word sums hold |eta - shift| <= 60; beyond that AUTO refits with an FP64 engine
    if (rc != COX_E_RANGE || eng != COX_ENGINE_AUTO) return rc;
    if ((rc = init_state(h, beta0))) return rc;
  }
  const bool resident = (eng == COX_ENGINE_AUTO || eng == COX_ENGINE_RESIDENT) && h->sd->prep.res_T > 0;
  if (eng == COX_ENGINE_RESIDENT && !resident)
    return fail(h, COX_E_INVALID, "cox_fit: the data do not qualify for the resident kernel (binary X, sequence within shared memory)");
  if (resident) return fit_resident(h, beta_out, info);
  const int len = kSweepBody;
  if ((rc = build_graph(h, len))) return rc;
  // the step-launch budget bounds the device-driven loop whatever happens on the device
  const int64_t max_launches = (int64_t(h->opts.max_sweeps) + 2) * d.p + 2;
  LaunchCtl lc{0u, 0u, int32_t(h->n_items), 1, max_launches};
  if (cudaMemcpyAsync(h->lc, &lc, sizeof(lc), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return cuda_fail(h, "lc copy");
  if (!h->ev0 && (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess))
    return cuda_fail(h, "event create");
  cudaEventRecord(h->ev0, h->stream);
  if (cudaGraphLaunch(h->graph, h->stream) != cudaSuccess) return cuda_fail(h, "graph launch");
  cudaEventRecord(h->ev1, h->stream);
  LaunchCtl lc_after{};
  if (cudaMemcpyAsync(&lc_after, h->lc, sizeof(lc_after), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return cuda_fail(h, "lc read");
  if ((rc = read_ctl(h))) return rc;
  const int64_t launched = max_launches - lc_after.budget;
  count_launches(launched);
  if ((rc = device_error(h))) return rc;
  if (h->h_ctl->state == kRunning)
    return fail(h, COX_E_INVALID, "cox_fit: the launch budget ended the sweep loop before the fit stopped");
  const FitCtl &c = *h->h_ctl;
  rc = c.state == kConverged ? COX_OK : COX_W_NOT_CONVERGED;
  if (info) {
    info->sweeps = c.sweep;
    info->converged = c.state == kConverged;
    info->coord_updates = c.coord_updates;
    info->loglik = c.loglik;
    info->objective = c.obj;
    info->status = rc;
    info->engine = COX_ENGINE_STREAM;
    info->step_launches = launched;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    info->sweep_ms = ms;
  }
  int rc2 = copy_out(h, beta_out, h->hfit.beta, d.p);
  return rc2 ? rc2 : rc;
}

int cox_loglik(cox_handle *h, const double *beta, double *loglik_out) {
  if (!h || !loglik_out) return fail(h, COX_E_INVALID, "cox_loglik: null argument");
  int rc = init_state(h, beta);
  if (rc) return rc;
  if (D(h).T == 0) {
    *loglik_out = 0.0;
    return COX_OK;
  }
  if ((rc = launch_mode(h, kModeLL, -1)) || (rc = read_ctl(h)) || (rc = device_error(h))) return rc;
  *loglik_out = h->h_ctl->out_ll;
  return COX_OK;
}

int cox_gradient(cox_handle *h, const double *beta, double *grad, double *hess_diag) {
  if (!h || !grad) return fail(h, COX_E_INVALID, "cox_gradient: null argument");
  const DevData &d = D(h);
  int rc = init_state(h, beta);
  if (rc) return rc;
  h->hfit.gout = h->gout;
  if ((rc = push_desc(h))) return rc;
  if (d.T == 0 && d.p > 0) cudaMemsetAsync(h->gout, 0, 2 * d.p * sizeof(double), h->stream);
  for (int32_t j = 0; j < d.p; ++j)
    if ((rc = launch_mode(h, kModeEval, j))) break;
  h->hfit.gout = nullptr;
  int rc2 = push_desc(h);
  if (rc) return rc;
  if (rc2) return rc2;
  if ((rc = read_ctl(h)) || (rc = device_error(h))) return rc;
  std::vector<double> g(static_cast<size_t>(2 * std::max<int32_t>(d.p, 1)));
  if (d.p > 0 && cudaMemcpy(g.data(), h->gout, 2 * d.p * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_fail(h, "gradient read");
  std::vector<double> g1(d.p), g2(d.p);
  for (int32_t j = 0; j < d.p; ++j) {
    g1[j] = g[2 * j];
    g2[j] = g[2 * j + 1];
  }
  if (d.p > 0 && cudaMemcpy(grad, g1.data(), d.p * sizeof(double), cudaMemcpyDefault) != cudaSuccess)
    return cuda_fail(h, "gradient write");
  if (hess_diag && d.p > 0 && cudaMemcpy(hess_diag, g2.data(), d.p * sizeof(double), cudaMemcpyDefault) != cudaSuccess)
    return cuda_fail(h, "hessian write");
  return COX_OK;
}

int cox_risk_sums(cox_handle *h, const double *beta, int32_t j, double *S0, double *S1, int64_t *n_groups) {
  if (!h) return fail(h, COX_E_INVALID, "cox_risk_sums: null handle");
  const DevData &d = D(h);
  if (n_groups) *n_groups = d.G;
  if (!S0 && !S1) return COX_OK;
  if (j >= d.p) return fail(h, COX_E_INVALID, "cox_risk_sums: column out of range");
  int rc = init_state(h, beta);
  if (rc) return rc;
  if (d.G == 0) return COX_OK;
  cudaMemsetAsync(h->S1, 0, d.G * sizeof(double), h->stream);
  h->hfit.out_S0 = h->S0;
  h->hfit.out_S1 = h->S1;
  if ((rc = push_desc(h))) return rc;
  rc = launch_mode(h, j >= 0 ? kModeEval : kModeLL, j);
  h->hfit.out_S0 = h->hfit.out_S1 = nullptr;
  int rc2 = push_desc(h);
  if (rc) return rc;
  if (rc2) return rc2;
  if ((rc = read_ctl(h)) || (rc = device_error(h))) return rc;
  if (S0 && (rc = copy_out(h, S0, h->S0, d.G))) return rc;
  if (S1 && (rc = copy_out(h, S1, h->S1, d.G))) return rc;
  return COX_OK;
}

int cox_metadata(cox_handle *h, int64_t *n_groups, int64_t *n_strata, int32_t *group_stratum, int32_t *group_time,
                 int32_t *group_events, int64_t *group_at_risk, int64_t *strata_start) {
  if (!h) return fail(h, COX_E_INVALID, "cox_metadata: null handle");
  const DevData &d = D(h);
  const Prepared &P = h->sd->prep;
  if (n_groups) *n_groups = d.G;
  if (n_strata) *n_strata = d.K;
  auto copy_i32 = [&](int32_t *dst, const int32_t *src, int64_t n) -> int {
    if (!dst || n <= 0) return COX_OK;
    return cudaMemcpy(dst, src, n * sizeof(int32_t), cudaMemcpyDefault) == cudaSuccess ? COX_OK
                                                                                        : cuda_fail(h, "metadata copy");
  };
  int rc;
  if ((rc = copy_i32(group_stratum, P.g_stratum, d.G)) || (rc = copy_i32(group_time, P.g_time, d.G)) ||
      (rc = copy_i32(group_events, d.head_d, d.G)))
    return rc;
  if (strata_start) {
    std::vector<int32_t> ss(static_cast<size_t>(d.K) + 1);
    if (cudaMemcpy(ss.data(), P.strata_start, (d.K + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return cuda_fail(h, "metadata copy");
    std::vector<int64_t> s64(ss.begin(), ss.end());
    if (cudaMemcpy(strata_start, s64.data(), s64.size() * sizeof(int64_t), cudaMemcpyDefault) != cudaSuccess)
      return cuda_fail(h, "metadata copy");
  }
  if (group_at_risk && d.G > 0) {
    // with beta = 0 and no shift every position holds +-1, so the risk-set sums are counts
    std::vector<double> c(static_cast<size_t>(d.G));
    const double shift = h->hfit.shift;
    h->hfit.shift = 0.0;
    rc = cox_risk_sums(h, nullptr, -1, c.data(), nullptr, nullptr);
    h->hfit.shift = shift;
    push_desc(h);
    if (rc) return rc;
    std::vector<int64_t> ci(c.size());
    for (size_t g = 0; g < c.size(); ++g) ci[g] = int64_t(std::llround(c[g]));
    if (cudaMemcpy(group_at_risk, ci.data(), ci.size() * sizeof(int64_t), cudaMemcpyDefault) != cudaSuccess)
      return cuda_fail(h, "metadata copy");
  }
  return COX_OK;
}

int cox_dx(cox_handle *h, double *dx) {
  if (!h || !dx) return fail(h, COX_E_INVALID, "cox_dx: null argument");
  const DevData &d = D(h);
  if (d.p > 0 && cudaMemcpy(dx, d.dX, d.p * sizeof(double), cudaMemcpyDefault) != cudaSuccess)
    return cuda_fail(h, "dx copy");
  return COX_OK;
}

int64_t cox_launch_count(void) { return launch_count(); }

// ------------------------------------------------------------------ one fit sharded by stratum
int cox_shard_setup(cox_handle *h, const double *dx_global, int32_t last_continues) {
  if (!h || (!dx_global && D(h).p > 0)) return fail(h, COX_E_INVALID, "cox_shard_setup: null argument");
  if (h->sd->precision != COX_FP64) return fail(h, COX_E_INVALID, "cox_shard_setup: shards run in COX_FP64");
  const int64_t p = D(h).p;
  if (!h->sh_dx) {
    h->sh_dx = static_cast<double *>(h->bufs.get(std::max<int64_t>(p, 1) * sizeof(double)));
    h->sh_buf = static_cast<double *>(h->bufs.get(8 * sizeof(double)));
    h->sh_ext = static_cast<double *>(h->bufs.get(4 * sizeof(double)));
    if (!h->sh_dx || !h->sh_buf || !h->sh_ext) return fail(h, COX_E_OOM, "cox_shard_setup: allocation");
  }
  if (p > 0 && cudaMemcpyAsync(h->sh_dx, dx_global, p * sizeof(double), cudaMemcpyDefault, h->stream) != cudaSuccess)
    return cuda_fail(h, "cox_shard_setup: copy");
  int rc = init_state(h, nullptr);
  if (rc) return rc;
  if (last_continues && !h->sh_open) {
    if (launch_shard_open_end(h->sd->d_desc, const_cast<int32_t *>(D(h).tile_k), h->stream))
      return cuda_fail(h, "cox_shard_setup: launch");
    h->sh_open = 1;
  }
  return cudaStreamSynchronize(h->stream) == cudaSuccess ? COX_OK : cuda_fail(h, "cox_shard_setup");
}

int cox_shard_head(cox_handle *h, int32_t j, double *head) {
  if (!h || !head || j < 0 || j >= D(h).p || !h->sh_dx) return fail(h, COX_E_INVALID, "cox_shard_head: bad arguments");
  if (launch_shard_head(h->dfit, j, h->sh_buf, h->stream)) return cuda_fail(h, "cox_shard_head: launch");
  int rc;
  if ((rc = read_ctl(h)) || (rc = device_error(h))) return rc;
  return copy_out(h, head, h->sh_buf, 4);
}

int cox_shard_partial(cox_handle *h, int32_t j, const double *carry, int32_t need_ll, double *out) {
  if (!h || !out || j < 0 || j >= D(h).p || !h->sh_dx) return fail(h, COX_E_INVALID, "cox_shard_partial: bad arguments");
  const int32_t nl = need_ll ? 1 : 0;
  const double *ext = nullptr;
  if (h->sh_open && carry) {
    if (cudaMemcpyAsync(h->sh_ext, carry, 3 * sizeof(double), cudaMemcpyDefault, h->stream) != cudaSuccess)
      return cuda_fail(h, "cox_shard_partial: carry");
    ext = h->sh_ext;
  }
  if (cudaMemcpyAsync(&h->ctl->need_ll, &nl, sizeof(nl), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(&h->lc->ext, &ext, sizeof(ext), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return cuda_fail(h, "cox_shard_partial: control");
  int rc;
  if ((rc = launch_mode(h, kModeShard, j)) || (rc = read_ctl(h)) || (rc = device_error(h))) return rc;
  const FitCtl &c = *h->h_ctl;
  const double r[4] = {c.out_g1, c.out_g2, nl ? c.out_ll : 0.0, nl ? c.out_bdx : 0.0};
  if (cudaMemcpy(out, r, sizeof(r), cudaMemcpyDefault) != cudaSuccess) return cuda_fail(h, "cox_shard_partial: out");
  return COX_OK;
}

int cox_shard_step(cox_handle *h, int32_t j, const double *tot, int32_t need_ll, int32_t sweep, int32_t max_sweeps,
                   int32_t *state, double *loglik) {
  if (!h || !tot || j < 0 || j >= D(h).p || !h->sh_dx) return fail(h, COX_E_INVALID, "cox_shard_step: bad arguments");
  double t[4];
  if (cudaMemcpy(t, tot, sizeof(t), cudaMemcpyDefault) != cudaSuccess) return cuda_fail(h, "cox_shard_step: sums");
  if (launch_shard_step(h->dfit, h->sh_dx, j, t, need_ll ? 1 : 0, sweep, max_sweeps, h->sh_buf, h->stream))
    return cuda_fail(h, "cox_shard_step: launch");
  double r[2];
  if (cudaMemcpyAsync(r, h->sh_buf, sizeof(r), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return cuda_fail(h, "cox_shard_step: result");
  if (state) *state = int32_t(r[0]);
  if (loglik) *loglik = r[1];
  if (int32_t(r[0]) == kError) return fail(h, COX_E_CUDA, "cox_shard_step: device error");
  return COX_OK;
}

int cox_shard_beta(cox_handle *h, double *beta) {
  if (!h || !beta) return fail(h, COX_E_INVALID, "cox_shard_beta: null argument");
  return copy_out(h, beta, h->hfit.beta, D(h).p);
}

int cox_debug_set_wait_limit(long long clocks) {
  set_wait_limit(clocks);
  return COX_OK;
}

int cox_debug_set_cached_s0(int32_t enable) {
  g_cached_s0.store(enable != 0);
  return COX_OK;
}

int cox_set_chunk_plan(int32_t chunks_per_cta) {
  if (chunks_per_cta < 0 || chunks_per_cta > 8) return fail(nullptr, COX_E_INVALID, "cox_set_chunk_plan: 0 to 8");
  g_chunks_per_cta.store(chunks_per_cta == 0 ? kChunksPerCtaDefault : chunks_per_cta);
  return COX_OK;
}

int cox_debug_set_chunk_tiles(int32_t tiles) {
  if (tiles < 0 || tiles > kChunkMaxTiles) return fail(nullptr, COX_E_INVALID, "cox_debug_set_chunk_tiles: 0 to 64");
  g_chunk_tiles.store(tiles);
  return COX_OK;
}

int cox_footprint(const cox_data *data, const cox_options *opts, size_t *bytes) {
  if (!data || !bytes) return fail(nullptr, COX_E_INVALID, "cox_footprint: null argument");
  const int precision = opts ? opts->precision : COX_FP64;
  std::vector<int64_t> cp(2, 0);
  int64_t nnz = 0;
  if (data->p > 0 && cudaMemcpy(&nnz, data->col_ptr + data->p, sizeof(int64_t), cudaMemcpyDefault) != cudaSuccess)
    return fail(nullptr, COX_E_INVALID, "cox_footprint: cannot read col_ptr");
  const int64_t n = data->n_rows, p = data->p;
  const int64_t M = data->start ? 2 * n : n, nnzp = data->start ? 2 * nnz : nnz;
  const int64_t tile = opts && opts->tile > 0 ? opts->tile : ccd_tile(precision);
  const int64_t T = (M + tile - 1) / tile + 1;
  const int64_t sv = precision == COX_FP32C ? 4 : 8;
  int64_t b = 0;
  b += 8 * (p + 1) + 4 * nnzp + (data->val ? 8 * nnzp : 0);     // CSC
  b += 4 * p * (T + 1) + 12 * (T + 1) + 8 * p;                  // tables, dX
  b += 16 * n / 8 + 4 * n;                                       // tie groups / strata (upper bounds)
  b += 8 * M + sv * (M + tile + 64) + (data->start ? M / 8 + 8 : 0);   // eta, v, exit bits
  b += 8 * 5 * p + 4 * T + 72 * T + 8 * T + 2 * 8 * n / 4;       // beta, trust, gout; look-back; items; diagnostics
  *bytes = size_t(b) + 64 * 1024;
  return COX_OK;
}

// ------------------------------------------------------------------ batched fits
int cox_batch_fit(cox_handle *const *hs, int32_t n, const double *const *beta0, double *const *beta_out,
                  cox_fit_info *info) {
  if (!hs || n <= 0 || !beta_out) return fail(nullptr, COX_E_INVALID, "cox_batch_fit: bad arguments");
  const int precision = hs[0]->sd->precision;
  for (int i = 0; i < n; ++i) {
    if (!hs[i] || !beta_out[i]) return fail(nullptr, COX_E_INVALID, "cox_batch_fit: null handle or output");
    if (hs[i]->sd->precision != precision) return fail(nullptr, COX_E_INVALID, "cox_batch_fit: mixed precisions");
  }
  // every fit on the incremental kernel when each qualifies and its compact plan fits the GPU; in
  // FP64 (measured on a 256-fit cross-validation batch: 424 fits/s against 277 for the streaming
  // batch), while the compensated-FP32 streaming batch stays the faster FP32C path (567 fits/s)
  bool incr = precision == COX_FP64;
  for (int i = 0; i < n && incr; ++i) {
    const int eng = hs[i]->opts.engine;
    incr = (eng == COX_ENGINE_AUTO || eng == COX_ENGINE_INCR) && hs[i]->sd->prep.inc_T > 0 && D(hs[i]).p > 0;
  }
  for (int i = 0; i < n && incr; ++i) {
    std::string err;
    const int rc = prepare_compact_incr(&hs[i]->sd->prep, precision, hs[0]->stream, &err);
    if (rc) return fail(nullptr, rc, err);
    incr = hs[i]->sd->prep.cinc_T > 0;
  }
  if (incr) return batch_incr(hs, n, beta0, beta_out, info);
  cox_handle *h0 = hs[0];
  cudaStream_t s = h0->stream;
  // per-fit init on the shared stream
  std::vector<cudaStream_t> saved(n);
  int rc = COX_OK;
  for (int i = 0; i < n && !rc; ++i) {
    saved[i] = hs[i]->stream;
    hs[i]->stream = s;
    rc = init_state(hs[i], beta0 ? beta0[i] : nullptr);
  }
  // batch-owned descriptors, control blocks and work list
  BufferSet B;
  DevFit *fits = static_cast<DevFit *>(B.get(n * sizeof(DevFit)));
  FitCtl *ctls = static_cast<FitCtl *>(B.get(n * sizeof(FitCtl)));
  LaunchCtl *lc = static_cast<LaunchCtl *>(B.get(sizeof(LaunchCtl)));
  int64_t total_items = 0;
  int valued = 0;
  for (int i = 0; i < n; ++i) {
    total_items += D(hs[i]).T;
    valued |= hs[i]->valued;
  }
  WorkItem *items = static_cast<WorkItem *>(B.get(std::max<int64_t>(total_items, 1) * sizeof(WorkItem)));
  FitCtl *hc = nullptr;
  if (!rc && (!fits || !ctls || !lc || !items)) rc = fail(nullptr, COX_E_OOM, "cox_batch_fit: allocation");
  if (!rc && cudaMallocHost(&hc, n * sizeof(FitCtl)) != cudaSuccess) rc = cuda_fail(nullptr, "pinned alloc");
  std::vector<DevFit> hf(n);
  for (int i = 0; i < n && !rc; ++i) {
    hf[i] = hs[i]->hfit;
    hf[i].ctl = ctls + i;
    if (cudaMemcpyAsync(ctls + i, hs[i]->ctl, sizeof(FitCtl), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      rc = cuda_fail(nullptr, "ctl copy");
  }
  if (!rc && cudaMemcpyAsync(fits, hf.data(), n * sizeof(DevFit), cudaMemcpyHostToDevice, s) != cudaSuccess)
    rc = cuda_fail(nullptr, "fits copy");
  std::vector<int> running(n, 1);
  const int slots = std::max(1, ccd_max_grid(precision, valued));
  auto rebuild_items = [&]() -> int {
    // the running fits' chunks re-planned over the resident CTAs (their look-back words cleared:
    // a new chunk layout), interleaved item by item (each fit's items in their look-back order)
    std::vector<int64_t> tiles;
    for (int i = 0; i < n; ++i)
      if (running[i]) tiles.push_back(D(hs[i]).T);
    const std::vector<int> nck = plan_chunks(tiles, slots);
    std::vector<std::vector<WorkItem>> lists;
    for (int i = 0, r = 0; i < n; ++i)
      if (running[i]) {
        if (precision == COX_FP32C && clear_lookback(hs[i], s)) return cuda_fail(nullptr, "memset");
        // the cached-S0 path was admitted under the old chunk layout: the next launch takes the full one
        if (cudaMemsetAsync(&ctls[i].s0c_tag, 0, sizeof(uint32_t), s) != cudaSuccess) return cuda_fail(nullptr, "memset");
        lists.push_back(fit_items(hs[i], i, nck[r++]));
      }
    const std::vector<WorkItem> it = interleave(lists);
    int act = 0;
    for (int i = 0; i < n; ++i) act += running[i];
    LaunchCtl l{0u, 0u, int32_t(it.size()), act, 0};
    if (!it.empty() && cudaMemcpyAsync(items, it.data(), it.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return cuda_fail(nullptr, "items copy");
    if (cudaMemcpyAsync(lc, &l, sizeof(l), cudaMemcpyHostToDevice, s) != cudaSuccess) return cuda_fail(nullptr, "lc copy");
    return cudaStreamSynchronize(s) == cudaSuccess ? COX_OK : cuda_fail(nullptr, "items");
  };
  int64_t maxp = 1, max_launches = 0;
  for (int i = 0; i < n; ++i) {
    maxp = std::max<int64_t>(maxp, D(hs[i]).p);
    max_launches = std::max<int64_t>(max_launches, (int64_t(hs[i]->opts.max_sweeps) + 2) * D(hs[i]).p + 2);
    if (D(hs[i]).p == 0 || D(hs[i]).T == 0) running[i] = 0;
  }
  if (!rc) rc = rebuild_items();
  // A fit can stop only at the first step of a sweep (where its objective is tested): launch s p
  // (s >= 1, counted from 0) of a fit of p columns. The host runs segments of launches that end
  // right after the next such launch of any running fit, so that a stopped fit's chunks leave the
  // plan before the next launch. Graphs of 1, 2, 4, ... launches are captured once; a segment is
  // the binary decomposition of its length.
  const int len = int(std::min<int64_t>(std::max<int64_t>(maxp, 32), 2048));
  const int grid = std::max(1, ccd_max_grid(precision, valued));
  std::vector<cudaGraphExec_t> pow2;
  while (!rc && (int64_t(1) << pow2.size()) <= len) {
    const int k = 1 << pow2.size();
    cudaGraph_t g;
    cudaGraphExec_t ge = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = cuda_fail(nullptr, "capture");
      break;
    }
    for (int i = 0; i < k && !rc; ++i)
      if (launch_ccd(precision, fits, items, lc, grid, kModeFit, 0, valued, s)) rc = cuda_fail(nullptr, "capture launch");
    if (cudaStreamEndCapture(s, &g) != cudaSuccess && !rc) rc = cuda_fail(nullptr, "end capture");
    if (!rc) {
      if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) rc = cuda_fail(nullptr, "instantiate");
      cudaGraphDestroy(g);
    }
    if (!rc) pow2.push_back(ge);
  }
  auto segment_end = [&](int64_t done) {   // launches done when the next segment ends
    int64_t b = INT64_MAX;
    for (int i = 0; i < n; ++i)
      if (running[i]) {
        const int64_t pi = D(hs[i]).p;
        int64_t sw = std::max<int64_t>(1, done / pi);
        while (sw * pi + 1 <= done) ++sw;
        b = std::min(b, sw * pi + 1);
      }
    return std::min(b, done + 2 * int64_t(len));
  };
  int64_t launched = 0;
  while (!rc) {
    int any = 0;
    for (int i = 0; i < n; ++i) any |= running[i];
    if (!any) break;
    int64_t todo = segment_end(launched) - launched;
    for (int k = int(pow2.size()) - 1; k >= 0 && todo > 0 && !rc; --k)
      while (todo >= (int64_t(1) << k) && !rc) {
        if (cudaGraphLaunch(pow2[size_t(k)], s) != cudaSuccess) rc = cuda_fail(nullptr, "graph launch");
        count_launches(1 << k);
        launched += 1 << k;
        todo -= 1 << k;
      }
    if (rc) break;
    LaunchCtl lc_now{};
    if (cudaMemcpyAsync(hc, ctls, n * sizeof(FitCtl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&lc_now, lc, sizeof(LaunchCtl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = cuda_fail(nullptr, "batch execution");
      break;
    }
    if (lc_now.error) {
      rc = fail(nullptr, COX_E_TIMEOUT, "cox_batch_fit: a device-side wait exceeded its bound");
      break;
    }
    bool changed = false;
    for (int i = 0; i < n; ++i)
      if (running[i] && (hc[i].state != kRunning || hc[i].error)) {
        running[i] = 0;
        changed = true;
      }
    if (changed) rc = rebuild_items();
    if (launched > max_launches + len) { rc = fail(nullptr, COX_E_INVALID, "cox_batch_fit: launch bound exceeded"); break; }
  }
  for (cudaGraphExec_t ge : pow2) cudaGraphExecDestroy(ge);
  int worst = rc;
  if (!rc) {
    for (int i = 0; i < n; ++i) {
      cox_handle *h = hs[i];
      // results back into the handle; its own work list has another chunk layout
      cudaMemcpyAsync(h->ctl, ctls + i, sizeof(FitCtl), cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(h->h_ctl, ctls + i, sizeof(FitCtl), cudaMemcpyDeviceToHost, s);
      clear_lookback(h, s);
      cudaStreamSynchronize(s);
      const FitCtl &c = *h->h_ctl;
      int r = c.error ? device_error(h) : (D(h).p == 0 ? COX_OK : (c.state == kConverged ? COX_OK : COX_W_NOT_CONVERGED));
      if (D(h).p == 0 || D(h).T == 0) r = COX_OK;
      if (info) {
        info[i].sweeps = c.sweep;
        info[i].converged = c.state == kConverged || D(h).p == 0;
        info[i].coord_updates = c.coord_updates;
        info[i].loglik = c.loglik;
        info[i].objective = c.obj;
        info[i].status = r;
        info[i].engine = COX_ENGINE_STREAM;
        info[i].step_launches = launched;
      }
      int r2 = copy_out(h, beta_out[i], h->hfit.beta, D(h).p);
      if (r2) r = r2;
      if (r < 0 || (worst >= 0 && r > worst)) worst = r;
    }
  }
  for (int i = 0; i < n; ++i) hs[i]->stream = saved[i];
  if (hc) cudaFreeHost(hc);
  cudaStreamSynchronize(s);
  return worst;
}

}  // extern "C"

// =================================================================== serving
namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Owned host copy of one request's inputs (so the caller may free its buffers on return).
struct HostData {
  int64_t n = 0;
  int32_t p = 0;
  std::vector<int32_t> stop, start, stratum, row_idx;
  std::vector<uint8_t> event;
  std::vector<int64_t> col_ptr;
  std::vector<double> val;
  cox_data view() const {
    cox_data d{};
    d.n_rows = n;
    d.p = p;
    d.stop = stop.data();
    d.start = start.empty() ? nullptr : start.data();
    d.event = event.data();
    d.stratum = stratum.empty() ? nullptr : stratum.data();
    d.col_ptr = col_ptr.data();
    d.row_idx = row_idx.data();
    d.val = val.empty() ? nullptr : val.data();
    return d;
  }
};

template <class V>
bool copy_in(std::vector<V> &dst, const V *src, int64_t n) {
  dst.clear();
  if (!src || n <= 0) return true;
  dst.resize(static_cast<size_t>(n));
  return cudaMemcpy(dst.data(), src, n * sizeof(V), cudaMemcpyDefault) == cudaSuccess;
}

enum ReqState { kQueued, kPreparing, kReady, kInFlight, kDone };

struct Req {
  uint64_t id = 0;
  ReqState state = kQueued;
  HostData data;
  cox_options opts{};
  std::vector<uint8_t> penalize;
  size_t footprint = 0;
  cox_handle *h = nullptr;
  int slot = -1;
  bool incr = false;   // runs whole on the incremental kernel (between replays), not in the work list
  bool cancel = false;
  std::vector<double> beta;
  cox_fit_info info{};
  int rc = COX_OK;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
};

}  // namespace

struct cox_server {
  cox_server_options o{};
  std::mutex mu;
  std::condition_variable cv_prep, cv_run, cv_done;
  std::deque<Req *> queue;
  std::vector<Req *> ready;
  std::deque<Req *> incr_ready;   // prepared fits routed to the incremental kernel (counted in n_running)
  std::unordered_map<uint64_t, Req *> reqs;
  uint64_t next_id = 1;
  size_t bytes_in_use = 0;
  int n_preparing = 0, n_running = 0, n_done = 0;
  int64_t submitted = 0, completed = 0, failed = 0, replays = 0, step_launches = 0;
  bool stop = false;
  int device = 0;
  cudaStream_t prep_stream = nullptr, run_stream = nullptr;
  std::thread prep_thr, run_thr;
  // batch state (run thread only)
  BufferSet bufs;
  DevFit *fits = nullptr;
  FitCtl *ctls = nullptr;
  LaunchCtl *lc = nullptr;
  WorkItem *items = nullptr;
  int64_t items_cap = 0;
  FitCtl *h_ctls = nullptr;
  std::vector<Req *> slots;
  cudaGraphExec_t graph = nullptr;
  int graph_valued = -1;
  int grid = 0;
};

namespace {

void finish_locked(cox_server *S, Req *r, int rc) {
  r->rc = rc;
  r->state = kDone;
  r->t_done = now_ms();
  r->info.status = rc;
  r->info.wait_ms = (r->t_admit > 0.0 ? r->t_admit : r->t_done) - r->t_submit;
  r->info.total_ms = r->t_done - r->t_submit;
  S->n_done++;
  if (rc < 0) S->failed++;
  else S->completed++;
  S->cv_done.notify_all();
  S->cv_prep.notify_all();
}

bool can_admit_locked(cox_server *S) {
  if (S->queue.empty()) return false;
  if (S->queue.front()->cancel) return true;
  const int inflight = S->n_preparing + S->n_running + int(S->ready.size());
  return inflight < S->o.max_active && S->bytes_in_use + S->queue.front()->footprint <= S->o.memory_budget;
}

void prep_loop(cox_server *S) {
  cudaSetDevice(S->device);
  for (;;) {
    Req *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_prep.wait(lk, [&] { return S->stop || can_admit_locked(S); });
      if (S->stop) return;
      r = S->queue.front();
      S->queue.pop_front();
      if (r->cancel) {
        finish_locked(S, r, COX_E_INVALID);
        continue;
      }
      r->state = kPreparing;
      r->t_admit = now_ms();
      S->n_preparing++;
      S->bytes_in_use += r->footprint;
    }
    cox_options o = r->opts;
    o.stream = S->prep_stream;
    o.precision = S->o.precision;
    o.engine = COX_ENGINE_STREAM;
    o.penalize = r->penalize.empty() ? nullptr : r->penalize.data();
    const cox_data d = r->data.view();
    cox_handle *h = nullptr;
    int rc = cox_create(&d, &o, &h);
    bool direct = false;
    if (!rc && (D(h).p == 0 || D(h).T == 0)) direct = true;   // nothing to iterate: fit right here
    if (!rc && !direct) rc = init_state(h, nullptr);
    std::vector<double> beta;
    cox_fit_info info{};
    if (!rc && direct) {
      beta.assign(static_cast<size_t>(std::max<int32_t>(D(h).p, 1)), 0.0);
      rc = cox_fit(h, nullptr, beta.data(), &info);
    }
    std::unique_lock<std::mutex> lk(S->mu);
    S->n_preparing--;
    r->data = HostData{};
    if (rc < 0 || direct) {
      if (h) {
        lk.unlock();
        cox_destroy(h);
        lk.lock();
      }
      S->bytes_in_use -= r->footprint;
      if (direct && rc >= 0) {
        r->beta = beta;
        r->info = info;
      }
      finish_locked(S, r, rc);
      continue;
    }
    // account the actual device bytes instead of the estimate
    const size_t actual = h->bufs.bytes_total + h->sd->prep.bufs.bytes_total;
    S->bytes_in_use = S->bytes_in_use - r->footprint + actual;
    r->footprint = actual;
    r->h = h;
    // a fit whose data qualify for the incremental kernel runs whole on it: O(groups + nonzeros)
    // per coordinate against the work list's O(positions) (a launch of the list is latency-bound
    // at ~20 us, however few positions its fits hold); the others batch in the list
    r->incr = h->sd->prep.inc_T > 0;
    if (r->incr) {
      r->state = kInFlight;
      S->incr_ready.push_back(r);
      S->n_running++;
    } else {
      r->state = kReady;
      S->ready.push_back(r);
    }
    S->cv_run.notify_one();
  }
}

// One fit routed to the incremental kernel, run to its end on the run stream, and retired.
void run_incr_fit(cox_server *S, Req *r) {
  cox_handle *h = r->h;
  h->stream = S->run_stream;
  cox_fit_info info{};
  std::vector<double> beta(static_cast<size_t>(std::max<int32_t>(D(h).p, 1)), 0.0);
  int rc = r->cancel ? COX_E_INVALID : fit_incr(h, beta.data(), &info);
  if (rc == COX_E_RANGE && init_state(h, nullptr) == COX_OK) {
    // beyond the double-word range of the incremental sums: the work list (FP32C with a shift
    // check, or FP64) takes the fit from the start
    std::lock_guard<std::mutex> lk(S->mu);
    r->incr = false;
    r->state = kReady;
    S->n_running--;
    S->ready.push_back(r);
    return;
  }
  r->beta = beta;
  r->info = info;
  cox_destroy(h);
  r->h = nullptr;
  std::lock_guard<std::mutex> lk(S->mu);
  S->n_running--;
  S->bytes_in_use -= r->footprint;
  S->step_launches += info.step_launches;
  finish_locked(S, r, rc);
}

int rebuild_batch(cox_server *S) {
  int valued = 0, active = 0;
  std::vector<int64_t> tiles;
  for (size_t sl = 0; sl < S->slots.size(); ++sl)
    if (Req *r = S->slots[sl]) {
      valued |= r->h->valued;
      ++active;
      tiles.push_back(D(r->h).T);
    }
  // the in-flight fits' chunks re-planned over the resident CTAs (a new layout: look-back words
  // cleared on the run stream, ahead of the next replay)
  const std::vector<int> nck = plan_chunks(tiles, std::max(1, ccd_max_grid(S->o.precision, valued)));
  std::vector<std::vector<WorkItem>> lists;
  for (size_t sl = 0, r = 0; sl < S->slots.size(); ++sl)
    if (Req *q = S->slots[sl]) {
      if (S->o.precision == COX_FP32C && clear_lookback(q->h, S->run_stream)) return COX_E_CUDA;
      // the cached-S0 path was admitted under the old chunk layout: the next launch takes the full one
      if (cudaMemsetAsync(&S->ctls[sl].s0c_tag, 0, sizeof(uint32_t), S->run_stream) != cudaSuccess) return COX_E_CUDA;
      lists.push_back(fit_items(q->h, int(sl), nck[r++]));
    }
  const std::vector<WorkItem> it = interleave(lists);
  if (int64_t(it.size()) > S->items_cap || valued != S->graph_valued || !S->graph) {
    if (int64_t(it.size()) > S->items_cap) {
      const int64_t cap = std::max<int64_t>(int64_t(it.size()) * 2, S->items_cap * 2);
      WorkItem *ni = static_cast<WorkItem *>(S->bufs.get(cap * sizeof(WorkItem)));
      if (!ni) return COX_E_OOM;
      S->items = ni;   // the old buffer stays in the set until the server is destroyed
      S->items_cap = cap;
    }
    if (S->graph) {
      cudaGraphExecDestroy(S->graph);
      S->graph = nullptr;
    }
    cudaGraph_t g;
    if (cudaStreamBeginCapture(S->run_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return COX_E_CUDA;
    int rc = COX_OK;
    for (int i = 0; i < S->o.steps_per_replay && !rc; ++i)
      // the streaming kernel's CTAs must all be resident at once: the grid of the variant launched
      rc = launch_ccd(S->o.precision, S->fits, S->items, S->lc, std::max(1, ccd_max_grid(S->o.precision, valued)),
                      kModeFit, 0, valued, S->run_stream);
    const cudaError_t e = cudaStreamEndCapture(S->run_stream, &g);
    if (rc || e != cudaSuccess) return COX_E_CUDA;
    const cudaError_t ei = cudaGraphInstantiate(&S->graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return COX_E_CUDA;
    S->graph_valued = valued;
  }
  LaunchCtl l{0u, 0u, int32_t(it.size()), active, 0};
  if (!it.empty() && cudaMemcpyAsync(S->items, it.data(), it.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                                     S->run_stream) != cudaSuccess)
    return COX_E_CUDA;
  if (cudaMemcpyAsync(S->lc, &l, sizeof(l), cudaMemcpyHostToDevice, S->run_stream) != cudaSuccess) return COX_E_CUDA;
  return cudaStreamSynchronize(S->run_stream) == cudaSuccess ? COX_OK : COX_E_CUDA;
}

void run_loop(cox_server *S) {
  cudaSetDevice(S->device);
  bool dirty = false;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_run.wait_for(lk, std::chrono::milliseconds(20),
                         [&] { return S->stop || !S->ready.empty() || S->n_running > 0; });
      if (S->stop) return;
      // join prepared fits
      for (Req *r : S->ready) {
        size_t sl = 0;
        while (sl < S->slots.size() && S->slots[sl]) ++sl;
        if (sl == S->slots.size()) break;   // cannot happen: slots == max_active
        DevFit df = r->h->hfit;
        df.ctl = S->ctls + sl;
        cudaMemcpyAsync(S->fits + sl, &df, sizeof(df), cudaMemcpyHostToDevice, S->run_stream);
        cudaMemcpyAsync(S->ctls + sl, r->h->ctl, sizeof(FitCtl), cudaMemcpyDeviceToDevice, S->run_stream);
        r->h->stream = S->run_stream;
        r->slot = int(sl);
        r->state = kInFlight;
        S->slots[sl] = r;
        S->n_running++;
        dirty = true;
      }
      S->ready.clear();
      if (S->n_running == 0) continue;
    }
    // one fit routed to the incremental kernel, then a replay of the work list (if it holds any)
    Req *ri = nullptr;
    bool listed = false;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (!S->incr_ready.empty()) {
        ri = S->incr_ready.front();
        S->incr_ready.pop_front();
      }
      for (Req *r : S->slots) listed = listed || r != nullptr;
    }
    if (ri) run_incr_fit(S, ri);
    if (!listed) continue;
    // cancellations are honoured here, at a replay boundary
    std::vector<Req *> retire;
    bool waits_failed = false;   // a launch of the work list gave up a device-side wait
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (Req *r : S->slots)
        if (r && r->cancel) retire.push_back(r);
    }
    if (retire.empty()) {
      int rc = dirty ? rebuild_batch(S) : COX_OK;
      dirty = false;
      if (!rc && cudaGraphLaunch(S->graph, S->run_stream) != cudaSuccess) rc = COX_E_CUDA;
      if (!rc) count_launches(S->o.steps_per_replay);
      LaunchCtl lc_now{};
      if (!rc && (cudaMemcpyAsync(S->h_ctls, S->ctls, S->slots.size() * sizeof(FitCtl), cudaMemcpyDeviceToHost,
                                  S->run_stream) != cudaSuccess ||
                  cudaMemcpyAsync(&lc_now, S->lc, sizeof(LaunchCtl), cudaMemcpyDeviceToHost, S->run_stream) !=
                      cudaSuccess ||
                  cudaStreamSynchronize(S->run_stream) != cudaSuccess))
        rc = COX_E_CUDA;
      waits_failed = !rc && lc_now.error != 0;
      if (rc) {   // a CUDA failure ends every fit in flight with that error
        std::lock_guard<std::mutex> lk(S->mu);
        for (Req *r : S->slots)
          if (r) r->cancel = true;
        continue;
      }
      S->replays++;
      S->step_launches += S->o.steps_per_replay;
      for (size_t sl = 0; sl < S->slots.size(); ++sl)
        if (Req *r = S->slots[sl])
          if (waits_failed || S->h_ctls[sl].state != kRunning || S->h_ctls[sl].error) retire.push_back(r);
    }
    for (Req *r : retire) {
      const int sl = r->slot;
      const FitCtl &c = S->h_ctls[sl];
      int rc;
      if (r->cancel) rc = COX_E_INVALID;
      else if (c.error) rc = c.error;
      else if (waits_failed) rc = COX_E_TIMEOUT;
      else rc = c.state == kConverged ? COX_OK : COX_W_NOT_CONVERGED;
      r->beta.assign(static_cast<size_t>(std::max<int32_t>(D(r->h).p, 1)), 0.0);
      if (rc >= 0 && D(r->h).p > 0)
        cudaMemcpy(r->beta.data(), r->h->hfit.beta, D(r->h).p * sizeof(double), cudaMemcpyDeviceToHost);
      r->info.sweeps = c.sweep;
      r->info.converged = c.state == kConverged;
      r->info.engine = COX_ENGINE_STREAM;
      r->info.coord_updates = c.coord_updates;
      r->info.loglik = c.loglik;
      r->info.objective = c.obj;
      cox_destroy(r->h);
      r->h = nullptr;
      std::lock_guard<std::mutex> lk(S->mu);
      S->slots[sl] = nullptr;
      r->slot = -1;
      S->n_running--;
      S->bytes_in_use -= r->footprint;
      finish_locked(S, r, rc);
      dirty = true;
    }
  }
}

int server_result(cox_server *S, Req *r, double *beta_out, cox_fit_info *info) {
  // called with S->mu held; forgets the request
  const int rc = r->rc;
  if (info) *info = r->info;
  if (beta_out && rc >= 0 && !r->beta.empty()) {
    const size_t p = r->beta.size();
    if (cudaMemcpy(beta_out, r->beta.data(), p * sizeof(double), cudaMemcpyDefault) != cudaSuccess) return COX_E_CUDA;
  }
  S->reqs.erase(r->id);
  S->n_done--;
  delete r;
  return rc;
}

}  // namespace

extern "C" {

int cox_server_create(const cox_server_options *opts, cox_server **out) {
  if (!out) return fail(nullptr, COX_E_INVALID, "cox_server_create: null argument");
  *out = nullptr;
  std::unique_ptr<cox_server> S(new cox_server());
  if (opts) S->o = *opts;
  if (S->o.precision != COX_FP64 && S->o.precision != COX_FP32C)
    return fail(nullptr, COX_E_INVALID, "cox_server_create: precision");
  if (S->o.max_active <= 0) S->o.max_active = 256;
  if (S->o.steps_per_replay <= 0) S->o.steps_per_replay = 64;
  if (cudaGetDevice(&S->device) != cudaSuccess) return cuda_fail(nullptr, "cox_server_create: no device");
  if (S->o.memory_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return cuda_fail(nullptr, "cox_server_create: memory info");
    S->o.memory_budget = size_t(double(fr) * 0.8);
  }
  if (cudaStreamCreateWithFlags(&S->prep_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->run_stream, cudaStreamNonBlocking) != cudaSuccess)
    return cuda_fail(nullptr, "cox_server_create: streams");
  const int n = S->o.max_active;
  S->fits = static_cast<DevFit *>(S->bufs.get(n * sizeof(DevFit)));
  S->ctls = static_cast<FitCtl *>(S->bufs.get(n * sizeof(FitCtl)));
  S->lc = static_cast<LaunchCtl *>(S->bufs.get(sizeof(LaunchCtl)));
  S->items_cap = 1 << 16;
  S->items = static_cast<WorkItem *>(S->bufs.get(S->items_cap * sizeof(WorkItem)));
  if (!S->fits || !S->ctls || !S->lc || !S->items) return fail(nullptr, COX_E_OOM, "cox_server_create: allocation");
  if (cudaMallocHost(&S->h_ctls, n * sizeof(FitCtl)) != cudaSuccess) return cuda_fail(nullptr, "cox_server_create: pinned");
  S->slots.assign(static_cast<size_t>(n), nullptr);
  S->grid = std::max(1, std::max(ccd_max_grid(S->o.precision, 0), ccd_max_grid(S->o.precision, 1)));
  cox_server *raw = S.get();
  S->prep_thr = std::thread(prep_loop, raw);
  S->run_thr = std::thread(run_loop, raw);
  *out = S.release();
  return COX_OK;
}

int cox_server_submit(cox_server *S, const cox_data *data, const cox_options *opts, uint64_t *request_id) {
  if (!S || !data || !request_id) return fail(nullptr, COX_E_INVALID, "cox_server_submit: null argument");
  if (check_options(opts)) return fail(nullptr, COX_E_INVALID, "cox_server_submit: invalid options");
  std::unique_ptr<Req> r(new Req());
  cox_options o = opts ? *opts : default_options();
  o.precision = S->o.precision;
  size_t fp = 0;
  int rc = cox_footprint(data, &o, &fp);
  if (rc) return rc;
  if (fp > S->o.memory_budget) return fail(nullptr, COX_E_ADMISSION, "cox_server_submit: request exceeds the memory budget");
  HostData &h = r->data;
  h.n = data->n_rows;
  h.p = data->p;
  if (h.n < 0 || h.p < 0 || !data->stop || !data->event || !data->col_ptr)
    return fail(nullptr, COX_E_INVALID, "cox_server_submit: null or negative argument");
  bool ok = copy_in(h.col_ptr, data->col_ptr, int64_t(h.p) + 1);
  const int64_t nnz = ok && h.p >= 0 ? h.col_ptr[h.p] : 0;
  ok = ok && nnz >= 0 && copy_in(h.stop, data->stop, h.n) && copy_in(h.event, data->event, h.n) &&
       copy_in(h.start, data->start, h.n) && copy_in(h.stratum, data->stratum, h.n) &&
       copy_in(h.row_idx, data->row_idx, nnz) && copy_in(h.val, data->val, nnz);
  if (ok && opts && opts->penalize && h.p > 0) ok = copy_in(r->penalize, opts->penalize, h.p);
  if (!ok) return cuda_fail(nullptr, "cox_server_submit: copying the inputs");
  if (h.stop.empty()) h.stop.resize(1);   // keep non-null pointers for empty data
  if (h.event.empty()) h.event.resize(1);
  if (h.row_idx.empty()) h.row_idx.resize(1);
  o.penalize = nullptr;
  r->opts = o;
  r->footprint = fp;
  r->t_submit = now_ms();
  std::lock_guard<std::mutex> lk(S->mu);
  r->id = S->next_id++;
  *request_id = r->id;
  S->reqs[r->id] = r.get();
  S->queue.push_back(r.release());
  S->submitted++;
  S->cv_prep.notify_one();
  return COX_OK;
}

int cox_server_poll(cox_server *S, uint64_t id, double *beta_out, cox_fit_info *info) {
  if (!S) return fail(nullptr, COX_E_INVALID, "cox_server_poll: null server");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return fail(nullptr, COX_E_NOT_FOUND, "cox_server_poll: unknown request");
  if (it->second->state != kDone) return COX_E_BUSY;
  return server_result(S, it->second, beta_out, info);
}

int cox_server_wait(cox_server *S, uint64_t id, double timeout_s, double *beta_out, cox_fit_info *info) {
  if (!S) return fail(nullptr, COX_E_INVALID, "cox_server_wait: null server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto done = [&] {
    auto it = S->reqs.find(id);
    return it == S->reqs.end() || it->second->state == kDone;
  };
  if (timeout_s < 0) S->cv_done.wait(lk, done);
  else S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return fail(nullptr, COX_E_NOT_FOUND, "cox_server_wait: unknown request");
  if (it->second->state != kDone) return COX_E_BUSY;
  return server_result(S, it->second, beta_out, info);
}

int cox_server_cancel(cox_server *S, uint64_t id) {
  if (!S) return fail(nullptr, COX_E_INVALID, "cox_server_cancel: null server");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return fail(nullptr, COX_E_NOT_FOUND, "cox_server_cancel: unknown request");
  it->second->cancel = true;
  S->cv_prep.notify_all();
  return COX_OK;
}

int cox_server_stats_get(cox_server *S, cox_server_stats *out) {
  if (!S || !out) return fail(nullptr, COX_E_INVALID, "cox_server_stats_get: null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->queued = int32_t(S->queue.size());
  out->preparing = S->n_preparing + int32_t(S->ready.size());
  out->running = S->n_running;
  out->done_unpolled = S->n_done;
  out->bytes_in_use = S->bytes_in_use;
  out->memory_budget = S->o.memory_budget;
  out->replays = S->replays;
  out->step_launches = S->step_launches;
  return COX_OK;
}

void cox_server_destroy(cox_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_prep.notify_all();
  S->cv_run.notify_all();
  if (S->prep_thr.joinable()) S->prep_thr.join();
  if (S->run_thr.joinable()) S->run_thr.join();
  cudaStreamSynchronize(S->run_stream);
  for (auto &kv : S->reqs) {
    if (kv.second->h) cox_destroy(kv.second->h);
    delete kv.second;
  }
  if (S->graph) cudaGraphExecDestroy(S->graph);
  if (S->h_ctls) cudaFreeHost(S->h_ctls);
  S->bufs.release();
  if (S->prep_stream) cudaStreamDestroy(S->prep_stream);
  if (S->run_stream) cudaStreamDestroy(S->run_stream);
  delete S;
}

}  // extern "C"
