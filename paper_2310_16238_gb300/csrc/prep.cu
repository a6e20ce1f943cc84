// Device-side preparation of a data set for the fused coordinate-step kernel
// (arXiv 2310.16238 §2.7: time-ordered, stratum-concatenated rows with segment heads).
//
// Integer work only (plus delta'X in FP64), all on the device:
//   * validation of the sort order and of the CSC,
//   * strata (segments) and tie groups (a (stratum, time) with >= 1 event; Breslow),
//   * delta'X_j, the first term of eq. (parallel_g),
//   * for counting-process rows (start, stop] the merged risk sequence: per stratum the
//     entries (at stop, +exp) and exits (at start, -exp) ordered by time, and the
//     position-space CSC that lists both positions of every nonzero,
//   * the tile plan and the per-(tile) / per-(column, tile) lookup tables.
// Building blocks: a three-phase exclusive scan, flag compaction and a stable LSD radix
// sort that splits on one key bit per pass (Blelloch's split primitive, "Vector Models for
// Data-Parallel Computing", 1990).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "cox.h"
#include "cox_internal.h"
#include "prep.h"

namespace coxgb {

// ------------------------------------------------------------------ allocation
static cox_alloc_fn g_alloc = nullptr;
static cox_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;

void set_allocator(cox_alloc_fn a, cox_free_fn f, void *ctx) {
  g_alloc = a;
  g_free = f;
  g_alloc_ctx = ctx;
}

static std::atomic<long long> g_wait_limit{0};
long long wait_limit() {
  const long long v = g_wait_limit.load(std::memory_order_relaxed);
  return v > 0 ? v : 4000000000LL;   // ~2 s of SM clock
}
void set_wait_limit(long long clocks) { g_wait_limit.store(clocks > 0 ? clocks : 0, std::memory_order_relaxed); }

static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

void *dev_alloc(size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes == 0) bytes = 256;
  if (g_alloc) return g_alloc(bytes, g_alloc_ctx);
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void *p, size_t bytes) {
  if (!p) return;
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes == 0) bytes = 256;
  if (g_free) g_free(p, bytes, g_alloc_ctx);
  else cudaFree(p);
}

void BufferSet::release() {
  for (auto &b : bufs) dev_free(b.first, b.second);
  bufs.clear();
  bytes_total = 0;
  slab = nullptr;
  slab_left = 0;
}

void *BufferSet::get(size_t bytes) {
  const size_t r = ((bytes ? bytes : 1) + 255) & ~size_t(255);   // 256-byte aligned pieces
  if (r <= kSlabMax) {
    if (r > slab_left) {
      void *s = dev_alloc(kSlabBytes);
      if (!s) return nullptr;
      bufs.emplace_back(s, kSlabBytes);
      slab = static_cast<char *>(s);
      slab_left = kSlabBytes;
    }
    void *p = slab;
    slab += r;
    slab_left -= r;
    bytes_total += r;
    return p;
  }
  void *p = dev_alloc(bytes);
  if (p) {
    bufs.emplace_back(p, bytes);
    bytes_total += r;
  }
  return p;
}

// ------------------------------------------------------------------ scan / compaction
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanBlock = kScanThreads * kScanItems;

// exclusive block-level scan of per-thread counts (int64)
__device__ int64_t block_excl_scan(int64_t v, int64_t *warp_tot, int64_t *block_total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t incl = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
    int64_t wi = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, wi, off);
      if (lane >= off) wi += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;
    if (lane == kScanThreads / 32 - 1) *block_total = wi;
  }
  __syncthreads();
  int64_t r = warp_tot[warp] + incl - v;
  __syncthreads();
  return r;
}

__global__ void scan_reduce_kernel(const int32_t *in, int64_t n, int64_t *bsum) {
  __shared__ int64_t wt[32];
  __shared__ int64_t tot;
  const int64_t base = int64_t(blockIdx.x) * kScanBlock + int64_t(threadIdx.x) * kScanItems;
  int64_t s = 0;
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) s += in[base + k];
  block_excl_scan(s, wt, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void scan_bsums_kernel(int64_t *bsum, int64_t nb, int64_t *total) {
  __shared__ int64_t wt[32];
  __shared__ int64_t tot;
  int64_t carry = 0;
  for (int64_t base = 0; base < nb; base += kScanThreads) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < nb ? bsum[i] : 0;
    const int64_t ex = block_excl_scan(v, wt, &tot);
    if (i < nb) bsum[i] = carry + ex;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void scan_final_kernel(const int32_t *in, int64_t n, const int64_t *boff, int64_t *out) {
  __shared__ int64_t wt[32];
  __shared__ int64_t tot;
  const int64_t base = int64_t(blockIdx.x) * kScanBlock + int64_t(threadIdx.x) * kScanItems;
  int64_t s = 0;
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) s += in[base + k];
  int64_t ex = block_excl_scan(s, wt, &tot) + boff[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) {
      out[base + k] = ex;
      ex += in[base + k];
    }
}

// out[i] = sum_{k<i} in[k]; returns the total (synchronizes the stream).
static int exclusive_scan(const int32_t *in, int64_t n, int64_t *out, int64_t *total_host, Scratch &sc,
                          cudaStream_t s) {
  if (n <= 0) {
    *total_host = 0;
    return COX_OK;
  }
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  int64_t *bsum = static_cast<int64_t *>(sc.get((nb + 1) * sizeof(int64_t)));
  int64_t *tot = static_cast<int64_t *>(sc.get(sizeof(int64_t)));
  if (!bsum || !tot) return COX_E_OOM;
  count_launches(1);
  scan_reduce_kernel<<<unsigned(nb), kScanThreads, 0, s>>>(in, n, bsum);
  count_launches(1);
  scan_bsums_kernel<<<1, kScanThreads, 0, s>>>(bsum, nb, tot);
  count_launches(1);
  scan_final_kernel<<<unsigned(nb), kScanThreads, 0, s>>>(in, n, bsum, out);
  if (cudaMemcpyAsync(total_host, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return COX_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return COX_E_CUDA;
  return COX_OK;
}

__global__ void compact_kernel(const int32_t *flag, const int64_t *pre, int64_t n, int32_t *out) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    if (flag[i]) out[pre[i]] = int32_t(i);
}

static unsigned grid_for(int64_t n, int threads = 256, int64_t cap = 65536) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return unsigned(g);
}

// ------------------------------------------------------------------ stable LSD radix sort
// Keys are sorted on a listed set of bit positions, four at a time (16 buckets per pass): per
// tile of kSortTile keys a digit histogram, one exclusive scan of the histograms in
// (digit, tile) order, then a stable scatter that ranks each key among the equal digits before
// it in its tile (per round of 256 keys: warp match masks, then the counts of the earlier warps).
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

struct SortDigit {
  int32_t nb;       // bits in this digit (1..4)
  int32_t pos[4];   // their positions in the key, least significant first
};

__device__ __forceinline__ int sort_digit(uint64_t k, const SortDigit &d) {
  int v = 0;
  for (int i = 0; i < d.nb; ++i) v |= int((k >> d.pos[i]) & 1u) << i;
  return v;
}

__global__ void digit_hist_kernel(const uint64_t *key, int64_t n, SortDigit dg, int64_t ntiles, int32_t *counts) {
  __shared__ int h[16];
  if (threadIdx.x < 16) h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = base + int64_t(r) * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[sort_digit(key[i], dg)], 1);
  }
  __syncthreads();
  if (threadIdx.x < 16) counts[int64_t(threadIdx.x) * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void digit_scatter_kernel(const uint64_t *key, const uint32_t *pay, int64_t n, SortDigit dg, int64_t ntiles,
                                     const int64_t *offs, uint64_t *key_out, uint32_t *pay_out) {
  constexpr int kW = kSortThreads / 32;
  __shared__ int64_t base_d[16];
  __shared__ int wcnt[kW][17];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < 16) base_d[threadIdx.x] = offs[int64_t(threadIdx.x) * ntiles + blockIdx.x];
  const int64_t tile0 = int64_t(blockIdx.x) * kSortTile;
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = tile0 + int64_t(r) * kSortThreads + threadIdx.x;
    uint64_t k = 0;
    uint32_t v = 0;
    int d = 16;   // past the end: a bucket of its own
    if (i < n) {
      k = key[i];
      v = pay[i];
      d = sort_digit(k, dg);
    }
    const unsigned same = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(same & ((1u << lane) - 1u));
    __syncthreads();   // the previous round's positions are written and its counts folded in
    for (int q = threadIdx.x; q < kW * 17; q += kSortThreads) wcnt[q / 17][q % 17] = 0;
    __syncthreads();
    if (rank == 0) wcnt[warp][d] = __popc(same);
    __syncthreads();
    if (d < 16) {
      int64_t pos = base_d[d] + rank;
      for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
      key_out[pos] = k;
      pay_out[pos] = v;
    }
    __syncthreads();
    if (threadIdx.x < 16) {
      int add = 0;
      for (int w = 0; w < kW; ++w) add += wcnt[w][threadIdx.x];
      base_d[threadIdx.x] += add;
    }
  }
}

// Sorts (key, payload) by the listed key bits, least significant first; stable.
static int radix_sort(uint64_t *&key, uint32_t *&pay, int64_t n, const std::vector<int> &bits, Scratch &sc,
                      cudaStream_t s) {
  if (n <= 1 || bits.empty()) return COX_OK;
  const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
  uint64_t *k2 = static_cast<uint64_t *>(sc.get(n * sizeof(uint64_t)));
  uint32_t *p2 = static_cast<uint32_t *>(sc.get(n * sizeof(uint32_t)));
  int32_t *counts = static_cast<int32_t *>(sc.get(16 * ntiles * sizeof(int32_t)));
  int64_t *offs = static_cast<int64_t *>(sc.get(16 * ntiles * sizeof(int64_t)));
  if (!k2 || !p2 || !counts || !offs) return COX_E_OOM;
  for (size_t b0 = 0; b0 < bits.size(); b0 += 4) {
    SortDigit dg{};
    dg.nb = int32_t(std::min<size_t>(4, bits.size() - b0));
    for (int i = 0; i < dg.nb; ++i) dg.pos[i] = bits[b0 + i];
    count_launches(1);
    digit_hist_kernel<<<unsigned(ntiles), kSortThreads, 0, s>>>(key, n, dg, ntiles, counts);
    int64_t total = 0;
    int rc = exclusive_scan(counts, 16 * ntiles, offs, &total, sc, s);
    if (rc) return rc;
    count_launches(1);
    digit_scatter_kernel<<<unsigned(ntiles), kSortThreads, 0, s>>>(key, pay, n, dg, ntiles, offs, k2, p2);
    std::swap(key, k2);
    std::swap(pay, p2);
  }
  return cudaPeekAtLastError() == cudaSuccess ? COX_OK : COX_E_CUDA;
}

static int bits_needed(uint64_t maxval) {
  int b = 0;
  while (b < 64 && (maxval >> b) != 0) ++b;
  return b;
}

// ------------------------------------------------------------------ validation
enum : int32_t {
  kErrEvent = 1, kErrStartStop = 2, kErrUnsorted = 4, kErrRowIdx = 8, kErrColOrder = 16, kErrColPtr = 32
};

__global__ void validate_rows_kernel(int64_t n, const int32_t *stop, const int32_t *start, const uint8_t *event,
                                     const int32_t *stratum, int32_t *err) {
  int32_t e = 0;
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
    if (event[r] > 1) e |= kErrEvent;
    if (start && !(start[r] < stop[r])) e |= kErrStartStop;
    if (r > 0) {
      const int32_t k0 = stratum ? stratum[r - 1] : 0, k1 = stratum ? stratum[r] : 0;
      if (k1 < k0 || (k1 == k0 && stop[r] < stop[r - 1])) e |= kErrUnsorted;
    }
  }
  if (e) atomicOr(err, e);
}

// ------------------------------------------------------------------ column segments
// Per-column passes over the CSC run one block per segment of at most kSegLen entries of one
// column, so one long column no longer serialises a pass (column lengths span three orders of
// magnitude in the sparse workloads).
constexpr int64_t kSegLen = 8192;
constexpr int kSegThreads = 256;

struct ColSeg {
  int64_t a, b;     // entries [a, b) of column j (row-space CSC)
  int64_t end;      // the column's end (col_ptr[j + 1])
  int32_t j, pad;
};

// Segments of every non-empty column, in column order; first[j] = index of column j's first
// segment (first[p] = number of segments).
static void column_segments(const std::vector<int64_t> &col_ptr, std::vector<ColSeg> *segs, std::vector<int32_t> *first) {
  const int32_t p = int32_t(col_ptr.size()) - 1;
  segs->clear();
  first->assign(size_t(p) + 1, 0);
  for (int32_t j = 0; j < p; ++j) {
    (*first)[j] = int32_t(segs->size());
    for (int64_t a = col_ptr[j]; a < col_ptr[j + 1]; a += kSegLen)
      segs->push_back({a, std::min(a + kSegLen, col_ptr[j + 1]), col_ptr[j + 1], j, 0});
  }
  (*first)[p] = int32_t(segs->size());
}

__global__ void validate_cols_kernel(const ColSeg *segs, const int64_t *col_ptr, const int32_t *row_idx, int64_t n,
                                     int32_t *err) {
  const ColSeg sg = segs[blockIdx.x];
  const int64_t col_lo = col_ptr[sg.j];
  int32_t e = 0;
#pragma unroll 4
  for (int64_t q = sg.a + threadIdx.x; q < sg.b; q += kSegThreads) {
    const int32_t r = row_idx[q];
    if (r < 0 || r >= n) e |= kErrRowIdx;
    if (q > col_lo && !(row_idx[q - 1] < r)) e |= kErrColOrder;
  }
  if (e) atomicOr(err, e);
}

// ------------------------------------------------------------------ metadata kernels
__device__ __forceinline__ int32_t stratum_at(const int32_t *stratum, int64_t r) { return stratum ? stratum[r] : 0; }

__global__ void row_flags_kernel(int64_t n, const int32_t *stop, const uint8_t *event, const int32_t *stratum,
                                 int32_t *seg_start_flag, int32_t *event_flag) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
    seg_start_flag[r] = (r == 0 || stratum_at(stratum, r) != stratum_at(stratum, r - 1)) ? 1 : 0;
    event_flag[r] = event[r] ? 1 : 0;
  }
}

// a new tie group starts at event row i when its (stratum, stop) differs from the previous event row
__global__ void group_flags_kernel(int64_t E, const int32_t *ev_rows, const int32_t *stop, const int32_t *stratum,
                                   int32_t *gflag) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < E; i += int64_t(gridDim.x) * blockDim.x) {
    const int32_t r = ev_rows[i];
    bool f = i == 0;
    if (!f) {
      const int32_t q = ev_rows[i - 1];
      f = stop[q] != stop[r] || stratum_at(stratum, q) != stratum_at(stratum, r);
    }
    gflag[i] = f ? 1 : 0;
  }
}

// stratum index of every row: inclusive count of segment starts minus one
__global__ void row_stratum_index_kernel(int64_t n, const int32_t *seg_start_flag, const int64_t *seg_pre, int32_t *kidx) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x)
    kidx[r] = int32_t(seg_pre[r] + seg_start_flag[r] - 1);
}

template <class V>
__device__ __forceinline__ int64_t lower_bound_dev(const V *a, int64_t n, V x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t m = (lo + hi) >> 1;
    if (a[m] < x) lo = m + 1;
    else hi = m;
  }
  return lo;
}
template <class V>
__device__ __forceinline__ int64_t upper_bound_dev(const V *a, int64_t n, V x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t m = (lo + hi) >> 1;
    if (!(x < a[m])) lo = m + 1;
    else hi = m;
  }
  return lo;
}

// per tie group: time, stratum, events and read position in the risk sequence
__global__ void group_build_kernel(int64_t G, int64_t E, const int32_t *gstart, const int32_t *ev_rows,
                                   const int32_t *stop, const int32_t *stratum, const int32_t *kidx,
                                   const int32_t *seg_start /*K+1*/, const int32_t *sorted_start /*n or null*/,
                                   int counting, int32_t *head_pos, int32_t *head_d, int32_t *g_time, int32_t *g_stratum,
                                   int32_t *g_kidx) {
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < G; g += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i0 = gstart[g], i1 = g + 1 < G ? gstart[g + 1] : E;
    const int32_t r = ev_rows[i0];
    const int32_t t = stop[r];
    const int32_t k = kidx[r];
    const int64_t a = seg_start[k], nk = int64_t(seg_start[k + 1]) - a;
    const int64_t n_entries_before = lower_bound_dev<int32_t>(stop + a, nk, t);
    int64_t pos;
    if (counting) pos = 2 * a + n_entries_before + lower_bound_dev<int32_t>(sorted_start + a, nk, t);
    else pos = a + n_entries_before;
    head_pos[g] = int32_t(pos);
    head_d[g] = int32_t(i1 - i0);
    g_time[g] = t;
    g_stratum[g] = stratum_at(stratum, r);
    g_kidx[g] = k;
  }
}

__global__ void cut_build_kernel(int32_t K, const int32_t *seg_start, int counting, int32_t *cut_pos) {
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < K; k += int64_t(gridDim.x) * blockDim.x) {
    const int64_t b = seg_start[k + 1];
    cut_pos[k] = int32_t(counting ? 2 * b - 1 : b - 1);
  }
}

// bit pos[i] of a bitmap, for every i (the bitmap starts zeroed)
__global__ void set_bits_kernel(const int32_t *pos, int64_t n, uint32_t *bits) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int32_t q = pos[i];
    atomicOr(&bits[q >> 5], 1u << (q & 31));
  }
}

// delta'X_j in two passes with a fixed summation order: one block per column segment (each
// thread a strided subset, then a fixed tree), then one thread per column over its segments.
__global__ void dx_seg_kernel(const ColSeg *segs, const int32_t *row_idx, const double *val, const uint8_t *event,
                              double *partial) {
  __shared__ double red[kSegThreads / 32];
  const ColSeg sg = segs[blockIdx.x];
  double s = 0.0;
#pragma unroll 4
  for (int64_t q = sg.a + threadIdx.x; q < sg.b; q += kSegThreads)
    if (event[row_idx[q]]) s += val ? val[q] : 1.0;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kSegThreads / 32; ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void dx_final_kernel(int32_t p, const int32_t *first, const double *partial, double *dX) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < p; j += int64_t(gridDim.x) * blockDim.x) {
    double s = 0.0;
    for (int32_t i = first[j]; i < first[j + 1]; ++i) s += partial[i];
    dX[j] = s;
  }
}

// ---- counting-process sequence
__global__ void start_keys_kernel(int64_t n, const int32_t *start, const int32_t *kidx, int32_t min_start, uint64_t *key,
                                  uint32_t *pay) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
    key[r] = (uint64_t(uint32_t(kidx[r])) << 32) | uint64_t(uint32_t(start[r] - min_start));
    pay[r] = uint32_t(r);
  }
}

__global__ void gather_start_kernel(int64_t n, const uint32_t *sidx, const int32_t *start, int32_t *sorted_start) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    sorted_start[i] = start[sidx[i]];
}

// entry position of row r and exit position of the row at start-order rank i
__global__ void merge_positions_kernel(int64_t n, const int32_t *stop, const int32_t *start, const int32_t *kidx,
                                       const int32_t *seg_start, const uint32_t *sidx, const int32_t *sorted_start,
                                       int32_t *pos_entry, int32_t *pos_exit, uint32_t *exit_bits) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    // entry of row i: entries before it in its stratum + exits with start < stop_i
    {
      const int32_t k = kidx[i];
      const int64_t a = seg_start[k], nk = int64_t(seg_start[k + 1]) - a;
      pos_entry[i] = int32_t(2 * a + (i - a) + lower_bound_dev<int32_t>(sorted_start + a, nk, stop[i]));
    }
    // exit at start-order rank i: exits before it + entries with stop <= start (entries first on ties)
    {
      const uint32_t r = sidx[i];
      const int32_t k = kidx[r];
      const int64_t a = seg_start[k], nk = int64_t(seg_start[k + 1]) - a;
      const int32_t pe = int32_t(2 * a + (i - a) + upper_bound_dev<int32_t>(stop + a, nk, start[r]));
      pos_exit[r] = pe;
      atomicOr(&exit_bits[pe >> 5], 1u << (pe & 31));
    }
  }
}

// two position-space entries per nonzero: key = (column << 32) | position
__global__ void pos_csc_keys_kernel(const ColSeg *segs, const int32_t *row_idx, const int32_t *pos_entry,
                                    const int32_t *pos_exit, uint64_t *key, uint32_t *pay) {
  const ColSeg sg = segs[blockIdx.x];
  const uint64_t j = uint64_t(sg.j) << 32;
  for (int64_t q = sg.a + threadIdx.x; q < sg.b; q += kSegThreads) {
    const int32_t r = row_idx[q];
    key[2 * q] = j | uint64_t(uint32_t(pos_entry[r]));
    pay[2 * q] = uint32_t(q) << 1;
    key[2 * q + 1] = j | uint64_t(uint32_t(pos_exit[r]));
    pay[2 * q + 1] = (uint32_t(q) << 1) | 1u;
  }
}

__global__ void pos_csc_fill_kernel(int64_t nnz2, const uint64_t *key, const uint32_t *pay, const double *val_row,
                                    uint32_t *idx, double *val) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nnz2; i += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t pos = uint32_t(key[i] & 0xffffffffu);
    idx[i] = pos | ((pay[i] & 1u) ? kExitBit : 0u);
    if (val) val[i] = val_row[pay[i] >> 1];
  }
}

__global__ void double_ptr_kernel(int32_t p, const int64_t *col_ptr, int64_t *col_ptr2) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j <= p; j += int64_t(gridDim.x) * blockDim.x)
    col_ptr2[j] = 2 * col_ptr[j];
}

// ---- tile tables
__global__ void tile_tables_kernel(int32_t T, const int32_t *tile_lo, const int32_t *head_pos, int32_t G,
                                   const int32_t *cut_pos, int32_t K, int32_t *tile_g, int32_t *tile_k) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t <= T; t += int64_t(gridDim.x) * blockDim.x) {
    tile_g[t] = int32_t(lower_bound_dev<int32_t>(head_pos, G, tile_lo[t]));
    tile_k[t] = int32_t(lower_bound_dev<int32_t>(cut_pos, K, tile_lo[t]));
  }
}

__device__ __forceinline__ int64_t lower_bound_pos(const uint32_t *idx, int64_t n, uint32_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t m = (lo + hi) >> 1;
    if ((idx[m] & kPosMask) < x) lo = m + 1;
    else hi = m;
  }
  return lo;
}

__global__ void col_tile_kernel(int32_t p, int32_t T, const int64_t *col_ptr, const uint32_t *idx, const int32_t *tile_lo,
                                int32_t *col_tile) {
  const int64_t total = int64_t(p) * (T + 1);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t j = i / (T + 1), t = i % (T + 1);
    const int64_t a = col_ptr[j], b = col_ptr[j + 1];
    col_tile[i] = int32_t(lower_bound_pos(idx + a, b - a, uint32_t(tile_lo[t])));
  }
}

// Per column, the shortest run of risk positions that holds cap + 1 of its entries (one block per
// column segment; `scale` = position-space entries per nonzero): a tile shorter than it holds at
// most cap entries of the column. out_min[j] starts at INT32_MAX.
__global__ void window_kernel(const ColSeg *segs, int32_t scale, const uint32_t *idx, int32_t cap, int32_t *out_min) {
  const ColSeg sg = segs[blockIdx.x];
  const int64_t a = scale * sg.a, b = scale * sg.b, end = scale * sg.end;
  int32_t best = 0x7fffffff;
#pragma unroll 4
  for (int64_t k = a + threadIdx.x; k < b && k + cap < end; k += kSegThreads) {
    const int32_t w = int32_t(idx[k + cap] & kPosMask) - int32_t(idx[k] & kPosMask) + 1;
    best = min(best, w);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) best = min(best, __shfl_down_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0 && best < 0x7fffffff) atomicMin(&out_min[sg.j], best);
}

static bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool pointer_on_device(const void *p) { return is_device_ptr(p); }

// Make a device-resident view of an input array (copy host arrays into scratch).
template <class V>
static const V *device_view(const V *p, int64_t count, Scratch &sc, cudaStream_t s, int *rc) {
  if (!p || count <= 0) return p;
  if (is_device_ptr(p)) return p;
  V *d = static_cast<V *>(sc.get(count * sizeof(V)));
  if (!d) { *rc = COX_E_OOM; return nullptr; }
  if (cudaMemcpyAsync(d, p, count * sizeof(V), cudaMemcpyHostToDevice, s) != cudaSuccess) { *rc = COX_E_CUDA; return nullptr; }
  return d;
}

// Greedy tile plan: tiles of `tile` positions, shortened when they would hold more than
// kHeadCap tie-group read positions. Boundaries are multiples of 32.
// Tiles of at most `per` positions (multiples of 32), each shortened so that it holds at most
// `cap` tie-group read positions.
static std::vector<int32_t> capped_plan(int64_t M, int64_t per, size_t cap, const std::vector<int32_t> &h_head) {
  std::vector<int32_t> rl;
  int64_t cur = 0;
  size_t hh = 0;
  while (cur < M) {
    rl.push_back(int32_t(cur));
    int64_t hi = std::min<int64_t>(cur + per, M);
    while (hh < h_head.size() && h_head[hh] < cur) ++hh;
    if (hh + cap < h_head.size() && h_head[hh + cap] < hi) {
      const int64_t cut = (int64_t(h_head[hh + cap]) / 32) * 32;
      if (cut > cur) hi = cut;
    }
    cur = hi;
  }
  rl.push_back(int32_t(M));
  return rl;
}

// The shortest tile length (best balance across CTAs, at most pmax) whose capped plan has at
// most `grid` tiles; empty when none has.
static std::vector<int32_t> fit_plan(int64_t M, int64_t pmax, size_t cap, int64_t grid, const std::vector<int32_t> &h_head) {
  int64_t plo = ((M + grid - 1) / grid + 31) / 32 * 32, phi = pmax;
  if (plo > pmax || int64_t(capped_plan(M, pmax, cap, h_head).size()) - 1 > grid) return {};
  while (plo < phi) {   // the plan size is nonincreasing in the tile length
    const int64_t mid = ((plo + phi) / 2) / 32 * 32;
    if (mid <= plo) break;
    if (int64_t(capped_plan(M, mid, cap, h_head).size()) - 1 <= grid) phi = mid;
    else plo = mid + 32;
  }
  std::vector<int32_t> rl = capped_plan(M, phi, cap, h_head);
  if (int64_t(rl.size()) - 1 > grid) rl.clear();
  return rl;
}

// Tiles holding equal numbers of tie-group read positions (at most `per_g` each; the
// incremental kernel's step cost grows with its groups), each cut again after `pos_cap`
// positions. Every tile but the first starts at a read position.
static std::vector<int32_t> group_tiles(int64_t M, int64_t per_g, int64_t pos_cap, const std::vector<int32_t> &h_head) {
  const int64_t G = int64_t(h_head.size());
  std::vector<int32_t> rl{0};
  int64_t cur = 0, g = 0;   // g: first group whose read position is >= cur
  while (cur < M) {
    int64_t hi = g + per_g < G ? int64_t(h_head[g + per_g]) : M;
    hi = std::min(hi, cur + pos_cap);
    if (hi <= cur) hi = std::min<int64_t>(M, cur + 1);
    rl.push_back(int32_t(hi));
    cur = hi;
    g = int64_t(std::lower_bound(h_head.begin() + g, h_head.end(), int32_t(std::min<int64_t>(cur, INT32_MAX))) -
                h_head.begin());
  }
  return rl;
}

// The smallest group count per tile whose group-balanced plan has at most `grid` tiles; empty
// when none within `cap` groups per tile has.
static std::vector<int32_t> group_plan(int64_t M, int64_t pos_cap, int64_t cap, int64_t grid, const std::vector<int32_t> &h_head) {
  const int64_t G = int64_t(h_head.size());
  int64_t lo = std::max<int64_t>(1, (G + grid - 1) / grid), hi = cap;
  if (lo > hi || int64_t(group_tiles(M, hi, pos_cap, h_head).size()) - 1 > grid) return {};
  while (lo < hi) {   // the tile count is nonincreasing in the groups per tile
    const int64_t mid = (lo + hi) / 2;
    if (int64_t(group_tiles(M, mid, pos_cap, h_head).size()) - 1 <= grid) hi = mid;
    else lo = mid + 1;
  }
  return group_tiles(M, hi, pos_cap, h_head);
}

static std::vector<int32_t> plan_tiles(int64_t M, int tile, const std::vector<int32_t> &head_pos) {
  std::vector<int32_t> lo;
  int64_t cur = 0;
  size_t h = 0;
  while (cur < M) {
    lo.push_back(int32_t(cur));
    int64_t hi = std::min<int64_t>(cur + tile, M);
    while (h < head_pos.size() && head_pos[h] < cur) ++h;
    if (h + kHeadCap < head_pos.size() && head_pos[h + kHeadCap] < hi) {
      int64_t cut = (int64_t(head_pos[h + kHeadCap]) / 32) * 32;
      if (cut > cur) hi = cut;
    }
    cur = hi;
  }
  lo.push_back(int32_t(M));
  return lo;
}

// Device tables of a one-tile-per-CTA plan: first tie group and first stratum end of every tile,
// and every column's first entry in every tile.
static int build_tile_tables(BufferSet &B, cudaStream_t s, const DevData &D, const std::vector<int32_t> &rl, int32_t **lo_out,
                             int32_t **g_out, int32_t **k_out, int32_t **ct_out) {
  const int32_t RT = int32_t(rl.size()) - 1;
  const int32_t p = D.p;
  int32_t *r_lo = static_cast<int32_t *>(B.get((RT + 1) * sizeof(int32_t)));
  int32_t *r_g = static_cast<int32_t *>(B.get((RT + 1) * sizeof(int32_t)));
  int32_t *r_k = static_cast<int32_t *>(B.get((RT + 1) * sizeof(int32_t)));
  int32_t *r_ct = static_cast<int32_t *>(B.get(std::max<int64_t>(int64_t(p) * (RT + 1), 1) * sizeof(int32_t)));
  if (!r_lo || !r_g || !r_k || !r_ct) return COX_E_OOM;
  cudaMemcpyAsync(r_lo, rl.data(), (RT + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  count_launches(1);
  tile_tables_kernel<<<grid_for(int64_t(RT) + 1), 256, 0, s>>>(RT, r_lo, D.head_pos, D.G, D.cut_pos, D.K, r_g, r_k);
  if (p > 0) {
    count_launches(1);
    col_tile_kernel<<<grid_for(int64_t(p) * (RT + 1)), 256, 0, s>>>(p, RT, D.col_ptr, D.idx, r_lo, r_ct);
  }
  *lo_out = r_lo;
  *g_out = r_g;
  *k_out = r_k;
  *ct_out = r_ct;
  return COX_OK;
}

// Whether every column's entries in every tile of a plan fit the incremental kernel's lists.
// Columns holding more than the list capacity of entries in some tile of a plan (over[j] = 1):
// one thread per column over its per-tile entry offsets, then p bytes to the host.
__global__ void list_over_kernel(int32_t p, int32_t T, const int32_t *ct, int32_t cap, uint8_t *over) {
  // one warp per column, lanes over its tiles
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t j = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; j < p; j += nw) {
    const int32_t *c = ct + j * (T + 1);
    bool o = false;
    for (int32_t t = lane; t < T; t += 32) o = o || c[t + 1] - c[t] > cap;
    o = __any_sync(0xffffffffu, o);
    if (lane == 0) over[j] = o ? 1 : 0;
  }
}

static int list_overflow(const DevData &D, const int32_t *ct, int32_t T, cudaStream_t s, std::vector<uint8_t> *over,
                         int cap) {
  over->assign(size_t(D.p), 0);
  if (D.p <= 0) return COX_OK;
  uint8_t *d_over = static_cast<uint8_t *>(dev_alloc(size_t(D.p)));
  if (!d_over) return COX_E_OOM;
  count_launches(1);
  list_over_kernel<<<grid_for(int64_t(D.p) * 32), 256, 0, s>>>(D.p, T, ct, cap, d_over);
  const bool ok = cudaMemcpyAsync(over->data(), d_over, size_t(D.p), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                  cudaStreamSynchronize(s) == cudaSuccess;
  dev_free(d_over, size_t(D.p));
  return ok ? COX_OK : COX_E_CUDA;
}

static int lists_fit(const DevData &D, const int32_t *ct, int32_t T, cudaStream_t s, bool *fits) {
  std::vector<uint8_t> over;
  const int rc = list_overflow(D, ct, T, s, &over, inc_list_cap(0));
  *fits = rc == COX_OK && std::find(over.begin(), over.end(), uint8_t(1)) == over.end();
  return rc;
}

int prepare_compact_incr(Prepared *P, int precision, cudaStream_t s, std::string *err) {
  if (P->cinc_T != 0) return COX_OK;
  P->cinc_T = -1;
  const DevData &D = P->desc;
  const int grid = inc_max_grid(precision, 0);
  // batches: configuration 0 only, and no dense-column hand-over
  if (P->inc_T <= 0 || P->inc_n_halt > 0 || P->inc_variant != 0 || grid <= 0) return COX_OK;
  std::vector<int32_t> h_head(size_t(D.G));
  if (D.G > 0 && (cudaMemcpyAsync(h_head.data(), D.head_pos, size_t(D.G) * sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
                      cudaSuccess ||
                  cudaStreamSynchronize(s) != cudaSuccess)) {
    *err = "cox_batch_fit: plan tables";
    return COX_E_CUDA;
  }
  // as many tie groups per tile as a CTA holds, tiles shorter than the run of positions that
  // would overflow a column's list (shortened further if a list still overflows)
  for (int64_t pos_cap = std::min<int64_t>(inc_pos_cap(0), int64_t(P->inc_wmin) - 1); pos_cap >= 32; pos_cap /= 2) {
    std::vector<int32_t> rl = group_tiles(D.M, inc_group_cap(0), pos_cap, h_head);
    const int32_t T = int32_t(rl.size()) - 1;
    if (T > grid) return COX_OK;
    int32_t *lo = nullptr, *g = nullptr, *k = nullptr, *ct = nullptr;
    int rc = build_tile_tables(P->bufs, s, D, rl, &lo, &g, &k, &ct);
    if (rc) return rc;
    bool fits = false;
    if ((rc = lists_fit(D, ct, T, s, &fits))) {
      *err = "cox_batch_fit: plan tables";
      return rc;
    }
    if (fits) {
      P->cinc_T = T;
      P->cinc_tile_lo = lo;
      P->cinc_tile_g = g;
      P->cinc_tile_k = k;
      P->cinc_col_tile = ct;
      return COX_OK;
    }
  }
  return COX_OK;
}

// Inputs staged on the device and validated (shared by cox_create and the time-split view).
struct Staged {
  int64_t n = 0, nnz = 0, nseg = 0;
  int32_t p = 0;
  const int32_t *stop = nullptr, *start = nullptr, *stratum = nullptr, *row_idx = nullptr;
  const uint8_t *event = nullptr;
  const double *val = nullptr;
  const int64_t *col_ptr = nullptr;
  std::vector<int64_t> h_col_ptr;
  std::vector<int32_t> h_seg_first;
  ColSeg *segs = nullptr;
  int32_t *seg_first = nullptr;
};

static int stage_inputs(const cox_data *in, Scratch &sc, cudaStream_t s, Staged *st, std::string *err) {
  const int64_t n = in->n_rows;
  const int32_t p = in->p;
  if (n < 0 || p < 0 || !in->stop || !in->event || !in->col_ptr || (n > 0 && p > 0 && !in->row_idx)) {
    *err = "cox_create: null or negative argument";
    return COX_E_INVALID;
  }
  if (n >= (int64_t(1) << 30)) {
    *err = "cox_create: n_rows must be < 2^30";
    return COX_E_INVALID;
  }
  // column pointers (host copy for nnz and launch sizes)
  std::vector<int64_t> &h_col_ptr = st->h_col_ptr;
  h_col_ptr.assign(size_t(p) + 1, 0);
  if (cudaMemcpy(h_col_ptr.data(), in->col_ptr, (size_t(p) + 1) * sizeof(int64_t), cudaMemcpyDefault) != cudaSuccess) {
    *err = "cox_create: cannot read col_ptr";
    return COX_E_CUDA;
  }
  const int64_t nnz = h_col_ptr[p];
  if (h_col_ptr[0] != 0 || nnz < 0) {
    *err = "cox_create: col_ptr[0] must be 0 and col_ptr[p] >= 0";
    return COX_E_INVALID;
  }
  for (int32_t j = 0; j < p; ++j)
    if (h_col_ptr[j + 1] < h_col_ptr[j]) {
      *err = "cox_create: col_ptr must be nondecreasing";
      return COX_E_INVALID;
    }
  int rc = COX_OK;
  st->n = n;
  st->p = p;
  st->nnz = nnz;
  st->stop = device_view(in->stop, n, sc, s, &rc);
  st->start = device_view(in->start, n, sc, s, &rc);
  st->event = device_view(in->event, n, sc, s, &rc);
  st->stratum = device_view(in->stratum, n, sc, s, &rc);
  st->row_idx = device_view(in->row_idx, nnz, sc, s, &rc);
  st->val = device_view(in->val, nnz, sc, s, &rc);
  st->col_ptr = device_view(in->col_ptr, int64_t(p) + 1, sc, s, &rc);
  if (rc) {
    *err = "cox_create: staging inputs failed";
    return rc;
  }
  // column segments for the per-column passes (validation, delta'X, list windows)
  std::vector<ColSeg> h_segs;
  column_segments(h_col_ptr, &h_segs, &st->h_seg_first);
  const int64_t nseg = st->nseg = int64_t(h_segs.size());
  st->segs = static_cast<ColSeg *>(sc.get((nseg > 0 ? nseg : 1) * sizeof(ColSeg)));
  st->seg_first = static_cast<int32_t *>(sc.get((size_t(p) + 1) * sizeof(int32_t)));
  if (!st->segs || !st->seg_first) return COX_E_OOM;
  if ((nseg > 0 && cudaMemcpyAsync(st->segs, h_segs.data(), nseg * sizeof(ColSeg), cudaMemcpyHostToDevice, s) != cudaSuccess) ||
      cudaMemcpyAsync(st->seg_first, st->h_seg_first.data(), (size_t(p) + 1) * sizeof(int32_t), cudaMemcpyHostToDevice,
                      s) != cudaSuccess) {
    *err = "cox_create: staging column segments failed";
    return COX_E_CUDA;
  }
  int32_t *d_err = static_cast<int32_t *>(sc.get(sizeof(int32_t)));
  if (!d_err) return COX_E_OOM;
  cudaMemsetAsync(d_err, 0, sizeof(int32_t), s);
  if (n > 0) {
    count_launches(1);
    validate_rows_kernel<<<grid_for(n), 256, 0, s>>>(n, st->stop, st->start, st->event, st->stratum, d_err);
  }
  if (nseg > 0) {
    count_launches(1);
    validate_cols_kernel<<<unsigned(nseg), kSegThreads, 0, s>>>(st->segs, st->col_ptr, st->row_idx, n, d_err);
  }
  int32_t h_err = 0;
  cudaMemcpyAsync(&h_err, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    *err = "cox_create: validation kernels failed";
    return COX_E_CUDA;
  }
  if (h_err & kErrUnsorted) { *err = "cox_create: rows are not sorted by (stratum, stop)"; return COX_E_UNSORTED; }
  if (h_err & kErrEvent) { *err = "cox_create: event must be 0 or 1"; return COX_E_INVALID; }
  if (h_err & kErrStartStop) { *err = "cox_create: start must be < stop"; return COX_E_INVALID; }
  if (h_err & kErrRowIdx) { *err = "cox_create: row_idx out of range"; return COX_E_INVALID; }
  if (h_err & kErrColOrder) { *err = "cox_create: row_idx must be strictly ascending within a column"; return COX_E_INVALID; }
  if (h_err & kErrColPtr) { *err = "cox_create: col_ptr must be nondecreasing"; return COX_E_INVALID; }
  return COX_OK;
}

int prepare_data(const cox_data *in, int precision, int tile_req, cudaStream_t s, Prepared *out, std::string *err) {
  Scratch sc;   // temporaries, freed on return
  const int counting = in->start != nullptr;
  const int kernel_tile = ccd_tile(precision);
  int tile = tile_req > 0 ? tile_req : kernel_tile;
  if (tile % 32 != 0 || tile > kernel_tile || tile < 1024) {
    *err = "cox_create: tile must be a multiple of 32 in [1024, " + std::to_string(kernel_tile) + "]";
    return COX_E_INVALID;
  }
  Staged st;
  int rc = stage_inputs(in, sc, s, &st, err);
  if (rc) return rc;
  const int64_t n = st.n, nnz = st.nnz, nseg = st.nseg;
  const int32_t p = st.p;
  const int32_t *stop = st.stop, *start = st.start, *stratum = st.stratum, *row_idx = st.row_idx;
  const uint8_t *event = st.event;
  const double *val = st.val;
  const int64_t *col_ptr_in = st.col_ptr;
  const std::vector<int64_t> &h_col_ptr = st.h_col_ptr;
  const ColSeg *segs = st.segs;
  const int32_t *seg_first = st.seg_first;

  BufferSet &B = out->bufs;
  DevData &D = out->desc;
  D = DevData{};
  D.n_rows = n;
  D.p = p;
  D.counting = counting;
  D.binary = in->val == nullptr;
  D.M = counting ? 2 * n : n;
  D.tile = tile;
  out->nnz_rows = nnz;
  out->h_col_ptr_rows = h_col_ptr;

  // ---- strata and tie groups
  const int64_t nn = n > 0 ? n : 1;
  int32_t *seg_flag = static_cast<int32_t *>(sc.get(nn * sizeof(int32_t)));
  int32_t *ev_flag = static_cast<int32_t *>(sc.get(nn * sizeof(int32_t)));
  int64_t *seg_pre = static_cast<int64_t *>(sc.get(nn * sizeof(int64_t)));
  int64_t *ev_pre = static_cast<int64_t *>(sc.get(nn * sizeof(int64_t)));
  if (!seg_flag || !ev_flag || !seg_pre || !ev_pre) return COX_E_OOM;
  int64_t K = 0, E = 0;
  if (n > 0) {
    count_launches(1);
    row_flags_kernel<<<grid_for(n), 256, 0, s>>>(n, stop, event, stratum, seg_flag, ev_flag);
    if ((rc = exclusive_scan(seg_flag, n, seg_pre, &K, sc, s))) return rc;
    if ((rc = exclusive_scan(ev_flag, n, ev_pre, &E, sc, s))) return rc;
  }
  D.K = int32_t(K);
  D.sum_d = double(E);
  int32_t *seg_start = static_cast<int32_t *>(B.get((K + 1) * sizeof(int32_t)));
  int32_t *kidx = static_cast<int32_t *>(sc.get(nn * sizeof(int32_t)));
  int32_t *ev_rows = static_cast<int32_t *>(sc.get((E > 0 ? E : 1) * sizeof(int32_t)));
  if (!seg_start || !kidx || !ev_rows) return COX_E_OOM;
  if (n > 0) {
    count_launches(1);
    compact_kernel<<<grid_for(n), 256, 0, s>>>(seg_flag, seg_pre, n, seg_start);
    count_launches(1);
    compact_kernel<<<grid_for(n), 256, 0, s>>>(ev_flag, ev_pre, n, ev_rows);
    count_launches(1);
    row_stratum_index_kernel<<<grid_for(n), 256, 0, s>>>(n, seg_flag, seg_pre, kidx);
  }
  {
    const int32_t nv = int32_t(n);
    cudaMemcpyAsync(seg_start + K, &nv, sizeof(int32_t), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);   // nv lives on this stack frame
  }
  out->strata_start = seg_start;

  // counting process: start order within strata
  const int32_t *sorted_start = nullptr;
  uint32_t *sidx = nullptr;
  if (counting && n > 0) {
    std::vector<int32_t> hs(static_cast<size_t>(n));
    // min start for the key offset (host reduction over a copy; small relative to the fit)
    if (cudaMemcpyAsync(hs.data(), start, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return COX_E_CUDA;
    int32_t mn = *std::min_element(hs.begin(), hs.end()), mx = *std::max_element(hs.begin(), hs.end());
    uint64_t *key = static_cast<uint64_t *>(sc.get(n * sizeof(uint64_t)));
    uint32_t *pay = static_cast<uint32_t *>(sc.get(n * sizeof(uint32_t)));
    if (!key || !pay) return COX_E_OOM;
    count_launches(1);
    start_keys_kernel<<<grid_for(n), 256, 0, s>>>(n, start, kidx, mn, key, pay);
    std::vector<int> bits;
    const int lob = bits_needed(uint64_t(uint32_t(mx - mn))), hib = bits_needed(uint64_t(K > 0 ? K - 1 : 0));
    for (int b = 0; b < lob; ++b) bits.push_back(b);
    for (int b = 0; b < hib; ++b) bits.push_back(32 + b);
    if ((rc = radix_sort(key, pay, n, bits, sc, s))) return rc;
    sidx = pay;
    int32_t *ss = static_cast<int32_t *>(sc.get(n * sizeof(int32_t)));
    if (!ss) return COX_E_OOM;
    count_launches(1);
    gather_start_kernel<<<grid_for(n), 256, 0, s>>>(n, sidx, start, ss);
    sorted_start = ss;
  }

  // tie groups
  int32_t *gflag = static_cast<int32_t *>(sc.get((E > 0 ? E : 1) * sizeof(int32_t)));
  int64_t *gpre = static_cast<int64_t *>(sc.get((E > 0 ? E : 1) * sizeof(int64_t)));
  if (!gflag || !gpre) return COX_E_OOM;
  int64_t G = 0;
  if (E > 0) {
    count_launches(1);
    group_flags_kernel<<<grid_for(E), 256, 0, s>>>(E, ev_rows, stop, stratum, gflag);
    if ((rc = exclusive_scan(gflag, E, gpre, &G, sc, s))) return rc;
  }
  D.G = int32_t(G);
  const int64_t Gs = G > 0 ? G : 1;
  int32_t *gstart = static_cast<int32_t *>(sc.get(Gs * sizeof(int32_t)));
  int32_t *head_pos = static_cast<int32_t *>(B.get(Gs * sizeof(int32_t)));
  int32_t *head_d = static_cast<int32_t *>(B.get(Gs * sizeof(int32_t)));
  int32_t *g_time = static_cast<int32_t *>(B.get(Gs * sizeof(int32_t)));
  int32_t *g_stratum = static_cast<int32_t *>(B.get(Gs * sizeof(int32_t)));
  int32_t *g_kidx = static_cast<int32_t *>(sc.get(Gs * sizeof(int32_t)));
  if (!gstart || !head_pos || !head_d || !g_time || !g_stratum || !g_kidx) return COX_E_OOM;
  if (G > 0) {
    count_launches(1);
    compact_kernel<<<grid_for(E), 256, 0, s>>>(gflag, gpre, E, gstart);
    count_launches(1);
    group_build_kernel<<<grid_for(G), 256, 0, s>>>(G, E, gstart, ev_rows, stop, stratum, kidx, seg_start, sorted_start,
                                                    counting, head_pos, head_d, g_time, g_stratum, g_kidx);
  }
  D.head_pos = head_pos;
  D.head_d = head_d;
  out->g_time = g_time;
  out->g_stratum = g_stratum;
  int32_t *cut_pos = static_cast<int32_t *>(B.get((K > 0 ? K : 1) * sizeof(int32_t)));
  if (!cut_pos) return COX_E_OOM;
  if (K > 0) { count_launches(1); cut_build_kernel<<<grid_for(K), 256, 0, s>>>(int32_t(K), seg_start, counting, cut_pos); }
  D.cut_pos = cut_pos;
  // the same positions as bitmaps over the risk sequence (the streaming kernels stage a tile's
  // words beside its values: up to 128 words from a tile's first position, so 128 zero words
  // follow the end)
  {
    const int64_t words = (D.M + 31) / 32 + 128;
    uint32_t *hb = static_cast<uint32_t *>(B.get(words * sizeof(uint32_t)));
    uint32_t *cb = static_cast<uint32_t *>(B.get(words * sizeof(uint32_t)));
    if (!hb || !cb) return COX_E_OOM;
    cudaMemsetAsync(hb, 0, words * sizeof(uint32_t), s);
    cudaMemsetAsync(cb, 0, words * sizeof(uint32_t), s);
    if (G > 0) { count_launches(1); set_bits_kernel<<<grid_for(G), 256, 0, s>>>(head_pos, G, hb); }
    if (K > 0) { count_launches(1); set_bits_kernel<<<grid_for(K), 256, 0, s>>>(cut_pos, K, cb); }
    D.head_bits = hb;
    D.cut_bits = cb;
  }

  // delta'X
  double *dX = static_cast<double *>(B.get((p > 0 ? p : 1) * sizeof(double)));
  if (!dX) return COX_E_OOM;
  if (p > 0) {
    double *partial = static_cast<double *>(sc.get((nseg > 0 ? nseg : 1) * sizeof(double)));
    if (!partial) return COX_E_OOM;
    if (nseg > 0) { count_launches(1); dx_seg_kernel<<<unsigned(nseg), kSegThreads, 0, s>>>(segs, row_idx, val, event, partial); }
    count_launches(1);
    dx_final_kernel<<<grid_for(p), 256, 0, s>>>(p, seg_first, partial, dX);
  }
  D.dX = dX;

  // ---- the position-space CSC
  const int64_t nnz_pos = counting ? 2 * nnz : nnz;
  int64_t *col_ptr = static_cast<int64_t *>(B.get((int64_t(p) + 1) * sizeof(int64_t)));
  uint32_t *idx = static_cast<uint32_t *>(B.get((nnz_pos > 0 ? nnz_pos : 1) * sizeof(uint32_t)));
  double *vpos = nullptr;
  if (in->val) vpos = static_cast<double *>(B.get((nnz_pos > 0 ? nnz_pos : 1) * sizeof(double)));
  if (!col_ptr || !idx || (in->val && !vpos)) return COX_E_OOM;
  uint32_t *exit_bits = nullptr;
  if (!counting) {
    cudaMemcpyAsync(col_ptr, col_ptr_in, (int64_t(p) + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    if (nnz > 0) cudaMemcpyAsync(idx, row_idx, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (vpos && nnz > 0) cudaMemcpyAsync(vpos, val, nnz * sizeof(double), cudaMemcpyDeviceToDevice, s);
  } else {
    const int64_t M = D.M;
    exit_bits = static_cast<uint32_t *>(B.get(((M + 31) / 32 + 1) * sizeof(uint32_t)));
    int32_t *pos_entry = static_cast<int32_t *>(sc.get(nn * sizeof(int32_t)));
    int32_t *pos_exit = static_cast<int32_t *>(sc.get(nn * sizeof(int32_t)));
    if (!exit_bits || !pos_entry || !pos_exit) return COX_E_OOM;
    cudaMemsetAsync(exit_bits, 0, ((M + 31) / 32 + 1) * sizeof(uint32_t), s);
    if (n > 0) {
      count_launches(1);
      merge_positions_kernel<<<grid_for(n), 256, 0, s>>>(n, stop, start, kidx, seg_start, sidx, sorted_start, pos_entry,
                                                         pos_exit, exit_bits);
    }
    count_launches(1);
    double_ptr_kernel<<<grid_for(int64_t(p) + 1), 256, 0, s>>>(p, col_ptr_in, col_ptr);
    if (nnz > 0) {
      uint64_t *key = static_cast<uint64_t *>(sc.get(nnz_pos * sizeof(uint64_t)));
      uint32_t *pay = static_cast<uint32_t *>(sc.get(nnz_pos * sizeof(uint32_t)));
      if (!key || !pay) return COX_E_OOM;
      count_launches(1);
      pos_csc_keys_kernel<<<unsigned(nseg), kSegThreads, 0, s>>>(segs, row_idx, pos_entry, pos_exit, key, pay);
      std::vector<int> bits;
      const int pb = bits_needed(uint64_t(M > 0 ? M - 1 : 0)), jb = bits_needed(uint64_t(p > 0 ? p - 1 : 0));
      for (int b = 0; b < pb; ++b) bits.push_back(b);
      for (int b = 0; b < jb; ++b) bits.push_back(32 + b);
      if ((rc = radix_sort(key, pay, nnz_pos, bits, sc, s))) return rc;
      count_launches(1);
      pos_csc_fill_kernel<<<grid_for(nnz_pos), 256, 0, s>>>(nnz_pos, key, pay, val, idx, vpos);
    }
  }
  D.col_ptr = col_ptr;
  D.idx = idx;
  D.val = vpos;
  D.exit_bits = exit_bits;
  out->h_col_ptr.resize(size_t(p) + 1);
  for (int32_t j = 0; j <= p; ++j) out->h_col_ptr[j] = counting ? 2 * h_col_ptr[j] : h_col_ptr[j];

  // ---- tile plan and tables
  std::vector<int32_t> h_head(static_cast<size_t>(G));
  if (G > 0 && cudaMemcpyAsync(h_head.data(), head_pos, G * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return COX_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    *err = "cox_create: preparation kernels failed";
    return COX_E_CUDA;
  }
  std::vector<int32_t> h_lo = plan_tiles(D.M, tile, h_head);
  const int32_t T = int32_t(h_lo.size()) - 1;
  D.T = T;
  int32_t *tile_lo = static_cast<int32_t *>(B.get((T + 1) * sizeof(int32_t)));
  int32_t *tile_g = static_cast<int32_t *>(B.get((T + 1) * sizeof(int32_t)));
  int32_t *tile_k = static_cast<int32_t *>(B.get((T + 1) * sizeof(int32_t)));
  int32_t *col_tile = static_cast<int32_t *>(B.get((int64_t(p) * (T + 1) > 0 ? int64_t(p) * (T + 1) : 1) * sizeof(int32_t)));
  if (!tile_lo || !tile_g || !tile_k || !col_tile) return COX_E_OOM;
  cudaMemcpyAsync(tile_lo, h_lo.data(), (T + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  count_launches(1);
  tile_tables_kernel<<<grid_for(int64_t(T) + 1), 256, 0, s>>>(T, tile_lo, head_pos, int32_t(G), cut_pos, int32_t(K), tile_g,
                                                              tile_k);
  if (p > 0) { count_launches(1); col_tile_kernel<<<grid_for(int64_t(p) * (T + 1)), 256, 0, s>>>(p, T, col_ptr, idx, tile_lo, col_tile); }
  D.tile_lo = tile_lo;
  D.tile_g = tile_g;
  D.tile_k = tile_k;
  D.col_tile = col_tile;
  out->h_tile_lo = h_lo;
  out->h_tile_g.resize(h_lo.size());
  for (size_t t = 0; t < h_lo.size(); ++t)
    out->h_tile_g[t] = int32_t(std::lower_bound(h_head.begin(), h_head.end(), h_lo[t]) - h_head.begin());

  // one-tile-per-CTA plans of the resident and incremental kernels (binary X only)
  auto tables = [&](const std::vector<int32_t> &rl, int32_t **lo_out, int32_t **g_out, int32_t **k_out,
                    int32_t **ct_out) -> int { return build_tile_tables(B, s, D, rl, lo_out, g_out, k_out, ct_out); };
  if (in->val == nullptr && p > 0 && D.M > 0) {
    const int res_grid = res_max_grid(precision);
    if (res_grid > 0) {
      std::vector<int32_t> rl = fit_plan(D.M, res_tile(precision), size_t(res_head_cap()), res_grid, h_head);
      if (!rl.empty()) {
        if ((rc = tables(rl, &out->res_tile_lo, &out->res_tile_g, &out->res_tile_k, &out->res_col_tile))) return rc;
        out->res_T = int32_t(rl.size()) - 1;
      }
    }
    // configuration 0 first (one tie group per thread); configuration 1 for group-dense data
    for (int variant = 0; variant < 2 && out->inc_T == 0; ++variant) {
      const int inc_grid = inc_max_grid(precision, variant);
      if (inc_grid <= 0) continue;
      // candidate plans: equal tie groups per tile (the step's cost) with tiles shorter than the
      // shortest run of positions holding more entries of one column than the kernel's list
      // capacity; then equal positions. The first whose lists fit is taken. A few columns too
      // dense for any plan of at most inc_grid tiles (a treatment indicator held by half the
      // rows) are left to the resident kernel: the incremental launch halts before them.
      std::vector<int32_t> wcol(size_t(p), 0x7fffffff);
      {
        int32_t *d_w = static_cast<int32_t *>(sc.get(size_t(p) * sizeof(int32_t)));
        if (!d_w) return COX_E_OOM;
        cudaMemcpyAsync(d_w, wcol.data(), size_t(p) * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (nseg > 0) count_launches(1);
        if (nseg > 0)
          window_kernel<<<unsigned(nseg), kSegThreads, 0, s>>>(segs, counting ? 2 : 1, idx, inc_list_cap(variant), d_w);
        if (cudaMemcpyAsync(wcol.data(), d_w, size_t(p) * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
          *err = "cox_create: table kernels failed";
          return COX_E_CUDA;
        }
      }
      // Plans in order of preference; a plan is taken when at most `allowed` columns overflow its
      // lists (those become halt columns). First every column on the lists; failing that, the
      // columns that overflow the equal-positions plan are handed over (at most max(2, p / 16)),
      // and the group-balanced plan is built for the others.
      const int64_t max_halt = out->res_T > 0 ? std::max<int64_t>(2, p / 16) : 0;
      auto take = [&](const std::vector<int32_t> &il, int64_t allowed, const std::vector<uint8_t> &pre,
                      bool *taken, std::vector<uint8_t> *halt_out) -> int {
        *taken = false;
        if (il.empty()) return COX_OK;
        int32_t *ilo = nullptr, *ig = nullptr, *ik = nullptr, *ict = nullptr;
        int r = tables(il, &ilo, &ig, &ik, &ict);
        if (r) return r;
        const int32_t IT = int32_t(il.size()) - 1;
        std::vector<uint8_t> over;
        if ((r = list_overflow(D, ict, IT, s, &over, inc_list_cap(variant)))) return r;
        int64_t n2 = 0;
        for (int32_t j = 0; j < p; ++j) {
          over[j] = over[j] | pre[j];
          n2 += over[j];
        }
        *halt_out = over;
        if (n2 > allowed || n2 >= p) return COX_OK;
        out->inc_T = IT;
        out->inc_tile_lo = ilo;
        out->inc_tile_g = ig;
        out->inc_tile_k = ik;
        out->inc_col_tile = ict;
        out->inc_n_halt = int32_t(n2);
        out->inc_variant = variant;
        if (n2 > 0) {
          uint8_t *dh = static_cast<uint8_t *>(B.get(size_t(p)));
          if (!dh || cudaMemcpyAsync(dh, over.data(), size_t(p), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return COX_E_OOM;
          out->inc_halt = dh;
          out->h_inc_halt = over;
        }
        *taken = true;
        return COX_OK;
      };
      auto group_for = [&](const std::vector<uint8_t> &excl) {
        int32_t wmin = 0x7fffffff;
        for (int32_t j = 0; j < p; ++j)
          if (!excl[j]) wmin = std::min(wmin, wcol[j]);
        const int64_t pos_cap = std::min<int64_t>(inc_pos_cap(variant), int64_t(wmin) - 1);
        return pos_cap >= 32 ? group_plan(D.M, pos_cap, inc_group_cap(variant), inc_grid, h_head) : std::vector<int32_t>{};
      };
      const std::vector<uint8_t> none(size_t(p), 0);
      std::vector<uint8_t> hset;
      bool taken = false;
      {
        int32_t wmin = 0x7fffffff;
        for (int32_t j = 0; j < p; ++j) wmin = std::min(wmin, wcol[j]);
        if (variant == 0) out->inc_wmin = wmin;
      }
      const std::vector<int32_t> fp =
          fit_plan(D.M, inc_pos_cap(variant), size_t(inc_group_cap(variant)), inc_grid, h_head);
      if ((rc = take(group_for(none), 0, none, &taken, &hset))) return rc;
      if (!taken && (rc = take(fp, 0, none, &taken, &hset))) return rc;
      if (!taken && max_halt > 0 && !fp.empty()) {
        const std::vector<uint8_t> over_f = hset;   // the equal-positions plan's overflow set
        int64_t nf = 0;
        for (uint8_t v : over_f) nf += v;
        if (nf > 0 && nf <= max_halt) {
          if ((rc = take(group_for(over_f), max_halt, over_f, &taken, &hset))) return rc;
          if (!taken && (rc = take(fp, max_halt, over_f, &taken, &hset))) return rc;
        }
      }
    }
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    *err = "cox_create: table kernels failed";
    return COX_E_CUDA;
  }
  return COX_OK;
}

// ------------------------------------------------------------------ time-split view (§2.2, §2.3)
// Intervals a row can be at risk in: I_k (k = 0..C, I_k = [t_k, t_{k+1}), t_0 = -inf,
// t_{C+1} = +inf) holds an integer time t with start < t <= stop iff t_k <= stop and
// start + 1 < t_{k+1}; both bounds are counts of cuts, so the intervals form the range [klo, khi].
__device__ __forceinline__ void split_range(const int32_t *cuts, int32_t C, int32_t stop, const int32_t *start,
                                            int64_t r, int32_t *klo, int32_t *khi) {
  *khi = int32_t(upper_bound_dev<int32_t>(cuts, C, stop));
  *klo = start ? int32_t(upper_bound_dev<int32_t>(cuts, C, start[r] + 1)) : 0;
}

__global__ void split_count_kernel(int64_t n, const int32_t *stop, const int32_t *start, const int32_t *cuts, int32_t C,
                                   int32_t *cnt) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
    int32_t klo, khi;
    split_range(cuts, C, stop[r], start, r, &klo, &khi);
    cnt[r] = khi - klo + 1;
  }
}

// one (row, interval) pair per view row; key = view stratum (input stratum index, interval)
__global__ void split_pairs_kernel(int64_t n, const int32_t *stop, const int32_t *start, const int32_t *kidx,
                                   const int32_t *cuts, int32_t C, const int64_t *pair_off, uint64_t *key, uint32_t *pay) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
    int32_t klo, khi;
    split_range(cuts, C, stop[r], start, r, &klo, &khi);
    for (int32_t k = klo; k <= khi; ++k) {
      const int64_t q = pair_off[r] + (k - klo);
      key[q] = uint64_t(kidx[r]) * uint64_t(C + 1) + uint64_t(k);
      pay[q] = uint32_t(r);
    }
  }
}

// view rows in (stratum, interval, input row) order; inv maps each pair to its view row
__global__ void split_rows_kernel(int64_t M, const uint64_t *key, const uint32_t *pay, const int32_t *cuts, int32_t C,
                                  const int32_t *stop, const int32_t *start, const uint8_t *event, const int64_t *pair_off,
                                  int32_t *v_stop, int32_t *v_start, uint8_t *v_event, int32_t *v_stratum, int32_t *inv) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < M; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = pay[i];
    const int32_t k = int32_t(key[i] % uint64_t(C + 1));
    int32_t klo, khi;
    split_range(cuts, C, stop[r], start, r, &klo, &khi);
    v_stop[i] = k < C ? min(stop[r], cuts[k]) : stop[r];
    v_event[i] = (event[r] && k == khi) ? 1 : 0;
    if (v_start) v_start[i] = start[r];
    v_stratum[i] = int32_t(key[i]);
    inv[pair_off[r] + (k - klo)] = int32_t(i);
  }
}

__global__ void split_entry_count_kernel(int64_t nnz, const int32_t *row_idx, const int32_t *cnt, int32_t *ecnt) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < nnz; q += int64_t(gridDim.x) * blockDim.x)
    ecnt[q] = cnt[row_idx[q]];
}

// one view entry per (nonzero, interval of its row): key = (view column, view stratum); a
// stable sort on the key leaves the entries of one (column, stratum) in input-row order,
// which is view-row order
__global__ void split_entries_kernel(const ColSeg *segs, const int32_t *row_idx, const int32_t *stop,
                                     const int32_t *start, const int32_t *kidx, const int32_t *cuts, int32_t C, uint64_t Kv,
                                     const int32_t *col_base, const uint8_t *col_tvc, const int64_t *pair_off,
                                     const int32_t *inv, const int64_t *eoff, uint64_t *key, uint32_t *pay, int32_t *g_row,
                                     int64_t *g_src) {
  const ColSeg sg = segs[blockIdx.x];
  const int32_t base = col_base[sg.j];
  const bool tvc = col_tvc[sg.j] != 0;
  for (int64_t q = sg.a + threadIdx.x; q < sg.b; q += kSegThreads) {
    const int32_t r = row_idx[q];
    int32_t klo, khi;
    split_range(cuts, C, stop[r], start, r, &klo, &khi);
    for (int32_t k = klo; k <= khi; ++k) {
      const int64_t g = eoff[q] + (k - klo);
      const uint64_t c = uint64_t(base + (tvc ? k : 0));
      key[g] = c * Kv + uint64_t(kidx[r]) * uint64_t(C + 1) + uint64_t(k);
      pay[g] = uint32_t(g);
      g_row[g] = inv[pair_off[r] + (k - klo)];
      if (g_src) g_src[g] = q;
    }
  }
}

__global__ void split_fill_kernel(int64_t E, const uint64_t *key, const uint32_t *pay, uint64_t Kv, int32_t p_view,
                                  const int32_t *g_row, const int64_t *g_src, const double *val, int32_t *v_row,
                                  double *v_val, int64_t *v_col_ptr) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < E; e += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t g = pay[e];
    v_row[e] = g_row[g];
    if (v_val) v_val[e] = val[g_src[g]];
    const int64_t c = int64_t(key[e] / Kv);
    const int64_t cp = e == 0 ? -1 : int64_t(key[e - 1] / Kv);
    for (int64_t cc = cp + 1; cc <= c; ++cc) v_col_ptr[cc] = e;
    if (e == E - 1)
      for (int64_t cc = c + 1; cc <= p_view; ++cc) v_col_ptr[cc] = E;
  }
}

int split_columns(int32_t p, const cox_split *sp, int32_t *p_view, std::string *err) {
  if (!sp || sp->n_cuts < 1 || !sp->cuts || sp->n_tvc < 0 || sp->n_tvc > p || (sp->n_tvc > 0 && !sp->tvc_cols)) {
    *err = "cox_split: need n_cuts >= 1 with cuts, and 0 <= n_tvc <= p with tvc_cols";
    return COX_E_INVALID;
  }
  for (int32_t c = 1; c < sp->n_cuts; ++c)
    if (!(sp->cuts[c - 1] < sp->cuts[c])) {
      *err = "cox_split: cuts must be strictly ascending";
      return COX_E_INVALID;
    }
  for (int32_t m = 0; m < sp->n_tvc; ++m)
    if (sp->tvc_cols[m] < 0 || sp->tvc_cols[m] >= p || (m > 0 && !(sp->tvc_cols[m - 1] < sp->tvc_cols[m]))) {
      *err = "cox_split: tvc_cols must be strictly ascending column indices in [0, p)";
      return COX_E_INVALID;
    }
  const int64_t pv = int64_t(p) + int64_t(sp->n_tvc) * sp->n_cuts;
  if (pv >= (int64_t(1) << 31)) {
    *err = "cox_split: too many view columns";
    return COX_E_INVALID;
  }
  *p_view = int32_t(pv);
  return COX_OK;
}

int build_split_view(const cox_data *in, const cox_split *sp, cudaStream_t s, BufferSet &B, cox_data *view,
                     std::string *err) {
  Scratch sc;
  int32_t p_view = 0;
  int rc = split_columns(in ? in->p : 0, sp, &p_view, err);
  if (rc) return rc;
  Staged st;
  if ((rc = stage_inputs(in, sc, s, &st, err))) return rc;
  const int64_t n = st.n, nnz = st.nnz;
  const int32_t p = st.p, C = sp->n_cuts;
  // cuts and the column map on the device
  std::vector<int32_t> h_base(size_t(p) + 1, 0);
  std::vector<uint8_t> h_tvc(size_t(p) + 1, 0);
  for (int32_t m = 0; m < sp->n_tvc; ++m) h_tvc[sp->tvc_cols[m]] = 1;
  for (int32_t j = 0, c = 0; j < p; ++j) {
    h_base[j] = c;
    c += h_tvc[j] ? C + 1 : 1;
  }
  int32_t *cuts = static_cast<int32_t *>(sc.get(size_t(C) * sizeof(int32_t)));
  int32_t *col_base = static_cast<int32_t *>(sc.get((size_t(p) + 1) * sizeof(int32_t)));
  uint8_t *col_tvc = static_cast<uint8_t *>(sc.get(size_t(p) + 1));
  if (!cuts || !col_base || !col_tvc) return COX_E_OOM;
  if (cudaMemcpyAsync(cuts, sp->cuts, size_t(C) * sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(col_base, h_base.data(), (size_t(p) + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(col_tvc, h_tvc.data(), size_t(p) + 1, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return COX_E_CUDA;

  // stratum index of every row
  const int64_t nn = n > 0 ? n : 1;
  int32_t *seg_flag = static_cast<int32_t *>(sc.get(nn * sizeof(int32_t)));
  int32_t *ev_flag = static_cast<int32_t *>(sc.get(nn * sizeof(int32_t)));
  int64_t *seg_pre = static_cast<int64_t *>(sc.get(nn * sizeof(int64_t)));
  int32_t *kidx = static_cast<int32_t *>(sc.get(nn * sizeof(int32_t)));
  int32_t *cnt = static_cast<int32_t *>(sc.get(nn * sizeof(int32_t)));
  int64_t *pair_off = static_cast<int64_t *>(sc.get(nn * sizeof(int64_t)));
  if (!seg_flag || !ev_flag || !seg_pre || !kidx || !cnt || !pair_off) return COX_E_OOM;
  int64_t K = 0, M = 0;
  if (n > 0) {
    count_launches(1);
    row_flags_kernel<<<grid_for(n), 256, 0, s>>>(n, st.stop, st.event, st.stratum, seg_flag, ev_flag);
    if ((rc = exclusive_scan(seg_flag, n, seg_pre, &K, sc, s))) return rc;
    count_launches(1);
    row_stratum_index_kernel<<<grid_for(n), 256, 0, s>>>(n, seg_flag, seg_pre, kidx);
    count_launches(1);
    split_count_kernel<<<grid_for(n), 256, 0, s>>>(n, st.stop, st.start, cuts, C, cnt);
    if ((rc = exclusive_scan(cnt, n, pair_off, &M, sc, s))) return rc;
  }
  const uint64_t Kv = uint64_t(K > 0 ? K : 1) * uint64_t(C + 1);
  if (M >= (int64_t(1) << 30) || Kv >= (uint64_t(1) << 31)) {
    *err = "cox_split: the view needs fewer than 2^30 rows and 2^31 strata";
    return COX_E_INVALID;
  }
  // view rows
  const int64_t mm = M > 0 ? M : 1;
  int32_t *v_stop = static_cast<int32_t *>(B.get(mm * sizeof(int32_t)));
  int32_t *v_start = st.start ? static_cast<int32_t *>(B.get(mm * sizeof(int32_t))) : nullptr;
  uint8_t *v_event = static_cast<uint8_t *>(B.get(mm));
  int32_t *v_stratum = static_cast<int32_t *>(B.get(mm * sizeof(int32_t)));
  int32_t *inv = static_cast<int32_t *>(sc.get(mm * sizeof(int32_t)));
  if (!v_stop || (st.start && !v_start) || !v_event || !v_stratum || !inv) return COX_E_OOM;
  if (M > 0) {
    uint64_t *key = static_cast<uint64_t *>(sc.get(M * sizeof(uint64_t)));
    uint32_t *pay = static_cast<uint32_t *>(sc.get(M * sizeof(uint32_t)));
    if (!key || !pay) return COX_E_OOM;
    count_launches(1);
    split_pairs_kernel<<<grid_for(n), 256, 0, s>>>(n, st.stop, st.start, kidx, cuts, C, pair_off, key, pay);
    std::vector<int> bits;
    for (int b = 0; b < bits_needed(Kv - 1); ++b) bits.push_back(b);
    if ((rc = radix_sort(key, pay, M, bits, sc, s))) return rc;
    count_launches(1);
    split_rows_kernel<<<grid_for(M), 256, 0, s>>>(M, key, pay, cuts, C, st.stop, st.start, st.event, pair_off, v_stop,
                                                    v_start, v_event, v_stratum, inv);
  }
  // view columns
  int64_t E = 0;
  int32_t *ecnt = static_cast<int32_t *>(sc.get((nnz > 0 ? nnz : 1) * sizeof(int32_t)));
  int64_t *eoff = static_cast<int64_t *>(sc.get((nnz > 0 ? nnz : 1) * sizeof(int64_t)));
  if (!ecnt || !eoff) return COX_E_OOM;
  if (nnz > 0) {
    count_launches(1);
    split_entry_count_kernel<<<grid_for(nnz), 256, 0, s>>>(nnz, st.row_idx, cnt, ecnt);
    if ((rc = exclusive_scan(ecnt, nnz, eoff, &E, sc, s))) return rc;
  }
  if (E >= (int64_t(1) << 32)) {
    *err = "cox_split: the view needs fewer than 2^32 nonzeros";
    return COX_E_INVALID;
  }
  const int64_t ee = E > 0 ? E : 1;
  int64_t *v_col_ptr = static_cast<int64_t *>(B.get((size_t(p_view) + 1) * sizeof(int64_t)));
  int32_t *v_row = static_cast<int32_t *>(B.get(ee * sizeof(int32_t)));
  double *v_val = st.val ? static_cast<double *>(B.get(ee * sizeof(double))) : nullptr;
  if (!v_col_ptr || !v_row || (st.val && !v_val)) return COX_E_OOM;
  cudaMemsetAsync(v_col_ptr, 0, (size_t(p_view) + 1) * sizeof(int64_t), s);
  if (E > 0) {
    uint64_t *key = static_cast<uint64_t *>(sc.get(E * sizeof(uint64_t)));
    uint32_t *pay = static_cast<uint32_t *>(sc.get(E * sizeof(uint32_t)));
    int32_t *g_row = static_cast<int32_t *>(sc.get(E * sizeof(int32_t)));
    int64_t *g_src = st.val ? static_cast<int64_t *>(sc.get(E * sizeof(int64_t))) : nullptr;
    if (!key || !pay || !g_row || (st.val && !g_src)) return COX_E_OOM;
    count_launches(1);
    split_entries_kernel<<<unsigned(st.nseg), kSegThreads, 0, s>>>(st.segs, st.row_idx, st.stop, st.start, kidx, cuts, C,
                                                                   Kv, col_base, col_tvc, pair_off, inv, eoff, key, pay,
                                                                   g_row, g_src);
    std::vector<int> bits;
    for (int b = 0; b < bits_needed(uint64_t(p_view) * Kv - 1); ++b) bits.push_back(b);
    if ((rc = radix_sort(key, pay, E, bits, sc, s))) return rc;
    count_launches(1);
    split_fill_kernel<<<grid_for(E), 256, 0, s>>>(E, key, pay, Kv, p_view, g_row, g_src, st.val, v_row, v_val,
                                                   v_col_ptr);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaPeekAtLastError() != cudaSuccess) {
    *err = "cox_split: view kernels failed";
    return COX_E_CUDA;
  }
  *view = cox_data{};
  view->n_rows = M;
  view->p = p_view;
  view->stop = v_stop;
  view->start = v_start;
  view->event = v_event;
  view->stratum = v_stratum;
  view->col_ptr = v_col_ptr;
  view->row_idx = v_row;
  view->val = v_val;
  return COX_OK;
}

// ------------------------------------------------------------------ training-fold view
// The rows of a data set whose fold id differs from k, in their order (so still sorted), with
// the CSC restricted to them: row ranks by a prefix count of the kept rows, entries by a prefix
// count of the kept entries (a column's kept entries stay contiguous and ascending).
__global__ void fold_keep_kernel(int64_t n, const int32_t *fold, int32_t k, int32_t K, int32_t *keep, int32_t *err) {
  int32_t e = 0;
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
    const int32_t f = fold[r];
    if (f < 0 || f >= K) e = 1;
    keep[r] = f != k ? 1 : 0;
  }
  if (e) atomicOr(err, e);
}

__global__ void subset_rows_kernel(int64_t n, const int32_t *keep, const int64_t *pre, const int32_t *stop,
                                   const int32_t *start, const uint8_t *event, const int32_t *stratum, int32_t *v_stop,
                                   int32_t *v_start, uint8_t *v_event, int32_t *v_stratum) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
    if (!keep[r]) continue;
    const int64_t i = pre[r];
    v_stop[i] = stop[r];
    v_event[i] = event[r];
    if (v_start) v_start[i] = start[r];
    if (v_stratum) v_stratum[i] = stratum[r];
  }
}

__global__ void subset_entry_flags_kernel(int64_t nnz, const int32_t *row_idx, const int32_t *keep, int32_t *eflag) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < nnz; q += int64_t(gridDim.x) * blockDim.x)
    eflag[q] = keep[row_idx[q]];
}

__global__ void subset_entries_kernel(int64_t nnz, const int32_t *row_idx, const double *val, const int32_t *eflag,
                                      const int64_t *epre, const int64_t *row_pre, int32_t *v_row, double *v_val) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < nnz; q += int64_t(gridDim.x) * blockDim.x) {
    if (!eflag[q]) continue;
    const int64_t e = epre[q];
    v_row[e] = int32_t(row_pre[row_idx[q]]);
    if (v_val) v_val[e] = val[q];
  }
}

__global__ void subset_colptr_kernel(int32_t p, const int64_t *col_ptr, int64_t nnz, const int64_t *epre, int64_t E,
                                     int64_t *v_col_ptr) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j <= p; j += int64_t(gridDim.x) * blockDim.x) {
    const int64_t a = j < p ? col_ptr[j] : nnz;
    v_col_ptr[j] = a < nnz ? epre[a] : E;
  }
}

int build_fold_view(const cox_data *in, const int32_t *fold, int32_t k, int32_t K, cudaStream_t s, BufferSet &B,
                    cox_data *view, std::string *err) {
  Scratch sc;
  if (!fold || K < 2 || k < 0 || k >= K) {
    *err = "cox_cv_path: need fold ids and 0 <= k < n_folds, n_folds >= 2";
    return COX_E_INVALID;
  }
  Staged st;
  int rc = stage_inputs(in, sc, s, &st, err);
  if (rc) return rc;
  const int64_t n = st.n, nnz = st.nnz;
  const int32_t p = st.p;
  const int64_t nn = n > 0 ? n : 1;
  const int32_t *dfold = device_view(fold, n, sc, s, &rc);
  int32_t *keep = static_cast<int32_t *>(sc.get(nn * sizeof(int32_t)));
  int64_t *row_pre = static_cast<int64_t *>(sc.get(nn * sizeof(int64_t)));
  int32_t *d_err = static_cast<int32_t *>(sc.get(sizeof(int32_t)));
  if (rc || !keep || !row_pre || !d_err) return rc ? rc : COX_E_OOM;
  cudaMemsetAsync(d_err, 0, sizeof(int32_t), s);
  int64_t M = 0;
  if (n > 0) {
    count_launches(1);
    fold_keep_kernel<<<grid_for(n), 256, 0, s>>>(n, dfold, k, K, keep, d_err);
    if ((rc = exclusive_scan(keep, n, row_pre, &M, sc, s))) return rc;   // synchronizes
  }
  int32_t h_err = 0;
  if (cudaMemcpy(&h_err, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return COX_E_CUDA;
  if (h_err) {
    *err = "cox_cv_path: fold ids must lie in [0, n_folds)";
    return COX_E_INVALID;
  }
  const int64_t mm = M > 0 ? M : 1;
  int32_t *v_stop = static_cast<int32_t *>(B.get(mm * sizeof(int32_t)));
  int32_t *v_start = st.start ? static_cast<int32_t *>(B.get(mm * sizeof(int32_t))) : nullptr;
  uint8_t *v_event = static_cast<uint8_t *>(B.get(mm));
  int32_t *v_stratum = st.stratum ? static_cast<int32_t *>(B.get(mm * sizeof(int32_t))) : nullptr;
  if (!v_stop || (st.start && !v_start) || !v_event || (st.stratum && !v_stratum)) return COX_E_OOM;
  if (n > 0) {
    count_launches(1);
    subset_rows_kernel<<<grid_for(n), 256, 0, s>>>(n, keep, row_pre, st.stop, st.start, st.event, st.stratum, v_stop,
                                                   v_start, v_event, v_stratum);
  }
  const int64_t ne = nnz > 0 ? nnz : 1;
  int32_t *eflag = static_cast<int32_t *>(sc.get(ne * sizeof(int32_t)));
  int64_t *epre = static_cast<int64_t *>(sc.get(ne * sizeof(int64_t)));
  if (!eflag || !epre) return COX_E_OOM;
  int64_t E = 0;
  if (nnz > 0) {
    count_launches(1);
    subset_entry_flags_kernel<<<grid_for(nnz), 256, 0, s>>>(nnz, st.row_idx, keep, eflag);
    if ((rc = exclusive_scan(eflag, nnz, epre, &E, sc, s))) return rc;
  }
  int64_t *v_col_ptr = static_cast<int64_t *>(B.get((size_t(p) + 1) * sizeof(int64_t)));
  int32_t *v_row = static_cast<int32_t *>(B.get((E > 0 ? E : 1) * sizeof(int32_t)));
  double *v_val = st.val ? static_cast<double *>(B.get((E > 0 ? E : 1) * sizeof(double))) : nullptr;
  if (!v_col_ptr || !v_row || (st.val && !v_val)) return COX_E_OOM;
  if (nnz > 0) {
    count_launches(1);
    subset_entries_kernel<<<grid_for(nnz), 256, 0, s>>>(nnz, st.row_idx, st.val, eflag, epre, row_pre, v_row, v_val);
  }
  count_launches(1);
  subset_colptr_kernel<<<grid_for(int64_t(p) + 1), 256, 0, s>>>(p, st.col_ptr, nnz, epre, E, v_col_ptr);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaPeekAtLastError() != cudaSuccess) {
    *err = "cox_cv_path: fold view kernels failed";
    return COX_E_CUDA;
  }
  *view = cox_data{};
  view->n_rows = M;
  view->p = p;
  view->stop = v_stop;
  view->start = v_start;
  view->event = v_event;
  view->stratum = v_stratum;
  view->col_ptr = v_col_ptr;
  view->row_idx = v_row;
  view->val = v_val;
  return COX_OK;
}

}  // namespace coxgb
