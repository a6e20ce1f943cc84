// Segmented inclusive scan with the paper's flag-value operator (arXiv 2310.16238 §2.6):
//   (f_i, a_i) (+)s (f_j, a_j) = (f_i | f_j, f_j ? a_j : a_i + a_j),
// i.e. b_i = sum of a over [last head at or before i, i]. One pass over the data: each CTA
// scans a tile of 4096 values in registers (16 consecutive values per thread), combines
// threads with a warp-shuffle segmented scan, and takes its carry from earlier tiles by a
// decoupled look-back (Merrill & Garland, "Single-pass Parallel Prefix Scan with Decoupled
// Look-back", 2016) over per-tile tagged records kept in scratch memory.
#include <cuda_runtime.h>

#include <cstdint>
#include <atomic>
#include <mutex>
#include <string>

#include "cox.h"
#include "cox_internal.h"
#include "prep.h"

namespace coxgb {

constexpr int kSegThreads = 256;
constexpr int kSegItems = 16;
constexpr int kSegTile = kSegThreads * kSegItems;

// Scratch layout (bytes): [0] ticket, [4] exited, [8] error, then per tile two records of 16 bytes,
// its aggregate and its inclusive value. A record is two 64-bit words, (tag << 32) | the low and
// (tag << 32) | the high 32 bits of the double: each word is stored and loaded whole, so a reader
// that sees the tag in both words has the value (no fence to publish, no flag to acquire). The
// whole scratch is zeroed before every call, so the tag is a constant.
constexpr uint64_t kSegTag = 0x5ca1ull;
struct SegScratchView {
  uint32_t *ticket, *exited, *error;
  uint64_t *rec;   // [tile][2 records][2 words]
};

__host__ __device__ constexpr size_t seg_scratch_bytes(int64_t tiles) { return 16 + 32 * size_t(tiles); }

__device__ inline SegScratchView seg_view(unsigned char *s, int64_t) {
  SegScratchView v;
  v.ticket = reinterpret_cast<uint32_t *>(s);
  v.exited = reinterpret_cast<uint32_t *>(s + 4);
  v.error = reinterpret_cast<uint32_t *>(s + 8);
  v.rec = reinterpret_cast<uint64_t *>(s + 16);
  return v;
}

__device__ __forceinline__ void seg_put(uint64_t *r, double x) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x));
  const uint64_t w0 = (kSegTag << 32) | (b & 0xffffffffull), w1 = (kSegTag << 32) | (b >> 32);
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(r), "l"(w0), "l"(w1) : "memory");
}
// the record's value when both words carry the tag
__device__ __forceinline__ bool seg_get(const uint64_t *r, double *x) {
  uint64_t w0, w1;
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(w0), "=l"(w1) : "l"(r) : "memory");
  if ((w0 >> 32) != kSegTag || (w1 >> 32) != kSegTag) return false;
  *x = __longlong_as_double(static_cast<long long>((w1 << 32) | (w0 & 0xffffffffull)));
  return true;
}

__device__ __forceinline__ double seg_ld_nc(const double2 *p, double &hi) {
  const double2 x = __ldg(p);
  hi = x.y;
  return x.x;
}

__global__ void __launch_bounds__(kSegThreads, 3) segscan_kernel(const double *a, const uint8_t *__restrict__ f,
                                                                 int64_t n, double *b, unsigned char *scratch,
                                                                 int64_t tiles, long long spin) {
  constexpr int kW = kSegThreads / 32;
  const SegScratchView S = seg_view(scratch, tiles);
  __shared__ int64_t s_tile;
  __shared__ double s_wsum[kW];
  __shared__ int s_wflag[kW];
  __shared__ double s_wex[kW];    // carry into each warp from the tile's earlier warps
  __shared__ int s_wexf[kW];      // ... which stops at a head
  __shared__ double s_carry;      // carry into the tile from earlier tiles
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // 16-byte loads and stores of a thread's 16 values and flags when every array is 16-byte aligned
  const bool vec = ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(f) |
                     reinterpret_cast<uintptr_t>(b)) & 15u) == 0u;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(S.ticket, 1u);
    __syncthreads();
    const int64_t t = s_tile;
    if (t >= tiles) break;
    const int64_t base = t * kSegTile + int64_t(tid) * kSegItems;
    const bool full = vec && (t + 1) * kSegTile <= n;   // uniform over the tile
    double v[kSegItems];
    uint32_t fm = 0;
    if (full) {
      const double2 *a2 = reinterpret_cast<const double2 *>(a + base);
#pragma unroll
      for (int k = 0; k < kSegItems / 2; ++k) v[2 * k] = seg_ld_nc(a2 + k, v[2 * k + 1]);
      const uint4 fw = __ldg(reinterpret_cast<const uint4 *>(f + base));
      const uint32_t w4[4] = {fw.x, fw.y, fw.z, fw.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {   // a nonzero flag byte -> its bit
        const uint32_t m = __vcmpne4(w4[q], 0u);
        fm |= (((m >> 7) & 1u) | ((m >> 14) & 2u) | ((m >> 21) & 4u) | ((m >> 28) & 8u)) << (4 * q);
      }
    } else {
#pragma unroll
      for (int k = 0; k < kSegItems; ++k) {
        const int64_t i = base + k;
        v[k] = i < n ? a[i] : 0.0;
        if (i < n && f[i]) fm |= 1u << k;
      }
    }
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kSegItems; ++k) {
      acc = ((fm >> k) & 1u) ? v[k] : acc + v[k];
      v[k] = acc;
    }
    // warp inclusive scan of (flag, value) pairs, left to right
    int fl = fm != 0u;
    double x = acc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, x, off);
      const int yf = __shfl_up_sync(0xffffffffu, fl, off);
      if (lane >= off) {
        if (!fl) x = y + x;
        fl |= yf;
      }
    }
    if (lane == 31) {
      s_wsum[warp] = x;
      s_wflag[warp] = fl;
    }
    double ex = __shfl_up_sync(0xffffffffu, x, 1);
    int exf = __shfl_up_sync(0xffffffffu, fl, 1);
    if (lane == 0) {
      ex = 0.0;
      exf = 0;
    }
    __syncthreads();
    if (warp == 0) {
      // the tile's warps combined by shuffles; the tile aggregate published; then one look-back
      // over up to 32 earlier tiles at a time
      double w = lane < kW ? s_wsum[lane] : 0.0;
      int wf = lane < kW ? s_wflag[lane] : 0;
#pragma unroll
      for (int off = 1; off < kW; off <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, w, off);
        const int yf = __shfl_up_sync(0xffffffffu, wf, off);
        if (lane >= off) {
          if (!wf) w = y + w;
          wf |= yf;
        }
      }
      double we = __shfl_up_sync(0xffffffffu, w, 1);
      int wef = __shfl_up_sync(0xffffffffu, wf, 1);
      if (lane < kW) {
        s_wex[lane] = lane == 0 ? 0.0 : we;
        s_wexf[lane] = lane == 0 ? 0 : wef;
      }
      const double c = __shfl_sync(0xffffffffu, w, kW - 1);
      const int cf = __shfl_sync(0xffffffffu, wf, kW - 1);
      // a tile with a head publishes its sums from that head on as final (inclusive) at once
      if (lane == 0) seg_put(S.rec + 4 * t + (cf ? 2 : 0), c);
      double carry = 0.0;
      bool timed_out = false;
      const long long t0 = clock64();
      for (int64_t u0 = t - 1; u0 >= 0;) {
        const int64_t u = u0 - lane;   // lane 0 the nearest earlier tile; before tile 0 an inclusive 0
        double val = 0.0;
        int first = 32;
        for (;;) {
          int vi = 1, va = 0;
          val = 0.0;
          if (u >= 0) {
            vi = seg_get(S.rec + 4 * u + 2, &val);
            if (!vi) va = seg_get(S.rec + 4 * u, &val);
          }
          const uint32_t inc = __ballot_sync(0xffffffffu, vi);
          const uint32_t pend = __ballot_sync(0xffffffffu, !(vi || va));
          first = inc ? __ffs(inc) - 1 : 32;
          const uint32_t need = first >= 31 ? 0xffffffffu : ((2u << first) - 1u);   // lanes 0..first
          if ((pend & need) == 0u) break;
          if (clock64() - t0 > spin) {
            timed_out = true;
            break;
          }
          __nanosleep(32);
        }
        if (timed_out) {
          if (lane == 0) atomicExch(S.error, 1u);
          break;
        }
        if (lane > first) val = 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) val += __shfl_xor_sync(0xffffffffu, val, off);
        carry += val;
        if (first < 32) break;
        u0 -= 32;
      }
      if (lane == 0) {
        s_carry = carry;
        if (!cf) seg_put(S.rec + 4 * t + 2, carry + c);
      }
    }
    __syncthreads();
    // exclusive carry of this thread: earlier threads of the warp, earlier warps, earlier tiles
    if (!exf) {
      ex = s_wex[warp] + ex;
      exf = s_wexf[warp];
      if (!exf) ex = s_carry + ex;
    }
#pragma unroll
    for (int k = 0; k < kSegItems; ++k)
      if ((fm & ((2u << k) - 1u)) == 0u) v[k] = ex + v[k];
    if (full) {
      double2 *b2 = reinterpret_cast<double2 *>(b + base);
#pragma unroll
      for (int k = 0; k < kSegItems / 2; ++k) b2[k] = make_double2(v[2 * k], v[2 * k + 1]);
    } else {
#pragma unroll
      for (int k = 0; k < kSegItems; ++k) {
        const int64_t i = base + k;
        if (i < n) b[i] = v[k];
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(S.exited, 1u) == gridDim.x - 1) {
      *S.ticket = 0u;
      *S.exited = 0u;
    }
  }
}

// Resident CTAs of segscan_kernel on a device (occupancy x SMs), computed once per device; the
// array is indexed by device ordinal and written under a lock, so concurrent first calls and
// devices with different SM counts each get their own value.
constexpr int kGridDevices = 64;
static std::atomic<int> g_seg_cap[kGridDevices];

static int seg_grid(int64_t tiles) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kGridDevices) {
    cudaGetLastError();
    dev = -1;
  }
  int cap = dev >= 0 ? g_seg_cap[dev].load(std::memory_order_acquire) : 0;
  if (!cap) {
    int per = 0, nsm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, segscan_kernel, kSegThreads, 0);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev >= 0 ? dev : 0);
    cap = (per > 0 ? per : 1) * (nsm > 0 ? nsm : 1);
    if (dev >= 0) g_seg_cap[dev].store(cap, std::memory_order_release);
  }
  return int(tiles < cap ? tiles : cap);
}

// Runs the scan with scratch at `scratch` (already zeroed: seg_scratch_bytes(T) bytes).
static int segscan_run(const double *a, const uint8_t *f, int64_t n, double *b, unsigned char *scratch, int64_t tiles,
                       cudaStream_t s, std::string *err) {
  count_launches(1);
  segscan_kernel<<<seg_grid(tiles), kSegThreads, 0, s>>>(a, f, n, b, scratch, tiles, wait_limit());
  if (cudaGetLastError() != cudaSuccess) { *err = "cox_segscan: launch failed"; return COX_E_CUDA; }
  uint32_t e = 0;
  if (cudaMemcpyAsync(&e, scratch + 8, sizeof(e), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    *err = "cox_segscan: execution failed";
    return COX_E_CUDA;
  }
  if (e) { *err = "cox_segscan: a look-back wait exceeded its bound"; return COX_E_TIMEOUT; }
  return COX_OK;
}

static int segscan_check(const double *a, const uint8_t *f, int64_t n, double *b, std::string *err) {
  if (n < 0 || (n > 0 && (!a || !f || !b))) { *err = "cox_segscan: null or negative argument"; return COX_E_INVALID; }
  if (n > 0 && (!pointer_on_device(a) || !pointer_on_device(f) || !pointer_on_device(b))) {
    *err = "cox_segscan: a, head_flags and out must be device memory";
    return COX_E_INVALID;
  }
  return COX_OK;
}

}  // namespace coxgb

using namespace coxgb;

extern "C" int cox_segscan(const double *a, const uint8_t *head_flags, int64_t n, double *out, void *stream) {
  std::string err;
  int rc = segscan_check(a, head_flags, n, out, &err);
  if (rc || n == 0) return rc ? set_last_error(rc, err.c_str()) : COX_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t tiles = (n + kSegTile - 1) / kSegTile;
  const size_t bytes = seg_scratch_bytes(tiles);
  unsigned char *scratch = static_cast<unsigned char *>(dev_alloc(bytes));
  if (!scratch) return set_last_error(COX_E_OOM, "cox_segscan: scratch allocation failed");
  rc = cudaMemsetAsync(scratch, 0, bytes, s) == cudaSuccess ? COX_OK : COX_E_CUDA;
  if (!rc) rc = segscan_run(a, head_flags, n, out, scratch, tiles, s, &err);
  else err = "cox_segscan: memset failed";
  cudaStreamSynchronize(s);
  dev_free(scratch, bytes);
  return rc ? set_last_error(rc, err.c_str()) : COX_OK;
}

// ---------------------------------------------------------------- allocation-free variant
// Callers that must not allocate device memory during a call use cox_segscan_noalloc: the
// look-back scratch lives in this file-scope array instead of the library allocator. Every
// GPU that loads the library holds these bytes until the process exits.
namespace coxgb {
constexpr int64_t kStaticMaxTiles = 4096;   // 4096 tiles x 4096 values = 16,777,216 values
constexpr size_t kStaticScratchBytes = seg_scratch_bytes(kStaticMaxTiles);
static __device__ __align__(256) unsigned char g_segscan_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
// Per device: the array's device address and the CUDA context it was looked up in. A context
// destroyed and recreated (cudaDeviceReset) may load the module at another address, so a cached
// address is reused only while the current context is the one it came from.
struct StaticSlot {
  void *ctx;
  unsigned char *addr;
};
static StaticSlot g_static_slot[kMaxDevices] = {};

// The driver's cuCtxGetCurrent, fetched through the runtime (no link-time dependency on libcuda).
using CtxGetCurrentFn = int (*)(void **);
static CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  return fn;
}

static void *current_context() {
  void *c = nullptr;
  if (CtxGetCurrentFn f = ctx_get_current())
    if (f(&c) != 0) c = nullptr;
  return c;
}

// Device address of the static scratch on the current device (host code cannot use the array's
// name as a device address): looked up with cudaGetSymbolAddress on the first call on each device
// and again whenever the device's current context has changed since.
static int static_scratch_address(unsigned char **out, std::string *err) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    *err = "cox_segscan_noalloc: no usable current device";
    return COX_E_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  StaticSlot &slot = g_static_slot[dev];
  void *ctx = current_context();
  if (!slot.addr || !ctx || slot.ctx != ctx) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_segscan_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      *err = std::string("cox_segscan_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      return COX_E_CUDA;
    }
    slot.addr = static_cast<unsigned char *>(p);
    slot.ctx = current_context();   // the lookup makes the device's primary context current
  }
  *out = slot.addr;
  return COX_OK;
}
}  // namespace coxgb

extern "C" int cox_segscan_noalloc(const double *a, const uint8_t *head_flags, int64_t n, double *out, void *stream) {
  std::string err;
  int rc = segscan_check(a, head_flags, n, out, &err);
  if (rc) return set_last_error(rc, err.c_str());
  if (n == 0) return COX_OK;
  const int64_t tiles = (n + kSegTile - 1) / kSegTile;
  if (tiles > kStaticMaxTiles)
    return set_last_error(COX_E_INVALID, "cox_segscan_noalloc: n exceeds 16,777,216 values (the static scratch limit)");
  unsigned char *scratch = nullptr;
  if ((rc = static_scratch_address(&scratch, &err))) return set_last_error(rc, err.c_str());
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: clear the ticket, error and the tiles' records
  if (cudaMemsetAsync(scratch, 0, seg_scratch_bytes(tiles), s) != cudaSuccess)
    return set_last_error(COX_E_CUDA, "cox_segscan_noalloc: clearing the static scratch failed");
  rc = segscan_run(a, head_flags, n, out, scratch, tiles, s, &err);
  return rc ? set_last_error(rc, err.c_str()) : COX_OK;
}
