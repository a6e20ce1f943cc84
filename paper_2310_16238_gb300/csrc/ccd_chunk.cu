// FP32C coordinate-step kernel for cyclic coordinate descent on the stratified / time-varying
// Cox partial likelihood (arXiv 2310.16238, §2.4-§2.7): one launch advances every fit in its work
// list by one coordinate.
//
// A fit's risk sequence is cut into tiles of up to 4,096 positions and its tiles into contiguous
// chunks; a work item is one chunk. One CTA of 128 threads streams the chunk's tiles right to left,
// the direction of the suffix sums, staging the next tile with cp.async while it scans the current:
//   * at the chunk's start, the previous coordinate's pending update at the chunk's entries of that
//     column (eta += x dbeta, eq. parallel_xb; v = +-exp(eta - shift), eq. parallel_d);
//   * per tile, each thread owns 32 consecutive positions. The stratum-segmented suffix sums of v
//     (strata are segments of §2.6's flag-value operator) are plain float sums inside blocks of 8
//     positions and compensated (TwoSum) sums above them; the column's x v and x^2 v sums come
//     from a walk over the thread's nonzeros only. Warp-shuffle segmented scans and a combine over
//     the 4 warps give each thread its carry from the chunk's later positions, and the tile's tie
//     groups then read their risk-set sums head-parallel and add the ratios of eqs.
//     (parallel_g)/(parallel_h) to the chunk's partial;
//   * tie groups whose risk set runs past the chunk's end keep their local sums in a per-group
//     scratch until the chunk's carry arrives: one decoupled look-back per chunk over epoch-tagged
//     64-bit words (each word carries its own tag in its low mantissa bits, so publishing needs no
//     memory fence and a reader needs no second load);
//   * the CTA that finishes a fit's last chunk reduces the chunk partials in a fixed order and
//     takes the coordinate step (§2.4).
// A tile's sums are thus written to shared memory once and read at its tie groups only; the only
// global writes are the pending update's eta and v, the deferred groups' scratch and the partials.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <climits>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "ccd_common.cuh"
#include "cox.h"
#include "cox_internal.h"

namespace coxgb {
namespace {

constexpr int kCT = 128;        // threads per CTA
constexpr int kCI = 32;         // positions per thread
constexpr int kCW = kCT / 32;   // warps per CTA
constexpr int kPF = 2;          // events-per-group values each thread prefetches for its first groups
constexpr int kES = 2 * kCT;    // column entries of the next tile copied ahead with its tile (2 per thread)
#ifndef COXGB_CHUNK_MIN_CTAS
#define COXGB_CHUNK_MIN_CTAS 4  // resident CTAs per SM the register allocation is held to
#endif
static_assert(kCT * kCI == kChunkTile, "a tile is one position range per thread");

using P = PF32C;
using Acc = P::Acc;

#if COX_TRACE_ON
// Phase stamps (ns) of one traced launch: [work item][8] (diagnostic builds only).
__device__ uint64_t *g_chunk_trace = nullptr;
#define CHUNK_STAMP(k)                                                              \
  do {                                                                              \
    if (g_chunk_trace && tid == 0) {                                                \
      uint64_t t_;                                                                  \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));                        \
      g_chunk_trace[8 * int64_t(w) + (k)] = t_;                                     \
    }                                                                               \
  } while (0)
#else
#define CHUNK_STAMP(k) \
  do {                 \
  } while (0)
#endif

template <int NV>
struct ChunkSmem {
  float v[2][kChunkTile];                                  // staged tiles (16-byte chunks swizzled);
                                                           // the current tile's S0 partials overwrite it
  float xs[NV == 3 ? 2 : 1][NV == 3 ? kChunkTile : 4];     // column values at the tile's nonzeros
  float s1h[NV - 1][kHeadCap];                             // tie groups' thread-local S1 (and S2) sums
  uint32_t cw[2][kCT], hw[2][kCT];                         // stratum-end and tie-group bits per thread
  uint32_t nzw[3][kCT];                                    // column-j bits per thread, by tile mod 3
  uint32_t ib[2][kES];                                     // column j's first entries of a staged tile
  double vb[NV == 3 ? 2 : 1][NV == 3 ? kES : 1];           // their values (valued fits)
  int32_t tlo[kChunkMaxTiles + 1], tg[kChunkMaxTiles + 1]; // the chunk's tile positions and first groups
  int32_t ctj[kChunkMaxTiles + 1], ctp[kChunkMaxTiles + 1];// column j's / the pending column's first entries
  uint16_t hpos[kHeadCap];                                 // the tile's tie-group positions
  Acc bs[4][kCT];                                          // S0 suffix of a thread's blocks right of block b
  Acc E[NV][kCT];                                          // each thread's carry from the chunk's later positions
  uint8_t Eo[kCT], zf[kCT];                                // that carry runs to the chunk's end / the thread's
                                                           // column positions: 0 none, 1 some, 2 all (binary x)
  Acc wa[NV][kCW];                                         // warp sums from the warp's first position
  int32_t wf[kCW];                                         // warp holds a stratum end
  Acc cc[2][NV];                                           // the chunk carry into the current tile
  int32_t ccf[2];                                          // that carry stopped at a stratum end
  int32_t hopen, last, next;
  int32_t fsc[2][kCW];                                     // cached-S0 path: stratum ends / tie groups per warp
  uint64_t mbar[2];                                        // tile copy completion, per buffer
  double red[3][kCW];
  double scratch[3 * 32];
  double cr[NV];
};

// position e of a staged tile -> its float slot (16-byte chunks XOR-swizzled within 128-byte rows,
// so a thread's eight 16-byte reads of its own 128 bytes hit distinct banks)
__device__ __forceinline__ int swz(int e) {
  const int c = e >> 2;
  return ((c ^ ((c >> 3) & 7)) << 2) | (e & 3);
}

// a double with a 4-bit tag in its lowest mantissa bits (a relative change below 2^-48)
__device__ __forceinline__ uint64_t tag_word(double v, uint32_t tg) {
  return (static_cast<uint64_t>(__double_as_longlong(v)) & ~uint64_t(15)) | uint64_t(tg);
}
__device__ __forceinline__ double word_value(uint64_t w) {
  return __longlong_as_double(static_cast<long long>(w & ~uint64_t(15)));
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---- tile copies: one bulk tensor copy (TMA) per tile, completion counted on an mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// rows [y, y + 128) of the 32-float-wide view of v into dst (1024-byte aligned), 128-byte swizzle
__device__ __forceinline__ void tma_load_rows(void *dst, const void *map, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(0), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// generic-proxy accesses before async-proxy (TMA) accesses of the same memory
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
// a tile copy that has not landed within this many SM clocks (about 2 s) is an error
constexpr long long kTmaWait = 1ll << 32;

// One tie group's terms of eqs. (parallel_g)/(parallel_h) (and d log S0 when the log-likelihood
// is due) from its risk-set sums sh = (S0, S1[, S2]).
template <int NV>
__device__ __forceinline__ void add_group(const Acc (&sh)[NV], int dgi, int j, bool need_ll, Acc &g1q, Acc &g2q,
                                          double &llq, const DevFit &F, int gidx, bool cache) {
  const float S0 = sh[0].s + sh[0].c, S1 = sh[1].s + sh[1].c;
  const float fd = float(dgi);
  if (j >= 0) {
    const float inv = __frcp_rn(S0);
    const float r = __fdiv_rn(S1, S0);
    P::add(g1q, fd * r);
    if constexpr (NV == 3) P::add(g2q, fd * ((sh[2].s + sh[2].c) * inv - r * r));
    else P::add(g2q, fd * (r * (1.0f - r)));
  }
  if (need_ll) llq += double(dgi) * log(P::to64(sh[0]));
  if (F.out_S0) {
    F.out_S0[gidx] = P::to64(sh[0]);
    F.out_S1[gidx] = P::to64(sh[1]);
  }
  // the group's risk-set sum, kept for the fit's next launch (read when eta has not changed)
  if (cache) reinterpret_cast<float2 *>(F.hscr)[3 * int64_t(gidx)] = make_float2(sh[0].s, sh[0].c);
}

// Warp 0: publish the chunk's aggregate (its sums from its first position up to its first stratum
// end, final when a stratum ends in the chunk: AF) and, when need_lb, look back over the fit's later
// chunks for the carry into the chunk's last stratum (epoch-tagged words: aggregate 0..2,
// inclusive 3..5 per chunk). The carry goes to cr_out; a chunk without a stratum end then publishes
// aggregate + carry as its inclusive value. A wait past `spin` clocks raises COX_E_TIMEOUT.
template <int NV>
__device__ void chunk_lookback(uint64_t *cwd, int c, int nc, const double (&agg)[NV], int AF, bool need_lb,
                               uint32_t etag, long long spin, FitCtl *ctl, LaunchCtl *lc, double *cr_out) {
  const int lane = threadIdx.x & 31;
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) st_relaxed_u64(&cwd[6 * c + (AF ? 3 : 0) + i], tag_word(agg[i], etag));
  double cr[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) cr[i] = 0.0;
  if (need_lb) {
    int base = c + 1;
    const long long t0 = clock64();
    bool timed_out = false;
    for (;;) {
      const int u = base + lane;
      double val[NV];
      int vi = 0, va = 0;
      for (;;) {
        vi = 0;
        va = 0;
        if (u < nc) {
          uint64_t wv[NV];
          bool ok = true;
#pragma unroll
          for (int i = 0; i < NV; ++i) {
            wv[i] = ld_relaxed_u64(&cwd[6 * u + 3 + i]);
            ok = ok && (wv[i] & 15u) == etag;
          }
          if (!ok) {
            ok = true;
#pragma unroll
            for (int i = 0; i < NV; ++i) {
              wv[i] = ld_relaxed_u64(&cwd[6 * u + i]);
              ok = ok && (wv[i] & 15u) == etag;
            }
            va = ok;
          } else {
            vi = 1;
          }
#pragma unroll
          for (int i = 0; i < NV; ++i) val[i] = word_value(wv[i]);
        } else {   // past the fit's last chunk
          vi = 1;
#pragma unroll
          for (int i = 0; i < NV; ++i) val[i] = 0.0;
        }
        const uint32_t inv = __ballot_sync(0xffffffffu, !(vi || va));
        const uint32_t inc = __ballot_sync(0xffffffffu, vi);
        if (inv == 0u || (inc != 0u && __ffs(inc) < __ffs(inv))) break;
        if (clock64() - t0 > spin) {
          timed_out = true;
          break;
        }
        __nanosleep(32);
      }
      if (timed_out) {
        if (lane == 0) {
          atomicExch(&ctl->error, COX_E_TIMEOUT);
          atomicExch(&lc->error, COX_E_TIMEOUT);
        }
        break;
      }
      const uint32_t inc = __ballot_sync(0xffffffffu, vi);
      const int stop = inc ? __ffs(inc) - 1 : 31;
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        double xv = lane <= stop ? val[i] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) xv += __shfl_down_sync(0xffffffffu, xv, off);
        cr[i] += __shfl_sync(0xffffffffu, xv, 0);
      }
      if (inc) break;
      base += 32;
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) cr_out[i] = cr[i];
    if (!AF && (need_lb || c + 1 == nc))
#pragma unroll
      for (int i = 0; i < NV; ++i) st_relaxed_u64(&cwd[6 * c + 3 + i], tag_word(agg[i] + cr[i], etag));
  }
}

// ---- the cached-S0 path: a launch of a fit whose eta is unchanged since its previous launch (no
// pending update) reads every tie group's S0 from that launch (kept beside the group's scratch) and
// computes column j's S1 (S2) from its entries alone: per chunk O(entries + tie groups) instead of
// a pass over every position. Its arrays lie over the tile buffers (and, valued, the value buffers).
template <int NV>
struct FastView {
  uint32_t epos[kChunkFastE];         // column j's entries in the chunk: position from the chunk's first
  uint16_t erk[kChunkFastE];          // their stratum rank in the chunk (stratum ends before them)
  int32_t cut[kChunkFastCuts];        // the chunk's stratum ends (positions from its first)
  uint16_t hcode[kChunkFastH];        // per tie group: its first entry at or after its position
                                      // (bits 0-11), that entry lies in its stratum (bit 12), its
                                      // stratum continues past the chunk (bit 13)
  Acc es[NV - 1][kChunkFastE];        // x v (x^2 v) per entry, then their segmented suffix sums
};
static_assert(kChunkFastE <= 4096, "entry index in 12 bits");
static_assert(sizeof(FastView<2>) <= sizeof(float) * 2 * kChunkTile, "cached-S0 arrays fit the tile buffers");
static_assert(sizeof(FastView<3>) <= sizeof(float) * 4 * kChunkTile, "cached-S0 arrays fit the tile and value buffers");

// The chunk's partial (G1, G2[, sum d log S0]) on the cached-S0 path, into g1q, g2q, llq. The
// caller staged the chunk's last tile before it knew the path: its copy lands before the buffers
// are reused. Limits (strata, tie groups, entries) are admitted by the host plan and the previous
// launch; a chunk past them raises COX_E_INVALID and adds nothing.
template <int NV>
__device__ void fast_chunk(ChunkSmem<NV> &S, const DevFit &F, FitCtl *ctl, LaunchCtl *lc, int c, int nc, int nt, int tb,
                           int j, int64_t cbj, bool vf, bool need_ll, uint32_t etag, long long spin, uint32_t &ph,
                           bool &tma_late, Acc &g1q, Acc &g2q, double &llq) {
  constexpr bool VAL = NV == 3;
  constexpr int NS = NV - 1;
  FastView<NV> &V = *reinterpret_cast<FastView<NV> *>(&S.v[0][0]);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int P0 = S.tlo[0], span = S.tlo[nt] - P0;
  const int W0 = P0 >> 5, nw = (span + 31) >> 5;     // the chunk's bitmap words (P0 is a multiple of 32)
  const int wpt = (nw + kCT - 1) / kCT;                // a run of consecutive words per thread
  const int wa = min(nw, tid * wpt), wb = min(nw, wa + wpt);
  const int64_t q0 = cbj + S.ctj[0];
  const int ne = S.ctj[nt] - S.ctj[0];
  auto wmask = [&](int w) {
    const int r = span - 32 * w;
    return r >= 32 ? 0xffffffffu : ((1u << r) - 1u);
  };
  // 1. stratum ends and tie groups per thread; their bases over the CTA
  int ncut = 0, nhd = 0;
#pragma unroll 4
  for (int w = wa; w < wb; ++w) {
    const uint32_t m = wmask(w);
    ncut += __popc(F.cut_bits[W0 + w] & m);
    nhd += __popc(F.head_bits[W0 + w] & m);
  }
  int ic = ncut, ih = nhd;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, ic, off), z = __shfl_up_sync(0xffffffffu, ih, off);
    if (lane >= off) {
      ic += y;
      ih += z;
    }
  }
  if (lane == 31) {
    S.fsc[0][warp] = ic;
    S.fsc[1][warp] = ih;
  }
  // the staged tile's copy lands before its buffer is reused
  {
    const int b = (tb - 1) & 1;
    const long long t0 = clock64();
    while (!mbar_try_wait(&S.mbar[b], (ph >> b) & 1u))
      if (clock64() - t0 > kTmaWait) {
        tma_late = true;
        break;
      }
    ph ^= 1u << b;
  }
  cp_async_wait_all();
  __syncthreads();
  int cb = ic - ncut, hb = ih - nhd, nC = 0, nH = 0;
#pragma unroll
  for (int q = 0; q < kCW; ++q) {
    if (q < warp) {
      cb += S.fsc[0][q];
      hb += S.fsc[1][q];
    }
    nC += S.fsc[0][q];
    nH += S.fsc[1][q];
  }
  if (nC > kChunkFastCuts || nH > kChunkFastH || ne > kChunkFastE || ne < 0 || tma_late) {   // uniform
    if (tid == 0) atomicCAS(&ctl->error, 0, tma_late ? COX_E_TIMEOUT : COX_E_INVALID);
    if (warp == 0) {   // final zeros, so that no chunk of the fit waits for this one
      const double z[NV] = {};
      chunk_lookback<NV>(reinterpret_cast<uint64_t *>(F.tval), c, nc, z, 1, false, etag, spin, ctl, lc, S.cr);
    }
    return;
  }
  // 2. the stratum ends in order; column j's entries: positions, x v (x^2 v)
  {
    int k = cb;
    for (int w = wa; w < wb; ++w)
      for (uint32_t m = F.cut_bits[W0 + w] & wmask(w); m; m &= m - 1u) V.cut[k++] = 32 * w + __ffs(m) - 1;
  }
  // kFB entries per thread at a time: their positions, then v at them (and x), loaded together
  constexpr int kFB = 4;
  const float *vg = static_cast<const float *>(F.v);
  for (int k0 = tid; k0 < ne; k0 += kFB * kCT) {
    int pos[kFB];
    float vv[kFB], x[kFB];
#pragma unroll
    for (int u = 0; u < kFB; ++u) {
      const int k = k0 + u * kCT;
      pos[u] = k < ne ? int(F.idx[q0 + k] & kPosMask) - P0 : 0;
      x[u] = vf && k < ne ? float(F.val[q0 + k]) : 1.0f;
    }
#pragma unroll
    for (int u = 0; u < kFB; ++u) vv[u] = k0 + u * kCT < ne ? vg[P0 + pos[u]] : 0.f;
#pragma unroll
    for (int u = 0; u < kFB; ++u) {
      const int k = k0 + u * kCT;
      if (k < ne) {
        V.epos[k] = uint32_t(pos[u]);
        V.es[0][k] = Acc{x[u] * vv[u], 0.f};
        if constexpr (VAL) V.es[1][k] = Acc{x[u] * (x[u] * vv[u]), 0.f};
      }
    }
  }
  __syncthreads();
  for (int k = tid; k < ne; k += kCT) {   // stratum ends before each entry
    const int pos = int(V.epos[k]);
    int lo = 0, hi = nC;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (V.cut[mid] < pos) lo = mid + 1;
      else hi = mid;
    }
    V.erk[k] = uint16_t(lo);
  }
  __syncthreads();
  // 3. segmented suffix sums over the entries (a stratum end between two entries ends a segment),
  //    compensated: thread-local runs over consecutive entries, a warp scan of the runs, the warps
  const int me = (ne + kCT - 1) / kCT;
  const int ka = min(ne, tid * me), kb = min(ne, ka + me);
  auto seg_end = [&](int k) { return k == ne - 1 || V.erk[k] != V.erk[k + 1]; };
  int brk = 0;
  {
    Acc run[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) run[i] = P::zero();
    for (int k = kb - 1; k >= ka; --k) {
      if (seg_end(k)) {
        brk = 1;
#pragma unroll
        for (int i = 0; i < NS; ++i) run[i] = V.es[i][k];
      } else {
#pragma unroll
        for (int i = 0; i < NS; ++i) run[i] = P::comb(V.es[i][k], run[i]);
      }
#pragma unroll
      for (int i = 0; i < NS; ++i) V.es[i][k] = run[i];
    }
  }
  Acc I[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) I[i] = ka < kb ? V.es[i][ka] : P::zero();
  int If = brk;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    Acc y[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) y[i] = P::shfl_down(I[i], off);
    const int yf = __shfl_down_sync(0xffffffffu, If, off);
    if (lane + off < 32) {
      if (!If) {
#pragma unroll
        for (int i = 0; i < NS; ++i) I[i] = P::comb(I[i], y[i]);
      }
      If |= yf;
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NS; ++i) S.wa[i][warp] = I[i];
    S.wf[warp] = If;
  }
  __syncthreads();
  {
    Acc Cw[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) Cw[i] = P::zero();
    for (int q = kCW - 1; q > warp; --q) {
      if (S.wf[q]) {
#pragma unroll
        for (int i = 0; i < NS; ++i) Cw[i] = S.wa[i][q];
      } else {
#pragma unroll
        for (int i = 0; i < NS; ++i) Cw[i] = P::comb(S.wa[i][q], Cw[i]);
      }
    }
    Acc E[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) E[i] = P::shfl_down(I[i], 1);
    const int Ef = __shfl_down_sync(0xffffffffu, If, 1);
    if (lane == 31) {
#pragma unroll
      for (int i = 0; i < NS; ++i) E[i] = Cw[i];
    } else if (!Ef) {
#pragma unroll
      for (int i = 0; i < NS; ++i) E[i] = P::comb(E[i], Cw[i]);
    }
    for (int k = kb - 1; k >= ka && !seg_end(k); --k)   // the entries after the thread's last segment end
#pragma unroll
      for (int i = 0; i < NS; ++i) V.es[i][k] = P::comb(V.es[i][k], E[i]);
  }
  __syncthreads();
  // 4. warp 0 publishes the chunk's sums up to its first stratum end and looks back for the carry
  //    into its last stratum (S0 is not carried: every chunk of the fit reads its groups' S0);
  //    meanwhile every thread codes its tie groups
  if (warp == 0) {
    double agg[NV];
    agg[0] = 0.0;
#pragma unroll
    for (int i = 0; i < NS; ++i) agg[i + 1] = (ne > 0 && V.erk[0] == 0) ? P::to64(V.es[i][0]) : 0.0;
    chunk_lookback<NV>(reinterpret_cast<uint64_t *>(F.tval), c, nc, agg, nC > 0, c + 1 < nc, etag, spin, ctl, lc, S.cr);
  }
  {
    int r = cb, o = hb;
    int k = 0;
    {
      int hi = ne;
      const int p0 = 32 * wa;
      while (k < hi) {
        const int mid = (k + hi) >> 1;
        if (int(V.epos[mid]) < p0) k = mid + 1;
        else hi = mid;
      }
    }
#pragma unroll 2
    for (int w = wa; w < wb; ++w) {
      const uint32_t msk = wmask(w);
      const uint32_t hm = F.head_bits[W0 + w] & msk, cm = F.cut_bits[W0 + w] & msk;
      for (uint32_t m = hm | cm; m; m &= m - 1u) {
        const int bit = __ffs(m) - 1, pos = 32 * w + bit;
        if ((hm >> bit) & 1u) {
          while (k < ne && int(V.epos[k]) < pos) ++k;
          const uint32_t in = (k < ne && int(V.erk[k]) == r) ? 1u : 0u;
          V.hcode[o++] = uint16_t((k < ne ? k : 0) | (in << 12) | (uint32_t(r == nC) << 13));
        }
        if ((cm >> bit) & 1u) ++r;
      }
    }
  }
  __syncthreads();
  // 5. the tie groups' terms (consecutive threads take consecutive groups)
  Acc CR[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) CR[i] = P::from64(S.cr[i + 1]);
  const float2 *s0c = reinterpret_cast<const float2 *>(F.hscr);
  const int g0 = S.tg[0];
  for (int h0 = tid; h0 < nH; h0 += kFB * kCT) {   // kFB groups per thread: their loads together
    float2 z[kFB];
    int dg[kFB];
#pragma unroll
    for (int u = 0; u < kFB; ++u) {
      const int h = h0 + u * kCT;
      z[u] = h < nH ? s0c[3 * int64_t(g0 + h)] : make_float2(1.f, 0.f);
      dg[u] = h < nH ? F.head_d[g0 + h] : 0;
    }
#pragma unroll
    for (int u = 0; u < kFB; ++u) {
      const int h = h0 + u * kCT;
      if (h >= nH) break;
      const int code = V.hcode[h];
      Acc sh[NV];
      sh[0] = Acc{z[u].x, z[u].y};
#pragma unroll
      for (int i = 0; i < NS; ++i) sh[i + 1] = (code & (1 << 12)) ? V.es[i][code & 4095] : P::zero();
      if (code & (1 << 13))
#pragma unroll
        for (int i = 0; i < NS; ++i) sh[i + 1] = P::comb(sh[i + 1], CR[i]);
      add_group<NV>(sh, dg[u], j, need_ll, g1q, g2q, llq, F, g0 + h, false);
    }
  }
  fence_proxy_async_smem();   // the tile buffers are rewritten by the next chunk's copies
}

template <int NV, bool kCond>
__global__ void __launch_bounds__(kCT, COXGB_CHUNK_MIN_CTAS) chunk_kernel(const DevFit *__restrict__ fits, const ChunkItem *__restrict__ items,
                                                    LaunchCtl *lc, int mode, int j_eval, unsigned long long cond,
                                                    long long spin) {
  constexpr bool VAL = NV == 3;
  extern __shared__ __align__(16) unsigned char smraw[];
  // the tile buffers start on a 1024-byte boundary (the period of the copies' 128-byte swizzle)
  ChunkSmem<NV> &S = *reinterpret_cast<ChunkSmem<NV> *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&S.mbar[0], 1);
    mbar_init(&S.mbar[1], 1);
    mbar_init_fence();
  }
  uint32_t ph = 0;   // bit b: the phase of buffer b's barrier that the next wait expects
  bool tma_late = false;
  const int n_items = lc->n_items;
  ChunkItem it = blockIdx.x < n_items ? items[blockIdx.x] : ChunkItem{};   // issued before the check below
  // nothing to do once every fit stopped, or after a launch of this work list gave up a wait
  const int active = __syncthreads_or(
      tid == 0 && *reinterpret_cast<volatile int32_t *>(&lc->error) == 0 &&
      (mode != kModeFit || *reinterpret_cast<volatile int32_t *>(&lc->active) > 0));

  // a CTA's first item is its index; later ones are taken in work-list order from the launch's
  // ticket (a look-back waits only for items earlier in the list, all held by running CTAs)
  auto next_item = [&]() {
    if (n_items <= int(gridDim.x)) return n_items;
    if (tid == 0) S.next = int(gridDim.x) + int(atomicAdd(&lc->ticket, 1u));
    __syncthreads();
    return S.next;
  };
  for (int w = blockIdx.x; active && w < n_items; w = next_item()) {
    CHUNK_STAMP(0);
    if (w != int(blockIdx.x)) it = items[w];
    const DevFit &F = fits[it.f];
    FitCtl *ctl = F.ctl;
    const int c = it.c, ta = it.ta, tb = it.tb, nc = it.nc, nt = tb - ta;
    const float *vg = static_cast<const float *>(F.v);   // the patch below reads v directly
    int j = -1;            // the launch's column (set once the fit's control block is read)
    int64_t cbj = 0;       // its first entry
    bool vf = false;       // valued fit (binary fits in a valued launch use x = 1)
    // tile t's values (one tensor copy), bits and, once the tables are in (cols), the first kES of
    // column j's entries in the tile (each thread copies, and later scatters, its own), asynchronously
    auto stage = [&](int t, int lo, bool cols) {
      const int b = t & 1;
      if (tid == 0) {
        mbar_expect_tx(&S.mbar[b], uint32_t(kChunkTile * sizeof(float)));
        tma_load_rows(&S.v[b][0], F.vmap, lo >> 5, &S.mbar[b]);
      }
      cp_async4(&S.cw[b][tid], F.cut_bits + (lo >> 5) + tid);
      cp_async4(&S.hw[b][tid], F.head_bits + (lo >> 5) + tid);
      if (cols && j >= 0) {
        const int tq = t - ta;
        const int64_t q0 = cbj + S.ctj[tq], q1 = cbj + S.ctj[tq + 1];
#pragma unroll
        for (int u = 0; u < kES / kCT; ++u) {
          const int64_t q = q0 + tid + u * kCT;
          if (q < q1) {
            cp_async4(&S.ib[b][tid + u * kCT], F.idx + q);
            if constexpr (VAL) {
              if (vf) cp_async8(&S.vb[b][tid + u * kCT], F.val + q);
            }
          }
        }
      }
      cp_async_commit();
    };
    if (__syncthreads_or(tid == 0 && mode == kModeFit && ctl->state != kRunning)) continue;
    stage(tb - 1, it.lo_last, false);   // the chunk's last tile, before its tables arrive
    const int T_ = F.T;
    j = (mode == kModeEval || mode == kModeShard) ? j_eval : (mode == kModeFit ? ctl->j : -1);
    const bool need_ll = mode == kModeLL || ((mode == kModeFit || mode == kModeShard) && ctl->need_ll);
    const int pend_j = mode == kModeFit ? ctl->pend_j : -1;
    const double pend_db = ctl->pend_db;
    const uint32_t epoch = ctl->epoch;
    const uint32_t etag = epoch % 15u + 1u;   // never 0: zeroed words are never current
    // fit launches and evaluation launches (cox_gradient: columns in order at one eta) keep and
    // read the tie groups' S0
    const bool keeps_s0 = mode == kModeFit || mode == kModeEval;
    const uint32_t s0tag = keeps_s0 ? ctl->s0c_tag : 0u;
    const double shift = F.shift;
    vf = VAL && F.val != nullptr;
    cbj = j >= 0 ? F.col_ptr[j] : 0;
    // the next column's entries in this chunk: whether the next launch's cached-S0 path admits it
    int ent_next = 0;
    if (keeps_s0 && tid == 0 && j >= 0) {
      const int32_t *ctn = F.col_tile + int64_t(j + 1 < F.p ? j + 1 : 0) * (T_ + 1);
      ent_next = ctn[tb] - ctn[ta];
    }

    // ---- the chunk's tables
    for (int q = tid; q <= nt; q += kCT) {
      S.tlo[q] = F.tile_lo[ta + q];
      S.tg[q] = F.tile_g[ta + q];
      S.ctj[q] = j >= 0 ? F.col_tile[int64_t(j) * (T_ + 1) + ta + q] : 0;
      S.ctp[q] = pend_j >= 0 ? F.col_tile[int64_t(pend_j) * (T_ + 1) + ta + q] : 0;
    }
    for (int q = tid; q < 3 * kCT; q += kCT) S.nzw[q / kCT][q % kCT] = 0u;
    if (tid == 0) {
      for (int i = 0; i < NV; ++i) S.cc[0][i] = P::zero();
      S.ccf[0] = 0;
      S.hopen = INT_MAX;
    }
    __syncthreads();

    // eta unchanged since the fit's previous launch (no pending update), which admitted the cached-S0
    // path for this one: every chunk of the fit reads its tie groups' S0 from that launch
    const bool fastfit = keeps_s0 && pend_j < 0 && s0tag == epoch && it.fast_ok != 0;
    Acc g1q = P::zero(), g2q = P::zero();
    double llq = 0.0;
    if (fastfit) {
      fast_chunk<NV>(S, F, ctl, lc, c, nc, nt, tb, j, cbj, vf, need_ll, etag, spin, ph, tma_late, g1q, g2q, llq);
    } else {

    // column j's entries of tile t -> per-thread bits (and values): the thread's entries that
    // stage() copied (staged), then any beyond them from global memory
    auto scatter = [&](int t, bool staged) {
      if (j < 0) return;
      const int tq = t - ta, lo = S.tlo[tq], b = t & 1;
      const int64_t q1 = cbj + S.ctj[tq + 1];
      int64_t q = cbj + S.ctj[tq] + tid;
      if (staged) {
#pragma unroll
        for (int u = 0; u < kES / kCT; ++u, q += kCT) {
          if (q < q1) {
            const int e = int(S.ib[b][tid + u * kCT] & kPosMask) - lo;
            atomicOr(&S.nzw[t % 3][e >> 5], 1u << (e & 31));
            if constexpr (VAL) {
              if (vf) S.xs[b][e] = float(S.vb[b][tid + u * kCT]);
            }
          }
        }
      }
      for (; q < q1; q += kCT) {
        const int e = int(F.idx[q] & kPosMask) - lo;
        atomicOr(&S.nzw[t % 3][e >> 5], 1u << (e & 31));
        if constexpr (VAL) {
          if (vf) S.xs[b][e] = float(F.val[q]);
        }
      }
    };

    // ---- the pending update at the chunk's entries of column pend_j (global eta and v); the new
    //      values at the last tile's positions (staged before the update) are kept for its patch
    constexpr int kKeep = 4;
    int np = 0, keep_pos[kKeep];
    float keep_v[kKeep];
    bool overflow = false;
    if (pend_j >= 0) {
      const int64_t cb = F.col_ptr[pend_j];
      const int lo_l = S.tlo[nt - 1], hi_l = S.tlo[nt];
      const int64_t qa = cb + S.ctp[0], qb = cb + S.ctp[nt];
      // kPU of the thread's entries at a time: their positions, then their eta, are loaded together
      // (a chunk of many tiles holds several entries per thread; one at a time, each would cost two
      // dependent round trips to memory)
      constexpr int kPU = 4;
      for (int64_t q0 = qa + tid; q0 < qb; q0 += kPU * kCT) {
        uint32_t e[kPU];
        double x[kPU], eo[kPU];
#pragma unroll
        for (int u = 0; u < kPU; ++u) {
          const int64_t q = q0 + int64_t(u) * kCT;
          e[u] = q < qb ? F.idx[q] : 0u;
          x[u] = F.val && q < qb ? F.val[q] : 1.0;
        }
#pragma unroll
        for (int u = 0; u < kPU; ++u) eo[u] = q0 + int64_t(u) * kCT < qb ? F.eta[e[u] & kPosMask] : 0.0;
#pragma unroll
        for (int u = 0; u < kPU; ++u) {
          if (q0 + int64_t(u) * kCT >= qb) break;
          const int64_t pos = e[u] & kPosMask;
          const double et = __dadd_rn(eo[u], __dmul_rn(x[u], pend_db));
          F.eta[pos] = et;
          const float nv = make_v<P>(et, shift, (e[u] & kExitBit) != 0, &ctl->error);
          static_cast<float *>(F.v)[pos] = nv;
          if (pos >= lo_l && pos < hi_l) {
            if (np < kKeep) {
#pragma unroll
              for (int k = 0; k < kKeep; ++k)
                if (k == np) { keep_pos[k] = int(pos - lo_l); keep_v[k] = nv; }
              ++np;
            } else {
              overflow = true;
            }
          }
        }
      }
      // the chunk's earlier tiles are read by tensor copies (the async proxy, through L2): the new
      // values must be there, and ordered before those copies, by the barrier that precedes them
      __threadfence();
      fence_proxy_async_global();
    }
    scatter(tb - 1, false);
    CHUNK_STAMP(1);

    int slot = 0;
    for (int t = tb - 1; t >= ta; --t) {
      const int b = t & 1, tq = t - ta;
      const int lo = S.tlo[tq], hi = S.tlo[tq + 1], ga = S.tg[tq], gb = S.tg[tq + 1];
      {   // tile t's copy landed (bounded wait), its bits too
        const long long t0 = clock64();
        while (!mbar_try_wait(&S.mbar[b], (ph >> b) & 1u))
          if (clock64() - t0 > kTmaWait) {
            tma_late = true;
            break;
          }
        ph ^= 1u << b;
      }
      cp_async_wait_all();
      __syncthreads();   // tile t staged, its bits scattered; tile t+1 finished
      if (t == tb - 1) CHUNK_STAMP(2);
      if (t == tb - 1 && pend_j >= 0) {
        // the tile was staged before the pending update: put in the updated values (from registers;
        // from global memory where a thread had more of them than it kept)
        if (__syncthreads_or(overflow)) {
          const int64_t cb = F.col_ptr[pend_j];
          for (int64_t q = cb + S.ctp[tq] + tid; q < cb + S.ctp[tq + 1]; q += kCT) {
            const int64_t pos = F.idx[q] & kPosMask;
            S.v[b][swz(int(pos - lo))] = vg[pos];
          }
        } else {
#pragma unroll
          for (int u = 0; u < kKeep; ++u)
            if (u < np) S.v[b][swz(keep_pos[u])] = keep_v[u];
        }
        __syncthreads();
      }
      if (t - 1 >= ta) stage(t - 1, S.tlo[tq - 1], true);
      S.nzw[(t + 1) % 3][tid] = 0u;   // tile t+1's bits are no longer read
      const int nh = gb - ga;
      int dpre[kPF];
#pragma unroll
      for (int u = 0; u < kPF; ++u) dpre[u] = tid + u * kCT < nh ? F.head_d[ga + tid + u * kCT] : 0;

      const bool act = tid * kCI < hi - lo;   // positions past the tile's end belong to the next tile
      const uint32_t cm = act ? S.cw[b][tid] : 0u, hm = act ? S.hw[b][tid] : 0u;
      const uint32_t zm = S.nzw[t % 3][tid];
      // this thread's first tie group within the tile: earlier lanes, then earlier warps
      const int hc = __popc(hm);
      int hinc = hc;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, hinc, off);
        if (lane >= off) hinc += y;
      }
      int wpre = 0;
      for (int q = lane; q < warp * 32; q += 32) wpre += q * kCI < hi - lo ? __popc(S.hw[b][q]) : 0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) wpre += __shfl_xor_sync(0xffffffffu, wpre, off);
      const int hbase = wpre + hinc - hc;

      // ---- S1 (S2) over the thread's nonzeros, right to left (reads v before it is overwritten).
      //      A thread whose every position is a nonzero of a binary column takes S0's sums instead
      //      (the same additions in the same order), so that a column that is nonzero everywhere
      //      gives S1 bitwise equal to S0 (ratios of exactly 1, the paper's degenerate column).
      const bool full = !vf && zm == 0xffffffffu;
      float a1 = 0.f, a2 = 0.f;
      if (zm && !full) {
        float r1 = 0.f, r2 = 0.f;
        int rank = hc;
        for (uint32_t m = zm | hm | cm; m;) {
          const int k = 31 - __clz(m);
          m &= ~(1u << k);
          if ((cm >> k) & 1u) { r1 = 0.f; r2 = 0.f; }   // k ends its stratum: later positions are another
          if ((zm >> k) & 1u) {
            const float vv = S.v[b][swz(tid * kCI + k)];
            if constexpr (VAL) {
              const float x = vf ? S.xs[t & 1][tid * kCI + k] : 1.0f;
              const float xv = x * vv;
              r1 += xv;
              r2 += x * xv;
            } else {
              r1 += vv;
            }
          }
          if ((hm >> k) & 1u) {
            --rank;
            S.s1h[0][hbase + rank] = r1;
            if constexpr (VAL) S.s1h[1][hbase + rank] = r2;
          }
        }
        a1 = r1;
        a2 = r2;
      }
      S.zf[tid] = uint8_t(full ? 2 : (zm != 0u ? 1 : 0));

      // ---- S0: plain sums within blocks of 8, compensated above; partials replace v in place
      float x[kCI];
#pragma unroll
      for (int q = 0; q < kCI / 4; ++q) {
        const int ch = tid * (kCI / 4) + q;
        const float4 f = *reinterpret_cast<const float4 *>(&S.v[b][(ch ^ ((ch >> 3) & 7)) * 4]);
        x[4 * q] = f.x;
        x[4 * q + 1] = f.y;
        x[4 * q + 2] = f.z;
        x[4 * q + 3] = f.w;
      }
      if (__any_sync(0xffffffffu, !act)) {   // the warp holding the tile's end (the staged window runs on)
        if (!act) {
#pragma unroll
          for (int i = 0; i < kCI; ++i) x[i] = 0.f;
        }
      }
      Acc run = P::zero();
      int rf = 0;
      const bool nocut = __all_sync(0xffffffffu, cm == 0u);
#pragma unroll
      for (int bl = 3; bl >= 0; --bl) {
        S.bs[bl][tid] = run;
        float p = 0.f, pr[8];
        if (nocut) {
#pragma unroll
          for (int i = 7; i >= 0; --i) {
            p += x[8 * bl + i];
            pr[i] = p;
          }
        } else {
#pragma unroll
          for (int i = 7; i >= 0; --i) {
            if ((cm >> (8 * bl + i)) & 1u) p = 0.f;
            p += x[8 * bl + i];
            pr[i] = p;
          }
        }
#pragma unroll
        for (int hq = 0; hq < 2; ++hq) {
          const int ch = tid * (kCI / 4) + 2 * bl + hq;
          *reinterpret_cast<float4 *>(&S.v[b][(ch ^ ((ch >> 3) & 7)) * 4]) =
              make_float4(pr[4 * hq], pr[4 * hq + 1], pr[4 * hq + 2], pr[4 * hq + 3]);
        }
        const bool bc = ((cm >> (8 * bl)) & 0xffu) != 0u;
        run = bc ? Acc{p, 0.f} : P::comb(Acc{p, 0.f}, run);
        rf |= int(bc);
      }

      // ---- warp segmented suffix scan of the thread sums (from each thread's first position)
      Acc I[NV];
      I[0] = run;
      I[1] = full ? run : Acc{a1, 0.f};
      if constexpr (VAL) I[2] = full ? run : Acc{a2, 0.f};
      int If = rf;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        Acc y[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) y[i] = P::shfl_down(I[i], off);
        const int yf = __shfl_down_sync(0xffffffffu, If, off);
        if (lane + off < 32) {
          if (!If) {
#pragma unroll
            for (int i = 0; i < NV; ++i) I[i] = P::comb(I[i], y[i]);
          }
          If |= yf;
        }
      }
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) S.wa[i][warp] = I[i];
        S.wf[warp] = If;
      }
      {   // the tile's tie-group positions, in order
        int hq = hbase;
        for (uint32_t m = hm; m; m &= m - 1u) S.hpos[hq++] = uint16_t(tid * kCI + __ffs(m) - 1);
      }
      __syncthreads();

      // ---- each thread's carry from the chunk's later positions (known part) and the tile total
      Acc CC[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) CC[i] = S.cc[slot][i];
      const int CCf = S.ccf[slot];
      Acc Cw[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) Cw[i] = CC[i];
      int Cwo = !CCf;
      for (int q = kCW - 1; q > warp; --q) {
        if (S.wf[q]) {
#pragma unroll
          for (int i = 0; i < NV; ++i) Cw[i] = S.wa[i][q];
          Cwo = 0;
        } else {
#pragma unroll
          for (int i = 0; i < NV; ++i) Cw[i] = P::comb(S.wa[i][q], Cw[i]);
        }
      }
      Acc E[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) E[i] = P::shfl_down(I[i], 1);
      const int Ef = __shfl_down_sync(0xffffffffu, If, 1);
      int Eo;
      if (lane == 31) {
#pragma unroll
        for (int i = 0; i < NV; ++i) E[i] = Cw[i];
        Eo = Cwo;
      } else if (Ef) {
        Eo = 0;
      } else {
#pragma unroll
        for (int i = 0; i < NV; ++i) E[i] = P::comb(E[i], Cw[i]);
        Eo = Cwo;
      }
#pragma unroll
      for (int i = 0; i < NV; ++i) S.E[i][tid] = E[i];
      S.Eo[tid] = uint8_t(Eo);
      if (tid == 0) {
        Acc TI[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) TI[i] = P::zero();
        int TF = 0;
        for (int q = kCW - 1; q >= 0; --q) {
          if (S.wf[q]) {
#pragma unroll
            for (int i = 0; i < NV; ++i) TI[i] = S.wa[i][q];
            TF = 1;
          } else {
#pragma unroll
            for (int i = 0; i < NV; ++i) TI[i] = P::comb(S.wa[i][q], TI[i]);
          }
        }
#pragma unroll
        for (int i = 0; i < NV; ++i) S.cc[slot ^ 1][i] = TF ? TI[i] : P::comb(TI[i], CC[i]);
        S.ccf[slot ^ 1] = TF | CCf;
      }
      __syncthreads();

      // ---- the tile's tie groups (head-parallel)
      int myopen = INT_MAX;
      for (int u = 0, h = tid; h < nh; ++u, h += kCT) {
        const int pos = S.hpos[h], o = pos >> 5, k = pos & 31, bl = k >> 3;
        const uint32_t m = S.cw[b][o];
        const uint32_t toend = 0xffffffffu << k;
        const uint32_t upto = bl == 3 ? toend : (toend & ((1u << (8 * bl + 8)) - 1u));
        Acc sh[NV];
        sh[0] = Acc{S.v[b][swz(pos)], 0.f};
        if ((m & upto) == 0u) sh[0] = P::comb(sh[0], S.bs[bl][o]);
        const int z = S.zf[o];
        sh[1] = z == 2 ? sh[0] : Acc{z ? S.s1h[0][h] : 0.f, 0.f};
        if constexpr (VAL) sh[2] = z == 2 ? sh[0] : Acc{z ? S.s1h[1][h] : 0.f, 0.f};
        int open = 0;
        if ((m & toend) == 0u) {   // the risk set runs past the thread's positions
#pragma unroll
          for (int i = 0; i < NV; ++i) sh[i] = P::comb(sh[i], S.E[i][o]);
          open = S.Eo[o];
        }
        const int gidx = ga + h;
        const int dgi = u == 0 ? dpre[0] : (u == 1 ? dpre[1] : F.head_d[gidx]);
        if (open) {   // wait for the chunk's carry
          float2 *hs = reinterpret_cast<float2 *>(F.hscr) + 3 * int64_t(gidx);
#pragma unroll
          for (int i = 0; i < NV; ++i) hs[i] = make_float2(sh[i].s, sh[i].c);
          myopen = min(myopen, gidx);
        } else {
          add_group<NV>(sh, dgi, j, need_ll, g1q, g2q, llq, F, gidx, keeps_s0);
        }
      }
      if (myopen != INT_MAX) atomicMin(&S.hopen, myopen);
      // tile t-1's column bits (its entries were copied with the tile, a tile's work ago), ordered
      // before their reads by the barrier at the top of the next iteration
      if (t - 1 >= ta) {
        cp_async_wait_all();
        scatter(t - 1, true);
      }
      fence_proxy_async_smem();   // this tile's buffer is rewritten by a later copy
      slot ^= 1;
    }
    __syncthreads();

    CHUNK_STAMP(3);
    // ---- publish the chunk's sums; look back for its carry
    const int hopen = S.hopen;
    const int gac = S.tg[0], gbc = S.tg[nt];
    const int q0 = min(max(hopen, gac), gbc);   // deferred groups: [q0, gbc) (hopen is INT_MAX when none)
    // while warp 0 looks back, the other warps copy the deferred groups' sums and event counts
    // into the (now idle) tile buffers, when they fit there
    const int ndef = gbc - q0;
    constexpr int kDefCap = int(sizeof(S.v) / (NV * sizeof(float2) + sizeof(int32_t)));
    float2 *dsum = reinterpret_cast<float2 *>(&S.v[0][0]);                  // [NV][kDefCap]
    int32_t *dcnt = reinterpret_cast<int32_t *>(dsum + NV * kDefCap);      // [kDefCap]
    const bool on_chip = ndef <= kDefCap;
    if (on_chip && warp > 0) {
      const float2 *hs = reinterpret_cast<const float2 *>(F.hscr) + 3 * int64_t(q0);
#pragma unroll 4
      for (int q = tid - 32; q < ndef; q += kCT - 32) {
#pragma unroll
        for (int i = 0; i < NV; ++i) dsum[i * kDefCap + q] = hs[3 * q + i];
        dcnt[q] = F.head_d[q0 + q];
      }
    }
    uint64_t *cwd = reinterpret_cast<uint64_t *>(F.tval);   // per chunk: aggregate words 0..2, inclusive 3..5
    if (warp == 0) {
      double agg[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) agg[i] = P::to64(S.cc[slot][i]);
      const int AF = S.ccf[slot];   // a stratum ends in the chunk: its sums from the first position are final
      chunk_lookback<NV>(cwd, c, nc, agg, AF, c + 1 < nc && (hopen < gbc || !AF), etag, spin, ctl, lc, S.cr);
    }
    __syncthreads();

    CHUNK_STAMP(4);
    // ---- the deferred tie groups: a contiguous run of the chunk's last groups
    {
      Acc CR[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) CR[i] = P::from64(S.cr[i]);
      const float2 *hs = reinterpret_cast<const float2 *>(F.hscr) + 3 * int64_t(q0);
      for (int q = tid; q < ndef; q += kCT) {
        Acc sh[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
          const float2 f2 = on_chip ? dsum[i * kDefCap + q] : hs[3 * q + i];
          sh[i] = P::comb(Acc{f2.x, f2.y}, CR[i]);
        }
        add_group<NV>(sh, on_chip ? dcnt[q] : F.head_d[q0 + q], j, need_ll, g1q, g2q, llq, F, q0 + q,
                      keeps_s0);
      }
      fence_proxy_async_smem();   // the tile buffers are rewritten by the next chunk's copies
    }
    }   // the full path

    // ---- the chunk's partial, then the step by the CTA that finishes the fit's last chunk
    double r[3] = {P::to64(g1q), P::to64(g2q), llq};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) r[i] += __shfl_down_sync(0xffffffffu, r[i], off);
    if (lane == 0)
#pragma unroll
      for (int i = 0; i < 3; ++i) S.red[i][warp] = r[i];
    __syncthreads();
    if (tid == 0) {
      if (keeps_s0) {   // a chunk the next launch's cached-S0 path would not hold rules it out
        const int span = S.tlo[nt] - S.tlo[0];
        if (!it.fast_ok || ent_next > kChunkFastE || (F.val == nullptr && ent_next >= span))
          atomicOr(&ctl->fast_no, 1u);
      }
      double p0 = 0.0, p1 = 0.0, p2 = 0.0;
      for (int q = 0; q < kCW; ++q) { p0 += S.red[0][q]; p1 += S.red[1][q]; p2 += S.red[2][q]; }
      F.part[3 * c + 0] = p0;
      F.part[3 * c + 1] = p1;
      F.part[3 * c + 2] = p2;
      // release: the partials before the count; acquire for the CTA that finds itself last
      uint32_t prev;
      asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(&ctl->done_tiles) : "memory");
      S.last = prev == uint32_t(nc - 1);
    }
    __syncthreads();
    CHUNK_STAMP(5);
    if (S.last) {
      if (keeps_s0 && tid == 0) {   // every tie group's S0 now holds for the fit's eta
        ctl->s0c_tag = ctl->fast_no == 0u ? epoch + 1u : 0u;
        ctl->fast_no = 0u;
      }
      finish_launch_step<kCT, false>(F, lc, mode, j, need_ll, nc, epoch, S.scratch);
    }
    __syncthreads();
    CHUNK_STAMP(6);
  }
  cp_async_wait_all();
  if (tma_late) {   // a copy that missed its bound: flag it, then give it one more bound before exit
    if (tid == 0) {
      atomicExch(&lc->error, COX_E_TIMEOUT);
      for (int b = 0; b < 2; ++b) {
        const long long t0 = clock64();
        while (!mbar_try_wait(&S.mbar[b], (ph >> b) & 1u) && clock64() - t0 < kTmaWait) {
        }
      }
    }
    __syncthreads();
  }
  // the last CTA of the launch resets the ticket (when items were taken from it) and, in a graph's
  // sweep loop, ends the loop when nothing is left
  if (kCond || n_items > int(gridDim.x)) {
    if (tid == 0) {
      __threadfence();
      if (atomicAdd(&lc->exited, 1u) == gridDim.x - 1) {
        lc->exited = 0u;
        lc->ticket = 0u;
        if constexpr (kCond) {
          if (mode == kModeFit && cond) {
            const long long left = --lc->budget;
            if (*reinterpret_cast<volatile int32_t *>(&lc->active) <= 0 || left <= 0 ||
                *reinterpret_cast<volatile int32_t *>(&lc->error) != 0)
              cudaGraphSetConditional(cond, 0u);
          }
        }
      }
    }
  }
}

template <int NV, bool kCond>
int occupancy_one() {
  const int sm = int(sizeof(ChunkSmem<NV>)) + 1024;
  if (cudaFuncSetAttribute(chunk_kernel<NV, kCond>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess)
    return -1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chunk_kernel<NV, kCond>, kCT, sm) != cudaSuccess) return -1;
  return per_sm > 0 ? per_sm : 1;
}

// Resident CTAs of a variant on the current device (both graph variants share the smaller figure).
template <int NV>
int max_grid_nv() {
  static int cached[64] = {0};
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  if (cached[dev]) return cached[dev];
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  const int a = occupancy_one<NV, false>(), b = occupancy_one<NV, true>();
  if (a < 0 || b < 0) return -1;
  cached[dev] = (a < b ? a : b) * nsm;
  return cached[dev];
}

template <int NV>
int launch_nv(const DevFit *fits, const ChunkItem *items, LaunchCtl *lc, int grid, int mode, int j_eval, cudaStream_t s,
              unsigned long long cond) {
  if (max_grid_nv<NV>() < 0) return COX_E_CUDA;
  const long long spin = wait_limit();
  const size_t sm = sizeof(ChunkSmem<NV>) + 1024;
  if (cond) chunk_kernel<NV, true><<<grid, kCT, sm, s>>>(fits, items, lc, mode, j_eval, cond, spin);
  else chunk_kernel<NV, false><<<grid, kCT, sm, s>>>(fits, items, lc, mode, j_eval, 0ull, spin);
  return COX_OK;
}

}  // namespace

int chunk_max_grid(int valued) { return valued ? max_grid_nv<3>() : max_grid_nv<2>(); }

int chunk_encode_vmap(void *v, int64_t n_floats, void *out) {
  // the driver's encoder, fetched through the runtime (no link-time dependency on libcuda)
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  if (!enc || !v || n_floats < 32 * 128 || (reinterpret_cast<uintptr_t>(v) & 15u)) return COX_E_CUDA;
  const cuuint64_t dims[2] = {32, cuuint64_t(n_floats / 32)};
  const cuuint64_t strides[1] = {32 * sizeof(float)};
  const cuuint32_t box[2] = {32, kChunkTile / 32};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(static_cast<CUtensorMap *>(out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, v, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? COX_OK : COX_E_CUDA;
}

int launch_chunk(const DevFit *fits, const ChunkItem *items, LaunchCtl *lc, int grid, int mode, int j_eval, int valued,
                 void *stream, unsigned long long cond) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
#if COX_TRACE_ON
  // COXGB_CHUNK_TRACE=<k>: stamp the phases of the k-th launch made outside a graph capture and
  // print, per phase, the mean and largest time over the launch's work items
  static long long seen = 0;
  static const long long want = std::getenv("COXGB_CHUNK_TRACE") ? std::atoll(std::getenv("COXGB_CHUNK_TRACE")) : -1;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  uint64_t *tr = nullptr;
  const int kMaxItems = 1 << 16;
  if (cs == cudaStreamCaptureStatusNone && want >= 0 && seen++ == want) {
    cudaMalloc(&tr, size_t(kMaxItems) * 8 * sizeof(uint64_t));
    cudaMemset(tr, 0, size_t(kMaxItems) * 8 * sizeof(uint64_t));
    cudaMemcpyToSymbol(g_chunk_trace, &tr, sizeof(tr));
  }
#endif
  const int rc = valued ? launch_nv<3>(fits, items, lc, grid, mode, j_eval, s, cond)
                        : launch_nv<2>(fits, items, lc, grid, mode, j_eval, s, cond);
#if COX_TRACE_ON
  if (tr) {
    cudaStreamSynchronize(s);
    std::vector<uint64_t> h(size_t(kMaxItems) * 8);
    cudaMemcpy(h.data(), tr, h.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost);
    uint64_t *null = nullptr;
    cudaMemcpyToSymbol(g_chunk_trace, &null, sizeof(null));
    cudaFree(tr);
    double sum[6] = {0}, mx[6] = {0};
    uint64_t t0 = ~0ull, t1 = 0;
    int n = 0;
    for (int i = 0; i < kMaxItems; ++i) {
      const uint64_t *r = &h[size_t(i) * 8];
      if (!r[0] || !r[6]) continue;
      ++n;
      t0 = std::min(t0, r[0]);
      t1 = std::max(t1, r[6]);
      for (int k = 0; k < 6; ++k) {
        const double d = double(r[k + 1] - r[k]);
        sum[k] += d;
        mx[k] = std::max(mx[k], d);
      }
    }
    static const char *names[6] = {"tables+update", "first tile wait", "tiles", "look-back", "deferred+partial",
                                   "final step"};
    std::fprintf(stderr, "[chunk trace] %d items, span %.2f us\n", n, n ? (t1 - t0) * 1e-3 : 0.0);
    for (int k = 0; k < 6; ++k)
      std::fprintf(stderr, "  %-18s mean %7.2f us  max %7.2f us\n", names[k], n ? sum[k] / n * 1e-3 : 0.0, mx[k] * 1e-3);
  }
#endif
  if (rc) return rc;
  return cudaPeekAtLastError() == cudaSuccess ? COX_OK : COX_E_CUDA;
}

}  // namespace coxgb
