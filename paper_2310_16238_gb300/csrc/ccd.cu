// Streaming coordinate-step kernel for cyclic coordinate descent on the stratified /
// time-varying Cox partial likelihood (arXiv 2310.16238, §2.4-§2.7).
//
// One launch advances every fit in its work list by one coordinate. A work item is one tile (a
// contiguous range of risk-sequence positions) of one fit; items are handed out by a ticket
// counter, and every tile of a fit comes after the tiles to its right (later positions), whose
// sums it needs. The CTAs are persistent and pipelined: while a CTA works on one item, the tile
// of exp(eta) of its next item streams into the other shared-memory stage (cp.async), and the
// ticket and work-item record of the item after that are fetched between the phases of the
// current one. Per item:
//   1. column j's entries in the tile, the tie-group read positions and the stratum ends are
//      marked in bitmasks; the previous coordinate's pending update is applied at the tile's
//      entries of that column (eta += x dbeta, eq. parallel_xb; v = +-exp(eta - shift),
//      eq. parallel_d), in global memory and in the staged tile;
//   2. pass 1: each thread sums its ITEMS consecutive positions right to left, restarting at
//      stratum ends (strata are the segments of the paper's flag-value operator, §2.6), for
//      D = v, N1 = x_j v and N2 = x_j^2 v;
//   3. a block-wide segmented suffix scan of the thread sums gives every thread the sum of the
//      positions to its right in the tile, and the tile's own sum (up to its first stratum end);
//   4. the tile sum is published and the tiles to the right are summed with a decoupled
//      look-back (FP64 carries);
//   5. pass 2: each thread walks its positions again from the carried-in sums and evaluates the
//      ratios of eqs. (parallel_g)/(parallel_h) at its tie groups (Breslow: the suffix sum at the
//      first row of the tie block, weighted by the group's event count);
//   6. the tile's partial (G1, G2[, sum d log S0]) is stored, and the last tile of a fit reduces
//      the partials in a fixed order and takes the coordinate step (§2.4: Newton eq. newton,
//      trust region, L1 directional derivatives).
// No N-length vector is written except at the nonzeros of the updated column.
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

#include "ccd_common.cuh"
#include "cox.h"
#include "cox_internal.h"

namespace coxgb {

// ------------------------------------------------------------------ shared memory plan
// NV = number of running sums: 2 for binary X (D and N1; N2 = N1), 3 for valued X.
// NST stages, each holding one work item: its tile of v, the bitmasks of its tie groups,
// stratum ends and column-j entries, the events of its tie groups, x at column j's entries
// (valued X) and a header with what the consumers need to know about the item.
constexpr int kStages = 2;
constexpr int kConsumers = kThreads;             // warps 0..7 scan; warp 8 + s produces stage s
constexpr int kBlock = kConsumers + 32 * kStages;

struct StageHdr {
  int32_t end;       // 1: no more items for this CTA; 2: this item's fit has stopped (skip it)
  int32_t f, t;      // fit and tile
  int32_t lo, len;   // first position and number of positions
  int32_t ga, nh;    // first tie group of the tile and their number
  int32_t j;         // column evaluated (-1: none)
  int32_t need_ll;   // the log-likelihood is due
  uint32_t epoch;    // the fit's launch counter
  int32_t pad[2];
};

template <class P, int NV>
struct Smem {
  using T = typename P::T;
  static constexpr int TILE = kThreads * P::ITEMS;
  static constexpr int WORDS = TILE / 32;
  static constexpr size_t al(size_t x) { return (x + 127) & ~size_t(127); }
  static constexpr size_t o_v = 0;                                        // the tile of v, swizzled chunks
  static constexpr size_t o_head = o_v + sizeof(T) * TILE;                // tie-group read positions
  static constexpr size_t o_cut = o_head + 4 * WORDS;                     // stratum ends
  static constexpr size_t o_nz = o_cut + 4 * WORDS;                       // column j's entries
  static constexpr size_t o_hd = o_nz + 4 * WORDS;                        // events per tie group
  static constexpr size_t o_hdr = o_hd + 4 * kHeadCap;                    // StageHdr
  static constexpr size_t o_x = al(o_hdr + sizeof(StageHdr));             // x at column j's entries (valued X)
  static constexpr size_t stage = al(NV == 3 ? o_x + sizeof(T) * TILE : o_x);
  static constexpr size_t o_bar = kStages * stage;                        // full[kStages], empty[kStages]
  static constexpr size_t bytes = o_bar + 16 * kStages;
};

// 16-byte chunk c of a tile lives at chunk c ^ ((c >> 3) & 7) of its stage: the eight chunks one
// consumer thread owns (c = 8 tid + k) land in eight different bank groups for the eight threads
// of a quarter warp, so the per-thread reads do not conflict.
__device__ __forceinline__ int swz(int c) { return c ^ ((c >> 3) & 7); }

// ------------------------------------------------------------------ mbarriers (CTA scope)
static __device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
static __device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
static __device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
static __device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
// Wait until the phase of the given parity has completed; false when `budget` clocks passed first.
static __device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long budget) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (clock64() - t0 > budget) return false;
    __nanosleep(20);
  }
  return true;
}
// Barrier of the consumer warps only (the producer warp runs ahead on its own).
static __device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory"); }

template <int NV>
static __device__ void consumer_sum(double (&v)[NV], double *scratch /* [NV*32] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
  consumers_sync();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) scratch[i * 32 + warp] = v[i];
  consumers_sync();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double x = lane < kConsumers / 32 ? scratch[i * 32 + lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      v[i] = x;   // valid in thread 0
    }
  }
  consumers_sync();
}

// ------------------------------------------------------------------ the kernel
// One producer warp (warp 8) takes tickets and prepares each item in a free stage: it reads the
// work item and the fit's control block, copies the tile of v (cp.async), marks the tile's tie
// groups, stratum ends and column-j entries in the stage's bitmasks, applies the previous
// coordinate's pending update (eta and v in global memory, and in the staged tile), and signals
// the stage full. The eight consumer warps take the stages in order: the two passes over the
// tile, the block scan, the look-back, the ratios, the tile partial and, in the last tile of a
// fit, the coordinate step. Only the look-back reads global memory on their path.
template <class P, int NV, bool kCond>
__global__ void __launch_bounds__(kBlock, NV == 3 ? 1 : 2)
    ccd_kernel(const DevFit *__restrict__ fits, const WorkItem *__restrict__ items, LaunchCtl *lc, int mode, int j_eval,
               unsigned long long cond, long long spin) {
  using T = typename P::T;
  using Acc = typename P::Acc;
  using S = Smem<P, NV>;
  constexpr bool VAL = NV == 3;
  constexpr int ITEMS = P::ITEMS;
  constexpr int PC = 16 / sizeof(T);          // elements per 16-byte chunk
  constexpr int TCH = ITEMS / PC;             // chunks per consumer thread (8)
  constexpr int NW = kConsumers / 32;
  static_assert(TCH == 8, "each consumer thread owns 128 bytes");
  static_assert(ITEMS <= 32, "a thread's positions fit one bitmask word");

  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + S::o_bar);
  uint64_t *empty = full + kStages;

  __shared__ int s_last;
  __shared__ Acc s_wagg[NV][NW];              // per warp: inclusive suffix from its first thread
  __shared__ int s_wflag[NW];
  __shared__ int s_whc[NW];                   // per warp: tie-group read positions it holds
  __shared__ double s_carry[NV];              // the tile's carry from the tiles to its right
  __shared__ double s_wred[3][NW];
  __shared__ double s_red[3 * 32];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n_items = lc->n_items;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
  }
  __syncthreads();

  if (warp >= NW) {
    // =========================================================== producer warps
    // Items are assigned statically: CTA c takes items c, c + G, c + 2G, ... (G CTAs), in that
    // order; producer warp s stages the CTA's items k = s, s + kStages, ... into stage s. Every
    // item needs only items before it in the list (the tiles to its right), so the earliest
    // unfinished item is always being worked on. A producer reads the record of its next item
    // and that fit's control block while it stages the current one.
    const int s = warp - NW;
    unsigned char *sb = smem + size_t(s) * S::stage;
    StageHdr *hdr = reinterpret_cast<StageHdr *>(sb + S::o_hdr);
    uint32_t *headbits = reinterpret_cast<uint32_t *>(sb + S::o_head);
    uint32_t *cutbits = reinterpret_cast<uint32_t *>(sb + S::o_cut);
    uint32_t *nzbits = reinterpret_cast<uint32_t *>(sb + S::o_nz);
    int32_t *hd = reinterpret_cast<int32_t *>(sb + S::o_hd);
    T *xs = reinterpret_cast<T *>(sb + S::o_x);
    T *sv = reinterpret_cast<T *>(sb + S::o_v);
    // nothing to do once every fit stopped, or after a launch of this work list gave up a wait
    const bool active = (mode != kModeFit || *reinterpret_cast<volatile int32_t *>(&lc->active) > 0) &&
                        *reinterpret_cast<volatile int32_t *>(&lc->error) == 0;
    const int64_t stride = int64_t(kStages) * gridDim.x;
    int64_t i = int64_t(blockIdx.x) + int64_t(s) * gridDim.x;
    // what a producer needs to know about an item's fit in this launch
    struct FitView {
      FitCtl *ctl;
      const DevData *D;
      T *v;
      double *eta;
      double shift, db;
      int32_t j, pj, need, run;
      uint32_t ep;
    };
    auto view = [&](int f) {
      const DevFit &F = fits[f];
      FitView fv;
      fv.ctl = F.ctl;
      fv.D = F.d;
      fv.v = static_cast<T *>(F.v);
      fv.eta = F.eta;
      fv.shift = F.shift;
      const FitCtl *c = F.ctl;
      fv.run = mode != kModeFit || c->state == kRunning;
      fv.j = mode == kModeEval ? j_eval : (mode == kModeFit ? c->j : -1);
      fv.pj = mode == kModeFit ? c->pend_j : -1;
      fv.db = c->pend_db;
      fv.need = mode == kModeLL || (mode == kModeFit && c->need_ll);
      fv.ep = c->epoch;
      return fv;
    };
    WorkItem it{};
    FitView fv{};
    if (active && i < n_items) {
      it = items[i];
      fv = view(it.f);
    }
    for (int u = 0;; ++u, i += stride) {
      // the stage is free once the consumers released its previous item
      if (u > 0 && !mbar_wait(&empty[s], uint32_t((u - 1) & 1), spin)) {
        if (lane == 0) atomicExch(&lc->error, COX_E_TIMEOUT);
        break;
      }
      if (!active || i >= n_items) {
        if (lane == 0) {
          hdr->end = 1;
          mbar_arrive(&full[s]);
        }
        break;
      }
      if (!fv.run) {   // a fit that stopped: its tiles are skipped (the stage still passes in order)
        if (lane == 0) {
          hdr->end = 2;
          mbar_arrive(&full[s]);
        }
        if (i + stride < n_items) {
          it = items[i + stride];
          fv = view(it.f);
        }
        continue;
      }
      const DevData *D = fv.D;
      const int t = it.t, lo = it.lo, len = it.hi - it.lo, ga = it.ga, nh = it.gb - it.ga;
      {   // asynchronous copies: the tile of v, its words of the tie-group and stratum-end bitmaps,
          // and its tie groups' event counts
        const unsigned char *g = reinterpret_cast<const unsigned char *>(fv.v + lo);
        const int nch = (len + PC - 1) / PC;
        for (int c = lane; c < nch; c += 32) cp_async16(sb + S::o_v + size_t(swz(c)) * 16, g + size_t(c) * 16);
        const int nw = (len + 31) >> 5;
        const uint32_t *hw = D->head_bits + (lo >> 5), *cw = D->cut_bits + (lo >> 5);
        for (int q = lane; q < nw; q += 32) {
          cp_async4(&headbits[q], hw + q);
          cp_async4(&cutbits[q], cw + q);
        }
        for (int h = lane; h < nh; h += 32) cp_async4(&hd[h], D->head_d + ga + h);
        cp_async_commit();
      }
      const int T_ = D->T;
      int64_t qa = 0, qb = 0, ua = 0, ub = 0;
      if (fv.j >= 0) {
        const int64_t cb = D->col_ptr[fv.j];
        const int32_t *ct = D->col_tile + int64_t(fv.j) * (T_ + 1);
        qa = cb + ct[t];
        qb = cb + ct[t + 1];
      }
      if (fv.pj >= 0) {
        const int64_t cb = D->col_ptr[fv.pj];
        const int32_t *ct = D->col_tile + int64_t(fv.pj) * (T_ + 1);
        ua = cb + ct[t];
        ub = cb + ct[t + 1];
      }
      const FitView cur = fv;
      const int cur_f = it.f;
      if (i + stride < n_items) {   // the next item's record and its fit's control block, early
        it = items[i + stride];
        fv = view(it.f);
      }
      for (int q = lane; q < S::WORDS; q += 32) nzbits[q] = 0u;
      __syncwarp();
      // column j's entries in the tile (eight loads in flight per lane)
      const bool vf = VAL && D->val != nullptr;
      for (int64_t base = qa; base < qb; base += 32 * 8) {
        uint32_t e[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int64_t q = base + lane + 32 * r;
          e[r] = q < qb ? D->idx[q] : 0u;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int64_t q = base + lane + 32 * r;
          if (q < qb) {
            const int pos = int(e[r] & kPosMask) - lo;
            atomicOr(&nzbits[pos >> 5], 1u << (pos & 31));
            if (vf) xs[pos] = T(D->val[q]);
          }
        }
      }
      cp_async_wait_all();   // this lane's copies; the warp barrier below makes all of them visible
      __syncwarp();
      // the previous coordinate's step at this tile's entries: eta and v in global memory and in
      // the staged tile (eight entries in flight per lane)
      for (int64_t base = ua; base < ub; base += 32 * 8) {
        uint32_t e[8];
        double et[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int64_t q = base + lane + 32 * r;
          e[r] = q < ub ? D->idx[q] : 0u;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int64_t q = base + lane + 32 * r;
          et[r] = q < ub ? cur.eta[e[r] & kPosMask] : 0.0;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int64_t q = base + lane + 32 * r;
          if (q < ub) {
            const int64_t pos = e[r] & kPosMask;
            const double x = D->val ? D->val[q] : 1.0;
            const double nt = __dadd_rn(et[r], __dmul_rn(x, cur.db));
            cur.eta[pos] = nt;
            const T nv = make_v<P>(nt, cur.shift, (e[r] & kExitBit) != 0, &cur.ctl->error);
            cur.v[pos] = nv;
            const int el = int(pos) - lo, c = el / PC;
            sv[swz(c) * PC + (el % PC)] = nv;
          }
        }
      }
      if (lane == 0) {
        hdr->end = 0;
        hdr->f = cur_f;
        hdr->t = t;
        hdr->lo = lo;
        hdr->len = len;
        hdr->ga = ga;
        hdr->nh = nh;
        hdr->j = cur.j;
        hdr->need_ll = cur.need;
        hdr->epoch = cur.ep;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[s]);
    }
  } else {
    // =========================================================== consumer warps
    // The last tile of a fit (the one whose count of finished tiles reaches T) takes the fit's
    // coordinate step. Thread 0 issues that count's atomic after an item and reads its result one
    // item later (or at the end), so its round trip stays off the per-item path.
    uint32_t pend_prev = 0u;          // thread 0: result of the previous item's count
    bool pend = false;                // thread 0: a count is outstanding
    StageHdr prev{};                  // the previous item (its fit's step may be due)
    auto fit_step = [&](const StageHdr &ph) {
      const DevFit &F = fits[ph.f];
      FitCtl *ctl = F.ctl;
      const DevData *D = F.d;
      const int T_ = D->T, j = ph.j;
      const bool need_ll = ph.need_ll != 0;
        __threadfence();
        double acc[3] = {0.0, 0.0, 0.0};
        for (int u = tid; u < T_; u += kConsumers) {
          acc[0] += ld_relaxed_f64(&F.part[3 * u + 0]);
          acc[1] += ld_relaxed_f64(&F.part[3 * u + 1]);
          acc[2] += ld_relaxed_f64(&F.part[3 * u + 2]);
        }
        consumer_sum<3>(acc, s_red);
        double extra[2] = {0.0, 0.0};   // beta'dX and the penalty, when the log-likelihood is due
        if (need_ll) {
          for (int jj = tid; jj < D->p; jj += kConsumers) {
            const double b = F.beta[jj];
            extra[0] += b * D->dX[jj];
            const bool pen = F.penalize ? F.penalize[jj] != 0 : true;
            if (pen && F.penalty == COX_PEN_L1) extra[1] += F.lambda * fabs(b);
            if (pen && F.penalty == COX_PEN_L2) extra[1] += b * b / (2.0 * F.l2_var);
          }
          consumer_sum<2>(extra, s_red);
        }
        if (tid == 0) {
          const double G1 = acc[0], G2 = acc[1], LL = acc[2];
          const double shift = F.shift;
          if (ctl->error != 0) {
            if (mode == kModeFit && ctl->state == kRunning) atomicSub(&lc->active, 1);
            ctl->state = kError;
          } else if (mode == kModeEval) {
            ctl->out_g1 = -D->dX[j] + G1;
            ctl->out_g2 = G2;
            if (F.gout) { F.gout[2 * j] = -D->dX[j] + G1; F.gout[2 * j + 1] = G2; }
          } else if (mode == kModeLL) {
            ctl->out_ll = extra[0] - LL - shift * D->sum_d;
          } else {
            bool stop = false;
            if (need_ll) {
              const double ll = extra[0] - LL - shift * D->sum_d;
              const double obj = -ll + extra[1];
              ctl->loglik = ll;
              ctl->obj = obj;
              if (ctl->sweep > 0 && fabs(obj - ctl->obj_prev) <= F.tol * fabs(obj)) {
                ctl->state = kConverged;
                stop = true;
              } else if (ctl->sweep >= F.max_sweeps) {
                ctl->state = kMaxed;
                stop = true;
              }
              if (stop) {
                atomicSub(&lc->active, 1);
                ctl->pend_j = -1;   // this launch's tiles already applied the pending update
              } else {
                ctl->obj_prev = obj;
              }
            }
            if (!stop) {
              const double g1 = -D->dX[j] + G1, g2 = G2;
              const int pen = F.penalize ? F.penalize[j] != 0 : 1;
              double tr = F.trust[j];
              const double s = ccd_step_rule(g1, g2, F.beta[j], &tr, F.penalty, F.lambda, F.l2_var, pen);
              F.trust[j] = tr;
              if (s != 0.0) {
                F.beta[j] = F.beta[j] + s;
                ctl->pend_j = j;
                ctl->pend_db = s;
              } else {
                ctl->pend_j = -1;
                ctl->pend_db = 0.0;
              }
              ctl->coord_updates += 1;
              int jn = j + 1;
              if (jn >= D->p) {
                jn = 0;
                ctl->sweep += 1;
                ctl->need_ll = 1;
              } else {
                ctl->need_ll = 0;
              }
              ctl->j = jn;
            }
          }
          ctl->done_tiles = 0u;
          ctl->epoch = ph.epoch + 1u;
        }
          };
    for (int k = 0;; ++k) {
      const int st = k % kStages;
      unsigned char *sb = smem + size_t(st) * S::stage;
      if (!mbar_wait(&full[st], uint32_t((k / kStages) & 1), spin)) {
        if (tid == 0) atomicExch(&lc->error, COX_E_TIMEOUT);
        break;
      }
      const StageHdr hdr = *reinterpret_cast<const StageHdr *>(sb + S::o_hdr);
      if (hdr.end == 1) break;
      if (hdr.end == 2) {   // a stopped fit's tile: release the stage
        consumers_sync();
        if (tid == 0) mbar_arrive(&empty[st]);
        continue;
      }
      const uint32_t *headbits = reinterpret_cast<const uint32_t *>(sb + S::o_head);
      const uint32_t *cutbits = reinterpret_cast<const uint32_t *>(sb + S::o_cut);
      const uint32_t *nzbits = reinterpret_cast<const uint32_t *>(sb + S::o_nz);
      const int32_t *hd = reinterpret_cast<const int32_t *>(sb + S::o_hd);
      const T *xs = reinterpret_cast<const T *>(sb + S::o_x);
      const T *sv = reinterpret_cast<const T *>(sb + S::o_v);
      const DevFit &F = fits[hdr.f];
      FitCtl *ctl = F.ctl;
      const DevData *D = F.d;
      const int t = hdr.t, T_ = D->T, len = hdr.len, j = hdr.j, ga = hdr.ga;
      const bool need_ll = hdr.need_ll != 0;
      const bool vf = VAL && D->val != nullptr;   // binary fits in a valued launch use x = 1

      // ---- pass 1: this thread's positions b0 .. b0 + ITEMS - 1, right to left
      const int b0 = tid * ITEMS;
      const uint32_t wmask = ITEMS == 32 ? 0xffffffffu : ((1u << ITEMS) - 1u);
      const int vlen = len - b0;   // positions of this thread inside the tile (may be <= 0)
      const uint32_t lmask = vlen >= ITEMS ? wmask : (vlen <= 0 ? 0u : ((1u << vlen) - 1u));
      // (words past the tile's length were not copied: only bits of its own positions are read)
      const uint32_t hm = lmask ? (headbits[b0 >> 5] >> (b0 & 31)) & lmask : 0u;
      const uint32_t cm = lmask ? (cutbits[b0 >> 5] >> (b0 & 31)) & lmask : 0u;
      const uint32_t zm = lmask ? (nzbits[b0 >> 5] >> (b0 & 31)) & lmask : 0u;
      const bool warp_nz = __any_sync(0xffffffffu, zm != 0u);
      auto load_vals = [&](T (&vals)[ITEMS]) {
#pragma unroll
        for (int kc = 0; kc < TCH; ++kc) {
          const float4 q = *reinterpret_cast<const float4 *>(sv + swz(tid * TCH + kc) * PC);
          const T *qq = reinterpret_cast<const T *>(&q);
#pragma unroll
          for (int u = 0; u < PC; ++u) vals[kc * PC + u] = ((lmask >> (kc * PC + u)) & 1u) ? qq[u] : T(0);
        }
      };
      Acc a[NV];
      {
        T vals[ITEMS];
        load_vals(vals);
#pragma unroll
        for (int i = 0; i < NV; ++i) a[i] = P::zero();
#pragma unroll
        for (int kk = ITEMS - 1; kk >= 0; --kk) {
          if ((cm >> kk) & 1u) {
#pragma unroll
            for (int i = 0; i < NV; ++i) a[i] = P::zero();
          }
          P::add(a[0], vals[kk]);
          if (warp_nz && ((zm >> kk) & 1u)) {
            if constexpr (VAL) {
              const T x = vf ? xs[b0 + kk] : T(1);
              const T wv = T(x * vals[kk]);
              P::add(a[1], wv);
              P::add(a[2], T(x * wv));
            } else {
              P::add(a[1], vals[kk]);
            }
          }
        }
      }
      // ---- block-wide segmented suffix scan of the thread sums; head counts left to right
      int xf = cm != 0u;
      Acc x[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) x[i] = a[i];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        Acc y[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) y[i] = P::shfl_down(x[i], off);
        const int yf = __shfl_down_sync(0xffffffffu, xf, off);
        if (lane + off < 32) {
          if (!xf) comb_n<Acc, P, NV>(x, y);
          xf |= yf;
        }
      }
      Acc ex[NV];   // this thread's carry within its warp: lane + 1's inclusive value
#pragma unroll
      for (int i = 0; i < NV; ++i) ex[i] = P::shfl_down(x[i], 1);
      int exf = __shfl_down_sync(0xffffffffu, xf, 1);
      if (lane == 31) {
#pragma unroll
        for (int i = 0; i < NV; ++i) ex[i] = P::zero();
        exf = 0;
      }
      const int hcnt = __popc(hm);
      int hinc = hcnt;   // inclusive prefix of head counts within the warp
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, hinc, off);
        if (lane >= off) hinc += y;
      }
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) s_wagg[i][warp] = x[i];
        s_wflag[warp] = xf;
      }
      if (lane == 31) s_whc[warp] = hinc;
      consumers_sync();
      Acc wc[NV];   // carry from the warps to the right
      int wcf = 0;
#pragma unroll
      for (int i = 0; i < NV; ++i) wc[i] = P::zero();
      int hb = hinc - hcnt;   // this thread's first tie group in the tile
      for (int w2 = NW - 1; w2 > warp; --w2) {   // wc = warp w2 (+) wc, right to left
        Acc r[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) r[i] = s_wagg[i][w2];
        if (!s_wflag[w2]) comb_n<Acc, P, NV>(r, wc);
#pragma unroll
        for (int i = 0; i < NV; ++i) wc[i] = r[i];
        wcf |= s_wflag[w2];
      }
      for (int w2 = 0; w2 < warp; ++w2) hb += s_whc[w2];
      if (!exf) comb_n<Acc, P, NV>(ex, wc);
      exf |= wcf;

      // ---- publish the tile sum and look back over the tiles to the right (FP64 carries)
      if (warp == 0) {
        Acc tot[NV];   // thread 0's inclusive value with the warps to its right: the tile's sum
#pragma unroll
        for (int i = 0; i < NV; ++i) tot[i] = x[i];
        if (!xf) comb_n<Acc, P, NV>(tot, wc);
        const int tf = __shfl_sync(0xffffffffu, xf | wcf, 0);
        double agg[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) agg[i] = __shfl_sync(0xffffffffu, P::to64(tot[i]), 0);
        const uint32_t ep = (hdr.epoch & 0x1fffffffu) << 3;
        if (lane == 0) {   // slots 0..2: aggregate, 3..5: inclusive (a tile holding a stratum end is complete)
          const int o = tf ? 3 : 0;
#pragma unroll
          for (int i = 0; i < NV; ++i) F.tval[6 * t + o + i] = agg[i];
          __threadfence();
          st_release_u32(&F.tstat[t], ep | (tf ? 4u | 2u : 1u));
        }
        double cr[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) cr[i] = 0.0;
        const bool last_is_cut = len > 0 && ((cutbits[(len - 1) >> 5] >> ((len - 1) & 31)) & 1u) != 0u;
        if (t + 1 < T_ && !last_is_cut) {
          int base = t + 1;
          const long long tstart = clock64();
          bool timed_out = false;
          for (;;) {
            const int u = base + lane;
            uint32_t stw = 0;
            bool valid = false;
            for (;;) {
              if (u < T_) {
                stw = ld_acquire_u32(&F.tstat[u]);
                valid = (stw & ~7u) == ep && (stw & 3u) != 0u;
              } else {
                valid = true;
                stw = ep | 2u;
              }
              const uint32_t inv = __ballot_sync(0xffffffffu, !valid);
              const uint32_t inc = __ballot_sync(0xffffffffu, valid && (stw & 3u) == 2u);
              if (inv == 0u || (inc != 0u && (__ffs(inc) < __ffs(inv)))) break;
              if (clock64() - tstart > spin) { timed_out = true; break; }
              __nanosleep(32);
            }
            if (timed_out) {
              if (lane == 0) atomicExch(&ctl->error, COX_E_TIMEOUT);
              break;
            }
            const uint32_t inc = __ballot_sync(0xffffffffu, valid && (stw & 3u) == 2u);
            const int stop = inc ? __ffs(inc) - 1 : 31;
            double v[NV];
#pragma unroll
            for (int i = 0; i < NV; ++i) v[i] = 0.0;
            if (lane <= stop && u < T_) {
              const int o = (stw & 3u) == 2u ? 3 : 0;
#pragma unroll
              for (int i = 0; i < NV; ++i) v[i] = ld_relaxed_f64(&F.tval[6 * u + o + i]);
            }
#pragma unroll
            for (int i = 0; i < NV; ++i) {
#pragma unroll
              for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
              cr[i] += __shfl_sync(0xffffffffu, v[i], 0);
            }
            if (inc) break;
            base += 32;
          }
        }
          if (lane == 0) {
          // the previous item's count of finished tiles (its round trip overlapped this item)
          s_last = pend && pend_prev == uint32_t(fits[prev.f].d->T - 1);
          pend = false;
#pragma unroll
          for (int i = 0; i < NV; ++i) s_carry[i] = cr[i];
          if (!tf) {
#pragma unroll
            for (int i = 0; i < NV; ++i) F.tval[6 * t + 3 + i] = agg[i] + cr[i];
            __threadfence();
            st_release_u32(&F.tstat[t], ep | 2u);
          }
        }
      }
      consumers_sync();
      if (s_last) {   // the previous item was its fit's last tile in this launch: the step
        fit_step(prev);
        if (tid == 0) s_last = 0;
        consumers_sync();
      }

      // ---- pass 2: running sums from the carried-in values; ratios at the tie groups
      double r_g1 = 0.0, r_g2 = 0.0, r_ll = 0.0;
      {
        Acc run[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) run[i] = ex[i];
        if (!exf) {
#pragma unroll
          for (int i = 0; i < NV; ++i) run[i] = P::comb(run[i], P::from64(s_carry[i]));
        }
        Acc q_g1 = P::zero(), q_g2 = P::zero();
        if (__any_sync(0xffffffffu, hm != 0u)) {
          T vals[ITEMS];
          load_vals(vals);
#pragma unroll
          for (int kk = ITEMS - 1; kk >= 0; --kk) {
            if ((cm >> kk) & 1u) {
#pragma unroll
              for (int i = 0; i < NV; ++i) run[i] = P::zero();
            }
            P::add(run[0], vals[kk]);
            if (warp_nz && ((zm >> kk) & 1u)) {
              if constexpr (VAL) {
                const T xx = vf ? xs[b0 + kk] : T(1);
                const T wv = T(xx * vals[kk]);
                P::add(run[1], wv);
                P::add(run[2], T(xx * wv));
              } else {
                P::add(run[1], vals[kk]);
              }
            }
            if ((hm >> kk) & 1u) {
              const int h = hb + __popc(hm & ((1u << kk) - 1u));
              const int dgi = hd[h];
              if constexpr (sizeof(T) == 8) {
                const double S0 = P::to64(run[0]), S1 = P::to64(run[1]);
                const double dg = double(dgi);
                if (j >= 0) {
                  const double inv = 1.0 / S0;
                  const double r = S1 * inv;
                  P::add(q_g1, dg * r);
                  if constexpr (VAL) P::add(q_g2, dg * (P::to64(run[2]) * inv - r * r));
                  else P::add(q_g2, dg * (r * (1.0 - r)));
                }
                if (need_ll) r_ll += dg * log(S0);
                if (F.out_S0) { F.out_S0[ga + h] = S0; F.out_S1[ga + h] = S1; }
              } else {
                const float S0 = run[0].s + run[0].c, S1 = run[1].s + run[1].c;
                const float fd = float(dgi);
                if (j >= 0) {
                  const float inv = __frcp_rn(S0);
                  const float r = __fdiv_rn(S1, S0);
                  P::add(q_g1, fd * r);
                  if constexpr (VAL) P::add(q_g2, fd * ((run[2].s + run[2].c) * inv - r * r));
                  else P::add(q_g2, fd * (r * (1.0f - r)));
                }
                if (need_ll) r_ll += double(dgi) * log(P::to64(run[0]));
                if (F.out_S0) { F.out_S0[ga + h] = P::to64(run[0]); F.out_S1[ga + h] = P::to64(run[1]); }
              }
            }
          }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {   // warp sums (compensated for FP32)
          q_g1 = P::comb(q_g1, P::shfl_down(q_g1, off));
          q_g2 = P::comb(q_g2, P::shfl_down(q_g2, off));
        }
        r_g1 = P::to64(q_g1);
        r_g2 = P::to64(q_g2);
        if (need_ll) {
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) r_ll += __shfl_down_sync(0xffffffffu, r_ll, off);
        }
      }
      if (lane == 0) { s_wred[0][warp] = r_g1; s_wred[1][warp] = r_g2; s_wred[2][warp] = r_ll; }
      consumers_sync();
      // the stage's contents are consumed: the producer may refill it
      if (tid == 0) {
        mbar_arrive(&empty[st]);
        double p0 = 0.0, p1 = 0.0, p2 = 0.0;
        for (int ww = 0; ww < NW; ++ww) { p0 += s_wred[0][ww]; p1 += s_wred[1][ww]; p2 += s_wred[2][ww]; }
        F.part[3 * t + 0] = p0; F.part[3 * t + 1] = p1; F.part[3 * t + 2] = p2;
        __threadfence();
        pend_prev = atomicAdd(&ctl->done_tiles, 1u);   // read one item later
        pend = true;
      }
      prev = hdr;
    }
    // the last item's count
    if (tid == 0) {
      s_last = pend && pend_prev == uint32_t(fits[prev.f].d->T - 1);
      pend = false;
    }
    consumers_sync();
    if (s_last) fit_step(prev);
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&lc->exited, 1u) == gridDim.x - 1) {   // the last CTA of this launch
      lc->ticket = 0u;
      lc->exited = 0u;
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

// Apply one column step to eta and v over all of the column's nonzeros (warm starts and
// coefficient vectors given to cox_loglik / cox_gradient), in column order.
template <class P>
__global__ void column_update_kernel(const DevFit *__restrict__ fit, int32_t j, double db, int64_t nnz_j) {
  const DevFit &F = *fit;
  const DevData *D = F.d;
  const int64_t cb = D->col_ptr[j];
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < nnz_j; k += int64_t(gridDim.x) * blockDim.x) {
    const int64_t q = cb + k;
    const uint32_t e = D->idx[q];
    const int64_t pos = e & kPosMask;
    const double x = D->val ? D->val[q] : 1.0;
    const double et = __dadd_rn(F.eta[pos], __dmul_rn(x, db));
    F.eta[pos] = et;
    static_cast<typename P::T *>(F.v)[pos] = make_v<P>(et, F.shift, (e & kExitBit) != 0, &F.ctl->error);
  }
}

// eta = 0 and v = +-exp(-shift) at every position (exits negative); padding stays 0.
template <class P>
__global__ void fill_v_kernel(const DevFit *__restrict__ fit, int64_t M, const uint32_t *__restrict__ exit_bits) {
  const DevFit &F = *fit;
  for (int64_t pos = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; pos < M; pos += int64_t(gridDim.x) * blockDim.x) {
    const bool ex = exit_bits ? ((exit_bits[pos >> 5] >> (pos & 31)) & 1u) != 0u : false;
    F.eta[pos] = 0.0;
    static_cast<typename P::T *>(F.v)[pos] = make_v<P>(0.0, F.shift, ex, &F.ctl->error);
  }
}

// ------------------------------------------------------------------ launchers
template <class P, int NV, bool kCond>
static int max_grid_one() {
  const size_t sm = Smem<P, NV>::bytes;
  if (cudaFuncSetAttribute(ccd_kernel<P, NV, kCond>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)) !=
      cudaSuccess)
    return -1;
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ccd_kernel<P, NV, kCond>, kBlock, sm) != cudaSuccess)
    return -1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return (per_sm > 0 ? per_sm : 1) * nsm;
}

// Resident CTAs of a variant (occupancy x SMs); both graph variants share the smaller figure.
template <class P, int NV>
static int max_grid_impl() {
  static int cached = 0;
  if (cached) return cached;
  const int a = max_grid_one<P, NV, false>(), b = max_grid_one<P, NV, true>();
  if (a < 0 || b < 0) return -1;
  cached = a < b ? a : b;
  return cached;
}

int ccd_max_grid(int precision, int valued) {
  if (precision == COX_FP32C) return valued ? max_grid_impl<PF32C, 3>() : max_grid_impl<PF32C, 2>();
  return valued ? max_grid_impl<PF64, 3>() : max_grid_impl<PF64, 2>();
}

int ccd_tile(int precision) { return precision == COX_FP32C ? kThreads * PF32C::ITEMS : kThreads * PF64::ITEMS; }

template <class P, int NV>
static int launch_impl(const DevFit *fits, const WorkItem *items, LaunchCtl *lc, int grid, int mode, int j_eval,
                       cudaStream_t s, unsigned long long cond) {
  if (max_grid_impl<P, NV>() < 0) return COX_E_CUDA;
  // the variant that can end a conditional graph loop only where there is one to end: kernels that
  // set conditional handles cannot be captured by profilers as single kernels
  const long long spin = wait_limit();
  if (cond)
    ccd_kernel<P, NV, true><<<grid, kBlock, Smem<P, NV>::bytes, s>>>(fits, items, lc, mode, j_eval, cond, spin);
  else
    ccd_kernel<P, NV, false><<<grid, kBlock, Smem<P, NV>::bytes, s>>>(fits, items, lc, mode, j_eval, 0ull, spin);
  return COX_OK;
}

int launch_ccd(int precision, const DevFit *fits, const WorkItem *items, LaunchCtl *lc, int grid, int mode, int j_eval,
               int valued, void *stream, unsigned long long cond) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs == cudaStreamCaptureStatusNone) count_launches(1);   // graph nodes are counted per replay
  int rc;
  if (precision == COX_FP32C)
    rc = valued ? launch_impl<PF32C, 3>(fits, items, lc, grid, mode, j_eval, s, cond)
                : launch_impl<PF32C, 2>(fits, items, lc, grid, mode, j_eval, s, cond);
  else
    rc = valued ? launch_impl<PF64, 3>(fits, items, lc, grid, mode, j_eval, s, cond)
                : launch_impl<PF64, 2>(fits, items, lc, grid, mode, j_eval, s, cond);
  if (rc) return rc;
  return cudaPeekAtLastError() == cudaSuccess ? COX_OK : COX_E_CUDA;
}

int launch_column_update(int precision, const DevFit *fit_dev, int32_t j, double db, int64_t nnz_j, void *stream) {
  if (nnz_j <= 0) return COX_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  count_launches(1);
  int blocks = int((nnz_j + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (precision == COX_FP32C) column_update_kernel<PF32C><<<blocks, 256, 0, s>>>(fit_dev, j, db, nnz_j);
  else column_update_kernel<PF64><<<blocks, 256, 0, s>>>(fit_dev, j, db, nnz_j);
  return cudaPeekAtLastError() == cudaSuccess ? COX_OK : COX_E_CUDA;
}

int launch_fill_v(int precision, const DevFit *fit_dev, int64_t M, const uint32_t *exit_bits, void *stream) {
  if (M <= 0) return COX_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  count_launches(1);
  int blocks = int((M + 255) / 256);
  if (blocks > 8192) blocks = 8192;
  if (precision == COX_FP32C) fill_v_kernel<PF32C><<<blocks, 256, 0, s>>>(fit_dev, M, exit_bits);
  else fill_v_kernel<PF64><<<blocks, 256, 0, s>>>(fit_dev, M, exit_bits);
  return cudaPeekAtLastError() == cudaSuccess ? COX_OK : COX_E_CUDA;
}

}  // namespace coxgb
