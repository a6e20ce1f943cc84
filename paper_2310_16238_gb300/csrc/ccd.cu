// Fused coordinate-step kernel for cyclic coordinate descent on the stratified /
// time-varying Cox partial likelihood (arXiv 2310.16238, §2.4-§2.7).
//
// One launch advances every fit in its work list by one coordinate. A work item is one
// tile (a contiguous range of risk-sequence positions) of one fit. Per item, one CTA:
//   1. applies the previous coordinate's pending update at the tile's nonzeros
//      (eta += x_j * dbeta, eq. parallel_xb; v = +-exp(eta - shift), eq. parallel_d),
//   2. stages the tile of v in shared memory (cp.async, XOR-swizzled 16-byte chunks),
//   3. runs a stratum-segmented suffix scan of D = v, N1 = x_j v, N2 = x_j^2 v in registers
//      (one thread = ITEMS consecutive positions), recording local sums at tie-group read
//      positions; strata are segments of the paper's flag-value operator (§2.6), applied
//      right to left,
//   4. combines threads with a warp-shuffle segmented scan and tiles with a decoupled
//      look-back over FP64 tile carries,
//   5. evaluates the ratios of eqs. (parallel_g)/(parallel_h) at its tie groups and reduces
//      them to a tile partial (G1, G2[, sum d log S0]),
//   6. and the last CTA of a fit reduces the partials in a fixed order and takes the
//      coordinate step (§2.4: Newton eq. newton, trust region, L1 directional derivatives).
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
template <class P, int NV>
struct Smem {
  using T = typename P::T;
  using Acc = typename P::Acc;
  static constexpr int TILE = kThreads * P::ITEMS;
  static constexpr int WORDS = TILE / 32;
  static constexpr size_t al(size_t x) { return (x + 15) & ~size_t(15); }
  static constexpr size_t o_v = 0;                                        // TILE values, swizzled
  static constexpr size_t o_head = o_v + sizeof(T) * TILE;                 // head bitmask
  static constexpr size_t o_cut = o_head + 4 * WORDS;                      // stratum-end bitmask
  static constexpr size_t o_nz = o_cut + 4 * WORDS;                        // column-j bitmask
  static constexpr size_t o_hpre = o_nz + 4 * WORDS;                       // popcount prefix of heads
  static constexpr size_t o_hloc = al(o_hpre + 4 * WORDS);                 // local sums at heads
  static constexpr size_t o_hpos = o_hloc + sizeof(Acc) * NV * kHeadCap;   // head offsets in tile
  static constexpr size_t o_hd = al(o_hpos + 2 * kHeadCap);                // events per head
  static constexpr size_t o_hcut = o_hd + 4 * kHeadCap;                    // cut after head in its thread
  static constexpr size_t o_tc = al(o_hcut + kHeadCap);                    // thread aggregates, then carries
  static constexpr size_t o_tflag = o_tc + sizeof(Acc) * NV * kThreads;
  static constexpr size_t o_x = al(o_tflag + kThreads);                    // x values (valued X only)
  static constexpr size_t bytes = NV == 3 ? o_x + sizeof(T) * TILE : o_x;
};

// ------------------------------------------------------------------ the kernel
template <class P, int NV, bool kCond>
__global__ void __launch_bounds__(kThreads) ccd_kernel(const DevFit *__restrict__ fits, const WorkItem *__restrict__ items,
                                                       LaunchCtl *lc, int mode, int j_eval, unsigned long long cond,
                                                       long long spin) {
  using T = typename P::T;
  using Acc = typename P::Acc;
  using S = Smem<P, NV>;
  constexpr bool VAL = NV == 3;
  constexpr int ITEMS = P::ITEMS;
  constexpr int TILE = S::TILE;
  constexpr int WORDS = S::WORDS;
  constexpr int PC = 16 / sizeof(T);          // elements per 16-byte chunk
  constexpr int CHUNKS = TILE / PC;
  constexpr int TCH = ITEMS / PC;             // chunks per thread (8)
  constexpr int RAKE = kThreads / 32;         // thread aggregates per lane of the raking warp
  static_assert(TCH == 8, "each thread owns 128 bytes");

  extern __shared__ __align__(16) unsigned char smem[];
  T *sv = reinterpret_cast<T *>(smem + S::o_v);
  uint32_t *headbits = reinterpret_cast<uint32_t *>(smem + S::o_head);
  uint32_t *cutbits = reinterpret_cast<uint32_t *>(smem + S::o_cut);
  uint32_t *nzbits = reinterpret_cast<uint32_t *>(smem + S::o_nz);
  int32_t *hpre = reinterpret_cast<int32_t *>(smem + S::o_hpre);
  Acc *hloc = reinterpret_cast<Acc *>(smem + S::o_hloc);
  uint16_t *hpos = reinterpret_cast<uint16_t *>(smem + S::o_hpos);
  int32_t *hd = reinterpret_cast<int32_t *>(smem + S::o_hd);
  uint8_t *hcut = reinterpret_cast<uint8_t *>(smem + S::o_hcut);
  Acc *tc = reinterpret_cast<Acc *>(smem + S::o_tc);
  uint8_t *tflag = reinterpret_cast<uint8_t *>(smem + S::o_tflag);
  T *xs = reinterpret_cast<T *>(smem + S::o_x);

  __shared__ int s_item;
  __shared__ int s_last;
  __shared__ int s_active;
  __shared__ double s_red[3 * 32];
  __shared__ Acc s_carry[NV];
  __shared__ double s_wred[3][kThreads / 32];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n_items = lc->n_items;
  // nothing to do once every fit stopped, or after a launch of this work list gave up a wait
  if (tid == 0)
    s_active = *reinterpret_cast<volatile int32_t *>(&lc->error) != 0
                   ? 0
                   : (mode == kModeFit ? *reinterpret_cast<volatile int32_t *>(&lc->active) : 1);
  __syncthreads();

  for (; s_active > 0;) {   // a launch after every fit stopped only does the exit accounting
    if (tid == 0) s_item = atomicAdd(&lc->ticket, 1u);
    __syncthreads();
    const int w = s_item;
    if (w >= n_items) break;
    const WorkItem it = items[w];
    const DevFit &F = fits[it.f];
    const int t = it.t;
    FitCtl *ctl = F.ctl;
    if (mode == kModeFit && ctl->state != kRunning) {
      __syncthreads();
      continue;
    }
    const DevData *D = F.d;
    const int T_ = D->T;
    const int lo = D->tile_lo[t], hi = D->tile_lo[t + 1];
    const int j = (mode == kModeEval || mode == kModeShard) ? j_eval : (mode == kModeFit ? ctl->j : -1);
    const bool need_ll = mode == kModeLL || ((mode == kModeFit || mode == kModeShard) && ctl->need_ll);
    const int pend_j = mode == kModeFit ? ctl->pend_j : -1;
    const double pend_db = ctl->pend_db;
    const uint32_t epoch = ctl->epoch;
    const double shift = F.shift;
    const bool vf = VAL && D->val != nullptr;   // binary fits in a valued launch use x = 1

    // ---- 1. stage the tile of v (async), overlapped with the metadata below
    {
      const unsigned char *g = reinterpret_cast<const unsigned char *>(static_cast<const T *>(F.v) + lo);
      for (int c = tid; c < CHUNKS; c += kThreads) {
        const int phys = c ^ ((c >> 3) & 7);
        cp_async16(smem + S::o_v + size_t(phys) * 16, g + size_t(c) * 16);
      }
      cp_async_commit();
    }
    for (int q = tid; q < WORDS; q += kThreads) { headbits[q] = 0u; cutbits[q] = 0u; nzbits[q] = 0u; }
    if (VAL)
      for (int q = tid; q < TILE; q += kThreads) xs[q] = T(0);
    __syncthreads();
    const int ga = D->tile_g[t], nh = D->tile_g[t + 1] - ga;
    for (int h = tid; h < nh; h += kThreads) {
      const int pos = D->head_pos[ga + h] - lo;
      hpos[h] = uint16_t(pos);
      hd[h] = D->head_d[ga + h];
      atomicOr(&headbits[pos >> 5], 1u << (pos & 31));
    }
    {
      const int ka = D->tile_k[t], kb = D->tile_k[t + 1];
      for (int k = ka + tid; k < kb; k += kThreads) {
        const int pos = D->cut_pos[k] - lo;
        atomicOr(&cutbits[pos >> 5], 1u << (pos & 31));
      }
    }
    if (j >= 0) {
      const int64_t cb = D->col_ptr[j];
      const int32_t *ct = D->col_tile + int64_t(j) * (T_ + 1);
      const int64_t qa = cb + ct[t], qb = cb + ct[t + 1];
      for (int64_t q = qa + tid; q < qb; q += kThreads) {
        const int pos = int(D->idx[q] & kPosMask) - lo;
        atomicOr(&nzbits[pos >> 5], 1u << (pos & 31));
        if (vf) xs[pos] = T(D->val[q]);
      }
    }
    // ---- pending update of the previous coordinate at this tile's nonzeros (global)
    int64_t ua = 0, ub = 0;
    if (pend_j >= 0) {
      const int64_t cb = D->col_ptr[pend_j];
      const int32_t *ct = D->col_tile + int64_t(pend_j) * (T_ + 1);
      ua = cb + ct[t];
      ub = cb + ct[t + 1];
      for (int64_t q = ua + tid; q < ub; q += kThreads) {
        const uint32_t e = D->idx[q];
        const int64_t pos = e & kPosMask;
        const double x = D->val ? D->val[q] : 1.0;
        const double et = __dadd_rn(F.eta[pos], __dmul_rn(x, pend_db));
        F.eta[pos] = et;
        static_cast<T *>(F.v)[pos] = make_v<P>(et, shift, (e & kExitBit) != 0, &ctl->error);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    // patch the staged tile with the updated values (each thread rereads its own writes)
    for (int64_t q = ua + tid; q < ub; q += kThreads) {
      const int e = int(D->idx[q] & kPosMask) - lo;
      const int c = e / PC;
      sv[(c ^ ((c >> 3) & 7)) * PC + (e % PC)] = static_cast<const T *>(F.v)[lo + e];
    }
    if (hi - lo < TILE)
      for (int e = hi - lo + tid; e < TILE; e += kThreads) {
        const int c = e / PC;
        sv[(c ^ ((c >> 3) & 7)) * PC + (e % PC)] = T(0);
      }
    if (warp == 0) {   // exclusive popcount prefix of the head bitmask
      int run = 0;
      for (int base = 0; base < WORDS; base += 32) {
        const int c = base + lane < WORDS ? __popc(headbits[base + lane]) : 0;
        int incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, off);
          if (lane >= off) incl += y;
        }
        if (base + lane < WORDS) hpre[base + lane] = run + incl - c;
        run += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    __syncthreads();

    // ---- 3. per-thread segmented suffix over ITEMS consecutive positions
    T vals[ITEMS];
    {
      const int c0 = tid * TCH;
#pragma unroll
      for (int k = 0; k < TCH; ++k) {
        const int c = c0 + k;
        const int phys = c ^ ((c >> 3) & 7);
        const float4 q = *reinterpret_cast<const float4 *>(smem + S::o_v + size_t(phys) * 16);
        const T *qq = reinterpret_cast<const T *>(&q);
#pragma unroll
        for (int u = 0; u < PC; ++u) vals[k * PC + u] = qq[u];
      }
    }
    const int b0 = tid * ITEMS;
    const uint32_t wmask = ITEMS == 32 ? 0xffffffffu : ((1u << ITEMS) - 1u);
    const uint32_t hm = (headbits[b0 >> 5] >> (b0 & 31)) & wmask;
    const uint32_t cm = (cutbits[b0 >> 5] >> (b0 & 31)) & wmask;
    const uint32_t zm = (nzbits[b0 >> 5] >> (b0 & 31)) & wmask;
    const int hb = hpre[b0 >> 5] + __popc(headbits[b0 >> 5] & ((1u << (b0 & 31)) - 1u));
    Acc a[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) a[i] = P::zero();
    int seen = 0;
    const bool any_nz = __any_sync(0xffffffffu, zm != 0u);
#pragma unroll
    for (int k = ITEMS - 1; k >= 0; --k) {
      if ((cm >> k) & 1u) {
#pragma unroll
        for (int i = 0; i < NV; ++i) a[i] = P::zero();
        seen = 1;
      }
      P::add(a[0], vals[k]);
      if (any_nz && __any_sync(0xffffffffu, (zm >> k) & 1u)) {
        if ((zm >> k) & 1u) {
          if constexpr (VAL) {
            const T x = vf ? xs[b0 + k] : T(1);
            const T wv = T(x * vals[k]);
            P::add(a[1], wv);
            P::add(a[2], T(x * wv));
          } else {
            P::add(a[1], vals[k]);
          }
        }
      }
      if ((hm >> k) & 1u) {
        const int h = hb + __popc(hm & ((1u << k) - 1u));
#pragma unroll
        for (int i = 0; i < NV; ++i) hloc[NV * h + i] = a[i];
        hcut[h] = uint8_t(seen);
      }
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) tc[NV * tid + i] = a[i];
    tflag[tid] = uint8_t(cm != 0u);
    __syncthreads();

    // ---- 4. one warp: raking segmented suffix over the thread aggregates, tile aggregate,
    //         per-thread exclusive carries, then the decoupled look-back over earlier tiles
    if (warp == 0) {
      const int t0 = lane * RAKE;
      Acc r[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) r[i] = P::zero();
      int rf = 0;
#pragma unroll
      for (int q = RAKE - 1; q >= 0; --q) {
        const int th = t0 + q;
        if (tflag[th]) {
#pragma unroll
          for (int i = 0; i < NV; ++i) r[i] = tc[NV * th + i];
          rf = 1;
        } else {
#pragma unroll
          for (int i = 0; i < NV; ++i) r[i] = P::comb(tc[NV * th + i], r[i]);
        }
      }
      Acc x[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) x[i] = r[i];
      int xf = rf;
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
      // lane 0 holds the tile's inclusive value from its first position
      const int tf = __shfl_sync(0xffffffffu, xf, 0);
      double agg[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) agg[i] = __shfl_sync(0xffffffffu, P::to64(x[i]), 0);
      const uint32_t ep = (epoch & 0x1fffffffu) << 3;
      if (lane == 0) {   // slots 0..2: aggregate, 3..5: inclusive (a tile holding a stratum end is complete)
        const int o = tf ? 3 : 0;
#pragma unroll
        for (int i = 0; i < NV; ++i) F.tval[6 * t + o + i] = agg[i];
        st_release_u32(&F.tstat[t], ep | (tf ? 4u | 2u : 1u));   // release: the values above first
      }
      // exclusive carries of this lane's threads: start from lane + 1's inclusive value
      Acc c[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) c[i] = P::shfl_down(x[i], 1);
      int cf = __shfl_down_sync(0xffffffffu, xf, 1);
      if (lane == 31) {
#pragma unroll
        for (int i = 0; i < NV; ++i) c[i] = P::zero();
        cf = 0;
      }
#pragma unroll
      for (int q = RAKE - 1; q >= 0; --q) {
        const int th = t0 + q;
        Acc own[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) own[i] = tc[NV * th + i];
        const int of = tflag[th];
#pragma unroll
        for (int i = 0; i < NV; ++i) tc[NV * th + i] = c[i];
        tflag[th] = uint8_t(cf);
        if (of) {
#pragma unroll
          for (int i = 0; i < NV; ++i) c[i] = own[i];
          cf = 1;
        } else {
#pragma unroll
          for (int i = 0; i < NV; ++i) c[i] = P::comb(own[i], c[i]);
        }
      }
      // look back over the tiles to the right (they hold the later positions)
      double cr[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) cr[i] = 0.0;
      const bool last_is_cut = ((cutbits[(hi - lo - 1) >> 5] >> ((hi - lo - 1) & 31)) & 1u) != 0u;
      if (t + 1 < T_ && !last_is_cut) {
        int base = t + 1;
        const long long tstart = clock64();
        bool timed_out = false;
        for (;;) {
          const int u = base + lane;
          uint32_t st = 0;
          bool valid = false;
          for (;;) {
            if (u < T_) {
              st = ld_acquire_u32(&F.tstat[u]);
              valid = (st & ~7u) == ep && (st & 3u) != 0u;
            } else {
              valid = true;
              st = ep | 2u;
            }
            const uint32_t inv = __ballot_sync(0xffffffffu, !valid);
            const uint32_t inc = __ballot_sync(0xffffffffu, valid && (st & 3u) == 2u);
            if (inv == 0u || (inc != 0u && (__ffs(inc) < __ffs(inv)))) break;
            if (clock64() - tstart > spin) { timed_out = true; break; }
            __nanosleep(32);
          }
          if (timed_out) {
            if (lane == 0) atomicExch(&ctl->error, COX_E_TIMEOUT);
            break;
          }
          const uint32_t inc = __ballot_sync(0xffffffffu, valid && (st & 3u) == 2u);
          const int stop = inc ? __ffs(inc) - 1 : 31;
          double v[NV];
#pragma unroll
          for (int i = 0; i < NV; ++i) v[i] = 0.0;
          if (lane <= stop && u < T_) {
            const int o = (st & 3u) == 2u ? 3 : 0;
#pragma unroll
            for (int i = 0; i < NV; ++i) v[i] = ld_relaxed_f64(&F.tval[6 * u + o + i]);
          } else if (lane == stop && u == T_ && lc->ext) {
            // past the data's end: the continuation of its last stratum (the last tile may not have
            // published its inclusive value yet, so a walk can reach here through its aggregate)
#pragma unroll
            for (int i = 0; i < NV; ++i) v[i] = lc->ext[i];
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
      if (t + 1 == T_ && !last_is_cut && lc->ext) {   // the last stratum continues past the data
#pragma unroll
        for (int i = 0; i < NV; ++i) cr[i] = lc->ext[i];
      }
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) s_carry[i] = P::from64(cr[i]);
        if (!tf) {
#pragma unroll
          for (int i = 0; i < NV; ++i) F.tval[6 * t + 3 + i] = agg[i] + cr[i];
          st_release_u32(&F.tstat[t], ep | 2u);
        }
      }
    }
    __syncthreads();

    // ---- 5. tie-group ratios (eqs. parallel_g / parallel_h), head-parallel
    double r_g1 = 0.0, r_g2 = 0.0, r_ll = 0.0;
    if (warp * 32 < nh) {
      Acc C[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) C[i] = s_carry[i];
      Acc q_g1 = P::zero(), q_g2 = P::zero();
      for (int h = tid; h < nh; h += kThreads) {
        const int pos = hpos[h];
        const int o = pos / ITEMS;
        Acc sh[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) sh[i] = hloc[NV * h + i];
        if (!hcut[h]) {
          Acc k[NV];
#pragma unroll
          for (int i = 0; i < NV; ++i) k[i] = tc[NV * o + i];
          if (!tflag[o]) comb_n<Acc, P, NV>(k, C);
          comb_n<Acc, P, NV>(sh, k);
        }
        const int dgi = hd[h];
        if constexpr (sizeof(T) == 8) {
          const double S0 = P::to64(sh[0]), S1 = P::to64(sh[1]);
          const double dg = double(dgi);
          if (j >= 0) {
            const double inv = 1.0 / S0;
            const double r = S1 * inv;
            r_g1 += dg * r;
            if constexpr (VAL) r_g2 += dg * (P::to64(sh[2]) * inv - r * r);
            else r_g2 += dg * (r * (1.0 - r));
          }
          if (need_ll) r_ll += dg * log(S0);
          if (F.out_S0) { F.out_S0[ga + h] = S0; F.out_S1[ga + h] = S1; }
        } else {
          const float S0 = sh[0].s + sh[0].c, S1 = sh[1].s + sh[1].c;
          const float fd = float(dgi);
          if (j >= 0) {
            const float inv = __frcp_rn(S0);
            const float r = __fdiv_rn(S1, S0);
            P::add(q_g1, fd * r);
            if constexpr (VAL) P::add(q_g2, fd * ((sh[2].s + sh[2].c) * inv - r * r));
            else P::add(q_g2, fd * (r * (1.0f - r)));
          }
          if (need_ll) r_ll += double(dgi) * log(P::to64(sh[0]));
          if (F.out_S0) { F.out_S0[ga + h] = P::to64(sh[0]); F.out_S1[ga + h] = P::to64(sh[1]); }
        }
      }
      if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          q_g1 = P::comb(q_g1, P::shfl_down(q_g1, off));
          q_g2 = P::comb(q_g2, P::shfl_down(q_g2, off));
        }
        if (lane == 0) { r_g1 = P::to64(q_g1); r_g2 = P::to64(q_g2); }
      } else {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          r_g1 += __shfl_down_sync(0xffffffffu, r_g1, off);
          r_g2 += __shfl_down_sync(0xffffffffu, r_g2, off);
        }
      }
      if (need_ll) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) r_ll += __shfl_down_sync(0xffffffffu, r_ll, off);
      }
    }
    if (lane == 0) { s_wred[0][warp] = r_g1; s_wred[1][warp] = r_g2; s_wred[2][warp] = r_ll; }
    __syncthreads();
    if (tid == 0) {
      double p0 = 0.0, p1 = 0.0, p2 = 0.0;
      for (int ww = 0; ww < kThreads / 32; ++ww) { p0 += s_wred[0][ww]; p1 += s_wred[1][ww]; p2 += s_wred[2][ww]; }
      F.part[3 * t + 0] = p0; F.part[3 * t + 1] = p1; F.part[3 * t + 2] = p2;
      __threadfence();
      const uint32_t prev = atomicAdd(&ctl->done_tiles, 1u);
      s_last = prev == uint32_t(T_ - 1);
    }
    __syncthreads();

    // ---- 6. last CTA of this fit: fixed-order reduction and the coordinate step
    if (s_last) finish_launch_step<kThreads>(F, lc, mode, j, need_ll, T_, epoch, s_red);
    __syncthreads();
  }
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
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ccd_kernel<P, NV, kCond>, kThreads, sm) != cudaSuccess)
    return -1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return (per_sm > 0 ? per_sm : 1) * nsm;
}

// Resident CTAs of a variant on the current device (occupancy x SMs); both graph variants share
// the smaller figure.
template <class P, int NV>
static int max_grid_impl() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  if (cached[dev]) return cached[dev];
  const int a = max_grid_one<P, NV, false>(), b = max_grid_one<P, NV, true>();
  if (a < 0 || b < 0) return -1;
  cached[dev] = a < b ? a : b;
  return cached[dev];
}

// FP32C runs the chunked kernel (ccd_chunk.cu); this kernel serves FP64.
int ccd_max_grid(int precision, int valued) {
  if (precision == COX_FP32C) return chunk_max_grid(valued);
  return valued ? max_grid_impl<PF64, 3>() : max_grid_impl<PF64, 2>();
}

int ccd_tile(int precision) { return precision == COX_FP32C ? kChunkTile : kThreads * PF64::ITEMS; }

template <class P, int NV>
static int launch_impl(const DevFit *fits, const WorkItem *items, LaunchCtl *lc, int grid, int mode, int j_eval,
                       cudaStream_t s, unsigned long long cond) {
  if (max_grid_impl<P, NV>() < 0) return COX_E_CUDA;
  // the variant that can end a conditional graph loop only where there is one to end: kernels that
  // can set a conditional handle cannot be profiled as single graph kernel nodes
  const long long spin = wait_limit();
  if (cond)
    ccd_kernel<P, NV, true><<<grid, kThreads, Smem<P, NV>::bytes, s>>>(fits, items, lc, mode, j_eval, cond, spin);
  else
    ccd_kernel<P, NV, false><<<grid, kThreads, Smem<P, NV>::bytes, s>>>(fits, items, lc, mode, j_eval, 0ull, spin);
  return COX_OK;
}

int launch_ccd(int precision, const DevFit *fits, const WorkItem *items, LaunchCtl *lc, int grid, int mode, int j_eval,
               int valued, void *stream, unsigned long long cond) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs == cudaStreamCaptureStatusNone) count_launches(1);   // graph nodes are counted per replay
  if (precision == COX_FP32C)
    return launch_chunk(fits, reinterpret_cast<const ChunkItem *>(items), lc, grid, mode, j_eval, valued, stream, cond);
  const int rc = valued ? launch_impl<PF64, 3>(fits, items, lc, grid, mode, j_eval, s, cond)
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
