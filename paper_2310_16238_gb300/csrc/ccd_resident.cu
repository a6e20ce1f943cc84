// Resident coordinate-descent kernel: the whole risk sequence of one fit stays in shared
// memory across coordinate steps (arXiv 2310.16238 §2.4-§2.7 for the method).
//
// One cooperative launch of one 1024-thread CTA per SM runs many coordinate steps. CTA t owns
// the positions [tile_lo[t], tile_lo[t+1]) and keeps their values v = +-exp(eta - shift) in
// shared memory for the whole launch, with its tie-group read positions and stratum ends.
// Each step:
//   1. applies the previous step's update at its nonzeros (eta += dbeta, eq. parallel_xb;
//      v = +-exp(eta - shift), eq. parallel_d) directly in shared memory,
//   2. scans its positions for D = v and N1 = x_j v (segmented suffix, strata are segments),
//      combines threads with warp-shuffle scans and CTAs by reading the published aggregates
//      of the later CTAs of the stratum (all CTAs are co-resident, so no carry chain),
//   3. evaluates the tie-group ratios of eqs. (parallel_g)/(parallel_h) into a CTA partial,
//   4. all-gathers the partials of every CTA and reduces them in a fixed order, so every CTA
//      computes the same Newton / trust-region / L1 step (§2.4) without another launch.
// Column j+1's entries are fetched while step j waits on other CTAs; their eta values are read
// after step j's own update is applied. Binary X only (x = 1 at every stored entry).
#include <cuda_runtime.h>

#include <cstdint>

#include "ccd_common.cuh"
#include "cox.h"
#include "cox_internal.h"

namespace coxgb {

constexpr int kResThreads = 1024;
constexpr int kResHeadCap = 1024;    // tie-group read positions per CTA
constexpr int kResListCap = 1024;    // column entries per CTA held in shared memory
constexpr int kResMaxCtas = 256;     // grid limit (one CTA per SM; GB300 has 152 SMs)

template <class P>
struct ResSmem {
  using T = typename P::T;
  using Acc = typename P::Acc;
  static constexpr int NV = 2;
  static constexpr int TILE = kResThreads * P::ITEMS;
  static constexpr int WORDS = TILE / 32;
  static constexpr size_t al(size_t x) { return (x + 15) & ~size_t(15); }
  static constexpr size_t o_v = 0;
  static constexpr size_t o_head = o_v + sizeof(T) * TILE;
  static constexpr size_t o_cut = o_head + 4 * WORDS;
  static constexpr size_t o_nz = o_cut + 4 * WORDS;
  static constexpr size_t o_hpre = o_nz + 4 * WORDS;
  static constexpr size_t o_hloc = al(o_hpre + 4 * WORDS);
  static constexpr size_t o_hpos = o_hloc + sizeof(Acc) * NV * kResHeadCap;
  static constexpr size_t o_hd = al(o_hpos + 2 * kResHeadCap);
  static constexpr size_t o_hcut = o_hd + 4 * kResHeadCap;
  static constexpr size_t o_tc = al(o_hcut + kResHeadCap);
  static constexpr size_t o_tflag = o_tc + sizeof(Acc) * NV * (kResThreads + 32);
  static constexpr size_t o_lpos = al(o_tflag + kResThreads + 32);          // [2][cap] entry positions
  static constexpr size_t o_leta = al(o_lpos + 2 * 4 * kResListCap);         // [2][cap] eta at entries
  static constexpr size_t o_part = o_leta + 2 * 8 * kResListCap;             // [T][3] gathered partials
  static constexpr size_t bytes = o_part + 3 * 8 * kResMaxCtas;
};

int res_tile(int precision) { return precision == COX_FP32C ? kResThreads * PF32C::ITEMS : kResThreads * PF64::ITEMS; }
int res_head_cap() { return kResHeadCap; }

// Step-synchronous control state, identical in every CTA.
struct ResState {
  int32_t j, sweep, need_ll, pend_j, state, list_over[2];
  double pend_db, obj_prev, bdx, pen, loglik, obj;
  int64_t coord_updates;
  uint32_t epoch;
};

// Thread aggregates live at slot(th) = (th % 32) * 33 + th / 32 (per value array), so the raking
// lane l, which walks threads 32 l .. 32 l + 31, reads 32 consecutive slots across the warp.
static __device__ __forceinline__ int tslot(int th) { return (th & 31) * 33 + (th >> 5); }
constexpr int kTcStride = kResThreads + 32;   // slots per value array

template <int NV, int NT>
static __device__ void block_sum_t(double (&v)[NV], double *scratch /* [NV*32] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) scratch[i * 32 + warp] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double x = lane < NT / 32 ? scratch[i * 32 + lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      v[i] = x;   // valid in thread 0
    }
  }
  __syncthreads();
}


// ---- epoch-tagged exchange records: every 8-byte word is (epoch << 32) | 32 data bits, so a
// reader validates and receives a record with one round trip (aligned 8-byte accesses are
// single-copy atomic; no status word, release or fence is needed)
static __device__ __forceinline__ void st_cg_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.global.cg.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
static __device__ __forceinline__ void ld_cg_v2(const uint64_t *p, uint64_t &a, uint64_t &b) {
  asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
static __device__ __forceinline__ void put_tagged(uint64_t *w, uint32_t tag, double v) {
  const uint64_t b = uint64_t(__double_as_longlong(v));
  st_cg_u64(w, (uint64_t(tag) << 32) | (b & 0xffffffffull));
  st_cg_u64(w + 1, (uint64_t(tag) << 32) | (b >> 32));
}
static __device__ __forceinline__ bool tag_ok(uint64_t w, uint32_t tag) { return uint32_t(w >> 32) == tag; }
static __device__ __forceinline__ double untag(uint64_t lo, uint64_t hi) {
  return __longlong_as_double(static_cast<long long>((lo & 0xffffffffull) | ((hi & 0xffffffffull) << 32)));
}

static __device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

static __device__ double penalty_of(const DevFit &F, int j, double b) {
  const bool pen = F.penalize ? F.penalize[j] != 0 : true;
  if (!pen) return 0.0;
  if (F.penalty == COX_PEN_L1) return F.lambda * fabs(b);
  if (F.penalty == COX_PEN_L2) return b * b / (2.0 * F.l2_var);
  return 0.0;
}

// Stage column j's entries in [lo, hi) into list slot `b` (positions relative to lo, exit bit kept);
// returns through s->list_over[b] whether they did not fit.
static __device__ void res_load_list(const DevData &D, const int32_t *col_tile, int t, int T_, int j, int lo, uint32_t *lpos,
                                     int *count, int *over) {
  const int64_t cb = D.col_ptr[j];
  const int32_t *ct = col_tile + int64_t(j) * (T_ + 1);
  const int64_t qa = cb + ct[t], qb = cb + ct[t + 1];
  const int n = int(qb - qa);
  for (int m = threadIdx.x; m < n && m < kResListCap; m += kResThreads) {
    const uint32_t e = D.idx[qa + m];
    lpos[m] = (uint32_t(int(e & kPosMask) - lo)) | (e & kExitBit);
  }
  if (threadIdx.x == 0) {
    *count = n;
    *over = n > kResListCap;
  }
}

template <class P>
__global__ void __launch_bounds__(kResThreads, 1) ccd_resident_kernel(const ResParams prm) {
  using T = typename P::T;
  using Acc = typename P::Acc;
  using S = ResSmem<P>;
  constexpr int NV = 2;
  constexpr int ITEMS = P::ITEMS;
  constexpr int TILE = S::TILE;
  constexpr int WORDS = S::WORDS;
  constexpr int PC = 16 / sizeof(T);
  constexpr int TCH = ITEMS / PC;
  constexpr int RAKE = kResThreads / 32;
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
  uint32_t *lpos = reinterpret_cast<uint32_t *>(smem + S::o_lpos);
  double *leta = reinterpret_cast<double *>(smem + S::o_leta);
  double *gpart = reinterpret_cast<double *>(smem + S::o_part);

  __shared__ ResState st;
  __shared__ int s_count[2];
  __shared__ double s_red[3 * 32];
  __shared__ Acc s_carry[NV];
  __shared__ double s_wred[3][kResThreads / 32];
  __shared__ double s_G[3];
  __shared__ Acc s_wagg[2][32];
  __shared__ int s_wflag[32];
  __shared__ Acc s_wcar[2][32];
  __shared__ int s_wcflag[32];

  const DevFit &F = prm.F;
  const DevData &D = prm.D;
  FitCtl *ctl = F.ctl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int t = blockIdx.x, T_ = gridDim.x;
  const int lo = prm.tile_lo[t], hi = prm.tile_lo[t + 1];
  const double shift = F.shift;
  T *vglob = static_cast<T *>(F.v);

  // ---- one-time staging: values, tie groups, stratum ends, control state
  {
    const int nch = (hi - lo + PC - 1) / PC;
    const unsigned char *g = reinterpret_cast<const unsigned char *>(vglob + lo);
    for (int c = tid; c < nch; c += kResThreads) {
      const int phys = c ^ ((c >> 3) & 7);
      cp_async16(smem + S::o_v + size_t(phys) * 16, g + size_t(c) * 16);
    }
    cp_async_commit();
  }
  for (int q = tid; q < WORDS; q += kResThreads) { headbits[q] = 0u; cutbits[q] = 0u; }
  if (tid == 0) {
    st.j = ctl->j;
    st.sweep = ctl->sweep;
    st.need_ll = ctl->need_ll;
    st.pend_j = ctl->pend_j;
    st.pend_db = ctl->pend_db;
    st.state = ctl->state;
    st.obj_prev = ctl->obj_prev;
    st.loglik = ctl->loglik;
    st.obj = ctl->obj;
    st.coord_updates = ctl->coord_updates;
    st.epoch = ctl->epoch;
  }
  __syncthreads();
  const int ga = prm.tile_g[t], nh = prm.tile_g[t + 1] - ga;
  for (int h = tid; h < nh; h += kResThreads) {
    const int pos = D.head_pos[ga + h] - lo;
    hpos[h] = uint16_t(pos);
    hd[h] = D.head_d[ga + h];
    atomicOr(&headbits[pos >> 5], 1u << (pos & 31));
  }
  for (int k = prm.tile_k[t] + tid; k < prm.tile_k[t + 1]; k += kResThreads) {
    const int pos = D.cut_pos[k] - lo;
    atomicOr(&cutbits[pos >> 5], 1u << (pos & 31));
  }
  {   // beta'dX and the penalty at the starting coefficients (same order in every CTA)
    double ex[2] = {0.0, 0.0};
    for (int jj = tid; jj < D.p; jj += kResThreads) {
      const double b = F.beta[jj];
      ex[0] += b * D.dX[jj];
      ex[1] += penalty_of(F, jj, b);
    }
    block_sum_t<2, kResThreads>(ex, s_red);
    if (tid == 0) { st.bdx = ex[0]; st.pen = ex[1]; }
  }
  cp_async_wait_all();
  __syncthreads();
  for (int e = (hi - lo) + tid; e < TILE; e += kResThreads) {
    const int c = e / PC;
    sv[(c ^ ((c >> 3) & 7)) * PC + (e % PC)] = T(0);
  }
  if (warp == 0) {
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
  // entries of the pending column (if resuming with an update) and of the first column
  int cur = 0;   // list slot of the column scanned in this step; slot cur^1 holds the pending column
  if (st.pend_j >= 0) res_load_list(D, prm.col_tile, t, T_, st.pend_j, lo, lpos + kResListCap, &s_count[1], &st.list_over[1]);
  __syncthreads();
  if (st.pend_j >= 0 && !st.list_over[1])
    for (int m = tid; m < s_count[1] && m < kResListCap; m += kResThreads) {
      const int pos = int(lpos[kResListCap + m] & kPosMask);
      leta[kResListCap + m] = pos < hi - lo ? F.eta[lo + pos] : 0.0;
    }
  if (st.state == kRunning) res_load_list(D, prm.col_tile, t, T_, st.j, lo, lpos, &s_count[0], &st.list_over[0]);
  __syncthreads();

  for (int64_t step = 0; step < prm.max_steps && st.state == kRunning; ++step) {
    const int j = st.j, pend_j = st.pend_j;
    const double pend_db = st.pend_db;
    const bool need_ll = st.need_ll != 0;
    const uint32_t epoch = st.epoch;
    const int pslot = cur ^ 1;
    uint64_t *trace = (COX_TRACE_ON && prm.trace && step < prm.trace_steps && tid == 0) ? prm.trace + (step * T_ + t) * 8 : nullptr;
    if (trace) trace[0] = gtimer();
    // this coordinate's inputs to the step, loaded now so their latency overlaps the step
    // (beta_j and trust_j were last written by CTA 0 at least one all-gather ago when p >= 2)
    double pre_dx = 0.0, pre_b = 0.0, pre_tr = 0.0;
    int pre_pen = 1;
    if (tid == 0) {
      pre_dx = D.dX[j];
      pre_pen = F.penalize ? F.penalize[j] != 0 : 1;
      if (D.p >= 2) {
        pre_b = ld_relaxed_f64(&F.beta[j]);
        pre_tr = ld_relaxed_f64(&F.trust[j]);
      }
    }
    // ---- 1. the pending update, in shared memory (eta also written back to global)
    if (pend_j >= 0) {
      if (!st.list_over[pslot]) {
        for (int m = tid; m < s_count[pslot]; m += kResThreads) {
          const uint32_t e = lpos[pslot * kResListCap + m];
          const int pos = int(e & kPosMask);
          if (pos >= hi - lo) {   // never expected: a list entry outside this CTA's positions
            atomicCAS(&ctl->error, 0, COX_E_INVALID);
            continue;
          }
          const double et = __dadd_rn(leta[pslot * kResListCap + m], pend_db);
          F.eta[lo + pos] = et;
          const int c = pos / PC;
          sv[(c ^ ((c >> 3) & 7)) * PC + (pos % PC)] = make_v<P>(et, shift, (e & kExitBit) != 0, &ctl->error);
        }
      } else {   // more entries than the list holds: walk the column in global memory
        const int64_t cb = D.col_ptr[pend_j];
        const int32_t *ct = prm.col_tile + int64_t(pend_j) * (T_ + 1);
        for (int64_t q = cb + ct[t] + tid; q < cb + ct[t + 1]; q += kResThreads) {
          const uint32_t e = D.idx[q];
          const int pos = int(e & kPosMask) - lo;
          if (pos < 0 || pos >= hi - lo) {
            atomicCAS(&ctl->error, 0, COX_E_INVALID);
            continue;
          }
          const double et = __dadd_rn(F.eta[lo + pos], pend_db);
          F.eta[lo + pos] = et;
          const int c = pos / PC;
          sv[(c ^ ((c >> 3) & 7)) * PC + (pos % PC)] = make_v<P>(et, shift, (e & kExitBit) != 0, &ctl->error);
        }
      }
    }
    // ---- 2. column j's bitmask
    for (int q = tid; q < WORDS; q += kResThreads) nzbits[q] = 0u;
    __syncthreads();
    if (!st.list_over[cur]) {
      for (int m = tid; m < s_count[cur]; m += kResThreads) {
        const int pos = int(lpos[cur * kResListCap + m] & kPosMask);
        if (pos < hi - lo) atomicOr(&nzbits[pos >> 5], 1u << (pos & 31));
      }
    } else {
      const int64_t cb = D.col_ptr[j];
      const int32_t *ct = prm.col_tile + int64_t(j) * (T_ + 1);
      for (int64_t q = cb + ct[t] + tid; q < cb + ct[t + 1]; q += kResThreads) {
        const int pos = int(D.idx[q] & kPosMask) - lo;
        atomicOr(&nzbits[pos >> 5], 1u << (pos & 31));
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
    Acc a0 = P::zero(), a1 = P::zero();
    int seen = 0;
    const bool any_nz = __any_sync(0xffffffffu, zm != 0u);
    // warps whose slots all lie past the tile's end hold zeros only: nothing to scan
    if (__any_sync(0xffffffffu, b0 < hi - lo))
#pragma unroll
    for (int k = ITEMS - 1; k >= 0; --k) {
      if ((cm >> k) & 1u) { a0 = P::zero(); a1 = P::zero(); seen = 1; }
      P::add(a0, vals[k]);
      if (any_nz && __any_sync(0xffffffffu, (zm >> k) & 1u))
        if ((zm >> k) & 1u) P::add(a1, vals[k]);
      if ((hm >> k) & 1u) {
        const int h = hb + __popc(hm & ((1u << k) - 1u));
        hloc[NV * h + 0] = a0;
        hloc[NV * h + 1] = a1;
        hcut[h] = uint8_t(seen);
      }
    }
    // ---- 4. segmented suffix over the thread aggregates: every warp scans its 32 threads,
    //         then warp 0 scans the 32 warp aggregates, publishes the tile aggregate and looks back
    {
      Acc x0 = a0, x1 = a1;
      int xf = cm != 0u;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const Acc y0 = P::shfl_down(x0, off), y1 = P::shfl_down(x1, off);
        const int yf = __shfl_down_sync(0xffffffffu, xf, off);
        if (lane + off < 32) {
          if (!xf) { x0 = P::comb(x0, y0); x1 = P::comb(x1, y1); }
          xf |= yf;
        }
      }
      // exclusive within the warp: the inclusive value of lane + 1
      Acc e0 = P::shfl_down(x0, 1), e1 = P::shfl_down(x1, 1);
      int ef = __shfl_down_sync(0xffffffffu, xf, 1);
      if (lane == 31) { e0 = P::zero(); e1 = P::zero(); ef = 0; }
      tc[tslot(tid)] = e0;
      tc[kTcStride + tslot(tid)] = e1;
      tflag[tslot(tid)] = uint8_t(ef);
      if (lane == 0) { s_wagg[0][warp] = x0; s_wagg[1][warp] = x1; s_wflag[warp] = xf; }
    }
    __syncthreads();
    if (trace) trace[1] = gtimer();
    if (warp == 0) {
      Acc x0 = s_wagg[0][lane], x1 = s_wagg[1][lane];
      int xf = s_wflag[lane];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const Acc y0 = P::shfl_down(x0, off), y1 = P::shfl_down(x1, off);
        const int yf = __shfl_down_sync(0xffffffffu, xf, off);
        if (lane + off < 32) {
          if (!xf) { x0 = P::comb(x0, y0); x1 = P::comb(x1, y1); }
          xf |= yf;
        }
      }
      Acc c0 = P::shfl_down(x0, 1), c1 = P::shfl_down(x1, 1);
      int cf = __shfl_down_sync(0xffffffffu, xf, 1);
      if (lane == 31) { c0 = P::zero(); c1 = P::zero(); cf = 0; }
      s_wcar[0][lane] = c0;   // carry into warp `lane` from the later warps of this tile
      s_wcar[1][lane] = c1;
      s_wcflag[lane] = cf;
      const int tf = __shfl_sync(0xffffffffu, xf, 0);
      const double agg0 = __shfl_sync(0xffffffffu, P::to64(x0), 0), agg1 = __shfl_sync(0xffffffffu, P::to64(x1), 0);
      const uint32_t tag = epoch;
      if (lane == 0) {   // publish the aggregate; a tile holding a stratum end is flagged
        uint64_t *w = prm.tagg + 6 * int64_t(t);
        put_tagged(w, tag, agg0);
        put_tagged(w + 2, tag, agg1);
        st_cg_u64(w + 4, (uint64_t(tag) << 32) | uint64_t(tf));
      }
      // carry from the later tiles of this stratum: every CTA publishes its aggregate each step,
      // so read them all (up to the first tile holding a stratum end) and sum them in a fixed
      // order -- no tile waits for another tile's carry, and the result is deterministic
      double cr0 = 0.0, cr1 = 0.0;
      const bool last_is_cut = ((cutbits[(hi - lo - 1) >> 5] >> ((hi - lo - 1) & 31)) & 1u) != 0u;
      if (t + 1 < T_ && !last_is_cut) {
        const long long tstart = clock64();
        for (int base = t + 1; base < T_; base += 32) {
          const int u = base + lane;
          uint64_t w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
          bool quit = false;
          if (u < T_) {
            const uint64_t *w = prm.tagg + 6 * int64_t(u);
            for (;;) {
              ld_cg_v2(w, w0, w1);
              ld_cg_v2(w + 2, w2, w3);
              ld_cg_v2(w + 4, w4, w5);
              if (tag_ok(w0, tag) && tag_ok(w1, tag) && tag_ok(w2, tag) && tag_ok(w3, tag) && tag_ok(w4, tag)) break;
              if (clock64() - tstart > prm.spin || *reinterpret_cast<volatile int32_t *>(&ctl->error) != 0) {
                quit = true;
                break;
              }
              __nanosleep(20);
            }
          }
          if (__any_sync(0xffffffffu, quit)) {
            if (lane == 0) atomicCAS(&ctl->error, 0, COX_E_TIMEOUT);
            break;
          }
          const uint32_t fm = __ballot_sync(0xffffffffu, u < T_ && (w4 & 1ull));
          const int stop = fm ? __ffs(fm) - 1 : 31;
          double v0 = 0.0, v1 = 0.0;
          if (u < T_ && lane <= stop) {
            v0 = untag(w0, w1);
            v1 = untag(w2, w3);
          }
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) {
            v0 += __shfl_down_sync(0xffffffffu, v0, off);
            v1 += __shfl_down_sync(0xffffffffu, v1, off);
          }
          cr0 += __shfl_sync(0xffffffffu, v0, 0);
          cr1 += __shfl_sync(0xffffffffu, v1, 0);
          if (fm) break;
        }
      }
      if (lane == 0) {
        s_carry[0] = P::from64(cr0);
        s_carry[1] = P::from64(cr1);
      }
    }
    // the next column's entries, fetched while other CTAs are still scanning (its eta values
    // are read after the next update, in the next step)
    const int jn = j + 1 >= D.p ? 0 : j + 1;
    if (warp != 0) {
      // warps 1.. stage the entries; warp 0 is busy with the look-back
      const int64_t cb = D.col_ptr[jn];
      const int32_t *ct = prm.col_tile + int64_t(jn) * (T_ + 1);
      const int64_t qa = cb + ct[t], qb = cb + ct[t + 1];
      const int n = int(qb - qa);
      for (int m = tid - 32; m < n && m < kResListCap; m += kResThreads - 32) {
        const uint32_t e = D.idx[qa + m];
        lpos[pslot * kResListCap + m] = (uint32_t(int(e & kPosMask) - lo)) | (e & kExitBit);
      }
      if (tid == 32) { s_count[pslot] = n; st.list_over[pslot] = n > kResListCap; }
    }
    __syncthreads();

    if (trace) trace[2] = gtimer();
    // ---- 5. tie-group ratios into this CTA's partial
    double r_g1 = 0.0, r_g2 = 0.0, r_ll = 0.0;
    if (warp * 32 < nh) {
      const Acc C0 = s_carry[0], C1 = s_carry[1];
      Acc q_g1 = P::zero(), q_g2 = P::zero();
      for (int h = tid; h < nh; h += kResThreads) {
        const int ot = hpos[h] / ITEMS, o = tslot(ot), ow = ot >> 5;
        Acc s0 = hloc[NV * h], s1 = hloc[NV * h + 1];
        if (!hcut[h]) {
          // carry of the owner thread: later threads of its warp, then later warps, then later tiles
          Acc k0 = tc[o], k1 = tc[kTcStride + o];
          if (!tflag[o]) {
            k0 = P::comb(k0, s_wcar[0][ow]);
            k1 = P::comb(k1, s_wcar[1][ow]);
            if (!s_wcflag[ow]) { k0 = P::comb(k0, C0); k1 = P::comb(k1, C1); }
          }
          s0 = P::comb(s0, k0);
          s1 = P::comb(s1, k1);
        }
        const int dgi = hd[h];
        if constexpr (sizeof(T) == 8) {
          const double S0 = P::to64(s0), S1 = P::to64(s1), dg = double(dgi);
          const double r = S1 * (1.0 / S0);
          r_g1 += dg * r;
          r_g2 += dg * (r * (1.0 - r));
          if (need_ll) r_ll += dg * log(S0);
        } else {
          const float S0 = s0.s + s0.c, S1 = s1.s + s1.c, fd = float(dgi);
          const float r = __fdiv_rn(S1, S0);
          P::add(q_g1, fd * r);
          P::add(q_g2, fd * (r * (1.0f - r)));
          if (need_ll) r_ll += double(dgi) * log(P::to64(s0));
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
      if (need_ll)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) r_ll += __shfl_down_sync(0xffffffffu, r_ll, off);
    }
    if (lane == 0) { s_wred[0][warp] = r_g1; s_wred[1][warp] = r_g2; s_wred[2][warp] = r_ll; }
    __syncthreads();
    const int par = int(epoch & 1u);
    const uint32_t ptag = epoch;
    if (warp == 0) {
      double p0 = s_wred[0][lane], p1 = s_wred[1][lane], p2 = s_wred[2][lane];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        p0 += __shfl_down_sync(0xffffffffu, p0, off);
        p1 += __shfl_down_sync(0xffffffffu, p1, off);
        p2 += __shfl_down_sync(0xffffffffu, p2, off);
      }
      if (lane == 0) {
        uint64_t *w = prm.tpart + 6 * (int64_t(par) * T_ + t);
        put_tagged(w, ptag, p0);
        put_tagged(w + 2, ptag, p1);
        put_tagged(w + 4, ptag, p2);
        if (trace) trace[3] = gtimer();
      }
    }
    // ---- 6. all-gather of the CTA partials (one thread per CTA), fixed-order reduction
    if (tid < T_) {
      const long long tstart = clock64();
      const uint64_t *w = prm.tpart + 6 * (int64_t(par) * T_ + tid);
      uint64_t w0, w1, w2, w3, w4, w5;
      for (;;) {
        ld_cg_v2(w, w0, w1);
        ld_cg_v2(w + 2, w2, w3);
        ld_cg_v2(w + 4, w4, w5);
        if (tag_ok(w0, ptag) && tag_ok(w1, ptag) && tag_ok(w2, ptag) && tag_ok(w3, ptag) && tag_ok(w4, ptag) &&
            tag_ok(w5, ptag))
          break;
        if (clock64() - tstart > prm.spin) { atomicCAS(&ctl->error, 0, COX_E_TIMEOUT); break; }
        if (*reinterpret_cast<volatile int32_t *>(&ctl->error) != 0) break;   // another CTA gave up
        __nanosleep(20);
      }
      gpart[3 * tid] = untag(w0, w1);
      gpart[3 * tid + 1] = untag(w2, w3);
      gpart[3 * tid + 2] = untag(w4, w5);
    } else if (!st.list_over[cur]) {
      // meanwhile the other threads read eta at column j's entries (current since this step's
      // update): the next step's update starts from these values
      for (int m = tid - T_; m < s_count[cur]; m += kResThreads - T_) {
        const int pos = int(lpos[cur * kResListCap + m] & kPosMask);
        leta[cur * kResListCap + m] = pos < hi - lo ? F.eta[lo + pos] : 0.0;
      }
    }
    __syncthreads();
    if (warp == 0) {
      double g0 = 0.0, g1 = 0.0, g2 = 0.0;
      for (int u = lane; u < T_; u += 32) { g0 += gpart[3 * u]; g1 += gpart[3 * u + 1]; g2 += gpart[3 * u + 2]; }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        g0 += __shfl_down_sync(0xffffffffu, g0, off);
        g1 += __shfl_down_sync(0xffffffffu, g1, off);
        g2 += __shfl_down_sync(0xffffffffu, g2, off);
      }
      if (lane == 0) { s_G[0] = g0; s_G[1] = g1; s_G[2] = g2; }
    }
    __syncthreads();
    if (trace) trace[4] = gtimer();
    // ---- 7. the coordinate step, computed identically by every CTA
    if (tid == 0) {
      const double G1 = s_G[0], G2 = s_G[1], LL = s_G[2];
      bool stop = false;
      if (*reinterpret_cast<volatile int32_t *>(&ctl->error) != 0) {
        st.state = kError;
        stop = true;
      } else if (need_ll) {
        const double ll = st.bdx - LL - shift * D.sum_d;
        const double obj = -ll + st.pen;
        st.loglik = ll;
        st.obj = obj;
        if (st.sweep > 0 && fabs(obj - st.obj_prev) <= F.tol * fabs(obj)) {
          st.state = kConverged;
          stop = true;
        } else if (st.sweep >= F.max_sweeps) {
          st.state = kMaxed;
          stop = true;
        } else {
          st.obj_prev = obj;
        }
      }
      if (stop) st.pend_j = -1;   // this step already applied the pending update
      if (!stop) {
        const double g1 = -pre_dx + G1, g2 = G2;
        const int pen = pre_pen;
        // with one column, CTA 0 wrote beta_0 in the previous step: read it after this all-gather
        const double b_old = D.p >= 2 ? pre_b : ld_relaxed_f64(&F.beta[j]);
        double tr = D.p >= 2 ? pre_tr : ld_relaxed_f64(&F.trust[j]);
        const double s = ccd_step_rule(g1, g2, b_old, &tr, F.penalty, F.lambda, F.l2_var, pen);
        const double b_new = b_old + s;
        if (t == 0) {
          F.trust[j] = tr;
          F.beta[j] = b_new;
        }
        if (s != 0.0) {
          st.pend_j = j;
          st.pend_db = s;
          st.bdx = st.bdx + s * pre_dx;
          st.pen = st.pen + (penalty_of(F, j, b_new) - penalty_of(F, j, b_old));
        } else {
          st.pend_j = -1;
          st.pend_db = 0.0;
        }
        st.coord_updates += 1;
        if (jn == 0) {
          st.sweep += 1;
          st.need_ll = 1;
        } else {
          st.need_ll = 0;
        }
        st.j = jn;
      }
      st.epoch = epoch + 1u;
      if (trace) trace[5] = gtimer();
    }
    __syncthreads();
    cur ^= 1;
  }

  // ---- write back the resident values and (CTA 0) the control state
  for (int e = tid; e < hi - lo; e += kResThreads) {
    const int c = e / PC;
    vglob[lo + e] = sv[(c ^ ((c >> 3) & 7)) * PC + (e % PC)];
  }
  if (t == 0 && tid == 0) {
    ctl->j = st.j;
    ctl->sweep = st.sweep;
    ctl->need_ll = st.need_ll;
    ctl->pend_j = st.pend_j;
    ctl->pend_db = st.pend_db;
    ctl->state = st.state;
    ctl->obj_prev = st.obj_prev;
    ctl->loglik = st.loglik;
    ctl->obj = st.obj;
    ctl->coord_updates = st.coord_updates;
    ctl->epoch = st.epoch;
  }
}

int res_smem_bytes(int precision) {
  return int(precision == COX_FP32C ? ResSmem<PF32C>::bytes : ResSmem<PF64>::bytes);
}

template <class P>
static int res_max_ctas() {
  static int cached = -2;
  if (cached != -2) return cached;
  const size_t sm = ResSmem<P>::bytes;
  if (cudaFuncSetAttribute(ccd_resident_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)) != cudaSuccess) {
    cudaGetLastError();
    return cached = 0;
  }
  int per_sm = 0, dev = 0, nsm = 0, coop = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ccd_resident_kernel<P>, kResThreads, sm) != cudaSuccess) {
    cudaGetLastError();
    return cached = 0;
  }
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  const int g = coop ? per_sm * nsm : 0;
  return cached = g < kResMaxCtas ? g : kResMaxCtas;
}

int res_max_grid(int precision) { return precision == COX_FP32C ? res_max_ctas<PF32C>() : res_max_ctas<PF64>(); }

int launch_resident(int precision, const ResParams &prm, int grid, void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void *args[] = {const_cast<ResParams *>(&prm)};
  count_launches(1);
  cudaError_t e;
  if (precision == COX_FP32C) {
    if (res_max_ctas<PF32C>() < grid) return COX_E_INVALID;
    e = cudaLaunchCooperativeKernel(reinterpret_cast<void *>(ccd_resident_kernel<PF32C>), dim3(grid), dim3(kResThreads),
                                    args, ResSmem<PF32C>::bytes, s);
  } else {
    if (res_max_ctas<PF64>() < grid) return COX_E_INVALID;
    e = cudaLaunchCooperativeKernel(reinterpret_cast<void *>(ccd_resident_kernel<PF64>), dim3(grid), dim3(kResThreads),
                                    args, ResSmem<PF64>::bytes, s);
  }
  return e == cudaSuccess ? COX_OK : COX_E_CUDA;
}

}  // namespace coxgb
