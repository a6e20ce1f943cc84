// Incremental risk-set kernel: the per-tie-group risk-set sums S0 stay on chip (shared memory)
// across coordinate steps and are updated from the changed positions only (arXiv 2310.16238 §2.4-§2.7
// for the method; this is an exact reformulation of its segmented scans, not the paper's layout).
//
// One cooperative launch of one 1024-thread CTA per SM runs the whole fit. CTA t owns the risk
// positions [tile_lo[t], tile_lo[t+1]) and the tie groups whose read position lies there (thread
// h holds group h, or groups h + 1024 i in the group-dense configuration: S0, read position,
// stratum segment and events). A coordinate step for
// column j touches only the positions of column j's nonzeros:
//   * the previous step's update (eta += dbeta, eq. parallel_xb; v = +-exp(eta - shift), eq.
//     parallel_d) changes v at column j-1's entries by dD = v (e^dbeta - 1); S0 of every group
//     grows by the segmented suffix sum of dD from its read position (strata are segments),
//     which is (e^dbeta - 1) times the group's S1 of the previous step (binary X), plus, for
//     groups whose stratum continues past the tile, the change in the later tiles;
//   * S1 of every group is the segmented suffix sum of v over column j's entries, plus the later
//     tiles' share, so the tie-group ratios of eqs. (parallel_g)/(parallel_h) cost
//     O(groups + entries) per tile instead of O(positions);
//   * the later tiles' shares come from the previous step's exchange: with binary X a tile's
//     head-segment sums after an update by d are R + (e^d - 1) I, so every CTA publishes the sums
//     it will need one step ahead, and one all-gather per step serves both the carries and the
//     Newton / trust-region / L1 step (§2.4), which every CTA computes identically.
// At the first step of a launch and of every sweep (where the log-likelihood is evaluated) v is
// recomputed from eta at every position and S0 rebuilt from a dense scan, which bounds the
// rounding that the multiplicative updates and the incremental sums accumulate within a sweep.
//
// Arithmetic: sums, scans and ratios use double-word floats (dw.cuh, about 48 bits; FP64 issue
// is 64 cycles per warp instruction per sub-partition on this GPU); eta, beta, the step rule and
// the log-likelihood are FP64. v is held as a double-word per position (vdw), so the float
// exponent range applies: |eta - shift| above kIncRange raises COX_E_RANGE (the library then
// falls back to an FP64 engine). Column j+2's entries and their eta and v are fetched while step
// j waits on the exchange, and column j+1's suffix sums are prepared while thread 0 computes
// step j, in a form that takes step j's update as one multiply-add per tie group.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "ccd_common.cuh"
#include "cox.h"
#include "cox_internal.h"
#include "dw.cuh"
#include "step_rule.cuh"

namespace coxgb {

constexpr int kIncThreads = 1024;
constexpr int kIncMaxCtas = 160;   // CTAs of one fit at most (one per SM; 152 on GB300)
constexpr int kIncRec = kIncRecWords / 2;   // step record payloads: G1, G2, LL, H1, R, I
constexpr uint32_t kTagErr = 0x80000000u;   // tag bit: the writer raised an error
constexpr double kIncRange = 60.0;          // |eta - shift| that keeps every sum inside float range
constexpr unsigned kFull = 0xffffffffu;
constexpr int kIncTraceSlots = 24;        // phase timestamps per step and CTA (COXGB_PHASE_TRACE)

constexpr size_t inc_al16(size_t x) { return (x + 15) & ~size_t(15); }

// Capacities of one kernel configuration: tie groups per CTA (kGpt per thread), entries of one
// column per CTA (at most one per thread), positions per CTA (bitmask capacity).
template <int GPT, int LCAP, int PCAP>
struct IncCfg {
  static constexpr int kGpt = GPT;
  static constexpr int kGroupCap = GPT * kIncThreads;
  static constexpr int kListCap = LCAP;
  static constexpr int kPosCap = PCAP;
  static constexpr int kWords = PCAP / 32;
  static_assert(LCAP <= kIncThreads, "one list entry per thread");
};
using IncWide = IncCfg<1, 1024, 65536>;   // one tie group and up to one list entry per thread
using IncDeep = IncCfg<4, 512, 32768>;    // group-dense data: up to four tie groups per thread

template <class Cfg>
struct IncSmem {
  static constexpr int LC = Cfg::kListCap, GC = Cfg::kGroupCap, W = Cfg::kWords;
  static constexpr size_t o_lpos = 0;                                   // u32 [4][cap] entry positions
  static constexpr size_t o_lv = o_lpos + 4 * 4 * LC;                   // dw  [4][cap] v at the entries
  static constexpr size_t o_le = o_lv + 4 * 8 * LC;                     // f64 [4][cap] eta at the entries
  // dw [cap] x 2: segmented suffix sums of v over the current column's entries before the pending
  // update (A), and over those of its entries that the pending update changes (B)
  static constexpr size_t o_ua = o_le + 4 * 8 * LC;
  static constexpr size_t o_ub = o_ua + 8 * LC;
  static constexpr size_t o_cutb = o_ub + 8 * LC;                       // u32 [W] stratum ends
  static constexpr size_t o_cutp = o_cutb + 4 * W;                      // i32 [W] prefix counts
  static constexpr size_t o_headb = o_cutp + 4 * W;                     // u32 [W] read positions
  static constexpr size_t o_headp = o_headb + 4 * W;                    // i32 [W]
  // dw [gcap]: a rebuild's dense-scan S0 per group; otherwise each group's S1 of the last step
  // (without the later tiles' share), which times e^dbeta - 1 is the change of its S0
  static constexpr size_t o_gs0 = o_headp + 4 * W;
  static constexpr size_t o_gseen = o_gs0 + 8 * GC;                     // u8  [gcap]
  static constexpr size_t o_rec = inc_al16(o_gseen + GC);               // 8-byte slots [6][C] record payloads
  static constexpr size_t o_rref = o_rec + 8 * kIncRec * kIncMaxCtas;   // dw [C][2] refresh records
  static constexpr size_t o_grp = o_rref + 8 * 2 * kIncMaxCtas;         // GroupSlot [gcap]
  static constexpr size_t o_pmask = o_grp + 24 * GC;                    // u32 [W] the previous column's positions
  static constexpr size_t o_cmask = o_pmask + 4 * W;                    // u32 [W] the current column's positions
  // u16 [gcap]: per tie group, the first entry of the current column's list at or after the
  // group's read position in its stratum segment (kNoEntry: none). A step reads it for its own
  // column before the exchange wait, where it is rebuilt for the next column, so one copy serves.
  // Kept for one group per thread only: with four, building it off the chain (binary searches of
  // 4,096 groups by the threads not polling) outlasts the wait, and the step searches instead.
  static constexpr int KG = Cfg::kGpt == 1 ? GC : 0;
  static constexpr size_t o_kg = o_cmask + 4 * W;
  static constexpr size_t o_ginv = inc_al16(o_kg + 2 * KG);               // dw [gcap] 1 / S0 per group (same)
  static constexpr size_t o_fce = o_ginv + 8 * KG;                        // u8 [cap] segment ends of a list (as kg)
  static constexpr size_t o_mfl = o_fce + LC;                             // u8 [cap] next-list entries in the current column
  static constexpr size_t bytes = o_mfl + LC;
};

// One tie group of this CTA (thread h owns group h): its risk-set sum S0, read position (relative
// to the tile), events, stratum segment within the tile, and whether the later tiles' carry
// reaches it. Kept in shared memory rather than registers: the step loop is register-bound at
// 1024 threads, and spilled registers would go to memory.
struct GroupSlot {
  dw S0;
  int32_t q;
  float d;
  int32_t seg;
  int32_t tail;
};
static_assert(sizeof(GroupSlot) == 24, "group slot layout");

constexpr uint16_t kNoEntry = 0xffffu;

// First entry of the sorted list lp[0, n) at or after position q that lies in q's stratum
// segment `seg` (kNoEntry: none).
static __device__ __forceinline__ uint16_t inc_first_entry(const uint32_t *lp, int n, int q, int seg,
                                                           const uint32_t *cutb, const int32_t *cutp);

int inc_group_cap(int variant) { return variant ? IncDeep::kGroupCap : IncWide::kGroupCap; }
int inc_list_cap(int variant) { return variant ? IncDeep::kListCap : IncWide::kListCap; }
int inc_pos_cap(int variant) { return variant ? IncDeep::kPosCap : IncWide::kPosCap; }

// Step-synchronous control state, identical in every CTA.
struct IncState {
  int32_t j, sweep, need_ll, pend_j, state;
  int32_t halt;              // the next column is a halt column: end the launch before it
  double pend_db, obj_prev, bdx, pen, loglik, obj;
  dw E;                      // e^pend_db - 1
  int64_t coord_updates;
  uint32_t epoch;
  // the last step's coefficient bookkeeping, done off the critical path at the next step
  int32_t book, book_j, book_pen;
  double book_s, book_b, book_dx, book_t;
};

// This step's column inputs, loaded and converted by an idle thread while the step runs.
struct IncPre {
  double dx, b, t;
  dw dxw, bw, tw;
  int32_t pen, halt_next;
};

// ---- epoch-tagged exchange words: (epoch << 32) | 32 data bits; relaxed 8-byte accesses are
// single-copy atomic, so a reader that sees the tag has the data of that epoch
static __device__ __forceinline__ void st_rlx_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
static __device__ __forceinline__ void st_rlx_v2(uint64_t *p, uint64_t a, uint64_t b) {
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
static __device__ __forceinline__ void ld_rlx_v2(const uint64_t *p, uint64_t &a, uint64_t &b) {
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
static __device__ __forceinline__ void put_tag2(uint64_t *w, uint32_t tag, uint32_t a, uint32_t b) {
  st_rlx_u64(w, (uint64_t(tag) << 32) | a);
  st_rlx_u64(w + 1, (uint64_t(tag) << 32) | b);
}
static __device__ __forceinline__ void put_dw(uint64_t *w, uint32_t tag, dw v) {
  put_tag2(w, tag, __float_as_uint(v.h), __float_as_uint(v.l));
}
static __device__ __forceinline__ bool tagged(uint64_t a, uint64_t b, uint32_t tag) {
  return uint32_t(a >> 32) == tag && uint32_t(b >> 32) == tag;
}
static __device__ __forceinline__ uint64_t inc_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// a record slot holds either a double-word or an FP64 value in 8 bytes
static __device__ __forceinline__ dw slot_dw(const uint64_t *s) { return *reinterpret_cast<const dw *>(s); }
static __device__ __forceinline__ double slot_f64(const uint64_t *s) { return *reinterpret_cast<const double *>(s); }

// Wait for N tagged 8-byte payloads at w (2 words each; all loads of a poll in flight together)
// and store the payloads (low halves of the word pairs) in out. false: the wait gave up (bound
// reached or another CTA raised an error).
template <int N>
static __device__ bool wait_tagged(const uint64_t *w, uint32_t tag, uint64_t *out, int32_t *err, long long spin) {
  const long long t0 = clock64();
  unsigned polls = 0;
  for (;;) {
    uint64_t a[N], b[N];
#pragma unroll
    for (int i = 0; i < N; ++i) ld_rlx_v2(w + 2 * i, a[i], b[i]);
    bool ok = true;
#pragma unroll
    for (int i = 0; i < N; ++i) ok = ok && tagged(a[i], b[i], tag);
    if (ok) {
#pragma unroll
      for (int i = 0; i < N; ++i) out[i] = (a[i] & 0xffffffffull) | ((b[i] & 0xffffffffull) << 32);
      return true;
    }
    if ((++polls & 63) == 0) {   // off the fast path: the bound and another CTA's failure
      if (clock64() - t0 > spin) {
        atomicCAS(err, 0, COX_E_TIMEOUT);
        return false;
      }
      if (*reinterpret_cast<volatile int32_t *>(err) != 0) return false;
    }
    __nanosleep(32);
  }
}

// Wait for the first n (<= N) tagged payloads of a record at w whose tags carry `tag` or `tag` with
// the error bit; the payloads go to out. Returns 1 (clean), 2 (the writer raised an error) or 0
// (the wait gave up: bound reached or another CTA raised an error).
template <int N>
static __device__ int wait_record(const uint64_t *w, int n, uint32_t tag, uint64_t *out, int32_t *err, long long spin,
                                  unsigned *npolls = nullptr) {
  const long long t0 = clock64();
  unsigned polls = 0;
  for (;;) {
    uint64_t a[N], b[N];
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) ld_rlx_v2(w + 2 * i, a[i], b[i]);
    bool ok = true, bad = false;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) {
        const uint32_t ta = uint32_t(a[i] >> 32), tb = uint32_t(b[i] >> 32);
        ok = ok && (ta & ~kTagErr) == tag && (tb & ~kTagErr) == tag;
        bad = bad || ((ta | tb) & kTagErr) != 0;
      }
    if (ok) {
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i < n) out[i] = (a[i] & 0xffffffffull) | ((b[i] & 0xffffffffull) << 32);
      if (npolls) *npolls = polls + 1;
      return bad ? 2 : 1;
    }
    if ((++polls & 63) == 0) {   // off the fast path: the bound and another CTA's failure
      if (clock64() - t0 > spin) {
        atomicCAS(err, 0, COX_E_TIMEOUT);
        return 0;
      }
      if (*reinterpret_cast<volatile int32_t *>(err) != 0) return 0;
    }
    __nanosleep(32);
  }
}

static __device__ __forceinline__ int inc_rank(const uint32_t *bits, const int32_t *pre, int q) {
  return pre[q >> 5] + __popc(bits[q >> 5] & ((1u << (q & 31)) - 1u));
}
static __device__ __forceinline__ int inc_lower_bound(const uint32_t *lp, int n, int q) {
  int a = 0, b = n;
  while (a < b) {
    const int m = (a + b) >> 1;
    if (int(lp[m] & kPosMask) < q) a = m + 1;
    else b = m;
  }
  return a;
}

// Entry k of a sorted list ends its stratum segment within the list (the last entry, or the next
// one lies past a stratum end).
static __device__ __forceinline__ uint8_t inc_seg_end(const uint32_t *lp, int n, int k, const uint32_t *cutb,
                                                      const int32_t *cutp) {
  return (k + 1 >= n ||
          inc_rank(cutb, cutp, int(lp[k + 1] & kPosMask)) != inc_rank(cutb, cutp, int(lp[k] & kPosMask))) ? 1 : 0;
}

static __device__ __forceinline__ uint16_t inc_first_entry(const uint32_t *lp, int n, int q, int seg,
                                                           const uint32_t *cutb, const int32_t *cutp) {
  const int k = inc_lower_bound(lp, n, q);
  return (k < n && inc_rank(cutb, cutp, int(lp[k] & kPosMask)) == seg) ? uint16_t(k) : kNoEntry;
}

static __device__ double inc_penalty(const DevFit &F, int j, double b) {
  const bool pen = F.penalize ? F.penalize[j] != 0 : true;
  if (!pen) return 0.0;
  if (F.penalty == COX_PEN_L1) return F.lambda * fabs(b);
  if (F.penalty == COX_PEN_L2) return b * b / (2.0 * F.l2_var);
  return 0.0;
}

// The bookkeeping of a coordinate step (FP64): the new coefficient and trust half-width
// (max(2 |s|, t / 2), §2.4) in this CTA's copies, beta'dX and the penalty.
template <class St>
static __device__ void inc_book(St &st, double *bet, double *tru, const DevFit &F, double half_inv_var) {
  const int j = st.book_j;
  const double s = st.book_s, b = st.book_b, bn = b + s;
  bet[j] = bn;
  const double a2 = 2.0 * fabs(s), h = 0.5 * st.book_t;
  tru[j] = a2 > h ? a2 : h;
  if (s != 0.0) {
    st.bdx = fma(s, st.book_dx, st.bdx);
    if (st.book_pen && F.penalty == COX_PEN_L1) st.pen += F.lambda * (fabs(bn) - fabs(b));
    else if (st.book_pen && F.penalty == COX_PEN_L2) st.pen += (bn - b) * (bn + b) * half_inv_var;
  }
  st.book = 0;
}

// v at a position from eta (eq. parallel_d): FP64 exp split into a double-word, or the float
// exp of the compensated-FP32 precision; exits hold the negative. Raises COX_E_RANGE through
// serr when |eta - shift| leaves the range the double-word sums can hold.
template <class P>
static __device__ __forceinline__ dw inc_v(double eta, double shift, bool exitp, typename P::T *out, int *serr) {
  const double a = eta - shift;
  if (!(fabs(a) <= kIncRange)) atomicCAS(serr, 0, COX_E_RANGE);
  if constexpr (sizeof(typename P::T) == 8) {
    const double e = exitp ? -exp(a) : exp(a);
    *out = e;
    return dw_from(e);
  } else {
    const float e = exitp ? -expf(__double2float_rn(a)) : expf(__double2float_rn(a));
    *out = e;
    return dw_make(e);
  }
}

// Stage column j's entries in this tile (positions relative to lo, exit bit kept) with eta and v
// at them, using threads [th0, th0 + nth).
static __device__ void inc_load_list(const IncParams &prm, int t, int j, int lo, int npos, uint32_t *lp, dw *lv,
                                     double *le, int *cnt, int th0, int nth, int *serr, int cap) {
  const DevData &D = prm.D;
  const int C = prm.T;
  const int64_t cb = D.col_ptr[j];
  const int32_t *ct = prm.col_tile + int64_t(j) * (C + 1);
  const int64_t qa = cb + ct[t];
  int n = ct[t + 1] - ct[t];
  if (n > cap || n < 0) {   // the plan keeps every column within the cap
    if (int(threadIdx.x) == th0) atomicCAS(serr, 0, COX_E_INVALID);
    n = 0;
  }
#pragma unroll 1
  for (int m = int(threadIdx.x) - th0; m >= 0 && m < n; m += nth) {
    const uint32_t e = D.idx[qa + m];
    int q = int(e & kPosMask) - lo;
    if (q < 0 || q >= npos) {
      atomicCAS(serr, 0, COX_E_INVALID);
      q = 0;
    }
    lp[m] = uint32_t(q) | (e & kExitBit);
    lv[m] = prm.vdw[lo + q];
    le[m] = prm.F.eta[lo + q];
  }
  if (int(threadIdx.x) == th0) *cnt = n;
}

// inc_load_list for a column whose entry range in the tile (first entry qa, n entries) is known: the
// positions are stored at once, eta and v at them are copied asynchronously (cp.async; each thread
// waits for its own copies with cp_async_wait_all before the barrier that precedes their use).
static __device__ void inc_load_list_async(const IncParams &prm, int64_t qa, int n, int lo, int npos, uint32_t *lp,
                                           dw *lv, double *le, int *cnt, int th0, int nth, int *serr, int cap) {
  const DevData &D = prm.D;
  if (n > cap || n < 0) {
    if (int(threadIdx.x) == th0) atomicCAS(serr, 0, COX_E_INVALID);
    n = 0;
  }
#pragma unroll 1
  for (int m = int(threadIdx.x) - th0; m >= 0 && m < n; m += nth) {
    const uint32_t e = D.idx[qa + m];
    int q = int(e & kPosMask) - lo;
    if (q < 0 || q >= npos) {
      atomicCAS(serr, 0, COX_E_INVALID);
      q = 0;
    }
    lp[m] = uint32_t(q) | (e & kExitBit);
    cp_async8(&lv[m], &prm.vdw[lo + q]);
    cp_async8(&le[m], &prm.F.eta[lo + q]);
  }
  if (int(threadIdx.x) == th0) *cnt = n;
}

// Inclusive segmented suffix sum of one sequence held one element per thread (element k = thread
// k, k < nact; later elements are 0 and end their segments); f = 1 marks the last element of a
// segment. Warps past nact skip the arithmetic. Results go to out[k] for k < nact.
static __device__ void inc_seg_suffix1(dw x, int f, int nact, dw *out, dw (*s_agg)[32], int (*s_flg)[32]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool act = warp * 32 < nact;   // warp-uniform
  if (act) {
#pragma unroll 1
    for (int off = 1; off < 32; off <<= 1) {
      const dw y = dw_shfl_down(x, off);
      const int g = __shfl_down_sync(kFull, f, off);
      if (lane + off < 32) {
        if (!f) x = dw_add(x, y);
        f |= g;
      }
    }
  }
  if (lane == 0) {
    s_agg[0][warp] = act ? x : dw_make(0.0f);
    s_flg[0][warp] = act ? f : 1;
  }
  __syncthreads();
  const int nwa = (nact + 31) >> 5;
  if (warp == 0 && nwa > 1) {
    dw a = s_agg[0][lane];
    int h = s_flg[0][lane];
#pragma unroll 1
    for (int off = 1; off < nwa; off <<= 1) {
      const dw y = dw_shfl_down(a, off);
      const int g = __shfl_down_sync(kFull, h, off);
      if (lane + off < 32) {
        if (!h) a = dw_add(a, y);
        h |= g;
      }
    }
    dw c = dw_shfl_down(a, 1);
    if (lane == 31) c = dw_make(0.0f);
    s_agg[0][lane] = c;   // carry into warp `lane` from the later warps
  }
  __syncthreads();
  if (act) {
    if (nwa > 1 && !f) x = dw_add(x, s_agg[0][warp]);
    out[tid] = x;
  }
}

// The scan of the next step's column, run one step ahead by warps [kPsWarp0, 32) while thread 0
// computes the step. Two inclusive segmented suffix sums over the list's entries: of v (A)
// and of v at the entries that mfl marks (B: those the pending update will change); fend = 1 marks
// the last entry of a segment. After the update by e^dbeta - 1 = E at the marked entries, the
// suffix sums of v are A + E B. Each warp takes 64 consecutive entries (two per lane); the warps'
// aggregates meet in shared memory behind one named barrier of these warps only, which all of
// them reach whatever the list's length.
constexpr int kPsWarp0 = 16;
constexpr int kPsThreads = (32 - kPsWarp0) * 32;
constexpr int kPsBarrier = 1;   // named barrier id (0 is __syncthreads)
static_assert((32 - kPsWarp0) * 64 >= kIncThreads, "the pre-scan warps cover a full list");

static __device__ void inc_prescan(const dw *lv, const uint8_t *mfl, const uint8_t *fend, int n, dw *ua, dw *ub,
                                   dw (*s_agg)[32], int (*s_flg)[32]) {
  const int lane = threadIdx.x & 31, c = (int(threadIdx.x) >> 5) - kPsWarp0;   // this warp's chunk
  const int e0 = 64 * c + 2 * lane, e1 = e0 + 1;
  const int nch = (n + 63) >> 6;
  dw a1 = dw_make(0.0f), b1 = dw_make(0.0f), xa = dw_make(0.0f), xb = dw_make(0.0f);
  int f1 = 1, fl = 1;
  if (c < nch) {   // warp-uniform
    dw a0 = dw_make(0.0f), b0 = dw_make(0.0f);
    int f0 = 1;
    if (e0 < n) {
      a0 = lv[e0];
      b0 = mfl[e0] ? a0 : dw_make(0.0f);
      f0 = int(fend[e0]);
    }
    if (e1 < n) {
      a1 = lv[e1];
      b1 = mfl[e1] ? a1 : dw_make(0.0f);
      f1 = int(fend[e1]);
    }
    // the lane's pair from e0 to its segment end within the pair, then across the warp's lanes
    xa = f0 ? a0 : dw_add(a0, a1);
    xb = f0 ? b0 : dw_add(b0, b1);
    fl = f0 | f1;
#pragma unroll 1
    for (int off = 1; off < 32; off <<= 1) {
      const dw ya = dw_shfl_down(xa, off), yb = dw_shfl_down(xb, off);
      const int g = __shfl_down_sync(kFull, fl, off);
      if (lane + off < 32) {
        if (!fl) {
          xa = dw_add(xa, ya);
          xb = dw_add(xb, yb);
        }
        fl |= g;
      }
    }
    if (lane == 0) {
      s_agg[0][c] = xa;
      s_agg[1][c] = xb;
      s_flg[0][c] = fl;
    }
  }
  __syncwarp();
  asm volatile("bar.sync %0, %1;" ::"n"(kPsBarrier), "n"(kPsThreads) : "memory");
  if (c < nch) {
    // carry into this chunk: the later chunks' sums up to the first one that ends a segment
    dw za = lane < nch ? s_agg[0][lane] : dw_make(0.0f), zb = lane < nch ? s_agg[1][lane] : dw_make(0.0f);
    int h = lane < nch ? s_flg[0][lane] : 1;
#pragma unroll 1
    for (int off = 1; off < 32; off <<= 1) {
      const dw ya = dw_shfl_down(za, off), yb = dw_shfl_down(zb, off);
      const int g = __shfl_down_sync(kFull, h, off);
      if (lane + off < 32) {
        if (!h) {
          za = dw_add(za, ya);
          zb = dw_add(zb, yb);
        }
        h |= g;
      }
    }
    dw ca = dw_shfl(za, c + 1), cb = dw_shfl(zb, c + 1);   // c + 1 <= 16
    if (c + 1 >= nch) ca = cb = dw_make(0.0f);
    // e1: its own value plus, when its segment goes on, the next lane's sum
    const dw na = dw_shfl_down(xa, 1), nb = dw_shfl_down(xb, 1);
    const int nf = __shfl_down_sync(kFull, fl, 1);
    dw sa1 = a1, sb1 = b1;
    bool open1 = !f1;   // e1's segment reaches the chunk's end
    if (!f1 && lane < 31) {
      sa1 = dw_add(a1, na);
      sb1 = dw_add(b1, nb);
      open1 = !nf;
    }
    if (!fl) {
      xa = dw_add(xa, ca);
      xb = dw_add(xb, cb);
    }
    if (open1) {
      sa1 = dw_add(sa1, ca);
      sb1 = dw_add(sb1, cb);
    }
    if (e0 < n) {
      ua[e0] = xa;
      ub[e0] = xb;
    }
    if (e1 < n) {
      ua[e1] = sa1;
      ub[e1] = sb1;
    }
  }
}

// The rebuild: v recomputed from eta at every position of the tile (written to vdw and to the
// fit's v), then a dense segmented suffix of v: every tie group's in-tile S0 (before the carry
// from the later tiles) into gs0, and the tile's head aggregate (sum from its first position to
// its first stratum end), returned in warp 0.
template <class P>
static __device__ dw inc_dense(const IncParams &prm, int lo, int npos, const uint32_t *cutb, const uint32_t *headb,
                               const int32_t *headp, dw *gs0, uint8_t *gseen, dw *s_wagg, int *s_wflag, dw *s_wk, int RW,
                               int *serr) {
  using T = typename P::T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ws = warp * RW, we = min(ws + RW, npos);
  const double *etat = prm.F.eta + lo;
  T *vt = static_cast<T *>(prm.F.v) + lo;
  dw *vd = prm.vdw + lo;
  const uint32_t *exitb = prm.D.exit_bits;
  const double shift = prm.F.shift;
  dw carry = dw_make(0.0f);
  int seen = 0;
  if (ws < we) {
    const int top = ws + ((we - ws - 1) >> 5) * 32;
    for (int b = top; b >= ws; b -= 128) {
      dw xs[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int bb = b - 32 * u, p = bb + lane;
        xs[u] = dw_make(0.0f);
        if (bb >= ws && p < we) {
          const int g = lo + p;
          const bool ex = exitb != nullptr && ((exitb[g >> 5] >> (g & 31)) & 1u);
          T vv;
          xs[u] = inc_v<P>(etat[p], shift, ex, &vv, serr);
          vt[p] = vv;
          vd[p] = xs[u];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int bb = b - 32 * u;
        if (bb < ws) break;
        const int p = bb + lane;
        const bool in = p < we;
        const uint32_t cw = cutb[bb >> 5], hw = headb[bb >> 5];
        dw x = xs[u];
        int f = in ? int((cw >> lane) & 1u) : 0;
#pragma unroll 1
        for (int off = 1; off < 32; off <<= 1) {
          const dw y = dw_shfl_down(x, off);
          const int g = __shfl_down_sync(kFull, f, off);
          if (lane + off < 32) {
            if (!f) x = dw_add(x, y);
            f |= g;
          }
        }
        if (!f) x = dw_add(x, carry);
        if (in && ((hw >> lane) & 1u)) {
          const int h = headp[bb >> 5] + __popc(hw & ((1u << lane) - 1u));
          gs0[h] = x;
          gseen[h] = uint8_t(f | seen);
        }
        carry = dw_shfl(x, 0);
        seen |= __shfl_sync(kFull, f, 0);
      }
    }
  }
  if (lane == 0) {
    s_wagg[warp] = carry;
    s_wflag[warp] = seen;
  }
  __syncthreads();
  dw head = dw_make(0.0f);
  if (warp == 0) {
    dw a = s_wagg[lane];
    int h = s_wflag[lane];
#pragma unroll 1
    for (int off = 1; off < 32; off <<= 1) {
      const dw y = dw_shfl_down(a, off);
      const int g = __shfl_down_sync(kFull, h, off);
      if (lane + off < 32) {
        if (!h) a = dw_add(a, y);
        h |= g;
      }
    }
    dw c = dw_shfl_down(a, 1);
    if (lane == 31) c = dw_make(0.0f);
    s_wk[lane] = c;
    head = dw_shfl(a, 0);
  }
  __syncthreads();
  return head;
}

template <class P, class Cfg, bool kTrace>
static __device__ __forceinline__ void incr_body(const IncParams &prm, const int t) {
  using T = typename P::T;
  using S = IncSmem<Cfg>;
  constexpr int LC = Cfg::kListCap;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *lpos = reinterpret_cast<uint32_t *>(smem + S::o_lpos);
  dw *lv = reinterpret_cast<dw *>(smem + S::o_lv);
  double *le = reinterpret_cast<double *>(smem + S::o_le);
  dw *ua = reinterpret_cast<dw *>(smem + S::o_ua);
  dw *ub = reinterpret_cast<dw *>(smem + S::o_ub);
  uint32_t *cutb = reinterpret_cast<uint32_t *>(smem + S::o_cutb);
  int32_t *cutp = reinterpret_cast<int32_t *>(smem + S::o_cutp);
  uint32_t *headb = reinterpret_cast<uint32_t *>(smem + S::o_headb);
  int32_t *headp = reinterpret_cast<int32_t *>(smem + S::o_headp);
  dw *gs0 = reinterpret_cast<dw *>(smem + S::o_gs0);
  dw *s1p = gs0;   // outside a rebuild: each group's S1 of the last step
  uint8_t *gseen = reinterpret_cast<uint8_t *>(smem + S::o_gseen);
  uint64_t *srec = reinterpret_cast<uint64_t *>(smem + S::o_rec);
  dw *sref = reinterpret_cast<dw *>(smem + S::o_rref);
  GroupSlot *grp = reinterpret_cast<GroupSlot *>(smem + S::o_grp);
  uint32_t *pmask = reinterpret_cast<uint32_t *>(smem + S::o_pmask);
  uint32_t *cmask = reinterpret_cast<uint32_t *>(smem + S::o_cmask);
  uint16_t *kg = reinterpret_cast<uint16_t *>(smem + S::o_kg);   // [gcap]
  dw *ginv = reinterpret_cast<dw *>(smem + S::o_ginv);            // [gcap], one group per thread only
  uint8_t *fce = smem + S::o_fce;                                 // [cap]
  uint8_t *mfl = smem + S::o_mfl;                                 // [cap] next-list entries in the current column

  __shared__ IncState st;
  __shared__ int s_cnt[4];
  __shared__ dw s_agg[2][32];
  __shared__ int s_flg[2][32];
  __shared__ dw s_red[4][32];
  __shared__ double s_rll[32];
  __shared__ dw s_Gq[2][4];   // G1, G2 over quarters of the CTAs
  __shared__ double s_LL;
  __shared__ dw s_chain[3];    // chain sums of the previous step's H1, R, I
  __shared__ dw s_carry[2];    // rebuild: carries of S0 and S1 from the later tiles
  __shared__ dw s_dagg[32], s_dcar[32];   // dense scan: warp aggregates, carries into warps
  __shared__ int s_dflg[32];
  __shared__ int s_chain_end, s_bad, s_err, s_anyerr;
  __shared__ int s_cut0;   // first stratum end in the tile (npos: none): positions up to it are the head segment
  __shared__ int s_ce[kIncMaxCtas];   // chain end of every CTA of the fit
  __shared__ uint64_t s_pay[kIncRec];   // this CTA's record payloads (bits): G1, G2, LL, H1, R, I
  __shared__ double s_half_inv_var;
  __shared__ dw s_inv_var_dw, s_lambda_dw;
  __shared__ IncPre s_pre;
  // the entry range in this tile of the column two steps ahead, fetched a step before its list:
  // its first entry (col_ptr), the column's tile offsets (col_tile [t], [t + 1]), halt flag
  __shared__ int64_t s_nbq[2];
  __shared__ int32_t s_nbt[2][2];
  __shared__ int32_t s_nbh[2];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const DevFit &F = prm.F;
  const DevData &D = prm.D;
  FitCtl *ctl = F.ctl;
  const int C = prm.T;
  const int lo = prm.tile_lo[t], hi = prm.tile_lo[t + 1], npos = hi - lo;
  const int ga = prm.tile_g[t], ng = prm.tile_g[t + 1] - ga;
  const int kc0 = prm.tile_k[t], nc = prm.tile_k[t + 1] - kc0;
  const double shift = F.shift;
  const int p = D.p;
  double *bet = prm.bcopy + size_t(t) * 2 * size_t(p);   // this CTA's copy of beta and trust
  double *tru = bet + p;

  // ---- one-time set-up: stratum ends and read positions as bitmasks, group slots, lists
  if (tid == 0) {
    s_cut0 = nc > 0 ? D.cut_pos[kc0] - lo : npos;
    s_bad = (npos > Cfg::kPosCap || ng > Cfg::kGroupCap || C > kIncMaxCtas || npos <= 0 || ng < 0) ? 1 : 0;
    s_err = 0;
  }
  __syncthreads();
  if (s_bad) {   // the plan never builds such a tile
    if (tid == 0) atomicCAS(&ctl->error, 0, COX_E_INVALID);
    return;
  }
  const int nw = (npos + 31) >> 5;
#pragma unroll 1
  for (int w = tid; w < nw; w += kIncThreads) { cutb[w] = 0u; headb[w] = 0u; pmask[w] = 0u; cmask[w] = 0u; }
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
    st.E = st.pend_j >= 0 ? dw_from(expm1(st.pend_db)) : dw_make(0.0f);
    st.halt = 0;
    s_half_inv_var = 0.5 / F.l2_var;
    s_inv_var_dw = dw_from(1.0 / F.l2_var);
    s_lambda_dw = dw_from(F.lambda);
    st.book = 0;
  }
#pragma unroll 1
  for (int jj = tid; jj < p; jj += kIncThreads) {
    bet[jj] = F.beta[jj];
    tru[jj] = F.trust[jj];
  }
  __syncthreads();
#pragma unroll 1
  for (int gi = tid; gi < ng; gi += kIncThreads) {
    int qg = D.head_pos[ga + gi] - lo;
    if (qg < 0 || qg >= npos) {
      atomicCAS(&s_err, 0, COX_E_INVALID);
      qg = 0;
    }
    grp[gi].q = qg;
    grp[gi].d = float(D.head_d[ga + gi]);   // events of the group (exact in float below 2^24)
    grp[gi].S0 = dw_make(0.0f);
    atomicOr(&headb[qg >> 5], 1u << (qg & 31));
  }
#pragma unroll 1
  for (int k = tid; k < nc; k += kIncThreads) {
    int q = D.cut_pos[kc0 + k] - lo;
    if (q < 0 || q >= npos) {
      atomicCAS(&s_err, 0, COX_E_INVALID);
      q = 0;
    }
    atomicOr(&cutb[q >> 5], 1u << (q & 31));
  }
  {   // beta'dX and the penalty at the starting coefficients (same order in every CTA)
    double ex[2] = {0.0, 0.0};
#pragma unroll 1
    for (int jj = tid; jj < p; jj += kIncThreads) {
      const double b = F.beta[jj];
      ex[0] += b * D.dX[jj];
      ex[1] += inc_penalty(F, jj, b);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll 1
      for (int off = 16; off > 0; off >>= 1) ex[i] += __shfl_down_sync(kFull, ex[i], off);
    if (lane == 0) { s_rll[warp] = ex[0]; s_red[0][warp] = dw_from(ex[1]); }
  }
  __syncthreads();
  if (warp == 0) {
    double a = s_rll[lane], b = dw_to(s_red[0][lane]);
#pragma unroll 1
    for (int off = 16; off > 0; off >>= 1) {
      a += __shfl_down_sync(kFull, a, off);
      b += __shfl_down_sync(kFull, b, off);
    }
    if (lane == 0) { st.bdx = a; st.pen = b; }
  } else if (warp == 1 || warp == 2) {   // prefix counts of the two bitmasks
    const uint32_t *bits = warp == 1 ? cutb : headb;
    int32_t *pre = warp == 1 ? cutp : headp;
    int run = 0;
#pragma unroll 1
    for (int base = 0; base < nw; base += 32) {
      const int c = base + lane < nw ? __popc(bits[base + lane]) : 0;
      int incl = c;
#pragma unroll 1
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += y;
      }
      if (base + lane < nw) pre[base + lane] = run + incl - c;
      run += __shfl_sync(kFull, incl, 31);
    }
  } else if (tid == 96) {
    // the later tiles whose head segments continue this tile's last stratum: up to and including
    // the first tile that holds a stratum end (none when this tile's last position ends one)
    const bool last_cut = nc > 0 && D.cut_pos[kc0 + nc - 1] == hi - 1;
    int e = t;
    if (!last_cut)
#pragma unroll 1
      for (int c = t + 1; c < C; ++c) {
        e = c;
        if (prm.tile_k[c + 1] > prm.tile_k[c]) break;
      }
    s_chain_end = e;
  }
  // chain end of CTA tid (thread tid pushes this CTA's record into CTA tid's inbox: the head sums
  // H1, R, I go only to CTAs whose last stratum continues into this tile)
  if (tid < C) {
    const int k1 = prm.tile_k[tid + 1];
    const bool lc = k1 > prm.tile_k[tid] && D.cut_pos[k1 - 1] == prm.tile_lo[tid + 1] - 1;
    int ce = tid;
    if (!lc)
#pragma unroll 1
      for (int c = tid + 1; c < C; ++c) {
        ce = c;
        if (prm.tile_k[c + 1] > prm.tile_k[c]) break;
      }
    s_ce[tid] = ce;
  }
  __syncthreads();
#pragma unroll 1
  for (int gi = tid; gi < ng; gi += kIncThreads) {
    const int seg = inc_rank(cutb, cutp, grp[gi].q);
    grp[gi].seg = seg;
    grp[gi].tail = seg == nc;
  }
  const int RW = max(32, ((npos + 1023) / 1024) * 32);   // positions per warp in the dense scan
  const double half_inv_var = s_half_inv_var;
  // list slots: previous column (pending update), current, next, and the one being fetched
  int base = 0;
  if (st.state == kRunning) {
    if (st.pend_j >= 0)
      inc_load_list(prm, t, st.pend_j, lo, npos, lpos, lv, le, &s_cnt[0], 0, kIncThreads, &s_err, LC);
    else if (tid == 0)
      s_cnt[0] = 0;
    const int j1 = st.j, j2 = st.j + 1 >= p ? 0 : st.j + 1;
    inc_load_list(prm, t, j1, lo, npos, lpos + LC, lv + LC, le + LC, &s_cnt[1], 0, kIncThreads, &s_err, LC);
    if (prm.halt && prm.halt[j2]) {   // the launch ends before it
      if (tid == 0) s_cnt[2] = 0;
    } else {
      inc_load_list(prm, t, j2, lo, npos, lpos + 2 * LC, lv + 2 * LC, le + 2 * LC, &s_cnt[2], 0, kIncThreads, &s_err,
                    LC);
    }
  }
  if (tid == 0 && st.state == kRunning) {   // the range of the column the first step fetches
    const int jf0 = (st.j + 2) % p;
    s_nbq[0] = D.col_ptr[jf0];
    s_nbt[0][0] = prm.col_tile[int64_t(jf0) * (C + 1) + t];
    s_nbt[0][1] = prm.col_tile[int64_t(jf0) * (C + 1) + t + 1];
    s_nbh[0] = prm.halt ? prm.halt[jf0] : 0;
  }
  __syncthreads();
  if (st.state == kRunning) {   // the first column's lookups (later ones are built a step ahead)
    if (Cfg::kGpt == 1 && tid < ng) kg[tid] = inc_first_entry(lpos + LC, s_cnt[1], grp[tid].q, grp[tid].seg, cutb, cutp);
    if (tid < s_cnt[1]) fce[tid] = inc_seg_end(lpos + LC, s_cnt[1], tid, cutb, cutp);
  }
  __syncthreads();
  bool refreshed = false;  // the last step taken rebuilt v from eta

  for (int64_t step = 0; step < prm.max_steps && st.state == kRunning && !st.halt; ++step) {
    const int j = st.j, pj = st.pend_j;
    const double db = st.pend_db;
    const bool need_ll = st.need_ll != 0;
    const bool refresh = need_ll || step == 0;
    const uint32_t epoch = st.epoch;
    const int sp = base & 3, sc = (base + 1) & 3, sn = (base + 2) & 3, sf = (base + 3) & 3;
    uint32_t *lp_p = lpos + sp * LC, *lp_c = lpos + sc * LC, *lp_n = lpos + sn * LC;
    dw *lv_p = lv + sp * LC, *lv_c = lv + sc * LC, *lv_n = lv + sn * LC;
    double *le_p = le + sp * LC, *le_c = le + sc * LC, *le_n = le + sn * LC;
    const int np = pj >= 0 ? s_cnt[sp] : 0, ncur = s_cnt[sc], nnx = s_cnt[sn];
    uint64_t *trace =
        (kTrace && prm.trace && step < prm.trace_steps && tid == 0) ? prm.trace + (step * C + t) * kIncTraceSlots : nullptr;
    if (trace) { trace[0] = uint64_t(clock64()); trace[21] = inc_timer(); }
    if (tid == 0) s_anyerr = 0;
    // ---- 1. the pending update at the previous column's entries (one per thread):
    //         eta += dbeta (eq. parallel_xb); v (1 + (e^dbeta - 1)) (eq. parallel_d)
    if (tid < np) {
      const uint32_t e = lp_p[tid];
      const int q = int(e & kPosMask);
      const double et = __dadd_rn(le_p[tid], db);
      if (!(fabs(et - shift) <= kIncRange)) atomicCAS(&s_err, 0, COX_E_RANGE);
      const dw nv = dw_add(lv_p[tid], dw_mul(lv_p[tid], st.E));
      atomicOr(&pmask[q >> 5], 1u << (q & 31));
      prm.vdw[lo + q] = nv;
      F.eta[lo + q] = et;
      le_p[tid] = et;
      lv_p[tid] = nv;
    }
    __syncthreads();
    if (trace) trace[1] = uint64_t(clock64());
    // ---- 2. a sweep start rebuilds v and S0 from eta; otherwise the current and next lists
    //         take the update at the entries they share with the previous column
    dw HA0 = dw_make(0.0f);
    if (refresh) {
      HA0 = inc_dense<P>(prm, lo, npos, cutb, headb, headp, gs0, gseen, s_dagg, s_dflg, s_dcar, RW, &s_err);
      if (tid < ncur) {
        const int q = int(lp_c[tid] & kPosMask);
        lv_c[tid] = prm.vdw[lo + q];
        le_c[tid] = F.eta[lo + q];
      }
      if (tid < nnx) {
        const int q = int(lp_n[tid] & kPosMask);
        lv_n[tid] = prm.vdw[lo + q];
        le_n[tid] = F.eta[lo + q];
      }
    } else if (np > 0) {
      // an entry at a position of the previous column takes the same update (the copies of v
      // and eta in every list agree, so the result is the previous list's to the bit)
      if (tid < ncur) {
        const int q = int(lp_c[tid] & kPosMask);
        if ((pmask[q >> 5] >> (q & 31)) & 1u) {
          lv_c[tid] = dw_add(lv_c[tid], dw_mul(lv_c[tid], st.E));
          le_c[tid] = __dadd_rn(le_c[tid], db);
        }
      }
      if (tid < nnx) {
        const int q = int(lp_n[tid] & kPosMask);
        if ((pmask[q >> 5] >> (q & 31)) & 1u) {
          lv_n[tid] = dw_add(lv_n[tid], dw_mul(lv_n[tid], st.E));
          le_n[tid] = __dadd_rn(le_n[tid], db);
        }
      }
    }
    refreshed = refresh;
    if (tid < ncur) {
      const int q = int(lp_c[tid] & kPosMask);
      atomicOr(&cmask[q >> 5], 1u << (q & 31));
    }
    // ---- 3. suffix sums of v over the current column: after a rebuild a segmented scan of the
    //         reloaded list (into A, B unused); otherwise A + E B from the scan run one step ahead
    //         (binary X: the pending update multiplies v by e^dbeta at the previous column's
    //         entries). The previous step's S1 per group, times E, is the change of S0.
    if (trace) trace[2] = uint64_t(clock64());
    if (refresh) {
      dw x1 = dw_make(0.0f);
      int fc = 1;
      if (tid < ncur) {
        x1 = lv_c[tid];
        fc = int(fce[tid]);
      }
      inc_seg_suffix1(x1, fc, ncur, ua, s_agg, s_flg);
    }
    if (trace) trace[3] = uint64_t(clock64());
    __syncthreads();
    if (tid < np) {   // the marks of the previous column are read; clear them for the next step
      const int q = int(lp_p[tid] & kPosMask);
      atomicAnd(&pmask[q >> 5], ~(1u << (q & 31)));
    }
    const dw Es = refresh ? dw_make(0.0f) : st.E;
    auto s1_at = [&](int k) { return refresh ? ua[k] : dw_add(ua[k], dw_mul(Es, ub[k])); };
    // head-segment sum of column j's v in this tile (what the earlier tiles of the stratum need)
    auto head1 = [&]() { return (ncur > 0 && inc_rank(cutb, cutp, int(lp_c[0] & kPosMask)) == 0) ? s1_at(0) : dw_make(0.0f); };
    if (trace) trace[4] = uint64_t(clock64());
    dw C1;
    if (refresh) {
      // ---- carries of the rebuilt S0 and of S1 from one exchange of the tiles' head sums
      const uint32_t tag = epoch;
      if (tid == 0) {
        uint64_t *w = prm.tref + 4 * int64_t(t);
        put_dw(w, tag, HA0);
        put_dw(w + 2, tag, head1());
      }
      if (tid < C) {
        uint64_t r[2] = {0, 0};
        if (!wait_tagged<2>(prm.tref + 4 * int64_t(tid), tag, r, &ctl->error, prm.spin)) {
          atomicCAS(&s_err, 0, COX_E_TIMEOUT);
          r[0] = r[1] = 0;
        }
        sref[2 * tid] = slot_dw(&r[0]);
        sref[2 * tid + 1] = slot_dw(&r[1]);
      }
      __syncthreads();
      if (warp < 2) {
        dw c0 = dw_make(0.0f);
#pragma unroll 1
        for (int c = t + 1 + lane; c <= s_chain_end; c += 32) c0 = dw_add(c0, sref[2 * c + warp]);
#pragma unroll 1
        for (int off = 16; off > 0; off >>= 1) c0 = dw_add(c0, dw_shfl_down(c0, off));
        if (lane == 0) s_carry[warp] = c0;
      }
      __syncthreads();
#pragma unroll 1
      for (int gi = tid; gi < ng; gi += kIncThreads) {
        dw S0 = gs0[gi];
        if (!gseen[gi]) S0 = dw_add(S0, s_dcar[grp[gi].q / RW]);
        if (grp[gi].tail) S0 = dw_add(S0, s_carry[0]);
        grp[gi].S0 = S0;
        if (Cfg::kGpt == 1) ginv[gi] = dw_div(dw_make(1.0f), S0);
      }
      C1 = s_carry[1];
    } else {
      // ---- S0 += the suffix of dD from the read position, and the later tiles' change
#pragma unroll
      for (int i = 0; i < Cfg::kGpt; ++i) {
        const int gi = tid + i * kIncThreads;
        if (gi < ng) {
          dw S0 = grp[gi].S0;
          bool upd = false;
          if (np > 0) {
            const dw sp1 = s1p[gi];
            if (!dw_is_zero(sp1)) {
              S0 = dw_add(S0, dw_mul(st.E, sp1));
              upd = true;
            }
          }
          if (grp[gi].tail && !dw_is_zero(st.E)) {
            S0 = dw_add(S0, dw_mul(st.E, s_chain[0]));
            upd = true;
          }
          if (upd) {
            grp[gi].S0 = S0;
            if (Cfg::kGpt == 1) ginv[gi] = dw_div(dw_make(1.0f), S0);
          }
        }
      }
      C1 = dw_add(s_chain[1], dw_mul(st.E, s_chain[2]));
    }
    if (trace) trace[5] = uint64_t(clock64());
    // ---- 4. tie-group ratios (warps holding groups); the next column's head-segment sums R,
    //         and I over the entries this step's update may change (warps holding its entries)
    const bool gwarp = warp * 32 < ng, nwarp = warp * 32 < nnx;   // warp-uniform
    dw r_g1 = dw_make(0.0f), r_g2 = dw_make(0.0f), r_R = dw_make(0.0f), r_I = dw_make(0.0f);
    double r_ll = 0.0;
    if (gwarp) {
#pragma unroll
      for (int i = 0; i < Cfg::kGpt; ++i) {
        const int gi = tid + i * kIncThreads;
        if (gi < ng) {
          const GroupSlot g = grp[gi];
          dw s1 = dw_make(0.0f);
          if (ncur > 0) {
            const int k = Cfg::kGpt == 1 ? int(kg[gi]) : int(inc_first_entry(lp_c, ncur, g.q, g.seg, cutb, cutp));
            if (k != kNoEntry) s1 = s1_at(k);
          }
          s1p[gi] = s1;
          if (g.tail) s1 = dw_add(s1, C1);
          if (!dw_is_zero(s1)) {
            const dw r = Cfg::kGpt == 1 ? dw_mul(s1, ginv[gi]) : dw_div(s1, g.S0);
            const dw a1 = dw_mul_f(r, g.d);
            const dw a2 = dw_mul(a1, dw_sub(dw_make(1.0f), r));
            if (Cfg::kGpt == 1) {
              r_g1 = a1;
              r_g2 = a2;
            } else {
              r_g1 = dw_add_same(r_g1, a1);
              r_g2 = dw_add_same(r_g2, a2);
            }
          }
          if (need_ll) r_ll += double(g.d) * log(dw_to(g.S0));
        }
      }
      if (trace) trace[6] = uint64_t(clock64());
#pragma unroll 1
      for (int off = 16; off > 0; off >>= 1) {
        r_g1 = dw_add_same(r_g1, dw_shfl_down(r_g1, off));
        r_g2 = dw_add_same(r_g2, dw_shfl_down(r_g2, off));
      }
      if (need_ll)
#pragma unroll 1
        for (int off = 16; off > 0; off >>= 1) r_ll += __shfl_down_sync(kFull, r_ll, off);
    }
    if (trace && !gwarp) trace[6] = uint64_t(clock64());
    if (nwarp) {
      const int qnx = tid < nnx ? int(lp_n[tid] & kPosMask) : 0;
      const bool inj = tid < nnx && ((cmask[qnx >> 5] >> (qnx & 31)) & 1u);
      if (tid < nnx) mfl[tid] = uint8_t(inj);
      if (tid < nnx && qnx <= s_cut0) {
        const dw vnx = lv_n[tid];
        r_R = vnx;
        if (inj) r_I = vnx;
      }
      if (__any_sync(kFull, !dw_is_zero(r_R))) {
#pragma unroll 1
        for (int off = 16; off > 0; off >>= 1) {
          r_R = dw_add(r_R, dw_shfl_down(r_R, off));
          r_I = dw_add(r_I, dw_shfl_down(r_I, off));
        }
      }
    }
    if (lane == 0) {
      s_red[0][warp] = r_g1;
      s_red[1][warp] = r_g2;
      s_red[2][warp] = r_R;
      s_red[3][warp] = r_I;
      s_rll[warp] = r_ll;
    }
    if (trace) trace[7] = uint64_t(clock64());
    __syncthreads();
    if (trace) trace[8] = uint64_t(clock64());
    if (tid < ncur) {   // the marks of the current column are read; clear them for the next step
      const int q = int(lp_c[tid] & kPosMask);
      atomicAnd(&cmask[q >> 5], ~(1u << (q & 31)));
    }
    // ---- one value per warp: sums of the warp partials (G1, G2, R, I as double-words, LL in
    //      FP64), then this CTA's record, pushed into every CTA's inbox by thread r for reader r:
    //      (G1, G2[, LL]) to every CTA, and (H1, R, I) as well to the CTAs whose chain holds this tile
    const int par = int(epoch & 1u);
    if (warp < 2 || warp == 3 || warp == 4) {
      const int v = warp < 2 ? warp : warp - 1;           // s_red row: G1, G2, R, I
      const int nv = warp < 2 ? min((ng + 31) >> 5, 32) : (nnx + 31) >> 5;
      dw a = lane < nv ? s_red[v][lane] : dw_make(0.0f);
      if (warp < 2)
#pragma unroll 1
        for (int off = 1; off < nv; off <<= 1) a = dw_add_same(a, dw_shfl_down(a, off));
      else
#pragma unroll 1
        for (int off = 1; off < nv; off <<= 1) a = dw_add(a, dw_shfl_down(a, off));
      if (lane == 0) s_pay[warp < 2 ? warp : warp + 1] = *reinterpret_cast<const uint64_t *>(&a);   // 0 G1, 1 G2, 4 R, 5 I
      if (trace) trace[9] = uint64_t(clock64());
    } else if (warp == 2) {
      const int nv = min((ng + 31) >> 5, 32);
      double a = (need_ll && lane < nv) ? s_rll[lane] : 0.0;
      if (need_ll)
#pragma unroll 1
        for (int off = 1; off < nv; off <<= 1) a += __shfl_down_sync(kFull, a, off);
      if (lane == 0) s_pay[2] = uint64_t(__double_as_longlong(a));
    } else if (tid == 5 * 32) {
      const dw H1 = head1();
      s_pay[3] = *reinterpret_cast<const uint64_t *>(&H1);
    }
    __syncthreads();
    if (trace) trace[10] = uint64_t(clock64());
    const int nbase = need_ll ? 3 : 2;   // payloads every CTA gets
    const uint32_t tag = (epoch & ~kTagErr) | (s_err ? kTagErr : 0u);
    if (trace) trace[19] = inc_timer();   // global time of the push (cross-CTA comparison)
    if (tid < C) {
      uint64_t *w = prm.trec + int64_t(kIncRecWords) * ((int64_t(par) * C + tid) * C + t);
      const int nw_ = (tid < t && s_ce[tid] >= t) ? kIncRec : nbase;
#pragma unroll 1
      for (int i = 0; i < nw_; ++i) {
        const uint64_t v = s_pay[i];
        st_rlx_v2(w + 2 * i, (uint64_t(tag) << 32) | (v & 0xffffffffull), (uint64_t(tag) << 32) | (v >> 32));
      }
    }
    if (tid == 0 && s_err) atomicCAS(&ctl->error, 0, s_err);
    if (trace) trace[11] = uint64_t(clock64());
    // ---- 5. the inbox: one thread per writer; meanwhile the other threads fetch column j+2's
    //         entries (its range fetched a step ago) with eta and v as of this step's update,
    //         copied asynchronously: the barrier after the inbox waits for no memory round trip
    //         but the records'
    if (tid < C) {
      uint64_t r[kIncRec];
      unsigned polls = 0;
      const int nr = (tid > t && tid <= s_chain_end) ? kIncRec : nbase;
      const int got = wait_record<kIncRec>(prm.trec + int64_t(kIncRecWords) * ((int64_t(par) * C + t) * C + tid), nr,
                                           epoch & ~kTagErr, r, &ctl->error, prm.spin, &polls);
      if (trace) trace[20] = polls;
      if (got != 1) {
        for (int i = 0; i < kIncRec; ++i) r[i] = 0;
        atomicCAS(&s_anyerr, 0, got == 0 ? COX_E_TIMEOUT : 1);
      }
      for (int i = 0; i < nr; ++i) srec[i * kIncMaxCtas + tid] = r[i];
      if (trace) trace[12] = uint64_t(clock64());
    } else {
      if (tid == kIncThreads - 1) {
        // while the records travel: the previous step's coefficient bookkeeping, then this
        // coordinate's inputs to the step, converted for the double-word step rule
        if (st.book) inc_book(st, bet, tru, F, half_inv_var);
        IncPre q;
        q.dx = D.dX[j];
        q.b = bet[j];
        q.t = tru[j];
        q.pen = F.penalize ? F.penalize[j] != 0 : 1;
        q.halt_next = prm.halt ? prm.halt[j + 1 >= p ? 0 : j + 1] : 0;
        q.dxw = dw_from(q.dx);
        q.bw = dw_from(q.b);
        q.tw = dw_from(q.t);
        s_pre = q;
      }
      {   // the next column's first entries per group and segment ends, for its step (this
          // step's own were read before the exchange)
        if (Cfg::kGpt == 1)
#pragma unroll 1
          for (int gi = tid - C; gi < ng; gi += kIncThreads - C)
            kg[gi] = inc_first_entry(lp_n, nnx, grp[gi].q, grp[gi].seg, cutb, cutp);
#pragma unroll 1
        for (int k = tid - C; k < nnx; k += kIncThreads - C) fce[k] = inc_seg_end(lp_n, nnx, k, cutb, cutp);
      }
      const int nb = base & 1;
      if (tid == kIncThreads - 2) {   // the range of the column the next step fetches (j + 3)
        const int jn3 = (j + 3) % p;
        cp_async8(&s_nbq[nb ^ 1], D.col_ptr + jn3);
        cp_async4(&s_nbt[nb ^ 1][0], prm.col_tile + int64_t(jn3) * (C + 1) + t);
        cp_async4(&s_nbt[nb ^ 1][1], prm.col_tile + int64_t(jn3) * (C + 1) + t + 1);
        s_nbh[nb ^ 1] = prm.halt ? prm.halt[jn3] : 0;
      }
      if (s_nbh[nb]) {   // the launch ends before it
        if (tid == C) s_cnt[sf] = 0;
      } else {
        inc_load_list_async(prm, s_nbq[nb] + s_nbt[nb][0], s_nbt[nb][1] - s_nbt[nb][0], lo, npos, lpos + sf * LC,
                            lv + sf * LC, le + sf * LC, &s_cnt[sf], C, kIncThreads - C, &s_err, LC);
      }
    }
    __syncthreads();
    if (trace) trace[13] = uint64_t(clock64());
    // ---- 6. fixed-order reductions: G1 and G2 over every CTA by four warps each (quarters of the
    //         CTAs, combined by the step), LL when evaluated; H1, R, I over the later tiles this
    //         tile's last stratum continues into, one warp each
    if (warp < 8) {
      const int v = warp >> 2, qtr = warp & 3;   // payload 0 G1 / 1 G2, quarter of the CTAs
      const int c0 = (C * qtr) >> 2, c1 = (C * (qtr + 1)) >> 2;
      dw a = dw_make(0.0f);
#pragma unroll 1
      for (int c = c0 + lane; c < c1; c += 32) a = dw_add_same(a, slot_dw(&srec[v * kIncMaxCtas + c]));
#pragma unroll 1
      for (int off = 16; off > 0; off >>= 1) a = dw_add_same(a, dw_shfl_down(a, off));
      if (lane == 0) s_Gq[v][qtr] = a;
      if (trace) trace[16] = uint64_t(clock64());
    } else if (warp < 11) {
      const int v = warp - 5;   // payload 3 H1, 4 R, 5 I
      dw a = dw_make(0.0f);
#pragma unroll 1
      for (int c = t + 1 + lane; c <= s_chain_end; c += 32) a = dw_add(a, slot_dw(&srec[v * kIncMaxCtas + c]));
#pragma unroll 1
      for (int off = 16; off > 0; off >>= 1) a = dw_add(a, dw_shfl_down(a, off));
      if (lane == 0) s_chain[v - 3] = a;
    } else if (warp == 11 && need_ll) {
      double a = 0.0;
#pragma unroll 1
      for (int c = lane; c < C; c += 32) a += slot_f64(&srec[2 * kIncMaxCtas + c]);
#pragma unroll 1
      for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(kFull, a, off);
      if (lane == 0) s_LL = a;
    }
    __syncthreads();
    if (trace) trace[14] = uint64_t(clock64());
    // ---- 7. the coordinate step, computed identically by every CTA; meanwhile the next column's
    //         A and B (its list holds v after the pending update; the update this step decides
    //         changes the entries that mfl marks)
    if (warp >= kPsWarp0)
      inc_prescan(lv_n, mfl, fce, nnx, ua, ub, s_agg, s_flg);
    if (tid == 0) {
      bool stop = false;
      if (s_anyerr) {
        st.state = kError;
        stop = true;
      } else if (need_ll) {
        const double ll = st.bdx - s_LL - shift * D.sum_d;
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
      if (stop) {
        st.pend_j = -1;   // this step already applied the pending update
        st.E = dw_make(0.0f);
      } else {
        const dw G1 = dw_add_same(dw_add_same(s_Gq[0][0], s_Gq[0][1]), dw_add_same(s_Gq[0][2], s_Gq[0][3]));
        const dw G2 = dw_add_same(dw_add_same(s_Gq[1][0], s_Gq[1][1]), dw_add_same(s_Gq[1][2], s_Gq[1][3]));
        const IncPre q = s_pre;
        if (trace) trace[17] = uint64_t(clock64());
        int kind;
        const dw sw = inc_step_rule_dw(dw_sub(G1, q.dxw), G2, q.bw, q.b == 0.0, q.tw, F.penalty, s_lambda_dw,
                                       s_inv_var_dw, q.pen, &kind);
        if (trace) trace[18] = uint64_t(clock64());
        const double sd = inc_step_value(sw, kind, q.b, q.t);
        if (sd != 0.0) {
          st.pend_j = j;
          st.pend_db = sd;
          st.E = dw_from(exp(sd) - 1.0);   // its absolute error is what the sums see
        } else {
          st.pend_j = -1;
          st.pend_db = 0.0;
          st.E = dw_make(0.0f);
        }
        // coefficient, trust, beta'dX and penalty follow at the next step (inc_book)
        st.book = 1;
        st.book_j = j;
        st.book_s = sd;
        st.book_b = q.b;
        st.book_dx = q.dx;
        st.book_t = q.t;
        st.book_pen = q.pen;
        st.coord_updates += 1;
        const int jn = j + 1 >= p ? 0 : j + 1;
        if (jn == 0) {
          st.sweep += 1;
          st.need_ll = 1;
        } else {
          st.need_ll = 0;
        }
        st.j = jn;
        st.halt = q.halt_next;
      }
      st.epoch = epoch + 1u;
      if (trace) trace[15] = uint64_t(clock64());
    }
    cp_async_wait_all();   // the fetched list's eta and v, the next range (issued during the inbox wait)
    __syncthreads();
    ++base;
  }

  if (tid == kIncThreads - 1 && st.book) inc_book(st, bet, tru, F, half_inv_var);
  // ---- the fit's v in its own precision: current since the last rebuild unless later steps
  //      updated positions
  if (!refreshed) {
    T *vt = static_cast<T *>(F.v);
#pragma unroll 1
    for (int q = tid; q < npos; q += kIncThreads) {
      const int g = lo + q;
      const bool ex = D.exit_bits != nullptr && ((D.exit_bits[g >> 5] >> (g & 31)) & 1u);
      T vv;
      inc_v<P>(F.eta[g], shift, ex, &vv, &s_err);
      vt[g] = vv;
    }
  }
  __syncthreads();
  // ---- CTA 0 writes back the coefficients, trust half-widths and the control state
  if (t == 0) {
#pragma unroll 1
    for (int jj = tid; jj < p; jj += kIncThreads) {
      F.beta[jj] = bet[jj];
      F.trust[jj] = tru[jj];
    }
    if (tid == 0) {
      if (s_err) atomicCAS(&ctl->error, 0, s_err);
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
  } else if (tid == 0 && s_err) {
    atomicCAS(&ctl->error, 0, s_err);
  }
}

// One fit over the whole grid: its arguments stay in the kernel-parameter space. The traced
// instantiation records phase timestamps (its trace pointer costs registers, so the production
// instantiation has none).
template <class P, class Cfg, bool kTrace>
__global__ void __launch_bounds__(kIncThreads, 1) ccd_incr_kernel(const IncParams prm) {
  incr_body<P, Cfg, kTrace>(prm, int(blockIdx.x));
}

// Several fits per launch: CTA b runs tile cta_map[b].y of fit cta_map[b].x, whose arguments it
// copies into shared memory.
template <class P>
__global__ void __launch_bounds__(kIncThreads, 1) ccd_incr_multi_kernel(const IncParams *prms, const int2 *cta_map) {
  __shared__ IncParams sp;
  const int2 me = cta_map[blockIdx.x];
  static_assert(sizeof(IncParams) % 4 == 0, "copied in words");
  const uint32_t *src = reinterpret_cast<const uint32_t *>(prms + me.x);
  uint32_t *dst = reinterpret_cast<uint32_t *>(&sp);
  for (int w = int(threadIdx.x); w < int(sizeof(IncParams) / 4); w += kIncThreads) dst[w] = src[w];
  __syncthreads();
  incr_body<P, IncWide, false>(sp, me.y);
}

template <class K>
static int inc_max_ctas_of(K kernel, size_t sm) {
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0, dev = 0, nsm = 0, coop = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kIncThreads, sm) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  const int g = coop ? per_sm * nsm : 0;
  return g < kIncMaxCtas ? g : kIncMaxCtas;
}

// the largest cooperative grid of a configuration's entry points (the smallest of them)
template <class P, class Cfg>
static int inc_max_ctas() {
  static int cached = -2;
  if (cached != -2) return cached;
  const size_t sm = IncSmem<Cfg>::bytes;
  int g = inc_max_ctas_of(ccd_incr_kernel<P, Cfg, false>, sm);
#if COX_TRACE_ON
  g = std::min(g, inc_max_ctas_of(ccd_incr_kernel<P, Cfg, true>, sm));
#endif
  if (std::is_same<Cfg, IncWide>::value) g = std::min(g, inc_max_ctas_of(ccd_incr_multi_kernel<P>, sm));
  return cached = g;
}

int inc_max_grid(int precision, int variant) {
  if (variant)
    return precision == COX_FP32C ? inc_max_ctas<PF32C, IncDeep>() : inc_max_ctas<PF64, IncDeep>();
  return precision == COX_FP32C ? inc_max_ctas<PF32C, IncWide>() : inc_max_ctas<PF64, IncWide>();
}

template <class Cfg>
static const void *incr_entry(int precision, bool trace) {
#if COX_TRACE_ON
  if (trace)
    return precision == COX_FP32C ? reinterpret_cast<const void *>(ccd_incr_kernel<PF32C, Cfg, true>)
                                  : reinterpret_cast<const void *>(ccd_incr_kernel<PF64, Cfg, true>);
#else
  (void)trace;
#endif
  return precision == COX_FP32C ? reinterpret_cast<const void *>(ccd_incr_kernel<PF32C, Cfg, false>)
                                : reinterpret_cast<const void *>(ccd_incr_kernel<PF64, Cfg, false>);
}

int launch_incr(int precision, const IncParams &prm, int grid, void *stream, int variant) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void *args[] = {const_cast<IncParams *>(&prm)};
  if (grid <= 0 || grid > inc_max_grid(precision, variant) || grid != prm.T) return COX_E_INVALID;
  count_launches(1);
  const bool tr = prm.trace != nullptr;
  const void *fn = variant ? incr_entry<IncDeep>(precision, tr) : incr_entry<IncWide>(precision, tr);
  const size_t sm = variant ? IncSmem<IncDeep>::bytes : IncSmem<IncWide>::bytes;
  const cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kIncThreads), args, sm, s);
  return e == cudaSuccess ? COX_OK : COX_E_CUDA;
}

int launch_incr_multi(int precision, const IncParams *prms, const int2 *cta_map, int grid, void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void *args[] = {const_cast<IncParams **>(&prms), const_cast<int2 **>(&cta_map)};
  if (grid <= 0 || grid > inc_max_grid(precision, 0)) return COX_E_INVALID;
  count_launches(1);
  const void *fn = precision == COX_FP32C ? reinterpret_cast<const void *>(ccd_incr_multi_kernel<PF32C>)
                                          : reinterpret_cast<const void *>(ccd_incr_multi_kernel<PF64>);
  const cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kIncThreads), args, IncSmem<IncWide>::bytes, s);
  return e == cudaSuccess ? COX_OK : COX_E_CUDA;
}

}  // namespace coxgb
