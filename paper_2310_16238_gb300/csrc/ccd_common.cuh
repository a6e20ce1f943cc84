// Device building blocks shared by the coordinate-step kernels (ccd.cu, ccd_resident.cu):
// PTX memory-ordering helpers, the FP64 / compensated-FP32 precision policies, the §2.4 step
// rule and the exp(eta) value written at a risk-sequence position.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "cox.h"
#include "cox_internal.h"

namespace coxgb {

// ------------------------------------------------------------------ PTX helpers
static __device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
static __device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
static __device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Acquire side of a release/acquire pair that was observed with relaxed loads.
static __device__ __forceinline__ void fence_acquire_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
static __device__ __forceinline__ double ld_relaxed_f64(const double *p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}
static __device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
// 4-byte asynchronous copy (both addresses 4-byte aligned), for word-granular tables
static __device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
// 8-byte asynchronous copy (both addresses 8-byte aligned)
static __device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
static __device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
static __device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// all but the most recent commit group have completed
static __device__ __forceinline__ void cp_async_wait_group1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// ------------------------------------------------------------------ precision policies
// FP64: values, scans, ratios in double.
struct PF64 {
  using T = double;
  static constexpr int ITEMS = 16;
  struct Acc { double s; };
  __device__ static Acc zero() { return {0.0}; }
  __device__ static void add(Acc &a, double x) { a.s = a.s + x; }
  __device__ static Acc comb(Acc a, Acc b) { return {a.s + b.s}; }
  __device__ static double to64(Acc a) { return a.s; }
  __device__ static Acc from64(double x) { return {x}; }
  __device__ static Acc shfl_down(Acc a, int off) { return {__shfl_down_sync(0xffffffffu, a.s, off)}; }
};

// FP32 with a compensation term: a = s + c, additions by Knuth's TwoSum (error-free
// transformation, TAOCP vol. 2 §4.2.2), so tile sums carry ~2x float precision.
struct PF32C {
  using T = float;
  static constexpr int ITEMS = 32;
  struct Acc { float s, c; };
  __device__ static Acc zero() { return {0.0f, 0.0f}; }
  __device__ static void add(Acc &a, float x) {
    float t = __fadd_rn(a.s, x);
    float bp = __fsub_rn(t, a.s);
    float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    a.s = t;
    a.c = __fadd_rn(a.c, err);
  }
  __device__ static Acc comb(Acc a, Acc b) {
    Acc r = a;
    add(r, b.s);
    r.c = __fadd_rn(r.c, b.c);
    return r;
  }
  __device__ static double to64(Acc a) { return (double)a.s + (double)a.c; }
  __device__ static Acc from64(double x) {
    float hi = __double2float_rn(x);
    return {hi, __double2float_rn(x - (double)hi)};
  }
  __device__ static Acc shfl_down(Acc a, int off) {
    return {__shfl_down_sync(0xffffffffu, a.s, off), __shfl_down_sync(0xffffffffu, a.c, off)};
  }
};


// ------------------------------------------------------------------ the coordinate step
// §2.4, with these readings where the paper is silent: L2 adds beta/sigma^2 and 1/sigma^2; L1 uses the
// directional derivatives g' +- gamma at 0 and g' + gamma sgn(beta) elsewhere; the Newton
// step is clipped to the trust half-width, an L1 step that would cross 0 stops at 0, and
// the half-width becomes max(2 |step|, half-width / 2). g'' <= 0 skips the coordinate.
static __device__ double ccd_step_rule(double g1, double g2, double b, double *tr, int penalty, double lambda,
                                double l2_var, int penalized) {
  double gamma = 0.0;
  if (penalized && penalty == COX_PEN_L2) {
    g1 = g1 + b / l2_var;
    g2 = g2 + 1.0 / l2_var;
  }
  if (penalized && penalty == COX_PEN_L1) gamma = lambda;
  double s;
  if (!(g2 > 0.0) || !isfinite(g1) || !isfinite(g2)) {
    s = 0.0;
  } else if (gamma > 0.0) {
    if (b == 0.0) {
      if (g1 + gamma < 0.0) s = -(g1 + gamma) / g2;
      else if (g1 - gamma > 0.0) s = -(g1 - gamma) / g2;
      else s = 0.0;
    } else {
      s = -(g1 + (b > 0.0 ? gamma : -gamma)) / g2;
    }
  } else {
    s = -g1 / g2;
  }
  double t = *tr;
  if (fabs(s) > t) s = s > 0.0 ? t : -t;
  if (gamma > 0.0 && b != 0.0) {
    double nb = b + s;
    if ((b > 0.0 && nb < 0.0) || (b < 0.0 && nb > 0.0)) s = -b;
  }
  double a2 = 2.0 * fabs(s), h = 0.5 * t;
  *tr = a2 > h ? a2 : h;
  return s;
}

// Block-wide sum of NV doubles in a fixed order (deterministic for fixed inputs).
template <int NV>
static __device__ void block_sum(double (&v)[NV], double *scratch /* [NV*32] */) {
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
      double x = lane < (kThreads / 32) ? scratch[i * 32 + lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      v[i] = x;   // valid in thread 0
    }
  }
  __syncthreads();
}

// block_sum for a CTA of NT threads (NT a multiple of 32, at most 1024).
template <int NV, int NT>
static __device__ void block_sum_nt(double (&v)[NV], double *scratch /* [NV*32] */) {
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
      double x = lane < (NT / 32) ? scratch[i * 32 + lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      v[i] = x;   // valid in thread 0
    }
  }
  __syncthreads();
}

// The end of a launch for one fit, run by the CTA that finished its last unit of work: the units'
// partials (G1, G2, sum d log S0) summed in a fixed order, then by mode the evaluation result, the
// log-likelihood, or the convergence test (once per sweep) and the coordinate step of §2.4 with
// the update it leaves pending for the next launch. `nunits` partials sit in F.part[3u..3u+2].
// kFence: the caller's completion count was relaxed, so the partials need an acquire fence here
// (false where the count was an acquire-release atomic followed by a CTA barrier).
template <int NT, bool kFence = true>
static __device__ void finish_launch_step(const DevFit &F, LaunchCtl *lc, int mode, int j, bool need_ll, int nunits,
                                          uint32_t epoch, double *s_red) {
  const DevData *D = F.d;
  FitCtl *ctl = F.ctl;
  const int tid = threadIdx.x;
  const double shift = F.shift;
  const int T_ = nunits;
  if constexpr (kFence) __threadfence();
  // the step's scalars, loaded ahead of the reduction below (each would otherwise be a dependent
  // round trip of thread 0 after it)
  double dxj = 0.0, bj = 0.0, trj = 0.0, obj_prev = 0.0, sum_d = 0.0;
  int pzj = 1, err = 0, state = 0, sweep = 0, np_ = 0;
  if (tid == 0) {
    if (j >= 0) {
      dxj = D->dX[j];
      bj = F.beta[j];
      trj = F.trust[j];
      pzj = F.penalize ? F.penalize[j] != 0 : 1;
    }
    err = ctl->error;
    state = ctl->state;
    sweep = ctl->sweep;
    obj_prev = ctl->obj_prev;
    sum_d = D->sum_d;
    np_ = D->p;
  }
  double acc[3] = {0.0, 0.0, 0.0};
  for (int u = tid; u < T_; u += NT) {
    acc[0] += ld_relaxed_f64(&F.part[3 * u + 0]);
    acc[1] += ld_relaxed_f64(&F.part[3 * u + 1]);
    acc[2] += ld_relaxed_f64(&F.part[3 * u + 2]);
  }
  block_sum_nt<3, NT>(acc, s_red);
  double extra[2] = {0.0, 0.0};   // beta'dX and the penalty, when the log-likelihood is due
  if (need_ll) {
    for (int jj = tid; jj < D->p; jj += NT) {
      const double b = F.beta[jj];
      extra[0] += b * D->dX[jj];
      const bool pen = F.penalize ? F.penalize[jj] != 0 : true;
      if (pen && F.penalty == COX_PEN_L1) extra[1] += F.lambda * fabs(b);
      if (pen && F.penalty == COX_PEN_L2) extra[1] += b * b / (2.0 * F.l2_var);
    }
    block_sum_nt<2, NT>(extra, s_red);
  }
  if (tid == 0) {
    const double G1 = acc[0], G2 = acc[1], LL = acc[2];
    if (err != 0) {   // raised by this fit's work in this launch (every unit finished before the fence)
      if (mode == kModeFit && state == kRunning) atomicSub(&lc->active, 1);
      ctl->state = kError;
    } else if (mode == kModeShard) {
      ctl->out_g1 = G1;
      ctl->out_g2 = G2;
      ctl->out_ll = LL;
      ctl->out_bdx = extra[0];
    } else if (mode == kModeEval) {
      ctl->out_g1 = -dxj + G1;
      ctl->out_g2 = G2;
      if (F.gout) { F.gout[2 * j] = -dxj + G1; F.gout[2 * j + 1] = G2; }
    } else if (mode == kModeLL) {
      ctl->out_ll = extra[0] - LL - shift * sum_d;
    } else {
      bool stop = false;
      if (need_ll) {
        const double ll = extra[0] - LL - shift * sum_d;
        const double obj = -ll + extra[1];
        ctl->loglik = ll;
        ctl->obj = obj;
        if (sweep > 0 && fabs(obj - obj_prev) <= F.tol * fabs(obj)) {
          ctl->state = kConverged;
          stop = true;
        } else if (sweep >= F.max_sweeps) {
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
        const double g1 = -dxj + G1, g2 = G2;
        double tr = trj;
        const double s = ccd_step_rule(g1, g2, bj, &tr, F.penalty, F.lambda, F.l2_var, pzj);
        F.trust[j] = tr;
        if (s != 0.0) {
          F.beta[j] = bj + s;
          ctl->pend_j = j;
          ctl->pend_db = s;
        } else {
          ctl->pend_j = -1;
          ctl->pend_db = 0.0;
        }
        ctl->coord_updates += 1;
        int jn = j + 1;
        if (jn >= np_) {
          jn = 0;
          ctl->sweep = sweep + 1;
          ctl->need_ll = 1;
        } else {
          ctl->need_ll = 0;
        }
        ctl->j = jn;
      }
    }
    ctl->done_tiles = 0u;
    ctl->epoch = epoch + 1u;
  }
}

// value written at a position for exp(eta - shift); exits hold the negative
template <class P>
static __device__ __forceinline__ typename P::T make_v(double eta, double shift, bool exitp, int32_t *err) {
  if constexpr (sizeof(typename P::T) == 8) {
    double e = exp(eta - shift);
    return exitp ? -e : e;
  } else {
    double a = eta - shift;
    if (!(fabs(a) < 80.0)) atomicExch(err, COX_E_RANGE);
    float e = expf(__double2float_rn(a));
    return exitp ? -e : e;
  }
}

template <class Acc, class P, int NV>
static __device__ __forceinline__ void comb_n(Acc (&a)[NV], const Acc (&b)[NV]) {
#pragma unroll
  for (int i = 0; i < NV; ++i) a[i] = P::comb(a[i], b[i]);
}

}  // namespace coxgb
