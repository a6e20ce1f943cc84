// Double-word arithmetic on the FP32 pipe: a value is the unevaluated sum h + l of two floats
// with |l| <= ulp(h)/2 (about 48 significant bits). On GB300 an FP64 instruction occupies its
// sub-partition's FP64 unit for 64 cycles, while these sequences run on the FP32 pipe at one
// warp instruction per cycle, so sums and ratios over many positions or tie groups are done here.
//
// Building blocks (error-free transformations): Knuth's TwoSum (TAOCP vol. 2 §4.2.2), Dekker's
// Fast2Sum and an FMA-based TwoProd (T. J. Dekker, "A floating-point technique for extending the
// available precision", Numer. Math. 18, 1971). Double-word operations follow the algorithms
// analysed by M. Joldes, J.-M. Muller and V. Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic", ACM TOMS 44(2), 2017: the accurate DW+DW sum
// (relative error <= 3u^2 + 13u^3; the sloppy sum for same-sign operands), DW*FP (<= 2u^2),
// DW*DW with FMA (<= 5u^2) and DW/DW
// (<= 15u^2 + 56u^3), u = 2^-24. Every step uses explicitly rounded intrinsics so that no
// compiler contraction can change the error-free transformations.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#include <cuda_runtime.h>
#define DW_FN static __host__ __device__ __forceinline__
#else   // host-only builds (the arithmetic's CPU test): plain IEEE float, no contraction
#include <cmath>
#define DW_FN static inline
#endif

namespace coxgb {

// correctly rounded float operations that the compiler may not contract or reorder
#if defined(__CUDA_ARCH__)
DW_FN float dw_fadd(float a, float b) { return __fadd_rn(a, b); }
DW_FN float dw_fsub(float a, float b) { return __fsub_rn(a, b); }
DW_FN float dw_fmul(float a, float b) { return __fmul_rn(a, b); }
DW_FN float dw_ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
DW_FN float dw_fdiv(float a, float b) { return __fdiv_rn(a, b); }
#else
DW_FN float dw_fadd(float a, float b) { volatile float r = a + b; return r; }
DW_FN float dw_fsub(float a, float b) { volatile float r = a - b; return r; }
DW_FN float dw_fmul(float a, float b) { volatile float r = a * b; return r; }
DW_FN float dw_ffma(float a, float b, float c) { return std::fmaf(a, b, c); }
DW_FN float dw_fdiv(float a, float b) { volatile float r = a / b; return r; }
#endif

struct dw {
  float h, l;
};

DW_FN dw dw_make(float h) { return {h, 0.0f}; }

// a + b = s + e exactly
DW_FN dw two_sum(float a, float b) {
  const float s = dw_fadd(a, b);
  const float bb = dw_fsub(s, a);
  const float e = dw_fadd(dw_fsub(a, dw_fsub(s, bb)), dw_fsub(b, bb));
  return {s, e};
}
// a + b = s + e exactly when |a| >= |b| (or a == 0)
DW_FN dw fast_two_sum(float a, float b) {
  const float s = dw_fadd(a, b);
  const float e = dw_fsub(b, dw_fsub(s, a));
  return {s, e};
}
// a * b = p + e exactly (barring underflow)
DW_FN dw two_prod(float a, float b) {
  const float p = dw_fmul(a, b);
  const float e = dw_ffma(a, b, -p);
  return {p, e};
}

// x + y, the accurate double-word sum (valid for operands of any signs)
DW_FN dw dw_add(dw x, dw y) {
  const dw s = two_sum(x.h, y.h);
  const dw t = two_sum(x.l, y.l);
  const float c = dw_fadd(s.l, t.h);
  const dw v = fast_two_sum(s.h, c);
  const float w = dw_fadd(t.l, v.l);
  return fast_two_sum(v.h, w);
}
// x + y for operands of the same sign (the sloppy double-word sum of the same paper: fewer
// operations, relative error within 3u^2 when x and y do not cancel)
DW_FN dw dw_add_same(dw x, dw y) {
  const dw s = two_sum(x.h, y.h);
  const float v = dw_fadd(x.l, y.l);
  const float w = dw_fadd(s.l, v);
  return fast_two_sum(s.h, w);
}
DW_FN dw dw_neg(dw x) { return {-x.h, -x.l}; }
DW_FN dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }

// x * y for a float y
DW_FN dw dw_mul_f(dw x, float y) {
  const dw c = two_prod(x.h, y);
  const float cl3 = dw_ffma(x.l, y, c.l);
  return fast_two_sum(c.h, cl3);
}
// x * y
DW_FN dw dw_mul(dw x, dw y) {
  const dw c = two_prod(x.h, y.h);
  const float tl0 = dw_fmul(x.l, y.l);
  const float tl1 = dw_ffma(x.h, y.l, tl0);
  const float cl2 = dw_ffma(x.l, y.h, tl1);
  const float cl3 = dw_fadd(c.l, cl2);
  return fast_two_sum(c.h, cl3);
}
// x / y (y != 0)
DW_FN dw dw_div(dw x, dw y) {
  const float th = dw_fdiv(x.h, y.h);
  const dw r = dw_mul_f(y, th);
  const float pih = dw_fsub(x.h, r.h);
  const float dl = dw_fsub(x.l, r.l);
  const float d = dw_fadd(pih, dl);
  const float tl = dw_fdiv(d, y.h);
  return fast_two_sum(th, tl);
}

// conversions (FP64 instructions on the GPU: used at the edges only)
DW_FN dw dw_from(double x) {
  const float h = float(x);
  return {h, float(x - double(h))};
}
DW_FN double dw_to(dw x) { return double(x.h) + double(x.l); }
DW_FN bool dw_is_zero(dw x) { return x.h == 0.0f && x.l == 0.0f; }

#if defined(__CUDACC__)
// warp shuffles
static __device__ __forceinline__ dw dw_shfl_down(dw x, int off) {
  return {__shfl_down_sync(0xffffffffu, x.h, off), __shfl_down_sync(0xffffffffu, x.l, off)};
}
static __device__ __forceinline__ dw dw_shfl(dw x, int src) {
  return {__shfl_sync(0xffffffffu, x.h, src), __shfl_sync(0xffffffffu, x.l, src)};
}
#endif

}  // namespace coxgb
