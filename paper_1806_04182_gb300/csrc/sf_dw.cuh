// Arithmetic of the "island" quantities of the FP32-bulk CCZ4 path (conformal
// metric determinant, inverse, ln det and the trace removals), in one of two
// types:
//   double - native FP64;
//   dw     - an unevaluated sum hi + lo of two floats ("double-word"), built
//            from error-free transformations: TwoSum (Knuth, TAOCP vol. 2),
//            FastTwoSum (Dekker 1971), TwoProd via FMA, and the double-word
//            sum/product algorithms of Joldes, Muller & Popescu, "Tight and
//            rigorous error bounds for basic building blocks of double-word
//            arithmetic", ACM TOMS 44 (2017) (AccurateDWPlusDW, DWTimesFP3,
//            DWTimesDW3).  Relative error of each operation is a few 2^-48,
//            i.e. within a small factor of FP64, while every instruction runs
//            on the FP32 pipe (GB300's FP64 pipe is ~1/58 of its FP32 rate).
// The explicit __fadd_rn/__fmul_rn intrinsics keep the compiler from fusing
// the error-free transformations into FMAs.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace sf {

struct dw {
  float hi, lo;
};

__device__ __forceinline__ dw dw_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fadd_rn(s, -a);
  const float e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
  return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ dw dw_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float z = __fadd_rn(s, -a);
  return {s, __fadd_rn(b, -z)};
}

__device__ __forceinline__ dw dw_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dw dw_add(dw x, dw y) {  // AccurateDWPlusDW
  const dw s = dw_two_sum(x.hi, y.hi);
  const dw t = dw_two_sum(x.lo, y.lo);
  const float c = __fadd_rn(s.lo, t.hi);
  const dw v = dw_fast_two_sum(s.hi, c);
  const float w = __fadd_rn(t.lo, v.lo);
  return dw_fast_two_sum(v.hi, w);
}

__device__ __forceinline__ dw dw_neg(dw x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ dw dw_mulf(dw x, float y) {  // DWTimesFP3
  const dw c = dw_two_prod(x.hi, y);
  const float cl3 = __fmaf_rn(x.lo, y, c.lo);
  return dw_fast_two_sum(c.hi, cl3);
}

__device__ __forceinline__ dw dw_mul(dw x, dw y) {  // DWTimesDW3
  const dw c = dw_two_prod(x.hi, y.hi);
  const float tl0 = __fmul_rn(x.lo, y.lo);
  const float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
  const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  const float cl3 = __fadd_rn(c.lo, cl2);
  return dw_fast_two_sum(c.hi, cl3);
}

// 1/x by one Newton step from the float reciprocal r0: with the residual
// e = 1 - x r0 (|e| ~ 2^-24, formed by an FMA, which is exact for it, minus
// x.lo r0), 1/x = r0 + r0 e + O(e^2); the two terms are normalised by
// FastTwoSum (|r0| > |r0 e|).
__device__ __forceinline__ dw dw_recip(dw x) {
  const float r0 = __frcp_rn(x.hi);
  const float e = __fmaf_rn(-x.lo, r0, __fmaf_rn(-x.hi, r0, 1.0f));
  return dw_fast_two_sum(r0, __fmul_rn(r0, e));
}

// Dot product sum_q a_q x_q of double-word a_q and float x_q, in the manner
// of Ogita, Rump & Oishi, "Accurate sum and dot product", SIAM J. Sci.
// Comput. 26 (2005) (Dot2): each product's high part is exact by TwoProd,
// the high parts are added by a cascade of TwoSums, and every rounding error
// (and the low parts a_q.lo x_q) is summed in float; the result is as
// accurate as a dot product evaluated in twice the float precision.
template <int N>
__device__ __forceinline__ dw dw_dot(const dw* a, const float* x) {
  float s = __fmul_rn(a[0].hi, x[0]);
  float err = __fmaf_rn(a[0].lo, x[0], __fmaf_rn(a[0].hi, x[0], -s));
#pragma unroll
  for (int q = 1; q < N; ++q) {
    const float p = __fmul_rn(a[q].hi, x[q]);
    const float pe = __fmaf_rn(a[q].lo, x[q], __fmaf_rn(a[q].hi, x[q], -p));
    const dw t = dw_two_sum(s, p);
    s = t.hi;
    err = __fadd_rn(err, __fadd_rn(t.lo, pe));
  }
  return dw_two_sum(s, err);
}

// x - a y rounded to float, for float x, y and double-word a: the product's
// high part is exact (TwoProd), its subtraction from x exact (TwoSum), and
// the remaining small terms are added once.
__device__ __forceinline__ float dw_sub_prod_f(float x, dw a, float y) {
  const float p = __fmul_rn(a.hi, y);
  const float pe = __fmaf_rn(a.lo, y, __fmaf_rn(a.hi, y, -p));
  const dw t = dw_two_sum(x, -p);
  return __fadd_rn(t.hi, __fadd_rn(t.lo, -pe));
}

// ------------------------------------------------------------ island ops
// Uniform interface over H = double and H = dw.
template <typename H> struct Isl;

template <> struct Isl<double> {
  using H = double;
  static __device__ __forceinline__ H from(float a) { return double(a); }
  static __device__ __forceinline__ H from(double a) { return a; }
  static __device__ __forceinline__ H sum2(float a, float b) { return double(a) + double(b); }
  static __device__ __forceinline__ H sum2(double a, double b) { return a + b; }
  static __device__ __forceinline__ H prod(float a, float b) { return double(a) * double(b); }
  static __device__ __forceinline__ H prod(double a, double b) { return a * b; }
  static __device__ __forceinline__ H add(H a, H b) { return a + b; }
  static __device__ __forceinline__ H sub(H a, H b) { return a - b; }
  static __device__ __forceinline__ H mul(H a, H b) { return a * b; }
  static __device__ __forceinline__ H mulf(H a, float b) { return a * double(b); }
  static __device__ __forceinline__ H mulf(H a, double b) { return a * b; }
  static __device__ __forceinline__ H recip(H a) { return 1.0 / a; }
  static __device__ __forceinline__ H third(H a) { return a * (1.0 / 3.0); }
  // a_0 x_0 + a_3 x_3 + a_5 x_5 + 2 (a_1 x_1 + a_2 x_2 + a_4 x_4): the trace
  // of a symmetric X stored as xx, xy, xz, yy, yz, zz against symmetric a
  template <typename T> static __device__ __forceinline__ H trace_sym(const H* a, const T* x) {
    return (a[0] * double(x[0]) + a[3] * double(x[3]) + a[5] * double(x[5])) +
           2.0 * (a[1] * double(x[1]) + a[2] * double(x[2]) + a[4] * double(x[4]));
  }
  // x - a y in the bulk type
  template <typename T> static __device__ __forceinline__ T sub_prod(T x, H a, T y) {
    return T(double(x) - a * double(y));
  }
  template <typename T> static __device__ __forceinline__ T to(H a) { return T(a); }
  // a kept as its bulk rounding v plus the exact remainder (nothing kept
  // when the bulk type is double itself)
  template <typename V> using Resid = double;
  template <typename V> static __device__ __forceinline__ double resid(H a, V v) {
    if constexpr (std::is_same<V, double>::value) return 0.0;
    else return a - double(v);
  }
  template <typename V> static __device__ __forceinline__ H join(V v, double r) {
    if constexpr (std::is_same<V, double>::value) return v;
    else return double(v) + r;
  }
  // ln of a value close to 1, returned in the bulk type (r: 1/a, unused here)
  template <typename T> static __device__ __forceinline__ T log(H a, H) { return T(::log(a)); }
};

template <> struct Isl<dw> {
  using H = dw;
  static __device__ __forceinline__ H from(float a) { return {a, 0.0f}; }
  static __device__ __forceinline__ H sum2(float a, float b) { return dw_two_sum(a, b); }
  static __device__ __forceinline__ H prod(float a, float b) { return dw_two_prod(a, b); }
  static __device__ __forceinline__ H add(H a, H b) { return dw_add(a, b); }
  static __device__ __forceinline__ H sub(H a, H b) { return dw_add(a, dw_neg(b)); }
  static __device__ __forceinline__ H mul(H a, H b) { return dw_mul(a, b); }
  static __device__ __forceinline__ H mulf(H a, float b) { return dw_mulf(a, b); }
  static __device__ __forceinline__ H recip(H a) { return dw_recip(a); }
  static __device__ __forceinline__ H third(H a) {
    // multiply by 1/3 represented as a double-word constant
    return dw_mul(a, dw{0.333333343267f, -9.93410746e-09f});
  }
  template <typename T> static __device__ __forceinline__ H trace_sym(const H* a, const T* x) {
    const dw aa[6] = {a[0], a[3], a[5], a[1], a[2], a[4]};
    const float xx[6] = {x[0], x[3], x[5], 2.0f * x[1], 2.0f * x[2], 2.0f * x[4]};
    return dw_dot<6>(aa, xx);
  }
  template <typename T> static __device__ __forceinline__ T sub_prod(T x, H a, T y) {
    return dw_sub_prod_f(x, a, y);
  }
  template <typename T> static __device__ __forceinline__ T to(H a) { return T(a.hi + a.lo); }
  // a as its float rounding v = fl(hi + lo) plus the exact remainder
  // (FastTwoSum's error term), which together represent a exactly
  template <typename V> using Resid = float;
  template <typename V> static __device__ __forceinline__ float resid(H a, V v) {
    return __fadd_rn(a.lo, -__fadd_rn(v, -a.hi));
  }
  template <typename V> static __device__ __forceinline__ H join(V v, float r) { return {v, r}; }
  // ln(hi + lo) = ln(hi) + ln(1 + lo/hi) ~ logf(hi) + lo/hi (|lo/hi| < 2^-24);
  // r is 1/a, so lo/hi = lo r.hi to far better than the term's own size
  template <typename T> static __device__ __forceinline__ T log(H a, H r) {
    return T(::logf(a.hi) + a.lo * r.hi);
  }
};

}  // namespace sf
