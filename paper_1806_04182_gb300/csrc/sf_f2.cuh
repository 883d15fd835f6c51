// Two float lanes computed by one instruction: the value type of the CCZ4
// float kernels that give each thread two neighbouring points along x.
//
// sm_100-class GPUs issue add/sub/mul/fma on a pair of floats (.f32x2) as
// one instruction, each lane rounded exactly as the scalar instruction
// would round it.  F2 carries the two points' values of one quantity, so
// every step of the per-point right-hand side advances both points at the
// cost of one issue slot.  Products are kept unevaluated (F2Prod) until they
// meet an addition, so that `s + a * b` and `s += a * b` become one fused
// multiply-add, as the compiler contracts them for scalar floats.  PTX has
// no paired negation, so a product subtracted from a value, or a value
// subtracted from a product, is formed as a multiply followed by a
// subtraction.
//
// The island arithmetic of the FP32-bulk CCZ4 path on pairs is here too:
// DW2, a double-word (hi + lo) per lane built from the error-free
// transformations of sf_dw.cuh, and D2, native FP64 per lane.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "sf_dw.cuh"

namespace sf {

struct alignas(8) F2 {
  float x, y;
  F2() = default;
  __device__ __forceinline__ constexpr F2(float a, float b) : x(a), y(b) {}
  // broadcast of a scalar (the algebra's constants: T(0), T(2.0 / 3.0), ...)
  template <typename S, typename = std::enable_if_t<std::is_arithmetic<S>::value>>
  __device__ __forceinline__ explicit constexpr F2(S v) : x(float(v)), y(float(v)) {}
};

__device__ __forceinline__ unsigned long long f2_bits(F2 a) {
  return *reinterpret_cast<const unsigned long long*>(&a);
}
__device__ __forceinline__ F2 f2_from(unsigned long long r) { return *reinterpret_cast<const F2*>(&r); }

__device__ __forceinline__ F2 add2(F2 a, F2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_from(r);
}
__device__ __forceinline__ F2 sub2(F2 a, F2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_from(r);
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_from(r);
}
// a * b + c, one rounding per lane
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
  return f2_from(r);
}
__device__ __forceinline__ F2 neg2(F2 a) { return F2(-a.x, -a.y); }

// ------------------------------------------------------------ expressions
struct F2Prod {
  F2 a, b;
  __device__ __forceinline__ operator F2() const { return mul2(a, b); }
};

__device__ __forceinline__ F2Prod operator*(F2 a, F2 b) { return {a, b}; }
__device__ __forceinline__ F2Prod operator*(F2Prod p, F2 c) { return {F2(p), c}; }
__device__ __forceinline__ F2Prod operator*(F2 c, F2Prod p) { return {c, F2(p)}; }
__device__ __forceinline__ F2Prod operator*(F2Prod p, F2Prod q) { return {F2(p), F2(q)}; }

__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return add2(a, b); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return sub2(a, b); }
__device__ __forceinline__ F2 operator+(F2Prod p, F2 c) { return fma2(p.a, p.b, c); }
__device__ __forceinline__ F2 operator+(F2 c, F2Prod p) { return fma2(p.a, p.b, c); }
__device__ __forceinline__ F2 operator+(F2Prod p, F2Prod q) { return fma2(p.a, p.b, F2(q)); }
__device__ __forceinline__ F2 operator-(F2Prod p, F2 c) { return sub2(F2(p), c); }
__device__ __forceinline__ F2 operator-(F2 c, F2Prod p) { return sub2(c, F2(p)); }
__device__ __forceinline__ F2 operator-(F2Prod p, F2Prod q) { return sub2(F2(p), F2(q)); }
__device__ __forceinline__ F2 operator-(F2 a) { return neg2(a); }
__device__ __forceinline__ F2Prod operator-(F2Prod p) { return {neg2(p.a), p.b}; }

__device__ __forceinline__ F2& operator+=(F2& s, F2 b) { return s = add2(s, b); }
__device__ __forceinline__ F2& operator+=(F2& s, F2Prod p) { return s = fma2(p.a, p.b, s); }
__device__ __forceinline__ F2& operator-=(F2& s, F2 b) { return s = sub2(s, b); }
__device__ __forceinline__ F2& operator-=(F2& s, F2Prod p) { return s = sub2(s, F2(p)); }
__device__ __forceinline__ F2& operator*=(F2& s, F2 b) { return s = mul2(s, b); }

// per lane, as the scalar code divides
__device__ __forceinline__ F2 operator/(F2 a, F2 b) { return F2(a.x / b.x, a.y / b.y); }
__device__ __forceinline__ F2 operator/(F2Prod a, F2 b) { return F2(a) / b; }

// ------------------------------------------------------------ pair islands
// Double-word per lane: the algorithms of sf_dw.cuh with every float
// operation on the pair.
struct DW2 {
  F2 hi, lo;
};

__device__ __forceinline__ DW2 dw2_two_sum(F2 a, F2 b) {
  const F2 s = add2(a, b);
  const F2 bb = sub2(s, a);
  const F2 e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
  return {s, e};
}
__device__ __forceinline__ DW2 dw2_fast_two_sum(F2 a, F2 b) {  // |a| >= |b| per lane
  const F2 s = add2(a, b);
  return {s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ DW2 dw2_two_prod(F2 a, F2 b) {
  const F2 p = mul2(a, b);
  return {p, fma2(a, b, neg2(p))};
}
__device__ __forceinline__ DW2 dw2_add(DW2 x, DW2 y) {
  const DW2 s = dw2_two_sum(x.hi, y.hi);
  const DW2 t = dw2_two_sum(x.lo, y.lo);
  const F2 c = add2(s.lo, t.hi);
  const DW2 v = dw2_fast_two_sum(s.hi, c);
  const F2 w = add2(t.lo, v.lo);
  return dw2_fast_two_sum(v.hi, w);
}
__device__ __forceinline__ DW2 dw2_sub(DW2 x, DW2 y) {
  // x + (-y), with the negation folded into the first level of TwoSums
  const F2 sh = sub2(x.hi, y.hi);
  const F2 bb = sub2(sh, x.hi);
  const F2 eh = sub2(sub2(x.hi, sub2(sh, bb)), add2(y.hi, bb));
  const F2 sl = sub2(x.lo, y.lo);
  const F2 bl = sub2(sl, x.lo);
  const F2 el = sub2(sub2(x.lo, sub2(sl, bl)), add2(y.lo, bl));
  const F2 c = add2(eh, sl);
  const DW2 v = dw2_fast_two_sum(sh, c);
  const F2 w = add2(el, v.lo);
  return dw2_fast_two_sum(v.hi, w);
}
__device__ __forceinline__ DW2 dw2_mulf(DW2 x, F2 y) {
  const DW2 c = dw2_two_prod(x.hi, y);
  return dw2_fast_two_sum(c.hi, fma2(x.lo, y, c.lo));
}
__device__ __forceinline__ DW2 dw2_mul(DW2 x, DW2 y) {
  const DW2 c = dw2_two_prod(x.hi, y.hi);
  const F2 t = fma2(x.hi, y.lo, mul2(x.lo, y.lo));
  return dw2_fast_two_sum(c.hi, add2(c.lo, fma2(x.lo, y.hi, t)));
}
__device__ __forceinline__ DW2 dw2_recip(DW2 x) {
  const F2 r0(__frcp_rn(x.hi.x), __frcp_rn(x.hi.y));
  const F2 e = fma2(neg2(x.lo), r0, fma2(neg2(x.hi), r0, F2(1.0f)));
  return dw2_fast_two_sum(r0, mul2(r0, e));
}

// Native FP64 per lane.
struct D2 {
  double x, y;
};

template <> struct Isl<DW2> {
  using H = DW2;
  static __device__ __forceinline__ H sum2(F2 a, F2 b) { return dw2_two_sum(a, b); }
  static __device__ __forceinline__ H prod(F2 a, F2 b) { return dw2_two_prod(a, b); }
  static __device__ __forceinline__ H add(H a, H b) { return dw2_add(a, b); }
  static __device__ __forceinline__ H sub(H a, H b) { return dw2_sub(a, b); }
  static __device__ __forceinline__ H mul(H a, H b) { return dw2_mul(a, b); }
  static __device__ __forceinline__ H mulf(H a, F2 b) { return dw2_mulf(a, b); }
  static __device__ __forceinline__ H recip(H a) { return dw2_recip(a); }
  static __device__ __forceinline__ H third(H a) {
    return dw2_mul(a, DW2{F2(0.333333343267f), F2(-9.93410746e-09f)});
  }
  // Dot2 of sf_dw.cuh on pairs: a_0 x_0 + a_3 x_3 + a_5 x_5 + 2 (a_1 x_1 + a_2 x_2 + a_4 x_4)
  template <typename V> static __device__ __forceinline__ H trace_sym(const H* a, const V* x) {
    const int ord[6] = {0, 3, 5, 1, 2, 4};
    F2 s, err;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int q = ord[k];
      const F2 xq = k < 3 ? x[q] : add2(x[q], x[q]);
      const F2 p = mul2(a[q].hi, xq);
      const F2 pe = fma2(a[q].lo, xq, fma2(a[q].hi, xq, neg2(p)));
      if (k == 0) {
        s = p;
        err = pe;
      } else {
        const DW2 t = dw2_two_sum(s, p);
        s = t.hi;
        err = add2(err, add2(t.lo, pe));
      }
    }
    return dw2_two_sum(s, err);
  }
  // x - a y rounded to float per lane
  template <typename V> static __device__ __forceinline__ V sub_prod(V x, H a, V y) {
    const F2 p = mul2(a.hi, y);
    const F2 pe = fma2(a.lo, y, fma2(a.hi, y, neg2(p)));
    const F2 th = sub2(x, p);
    const F2 bb = sub2(th, x);
    const F2 tl = sub2(sub2(x, sub2(th, bb)), add2(p, bb));  // TwoSum(x, -p) error
    return add2(th, sub2(tl, pe));
  }
  template <typename V> static __device__ __forceinline__ V to(H a) { return add2(a.hi, a.lo); }
  template <typename V> using Resid = F2;
  template <typename V> static __device__ __forceinline__ F2 resid(H a, V v) {
    return sub2(a.lo, sub2(v, a.hi));
  }
  template <typename V> static __device__ __forceinline__ H join(V v, F2 r) { return {v, r}; }
  template <typename V> static __device__ __forceinline__ V log(H a, H r) {
    return F2(::logf(a.hi.x) + a.lo.x * r.hi.x, ::logf(a.hi.y) + a.lo.y * r.hi.y);
  }
};

template <> struct Isl<D2> {
  using H = D2;
  static __device__ __forceinline__ H sum2(F2 a, F2 b) { return {double(a.x) + double(b.x), double(a.y) + double(b.y)}; }
  static __device__ __forceinline__ H prod(F2 a, F2 b) { return {double(a.x) * double(b.x), double(a.y) * double(b.y)}; }
  static __device__ __forceinline__ H add(H a, H b) { return {a.x + b.x, a.y + b.y}; }
  static __device__ __forceinline__ H sub(H a, H b) { return {a.x - b.x, a.y - b.y}; }
  static __device__ __forceinline__ H mul(H a, H b) { return {a.x * b.x, a.y * b.y}; }
  static __device__ __forceinline__ H mulf(H a, F2 b) { return {a.x * double(b.x), a.y * double(b.y)}; }
  static __device__ __forceinline__ H recip(H a) { return {1.0 / a.x, 1.0 / a.y}; }
  static __device__ __forceinline__ H third(H a) { return {a.x * (1.0 / 3.0), a.y * (1.0 / 3.0)}; }
  template <typename V> static __device__ __forceinline__ H trace_sym(const H* a, const V* x) {
    H r;
    r.x = (a[0].x * double(x[0].x) + a[3].x * double(x[3].x) + a[5].x * double(x[5].x)) +
          2.0 * (a[1].x * double(x[1].x) + a[2].x * double(x[2].x) + a[4].x * double(x[4].x));
    r.y = (a[0].y * double(x[0].y) + a[3].y * double(x[3].y) + a[5].y * double(x[5].y)) +
          2.0 * (a[1].y * double(x[1].y) + a[2].y * double(x[2].y) + a[4].y * double(x[4].y));
    return r;
  }
  template <typename V> static __device__ __forceinline__ V sub_prod(V x, H a, V y) {
    return F2(float(double(x.x) - a.x * double(y.x)), float(double(x.y) - a.y * double(y.y)));
  }
  template <typename V> static __device__ __forceinline__ V to(H a) { return F2(float(a.x), float(a.y)); }
  template <typename V> using Resid = D2;
  template <typename V> static __device__ __forceinline__ D2 resid(H a, V v) {
    return {a.x - double(v.x), a.y - double(v.y)};
  }
  template <typename V> static __device__ __forceinline__ H join(V v, D2 r) {
    return {double(v.x) + r.x, double(v.y) + r.y};
  }
  template <typename V> static __device__ __forceinline__ V log(H a, H) {
    return F2(float(::log(a.x)), float(::log(a.y)));
  }
};

}  // namespace sf
