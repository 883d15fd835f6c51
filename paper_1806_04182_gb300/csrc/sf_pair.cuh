// Two independent values advanced by one instruction.  On sm_100-class GPUs
// the FP32 pipe has paired instructions (add/sub/mul/fma .f32x2): one issue
// slot computes two lanes, each rounded exactly as the scalar instruction
// would round it.  The CCZ4 float kernels are bound by instruction issue, so
// stencil arithmetic that comes in pairs (two directions of one field, two
// mixed derivatives) is written with these.  The double instantiation is two
// scalar operations with the same rounding, for code shared with the FP64
// path.
#pragma once

#include <cuda_runtime.h>

namespace sf {

template <typename T>
struct P2 {
  T x, y;
};

template <typename T>
__device__ __forceinline__ P2<T> p2(T x, T y) {
  return {x, y};
}

template <typename T>
__device__ __forceinline__ P2<T> padd(P2<T> a, P2<T> b) {
  return {a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ P2<T> psub(P2<T> a, P2<T> b) {
  return {a.x - b.x, a.y - b.y};
}
template <typename T>
__device__ __forceinline__ P2<T> pmul(P2<T> a, P2<T> b) {
  return {a.x * b.x, a.y * b.y};
}
// a * b + c, fused
template <typename T>
__device__ __forceinline__ P2<T> pfma(P2<T> a, P2<T> b, P2<T> c) {
  return {fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)};
}

__device__ __forceinline__ float2 f2_(P2<float> a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ P2<float> p2_(float2 a) { return {a.x, a.y}; }

template <>
__device__ __forceinline__ P2<float> padd(P2<float> a, P2<float> b) {
  return p2_(__fadd2_rn(f2_(a), f2_(b)));
}
template <>
__device__ __forceinline__ P2<float> psub(P2<float> a, P2<float> b) {
  unsigned long long r;
  const float2 x = f2_(a), y = f2_(b);
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(r)
      : "l"(*reinterpret_cast<const unsigned long long*>(&x)),
        "l"(*reinterpret_cast<const unsigned long long*>(&y)));
  return p2_(*reinterpret_cast<const float2*>(&r));
}
template <>
__device__ __forceinline__ P2<float> pmul(P2<float> a, P2<float> b) {
  return p2_(__fmul2_rn(f2_(a), f2_(b)));
}
template <>
__device__ __forceinline__ P2<float> pfma(P2<float> a, P2<float> b, P2<float> c) {
  return p2_(__ffma2_rn(f2_(a), f2_(b), f2_(c)));
}

}  // namespace sf
