// Scalar wave equation, first-order form (Sec. IV.A): fields
// (phi, Pi, d_x, d_y, d_z) with d_i = partial_i phi,
//   d/dt phi = -Pi,  d/dt Pi = -sum_i D_i d_i,  d/dt d_i = -D_i Pi,
// plus Kreiss-Oliger dissipation on every field (Sec. II.B.1).  The adjoint
// variant applies the transpose on the periodic grid: D_i^T = -D_i,
// Q_d^T = Q_d, so d/dt l_phi = Q l_phi, d/dt l_Pi = -l_phi + sum_i D_i l_d_i,
// d/dt l_d_i = D_i l_Pi.
#pragma once
#include "sf_common.cuh"

namespace sf {

template <typename T, bool ADJ>
__device__ __forceinline__ void wave_point(const PatchArgs<T>& a, const T* __restrict__ u, T v[5],
                                           T r[5]) {
  const long long sf_ = a.sf, sy = a.sy, sz = a.sz;
#pragma unroll
  for (int f = 0; f < 5; ++f) v[f] = __ldg(u + f * sf_);
  const T div = d1(u + 2 * sf_, 1, a.i12h[0]) + d1(u + 3 * sf_, sy, a.i12h[1]) +
                d1(u + 4 * sf_, sz, a.i12h[2]);
  if (!ADJ) {
    r[0] = -v[1];
    r[1] = -div;
    r[2] = -d1(u + sf_, 1, a.i12h[0]);
    r[3] = -d1(u + sf_, sy, a.i12h[1]);
    r[4] = -d1(u + sf_, sz, a.i12h[2]);
  } else {
    r[0] = T(0);
    r[1] = div - v[0];
    r[2] = d1(u + sf_, 1, a.i12h[0]);
    r[3] = d1(u + sf_, sy, a.i12h[1]);
    r[4] = d1(u + sf_, sz, a.i12h[2]);
  }
#pragma unroll
  for (int f = 0; f < 5; ++f) r[f] += ko_all(u + f * sf_, sy, sz, v[f], a.ko);
}

}  // namespace sf
