// Ideal Newtonian MHD (Sec. IV.B), 8 conserved fields
//   U = (rho, S_x, S_y, S_z, E, B^x, B^y, B^z),
// in conservative form L(U)_i = -sum_d (F_{i+1/2} - F_{i-1/2}) / dx_d (Eq. 5).
// Interface fluxes: WENO reconstruction of the evolved fields from the left
// and right (WENO5 with JS or Z weights, App. B; WENO3, App. A), physical
// fluxes of both states and the local Lax-Friedrichs formula (Eq. LLF) with
// the largest fast magnetosonic signal speed of the two states; or, with
// flux_split, the same reconstructions applied to the Lax-Friedrichs split
// fluxes.  Fused with the RK stage update.
#include "sf_internal.cuh"

namespace sf {

template <typename T>
struct MhdCoef {
  T gamma;
  T eps[3];   // WENO epsilon per direction
  T q;        // WENO-Z exponent
  int variant;
  int split;  // 1: reconstruction of the Lax-Friedrichs split fluxes
  T idx[3];   // 1/dx_d
};

template <typename T>
__device__ __forceinline__ T wz_pow(T x, T q) {
  return q == T(2) ? x * x : (q == T(1) ? x : pow(x, q));
}

// App. B smoothness indicators of the three WENO5 stencils of cell c, from
// w[0..4] = U_{c-2..c+2}: beta_0 of cells c..c+2, beta_1 of c-1..c+1, beta_2
// of c-2..c.  They measure the candidate polynomials on cell c, so the
// reconstructions at both edges of the cell use the same three numbers.
template <typename T>
__device__ __forceinline__ void weno5_beta(const T* w, T& be0, T& be1, T& be2) {
  const T a0 = w[2] - T(2) * w[3] + w[4], b0 = T(3) * w[2] - T(4) * w[3] + w[4];
  const T a1 = w[1] - T(2) * w[2] + w[3], b1 = w[1] - w[3];
  const T a2 = w[0] - T(2) * w[1] + w[2], b2 = w[0] - T(4) * w[1] + T(3) * w[2];
  be0 = T(13.0 / 12.0) * a0 * a0 + T(0.25) * b0 * b0;
  be1 = T(13.0 / 12.0) * a1 * a1 + T(0.25) * b1 * b1;
  be2 = T(13.0 / 12.0) * a2 * a2 + T(0.25) * b2 * b2;
}

// App. B nonlinear combination of the candidates c_k of stencils k = 0, 1, 2
// with linear weights g_k and smoothness indicators be_k: JS weights
// g_k / (eps + be_k)^2, or with Z the WENO-Z weights g_k (1 + (tau / (eps +
// be_k))^q), tau = |be_0 - be_2|, normalised by their sum.  In double the
// weights are formed over the common denominator (eps + be_0)^2 (eps + be_1)^2
// (eps + be_2)^2 (WENO-Z for q = 2), which cancels in the normalisation: one
// division instead of four (the products of squares would underflow float on
// fine grids, so float keeps the per-weight divisions).
template <typename T, bool Z>
__device__ __forceinline__ T weno5_combine(T c0, T c1, T c2, T g0, T g1, T g2, T be0, T be1, T be2,
                                           T eps, const MhdCoef<T>& mc) {
  T al0, al1, al2;
  if constexpr (Z) {
    const T tau = fabs(be0 - be2);
    if (sizeof(T) == 8 && mc.q == T(2)) {
      const T e0 = eps + be0, e1 = eps + be1, e2 = eps + be2, t2 = tau * tau;
      const T q0 = e0 * e0, q1 = e1 * e1, q2 = e2 * e2;
      al0 = g0 * (q0 + t2) * (q1 * q2);
      al1 = g1 * (q1 + t2) * (q0 * q2);
      al2 = g2 * (q2 + t2) * (q0 * q1);
    } else {
      al0 = g0 * (T(1) + wz_pow(tau / (eps + be0), mc.q));
      al1 = g1 * (T(1) + wz_pow(tau / (eps + be1), mc.q));
      al2 = g2 * (T(1) + wz_pow(tau / (eps + be2), mc.q));
    }
  } else if constexpr (sizeof(T) == 8) {
    const T e0 = eps + be0, e1 = eps + be1, e2 = eps + be2;
    const T q0 = e0 * e0, q1 = e1 * e1, q2 = e2 * e2;
    al0 = g0 * (q1 * q2);
    al1 = g1 * (q0 * q2);
    al2 = g2 * (q0 * q1);
  } else {
    const T e0 = eps + be0, e1 = eps + be1, e2 = eps + be2;
    al0 = g0 / (e0 * e0);
    al1 = g1 / (e1 * e1);
    al2 = g2 / (e2 * e2);
  }
  return (al0 * c0 + al1 * c1 + al2 * c2) / (al0 + al1 + al2);
}

// App. B: left state at i+1/2 (the right edge of cell i) from w[0..4] =
// U_{i-2..i+2}; Z: WENO-Z weights
template <typename T, bool Z>
__device__ __forceinline__ T weno_left(const T* w, T eps, const MhdCoef<T>& mc) {
  const T c0 = (T(2) * w[2] + T(5) * w[3] - w[4]) * T(1.0 / 6.0);
  const T c1 = (-w[1] + T(5) * w[2] + T(2) * w[3]) * T(1.0 / 6.0);
  const T c2 = (T(2) * w[0] - T(7) * w[1] + T(11) * w[2]) * T(1.0 / 6.0);
  T be0, be1, be2;
  weno5_beta(w, be0, be1, be2);
  return weno5_combine<T, Z>(c0, c1, c2, T(0.3), T(0.6), T(0.1), be0, be1, be2, eps, mc);
}

// App. B: right state at i-1/2 (the left edge of cell i) from w[0..4] =
// U_{i-2..i+2}; Z: WENO-Z weights
template <typename T, bool Z>
__device__ __forceinline__ T weno_right(const T* w, T eps, const MhdCoef<T>& mc) {
  const T c0 = (T(2) * w[4] - T(7) * w[3] + T(11) * w[2]) * T(1.0 / 6.0);
  const T c1 = (-w[3] + T(5) * w[2] + T(2) * w[1]) * T(1.0 / 6.0);
  const T c2 = (T(2) * w[2] + T(5) * w[1] - w[0]) * T(1.0 / 6.0);
  T be0, be1, be2;
  weno5_beta(w, be0, be1, be2);
  return weno5_combine<T, Z>(c0, c1, c2, T(0.1), T(0.6), T(0.3), be0, be1, be2, eps, mc);
}

// Both edge values of cell c from w[0..4] = U_{c-2..c+2} (VAR 0 WENO5-JS,
// 1 WENO5-Z, 2 WENO3): er = the left state at c + 1/2, el = the right state
// at c - 1/2, with the smoothness indicators formed once
template <typename T, int VAR>
__device__ __forceinline__ void weno_edges(const T* w, T eps, const MhdCoef<T>& mc, T& er, T& el);

// App. A: WENO3 left state at i+1/2 from w[1..3] = U_{i-1..i+1}
template <typename T>
__device__ __forceinline__ T weno3_left(const T* w, T eps) {
  const T c0 = T(0.5) * w[2] + T(0.5) * w[3];
  const T c1 = T(-0.5) * w[1] + T(1.5) * w[2];
  const T b0 = (w[3] - w[2]) * (w[3] - w[2]);
  const T b1 = (w[2] - w[1]) * (w[2] - w[1]);
  const T e0 = eps + b0, e1 = eps + b1;
  if constexpr (sizeof(T) == 8) {  // common denominator e0^2 e1^2 (see weno5_combine)
    const T a0 = T(2.0 / 3.0) * (e1 * e1), a1 = T(1.0 / 3.0) * (e0 * e0);
    return (a0 * c0 + a1 * c1) / (a0 + a1);
  }
  const T a0 = T(2.0 / 3.0) / (e0 * e0), a1 = T(1.0 / 3.0) / (e1 * e1);
  return (a0 * c0 + a1 * c1) / (a0 + a1);
}

// App. A: WENO3 right state at i-1/2 from w[1..3] = U_{i-1..i+1}
template <typename T>
__device__ __forceinline__ T weno3_right(const T* w, T eps) {
  const T c0 = T(-0.5) * w[3] + T(1.5) * w[2];
  const T c1 = T(0.5) * w[2] + T(0.5) * w[1];
  const T b0 = (w[2] - w[3]) * (w[2] - w[3]);
  const T b1 = (w[1] - w[2]) * (w[1] - w[2]);
  const T e0 = eps + b0, e1 = eps + b1;
  if constexpr (sizeof(T) == 8) {  // common denominator e0^2 e1^2 (see weno5_combine)
    const T a0 = T(1.0 / 3.0) * (e1 * e1), a1 = T(2.0 / 3.0) * (e0 * e0);
    return (a0 * c0 + a1 * c1) / (a0 + a1);
  }
  const T a0 = T(1.0 / 3.0) / (e0 * e0), a1 = T(2.0 / 3.0) / (e1 * e1);
  return (a0 * c0 + a1 * c1) / (a0 + a1);
}

// one of three values by a direction d that may be known only at run time
// (selects, not an indexed array, so that nothing goes to local memory)
template <typename T>
__device__ __forceinline__ T by_dir(int d, T x, T y, T z) {
  return d == 0 ? x : (d == 1 ? y : z);
}

template <typename T, int VAR>
__device__ __forceinline__ void weno_edges(const T* w, T eps, const MhdCoef<T>& mc, T& er, T& el) {
  if constexpr (VAR == 2) {
    er = weno3_left(w, eps);
    el = weno3_right(w, eps);
  } else {
    T be0, be1, be2;
    weno5_beta(w, be0, be1, be2);
    er = weno5_combine<T, VAR == 1>((T(2) * w[2] + T(5) * w[3] - w[4]) * T(1.0 / 6.0),
                                    (-w[1] + T(5) * w[2] + T(2) * w[3]) * T(1.0 / 6.0),
                                    (T(2) * w[0] - T(7) * w[1] + T(11) * w[2]) * T(1.0 / 6.0), T(0.3),
                                    T(0.6), T(0.1), be0, be1, be2, eps, mc);
    el = weno5_combine<T, VAR == 1>((T(2) * w[4] - T(7) * w[3] + T(11) * w[2]) * T(1.0 / 6.0),
                                    (-w[3] + T(5) * w[2] + T(2) * w[1]) * T(1.0 / 6.0),
                                    (T(2) * w[2] + T(5) * w[1] - w[0]) * T(1.0 / 6.0), T(0.1),
                                    T(0.6), T(0.3), be0, be1, be2, eps, mc);
  }
}

// physical flux along d and the largest signal speed |v_d| + c_fast,d
template <typename T>
__device__ __forceinline__ T flux_speed(const T* q, int d, const MhdCoef<T>& mc, T* F) {
  const T rho = q[0], irho = T(1) / rho;
  const T v[3] = {q[1] * irho, q[2] * irho, q[3] * irho};
  const T B[3] = {q[5], q[6], q[7]};
  const T B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
  const T S2v = q[1] * v[0] + q[2] * v[1] + q[3] * v[2];
  const T pr = (mc.gamma - T(1)) * (q[4] - T(0.5) * S2v - T(0.5) * B2);
  const T ptot = pr + T(0.5) * B2;
  const T vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
  const T vd = by_dir(d, v[0], v[1], v[2]), Bd = by_dir(d, B[0], B[1], B[2]);
  const T Sd = by_dir(d, q[1], q[2], q[3]);
  F[0] = Sd;
#pragma unroll
  for (int a = 0; a < 3; ++a) F[1 + a] = Sd * v[a] - Bd * B[a] + (a == d ? ptot : T(0));
  F[4] = (q[4] + ptot) * vd - vB * Bd;
#pragma unroll
  for (int a = 0; a < 3; ++a) F[5 + a] = vd * B[a] - v[a] * Bd;
  const T a2 = mc.gamma * pr * irho, b2 = B2 * irho, bd2 = Bd * Bd * irho;
  const T s = a2 + b2;
  const T cf2 = T(0.5) * (s + sqrt(s * s - T(4) * a2 * bd2));
  return fabs(vd) + sqrt(cf2);
}

// LLF flux through the face between the cell at p and its +d neighbour;
// VAR: the reconstruction (0 WENO5-JS, 1 WENO5-Z, 2 WENO3)
template <typename T, int VAR>
__device__ __forceinline__ void face_flux(const T* __restrict__ p, long long F, long long s, int d,
                                          const MhdCoef<T>& mc, T* Fout) {
  const T eps = by_dir(d, mc.eps[0], mc.eps[1], mc.eps[2]);
  T UL[8], UR[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    const T* q = p + f * F;
    T w[6];
#pragma unroll
    for (int o = 0; o < 6; ++o) w[o] = __ldg(q + (o - 2) * s);
    if constexpr (VAR == 2) {
      UL[f] = weno3_left(w, eps);
      UR[f] = weno3_right(w + 1, eps);
    } else {
      UL[f] = weno_left<T, VAR == 1>(w, eps, mc);
      UR[f] = weno_right<T, VAR == 1>(w + 1, eps, mc);
    }
  }
  T FL[8], FR[8];
  const T sl = flux_speed(UL, d, mc, FL);
  const T sr = flux_speed(UR, d, mc, FR);
  const T S = sl > sr ? sl : sr;
#pragma unroll
  for (int f = 0; f < 8; ++f) Fout[f] = T(0.5) * (FL[f] + FR[f] - S * (UR[f] - UL[f]));
}

// z-faces of a thread marching up its column (double, reconstruction of the
// evolved fields): the flux at k + 1/2 from the carried right-edge values of
// cell k (er, 8 fields) and both edge values of cell k + 1 (cells k-1 .. k+3
// around p1), whose right-edge values then replace er.  Each cell is
// reconstructed once for both of its edges, its smoothness indicators formed
// once instead of twice.
template <typename T, int VAR>
__device__ __forceinline__ void zface_carry(const T* __restrict__ p1, long long F, long long s,
                                            const MhdCoef<T>& mc, T* er, T* Fout) {
  const T eps = mc.eps[2];
  T UR[8], ERn[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    const T* q = p1 + f * F;
    T w[5];
#pragma unroll
    for (int o = 0; o < 5; ++o) w[o] = __ldg(q + (o - 2) * s);
    weno_edges<T, VAR>(w, eps, mc, ERn[f], UR[f]);
  }
  T FL[8], FR[8];
  const T sl = flux_speed(er, 2, mc, FL);
  const T sr = flux_speed(UR, 2, mc, FR);
  const T S = sl > sr ? sl : sr;
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    Fout[f] = T(0.5) * (FL[f] + FR[f] - S * (UR[f] - er[f]));
    er[f] = ERn[f];
  }
}

// The right-edge values (left state at c + 1/2 along z) of the cell at p, to
// start the carry of zface_carry.
template <typename T, int VAR>
__device__ __forceinline__ void zedge_right(const T* __restrict__ p, long long F, long long s,
                                            const MhdCoef<T>& mc, T* er) {
  const T eps = mc.eps[2];
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    const T* q = p + f * F;
    T w[5];
#pragma unroll
    for (int o = 0; o < 5; ++o) w[o] = __ldg(q + (o - 2) * s);
    if constexpr (VAR == 2)
      er[f] = weno3_left(w, eps);
    else
      er[f] = weno_left<T, VAR == 1>(w, eps, mc);
  }
}

// Flux through the same face from the reconstruction of the split fluxes
// (Sec. II.B.2, Lax-Friedrichs splitting): S = the largest signal speed over
// the six cells p-2..p+3, F+- = (F(U) +- S U)/2 at each cell, F+ reconstructed
// from the left (cells p-2..p+2) plus F- from the right (cells p-1..p+3).
template <typename T, int VAR>
__device__ __forceinline__ void face_flux_split(const T* __restrict__ p, long long F, long long s,
                                                int d, const MhdCoef<T>& mc, T* Fout) {
  const T eps = by_dir(d, mc.eps[0], mc.eps[1], mc.eps[2]);
  T Uc[6][8], Fc[6][8];
  T S = T(0);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
#pragma unroll
    for (int f = 0; f < 8; ++f) Uc[c][f] = __ldg(p + f * F + (c - 2) * s);
    const T sp = flux_speed(Uc[c], d, mc, Fc[c]);
    S = sp > S ? sp : S;
  }
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    T wp[6], wm[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      wp[c] = T(0.5) * (Fc[c][f] + S * Uc[c][f]);
      wm[c] = T(0.5) * (Fc[c][f] - S * Uc[c][f]);
    }
    if constexpr (VAR == 2)
      Fout[f] = weno3_left(wp, eps) + weno3_right(wm + 1, eps);
    else
      Fout[f] = weno_left<T, VAR == 1>(wp, eps, mc) + weno_right<T, VAR == 1>(wm + 1, eps, mc);
  }
}

template <typename T, bool SPLIT, int VAR>
__device__ __forceinline__ void interface_flux(const T* __restrict__ p, long long F, long long s,
                                               int d, const MhdCoef<T>& mc, T* Fout) {
  if constexpr (SPLIT)
    face_flux_split<T, VAR>(p, F, s, d, mc, Fout);
  else
    face_flux<T, VAR>(p, F, s, d, mc, Fout);
}

// Stage kernel.  Each interface flux is evaluated once: a block of 32 x MY
// threads owns 31 x (MY - 1) output cells of a plane (MY = 12 for float
// without flux splitting, 8 otherwise: mhd_rows); thread (tx, ty) evaluates the
// x-face at i - 1/2 and the y-face at j - 1/2 of its column, so the +1/2
// faces of the output cells come from lane tx + 1 (warp shuffle) and row
// ty + 1 (shared memory).  Each thread marches mz planes in z and carries the
// z-face below the current plane in registers (the block also evaluates the
// z-face below its first plane, one face in 3 mz + 1, in a first pass of the
// plane loop that evaluates nothing else, so that the kernel holds one copy
// of the z-face code).  VAR is the reconstruction (0 WENO5-JS, 1 WENO5-Z,
// 2 WENO3), a template argument so that each instance carries one
// reconstruction: the kernel's code is large enough for instruction fetch to
// be its top stall.  mz is chosen per
// launch (mhd_planes_per_block) so that the grid fills whole waves of
// resident blocks.  Faces are only evaluated at positions 0..n along their
// direction, whose WENO stencils (cells p-3..p+2) lie inside the 3-point
// ghost zone.
constexpr int MX = 32;
template <typename T, bool SPLIT>
constexpr int mhd_rows() {
  return sizeof(T) == 4 && !SPLIT ? 12 : 8;
}

// Float without flux splitting: blocks of 32 x 12 threads, 2 resident per SM
// (at most 85 registers a thread, 24 warps per SM), so that 11 of 12 rows
// output cells (7 of 8 with 32 x 8: 2.51e9 against 2.83e9 cell-updates/s at
// 128^3; 32 x 24, one block per SM: 2.82e9; 32 x 8 left to the compiler's
// register choice, 96 a thread and 16 warps per SM, was 15% slower than
// 32 x 8 at 3 blocks per SM).  The other forms keep 32 x 8 and the compiler's
// register choice.
template <typename T, bool SPLIT>
constexpr int mhd_min_blocks() {
  return sizeof(T) == 4 && !SPLIT ? 2 : 1;
}

template <typename T, bool SPLIT, int VAR>
__global__ void __launch_bounds__(MX * mhd_rows<T, SPLIT>(), mhd_min_blocks<T, SPLIT>())
    mhd_stage_kernel(PatchArgs<T> a, StageArgs s, MhdCoef<T> mc, int mz) {
  constexpr int MY = mhd_rows<T, SPLIT>();
  __shared__ T fy[MY][MX][8];
  __shared__ double s_rate[MX * MY / 32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  double rate = 0.0;  // max signal rate of this thread's outputs (fused CFL reduction)
  const int i = blockIdx.x * (MX - 1) + tx;
  const int j = blockIdx.y * (MY - 1) + ty;
  const int k0 = blockIdx.z * mz;
  const int k1 = min(k0 + mz, a.n[2]);
  const int g = a.g;
  const bool out = tx < MX - 1 && ty < MY - 1 && i < a.n[0] && j < a.n[1];
  const bool xface = i <= a.n[0] && j < a.n[1];
  const bool yface = j <= a.n[1] && i < a.n[0];
  auto at = [&](int ii, int jj, int kk) {
    return a.us + (long long)(kk + g) * a.sz + (long long)(jj + g) * a.sy + (ii + g);
  };
  // double without flux splitting: the z-faces by zface_carry (each cell's
  // z reconstruction serves both of its z-faces), er its carried values
  constexpr bool ZC = sizeof(T) == 8 && !SPLIT;
  T Fzm[8], er[8];
  // pass k = k0 - 1 evaluates only the z-face below the first plane (Fzm);
  // `body` is the same for the whole block, so the barriers below are taken
  // by every thread or by none
  for (int k = k0 - 1; k < k1; ++k) {
    const bool body = k >= k0;
    T Fx[8], Fy[8], Fz[8];
    // the x-face at i - 1/2, the y-face at j - 1/2 and the z-face at k + 1/2
    // in one rolled loop over the direction (one copy of the face code); with
    // ZC the z-face comes from zface_carry after the loop
#pragma unroll 1
    for (int d = body ? 0 : 2; d < (ZC ? 2 : 3); ++d) {
      T Fd[8];
      if (d == 0 ? xface : (d == 1 ? yface : out)) {
        const T* base = d == 0 ? at(i - 1, j, k) : (d == 1 ? at(i, j - 1, k) : at(i, j, k));
        interface_flux<T, SPLIT, VAR>(base, a.sf, d == 0 ? 1LL : (d == 1 ? a.sy : a.sz), d, mc, Fd);
      } else {
#pragma unroll
        for (int f = 0; f < 8; ++f) Fd[f] = T(0);
      }
#pragma unroll
      for (int f = 0; f < 8; ++f) {
        Fx[f] = d == 0 ? Fd[f] : Fx[f];
        Fy[f] = d == 1 ? Fd[f] : Fy[f];
        Fz[f] = d == 2 ? Fd[f] : Fz[f];
      }
    }
    if constexpr (ZC) {
      if (out) {
        if (!body) zedge_right<T, VAR>(at(i, j, k), a.sf, a.sz, mc, er);
        zface_carry<T, VAR>(at(i, j, k + 1), a.sf, a.sz, mc, er, Fz);
      }
    }
    if (body) {
#pragma unroll
      for (int f = 0; f < 8; ++f) fy[ty][tx][f] = Fy[f];
    }
    if (!body) {
#pragma unroll
      for (int f = 0; f < 8; ++f) Fzm[f] = Fz[f];
      continue;
    }
    T Fxp[8];
#pragma unroll
    for (int f = 0; f < 8; ++f) Fxp[f] = __shfl_down_sync(0xffffffffu, Fx[f], 1);
    __syncthreads();
    if (out) {
      const long long c = (long long)(k + g) * a.sz + (long long)(j + g) * a.sy + (i + g);
      const Images im = ghost_images(a, s, i, j, k);
      T q[8];
#pragma unroll
      for (int f = 0; f < 8; ++f) {
        T r = T(0);
        r -= (Fxp[f] - Fx[f]) * mc.idx[0];
        r -= (fy[ty + 1][tx][f] - Fy[f]) * mc.idx[1];
        r -= (Fz[f] - Fzm[f]) * mc.idx[2];
        q[f] = write_field(a, s, im, f, c, i, j, k, __ldg(a.us + f * a.sf + c), r);
        Fzm[f] = Fz[f];
      }
      if (a.rate) {
        T Fd[8];
#pragma unroll
        for (int d = 0; d < 3; ++d) rate = fmax(rate, double(flux_speed(q, d, mc, Fd) * mc.idx[d]));
      }
    }
    __syncthreads();
  }
  if (a.rate) {  // block max, then one atomic per block (non-negative doubles order as their bits)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rate = fmax(rate, __shfl_down_sync(0xffffffffu, rate, o));
    const int lin = ty * MX + tx;
    if ((lin & 31) == 0) s_rate[lin >> 5] = rate;
    __syncthreads();
    if (lin == 0) {
      double m = 0.0;
      for (int w = 0; w < MX * MY / 32; ++w) m = fmax(m, s_rate[w]);
      atomicMax(reinterpret_cast<unsigned long long*>(a.rate), (unsigned long long)__double_as_longlong(m));
    }
  }
}

// CFL rate: max over cells and d of (|v_d| + c_fast,d) / dx_d
template <typename T>
__global__ void __launch_bounds__(256) mhd_rate_kernel(const T* __restrict__ u0, int nx, int ny,
                                                       int nz, int g, long long sy, long long sz,
                                                       long long F, MhdCoef<T> mc,
                                                       unsigned long long* out) {
  const long long total = (long long)nx * ny * nz;
  double best = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % nx);
    const int j = (int)((t / nx) % ny);
    const int k = (int)(t / ((long long)nx * ny));
    const T* p = u0 + (long long)(k + g) * sz + (long long)(j + g) * sy + (i + g);
    T q[8], Fd[8];
#pragma unroll
    for (int f = 0; f < 8; ++f) q[f] = __ldg(p + f * F);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double r = double(flux_speed(q, d, mc, Fd)) * double(mc.idx[d]);
      best = r > best ? r : best;
    }
  }
  // block max, then one atomic per block (non-negative doubles order like their bits)
  __shared__ double sm[256];
  sm[threadIdx.x] = best;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(sm[0]));
}

template <typename T>
static MhdCoef<T> coef(const sf_params& prm, const sf_patch& p) {
  MhdCoef<T> mc;
  mc.gamma = T(prm.gamma_eos);
  for (int d = 0; d < 3; ++d) {
    const double h = p.dx[d];
    mc.eps[d] = T(prm.weno_eps > 0 ? prm.weno_eps
                                   : (prm.weno_variant == 2 ? h * h : h * h * h * h));
    mc.idx[d] = T(1.0 / h);
  }
  mc.q = T(prm.weno_q);
  mc.variant = prm.weno_variant;
  mc.split = prm.flux_split;
  return mc;
}

// Planes per block along z: each block evaluates 3 mz + 1 interface fluxes
// per column, and a launch of B blocks takes ceil(B / resident) rounds of
// the resident blocks (blocks per SM x SMs), so mz in [4, 16] minimises
// ceil(B(mz) / resident) (3 mz + 1); ties go to the larger mz.  Only chunk
// lengths whose grid fits gridDim.z (65535) are considered.
static int mhd_planes_per_block(int gx, int gy, int nz, int resident) {
  int best = 16;
  long long best_cost = -1;
  for (int mz = 16; mz >= 4; --mz) {
    if ((nz + mz - 1) / mz > 65535) break;
    const long long blocks = (long long)gx * gy * ((nz + mz - 1) / mz);
    const long long rounds = resident > 0 ? (blocks + resident - 1) / resident : blocks;
    const long long cost = rounds * (3 * mz + 1);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = mz;
    }
  }
  return best;
}

// Resident blocks of the stage kernel instance on the current device
// (blocks per SM x SMs), cached per instance and device; 0 if unknown.
template <typename T, bool SPLIT, int VAR>
static int resident_blocks() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (!cache[dev]) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mhd_stage_kernel<T, SPLIT, VAR>,
                                                      MX * mhd_rows<T, SPLIT>(),
                                                      0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return 0;
    cache[dev] = per_sm * sms;
  }
  return cache[dev];
}

// One launch of the instance for (T, SPLIT, VAR) with its chunk length.
template <typename T, bool SPLIT, int VAR>
static void launch_instance(const PatchArgs<T>& a, const StageArgs& s, const MhdCoef<T>& mc,
                            const sf_patch& p, cudaStream_t st) {
  constexpr int MY = mhd_rows<T, SPLIT>();
  const dim3 block(MX, MY, 1);
  const int gx = (p.n[0] + MX - 2) / (MX - 1), gy = (p.n[1] + MY - 2) / (MY - 1);
  const int mz = mhd_planes_per_block(gx, gy, p.n[2], resident_blocks<T, SPLIT, VAR>());
  const dim3 grid(gx, gy, (p.n[2] + mz - 1) / mz);
  mhd_stage_kernel<T, SPLIT, VAR><<<grid, block, 0, st>>>(a, s, mc, mz);
}

template <typename T, bool SPLIT>
static void launch_variant(const PatchArgs<T>& a, const StageArgs& s, const MhdCoef<T>& mc,
                           const sf_patch& p, cudaStream_t st) {
  if (mc.variant == 1)
    launch_instance<T, SPLIT, 1>(a, s, mc, p, st);
  else if (mc.variant == 2)
    launch_instance<T, SPLIT, 2>(a, s, mc, p, st);
  else
    launch_instance<T, SPLIT, 0>(a, s, mc, p, st);
}

template <typename T>
static sf_status launch(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                        void* rhs_out, cudaStream_t st) {
  PatchArgs<T> a = make_args<T>(prm, p, stage, 8, rhs_out);
  const int last = prm.rk == SF_RK4 ? 3 : 2;
  if (p.cfl_rate && !rhs_out && stage == last) {
    if (cudaMemsetAsync(p.cfl_rate, 0, sizeof(double), st) != cudaSuccess)
      return set_error(SF_ECUDA, "reset of cfl_rate failed");
    a.rate = p.cfl_rate;
  }
  const MhdCoef<T> mc = coef<T>(prm, p);
  if (prm.flux_split)
    launch_variant<T, true>(a, s, mc, p, st);
  else
    launch_variant<T, false>(a, s, mc, p, st);
  return after_launch("mhd_stage_kernel");
}

sf_status launch_mhd(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                     void* rhs_out, cudaStream_t st) {
  if (p.precision == SF_FP64) return launch<double>(prm, p, s, stage, rhs_out, st);
  return launch<float>(prm, p, s, stage, rhs_out, st);
}

}  // namespace sf

using namespace sf;

extern "C" sf_status sf_mhd_max_rate(const sf_params* prm, const sf_patch* patch,
                                     const void* array, double* d_rate, void* stream) {
  if (!patch || !array || !d_rate) return set_error(SF_EINVAL, "NULL argument");
  sf_patch p = *patch;
  normalise_strides(p, 8);
  p.u_stage = const_cast<void*>(array);
  sf_status e = check_patch(prm, p, 0, 0);
  if (e) return e;
  if (p.system != SF_MHD) return set_error(SF_EINVAL, "sf_mhd_max_rate needs an SF_MHD patch");
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_rate, 0, sizeof(double), st) != cudaSuccess)
    return set_error(SF_ECUDA, "memset of d_rate failed");
  const long long total = (long long)p.n[0] * p.n[1] * p.n[2];
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (p.precision == SF_FP64)
    mhd_rate_kernel<double><<<blocks, 256, 0, st>>>((const double*)array, p.n[0], p.n[1], p.n[2],
                                                    p.ghost, p.sy, p.sz, p.sf, coef<double>(*prm, p),
                                                    (unsigned long long*)d_rate);
  else
    mhd_rate_kernel<float><<<blocks, 256, 0, st>>>((const float*)array, p.n[0], p.n[1], p.n[2],
                                                   p.ghost, p.sy, p.sz, p.sf, coef<float>(*prm, p),
                                                   (unsigned long long*)d_rate);
  return after_launch("mhd_rate_kernel");
}
