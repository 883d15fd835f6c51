// FP64 CPU oracle for the method-of-lines substep of arXiv:1806.04182.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference against
// which the CUDA path is checked.  Only the tests, the smoke check and the
// CPU-baseline leg of the benchmark may load it; the product path never does.
// It shares no code, header or constant table with the CUDA library.
//
// Everything is written as the paper states it, cell by cell, with no
// blocking, fusion or reordering:
//   * semi-discrete system dU/dt = L(U) + Q_d(U)                  Sec. II.A, Eq. (2)
//   * 4th-order centred D_i, D_ii, D_ij = D_j D_i                 Sec. II.B.1
//   * 6th-order Kreiss-Oliger dissipation Q_d                     Sec. II.B.1
//   * WENO5 (JS and Z) reconstruction of the evolved fields       Sec. II.B.2, App. B
//   * local Lax-Friedrichs interface flux, conservative form      Sec. II.B.2, Eq. (LLF), Eq. (5)
//   * RK(4,4) and SSP-RK(3,3)                                     Sec. II.C, App. C/D
//   * scalar wave equation (first-order reduction)                Sec. IV.A
//   * ideal Newtonian MHD (+ optional GLM cleaning field psi)     Sec. IV.B
//   * CCZ4 + Bona-Masso slicing + Gamma-driver shift (vacuum)     Sec. V
//
// Array layout (all arrays double): a "ghosted" array holds nf fields, each a
// box of (nz+2g) x (ny+2g) x (nx+2g) points, x fastest.  Interior point
// (i,j,k), 0 <= i < nx, sits at x offset i+g.  RHS outputs are interior-only
// arrays nf x nz x ny x nx.
//
// Parity status per function is stated in oracle/__init__.py.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {
typedef struct {
  double sigma;       // KO strength (Sec. II.B.1)
  double gamma_eos;   // ideal-gas adiabatic index (Sec. IV.B)
  double weno_eps;    // WENO epsilon; <= 0 means dx_d^4 (WENO5, App. B) or dx_d^2 (WENO3, App. A)
  double weno_q;      // WENO-Z exponent q (App. B)
  double kappa_z;     // Z4 damping (Sec. V)
  double kappa_c;     // conformal-constraint damping (Sec. V)
  double eta;         // Gamma-driver damping (Sec. V)
  double g_shift;     // Gamma-driver coefficient g (Sec. V)
  double ch;          // GLM cleaning speed (Sec. IV.B)
  double kappa_psi;   // GLM damping (Sec. IV.B)
  int32_t weno_variant;  // 0: WENO5-JS, 1: WENO5-Z, 2: WENO3 (App. A)
  int32_t slicing;       // 0: 1+log (f = 2/alpha), 1: harmonic (f = 1)
  int32_t shift_frozen;  // 1: d/dt beta = d/dt B = 0
  int32_t mhd_glm;       // 1: 9th MHD field psi
  int32_t lopsided;      // 1: CCZ4 advection beta^k d_k with the one-sided stencils (Sec. II.B.1)
  int32_t flux_split;    // 1: MHD reconstruction of the split fluxes (Lax-Friedrichs splitting)
} or_params;
}

namespace {

// ---------------------------------------------------------------- counting
// A scalar that counts its floating-point operations.  Instantiating the
// per-cell functions with it gives the algorithmic FLOP count of one cell.
struct OpCount { long add, mul, div, sqrt_, log_, cmp; };
static OpCount g_ops;

struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
};
inline Cnt operator+(Cnt a, Cnt b) { g_ops.add++; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { g_ops.add++; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { g_ops.mul++; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { g_ops.div++; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline Cnt& operator*=(Cnt& a, Cnt b) { a = a * b; return a; }
inline Cnt sqrt_(Cnt a) { g_ops.sqrt_++; return Cnt(std::sqrt(a.v)); }
inline Cnt log_(Cnt a) { g_ops.log_++; return Cnt(std::log(a.v)); }
inline Cnt fabs_(Cnt a) { return Cnt(std::fabs(a.v)); }
inline Cnt max_(Cnt a, Cnt b) { g_ops.cmp++; return Cnt(a.v > b.v ? a.v : b.v); }
inline Cnt pow_(Cnt a, double q) {
  // q in {1, 2} is all the method uses (WENO-Z); count it as multiplies.
  if (q == 1.0) return a;
  if (q == 2.0) return a * a;
  g_ops.log_++; g_ops.mul++;
  return Cnt(std::pow(a.v, q));
}
inline double val_(Cnt a) { return a.v; }

inline double sqrt_(double a) { return std::sqrt(a); }
inline double log_(double a) { return std::log(a); }
inline double fabs_(double a) { return std::fabs(a); }
inline double max_(double a, double b) { return a > b ? a : b; }
inline double pow_(double a, double q) { return q == 2.0 ? a * a : std::pow(a, q); }
inline double val_(double a) { return a; }

// ---------------------------------------------------------------- grid
struct Grid {
  int n[3];
  int g;
  long N[3];
  long sy, sz, sf;
  long ninterior;
  Grid(const int* n_, int g_) : g(g_) {
    for (int d = 0; d < 3; ++d) { n[d] = n_[d]; N[d] = n_[d] + 2L * g_; }
    sy = N[0];
    sz = N[0] * N[1];
    sf = N[0] * N[1] * N[2];
    ninterior = (long)n[0] * n[1] * n[2];
  }
  // ghosted offset of interior coordinates (i,j,k), each may be in [-g, n+g)
  long at(int f, int i, int j, int k) const {
    return f * sf + (long)(k + g) * sz + (long)(j + g) * sy + (i + g);
  }
  long out(int f, int i, int j, int k) const {
    return f * ninterior + ((long)k * n[1] + j) * n[0] + i;
  }
};

inline void step_(int d, int s, int& i, int& j, int& k) {
  if (d == 0) i += s; else if (d == 1) j += s; else k += s;
}

template <class T>
inline T U_(const double* u, const Grid& G, int f, int i, int j, int k) {
  return T(u[G.at(f, i, j, k)]);
}

template <class T>
inline T U_off(const double* u, const Grid& G, int f, int i, int j, int k, int d, int s) {
  step_(d, s, i, j, k);
  return U_<T>(u, G, f, i, j, k);
}

// Sec. II.B.1: D_d U = (U_{-2} - 8 U_{-1} + 8 U_{+1} - U_{+2}) / (12 dx_d)
template <class T>
T D1(const double* u, const Grid& G, int f, int i, int j, int k, int d, const double* dx) {
  T um2 = U_off<T>(u, G, f, i, j, k, d, -2);
  T um1 = U_off<T>(u, G, f, i, j, k, d, -1);
  T up1 = U_off<T>(u, G, f, i, j, k, d, +1);
  T up2 = U_off<T>(u, G, f, i, j, k, d, +2);
  return (um2 - T(8.0) * um1 + T(8.0) * up1 - up2) * T(1.0 / (12.0 * dx[d]));
}

// Sec. II.B.1: D_dd U = (-U_{-2} + 16 U_{-1} - 30 U_0 + 16 U_{+1} - U_{+2}) / (12 dx_d^2)
template <class T>
T D2(const double* u, const Grid& G, int f, int i, int j, int k, int d, const double* dx) {
  T um2 = U_off<T>(u, G, f, i, j, k, d, -2);
  T um1 = U_off<T>(u, G, f, i, j, k, d, -1);
  T u0 = U_<T>(u, G, f, i, j, k);
  T up1 = U_off<T>(u, G, f, i, j, k, d, +1);
  T up2 = U_off<T>(u, G, f, i, j, k, d, +2);
  return (-um2 + T(16.0) * um1 - T(30.0) * u0 + T(16.0) * up1 - up2) *
         T(1.0 / (12.0 * dx[d] * dx[d]));
}

// Sec. II.B.1: mixed derivative D_{d1 d2} U = D_{d2}( D_{d1} U ), d1 != d2
template <class T>
T Dmix(const double* u, const Grid& G, int f, int i, int j, int k, int d1, int d2,
       const double* dx) {
  const double c[5] = {1.0, -8.0, 0.0, 8.0, -1.0};
  T acc(0.0);
  for (int s = -2; s <= 2; ++s) {
    if (s == 0) continue;
    int ii = i, jj = j, kk = k;
    step_(d2, s, ii, jj, kk);
    acc = acc + T(c[s + 2]) * D1<T>(u, G, f, ii, jj, kk, d1, dx);
  }
  return acc * T(1.0 / (12.0 * dx[d2]));
}

// Sec. II.B.1: one-sided ("lopsided") advection derivative along d for an
// advecting velocity of sign `sgn`:
//   beta > 0: ( U_{+3} - 6 U_{+2} + 18 U_{+1} - 10 U_0 - 3 U_{-1}) / (12 dx_d)
//   beta < 0: (-U_{-3} + 6 U_{-2} - 18 U_{-1} + 10 U_0 + 3 U_{+1}) / (12 dx_d)
template <class T>
T Dlop(const double* u, const Grid& G, int f, int i, int j, int k, int d, double sgn,
       const double* dx) {
  T u0 = U_<T>(u, G, f, i, j, k);
  if (sgn > 0) {
    T a = U_off<T>(u, G, f, i, j, k, d, 3), b = U_off<T>(u, G, f, i, j, k, d, 2);
    T c = U_off<T>(u, G, f, i, j, k, d, 1), e = U_off<T>(u, G, f, i, j, k, d, -1);
    return (a - T(6.0) * b + T(18.0) * c - T(10.0) * u0 - T(3.0) * e) * T(1.0 / (12.0 * dx[d]));
  }
  T a = U_off<T>(u, G, f, i, j, k, d, -3), b = U_off<T>(u, G, f, i, j, k, d, -2);
  T c = U_off<T>(u, G, f, i, j, k, d, -1), e = U_off<T>(u, G, f, i, j, k, d, 1);
  return (-a + T(6.0) * b - T(18.0) * c + T(10.0) * u0 + T(3.0) * e) * T(1.0 / (12.0 * dx[d]));
}

// Sec. II.B.1: Q_d U = sum_d sigma/(64 dx_d) (U_{-3} - 6U_{-2} + 15U_{-1} - 20U_0 + 15U_{+1} - 6U_{+2} + U_{+3})
template <class T>
T KO(const double* u, const Grid& G, int f, int i, int j, int k, const double* dx, double sigma) {
  const double c[7] = {1.0, -6.0, 15.0, -20.0, 15.0, -6.0, 1.0};
  T total(0.0);
  for (int d = 0; d < 3; ++d) {
    T s(0.0);
    for (int o = -3; o <= 3; ++o) s = s + T(c[o + 3]) * U_off<T>(u, G, f, i, j, k, d, o);
    total = total + T(sigma / (64.0 * dx[d])) * s;
  }
  return total;
}

// ---------------------------------------------------------------- wave
// Sec. IV.A in first-order form: fields (phi, Pi, d_x, d_y, d_z) with
// d_i = partial_i phi, so dphi/dt = -Pi, dPi/dt = -sum_i D_i d_i,
// dd_i/dt = -D_i Pi; KO on every field.
template <class T>
void wave_cell(const or_params& p, const double* u, const Grid& G, const double* dx, int i, int j,
               int k, T rhs[5]) {
  T Pi = U_<T>(u, G, 1, i, j, k);
  T divd = D1<T>(u, G, 2, i, j, k, 0, dx) + D1<T>(u, G, 3, i, j, k, 1, dx) +
           D1<T>(u, G, 4, i, j, k, 2, dx);
  rhs[0] = -Pi;
  rhs[1] = -divd;
  for (int d = 0; d < 3; ++d) rhs[2 + d] = -D1<T>(u, G, 1, i, j, k, d, dx);
  for (int f = 0; f < 5; ++f) rhs[f] = rhs[f] + KO<T>(u, G, f, i, j, k, dx, p.sigma);
}

// Transpose L^T of the wave operator above on a periodic grid, acting on the
// adjoint fields lambda = (l_phi, l_Pi, l_d).  Uses D_i^T = -D_i (the centred
// stencil is antisymmetric) and Q_d^T = Q_d (symmetric stencil).
template <class T>
void wave_adj_cell(const or_params& p, const double* u, const Grid& G, const double* dx, int i,
                   int j, int k, T rhs[5]) {
  T lphi = U_<T>(u, G, 0, i, j, k);
  T divl = D1<T>(u, G, 2, i, j, k, 0, dx) + D1<T>(u, G, 3, i, j, k, 1, dx) +
           D1<T>(u, G, 4, i, j, k, 2, dx);
  rhs[0] = T(0.0);
  rhs[1] = -lphi + divl;
  for (int d = 0; d < 3; ++d) rhs[2 + d] = D1<T>(u, G, 1, i, j, k, d, dx);
  for (int f = 0; f < 5; ++f) rhs[f] = rhs[f] + KO<T>(u, G, f, i, j, k, dx, p.sigma);
}

// ---------------------------------------------------------------- MHD
// Sec. IV.B.  Conserved U = (rho, S_x, S_y, S_z, E, B^x, B^y, B^z [, psi]).
enum { MH_RHO = 0, MH_S = 1, MH_E = 4, MH_B = 5, MH_PSI = 8 };

template <class T>
T mhd_pressure(const or_params& p, const T* q) {
  T rho = q[MH_RHO];
  T S2 = q[MH_S] * q[MH_S] + q[MH_S + 1] * q[MH_S + 1] + q[MH_S + 2] * q[MH_S + 2];
  T B2 = q[MH_B] * q[MH_B] + q[MH_B + 1] * q[MH_B + 1] + q[MH_B + 2] * q[MH_B + 2];
  // E = rho v^2/2 + rho eps + B^2/2, p = (Gamma-1) rho eps
  T rhoeps = q[MH_E] - T(0.5) * S2 / rho - T(0.5) * B2;
  return T(p.gamma_eos - 1.0) * rhoeps;
}

// Physical flux F^d(U), Sec. IV.B.
template <class T>
void mhd_flux(const or_params& p, const T* q, int d, int nf, T* F) {
  T rho = q[MH_RHO];
  T v[3], B[3];
  for (int a = 0; a < 3; ++a) { v[a] = q[MH_S + a] / rho; B[a] = q[MH_B + a]; }
  T B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
  T pr = mhd_pressure<T>(p, q);
  T ptot = pr + T(0.5) * B2;
  T vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
  F[MH_RHO] = rho * v[d];
  for (int a = 0; a < 3; ++a) {
    F[MH_S + a] = rho * v[d] * v[a] - B[d] * B[a];
    if (a == d) F[MH_S + a] = F[MH_S + a] + ptot;
  }
  F[MH_E] = (q[MH_E] + ptot) * v[d] - vB * B[d];
  for (int a = 0; a < 3; ++a) F[MH_B + a] = v[d] * B[a] - v[a] * B[d];
  if (nf == 9) {
    F[MH_B + d] = F[MH_B + d] + q[MH_PSI];
    F[MH_PSI] = T(p.ch * p.ch) * B[d];
  }
}

// Largest characteristic speed along d: |v_d| + c_fast,d (standard ideal-MHD
// fast magnetosonic speed; with GLM the cleaning speed c_h bounds it too).
template <class T>
T mhd_speed(const or_params& p, const T* q, int d, int nf) {
  T rho = q[MH_RHO];
  T vd = q[MH_S + d] / rho;
  T B2 = q[MH_B] * q[MH_B] + q[MH_B + 1] * q[MH_B + 1] + q[MH_B + 2] * q[MH_B + 2];
  T pr = mhd_pressure<T>(p, q);
  T a2 = T(p.gamma_eos) * pr / rho;
  T b2 = B2 / rho;
  T bd2 = q[MH_B + d] * q[MH_B + d] / rho;
  T s = a2 + b2;
  T cf2 = T(0.5) * (s + sqrt_(s * s - T(4.0) * a2 * bd2));
  T sp = fabs_(vd) + sqrt_(cf2);
  if (nf == 9) sp = max_(sp, T(p.ch));
  return sp;
}

// App. B: WENO5 left state U^L_{i+1/2} from U_{i-2..i+2} (w[0..4]).
template <class T>
T weno5_left(const or_params& p, const T* w, double eps) {
  const T& um2 = w[0]; const T& um1 = w[1]; const T& u0 = w[2]; const T& up1 = w[3]; const T& up2 = w[4];
  T c0 = T(2.0 / 6.0) * u0 + T(5.0 / 6.0) * up1 - T(1.0 / 6.0) * up2;
  T c1 = T(-1.0 / 6.0) * um1 + T(5.0 / 6.0) * u0 + T(2.0 / 6.0) * up1;
  T c2 = T(2.0 / 6.0) * um2 - T(7.0 / 6.0) * um1 + T(11.0 / 6.0) * u0;
  T a0 = u0 - T(2.0) * up1 + up2, b0 = T(3.0) * u0 - T(4.0) * up1 + up2;
  T a1 = um1 - T(2.0) * u0 + up1, b1 = um1 - up1;
  T a2 = um2 - T(2.0) * um1 + u0, b2 = um2 - T(4.0) * um1 + T(3.0) * u0;
  T be0 = T(13.0 / 12.0) * a0 * a0 + T(0.25) * b0 * b0;
  T be1 = T(13.0 / 12.0) * a1 * a1 + T(0.25) * b1 * b1;
  T be2 = T(13.0 / 12.0) * a2 * a2 + T(0.25) * b2 * b2;
  const double d[3] = {3.0 / 10.0, 6.0 / 10.0, 1.0 / 10.0};
  T be[3] = {be0, be1, be2};
  T al[3];
  if (p.weno_variant == 1) {
    T tau = fabs_(be0 - be2);
    for (int r = 0; r < 3; ++r) al[r] = T(d[r]) * (T(1.0) + pow_(tau / (T(eps) + be[r]), p.weno_q));
  } else {
    for (int r = 0; r < 3; ++r) { T e = T(eps) + be[r]; al[r] = T(d[r]) / (e * e); }
  }
  T sum = al[0] + al[1] + al[2];
  return (al[0] * c0 + al[1] * c1 + al[2] * c2) / sum;
}

// App. B: WENO5 right state U^R_{i-1/2} from U_{i-2..i+2} (w[0..4]).
template <class T>
T weno5_right(const or_params& p, const T* w, double eps) {
  const T& um2 = w[0]; const T& um1 = w[1]; const T& u0 = w[2]; const T& up1 = w[3]; const T& up2 = w[4];
  T c0 = T(2.0 / 6.0) * up2 - T(7.0 / 6.0) * up1 + T(11.0 / 6.0) * u0;
  T c1 = T(-1.0 / 6.0) * up1 + T(5.0 / 6.0) * u0 + T(2.0 / 6.0) * um1;
  T c2 = T(2.0 / 6.0) * u0 + T(5.0 / 6.0) * um1 - T(1.0 / 6.0) * um2;
  T a0 = up2 - T(2.0) * up1 + u0, b0 = up2 - T(4.0) * up1 + T(3.0) * u0;
  T a1 = up1 - T(2.0) * u0 + um1, b1 = up1 - um1;
  T a2 = u0 - T(2.0) * um1 + um2, b2 = T(3.0) * u0 - T(4.0) * um1 + um2;
  T be0 = T(13.0 / 12.0) * a0 * a0 + T(0.25) * b0 * b0;
  T be1 = T(13.0 / 12.0) * a1 * a1 + T(0.25) * b1 * b1;
  T be2 = T(13.0 / 12.0) * a2 * a2 + T(0.25) * b2 * b2;
  const double d[3] = {1.0 / 10.0, 6.0 / 10.0, 3.0 / 10.0};  // d~_r = d_{k-1-r}
  T be[3] = {be0, be1, be2};
  T al[3];
  if (p.weno_variant == 1) {
    T tau = fabs_(be0 - be2);
    for (int r = 0; r < 3; ++r) al[r] = T(d[r]) * (T(1.0) + pow_(tau / (T(eps) + be[r]), p.weno_q));
  } else {
    for (int r = 0; r < 3; ++r) { T e = T(eps) + be[r]; al[r] = T(d[r]) / (e * e); }
  }
  T sum = al[0] + al[1] + al[2];
  return (al[0] * c0 + al[1] * c1 + al[2] * c2) / sum;
}

// App. A: WENO3 left state U^L_{i+1/2} from U_{i-1..i+1} (w[1..3] of w[0..4]).
template <class T>
T weno3_left(const T* w, double eps) {
  const T& um1 = w[1]; const T& u0 = w[2]; const T& up1 = w[3];
  T c0 = T(0.5) * u0 + T(0.5) * up1;
  T c1 = T(-0.5) * um1 + T(1.5) * u0;
  T b0 = (up1 - u0) * (up1 - u0);
  T b1 = (u0 - um1) * (u0 - um1);
  T e0 = T(eps) + b0, e1 = T(eps) + b1;
  T a0 = T(2.0 / 3.0) / (e0 * e0), a1 = T(1.0 / 3.0) / (e1 * e1);
  return (a0 * c0 + a1 * c1) / (a0 + a1);
}

// App. A: WENO3 right state U^R_{i-1/2} from U_{i-1..i+1}.
template <class T>
T weno3_right(const T* w, double eps) {
  const T& um1 = w[1]; const T& u0 = w[2]; const T& up1 = w[3];
  T c0 = T(-0.5) * up1 + T(1.5) * u0;
  T c1 = T(0.5) * u0 + T(0.5) * um1;
  T b0 = (u0 - up1) * (u0 - up1);
  T b1 = (um1 - u0) * (um1 - u0);
  T e0 = T(eps) + b0, e1 = T(eps) + b1;
  T a0 = T(1.0 / 3.0) / (e0 * e0), a1 = T(2.0 / 3.0) / (e1 * e1);
  return (a0 * c0 + a1 * c1) / (a0 + a1);
}

// Flux at the interface x_{i+1/2} along d.
//  flux_split = 0 (the paper's tests): WENO left state (stencil centred at i)
//    and right state (centred at i+1) of the evolved fields, then the LLF
//    formula (Eq. LLF).
//  flux_split = 1: reconstruction of the fluxes (Sec. II.B.2 lists it as the
//    alternative to reconstructing the fields), in Lax-Friedrichs splitting
//    form: S = the largest signal speed |v_d| + c_f over the six cells
//    i-2..i+3 of the stencil, F^(+-)_c = (F(U_c) +- S U_c)/2 at each cell,
//    F_{i+1/2} = F^+ reconstructed from the left + F^- from the right.
template <class T>
void mhd_interface_flux(const or_params& p, const double* u, const Grid& G, const double* dx,
                        int nf, int i, int j, int k, int d, T* Fout) {
  double eps = p.weno_eps > 0 ? p.weno_eps
                              : (p.weno_variant == 2 ? dx[d] * dx[d] : dx[d] * dx[d] * dx[d] * dx[d]);
  if (p.flux_split) {
    T Uc[6][9], Fc[6][9];
    T S = T(0.0);
    for (int c = 0; c < 6; ++c) {
      for (int f = 0; f < nf; ++f) Uc[c][f] = U_off<T>(u, G, f, i, j, k, d, c - 2);
      mhd_flux<T>(p, Uc[c], d, nf, Fc[c]);
      S = max_(S, mhd_speed<T>(p, Uc[c], d, nf));
    }
    for (int f = 0; f < nf; ++f) {
      T wp[5], wm[5];
      for (int c = 0; c < 5; ++c) {
        wp[c] = T(0.5) * (Fc[c][f] + S * Uc[c][f]);          // cells i-2..i+2
        wm[c] = T(0.5) * (Fc[c + 1][f] - S * Uc[c + 1][f]);  // cells i-1..i+3
      }
      if (p.weno_variant == 2)
        Fout[f] = weno3_left<T>(wp, eps) + weno3_right<T>(wm, eps);
      else
        Fout[f] = weno5_left<T>(p, wp, eps) + weno5_right<T>(p, wm, eps);
    }
    return;
  }
  T UL[9], UR[9];
  for (int f = 0; f < nf; ++f) {
    T wl[5], wr[5];
    for (int s = -2; s <= 2; ++s) {
      wl[s + 2] = U_off<T>(u, G, f, i, j, k, d, s);
      wr[s + 2] = U_off<T>(u, G, f, i, j, k, d, s + 1);
    }
    if (p.weno_variant == 2) {
      UL[f] = weno3_left<T>(wl, eps);
      UR[f] = weno3_right<T>(wr, eps);
    } else {
      UL[f] = weno5_left<T>(p, wl, eps);
      UR[f] = weno5_right<T>(p, wr, eps);
    }
  }
  T FL[9], FR[9];
  mhd_flux<T>(p, UL, d, nf, FL);
  mhd_flux<T>(p, UR, d, nf, FR);
  T S = max_(mhd_speed<T>(p, UL, d, nf), mhd_speed<T>(p, UR, d, nf));
  for (int f = 0; f < nf; ++f) Fout[f] = T(0.5) * (FL[f] + FR[f] - S * (UR[f] - UL[f]));
}

// Eq. (5): L(U)_i = -sum_d (F_{i+1/2} - F_{i-1/2}) / dx_d  (+ GLM source).
template <class T>
void mhd_cell(const or_params& p, const double* u, const Grid& G, const double* dx, int nf,
              int i, int j, int k, T* rhs) {
  for (int f = 0; f < nf; ++f) rhs[f] = T(0.0);
  for (int d = 0; d < 3; ++d) {
    T Fp[9], Fm[9];
    mhd_interface_flux<T>(p, u, G, dx, nf, i, j, k, d, Fp);
    int ii = i, jj = j, kk = k;
    step_(d, -1, ii, jj, kk);
    mhd_interface_flux<T>(p, u, G, dx, nf, ii, jj, kk, d, Fm);
    for (int f = 0; f < nf; ++f) rhs[f] = rhs[f] - (Fp[f] - Fm[f]) * T(1.0 / dx[d]);
  }
  if (nf == 9) rhs[MH_PSI] = rhs[MH_PSI] - T(p.kappa_psi) * U_<T>(u, G, MH_PSI, i, j, k);
}

// ---------------------------------------------------------------- CCZ4
// Field order: 0 chi | 1-6 gt_xx,xy,xz,yy,yz,zz | 7 Khat | 8-13 At_ij |
// 14-16 Gammahat^i | 17 Theta | 18 alpha | 19-21 beta^i | 22-24 B^i
enum { Z_CHI = 0, Z_GT = 1, Z_KH = 7, Z_AT = 8, Z_GH = 14, Z_TH = 17, Z_AL = 18, Z_BE = 19,
       Z_B = 22, Z_NF = 25 };
static const int SYM[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

template <class T>
void z4_cell(const or_params& p, const double* u, const Grid& G, const double* dx, int i, int j,
             int k, T rhs[Z_NF]) {
  // --- fields
  T chi = U_<T>(u, G, Z_CHI, i, j, k);
  T gt[3][3], At[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      gt[a][b] = U_<T>(u, G, Z_GT + SYM[a][b], i, j, k);
      At[a][b] = U_<T>(u, G, Z_AT + SYM[a][b], i, j, k);
    }
  T Kh = U_<T>(u, G, Z_KH, i, j, k);
  T Th = U_<T>(u, G, Z_TH, i, j, k);
  T al = U_<T>(u, G, Z_AL, i, j, k);
  T Gh[3], be[3], Bv[3];
  for (int a = 0; a < 3; ++a) {
    Gh[a] = U_<T>(u, G, Z_GH + a, i, j, k);
    be[a] = U_<T>(u, G, Z_BE + a, i, j, k);
    Bv[a] = U_<T>(u, G, Z_B + a, i, j, k);
  }

  // --- first derivatives d1[f][c] = D_c U_f of all 25 fields
  T d1[Z_NF][3];
  for (int f = 0; f < Z_NF; ++f)
    for (int c = 0; c < 3; ++c) d1[f][c] = D1<T>(u, G, f, i, j, k, c, dx);
  T dchi[3], dgt[3][3][3], dKh[3], dGh[3][3], dTh[3], dal[3], dbe[3][3];
  for (int c = 0; c < 3; ++c) {
    dchi[c] = d1[Z_CHI][c];
    dKh[c] = d1[Z_KH][c];
    dTh[c] = d1[Z_TH][c];
    dal[c] = d1[Z_AL][c];
    for (int a = 0; a < 3; ++a) {
      dGh[a][c] = d1[Z_GH + a][c];  // partial_c Gammahat^a
      dbe[a][c] = d1[Z_BE + a][c];  // partial_c beta^a
      for (int b = 0; b < 3; ++b) dgt[a][b][c] = d1[Z_GT + SYM[a][b]][c];
    }
  }

  // --- second derivatives of chi, gt_ij, alpha, beta^i (D_cc and D_ce = D_e D_c)
  auto dd = [&](int f, int c, int e) -> T {
    if (c == e) return D2<T>(u, G, f, i, j, k, c, dx);
    int lo = c < e ? c : e, hi = c < e ? e : c;
    return Dmix<T>(u, G, f, i, j, k, lo, hi, dx);
  };
  T ddchi[3][3], ddal[3][3], ddgt[3][3][3][3], ddbe[3][3][3];
  for (int c = 0; c < 3; ++c)
    for (int e = c; e < 3; ++e) {
      ddchi[c][e] = ddchi[e][c] = dd(Z_CHI, c, e);
      ddal[c][e] = ddal[e][c] = dd(Z_AL, c, e);
      for (int a = 0; a < 3; ++a) {
        ddbe[a][c][e] = ddbe[a][e][c] = dd(Z_BE + a, c, e);
        for (int b = a; b < 3; ++b) {
          T v = dd(Z_GT + SYM[a][b], c, e);
          ddgt[a][b][c][e] = ddgt[a][b][e][c] = ddgt[b][a][c][e] = ddgt[b][a][e][c] = v;
        }
      }
    }

  // --- conformal metric: determinant, inverse, ln det
  T det = gt[0][0] * (gt[1][1] * gt[2][2] - gt[1][2] * gt[1][2]) -
          gt[0][1] * (gt[0][1] * gt[2][2] - gt[1][2] * gt[0][2]) +
          gt[0][2] * (gt[0][1] * gt[1][2] - gt[1][1] * gt[0][2]);
  T idet = T(1.0) / det;
  T ig[3][3];
  ig[0][0] = (gt[1][1] * gt[2][2] - gt[1][2] * gt[1][2]) * idet;
  ig[0][1] = (gt[0][2] * gt[1][2] - gt[0][1] * gt[2][2]) * idet;
  ig[0][2] = (gt[0][1] * gt[1][2] - gt[0][2] * gt[1][1]) * idet;
  ig[1][1] = (gt[0][0] * gt[2][2] - gt[0][2] * gt[0][2]) * idet;
  ig[1][2] = (gt[0][1] * gt[0][2] - gt[0][0] * gt[1][2]) * idet;
  ig[2][2] = (gt[0][0] * gt[1][1] - gt[0][1] * gt[0][1]) * idet;
  ig[1][0] = ig[0][1]; ig[2][0] = ig[0][2]; ig[2][1] = ig[1][2];
  T lndet = log_(det);

  // --- Christoffel symbols: first kind Gl[a][b][c] = Gamma~_{abc} (first
  // index lowered) = 1/2 (d_b gt_ac + d_c gt_ab - d_a gt_bc); second kind
  // Gu[a][b][c] = Gamma~^a_{bc}; contracted Gt[a] = gt^{bc} Gamma~^a_{bc}.
  T Gl[3][3][3], Gu[3][3][3], Gt[3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c)
        Gl[a][b][c] = T(0.5) * (dgt[a][c][b] + dgt[a][b][c] - dgt[b][c][a]);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) {
        T s(0.0);
        for (int l = 0; l < 3; ++l) s = s + ig[a][l] * Gl[l][b][c];
        Gu[a][b][c] = s;
      }
  for (int a = 0; a < 3; ++a) {
    T s(0.0);
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) s = s + ig[b][c] * Gu[a][b][c];
    Gt[a] = s;
  }
  // Z^i = chi/2 (Gammahat^i - Gamma~^i), from Gammahat^i = Gamma~^i + 2 Z^i / chi
  T Z[3];
  for (int a = 0; a < 3; ++a) Z[a] = T(0.5) * chi * (Gh[a] - Gt[a]);

  // --- Ricci: Rhat_ij (conformal part) + Rchi_ij
  T Rt[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      T t1(0.0);
      for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n) t1 = t1 + ig[m][n] * ddgt[a][b][m][n];
      T t2(0.0);
      for (int c = 0; c < 3; ++c) t2 = t2 + gt[c][a] * dGh[c][b] + gt[c][b] * dGh[c][a];
      T t3(0.0);
      for (int c = 0; c < 3; ++c) t3 = t3 + Gh[c] * (Gl[a][b][c] + Gl[b][a][c]);
      T t4(0.0);
      for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n) {
          T s(0.0);
          for (int c = 0; c < 3; ++c)
            s = s + Gu[c][m][a] * Gl[b][c][n] + Gu[c][m][b] * Gl[a][c][n] + Gu[c][m][a] * Gl[c][n][b];
          t4 = t4 + ig[m][n] * s;
        }
      T Rhat = T(-0.5) * t1 + T(0.5) * t2 + T(0.5) * t3 + t4;

      T s1(0.0);
      for (int c = 0; c < 3; ++c) s1 = s1 + Gu[c][a][b] * dchi[c];
      T s2(0.0);
      for (int c = 0; c < 3; ++c) s2 = s2 + Z[c] * (gt[c][a] * dchi[b] + gt[c][b] * dchi[a]);
      T s3(0.0);
      for (int c = 0; c < 3; ++c)
        for (int m = 0; m < 3; ++m)
          s3 = s3 + ig[c][m] * (ddchi[c][m] - T(1.5) / chi * dchi[c] * dchi[m]);
      T s4(0.0);
      for (int c = 0; c < 3; ++c) s4 = s4 + Gh[c] * dchi[c];
      T Rchi = ddchi[a][b] / (T(2.0) * chi) - s1 / (T(2.0) * chi) -
               dchi[a] * dchi[b] / (T(4.0) * chi * chi) + T(2.0) / (chi * chi) * T(0.5) * s2 +
               gt[a][b] / (T(2.0) * chi) * (s3 - s4);
      Rt[a][b] = Rhat + Rchi;
    }
  // R + 2 nabla_i Z^i = gamma^{ij} (Rhat_ij + Rchi_ij), gamma^{ij} = chi gt^{ij}
  T RZ(0.0);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) RZ = RZ + ig[a][b] * Rt[a][b];
  RZ = chi * RZ;

  // --- nabla_i nabla_j alpha and its trace
  T gdadc(0.0);
  for (int c = 0; c < 3; ++c)
    for (int m = 0; m < 3; ++m) gdadc = gdadc + ig[c][m] * dal[c] * dchi[m];
  T DDal[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      T s(0.0);
      for (int c = 0; c < 3; ++c) s = s + Gu[c][a][b] * dal[c];
      DDal[a][b] = ddal[a][b] - s +
                   T(1.0) / (T(2.0) * chi) * (dal[a] * dchi[b] + dal[b] * dchi[a] - gt[a][b] * gdadc);
    }
  T LapAl(0.0);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) LapAl = LapAl + ig[a][b] * DDal[a][b];
  LapAl = chi * LapAl;

  // --- A~ contractions
  T trA(0.0);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) trA = trA + ig[a][b] * At[a][b];
  T Aud[3][3];  // A~^a_b = gt^{ac} A~_cb
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      T s(0.0);
      for (int c = 0; c < 3; ++c) s = s + ig[a][c] * At[c][b];
      Aud[a][b] = s;
    }
  T Auu[3][3];  // A~^{ab} = gt^{ac} gt^{bd} A~_cd
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      T s(0.0);
      for (int c = 0; c < 3; ++c)
        for (int e = 0; e < 3; ++e) s = s + ig[a][c] * ig[b][e] * At[c][e];
      Auu[a][b] = s;
    }
  T AA(0.0);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) AA = AA + At[a][b] * Auu[a][b];

  T divbe = dbe[0][0] + dbe[1][1] + dbe[2][2];
  // advection beta^k d_k U_f: centred D_k, or the one-sided stencil chosen by the sign of beta^k
  auto adv = [&](int f) -> T {
    if (!p.lopsided) return be[0] * d1[f][0] + be[1] * d1[f][1] + be[2] * d1[f][2];
    T s(0.0);
    for (int c = 0; c < 3; ++c) {
      const double b = val_(be[c]);
      if (b != 0.0) s = s + be[c] * Dlop<T>(u, G, f, i, j, k, c, b, dx);
    }
    return s;
  };
  const T kz(p.kappa_z), kc(p.kappa_c);

  // --- d/dt gt_ij  (Eq. syseq1)
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) {
      T s(0.0);
      for (int c = 0; c < 3; ++c) s = s + gt[a][c] * dbe[c][b] + gt[c][b] * dbe[c][a];
      rhs[Z_GT + SYM[a][b]] = adv(Z_GT + SYM[a][b]) + s - T(2.0 / 3.0) * gt[a][b] * divbe -
                              T(2.0) * al * (At[a][b] - T(1.0 / 3.0) * gt[a][b] * trA) -
                              kc / T(3.0) * al * gt[a][b] * lndet;
    }

  // --- d/dt A~_ij
  T M[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) M[a][b] = al * Rt[a][b] - DDal[a][b];
  T trM(0.0);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) trM = trM + ig[a][b] * M[a][b];
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) {
      T s(0.0);
      for (int c = 0; c < 3; ++c) s = s + At[a][c] * dbe[c][b] + At[c][b] * dbe[c][a];
      T AAd(0.0);
      for (int c = 0; c < 3; ++c) AAd = AAd + At[a][c] * Aud[c][b];
      T MTF = M[a][b] - T(1.0 / 3.0) * gt[a][b] * trM;
      rhs[Z_AT + SYM[a][b]] = adv(Z_AT + SYM[a][b]) + s - T(2.0 / 3.0) * At[a][b] * divbe -
                              kc / T(3.0) * al * gt[a][b] * trA + chi * MTF +
                              al * (Kh * At[a][b] - T(2.0) * AAd);
    }

  // --- d/dt chi
  rhs[Z_CHI] = adv(Z_CHI) + T(2.0 / 3.0) * chi * (al * (Kh + T(2.0) * Th) - divbe);

  // --- d/dt Khat
  T Zdal = Z[0] * dal[0] + Z[1] * dal[1] + Z[2] * dal[2];
  T Kt = Kh + T(2.0) * Th;
  rhs[Z_KH] = adv(Z_KH) - LapAl + al * (T(1.0 / 3.0) * Kt * Kt + AA + kz * Th) + T(2.0) * Zdal;

  // --- d/dt Theta
  rhs[Z_TH] = adv(Z_TH) +
              T(0.5) * al * (RZ + T(2.0 / 3.0) * Kh * Kh + T(2.0 / 3.0) * Th * (Kh - T(2.0) * Th) - AA) -
              Zdal - al * (T(2.0) * kz * Th);

  // --- d/dt Gammahat^i  (Eq. syseq2)
  T rGh[3];
  for (int a = 0; a < 3; ++a) {
    T s1(0.0);
    for (int b = 0; b < 3; ++b) s1 = s1 + Gh[b] * dbe[a][b];
    T s2(0.0);
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) s2 = s2 + ig[b][c] * ddbe[a][b][c];
    T s3(0.0);
    for (int b = 0; b < 3; ++b) {
      T ddiv = ddbe[0][b][0] + ddbe[1][b][1] + ddbe[2][b][2];  // partial_b partial_k beta^k
      s3 = s3 + ig[a][b] * ddiv;
    }
    T s4(0.0);
    for (int b = 0; b < 3; ++b) s4 = s4 + Auu[a][b] * dal[b];
    T s5(0.0);
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) s5 = s5 + Gu[a][b][c] * Auu[b][c];
    T s6(0.0);
    for (int b = 0; b < 3; ++b) s6 = s6 + Auu[a][b] * dchi[b];
    T s7(0.0);
    for (int b = 0; b < 3; ++b) s7 = s7 + ig[a][b] * dKh[b];
    T s8(0.0);
    for (int b = 0; b < 3; ++b) s8 = s8 + ig[a][b] * (T(1.0 / 3.0) * dTh[b] + Th / al * dal[b]);
    rGh[a] = -s1 + T(2.0 / 3.0) * Gh[a] * divbe + s2 + T(1.0 / 3.0) * s3 - T(2.0) * s4 +
             T(2.0) * al * (s5 - T(1.5) / chi * s6 - T(2.0 / 3.0) * s7) +
             T(2.0) * al * (-s8 - T(1.0) / chi * Z[a] * (kz + T(2.0 / 3.0) * Kt));
    rhs[Z_GH + a] = adv(Z_GH + a) + rGh[a];
  }

  // --- gauge: Bona-Masso slicing, Gamma-driver shift
  T f = p.slicing == 0 ? T(2.0) / al : T(1.0);
  rhs[Z_AL] = adv(Z_AL) - al * al * f * Kh;
  for (int a = 0; a < 3; ++a) {
    if (p.shift_frozen) {
      rhs[Z_BE + a] = T(0.0);
      rhs[Z_B + a] = T(0.0);
    } else {
      rhs[Z_BE + a] = adv(Z_BE + a) + T(p.g_shift) * Bv[a];
      // d/dt B^i = beta^j d_j B^i - eta B^i + d/dt Gammahat^i - beta^j d_j Gammahat^i
      rhs[Z_B + a] = adv(Z_B + a) - T(p.eta) * Bv[a] + rGh[a];
    }
  }

  // --- Kreiss-Oliger dissipation on every evolved field
  for (int fld = 0; fld < Z_NF; ++fld) {
    if (p.shift_frozen && fld >= Z_BE) continue;
    rhs[fld] = rhs[fld] + KO<T>(u, G, fld, i, j, k, dx, p.sigma);
  }
}

int nfields(int system, const or_params& p) {
  switch (system) {
    case 0: return 5;
    case 1: return p.mhd_glm ? 9 : 8;
    case 2: return Z_NF;
    case 3: return 5;
  }
  return -1;
}

template <class T>
void cell_rhs(int system, const or_params& p, const double* u, const Grid& G, const double* dx,
              int i, int j, int k, T* r) {
  switch (system) {
    case 0: wave_cell<T>(p, u, G, dx, i, j, k, r); break;
    case 1: mhd_cell<T>(p, u, G, dx, nfields(1, p), i, j, k, r); break;
    case 2: z4_cell<T>(p, u, G, dx, i, j, k, r); break;
    case 3: wave_adj_cell<T>(p, u, G, dx, i, j, k, r); break;
  }
}

void rhs_all(int system, const or_params& p, const Grid& G, const double* dx, const double* u,
             double* out) {
  int nf = nfields(system, p);
  // rows (k, j) are independent: parallel over both, so that a thin slab
  // still gives every host core work
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        double r[32];
        cell_rhs<double>(system, p, u, G, dx, i, j, k, r);
        for (int f = 0; f < nf; ++f) out[G.out(f, i, j, k)] = r[f];
      }
}

// ---------------------------------------------------------------- radiative boundaries
// Sec. V: radiative (outgoing-wave) boundary condition.  A field behaving as
// U = U_inf + f(r - v t)/r near the boundary obeys
//   dU/dt = -v x^i/r d_i U - v (U - U_inf)/r,
// with x the physical position of the point and r = |x|.  It is applied at
// every ghost point of a non-periodic patch, whose values are then evolved by
// the RK stages like the interior.  d_i is the centred 4th-order D_i where the
// ghosted array holds two points on both sides of the point, and a 4th-order
// one-sided stencil leaning into the array elsewhere:
//   one point behind:  (-3 U_{-1} - 10 U_0 + 18 U_{+1} - 6 U_{+2} + U_{+3}) / (12 h),
//   none behind:       (-25 U_0 + 48 U_{+1} - 36 U_{+2} + 16 U_{+3} - 3 U_{+4}) / (12 h),
// and their mirror images at the upper end.
static double rad_deriv(const double* u, const Grid& G, int f, int i, int j, int k, int d,
                        const double* dx) {
  const int ig = (d == 0 ? i : (d == 1 ? j : k)) + G.g;
  const long N = G.N[d];
  auto U = [&](int s) { return U_off<double>(u, G, f, i, j, k, d, s); };
  const double h12 = 12.0 * dx[d];
  if (ig >= 2 && ig <= N - 3) return (U(-2) - 8.0 * U(-1) + 8.0 * U(1) - U(2)) / h12;
  if (ig == 1) return (-3.0 * U(-1) - 10.0 * U(0) + 18.0 * U(1) - 6.0 * U(2) + U(3)) / h12;
  if (ig == 0) return (-25.0 * U(0) + 48.0 * U(1) - 36.0 * U(2) + 16.0 * U(3) - 3.0 * U(4)) / h12;
  if (ig == N - 2) return (3.0 * U(1) + 10.0 * U(0) - 18.0 * U(-1) + 6.0 * U(-2) - U(-3)) / h12;
  return (25.0 * U(0) - 48.0 * U(-1) + 36.0 * U(-2) - 16.0 * U(-3) + 3.0 * U(-4)) / h12;
}

static double rad_rhs_point(const double* u, const Grid& G, int f, int i, int j, int k,
                            const double* dx, const double* x0, double uinf, double v) {
  const double x[3] = {x0[0] + i * dx[0], x0[1] + j * dx[1], x0[2] + k * dx[2]};
  const double r = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  if (r == 0.0) return 0.0;
  double xdu = 0.0;
  for (int d = 0; d < 3; ++d) xdu += x[d] * rad_deriv(u, G, f, i, j, k, d, dx);
  return -v * xdu / r - v * (u[G.at(f, i, j, k)] - uinf) / r;
}

static bool is_ghost(const Grid& G, int i, int j, int k) {
  return !(i >= 0 && i < G.n[0] && j >= 0 && j < G.n[1] && k >= 0 && k < G.n[2]);
}

void fill_ghosts(int nf, const Grid& G, double* u) {
  // periodic: ghost (i,j,k) takes the value of interior ((i mod n), ...)
  for (int f = 0; f < nf; ++f)
    for (int k = -G.g; k < G.n[2] + G.g; ++k)
      for (int j = -G.g; j < G.n[1] + G.g; ++j)
        for (int i = -G.g; i < G.n[0] + G.g; ++i) {
          bool interior = i >= 0 && i < G.n[0] && j >= 0 && j < G.n[1] && k >= 0 && k < G.n[2];
          if (interior) continue;
          int ii = ((i % G.n[0]) + G.n[0]) % G.n[0];
          int jj = ((j % G.n[1]) + G.n[1]) % G.n[1];
          int kk = ((k % G.n[2]) + G.n[2]) % G.n[2];
          u[G.at(f, i, j, k)] = u[G.at(f, ii, jj, kk)];
        }
}

// Y_interior = X_interior + a * K  (K interior-only), then periodic ghosts.
void axpy_interior(int nf, const Grid& G, const double* X, double a, const double* K, double* Y) {
  for (int f = 0; f < nf; ++f)
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i)
          Y[G.at(f, i, j, k)] = X[G.at(f, i, j, k)] + a * K[G.out(f, i, j, k)];
  fill_ghosts(nf, G, Y);
}

void copy_interior_out(int nf, const Grid& G, const double* X, double* out) {
  for (int f = 0; f < nf; ++f)
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i) out[G.out(f, i, j, k)] = X[G.at(f, i, j, k)];
}

}  // namespace

extern "C" {

int or_nfields(int system, const or_params* p) { return nfields(system, *p); }

// Threads of the parallel sweeps (OpenMP); 1 when built without OpenMP.
void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_fill_ghosts_periodic(int nf, const int* n, int g, double* u) {
  Grid G(n, g);
  fill_ghosts(nf, G, u);
}

// L(U) + Q_d(U) on the interior of a ghost-filled array.
int or_rhs(int system, const or_params* p, const int* n, int g, const double* dx, const double* u,
           double* rhs) {
  if (nfields(system, *p) < 0 || g < 3) return 1;
  Grid G(n, g);
  rhs_all(system, *p, G, dx, u, rhs);
  return 0;
}

// One RK(4,4) step in the form of Sec. II.C:
//   U(1) = U^n, U(2) = U^n + k1/2, U(3) = U^n + k2/2, U(4) = U^n + k3,
//   U^{n+1} = U^n + (k1 + 2 k2 + 2 k3 + k4)/6,  k_j = dt (L + Q_d)(U(j)).
// U is ghosted and updated in place (ghosts refilled periodically).  If
// `stages` is non-null it receives U(2), U(3), U(4), U^{n+1} (interior-only).
int or_rk4_step(int system, const or_params* p, const int* n, int g, const double* dx, double dt,
                double* U, double* stages) {
  int nf = nfields(system, *p);
  if (nf < 0 || g < 3) return 1;
  Grid G(n, g);
  size_t tot = (size_t)nf * G.sf, inn = (size_t)nf * G.ninterior;
  std::vector<double> Us(tot), k1(inn), k2(inn), k3(inn), k4(inn);
  fill_ghosts(nf, G, U);
  rhs_all(system, *p, G, dx, U, k1.data());
  for (auto& v : k1) v *= dt;
  axpy_interior(nf, G, U, 0.5, k1.data(), Us.data());
  if (stages) copy_interior_out(nf, G, Us.data(), stages + 0 * inn);
  rhs_all(system, *p, G, dx, Us.data(), k2.data());
  for (auto& v : k2) v *= dt;
  axpy_interior(nf, G, U, 0.5, k2.data(), Us.data());
  if (stages) copy_interior_out(nf, G, Us.data(), stages + 1 * inn);
  rhs_all(system, *p, G, dx, Us.data(), k3.data());
  for (auto& v : k3) v *= dt;
  axpy_interior(nf, G, U, 1.0, k3.data(), Us.data());
  if (stages) copy_interior_out(nf, G, Us.data(), stages + 2 * inn);
  rhs_all(system, *p, G, dx, Us.data(), k4.data());
  for (auto& v : k4) v *= dt;
  for (int f = 0; f < nf; ++f)
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i) {
          long o = G.out(f, i, j, k);
          U[G.at(f, i, j, k)] += (k1[o] + 2.0 * k2[o] + 2.0 * k3[o] + k4[o]) / 6.0;
        }
  fill_ghosts(nf, G, U);
  if (stages) copy_interior_out(nf, G, U, stages + 3 * inn);
  return 0;
}

// One SSP-RK(3,3) step in the k-form of App. D (with the weights read so
// that they sum to one and agree with App. C's b_j(1) = (1/6, 1/6, 4/6)):
//   U(1) = U^n, U(2) = U^n + k1, U(3) = U^n + k1/4 + k2/4,
//   U^{n+1} = U^n + (k1 + k2 + 4 k3)/6.
// `stages` (optional) receives U(2), U(3), U^{n+1}.
int or_ssprk3_step(int system, const or_params* p, const int* n, int g, const double* dx,
                   double dt, double* U, double* stages) {
  int nf = nfields(system, *p);
  if (nf < 0 || g < 3) return 1;
  Grid G(n, g);
  size_t tot = (size_t)nf * G.sf, inn = (size_t)nf * G.ninterior;
  std::vector<double> Us(tot), k1(inn), k2(inn), k3(inn);
  fill_ghosts(nf, G, U);
  rhs_all(system, *p, G, dx, U, k1.data());
  for (auto& v : k1) v *= dt;
  axpy_interior(nf, G, U, 1.0, k1.data(), Us.data());
  if (stages) copy_interior_out(nf, G, Us.data(), stages + 0 * inn);
  rhs_all(system, *p, G, dx, Us.data(), k2.data());
  for (auto& v : k2) v *= dt;
  for (int f = 0; f < nf; ++f)
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i) {
          long o = G.out(f, i, j, k);
          Us[G.at(f, i, j, k)] = U[G.at(f, i, j, k)] + 0.25 * k1[o] + 0.25 * k2[o];
        }
  fill_ghosts(nf, G, Us.data());
  if (stages) copy_interior_out(nf, G, Us.data(), stages + 1 * inn);
  rhs_all(system, *p, G, dx, Us.data(), k3.data());
  for (auto& v : k3) v *= dt;
  for (int f = 0; f < nf; ++f)
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i) {
          long o = G.out(f, i, j, k);
          U[G.at(f, i, j, k)] += (k1[o] + k2[o] + 4.0 * k3[o]) / 6.0;
        }
  fill_ghosts(nf, G, U);
  if (stages) copy_interior_out(nf, G, U, stages + 2 * inn);
  return 0;
}

// CFL rate of the MHD system (Sec. II.A footnote): max over interior cells
// and directions of (|v_d| + c_fast,d) / dx_d.  dt = cfl / rate.
double or_mhd_max_rate(const or_params* p, const int* n, int g, const double* dx, const double* u) {
  Grid G(n, g);
  int nf = nfields(1, *p);
  double best = 0.0;
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        double q[9];
        for (int f = 0; f < nf; ++f) q[f] = u[G.at(f, i, j, k)];
        for (int d = 0; d < 3; ++d) best = std::max(best, mhd_speed<double>(*p, q, d, nf) / dx[d]);
      }
  return best;
}

// Wave energy E = 1/2 sum_cells (Pi^2 + |d|^2) dx dy dz.
double or_wave_energy(const int* n, int g, const double* dx, const double* u) {
  Grid G(n, g);
  double e = 0.0;
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i)
        for (int f = 1; f < 5; ++f) {
          double v = u[G.at(f, i, j, k)];
          e += 0.5 * v * v;
        }
  return e * dx[0] * dx[1] * dx[2];
}

// Z4 constraint monitors (root mean square over interior cells):
// out[0] = Theta, out[1] = |Z| with Z^i = chi/2 (Gammahat^i - Gamma~^i),
// out[2] = ln det gt, out[3] = tr A~ = gt^{ij} A~_ij.
void or_z4_monitors(const int* n, int g, const double* dx, const double* u, double* out) {
  Grid G(n, g);
  double s[4] = {0, 0, 0, 0};
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        double gt[3][3], At[3][3], dgt[3][3][3];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            gt[a][b] = u[G.at(Z_GT + SYM[a][b], i, j, k)];
            At[a][b] = u[G.at(Z_AT + SYM[a][b], i, j, k)];
            for (int c = 0; c < 3; ++c) dgt[a][b][c] = D1<double>(u, G, Z_GT + SYM[a][b], i, j, k, c, dx);
          }
        double det = gt[0][0] * (gt[1][1] * gt[2][2] - gt[1][2] * gt[1][2]) -
                     gt[0][1] * (gt[0][1] * gt[2][2] - gt[1][2] * gt[0][2]) +
                     gt[0][2] * (gt[0][1] * gt[1][2] - gt[1][1] * gt[0][2]);
        double ig[3][3];
        ig[0][0] = (gt[1][1] * gt[2][2] - gt[1][2] * gt[1][2]) / det;
        ig[0][1] = (gt[0][2] * gt[1][2] - gt[0][1] * gt[2][2]) / det;
        ig[0][2] = (gt[0][1] * gt[1][2] - gt[0][2] * gt[1][1]) / det;
        ig[1][1] = (gt[0][0] * gt[2][2] - gt[0][2] * gt[0][2]) / det;
        ig[1][2] = (gt[0][1] * gt[0][2] - gt[0][0] * gt[1][2]) / det;
        ig[2][2] = (gt[0][0] * gt[1][1] - gt[0][1] * gt[0][1]) / det;
        ig[1][0] = ig[0][1]; ig[2][0] = ig[0][2]; ig[2][1] = ig[1][2];
        double chi = u[G.at(Z_CHI, i, j, k)];
        double Z2 = 0.0;
        for (int a = 0; a < 3; ++a) {
          double Gt = 0.0;
          for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c)
              for (int l = 0; l < 3; ++l)
                Gt += ig[b][c] * ig[a][l] * 0.5 * (dgt[l][c][b] + dgt[l][b][c] - dgt[b][c][l]);
          double Za = 0.5 * chi * (u[G.at(Z_GH + a, i, j, k)] - Gt);
          Z2 += Za * Za;
        }
        double trA = 0.0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) trA += ig[a][b] * At[a][b];
        double Th = u[G.at(Z_TH, i, j, k)];
        double ld = std::log(det);
        s[0] += Th * Th;
        s[1] += Z2;
        s[2] += ld * ld;
        s[3] += trA * trA;
      }
  for (int q = 0; q < 4; ++q) out[q] = std::sqrt(s[q] / (double)G.ninterior);
}

// Gradient of the observer misfit J = 1/2 sum_{n=1..N} sum_o (phi^n(x_o) - ref[n-1][o])^2
// of the RK4 wave evolution with respect to the initial data (phi0, Pi0),
// where the initial state is (phi0, Pi0, D_x phi0, D_y phi0, D_z phi0).
// Discrete adjoint: lambda <- S^T (lambda + e_n) from n = N down to 1, with
// S^T = P(dt L^T) applied as one RK4 step of the transposed operator, then
// g_phi = lambda_phi + sum_i D_i^T lambda_{d_i} = lambda_phi - sum_i D_i lambda_{d_i},
// g_Pi = lambda_Pi.  phi0, Pi0, g_phi, g_Pi: interior arrays nz x ny x nx.
// obs: interior linear indices (k*ny + j)*nx + i.  Returns J.
double or_wave_misfit_gradient(const or_params* p, const int* n, const double* dx, double dt,
                               int nsteps, const double* phi0, const double* Pi0, int nobs,
                               const int64_t* obs, const double* ref, double* g_phi,
                               double* g_Pi) {
  const int g = 3;
  Grid G(n, g);
  size_t tot = 5 * (size_t)G.sf;
  std::vector<double> U(tot, 0.0);
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        long o = G.out(0, i, j, k);
        U[G.at(0, i, j, k)] = phi0[o];
        U[G.at(1, i, j, k)] = Pi0[o];
      }
  fill_ghosts(5, G, U.data());
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i)
        for (int d = 0; d < 3; ++d) U[G.at(2 + d, i, j, k)] = D1<double>(U.data(), G, 0, i, j, k, d, dx);
  fill_ghosts(5, G, U.data());

  auto obs_at = [&](const double* A, int f, int64_t lin) {
    int i = (int)(lin % G.n[0]);
    int j = (int)((lin / G.n[0]) % G.n[1]);
    int k = (int)(lin / ((int64_t)G.n[0] * G.n[1]));
    return G.at(f, i, j, k);
  };
  std::vector<double> res((size_t)nsteps * nobs);
  double J = 0.0;
  for (int s = 0; s < nsteps; ++s) {
    or_rk4_step(0, p, n, g, dx, dt, U.data(), nullptr);
    for (int o = 0; o < nobs; ++o) {
      double r = U[obs_at(U.data(), 0, obs[o])] - ref[(size_t)s * nobs + o];
      res[(size_t)s * nobs + o] = r;
      J += 0.5 * r * r;
    }
  }
  std::vector<double> L(tot, 0.0);
  for (int s = nsteps - 1; s >= 0; --s) {
    for (int o = 0; o < nobs; ++o) L[obs_at(L.data(), 0, obs[o])] += res[(size_t)s * nobs + o];
    or_rk4_step(3, p, n, g, dx, dt, L.data(), nullptr);
  }
  fill_ghosts(5, G, L.data());
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        long o = G.out(0, i, j, k);
        double s = L[G.at(0, i, j, k)];
        for (int d = 0; d < 3; ++d) s -= D1<double>(L.data(), G, 2 + d, i, j, k, d, dx);
        g_phi[o] = s;
        g_Pi[o] = L[G.at(1, i, j, k)];
      }
  return J;
}

// (L + Q_d)(U) at `npts` interior points given as linear indices
// (k*ny + j)*nx + i; out[f*npts + q].  For sampled checks of large grids.
int or_rhs_points(int system, const or_params* p, const int* n, int g, const double* dx,
                  const double* u, int npts, const int64_t* pts, double* out) {
  int nf = nfields(system, *p);
  if (nf < 0 || g < 3) return 1;
  Grid G(n, g);
#pragma omp parallel for schedule(static)
  for (int q = 0; q < npts; ++q) {
    int64_t lin = pts[q];
    int i = (int)(lin % G.n[0]);
    int j = (int)((lin / G.n[0]) % G.n[1]);
    int k = (int)(lin / ((int64_t)G.n[0] * G.n[1]));
    double r[32];
    cell_rhs<double>(system, *p, u, G, dx, i, j, k, r);
    for (int f = 0; f < nf; ++f) out[(size_t)f * npts + q] = r[f];
  }
  return 0;
}

// Sec. III.A prolongation: 6-point (5th-order) Lagrange interpolation in each
// direction, p(x) = sum_j U_j l_j(x), l_j(x) = prod_{m != j} (x - x_m)/(x_j - x_m),
// applied as a tensor product.  Fine point F (fine index, where fine index
// R*i sits on coarse interior point i) has coarse coordinate X = F/R; the
// nodes are the coarse points floor(X)-2 .. floor(X)+3.  `cu` is a ghost-filled
// coarse array (nf fields, interior n, ghost g); `out` is a dense array
// nf x ext[2] x ext[1] x ext[0] of the fine points origin .. origin+ext-1.
int or_prolong(int nf, const int* n, int g, const double* cu, int ratio, const int* origin,
               const int* ext, double* out) {
  Grid G(n, g);
  auto weights = [&](long F, int& base, double w[6]) {
    // floor division for negative fine indices
    long q = F >= 0 ? F / ratio : -((-F + ratio - 1) / ratio);
    base = (int)q;
    const double X = (double)F / (double)ratio;
    for (int j = 0; j < 6; ++j) {
      const double xj = (double)(base - 2 + j);
      double l = 1.0;
      for (int m = 0; m < 6; ++m) {
        if (m == j) continue;
        const double xm = (double)(base - 2 + m);
        l *= (X - xm) / (xj - xm);
      }
      w[j] = l;
    }
  };
  for (int k = 0; k < ext[2]; ++k)
    for (int jj = 0; jj < ext[1]; ++jj)
      for (int i = 0; i < ext[0]; ++i) {
        int bx, by, bz;
        double wx[6], wy[6], wz[6];
        weights(origin[0] + i, bx, wx);
        weights(origin[1] + jj, by, wy);
        weights(origin[2] + k, bz, wz);
        for (int a = 0; a < 3; ++a) {
          const int b = a == 0 ? bx : (a == 1 ? by : bz);
          if (b - 2 < -g || b + 3 > n[a] + g - 1) return 1;  // stencil leaves the coarse box
        }
        for (int f = 0; f < nf; ++f) {
          double acc = 0.0;
          for (int c = 0; c < 6; ++c)
            for (int bq = 0; bq < 6; ++bq)
              for (int a = 0; a < 6; ++a)
                acc += wz[c] * wy[bq] * wx[a] *
                       cu[G.at(f, bx - 2 + a, by - 2 + bq, bz - 2 + c)];
          out[(((long)f * ext[2] + k) * ext[1] + jj) * ext[0] + i] = acc;
        }
      }
  return 0;
}

// Sec. III.A restriction by injection: coarse interior point i takes the fine
// value at fine interior point R*i.  Coarse points origin .. origin+ext-1 are
// written into the dense array `out` (nf x ext).
int or_restrict(int nf, const int* nfine, int gf, const double* fu, int ratio, const int* origin,
                const int* ext, double* out) {
  Grid G(nfine, gf);
  for (int f = 0; f < nf; ++f)
    for (int k = 0; k < ext[2]; ++k)
      for (int j = 0; j < ext[1]; ++j)
        for (int i = 0; i < ext[0]; ++i) {
          const int I = ratio * (origin[0] + i), J = ratio * (origin[1] + j),
                    K = ratio * (origin[2] + k);
          if (I < -gf || I >= nfine[0] + gf || J < -gf || J >= nfine[1] + gf || K < -gf ||
              K >= nfine[2] + gf)
            return 1;
          out[(((long)f * ext[2] + k) * ext[1] + j) * ext[0] + i] = fu[G.at(f, I, J, K)];
        }
  return 0;
}

// One WENO reconstruction (Sec. II.B.2, App. A, App. B) of the five values
// w[0..4] = U_{i-2..i+2}: side 0 gives U^L_{i+1/2}, side 1 gives U^R_{i-1/2};
// variant as in or_params (0 JS, 1 Z, 2 WENO3 on w[1..3]).
double or_weno(int variant, int side, const double* w, double eps, double q) {
  or_params p;
  std::memset(&p, 0, sizeof(p));
  p.weno_variant = variant;
  p.weno_q = q;
  if (variant == 2) return side == 0 ? weno3_left<double>(w, eps) : weno3_right<double>(w, eps);
  return side == 0 ? weno5_left<double>(p, w, eps) : weno5_right<double>(p, w, eps);
}

// Radiative right-hand side (Sec. V) at every ghost point of the ghosted
// array u (nf fields); out has u's layout and receives it at ghost points
// (interior points are left untouched).  x0 = physical position of interior
// point (0,0,0); uinf, v = per-field value at infinity and speed.
int or_radiative_rhs(int nf, const int* n, int g, const double* dx, const double* x0,
                     const double* u, const double* uinf, const double* v, double* out) {
  if (g < 3 || nf < 1) return 1;
  Grid G(n, g);
  for (int d = 0; d < 3; ++d)
    if (G.N[d] < 7) return 1;
  for (int f = 0; f < nf; ++f)
    for (int k = -g; k < n[2] + g; ++k)
      for (int j = -g; j < n[1] + g; ++j)
        for (int i = -g; i < n[0] + g; ++i)
          if (is_ghost(G, i, j, k))
            out[G.at(f, i, j, k)] = rad_rhs_point(u, G, f, i, j, k, dx, x0, uinf[f], v[f]);
  return 0;
}

// One RK(4,4) step (Sec. II.C) of a non-periodic patch whose ghost points
// evolve under the radiative condition: interior k_j = dt (L + Q_d)(U(j)),
// ghost k_j = dt (radiative RHS)(U(j)); the stage inputs are formed at every
// point.  U is ghosted and updated in place; `stages` (optional) receives the
// ghosted U(2), U(3), U(4), U^{n+1}.
int or_rk4_step_radiative(int system, const or_params* p, const int* n, int g, const double* dx,
                          const double* x0, const double* uinf, const double* v, double dt,
                          double* U, double* stages) {
  const int nf = nfields(system, *p);
  if (nf < 0 || g < 3) return 1;
  Grid G(n, g);
  for (int d = 0; d < 3; ++d)
    if (G.N[d] < 7) return 1;
  const size_t tot = (size_t)nf * G.sf, inn = (size_t)nf * G.ninterior;
  std::vector<double> S(U, U + tot), kin(inn), K[4];
  for (int s = 0; s < 4; ++s) K[s].assign(tot, 0.0);
  const double a[3] = {0.5, 0.5, 1.0};
  for (int s = 0; s < 4; ++s) {
    // k_s = dt * RHS(S) at every point
    rhs_all(system, *p, G, dx, S.data(), kin.data());
    for (int f = 0; f < nf; ++f)
      for (int k = -g; k < n[2] + g; ++k)
        for (int j = -g; j < n[1] + g; ++j)
          for (int i = -g; i < n[0] + g; ++i) {
            const long o = G.at(f, i, j, k);
            K[s][o] = dt * (is_ghost(G, i, j, k)
                                ? rad_rhs_point(S.data(), G, f, i, j, k, dx, x0, uinf[f], v[f])
                                : kin[G.out(f, i, j, k)]);
          }
    if (s < 3) {
      for (size_t o = 0; o < tot; ++o) S[o] = U[o] + a[s] * K[s][o];
      if (stages) std::copy(S.begin(), S.end(), stages + s * tot);
    }
  }
  for (size_t o = 0; o < tot; ++o) U[o] += (K[0][o] + 2.0 * K[1][o] + 2.0 * K[2][o] + K[3][o]) / 6.0;
  if (stages) std::copy(U, U + tot, stages + 3 * tot);
  return 0;
}

// ---------------------------------------------------------------- sub-cycling
// App. C dense output of one coarse RK step, U(t^n + theta dt) =
// U^n + sum_j b_j(theta) k_j, and its theta-derivatives d^m b_j / d theta^m
// (m = 0..3) written out from the polynomials.
//   RK(4,4):    b_1 = theta - 3/2 theta^2 + 2/3 theta^3,
//               b_2 = b_3 = theta^2 - 2/3 theta^3,
//               b_4 = -1/2 theta^2 + 2/3 theta^3   (sign of the cubic term read
//               so that b_4(1) = 1/6, the RK weight);
//   SSP-RK(3,3): b_1 = theta - 5/6 theta^2, b_2 = 1/6 theta^2, b_3 = 4/6 theta^2.
static void dense_b(int rk, double th, int m, double b[4]) {
  const double t2 = th * th, t3 = t2 * th;
  if (rk == 0) {
    switch (m) {
      case 0: b[0] = th - 1.5 * t2 + (2.0 / 3.0) * t3; b[1] = t2 - (2.0 / 3.0) * t3;
              b[3] = -0.5 * t2 + (2.0 / 3.0) * t3; break;
      case 1: b[0] = 1.0 - 3.0 * th + 2.0 * t2; b[1] = 2.0 * th - 2.0 * t2; b[3] = -th + 2.0 * t2; break;
      case 2: b[0] = -3.0 + 4.0 * th; b[1] = 2.0 - 4.0 * th; b[3] = -1.0 + 4.0 * th; break;
      default: b[0] = 4.0; b[1] = -4.0; b[3] = 4.0; break;
    }
    b[2] = b[1];
  } else {
    switch (m) {
      case 0: b[0] = th - (5.0 / 6.0) * t2; b[1] = t2 / 6.0; b[2] = (4.0 / 6.0) * t2; break;
      case 1: b[0] = 1.0 - (5.0 / 3.0) * th; b[1] = th / 3.0; b[2] = (4.0 / 3.0) * th; break;
      case 2: b[0] = -5.0 / 3.0; b[1] = 1.0 / 3.0; b[2] = 4.0 / 3.0; break;
      default: b[0] = b[1] = b[2] = 0.0; break;
    }
    b[3] = 0.0;
  }
}

// Sec. III.B / App. D, Berger-Oliger without order reduction, for one fine
// step r (0 <= r < R) of the R fine steps inside one coarse step of size dt.
// Inputs per point q: the coarse U^n (un[q]) and the coarse stage increments
// k_j = dt L(U^(j)) (k[j*npts + q], j < s; s = 4 for RK4, 3 for SSP-RK3).
// Steps, in the order of App. D:
//   1. U_{n+r/R} from the dense output at theta = r/R;
//   2. the first three time derivatives of U from the theta-derivatives of
//      the dense output, d^m U/dt^m = dt^-m sum_j k_j b_j^(m)(theta), and
//      (RK4 only) the Jacobian term f_U U_tt = 4 (k_3 - k_2) / dt^3;
//   3. the fine increments with dt_F = dt / R (RK4: the four fine-grid
//      increments of App. D; SSP-RK3: k_1 = dt_F U_t, k_2 = dt_F U_t +
//      dt_F^2 U_tt, k_3 = dt_F U_t + dt_F^2 U_tt / 2);
//   4. the fine stage inputs and the end-of-step value: RK4 U^(1) = U_{n+r/R},
//      U^(2) = U^(1) + k_1/2, U^(3) = U^(1) + k_2/2, U^(4) = U^(1) + k_3,
//      U^{n+(r+1)/R} = U^(1) + (k_1 + 2k_2 + 2k_3 + k_4)/6; SSP-RK3 U^(1),
//      U^(2) = U^(1) + k_1, U^(3) = U^(1) + k_1/4 + k_2/4 (the printed
//      k_2/4 + k_3/4 read as the scheme's own third stage, as in the coarse
//      step), U^{n+(r+1)/R} = U^(1) + (k_1 + k_2 + 4 k_3)/6.
// out[m*npts + q], m = 0..s: U^(1..s) then U^{n+(r+1)/R}.
int or_bor_fine_stages(int rk, int npts, const double* un, const double* k, double dt, int R,
                       int r, double* out) {
  if ((rk != 0 && rk != 1) || R < 1 || r < 0 || r >= R || npts < 0) return 1;
  const int s = rk == 0 ? 4 : 3;
  const double th = (double)r / (double)R;
  const double dtF = dt / (double)R;
  double b0[4], b1[4], b2[4], b3[4];
  dense_b(rk, th, 0, b0);
  dense_b(rk, th, 1, b1);
  dense_b(rk, th, 2, b2);
  dense_b(rk, th, 3, b3);
  for (int q = 0; q < npts; ++q) {
    double kk[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < s; ++j) kk[j] = k[(size_t)j * npts + q];
    // step 1
    double U = un[q];
    for (int j = 0; j < s; ++j) U += b0[j] * kk[j];
    // step 2
    double d1 = 0.0, d2 = 0.0, d3 = 0.0;
    for (int j = 0; j < s; ++j) {
      d1 += b1[j] * kk[j];
      d2 += b2[j] * kk[j];
      d3 += b3[j] * kk[j];
    }
    const double Ut = d1 / dt, Utt = d2 / (dt * dt), Uttt = d3 / (dt * dt * dt);
    double* o = out + q;
    if (rk == 0) {
      const double fUtt = 4.0 * (kk[2] - kk[1]) / (dt * dt * dt);
      // step 3
      const double f1 = dtF * Ut;
      const double f2 = dtF * Ut + 0.5 * dtF * dtF * Utt + 0.125 * dtF * dtF * dtF * (Uttt - fUtt);
      const double f3 = dtF * Ut + 0.5 * dtF * dtF * Utt + 0.125 * dtF * dtF * dtF * (Uttt + fUtt);
      const double f4 = dtF * Ut + dtF * dtF * Utt + 0.5 * dtF * dtF * dtF * Uttt;
      // step 4
      o[0] = U;
      o[(size_t)npts] = U + 0.5 * f1;
      o[2 * (size_t)npts] = U + 0.5 * f2;
      o[3 * (size_t)npts] = U + f3;
      o[4 * (size_t)npts] = U + (f1 + 2.0 * f2 + 2.0 * f3 + f4) / 6.0;
    } else {
      const double f1 = dtF * Ut;
      const double f2 = dtF * Ut + dtF * dtF * Utt;
      const double f3 = dtF * Ut + 0.5 * dtF * dtF * Utt;
      o[0] = U;
      o[(size_t)npts] = U + f1;
      o[2 * (size_t)npts] = U + 0.25 * f1 + 0.25 * f2;
      o[3 * (size_t)npts] = U + (f1 + f2 + 4.0 * f3) / 6.0;
    }
  }
  return 0;
}

// Dense output U(t^n + theta dt) and its time derivatives (App. C):
// out[q] = dt^-m sum_j k_j b_j^(m)(theta) (+ U^n for m = 0).
int or_dense_output(int rk, int npts, const double* un, const double* k, double dt, double theta,
                    int m, double* out) {
  if ((rk != 0 && rk != 1) || m < 0 || m > 3) return 1;
  const int s = rk == 0 ? 4 : 3;
  double b[4];
  dense_b(rk, theta, m, b);
  const double scale = std::pow(dt, -(double)m);
  for (int q = 0; q < npts; ++q) {
    double v = 0.0;
    for (int j = 0; j < s; ++j) v += b[j] * k[(size_t)j * npts + q];
    out[q] = (m == 0 ? un[q] : 0.0) + scale * v;
  }
  return 0;
}

// One stencil of Sec. II.B.1 at interior point (i,j,k) of field f of a
// ghost-filled array: op 0 = D_d1, 1 = D_d1d1, 2 = D_d2(D_d1) (d1 != d2),
// 3 = Q_d with strength sigma (all three directions), 4 = one-sided D_d1 for
// an advecting velocity of sign d2 (> 0 or <= 0).
double or_stencil(int op, const int* n, int g, const double* dx, const double* u, int f, int i,
                  int j, int k, int d1, int d2, double sigma) {
  Grid G(n, g);
  switch (op) {
    case 0: return D1<double>(u, G, f, i, j, k, d1, dx);
    case 1: return D2<double>(u, G, f, i, j, k, d1, dx);
    case 2: return Dmix<double>(u, G, f, i, j, k, d1, d2, dx);
    case 3: return KO<double>(u, G, f, i, j, k, dx, sigma);
    case 4: return Dlop<double>(u, G, f, i, j, k, d1, d2 > 0 ? 1.0 : -1.0, dx);
  }
  return 0.0;
}

// Algorithmic operation count of one interior cell's right-hand side, from
// the per-cell function instantiated on the counting scalar.  The values are
// taken at cell (0,0,0) of the given ghost-filled array.
// out = {add, mul, div, sqrt, log, cmp}.
void or_count_ops(int system, const or_params* p, const int* n, int g, const double* dx,
                  const double* u, long* out) {
  Grid G(n, g);
  g_ops = OpCount{0, 0, 0, 0, 0, 0};
  Cnt r[32];
  cell_rhs<Cnt>(system, *p, u, G, dx, 0, 0, 0, r);
  out[0] = g_ops.add; out[1] = g_ops.mul; out[2] = g_ops.div;
  out[3] = g_ops.sqrt_; out[4] = g_ops.log_; out[5] = g_ops.cmp;
}

}  // extern "C"
