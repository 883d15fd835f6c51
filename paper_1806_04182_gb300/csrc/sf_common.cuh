// Shared device/host pieces of the GB300 substep library: patch layout
// passed to kernels, the 4th-order stencils of Sec. II.B.1, the RK stage
// combination of Sec. II.C / App. C-D, fused periodic ghost writes and the
// status-word bits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sf.h"

namespace sf {

// ------------------------------------------------------------ status word
// bit 0: non-finite output, bit 1: work-queue time-out.  The word lives in
// sf_api.cu; kernels get its device address through StageArgs::status.
constexpr unsigned int ST_NONFINITE = 1u;
constexpr unsigned int ST_TIMEOUT = 2u;

// ------------------------------------------------------------ kernel args
// Everything a stage kernel needs about one patch, by value.
template <typename T>
struct PatchArgs {
  int n[3];
  int g;
  long long sy, sz, sf;
  long long ninterior;
  const T* __restrict__ us;  // stage input (ghosted)
  const T* __restrict__ un;  // U^n (ghosted)
  T* acc;
  T* nx;                     // next stage / U^{n+1}, or the RHS output (unghosted)
  T* kh;
  double* rate;  // MHD: max signal rate of u_next (last stage only), or nullptr
  // precomputed coefficients
  T i12h[3];    // 1 / (12 dx_d)
  T i12h2[3];   // 1 / (12 dx_d^2)
  T i144hh[3];  // 1 / (144 dx_a dx_b) for (xy, xz, yz)
  T ko[3];      // sigma / (64 dx_d)
  // The same stencil weights folded into per-direction coefficients, for
  // kernels that evaluate two directions at once (sf_pair.cuh): entry k of
  // direction d is cst[k][d]; pairs (x, y) are 8-byte aligned.
  //   0: 1/(12 dx)    1: 8/(12 dx)                          (D_d)
  //   2: s   3: 15 s   4: -6 s   5: -20 s,  s = sigma/(64 dx)  (KO)
  //   6: 16 e   7: -e   8: -30 e,  e = 1/(12 dx^2)            (D_dd)
  // and mixed: cmx[k] = (w, 8 w, 64 w)[k] with w = 1/(144 dx_a dx_b) for
  // (xy, xz) as a pair and yz alone.
  struct alignas(8) Dir3 { T v[4]; };
  Dir3 cst[9];
  Dir3 cmx[3];
  T c_next;     // u_next = un + c_next * r   (or ssp weights)
  T c_acc;      // acc += c_acc * r
  T dt;
};

// RK stage selection, uniform over a launch
struct StageArgs {
  int mode;        // 0: stage update, 1: write RHS only
  int rk;          // SF_RK4 / SF_SSPRK3
  int stage;
  int kahan;       // FP32_BULK compensated last stage
  int un_alias;    // u_n == u_stage: reuse the centre value
  int ghosts;      // SF_GHOSTS_PERIODIC: also write the periodic ghost shell
  int check_finite;
  unsigned int* status;  // device status word
};

// ------------------------------------------------------------ stencils
// Sec. II.B.1.  `p` points at the centre value, `s` is the element stride
// of the direction.
template <typename T>
__device__ __forceinline__ T d1(const T* __restrict__ p, long long s, T i12h) {
  return ((__ldg(p - 2 * s) - __ldg(p + 2 * s)) + T(8) * (__ldg(p + s) - __ldg(p - s))) * i12h;
}

template <typename T>
__device__ __forceinline__ T d2(const T* __restrict__ p, long long s, T c0, T i12h2) {
  return (T(16) * (__ldg(p - s) + __ldg(p + s)) - (__ldg(p - 2 * s) + __ldg(p + 2 * s)) - T(30) * c0) *
         i12h2;
}

// D_b(D_a U): tensor product of two first-derivative stencils (16 points)
template <typename T>
__device__ __forceinline__ T dmix(const T* __restrict__ p, long long sa, long long sb, T i144) {
  auto row = [&](long long o) {
    const T* q = p + o;
    return (__ldg(q - 2 * sa) - __ldg(q + 2 * sa)) + T(8) * (__ldg(q + sa) - __ldg(q - sa));
  };
  return ((row(-2 * sb) - row(2 * sb)) + T(8) * (row(sb) - row(-sb))) * i144;
}

// 6th difference along one direction: U-3 - 6U-2 + 15U-1 - 20U0 + 15U+1 - 6U+2 + U+3
template <typename T>
__device__ __forceinline__ T delta6(const T* __restrict__ p, long long s, T c0) {
  return (__ldg(p - 3 * s) + __ldg(p + 3 * s)) - T(6) * (__ldg(p - 2 * s) + __ldg(p + 2 * s)) +
         T(15) * (__ldg(p - s) + __ldg(p + s)) - T(20) * c0;
}

template <typename T>
__device__ __forceinline__ T ko_all(const T* __restrict__ p, long long sy, long long sz, T c0,
                                    const T* kc) {
  return kc[0] * delta6(p, 1, c0) + kc[1] * delta6(p, sy, c0) + kc[2] * delta6(p, sz, c0);
}

__device__ __forceinline__ bool finite_(double v) { return isfinite(v); }
__device__ __forceinline__ bool finite_(float v) { return isfinite(v); }

// ------------------------------------------------------------ stage write
// RK stage combination of one field value at ghosted offset c (interior
// point i,j,k); `centre` is u_stage there and r = (L + Q_d)(u_stage).  The
// periodic ghost images of the point are computed once (ghost_images) and
// reused for every field (write_field).
struct Images {
  // bit 2d: the point lies within `ghost` of the low end of axis d (its image
  // shifted by +n_d is a ghost point); bit 2d+1: of the high end (shift -n_d).
  // Both bits of one axis are set when n_d < 2 ghost; up to 26 images.
  unsigned mask;
};

template <typename T>
__device__ __forceinline__ Images ghost_images(const PatchArgs<T>& a, const StageArgs& s, int i,
                                               int j, int k) {
  Images im;
  im.mask = 0;
  if (!s.ghosts || s.mode == 1) return im;
  const int g = a.g;
  im.mask = (i < g ? 1u : 0u) | (i >= a.n[0] - g ? 2u : 0u) | (j < g ? 4u : 0u) |
            (j >= a.n[1] - g ? 8u : 0u) | (k < g ? 16u : 0u) | (k >= a.n[2] - g ? 32u : 0u);
  return im;
}

// Periodic ghost images of the value `out` written at offset o.
template <typename T>
__device__ __forceinline__ void store_images(const PatchArgs<T>& a, const Images& im, long long o,
                                             T out) {
  if (!im.mask) return;
  // shift index 0: none, 1: +n_d (point near the low end), 2: -n_d
  const unsigned m = im.mask;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    if (p && !(m & (p == 1 ? 16u : 32u))) continue;
    const long long oz = p == 0 ? 0 : (p == 1 ? 1 : -1) * (long long)a.n[2] * a.sz;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (q && !(m & (q == 1 ? 4u : 8u))) continue;
      const long long oy = q == 0 ? 0 : (q == 1 ? 1 : -1) * (long long)a.n[1] * a.sy;
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        if (w && !(m & (w == 1 ? 1u : 2u))) continue;
        if (p | q | w) a.nx[o + oz + oy + (w == 0 ? 0 : (w == 1 ? a.n[0] : -a.n[0]))] = out;
      }
    }
  }
}

// RK stage combination at offset o from the values it reads (u_stage centre,
// U^n, accumulator, Kahan term; only those the stage uses are meaningful):
// writes the accumulator / Kahan term and returns the next stage input.
template <typename T>
__device__ __forceinline__ T stage_combine(const PatchArgs<T>& a, const StageArgs& s, long long o,
                                           T centre, T un_m, T acc, T kh, T r) {
  const T un = s.un_alias ? centre : un_m;
  T out;
  if (s.rk == SF_RK4) {
    if (s.stage == 0) {
      a.acc[o] = (s.kahan ? T(0) : un) + a.c_acc * r;
      out = un + a.c_next * r;
    } else if (s.stage < 3) {
      a.acc[o] = acc + a.c_acc * r;
      out = un + a.c_next * r;
    } else if (!s.kahan) {
      out = acc + a.c_next * r;
    } else {
      const T inc = acc + a.c_next * r;
      const T y = inc - kh;
      const T t = un + y;
      a.kh[o] = (t - un) - y;
      out = t;
    }
  } else {
    if (s.stage == 0) out = un + a.dt * r;
    else if (s.stage == 1) out = T(0.75) * un + T(0.25) * (centre + a.dt * r);
    else out = un * T(1.0 / 3.0) + T(2.0 / 3.0) * (centre + a.dt * r);
  }
  return out;
}

template <typename T>
__device__ __forceinline__ T write_field(const PatchArgs<T>& a, const StageArgs& s,
                                         const Images& im, int f, long long c, int i, int j,
                                         int k, T centre, T r) {
  if (s.mode == 1) {
    a.nx[f * a.ninterior + ((long long)k * a.n[1] + j) * a.n[0] + i] = r;
    return r;
  }
  const long long o = f * a.sf + c;
  const bool rk4 = s.rk == SF_RK4;
  const T un = s.un_alias ? centre : a.un[o];
  const T acc = (rk4 && s.stage > 0) ? a.acc[o] : T(0);
  const T kh = (rk4 && s.stage == 3 && s.kahan) ? a.kh[o] : T(0);
  const T out = stage_combine(a, s, o, centre, un, acc, kh, r);
  a.nx[o] = out;
  if (s.check_finite && !finite_(out)) atomicOr(s.status, ST_NONFINITE);
  store_images(a, im, o, out);
  return out;
}

// The stage write of all NF fields of one point whose right-hand sides were
// parked in memory (r[f * stride]), for kernels that produce the 25 CCZ4
// right-hand sides before writing any of them.  Fields go in batches of
// five: every read of a batch (u_stage centre, U^n, accumulator, Kahan term,
// as the stage needs them) is issued before its writes, so five reads of
// each array are in flight at once instead of one.  The new values replace
// the right-hand sides in r, and the periodic images (boundary points only)
// are written by one rolled pass at the end.
template <typename T, int NF>
__device__ __forceinline__ void write_fields(const PatchArgs<T>& a, const StageArgs& s,
                                             const Images& im, long long c, int i, int j, int k,
                                             T* r, int stride) {
  static_assert(NF % 5 == 0, "fields go in batches of five");
  if (s.mode == 1) {
    const long long oi = ((long long)k * a.n[1] + j) * a.n[0] + i;
#pragma unroll 1
    for (int f = 0; f < NF; ++f) a.nx[f * a.ninterior + oi] = r[f * stride];
    return;
  }
  const bool rk4 = s.rk == SF_RK4;
  const bool need_centre = s.un_alias || !rk4;
  const bool need_acc = rk4 && s.stage > 0;
  const bool need_kh = rk4 && s.stage == 3 && s.kahan;
#pragma unroll 1
  for (int f0 = 0; f0 < NF; f0 += 5) {
    T cen[5], un[5], acc[5], kh[5], rr[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const long long o = (f0 + q) * a.sf + c;
      rr[q] = r[(f0 + q) * stride];
      cen[q] = need_centre ? a.us[o] : T(0);
      un[q] = s.un_alias ? T(0) : a.un[o];
      acc[q] = need_acc ? a.acc[o] : T(0);
      kh[q] = need_kh ? a.kh[o] : T(0);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const long long o = (f0 + q) * a.sf + c;
      const T out = stage_combine(a, s, o, cen[q], un[q], acc[q], kh[q], rr[q]);
      a.nx[o] = out;
      if (s.check_finite && !finite_(out)) atomicOr(s.status, ST_NONFINITE);
      r[(f0 + q) * stride] = out;
    }
  }
  if (im.mask) {
#pragma unroll 1
    for (int f = 0; f < NF; ++f) store_images(a, im, f * a.sf + c, r[f * stride]);
  }
}

// ------------------------------------------------------------ launch plumbing
struct Launch {
  dim3 grid, block;
};

// Host-side construction of PatchArgs from the ABI structs.
template <typename T>
PatchArgs<T> make_args(const sf_params& prm, const sf_patch& p, int stage, int nf,
                       void* rhs_out) {
  PatchArgs<T> a;
  for (int d = 0; d < 3; ++d) a.n[d] = p.n[d];
  a.g = p.ghost;
  a.sy = p.sy;
  a.sz = p.sz;
  a.sf = p.sf;
  a.ninterior = (long long)p.n[0] * p.n[1] * p.n[2];
  a.us = static_cast<const T*>(p.u_stage);
  a.un = static_cast<const T*>(p.u_n);
  a.acc = static_cast<T*>(p.acc);
  a.nx = static_cast<T*>(rhs_out ? rhs_out : p.u_next);
  a.kh = static_cast<T*>(p.kahan);
  a.rate = nullptr;
  for (int d = 0; d < 3; ++d) {
    a.i12h[d] = T(1.0 / (12.0 * p.dx[d]));
    a.i12h2[d] = T(1.0 / (12.0 * p.dx[d] * p.dx[d]));
    a.ko[d] = T(prm.sigma_ko / (64.0 * p.dx[d]));
  }
  for (int d = 0; d < 3; ++d) {
    const double h = p.dx[d], sk = prm.sigma_ko / (64.0 * h), e = 1.0 / (12.0 * h * h);
    const double w[9] = {1.0 / (12.0 * h), 8.0 / (12.0 * h), sk, 15.0 * sk, -6.0 * sk, -20.0 * sk,
                         16.0 * e, -e, -30.0 * e};
    for (int k = 0; k < 9; ++k) a.cst[k].v[d] = T(w[k]);
  }
  for (int k = 0; k < 9; ++k) a.cst[k].v[3] = T(0);
  {
    const double wxy = 1.0 / (144.0 * p.dx[0] * p.dx[1]), wxz = 1.0 / (144.0 * p.dx[0] * p.dx[2]),
                 wyz = 1.0 / (144.0 * p.dx[1] * p.dx[2]);
    const double f[3] = {1.0, 8.0, 64.0};
    for (int k = 0; k < 3; ++k) {
      a.cmx[k].v[0] = T(f[k] * wxy);
      a.cmx[k].v[1] = T(f[k] * wxz);
      a.cmx[k].v[2] = T(f[k] * wyz);
      a.cmx[k].v[3] = T(0);
    }
  }
  a.i144hh[0] = T(1.0 / (144.0 * p.dx[0] * p.dx[1]));
  a.i144hh[1] = T(1.0 / (144.0 * p.dx[0] * p.dx[2]));
  a.i144hh[2] = T(1.0 / (144.0 * p.dx[1] * p.dx[2]));
  const double dt = p.dt;
  a.dt = T(dt);
  double cn = 0.0, ca = 0.0;
  if (prm.rk == SF_RK4) {
    const double cnext[4] = {0.5, 0.5, 1.0, 1.0 / 6.0};
    const double cacc[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 0.0};
    cn = cnext[stage] * dt;
    ca = cacc[stage] * dt;
  }
  a.c_next = T(cn);
  a.c_acc = T(ca);
  (void)nf;
  return a;
}

}  // namespace sf
