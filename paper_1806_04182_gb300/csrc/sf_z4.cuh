// CCZ4 (Sec. V) with Bona-Masso slicing and Gamma-driver shift, vacuum,
// 25 fields, fused with Kreiss-Oliger dissipation and the RK stage update.
//
// Field order: 0 chi | 1-6 gt_xx,xy,xz,yy,yz,zz | 7 Khat | 8-13 At_ij |
// 14-16 Gammahat^i | 17 Theta | 18 alpha | 19-21 beta^i | 22-24 B^i
//
// One thread per interior point.  Derivatives are taken straight from the
// ghosted SoA arrays (L1/L2-resident neighbours) and consumed as soon as
// they are formed, so only the 48 first derivatives the algebra reuses stay
// live.  T is the bulk (storage + stencil) type, H the type of the
// "island" quantities: conformal-metric determinant, inverse, ln det and
// the trace removals.  FP64: T = H = double.  FP32-bulk: T = float,
// H = double.
#pragma once
#include "sf_common.cuh"

namespace sf {

template <typename T>
struct Z4Coef {
  T kappa_z, kappa_c, eta, g_shift;
  int slicing;       // 0: 1+log, 1: harmonic
  int shift_frozen;
};

__host__ __device__ constexpr int S(int a, int b) {
  return a == b ? (a == 0 ? 0 : (a == 1 ? 3 : 5))
                : ((a + b) == 1 ? 1 : ((a + b) == 2 ? 2 : 4));
}

template <typename T, typename H>
__device__ __forceinline__ void z4_point(const PatchArgs<T>& a, const Z4Coef<T>& zc,
                                         const T* __restrict__ u, T v[25], T rhs[25]) {
  const long long F = a.sf;
  const long long st[3] = {1, a.sy, a.sz};
  const long long sy = a.sy, sz = a.sz;
  auto U = [&](int f) { return u + f * F; };

#pragma unroll
  for (int f = 0; f < 25; ++f) v[f] = __ldg(U(f));
  const T chi = v[0];
  T gt[6], At[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) { gt[q] = v[1 + q]; At[q] = v[8 + q]; }
  const T Kh = v[7], Th = v[17], al = v[18];
  const T Gh[3] = {v[14], v[15], v[16]};
  const T be[3] = {v[19], v[20], v[21]};
  const T Bv[3] = {v[22], v[23], v[24]};

  // ---- conformal metric inverse, determinant, ln det (island type H)
  const H g00 = gt[0], g01 = gt[1], g02 = gt[2], g11 = gt[3], g12 = gt[4], g22 = gt[5];
  const H c00 = g11 * g22 - g12 * g12, c01 = g02 * g12 - g01 * g22, c02 = g01 * g12 - g02 * g11;
  const H c11 = g00 * g22 - g02 * g02, c12 = g01 * g02 - g00 * g12, c22 = g00 * g11 - g01 * g01;
  const H det = g00 * c00 + g01 * c01 + g02 * c02;
  const H idet = H(1) / det;
  const H igH[6] = {c00 * idet, c01 * idet, c02 * idet, c11 * idet, c12 * idet, c22 * idet};
  const H lndet = log(det);
  T ig[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) ig[q] = T(igH[q]);
  // symmetric contraction weights: off-diagonal entries appear twice
  T w[6] = {ig[0], T(2) * ig[1], T(2) * ig[2], ig[3], T(2) * ig[4], ig[5]};

  // ---- first derivatives that the algebra reuses
  T dchi[3], dKh[3], dTh[3], dal[3], dgt[6][3], dbe[3][3], dGh[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T h = a.i12h[d];
    dchi[d] = d1(U(0), st[d], h);
    dKh[d] = d1(U(7), st[d], h);
    dTh[d] = d1(U(17), st[d], h);
    dal[d] = d1(U(18), st[d], h);
#pragma unroll
    for (int q = 0; q < 6; ++q) dgt[q][d] = d1(U(1 + q), st[d], h);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      dbe[q][d] = d1(U(19 + q), st[d], h);  // partial_d beta^q
      dGh[q][d] = d1(U(14 + q), st[d], h);  // partial_d Gammahat^q
    }
  }
  auto advk = [&](const T* dd) { return be[0] * dd[0] + be[1] * dd[1] + be[2] * dd[2]; };
  auto adv_direct = [&](int f) {
    T s = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) s += be[d] * d1(U(f), st[d], a.i12h[d]);
    return s;
  };
  const T divbe = dbe[0][0] + dbe[1][1] + dbe[2][2];

  // ---- second derivatives.  dd(f, m, n) for m <= n.
  auto dd = [&](int f, int m, int n) -> T {
    if (m == n) return d2(U(f), st[m], v[f], a.i12h2[m]);
    const int pi = (m == 0 && n == 1) ? 0 : ((m == 0 && n == 2) ? 1 : 2);
    return dmix(U(f), st[m], st[n], a.i144hh[pi]);
  };
  T ddchi[6], ddal[6];
  // conformal metric: t1[q] = gt^{mn} d_m d_n gt_q, consumed at once
  T t1[6];
  // shift: s2[a] = gt^{mn} d_m d_n beta^a, ddiv[b] = d_b d_k beta^k
  T s2[3] = {T(0), T(0), T(0)}, ddiv[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int n = m; n < 3; ++n) {
      const int q = S(m, n);
      ddchi[q] = dd(0, m, n);
      ddal[q] = dd(18, m, n);
    }
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    T s = T(0);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int n = m; n < 3; ++n) s += w[S(m, n)] * dd(1 + p, m, n);
    t1[p] = s;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int n = m; n < 3; ++n) {
        const T x = dd(19 + c, m, n);
        s2[c] += w[S(m, n)] * x;
        if (m == n) {
          if (m == c) ddiv[c] += x;
        } else {
          if (n == c) ddiv[m] += x;
          if (m == c) ddiv[n] += x;
        }
      }

  // ---- Christoffel symbols
  T Gl[3][6];  // Gamma~_{a bc}, first index lowered
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = b; c < 3; ++c)
        Gl[p][S(b, c)] = T(0.5) * (dgt[S(p, c)][b] + dgt[S(p, b)][c] - dgt[S(b, c)][p]);
  T Gu[3][6];  // Gamma~^a_{bc}
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 6; ++q)
      Gu[p][q] = ig[S(p, 0)] * Gl[0][q] + ig[S(p, 1)] * Gl[1][q] + ig[S(p, 2)] * Gl[2][q];
  T Gt[3], Z[3];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    T s = T(0);
#pragma unroll
    for (int q = 0; q < 6; ++q) s += w[q] * Gu[p][q];
    Gt[p] = s;
    Z[p] = T(0.5) * chi * (Gh[p] - Gt[p]);
  }

  // ---- Ricci tensor Rhat_ab + Rchi_ab (Sec. V)
  // Q[c][a][n] = gt^{nm} Gamma~^c_{ma}
  T Qm[3][3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int n = 0; n < 3; ++n)
        Qm[c][p][n] = ig[S(n, 0)] * Gu[c][S(0, p)] + ig[S(n, 1)] * Gu[c][S(1, p)] +
                      ig[S(n, 2)] * Gu[c][S(2, p)];
  const T ichi = T(1) / chi;
  T s3 = T(0);
#pragma unroll
  for (int q = 0; q < 6; ++q) s3 += w[q] * ddchi[q];
  T s3b = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int m = 0; m < 3; ++m) s3b += ig[S(c, m)] * dchi[c] * dchi[m];
  const T Ghdchi = Gh[0] * dchi[0] + Gh[1] * dchi[1] + Gh[2] * dchi[2];
  const T trace_chi = (s3 - T(1.5) * ichi * s3b) - Ghdchi;
  T Rt[6];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int b = p; b < 3; ++b) {
      const int q = S(p, b);
      T t2 = T(0), t3 = T(0), t4 = T(0), sG = T(0), sZ = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        t2 += gt[S(c, p)] * dGh[c][b] + gt[S(c, b)] * dGh[c][p];
        t3 += Gh[c] * (Gl[p][S(b, c)] + Gl[b][S(p, c)]);
        sG += Gu[c][q] * dchi[c];
        sZ += Z[c] * (gt[S(c, p)] * dchi[b] + gt[S(c, b)] * dchi[p]);
#pragma unroll
        for (int n = 0; n < 3; ++n)
          t4 += Qm[c][p][n] * Gl[b][S(c, n)] + Qm[c][b][n] * Gl[p][S(c, n)] +
                Qm[c][p][n] * Gl[c][S(n, b)];
      }
      const T Rhat = T(-0.5) * t1[q] + T(0.5) * t2 + T(0.5) * t3 + t4;
      const T Rchi = T(0.5) * ichi * (ddchi[q] - sG) - T(0.25) * ichi * ichi * dchi[p] * dchi[b] +
                     ichi * ichi * sZ + T(0.5) * ichi * gt[q] * trace_chi;
      Rt[q] = Rhat + Rchi;
    }
  T RZ = T(0);
#pragma unroll
  for (int q = 0; q < 6; ++q) RZ += w[q] * Rt[q];
  RZ *= chi;

  // ---- nabla_a nabla_b alpha and its trace
  T gdadc = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int m = 0; m < 3; ++m) gdadc += ig[S(c, m)] * dal[c] * dchi[m];
  T DDal[6];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int b = p; b < 3; ++b) {
      const int q = S(p, b);
      T sG = Gu[0][q] * dal[0] + Gu[1][q] * dal[1] + Gu[2][q] * dal[2];
      DDal[q] = ddal[q] - sG + T(0.5) * ichi * (dal[p] * dchi[b] + dal[b] * dchi[p] - gt[q] * gdadc);
    }
  T LapAl = T(0);
#pragma unroll
  for (int q = 0; q < 6; ++q) LapAl += w[q] * DDal[q];
  LapAl *= chi;

  // ---- A~ contractions
  H trAH = H(0);
  {
    const H wH[6] = {igH[0], H(2) * igH[1], H(2) * igH[2], igH[3], H(2) * igH[4], igH[5]};
#pragma unroll
    for (int q = 0; q < 6; ++q) trAH += wH[q] * H(At[q]);
  }
  const T trA = T(trAH);
  T Aud[3][3];  // A~^a_b = gt^{ac} A~_cb
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      Aud[p][b] = ig[S(p, 0)] * At[S(0, b)] + ig[S(p, 1)] * At[S(1, b)] + ig[S(p, 2)] * At[S(2, b)];
  T Auu[6];  // A~^{ab}
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int b = p; b < 3; ++b)
      Auu[S(p, b)] = ig[S(p, 0)] * Aud[b][0] + ig[S(p, 1)] * Aud[b][1] + ig[S(p, 2)] * Aud[b][2];
  T AA = T(0);
  {
    const T wA[6] = {T(1), T(2), T(2), T(1), T(2), T(1)};
#pragma unroll
    for (int q = 0; q < 6; ++q) AA += wA[q] * At[q] * Auu[q];
  }

  const T kz = zc.kappa_z, kc = zc.kappa_c;
  // ---- d/dt gt_ab  (Eq. syseq1); trace removal of A~ in H
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int b = p; b < 3; ++b) {
      const int q = S(p, b);
      T s = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) s += gt[S(p, c)] * dbe[c][b] + gt[S(c, b)] * dbe[c][p];
      const T AtTF = T(H(At[q]) - H(1.0 / 3.0) * H(gt[q]) * trAH);
      rhs[1 + q] = advk(dgt[q]) + s - T(2.0 / 3.0) * gt[q] * divbe - T(2) * al * AtTF -
                   kc * T(1.0 / 3.0) * al * gt[q] * T(lndet);
    }

  // ---- d/dt A~_ab; trace-free part of alpha R - D D alpha in H
  {
    T M[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) M[q] = al * Rt[q] - DDal[q];
    const H wH[6] = {igH[0], H(2) * igH[1], H(2) * igH[2], igH[3], H(2) * igH[4], igH[5]};
    H trM = H(0);
#pragma unroll
    for (int q = 0; q < 6; ++q) trM += wH[q] * H(M[q]);
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = p; b < 3; ++b) {
        const int q = S(p, b);
        T s = T(0), AAd = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          s += At[S(p, c)] * dbe[c][b] + At[S(c, b)] * dbe[c][p];
          AAd += At[S(p, c)] * Aud[c][b];
        }
        const T MTF = T(H(M[q]) - H(1.0 / 3.0) * H(gt[q]) * trM);
        rhs[8 + q] = adv_direct(8 + q) + s - T(2.0 / 3.0) * At[q] * divbe -
                     kc * T(1.0 / 3.0) * al * gt[q] * trA + chi * MTF +
                     al * (Kh * At[q] - T(2) * AAd);
      }
  }

  // ---- d/dt chi, Khat, Theta
  const T Kt = Kh + T(2) * Th;
  rhs[0] = advk(dchi) + T(2.0 / 3.0) * chi * (al * Kt - divbe);
  const T Zdal = Z[0] * dal[0] + Z[1] * dal[1] + Z[2] * dal[2];
  rhs[7] = advk(dKh) - LapAl + al * (T(1.0 / 3.0) * Kt * Kt + AA + kz * Th) + T(2) * Zdal;
  rhs[17] = advk(dTh) +
            T(0.5) * al * (RZ + T(2.0 / 3.0) * Kh * Kh + T(2.0 / 3.0) * Th * (Kh - T(2) * Th) - AA) -
            Zdal - T(2) * al * kz * Th;

  // ---- d/dt Gammahat^a  (Eq. syseq2)
  T rGh[3];
  const T ialpha = T(1) / al;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    T sb = T(0), s3v = T(0), s4 = T(0), s5 = T(0), s6 = T(0), s7 = T(0), s8 = T(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      sb += Gh[b] * dbe[p][b];
      s3v += ig[S(p, b)] * ddiv[b];
      s4 += Auu[S(p, b)] * dal[b];
      s6 += Auu[S(p, b)] * dchi[b];
      s7 += ig[S(p, b)] * dKh[b];
      s8 += ig[S(p, b)] * (T(1.0 / 3.0) * dTh[b] + Th * ialpha * dal[b]);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const T wA = (q == 0 || q == 3 || q == 5) ? T(1) : T(2);
      s5 += wA * Gu[p][q] * Auu[q];
    }
    rGh[p] = -sb + T(2.0 / 3.0) * Gh[p] * divbe + s2[p] + T(1.0 / 3.0) * s3v - T(2) * s4 +
             T(2) * al * (s5 - T(1.5) * ichi * s6 - T(2.0 / 3.0) * s7) +
             T(2) * al * (-s8 - ichi * Z[p] * (kz + T(2.0 / 3.0) * Kt));
    rhs[14 + p] = advk(dGh[p]) + rGh[p];
  }

  // ---- gauge (Sec. V): Bona-Masso slicing, Gamma-driver shift
  const T fsl = zc.slicing == 0 ? T(2) * ialpha : T(1);
  rhs[18] = advk(dal) - al * al * fsl * Kh;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    if (zc.shift_frozen) {
      rhs[19 + p] = T(0);
      rhs[22 + p] = T(0);
    } else {
      rhs[19 + p] = advk(dbe[p]) + zc.g_shift * Bv[p];
      rhs[22 + p] = adv_direct(22 + p) - zc.eta * Bv[p] + rGh[p];
    }
  }

  // ---- Kreiss-Oliger dissipation on every evolved field
  const int nko = zc.shift_frozen ? 19 : 25;
#pragma unroll
  for (int f = 0; f < 25; ++f)
    if (f < nko) rhs[f] += ko_all(U(f), sy, sz, v[f], a.ko);
}

}  // namespace sf
