// CCZ4 right-hand side at one point (Sec. V): Bona-Masso slicing,
// Gamma-driver shift, vacuum, 25 fields, plus Kreiss-Oliger dissipation.
//
// Field order: 0 chi | 1-6 gt_xx,xy,xz,yy,yz,zz | 7 Khat | 8-13 At_ij |
// 14-16 Gammahat^i | 17 Theta | 18 alpha | 19-21 beta^i | 22-24 B^i
//
// Each field's 19-point cross (centre and +-1..3 along x, y, z) is read once
// and gives its three first derivatives D_i, its KO term and, for the fields
// that need them, its pure second derivatives D_ii (Sec. II.B.1); mixed
// derivatives D_ij = D_j(D_i) read their 16 off-axis points.  Quantities are
// formed in the order they are consumed and every field is handed to
// `out(f, rhs, centre)` as soon as its right-hand side is complete:
//   islands (det, inverse, ln det) -> shift -> metric + d/dt gt ->
//   Christoffels -> chi, alpha -> Ricci -> D D alpha -> Khat, Theta ->
//   A~ -> Gammahat, beta, B.
// T is the bulk (storage + stencil) type; H the island type (double, or the
// double-word float pair of sf_dw.cuh).  With T = float the arrays store
// chi - 1, gt_xx - 1, gt_yy - 1, gt_zz - 1 and alpha - 1, so that values
// near flat space keep their small deviations (e.g. 1e-10 noise) in float.
// SY, SZ > 0 fix the y/z element strides at compile time, so every stencil
// read is an immediate offset from a per-field base pointer; 0 means
// runtime strides.
#pragma once
#include "sf_common.cuh"
#include "sf_dw.cuh"
#include "sf_pair.cuh"

namespace sf {

template <typename T>
struct Z4Coef {
  T kappa_z, kappa_c, eta, g_shift;
  int slicing;       // 0: 1+log, 1: harmonic
  int shift_frozen;
  int lopsided;      // 1: one-sided advection stencils (Sec. II.B.1); picks the LOP instance
};

template <typename T>
Z4Coef<T> z4_coef(const sf_params& prm) {
  Z4Coef<T> zc;
  zc.kappa_z = T(prm.kappa_z);
  zc.kappa_c = T(prm.kappa_c);
  zc.eta = T(prm.eta);
  zc.g_shift = T(prm.g_shift);
  zc.slicing = prm.slicing;
  zc.shift_frozen = prm.shift_frozen;
  zc.lopsided = prm.lopsided;
  return zc;
}

__host__ __device__ constexpr int S(int a, int b) {
  return a == b ? (a == 0 ? 0 : (a == 1 ? 3 : 5))
                : ((a + b) == 1 ? 1 : ((a + b) == 2 ? 2 : 4));
}

template <typename T>
struct Cross {
  T c;      // centre value
  T d[3];   // D_x, D_y, D_z
  T dd[3];  // D_xx, D_yy, D_zz (when requested)
  T ko;     // sum_d sigma/(64 dx_d) delta^6_d
  T adv;    // beta^k d_k U: centred D_k, or one-sided by the sign of beta^k
};

// Stencil source reading the ghosted SoA arrays in global memory.
template <typename T, int SY, int SZ>
struct GlobalSrc {
  const T* __restrict__ u;  // centre of field 0
  long long F, sy_, sz_;
  __device__ __forceinline__ long long sy() const { return SY ? (long long)SY : sy_; }
  __device__ __forceinline__ long long sz() const { return SZ ? (long long)SZ : sz_; }
  __device__ __forceinline__ const T* p(int f) const { return u + f * F; }
  __device__ __forceinline__ T ld(const T* q) const { return __ldg(q); }
  __device__ __forceinline__ T centre(int f) const { return __ldg(u + f * F); }
  __device__ __forceinline__ void begin(int) {}   // called before field f's first stencil
  __device__ __forceinline__ void finish() {}     // called once at the end
};

// LOP: one-sided advection stencils compiled in (Z4Coef::lopsided selects
// the instance at launch, so the centred instance carries no extra code).
template <typename T, typename H, bool LOP, typename Src, typename Out>
__device__ __forceinline__ void z4_cell(const PatchArgs<T>& a, const Z4Coef<T>& zc, Src& src,
                                        Out&& out) {
  using I = Isl<H>;
  const long long sy = src.sy();
  const long long sz = src.sz();
  const long long st[3] = {1, sy, sz};
  auto U = [&](int f) { return src.p(f); };
  auto c0 = [&](int f) { return src.centre(f); };
  T be[3], Gh[3];  // loaded with the other centre values below
  // Float storage with centred advection evaluates the x and y directions of
  // a field's cross (and the xy and xz mixed derivatives) as pairs, with the
  // stencil weights folded into per-direction coefficients (PatchArgs::cst):
  // the same stencils, one instruction for two lanes.
  constexpr bool PAIR = sizeof(T) == 4 && !LOP;
  auto cxy = [&](int k) { return p2<T>(a.cst[k].v[0], a.cst[k].v[1]); };
  // 19-point cross of field f: first derivatives, KO, optional D_ii
  auto cross = [&](int f, bool second) {
    src.begin(f);
    const T* p = U(f);
    Cross<T> x;
    x.c = src.ld(p);
    x.ko = T(0);
    x.adv = T(0);
    if constexpr (PAIR) {
      const P2<T> m1 = p2(src.ld(p - 1), src.ld(p - sy)), q1 = p2(src.ld(p + 1), src.ld(p + sy));
      const P2<T> m2 = p2(src.ld(p - 2), src.ld(p - 2 * sy)),
                  q2 = p2(src.ld(p + 2), src.ld(p + 2 * sy));
      const P2<T> m3 = p2(src.ld(p - 3), src.ld(p - 3 * sy)),
                  q3 = p2(src.ld(p + 3), src.ld(p + 3 * sy));
      const T zm1 = src.ld(p - sz), zq1 = src.ld(p + sz), zm2 = src.ld(p - 2 * sz),
              zq2 = src.ld(p + 2 * sz), zm3 = src.ld(p - 3 * sz), zq3 = src.ld(p + 3 * sz);
      const P2<T> cc = p2(x.c, x.c);
      const P2<T> d = pfma(psub(q1, m1), cxy(1), pmul(psub(m2, q2), cxy(0)));
      const P2<T> s1 = padd(m1, q1), s2 = padd(m2, q2), s3 = padd(m3, q3);
      const P2<T> ko = pfma(s1, cxy(3), pfma(s2, cxy(4), pfma(cc, cxy(5), pmul(s3, cxy(2)))));
      const T z1 = zm1 + zq1, z2 = zm2 + zq2, z3 = zm3 + zq3;
      x.d[0] = d.x;
      x.d[1] = d.y;
      x.d[2] = (zq1 - zm1) * a.cst[1].v[2] + (zm2 - zq2) * a.cst[0].v[2];
      x.ko = (ko.x + ko.y) + (z1 * a.cst[3].v[2] + (z2 * a.cst[4].v[2] +
                                                    (x.c * a.cst[5].v[2] + z3 * a.cst[2].v[2])));
      if (second) {
        const P2<T> dd = pfma(s1, cxy(6), pfma(s2, cxy(7), pmul(cc, cxy(8))));
        x.dd[0] = dd.x;
        x.dd[1] = dd.y;
        x.dd[2] = z1 * a.cst[6].v[2] + (z2 * a.cst[7].v[2] + x.c * a.cst[8].v[2]);
      } else {
        x.dd[0] = x.dd[1] = x.dd[2] = T(0);
      }
      return x;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const long long s = st[d];
      const T m1 = src.ld(p - s), p1 = src.ld(p + s);
      const T m2 = src.ld(p - 2 * s), p2 = src.ld(p + 2 * s);
      const T m3 = src.ld(p - 3 * s), p3 = src.ld(p + 3 * s);
      x.d[d] = ((m2 - p2) + T(8) * (p1 - m1)) * a.i12h[d];
      x.dd[d] = second ? (T(16) * (m1 + p1) - (m2 + p2) - T(30) * x.c) * a.i12h2[d] : T(0);
      x.ko += a.ko[d] * ((m3 + p3) - T(6) * (m2 + p2) + T(15) * (m1 + p1) - T(20) * x.c);
      // advection along d (Sec. II.B.1), one-sided on the side the
      // characteristic comes from; the centred instance forms beta^k D_k at
      // the point of use instead (advk)
      if (LOP) {
        T ad = x.d[d];
        if (be[d] != T(0))
          ad = (be[d] > T(0) ? (p3 - T(6) * p2 + T(18) * p1 - T(10) * x.c - T(3) * m1)
                             : (-m3 + T(6) * m2 - T(18) * m1 + T(10) * x.c + T(3) * p1)) *
               a.i12h[d];
        x.adv += be[d] * ad;
      }
    }
    return x;
  };
  auto advk = [&](const T* dd) { return be[0] * dd[0] + be[1] * dd[1] + be[2] * dd[2]; };
  auto adv = [&](const Cross<T>& x) { return LOP ? x.adv : advk(x.d); };
  auto MIX = [&](int f, int m, int n) -> T {
    const int pi = (m == 0 && n == 1) ? 0 : ((m == 0 && n == 2) ? 1 : 2);
    const T* p = U(f);
    const long long sa = st[m], sb = st[n];
    auto row = [&](long long o) {
      const T* q = p + o;
      return (src.ld(q - 2 * sa) - src.ld(q + 2 * sa)) + T(8) * (src.ld(q + sa) - src.ld(q - sa));
    };
    return ((row(-2 * sb) - row(2 * sb)) + T(8) * (row(sb) - row(-sb))) * a.i144hh[pi];
  };
  // the three mixed derivatives (xy, xz, yz) of field f.  The paired form
  // splits each 16-point tensor-product stencil by weight: with row
  // differences r1(o) = U(o - 2) - U(o + 2) and r8(o) = U(o + 1) - U(o - 1)
  // along x at the offsets o = +-1, +-2 across, D_xb = w (r1(-2) - r1(2)) +
  // 8 w (r8(-2) - r8(2) + r1(1) - r1(-1)) + 64 w (r8(1) - r8(-1)).
  auto mix3 = [&](int f, T* out) {
    if constexpr (PAIR) {
      const T* p = U(f);
      auto r1 = [&](int o) {
        return psub(p2(src.ld(p + o * sy - 2), src.ld(p + o * sz - 2)),
                    p2(src.ld(p + o * sy + 2), src.ld(p + o * sz + 2)));
      };
      auto r8 = [&](int o) {
        return psub(p2(src.ld(p + o * sy + 1), src.ld(p + o * sz + 1)),
                    p2(src.ld(p + o * sy - 1), src.ld(p + o * sz - 1)));
      };
      const P2<T> x1 = psub(r1(-2), r1(2));
      const P2<T> x8 = padd(psub(r8(-2), r8(2)), psub(r1(1), r1(-1)));
      const P2<T> x64 = psub(r8(1), r8(-1));
      const P2<T> w1 = p2<T>(a.cmx[0].v[0], a.cmx[0].v[1]), w8 = p2<T>(a.cmx[1].v[0], a.cmx[1].v[1]),
                  w64 = p2<T>(a.cmx[2].v[0], a.cmx[2].v[1]);
      const P2<T> r = pfma(x64, w64, pfma(x8, w8, pmul(x1, w1)));
      out[0] = r.x;
      out[1] = r.y;
      out[2] = MIX(f, 1, 2);
    } else {
      out[0] = MIX(f, 0, 1);
      out[1] = MIX(f, 0, 2);
      out[2] = MIX(f, 1, 2);
    }
  };

  // float storage holds chi, gt_xx, gt_yy, gt_zz and alpha minus their flat
  // value 1 (every stencil's weights sum to zero, so derivatives are the
  // same; only the point values used in the algebra get the 1 back)
  const T off = sizeof(T) == 4 ? T(1) : T(0);
  const T chi = c0(0) + off, Kh = c0(7), Th = c0(17), al = c0(18) + off;
  T gt[6], At[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    gt[q] = c0(1 + q) + ((q == 0 || q == 3 || q == 5) ? off : T(0));
    At[q] = c0(8 + q);
  }
#pragma unroll
  for (int p = 0; p < 3; ++p) { be[p] = c0(19 + p); Gh[p] = c0(14 + p); }
  const T kz = zc.kappa_z, kc = zc.kappa_c;

  // ---- islands: determinant, inverse and ln det of the conformal metric,
  // from the exact stored value + offset (not its rounding to the bulk type).
  // The diagonal entries 1 + h are exact sums in the island type; products
  // of two stored values are exact there too, so each cofactor costs one
  // island product (or product by a stored value) and one subtraction.
  const T sg1 = c0(2), sg2 = c0(3), sg4 = c0(5);  // xy, xz, yz
  const H g0 = I::sum2(c0(1), off), g3 = I::sum2(c0(4), off), g5 = I::sum2(c0(6), off);
  const H c00 = I::sub(I::mul(g3, g5), I::prod(sg4, sg4));
  const H c01 = I::sub(I::prod(sg2, sg4), I::mulf(g5, sg1));
  const H c02 = I::sub(I::prod(sg1, sg4), I::mulf(g3, sg2));
  const H c11 = I::sub(I::mul(g0, g5), I::prod(sg2, sg2));
  const H c12 = I::sub(I::prod(sg1, sg2), I::mulf(g0, sg4));
  const H c22 = I::sub(I::mul(g0, g3), I::prod(sg1, sg1));
  const H det = I::add(I::add(I::mul(c00, g0), I::mulf(c01, sg1)), I::mulf(c02, sg2));
  const H idet = I::recip(det);
  const H igH[6] = {I::mul(c00, idet), I::mul(c01, idet), I::mul(c02, idet),
                    I::mul(c11, idet), I::mul(c12, idet), I::mul(c22, idet)};
  const T lndet = I::template log<T>(det, idet);
  T ig[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) ig[q] = I::template to<T>(igH[q]);
  const T w[6] = {ig[0], T(2) * ig[1], T(2) * ig[2], ig[3], T(2) * ig[4], ig[5]};
  // island trace gt^{ij} X_ij (off-diagonal entries counted twice)
  auto trace_isl = [&](const T* X) { return I::trace_sym(igH, X); };
  // island trace removal X_q - gt_q tr / 3, rounded to the bulk type (tr3 = tr / 3)
  auto tf_isl = [&](T Xq, T gq, const H& tr3) { return I::template sub_prod<T>(Xq, tr3, gq); };
  const H trAH = trace_isl(At);
  const T trA = I::template to<T>(trAH);
  const H trA3 = I::third(trAH);

  // ---- shift: first derivatives, gt^{mn} d_m d_n beta^c and d_b d_k beta^k
  T dbe[3][3], koBe[3], advBe[3];
  T s2[3] = {T(0), T(0), T(0)}, ddiv[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Cross<T> x = cross(19 + c, true);
    koBe[c] = x.ko;
    if (LOP) advBe[c] = x.adv;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      dbe[c][d] = x.d[d];  // partial_d beta^c
      s2[c] += w[S(d, d)] * x.dd[d];
    }
    ddiv[c] += x.dd[c];
    T mx[3];
    mix3(19 + c, mx);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int n = m + 1; n < 3; ++n) {
        const T y = mx[m + n - 1];
        s2[c] += w[S(m, n)] * y;
        if (n == c) ddiv[m] += y;
        if (m == c) ddiv[n] += y;
      }
  }
  const T divbe = dbe[0][0] + dbe[1][1] + dbe[2][2];

  // ---- conformal metric: derivatives, gt^{mn} d_m d_n gt_q, d/dt gt (Eq. syseq1)
  T Gl[3][6];  // Gamma~_{a bc}, first index lowered
  T t1[6];
  {
    T dgt[6][3];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = p; b < 3; ++b) {
        const int q = S(p, b);
        const Cross<T> x = cross(1 + q, true);
        T s1 = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          dgt[q][d] = x.d[d];
          s1 += w[S(d, d)] * x.dd[d];
        }
        T mx[3];
        mix3(1 + q, mx);
        s1 += w[1] * mx[0] + w[2] * mx[1] + w[4] * mx[2];
        t1[q] = s1;
        T s = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) s += gt[S(p, c)] * dbe[c][b] + gt[S(c, b)] * dbe[c][p];
        const T AtTF = tf_isl(At[q], gt[q], trA3);
        out(1 + q,
            adv(x) + s - T(2.0 / 3.0) * gt[q] * divbe - T(2) * al * AtTF -
                kc * T(1.0 / 3.0) * al * gt[q] * lndet + x.ko,
            x.c);
      }
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = b; c < 3; ++c)
          Gl[p][S(b, c)] = T(0.5) * (dgt[S(p, c)][b] + dgt[S(p, b)][c] - dgt[S(b, c)][p]);
  }
  T Gu[3][6];  // Gamma~^a_{bc}
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 6; ++q)
      Gu[p][q] = ig[S(p, 0)] * Gl[0][q] + ig[S(p, 1)] * Gl[1][q] + ig[S(p, 2)] * Gl[2][q];
  T Z[3];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    T s = T(0);
#pragma unroll
    for (int q = 0; q < 6; ++q) s += w[q] * Gu[p][q];
    Z[p] = T(0.5) * chi * (Gh[p] - s);  // Z^i = chi/2 (Gammahat^i - Gamma~^i)
  }
  const T Kt = Kh + T(2) * Th;

  // ---- chi and alpha: derivatives; their right-hand sides are complete here
  T dchi[3], ddchi[6], dal[3], ddal[6];
  {
    const Cross<T> x = cross(0, true);
#pragma unroll
    for (int d = 0; d < 3; ++d) { dchi[d] = x.d[d]; ddchi[S(d, d)] = x.dd[d]; }
    {
      T mx[3];
      mix3(0, mx);
      ddchi[1] = mx[0];
      ddchi[2] = mx[1];
      ddchi[4] = mx[2];
    }
    out(0, adv(x) + T(2.0 / 3.0) * chi * (al * Kt - divbe) + x.ko, x.c);
  }
  const T ialpha = T(1) / al;
  {
    const Cross<T> x = cross(18, true);
#pragma unroll
    for (int d = 0; d < 3; ++d) { dal[d] = x.d[d]; ddal[S(d, d)] = x.dd[d]; }
    {
      T mx[3];
      mix3(18, mx);
      ddal[1] = mx[0];
      ddal[2] = mx[1];
      ddal[4] = mx[2];
    }
    const T fsl = zc.slicing == 0 ? T(2) * ialpha : T(1);
    out(18, adv(x) - al * al * fsl * Kh + x.ko, x.c);
  }

  // ---- Ricci tensor Rhat_ab + Rchi_ab
  const T ichi = T(1) / chi;
  T Rt[6];
  T dGh[3][3], koGh[3], advGh[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Cross<T> x = cross(14 + c, false);
    koGh[c] = x.ko;
    if (LOP) advGh[c] = x.adv;
#pragma unroll
    for (int d = 0; d < 3; ++d) dGh[c][d] = x.d[d];  // partial_d Gammahat^c
  }
  {
    T t4[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) t4[q] = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T Qc[3][3];  // gt^{nm} Gamma~^c_{mp}
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int n = 0; n < 3; ++n)
          Qc[p][n] = ig[S(n, 0)] * Gu[c][S(0, p)] + ig[S(n, 1)] * Gu[c][S(1, p)] +
                     ig[S(n, 2)] * Gu[c][S(2, p)];
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int b = p; b < 3; ++b) {
          T s = T(0);
#pragma unroll
          for (int n = 0; n < 3; ++n)
            s += Qc[p][n] * (Gl[b][S(c, n)] + Gl[c][S(n, b)]) + Qc[b][n] * Gl[p][S(c, n)];
          t4[S(p, b)] += s;
        }
    }
    T s3 = T(0), s3b = T(0);
#pragma unroll
    for (int q = 0; q < 6; ++q) s3 += w[q] * ddchi[q];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int m = 0; m < 3; ++m) s3b += ig[S(c, m)] * dchi[c] * dchi[m];
    const T Ghdchi = Gh[0] * dchi[0] + Gh[1] * dchi[1] + Gh[2] * dchi[2];
    const T trace_chi = (s3 - T(1.5) * ichi * s3b) - Ghdchi;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = p; b < 3; ++b) {
        const int q = S(p, b);
        T t2 = T(0), t3 = T(0), sG = T(0), sZ = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          t2 += gt[S(c, p)] * dGh[c][b] + gt[S(c, b)] * dGh[c][p];
          t3 += Gh[c] * (Gl[p][S(b, c)] + Gl[b][S(p, c)]);
          sG += Gu[c][q] * dchi[c];
          sZ += Z[c] * (gt[S(c, p)] * dchi[b] + gt[S(c, b)] * dchi[p]);
        }
        const T Rhat = T(-0.5) * t1[q] + T(0.5) * t2 + T(0.5) * t3 + t4[q];
        const T Rchi = T(0.5) * ichi * (ddchi[q] - sG) -
                       T(0.25) * ichi * ichi * dchi[p] * dchi[b] + ichi * ichi * sZ +
                       T(0.5) * ichi * gt[q] * trace_chi;
        Rt[q] = Rhat + Rchi;
      }
  }
  T RZ = T(0);
#pragma unroll
  for (int q = 0; q < 6; ++q) RZ += w[q] * Rt[q];
  RZ *= chi;  // R + 2 nabla_i Z^i = chi gt^{ij} (Rhat + Rchi)_ij

  // ---- nabla_a nabla_b alpha and its trace; M_ab = alpha R_ab - D_a D_b alpha
  T M[6];
  T LapAl = T(0);
  {
    T gdadc = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int m = 0; m < 3; ++m) gdadc += ig[S(c, m)] * dal[c] * dchi[m];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = p; b < 3; ++b) {
        const int q = S(p, b);
        const T sG = Gu[0][q] * dal[0] + Gu[1][q] * dal[1] + Gu[2][q] * dal[2];
        const T DDal = ddal[q] - sG +
                       T(0.5) * ichi * (dal[p] * dchi[b] + dal[b] * dchi[p] - gt[q] * gdadc);
        LapAl += w[q] * DDal;
        M[q] = al * Rt[q] - DDal;
      }
    LapAl *= chi;
  }

  // ---- A~ contractions
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
#pragma unroll
  for (int q = 0; q < 6; ++q) AA += ((q == 0 || q == 3 || q == 5) ? T(1) : T(2)) * At[q] * Auu[q];

  // ---- Khat and Theta
  const T Zdal = Z[0] * dal[0] + Z[1] * dal[1] + Z[2] * dal[2];
  T dKh[3], dTh[3];
  {
    const Cross<T> x = cross(7, false);
#pragma unroll
    for (int d = 0; d < 3; ++d) dKh[d] = x.d[d];
    out(7, adv(x) - LapAl + al * (T(1.0 / 3.0) * Kt * Kt + AA + kz * Th) + T(2) * Zdal + x.ko,
        Kh);
  }
  {
    const Cross<T> x = cross(17, false);
#pragma unroll
    for (int d = 0; d < 3; ++d) dTh[d] = x.d[d];
    out(17,
        adv(x) +
            T(0.5) * al * (RZ + T(2.0 / 3.0) * Kh * Kh + T(2.0 / 3.0) * Th * (Kh - T(2) * Th) - AA) -
            Zdal - T(2) * al * kz * Th + x.ko,
        Th);
  }

  // ---- d/dt A~_ab (trace removal of M in the island type)
  {
    const H trM3 = I::third(trace_isl(M));
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = p; b < 3; ++b) {
        const int q = S(p, b);
        const Cross<T> x = cross(8 + q, false);
        T s = T(0), AAd = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          s += At[S(p, c)] * dbe[c][b] + At[S(c, b)] * dbe[c][p];
          AAd += At[S(p, c)] * Aud[c][b];
        }
        const T MTF = tf_isl(M[q], gt[q], trM3);
        out(8 + q,
            adv(x) + s - T(2.0 / 3.0) * At[q] * divbe - kc * T(1.0 / 3.0) * al * gt[q] * trA +
                chi * MTF + al * (Kh * At[q] - T(2) * AAd) + x.ko,
            x.c);
      }
  }

  // ---- d/dt Gammahat^a (Eq. syseq2), shift and B (Gamma-driver)
  T rGh[3];
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
    for (int q = 0; q < 6; ++q)
      s5 += ((q == 0 || q == 3 || q == 5) ? T(1) : T(2)) * Gu[p][q] * Auu[q];
    rGh[p] = -sb + T(2.0 / 3.0) * Gh[p] * divbe + s2[p] + T(1.0 / 3.0) * s3v - T(2) * s4 +
             T(2) * al * (s5 - T(1.5) * ichi * s6 - T(2.0 / 3.0) * s7) +
             T(2) * al * (-s8 - ichi * Z[p] * (kz + T(2.0 / 3.0) * Kt));
    out(14 + p, (LOP ? advGh[p] : advk(dGh[p])) + rGh[p] + koGh[p], Gh[p]);
  }
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    if (zc.shift_frozen) {
      out(19 + p, T(0), be[p]);
      out(22 + p, T(0), c0(22 + p));
    } else {
      const Cross<T> x = cross(22 + p, false);
      out(19 + p, (LOP ? advBe[p] : advk(dbe[p])) + zc.g_shift * x.c + koBe[p], be[p]);
      out(22 + p, adv(x) - zc.eta * x.c + rGh[p] + x.ko, x.c);
    }
  }
  src.finish();
}

}  // namespace sf
