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
#include "sf_f2.cuh"
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

// Whether the stored values are floats (which hold chi, gt_ii and alpha
// minus their flat value 1).
template <typename V>
struct ValTraits {
  static constexpr bool float_storage = sizeof(V) == 4;
};
template <>
struct ValTraits<F2> {
  static constexpr bool float_storage = true;
};

// Stencils of field f at the point, read through a source `Src` (global
// memory, or boxes staged in shared memory): the 19-point cross (D_i, KO,
// optional D_ii, one-sided advection) and the three mixed derivatives.
// Float storage with centred advection evaluates the x and y directions of
// a field's cross (and the xy and xz mixed derivatives) as pairs, with the
// stencil weights folded into per-direction coefficients (PatchArgs::cst):
// the same stencils, one instruction for two lanes.
template <typename T, bool LOP, typename Src>
struct Z4Sten {
  const PatchArgs<T>& a;
  Src& src;
  const T* be;  // shift at the point (one-sided advection)
  static constexpr bool PAIR = sizeof(T) == 4 && !LOP;
  __device__ __forceinline__ const T* U(int f) const { return src.p(f); }
  __device__ __forceinline__ P2<T> cxy(int k) const { return p2<T>(a.cst[k].v[0], a.cst[k].v[1]); }
  __device__ __forceinline__ T centre(int f) { return src.centre(f); }
  __device__ __forceinline__ void finish() { src.finish(); }
  // 19-point cross of field f: first derivatives, KO, optional D_ii
  __device__ __forceinline__ Cross<T> cross(int f, bool second) {
    const long long sy = src.sy();
    const long long sz = src.sz();
    const long long st[3] = {1, sy, sz};
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
  }
  __device__ __forceinline__ T MIX(int f, int m, int n) {
    const int pi = (m == 0 && n == 1) ? 0 : ((m == 0 && n == 2) ? 1 : 2);
    const T* p = U(f);
    const long long st[3] = {1, src.sy(), src.sz()};
    const long long sa = st[m], sb = st[n];
    auto row = [&](long long o) {
      const T* q = p + o;
      return (src.ld(q - 2 * sa) - src.ld(q + 2 * sa)) + T(8) * (src.ld(q + sa) - src.ld(q - sa));
    };
    return ((row(-2 * sb) - row(2 * sb)) + T(8) * (row(sb) - row(-sb))) * a.i144hh[pi];
  }
  // the three mixed derivatives (xy, xz, yz) of field f.  The paired form
  // splits each 16-point tensor-product stencil by weight: with row
  // differences r1(o) = U(o - 2) - U(o + 2) and r8(o) = U(o + 1) - U(o - 1)
  // along x at the offsets o = +-1, +-2 across, D_xb = w (r1(-2) - r1(2)) +
  // 8 w (r8(-2) - r8(2) + r1(1) - r1(-1)) + 64 w (r8(1) - r8(-1)).
  __device__ __forceinline__ void mix3(int f, T* out) {
    if constexpr (PAIR) {
      const long long sy = src.sy();
      const long long sz = src.sz();
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
  }
};

// LOP: one-sided advection stencils compiled in (Z4Coef::lopsided selects
// the instance at launch, so the centred instance carries no extra code).
// The right-hand side of one point (V = T), or of two points at once (V =
// F2: every operation on a pair, H the pair island type), from the stencils
// `sten` provides; `be` receives the shift at the point(s).
template <typename V, typename H, bool LOP, typename Sten, typename ZC, typename Out>
__device__ __forceinline__ void z4_rhs(const ZC& zc, Sten& sten, V (&be)[3], Out&& out) {
  using I = Isl<H>;
  V Gh[3];  // loaded with the other centre values below
  auto advk = [&](const V* dd) { return be[0] * dd[0] + be[1] * dd[1] + be[2] * dd[2]; };
  auto adv = [&](const Cross<V>& x) { return LOP ? x.adv : V(advk(x.d)); };

  // float storage holds chi, gt_xx, gt_yy, gt_zz and alpha minus their flat
  // value 1 (every stencil's weights sum to zero, so derivatives are the
  // same; only the point values used in the algebra get the 1 back)
  const V off = ValTraits<V>::float_storage ? V(1) : V(0);
  const V chi = sten.centre(0) + off, Kh = sten.centre(7), Th = sten.centre(17), al = sten.centre(18) + off;
  V gt[6], At[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    gt[q] = sten.centre(1 + q) + ((q == 0 || q == 3 || q == 5) ? off : V(0));
    At[q] = sten.centre(8 + q);
  }
#pragma unroll
  for (int p = 0; p < 3; ++p) { be[p] = sten.centre(19 + p); Gh[p] = sten.centre(14 + p); }
  const V kz = V(zc.kappa_z), kc = V(zc.kappa_c);

  // ---- islands: determinant, inverse and ln det of the conformal metric,
  // from the exact stored value + offset (not its rounding to the bulk type).
  // The diagonal entries 1 + h are exact sums in the island type; products
  // of two stored values are exact there too, so each cofactor costs one
  // island product (or product by a stored value) and one subtraction.
  const V sg1 = sten.centre(2), sg2 = sten.centre(3), sg4 = sten.centre(5);  // xy, xz, yz
  const H g0 = I::sum2(sten.centre(1), off), g3 = I::sum2(sten.centre(4), off), g5 = I::sum2(sten.centre(6), off);
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
  const V lndet = I::template log<V>(det, idet);
  V ig[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) ig[q] = I::template to<V>(igH[q]);
  // gt^{ij} X_ij of a symmetric X stored as xx, xy, xz, yy, yz, zz: the
  // diagonal and the off-diagonal products accumulated apart, the latter
  // counted twice
  auto trg = [&](const V* X) {
    V dg = ig[0] * X[0];
    dg += ig[3] * X[3];
    dg += ig[5] * X[5];
    V od = ig[1] * X[1];
    od += ig[2] * X[2];
    od += ig[4] * X[4];
    return V(V(2) * od + dg);
  };
  // island trace gt^{ij} X_ij (off-diagonal entries counted twice)
  auto trace_isl = [&](const V* X) { return I::trace_sym(igH, X); };
  // island trace removal X_q - gt_q tr / 3, rounded to the bulk type (tr3 = tr / 3)
  auto tf_isl = [&](V Xq, V gq, const H& tr3) { return I::template sub_prod<V>(Xq, tr3, gq); };
  const H trAH = trace_isl(At);
  const V trA = I::template to<V>(trAH);
  const H trA3 = I::third(trAH);
  // the island inverse is needed once more, for the trace of M_ab: kept as
  // its bulk rounding ig plus the (exact) rounding error
  typename I::template Resid<V> igR[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) igR[q] = I::template resid<V>(igH[q], ig[q]);
  const V ichi = V(1) / chi;
  const V Kt = Kh + V(2) * Th;

  // Every right-hand side term is folded into an accumulator as soon as its
  // inputs exist, so that derivatives die early: rGh collects d/dt Gammahat^a
  // without its advection and KO terms (GhAK), which d/dt B^a reuses; betaAcc
  // the shift equation without g B^a; sA the shift terms of d/dt A~_ab.

  // ---- shift: first derivatives, gt^{mn} d_m d_n beta^c and d_b d_k beta^k
  V dbe[3][3], betaAcc[3], rGh[3], sA[6];
  V divbe;
  {
    V s2[3], ddiv[3] = {V(0), V(0), V(0)}, koBe[3], advBe[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const Cross<V> x = sten.cross(19 + c, true);
      koBe[c] = x.ko;
      if (LOP) advBe[c] = x.adv;
#pragma unroll
      for (int d = 0; d < 3; ++d) dbe[c][d] = x.d[d];  // partial_d beta^c
      ddiv[c] += x.dd[c];
      V mx[3];
      sten.mix3(19 + c, mx);
      const V hess[6] = {x.dd[0], mx[0], mx[1], x.dd[1], mx[2], x.dd[2]};
      s2[c] = trg(hess);  // gt^{mn} d_m d_n beta^c
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = m + 1; n < 3; ++n) {
          const V y = mx[m + n - 1];
          if (n == c) ddiv[m] += y;
          if (m == c) ddiv[n] += y;
        }
    }
    divbe = dbe[0][0] + dbe[1][1] + dbe[2][2];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      betaAcc[p] = (LOP ? advBe[p] : V(advk(dbe[p]))) + koBe[p];
      V sb = Gh[0] * dbe[p][0];
      sb += Gh[1] * dbe[p][1];
      sb += Gh[2] * dbe[p][2];
      V s3v = ig[S(p, 0)] * ddiv[0];
      s3v += ig[S(p, 1)] * ddiv[1];
      s3v += ig[S(p, 2)] * ddiv[2];
      rGh[p] = s2[p] - sb;
      rGh[p] += V(1.0 / 3.0) * s3v;
      rGh[p] += V(2.0 / 3.0) * Gh[p] * divbe;
    }
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = p; b < 3; ++b) {
        const int q = S(p, b);
        V t = V(-2.0 / 3.0) * At[q] * divbe;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          t += At[S(p, c)] * dbe[c][b];
          t += At[S(c, b)] * dbe[c][p];
        }
        sA[q] = t;
      }
  }

  // ---- conformal metric: derivatives, gt^{mn} d_m d_n gt_q, d/dt gt (Eq. syseq1)
  V Gl[3][6];  // Gamma~_{a bc}, first index lowered
  V t1[6];
  {
    V dgt[6][3];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = p; b < 3; ++b) {
        const int q = S(p, b);
        const Cross<V> x = sten.cross(1 + q, true);
#pragma unroll
        for (int d = 0; d < 3; ++d) dgt[q][d] = x.d[d];
        V mx[3];
        sten.mix3(1 + q, mx);
        const V hess[6] = {x.dd[0], mx[0], mx[1], x.dd[1], mx[2], x.dd[2]};
        t1[q] = trg(hess);
        V s = adv(x) + x.ko;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          s += gt[S(p, c)] * dbe[c][b];
          s += gt[S(c, b)] * dbe[c][p];
        }
        const V AtTF = tf_isl(At[q], gt[q], trA3);
        s -= V(2.0 / 3.0) * gt[q] * divbe;
        s -= V(2) * al * AtTF;
        s -= kc * V(1.0 / 3.0) * al * gt[q] * lndet;
        out(1 + q, s, x.c);
      }
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = b; c < 3; ++c)
          Gl[p][S(b, c)] = V(0.5) * (dgt[S(p, c)][b] + dgt[S(p, b)][c] - dgt[S(b, c)][p]);
  }
  V Gu[3][6];  // Gamma~^a_{bc}
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      V g = ig[S(p, 0)] * Gl[0][q];
      g += ig[S(p, 1)] * Gl[1][q];
      g += ig[S(p, 2)] * Gl[2][q];
      Gu[p][q] = g;
    }
  V Z[3];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    Z[p] = V(0.5) * chi * (Gh[p] - trg(Gu[p]));  // Z^i = chi/2 (Gammahat^i - Gamma~^i)
    rGh[p] -= V(2) * al * ichi * Z[p] * (kz + V(2.0 / 3.0) * Kt);
  }

  // ---- Gammahat: derivatives (Ricci), advection and KO of d/dt Gammahat
  V dGh[3][3], GhAK[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Cross<V> x = sten.cross(14 + c, false);
#pragma unroll
    for (int d = 0; d < 3; ++d) dGh[c][d] = x.d[d];  // partial_d Gammahat^c
    GhAK[c] = adv(x) + x.ko;
  }

  // ---- chi: derivatives; its right-hand side is complete here
  V dchi[3], ddchi[6];
  {
    const Cross<V> x = sten.cross(0, true);
#pragma unroll
    for (int d = 0; d < 3; ++d) { dchi[d] = x.d[d]; ddchi[S(d, d)] = x.dd[d]; }
    {
      V mx[3];
      sten.mix3(0, mx);
      ddchi[1] = mx[0];
      ddchi[2] = mx[1];
      ddchi[4] = mx[2];
    }
    out(0, adv(x) + V(2.0 / 3.0) * chi * (al * Kt - divbe) + x.ko, x.c);
  }

  // ---- Ricci tensor Rhat_ab + Rchi_ab
  V Rt[6];
  {
    V t4[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) t4[q] = V(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      V Qc[3][3];  // gt^{nm} Gamma~^c_{mp}
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int n = 0; n < 3; ++n) {
          V qv = ig[S(n, 0)] * Gu[c][S(0, p)];
          qv += ig[S(n, 1)] * Gu[c][S(1, p)];
          qv += ig[S(n, 2)] * Gu[c][S(2, p)];
          Qc[p][n] = qv;
        }
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int b = p; b < 3; ++b) {
          V s = t4[S(p, b)];
#pragma unroll
          for (int n = 0; n < 3; ++n) {
            s += Qc[p][n] * (Gl[b][S(c, n)] + Gl[c][S(n, b)]);
            s += Qc[b][n] * Gl[p][S(c, n)];
          }
          t4[S(p, b)] = s;
        }
    }
    V s3b = V(0);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int m = 0; m < 3; ++m) s3b += ig[S(c, m)] * dchi[c] * dchi[m];
    V Ghdchi = Gh[0] * dchi[0];
    Ghdchi += Gh[1] * dchi[1];
    Ghdchi += Gh[2] * dchi[2];
    const V trace_chi = (trg(ddchi) - V(1.5) * ichi * s3b) - Ghdchi;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = p; b < 3; ++b) {
        const int q = S(p, b);
        V t2 = V(0), t3 = V(0), sG = V(0), sZ = V(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          t2 += gt[S(c, p)] * dGh[c][b];
          t2 += gt[S(c, b)] * dGh[c][p];
          t3 += Gh[c] * (Gl[p][S(b, c)] + Gl[b][S(p, c)]);
          sG += Gu[c][q] * dchi[c];
          sZ += Z[c] * (gt[S(c, p)] * dchi[b] + gt[S(c, b)] * dchi[p]);
        }
        V Rhat = t4[q] - V(0.5) * t1[q];
        Rhat += V(0.5) * (t2 + t3);
        V Rchi = V(0.5) * ichi * (ddchi[q] - sG);
        Rchi -= V(0.25) * ichi * ichi * dchi[p] * dchi[b];
        Rchi += ichi * ichi * sZ;
        Rchi += V(0.5) * ichi * gt[q] * trace_chi;
        Rt[q] = Rhat + Rchi;
      }
  }
  const V RZ = chi * trg(Rt);  // R + 2 nabla_i Z^i = chi gt^{ij} (Rhat + Rchi)_ij

  // ---- alpha: derivatives; its right-hand side is complete here
  V dal[3], ddal[6];
  const V ialpha = V(1) / al;
  {
    const Cross<V> x = sten.cross(18, true);
#pragma unroll
    for (int d = 0; d < 3; ++d) { dal[d] = x.d[d]; ddal[S(d, d)] = x.dd[d]; }
    {
      V mx[3];
      sten.mix3(18, mx);
      ddal[1] = mx[0];
      ddal[2] = mx[1];
      ddal[4] = mx[2];
    }
    const V fsl = zc.slicing == 0 ? V(V(2) * ialpha) : V(1);
    out(18, adv(x) - al * al * fsl * Kh + x.ko, x.c);
  }

  // ---- nabla_a nabla_b alpha and its trace; M_ab = alpha R_ab - D_a D_b alpha
  V M[6];
  V LapAl;
  {
    V gdadc = V(0);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int m = 0; m < 3; ++m) gdadc += ig[S(c, m)] * dal[c] * dchi[m];
    V DDal[6];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = p; b < 3; ++b) {
        const int q = S(p, b);
        V sG = Gu[0][q] * dal[0];
        sG += Gu[1][q] * dal[1];
        sG += Gu[2][q] * dal[2];
        V dd = ddal[q] - sG;
        dd += V(0.5) * ichi * (dal[p] * dchi[b] + dal[b] * dchi[p] - gt[q] * gdadc);
        DDal[q] = dd;
        M[q] = al * Rt[q] - dd;
      }
    LapAl = chi * trg(DDal);
  }

  // ---- A~ contractions, and the Gammahat terms that use them
  V AAd[6];  // A~_ac gt^{cd} A~_db
  {
    V Aud[3][3];  // A~^a_b = gt^{ac} A~_cb
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        V v = ig[S(p, 0)] * At[S(0, b)];
        v += ig[S(p, 1)] * At[S(1, b)];
        v += ig[S(p, 2)] * At[S(2, b)];
        Aud[p][b] = v;
      }
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = p; b < 3; ++b) {
        V v = At[S(p, 0)] * Aud[0][b];
        v += At[S(p, 1)] * Aud[1][b];
        v += At[S(p, 2)] * Aud[2][b];
        AAd[S(p, b)] = v;
      }
    V Auu[6];  // A~^{ab}
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = p; b < 3; ++b) {
        V v = ig[S(p, 0)] * Aud[b][0];
        v += ig[S(p, 1)] * Aud[b][1];
        v += ig[S(p, 2)] * Aud[b][2];
        Auu[S(p, b)] = v;
      }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      V s4 = V(0), s6 = V(0), s8a = V(0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        s4 += Auu[S(p, b)] * dal[b];
        s6 += Auu[S(p, b)] * dchi[b];
        s8a += ig[S(p, b)] * dal[b];
      }
      V s5d = Gu[p][0] * Auu[0];
      s5d += Gu[p][3] * Auu[3];
      s5d += Gu[p][5] * Auu[5];
      V s5o = Gu[p][1] * Auu[1];
      s5o += Gu[p][2] * Auu[2];
      s5o += Gu[p][4] * Auu[4];
      const V s5 = V(2) * s5o + s5d;
      rGh[p] -= V(2) * s4;
      rGh[p] += V(2) * al * (s5 - V(1.5) * ichi * s6);
      // 2 alpha (Theta / alpha) gt^{pb} d_b alpha of the s8 term
      rGh[p] -= V(2) * Th * s8a;
    }
  }
  const V AA = trg(AAd);

  // ---- Khat and Theta
  V Zdal = Z[0] * dal[0];
  Zdal += Z[1] * dal[1];
  Zdal += Z[2] * dal[2];
  {
    const Cross<V> x = sten.cross(7, false);
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      V s7 = ig[S(p, 0)] * x.d[0];
      s7 += ig[S(p, 1)] * x.d[1];
      s7 += ig[S(p, 2)] * x.d[2];
      rGh[p] -= V(4.0 / 3.0) * al * s7;
    }
    V r = adv(x) - LapAl + x.ko;
    r += al * (V(1.0 / 3.0) * Kt * Kt + AA + kz * Th);
    r += V(2) * Zdal;
    out(7, r, Kh);
  }
  {
    const Cross<V> x = sten.cross(17, false);
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      V s8 = ig[S(p, 0)] * x.d[0];
      s8 += ig[S(p, 1)] * x.d[1];
      s8 += ig[S(p, 2)] * x.d[2];
      rGh[p] -= V(2.0 / 3.0) * al * s8;
    }
    V r = adv(x) - Zdal + x.ko;
    r += V(0.5) * al * (RZ + V(2.0 / 3.0) * Kh * Kh + V(2.0 / 3.0) * Th * (Kh - V(2) * Th) - AA);
    r -= V(2) * al * kz * Th;
    out(17, r, Th);
  }

  // ---- d/dt A~_ab (trace removal of M in the island type)
  {
    H igJ[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) igJ[q] = I::template join<V>(ig[q], igR[q]);
    const H trM3 = I::third(I::trace_sym(igJ, M));
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int b = p; b < 3; ++b) {
        const int q = S(p, b);
        const Cross<V> x = sten.cross(8 + q, false);
        const V MTF = tf_isl(M[q], gt[q], trM3);
        V r = adv(x) + sA[q] + x.ko;
        r -= kc * V(1.0 / 3.0) * al * gt[q] * trA;
        r += chi * MTF;
        r += al * (Kh * At[q] - V(2) * AAd[q]);
        out(8 + q, r, x.c);
      }
  }

  // ---- d/dt Gammahat^a (Eq. syseq2), shift and B (Gamma-driver)
#pragma unroll
  for (int p = 0; p < 3; ++p) out(14 + p, GhAK[p] + rGh[p], Gh[p]);
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    if (zc.shift_frozen) {
      out(19 + p, V(0), be[p]);
      out(22 + p, V(0), sten.centre(22 + p));
    } else {
      const Cross<V> x = sten.cross(22 + p, false);
      out(19 + p, betaAcc[p] + V(zc.g_shift) * x.c, be[p]);
      out(22 + p, adv(x) - V(zc.eta) * x.c + rGh[p] + x.ko, x.c);
    }
  }
  sten.finish();
}

template <typename T, typename H, bool LOP, typename Src, typename Out>
__device__ __forceinline__ void z4_cell(const PatchArgs<T>& a, const Z4Coef<T>& zc, Src& src,
                                        Out&& out) {
  T be[3];
  Z4Sten<T, LOP, Src> sten{a, src, be};
  z4_rhs<T, H, LOP>(zc, sten, be, out);
}

}  // namespace sf
