// CCZ4 stage kernel with two points per thread (Sec. V right-hand side with
// the Sec. II.B.1 stencils, fused with the RK stage of Sec. II.C), float
// storage, centred advection.
//
// Each thread computes two x-neighbours (i, i + 1), i even, and carries
// every quantity of the right-hand side as a pair (F2): each add, multiply
// and fused multiply-add of the per-point algebra is one .f32x2 instruction
// for both points, and so are most of the stencil operations.  The kernel
// is bound by instruction issue, so this halves the issue slots of the
// arithmetic, of the address and control work and of the ring waits per
// point.  It needs rows laid out so that points with even interior x sit on
// 8-byte boundaries: a row pitch of a multiple of 4 floats with one float
// before the first ghost point (arrays start 4 bytes past a 16-byte
// boundary).  Then every stencil read is a 64-bit shared-memory load of an
// aligned pair, and every RK read and write a 64-bit global access.
//
// Staging as in the one-point TMA kernel: a CTA of W warps computes a
// 32 x 2W x 1 tile (half-warps take rows, 16 threads x 2 points each); the
// 40 x (2W + 6) x 7 box of every field is brought into a ring of shared
// memory slots by a cp.async.bulk.tensor load, fields in the order the
// right-hand side opens them, with a "full" mbarrier (TMA transaction count)
// and an "empty" mbarrier (one arrival per warp) per slot.  Every wait is
// bounded (about a second of clock cycles); a wait that gives up sets
// ST_TIMEOUT in the status word, the kernel finishes with whatever the slot
// holds, waits (bounded) for its own loads in flight and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "sf_internal.cuh"
#include "sf_mbar.cuh"
#include "sf_z4.cuh"

namespace sf {
namespace {

constexpr int kXB = 40, kTZ = 7;                  // box: 40 x (2W + 6) x 7 floats
constexpr int kSY = 104, kSZ = 104 * 102;         // strides of the padded 96^3 layout
constexpr long long kWaitCycles = 2000000000LL;   // ~1 s at GB300 clocks

template <int W, int KS>
struct PCfg {
  static constexpr int BY = 2 * W;  // tile rows
  static constexpr int TY = BY + 6;
  static constexpr int kBoxBytes = kXB * TY * kTZ * 4;
  static constexpr int kSlotBytes = (kBoxBytes + 127) / 128 * 128;
  static constexpr int kSlotFloats = kSlotBytes / 4;
  static constexpr int kThreads = 32 * W;
  static constexpr int kBarOffset = KS * kSlotBytes;
  static constexpr int kRbufOffset = kBarOffset + 2 * KS * 8;
  static constexpr int kSmemBytes = kRbufOffset + 25 * kThreads * 8;
  static_assert(kSmemBytes <= 232448, "shared memory per CTA");
};

// RK inputs staged through the ring: boxes of 32 x 16 points x kRkChunk
// fields of one array (a tile's rows), three chunks per array.
constexpr int kRkChunk = 12;
constexpr int kRkBoxBytes = 32 * 16 * kRkChunk * 4;

// The configuration in use: 8 warps (a 32 x 16 tile), 7 slots.  Measured on
// the 96^3 patch against 6 warps with 9 slots (32 x 12 tiles; 2.35e9 against
// 2.81e9 cell-updates/s), 5 slots (2.75e9) and a persistent form in which
// one CTA per SM walks the tiles with the ring running on from tile to tile
// (1.84e9).
constexpr int kW = 8, kKS = 7;
static_assert(kRkBoxBytes <= PCfg<kW, kKS>::kSlotBytes && PCfg<kW, kKS>::BY == 16, "RK chunk fits a slot");
static_assert(3 * kRkChunk >= 25, "three chunks cover the fields");

// Order in which z4_rhs opens the fields' stencils.  Without the
// Gamma-driver (shift frozen) the last three are not used.
__constant__ signed char kPairFieldSeq[25] = {19, 20, 21, 1, 2, 3, 4, 5, 6, 14, 15, 16, 0,
                                              18, 7, 17, 8, 9, 10, 11, 12, 13, 22, 23, 24};

// Stencil weights as broadcast pairs (Sec. II.B.1), per direction d.
struct PairCoef {
  F2 d1[3], d2[3];         // D_d = (U+1 - U-1) d1 + (U-2 - U+2) d2: 8/(12 h), 1/(12 h)
  F2 k1[3], k2[3], k3[3];  // KO: 15 s, -6 s, s on the sums at distance 1, 2, 3
  F2 kc;                   // KO centre: -20 (s_x + s_y + s_z), s = sigma / (64 h)
  F2 e1[3], e2[3], e0[3];  // D_dd: 16 e, -e, -30 e with e = 1 / (12 h^2)
  F2 mx[3][3];             // mixed (xy, xz, yz): w, 8 w, 64 w with w = 1 / (144 h_a h_b)
};

PairCoef pair_coef(const sf_params& prm, const sf_patch& p) {
  PairCoef c;
  double kc = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double h = p.dx[d], s = prm.sigma_ko / (64.0 * h), e = 1.0 / (12.0 * h * h);
    auto b = [](double v) { F2 r; r.x = r.y = float(v); return r; };
    c.d1[d] = b(8.0 / (12.0 * h));
    c.d2[d] = b(1.0 / (12.0 * h));
    c.k1[d] = b(15.0 * s);
    c.k2[d] = b(-6.0 * s);
    c.k3[d] = b(s);
    kc += s;
    c.e1[d] = b(16.0 * e);
    c.e2[d] = b(-e);
    c.e0[d] = b(-30.0 * e);
  }
  c.kc.x = c.kc.y = float(-20.0 * kc);
  const double w[3] = {1.0 / (144.0 * p.dx[0] * p.dx[1]), 1.0 / (144.0 * p.dx[0] * p.dx[2]),
                       1.0 / (144.0 * p.dx[1] * p.dx[2])};
  for (int m = 0; m < 3; ++m)
    for (int k = 0; k < 3; ++k) c.mx[m][k].x = c.mx[m][k].y = float(w[m] * (k == 0 ? 1.0 : k == 1 ? 8.0 : 64.0));
  return c;
}

__device__ __forceinline__ void tma_load_4d(float* dst, const CUtensorMap* map, int x, int y, int z,
                                            int f, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(f), "r"(saddr(bar))
      : "memory");
}

// Stencil source of z4_rhs for the pair of points (i, i + 1): the staged
// boxes in shared memory, the centre values (all fields, at the start) from
// global memory.
template <int W, int KS, int NARR = 0>
struct PairSrc {
  using C = PCfg<W, KS>;
  static constexpr int kY = kXB;            // box row, floats
  static constexpr int kZ = kXB * C::TY;    // box plane, floats
  const float* __restrict__ u;  // global stage input at point i, field 0
  long long F;
  const PairCoef* pc;
  float* tiles;
  uint64_t* full;
  uint64_t* empty;
  const CUtensorMap* map;
  unsigned* status;
  int local;  // this thread's point i inside a box (an even float index)
  int use, cur, nuses, issued;
  int gx, gy, gz;  // tensor coordinates of the box origin
  bool leader, lane0, dead;
  // NARR > 0: after the nfu field uses, the RK inputs of the tile (NARR
  // arrays) follow as uses of the ring, 3 chunks of 12 fields per array,
  // chunk-major, from the maps rkmap[0 .. NARR - 1] at tensor coordinates
  // (rx, ry, rz); consumed by the write phase (acquire / release)
  int nfu, done;
  const CUtensorMap* rkmap;
  int rx, ry, rz;

  __device__ __forceinline__ void fail() {
    if (!dead) atomicOr(status, ST_TIMEOUT);
    dead = true;
  }
  // leader: load use j into its slot once the previous occupant (use j - KS)
  // has been released by every warp
  __device__ __forceinline__ void issue(int j) {
    const int sl = j % KS;
    if (j >= KS && !dead && !mbar_wait(&empty[sl], ((j / KS) - 1) & 1, kWaitCycles)) fail();
    if (dead) return;
    if (NARR == 0 || j < nfu) {
      mbar_expect(&full[sl], C::kBoxBytes);
      tma_load_4d(tiles + sl * C::kSlotFloats, map, gx, gy, gz, kPairFieldSeq[j], &full[sl]);
    } else if constexpr (NARR > 0) {
      const int r = j - nfu;
      mbar_expect(&full[sl], kRkBoxBytes);
      tma_load_4d(tiles + sl * C::kSlotFloats, rkmap + r % NARR, rx, ry, rz, kRkChunk * (r / NARR),
                  &full[sl]);
    }
    issued = j + 1;
  }
  // write phase: wait for RK use i (kept until release(i)), after issuing
  // the uses up to i + KS - NARR (their slots' previous uses are released)
  __device__ __forceinline__ const float* acquire(int i) {
    if (leader)
      for (int q = issued; q <= i + KS - NARR && q < nuses && !dead; ++q) issue(q);
    if (!dead && !mbar_wait(&full[i % KS], (i / KS) & 1, kWaitCycles)) fail();
    done = i + 1;
    return tiles + (i % KS) * C::kSlotFloats;
  }
  __device__ __forceinline__ void release(int i) {
    __syncwarp();
    if (lane0) mbar_arrive(&empty[i % KS]);
  }
  __device__ __forceinline__ void prologue() {
    if (leader)
      for (int j = 0; j < KS - 2 && j < nuses; ++j) issue(j);
  }
  __device__ __forceinline__ void begin() {
    const int i = use++;
    if (leader && i + KS - 2 < nuses) issue(i + KS - 2);
    if (i > 0) {
      __syncwarp();
      if (lane0) mbar_arrive(&empty[(i - 1) % KS]);
    }
    cur = i % KS;
    if (!dead && !mbar_wait(&full[cur], (i / KS) & 1, kWaitCycles)) fail();
  }
  // end of the field uses (z4_rhs's last call): with staged RK inputs the
  // last field's slot is released for them; without, a leader whose wait
  // gave up waits (bounded) for its loads still in flight
  __device__ __forceinline__ void finish() {
    if constexpr (NARR > 0) {
      release(use - 1);
      done = use;
    } else {
      final_finish();
    }
  }
  __device__ __forceinline__ void final_finish() {
    const int from = NARR > 0 ? done : use;
    if (leader && dead)
      for (int j = from; j < issued; ++j) mbar_wait(&full[j % KS], (j / KS) & 1, kWaitCycles);
  }

  __device__ __forceinline__ const float* box() const { return tiles + cur * C::kSlotFloats + local; }
  // aligned pair at float offset o (even) from point i
  static __device__ __forceinline__ F2 L(const float* p, int o) { return *reinterpret_cast<const F2*>(p + o); }

  __device__ __forceinline__ F2 centre(int f) const {
    return *reinterpret_cast<const F2*>(u + f * F);
  }

  // 19-point cross of both points.  Along x the neighbours at odd distance
  // straddle two aligned pairs: their sums and differences are formed lane
  // by lane (two scalar instructions straight into a pair), everything else
  // on pairs.
  __device__ __forceinline__ Cross<F2> cross(int f, bool second) {
    begin();
    const float* p = box();
    const PairCoef& c = *pc;
    const F2 am4 = L(p, -4), am2 = L(p, -2), a0 = L(p, 0), a2 = L(p, 2), a4 = L(p, 4);
    // x: values q(o) at offset o from point i; point i + 1 reads q(o + 1)
    const F2 xs1(am2.y + a0.y, a0.x + a2.x);   // U-1 + U+1
    const F2 xd1(a0.y - am2.y, a2.x - a0.x);   // U+1 - U-1
    const F2 xs3(am4.y + a2.y, am2.x + a4.x);  // U-3 + U+3
    const F2 xs2 = add2(am2, a2), xd2 = sub2(am2, a2);
    const F2 ym1 = L(p, -kY), yp1 = L(p, kY), ym2 = L(p, -2 * kY), yp2 = L(p, 2 * kY),
             ym3 = L(p, -3 * kY), yp3 = L(p, 3 * kY);
    const F2 zm1 = L(p, -kZ), zp1 = L(p, kZ), zm2 = L(p, -2 * kZ), zp2 = L(p, 2 * kZ),
             zm3 = L(p, -3 * kZ), zp3 = L(p, 3 * kZ);
    const F2 ys1 = add2(ym1, yp1), yd1 = sub2(yp1, ym1), ys2 = add2(ym2, yp2), yd2 = sub2(ym2, yp2),
             ys3 = add2(ym3, yp3);
    const F2 zs1 = add2(zm1, zp1), zd1 = sub2(zp1, zm1), zs2 = add2(zm2, zp2), zd2 = sub2(zm2, zp2),
             zs3 = add2(zm3, zp3);
    Cross<F2> x;
    x.c = a0;
    x.d[0] = fma2(xd1, c.d1[0], mul2(xd2, c.d2[0]));
    x.d[1] = fma2(yd1, c.d1[1], mul2(yd2, c.d2[1]));
    x.d[2] = fma2(zd1, c.d1[2], mul2(zd2, c.d2[2]));
    F2 ko = mul2(a0, c.kc);
    ko = fma2(xs3, c.k3[0], ko);
    ko = fma2(ys3, c.k3[1], ko);
    ko = fma2(zs3, c.k3[2], ko);
    ko = fma2(xs2, c.k2[0], ko);
    ko = fma2(ys2, c.k2[1], ko);
    ko = fma2(zs2, c.k2[2], ko);
    ko = fma2(xs1, c.k1[0], ko);
    ko = fma2(ys1, c.k1[1], ko);
    x.ko = fma2(zs1, c.k1[2], ko);
    if (second) {
      x.dd[0] = fma2(xs1, c.e1[0], fma2(xs2, c.e2[0], mul2(a0, c.e0[0])));
      x.dd[1] = fma2(ys1, c.e1[1], fma2(ys2, c.e2[1], mul2(a0, c.e0[1])));
      x.dd[2] = fma2(zs1, c.e1[2], fma2(zs2, c.e2[2], mul2(a0, c.e0[2])));
    } else {
      x.dd[0] = x.dd[1] = x.dd[2] = F2(0.0f);
    }
    x.adv = F2(0.0f);
    return x;
  }

  // D_xb with b = y (s = kY) or z (s = kZ): with r1(o) = U(-2) - U(+2) and
  // r8(o) = U(+1) - U(-1) along x in the row at offset o across,
  // D_xb = w (r1(-2) - r1(2)) + 8 w (r8(-2) - r8(2) + r1(1) - r1(-1)) + 64 w (r8(1) - r8(-1)).
  __device__ __forceinline__ F2 mix_x(const float* p, int s, const F2* w) const {
    F2 r1[4], r8[4];  // rows -2, -1, 1, 2
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int o = (q < 2 ? q - 2 : q - 1) * s;
      const F2 am2 = L(p, o - 2), a0 = L(p, o), a2 = L(p, o + 2);
      r1[q] = sub2(am2, a2);
      r8[q] = F2(a0.y - am2.y, a2.x - a0.x);
    }
    const F2 x1 = sub2(r1[0], r1[3]);
    const F2 x8 = add2(sub2(r8[0], r8[3]), sub2(r1[2], r1[1]));
    const F2 x64 = sub2(r8[2], r8[1]);
    return fma2(x64, w[2], fma2(x8, w[1], mul2(x1, w[0])));
  }
  // D_yz: the same along y, rows across in z
  __device__ __forceinline__ F2 mix_yz(const float* p, const F2* w) const {
    F2 r1[4], r8[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int o = (q < 2 ? q - 2 : q - 1) * kZ;
      r1[q] = sub2(L(p, o - 2 * kY), L(p, o + 2 * kY));
      r8[q] = sub2(L(p, o + kY), L(p, o - kY));
    }
    const F2 x1 = sub2(r1[0], r1[3]);
    const F2 x8 = add2(sub2(r8[0], r8[3]), sub2(r1[2], r1[1]));
    const F2 x64 = sub2(r8[2], r8[1]);
    return fma2(x64, w[2], fma2(x8, w[1], mul2(x1, w[0])));
  }
  // mixed derivatives (xy, xz, yz) of the field whose cross was just read
  __device__ __forceinline__ void mix3(int, F2* out) const {
    const float* p = box();
    out[0] = mix_x(p, kY, pc->mx[0]);
    out[1] = mix_x(p, kZ, pc->mx[1]);
    out[2] = mix_yz(p, pc->mx[2]);
  }
};

// Forms of the RK combination fixed at compile time: the kernel is
// instantiated per form, so that its write phase carries one form's code and
// no branches on the stage (the generic form decides at run time).
//   kRk4First: RK4 stage 0 with the Kahan accumulator (U^n = the stage input)
//   kRk4Mid:   RK4 stages 1 and 2
//   kRk4Last:  RK4 stage 3 with the Kahan compensation
enum : int { kRkGeneric = 0, kRk4First = 1, kRk4Mid = 2, kRk4Last = 3 };

int rk_form(const StageArgs& s) {
  if (s.mode != 0 || s.rk != SF_RK4 || !s.kahan) return kRkGeneric;
  if (s.stage == 0) return s.un_alias ? kRk4First : kRkGeneric;
  return s.stage < 3 ? kRk4Mid : kRk4Last;
}

// Store of a value pair; MASKED (tiles that overhang the patch): vm bit 0
// for point i, bit 1 for point i + 1 (never set without bit 0).
template <bool MASKED>
__device__ __forceinline__ void store2(float* p, F2 v, unsigned vm) {
  if constexpr (MASKED) {
    if (vm == 3u) *reinterpret_cast<F2*>(p) = v;
    else if (vm & 1u) p[0] = v.x;
  } else {
    *reinterpret_cast<F2*>(p) = v;
  }
}

// RK stage combination of one field value pair (sf_common.cuh's
// stage_combine on pairs): writes the accumulator / Kahan term and returns
// the next stage input.
template <int FORM, bool MASKED = false>
__device__ __forceinline__ F2 stage_combine2(const PatchArgs<float>& a, const StageArgs& s,
                                             long long o, F2 centre, F2 un_m, F2 acc, F2 kh, F2 r,
                                             unsigned vm = 3u) {
  const F2 cn(a.c_next), ca(a.c_acc);
  if constexpr (FORM == kRk4First) {
    store2<MASKED>(a.acc + o, mul2(ca, r), vm);
    return fma2(cn, r, centre);
  } else if constexpr (FORM == kRk4Mid) {
    store2<MASKED>(a.acc + o, fma2(ca, r, acc), vm);
    return fma2(cn, r, un_m);
  } else if constexpr (FORM == kRk4Last) {
    const F2 inc = fma2(cn, r, acc);
    const F2 y = sub2(inc, kh);
    const F2 t = add2(un_m, y);
    store2<MASKED>(a.kh + o, sub2(sub2(t, un_m), y), vm);
    return t;
  }
  const F2 un = s.un_alias ? centre : un_m;
  F2 out;
  if (s.rk == SF_RK4) {
    if (s.stage == 0) {
      *reinterpret_cast<F2*>(a.acc + o) = s.kahan ? mul2(ca, r) : fma2(ca, r, un);
      out = fma2(cn, r, un);
    } else if (s.stage < 3) {
      *reinterpret_cast<F2*>(a.acc + o) = fma2(ca, r, acc);
      out = fma2(cn, r, un);
    } else if (!s.kahan) {
      out = fma2(cn, r, acc);
    } else {
      const F2 inc = fma2(cn, r, acc);
      const F2 y = sub2(inc, kh);
      const F2 t = add2(un, y);
      *reinterpret_cast<F2*>(a.kh + o) = sub2(sub2(t, un), y);
      out = t;
    }
  } else {
    const F2 dt(a.dt);
    if (s.stage == 0) out = fma2(dt, r, un);
    else if (s.stage == 1) out = fma2(F2(0.75f), un, mul2(F2(0.25f), fma2(dt, r, centre)));
    else out = fma2(un, F2(float(1.0 / 3.0)), mul2(F2(float(2.0 / 3.0)), fma2(dt, r, centre)));
  }
  return out;
}

// The stage write of the 25 fields of both points, right-hand sides parked
// in shared memory (r[f * stride]); the scheme of write_fields (batches of
// five fields with every read issued before the writes, periodic images of
// boundary points in one rolled pass at the end) on 64-bit accesses.
template <int FORM>
__device__ __forceinline__ void write_fields_pair(const PatchArgs<float>& a, const StageArgs& s,
                                                  long long c, int i, int j, int k, F2* r,
                                                  int stride) {
  if (FORM == kRkGeneric && s.mode == 1) {
    const long long oi = ((long long)k * a.n[1] + j) * a.n[0] + i;
#pragma unroll 1
    for (int f = 0; f < 25; ++f) {
      const F2 v = r[f * stride];
      a.nx[f * a.ninterior + oi] = v.x;
      a.nx[f * a.ninterior + oi + 1] = v.y;
    }
    return;
  }
  const bool rk4 = s.rk == SF_RK4;
  const bool need_centre = FORM == kRk4First || (FORM == kRkGeneric && (s.un_alias || !rk4));
  const bool need_un = FORM == kRk4Mid || FORM == kRk4Last || (FORM == kRkGeneric && !s.un_alias);
  const bool need_acc = FORM == kRk4Mid || FORM == kRk4Last || (FORM == kRkGeneric && rk4 && s.stage > 0);
  const bool need_kh = FORM == kRk4Last || (FORM == kRkGeneric && rk4 && s.stage == 3 && s.kahan);
  auto ld = [](const float* q) { return *reinterpret_cast<const F2*>(q); };
#pragma unroll 1
  for (int f0 = 0; f0 < 25; f0 += 5) {
    F2 cen[5], un[5], acc[5], kh[5], rr[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const long long o = (f0 + q) * a.sf + c;
      rr[q] = r[(f0 + q) * stride];
      cen[q] = need_centre ? ld(a.us + o) : F2(0.0f);
      un[q] = need_un ? ld(a.un + o) : F2(0.0f);
      acc[q] = need_acc ? ld(a.acc + o) : F2(0.0f);
      kh[q] = need_kh ? ld(a.kh + o) : F2(0.0f);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const long long o = (f0 + q) * a.sf + c;
      const F2 out = stage_combine2<FORM>(a, s, o, cen[q], un[q], acc[q], kh[q], rr[q]);
      *reinterpret_cast<F2*>(a.nx + o) = out;
      if (s.check_finite && !(finite_(out.x) && finite_(out.y))) atomicOr(s.status, ST_NONFINITE);
      r[(f0 + q) * stride] = out;
    }
  }
}

// The y and z periodic images of the pair's new values (rows and planes next
// to a face; r holds the values written), as aligned pairs: a shift in y or z
// keeps the pair on its 8-byte boundary.  The x ghost columns are written by
// write_x_images (RK4 forms) or by pair_xghost_kernel after the stage.
template <bool MASKED = false>
__device__ __forceinline__ void write_yz_images(const PatchArgs<float>& a, const StageArgs& s,
                                                long long c, int i, int j, int k, const F2* r,
                                                int stride, unsigned vm = 3u) {
  if (MASKED && !(vm & 1u)) return;
  const unsigned m = ghost_images(a, s, i, j, k).mask & ~3u;
  if (!m) return;
#pragma unroll 1
  for (int f = 0; f < 25; ++f) {
    const F2 v = r[f * stride];
    float* q = a.nx + f * a.sf + c;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      if (p && !(m & (p == 1 ? 16u : 32u))) continue;
      const long long oz = p == 0 ? 0 : (p == 1 ? 1 : -1) * (long long)a.n[2] * a.sz;
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        if (w && !(m & (w == 1 ? 4u : 8u))) continue;
        const long long oy = w == 0 ? 0 : (w == 1 ? 1 : -1) * (long long)a.n[1] * a.sy;
        if (p | w) store2<MASKED>(q + oz + oy, v, vm);
      }
    }
  }
}

// The x periodic images of the patch's boundary columns that lie in a tile
// (x0 .. x0 + 31, rows y0 .. y0 + 15 of plane k), written by the CTA from the
// tile's new values in shared memory (r: the pair of thread t for field f at
// r[f * stride + t]).  Interior x = 0..2 go to ghost x = n0 .. n0 + 2 (past
// the interior), x = n0 - 3 .. n0 - 1 to x = -3 .. -1; each also at the y and
// z image rows of its point, so that with write_yz_images every ghost value
// of the tile's points is written.  Spread over the CTA's threads.
__device__ __forceinline__ void write_x_images(const PatchArgs<float>& a, const StageArgs& s,
                                               int x0, int y0, int k, const F2* r, int stride,
                                               int tid) {
  const int n0 = a.n[0];
  const int lo0 = x0, lo1 = min(min(3, n0), x0 + 32);          // columns with an image at +n0
  const int hi0 = max(n0 - 3, x0), hi1 = min(n0, x0 + 32);      // columns with an image at -n0
  const int nlo = max(0, lo1 - lo0), nhi = max(0, hi1 - hi0), ncol = nlo + nhi;
  if (!ncol) return;
  const int rows = min(16, a.n[1] - y0);
#pragma unroll 1
  for (int v = tid; v < ncol * 16 * 25; v += stride) {
    const int f = v / (ncol * 16), rem = v - f * (ncol * 16), row = rem / ncol, cc = rem - row * ncol;
    if (row >= rows) continue;
    const bool low = cc < nlo;
    const int x = low ? lo0 + cc : hi0 + (cc - nlo);
    const int xl = x - x0;  // tile-local x of the source point
    // owner of (row, xl): warp row / 2, half-warp row % 2, lane xl / 2
    const F2 pr = r[f * stride + (row >> 1) * 32 + (row & 1) * 16 + (xl >> 1)];
    const float val = (xl & 1) ? pr.y : pr.x;
    const int j = y0 + row;
    const unsigned m = ghost_images(a, s, x, j, k).mask;
    const long long o = f * a.sf + (long long)(k + 3) * a.sz + (long long)(j + 3) * a.sy + (x + 3) +
                        (low ? n0 : -n0);
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      if (p && !(m & (p == 1 ? 16u : 32u))) continue;
      const long long oz = p == 0 ? 0 : (p == 1 ? 1 : -1) * (long long)a.n[2] * a.sz;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (q && !(m & (q == 1 ? 4u : 8u))) continue;
        const long long oy = q == 0 ? 0 : (q == 1 ? 1 : -1) * (long long)a.n[1] * a.sy;
        a.nx[o + oz + oy] = val;
      }
    }
  }
}

// The x ghost columns of every ghosted row (y and z over the whole ghosted
// range) of every field of u, from the same row's interior: ghost x = m
// (m < 3) takes x = m + n0, ghost x = n0 + 3 + m takes x = 3 + m.  Run after
// the stage kernel, whose fused y and z images have filled the interior part
// of the ghost rows.  One thread per ghost value.
__global__ void __launch_bounds__(256) pair_xghost_kernel(float* __restrict__ u, int nx, int ny,
                                                          int nz, long long sf) {
  const int Y = ny + 6, rows = Y * (nz + 6);
  const long long total = 25LL * rows * 6;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t % 6);
    const long long row = t / 6;
    const int f = (int)(row / rows), r = (int)(row - (long long)f * rows);
    const int z = r / Y, y = r - z * Y;
    float* b = u + f * sf + (long long)z * kSZ + (long long)y * kSY;
    if (q < 3) b[q] = b[q + nx];
    else b[nx + q] = b[q];
  }
}

}  // namespace

// The stage write with the RK inputs staged in the ring (the specialised
// forms): per block of up to 12 fields, the chunks of the NARR input arrays
// are acquired, every field of the block combined and stored, and the
// chunks released.  Array order: kRk4First: u_stage (= U^n); kRk4Mid: U^n,
// accumulator; kRk4Last: U^n, accumulator, Kahan term.
template <int FORM, int NARR, bool MASKED = false, typename Src>
__device__ __forceinline__ void write_fields_staged(const PatchArgs<float>& a, const StageArgs& s,
                                                    long long c, F2* r, int stride, Src& src,
                                                    int lpos, unsigned vm = 3u) {
  static_assert(NARR >= 1 && NARR <= 3, "staged arrays");
  auto ld = [](const float* q) { return *reinterpret_cast<const F2*>(q); };
  bool bad = false;  // a non-finite value written (reported once, at the end)
#pragma unroll 1
  for (int blk = 0; blk < 3; ++blk) {
    const float* in[NARR];
#pragma unroll
    for (int t = 0; t < NARR; ++t) in[t] = src.acquire(src.nfu + blk * NARR + t) + lpos;
    const int nf = min(kRkChunk, 25 - kRkChunk * blk);
#pragma unroll 1
    for (int q = 0; q < nf; ++q) {
      const int f = kRkChunk * blk + q;
      const long long o = f * a.sf + c;
      const F2 v0 = ld(in[0] + q * 512);
      const F2 v1 = NARR > 1 ? ld(in[NARR > 1 ? 1 : 0] + q * 512) : F2(0.0f);
      const F2 v2 = NARR > 2 ? ld(in[NARR > 2 ? 2 : 0] + q * 512) : F2(0.0f);
      const F2 rr = r[f * stride];
      // the first array is U^n (kRk4First: the stage input, which is U^n)
      const F2 out = stage_combine2<FORM, MASKED>(a, s, o, v0, v0, v1, v2, rr, vm);
      store2<MASKED>(a.nx + o, out, vm);
      if constexpr (MASKED)
        bad |= ((vm & 1u) && !finite_(out.x)) || ((vm & 2u) && !finite_(out.y));
      else
        bad |= !(finite_(out.x) && finite_(out.y));
      r[f * stride] = out;
    }
#pragma unroll
    for (int t = 0; t < NARR; ++t) src.release(src.nfu + blk * NARR + t);
  }
  if (s.check_finite && bad) atomicOr(s.status, ST_NONFINITE);
}

// Tensor maps of the RK input arrays of a stage form (unused ones zero).
struct RkMaps {
  CUtensorMap m[3];
};

// One tile of 32 x 16 points of plane k, lower corner (x0, y0): the stencil
// boxes staged through the ring, the right-hand side, the stage write and the
// periodic images of its points.  BATCH: the patch's strides come from `a`
// and the tile may overhang the patch (points outside write nothing, their
// centre reads are clamped into the patch); otherwise the compile-time
// strides of the padded 96^3-class layout and whole tiles.
template <typename H2, int W, int KS, int FORM, bool BATCH>
__device__ __forceinline__ void pair_tile(const CUtensorMap* map, const CUtensorMap* rkmaps,
                                          const PatchArgs<float>& a, const StageArgs& s,
                                          const Z4Coef<float>& zc, const PairCoef* pc, int x0,
                                          int y0, int k, unsigned char* smem) {
  constexpr int NARR = FORM == kRk4First ? 1 : (FORM == kRk4Mid ? 2 : (FORM == kRk4Last ? 3 : 0));
  static_assert(!BATCH || NARR > 0, "batched tiles take the RK4 stage forms");
  using C = PCfg<W, KS>;
  float* tiles = reinterpret_cast<float*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::kBarOffset);
  uint64_t* empty = full + KS;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (tid == 0) {
    for (int q = 0; q < KS; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], W);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  const int px = 2 * (threadIdx.x & 15);
  const int ly = 2 * threadIdx.y + (threadIdx.x >> 4);
  const int i = x0 + px;
  const int j = y0 + ly;
  long long c;
  unsigned vm = 3u;  // bit 0: point i in the patch, bit 1: point i + 1
  if constexpr (BATCH) {
    vm = j < a.n[1] ? (i < a.n[0] ? 1u : 0u) | (i + 1 < a.n[0] ? 2u : 0u) : 0u;
    const int ic = min(i, (a.n[0] - 1) & ~1), jc = min(j, a.n[1] - 1);
    c = (long long)(k + 3) * a.sz + (long long)(jc + 3) * a.sy + (ic + 3);
  } else {
    c = (long long)(k + 3) * kSZ + (long long)(j + 3) * kSY + (i + 3);
  }
  if (NARR == 0 && (threadIdx.x & 15) == 0 && s.mode == 0) {
    // generic form (RK inputs read from global memory in the write phase):
    // the row's 32 points start on a 16-byte boundary, prefetch their 128 B
    // of every field the RK combination reads.  The RK4 forms stage those
    // inputs through the TMA ring, where a prefetch only competes with the
    // stencil boxes.
    if (!s.un_alias) prefetch_rows<128>(a.un + c, a.sf);
    if (s.rk == SF_RK4 && s.stage > 0) prefetch_rows<128>(a.acc + c, a.sf);
    if (s.kahan && s.stage == 3) prefetch_rows<128>(a.kh + c, a.sf);
  }
  PairSrc<W, KS, NARR> src;
  src.u = a.us + c;
  src.F = a.sf;
  src.pc = pc;
  src.tiles = tiles;
  src.full = full;
  src.empty = empty;
  src.map = map;
  src.status = s.status;
  src.local = (3 * C::TY + ly + 3) * kXB + px + 4;
  src.use = 0;
  src.cur = 0;
  src.nfu = zc.shift_frozen ? 22 : 25;
  src.nuses = src.nfu + 3 * NARR;
  src.done = 0;
  src.rkmap = rkmaps;
  src.rx = x0 + 4;  // tensor x = ghosted x + 1 of point x0
  src.ry = y0 + 3;
  src.rz = k + 3;
  src.issued = 0;
  src.gx = x0;  // tensor x = ghosted x + 1; the box starts 4 before point x0
  src.gy = y0;
  src.gz = k;
  src.leader = tid == 0;
  src.lane0 = threadIdx.x == 0;
  src.dead = false;
  src.prologue();
  F2* rbuf = reinterpret_cast<F2*>(smem + C::kRbufOffset);
  F2 be[3];
  z4_rhs<F2, H2, false>(zc, src, be, [&](int f, F2 r, F2) { rbuf[f * C::kThreads + tid] = r; });
  if constexpr (NARR > 0)
    write_fields_staged<FORM, NARR, BATCH>(a, s, c, rbuf + tid, C::kThreads, src, ly * 32 + px, vm);
  else
    write_fields_pair<FORM>(a, s, c, i, j, k, rbuf + tid, C::kThreads);
  write_yz_images<BATCH>(a, s, c, i, j, k, rbuf + tid, C::kThreads, vm);
  if constexpr (NARR > 0) {
    if (s.ghosts && s.mode == 0) {
      __syncthreads();  // every new value of the tile is in rbuf
      write_x_images(a, s, x0, y0, k, rbuf, C::kThreads, tid);
    }
    src.final_finish();
  }
}

template <typename H2, int W, int KS, int FORM>
__global__ void __launch_bounds__(32 * W, 1)
    z4_pair_kernel(const __grid_constant__ CUtensorMap map, PatchArgs<float> a, StageArgs s,
                   Z4Coef<float> zc, const __grid_constant__ PairCoef pc,
                   const __grid_constant__ RkMaps rk) {
  extern __shared__ __align__(128) unsigned char smem[];
  // planes next to the z faces first (their tiles also write the z images, the
  // slowest tiles), so that the partial last wave holds plain tiles
  const int k = (int)((blockIdx.z + 3 * gridDim.z - 3) % gridDim.z);
  pair_tile<H2, W, KS, FORM, false>(&map, rk.m, a, s, zc, &pc, blockIdx.x * 32,
                                    blockIdx.y * PCfg<W, KS>::BY, k, smem);
}

// Any patch size on the one-float row offset layout (runtime strides, tiles
// that overhang the patch), the RK4 Kahan forms: one CTA per 32 x 16 tile.
template <typename H2, int W, int KS, int FORM>
__global__ void __launch_bounds__(32 * W, 1)
    z4_pair_any_kernel(const __grid_constant__ CUtensorMap map, PatchArgs<float> a, StageArgs s,
                       Z4Coef<float> zc, const __grid_constant__ PairCoef pc,
                       const __grid_constant__ RkMaps rk) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int k = (int)((blockIdx.z + 3 * gridDim.z - 3) % gridDim.z);
  pair_tile<H2, W, KS, FORM, true>(&map, rk.m, a, s, zc, &pc, blockIdx.x * 32,
                                   blockIdx.y * PCfg<W, KS>::BY, k, smem);
}

// The same over the tiles of many patches (the float CCZ4 patches of a batch
// on the two-point layout): one CTA per tile, the tile's patch from `tl`, its
// stage arguments and stencil weights copied into shared memory, its tensor
// maps from `maps` (six per patch: RK chunks of U^n, accumulator and Kahan
// term, then the stencil boxes of the u_n, u_stage and u_next buffer roles;
// `role` picks the stage input).
template <typename H2, int W, int KS, int FORM>
__global__ void __launch_bounds__(32 * W, 1)
    z4_pair_batch_kernel(const CUtensorMap* __restrict__ maps, int role,
                         const PatchArgs<float>* __restrict__ args, const PairCoef* __restrict__ coefs,
                         const TmaTile* __restrict__ tl, StageArgs s, Z4Coef<float> zc) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ PatchArgs<float> pa;
  __shared__ PairCoef pcs;
  const TmaTile w = tl[blockIdx.x];
  {
    static_assert(sizeof(PatchArgs<float>) % 4 == 0 && sizeof(PairCoef) % 4 == 0, "word copy");
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int* from = reinterpret_cast<const int*>(args + w.patch);
    int* to = reinterpret_cast<int*>(&pa);
    for (int q = tid; q < (int)(sizeof(PatchArgs<float>) / 4); q += 32 * W) to[q] = from[q];
    from = reinterpret_cast<const int*>(coefs + w.patch);
    to = reinterpret_cast<int*>(&pcs);
    for (int q = tid; q < (int)(sizeof(PairCoef) / 4); q += 32 * W) to[q] = from[q];
  }
  // (pair_tile's first barrier orders these copies before their reads)
  const CUtensorMap* pm = maps + 6 * (size_t)w.patch;
  pair_tile<H2, W, KS, FORM, true>(pm + 3 + role, pm, pa, s, zc, &pcs, w.x0, w.y0, w.z0, smem);
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn_pair() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool offset_aligned(const void* q) {
  return q && reinterpret_cast<uintptr_t>(q) % 16 == 4;
}

template <typename H2, bool ANY = false>
sf_status launch_pair(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                      void* rhs_out, cudaStream_t st) {
  using C = PCfg<kW, kKS>;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn_pair();
  if (!enc) return set_error(SF_ECUDA, "cuTensorMapEncodeTiled not available");
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  // tensor x = ghosted x + 1: the map starts at the float before ghost point 0
  const cuuint64_t dims[4] = {(cuuint64_t)(p.n[0] + 7), (cuuint64_t)(p.n[1] + 6),
                              (cuuint64_t)(p.n[2] + 6), 25};
  const cuuint64_t strides[3] = {(cuuint64_t)p.sy * 4, (cuuint64_t)p.sz * 4, (cuuint64_t)p.sf * 4};
  const cuuint32_t box[4] = {kXB, (cuuint32_t)C::TY, kTZ, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  void* base = static_cast<char*>(p.u_stage) - 4;
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(SF_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(z4_pair_kernel<H2, kW, kKS, kRkGeneric>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    cudaFuncSetAttribute(z4_pair_kernel<H2, kW, kKS, kRk4First>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    cudaFuncSetAttribute(z4_pair_kernel<H2, kW, kKS, kRk4Mid>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    cudaFuncSetAttribute(z4_pair_kernel<H2, kW, kKS, kRk4Last>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    if constexpr (ANY) {
      cudaFuncSetAttribute(z4_pair_any_kernel<H2, kW, kKS, kRk4First>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
      cudaFuncSetAttribute(z4_pair_any_kernel<H2, kW, kKS, kRk4Mid>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
      cudaFuncSetAttribute(z4_pair_any_kernel<H2, kW, kKS, kRk4Last>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    }
  });
  PatchArgs<float> a = make_args<float>(prm, p, stage, 25, rhs_out);
  const Z4Coef<float> zc = z4_coef<float>(prm);
  const PairCoef pc = pair_coef(prm, p);
  const int form = rk_form(s);
  // the RK inputs of the form, staged through the ring: boxes of the tile's
  // 32 x 16 points x 12 fields
  RkMaps rk;
  memset(&rk, 0, sizeof(rk));
  {
    const void* arrs[3] = {nullptr, nullptr, nullptr};
    if (form == kRk4First) arrs[0] = p.u_stage;
    if (form == kRk4Mid || form == kRk4Last) {
      arrs[0] = p.u_n;
      arrs[1] = p.acc;
    }
    if (form == kRk4Last) arrs[2] = p.kahan;
    const cuuint32_t rbox[4] = {32, (cuuint32_t)C::BY, 1, kRkChunk};
    for (int q = 0; q < 3; ++q) {
      if (!arrs[q]) continue;
      CUresult rr = enc(&rk.m[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                        static_cast<char*>(const_cast<void*>(arrs[q])) - 4, dims, strides, rbox,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (rr != CUDA_SUCCESS) return set_error(SF_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)rr);
    }
  }
  const dim3 block(32, kW, 1);
  if constexpr (ANY) {
    const dim3 grid((p.n[0] + 31) / 32, (p.n[1] + C::BY - 1) / C::BY, p.n[2]);
    switch (form) {
      case kRk4First:
        z4_pair_any_kernel<H2, kW, kKS, kRk4First><<<grid, block, C::kSmemBytes, st>>>(map, a, s, zc, pc, rk);
        break;
      case kRk4Mid:
        z4_pair_any_kernel<H2, kW, kKS, kRk4Mid><<<grid, block, C::kSmemBytes, st>>>(map, a, s, zc, pc, rk);
        break;
      default:
        z4_pair_any_kernel<H2, kW, kKS, kRk4Last><<<grid, block, C::kSmemBytes, st>>>(map, a, s, zc, pc, rk);
    }
    return after_launch("z4_pair_any_kernel");
  }
  dim3 grid(p.n[0] / 32, p.n[1] / C::BY, p.n[2]);
  switch (form) {
    case kRk4First:
      z4_pair_kernel<H2, kW, kKS, kRk4First><<<grid, block, C::kSmemBytes, st>>>(map, a, s, zc, pc, rk);
      break;
    case kRk4Mid:
      z4_pair_kernel<H2, kW, kKS, kRk4Mid><<<grid, block, C::kSmemBytes, st>>>(map, a, s, zc, pc, rk);
      break;
    case kRk4Last:
      z4_pair_kernel<H2, kW, kKS, kRk4Last><<<grid, block, C::kSmemBytes, st>>>(map, a, s, zc, pc, rk);
      break;
    default:
      z4_pair_kernel<H2, kW, kKS, kRkGeneric><<<grid, block, C::kSmemBytes, st>>>(map, a, s, zc, pc, rk);
  }
  sf_status e = after_launch("z4_pair_kernel");
  // the RK4 forms write the x images themselves
  if (e || !s.ghosts || s.mode == 1 || form != kRkGeneric) return e;
  const long long total = 25LL * (p.n[1] + 6) * (p.n[2] + 6) * 6;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
  pair_xghost_kernel<<<blocks, 256, 0, st>>>(a.nx, p.n[0], p.n[1], p.n[2], p.sf);
  return after_launch("pair_xghost_kernel");
}

}  // namespace

// The two-point kernel serves float storage with centred advection on the
// padded 96^3-class layout with the one-float row offset: 3 ghosts, row
// pitch 104 floats, plane pitch 104 x 102, field pitch a multiple of 4
// floats, every array 4 bytes past a 16-byte boundary, whole 32 x 16 tiles.
bool z4_pair_eligible(const sf_params& prm, const sf_patch& p, const void* rhs_out) {
  using C = PCfg<kW, kKS>;
  if (p.system != SF_Z4 || p.precision == SF_FP64 || prm.lopsided) return false;
  if (p.ghost != 3 || p.sy != kSY || p.sz != kSZ || p.sf % 4) return false;
  if (p.n[0] % 32 || p.n[1] % C::BY || p.n[0] + 7 > kSY || p.n[1] + 6 > 102) return false;
  if (!offset_aligned(p.u_stage)) return false;
  if (rhs_out) return true;  // RHS output: scalar stores
  for (const void* q : {(const void*)p.u_n, (const void*)p.u_next, (const void*)p.acc})
    if (q && !offset_aligned(q)) return false;
  if (p.kahan && !offset_aligned(p.kahan)) return false;
  return true;
}

sf_status launch_z4_pair(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                         void* rhs_out, cudaStream_t st) {
  if (p.precision == SF_FP32_BULK_DW) return launch_pair<DW2>(prm, p, s, stage, rhs_out, st);
  return launch_pair<D2>(prm, p, s, stage, rhs_out, st);
}

// Any size on the one-float row offset layout: double-word islands, the RK4
// Kahan stage forms, pitches of a multiple of 4 floats with room for the
// float before each row, every array 4 bytes past a 16-byte boundary.
bool z4_pair_any_eligible(const sf_params& prm, const sf_patch& p, const StageArgs& s,
                          const void* rhs_out) {
  if (rhs_out || rk_form(s) == kRkGeneric) return false;
  return z4_pair_batch_eligible(prm, p);
}

sf_status launch_z4_pair_any(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                             cudaStream_t st) {
  return launch_pair<DW2, true>(prm, p, s, stage, nullptr, st);
}

// Batch form: float CCZ4 with double-word islands, centred advection, 3
// ghosts, row / plane / field pitches of a multiple of 4 floats with room for
// the float before each row (row pitch >= n0 + 7), every array 4 bytes past
// a 16-byte boundary; any interior size (tiles may overhang).
bool z4_pair_batch_eligible(const sf_params& prm, const sf_patch& p) {
  if (p.system != SF_Z4 || p.precision != SF_FP32_BULK_DW || prm.lopsided) return false;
  if (p.ghost != 3 || p.sy % 4 || p.sz % 4 || p.sf % 4 || p.sy < p.n[0] + 7) return false;
  for (const void* q : {(const void*)p.u_n, (const void*)p.u_stage, (const void*)p.u_next,
                        (const void*)p.acc, (const void*)p.kahan})
    if (!offset_aligned(q)) return false;
  return true;
}

size_t z4_pair_coef_bytes() { return sizeof(PairCoef); }

// The six tensor maps of a batch patch (RK chunks of u_n, acc, kahan; stencil
// boxes of u_n, u_stage, u_next) and its stencil weights.
sf_status encode_z4_pair_batch(void* maps6, void* coef, const sf_params& prm, const sf_patch& p) {
  using C = PCfg<kW, kKS>;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn_pair();
  if (!enc) return set_error(SF_ECUDA, "cuTensorMapEncodeTiled not available");
  const cuuint64_t dims[4] = {(cuuint64_t)(p.n[0] + 7), (cuuint64_t)(p.n[1] + 6),
                              (cuuint64_t)(p.n[2] + 6), 25};
  const cuuint64_t strides[3] = {(cuuint64_t)p.sy * 4, (cuuint64_t)p.sz * 4, (cuuint64_t)p.sf * 4};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const cuuint32_t rbox[4] = {32, (cuuint32_t)C::BY, 1, kRkChunk};
  const cuuint32_t sbox[4] = {kXB, (cuuint32_t)C::TY, kTZ, 1};
  const void* arr[6] = {p.u_n, p.acc, p.kahan, p.u_n, p.u_stage, p.u_next};
  for (int q = 0; q < 6; ++q) {
    CUtensorMap m;
    memset(&m, 0, sizeof(m));
    // tensor x = ghosted x + 1: the map starts at the float before ghost point 0
    CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                     static_cast<char*>(const_cast<void*>(arr[q])) - 4, dims, strides,
                     q < 3 ? rbox : sbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(SF_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    memcpy(static_cast<char*>(maps6) + q * sizeof(CUtensorMap), &m, sizeof(m));
  }
  const PairCoef pc = pair_coef(prm, p);
  memcpy(coef, &pc, sizeof(pc));
  return SF_OK;
}

sf_status launch_z4_pair_batch(const sf_params& prm, const void* d_maps, int role,
                               const PatchArgs<float>* d_args, const void* d_coefs,
                               const TmaTile* d_tiles, int ntiles, const StageArgs& s,
                               cudaStream_t st) {
  if (ntiles <= 0) return SF_OK;
  using C = PCfg<kW, kKS>;
  const int form = rk_form(s);
  if (form == kRkGeneric) return set_error(SF_EINVAL, "batched two-point tiles need the RK4 Kahan forms");
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(z4_pair_batch_kernel<DW2, kW, kKS, kRk4First>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    cudaFuncSetAttribute(z4_pair_batch_kernel<DW2, kW, kKS, kRk4Mid>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    cudaFuncSetAttribute(z4_pair_batch_kernel<DW2, kW, kKS, kRk4Last>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
  });
  const Z4Coef<float> zc = z4_coef<float>(prm);
  const CUtensorMap* maps = static_cast<const CUtensorMap*>(d_maps);
  const PairCoef* coefs = static_cast<const PairCoef*>(d_coefs);
  const dim3 block(32, kW, 1);
  switch (form) {
    case kRk4First:
      z4_pair_batch_kernel<DW2, kW, kKS, kRk4First><<<ntiles, block, C::kSmemBytes, st>>>(
          maps, role, d_args, coefs, d_tiles, s, zc);
      break;
    case kRk4Mid:
      z4_pair_batch_kernel<DW2, kW, kKS, kRk4Mid><<<ntiles, block, C::kSmemBytes, st>>>(
          maps, role, d_args, coefs, d_tiles, s, zc);
      break;
    default:
      z4_pair_batch_kernel<DW2, kW, kKS, kRk4Last><<<ntiles, block, C::kSmemBytes, st>>>(
          maps, role, d_args, coefs, d_tiles, s, zc);
  }
  return after_launch("z4_pair_batch_kernel");
}

}  // namespace sf
