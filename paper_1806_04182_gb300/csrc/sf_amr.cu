// Inter-patch data movement of the AMR level loop (Sec. III, Sec. III.A):
//   sf_copy_boxes  - same-level ghost synchronisation (box copies between
//                    patch arrays) and, with a source step R, restriction by
//                    injection (coarse point i <- fine point R i);
//   sf_prolong     - 6-point (5th-order) Lagrange prolongation from a coarse
//                    patch onto fine points, as a tensor product of 1D
//                    interpolations whose weights l_j(t) are tabulated on the
//                    host for the R fractional positions t = r/R;
//   sf_bor_prolong - the same prolongation of the fine-time values of
//                    Berger-Oliger without order reduction (Sec. III.B,
//                    App. C-D), a fixed linear combination of the coarse
//                    stage states whose coefficients the host derives.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "sf_internal.cuh"

namespace sf {

// 256 descriptors and their block offsets (27.7 KB) travel as kernel
// parameters, so a launch needs no device-side table: the 26 halo boxes of
// each of 8 patches, or the six slabs of many ghost shells, go in one launch.
constexpr int kBoxesPerLaunch = 256;

struct BoxBatch {
  sf_box_copy b[kBoxesPerLaunch];
  int end[kBoxesPerLaunch];  // cumulative blocks per box
  int n;
};

// Each box gets blocks in proportion to its size (a corner box one, a face
// box hundreds); block b of the launch belongs to the first box whose end
// exceeds b.  Threads run over the box's points with 32-bit index arithmetic
// (the host checks that a box holds < 2^31 values), kCopyIlp points per pass
// with their loads issued together: a copy is one load and one store, so a
// thread with a single point would spend its life waiting on one load.  The
// launch is latency-bound (thin boxes, rows of 3 values in the x faces); 8
// loads in flight per thread measured faster than 4 (0.044 against 0.046 ms
// for the 208 halo boxes of eight 48^3 patches) and than 16 (0.049 ms, 128
// registers).
constexpr int kCopyIlp = 8;

template <typename T>
__global__ void __launch_bounds__(256) copy_boxes_kernel(BoxBatch bb) {
  int lo = 0, hi = bb.n - 1;  // first box with end > blockIdx.x
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (bb.end[mid] > (int)blockIdx.x) hi = mid;
    else lo = mid + 1;
  }
  const sf_box_copy& b = bb.b[lo];
  const unsigned first = lo ? (unsigned)bb.end[lo - 1] : 0u;
  const unsigned nblk = (unsigned)bb.end[lo] - first;
  const unsigned ex = (unsigned)b.ext[0], ey = (unsigned)b.ext[1], ez = (unsigned)b.ext[2];
  const unsigned total = ex * ey * ez * (unsigned)b.nf;
  const T* src = static_cast<const T*>(b.src);
  T* dst = static_cast<T*>(b.dst);
  const unsigned stride = nblk * blockDim.x;  // <= 1024 x 256
  for (unsigned t0 = (blockIdx.x - first) * blockDim.x + threadIdx.x; t0 < total;
       t0 += kCopyIlp * stride) {
    T v[kCopyIlp];
    long long d[kCopyIlp];
#pragma unroll
    for (int u = 0; u < kCopyIlp; ++u) {
      const unsigned t = t0 + u * stride;
      if (t >= total) break;
      unsigned r = t;
      const unsigned x = r % ex;
      r /= ex;
      const unsigned y = r % ey;
      r /= ey;
      const unsigned z = r % ez;
      const unsigned f = r / ez;
      const long long si = b.src_off + f * b.src_sf + (long long)z * b.src_step * b.src_sz +
                           (long long)y * b.src_step * b.src_sy + (long long)x * b.src_step;
      d[u] = b.dst_off + f * b.dst_sf + (long long)z * b.dst_sz + (long long)y * b.dst_sy + x;
      v[u] = __ldg(src + si);
    }
#pragma unroll
    for (int u = 0; u < kCopyIlp; ++u)
      if (t0 + u * stride < total) dst[d[u]] = v[u];
  }
}

// One output box of a prolongation launch: fine points origin..origin+ext-1
// written to out with element strides (osy, osz, osf); kind = the box's tile
// shape (kTileShapes), p[3] = that tile of fine points, t[3] = tiles per axis.
struct PBox {
  int origin[3], ext[3], p[3], t[3];
  int kind;
  void* out;
  long long osy, osz, osf;
};
constexpr int kMaxPBoxes = 16;

struct ProlongArgs {
  double w[8][6];      // Lagrange weights l_j(r/R), r = 0..R-1, nodes -2..3
  float wf[8][6];      // the same, rounded to float (float arrays)
  int R;
  int n[3], g;
  long long sy, sz, sf;          // coarse strides
  int nf;
  int nbox;
  int tiles_end[kMaxPBoxes];     // cumulative CTA counts (tiles x fields) per box
  PBox box[kMaxPBoxes];
};

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Value of the coarse data at a node: NS == 0 reads one array; otherwise a
// fixed linear combination of NS+1 arrays,  S_0 + sum_m c_m (S_m - S_0)
// (the BOR fine-time values below).
template <typename T>
struct Combo {
  const T* s[5];
  double c[4];
};

// Formed in the arrays' own precision: float arrays hold values to float
// accuracy, and the combination and interpolation weights sum to one.
template <typename T, int NS>
__device__ __forceinline__ T node_value(const Combo<T>& cb, long long o) {
  T v = __ldg(cb.s[0] + o);
  if (NS > 0) {
    const T u = v;
#pragma unroll
    for (int m = 1; m <= NS; ++m) v += T(cb.c[m - 1]) * (__ldg(cb.s[m] + o) - u);
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T lagrange_w(const ProlongArgs& p, int r, int q);
template <>
__device__ __forceinline__ double lagrange_w<double>(const ProlongArgs& p, int r, int q) {
  return p.w[r][q];
}
template <>
__device__ __forceinline__ float lagrange_w<float>(const ProlongArgs& p, int r, int q) {
  return p.wf[r][q];
}

// Fine tile of PX x PY x PZ points per CTA, chosen per box: 32 x 8 x 4 for a
// thick box; for a box at most 4 points thin along one axis (the slabs of a
// ghost shell) a tile 4 points deep along that axis and wider along the
// others, 4 x 16 x 16, 32 x 4 x 16 or 32 x 16 x 4, so that the coarse nodes
// a tile stages serve more fine points.  Along each axis the tile's points
// reach coarse nodes floor(F/R) - 2 .. floor(F/R) + 3, at most (P - 1)/R + 7
// of them (P + 6 for R = 1).  The kernel stages those nodes in shared memory
// (after the BOR combination, once per node), then interpolates separably:
// along x into tx, along y into ty, along z into the output.  One field per
// CTA, so thin boxes still fill the GPU.  18 weighted sums per fine point and
// field instead of 216, and the 6-point order of summation is the tensor
// product's (x innermost).
//
// The tile shapes are compile-time constants of the tile body, so every
// index into the staged arrays splits by constant divisors; the fine offsets'
// coarse node and weight row along each axis come from small tables the CTA
// builds once (the only divisions by R).  The staged extents are sized for
// R = 1 (P + 6 nodes) or for any R >= 2 ((P - 1)/2 + 7 nodes, about half),
// a second instance of the body.
struct TileShape {
  int px, py, pz;
};
constexpr TileShape kTileShapes[4] = {{32, 8, 4}, {4, 16, 16}, {32, 4, 16}, {32, 16, 4}};
constexpr int kThick = 0, kThinX = 1, kThinY = 2, kThinZ = 3;
constexpr int kProlongThreads = 256;
constexpr int kProlongTableBytes = 8 * 6 * 8 + 3 * 32 * 4;  // weights [R][6], node/row tables [3][32]
// coarse nodes a tile of P fine points reaches along an axis, for R >= rmin
constexpr int node_span(int p, int rmin) { return (p - 1) / rmin + 7; }
constexpr int prolong_elems(TileShape t, int rmin) {
  return node_span(t.pz, rmin) * node_span(t.py, rmin) * node_span(t.px, rmin) +
         node_span(t.pz, rmin) * node_span(t.py, rmin) * t.px + node_span(t.pz, rmin) * t.py * t.px;
}
constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int kProlongMaxElems =
    cmax(cmax(prolong_elems(kTileShapes[0], 1), prolong_elems(kTileShapes[1], 1)),
         cmax(prolong_elems(kTileShapes[2], 1), prolong_elems(kTileShapes[3], 1)));
template <typename T>
constexpr int prolong_smem_bytes(int elems) {
  return elems * (int)sizeof(T) + kProlongTableBytes;
}
template <typename T>
constexpr int prolong_smem_max() {
  return prolong_smem_bytes<T>(kProlongMaxElems);
}
static_assert(prolong_smem_max<double>() <= 227 * 1024, "prolongation tile fits shared memory");

static int tile_for(const int* ext) {
  if (ext[0] <= 4) return kThinX;
  if (ext[1] <= 4) return kThinY;
  if (ext[2] <= 4) return kThinZ;
  return kThick;
}

template <typename T, int NS, int RMIN, int PX, int PY, int PZ>
__device__ __forceinline__ void prolong_tile(const Combo<T>& cb, const ProlongArgs& p, const PBox& B,
                                             int local, unsigned char* raw) {
  constexpr int CXM = node_span(PX, RMIN), CYM = node_span(PY, RMIN), CZM = node_span(PZ, RMIN);
  constexpr int NT = kProlongThreads;
  static_assert(NT % PX == 0 && PX <= 32 && PY <= 32 && PZ <= 32, "tile shape");
  constexpr int ROWS = NT / PX;           // rows of a pass per sweep of the CTA
  T* cn = reinterpret_cast<T*>(raw);      // [CZM][CYM][CXM] staged nodes
  T* tx = cn + CZM * CYM * CXM;           // [CZM][CYM][PX]
  T* ty = tx + CZM * CYM * PX;            // [CZM][PY][PX]
  T* wt = ty + CZM * PY * PX;             // [R][6] Lagrange weights
  int* tab = reinterpret_cast<int*>(wt + 48);  // [3][32]: 8 x first node + weight row
  const int R = p.R;
  const int xt = local % B.t[0];
  local /= B.t[0];
  const int yt = local % B.t[1];
  local /= B.t[1];
  const int zt = local % B.t[2];
  const int f = local / B.t[2];
  T* out = static_cast<T*>(B.out);
  const int F0[3] = {B.origin[0] + xt * PX, B.origin[1] + yt * PY, B.origin[2] + zt * PZ};
  const int P[3] = {PX, PY, PZ};
  int nv[3], lo[3], nc[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    nv[d] = min(P[d], B.origin[d] + B.ext[d] - F0[d]);        // valid fine points in the tile
    lo[d] = floordiv(F0[d], R) - 2;                            // first coarse node
    nc[d] = floordiv(F0[d] + nv[d] - 1, R) + 3 - lo[d] + 1;    // coarse nodes spanned
  }
  const int tid = threadIdx.x;
  if (tid < 48) {
    wt[tid] = tid < 6 * R ? lagrange_w<T>(p, tid / 6, tid % 6) : T(0);
  } else if (tid >= 64 && tid < 64 + 96) {
    const int d = (tid - 64) >> 5, i = tid & 31;
    const int F = (d == 0 ? F0[0] : d == 1 ? F0[1] : F0[2]) + i;
    const int b = floordiv(F, R);
    tab[tid - 64] = (b - 2 - (d == 0 ? lo[0] : d == 1 ? lo[1] : lo[2])) * 8 + (F - b * R);
  }
  // coarse nodes (the BOR combination formed once per node)
  {
    const long long o0 = f * p.sf + (long long)(lo[2] + p.g) * p.sz + (long long)(lo[1] + p.g) * p.sy +
                         (lo[0] + p.g);
    const int end = nc[2] * CYM * CXM;
#pragma unroll 4
    for (int t = tid; t < end; t += NT) {
      const int cx = t % CXM, cy = (t / CXM) % CYM, cz = t / (CXM * CYM);
      if (cx < nc[0] && cy < nc[1])
        cn[t] = node_value<T, NS>(cb, o0 + (long long)cz * p.sz + (long long)cy * p.sy + cx);
    }
  }
  __syncthreads();
  const int xi = tid % PX;  // the same x offset in every sweep (NT is a multiple of PX)
  {
    const int e = tab[xi];
    const T* w = wt + (e & 7) * 6;
    T wx[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) wx[q] = w[q];
    const int s0 = e >> 3;
    const int end = nc[2] * CYM;
    if (xi < nv[0])
      for (int row = tid / PX; row < end; row += ROWS) {
        if (row % CYM >= nc[1]) continue;
        const T* c = cn + row * CXM + s0;
        T v = T(0);
#pragma unroll
        for (int q = 0; q < 6; ++q) v += wx[q] * c[q];
        tx[row * PX + xi] = v;
      }
  }
  __syncthreads();
  {
    const int end = nc[2] * PY;
    if (xi < nv[0])
      for (int row = tid / PX; row < end; row += ROWS) {
        const int yi = row % PY, cz = row / PY;
        if (yi >= nv[1]) continue;
        const int e = tab[32 + yi];
        const T* c = tx + (cz * CYM + (e >> 3)) * PX + xi;
        const T* w = wt + (e & 7) * 6;
        T v = T(0);
#pragma unroll
        for (int q = 0; q < 6; ++q) v += w[q] * c[q * PX];
        ty[row * PX + xi] = v;
      }
  }
  __syncthreads();
  if (xi < nv[0]) {
    T* o = out + f * B.osf + (long long)(F0[2] - B.origin[2]) * B.osz +
           (long long)(F0[1] - B.origin[1]) * B.osy + (F0[0] - B.origin[0]) + xi;
    static_assert(PX * PY * PZ % NT == 0, "whole sweeps");
#pragma unroll
    for (int k = 0; k < PX * PY * PZ / NT; ++k) {
      const int t = tid + k * NT;
      const int yi = (t / PX) % PY, zi = t / (PX * PY);
      if (yi >= nv[1] || zi >= nv[2]) continue;
      const int e = tab[64 + zi];
      const T* c = ty + ((e >> 3) * PY + yi) * PX + xi;
      const T* w = wt + (e & 7) * 6;
      T v = T(0);
#pragma unroll
      for (int q = 0; q < 6; ++q) v += w[q] * c[q * PY * PX];
      o[(long long)zi * B.osz + (long long)yi * B.osy] = v;
    }
  }
}

template <typename T, int NS, int RMIN>
__device__ __forceinline__ void prolong_kind(const Combo<T>& cb, const ProlongArgs& p, const PBox& B,
                                             int local, unsigned char* raw) {
  switch (B.kind) {
    case kThinX:
      prolong_tile<T, NS, RMIN, kTileShapes[kThinX].px, kTileShapes[kThinX].py,
                   kTileShapes[kThinX].pz>(cb, p, B, local, raw);
      break;
    case kThinY:
      prolong_tile<T, NS, RMIN, kTileShapes[kThinY].px, kTileShapes[kThinY].py,
                   kTileShapes[kThinY].pz>(cb, p, B, local, raw);
      break;
    case kThinZ:
      prolong_tile<T, NS, RMIN, kTileShapes[kThinZ].px, kTileShapes[kThinZ].py,
                   kTileShapes[kThinZ].pz>(cb, p, B, local, raw);
      break;
    default:
      prolong_tile<T, NS, RMIN, kTileShapes[kThick].px, kTileShapes[kThick].py,
                   kTileShapes[kThick].pz>(cb, p, B, local, raw);
  }
}

template <typename T, int NS>
__global__ void __launch_bounds__(kProlongThreads) prolong_kernel(Combo<T> cb, ProlongArgs p) {
  extern __shared__ __align__(16) unsigned char psm_raw[];
  // the CTA's box, tile and field (one field per CTA, field slowest)
  int bi = 0;
  while (bi + 1 < p.nbox && (int)blockIdx.x >= p.tiles_end[bi]) ++bi;
  const PBox& B = p.box[bi];
  const int local = (int)blockIdx.x - (bi ? p.tiles_end[bi - 1] : 0);
  if (p.R == 1)
    prolong_kind<T, NS, 1>(cb, p, B, local, psm_raw);
  else
    prolong_kind<T, NS, 2>(cb, p, B, local, psm_raw);
}

// App. C dense-output polynomials b_j(theta) of one coarse step and their
// theta-derivatives of order m (RK(4,4): the cubic interpolant with b_4's
// cubic coefficient +2/3, so that b_4(1) = 1/6; SSP-RK(3,3): the quadratic
// one).  Unused entries are zero.
static void dense_poly(int rk, double th, int m, double b[4]) {
  for (int j = 0; j < 4; ++j) b[j] = 0.0;
  if (rk == SF_RK4) {
    // coefficients of 1, th, th^2, th^3
    static const double P[4][4] = {{0.0, 1.0, -1.5, 2.0 / 3.0},
                                   {0.0, 0.0, 1.0, -2.0 / 3.0},
                                   {0.0, 0.0, 1.0, -2.0 / 3.0},
                                   {0.0, 0.0, -0.5, 2.0 / 3.0}};
    for (int j = 0; j < 4; ++j)
      for (int e = m; e < 4; ++e) {
        double fall = 1.0;  // e (e-1) ... (e-m+1)
        for (int q = 0; q < m; ++q) fall *= double(e - q);
        b[j] += P[j][e] * fall * std::pow(th, double(e - m));
      }
  } else {
    static const double P[3][3] = {{0.0, 1.0, -5.0 / 6.0}, {0.0, 0.0, 1.0 / 6.0}, {0.0, 0.0, 4.0 / 6.0}};
    for (int j = 0; j < 3; ++j)
      for (int e = m; e < 3; ++e) {
        double fall = 1.0;
        for (int q = 0; q < m; ++q) fall *= double(e - q);
        b[j] += P[j][e] * fall * std::pow(th, double(e - m));
      }
  }
}

// BOR (App. D) as a linear map.  Every quantity of the algorithm is a linear
// combination of the coarse increments k_1..k_s; a[j] is the weight of k_j in
// the requested fine value minus U^n.  The increments are in turn fixed by
// the stored stage states, k = T (S - U^n); the result is the coefficient c_m
// of (S_m - U^n).
static void bor_coefficients(int rk, int R, int r, int stage, double c[4]) {
  const int s = rk == SF_RK4 ? 4 : 3;
  const double th = double(r) / double(R), q = 1.0 / double(R);  // q = dt_F / dt
  double b0[4], v1[4], v2[4], v3[4];
  dense_poly(rk, th, 0, b0);  // U_{n+r/R} - U^n
  dense_poly(rk, th, 1, v1);  // dt U_t
  dense_poly(rk, th, 2, v2);  // dt^2 U_tt
  dense_poly(rk, th, 3, v3);  // dt^3 U_ttt
  double f[4][4] = {};        // fine increments f[i][j]: weight of coarse k_j
  for (int j = 0; j < 4; ++j) {
    if (rk == SF_RK4) {
      const double vf = j == 2 ? 4.0 : (j == 1 ? -4.0 : 0.0);  // dt^3 f_U U_tt = 4 (k_3 - k_2)
      f[0][j] = q * v1[j];
      f[1][j] = q * v1[j] + 0.5 * q * q * v2[j] + 0.125 * q * q * q * (v3[j] - vf);
      f[2][j] = q * v1[j] + 0.5 * q * q * v2[j] + 0.125 * q * q * q * (v3[j] + vf);
      f[3][j] = q * v1[j] + q * q * v2[j] + 0.5 * q * q * q * v3[j];
    } else {
      f[0][j] = q * v1[j];
      f[1][j] = q * v1[j] + q * q * v2[j];
      f[2][j] = q * v1[j] + 0.5 * q * q * v2[j];
    }
  }
  double a[4];
  for (int j = 0; j < 4; ++j) {
    double w;
    if (rk == SF_RK4) {
      switch (stage) {
        case 0: w = 0.0; break;
        case 1: w = 0.5 * f[0][j]; break;
        case 2: w = 0.5 * f[1][j]; break;
        case 3: w = f[2][j]; break;
        default: w = (f[0][j] + 2.0 * f[1][j] + 2.0 * f[2][j] + f[3][j]) / 6.0; break;
      }
    } else {
      switch (stage) {
        case 0: w = 0.0; break;
        case 1: w = f[0][j]; break;
        case 2: w = 0.25 * f[0][j] + 0.25 * f[1][j]; break;
        default: w = (f[0][j] + f[1][j] + 4.0 * f[2][j]) / 6.0; break;
      }
    }
    a[j] = b0[j] + w;
  }
  // k in terms of D_m = S_m - U^n (m = 1..s):
  //   RK4:  k_1 = 2 D_1, k_2 = 2 D_2, k_3 = D_3, k_4 = 6 D_4 - k_1 - 2 k_2 - 2 k_3
  //   SSP:  k_1 = D_1, k_2 = 4 D_2 - D_1, k_3 = (6 D_3 - k_1 - k_2) / 4
  double Tm[4][4] = {};
  if (rk == SF_RK4) {
    Tm[0][0] = 2.0;
    Tm[1][1] = 2.0;
    Tm[2][2] = 1.0;
    Tm[3][0] = -2.0; Tm[3][1] = -4.0; Tm[3][2] = -2.0; Tm[3][3] = 6.0;
  } else {
    Tm[0][0] = 1.0;
    Tm[1][0] = -1.0; Tm[1][1] = 4.0;
    Tm[2][1] = -1.0; Tm[2][2] = 1.5;
  }
  for (int m = 0; m < 4; ++m) {
    c[m] = 0.0;
    for (int j = 0; j < s; ++j) c[m] += a[j] * Tm[j][m];
  }
}

// Host checks of a box-copy list (everything sf_copy_boxes rejects).
sf_status check_box_copies(const sf_box_copy* boxes, int nbox, int precision) {
  if (nbox < 0 || (nbox > 0 && !boxes)) return set_error(SF_EINVAL, "boxes NULL or nbox < 0");
  if (precision < SF_FP64 || precision > SF_FP32_BULK_DW)
    return set_error(SF_EINVAL, "unknown precision %d", precision);
  const size_t es = precision == SF_FP64 ? 8 : 4;
  for (int q = 0; q < nbox; ++q) {
    const sf_box_copy& b = boxes[q];
    if (!b.src || !b.dst) return set_error(SF_EINVAL, "box %d: NULL array", q);
    if (reinterpret_cast<uintptr_t>(b.src) % es || reinterpret_cast<uintptr_t>(b.dst) % es)
      return set_error(SF_EINVAL, "box %d: misaligned array", q);
    if (b.nf < 1 || b.src_step < 1 || b.ext[0] < 0 || b.ext[1] < 0 || b.ext[2] < 0)
      return set_error(SF_EINVAL, "box %d: nf >= 1, src_step >= 1 and ext >= 0 required", q);
    if ((long long)b.ext[0] * b.ext[1] * b.ext[2] * b.nf >= (1LL << 31))
      return set_error(SF_EINVAL, "box %d: more than 2^31 values", q);
  }
  return SF_OK;
}

// Kernel launches sf_copy_boxes makes for a list: one per group of
// kBoxesPerLaunch boxes that holds a non-empty box.
int box_copy_launches(const sf_box_copy* boxes, int nbox) {
  int n = 0;
  for (int q0 = 0; q0 < nbox; q0 += kBoxesPerLaunch) {
    bool any = false;
    for (int q = q0; q < nbox && q < q0 + kBoxesPerLaunch; ++q)
      any = any || (long long)boxes[q].ext[0] * boxes[q].ext[1] * boxes[q].ext[2] * boxes[q].nf > 0;
    n += any ? 1 : 0;
  }
  return n;
}

}  // namespace sf

using namespace sf;

extern "C" sf_status sf_copy_boxes(const sf_box_copy* boxes, int32_t nbox, int32_t precision,
                                   void* stream) {
  sf_status e0 = check_box_copies(boxes, nbox, precision);
  if (e0) return e0;
  cudaStream_t st = (cudaStream_t)stream;
  for (int q0 = 0; q0 < nbox; q0 += kBoxesPerLaunch) {
    static_assert(sizeof(BoxBatch) < 32000, "kernel parameter limit");
    BoxBatch bb;
    bb.n = 0;
    int blocks = 0;
    for (int q = q0; q < nbox && q < q0 + kBoxesPerLaunch; ++q) {
      const long long v = (long long)boxes[q].ext[0] * boxes[q].ext[1] * boxes[q].ext[2] * boxes[q].nf;
      if (v == 0) continue;  // writes nothing
      long long nb = (v + 256 * kCopyIlp - 1) / (256 * kCopyIlp);
      if (nb > 1024) nb = 1024;  // the threads stride over larger boxes
      bb.b[bb.n] = boxes[q];
      blocks += (int)nb;
      bb.end[bb.n] = blocks;
      ++bb.n;
    }
    if (bb.n == 0) continue;
    if (precision == SF_FP64)
      copy_boxes_kernel<double><<<blocks, 256, 0, st>>>(bb);
    else
      copy_boxes_kernel<float><<<blocks, 256, 0, st>>>(bb);
    sf_status e = after_launch("copy_boxes_kernel");
    if (e) return e;
  }
  return SF_OK;
}

// Shared set-up of sf_prolong, sf_bor_prolong and sf_bor_prolong_boxes:
// validation of every box against the ghosted coarse layout, the Lagrange
// weight table, and one launch per kMaxPBoxes boxes.
template <int NS>
static sf_status prolong_launch(const sf_patch* coarse, const void* const* arrays, const double* c,
                                int32_t nf, int32_t ratio, const sf_prolong_box* boxes,
                                int32_t nbox, void* stream) {
  if (!coarse || !arrays || (nbox > 0 && !boxes) || nbox < 0)
    return set_error(SF_EINVAL, "NULL argument or nbox < 0");
  if (ratio < 1 || ratio > 8) return set_error(SF_EINVAL, "ratio %d not in [1, 8]", ratio);
  if (nf < 1) return set_error(SF_EINVAL, "nf < 1");
  sf_patch p = *coarse;
  normalise_strides(p, nf);
  const size_t es = p.precision == SF_FP64 ? 8 : 4;
  for (int m = 0; m <= NS; ++m) {
    if (!arrays[m]) return set_error(SF_EINVAL, "coarse array %d is NULL", m);
    if (reinterpret_cast<uintptr_t>(arrays[m]) % es) return set_error(SF_EINVAL, "coarse array %d misaligned", m);
  }
  sf_params dummy;
  memset(&dummy, 0, sizeof(dummy));
  p.u_stage = const_cast<void*>(arrays[0]);
  sf_status e = check_patch(&dummy, p, 0, 0);
  if (e) return e;
  ProlongArgs a;
  for (int r = 0; r < ratio; ++r) {
    const double t = double(r) / double(ratio);
    for (int j = 0; j < 6; ++j) {
      double l = 1.0;
      for (int m = 0; m < 6; ++m)
        if (m != j) l *= (t - double(m - 2)) / (double(j - 2) - double(m - 2));
      a.w[r][j] = l;
      a.wf[r][j] = (float)l;
    }
  }
  a.R = ratio;
  for (int d = 0; d < 3; ++d) a.n[d] = p.n[d];
  a.g = p.ghost;
  a.sy = p.sy;
  a.sz = p.sz;
  a.sf = p.sf;
  a.nf = nf;
  cudaStream_t st = (cudaStream_t)stream;
  // validate every box before any launch
  for (int q = 0; q < nbox; ++q) {
    const sf_prolong_box& bx = boxes[q];
    if (bx.ext[0] < 0 || bx.ext[1] < 0 || bx.ext[2] < 0)
      return set_error(SF_EINVAL, "box %d: negative extent", q);
    if (bx.ext[0] == 0 || bx.ext[1] == 0 || bx.ext[2] == 0) continue;  // writes nothing
    if (!bx.out) return set_error(SF_EINVAL, "box %d: out is NULL", q);
    if (reinterpret_cast<uintptr_t>(bx.out) % es) return set_error(SF_EINVAL, "box %d: out misaligned", q);
    for (int d = 0; d < 3; ++d) {
      if (bx.ext[d] < 0) return set_error(SF_EINVAL, "box %d: ext[%d] < 0", q, d);
      if (bx.ext[d] == 0) continue;
      // coarse nodes floor(F/R)-2 .. floor(F/R)+3 must lie in the ghosted coarse box
      const int lo = bx.origin[d], hi = bx.origin[d] + bx.ext[d] - 1;
      const int blo = lo >= 0 ? lo / ratio : -((-lo + ratio - 1) / ratio);
      const int bhi = hi >= 0 ? hi / ratio : -((-hi + ratio - 1) / ratio);
      if (blo - 2 < -p.ghost || bhi + 3 > p.n[d] + p.ghost - 1)
        return set_error(SF_EINVAL, "box %d: prolongation stencil leaves the coarse box along %d", q, d);
    }
    if (bx.out_sy < bx.ext[0] || bx.out_sz < bx.out_sy * bx.ext[1] ||
        bx.out_sf < bx.out_sz * bx.ext[2])
      return set_error(SF_EINVAL, "box %d: output strides too small for the box", q);
  }
  for (int q0 = 0; q0 < nbox; q0 += kMaxPBoxes) {
    long long total = 0;
    int smem_elems = 0;
    a.nbox = 0;
    for (int q = q0; q < nbox && q < q0 + kMaxPBoxes; ++q) {
      const sf_prolong_box& bx = boxes[q];
      if (bx.ext[0] == 0 || bx.ext[1] == 0 || bx.ext[2] == 0) continue;
      PBox& B = a.box[a.nbox];
      for (int d = 0; d < 3; ++d) {
        B.origin[d] = bx.origin[d];
        B.ext[d] = bx.ext[d];
      }
      B.kind = tile_for(bx.ext);
      const TileShape ts = kTileShapes[B.kind];
      B.p[0] = ts.px;
      B.p[1] = ts.py;
      B.p[2] = ts.pz;
      B.t[0] = (bx.ext[0] + ts.px - 1) / ts.px;
      B.t[1] = (bx.ext[1] + ts.py - 1) / ts.py;
      B.t[2] = (bx.ext[2] + ts.pz - 1) / ts.pz;
      smem_elems = std::max(smem_elems, prolong_elems(ts, ratio >= 2 ? 2 : 1));
      B.out = bx.out;
      B.osy = bx.out_sy;
      B.osz = bx.out_sz;
      B.osf = bx.out_sf;
      total += (long long)B.t[0] * B.t[1] * B.t[2] * nf;
      if (total >= (1LL << 31)) return set_error(SF_EINVAL, "boxes too large");
      a.tiles_end[a.nbox] = (int)total;
      ++a.nbox;
    }
    if (a.nbox == 0) continue;
    if (p.precision == SF_FP64) {
      Combo<double> cb;
      for (int m = 0; m < 5; ++m) cb.s[m] = m <= NS ? (const double*)arrays[m] : nullptr;
      for (int m = 0; m < 4; ++m) cb.c[m] = (c && m < NS) ? c[m] : 0.0;
      static std::once_flag once;
      std::call_once(once, [] {
        cudaFuncSetAttribute(prolong_kernel<double, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             prolong_smem_max<double>());
      });
      prolong_kernel<double, NS><<<(unsigned)total, kProlongThreads, prolong_smem_bytes<double>(smem_elems),
                                    st>>>(cb, a);
    } else {
      Combo<float> cb;
      for (int m = 0; m < 5; ++m) cb.s[m] = m <= NS ? (const float*)arrays[m] : nullptr;
      for (int m = 0; m < 4; ++m) cb.c[m] = (c && m < NS) ? c[m] : 0.0;
      static std::once_flag once;
      std::call_once(once, [] {
        cudaFuncSetAttribute(prolong_kernel<float, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             prolong_smem_max<float>());
      });
      prolong_kernel<float, NS><<<(unsigned)total, kProlongThreads, prolong_smem_bytes<float>(smem_elems),
                                   st>>>(cb, a);
    }
    e = after_launch("prolong_kernel");
    if (e) return e;
  }
  return SF_OK;
}

static sf_prolong_box one_box(const int32_t* origin, const int32_t* ext, void* out, int64_t sy,
                              int64_t sz, int64_t sf) {
  sf_prolong_box b;
  for (int d = 0; d < 3; ++d) {
    b.origin[d] = origin[d];
    b.ext[d] = ext[d];
  }
  b.out = out;
  b.out_sy = sy;
  b.out_sz = sz;
  b.out_sf = sf;
  return b;
}

extern "C" sf_status sf_prolong(const sf_patch* coarse, const void* coarse_array, int32_t nf,
                                int32_t ratio, const int32_t* origin, const int32_t* ext,
                                void* fine_out, int64_t out_sy, int64_t out_sz, int64_t out_sf,
                                void* stream) {
  if (!origin || !ext) return set_error(SF_EINVAL, "NULL argument");
  const void* arrays[1] = {coarse_array};
  const sf_prolong_box b = one_box(origin, ext, fine_out, out_sy, out_sz, out_sf);
  return prolong_launch<0>(coarse, arrays, nullptr, nf, ratio, &b, 1, stream);
}

static sf_status bor_args(int32_t rk, const void* const* states, int32_t ratio, int32_t r,
                          int32_t stage, double c[4]) {
  if (rk != SF_RK4 && rk != SF_SSPRK3) return set_error(SF_EINVAL, "unknown rk %d", rk);
  if (!states) return set_error(SF_EINVAL, "states NULL");
  if (ratio < 1 || ratio > 8) return set_error(SF_EINVAL, "ratio %d not in [1, 8]", ratio);
  if (r < 0 || r >= ratio) return set_error(SF_EINVAL, "fine step r = %d not in [0, %d)", r, ratio);
  const int s = rk == SF_RK4 ? 4 : 3;
  if (stage < 0 || stage > s) return set_error(SF_EINVAL, "stage %d not in [0, %d]", stage, s);
  bor_coefficients(rk, ratio, r, stage, c);
  return SF_OK;
}

extern "C" sf_status sf_bor_prolong_boxes(const sf_patch* coarse, int32_t rk,
                                          const void* const* states, int32_t nf, int32_t ratio,
                                          int32_t r, int32_t stage, const sf_prolong_box* boxes,
                                          int32_t nbox, void* stream) {
  double c[4];
  sf_status e = bor_args(rk, states, ratio, r, stage, c);
  if (e) return e;
  if (rk == SF_RK4) return prolong_launch<4>(coarse, states, c, nf, ratio, boxes, nbox, stream);
  return prolong_launch<3>(coarse, states, c, nf, ratio, boxes, nbox, stream);
}

extern "C" sf_status sf_bor_prolong(const sf_patch* coarse, int32_t rk, const void* const* states,
                                    int32_t nf, int32_t ratio, int32_t r, int32_t stage,
                                    const int32_t* origin, const int32_t* ext, void* fine_out,
                                    int64_t out_sy, int64_t out_sz, int64_t out_sf, void* stream) {
  if (!origin || !ext) return set_error(SF_EINVAL, "NULL argument");
  const sf_prolong_box b = one_box(origin, ext, fine_out, out_sy, out_sz, out_sf);
  return sf_bor_prolong_boxes(coarse, rk, states, nf, ratio, r, stage, &b, 1, stream);
}
