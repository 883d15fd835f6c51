// Radiative (outgoing-wave) boundary condition of Sec. V on the ghost shell of
// a non-periodic patch:  dU/dt = -v x^i/r d_i U - v (U - U_inf)/r,  x the
// physical position of the point, r = |x|.  One RK stage at every ghost
// point, the interior being advanced by sf_substep (ghost writes off) on the
// same arrays.  d_i is the centred 4th-order D_i where the ghosted array holds
// two points on both sides of the point and a 4th-order one-sided stencil
// leaning into the array elsewhere.
#include "sf_internal.cuh"

namespace sf {
namespace {

constexpr int kMaxFields = 32;

struct RadArgs {
  double x0[3];              // position of interior point (0,0,0)
  double dx[3];
  int nf;
  double uinf[kMaxFields];   // value at infinity, in the storage convention
  double v[kMaxFields];      // speed
};

// d/dx along one axis at a point with ghosted index ig of N along that axis;
// p points at the value, s is the element stride along the axis
template <typename T>
__device__ __forceinline__ T rad_d(const T* __restrict__ p, long long s, int ig, int N, T i12h) {
  if (ig >= 2 && ig <= N - 3) return ((p[-2 * s] - p[2 * s]) + T(8) * (p[s] - p[-s])) * i12h;
  if (ig == 1)
    return (T(-3) * p[-s] - T(10) * p[0] + T(18) * p[s] - T(6) * p[2 * s] + p[3 * s]) * i12h;
  if (ig == 0)
    return (T(-25) * p[0] + T(48) * p[s] - T(36) * p[2 * s] + T(16) * p[3 * s] - T(3) * p[4 * s]) *
           i12h;
  if (ig == N - 2)
    return (T(3) * p[s] + T(10) * p[0] - T(18) * p[-s] + T(6) * p[-2 * s] - p[-3 * s]) * i12h;
  return (T(25) * p[0] - T(48) * p[-s] + T(36) * p[-2 * s] - T(16) * p[-3 * s] + T(3) * p[-4 * s]) *
         i12h;
}

// One thread per ghost point and group of five fields (gridDim.y groups);
// ghost points are enumerated as the two z slabs (full x-y planes), the two y
// slabs (interior z) and the two x slabs (interior y, z).  32-bit index
// arithmetic (the host checks the count); the five fields' reads are issued
// together.
constexpr int kFieldGroup = 5;

template <typename T>
__global__ void __launch_bounds__(256) radiative_kernel(PatchArgs<T> a, StageArgs s, RadArgs ra) {
  const unsigned g = (unsigned)a.g;
  const unsigned N0 = a.n[0] + 2 * g, N1 = a.n[1] + 2 * g;
  const unsigned zslab = 2 * g * N1 * N0;
  const unsigned yslab = (unsigned)a.n[2] * 2 * g * N0;
  const unsigned xslab = (unsigned)a.n[2] * a.n[1] * 2 * g;
  const unsigned total = zslab + yslab + xslab;
  const int f0 = blockIdx.y * kFieldGroup;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int i, j, k;  // interior coordinates; ghost points lie outside [0, n)
    if (t < zslab) {
      unsigned q = t;
      i = (int)(q % N0) - (int)g;
      q /= N0;
      j = (int)(q % N1) - (int)g;
      const int kk = (int)(q / N1);
      k = kk < (int)g ? kk - (int)g : a.n[2] + (kk - (int)g);
    } else if (t < zslab + yslab) {
      unsigned q = t - zslab;
      i = (int)(q % N0) - (int)g;
      q /= N0;
      const int jj = (int)(q % (2 * g));
      k = (int)(q / (2 * g));
      j = jj < (int)g ? jj - (int)g : a.n[1] + (jj - (int)g);
    } else {
      unsigned q = t - zslab - yslab;
      const int ii = (int)(q % (2 * g));
      q /= 2 * g;
      j = (int)(q % (unsigned)a.n[1]);
      k = (int)(q / (unsigned)a.n[1]);
      i = ii < (int)g ? ii - (int)g : a.n[0] + (ii - (int)g);
    }
    const long long c = (long long)(k + (int)g) * a.sz + (long long)(j + (int)g) * a.sy + (i + (int)g);
    // the point's position, then its radius and direction cosines in the
    // arrays' precision (float arrays: float sqrt and divide, since the FP64
    // pipe runs at 1/58 of the FP32 rate and every field group repeats this)
    const double x = ra.x0[0] + i * ra.dx[0], y = ra.x0[1] + j * ra.dx[1], z = ra.x0[2] + k * ra.dx[2];
    const T xt = T(x), yt = T(y), zt = T(z);
    const T r = sqrt(xt * xt + yt * yt + zt * zt);
    const T ir = r > T(0) ? T(1) / r : T(0);
    const T ex = xt * ir, ey = yt * ir, ez = zt * ir;
    const int N[3] = {a.n[0] + 2 * (int)g, a.n[1] + 2 * (int)g, a.n[2] + 2 * (int)g};
    const bool rk4 = s.rk == SF_RK4;
#pragma unroll
    for (int q = 0; q < kFieldGroup; ++q) {
      const int f = f0 + q;
      if (f >= ra.nf) break;
      const long long o = f * a.sf + c;
      const T* p = a.us + o;
      const T U = p[0];
      const T du = ex * rad_d(p, 1, i + (int)g, N[0], a.i12h[0]) +
                   ey * rad_d(p, a.sy, j + (int)g, N[1], a.i12h[1]) +
                   ez * rad_d(p, a.sz, k + (int)g, N[2], a.i12h[2]);
      const T rhs = -T(ra.v[f]) * (du + (U - T(ra.uinf[f])) * ir);
      const T un = s.un_alias ? U : a.un[o];
      const T acc = (rk4 && s.stage > 0) ? a.acc[o] : T(0);
      const T kh = (rk4 && s.stage == 3 && s.kahan) ? a.kh[o] : T(0);
      const T out = stage_combine(a, s, o, U, un, acc, kh, rhs);
      a.nx[o] = out;
      if (s.check_finite && !finite_(out)) atomicOr(s.status, ST_NONFINITE);
    }
  }
}

template <typename T>
sf_status launch(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                 const RadArgs& ra, cudaStream_t st) {
  PatchArgs<T> a = make_args<T>(prm, p, stage, ra.nf, nullptr);
  const int g = p.ghost;
  const long long N0 = p.n[0] + 2 * g, N1 = p.n[1] + 2 * g, N2 = p.n[2] + 2 * g;
  const long long ghosts = N0 * N1 * N2 - (long long)p.n[0] * p.n[1] * p.n[2];
  if (ghosts >= (1LL << 31)) return set_error(SF_EINVAL, "ghost shell too large");
  long long blocks = (ghosts + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  const dim3 grid((unsigned)blocks, (unsigned)((ra.nf + kFieldGroup - 1) / kFieldGroup));
  radiative_kernel<T><<<grid, 256, 0, st>>>(a, s, ra);
  return after_launch("radiative_kernel");
}

}  // namespace

sf_status launch_radiative(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                           const double* x0, const double* u_inf, const double* speed,
                           cudaStream_t st) {
  const int nf = sf_nfields(p.system);
  if (nf < 1 || nf > kMaxFields) return set_error(SF_EINVAL, "unsupported field count");
  RadArgs ra;
  for (int d = 0; d < 3; ++d) {
    ra.x0[d] = x0[d];
    ra.dx[d] = p.dx[d];
  }
  ra.nf = nf;
  // float CCZ4 arrays store chi, gt_xx, gt_yy, gt_zz and alpha minus 1
  const bool offset = p.system == SF_Z4 && p.precision != SF_FP64;
  for (int f = 0; f < nf; ++f) {
    const bool off = offset && (f == 0 || f == 1 || f == 4 || f == 6 || f == 18);
    ra.uinf[f] = u_inf[f] - (off ? 1.0 : 0.0);
    ra.v[f] = speed[f];
  }
  if (p.precision == SF_FP64) return launch<double>(prm, p, s, stage, ra, st);
  return launch<float>(prm, p, s, stage, ra, st);
}

}  // namespace sf
