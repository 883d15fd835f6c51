// FP64 diagnostics of a patch: wave energy, CCZ4 constraint monitors
// (Theta, Z^i = chi/2 (Gammahat^i - Gamma~^i), ln det gt, tr A~; Sec. V) and a
// count of non-finite values.  Block partial sums are combined with double
// atomics into a 5-double device array that the caller owns.
#include "sf_internal.cuh"

namespace sf {

template <typename T>
__global__ void __launch_bounds__(256) diag_kernel(const T* __restrict__ u0, int system, int nx,
                                                   int ny, int nz, int g, long long sy,
                                                   long long sz, long long F, double hx, double hy,
                                                   double hz, double* out) {
  const long long total = (long long)nx * ny * nz;
  const int nf = system == SF_WAVE ? 5 : (system == SF_Z4 ? 25 : 8);
  double acc[5] = {0, 0, 0, 0, 0};
  const double ih[3] = {1.0 / (12.0 * hx), 1.0 / (12.0 * hy), 1.0 / (12.0 * hz)};
  const long long st[3] = {1, sy, sz};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % nx);
    const int j = (int)((t / nx) % ny);
    const int k = (int)(t / ((long long)nx * ny));
    const T* p = u0 + (long long)(k + g) * sz + (long long)(j + g) * sy + (i + g);
    for (int f = 0; f < nf; ++f)
      if (!isfinite(double(p[f * F]))) acc[4] += 1.0;
    if (system == SF_WAVE) {
      double e = 0.0;
      for (int f = 1; f < 5; ++f) {
        const double v = double(p[f * F]);
        e += 0.5 * v * v;
      }
      acc[0] += e * hx * hy * hz;
    } else if (system == SF_Z4) {
      // float arrays hold chi, gt_ii and alpha minus 1 (flat-space offset)
      const double off = sizeof(T) == 4 ? 1.0 : 0.0;
      double gt[6], At[6];
      for (int q = 0; q < 6; ++q) {
        gt[q] = double(p[(1 + q) * F]) + ((q == 0 || q == 3 || q == 5) ? off : 0.0);
        At[q] = double(p[(8 + q) * F]);
      }
      const double c00 = gt[3] * gt[5] - gt[4] * gt[4], c01 = gt[2] * gt[4] - gt[1] * gt[5],
                   c02 = gt[1] * gt[4] - gt[2] * gt[3], c11 = gt[0] * gt[5] - gt[2] * gt[2],
                   c12 = gt[1] * gt[2] - gt[0] * gt[4], c22 = gt[0] * gt[3] - gt[1] * gt[1];
      const double det = gt[0] * c00 + gt[1] * c01 + gt[2] * c02;
      const double ig[6] = {c00 / det, c01 / det, c02 / det, c11 / det, c12 / det, c22 / det};
      const int Sx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
      double dg[6][3];
      for (int q = 0; q < 6; ++q)
        for (int d = 0; d < 3; ++d) {
          const T* c = p + (1 + q) * F;
          const long long s = st[d];
          dg[q][d] = (double(c[-2 * s]) - double(c[2 * s]) + 8.0 * (double(c[s]) - double(c[-s]))) * ih[d];
        }
      const double chi = double(p[0]) + off;
      double Z2 = 0.0;
      for (int a = 0; a < 3; ++a) {
        double Gt = 0.0;
        for (int b = 0; b < 3; ++b)
          for (int c = 0; c < 3; ++c)
            for (int l = 0; l < 3; ++l)
              Gt += ig[Sx[b][c]] * ig[Sx[a][l]] * 0.5 *
                    (dg[Sx[l][c]][b] + dg[Sx[l][b]][c] - dg[Sx[b][c]][l]);
        const double Za = 0.5 * chi * (double(p[(14 + a) * F]) - Gt);
        Z2 += Za * Za;
      }
      const double w[6] = {1, 2, 2, 1, 2, 1};
      double trA = 0.0;
      for (int q = 0; q < 6; ++q) trA += w[q] * ig[q] * At[q];
      const double Th = double(p[17 * F]);
      const double ld = log(det);
      acc[0] += Th * Th;
      acc[1] += Z2;
      acc[2] += ld * ld;
      acc[3] += trA * trA;
    }
  }
  __shared__ double sm[5][256];
  for (int q = 0; q < 5; ++q) sm[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 5; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 5; ++q) atomicAdd(out + q, sm[q][0]);
}

}  // namespace sf

using namespace sf;

extern "C" sf_status sf_diagnostics(const sf_params* prm, const sf_patch* patch, const void* array,
                                    double* d_out, void* stream) {
  if (!patch || !array || !d_out) return set_error(SF_EINVAL, "NULL argument");
  sf_patch p = *patch;
  normalise_strides(p, sf_nfields(p.system));
  p.u_stage = const_cast<void*>(array);
  sf_status e = check_patch(prm, p, 0, 0);
  if (e) return e;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_out, 0, 5 * sizeof(double), st) != cudaSuccess)
    return set_error(SF_ECUDA, "memset of d_out failed");
  const long long total = (long long)p.n[0] * p.n[1] * p.n[2];
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 4) blocks = 152 * 4;
  if (p.precision == SF_FP64)
    diag_kernel<double><<<blocks, 256, 0, st>>>((const double*)array, p.system, p.n[0], p.n[1],
                                                p.n[2], p.ghost, p.sy, p.sz, p.sf, p.dx[0],
                                                p.dx[1], p.dx[2], d_out);
  else
    diag_kernel<float><<<blocks, 256, 0, st>>>((const float*)array, p.system, p.n[0], p.n[1],
                                               p.n[2], p.ghost, p.sy, p.sz, p.sf, p.dx[0],
                                               p.dx[1], p.dx[2], d_out);
  return after_launch("diag_kernel");
}
