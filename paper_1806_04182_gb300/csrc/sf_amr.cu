// Inter-patch data movement of the AMR level loop (Sec. III, Sec. III.A):
//   sf_copy_boxes  - same-level ghost synchronisation (box copies between
//                    patch arrays) and, with a source step R, restriction by
//                    injection (coarse point i <- fine point R i);
//   sf_prolong     - 6-point (5th-order) Lagrange prolongation from a coarse
//                    patch onto fine points, as a tensor product of 1D
//                    interpolations whose weights l_j(t) are tabulated on the
//                    host for the R fractional positions t = r/R.
#include <cstring>

#include "sf_internal.cuh"

namespace sf {

constexpr int kBoxesPerLaunch = 16;

struct BoxBatch {
  sf_box_copy b[kBoxesPerLaunch];
  int n;
};

template <typename T>
__global__ void __launch_bounds__(256) copy_boxes_kernel(BoxBatch bb) {
  const sf_box_copy& b = bb.b[blockIdx.y];
  const long long vol = (long long)b.ext[0] * b.ext[1] * b.ext[2];
  const long long total = vol * b.nf;
  const T* src = static_cast<const T*>(b.src);
  T* dst = static_cast<T*>(b.dst);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long r = t;
    const int x = (int)(r % b.ext[0]); r /= b.ext[0];
    const int y = (int)(r % b.ext[1]); r /= b.ext[1];
    const int z = (int)(r % b.ext[2]); r /= b.ext[2];
    const int f = (int)r;
    const long long s = b.src_off + f * b.src_sf + (long long)z * b.src_step * b.src_sz +
                        (long long)y * b.src_step * b.src_sy + (long long)x * b.src_step;
    const long long d = b.dst_off + f * b.dst_sf + (long long)z * b.dst_sz + (long long)y * b.dst_sy + x;
    dst[d] = src[s];
  }
}

struct ProlongArgs {
  double w[8][6];      // Lagrange weights l_j(r/R), r = 0..R-1, nodes -2..3
  int R;
  int n[3], g;
  long long sy, sz, sf;          // coarse strides
  int origin[3], ext[3];
  long long osy, osz, osf;       // output strides
  int nf;
};

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

template <typename T>
__global__ void __launch_bounds__(128) prolong_kernel(const T* __restrict__ cu, T* out, ProlongArgs p) {
  const long long vol = (long long)p.ext[0] * p.ext[1] * p.ext[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < vol;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % p.ext[0]);
    const int j = (int)((t / p.ext[0]) % p.ext[1]);
    const int k = (int)(t / ((long long)p.ext[0] * p.ext[1]));
    const int F[3] = {p.origin[0] + i, p.origin[1] + j, p.origin[2] + k};
    int base[3], r[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      base[d] = floordiv(F[d], p.R);
      r[d] = F[d] - base[d] * p.R;
    }
    // coarse node (base-2, base-2, base-2) in the ghosted array
    const long long c0 = (long long)(base[2] - 2 + p.g) * p.sz + (long long)(base[1] - 2 + p.g) * p.sy +
                         (base[0] - 2 + p.g);
    for (int f = 0; f < p.nf; ++f) {
      const T* q = cu + f * p.sf + c0;
      double acc = 0.0;
      for (int c = 0; c < 6; ++c) {
        double ay = 0.0;
        for (int b = 0; b < 6; ++b) {
          const T* row = q + c * p.sz + b * p.sy;
          double ax = 0.0;
#pragma unroll
          for (int a = 0; a < 6; ++a) ax += p.w[r[0]][a] * double(__ldg(row + a));
          ay += p.w[r[1]][b] * ax;
        }
        acc += p.w[r[2]][c] * ay;
      }
      out[f * p.osf + (long long)k * p.osz + (long long)j * p.osy + i] = T(acc);
    }
  }
}

}  // namespace sf

using namespace sf;

extern "C" sf_status sf_copy_boxes(const sf_box_copy* boxes, int32_t nbox, int32_t precision,
                                   void* stream) {
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
  }
  cudaStream_t st = (cudaStream_t)stream;
  for (int q0 = 0; q0 < nbox; q0 += kBoxesPerLaunch) {
    BoxBatch bb;
    bb.n = nbox - q0 < kBoxesPerLaunch ? nbox - q0 : kBoxesPerLaunch;
    long long maxv = 1;
    for (int q = 0; q < bb.n; ++q) {
      bb.b[q] = boxes[q0 + q];
      const long long v = (long long)bb.b[q].ext[0] * bb.b[q].ext[1] * bb.b[q].ext[2] * bb.b[q].nf;
      maxv = v > maxv ? v : maxv;
    }
    int gx = (int)((maxv + 255) / 256);
    if (gx > 1024) gx = 1024;
    if (precision == SF_FP64)
      copy_boxes_kernel<double><<<dim3(gx, bb.n), 256, 0, st>>>(bb);
    else
      copy_boxes_kernel<float><<<dim3(gx, bb.n), 256, 0, st>>>(bb);
    sf_status e = after_launch("copy_boxes_kernel");
    if (e) return e;
  }
  return SF_OK;
}

extern "C" sf_status sf_prolong(const sf_patch* coarse, const void* coarse_array, int32_t nf,
                                int32_t ratio, const int32_t* origin, const int32_t* ext,
                                void* fine_out, int64_t out_sy, int64_t out_sz, int64_t out_sf,
                                void* stream) {
  if (!coarse || !coarse_array || !origin || !ext || !fine_out)
    return set_error(SF_EINVAL, "NULL argument");
  if (ratio < 1 || ratio > 8) return set_error(SF_EINVAL, "ratio %d not in [1, 8]", ratio);
  if (nf < 1) return set_error(SF_EINVAL, "nf < 1");
  sf_patch p = *coarse;
  normalise_strides(p, nf);
  sf_params dummy;
  memset(&dummy, 0, sizeof(dummy));
  p.u_stage = const_cast<void*>(coarse_array);
  sf_status e = check_patch(&dummy, p, 0, 0);
  if (e) return e;
  for (int d = 0; d < 3; ++d) {
    if (ext[d] < 0) return set_error(SF_EINVAL, "ext[%d] < 0", d);
    if (ext[d] == 0) return SF_OK;
    // coarse nodes floor(F/R)-2 .. floor(F/R)+3 must lie in the ghosted coarse box
    const int lo = origin[d], hi = origin[d] + ext[d] - 1;
    const int blo = lo >= 0 ? lo / ratio : -((-lo + ratio - 1) / ratio);
    const int bhi = hi >= 0 ? hi / ratio : -((-hi + ratio - 1) / ratio);
    if (blo - 2 < -p.ghost || bhi + 3 > p.n[d] + p.ghost - 1)
      return set_error(SF_EINVAL, "prolongation stencil leaves the coarse box along %d", d);
  }
  if (out_sy < ext[0] || out_sz < out_sy * ext[1] || out_sf < out_sz * ext[2])
    return set_error(SF_EINVAL, "output strides too small for the box");
  ProlongArgs a;
  for (int r = 0; r < ratio; ++r) {
    const double t = double(r) / double(ratio);
    for (int j = 0; j < 6; ++j) {
      double l = 1.0;
      for (int m = 0; m < 6; ++m)
        if (m != j) l *= (t - double(m - 2)) / (double(j - 2) - double(m - 2));
      a.w[r][j] = l;
    }
  }
  a.R = ratio;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = p.n[d];
    a.origin[d] = origin[d];
    a.ext[d] = ext[d];
  }
  a.g = p.ghost;
  a.sy = p.sy;
  a.sz = p.sz;
  a.sf = p.sf;
  a.osy = out_sy;
  a.osz = out_sz;
  a.osf = out_sf;
  a.nf = nf;
  const long long vol = (long long)ext[0] * ext[1] * ext[2];
  int blocks = (int)((vol + 127) / 128);
  if (blocks > 152 * 16) blocks = 152 * 16;
  cudaStream_t st = (cudaStream_t)stream;
  if (p.precision == SF_FP64)
    prolong_kernel<double><<<blocks, 128, 0, st>>>((const double*)coarse_array, (double*)fine_out, a);
  else
    prolong_kernel<float><<<blocks, 128, 0, st>>>((const float*)coarse_array, (float*)fine_out, a);
  return after_launch("prolong_kernel");
}
