// Standalone CCZ4 stage kernel (one launch per patch); the per-point
// right-hand side lives in sf_z4.cuh.  Layouts with the strides of a 96^3
// patch with 3 ghosts (the benchmark configuration) get a kernel with
// compile-time strides; every other layout, and one-sided advection, uses
// runtime strides.
#include "sf_internal.cuh"
#include "sf_z4.cuh"

namespace sf {

// 128 threads and at least 3 CTAs per SM for the float kernels (<= 168
// registers): on the 96^3 benchmark patch this measured faster than 2 CTAs
// (255 registers) and than 4+ CTAs (128 registers or fewer, with spills).
template <typename T, typename H, int SY, int SZ, bool LOP>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 3 : 2)
    z4_stage_kernel(PatchArgs<T> a, StageArgs s, Z4Coef<T> zc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= a.n[0] || j >= a.n[1]) return;
  const int g = a.g;
  const long long sy = SY ? (long long)SY : a.sy;
  const long long sz = SZ ? (long long)SZ : a.sz;
  const long long c = (long long)(k + g) * sz + (long long)(j + g) * sy + (i + g);
  GlobalSrc<T, SY, SZ> src{a.us + c, a.sf, a.sy, a.sz};
  const Images im = ghost_images(a, s, i, j, k);
  z4_cell<T, H, LOP>(a, zc, src, [&](int f, T r, T centre) {
    write_field(a, s, im, f, c, i, j, k, centre, r);
  });
}

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

template <typename T, typename H>
static sf_status launch(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                        void* rhs_out, cudaStream_t st) {
  PatchArgs<T> a = make_args<T>(prm, p, stage, 25, rhs_out);
  const Z4Coef<T> zc = z4_coef<T>(prm);
  dim3 block(32, 4, 1);
  dim3 grid((p.n[0] + 31) / 32, (p.n[1] + 3) / 4, p.n[2]);
  if (prm.lopsided)
    z4_stage_kernel<T, H, 0, 0, true><<<grid, block, 0, st>>>(a, s, zc);
  else if (p.sy == 102 && p.sz == 102 * 102)
    z4_stage_kernel<T, H, 102, 102 * 102, false><<<grid, block, 0, st>>>(a, s, zc);
  else
    z4_stage_kernel<T, H, 0, 0, false><<<grid, block, 0, st>>>(a, s, zc);
  return after_launch("z4_stage_kernel");
}

sf_status launch_z4(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                    void* rhs_out, cudaStream_t st) {
  if (p.precision == SF_FP64) return launch<double, double>(prm, p, s, stage, rhs_out, st);
  if (p.precision == SF_FP32_BULK_DW) return launch<float, dw>(prm, p, s, stage, rhs_out, st);
  return launch<float, double>(prm, p, s, stage, rhs_out, st);
}

}  // namespace sf
