// Standalone CCZ4 stage kernel (one launch per patch); the per-point
// right-hand side lives in sf_z4.cuh.
#include "sf_internal.cuh"
#include "sf_z4.cuh"

namespace sf {

template <typename T, typename H>
__global__ void __launch_bounds__(128) z4_stage_kernel(PatchArgs<T> a, StageArgs s, Z4Coef<T> zc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= a.n[0] || j >= a.n[1]) return;
  const int g = a.g;
  const long long c = (long long)(k + g) * a.sz + (long long)(j + g) * a.sy + (i + g);
  T v[25], r[25];
  z4_point<T, H>(a, zc, a.us + c, v, r);
#pragma unroll
  for (int f = 0; f < 25; ++f) stage_write(a, s, f, c, i, j, k, v[f], r[f]);
}

template <typename T, typename H>
static sf_status launch(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                        void* rhs_out, cudaStream_t st) {
  PatchArgs<T> a = make_args<T>(prm, p, stage, 25, rhs_out);
  Z4Coef<T> zc;
  zc.kappa_z = T(prm.kappa_z);
  zc.kappa_c = T(prm.kappa_c);
  zc.eta = T(prm.eta);
  zc.g_shift = T(prm.g_shift);
  zc.slicing = prm.slicing;
  zc.shift_frozen = prm.shift_frozen;
  dim3 block(32, 4, 1);
  dim3 grid((p.n[0] + 31) / 32, (p.n[1] + 3) / 4, p.n[2]);
  z4_stage_kernel<T, H><<<grid, block, 0, st>>>(a, s, zc);
  return after_launch("z4_stage_kernel");
}

sf_status launch_z4(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                    void* rhs_out, cudaStream_t st) {
  if (p.precision == SF_FP64) return launch<double, double>(prm, p, s, stage, rhs_out, st);
  return launch<float, double>(prm, p, s, stage, rhs_out, st);
}

}  // namespace sf
