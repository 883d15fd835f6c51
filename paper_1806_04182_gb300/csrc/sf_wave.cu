// Standalone wave stage kernel (one launch per patch), forward or adjoint;
// the per-point right-hand side lives in sf_wave.cuh.
#include "sf_internal.cuh"
#include "sf_wave.cuh"

namespace sf {

template <typename T, bool ADJ>
__global__ void __launch_bounds__(128) wave_stage_kernel(PatchArgs<T> a, StageArgs s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= a.n[0] || j >= a.n[1]) return;
  const int g = a.g;
  const long long c = (long long)(k + g) * a.sz + (long long)(j + g) * a.sy + (i + g);
  T v[5], r[5];
  wave_point<T, ADJ>(a, a.us + c, v, r);
  const Images im = ghost_images(a, s, i, j, k);
#pragma unroll
  for (int f = 0; f < 5; ++f) write_field(a, s, im, f, c, i, j, k, v[f], r[f]);
}

template <typename T>
static sf_status launch(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                        void* rhs_out, bool adj, cudaStream_t st) {
  PatchArgs<T> a = make_args<T>(prm, p, stage, 5, rhs_out);
  dim3 block(32, 4, 1);
  dim3 grid((p.n[0] + 31) / 32, (p.n[1] + 3) / 4, p.n[2]);
  if (adj)
    wave_stage_kernel<T, true><<<grid, block, 0, st>>>(a, s);
  else
    wave_stage_kernel<T, false><<<grid, block, 0, st>>>(a, s);
  return after_launch("wave_stage_kernel");
}

sf_status launch_wave(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                      void* rhs_out, bool adjoint, cudaStream_t st) {
  if (p.precision == SF_FP64) return launch<double>(prm, p, s, stage, rhs_out, adjoint, st);
  return launch<float>(prm, p, s, stage, rhs_out, adjoint, st);
}

}  // namespace sf
