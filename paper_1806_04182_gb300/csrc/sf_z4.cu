// Standalone CCZ4 stage kernel (one launch per patch); the per-point
// right-hand side lives in sf_z4.cuh.  Float storage with centred advection
// and row / plane / field pitches on 16-byte boundaries goes to the
// TMA-staged kernels (sf_z4_tma.cu).  Layouts with the
// strides of a dense 96^3 patch with 3 ghosts get a kernel with compile-time
// strides; every other layout, and one-sided advection, uses runtime strides.
#include "sf_internal.cuh"
#include "sf_z4.cuh"

namespace sf {

// 128 threads and at least 3 CTAs per SM for the float kernels (<= 168
// registers): on the 96^3 benchmark patch this measured faster than 2 CTAs
// (255 registers) and than 4+ CTAs (128 registers or fewer, with spills).
//
// The right-hand sides of the 25 fields are parked in shared memory as
// z4_cell produces them, and the RK stage combination (which reads U^n, the
// accumulator and the Kahan term from memory) runs once at the end as a
// rolled loop over the fields.  Inlined after every field, the combination
// put 25 copies of its code and 25 dependent DRAM reads into the middle of the
// computation; the deferred form measured 7-10% faster on the 96^3 patch.
template <typename T, typename H, int SY, int SZ, bool LOP>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 3 : 2)
    z4_stage_kernel(PatchArgs<T> a, StageArgs s, Z4Coef<T> zc) {
  __shared__ T rbuf[25 * 128];
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
  const int tid = threadIdx.y * 32 + threadIdx.x;
  z4_cell<T, H, LOP>(a, zc, src, [&](int f, T r, T) { rbuf[f * 128 + tid] = r; });
  write_fields<T, 25>(a, s, im, c, i, j, k, rbuf + tid, 128);
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
  if (z4_pair_eligible(prm, p, rhs_out)) return launch_z4_pair(prm, p, s, stage, rhs_out, st);
  if (z4_pair_any_eligible(prm, p, s, rhs_out)) return launch_z4_pair_any(prm, p, s, stage, st);
  if (z4_tma_any_eligible(prm, p)) return launch_z4_tma(prm, p, s, stage, rhs_out, st);
  if (p.precision == SF_FP64) return launch<double, double>(prm, p, s, stage, rhs_out, st);
  if (p.precision == SF_FP32_BULK_DW) return launch<float, dw>(prm, p, s, stage, rhs_out, st);
  return launch<float, double>(prm, p, s, stage, rhs_out, st);
}

}  // namespace sf
