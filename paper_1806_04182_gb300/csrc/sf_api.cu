// C ABI entry points of libsf.so: argument validation, dispatch to the
// per-system stage kernels, periodic ghost fill, observer gather/scatter,
// device status word and error reporting.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "sf_internal.cuh"
#include "sf_mbar.cuh"

namespace sf {

__device__ unsigned int g_status_word;

static thread_local char t_err[512] = "";
static std::atomic<long long> g_launches{0};

sf_status set_error(sf_status code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_err, sizeof(t_err), fmt, ap);
  va_end(ap);
  return code;
}

sf_status after_launch(const char* what) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(SF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return SF_OK;
}

// Device address of the status word, cached per device.
unsigned int* status_ptr() {
  static unsigned int* cache[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!cache[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
    cache[dev] = static_cast<unsigned int*>(p);
  }
  return cache[dev];
}

void normalise_strides(sf_patch& p, int nf) {
  (void)nf;
  const long long g2 = 2LL * p.ghost;
  if (p.sy == 0) p.sy = p.n[0] + g2;
  if (p.sz == 0) p.sz = p.sy * (p.n[1] + g2);
  if (p.sf == 0) p.sf = p.sz * (p.n[2] + g2);
}

static bool aligned(const void* ptr, size_t a) { return (reinterpret_cast<uintptr_t>(ptr) % a) == 0; }

sf_status check_patch(const sf_params* prm, const sf_patch& p, int need_stage_arrays, int stage) {
  if (!prm) return set_error(SF_EINVAL, "params is NULL");
  if (p.system < 0 || p.system > 2) return set_error(SF_EINVAL, "unknown system %d", p.system);
  if (p.precision != SF_FP64 && p.precision != SF_FP32_BULK && p.precision != SF_FP32_BULK_DW)
    return set_error(SF_EINVAL, "unknown precision %d", p.precision);
  for (int d = 0; d < 3; ++d) {
    if (p.n[d] < 1) return set_error(SF_EINVAL, "n[%d] = %d < 1", d, p.n[d]);
    if (p.n[d] > 65535) return set_error(SF_EINVAL, "n[%d] = %d > 65535", d, p.n[d]);
    if (!(p.dx[d] > 0.0) || !(p.dx[d] < 1e300)) return set_error(SF_EINVAL, "dx[%d] must be > 0", d);
  }
  if (p.ghost < 3) return set_error(SF_EINVAL, "ghost = %d < 3 (4th-order FD + 6th-order KO need 3)", p.ghost);
  const long long g2 = 2LL * p.ghost;
  if (p.sy < p.n[0] + g2 || p.sz < p.sy * (p.n[1] + g2) || p.sf < p.sz * (p.n[2] + g2))
    return set_error(SF_EINVAL, "strides too small for the ghosted box");
  if (p.sf > (1LL << 40)) return set_error(SF_EINVAL, "field stride too large");
  const size_t es = p.precision == SF_FP64 ? 8 : 4;
  if (!p.u_stage || !aligned(p.u_stage, es)) return set_error(SF_EINVAL, "u_stage NULL or misaligned");
  if (need_stage_arrays) {
    if (prm->rk != SF_RK4 && prm->rk != SF_SSPRK3) return set_error(SF_EINVAL, "unknown rk %d", prm->rk);
    const int nst = prm->rk == SF_RK4 ? 4 : 3;
    if (stage < 0 || stage >= nst) return set_error(SF_EINVAL, "stage %d out of range [0,%d)", stage, nst);
    if (!p.u_n || !aligned(p.u_n, es)) return set_error(SF_EINVAL, "u_n NULL or misaligned");
    if (!p.u_next || !aligned(p.u_next, es)) return set_error(SF_EINVAL, "u_next NULL or misaligned");
    const bool last = stage == nst - 1;
    if (p.u_next == p.u_stage || p.u_next == p.acc || (p.u_next == p.u_n && !last))
      return set_error(SF_EINVAL,
                       "u_next must not alias u_stage or acc, nor u_n before the last stage");
    if (prm->rk == SF_RK4 && (!p.acc || !aligned(p.acc, es)))
      return set_error(SF_EINVAL, "RK4 needs an acc array");
    if (prm->rk == SF_RK4 && p.precision != SF_FP64 && (!p.kahan || !aligned(p.kahan, es)))
      return set_error(SF_EINVAL, "FP32_BULK RK4 needs a kahan array");
    if (!(p.dt == p.dt) || p.dt < 0) return set_error(SF_EINVAL, "dt must be >= 0");
    if (prm->ghosts == SF_GHOSTS_PERIODIC)
      for (int d = 0; d < 3; ++d)
        if (p.n[d] < p.ghost)
          return set_error(SF_EINVAL, "fused periodic ghosts need n[%d] >= ghost; use sf_fill_ghosts_periodic", d);
  }
  if (!(prm->sigma_ko >= 0)) return set_error(SF_EINVAL, "sigma_ko must be >= 0");
  if (prm->weno_variant < 0 || prm->weno_variant > 2)
    return set_error(SF_EINVAL, "weno_variant %d not in {0, 1, 2}", prm->weno_variant);
  if (prm->flux_split != 0 && prm->flux_split != 1)
    return set_error(SF_EINVAL, "flux_split %d not in {0, 1}", prm->flux_split);
  if (p.cfl_rate && p.system != SF_MHD)
    return set_error(SF_EINVAL, "cfl_rate is an SF_MHD output");
  if (p.cfl_rate && !aligned(p.cfl_rate, 8)) return set_error(SF_EINVAL, "cfl_rate misaligned");
  return SF_OK;
}

// ---------------------------------------------------------------- ghosts
// Periodic images into the ghost shell only, enumerated as six slabs (z
// slabs over the whole ghosted x-y plane, then y slabs over the interior z
// range, then x slabs over the interior y-z range): blockIdx.y is the field,
// the threads stride over the field's shell points with 32-bit indices (the
// host checks the count).  Every ghost reads an interior point, so the order
// of the writes does not matter.
template <typename T>
__global__ void __launch_bounds__(256) ghost_fill_kernel(T* u, int nx, int ny, int nz, int g,
                                                         long long sy, long long sz, long long sf) {
  const unsigned X = nx + 2 * g, Y = ny + 2 * g, G2 = 2 * g;
  const unsigned s1 = G2 * X * Y, s2 = G2 * X * nz, total = s1 + s2 + G2 * ny * nz;
  T* uf = u + blockIdx.y * sf;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int x, y, z;  // ghosted coordinates of the ghost point
    if (t < s1) {
      x = t % X;
      y = (t / X) % Y;
      const int q = t / (X * Y);
      z = q < g ? q : nz + q;
    } else if (t < s1 + s2) {
      const unsigned r = t - s1;
      x = r % X;
      const int q = (r / X) % G2;
      y = q < g ? q : ny + q;
      z = g + (int)(r / (X * G2));
    } else {
      const unsigned r = t - s1 - s2;
      const int q = r % G2;
      x = q < g ? q : nx + q;
      y = g + (int)((r / G2) % ny);
      z = g + (int)(r / (G2 * ny));
    }
    // interior source: the periodic image of (x, y, z) - g (more than one
    // wrap only when the patch is thinner than its ghost zone)
    int i = x - g, j = y - g, k = z - g;
    while (i < 0) i += nx;
    while (i >= nx) i -= nx;
    while (j < 0) j += ny;
    while (j >= ny) j -= ny;
    while (k < 0) k += nz;
    while (k >= nz) k -= nz;
    i += g;
    j += g;
    k += g;
    uf[(long long)z * sz + (long long)y * sy + x] = uf[(long long)k * sz + (long long)j * sy + i];
  }
}

// ---------------------------------------------------------------- observers
template <typename T>
__global__ void gather_kernel(const T* a, long long off, int nx, int ny, int g, long long sy,
                              long long sz, long long total, const int64_t* obs, int nobs, T* out) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nobs) return;
  long long lin = obs[o];
  if (lin < 0 || lin >= total) return;  // out-of-range observer: skipped
  int i = (int)(lin % nx);
  int j = (int)((lin / nx) % ny);
  int k = (int)(lin / ((long long)nx * ny));
  out[o] = a[off + (long long)(k + g) * sz + (long long)(j + g) * sy + (i + g)];
}

template <typename T>
__global__ void scatter_add_kernel(T* a, long long off, int nx, int ny, int g, long long sy,
                                   long long sz, long long total, const int64_t* obs, int nobs,
                                   const T* vals) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nobs) return;
  long long lin = obs[o];
  if (lin < 0 || lin >= total) return;  // out-of-range observer: skipped
  int i = (int)(lin % nx);
  int j = (int)((lin / nx) % ny);
  int k = (int)(lin / ((long long)nx * ny));
  a[off + (long long)(k + g) * sz + (long long)(j + g) * sy + (i + g)] += vals[o];
}

static StageArgs stage_args(const sf_params& prm, const sf_patch& p, int stage, int mode) {
  StageArgs s;
  s.mode = mode;
  s.rk = prm.rk;
  s.stage = stage;
  s.kahan = (p.precision != SF_FP64 && prm.rk == SF_RK4) ? 1 : 0;
  s.un_alias = p.u_n == p.u_stage ? 1 : 0;
  s.ghosts = prm.ghosts == SF_GHOSTS_PERIODIC ? 1 : 0;
  s.check_finite = prm.check_finite;
  s.status = status_ptr();
  return s;
}

static sf_status dispatch(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                          void* rhs_out, bool adjoint, cudaStream_t st) {
  if (!s.status) return set_error(SF_ECUDA, "no CUDA device / status word unavailable");
  switch (p.system) {
    case SF_WAVE: return launch_wave(prm, p, s, stage, rhs_out, adjoint, st);
    case SF_Z4: return launch_z4(prm, p, s, stage, rhs_out, st);
    case SF_MHD: return launch_mhd(prm, p, s, stage, rhs_out, st);
  }
  return set_error(SF_EINVAL, "unknown system");
}

}  // namespace sf

using namespace sf;

namespace sf {
namespace {

// Longest self-test wait accepted: about a second at GB300 clocks, the limit
// the stage kernels themselves use.
constexpr long long kMaxSelftestCycles = 2000000000LL;

// One warp waits on an mbarrier that nothing ever arrives on, through the
// same bounded wait the TMA-staged kernels use; the wait gives up after
// `limit` cycles and the kernel records ST_TIMEOUT.
__global__ void wait_selftest_kernel(long long limit, unsigned int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const bool ok = mbar_wait(&bar, 0, limit);
  if (!ok && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}

}  // namespace
}  // namespace sf

extern "C" {

int32_t sf_nfields(int32_t system) {
  switch (system) {
    case SF_WAVE: return 5;
    case SF_MHD: return 8;
    case SF_Z4: return 25;
  }
  return -1;
}

const char* sf_last_error(void) { return t_err; }

int64_t sf_launch_count(void) { return g_launches.load(); }

sf_status sf_radiative_substep(const sf_params* prm, const sf_patch* patch, const double* x0,
                               const double* u_inf, const double* speed, int32_t stage,
                               void* stream) {
  t_err[0] = 0;
  if (!prm || !patch || !x0 || !u_inf || !speed) return set_error(SF_EINVAL, "NULL argument");
  sf_patch p = *patch;
  const int nf = sf_nfields(p.system);
  normalise_strides(p, nf);
  sf_status e = check_patch(prm, p, 1, stage);
  if (e) return e;
  if (prm->ghosts != SF_GHOSTS_NONE)
    return set_error(SF_EINVAL, "radiative boundaries need ghosts = SF_GHOSTS_NONE");
  for (int d = 0; d < 3; ++d)
    if (!(x0[d] == x0[d]) || x0[d] > 1e300 || x0[d] < -1e300)
      return set_error(SF_EINVAL, "x0[%d] not finite", d);
  for (int f = 0; f < nf; ++f) {
    if (!(speed[f] >= 0.0) || speed[f] > 1e300) return set_error(SF_EINVAL, "speed[%d] must be >= 0", f);
    if (!(u_inf[f] == u_inf[f]) || u_inf[f] > 1e300 || u_inf[f] < -1e300)
      return set_error(SF_EINVAL, "u_inf[%d] not finite", f);
  }
  StageArgs s = stage_args(*prm, p, stage, 0);
  if (!s.status) return set_error(SF_ECUDA, "no CUDA device / status word unavailable");
  return launch_radiative(*prm, p, s, stage, x0, u_inf, speed, (cudaStream_t)stream);
}

sf_status sf_substep(const sf_params* prm, const sf_patch* patches, int32_t npatch, int32_t stage,
                     void* stream) {
  t_err[0] = 0;
  if (!patches || npatch < 0) return set_error(SF_EINVAL, "patches NULL or npatch < 0");
  if (!prm) return set_error(SF_EINVAL, "params is NULL");
  for (int q = 0; q < npatch; ++q) {
    sf_patch p = patches[q];
    normalise_strides(p, sf_nfields(p.system));
    sf_status e = check_patch(prm, p, 1, stage);
    if (e) return e;
    if (q > 0 && (p.system != patches[0].system || p.precision != patches[0].precision))
      return set_error(SF_EINVAL, "sf_substep needs one system and precision; use sf_batch");
  }
  for (int q = 0; q < npatch; ++q) {
    sf_patch p = patches[q];
    normalise_strides(p, sf_nfields(p.system));
    StageArgs s = stage_args(*prm, p, stage, 0);
    sf_status e = dispatch(*prm, p, s, stage, nullptr, false, (cudaStream_t)stream);
    if (e) return e;
  }
  return SF_OK;
}

sf_status sf_adjoint_substep(const sf_params* prm, const sf_patch* adj, int32_t npatch,
                             int32_t stage, void* stream) {
  t_err[0] = 0;
  if (!adj || npatch < 0) return set_error(SF_EINVAL, "patches NULL or npatch < 0");
  for (int q = 0; q < npatch; ++q) {
    sf_patch p = adj[q];
    normalise_strides(p, 5);
    sf_status e = check_patch(prm, p, 1, stage);
    if (e) return e;
    if (p.system != SF_WAVE) return set_error(SF_ENOTSUP, "adjoint substep exists for SF_WAVE only");
  }
  for (int q = 0; q < npatch; ++q) {
    sf_patch p = adj[q];
    normalise_strides(p, 5);
    StageArgs s = stage_args(*prm, p, stage, 0);
    if (!s.status) return set_error(SF_ECUDA, "no CUDA device");
    sf_status e = launch_wave(*prm, p, s, stage, nullptr, true, (cudaStream_t)stream);
    if (e) return e;
  }
  return SF_OK;
}

sf_status sf_rhs(const sf_params* prm, const sf_patch* patch, void* rhs_out, void* stream) {
  t_err[0] = 0;
  if (!patch || !rhs_out) return set_error(SF_EINVAL, "patch or rhs_out NULL");
  sf_patch p = *patch;
  normalise_strides(p, sf_nfields(p.system));
  sf_status e = check_patch(prm, p, 0, 0);
  if (e) return e;
  const size_t es = p.precision == SF_FP64 ? 8 : 4;
  if (!aligned(rhs_out, es)) return set_error(SF_EINVAL, "rhs_out misaligned");
  sf_params q = *prm;
  q.rk = SF_RK4;
  StageArgs s = stage_args(q, p, 0, 1);
  s.ghosts = 0;
  return dispatch(q, p, s, 0, rhs_out, false, (cudaStream_t)stream);
}

sf_status sf_fill_ghosts_periodic(const sf_patch* patch, void* array, int32_t nf, void* stream) {
  t_err[0] = 0;
  if (!patch || !array || nf < 1) return set_error(SF_EINVAL, "patch/array NULL or nf < 1");
  sf_patch p = *patch;
  normalise_strides(p, nf);
  sf_params dummy;
  memset(&dummy, 0, sizeof(dummy));
  p.u_stage = array;
  sf_status e = check_patch(&dummy, p, 0, 0);
  if (e) return e;
  const long long g = p.ghost, X = p.n[0] + 2 * g, Y = p.n[1] + 2 * g;
  const long long shell = 2 * g * (X * Y + X * p.n[2] + (long long)p.n[1] * p.n[2]);
  if (shell >= (1LL << 31)) return set_error(SF_EINVAL, "ghost shell of %lld points too large", shell);
  if (nf > 65535) return set_error(SF_EINVAL, "nf = %d > 65535", nf);
  long long gx = (shell + 255) / 256;
  if (gx > 1024) gx = 1024;
  const dim3 grid((unsigned)gx, (unsigned)nf);
  if (p.precision == SF_FP64)
    ghost_fill_kernel<double><<<grid, 256, 0, (cudaStream_t)stream>>>(
        (double*)array, p.n[0], p.n[1], p.n[2], p.ghost, p.sy, p.sz, p.sf);
  else
    ghost_fill_kernel<float><<<grid, 256, 0, (cudaStream_t)stream>>>(
        (float*)array, p.n[0], p.n[1], p.n[2], p.ghost, p.sy, p.sz, p.sf);
  return after_launch("ghost_fill_kernel");
}

static sf_status obs_check(const sf_patch* patch, const void* array, int32_t field,
                           const int64_t* obs, int32_t nobs, const void* other, sf_patch& p) {
  if (!patch || !array || !obs || !other || nobs < 0) return set_error(SF_EINVAL, "NULL argument");
  p = *patch;
  normalise_strides(p, sf_nfields(p.system));
  if (field < 0 || field >= sf_nfields(p.system)) return set_error(SF_EINVAL, "field out of range");
  sf_params dummy;
  memset(&dummy, 0, sizeof(dummy));
  p.u_stage = const_cast<void*>(array);
  return check_patch(&dummy, p, 0, 0);
}

sf_status sf_gather(const sf_patch* patch, const void* array, int32_t field, const int64_t* obs,
                    int32_t nobs, void* out, void* stream) {
  t_err[0] = 0;
  sf_patch p;
  sf_status e = obs_check(patch, array, field, obs, nobs, out, p);
  if (e) return e;
  if (nobs == 0) return SF_OK;
  int blocks = (nobs + 127) / 128;
  if (p.precision == SF_FP64)
    gather_kernel<double><<<blocks, 128, 0, (cudaStream_t)stream>>>(
        (const double*)array, field * p.sf, p.n[0], p.n[1], p.ghost, p.sy, p.sz,
        (long long)p.n[0] * p.n[1] * p.n[2], obs, nobs, (double*)out);
  else
    gather_kernel<float><<<blocks, 128, 0, (cudaStream_t)stream>>>(
        (const float*)array, field * p.sf, p.n[0], p.n[1], p.ghost, p.sy, p.sz,
        (long long)p.n[0] * p.n[1] * p.n[2], obs, nobs, (float*)out);
  return after_launch("gather_kernel");
}

sf_status sf_scatter_add(const sf_patch* patch, void* array, int32_t field, const int64_t* obs,
                         int32_t nobs, const void* vals, void* stream) {
  t_err[0] = 0;
  sf_patch p;
  sf_status e = obs_check(patch, array, field, obs, nobs, vals, p);
  if (e) return e;
  if (nobs == 0) return SF_OK;
  int blocks = (nobs + 127) / 128;
  if (p.precision == SF_FP64)
    scatter_add_kernel<double><<<blocks, 128, 0, (cudaStream_t)stream>>>(
        (double*)array, field * p.sf, p.n[0], p.n[1], p.ghost, p.sy, p.sz,
        (long long)p.n[0] * p.n[1] * p.n[2], obs, nobs, (const double*)vals);
  else
    scatter_add_kernel<float><<<blocks, 128, 0, (cudaStream_t)stream>>>(
        (float*)array, field * p.sf, p.n[0], p.n[1], p.ghost, p.sy, p.sz,
        (long long)p.n[0] * p.n[1] * p.n[2], obs, nobs, (const float*)vals);
  return after_launch("scatter_add_kernel");
}

sf_status sf_selftest_wait_timeout(int64_t limit_cycles, void* stream) {
  t_err[0] = 0;
  if (limit_cycles < 1 || limit_cycles > kMaxSelftestCycles)
    return set_error(SF_EINVAL, "limit_cycles must be in [1, %lld]", kMaxSelftestCycles);
  unsigned int* st = status_ptr();
  if (!st) return set_error(SF_ECUDA, "no CUDA device / status word unavailable");
  wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>((long long)limit_cycles, st);
  return after_launch("wait_selftest_kernel");
}

sf_status sf_get_device_status(void* stream) {
  t_err[0] = 0;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return set_error(SF_ECUDA, "sync: %s", cudaGetErrorString(e));
  unsigned int* p = status_ptr();
  if (!p) return set_error(SF_ECUDA, "no status word");
  unsigned int v = 0;
  e = cudaMemcpy(&v, p, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_error(SF_ECUDA, "status read: %s", cudaGetErrorString(e));
  unsigned int zero = 0;
  e = cudaMemcpy(p, &zero, sizeof(zero), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return set_error(SF_ECUDA, "status reset: %s", cudaGetErrorString(e));
  if (v & ST_TIMEOUT) return set_error(SF_ETIMEOUT, "a device wait timed out");
  if (v & ST_NONFINITE) return set_error(SF_ENONFINITE, "non-finite value written");
  return SF_OK;
}

}  // extern "C"
