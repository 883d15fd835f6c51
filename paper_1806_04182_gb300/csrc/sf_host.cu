// RK steps of patch states held in host memory: each step copies its input
// state to the device, runs every stage of the RK method there (Sec. II.C,
// the fused substep of sf_substep) and copies the new state back.  With two
// or more device slots the uploads of the next steps and the downloads of the
// previous ones run on copy streams of their own while a step computes (a
// slot is uploaded again once the download of its previous step is done, so
// with three slots an upload no longer waits on the download just before it);
// a step whose input is an earlier step's output (an evolution kept in host
// memory) waits for that download first.
#include <algorithm>
#include <cstring>

#include "sf_internal.cuh"

namespace sf {
namespace {

// Events of the pipeline, per host thread and device; created once and kept
// (a step's events are re-recorded two steps later, after every wait on
// them has been enqueued).
constexpr int kMaxSlots = 4;
// Copies go in kChunks pieces of the image, each download piece with an
// event of its own: the upload of a piece that an earlier step's download
// writes waits for that piece only, so in an evolution kept in host memory
// the next step's upload runs beside the rest of this step's download.
constexpr int kChunks = 8;
struct HostEvents {
  int dev = -1;
  cudaEvent_t up[kMaxSlots], comp[kMaxSlots], down[kMaxSlots][kChunks], entry;
};
thread_local HostEvents t_ev;

sf_status host_events(HostEvents** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return set_error(SF_ECUDA, "no CUDA device");
  HostEvents& e = t_ev;
  if (e.dev != dev) {
    cudaEvent_t* all[(2 + kChunks) * kMaxSlots + 1];
    int na = 0;
    for (int q = 0; q < kMaxSlots; ++q) {
      all[na++] = &e.up[q];
      all[na++] = &e.comp[q];
      for (int c = 0; c < kChunks; ++c) all[na++] = &e.down[q][c];
    }
    all[na++] = &e.entry;
    if (e.dev >= 0)
      for (cudaEvent_t* q : all) cudaEventDestroy(*q);
    e.dev = -1;
    for (cudaEvent_t* q : all)
      if (cudaEventCreateWithFlags(q, cudaEventDisableTiming) != cudaSuccess)
        return set_error(SF_ECUDA, "event creation failed");
    e.dev = dev;
  }
  *out = &e;
  return SF_OK;
}

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

struct Layout {
  int n0, n1, n2, g, nf;
  long long sy, sz, sf;
};

// Interior host images (SF_HOST_INTERIOR): the dense interior (field, z, y,
// x) copied into the patch layout, every ghost point taking the interior
// point congruent to it modulo n (the periodic shell).  Each warp walks whole
// rows (ghosted rows of every ghosted plane of every field), its lanes along
// x with four values in flight; a few CTAs per SM loop over the rows.
__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

template <typename T>
__global__ void __launch_bounds__(256) interior_scatter_kernel(T* __restrict__ u,
                                                               const T* __restrict__ dense, Layout L) {
  const int X = L.n0 + 2 * L.g, Y = L.n1 + 2 * L.g, Z = L.n2 + 2 * L.g;
  const int rows = L.nf * Z * Y;
  const int lane = threadIdx.x & 31;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += (gridDim.x * blockDim.x) >> 5) {
    const int y = r % Y, zf = r / Y, z = zf % Z, f = zf / Z;
    const int yi = wrap(y - L.g, L.n1), zi = wrap(z - L.g, L.n2);
    const T* src = dense + (((long long)f * L.n2 + zi) * L.n1 + yi) * L.n0;
    T* dst = u + f * L.sf + (long long)z * L.sz + (long long)y * L.sy;
    for (int x0 = 0; x0 < X; x0 += 128) {
      T v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int x = x0 + 32 * q + lane;
        if (x < X) v[q] = src[wrap(x - L.g, L.n0)];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int x = x0 + 32 * q + lane;
        if (x < X) dst[x] = v[q];
      }
    }
  }
}

// The interior of the patch layout gathered into a dense array, warps along
// interior rows.
template <typename T>
__global__ void __launch_bounds__(256) interior_gather_kernel(T* __restrict__ dense,
                                                              const T* __restrict__ u, Layout L) {
  const int rows = L.nf * L.n2 * L.n1;
  const int lane = threadIdx.x & 31;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += (gridDim.x * blockDim.x) >> 5) {
    const int y = r % L.n1, zf = r / L.n1, z = zf % L.n2, f = zf / L.n2;
    const T* src = u + f * L.sf + (long long)(z + L.g) * L.sz + (long long)(y + L.g) * L.sy + L.g;
    T* dst = dense + (long long)r * L.n0;
    for (int x0 = 0; x0 < L.n0; x0 += 128) {
      T v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int x = x0 + 32 * q + lane;
        if (x < L.n0) v[q] = src[x];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int x = x0 + 32 * q + lane;
        if (x < L.n0) dst[x] = v[q];
      }
    }
  }
}

sf_status interior_copy(bool scatter, bool fp64, void* arr, void* dense, const Layout& L,
                        cudaStream_t st) {
  const long long rows = scatter ? (long long)L.nf * (L.n2 + 2 * L.g) * (L.n1 + 2 * L.g)
                                 : (long long)L.nf * L.n2 * L.n1;
  if (rows > 0x7fffffffLL) return set_error(SF_EINVAL, "patch too large for an interior host image");
  const int blocks = (int)std::min<long long>((rows + 7) / 8, 152LL * 8);
  if (scatter) {
    if (fp64)
      interior_scatter_kernel<double><<<blocks, 256, 0, st>>>(static_cast<double*>(arr),
                                                              static_cast<const double*>(dense), L);
    else
      interior_scatter_kernel<float><<<blocks, 256, 0, st>>>(static_cast<float*>(arr),
                                                             static_cast<const float*>(dense), L);
    return after_launch("interior_scatter_kernel");
  }
  if (fp64)
    interior_gather_kernel<double><<<blocks, 256, 0, st>>>(static_cast<double*>(dense),
                                                           static_cast<const double*>(arr), L);
  else
    interior_gather_kernel<float><<<blocks, 256, 0, st>>>(static_cast<float*>(dense),
                                                          static_cast<const float*>(arr), L);
  return after_launch("interior_gather_kernel");
}

}  // namespace
}  // namespace sf

using namespace sf;

extern "C" {

int64_t sf_interior_span(const sf_patch* geom) {
  if (!geom) return -1;
  const int nf = sf_nfields(geom->system);
  if (nf < 0) return -1;
  return (long long)nf * geom->n[0] * geom->n[1] * geom->n[2];
}

int64_t sf_state_span(const sf_patch* geom) {
  if (!geom) return -1;
  sf_patch p = *geom;
  const int nf = sf_nfields(p.system);
  if (nf < 0) return -1;
  normalise_strides(p, nf);
  const long long g2 = 2LL * p.ghost;
  return (long long)(nf - 1) * p.sf + (p.n[2] + g2 - 1) * p.sz + (p.n[1] + g2 - 1) * p.sy +
         (p.n[0] + g2);
}

sf_status sf_step_host(const sf_params* prm, const sf_patch* geom, const sf_state* slots,
                       int32_t nslots, const void* const* host_in, void* const* host_out,
                       int32_t nsteps, uint32_t flags, void* compute_stream, void* h2d_stream,
                       void* d2h_stream) {
  if (!prm || !geom || !slots || !host_in || !host_out) return set_error(SF_EINVAL, "NULL argument");
  if (nslots < 1 || nslots > kMaxSlots)
    return set_error(SF_EINVAL, "nslots = %d not in 1..%d", nslots, kMaxSlots);
  if (nsteps < 0) return set_error(SF_EINVAL, "nsteps = %d < 0", nsteps);
  if (flags & ~(SF_HOST_RESET_KAHAN | SF_HOST_INTERIOR)) return set_error(SF_EINVAL, "unknown flags 0x%x", flags);
  const bool interior = (flags & SF_HOST_INTERIOR) != 0;
  if (interior && prm->ghosts != SF_GHOSTS_PERIODIC)
    return set_error(SF_EINVAL, "SF_HOST_INTERIOR needs periodic ghosts (prm->ghosts)");
  const int nst = prm->rk == SF_RK4 ? 4 : (prm->rk == SF_SSPRK3 ? 3 : 0);
  if (!nst) return set_error(SF_EINVAL, "unknown rk %d", prm->rk);
  const long long span = sf_state_span(geom);
  if (span <= 0) return set_error(SF_EINVAL, "unknown system %d", geom->system);
  const size_t es = geom->precision == SF_FP64 ? 8 : 4;
  const size_t bytes = (size_t)span * es;
  // what crosses the host link per step: the state image, or its interior
  const size_t hbytes = interior ? (size_t)sf_interior_span(geom) * es : bytes;
  sf_patch gp = *geom;
  normalise_strides(gp, sf_nfields(gp.system));
  const Layout lay{gp.n[0], gp.n[1], gp.n[2], gp.ghost, sf_nfields(gp.system), gp.sy, gp.sz, gp.sf};
  // every stage of every slot, checked before anything is enqueued
  for (int q = 0; q < nslots; ++q) {
    const sf_state& d = slots[q];
    void* us[4] = {d.u, d.s1, d.s2, d.s1};
    void* nx[4] = {d.s1, d.s2, d.s1, d.u};
    if (nst == 3) {
      nx[2] = d.u;
    }
    for (int s = 0; s < nst; ++s) {
      sf_patch p = *geom;
      p.u_n = d.u;
      p.u_stage = us[s];
      p.u_next = nx[s];
      p.acc = d.acc;
      p.kahan = d.kahan;
      normalise_strides(p, sf_nfields(p.system));
      sf_status e = check_patch(prm, p, 1, s);
      if (e) return e;
    }
    if ((flags & SF_HOST_RESET_KAHAN) && !d.kahan)
      return set_error(SF_EINVAL, "SF_HOST_RESET_KAHAN without a kahan array");
  }
  for (int k = 0; k < nsteps; ++k)
    if (!host_in[k] || !host_out[k]) return set_error(SF_EINVAL, "host buffer %d is NULL", k);
  HostEvents* ev = nullptr;
  sf_status e = host_events(&ev);
  if (e) return e;
  cudaStream_t cs = (cudaStream_t)compute_stream;
  cudaStream_t up = h2d_stream ? (cudaStream_t)h2d_stream : cs;
  cudaStream_t dn = d2h_stream ? (cudaStream_t)d2h_stream : cs;
  // earlier calls' downloads finish before this call's uploads start, and
  // this call's work follows what the compute stream already holds
  if (cudaEventRecord(ev->entry, dn) != cudaSuccess || cudaStreamWaitEvent(up, ev->entry, 0) != cudaSuccess ||
      cudaEventRecord(ev->entry, cs) != cudaSuccess || cudaStreamWaitEvent(up, ev->entry, 0) != cudaSuccess)
    return set_error(SF_ECUDA, "stream ordering failed");
  for (int k = 0; k < nsteps; ++k) {
    const sf_state& d = slots[k % nslots];
    const int b = k % nslots;
    // the image in kChunks pieces [piece(c), piece(c + 1)), 256-byte aligned
    auto piece = [&](int c) -> size_t {
      return c >= kChunks ? hbytes : hbytes / kChunks / 256 * 256 * c;
    };
    char* dbuf = static_cast<char*>(interior ? d.s2 : d.u);
    const char* hin = static_cast<const char*>(host_in[k]);
    // interior images land in the slot's s2 (stage scratch, free until stage
    // 1 writes it) and are spread into u with their periodic ghost shell
    for (int c = 0; c < kChunks; ++c) {
      const size_t lo = piece(c), hi = piece(c + 1);
      if (hi <= lo) continue;
      // the slot's previous download of this piece of its device buffer, and
      // the downloads of earlier steps of this call into the host memory it reads
      if (k >= nslots && cudaStreamWaitEvent(up, ev->down[b][c], 0) != cudaSuccess)
        return set_error(SF_ECUDA, "stream ordering failed");
      for (int j = std::max(0, k - nslots + 1); j < k; ++j)
        for (int c2 = 0; c2 < kChunks; ++c2) {
          const size_t lo2 = piece(c2), hi2 = piece(c2 + 1);
          if (hi2 > lo2 &&
              overlap(hin + lo, hi - lo, static_cast<const char*>(host_out[j]) + lo2, hi2 - lo2) &&
              cudaStreamWaitEvent(up, ev->down[j % nslots][c2], 0) != cudaSuccess)
            return set_error(SF_ECUDA, "stream ordering failed");
        }
      if (cudaMemcpyAsync(dbuf + lo, hin + lo, hi - lo, cudaMemcpyHostToDevice, up) != cudaSuccess)
        return set_error(SF_ECUDA, "upload of step %d failed", k);
    }
    if (interior && (e = interior_copy(true, geom->precision == SF_FP64, d.u, d.s2, lay, up))) return e;
    if ((flags & SF_HOST_RESET_KAHAN) && cudaMemsetAsync(d.kahan, 0, bytes, up) != cudaSuccess)
      return set_error(SF_ECUDA, "Kahan reset of step %d failed", k);
    if (cudaEventRecord(ev->up[b], up) != cudaSuccess || cudaStreamWaitEvent(cs, ev->up[b], 0) != cudaSuccess)
      return set_error(SF_ECUDA, "stream ordering failed");
    void* us[4] = {d.u, d.s1, d.s2, d.s1};
    void* nx[4] = {d.s1, d.s2, d.s1, d.u};
    if (nst == 3) nx[2] = d.u;
    for (int s = 0; s < nst; ++s) {
      sf_patch p = *geom;
      p.u_n = d.u;
      p.u_stage = us[s];
      p.u_next = nx[s];
      p.acc = d.acc;
      p.kahan = d.kahan;
      e = sf_substep(prm, &p, 1, s, compute_stream);
      if (e) return e;
    }
    // interior images: U^{n+1}'s interior gathered into s2 (free after the
    // last stage) for the download
    if (interior && (e = interior_copy(false, geom->precision == SF_FP64, d.u, d.s2, lay, cs))) return e;
    if (cudaEventRecord(ev->comp[b], cs) != cudaSuccess || cudaStreamWaitEvent(dn, ev->comp[b], 0) != cudaSuccess)
      return set_error(SF_ECUDA, "stream ordering failed");
    for (int c = 0; c < kChunks; ++c) {
      const size_t lo = piece(c), hi = piece(c + 1);
      if (hi <= lo) continue;
      if (cudaMemcpyAsync(static_cast<char*>(host_out[k]) + lo, dbuf + lo, hi - lo,
                          cudaMemcpyDeviceToHost, dn) != cudaSuccess)
        return set_error(SF_ECUDA, "download of step %d failed", k);
      if (cudaEventRecord(ev->down[b][c], dn) != cudaSuccess) return set_error(SF_ECUDA, "event record failed");
    }
  }
  return SF_OK;
}

}  // extern "C"
