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
struct HostEvents {
  int dev = -1;
  cudaEvent_t up[kMaxSlots], comp[kMaxSlots], down[kMaxSlots], entry;
};
thread_local HostEvents t_ev;

sf_status host_events(HostEvents** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return set_error(SF_ECUDA, "no CUDA device");
  HostEvents& e = t_ev;
  if (e.dev != dev) {
    cudaEvent_t* all[3 * kMaxSlots + 1];
    for (int q = 0; q < kMaxSlots; ++q) {
      all[3 * q] = &e.up[q];
      all[3 * q + 1] = &e.comp[q];
      all[3 * q + 2] = &e.down[q];
    }
    all[3 * kMaxSlots] = &e.entry;
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

bool overlap(const void* a, const void* b, size_t n) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + n && y < x + n;
}

}  // namespace
}  // namespace sf

using namespace sf;

extern "C" {

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
  if (flags & ~SF_HOST_RESET_KAHAN) return set_error(SF_EINVAL, "unknown flags 0x%x", flags);
  const int nst = prm->rk == SF_RK4 ? 4 : (prm->rk == SF_SSPRK3 ? 3 : 0);
  if (!nst) return set_error(SF_EINVAL, "unknown rk %d", prm->rk);
  const long long span = sf_state_span(geom);
  if (span <= 0) return set_error(SF_EINVAL, "unknown system %d", geom->system);
  const size_t bytes = (size_t)span * (geom->precision == SF_FP64 ? 8 : 4);
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
    // the slot's previous download, and the downloads this input depends on
    // (an earlier step of this call whose output it overlaps)
    if (k >= nslots && cudaStreamWaitEvent(up, ev->down[b], 0) != cudaSuccess)
      return set_error(SF_ECUDA, "stream ordering failed");
    for (int j = std::max(0, k - nslots + 1); j < k; ++j)
      if (overlap(host_in[k], host_out[j], bytes) &&
          cudaStreamWaitEvent(up, ev->down[j % nslots], 0) != cudaSuccess)
        return set_error(SF_ECUDA, "stream ordering failed");
    if (cudaMemcpyAsync(d.u, host_in[k], bytes, cudaMemcpyHostToDevice, up) != cudaSuccess)
      return set_error(SF_ECUDA, "upload of step %d failed", k);
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
    if (cudaEventRecord(ev->comp[b], cs) != cudaSuccess || cudaStreamWaitEvent(dn, ev->comp[b], 0) != cudaSuccess)
      return set_error(SF_ECUDA, "stream ordering failed");
    if (cudaMemcpyAsync(host_out[k], d.u, bytes, cudaMemcpyDeviceToHost, dn) != cudaSuccess)
      return set_error(SF_ECUDA, "download of step %d failed", k);
    if (cudaEventRecord(ev->down[b], dn) != cudaSuccess) return set_error(SF_ECUDA, "event record failed");
  }
  return SF_OK;
}

}  // extern "C"
