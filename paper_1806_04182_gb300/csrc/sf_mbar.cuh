// Shared-memory mbarrier operations (PTX mbarrier.*), the bounded wait used by
// every kernel that waits on one, and a bulk L2 prefetch of row segments.  A
// wait that runs past its cycle limit gives up and reports false, so no
// kernel of this library can wait forever; the caller records the failure in
// the status word (ST_TIMEOUT).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sf {

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity, for at most `limit` clock
// cycles; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, long long limit) {
  if (mbar_try(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(b, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes)
               : "memory");
}

// Bulk L2 prefetch of the 128-byte row segment of every field that the RK
// combination of this stage reads (U^n, the accumulator, the Kahan term):
// those reads come late in the point's computation, one field at a time, and
// would otherwise each wait for DRAM.
template <int kBytes = 144>
__device__ __forceinline__ void prefetch_rows(const float* base, long long F) {
  static_assert(kBytes % 16 == 0, "bulk prefetch size");
#pragma unroll 1
  for (int f = 0; f < 25; ++f)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(base + f * F), "n"(kBytes)
                 : "memory");
}

}  // namespace sf
