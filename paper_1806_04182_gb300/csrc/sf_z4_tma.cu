// CCZ4 stage kernels with TMA-staged stencils (float storage, centred
// advection).  The per-point right-hand side is the same z4_cell as the
// global-load kernel; only its stencil source differs.  Three kernels share
// the staging scheme below:
//   z4_tma_kernel        the padded 96^3 layout, compile-time global strides
//                        (the benchmark's configuration);
//   z4_tma_any_kernel    any patch size with row, plane and field pitches on
//                        16-byte boundaries, runtime strides, tiles that may
//                        overhang the patch;
//   z4_tma_batch_kernel  the tiles of many such patches in one launch (the
//                        CCZ4 patches of sf_batch), arguments and tensor maps
//                        read from device memory.
//
// Each CTA computes a 32 x 12 x 1 tile of points, one warp per row.  The
// CCZ4 right-hand side consumes the 25 fields' stencils one field at a time in
// a fixed order (the shift, the conformal metric, chi, alpha, Gammahat, Khat,
// Theta, A~, B), so the halo box of every field (40 x 18 x 7 floats: the
// 38 x 18 x 7 the 4th-order and Kreiss-Oliger stencils reach, x rounded up to
// 16 bytes) is copied into shared memory by a cp.async.bulk.tensor load ahead
// of its use.  A ring of slots, each with a "full" mbarrier (the TMA
// transaction count) and an "empty" mbarrier (one arrival per warp), keeps
// all but two slots in flight: thread 0 issues the load for field use
// u + slots - 2 when the warps reach field use u.  Warps wait only for the
// field they need, so there is no CTA-wide barrier after the barrier
// initialisation.
//
// Every wait is bounded (about a second of clock cycles); a wait that gives up
// sets ST_TIMEOUT in the status word, and the kernel finishes its points with
// whatever the slot holds, waits (bounded) for its own loads still in flight
// and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "sf_internal.cuh"
#include "sf_mbar.cuh"
#include "sf_z4.cuh"

namespace sf {
namespace {

// A CTA computes an XP x BY x 1 tile of points (32 / XP rows per warp: one
// row of 32 points, or two rows of 16); the staged box of a field is
// XB x (BY + 6) x TZ floats with XB = XP + 6 rounded up to 16 bytes, each slot
// rounded up to 128 B.  Shared memory: KS slots, 2 KS mbarriers, and the 25
// right-hand sides of every thread (parked until the RK combination at the
// end).
constexpr int TX = 40, TZ = 7;
constexpr int kSY = 104, kSZ = 104 * 102;         // global strides of the padded 96^3 layout
constexpr long long kWaitCycles = 2000000000LL;   // ~1 s at GB300 clocks

template <int BY, int KS, int XP = 32>
struct Cfg {
  static constexpr int XB = ((XP + 6 + 3) / 4) * 4;  // 40 for XP = 32, 24 for XP = 16
  static constexpr int TY = BY + 6;
  static constexpr int kBoxBytes = XB * TY * TZ * 4;
  static constexpr int kSlotFloats = ((kBoxBytes + 127) / 128) * 32;
  static constexpr int kSlots = KS;
  static constexpr int kThreads = XP * BY;
  static constexpr int kRbufOffset = KS * kSlotFloats * 4 + 2 * KS * 8;
  static constexpr int kSmemBytes = kRbufOffset + 25 * kThreads * 4;
  static constexpr int kMinBlocks = BY <= 4 ? 3 : 1;  // 168 registers a thread
};

// The configuration in use: one CTA of 12 warps per SM (168 registers x 384
// threads), a ring of 8 slots (6 fields in flight), 200 KB of shared memory.
// Measured on the 96^3 patch against 4-warp CTAs (3 per SM) and 6- or
// 10-slot rings: the 12 warps of one CTA stay within two fields of each
// other (the ring couples them), so they share the instruction cache, and
// the kernel is bound by instruction fetch.
constexpr int kBY = 12, kKS = 8;
static_assert(kTmaTileX == 32 && kTmaTileY == kBY, "batch tiles are the kernel's tiles");
static_assert(Cfg<kBY, kKS>::XB == TX, "the 32-wide box");
// The second tile of the batch kernel: 16 x 24 points, same 12 warps, same
// slot size (24 x 30 x 7 floats), for patches that a 32-wide tile overhangs.
constexpr int kBY16 = 24;
static_assert(Cfg<kBY16, kKS, 16>::kThreads == Cfg<kBY, kKS>::kThreads, "12 warps either way");
static_assert(Cfg<kBY16, kKS, 16>::kSlotFloats == Cfg<kBY, kKS>::kSlotFloats, "same slots");
static_assert(kTmaTileX16 == 16 && kTmaTileY16 == kBY16, "batch narrow tiles are the kernel's tiles");

// Order in which z4_cell opens the fields' stencils (cross, then the mixed
// derivatives of the same field).  Without the Gamma-driver (shift frozen)
// the last three are not used.
__constant__ signed char kFieldSeq[25] = {19, 20, 21, 1, 2, 3, 4, 5, 6, 14, 15, 16, 0,
                                          18, 7, 17, 8, 9, 10, 11, 12, 13, 22, 23, 24};

__device__ __forceinline__ void tma_load_4d(float* dst, const CUtensorMap* map, int x, int y, int z,
                                            int f, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(f), "r"(saddr(bar))
      : "memory");
}

// Stencil source for z4_cell reading the staged boxes.
template <int BY, int KS, int XP = 32>
struct TmaSrc {
  using C = Cfg<BY, KS, XP>;
  static constexpr int XB = C::XB;
  static constexpr int TY = C::TY;
  static constexpr int kSlots = KS;
  static constexpr int kSlotFloats = C::kSlotFloats;
  static constexpr int kBoxBytes = C::kBoxBytes;
  const float* __restrict__ u;  // global stage input at this point, field 0
  long long F;
  float* tiles;
  uint64_t* full;
  uint64_t* empty;
  const CUtensorMap* map;
  unsigned* status;
  int local;          // this thread's centre inside a box
  int use, cur, nuses, issued;
  int gx, gy, gz;     // ghosted coordinates of the box origin
  bool leader, lane0, dead;

  __device__ __forceinline__ static constexpr long long sy() { return XB; }
  __device__ __forceinline__ static constexpr long long sz() { return XB * TY; }
  __device__ __forceinline__ const float* p(int) const { return tiles + cur * kSlotFloats + local; }
  __device__ __forceinline__ float ld(const float* q) const { return *q; }
  __device__ __forceinline__ float centre(int f) const { return __ldg(u + f * F); }

  __device__ __forceinline__ void fail() {
    if (!dead) atomicOr(status, ST_TIMEOUT);
    dead = true;
  }

  // leader: load field use j into its slot once the previous occupant
  // (use j - kSlots) has been released by every warp
  __device__ __forceinline__ void issue(int j) {
    const int sl = j % kSlots;
    if (j >= kSlots && !dead && !mbar_wait(&empty[sl], ((j / kSlots) - 1) & 1, kWaitCycles)) fail();
    if (dead) return;
    mbar_expect(&full[sl], kBoxBytes);
    tma_load_4d(tiles + sl * kSlotFloats, map, gx, gy, gz, kFieldSeq[j], &full[sl]);
    issued = j + 1;
  }

  __device__ __forceinline__ void prologue() {
    if (leader)
      for (int j = 0; j < kSlots - 2 && j < nuses; ++j) issue(j);
  }

  __device__ __forceinline__ void begin(int) {
    const int i = use++;
    if (leader && i + kSlots - 2 < nuses) issue(i + kSlots - 2);
    if (i > 0) {
      __syncwarp();
      if (lane0) mbar_arrive(&empty[(i - 1) % kSlots]);
    }
    cur = i % kSlots;
    if (!dead && !mbar_wait(&full[cur], (i / kSlots) & 1, kWaitCycles)) fail();
  }

  // the leader's warp consumed every load it issued unless a wait gave up;
  // then it waits (bounded) for the loads still in flight before exiting
  __device__ __forceinline__ void finish() {
    if (leader && dead)
      for (int j = use; j < issued; ++j) mbar_wait(&full[j % kSlots], (j / kSlots) & 1, kWaitCycles);
  }
};

}  // namespace

template <typename H, int BY, int KS>
__global__ void __launch_bounds__(Cfg<BY, KS>::kThreads, Cfg<BY, KS>::kMinBlocks)
    z4_tma_kernel(const __grid_constant__ CUtensorMap map, PatchArgs<float> a, StageArgs s,
                  Z4Coef<float> zc) {
  using C = Cfg<BY, KS>;
  constexpr int kSlots = KS;
  extern __shared__ __align__(128) unsigned char smem[];
  float* tiles = reinterpret_cast<float*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kSlots * C::kSlotFloats * 4);
  uint64_t* empty = full + kSlots;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (tid == 0) {
    for (int q = 0; q < kSlots; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], BY);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  // whole tiles only (checked on the host): every thread has a point
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const long long c = (long long)(k + 3) * kSZ + (long long)(j + 3) * kSY + (i + 3);
  TmaSrc<BY, KS> src;
  src.u = a.us + c;
  src.F = a.sf;
  src.tiles = tiles;
  src.full = full;
  src.empty = empty;
  src.map = &map;
  src.status = s.status;
  src.local = (3 * C::TY + threadIdx.y + 3) * TX + threadIdx.x + 3;
  src.use = 0;
  src.cur = 0;
  src.nuses = zc.shift_frozen ? 22 : 25;
  src.issued = 0;
  src.gx = blockIdx.x * 32;  // interior x0 - 3, in ghosted coordinates
  src.gy = blockIdx.y * BY;
  src.gz = k;
  src.leader = tid == 0;
  src.lane0 = threadIdx.x == 0;
  src.dead = false;
  src.prologue();
  const Images im = ghost_images(a, s, i, j, k);
  // right-hand sides parked in shared memory; the RK combination runs once at
  // the end as a rolled loop over the fields (as in the global-load kernel)
  float* rbuf = reinterpret_cast<float*>(smem + C::kRbufOffset);
  z4_cell<float, H, false>(a, zc, src, [&](int f, float r, float) { rbuf[f * C::kThreads + tid] = r; });
  write_fields<float, 25>(a, s, im, c, i, j, k, rbuf + tid, C::kThreads);
}

// One XP x BY x 1 tile at interior (x0, y0, z0) of a patch with runtime
// strides (row, plane and field pitches multiples of 4 floats): 32 x 12 (one
// row per warp) or 16 x 24 (two rows per warp, lanes 0-15 and 16-31).  The
// tile may overhang the patch in x and y: the TMA box reads zeros beyond the
// array, the overhanging threads still take part in the ring (they compute on
// clamped centre values) and write nothing.  `a` may live in shared memory.
template <typename H, int XP>
__device__ __forceinline__ void tma_tile_runtime(const CUtensorMap* map, const PatchArgs<float>& a,
                                                 const StageArgs& s, const Z4Coef<float>& zc,
                                                 int x0, int y0, int k, unsigned char* smem) {
  constexpr int BY = XP == 32 ? kBY : kBY16;
  using C = Cfg<BY, kKS, XP>;
  constexpr int kSlots = kKS;
  float* tiles = reinterpret_cast<float*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kSlots * C::kSlotFloats * 4);
  uint64_t* empty = full + kSlots;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  // 16-wide tiles: the half-warps take rows two apart (warp w: rows
  // 4 (w / 2) + w % 2 and that + 2), so that their shared-memory rows, 24
  // floats each, start 48 floats = 16 banks apart and never share a bank
  const int lx = threadIdx.x % XP;
  const int ly = XP == 32 ? (int)threadIdx.y
                          : 4 * (threadIdx.y / 2) + threadIdx.y % 2 + 2 * (threadIdx.x / 16);
  const int i = x0 + lx, j = y0 + ly;
  const bool valid = i < a.n[0] && j < a.n[1];
  const int ic = min(i, a.n[0] - 1), jc = min(j, a.n[1] - 1);
  const long long c = (long long)(k + 3) * a.sz + (long long)(jc + 3) * a.sy + (ic + 3);
  TmaSrc<BY, kKS, XP> src;
  src.u = a.us + c;
  src.F = a.sf;
  src.tiles = tiles;
  src.full = full;
  src.empty = empty;
  src.map = map;
  src.status = s.status;
  src.local = (3 * C::TY + ly + 3) * C::XB + lx + 3;
  src.use = 0;
  src.cur = 0;
  src.nuses = zc.shift_frozen ? 22 : 25;
  src.issued = 0;
  src.gx = x0;  // interior x0 - 3, in ghosted coordinates
  src.gy = y0;
  src.gz = k;
  src.leader = tid == 0;
  src.lane0 = threadIdx.x == 0;
  src.dead = false;
  src.prologue();
  float* rbuf = reinterpret_cast<float*>(smem + C::kRbufOffset);
  z4_cell<float, H, false>(a, zc, src, [&](int f, float r, float) { rbuf[f * C::kThreads + tid] = r; });
  if (valid) {
    const Images im = ghost_images(a, s, i, j, k);
    write_fields<float, 25>(a, s, im, c, i, j, k, rbuf + tid, C::kThreads);
  }
}

__device__ __forceinline__ void init_ring(unsigned char* smem) {
  using C = Cfg<kBY, kKS>;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kKS * C::kSlotFloats * 4);
  uint64_t* empty = full + kKS;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    for (int q = 0; q < kKS; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kBY);  // one arrival per warp: 12 warps for either tile
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
}

// Any patch size and any 16-byte pitches (one patch, map and arguments as
// kernel parameters): grid (ceil(nx / 32), ceil(ny / 12), nz).
template <typename H>
__global__ void __launch_bounds__(Cfg<kBY, kKS>::kThreads, 1)
    z4_tma_any_kernel(const __grid_constant__ CUtensorMap map, PatchArgs<float> a, StageArgs s,
                      Z4Coef<float> zc) {
  extern __shared__ __align__(128) unsigned char smem[];
  init_ring(smem);
  __syncthreads();
  tma_tile_runtime<H, 32>(&map, a, s, zc, blockIdx.x * 32, blockIdx.y * kBY, blockIdx.z, smem);
}

// The same over the tiles of many patches (the CCZ4 patches of a batch): one
// CTA per tile, the tile's patch from `tl`, its arguments copied from `args`
// into shared memory (uniform reads), its stage input's tensor map from
// `maps` (three per patch, for the u_n, u_stage and u_next buffer roles;
// `role` picks this stage's input; the maps' boxes match the tile width XP).
template <typename H, int XP>
__global__ void __launch_bounds__(Cfg<kBY, kKS>::kThreads, 1)
    z4_tma_batch_kernel(const CUtensorMap* __restrict__ maps, int role,
                        const PatchArgs<float>* __restrict__ args, const TmaTile* __restrict__ tl,
                        StageArgs s, Z4Coef<float> zc) {
  using C = Cfg<kBY, kKS>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ PatchArgs<float> pa;
  const TmaTile w = tl[blockIdx.x];
  {
    static_assert(sizeof(PatchArgs<float>) % 4 == 0, "word copy");
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int* from = reinterpret_cast<const int*>(args + w.patch);
    int* to = reinterpret_cast<int*>(&pa);
    for (int q = tid; q < (int)(sizeof(PatchArgs<float>) / 4); q += C::kThreads) to[q] = from[q];
  }
  init_ring(smem);
  __syncthreads();
  tma_tile_runtime<H, XP>(maps + 3 * w.patch + role, pa, s, zc, w.x0, w.y0, w.z0, smem);
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

template <typename H, int BY, int KS>
sf_status launch_tma(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                     void* rhs_out, cudaStream_t st) {
  using C = Cfg<BY, KS>;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return set_error(SF_ECUDA, "cuTensorMapEncodeTiled not available");
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  const cuuint64_t dims[4] = {(cuuint64_t)(p.n[0] + 6), (cuuint64_t)(p.n[1] + 6),
                              (cuuint64_t)(p.n[2] + 6), 25};
  const cuuint64_t strides[3] = {(cuuint64_t)p.sy * 4, (cuuint64_t)p.sz * 4, (cuuint64_t)p.sf * 4};
  const cuuint32_t box[4] = {TX, (cuuint32_t)C::TY, TZ, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p.u_stage, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(SF_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(z4_tma_kernel<H, BY, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         C::kSmemBytes);
  });
  PatchArgs<float> a = make_args<float>(prm, p, stage, 25, rhs_out);
  const Z4Coef<float> zc = z4_coef<float>(prm);
  dim3 block(32, BY, 1);
  dim3 grid(p.n[0] / 32, p.n[1] / BY, p.n[2]);
  z4_tma_kernel<H, BY, KS><<<grid, block, C::kSmemBytes, st>>>(map, a, s, zc);
  return after_launch("z4_tma_kernel");
}

}  // namespace

// The staged kernel serves float storage with centred advection on the
// padded 96^3 layout: 3 ghosts, row pitch 104 floats (416 bytes), plane
// pitch 104 x 102, field pitch a multiple of 4 floats, 16-byte aligned
// arrays, and whole 32 x 12 tiles in x and y.
bool z4_tma_eligible(const sf_params& prm, const sf_patch& p) {
  if (p.precision == SF_FP64 || prm.lopsided) return false;
  if (p.ghost != 3 || p.sy != kSY || p.sz != kSZ || p.sf % 4) return false;
  if (p.n[0] % 32 || p.n[1] % kBY || p.n[0] + 6 > kSY || p.n[1] + 6 > 102) return false;
  if (reinterpret_cast<uintptr_t>(p.u_stage) % 16) return false;
  return true;
}

// Batch form: float storage, centred advection, 3 ghosts, row / plane /
// field pitches that are multiples of 4 floats (16 bytes, as TMA requires)
// and 16-byte aligned arrays; any interior size (tiles may overhang).
bool z4_tma_batch_eligible(const sf_params& prm, const sf_patch& p) {
  if (p.system != SF_Z4 || p.precision == SF_FP64 || prm.lopsided) return false;
  if (p.ghost != 3 || p.sy % 4 || p.sz % 4 || p.sf % 4) return false;
  for (const void* q : {(const void*)p.u_n, (const void*)p.u_stage, (const void*)p.u_next})
    if (reinterpret_cast<uintptr_t>(q) % 16) return false;
  return true;
}

// Tensor map of the ghosted float array `base` with p's extents and strides,
// boxes of the staged kernel for tiles xp wide: 40 x 18 x 7 x 1 (xp = 32) or
// 24 x 30 x 7 x 1 (xp = 16).
sf_status encode_z4_tma_map(void* out, const sf_patch& p, const void* base, int xp) {
  static_assert(sizeof(CUtensorMap) == kTmaMapBytes, "tensor map size");
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return set_error(SF_ECUDA, "cuTensorMapEncodeTiled not available");
  if (xp != 32 && xp != 16) return set_error(SF_EINVAL, "tile width %d is not 32 or 16", xp);
  using C32 = Cfg<kBY, kKS>;
  using C16 = Cfg<kBY16, kKS, 16>;
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  const cuuint64_t dims[4] = {(cuuint64_t)(p.n[0] + 6), (cuuint64_t)(p.n[1] + 6),
                              (cuuint64_t)(p.n[2] + 6), 25};
  const cuuint64_t strides[3] = {(cuuint64_t)p.sy * 4, (cuuint64_t)p.sz * 4, (cuuint64_t)p.sf * 4};
  const cuuint32_t box[4] = {(cuuint32_t)(xp == 32 ? C32::XB : C16::XB),
                             (cuuint32_t)(xp == 32 ? C32::TY : C16::TY), TZ, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(SF_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  memcpy(out, &map, sizeof(map));
  return SF_OK;
}

namespace {
template <typename H, int XP>
sf_status launch_tma_batch(const sf_params& prm, const void* d_maps, int role,
                           const PatchArgs<float>* d_args, const TmaTile* d_tiles, int ntiles,
                           const StageArgs& s, cudaStream_t st) {
  using C = Cfg<XP == 32 ? kBY : kBY16, kKS, XP>;
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(z4_tma_batch_kernel<H, XP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         C::kSmemBytes);
  });
  const Z4Coef<float> zc = z4_coef<float>(prm);
  z4_tma_batch_kernel<H, XP><<<ntiles, dim3(32, kBY, 1), C::kSmemBytes, st>>>(
      static_cast<const CUtensorMap*>(d_maps), role, d_args, d_tiles, s, zc);
  return after_launch("z4_tma_batch_kernel");
}
}  // namespace

sf_status launch_z4_tma_batch(const sf_params& prm, int precision, const void* d_maps, int role,
                              const PatchArgs<float>* d_args, const TmaTile* d_tiles, int ntiles,
                              int xp, const StageArgs& s, cudaStream_t st) {
  if (ntiles <= 0) return SF_OK;
  const bool d = precision == SF_FP32_BULK_DW;
  if (xp == 16)
    return d ? launch_tma_batch<dw, 16>(prm, d_maps, role, d_args, d_tiles, ntiles, s, st)
             : launch_tma_batch<double, 16>(prm, d_maps, role, d_args, d_tiles, ntiles, s, st);
  return d ? launch_tma_batch<dw, 32>(prm, d_maps, role, d_args, d_tiles, ntiles, s, st)
           : launch_tma_batch<double, 32>(prm, d_maps, role, d_args, d_tiles, ntiles, s, st);
}

namespace {
template <typename H>
sf_status launch_tma_any(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                         void* rhs_out, cudaStream_t st) {
  using C = Cfg<kBY, kKS>;
  alignas(64) unsigned char map[kTmaMapBytes];
  sf_status e = encode_z4_tma_map(map, p, p.u_stage, 32);
  if (e) return e;
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(z4_tma_any_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         C::kSmemBytes);
  });
  PatchArgs<float> a = make_args<float>(prm, p, stage, 25, rhs_out);
  const Z4Coef<float> zc = z4_coef<float>(prm);
  dim3 grid((p.n[0] + 31) / 32, (p.n[1] + kBY - 1) / kBY, p.n[2]);
  z4_tma_any_kernel<H><<<grid, dim3(32, kBY, 1), C::kSmemBytes, st>>>(
      *reinterpret_cast<const CUtensorMap*>(map), a, s, zc);
  return after_launch("z4_tma_any_kernel");
}
}  // namespace

// Float storage with centred advection and 16-byte pitches and arrays, any
// interior size: the compile-time-stride kernel for the padded 96^3 layout,
// the runtime-stride kernel (tiles may overhang) for every other.
bool z4_tma_any_eligible(const sf_params& prm, const sf_patch& p) {
  if (p.precision == SF_FP64 || prm.lopsided) return false;
  if (p.ghost != 3 || p.sy % 4 || p.sz % 4 || p.sf % 4) return false;
  return reinterpret_cast<uintptr_t>(p.u_stage) % 16 == 0;
}

sf_status launch_z4_tma(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                        void* rhs_out, cudaStream_t st) {
  if (z4_tma_eligible(prm, p)) {
    if (p.precision == SF_FP32_BULK_DW) return launch_tma<dw, kBY, kKS>(prm, p, s, stage, rhs_out, st);
    return launch_tma<double, kBY, kKS>(prm, p, s, stage, rhs_out, st);
  }
  if (p.precision == SF_FP32_BULK_DW) return launch_tma_any<dw>(prm, p, s, stage, rhs_out, st);
  return launch_tma_any<double>(prm, p, s, stage, rhs_out, st);
}

}  // namespace sf
