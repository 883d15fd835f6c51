// Batched AMR-patch dispatch.  A table of patches of mixed systems (wave,
// CCZ4) and sizes, each with its own dx and dt (the level loop of Sec. III
// runs every patch of every level through "calculate rhs" + "integrate
// time"), is advanced by ONE persistent launch per RK stage.  CTAs pull
// (patch, tile) work items from a device counter until the list is empty;
// CCZ4 tiles are queued first so the heavy items start early.  No CTA ever
// waits on another, so the queue has no spin-waits.
// Float CCZ4 patches whose layout suits TMA (pitches and arrays on 16-byte
// boundaries, centred advection) go instead to the TMA-staged kernel, one
// launch per stage and tile width over all their 32 x 12 x 1 or 16 x 24 x 1
// tiles, ahead of the persistent launch that takes the remaining patches;
// all are captured in the graph.
//
// Buffer roles per patch (sf_patch fields as passed to sf_batch_create):
//   u_n = A: the state U^n, updated in place by the last stage
//   u_stage = B, u_next = C: stage scratch
//   acc = D: RK4 accumulator, kahan = E (FP32_BULK)
// stage 0: A -> B, stage 1: B -> C, stage 2: C -> B, stage 3: B -> A.
// Patches that tile a level (ghosts = SF_GHOSTS_NONE) get their ghost shells
// from their neighbours: sf_batch_set_halo gives, per buffer role, the box
// copies that fill them, and each stage ends with one sf_copy_boxes launch
// for the role it wrote (inside the captured graph too).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "sf_internal.cuh"
#include "sf_wave.cuh"
#include "sf_z4.cuh"

namespace sf {

// tile shapes (TX, TY, TZ); blockDim is always 128 = TX * TY
struct Shape {
  int tx, ty, tz;
};
static const Shape kShapes[] = {{32, 4, 1}, {32, 4, 2}, {32, 4, 4}, {64, 2, 1},
                                {64, 2, 2}, {16, 8, 1}, {16, 8, 2}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);
constexpr int kClasses = 4;  // (wave, z4) x (small: max n <= 32, large)

struct Item {
  int patch, x0, y0, z0;
};

template <typename T, typename H, bool LOP>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 3 : 2) batch_stage_kernel(const PatchArgs<T>* __restrict__ pa,
                                                          const int* __restrict__ psys,
                                                          const int2* __restrict__ pshape,
                                                          const Item* __restrict__ items, int nitems,
                                                          unsigned int* counter, StageArgs s,
                                                          Z4Coef<T> zc) {
  __shared__ int s_item;
  __shared__ T rbuf[25 * 128];  // parked CCZ4 right-hand sides (see write_fields)
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= nitems) return;
    const Item w = items[it];
    const PatchArgs<T>& a = pa[w.patch];
    const int2 sh = pshape[w.patch];  // (tx, tz)
    const int lx = threadIdx.x % sh.x, ly = threadIdx.x / sh.x;
    const int i = w.x0 + lx, j = w.y0 + ly;
    if (i >= a.n[0] || j >= a.n[1]) continue;
    const int g = a.g;
    const int zend = min(w.z0 + sh.y, a.n[2]);
    const int system = psys[w.patch];
    for (int k = w.z0; k < zend; ++k) {
      const long long c = (long long)(k + g) * a.sz + (long long)(j + g) * a.sy + (i + g);
      if (system == SF_Z4) {
        GlobalSrc<T, 0, 0> src{a.us + c, a.sf, a.sy, a.sz};
        const Images im = ghost_images(a, s, i, j, k);
        z4_cell<T, H, LOP>(a, zc, src, [&](int f, T r, T) { rbuf[f * 128 + threadIdx.x] = r; });
        write_fields<T, 25>(a, s, im, c, i, j, k, rbuf + threadIdx.x, 128);
      } else {
        T v[5], r[5];
        wave_point<T, false>(a, a.us + c, v, r);
        const Images im = ghost_images(a, s, i, j, k);
#pragma unroll
        for (int f = 0; f < 5; ++f) write_field(a, s, im, f, c, i, j, k, v[f], r[f]);
      }
    }
  }
}

}  // namespace sf

using namespace sf;

struct sf_batch {
  sf_params prm;
  int precision;
  int npatch;
  std::vector<sf_patch> patches;
  int shape_of_class[kClasses];
  int tma_width_of_class[kClasses];  // TMA tile width per class: -1 the fewer-tiles rule, 0: 32 x 12, 1: 16 x 24
  int device;
  int grid[3];            // persistent grid size per precision
  void* d_args = nullptr; // PatchArgs<T>[4][npatch]
  int* d_sys = nullptr;
  int2* d_shape = nullptr;
  Item* d_items = nullptr;
  int nitems = 0;
  unsigned int* d_counter = nullptr;
  std::vector<char> tma;  // patch q goes to the TMA-staged CCZ4 kernel
  std::vector<char> pair;  // patch q goes to the two-point CCZ4 kernel (takes precedence)
  void* d_pmaps = nullptr;   // its tensor maps, 6 per patch
  void* d_pcoefs = nullptr;  // its stencil weights, one block per patch
  TmaTile* d_ptiles = nullptr;  // its 32 x 16 tiles
  int npair = 0;                // two-point tiles
  void* d_maps = nullptr; // tensor maps, 3 per patch (u_n, u_stage, u_next roles)
  TmaTile* d_tiles = nullptr;   // 32 x 12 tiles, then 16 x 24 tiles
  int ntiles = 0;               // all TMA tiles
  int ntiles16 = 0;             // of which the last ntiles16 are 16 x 24
  std::vector<sf_box_copy> halo[3];  // ghost-shell copies per buffer role (u_n, u_stage, u_next)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {
// buffer role each stage writes: B, C, B, A
constexpr int kOutRole[4] = {1, 2, 1, 0};
}  // namespace

namespace {

int class_of(const sf_patch& p) {
  const int m = std::max(p.n[0], std::max(p.n[1], p.n[2]));
  return (p.system == SF_Z4 ? 2 : 0) + (m > 32 ? 1 : 0);
}

template <typename T>
sf_status upload_args(sf_batch* b) {
  const int np = b->npatch;
  std::vector<PatchArgs<T>> h(4 * (size_t)np);
  for (int st = 0; st < 4; ++st)
    for (int q = 0; q < np; ++q) {
      sf_patch p = b->patches[q];
      void* A = p.u_n;
      void* B = p.u_stage;
      void* C = p.u_next;
      void* us[4] = {A, B, C, B};
      void* nx[4] = {B, C, B, A};
      p.u_stage = us[st];
      p.u_n = A;
      p.u_next = nx[st];
      h[(size_t)st * np + q] = make_args<T>(b->prm, p, st, sf_nfields(p.system), nullptr);
    }
  if (!b->d_args && cudaMalloc(&b->d_args, h.size() * sizeof(PatchArgs<T>)) != cudaSuccess)
    return set_error(SF_ECUDA, "batch: cudaMalloc of patch table failed");
  if (cudaMemcpy(b->d_args, h.data(), h.size() * sizeof(PatchArgs<T>), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return set_error(SF_ECUDA, "batch: upload of patch table failed");
  return SF_OK;
}

// Work list for the current shape choice; CCZ4 items first.  If `only_class`
// >= 0, only patches of that class are listed (tuning).
sf_status build_items(sf_batch* b, int only_class) {
  std::vector<Item> items;
  std::vector<int2> shapes(b->npatch);
  for (int pass = 0; pass < 2; ++pass)
    for (int q = 0; q < b->npatch; ++q) {
      const sf_patch& p = b->patches[q];
      const bool z4 = p.system == SF_Z4;
      if ((pass == 0) != z4) continue;
      if (!b->tma.empty() && b->tma[q]) continue;
      if (!b->pair.empty() && b->pair[q]) continue;
      const int cls = class_of(p);
      const Shape sh = kShapes[b->shape_of_class[cls]];
      shapes[q] = make_int2(sh.tx, sh.tz);
      if (only_class >= 0 && cls != only_class) continue;
      for (int z = 0; z < p.n[2]; z += sh.tz)
        for (int y = 0; y < p.n[1]; y += sh.ty)
          for (int x = 0; x < p.n[0]; x += sh.tx) items.push_back(Item{q, x, y, z});
    }
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  b->nitems = (int)items.size();
  if (!items.empty()) {
    if (cudaMalloc(&b->d_items, items.size() * sizeof(Item)) != cudaSuccess)
      return set_error(SF_ECUDA, "batch: cudaMalloc of work list failed");
    if (cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(Item), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return set_error(SF_ECUDA, "batch: upload of work list failed");
  }
  if (cudaMemcpy(b->d_shape, shapes.data(), shapes.size() * sizeof(int2), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return set_error(SF_ECUDA, "batch: upload of shapes failed");
  return SF_OK;
}

// Tensor maps, stencil weights and tile lists of the patches served by the
// two-point CCZ4 kernel (double-word islands, the one-float row offset
// layout): 32 x 16 tiles of every plane, overhanging the patch where its
// size is not a multiple.
sf_status build_pair(sf_batch* b) {
  b->pair.assign(b->npatch, 0);
  b->npair = 0;
  if (b->precision != SF_FP32_BULK_DW) return SF_OK;
  const size_t cb = z4_pair_coef_bytes();
  std::vector<unsigned char> maps((size_t)6 * b->npatch * kTmaMapBytes, 0), coefs(cb * b->npatch, 0);
  std::vector<TmaTile> tiles;
  for (int q = 0; q < b->npatch; ++q) {
    const sf_patch& p = b->patches[q];
    if (!z4_pair_batch_eligible(b->prm, p)) continue;
    b->pair[q] = 1;
    sf_status e = encode_z4_pair_batch(maps.data() + (size_t)6 * q * kTmaMapBytes, coefs.data() + cb * q,
                                       b->prm, p);
    if (e) return e;
    for (int z = 0; z < p.n[2]; ++z)
      for (int y = 0; y < p.n[1]; y += kPairTileY)
        for (int x = 0; x < p.n[0]; x += kPairTileX) tiles.push_back(TmaTile{q, x, y, z});
  }
  b->npair = (int)tiles.size();
  if (tiles.empty()) return SF_OK;
  if (cudaMalloc(&b->d_pmaps, maps.size()) != cudaSuccess ||
      cudaMalloc(&b->d_pcoefs, coefs.size()) != cudaSuccess ||
      cudaMalloc(&b->d_ptiles, tiles.size() * sizeof(TmaTile)) != cudaSuccess)
    return set_error(SF_ECUDA, "batch: cudaMalloc of two-point tiles failed");
  if (cudaMemcpy(b->d_pmaps, maps.data(), maps.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_pcoefs, coefs.data(), coefs.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_ptiles, tiles.data(), tiles.size() * sizeof(TmaTile), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return set_error(SF_ECUDA, "batch: upload of two-point tiles failed");
  return SF_OK;
}

// Tensor maps and the tile lists of the patches served by the TMA-staged
// CCZ4 kernel (float precision, eligible layouts).  A patch takes its size
// class's tile width where sf_batch_tune has measured one, else the width
// (32 x 12 or 16 x 24 points) that covers it with fewer tiles, i.e. with
// fewer idle lanes where tiles overhang it.  only_class >= 0 lists the tiles
// of that class only (tuning); every eligible patch is still marked TMA.
sf_status build_tma(sf_batch* b, int only_class = -1) {
  b->tma.assign(b->npatch, 0);
  b->ntiles = b->ntiles16 = 0;
  if (b->d_maps) cudaFree(b->d_maps);
  if (b->d_tiles) cudaFree(b->d_tiles);
  b->d_maps = nullptr;
  b->d_tiles = nullptr;
  if (b->precision == SF_FP64) return SF_OK;
  std::vector<unsigned char> maps((size_t)3 * b->npatch * kTmaMapBytes, 0);
  std::vector<TmaTile> tiles[2];  // [0]: 32 x 12, [1]: 16 x 24
  for (int q = 0; q < b->npatch; ++q) {
    const sf_patch& p = b->patches[q];
    if (!z4_tma_batch_eligible(b->prm, p) || (!b->pair.empty() && b->pair[q])) continue;
    b->tma[q] = 1;
    auto count = [&](int tx, int ty) {
      return (long long)((p.n[0] + tx - 1) / tx) * ((p.n[1] + ty - 1) / ty);
    };
    const int cls = class_of(p);
    const int w = b->tma_width_of_class[cls] >= 0
                      ? b->tma_width_of_class[cls]
                      : (count(kTmaTileX16, kTmaTileY16) < count(kTmaTileX, kTmaTileY) ? 1 : 0);
    if (only_class >= 0 && cls != only_class) continue;
    const int tx = w ? kTmaTileX16 : kTmaTileX, ty = w ? kTmaTileY16 : kTmaTileY;
    const void* arr[3] = {p.u_n, p.u_stage, p.u_next};
    for (int r = 0; r < 3; ++r) {
      sf_status e = encode_z4_tma_map(maps.data() + ((size_t)3 * q + r) * kTmaMapBytes, p, arr[r], tx);
      if (e) return e;
    }
    for (int z = 0; z < p.n[2]; ++z)
      for (int y = 0; y < p.n[1]; y += ty)
        for (int x = 0; x < p.n[0]; x += tx) tiles[w].push_back(TmaTile{q, x, y, z});
  }
  b->ntiles16 = (int)tiles[1].size();
  tiles[0].insert(tiles[0].end(), tiles[1].begin(), tiles[1].end());
  std::vector<TmaTile>& all = tiles[0];
  b->ntiles = (int)all.size();
  if (all.empty()) return SF_OK;
  if (cudaMalloc(&b->d_maps, maps.size()) != cudaSuccess ||
      cudaMalloc(&b->d_tiles, all.size() * sizeof(TmaTile)) != cudaSuccess)
    return set_error(SF_ECUDA, "batch: cudaMalloc of tensor maps failed");
  if (cudaMemcpy(b->d_maps, maps.data(), maps.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_tiles, all.data(), all.size() * sizeof(TmaTile), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return set_error(SF_ECUDA, "batch: upload of tensor maps failed");
  return SF_OK;
}

StageArgs batch_stage_args(const sf_batch* b, int stage, unsigned int* status) {
  StageArgs s;
  s.mode = 0;
  s.rk = SF_RK4;
  s.stage = stage;
  s.kahan = b->precision != SF_FP64 ? 1 : 0;
  s.un_alias = stage == 0 ? 1 : 0;
  s.ghosts = b->prm.ghosts == SF_GHOSTS_PERIODIC ? 1 : 0;
  s.check_finite = b->prm.check_finite;
  s.status = status;
  return s;
}

template <typename T, typename H>
sf_status launch_stage(sf_batch* b, int stage, cudaStream_t st, unsigned int* status) {
  if (b->ntiles > 0 || b->npair > 0) {
    // stage roles of the stage input: A (u_n), B (u_stage), C (u_next), B
    const int role[4] = {0, 1, 2, 1};
    const PatchArgs<float>* fargs =
        static_cast<const PatchArgs<float>*>(b->d_args) + (size_t)stage * b->npatch;
    const StageArgs sa = batch_stage_args(b, stage, status);
    sf_status e = launch_z4_pair_batch(b->prm, b->d_pmaps, role[stage], fargs, b->d_pcoefs,
                                       b->d_ptiles, b->npair, sa, st);
    const int n32 = b->ntiles - b->ntiles16;
    if (!e)
      e = launch_z4_tma_batch(b->prm, b->precision, b->d_maps, role[stage], fargs, b->d_tiles, n32,
                              kTmaTileX, sa, st);
    if (!e)
      e = launch_z4_tma_batch(b->prm, b->precision, b->d_maps, role[stage], fargs, b->d_tiles + n32,
                              b->ntiles16, kTmaTileX16, sa, st);
    if (e) return e;
    if (b->nitems == 0) return SF_OK;
  }
  if (cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), st) != cudaSuccess)
    return set_error(SF_ECUDA, "batch: counter reset failed");
  Z4Coef<T> zc;
  zc.kappa_z = T(b->prm.kappa_z);
  zc.kappa_c = T(b->prm.kappa_c);
  zc.eta = T(b->prm.eta);
  zc.g_shift = T(b->prm.g_shift);
  zc.slicing = b->prm.slicing;
  zc.shift_frozen = b->prm.shift_frozen;
  zc.lopsided = b->prm.lopsided;
  const PatchArgs<T>* args = static_cast<const PatchArgs<T>*>(b->d_args) + (size_t)stage * b->npatch;
  const int grid = b->grid[b->precision];
  const StageArgs sa = batch_stage_args(b, stage, status);
  if (b->prm.lopsided)
    batch_stage_kernel<T, H, true><<<grid, 128, 0, st>>>(args, b->d_sys, b->d_shape, b->d_items,
                                                         b->nitems, b->d_counter, sa, zc);
  else
    batch_stage_kernel<T, H, false><<<grid, 128, 0, st>>>(args, b->d_sys, b->d_shape, b->d_items,
                                                          b->nitems, b->d_counter, sa, zc);
  return after_launch("batch_stage_kernel");
}

}  // namespace

extern "C" {

sf_status sf_batch_create(const sf_params* prm, const sf_patch* patches, int32_t npatch,
                          sf_batch** out) {
  if (!prm || !patches || !out || npatch < 1) return set_error(SF_EINVAL, "NULL argument or npatch < 1");
  if (prm->rk != SF_RK4) return set_error(SF_ENOTSUP, "sf_batch runs RK4");
  if (prm->ghosts != SF_GHOSTS_NONE && prm->ghosts != SF_GHOSTS_PERIODIC)
    return set_error(SF_EINVAL, "ghosts %d not SF_GHOSTS_NONE or SF_GHOSTS_PERIODIC", prm->ghosts);
  *out = nullptr;
  sf_batch* b = new sf_batch();
  b->prm = *prm;
  b->npatch = npatch;
  b->precision = patches[0].precision;
  b->patches.assign(patches, patches + npatch);
  for (int q = 0; q < npatch; ++q) {
    sf_patch& p = b->patches[q];
    normalise_strides(p, sf_nfields(p.system));
    if (p.system != SF_WAVE && p.system != SF_Z4) {
      delete b;
      return set_error(SF_ENOTSUP, "sf_batch takes SF_WAVE and SF_Z4 patches");
    }
    if (p.precision != b->precision) {
      delete b;
      return set_error(SF_EINVAL, "all patches of a batch need one precision");
    }
    // the four stage roles must be valid sf_substep patches
    for (int st = 0; st < 4; ++st) {
      sf_patch r = p;
      void* us[4] = {p.u_n, p.u_stage, p.u_next, p.u_stage};
      void* nx[4] = {p.u_stage, p.u_next, p.u_stage, p.u_n};
      r.u_stage = us[st];
      r.u_next = nx[st];
      sf_status e = check_patch(&b->prm, r, 1, st);
      if (e) {
        delete b;
        return e;
      }
    }
    if (p.u_stage == p.u_next || p.u_stage == p.u_n || p.u_next == p.u_n) {
      delete b;
      return set_error(SF_EINVAL, "batch patches need distinct u_n, u_stage and u_next buffers");
    }
  }
  for (int c = 0; c < kClasses; ++c) {
    b->shape_of_class[c] = 0;
    b->tma_width_of_class[c] = -1;
  }
  cudaGetDevice(&b->device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  int occ[3] = {0, 0, 0};
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], batch_stage_kernel<double, double, false>, 128, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], batch_stage_kernel<float, double, false>, 128, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[2], batch_stage_kernel<float, dw, false>, 128, 0);
  for (int q = 0; q < 3; ++q) b->grid[q] = std::max(1, sms * std::max(1, occ[q]));
  std::vector<int> sys(npatch);
  for (int q = 0; q < npatch; ++q) sys[q] = b->patches[q].system;
  if (cudaMalloc(&b->d_sys, npatch * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->d_shape, npatch * sizeof(int2)) != cudaSuccess ||
      cudaMalloc(&b->d_counter, sizeof(unsigned int)) != cudaSuccess) {
    sf_batch_destroy(b);
    return set_error(SF_ECUDA, "batch: cudaMalloc failed");
  }
  cudaMemcpy(b->d_sys, sys.data(), npatch * sizeof(int), cudaMemcpyHostToDevice);
  sf_status e = b->precision == SF_FP64 ? upload_args<double>(b) : upload_args<float>(b);
  if (!e) e = build_pair(b);
  if (!e) e = build_tma(b);
  if (!e) e = build_items(b, -1);
  if (e) {
    sf_batch_destroy(b);
    return e;
  }
  *out = b;
  return SF_OK;
}

sf_status sf_batch_substep(sf_batch* b, int32_t stage, void* stream) {
  if (!b) return set_error(SF_EINVAL, "batch is NULL");
  if (stage < 0 || stage > 3) return set_error(SF_EINVAL, "stage %d out of range [0,4)", stage);
  unsigned int* status = status_ptr();
  if (!status) return set_error(SF_ECUDA, "no status word");
  sf_status e;
  if (b->precision == SF_FP64)
    e = launch_stage<double, double>(b, stage, (cudaStream_t)stream, status);
  else if (b->precision == SF_FP32_BULK_DW)
    e = launch_stage<float, dw>(b, stage, (cudaStream_t)stream, status);
  else
    e = launch_stage<float, double>(b, stage, (cudaStream_t)stream, status);
  if (e) return e;
  const std::vector<sf_box_copy>& h = b->halo[kOutRole[stage]];
  if (h.empty()) return SF_OK;
  return sf_copy_boxes(h.data(), (int32_t)h.size(), b->precision, stream);
}

sf_status sf_batch_set_halo(sf_batch* b, int32_t role, const sf_box_copy* boxes, int32_t nbox) {
  if (!b) return set_error(SF_EINVAL, "batch is NULL");
  if (role < 0 || role > 2) return set_error(SF_EINVAL, "role %d not in {0, 1, 2}", role);
  sf_status e = check_box_copies(boxes, nbox, b->precision);
  if (e) return e;
  if (nbox > 0)
    b->halo[role].assign(boxes, boxes + nbox);
  else
    b->halo[role].clear();
  if (b->exec) {  // a captured step no longer matches: capture again
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  return SF_OK;
}

sf_status sf_batch_tune(sf_batch* b, void* stream) {
  if (!b) return set_error(SF_EINVAL, "batch is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  sf_status err = SF_OK;
  // the TMA-staged patches have a fixed tile: time the persistent kernel alone
  const int ntiles = b->ntiles, ntiles16 = b->ntiles16, npair = b->npair;
  b->ntiles = b->ntiles16 = b->npair = 0;
  for (int cls = 0; cls < kClasses && !err; ++cls) {
    bool any = false;
    for (int q = 0; q < b->npatch; ++q) any |= class_of(b->patches[q]) == cls && !b->tma[q];
    if (!any) continue;
    float best = 1e30f;
    int best_shape = 0;
    for (int s = 0; s < kNumShapes && !err; ++s) {
      b->shape_of_class[cls] = s;
      if ((err = build_items(b, cls))) break;
      // stage 1 writes only scratch (u_next role C and acc), never U^n
      for (int rep = 0; rep < 2 && !err; ++rep) err = sf_batch_substep(b, 1, stream);
      cudaEventRecord(e0, st);
      for (int rep = 0; rep < 3 && !err; ++rep) err = sf_batch_substep(b, 1, stream);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_shape = s;
      }
    }
    b->shape_of_class[cls] = best_shape;
  }
  b->ntiles = ntiles;
  b->ntiles16 = ntiles16;
  // the TMA tile width of each class with TMA patches: the tiles of that
  // class alone, stage 1 (it writes scratch only), each width timed
  const int nitems = b->nitems;
  b->nitems = 0;  // sf_batch_substep then launches the TMA tiles only
  for (int cls = 0; cls < kClasses && !err && ntiles > 0; ++cls) {
    bool any = false;
    for (int q = 0; q < b->npatch; ++q)
      any |= class_of(b->patches[q]) == cls && z4_tma_batch_eligible(b->prm, b->patches[q]);
    if (!any) continue;
    float best = 1e30f;
    int best_w = 0;
    for (int w = 0; w < 2 && !err; ++w) {
      b->tma_width_of_class[cls] = w;
      if ((err = build_tma(b, cls))) break;
      for (int rep = 0; rep < 2 && !err; ++rep) err = sf_batch_substep(b, 1, stream);
      cudaEventRecord(e0, st);
      for (int rep = 0; rep < 3 && !err; ++rep) err = sf_batch_substep(b, 1, stream);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_w = w;
      }
    }
    b->tma_width_of_class[cls] = best_w;
  }
  b->nitems = nitems;
  b->npair = npair;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!err) err = build_tma(b, -1);
  if (!err) err = build_items(b, -1);
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  return err;
}

sf_status sf_batch_capture(sf_batch* b, void* stream) {
  if (!b) return set_error(SF_EINVAL, "batch is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (!st) return set_error(SF_EINVAL, "graph capture needs a non-default stream");
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  status_ptr();  // resolve the symbol address before capture
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return set_error(SF_ECUDA, "begin capture failed");
  sf_status err = SF_OK;
  for (int s = 0; s < 4 && !err; ++s) err = sf_batch_substep(b, s, stream);
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(st, &g);
  if (err) {
    if (g) cudaGraphDestroy(g);
    return err;
  }
  if (ce != cudaSuccess) return set_error(SF_ECUDA, "end capture: %s", cudaGetErrorString(ce));
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    return set_error(SF_ECUDA, "graph instantiate failed");
  }
  b->graph = g;
  return SF_OK;
}

sf_status sf_batch_launch(sf_batch* b, void* stream) {
  if (!b || !b->exec) return set_error(SF_EINVAL, "batch NULL or not captured");
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return set_error(SF_ECUDA, "graph launch: %s", cudaGetErrorString(e));
  return after_launch("batch graph");
}

int32_t sf_batch_launches_per_step(const sf_batch* b) {
  if (!b) return 0;
  const int n32 = b->ntiles - b->ntiles16;
  const int per_stage = (b->npair > 0 ? 1 : 0) + (n32 > 0 ? 1 : 0) + (b->ntiles16 > 0 ? 1 : 0) +
                        ((b->ntiles == 0 && b->npair == 0) || b->nitems > 0 ? 1 : 0);
  int halo = 0;
  for (int s = 0; s < 4; ++s) {
    const std::vector<sf_box_copy>& h = b->halo[kOutRole[s]];
    halo += box_copy_launches(h.data(), (int)h.size());
  }
  return 4 * per_stage + halo;
}

sf_status sf_batch_tuned(const sf_batch* b, int32_t* shape_of_class, int32_t* tma_width_of_class) {
  if (!b) return set_error(SF_EINVAL, "batch is NULL");
  for (int c = 0; c < kClasses; ++c) {
    if (shape_of_class) {
      const Shape sh = kShapes[b->shape_of_class[c]];
      shape_of_class[3 * c] = sh.tx;
      shape_of_class[3 * c + 1] = sh.ty;
      shape_of_class[3 * c + 2] = sh.tz;
    }
    if (tma_width_of_class) {
      bool any = false;
      for (int q = 0; q < b->npatch; ++q) any |= class_of(b->patches[q]) == c && b->tma[q];
      const int w = b->tma_width_of_class[c];
      tma_width_of_class[c] = !any ? 0 : (w < 0 ? -1 : (w ? kTmaTileX16 : kTmaTileX));
    }
  }
  return SF_OK;
}

sf_status sf_batch_destroy(sf_batch* b) {
  if (!b) return SF_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_args) cudaFree(b->d_args);
  if (b->d_sys) cudaFree(b->d_sys);
  if (b->d_shape) cudaFree(b->d_shape);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->d_maps) cudaFree(b->d_maps);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_pmaps) cudaFree(b->d_pmaps);
  if (b->d_pcoefs) cudaFree(b->d_pcoefs);
  if (b->d_ptiles) cudaFree(b->d_ptiles);
  delete b;
  return SF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free batched stage.  Some callers cannot call cudaMalloc at the
// point where they advance their patches: codes that hand all device memory
// to their own pool or arena up front, and codes that must not allocate
// while other work is in flight (cudaMalloc may synchronise the device and
// cudaFree always does).  sf_batch_substep_static serves them: it runs the
// same persistent kernel as sf_batch_substep, but keeps the kernel's scratch
// (queue counter, per-patch stage table, work list) in one file-scope
// device array of fixed size instead of memory from sf_batch_create.
namespace {

constexpr int kStaticMaxPatches = 64;
constexpr int kStaticMaxItems = 8192;
constexpr Shape kStaticShape = {32, 4, 4};
constexpr int kStaticTX = 32, kStaticTY = 4, kStaticTZ = 4;  // kStaticShape, for device code
static_assert(kStaticShape.tx == kStaticTX && kStaticShape.ty == kStaticTY && kStaticShape.tz == kStaticTZ, "tile");
constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kArgsBytes = align256(kStaticMaxPatches * (sizeof(PatchArgs<double>) > sizeof(PatchArgs<float>)
                                                               ? sizeof(PatchArgs<double>)
                                                               : sizeof(PatchArgs<float>)));
constexpr size_t kOffArgs = 256;  // [0, 256): queue counter
constexpr size_t kOffSys = kOffArgs + kArgsBytes;
constexpr size_t kOffShape = kOffSys + align256(kStaticMaxPatches * sizeof(int));
constexpr size_t kOffItems = kOffShape + align256(kStaticMaxPatches * sizeof(int2));
constexpr size_t kStaticBytes = kOffItems + align256(kStaticMaxItems * sizeof(Item));
static_assert(kStaticBytes == 170496, "the scratch size is stated in sf.h: update it there");

}  // namespace

// Scratch of sf_batch_substep_static: 170,496 bytes (about 167 KB).  Every GPU that loads
// the library holds one copy until the process exits.  Host code must not
// use this name as a device address; it asks the runtime for the address.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

namespace {

// The stage table reaches the scratch array through kernel parameters: each
// upload launch carries up to kChunkBytes of it by value, so every call's
// table is its own (nothing is read from host memory after the call returns)
// and no host buffer is shared between calls.
constexpr unsigned kChunkBytes = 28 * 1024;
struct StaticChunk {
  unsigned off, nbytes;  // destination offset in the scratch, bytes (multiples of 4)
  unsigned data[kChunkBytes / 4];
};
static_assert(sizeof(StaticChunk) <= 32764, "kernel parameter limit");

__global__ void static_upload_kernel(const __grid_constant__ StaticChunk c, unsigned char* base) {
  unsigned* dst = reinterpret_cast<unsigned*>(base + c.off);
  for (unsigned w = blockIdx.x * blockDim.x + threadIdx.x; w < c.nbytes / 4; w += gridDim.x * blockDim.x)
    dst[w] = c.data[w];
}

// Work list of one call, expanded on the device: queue position t belongs to
// the q-th patch in queue order (CCZ4 patches first) when first[q] <= t <
// first[q + 1]; within a patch the 32x4x4 tiles run x fastest, then y, z.
struct StaticPlan {
  int np, nitems;
  int patch[kStaticMaxPatches];
  int first[kStaticMaxPatches + 1];
  int tiles_x[kStaticMaxPatches], tiles_y[kStaticMaxPatches];
};

__global__ void static_items_kernel(const __grid_constant__ StaticPlan plan, Item* items,
                                    unsigned int* counter) {
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 == 0) *counter = 0u;  // the queue starts at zero on every call
  for (int t = t0; t < plan.nitems; t += gridDim.x * blockDim.x) {
    int q = 0;
    while (q + 1 < plan.np && plan.first[q + 1] <= t) ++q;
    const int l = t - plan.first[q];
    const int tx = l % plan.tiles_x[q], r = l / plan.tiles_x[q];
    const int ty = r % plan.tiles_y[q], tz = r / plan.tiles_y[q];
    items[t] = Item{plan.patch[q], tx * kStaticTX, ty * kStaticTY, tz * kStaticTZ};
  }
}

std::mutex g_static_mu;                       // guards the per-device set-up
unsigned char* g_static_dev[64] = {nullptr};  // scratch address per device
int g_static_grid[64][3] = {{0}};

// Per-device set-up, done once with that device current: the device address
// of the scratch array and the persistent grid sizes.
sf_status static_setup(int dev) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (g_static_dev[dev]) return SF_OK;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return set_error(SF_ECUDA, "scratch address: %s", cudaGetErrorString(e));
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return set_error(SF_ECUDA, "SM count query failed");
  int occ[3] = {0, 0, 0};
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], batch_stage_kernel<double, double, false>, 128, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], batch_stage_kernel<float, double, false>, 128, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[2], batch_stage_kernel<float, dw, false>, 128, 0);
  for (int q = 0; q < 3; ++q) g_static_grid[dev][q] = std::max(1, sms * std::max(1, occ[q]));
  g_static_dev[dev] = static_cast<unsigned char*>(p);
  return SF_OK;
}

// Copy `n` bytes (a multiple of 4) of `src` to scratch offset `off`, one
// launch per chunk.
sf_status static_upload(unsigned char* d, size_t off, const void* src, size_t n, cudaStream_t st) {
  StaticChunk c;
  for (size_t done = 0; done < n; done += kChunkBytes) {
    const size_t len = std::min<size_t>(kChunkBytes, n - done);
    c.off = (unsigned)(off + done);
    c.nbytes = (unsigned)len;
    memcpy(c.data, static_cast<const unsigned char*>(src) + done, len);
    static_upload_kernel<<<(unsigned)((len / 4 + 255) / 256), 256, 0, st>>>(c, d);
    sf_status e = after_launch("static_upload_kernel");
    if (e) return e;
  }
  return SF_OK;
}

template <typename T, typename H>
sf_status static_stage(const sf_params& prm, const sf_patch* pin, int np, int stage, int dev,
                       cudaStream_t st) {
  unsigned char* d = g_static_dev[dev];
  PatchArgs<T> args[kStaticMaxPatches];
  // sys at [0, 256), shapes at [256, 768): the layout of [kOffSys, kOffItems)
  static_assert(kOffShape - kOffSys == kStaticMaxPatches * sizeof(int), "sys block");
  struct {
    int sys[kStaticMaxPatches];
    int2 shape[kStaticMaxPatches];
  } small;
  StaticPlan plan;
  plan.np = np;
  int nq = 0, nitems = 0;
  for (int pass = 0; pass < 2; ++pass)  // CCZ4 items first, as in sf_batch_substep
    for (int q = 0; q < np; ++q) {
      const sf_patch& p = pin[q];
      if ((pass == 0) != (p.system == SF_Z4)) continue;
      plan.patch[nq] = q;
      plan.first[nq] = nitems;
      plan.tiles_x[nq] = (p.n[0] + kStaticShape.tx - 1) / kStaticShape.tx;
      plan.tiles_y[nq] = (p.n[1] + kStaticShape.ty - 1) / kStaticShape.ty;
      nitems += plan.tiles_x[nq] * plan.tiles_y[nq] * ((p.n[2] + kStaticShape.tz - 1) / kStaticShape.tz);
      ++nq;
    }
  plan.first[nq] = nitems;
  plan.nitems = nitems;
  for (int q = 0; q < np; ++q) {
    sf_patch p = pin[q];
    void* A = p.u_n;
    void* us[4] = {A, p.u_stage, p.u_next, p.u_stage};
    void* nx[4] = {p.u_stage, p.u_next, p.u_stage, A};
    p.u_stage = us[stage];
    p.u_next = nx[stage];
    args[q] = make_args<T>(prm, p, stage, sf_nfields(p.system), nullptr);
    small.sys[q] = p.system;
    small.shape[q] = make_int2(kStaticShape.tx, kStaticShape.tz);
  }
  sf_status e = static_upload(d, kOffArgs, args, np * sizeof(PatchArgs<T>), st);
  if (!e) e = static_upload(d, kOffSys, small.sys, np * sizeof(int), st);
  if (!e) e = static_upload(d, kOffShape, small.shape, np * sizeof(int2), st);
  if (e) return e;
  unsigned int* tcounter = reinterpret_cast<unsigned int*>(d);
  Item* titems = reinterpret_cast<Item*>(d + kOffItems);
  static_items_kernel<<<(nitems + 255) / 256, 256, 0, st>>>(plan, titems, tcounter);
  e = after_launch("static_items_kernel");
  if (e) return e;
  sf_batch tmp;  // only carries the fields batch_stage_args reads
  tmp.prm = prm;
  tmp.precision = pin[0].precision;
  Z4Coef<T> zc;
  zc.kappa_z = T(prm.kappa_z);
  zc.kappa_c = T(prm.kappa_c);
  zc.eta = T(prm.eta);
  zc.g_shift = T(prm.g_shift);
  zc.slicing = prm.slicing;
  zc.shift_frozen = prm.shift_frozen;
  zc.lopsided = prm.lopsided;
  const StageArgs sa = batch_stage_args(&tmp, stage, status_ptr());
  const int grid = g_static_grid[dev][pin[0].precision];
  const PatchArgs<T>* targs = reinterpret_cast<const PatchArgs<T>*>(d + kOffArgs);
  const int* tsys = reinterpret_cast<const int*>(d + kOffSys);
  const int2* tshape = reinterpret_cast<const int2*>(d + kOffShape);
  if (prm.lopsided)
    batch_stage_kernel<T, H, true><<<grid, 128, 0, st>>>(targs, tsys, tshape, titems, nitems,
                                                         tcounter, sa, zc);
  else
    batch_stage_kernel<T, H, false><<<grid, 128, 0, st>>>(targs, tsys, tshape, titems, nitems,
                                                          tcounter, sa, zc);
  return after_launch("batch_stage_kernel (static scratch)");
}

}  // namespace

extern "C" sf_status sf_batch_substep_static(const sf_params* prm, const sf_patch* patches,
                                             int32_t npatch, int32_t stage, void* stream) {
  if (!prm || !patches) return set_error(SF_EINVAL, "NULL argument");
  if (npatch < 1 || npatch > kStaticMaxPatches)
    return set_error(SF_EINVAL, "npatch = %d outside [1, %d], the static scratch maximum", npatch,
                     kStaticMaxPatches);
  if (stage < 0 || stage > 3) return set_error(SF_EINVAL, "stage %d out of range [0,4)", stage);
  if (prm->rk != SF_RK4) return set_error(SF_ENOTSUP, "sf_batch_substep_static runs RK4");
  if (prm->ghosts != SF_GHOSTS_NONE && prm->ghosts != SF_GHOSTS_PERIODIC)
    return set_error(SF_EINVAL, "ghosts %d not SF_GHOSTS_NONE or SF_GHOSTS_PERIODIC", prm->ghosts);
  const sf_params q = *prm;
  sf_patch local[kStaticMaxPatches];
  long long items = 0;
  for (int i = 0; i < npatch; ++i) {
    sf_patch p = patches[i];
    normalise_strides(p, sf_nfields(p.system));
    if (p.system != SF_WAVE && p.system != SF_Z4)
      return set_error(SF_ENOTSUP, "sf_batch_substep_static takes SF_WAVE and SF_Z4 patches");
    if (p.precision != patches[0].precision)
      return set_error(SF_EINVAL, "all patches of a call need one precision");
    if (p.u_stage == p.u_next || p.u_stage == p.u_n || p.u_next == p.u_n)
      return set_error(SF_EINVAL, "patches need distinct u_n, u_stage and u_next buffers");
    void* us[4] = {p.u_n, p.u_stage, p.u_next, p.u_stage};
    void* nx[4] = {p.u_stage, p.u_next, p.u_stage, p.u_n};
    sf_patch r = p;
    r.u_stage = us[stage];
    r.u_next = nx[stage];
    sf_status e = check_patch(&q, r, 1, stage);
    if (e) return e;
    items += (long long)((p.n[0] + kStaticShape.tx - 1) / kStaticShape.tx) *
             ((p.n[1] + kStaticShape.ty - 1) / kStaticShape.ty) *
             ((p.n[2] + kStaticShape.tz - 1) / kStaticShape.tz);
    local[i] = p;
  }
  if (items > kStaticMaxItems)
    return set_error(SF_EINVAL,
                     "%lld work items of 32x4x4 points exceed the static scratch maximum of %d",
                     items, kStaticMaxItems);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return set_error(SF_ECUDA, "no usable CUDA device");
  if (!status_ptr()) return set_error(SF_ECUDA, "no status word");
  sf_status e = static_setup(dev);
  if (e) return e;
  cudaStream_t st = (cudaStream_t)stream;
  switch (local[0].precision) {
    case SF_FP64: return static_stage<double, double>(q, local, npatch, stage, dev, st);
    case SF_FP32_BULK_DW: return static_stage<float, dw>(q, local, npatch, stage, dev, st);
    default: return static_stage<float, double>(q, local, npatch, stage, dev, st);
  }
}
