// Internal declarations shared by the translation units of libsf.so.
#pragma once

#include "sf_common.cuh"

namespace sf {

// thread-local error message + launch bookkeeping (sf_api.cu)
sf_status set_error(sf_status code, const char* fmt, ...);
sf_status after_launch(const char* what);
// device address of the status word on the current device (nullptr if none)
unsigned int* status_ptr();

// per-system stage launchers; rhs_out != nullptr selects "RHS only" output
sf_status launch_wave(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                      void* rhs_out, bool adjoint, cudaStream_t st);
sf_status launch_z4(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                    void* rhs_out, cudaStream_t st);
// TMA-staged CCZ4 kernel (sf_z4_tma.cu) and the layouts it serves
bool z4_tma_eligible(const sf_params& prm, const sf_patch& p);      // padded 96^3, compile-time strides
bool z4_tma_any_eligible(const sf_params& prm, const sf_patch& p);  // any size, 16-byte pitches
sf_status launch_z4_tma(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                        void* rhs_out, cudaStream_t st);
// Two-point (f32x2) TMA-staged CCZ4 kernel (sf_z4_pair.cu): padded 96^3-class
// layout with a one-float row offset
bool z4_pair_eligible(const sf_params& prm, const sf_patch& p, const void* rhs_out);
sf_status launch_z4_pair(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                         void* rhs_out, cudaStream_t st);
// the same tile body for any patch size on that layout (runtime strides,
// overhanging tiles; double-word islands, RK4 Kahan stage forms)
bool z4_pair_any_eligible(const sf_params& prm, const sf_patch& p, const StageArgs& s,
                          const void* rhs_out);
sf_status launch_z4_pair_any(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                             cudaStream_t st);
// TMA-staged CCZ4 kernel over the tiles of many patches (sf_z4_tma.cu), for
// sf_batch: 32 x 12 x 1 or 16 x 24 x 1 tiles (a patch's maps are encoded for
// its tile width), tensor maps in device memory (3 per patch: u_n, u_stage,
// u_next roles), the stage's u_stage role picked by `role`.
struct TmaTile {
  int patch, x0, y0, z0;
};
constexpr int kTmaTileX = 32, kTmaTileY = 12;      // the wide tile
constexpr int kTmaTileX16 = 16, kTmaTileY16 = 24;  // the narrow tile
constexpr size_t kTmaMapBytes = 128;  // sizeof(CUtensorMap)
bool z4_tma_batch_eligible(const sf_params& prm, const sf_patch& p);
// Two-point tiles of many patches (sf_z4_pair.cu), 32 x 16 x 1, for float
// CCZ4 batch patches with double-word islands on the one-float row offset
// layout: six tensor maps per patch (RK chunks of u_n, acc, kahan; stencil
// boxes of the u_n, u_stage, u_next roles) and the patch's stencil weights
// (z4_pair_coef_bytes each) in device memory.
constexpr int kPairTileX = 32, kPairTileY = 16;
bool z4_pair_batch_eligible(const sf_params& prm, const sf_patch& p);
size_t z4_pair_coef_bytes();
sf_status encode_z4_pair_batch(void* maps6, void* coef, const sf_params& prm, const sf_patch& p);
sf_status launch_z4_pair_batch(const sf_params& prm, const void* d_maps, int role,
                               const PatchArgs<float>* d_args, const void* d_coefs,
                               const TmaTile* d_tiles, int ntiles, const StageArgs& s,
                               cudaStream_t st);
sf_status encode_z4_tma_map(void* map, const sf_patch& p, const void* base, int xp);
sf_status launch_z4_tma_batch(const sf_params& prm, int precision, const void* d_maps, int role,
                              const PatchArgs<float>* d_args, const TmaTile* d_tiles, int ntiles,
                              int xp, const StageArgs& s, cudaStream_t st);
// box copies (sf_amr.cu): the host checks of sf_copy_boxes, and the number of
// launches it makes for a list
sf_status check_box_copies(const sf_box_copy* boxes, int nbox, int precision);
int box_copy_launches(const sf_box_copy* boxes, int nbox);
// radiative boundary stage on the ghost shell (sf_radiative.cu)
sf_status launch_radiative(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                           const double* x0, const double* u_inf, const double* speed,
                           cudaStream_t st);
sf_status launch_mhd(const sf_params& prm, const sf_patch& p, const StageArgs& s, int stage,
                     void* rhs_out, cudaStream_t st);

// argument validation shared by the entry points (sf_api.cu)
sf_status check_patch(const sf_params* prm, const sf_patch& p, int need_stage_arrays, int stage);
void normalise_strides(sf_patch& p, int nf);

}  // namespace sf
