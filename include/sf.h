/*
 * sf.h - C ABI of the GB300 method-of-lines substep library (libsf.so).
 *
 * The library advances ghosted grid patches by one Runge-Kutta substep of the
 * semi-discrete system dU/dt = L(U) + Q_d(U) (arXiv:1806.04182, Sec. II.A,
 * Eq. (2)), with
 *   - SF_WAVE: scalar wave equation in first-order form (phi, Pi, d_x, d_y, d_z)
 *     (Sec. IV.A), 4th-order centred derivatives (Sec. II.B.1),
 *   - SF_Z4:   CCZ4 with Bona-Masso slicing and Gamma-driver shift, vacuum,
 *     25 fields (Sec. V), 4th-order centred first, second and mixed
 *     derivatives (Sec. II.B.1),
 *   - SF_MHD:  ideal Newtonian MHD, 8 conserved fields (Sec. IV.B), WENO5
 *     reconstruction of the evolved fields (App. B) and local Lax-Friedrichs
 *     flux (Sec. II.B.2, Eq. LLF) in conservative form (Eq. 5),
 * and 6th-order Kreiss-Oliger dissipation Q_d on the wave and Z4 systems
 * (Sec. II.B.1).  Time integration: RK(4,4) (Sec. II.C, Table RK44) or
 * SSP-RK(3,3) (App. C/D), one call per stage.
 *
 * Memory: the caller owns every buffer (device memory for all pointers
 * unless stated).  The library keeps no pointer after a call returns, except
 * inside an sf_batch object, which records the patch table it was created
 * with.  Calls are asynchronous on the given CUDA stream (NULL = legacy
 * default stream) and return after enqueueing work.
 *
 * Errors: argument errors are reported synchronously as SF_EINVAL with a
 * message from sf_last_error() (thread-local) and nothing is enqueued.  CUDA
 * launch errors return SF_ECUDA.  Conditions found on the device (non-finite
 * values, work-queue time-outs) set a device status word that
 * sf_get_device_status() reads.  Nothing aborts, traps or throws across the
 * ABI.
 */
#ifndef SF_H
#define SF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SF_OK = 0,
  SF_EINVAL = 1,      /* bad argument; see sf_last_error() */
  SF_ENOTSUP = 2,     /* valid but unsupported combination */
  SF_ECUDA = 3,       /* a CUDA runtime call failed */
  SF_ENONFINITE = 4,  /* device found NaN/Inf in an output */
  SF_ETIMEOUT = 5     /* a bounded device wait gave up */
} sf_status;

typedef enum { SF_WAVE = 0, SF_MHD = 1, SF_Z4 = 2 } sf_system;

/* SF_FP64: storage and arithmetic in double.
 * SF_FP32_BULK: storage and stencil arithmetic in float; the Z4 conformal
 * metric determinant, inverse, ln det and the trace removals are evaluated
 * in double; the last RK4 stage adds the step increment to U^n with a
 * compensated (Kahan) sum carried across steps in the `kahan` array.
 * SF_FP32_BULK_DW: as SF_FP32_BULK, but the island quantities are evaluated
 * in double-word arithmetic (a float pair hi + lo built from error-free
 * transformations, relative error a few 2^-48) on the FP32 pipe instead of
 * the FP64 pipe, which on GB300 runs at ~1/58 of the FP32 rate.  The paper
 * has no counterpart; it is this library's way to keep FP64-class islands
 * cheap on this GPU.
 * In both FP32 modes the SF_Z4 arrays store chi, gt_xx, gt_yy, gt_zz and alpha
 * MINUS their flat-space value 1 (fields 0, 1, 4, 6 and 18), so that small
 * deviations from flat space (noise of 1e-10, say) survive float storage;
 * all other fields, and every field in SF_FP64, are stored as they are. */
typedef enum { SF_FP64 = 0, SF_FP32_BULK = 1, SF_FP32_BULK_DW = 2 } sf_precision;

typedef enum { SF_RK4 = 0, SF_SSPRK3 = 1 } sf_rk;

/* Ghost handling of the stage output. */
typedef enum {
  SF_GHOSTS_NONE = 0,     /* caller fills ghosts of u_next (e.g. from neighbours) */
  SF_GHOSTS_PERIODIC = 1  /* the substep also writes u_next's periodic ghost shell
                             (the patch is periodic onto itself; needs n >= ghost) */
} sf_ghosts;

/*
 * One ghosted box (Sec. III: a patch with a ghost zone of `ghost` points).
 * Every array of a patch has the same layout: nf fields, field f, interior
 * point (i,j,k) (0 <= i < n[0], ...) at element
 *     f*sf + (k+ghost)*sz + (j+ghost)*sy + (i+ghost)
 * with x fastest.  Elements are double (SF_FP64) or float (both FP32 modes).
 * Strides may be 0, meaning contiguous: sy = n[0]+2g, sz = sy*(n[1]+2g),
 * sf = sz*(n[2]+2g).
 *
 * Stage semantics, RK4 (k_j = dt (L+Q_d)(U(j)), r = (L+Q_d)(u_stage)):
 *   stage 0: u_stage = U^n (may alias u_n); acc = U^n + dt/6 r; u_next = U^n + dt/2 r
 *   stage 1: acc += dt/3 r;  u_next = U^n + dt/2 r
 *   stage 2: acc += dt/3 r;  u_next = U^n + dt r
 *   stage 3: u_next = acc + dt/6 r  (= U^{n+1})
 * In SF_FP32_BULK acc holds only the increment (acc = dt/6 r at stage 0) and
 * stage 3 forms U^{n+1} = U^n + (acc + dt/6 r) with Kahan compensation:
 * kahan is read and written in stage 3 and must start at zero.
 * SSP-RK3 (Shu-Osher form; acc unused):
 *   stage 0: u_next = U^n + dt r
 *   stage 1: u_next = 3/4 U^n + 1/4 (u_stage + dt r)
 *   stage 2: u_next = 1/3 U^n + 2/3 (u_stage + dt r)
 * u_next must not alias u_stage or acc; it may alias u_n in the last stage
 * only (each point reads its own U^n before overwriting it, and no stencil
 * reads U^n), which updates the state in place.  Only interior points of
 * u_next/acc/kahan are written (plus u_next's ghost shell under
 * SF_GHOSTS_PERIODIC).  u_stage must have valid ghosts.
 */
typedef struct {
  int32_t n[3];      /* interior points x, y, z (>= 1) */
  int32_t ghost;     /* ghost width, >= 3 */
  double dx[3];      /* grid spacing per direction (> 0) */
  double dt;         /* time step of this patch */
  int32_t system;    /* sf_system */
  int32_t precision; /* sf_precision */
  int64_t sy, sz, sf;/* element strides (0 = contiguous) */
  void* u_stage;     /* in:  stage input U(i) */
  void* u_n;         /* in:  U^n */
  void* acc;         /* in/out: RK4 accumulator (unused by SSP-RK3) */
  void* u_next;      /* out: next stage input, or U^{n+1} after the last stage */
  void* kahan;       /* in/out: FP32_BULK compensation (NULL otherwise) */
  double* cfl_rate;  /* SF_MHD only, optional (NULL = off): device double that the
                        LAST stage sets to max over interior points and directions
                        d of (|v_d| + c_fast,d)/dx_d of u_next (Sec. II.A footnote),
                        so the next step's dt = cfl / rate needs no extra sweep */
} sf_patch;

typedef struct {
  int32_t rk;           /* sf_rk */
  int32_t ghosts;       /* sf_ghosts */
  double sigma_ko;      /* KO strength sigma (Sec. II.B.1), >= 0 */
  double gamma_eos;     /* MHD adiabatic index (Sec. IV.B) */
  double weno_eps;      /* WENO epsilon; <= 0 means dx_d^4 (WENO5, App. B) or dx_d^2 (WENO3, App. A) */
  double weno_q;        /* WENO-Z exponent (App. B) */
  int32_t weno_variant; /* 0: WENO5-JS, 1: WENO5-Z, 2: WENO3 (App. A) */
  int32_t slicing;      /* 0: 1+log (f = 2/alpha), 1: harmonic (f = 1) (Sec. V) */
  int32_t shift_frozen; /* 1: d/dt beta = d/dt B = 0 */
  int32_t check_finite; /* 1: flag NaN/Inf written to u_next in the status word */
  double kappa_z;       /* Z4 damping kappa_z (Sec. V) */
  double kappa_c;       /* conformal-constraint damping kappa_c (Sec. V) */
  double eta;           /* Gamma-driver damping eta (Sec. V) */
  double g_shift;       /* Gamma-driver coefficient g (Sec. V) */
  int32_t lopsided;     /* SF_Z4: 1 = advection terms beta^k d_k with the 4th-order
                           one-sided stencils of Sec. II.B.1, chosen by the sign
                           of beta^k; 0 = centred D_k */
  int32_t flux_split;   /* SF_MHD: 0 = WENO reconstruction of the evolved fields at
                           each interface, then the LLF formula (Eq. LLF; the paper's
                           tests); 1 = reconstruction of the fluxes (Sec. II.B.2) in
                           Lax-Friedrichs splitting form: S = largest signal speed
                           over the interface's six-cell stencil, F+- = (F(U) +- S U)/2
                           at each cell, F+ reconstructed from the left plus F- from
                           the right */
} sf_params;

/* Number of evolved fields of a system (5, 8 or 25); -1 if unknown. */
int32_t sf_nfields(int32_t system);

/*
 * One RK stage on each of `npatch` patches (Sec. II.C; one launch per patch).
 * stage in [0,4) for RK4, [0,3) for SSP-RK3.  All patches must use the
 * same system and precision in this entry point (see sf_batch for mixed).
 */
sf_status sf_substep(const sf_params* prm, const sf_patch* patches, int32_t npatch,
                     int32_t stage, void* stream);

/*
 * The device arrays of one patch state, in the buffer roles of sf_batch: u
 * holds U^n and receives U^{n+1} from the last stage; s1 and s2 are stage
 * scratch; acc is the RK4 accumulator (NULL under SSP-RK3); kahan the
 * FP32-bulk compensation under RK4 (else NULL).  All share the layout
 * (strides) of the patch they belong to.
 */
typedef struct {
  void* u;
  void* s1;
  void* s2;
  void* acc;
  void* kahan;
} sf_state;

/* sf_step_host flag: zero the Kahan compensation of the slot at every upload. */
#define SF_HOST_RESET_KAHAN 1u
/* sf_step_host flag: host images are the interior only (sf_interior_span
 * elements, see there); needs periodic ghosts. */
#define SF_HOST_INTERIOR 2u

/* Elements of a state's interior host image: nf * n[0] * n[1] * n[2], dense,
 * field-major then z, y, x (x fastest), in the storage convention of the
 * stages.  -1 for an unknown system. */
int64_t sf_interior_span(const sf_patch* geom);

/*
 * Elements of a state's host image: from ghosted point (0,0,0) of field 0 to
 * the last ghosted point of field nf - 1 in the patch's strides,
 * (nf - 1) sf + (n2 + 2g - 1) sz + (n1 + 2g - 1) sy + n0 + 2g (row padding
 * in between included).  -1 for an unknown system.
 */
int64_t sf_state_span(const sf_patch* geom);

/*
 * RK steps of patch states held in host memory (Sec. II.C steps of the
 * fused substep; the paper's patches live in host memory under SAMRAI).
 * For k = 0 .. nsteps - 1: the host image host_in[k] (sf_state_span
 * elements, the patch's layout and the storage convention of the stages:
 * float CCZ4 fields chi, gt_ii, alpha minus 1) is copied to slot
 * slots[k % nslots].u on h2d_stream, one full RK step of prm->rk runs on
 * compute_stream (the stages of sf_substep, buffer roles u -> s1 -> s2 -> s1
 * -> u for RK4, u -> s1 -> s2 -> u for SSP-RK3), and U^{n+1} is copied from
 * slot.u to host_out[k] on d2h_stream.
 *   geom: n, ghost, dx, strides, dt, system, precision of every step (its
 *         pointer fields are ignored); nslots: 1 to 4 device states.
 *   Ordering: with two or more slots the uploads of later steps and the
 *   downloads of earlier ones overlap the stages of step k.  An upload waits
 *   for the download of the step that last used its slot and, when host_in[k]
 *   overlaps the host_out of a step still in flight, for that download, so
 *   an evolution kept in host memory (host_in[k] = host_out[k - 1]) is
 *   correct with any slot count.  Copies go in eight pieces of the image,
 *   and an upload piece waits only for the download pieces it overlaps, so
 *   in such an evolution the next upload runs beside the rest of the
 *   download.  With two slots the upload of step k + 1
 *   waits for the download of step k - 1; with three it does not, so
 *   independent steps run at the rate of the stages when the copies are
 *   shorter.  The first upload of a call waits for the work already queued on
 *   compute_stream and d2h_stream (earlier calls).
 *   Kahan compensation: with SF_HOST_RESET_KAHAN it restarts from zero at
 *   every upload (independent states); without it the slot's compensation
 *   carries over, which continues an evolution exactly when each slot is
 *   handed back the state it produced (one slot, chained buffers).
 *   With SF_HOST_INTERIOR the host images hold the interior only (no ghost
 *   shell, no row padding: 18% fewer bytes over the host link at 96^3); the
 *   upload lands in the slot's s2 array and a kernel spreads it into u with
 *   its periodic ghost shell, and the last stage's interior is gathered into
 *   s2 for the download.  It needs prm->ghosts == SF_GHOSTS_PERIODIC.
 *   Host buffers should be pinned (page-locked) for the copies to overlap;
 *   host_out[k] holds U^{n+1} once d2h_stream has passed the call's work.
 *   NULL h2d_stream or d2h_stream means compute_stream.
 * Asynchronous.  Errors (SF_EINVAL, nothing enqueued): NULL arguments,
 * nslots not in 1..4, unknown flags, SF_HOST_INTERIOR without periodic
 * ghosts, a slot the stages would reject.
 */
sf_status sf_step_host(const sf_params* prm, const sf_patch* geom, const sf_state* slots,
                       int32_t nslots, const void* const* host_in, void* const* host_out,
                       int32_t nsteps, uint32_t flags, void* compute_stream, void* h2d_stream,
                       void* d2h_stream);

/*
 * Right-hand side only: rhs_out[f][k][j][i] = (L + Q_d)(u_stage) on the
 * interior, an unghosted contiguous array of nf * n[0]*n[1]*n[2] elements of
 * the patch's precision.  For tests and diagnostics.
 */
sf_status sf_rhs(const sf_params* prm, const sf_patch* patch, void* rhs_out, void* stream);

/*
 * Periodic ghost fill of `array` (layout of `patch`, `nf` fields): every ghost
 * point takes the value of the interior point congruent to it modulo n
 * (the periodic boundary of Sec. IV tests).  Works for any n >= 1.
 */
sf_status sf_fill_ghosts_periodic(const sf_patch* patch, void* array, int32_t nf, void* stream);

/*
 * MHD CFL rate (Sec. II.A footnote): *d_rate = max over interior points and
 * directions d of (|v_d| + c_fast,d) / dx_d of `array` (layout of `patch`,
 * FP64 or FP32 per patch).  d_rate is one device double; dt = cfl / rate.
 */
sf_status sf_mhd_max_rate(const sf_params* prm, const sf_patch* patch, const void* array,
                          double* d_rate, void* stream);

/*
 * Adjoint RK stage of the wave system: same stage semantics as sf_substep
 * with L replaced by its transpose L^T on the periodic grid (D_i^T = -D_i,
 * Q_d^T = Q_d), acting on adjoint fields (l_phi, l_Pi, l_d).  Because the
 * wave operator is linear and autonomous, four such stages apply
 * P(dt L)^T = P(dt L^T), the exact transpose of one forward RK4 step.
 */
sf_status sf_adjoint_substep(const sf_params* prm, const sf_patch* adj, int32_t npatch,
                             int32_t stage, void* stream);

/*
 * out[o] = array[field][obs[o]] for nobs interior linear indices
 * obs[o] = (k*n[1] + j)*n[0] + i (device int64 array); out is a device
 * array of the patch's precision.  sf_scatter_add does array[field][obs[o]] += vals[o]
 * (observer indices must be distinct).
 */
sf_status sf_gather(const sf_patch* patch, const void* array, int32_t field, const int64_t* obs,
                    int32_t nobs, void* out, void* stream);
sf_status sf_scatter_add(const sf_patch* patch, void* array, int32_t field, const int64_t* obs,
                         int32_t nobs, const void* vals, void* stream);

/*
 * FP64 diagnostics of `array` (interior), written to device doubles d_out:
 *   SF_WAVE: d_out[0] = 1/2 sum (Pi^2 + |d|^2) dx dy dz (wave energy)
 *   SF_Z4:   d_out[0..3] = sums over points of Theta^2, |Z|^2, (ln det gt)^2,
 *            (tr A~)^2, with Z^i = chi/2 (Gammahat^i - Gamma~^i) (Sec. V)
 *   all:     d_out[4] = number of non-finite values (as a double)
 * d_out must hold 5 doubles.
 */
sf_status sf_diagnostics(const sf_params* prm, const sf_patch* patch, const void* array,
                         double* d_out, void* stream);

/*
 * Radiative (outgoing-wave) boundary condition of Sec. V: one RK stage at
 * every ghost point of a non-periodic patch, with the right-hand side
 *   dU/dt = -speed[f] ( x^i/r d_i U + (U - u_inf[f]) / r ),
 * x = x0 + (i, j, k) dx the physical position of the point (x0 = position of
 * interior point (0,0,0)), r = |x|, and d_i the centred 4th-order stencil
 * where the ghosted array holds two points on both sides, else the 4th-order
 * one-sided stencil leaning into the array.  The stage combination and the
 * array roles are those of sf_substep, which advances the interior of the
 * same patch for the same stage (with prm->ghosts = SF_GHOSTS_NONE, so that
 * it leaves the ghost shell to this call; both only read u_stage).  u_inf
 * and speed hold one value per field (u_inf in field values: the flat-space
 * offsets of float CCZ4 storage are applied here).  SF_EINVAL if
 * prm->ghosts is not SF_GHOSTS_NONE, for non-finite x0 or u_inf, negative
 * speeds, or any argument sf_substep rejects.
 */
sf_status sf_radiative_substep(const sf_params* prm, const sf_patch* patch, const double* x0,
                               const double* u_inf, const double* speed, int32_t stage,
                               void* stream);

/*
 * Box copies between patch arrays, for the AMR level loop (Sec. III): same-
 * level ghost synchronisation between neighbouring patches, and, with
 * src_step = R, restriction by injection (Sec. III.A: coarse point i takes
 * the fine value at fine point R i).  Box point (x, y, z) of field f is read
 * at  src_off + f*src_sf + R*(z*src_sz + y*src_sy + x)  and written at
 *      dst_off + f*dst_sf + z*dst_sz + y*dst_sy + x  (element offsets; the
 * element type follows `precision`).  The caller guarantees both ranges lie
 * inside its arrays and that destination boxes do not overlap sources or each
 * other.  One launch per 256 boxes; nothing is allocated.  Each box holds fewer
 * than 2^31 values.
 */
typedef struct {
  const void* src;
  void* dst;
  int64_t src_off, src_sy, src_sz, src_sf;
  int64_t dst_off, dst_sy, dst_sz, dst_sf;
  int32_t ext[3];    /* box extent x, y, z (>= 0) */
  int32_t nf;        /* fields (>= 1) */
  int32_t src_step;  /* 1: copy; R: injection from a level R times finer */
  int32_t reserved;  /* set to 0 */
} sf_box_copy;

sf_status sf_copy_boxes(const sf_box_copy* boxes, int32_t nbox, int32_t precision, void* stream);

/*
 * Prolongation (Sec. III.A): 6-point (5th-order) Lagrange interpolation of
 * `coarse_array` (layout of `coarse`, nf fields, ghost-filled) onto the fine
 * points origin .. origin+ext-1 of a level `ratio` times finer, where fine
 * index R i coincides with coarse interior point i.  In each direction the
 * nodes are the coarse points floor(F/R)-2 .. floor(F/R)+3 and the weights
 * are the Lagrange basis l_j at the fractional position (F mod R)/R; 3D is
 * the tensor product.  Coincident points reduce to injection.  The result
 * goes to fine_out with element strides (out_sy, out_sz, out_sf), for example
 * straight into a fine patch's ghost zone.  SF_EINVAL if a stencil node falls
 * outside the ghosted coarse box.  ratio in [1, 8].
 */
sf_status sf_prolong(const sf_patch* coarse, const void* coarse_array, int32_t nf, int32_t ratio,
                     const int32_t* origin, const int32_t* ext, void* fine_out, int64_t out_sy,
                     int64_t out_sz, int64_t out_sf, void* stream);

/*
 * Sub-cycling in time by Berger-Oliger without order reduction (Sec. III.B;
 * dense output App. C; BOR App. D), fused with the prolongation above: the
 * fine-grid value needed at fine points origin .. origin+ext-1 for fine step
 * r (0 <= r < ratio) of the `ratio` fine steps (dt_F = dt / ratio) inside
 * one coarse step.
 *   rk = SF_RK4:    states[0..4] = coarse U^n, U^(2) = U^n + k_1/2,
 *                   U^(3) = U^n + k_2/2, U^(4) = U^n + k_3, U^{n+1};
 *   rk = SF_SSPRK3: states[0..3] = coarse U^n, U^(2) = U^n + k_1,
 *                   U^(3) = U^n + (k_1 + k_2)/4, U^{n+1}
 * (the stage inputs the coarse substeps produce, each ghost-filled, layout
 * of `coarse`).  The coarse increments k_j follow from them exactly; the
 * value is that of App. D: the dense output at theta = r/ratio, its time
 * derivatives, the fine increments with dt_F, and the fine RK formula:
 *   stage = 0 .. s-1  ->  fine stage input U^(stage+1) of fine step r,
 *   stage = s         ->  U^{n+(r+1)/ratio},
 * with s = 4 (RK4) or 3 (SSP-RK3).  The result is then prolonged in space as
 * sf_prolong does (ratio 1: a copy) and written to fine_out.  Values are
 * formed in the arrays' element type (float arrays: float arithmetic, which
 * holds their accuracy since every weight set sums to one).
 * SF_EINVAL for a NULL or misaligned state, stage or r out of range, or a
 * stencil node outside the ghosted coarse box.
 */
sf_status sf_bor_prolong(const sf_patch* coarse, int32_t rk, const void* const* states, int32_t nf,
                         int32_t ratio, int32_t r, int32_t stage, const int32_t* origin,
                         const int32_t* ext, void* fine_out, int64_t out_sy, int64_t out_sz,
                         int64_t out_sf, void* stream);

/*
 * sf_bor_prolong for several output boxes at once (for example the six slabs
 * of a fine patch's ghost shell): one launch per 16 boxes.  Each box names its
 * fine points (origin, ext, as in sf_bor_prolong) and its output (pointer and
 * element strides).  Every box is validated before anything is launched;
 * boxes with a zero extent write nothing and may have a NULL output.
 */
typedef struct {
  int32_t origin[3];
  int32_t ext[3];
  void* out;
  int64_t out_sy, out_sz, out_sf;
} sf_prolong_box;

sf_status sf_bor_prolong_boxes(const sf_patch* coarse, int32_t rk, const void* const* states,
                               int32_t nf, int32_t ratio, int32_t r, int32_t stage,
                               const sf_prolong_box* boxes, int32_t nbox, void* stream);

/*
 * Batched AMR-patch dispatch (the level loop of Sec. III over many patches):
 * one persistent launch per stage over a table of patches of mixed systems
 * (SF_WAVE and SF_Z4) and sizes, each with its own dx and dt.  CTAs take
 * (patch, tile) work items from a device queue.  Float CCZ4 patches with
 * centred advection whose row, plane and field pitches are multiples of 4
 * floats and whose arrays are 16-byte aligned go instead to the TMA-staged
 * stage kernel: one launch per stage for each tile width in use (32 x 12 or
 * 16 x 24 points; each patch takes the width that covers it with fewer
 * tiles), ahead of the persistent launch for the other patches.
 * prm->ghosts applies to every patch: SF_GHOSTS_PERIODIC, each patch
 * periodic on its own (the stages write its periodic ghost shell), or
 * SF_GHOSTS_NONE, ghosts left to sf_batch_set_halo or the caller.
 * sf_batch_create copies the patch table (and the TMA patches' tensor maps
 * and tile lists) to the device (allocates; not in the hot path).
 * sf_batch_tune times the tile shapes of the persistent kernel for each
 * (system, size class) on `stream` and keeps the fastest, then, for each size
 * class with TMA patches, both TMA tile widths (that class's tiles alone) and
 * keeps the faster; it runs stage 1, which writes scratch roles only (the
 * u_next role and the accumulator), never U^n.  sf_batch_capture
 * records the RK stages of one full step into a CUDA graph; sf_batch_launch
 * replays it.
 */
typedef struct sf_batch sf_batch;
sf_status sf_batch_create(const sf_params* prm, const sf_patch* patches, int32_t npatch,
                          sf_batch** out);
sf_status sf_batch_substep(sf_batch* b, int32_t stage, void* stream);
sf_status sf_batch_tune(sf_batch* b, void* stream);
sf_status sf_batch_capture(sf_batch* b, void* stream);
sf_status sf_batch_launch(sf_batch* b, void* stream);
/*
 * Patches that tile a level (Sec. III: the patches of one level exchange
 * ghost zones, "level synchronisation"), created with ghosts =
 * SF_GHOSTS_NONE: sf_batch_set_halo gives, for buffer role `role` (0: the
 * u_n arrays, 1: u_stage, 2: u_next, as passed to sf_batch_create), the box
 * copies that fill every patch's ghost shell from its neighbours' interiors
 * (sf_box_copy semantics).  Each stage then ends with the copies of the role
 * it wrote (stage 0: u_stage, 1: u_next, 2: u_stage, 3: u_n), launched by
 * sf_batch_substep on its stream and recorded by sf_batch_capture.  The list
 * is copied (nbox = 0 clears it); the caller keeps the arrays alive.  Setting
 * a list drops a captured graph (capture again).  Errors: SF_EINVAL for a
 * NULL batch, a role outside 0..2, or a box sf_copy_boxes would reject.
 */
sf_status sf_batch_set_halo(sf_batch* b, int32_t role, const sf_box_copy* boxes, int32_t nbox);
/* Number of kernel launches (TMA tile launches, persistent launches and halo
 * box-copy launches) made by one sf_batch_launch, i.e. one RK4 step. */
int32_t sf_batch_launches_per_step(const sf_batch* b);
/* The batch's tile choices per size class c (0: wave, max n <= 32; 1: wave,
 * larger; 2: CCZ4, max n <= 32; 3: CCZ4, larger): shape_of_class[3c .. 3c+2]
 * the persistent kernel's tile (x, y, z extents), tma_width_of_class[c] the
 * TMA tile width (32: 32 x 12 points, 16: 16 x 24; -1 each patch of the class
 * takes the width that covers it with fewer tiles, as before sf_batch_tune;
 * 0 no TMA patch in the class).  Either array may be NULL (else 12 and 4
 * entries).  Errors: SF_EINVAL for a NULL batch. */
sf_status sf_batch_tuned(const sf_batch* b, int32_t* shape_of_class, int32_t* tma_width_of_class);
sf_status sf_batch_destroy(sf_batch* b);

/*
 * Allocation-free form of sf_batch_substep (the paper has no counterpart).
 * For callers that cannot call cudaMalloc when they advance their patches:
 * codes that give all device memory to their own pool or arena up front, and
 * codes that must not allocate while other work is in flight (cudaMalloc may
 * synchronise the device; cudaFree always does).  One RK4 stage of the
 * batched persistent kernel over `patches` (same buffer roles as sf_batch:
 * u_n = state, u_stage and u_next = scratch, acc, kahan), with the kernel's
 * scratch (queue counter, per-patch stage table, work list) kept in a
 * file-scope device array of 170,496 bytes that every GPU loading the
 * library holds until the process exits.  The call allocates nothing: on
 * `stream`, ahead of the persistent launch, small kernels whose parameters
 * carry this call's stage table write it into that array, expand the work
 * list and reset the queue counter (the call keeps no host buffer and reads
 * no host memory after it returns).
 * prm->ghosts: SF_GHOSTS_PERIODIC writes the periodic ghost shell of every
 * output (as sf_substep does), SF_GHOSTS_NONE leaves ghost shells to the
 * caller (patches that tile a level); any other value returns SF_EINVAL.
 * Limits: at most 64 patches and 8192 work items of 32x4x4 points per call;
 * larger requests return SF_EINVAL and enqueue nothing.
 * The first call on a device looks up the scratch address and the grid size
 * (with that device current); make that first call before any stream
 * capture.  All calls share the one scratch array, which keeps the last
 * call's contents: calls that overlap on the GPU (different streams, or
 * other host threads' streams) race; issue them in order on one stream.
 */
sf_status sf_batch_substep_static(const sf_params* prm, const sf_patch* patches, int32_t npatch,
                                  int32_t stage, void* stream);

/*
 * Self-test of failure detection (the paper has no counterpart).  Launches
 * one warp that waits, through the bounded mbarrier wait of the TMA-staged
 * stage kernels, on a barrier that nothing ever completes; after
 * `limit_cycles` SM clock cycles (1 .. 2e9, about a second at most) the wait
 * gives up and the kernel sets the time-out bit of the status word, which the
 * next sf_get_device_status() returns as SF_ETIMEOUT.  Nothing faults, traps
 * or hangs; the context stays usable.  Asynchronous on `stream`; a limit out
 * of range returns SF_EINVAL and enqueues nothing.
 */
sf_status sf_selftest_wait_timeout(int64_t limit_cycles, void* stream);

/*
 * Synchronises `stream`, returns and clears the device status word:
 * SF_OK, SF_ENONFINITE or SF_ETIMEOUT.
 */
sf_status sf_get_device_status(void* stream);

/* Message for the last failing call on this host thread ("" if none). */
const char* sf_last_error(void);

/* Count of kernel launches enqueued by this library since load (all threads). */
int64_t sf_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* SF_H */
