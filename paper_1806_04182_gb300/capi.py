"""ctypes binding of libsf.so with the names and arguments of include/sf.h.

Argument marshalling only: every step of the substep runs in the CUDA
kernels of the library.  Pointers are raw device addresses (for example
``tensor.data_ptr()``) and streams are raw ``cudaStream_t`` handles (for
example ``torch.cuda.current_stream().cuda_stream``).  A non-OK status
raises :class:`SfError` carrying ``sf_last_error()``.  There is no CPU
fallback: if the library is not built, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

SF_OK, SF_EINVAL, SF_ENOTSUP, SF_ECUDA, SF_ENONFINITE, SF_ETIMEOUT = range(6)
SF_WAVE, SF_MHD, SF_Z4 = 0, 1, 2
SF_FP64, SF_FP32_BULK, SF_FP32_BULK_DW = 0, 1, 2
SF_RK4, SF_SSPRK3 = 0, 1
SF_GHOSTS_NONE, SF_GHOSTS_PERIODIC = 0, 1
STATUS_NAMES = {0: "SF_OK", 1: "SF_EINVAL", 2: "SF_ENOTSUP", 3: "SF_ECUDA", 4: "SF_ENONFINITE",
                5: "SF_ETIMEOUT"}

EXPORTS = ["sf_nfields", "sf_substep", "sf_rhs", "sf_fill_ghosts_periodic", "sf_mhd_max_rate",
           "sf_adjoint_substep", "sf_gather", "sf_scatter_add", "sf_diagnostics",
           "sf_batch_create", "sf_batch_substep", "sf_batch_tune", "sf_batch_capture",
           "sf_batch_launch", "sf_batch_launches_per_step", "sf_batch_destroy",
           "sf_batch_set_halo", "sf_batch_substep_static", "sf_copy_boxes", "sf_prolong", "sf_bor_prolong", "sf_bor_prolong_boxes", "sf_radiative_substep",
           "sf_selftest_wait_timeout", "sf_get_device_status", "sf_last_error", "sf_launch_count",
           "sf_state_span", "sf_step_host", "sf_batch_tuned", "sf_interior_span"]
SF_HOST_RESET_KAHAN = 1
SF_HOST_INTERIOR = 2


class SfError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class sf_params(ctypes.Structure):
    _fields_ = [
        ("rk", ctypes.c_int32),
        ("ghosts", ctypes.c_int32),
        ("sigma_ko", ctypes.c_double),
        ("gamma_eos", ctypes.c_double),
        ("weno_eps", ctypes.c_double),
        ("weno_q", ctypes.c_double),
        ("weno_variant", ctypes.c_int32),
        ("slicing", ctypes.c_int32),
        ("shift_frozen", ctypes.c_int32),
        ("check_finite", ctypes.c_int32),
        ("kappa_z", ctypes.c_double),
        ("kappa_c", ctypes.c_double),
        ("eta", ctypes.c_double),
        ("g_shift", ctypes.c_double),
        ("lopsided", ctypes.c_int32),
        ("flux_split", ctypes.c_int32),
    ]


class sf_prolong_box(ctypes.Structure):
    _fields_ = [
        ("origin", ctypes.c_int32 * 3),
        ("ext", ctypes.c_int32 * 3),
        ("out", ctypes.c_void_p),
        ("out_sy", ctypes.c_int64),
        ("out_sz", ctypes.c_int64),
        ("out_sf", ctypes.c_int64),
    ]


class sf_patch(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3),
        ("ghost", ctypes.c_int32),
        ("dx", ctypes.c_double * 3),
        ("dt", ctypes.c_double),
        ("system", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("sy", ctypes.c_int64),
        ("sz", ctypes.c_int64),
        ("sf", ctypes.c_int64),
        ("u_stage", ctypes.c_void_p),
        ("u_n", ctypes.c_void_p),
        ("acc", ctypes.c_void_p),
        ("u_next", ctypes.c_void_p),
        ("kahan", ctypes.c_void_p),
        ("cfl_rate", ctypes.c_void_p),
    ]


class sf_state(ctypes.Structure):
    _fields_ = [
        ("u", ctypes.c_void_p),
        ("s1", ctypes.c_void_p),
        ("s2", ctypes.c_void_p),
        ("acc", ctypes.c_void_p),
        ("kahan", ctypes.c_void_p),
    ]


class sf_box_copy(ctypes.Structure):
    _fields_ = [
        ("src", ctypes.c_void_p),
        ("dst", ctypes.c_void_p),
        ("src_off", ctypes.c_int64), ("src_sy", ctypes.c_int64), ("src_sz", ctypes.c_int64),
        ("src_sf", ctypes.c_int64),
        ("dst_off", ctypes.c_int64), ("dst_sy", ctypes.c_int64), ("dst_sz", ctypes.c_int64),
        ("dst_sf", ctypes.c_int64),
        ("ext", ctypes.c_int32 * 3),
        ("nf", ctypes.c_int32),
        ("src_step", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


def params(**kw) -> sf_params:
    """Defaults: RK4, periodic ghosts written by the substep, sigma = 0.1,
    Gamma = 5/3, eps = dx^4, WENO5-JS, kappa_z = kappa_c = 1, eta = 2,
    g = 3/4, 1+log slicing (Sec. V with M = 1)."""
    d = dict(rk=SF_RK4, ghosts=SF_GHOSTS_PERIODIC, sigma_ko=0.1, gamma_eos=5.0 / 3.0,
             weno_eps=0.0, weno_q=2.0, weno_variant=0, slicing=0, shift_frozen=0,
             check_finite=0, kappa_z=1.0, kappa_c=1.0, eta=2.0, g_shift=0.75, lopsided=0,
             flux_split=0)
    d.update(kw)
    return sf_params(**d)


_lib = None


def lib() -> ctypes.CDLL:
    """Load libsf.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1806_04182_gb300.build.build()")
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.sf_nfields.argtypes = [i32]
        L.sf_nfields.restype = i32
        L.sf_substep.argtypes = [P(sf_params), P(sf_patch), i32, i32, vp]
        L.sf_rhs.argtypes = [P(sf_params), P(sf_patch), vp, vp]
        L.sf_fill_ghosts_periodic.argtypes = [P(sf_patch), vp, i32, vp]
        L.sf_mhd_max_rate.argtypes = [P(sf_params), P(sf_patch), vp, vp, vp]
        L.sf_adjoint_substep.argtypes = [P(sf_params), P(sf_patch), i32, i32, vp]
        L.sf_gather.argtypes = [P(sf_patch), vp, i32, vp, i32, vp, vp]
        L.sf_scatter_add.argtypes = [P(sf_patch), vp, i32, vp, i32, vp, vp]
        L.sf_diagnostics.argtypes = [P(sf_params), P(sf_patch), vp, vp, vp]
        L.sf_batch_create.argtypes = [P(sf_params), P(sf_patch), i32, P(vp)]
        L.sf_batch_substep.argtypes = [vp, i32, vp]
        L.sf_batch_tune.argtypes = [vp, vp]
        L.sf_batch_capture.argtypes = [vp, vp]
        L.sf_batch_launch.argtypes = [vp, vp]
        L.sf_batch_launches_per_step.argtypes = [vp]
        L.sf_batch_launches_per_step.restype = i32
        L.sf_batch_destroy.argtypes = [vp]
        L.sf_batch_substep_static.argtypes = [P(sf_params), P(sf_patch), i32, i32, vp]
        L.sf_copy_boxes.argtypes = [P(sf_box_copy), i32, i32, vp]
        L.sf_batch_set_halo.argtypes = [vp, i32, P(sf_box_copy), i32]
        L.sf_prolong.argtypes = [P(sf_patch), vp, i32, i32, P(i32), P(i32), vp, i64, i64, i64, vp]
        L.sf_bor_prolong_boxes.argtypes = [P(sf_patch), i32, P(vp), i32, i32, i32, i32,
                                           P(sf_prolong_box), i32, vp]
        L.sf_radiative_substep.argtypes = [P(sf_params), P(sf_patch), P(ctypes.c_double),
                                           P(ctypes.c_double), P(ctypes.c_double), i32, vp]
        L.sf_bor_prolong.argtypes = [P(sf_patch), i32, P(vp), i32, i32, i32, i32, P(i32), P(i32), vp,
                                     i64, i64, i64, vp]
        L.sf_state_span.argtypes = [P(sf_patch)]
        L.sf_state_span.restype = i64
        L.sf_interior_span.argtypes = [P(sf_patch)]
        L.sf_interior_span.restype = i64
        L.sf_step_host.argtypes = [P(sf_params), P(sf_patch), P(sf_state), i32, P(vp), P(vp), i32,
                                   ctypes.c_uint32, vp, vp, vp]
        L.sf_batch_tuned.argtypes = [vp, P(i32), P(i32)]
        L.sf_get_device_status.argtypes = [vp]
        L.sf_selftest_wait_timeout.argtypes = [i64, vp]
        L.sf_last_error.argtypes = []
        L.sf_last_error.restype = ctypes.c_char_p
        L.sf_launch_count.argtypes = []
        L.sf_launch_count.restype = i64
        for name in ("sf_substep", "sf_rhs", "sf_fill_ghosts_periodic", "sf_mhd_max_rate",
                     "sf_adjoint_substep", "sf_gather", "sf_scatter_add", "sf_diagnostics",
                     "sf_batch_create", "sf_batch_substep", "sf_batch_tune", "sf_batch_capture",
                     "sf_batch_launch", "sf_batch_destroy", "sf_get_device_status",
                     "sf_batch_substep_static", "sf_copy_boxes", "sf_prolong",
                     "sf_batch_set_halo", "sf_selftest_wait_timeout", "sf_step_host",
                     "sf_batch_tuned"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status: int, where: str) -> None:
    if status != SF_OK:
        raise SfError(status, where, lib().sf_last_error().decode(errors="replace"))


def _patches(patches):
    if isinstance(patches, sf_patch):
        patches = [patches]
    arr = (sf_patch * len(patches))(*patches)
    return arr, len(patches)


def sf_interior_span(geom: sf_patch) -> int:
    return int(lib().sf_interior_span(ctypes.byref(geom)))


def sf_state_span(geom: sf_patch) -> int:
    return lib().sf_state_span(ctypes.byref(geom))


def sf_step_host(prm: sf_params, geom: sf_patch, slots, host_in, host_out, flags: int = 0,
                 compute_stream: int = 0, h2d_stream: int = 0, d2h_stream: int = 0) -> None:
    """slots: one or two sf_state; host_in / host_out: host addresses, one per step."""
    if isinstance(slots, sf_state):
        slots = [slots]
    sl = (sf_state * len(slots))(*slots)
    n = len(host_in)
    if len(host_out) != n:
        raise ValueError("host_in and host_out need one buffer per step")
    hin = (ctypes.c_void_p * max(n, 1))(*host_in)
    hout = (ctypes.c_void_p * max(n, 1))(*host_out)
    _check(lib().sf_step_host(ctypes.byref(prm), ctypes.byref(geom), sl, len(slots), hin, hout, n,
                              flags, compute_stream, h2d_stream, d2h_stream), "sf_step_host")


def sf_nfields(system: int) -> int:
    return lib().sf_nfields(system)


def sf_substep(prm: sf_params, patches, stage: int, stream: int = 0) -> None:
    arr, n = _patches(patches)
    _check(lib().sf_substep(ctypes.byref(prm), arr, n, stage, stream), "sf_substep")


def sf_adjoint_substep(prm: sf_params, patches, stage: int, stream: int = 0) -> None:
    arr, n = _patches(patches)
    _check(lib().sf_adjoint_substep(ctypes.byref(prm), arr, n, stage, stream), "sf_adjoint_substep")


def sf_rhs(prm: sf_params, patch: sf_patch, rhs_out: int, stream: int = 0) -> None:
    _check(lib().sf_rhs(ctypes.byref(prm), ctypes.byref(patch), rhs_out, stream), "sf_rhs")


def sf_fill_ghosts_periodic(patch: sf_patch, array: int, nf: int, stream: int = 0) -> None:
    _check(lib().sf_fill_ghosts_periodic(ctypes.byref(patch), array, nf, stream),
           "sf_fill_ghosts_periodic")


def sf_mhd_max_rate(prm: sf_params, patch: sf_patch, array: int, d_rate: int, stream: int = 0) -> None:
    _check(lib().sf_mhd_max_rate(ctypes.byref(prm), ctypes.byref(patch), array, d_rate, stream),
           "sf_mhd_max_rate")


def sf_gather(patch: sf_patch, array: int, field: int, obs: int, nobs: int, out: int,
              stream: int = 0) -> None:
    _check(lib().sf_gather(ctypes.byref(patch), array, field, obs, nobs, out, stream), "sf_gather")


def sf_scatter_add(patch: sf_patch, array: int, field: int, obs: int, nobs: int, vals: int,
                   stream: int = 0) -> None:
    _check(lib().sf_scatter_add(ctypes.byref(patch), array, field, obs, nobs, vals, stream),
           "sf_scatter_add")


def sf_diagnostics(prm: sf_params, patch: sf_patch, array: int, d_out: int, stream: int = 0) -> None:
    _check(lib().sf_diagnostics(ctypes.byref(prm), ctypes.byref(patch), array, d_out, stream),
           "sf_diagnostics")


def sf_batch_create(prm: sf_params, patches) -> int:
    arr, n = _patches(patches)
    out = ctypes.c_void_p()
    _check(lib().sf_batch_create(ctypes.byref(prm), arr, n, ctypes.byref(out)), "sf_batch_create")
    return out.value


def sf_batch_substep(batch: int, stage: int, stream: int = 0) -> None:
    _check(lib().sf_batch_substep(batch, stage, stream), "sf_batch_substep")


def sf_batch_tune(batch: int, stream: int = 0) -> None:
    _check(lib().sf_batch_tune(batch, stream), "sf_batch_tune")


def sf_batch_capture(batch: int, stream: int) -> None:
    _check(lib().sf_batch_capture(batch, stream), "sf_batch_capture")


def sf_batch_launch(batch: int, stream: int = 0) -> None:
    _check(lib().sf_batch_launch(batch, stream), "sf_batch_launch")


def sf_batch_set_halo(batch: int, role: int, boxes) -> None:
    """Ghost-shell box copies run after every stage that writes buffer role
    `role` (0: u_n, 1: u_stage, 2: u_next)."""
    arr = (sf_box_copy * max(1, len(boxes)))(*boxes)
    _check(lib().sf_batch_set_halo(batch, role, arr, len(boxes)), "sf_batch_set_halo")


def sf_batch_launches_per_step(batch: int) -> int:
    return lib().sf_batch_launches_per_step(batch)


def sf_batch_tuned(batch: int) -> dict:
    """Tile choices per size class (wave small/large, CCZ4 small/large): the
    persistent kernel's tile and the TMA tile width (0: no TMA patch; -1:
    per-patch rule, not tuned)."""
    shapes = (ctypes.c_int32 * 12)()
    widths = (ctypes.c_int32 * 4)()
    _check(lib().sf_batch_tuned(batch, shapes, widths), "sf_batch_tuned")
    names = ("wave_small", "wave_large", "z4_small", "z4_large")
    return {n: {"persistent_tile": tuple(shapes[3 * c:3 * c + 3]), "tma_tile_width": widths[c]}
            for c, n in enumerate(names)}


def sf_batch_destroy(batch: int) -> None:
    _check(lib().sf_batch_destroy(batch), "sf_batch_destroy")


def sf_batch_substep_static(prm: sf_params, patches, stage: int, stream: int = 0) -> None:
    """Allocation-free batched RK4 stage (scratch in a fixed device array)."""
    arr, n = _patches(patches)
    _check(lib().sf_batch_substep_static(ctypes.byref(prm), arr, n, stage, stream),
           "sf_batch_substep_static")


def sf_copy_boxes(boxes, precision: int, stream: int = 0) -> None:
    arr = (sf_box_copy * max(1, len(boxes)))(*boxes)
    _check(lib().sf_copy_boxes(arr, len(boxes), precision, stream), "sf_copy_boxes")


def sf_prolong(coarse: sf_patch, coarse_array: int, nf: int, ratio: int, origin, ext,
               fine_out: int, out_sy: int, out_sz: int, out_sf: int, stream: int = 0) -> None:
    o = (ctypes.c_int32 * 3)(*origin)
    e = (ctypes.c_int32 * 3)(*ext)
    _check(lib().sf_prolong(ctypes.byref(coarse), coarse_array, nf, ratio, o, e, fine_out, out_sy,
                            out_sz, out_sf, stream), "sf_prolong")


def sf_radiative_substep(prm: sf_params, patch: sf_patch, x0, u_inf, speed, stage: int,
                         stream: int = 0) -> None:
    """RK stage of the radiative boundary condition on the ghost shell (Sec. V)."""
    d3 = (ctypes.c_double * 3)(*[float(v) for v in x0])
    ui = (ctypes.c_double * len(u_inf))(*[float(v) for v in u_inf])
    sp = (ctypes.c_double * len(speed))(*[float(v) for v in speed])
    _check(lib().sf_radiative_substep(ctypes.byref(prm), ctypes.byref(patch), d3, ui, sp, stage,
                                      stream), "sf_radiative_substep")


def sf_bor_prolong(coarse: sf_patch, rk: int, states, nf: int, ratio: int, r: int, stage: int,
                   origin, ext, fine_out: int, out_sy: int, out_sz: int, out_sf: int,
                   stream: int = 0) -> None:
    """Fine-time value of BOR sub-cycling (fine step r, fine stage `stage`, or
    the end of the fine step for stage = number of RK stages) prolonged onto
    fine points origin..origin+ext-1.  `states` are device pointers of the
    coarse stage states (5 for RK4, 4 for SSP-RK3)."""
    arr = (ctypes.c_void_p * len(states))(*states)
    o = (ctypes.c_int32 * 3)(*origin)
    e = (ctypes.c_int32 * 3)(*ext)
    _check(lib().sf_bor_prolong(ctypes.byref(coarse), rk, arr, nf, ratio, r, stage, o, e, fine_out,
                                out_sy, out_sz, out_sf, stream), "sf_bor_prolong")


def prolong_box(origin, ext, out: int, out_sy: int, out_sz: int, out_sf: int) -> sf_prolong_box:
    b = sf_prolong_box()
    b.origin[:] = origin
    b.ext[:] = ext
    b.out = out
    b.out_sy, b.out_sz, b.out_sf = out_sy, out_sz, out_sf
    return b


def sf_bor_prolong_boxes(coarse: sf_patch, rk: int, states, nf: int, ratio: int, r: int,
                         stage: int, boxes, stream: int = 0) -> None:
    """sf_bor_prolong over several output boxes (sf_prolong_box) in one launch."""
    arr = (ctypes.c_void_p * len(states))(*states)
    bx = (sf_prolong_box * max(1, len(boxes)))(*boxes)
    _check(lib().sf_bor_prolong_boxes(ctypes.byref(coarse), rk, arr, nf, ratio, r, stage, bx,
                                      len(boxes), stream), "sf_bor_prolong_boxes")


def sf_selftest_wait_timeout(limit_cycles: int, stream: int = 0) -> None:
    """Launches a bounded wait that must give up (see sf.h); the next
    sf_get_device_status() then returns SF_ETIMEOUT."""
    _check(lib().sf_selftest_wait_timeout(limit_cycles, stream), "sf_selftest_wait_timeout")


def sf_get_device_status(stream: int = 0) -> int:
    """Synchronises the stream; returns SF_OK, SF_ENONFINITE or SF_ETIMEOUT (and clears it)."""
    return lib().sf_get_device_status(stream)


def sf_last_error() -> str:
    return lib().sf_last_error().decode(errors="replace")


def sf_launch_count() -> int:
    return lib().sf_launch_count()
