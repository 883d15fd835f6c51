"""FP64 CPU oracle for the method-of-lines substep of arXiv:1806.04182.

TEST INFRASTRUCTURE.  This package is the plain, slow reference that the CUDA
path is checked against.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product package never
does, and it shares no code with the CUDA library.

The arithmetic lives in ``sf_oracle.cpp`` (plain C++17, FP64, one cell at a
time, OpenMP only over the (z, y) rows of the right-hand-side sweep).  This
module compiles it with g++ on first use and wraps it with ctypes.

Functions and what pins them (tests/test_oracle_*.py):
  rhs(WAVE)        Sec. IV.A (first-order form) + Sec. II.B.1 stencils.
                   Pinned: exact per-Fourier-mode symbols, closed-form RK4
                   evolution of a single mode, 4th-order convergence to the
                   continuum plane wave, energy decay.
  rhs(WAVE_ADJ)    transpose of the wave operator.  Pinned: <L u, v> = <u, L^T v>.
  rhs(MHD)         Sec. IV.B + Sec. II.B.2 + App. B.  Pinned: uniform state
                   gives zero, telescoping conservation, 1D data, axis
                   permutation equivariance, WENO5 exactness on quartic data
                   (JS weights reduce to the linear ones), convergence on the
                   circularly polarised Alfven wave (Sec. IV.B.1).
  rhs(Z4)          Sec. V.  Pinned: Minkowski gives zero, gauge-wave exact
                   solution (4th-order truncation), flat metric in curvilinear
                   coordinates (Ricci and Christoffels), lapse Laplacian;
                   every algebraic term (Theta, Z, K, A~ products, damping,
                   gauge) on homogeneous states, and the whole right-hand
                   side (gradient couplings of Z and Theta, conformal Ricci,
                   shift terms) on polynomial states where the stencils are
                   exact, both against the damped covariant Z4 equations in
                   3+1 form mapped to the CCZ4 variables.
  rk4_step         Sec. II.C Table RK44.  Pinned: amplification polynomial
                   of a single Fourier mode.
  ssprk3_step      App. C/D, read as U(3) = U + k1/4 + k2/4 and
                   U^{n+1} = U + (k1 + k2 + 4 k3)/6 (the printed k2/4 + k3/4
                   and (k1 + 2 k2 + 4 k3)/6 are inconsistent).  Pinned:
                   third-order amplification polynomial; equal to the
                   Shu-Osher form.
  z4_monitors      root mean squares of Theta, |Z| (Z^i = chi/2 (Gammahat^i -
                   Gamma~^i)), ln det gt~ and gt~^{ij} A~_ij (Sec. V).  Pinned:
                   closed forms on a rotated homogeneous metric with det != 1
                   and on a diagonal metric varying along x (closed-form
                   Gamma~^i), every monitor non-zero.
  rhs_points       rhs at listed interior points.  Pinned: equal bit for bit
                   to the columns of rhs, any order, ragged grid.
  misfit_gradient  discrete adjoint of the RK4 wave evolution.  Pinned:
                   central finite differences (exact for the quadratic misfit).
  weno             one reconstruction of five values (App. A, App. B).
                   Pinned: each candidate and the linear weights reproduce the
                   coefficient tables the paper prints (tests/golden).
  radiative_rhs    Sec. V radiative boundary condition at ghost points.
                   Pinned: zero on U = U_inf; closed form on linear data
                   (every one-sided stencil exact); 4th-order convergence to
                   the time derivative of an exact outgoing spherical wave.
  rk4_step_radiative  RK4 with radiative ghost points.  Pinned: reduces to
                   the plain step's interior on data that the boundary does
                   not reach within one step; outgoing wave convergence.
  stencil(DLOP)    Sec. II.B.1 one-sided advection stencils.  Pinned:
                   exactness on quartics, one-sidedness, truncation term.
  prolong          Sec. III.A quintic Lagrange prolongation.  Pinned:
                   exactness on quintic polynomials, injection at coincident
                   points, 6th-order convergence on smooth data.
  restrict         Sec. III.A injection.  Pinned: brute-force copy.
  dense_output     App. C interpolators.  Pinned: theta = 0 and 1 give U^n
                   and U^{n+1}; exact on polynomial-in-time solutions of the
                   interpolator's order; derivatives against finite
                   differences in theta.
  bor_fine_stages  App. D (BOR).  Pinned: with R = 1 the fine stages equal
                   the coarse RK4 stages for any increments; for a forcing
                   f(t) of degree 2 (RK4) or 1 (SSP-RK3) the fine stages equal
                   those of a fine RK step; 4th-order (RK4) error of the
                   sub-cycled solution of a linear ODE system.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

WAVE, MHD, Z4, WAVE_ADJ = 0, 1, 2, 3
RK4, SSPRK3 = 0, 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sf_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Params(ctypes.Structure):
    """Mirror of ``or_params`` in sf_oracle.cpp."""

    _fields_ = [
        ("sigma", ctypes.c_double),
        ("gamma_eos", ctypes.c_double),
        ("weno_eps", ctypes.c_double),
        ("weno_q", ctypes.c_double),
        ("kappa_z", ctypes.c_double),
        ("kappa_c", ctypes.c_double),
        ("eta", ctypes.c_double),
        ("g_shift", ctypes.c_double),
        ("ch", ctypes.c_double),
        ("kappa_psi", ctypes.c_double),
        ("weno_variant", ctypes.c_int32),
        ("slicing", ctypes.c_int32),
        ("shift_frozen", ctypes.c_int32),
        ("mhd_glm", ctypes.c_int32),
        ("lopsided", ctypes.c_int32),
        ("flux_split", ctypes.c_int32),
    ]


def params(**kw) -> Params:
    """Defaults: sigma = 0.1, Gamma = 5/3, eps = dx^4, JS weights, q = 2,
    kappa_z = kappa_c = 1, eta = 2, g = 3/4, 1+log slicing (Sec. V with M = 1)."""
    d = dict(sigma=0.1, gamma_eos=5.0 / 3.0, weno_eps=0.0, weno_q=2.0, kappa_z=1.0,
             kappa_c=1.0, eta=2.0, g_shift=0.75, ch=0.0, kappa_psi=0.0, weno_variant=0,
             slicing=0, shift_frozen=0, mhd_glm=0, lopsided=0, flux_split=0)
    d.update(kw)
    return Params(**d)


def build(force: bool = False) -> str:
    """Compile sf_oracle.cpp into oracle/_build/liboracle.so (g++, -O2, OpenMP)."""
    with _lock:
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
            return _SO
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
        return _SO


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        pp = ctypes.POINTER(Params)
        L.or_nfields.argtypes = [ctypes.c_int, pp]
        L.or_fill_ghosts_periodic.argtypes = [ctypes.c_int, ip, ctypes.c_int, dp]
        L.or_rhs.argtypes = [ctypes.c_int, pp, ip, ctypes.c_int, dp, dp, dp]
        L.or_rk4_step.argtypes = [ctypes.c_int, pp, ip, ctypes.c_int, dp, ctypes.c_double, dp, dp]
        L.or_ssprk3_step.argtypes = [ctypes.c_int, pp, ip, ctypes.c_int, dp, ctypes.c_double, dp, dp]
        L.or_mhd_max_rate.argtypes = [pp, ip, ctypes.c_int, dp, dp]
        L.or_mhd_max_rate.restype = ctypes.c_double
        L.or_wave_energy.argtypes = [ip, ctypes.c_int, dp, dp]
        L.or_wave_energy.restype = ctypes.c_double
        L.or_z4_monitors.argtypes = [ip, ctypes.c_int, dp, dp, dp]
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_max_threads.restype = ctypes.c_int
        L.or_wave_misfit_gradient.argtypes = [pp, ip, dp, ctypes.c_double, ctypes.c_int, dp, dp,
                                              ctypes.c_int, ctypes.POINTER(ctypes.c_int64), dp,
                                              dp, dp]
        L.or_wave_misfit_gradient.restype = ctypes.c_double
        L.or_count_ops.argtypes = [ctypes.c_int, pp, ip, ctypes.c_int, dp, dp,
                                   ctypes.POINTER(ctypes.c_long)]
        L.or_rhs_points.argtypes = [ctypes.c_int, pp, ip, ctypes.c_int, dp, dp, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int64), dp]
        L.or_prolong.argtypes = [ctypes.c_int, ip, ctypes.c_int, dp, ctypes.c_int, ip, ip, dp]
        L.or_restrict.argtypes = [ctypes.c_int, ip, ctypes.c_int, dp, ctypes.c_int, ip, ip, dp]
        L.or_stencil.argtypes = [ctypes.c_int, ip, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double]
        L.or_stencil.restype = ctypes.c_double
        L.or_weno.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ctypes.c_double]
        L.or_weno.restype = ctypes.c_double
        L.or_radiative_rhs.argtypes = [ctypes.c_int, ip, ctypes.c_int, dp, dp, dp, dp, dp, dp]
        L.or_rk4_step_radiative.argtypes = [ctypes.c_int, pp, ip, ctypes.c_int, dp, dp, dp, dp,
                                            ctypes.c_double, dp, dp]
        L.or_bor_fine_stages.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int, dp]
        L.or_dense_output.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, dp]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ivec(n):
    return (ctypes.c_int * 3)(*[int(x) for x in n])


def _dvec(d):
    return (ctypes.c_double * 3)(*[float(x) for x in d])


def _darr(d):
    d = [float(x) for x in d]
    return (ctypes.c_double * len(d))(*d)


def shape_info(U: np.ndarray, g: int):
    """(nf, n=(nx,ny,nz)) of a ghosted array of shape (nf, nz+2g, ny+2g, nx+2g)."""
    nf, Nz, Ny, Nx = U.shape
    return nf, (Nx - 2 * g, Ny - 2 * g, Nz - 2 * g)


def nfields(system: int, p: Params | None = None) -> int:
    return lib().or_nfields(system, ctypes.byref(p or params()))


def fill_ghosts(U: np.ndarray, g: int) -> np.ndarray:
    nf, n = shape_info(U, g)
    lib().or_fill_ghosts_periodic(nf, _ivec(n), g, _dp(U))
    return U


def rhs(system: int, U: np.ndarray, dx, p: Params | None = None, g: int = 3) -> np.ndarray:
    """(L + Q_d)(U) on the interior; U ghosted and ghost-filled."""
    p = p or params()
    nf, n = shape_info(U, g)
    out = np.zeros((nf, n[2], n[1], n[0]))
    rc = lib().or_rhs(system, ctypes.byref(p), _ivec(n), g, _dvec(dx), _dp(U), _dp(out))
    if rc:
        raise ValueError("oracle rhs: bad arguments")
    return out


def rhs_points(system: int, U: np.ndarray, dx, pts: np.ndarray, p: Params | None = None,
               g: int = 3) -> np.ndarray:
    """(L + Q_d)(U) at interior linear indices pts; returns shape (nf, npts)."""
    p = p or params()
    nf, n = shape_info(U, g)
    pts = np.ascontiguousarray(pts, dtype=np.int64)
    out = np.zeros((nf, pts.size))
    rc = lib().or_rhs_points(system, ctypes.byref(p), _ivec(n), g, _dvec(dx), _dp(U), pts.size,
                             pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out))
    if rc:
        raise ValueError("oracle rhs_points: bad arguments")
    return out


def prolong(Uc: np.ndarray, ratio: int, origin, ext, g: int = 3) -> np.ndarray:
    """Sec. III.A quintic Lagrange prolongation of a ghost-filled coarse array
    onto fine points origin..origin+ext-1 (fine index R*i = coarse point i)."""
    nf, n = shape_info(Uc, g)
    out = np.zeros((nf, ext[2], ext[1], ext[0]))
    rc = lib().or_prolong(nf, _ivec(n), g, _dp(Uc), ratio, _ivec(origin), _ivec(ext), _dp(out))
    if rc:
        raise ValueError("oracle prolong: stencil leaves the coarse box")
    return out


def restrict(Uf: np.ndarray, ratio: int, origin, ext, g: int = 3) -> np.ndarray:
    """Sec. III.A injection of fine point R*i into coarse points origin..origin+ext-1."""
    nf, n = shape_info(Uf, g)
    out = np.zeros((nf, ext[2], ext[1], ext[0]))
    rc = lib().or_restrict(nf, _ivec(n), g, _dp(Uf), ratio, _ivec(origin), _ivec(ext), _dp(out))
    if rc:
        raise ValueError("oracle restrict: out of the fine box")
    return out


def weno(variant: int, side: int, w, eps: float, q: float = 2.0) -> float:
    """One reconstruction of w = U_{i-2..i+2}: side 0 -> U^L_{i+1/2}, 1 -> U^R_{i-1/2}."""
    a = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    assert a.shape == (5,)
    return lib().or_weno(variant, side, _dp(a), eps, q)


def radiative_rhs(U: np.ndarray, dx, x0, uinf, v, g: int = 3) -> np.ndarray:
    """Sec. V radiative RHS at every ghost point of the ghosted array U (zero
    at interior points).  x0 = position of interior point (0,0,0)."""
    nf, n = shape_info(U, g)
    out = np.zeros_like(np.ascontiguousarray(U, dtype=np.float64))
    U = np.ascontiguousarray(U, dtype=np.float64)
    rc = lib().or_radiative_rhs(nf, _ivec(n), g, _dvec(dx), _dvec(x0), _dp(U),
                                _darr(np.broadcast_to(uinf, nf)), _darr(np.broadcast_to(v, nf)),
                                _dp(out))
    if rc:
        raise ValueError("oracle radiative_rhs: bad arguments")
    return out


def rk4_step_radiative(system: int, U: np.ndarray, dx, x0, uinf, v, dt: float,
                       p: Params | None = None, g: int = 3, stages: bool = False):
    """One RK(4,4) step in place with radiative ghost points (Sec. V); returns
    the ghosted U(2), U(3), U(4), U^{n+1} if asked."""
    p = p or params()
    nf, n = shape_info(U, g)
    st = np.zeros((4,) + U.shape) if stages else None
    rc = lib().or_rk4_step_radiative(system, ctypes.byref(p), _ivec(n), g, _dvec(dx), _dvec(x0),
                                     _darr(np.broadcast_to(uinf, nf)),
                                     _darr(np.broadcast_to(v, nf)), dt, _dp(U),
                                     _dp(st) if stages else None)
    if rc:
        raise ValueError("oracle rk4_step_radiative: bad arguments")
    return st


def bor_fine_stages(rk: int, Un: np.ndarray, k: np.ndarray, dt: float, R: int, r: int) -> np.ndarray:
    """Sec. III.B / App. D (BOR): fine stage inputs U^(1..s) and the end value
    U^{n+(r+1)/R} of fine step r of R, from the coarse U^n (any shape) and the
    coarse increments k (s x Un.shape), s = 4 (RK4, rk = 0) or 3 (SSP-RK3).
    Returns an array (s + 1) x Un.shape."""
    s = 4 if rk == RK4 else 3
    un = np.ascontiguousarray(Un, dtype=np.float64).ravel()
    kk = np.ascontiguousarray(k, dtype=np.float64).reshape(s, un.size)
    out = np.zeros((s + 1, un.size))
    rc = lib().or_bor_fine_stages(rk, un.size, _dp(un), _dp(kk), dt, R, r, _dp(out))
    if rc:
        raise ValueError("oracle bor_fine_stages: bad arguments")
    return out.reshape((s + 1,) + np.shape(Un))


def dense_output(rk: int, Un: np.ndarray, k: np.ndarray, dt: float, theta: float, m: int = 0) -> np.ndarray:
    """App. C dense output (m = 0) or its m-th time derivative at t^n + theta dt."""
    s = 4 if rk == RK4 else 3
    un = np.ascontiguousarray(Un, dtype=np.float64).ravel()
    kk = np.ascontiguousarray(k, dtype=np.float64).reshape(s, un.size)
    out = np.zeros(un.size)
    rc = lib().or_dense_output(rk, un.size, _dp(un), _dp(kk), dt, theta, m, _dp(out))
    if rc:
        raise ValueError("oracle dense_output: bad arguments")
    return out.reshape(np.shape(Un))


def rk4_step(system: int, U: np.ndarray, dx, dt: float, p: Params | None = None, g: int = 3,
             stages: bool = False):
    """One RK(4,4) step in place; returns the interior U(2), U(3), U(4), U^{n+1} if asked."""
    p = p or params()
    nf, n = shape_info(U, g)
    st = np.zeros((4, nf, n[2], n[1], n[0])) if stages else None
    rc = lib().or_rk4_step(system, ctypes.byref(p), _ivec(n), g, _dvec(dx), dt, _dp(U),
                           _dp(st) if stages else None)
    if rc:
        raise ValueError("oracle rk4: bad arguments")
    return st


def ssprk3_step(system: int, U: np.ndarray, dx, dt: float, p: Params | None = None, g: int = 3,
                stages: bool = False):
    """One SSP-RK(3,3) step in place; returns the interior U(2), U(3), U^{n+1} if asked."""
    p = p or params()
    nf, n = shape_info(U, g)
    st = np.zeros((3, nf, n[2], n[1], n[0])) if stages else None
    rc = lib().or_ssprk3_step(system, ctypes.byref(p), _ivec(n), g, _dvec(dx), dt, _dp(U),
                              _dp(st) if stages else None)
    if rc:
        raise ValueError("oracle ssprk3: bad arguments")
    return st


def mhd_max_rate(U: np.ndarray, dx, p: Params | None = None, g: int = 3) -> float:
    p = p or params()
    nf, n = shape_info(U, g)
    return lib().or_mhd_max_rate(ctypes.byref(p), _ivec(n), g, _dvec(dx), _dp(U))


def wave_energy(U: np.ndarray, dx, g: int = 3) -> float:
    nf, n = shape_info(U, g)
    return lib().or_wave_energy(_ivec(n), g, _dvec(dx), _dp(U))


def set_threads(n: int) -> int:
    """Use n threads in the parallel sweeps; returns the count now in effect."""
    lib().or_set_threads(int(n))
    return lib().or_max_threads()


def max_threads() -> int:
    return lib().or_max_threads()


def z4_monitors(U: np.ndarray, dx, g: int = 3) -> np.ndarray:
    nf, n = shape_info(U, g)
    out = np.zeros(4)
    lib().or_z4_monitors(_ivec(n), g, _dvec(dx), _dp(U), _dp(out))
    return out


def misfit_gradient(phi0: np.ndarray, Pi0: np.ndarray, dx, dt: float, nsteps: int,
                    obs: np.ndarray, ref: np.ndarray, p: Params | None = None):
    """(J, dJ/dphi0, dJ/dPi0) of the RK4 wave evolution; phi0/Pi0 shape (nz, ny, nx)."""
    p = p or params()
    nz, ny, nx = phi0.shape
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    Pi0 = np.ascontiguousarray(Pi0, dtype=np.float64)
    obs = np.ascontiguousarray(obs, dtype=np.int64)
    ref = np.ascontiguousarray(ref, dtype=np.float64)
    assert ref.shape == (nsteps, obs.size)
    gphi = np.zeros_like(phi0)
    gPi = np.zeros_like(Pi0)
    J = lib().or_wave_misfit_gradient(ctypes.byref(p), _ivec((nx, ny, nz)), _dvec(dx), dt,
                                      nsteps, _dp(phi0), _dp(Pi0), obs.size,
                                      obs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      _dp(ref), _dp(gphi), _dp(gPi))
    return J, gphi, gPi


D1, D2, DMIX, KO, DLOP = 0, 1, 2, 3, 4


def stencil(op: int, U: np.ndarray, dx, f: int, i: int, j: int, k: int, d1: int = 0,
            d2: int = 1, sigma: float = 0.1, g: int = 3) -> float:
    """One Sec. II.B.1 operator at interior point (i, j, k) of field f."""
    nf, n = shape_info(U, g)
    return lib().or_stencil(op, _ivec(n), g, _dvec(dx), _dp(U), f, i, j, k, d1, d2, sigma)


def count_ops(system: int, U: np.ndarray, dx, p: Params | None = None, g: int = 3) -> dict:
    """Per-cell operation counts of the right-hand side (counting scalar)."""
    p = p or params()
    nf, n = shape_info(U, g)
    out = (ctypes.c_long * 6)()
    lib().or_count_ops(system, ctypes.byref(p), _ivec(n), g, _dvec(dx), _dp(U), out)
    keys = ("add", "mul", "div", "sqrt", "log", "cmp")
    return dict(zip(keys, list(out)))


def ghosted(interior: np.ndarray, g: int = 3) -> np.ndarray:
    """Embed an interior array (nf, nz, ny, nx) into a ghost-filled periodic array."""
    nf, nz, ny, nx = interior.shape
    U = np.zeros((nf, nz + 2 * g, ny + 2 * g, nx + 2 * g))
    U[:, g:g + nz, g:g + ny, g:g + nx] = interior
    return fill_ghosts(U, g)


def interior(U: np.ndarray, g: int = 3) -> np.ndarray:
    return U[:, g:U.shape[1] - g, g:U.shape[2] - g, g:U.shape[3] - g]
