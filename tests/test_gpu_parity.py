"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerance (FP64): max over fields of ||gpu - oracle||_inf / max(||oracle||_inf, floor)
<= 1e-12 per substep, the bound stated for this path.  The floor (1e-3..1e-2 of
the O(1) state scale) exists because rounding of the O(1) metric's 1/dx^2
stencils enters every field's right-hand side, whatever that field's own size.  Summation order differs
between the two (the kernels fuse and reorder sums), so bit equality is not
expected except where the result is exactly zero.  FP32-bulk results are
checked against the same oracle with per-field bounds derived from float
rounding (stated at each test).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1806_04182_gb300 import build, capi, inputs
from paper_1806_04182_gb300.state import PatchState

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    return capi.lib()


def rel_err(got, want, floor=1e-300):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    errs = []
    for f in range(want.shape[0]):
        scale = max(np.abs(want[f]).max(), floor)
        errs.append(np.abs(got[f] - want[f]).max() / scale)
    return np.array(errs)


def oracle_params(prm: capi.sf_params):
    return oracle.params(sigma=prm.sigma_ko, gamma_eos=prm.gamma_eos, weno_eps=prm.weno_eps,
                         weno_q=prm.weno_q, kappa_z=prm.kappa_z, kappa_c=prm.kappa_c, eta=prm.eta,
                         g_shift=prm.g_shift, weno_variant=prm.weno_variant, slicing=prm.slicing,
                         shift_frozen=prm.shift_frozen, lopsided=prm.lopsided,
                         flux_split=prm.flux_split)


def run_stages(system, U0, dx, dt, prm, precision=capi.SF_FP64, pitch=None, x_offset=0):
    """GPU stage outputs (interior, numpy float64) of one full step."""
    n = (U0.shape[3], U0.shape[2], U0.shape[1])
    st = PatchState(system, n, dx, dt, precision=precision, prm=prm, x_pitch=pitch,
                    x_offset=x_offset)
    st.upload(U0)
    outs = []
    for s in range(st.nstages):
        arr = st.stage(s)
        outs.append(st.fields(arr).cpu().numpy())
    torch.cuda.synchronize()
    return outs


def oracle_stages(system, U0, dx, dt, prm):
    G = oracle.ghosted(U0.copy())
    if prm.rk == capi.SF_RK4:
        return list(oracle.rk4_step(system, G, dx, dt, oracle_params(prm), stages=True))
    return list(oracle.ssprk3_step(system, G, dx, dt, oracle_params(prm), stages=True))


# ------------------------------------------------------------------ wave
@pytest.mark.parametrize("n", [(37, 13, 11), (5, 6, 4), (64, 9, 3)])
def test_wave_fp64_stages(n):
    U0, dx = inputs.wave_plane(n, seed=2)
    U0 = U0 + inputs.wave_noise(n, seed=3, amp=0.3)
    prm = capi.params()
    dt = 0.25 * min(dx)
    got = run_stages(capi.SF_WAVE, U0, dx, dt, prm)
    want = oracle_stages(oracle.WAVE, U0, dx, dt, prm)
    for s in range(4):
        assert rel_err(got[s], want[s]).max() < TOL64, s


def test_wave_rhs_and_ghost_fill():
    n = (21, 10, 7)
    U0, dx = inputs.wave_plane(n, seed=4)
    U0 = U0 + inputs.wave_noise(n, seed=5, amp=0.5)
    st = PatchState(capi.SF_WAVE, n, dx, 0.01)
    st.upload(U0)
    G = oracle.ghosted(U0)
    # periodic ghost fill is a copy: bit-exact
    np.testing.assert_array_equal(st.A.cpu().numpy(), G)
    r = st.rhs().cpu().numpy()
    want = oracle.rhs(oracle.WAVE, G, dx)
    assert rel_err(r, want).max() < TOL64


@pytest.mark.parametrize("n", [(1, 2, 5), (2, 1, 1), (33, 4, 3)])
@pytest.mark.parametrize("precision", [capi.SF_FP64, capi.SF_FP32_BULK])
def test_periodic_ghost_fill_thin_patches(n, precision):
    # patches thinner than the ghost zone wrap more than once; the fill is a
    # copy, so it is bit-exact against the oracle's in either precision
    U0 = inputs.wave_noise(n, seed=7, amp=1.0)
    st = PatchState(capi.SF_WAVE, n, (0.1, 0.1, 0.1), 0.01, precision=precision)
    st.upload(U0)
    want = oracle.ghosted(U0.astype(np.float32).astype(np.float64) if precision else U0.copy())
    got = st.A.cpu().numpy()[..., :n[0] + 6].astype(np.float64)
    np.testing.assert_array_equal(got, want)


def test_wave_adjoint_step():
    n = (19, 11, 9)
    dx = (1 / 19, 1 / 11, 1 / 9)
    L0 = inputs.wave_noise(n, seed=8)
    dt = 0.2 * min(dx)
    prm = capi.params()
    st = PatchState(capi.SF_WAVE, n, dx, dt, prm=prm)
    st.upload(L0)
    st.adjoint_step(1)
    got = st.interior().cpu().numpy()
    G = oracle.ghosted(L0.copy())
    oracle.rk4_step(oracle.WAVE_ADJ, G, dx, dt, oracle_params(prm))
    assert rel_err(got, oracle.interior(G)).max() < TOL64


def test_wave_fp32_bulk_step():
    # float storage: relative error ~ a few ulp of float per stage
    n = (33, 10, 9)
    U0, dx = inputs.wave_plane(n, seed=6)
    prm = capi.params()
    dt = 0.25 * min(dx)
    got = run_stages(capi.SF_WAVE, U0, dx, dt, prm, precision=capi.SF_FP32_BULK)
    want = oracle_stages(oracle.WAVE, U0, dx, dt, prm)
    assert rel_err(got[3], want[3]).max() < 2e-6


# ------------------------------------------------------------------ Z4
@pytest.mark.parametrize("slicing,frozen,lop", [(0, 0, 0), (1, 1, 0), (0, 0, 1)])
def test_z4_fp64_stages(slicing, frozen, lop):
    n = (35, 9, 6)
    U0, dx = inputs.z4_perturbed(n, seed=1, amp=0.05)
    prm = capi.params(slicing=slicing, shift_frozen=frozen, lopsided=lop)
    dt = 0.25 * min(dx)
    got = run_stages(capi.SF_Z4, U0, dx, dt, prm)
    want = oracle_stages(oracle.Z4, U0, dx, dt, prm)
    for s in range(4):
        e = rel_err(got[s], want[s], floor=1e-3)
        assert e.max() < TOL64, (s, e)


@pytest.mark.parametrize("n", [(3, 5, 4), (7, 3, 5)])
def test_small_boxes_all_systems(n):
    # ghost <= n < 2 ghost: a point near both ends of an axis has periodic
    # images on both sides (up to 26 ghost copies per point)
    for system, osys, data, prm in (
            (capi.SF_WAVE, oracle.WAVE, inputs.wave_plane(n, seed=3), capi.params()),
            (capi.SF_Z4, oracle.Z4, inputs.z4_perturbed(n, seed=3, amp=0.03), capi.params()),
            (capi.SF_MHD, oracle.MHD, inputs.mhd_blast(n, seed=3, radius=0.4),
             capi.params(rk=capi.SF_SSPRK3))):
        U0, dx = data
        dt = 0.1 * min(dx)
        got = run_stages(system, U0, dx, dt, prm)
        want = oracle_stages(osys, U0, dx, dt, prm)
        for s_ in range(len(want)):
            assert rel_err(got[s_], want[s_], floor=1e-2).max() < TOL64, (system, s_)
        # the ghost shell written by the last stage equals a periodic fill
        st = PatchState(system, n, dx, dt, prm=prm)
        st.upload(U0)
        st.step(1)
        G = oracle.ghosted(st.interior().cpu().numpy().copy())
        np.testing.assert_array_equal(st.A.cpu().numpy(), G)


def test_z4_rhs_matches_oracle():
    n = (17, 12, 8)
    U0, dx = inputs.z4_perturbed(n, seed=3, amp=0.08)
    prm = capi.params()
    st = PatchState(capi.SF_Z4, n, dx, 0.01, prm=prm)
    st.upload(U0)
    r = st.rhs().cpu().numpy()
    want = oracle.rhs(oracle.Z4, oracle.ghosted(U0), dx, oracle_params(prm))
    e = rel_err(r, want, floor=1e-3)
    assert e.max() < TOL64, e


def test_z4_minkowski_rhs_is_exactly_zero():
    n = (12, 8, 8)
    U0 = inputs.z4_minkowski(n)
    for prec in (capi.SF_FP64, capi.SF_FP32_BULK):
        st = PatchState(capi.SF_Z4, n, (0.1, 0.1, 0.1), 0.01, precision=prec)
        st.upload(U0)
        assert torch.count_nonzero(st.rhs()).item() == 0


def test_z4_fp32_bulk_step():
    # Float rounding bound: a second-derivative stencil sums 64 ulp-sized
    # rounding terms of |U| <= ~1 and divides by 12 dx^2, so each stage adds
    # ~64 eps32 |U| / (12 dx^2) * dt ~ 1.3 eps32 / dx with dt = dx/4.  Over four
    # stages at dx = 1/33 that is ~2e-5 absolute, i.e. ~4e-4 relative to the
    # 5e-2 perturbation scale of the zero-background fields (floor 1e-2 caps it
    # at ~2e-3).  Fields with an O(1) background see ~1e-7.
    n = (33, 8, 8)
    U0, dx = inputs.z4_perturbed(n, seed=2, amp=0.05)
    prm = capi.params()
    dt = 0.25 * min(dx)
    eps32 = float(np.finfo(np.float32).eps)
    bound = 4 * 64 / 12 * eps32 * dt / min(dx) ** 2 / 1e-2
    got = run_stages(capi.SF_Z4, U0, dx, dt, prm, precision=capi.SF_FP32_BULK)
    want = oracle_stages(oracle.Z4, U0, dx, dt, prm)
    e = rel_err(got[3], want[3], floor=1e-2)
    assert e.max() < bound, (e, bound)
    # fields with an O(1) background (chi, gt_ii, alpha) stay at float rounding
    for f in (0, 1, 4, 6, 18):
        assert e[f] < 1e-6, (f, e[f])


# ------------------------------------------------------------------ MHD
@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_mhd_fp64_stages(variant, split):
    n = (35, 10, 7)
    U0, dx = inputs.mhd_blast(n, seed=4, radius=0.3)
    prm = capi.params(rk=capi.SF_SSPRK3, weno_variant=variant, flux_split=split)
    rate = oracle.mhd_max_rate(oracle.ghosted(U0), dx)
    dt = 0.3 / rate
    got = run_stages(capi.SF_MHD, U0, dx, dt, prm)
    want = oracle_stages(oracle.MHD, U0, dx, dt, prm)
    for s in range(3):
        e = rel_err(got[s], want[s], floor=1e-3)
        assert e.max() < TOL64, (s, e)


# The MHD stage kernel marches a number of planes per block that it picks per
# launch from the grid and the resident blocks (the last block of a column
# may hold fewer planes; a patch thinner than the smallest choice is one
# block deep).  Thin and ragged z extents (at least the 3 ghosts that fused
# periodic ghost writes need), both precisions, against the oracle's stages.
@pytest.mark.parametrize("precision", [capi.SF_FP64, capi.SF_FP32_BULK])
@pytest.mark.parametrize("nz", [3, 4, 5, 9, 17])
def test_mhd_plane_chunks_any_depth(nz, precision):
    n = (13, 9, nz)
    U0, dx = inputs.mhd_blast(n, seed=nz, radius=0.3)
    prm = capi.params(rk=capi.SF_SSPRK3)
    dt = 0.3 / oracle.mhd_max_rate(oracle.ghosted(U0), dx)
    got = run_stages(capi.SF_MHD, U0, dx, dt, prm, precision=precision)
    want = oracle_stages(oracle.MHD, U0, dx, dt, prm)
    tol = TOL64 if precision == capi.SF_FP64 else TOL32_MHD
    for s in range(3):
        e = rel_err(got[s], want[s], floor=1e-3)
        assert e.max() < tol, (nz, s, e)


# FP32 MHD (float storage and arithmetic; the suite's FP32 row) against the
# FP64 oracle.  Bound: a stage output is U plus dt/dx_d times differences of
# the six interface fluxes around the cell; each flux is formed with about
# ten roundings of relative size eps32/2 of |F| <= S |U| (S the LLF speed),
# and dt S / dx <= CFL = 0.3, so |error| <= (1 + 6 * 0.3 * 10) eps32 |U|
# ~ 19 eps32 |U| per stage, plus the rounding of the input state itself;
# the bound taken is 32 eps32 of each field's scale (floor 1e-3).  The
# WENO weights' sensitivity to rounding stays inside it: where a smoothness
# indicator is of rounding size the candidates agree to the same order.
EPS32 = float(np.finfo(np.float32).eps)
TOL32_MHD = 32 * EPS32


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_mhd_fp32_stages(variant, split):
    n = (35, 10, 7)
    U0, dx = inputs.mhd_blast(n, seed=4, radius=0.3)
    prm = capi.params(rk=capi.SF_SSPRK3, weno_variant=variant, flux_split=split)
    dt = 0.3 / oracle.mhd_max_rate(oracle.ghosted(U0), dx)
    got = run_stages(capi.SF_MHD, U0, dx, dt, prm, precision=capi.SF_FP32_BULK)
    want = oracle_stages(oracle.MHD, U0, dx, dt, prm)
    for s in range(3):
        e = rel_err(got[s], want[s], floor=1e-3)
        assert e.max() < TOL32_MHD, (s, e / EPS32)


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_mhd_fp32_brio_wu_stages(variant):
    n = (256, 3, 3)
    U0, dx = inputs.mhd_brio_wu(n)
    prm = capi.params(rk=capi.SF_SSPRK3, weno_variant=variant, gamma_eos=2.0)
    dt = 0.2 * dx[0]
    got = run_stages(capi.SF_MHD, U0, dx, dt, prm, precision=capi.SF_FP32_BULK)
    want = oracle_stages(oracle.MHD, U0, dx, dt, prm)
    for s in range(3):
        e = rel_err(got[s], want[s], floor=1e-3)
        assert e.max() < TOL32_MHD, (s, e / EPS32)


# The Brio & Wu shock tube (Sec. IV.B.2; Gamma = 2, dt = 0.2 dx): stage
# outputs on discontinuous data, where the WENO weights are far from the
# linear ones, from the initial jumps and from the developed waves after 30
# oracle steps, for every reconstruction.
@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("developed", [False, True])
def test_mhd_brio_wu_stages(variant, developed):
    n = (256, 3, 3)
    U0, dx = inputs.mhd_brio_wu(n)
    prm = capi.params(rk=capi.SF_SSPRK3, weno_variant=variant, gamma_eos=2.0)
    dt = 0.2 * dx[0]
    if developed:
        G = oracle.ghosted(U0.copy())
        for _ in range(30):
            oracle.ssprk3_step(oracle.MHD, G, dx, dt, oracle_params(prm))
        U0 = np.ascontiguousarray(oracle.interior(G))
    got = run_stages(capi.SF_MHD, U0, dx, dt, prm)
    want = oracle_stages(oracle.MHD, U0, dx, dt, prm)
    for s in range(3):
        e = rel_err(got[s], want[s], floor=1e-3)
        assert e.max() < TOL64, (s, e)


def test_mhd_max_rate_and_rhs():
    n = (20, 9, 8)
    U0, dx = inputs.mhd_blast(n, seed=5, radius=0.3)
    prm = capi.params(rk=capi.SF_SSPRK3)
    st = PatchState(capi.SF_MHD, n, dx, 0.001, prm=prm)
    st.upload(U0)
    G = oracle.ghosted(U0)
    assert st.mhd_max_rate().item() == pytest.approx(oracle.mhd_max_rate(G, dx), rel=1e-13)
    e = rel_err(st.rhs().cpu().numpy(), oracle.rhs(oracle.MHD, G, dx), floor=1e-3)
    assert e.max() < TOL64, e


def test_mhd_fused_cfl_rate_equals_separate_reduction():
    # the last SSP-RK3 stage reduces the signal rate of its output; it must equal
    # sf_mhd_max_rate of the new state exactly (max is order independent)
    n = (40, 17, 11)
    U0, dx = inputs.mhd_blast(n, seed=6, radius=0.3)
    st = PatchState(capi.SF_MHD, n, dx, 1e-3, prm=capi.params(rk=capi.SF_SSPRK3))
    st.upload(U0)
    rates = st.step_cfl(3, cfl=0.3)
    assert rates[0] == pytest.approx(oracle.mhd_max_rate(oracle.ghosted(U0), dx), rel=1e-13)
    st2 = PatchState(capi.SF_MHD, n, dx, 1e-3, prm=capi.params(rk=capi.SF_SSPRK3))
    st2.upload(U0)
    for r in rates[:-1]:
        st2.dt = 0.3 / r
        st2.step(1)
    assert st2.mhd_max_rate().item() == rates[-1]


def test_mhd_uniform_rhs_exactly_zero():
    n = (9, 8, 7)
    st = PatchState(capi.SF_MHD, n, (0.1, 0.1, 0.1), 0.01, prm=capi.params(rk=capi.SF_SSPRK3))
    st.upload(inputs.mhd_uniform(n))
    assert torch.count_nonzero(st.rhs()).item() == 0


# ------------------------------------------------------------------ diagnostics, status
def test_diagnostics_match_oracle():
    n = (16, 12, 10)
    U0, dx = inputs.wave_plane(n, seed=1)
    st = PatchState(capi.SF_WAVE, n, dx, 0.01)
    st.upload(U0)
    d = st.diagnostics().cpu().numpy()
    assert d[0] == pytest.approx(oracle.wave_energy(oracle.ghosted(U0), dx), rel=1e-12)
    assert d[4] == 0
    U0, dx = inputs.z4_perturbed(n, seed=2, amp=0.03)
    st = PatchState(capi.SF_Z4, n, dx, 0.01)
    st.upload(U0)
    d = st.diagnostics().cpu().numpy()
    m = oracle.z4_monitors(oracle.ghosted(U0), dx)
    N = np.prod(n)
    np.testing.assert_allclose(np.sqrt(d[:4] / N), m, rtol=1e-10)


def test_nonfinite_output_is_flagged():
    n = (8, 8, 8)
    U0, dx = inputs.wave_plane(n, seed=1)
    U0[1, 3, 4, 5] = np.nan
    prm = capi.params(check_finite=1)
    st = PatchState(capi.SF_WAVE, n, dx, 0.01, prm=prm)
    st.upload(U0)
    capi.sf_get_device_status()  # clear
    st.step(1)
    assert capi.sf_get_device_status() == capi.SF_ENONFINITE
    assert capi.sf_get_device_status() == capi.SF_OK  # cleared by the read


# ------------------------------------------------------------------ full size, sampled
def test_z4_full_size_sampled_parity():
    # The 96^3 CCZ4 workload of the benchmark, in its launch configuration
    # (compile-time-stride kernel): sampled points of the RHS and of the first
    # stage output against the oracle.  A 1/dx^2 stencil of O(1) values
    # carries ~64 eps64 |U| / (12 dx^2) of rounding whatever the summation
    # order, so the raw RHS gets that bound; the state after the substep
    # (U + dt/2 r) meets the 1e-12 bar.
    n = (96, 96, 96)
    U0, dx = inputs.z4_minkowski_noise(n, seed=0, amp=1e-10)
    pert, _ = inputs.z4_perturbed(n, seed=7, amp=0.05)
    U0 = U0 + (pert - inputs.z4_minkowski(n))
    prm = capi.params()
    dt = 0.25 * dx[0]
    st = PatchState(capi.SF_Z4, n, dx, dt, prm=prm)
    st.upload(U0)
    r = st.rhs().cpu().numpy().reshape(25, -1)
    out = st.interior(st.stage(0)).cpu().numpy().reshape(25, -1)
    pts = inputs.observers(n, 2000, seed=11)
    want = oracle.rhs_points(oracle.Z4, oracle.ghosted(U0), dx, pts, oracle_params(prm))
    eps64 = float(np.finfo(np.float64).eps)
    umax = np.abs(U0).max()
    for f in range(25):
        bound = 2 * 64 / 12 * eps64 * umax / dx[0] ** 2
        assert np.abs(r[f, pts] - want[f]).max() < bound, f
    want_out = U0.reshape(25, -1)[:, pts] + 0.5 * dt * want
    assert rel_err(out[:, pts], want_out, floor=1e-2).max() < TOL64


@pytest.mark.parametrize("n", [(96, 96, 96), (33, 10, 8)])
def test_z4_double_word_islands_match_fp64_islands(n):
    # Double-word islands (relative error a few 2^-48) and native FP64 islands
    # agree far below float resolution; what remains is the float rounding of
    # the bulk stencils, which differs between the two compiled kernels only
    # through FMA contraction.  Both must sit inside the FP32 rounding bound of
    # test_z4_fp32_bulk_step against the oracle, and within it of each other.
    U0, dx = inputs.z4_perturbed(n, seed=5, amp=0.03)
    prm = capi.params()
    dt = 0.25 * min(dx)
    eps32 = float(np.finfo(np.float32).eps)
    bound = 4 * 64 / 12 * eps32 * dt / min(dx) ** 2 / 1e-2
    a = run_stages(capi.SF_Z4, U0, dx, dt, prm, precision=capi.SF_FP32_BULK)[3]
    b = run_stages(capi.SF_Z4, U0, dx, dt, prm, precision=capi.SF_FP32_BULK_DW)[3]
    want = oracle_stages(oracle.Z4, U0, dx, dt, prm)[3]
    assert rel_err(a, want, floor=1e-2).max() < bound
    assert rel_err(b, want, floor=1e-2).max() < bound
    assert rel_err(b, a, floor=1e-2).max() < bound


def test_z4_double_word_minkowski_is_exactly_zero():
    n = (12, 8, 8)
    st = PatchState(capi.SF_Z4, n, (0.1, 0.1, 0.1), 0.01, precision=capi.SF_FP32_BULK_DW)
    st.upload(inputs.z4_minkowski(n))
    assert torch.count_nonzero(st.rhs()).item() == 0


# ------------------------------------------------------------------ checkpoint / resume
@pytest.mark.parametrize("precision", [capi.SF_FP64, capi.SF_FP32_BULK_DW])
def test_checkpoint_resume_is_bitwise(tmp_path, precision):
    n = (20, 12, 10)
    U0, dx = inputs.z4_perturbed(n, seed=4, amp=0.03)
    a = PatchState(capi.SF_Z4, n, dx, 0.25 * min(dx), precision=precision)
    a.upload(U0)
    a.step(4)
    b = PatchState(capi.SF_Z4, n, dx, 0.25 * min(dx), precision=precision)
    b.upload(U0)
    b.step(2)
    path = str(tmp_path / "ckpt.npz")
    b.save(path, step=2, t=2 * b.dt)
    c, step, t = PatchState.load(path)
    assert step == 2 and t == pytest.approx(2 * b.dt)
    c.step(2)
    assert torch.equal(a.A, c.A)


# ------------------------------------------------------------------ TMA-staged CCZ4 kernel
# Float CCZ4 on the padded layout (row pitch 104 floats, ny = 96, nx a
# multiple of 32) runs the kernel that stages every field's halo box in
# shared memory with cp.async.bulk.tensor loads.  Same right-hand side, same
# float rounding bound against the oracle; against the global-load kernel on
# the dense layout the only differences come from FMA contraction.
# x_offset 0: the one-point TMA kernel; x_offset 1 (rows 4 bytes past a
# 16-byte boundary): the two-point kernel, every stencil and the algebra on
# f32x2 pairs, 32 x 16 tiles.
@pytest.mark.parametrize("x_offset", [0, 1])
@pytest.mark.parametrize("precision", [capi.SF_FP32_BULK, capi.SF_FP32_BULK_DW])
@pytest.mark.parametrize("nx,nz", [(32, 7), (96, 5)])
def test_z4_tma_kernel_matches_oracle(precision, nx, nz, x_offset):
    n = (nx, 96, nz)
    U0, dx = inputs.z4_perturbed(n, seed=4, amp=0.05)
    prm = capi.params()
    dt = 0.25 * min(dx)
    eps32 = float(np.finfo(np.float32).eps)
    bound = 4 * 64 / 12 * eps32 * dt / min(dx) ** 2 / 1e-2
    got = run_stages(capi.SF_Z4, U0, dx, dt, prm, precision=precision, pitch=104, x_offset=x_offset)
    dense = run_stages(capi.SF_Z4, U0, dx, dt, prm, precision=precision)
    want = oracle_stages(oracle.Z4, U0, dx, dt, prm)
    for s in range(4):
        e = rel_err(got[s], want[s], floor=1e-2)
        assert e.max() < bound, (s, e, bound)
        assert rel_err(got[s], dense[s], floor=1e-2).max() < bound


# Any patch size with 16-byte row pitch: the runtime-stride TMA kernel, whose
# 32 x 12 tiles overhang the patch in x and y.  Against the oracle with the
# float bound, and against the global-load kernel on a pitch that is not a
# multiple of 4 floats.
@pytest.mark.parametrize("precision", [capi.SF_FP32_BULK, capi.SF_FP32_BULK_DW])
@pytest.mark.parametrize("n", [(37, 13, 5), (20, 30, 4), (64, 12, 3)])
def test_z4_tma_any_size_matches_oracle(precision, n):
    U0, dx = inputs.z4_perturbed(n, seed=6, amp=0.05)
    prm = capi.params()
    dt = 0.25 * min(dx)
    eps32 = float(np.finfo(np.float32).eps)
    bound = 4 * 64 / 12 * eps32 * dt / min(dx) ** 2 / 1e-2
    row = n[0] + 6
    got = run_stages(capi.SF_Z4, U0, dx, dt, prm, precision=precision, pitch=(row + 3) // 4 * 4)
    dense = run_stages(capi.SF_Z4, U0, dx, dt, prm, precision=precision,
                       pitch=row + 1 if row % 4 == 0 else row)
    want = oracle_stages(oracle.Z4, U0, dx, dt, prm)
    for s in range(4):
        assert rel_err(got[s], want[s], floor=1e-2).max() < bound, s
        assert rel_err(got[s], dense[s], floor=1e-2).max() < bound, s


# Any patch size on the two-point layout (rows of a multiple of 4 floats with
# one float before each row): the two-point tile body with runtime strides and
# 32 x 16 tiles overhanging the patch, odd widths included.  Against the
# oracle with the float bound, and against the global-load kernel on dense rows.
@pytest.mark.parametrize("n", [(37, 13, 5), (48, 21, 4), (7, 40, 3)])
def test_z4_two_point_any_size_matches_oracle(n):
    U0, dx = inputs.z4_perturbed(n, seed=8, amp=0.05)
    prm = capi.params()
    dt = 0.25 * min(dx)
    eps32 = float(np.finfo(np.float32).eps)
    bound = 4 * 64 / 12 * eps32 * dt / min(dx) ** 2 / 1e-2
    got = run_stages(capi.SF_Z4, U0, dx, dt, prm, precision=capi.SF_FP32_BULK_DW,
                     pitch=(n[0] + 7 + 3) // 4 * 4, x_offset=1)
    dense = run_stages(capi.SF_Z4, U0, dx, dt, prm, precision=capi.SF_FP32_BULK_DW)
    want = oracle_stages(oracle.Z4, U0, dx, dt, prm)
    for s in range(4):
        assert rel_err(got[s], want[s], floor=1e-2).max() < bound, s
        assert rel_err(got[s], dense[s], floor=1e-2).max() < bound, s


@pytest.mark.parametrize("x_offset", [0, 1])
def test_z4_tma_kernel_frozen_shift_gauge_wave(x_offset):
    # harmonic slicing and a frozen shift: the last three fields' stencils are
    # never opened, so the staged sequence is 22 boxes long
    n = (32, 96, 6)
    U0, dx = inputs.z4_gauge_wave(n, amp=0.01)
    prm = capi.params(slicing=1, shift_frozen=1)
    dt = 0.25 * min(dx)
    eps32 = float(np.finfo(np.float32).eps)
    bound = 4 * 64 / 12 * eps32 * dt / min(dx) ** 2 / 1e-2
    got = run_stages(capi.SF_Z4, U0, dx, dt, prm, precision=capi.SF_FP32_BULK_DW, pitch=104,
                     x_offset=x_offset)
    want = oracle_stages(oracle.Z4, U0, dx, dt, prm)
    assert rel_err(got[3], want[3], floor=1e-2).max() < bound


@pytest.mark.parametrize("x_offset", [0, 1])
def test_z4_tma_kernel_full_size_sampled(x_offset):
    # the benchmark's launch configuration (96^3, FP32-bulk with double-word
    # islands, row pitch 104, one float before each row's first ghost point
    # for the two-point kernel): sampled points of the RHS against the oracle.
    # Stored float values carry |U - U_flat| <= 0.05 here (flat-space offsets),
    # so a 1/dx^2 stencil holds ~64 eps32 * 0.05 / (12 dx^2) of rounding.
    n = (96, 96, 96)
    U0, dx = inputs.z4_minkowski_noise(n, seed=0, amp=1e-10)
    pert, _ = inputs.z4_perturbed(n, seed=7, amp=0.05)
    U0 = U0 + (pert - inputs.z4_minkowski(n))
    prm = capi.params()
    st = PatchState(capi.SF_Z4, n, dx, 0.25 * dx[0], precision=capi.SF_FP32_BULK_DW, prm=prm,
                    x_pitch=104, x_offset=x_offset)
    st.upload(U0)
    r = st.rhs().cpu().numpy().reshape(25, -1).astype(np.float64)
    pts = inputs.observers(n, 2000, seed=13)
    want = oracle.rhs_points(oracle.Z4, oracle.ghosted(U0), dx, pts, oracle_params(prm))
    eps32 = float(np.finfo(np.float32).eps)
    dev = np.abs(U0 - inputs.z4_minkowski(n)).max()
    bound = 4 * 64 / 12 * eps32 * dev / dx[0] ** 2
    for f in range(25):
        err = np.abs(r[f, pts] - want[f]).max()
        assert err < bound, (f, err, bound)
