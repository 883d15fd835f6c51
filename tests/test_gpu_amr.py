"""Inter-patch operations of the AMR level loop on the GPU.

* Same-level synchronisation: a periodic box split into 2 x 2 x 1 patches
  that exchange ghost shells with sf_copy_boxes between stages must give,
  bit for bit, the state of the undecomposed periodic run (the substep is a
  pure function of its ghosted input, and both runs use the same kernels).
* The same level as one sf_batch with the halo copies registered per buffer
  role (amr.level_batch), stepped through its captured graph: equal to the
  undecomposed run to rounding (the batch runs its own kernel instances).
* Prolongation (sf_prolong) against the oracle's Lagrange interpolation;
  restriction (sf_copy_boxes with src_step = R) against the oracle's
  injection, bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1806_04182_gb300 import amr, build, capi, inputs
from paper_1806_04182_gb300.state import PatchState

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    build.build()
    return capi.lib()


CASES = [
    (capi.SF_WAVE, capi.SF_FP64, lambda n: inputs.wave_plane(n, seed=2)),
    (capi.SF_Z4, capi.SF_FP64, lambda n: inputs.z4_perturbed(n, seed=2, amp=0.04)),
    (capi.SF_Z4, capi.SF_FP32_BULK_DW, lambda n: inputs.z4_perturbed(n, seed=2, amp=0.04)),
    (capi.SF_MHD, capi.SF_FP64, lambda n: inputs.mhd_blast(n, seed=2, radius=0.3)),
]


@pytest.mark.parametrize("system,precision,data", CASES)
def test_decomposed_run_equals_undecomposed(system, precision, data):
    N = (32, 24, 20)
    parts = (2, 2, 1)
    m = tuple(N[a] // parts[a] for a in range(3))
    U0, dx = data(N)
    rk = capi.SF_SSPRK3 if system == capi.SF_MHD else capi.SF_RK4
    dt = 0.2 * min(dx) if system != capi.SF_MHD else 1e-3
    whole = PatchState(system, N, dx, dt, precision=precision, prm=capi.params(rk=rk))
    whole.upload(U0)
    whole.step(2)
    prm_none = capi.params(rk=rk, ghosts=capi.SF_GHOSTS_NONE)
    grid = {}
    for a in range(parts[0]):
        for b in range(parts[1]):
            for c in range(parts[2]):
                st = PatchState(system, m, dx, dt, precision=precision, prm=prm_none)
                sub = U0[:, c * m[2]:(c + 1) * m[2], b * m[1]:(b + 1) * m[1], a * m[0]:(a + 1) * m[0]]
                st.upload(np.ascontiguousarray(sub))
                grid[(a, b, c)] = st
    h = torch.cuda.current_stream().cuda_stream
    capi.sf_copy_boxes(amr.halo_boxes(grid, "A"), precision, h)
    any_st = next(iter(grid.values()))
    for _ in range(2):
        for s in range(any_st.nstages):
            for st in grid.values():
                capi.sf_substep(st.prm, st.stage_patch(s), s, h)
            out_name = {id(any_st.A): "A", id(any_st.B): "B", id(any_st.C): "C"}[id(any_st.roles(s)[1])]
            capi.sf_copy_boxes(amr.halo_boxes(grid, out_name), precision, h)
    torch.cuda.synchronize()
    W = whole.interior().cpu().numpy()
    for (a, b, c), st in grid.items():
        part = W[:, c * m[2]:(c + 1) * m[2], b * m[1]:(b + 1) * m[1], a * m[0]:(a + 1) * m[0]]
        np.testing.assert_array_equal(st.interior().cpu().numpy(), part)


@pytest.mark.parametrize("system,precision,data", CASES[:3])
def test_level_batch_with_halo_equals_undecomposed(system, precision, data):
    # float CCZ4 on 16-byte rows: the parts go to the batch's TMA-staged
    # tiles, the whole patch to the TMA-staged kernel of sf_substep
    N, parts, steps = (32, 24, 20), (2, 2, 1), 2
    m = tuple(N[a] // parts[a] for a in range(3))
    pitch = (lambda n: (n[0] + 6 + 3) // 4 * 4) if precision != capi.SF_FP64 else (lambda n: None)
    U0, dx = data(N)
    dt = 0.2 * min(dx)
    whole = PatchState(system, N, dx, dt, precision=precision, x_pitch=pitch(N))
    whole.upload(U0)
    whole.step(steps)
    grid = {}
    for a in range(parts[0]):
        for b in range(parts[1]):
            st = PatchState(system, m, dx, dt, precision=precision,
                            prm=capi.params(ghosts=capi.SF_GHOSTS_NONE), x_pitch=pitch(m))
            st.upload(np.ascontiguousarray(U0[:, :, b * m[1]:(b + 1) * m[1], a * m[0]:(a + 1) * m[0]]))
            grid[(a, b, 0)] = st
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    batch = amr.level_batch(grid)
    try:
        plain = amr.level_batch(grid)  # the same patches without halo lists
        for role in range(3):
            capi.sf_batch_set_halo(plain, role, [])
        # one copy launch per stage (4 patches x 26 boxes < 256)
        assert capi.sf_batch_launches_per_step(batch) == capi.sf_batch_launches_per_step(plain) + 4
        capi.sf_batch_destroy(plain)
        with torch.cuda.stream(stream):
            capi.sf_copy_boxes(amr.halo_boxes(grid, "A"), precision, stream.cuda_stream)
            capi.sf_batch_capture(batch, stream.cuda_stream)
            for _ in range(steps):
                capi.sf_batch_launch(batch, stream.cuda_stream)
        stream.synchronize()
        assert capi.sf_get_device_status() == capi.SF_OK
    finally:
        capi.sf_batch_destroy(batch)
    W = whole.interior().cpu().numpy()
    h = min(dx)
    eps32 = float(np.finfo(np.float32).eps)
    for (a, b, _), st in grid.items():
        want = W[:, :, b * m[1]:(b + 1) * m[1], a * m[0]:(a + 1) * m[0]]
        got = st.interior().cpu().numpy()
        for f in range(W.shape[0]):
            scale = max(np.abs(want[f]).max(), 1e-2)
            err = np.abs(got[f] - want[f]).max() / scale
            # FP64: summation order; float: the float rounding of the 1/dx^2
            # stencils over dt per stage, 4 stages per step, against the floor
            bound = 1e-13 if precision == capi.SF_FP64 else \
                2 * steps * 4 * 64 / 12 * eps32 * dt / h ** 2 / 1e-2
            assert err < bound, (a, b, f, err, bound)


def test_level_batch_rejects_bad_halo_lists():
    st = PatchState(capi.SF_WAVE, (8, 8, 8), (0.1,) * 3, 0.01, prm=capi.params(ghosts=capi.SF_GHOSTS_NONE))
    grid = {(0, 0, 0): st}
    b = amr.level_batch(grid)
    try:
        with pytest.raises(capi.SfError, match="role"):
            capi.sf_batch_set_halo(b, 3, [])
        bad = amr.halo_boxes(grid, "A")[:1]
        bad[0].nf = 0
        with pytest.raises(capi.SfError, match="nf"):
            capi.sf_batch_set_halo(b, 0, bad)
    finally:
        capi.sf_batch_destroy(b)
    periodic = PatchState(capi.SF_WAVE, (8, 8, 8), (0.1,) * 3, 0.01)
    with pytest.raises(ValueError, match="GHOSTS_NONE"):
        amr.level_batch({(0, 0, 0): periodic})


@pytest.mark.parametrize("R", [2, 3, 4])
def test_prolongation_matches_oracle(R):
    n = (10, 9, 8)
    rng = np.random.default_rng(R)
    Uc = rng.standard_normal((5, n[2], n[1], n[0]))
    st = PatchState(capi.SF_WAVE, n, (0.1, 0.1, 0.1), 0.01)
    st.upload(Uc)
    origin, ext = (R * 2 - 1, R * 1 + 1, R * 3), (R * 5 + 2, R * 4, R * 2 + 1)
    out = torch.zeros((5, ext[2], ext[1], ext[0]), dtype=torch.float64, device="cuda")
    capi.sf_prolong(st.patch(st.A, st.A, st.B), st.A.data_ptr(), 5, R, origin, ext,
                    out.data_ptr(), ext[0], ext[0] * ext[1], ext[0] * ext[1] * ext[2])
    want = oracle.prolong(oracle.ghosted(Uc), R, origin, ext)
    got = out.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    # coincident fine points are exact injections
    off = [(-o) % R for o in origin]
    np.testing.assert_array_equal(got[:, off[2]::R, off[1]::R, off[0]::R],
                                  want[:, off[2]::R, off[1]::R, off[0]::R])


@pytest.mark.parametrize("R", [2, 3])
def test_prolongation_float_arrays(R):
    # float arrays interpolate in float: the weights of each 1D set sum to one
    # and |l_j| <= 1.6, so the result carries <= ~(1.6^3 + 1) ulps of max |U|
    n = (10, 9, 8)
    rng = np.random.default_rng(10 + R)
    Uc = rng.standard_normal((25, n[2], n[1], n[0]))
    st = PatchState(capi.SF_Z4, n, (0.1, 0.1, 0.1), 0.01, precision=capi.SF_FP32_BULK)
    st.upload(Uc)
    origin, ext = (R * 2 - 1, R * 1 + 1, R * 3), (R * 5 + 2, R * 4, R * 2 + 1)
    out = torch.zeros((25, ext[2], ext[1], ext[0]), dtype=torch.float32, device="cuda")
    capi.sf_prolong(st.patch(st.A, st.A, st.B), st.A.data_ptr(), 25, R, origin, ext,
                    out.data_ptr(), ext[0], ext[0] * ext[1], ext[0] * ext[1] * ext[2])
    # the oracle sees the stored float values (flat-space offsets included)
    stored = st.interior().double().cpu().numpy()
    want = oracle.prolong(oracle.ghosted(stored), R, origin, ext)
    got = out.double().cpu().numpy()
    eps32 = float(np.finfo(np.float32).eps)
    assert np.abs(got - want).max() <= 8 * eps32 * np.abs(stored).max()


def test_prolongation_rejects_stencil_outside_coarse_box():
    st = PatchState(capi.SF_WAVE, (6, 6, 6), (0.1,) * 3, 0.01)
    out = torch.zeros(5 * 8, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.SfError, match="leaves the coarse box"):
        capi.sf_prolong(st.patch(st.A, st.A, st.B), st.A.data_ptr(), 5, 2, (12, 0, 0), (2, 2, 2),
                        out.data_ptr(), 2, 4, 8)


@pytest.mark.parametrize("R", [2, 3])
def test_restriction_by_injection(R):
    nc = (6, 5, 4)
    nfine = tuple(R * v for v in nc)
    rng = np.random.default_rng(7)
    Uf = rng.standard_normal((5, nfine[2], nfine[1], nfine[0]))
    fine = PatchState(capi.SF_WAVE, nfine, (0.1,) * 3, 0.01)
    fine.upload(Uf)
    coarse = PatchState(capi.SF_WAVE, nc, (0.1,) * 3, 0.01)
    origin, ext = (1, 0, 1), (4, 5, 3)
    capi.sf_copy_boxes([amr.restrict_box(fine, coarse, R, origin, ext)], capi.SF_FP64)
    torch.cuda.synchronize()
    want = oracle.restrict(oracle.ghosted(Uf), R, origin, ext)
    got = coarse.interior().cpu().numpy()[:, origin[2]:origin[2] + ext[2],
                                          origin[1]:origin[1] + ext[1], origin[0]:origin[0] + ext[0]]
    np.testing.assert_array_equal(got, want)
