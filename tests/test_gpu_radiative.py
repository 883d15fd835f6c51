"""Radiative boundary condition (Sec. V) on the GPU: sf_radiative_substep on
the ghost shell together with sf_substep on the interior, on the puncture
initial data of Sec. V, against the oracle's RK4 step with radiative ghost
points (every stage, every point including the ghosts).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1806_04182_gb300 import amr, build, capi, inputs
from paper_1806_04182_gb300.state import PatchState

pytestmark = pytest.mark.gpu
SPEED = np.ones(25)


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    build.build()
    return capi.lib()


def ghosted_fields(st, arr):
    """Field values of a full ghosted array (flat-space offsets added back)."""
    nx = st.n[0] + 2 * st.g
    v = arr[:, :, :, :nx].double().clone()
    for f in st.offset_fields:
        v[f] += 1.0
    return v.cpu().numpy()


def run(n, precision, steps=1, length=6.0, pitch=None):
    U, dx, x0 = inputs.z4_puncture(n, length=length, ghost=3)
    dt = 0.25 * min(dx)
    st = PatchState(capi.SF_Z4, n, dx, dt, precision=precision,
                    prm=capi.params(ghosts=capi.SF_GHOSTS_NONE), x_pitch=pitch)
    st.upload_ghosted(U)
    outs = []
    h = torch.cuda.current_stream().cuda_stream
    for _ in range(steps):
        for s in range(4):
            p = st.stage_patch(s)
            capi.sf_substep(st.prm, p, s, h)
            capi.sf_radiative_substep(st.prm, p, x0, inputs.Z4_UINF, SPEED, s, h)
            outs.append(ghosted_fields(st, st.roles(s)[1]))
    torch.cuda.synchronize()
    return U, dx, x0, dt, outs


def rel(got, want, floor):
    return np.array([np.abs(got[f] - want[f]).max() / max(np.abs(want[f]).max(), floor)
                     for f in range(want.shape[0])])


def test_puncture_step_matches_oracle_fp64():
    n = (16, 14, 12)
    U, dx, x0, dt, outs = run(n, capi.SF_FP64)
    W = np.ascontiguousarray(U)
    st = oracle.rk4_step_radiative(oracle.Z4, W, dx, x0, inputs.Z4_UINF, SPEED, dt, stages=True)
    for s in range(4):
        e = rel(outs[s], st[s], 1e-2)
        assert e.max() < 1e-12, (s, e)


def test_puncture_step_float_bulk():
    # float storage: the bound of the periodic FP32 tests, 4 x 64/12 eps32 dt/dx^2
    n = (32, 24, 16)
    U, dx, x0, dt, outs = run(n, capi.SF_FP32_BULK_DW, length=8.0)
    W = np.ascontiguousarray(U)
    st = oracle.rk4_step_radiative(oracle.Z4, W, dx, x0, inputs.Z4_UINF, SPEED, dt, stages=True)
    eps32 = float(np.finfo(np.float32).eps)
    bound = 4 * 64 / 12 * eps32 * dt / min(dx) ** 2 / 1e-2
    e = rel(outs[3], st[3], 1e-2)
    assert e.max() < max(bound, 1e-5), (e, bound)


def test_puncture_tma_layout_matches_dense():
    # the padded layout runs the TMA-staged interior kernel; the ghost shell
    # goes through the same radiative kernel
    n = (32, 96, 6)
    _, _, _, _, a = run(n, capi.SF_FP32_BULK_DW, length=8.0, pitch=104)
    _, _, _, _, b = run(n, capi.SF_FP32_BULK_DW, length=8.0)
    eps32 = float(np.finfo(np.float32).eps)
    for s in range(4):
        assert rel(a[s], b[s], 1e-2).max() < 1e-4


def test_puncture_evolution_stays_finite():
    n = (48, 48, 48)
    U, dx, x0 = inputs.z4_puncture(n, length=8.0, ghost=3)
    st = PatchState(capi.SF_Z4, n, dx, 0.25 * min(dx), precision=capi.SF_FP64,
                    prm=capi.params(ghosts=capi.SF_GHOSTS_NONE, check_finite=1))
    st.upload_ghosted(U)
    st.step_radiative(40, x0, inputs.Z4_UINF, SPEED)
    assert capi.sf_get_device_status() == capi.SF_OK
    A = ghosted_fields(st, st.A)
    assert np.all(np.isfinite(A))
    # the outer shell stays close to flat space (the hole has mass 1 at the
    # centre of an 8^3 box: chi ~ (1 + 1/(2r))^-4 there)
    assert np.abs(A[0, 0] - 1).max() < 0.6


def test_rejects_periodic_ghost_mode():
    n = (8, 8, 8)
    st = PatchState(capi.SF_Z4, n, (0.1,) * 3, 0.01)
    with pytest.raises(capi.SfError, match="SF_GHOSTS_NONE"):
        capi.sf_radiative_substep(st.prm, st.stage_patch(0), (0, 0, 0), inputs.Z4_UINF, SPEED, 0)
    st2 = PatchState(capi.SF_Z4, n, (0.1,) * 3, 0.01, prm=capi.params(ghosts=capi.SF_GHOSTS_NONE))
    with pytest.raises(capi.SfError, match="speed"):
        capi.sf_radiative_substep(st2.prm, st2.stage_patch(0), (0, 0, 0), inputs.Z4_UINF,
                                  -SPEED, 0)


def test_fixed_refinement_ratio_one_equals_single_level():
    # a puncture box with radiative boundaries carrying a fine patch at the
    # same resolution around the hole (ratio 1): the BOR ghost values are then
    # the coarse stage values, so the fine patch evolves as the same region of
    # the single-level run
    n = (20, 20, 20)
    U, dx, x0 = inputs.z4_puncture(n, length=6.0, ghost=3)
    dt = 0.25 * min(dx)
    prm = capi.params(ghosts=capi.SF_GHOSTS_NONE)
    whole = PatchState(capi.SF_Z4, n, dx, dt, prm=prm)
    whole.upload_ghosted(U)
    whole.step_radiative(3, x0, inputs.Z4_UINF, SPEED)
    coarse = PatchState(capi.SF_Z4, n, dx, dt, prm=prm)
    coarse.upload_ghosted(U)
    at, m = (6, 6, 6), (8, 8, 8)
    fine = PatchState(capi.SF_Z4, m, dx, dt, prm=prm)
    g = 3
    fine.upload_ghosted(np.ascontiguousarray(U[:, at[2]:at[2] + m[2] + 2 * g,
                                               at[1]:at[1] + m[1] + 2 * g,
                                               at[0]:at[0] + m[0] + 2 * g]))
    pair = amr.SubcycledPair(coarse, fine, 1, at, coarse_radiative=(x0, inputs.Z4_UINF, SPEED))
    pair.step(3)
    torch.cuda.synchronize()
    W = whole.fields().cpu().numpy()
    want = W[:, at[2]:at[2] + m[2], at[1]:at[1] + m[1], at[0]:at[0] + m[0]]
    got = pair.fine.fields().cpu().numpy()
    assert rel(got, want, 1e-2).max() < 1e-11
    assert rel(pair.coarse.fields().cpu().numpy(), W, 1e-2).max() < 1e-11


def test_fixed_refinement_puncture_ratio_two_runs():
    # coarse 32^3 box (radiative boundary) with a ratio-2 fine patch of 32^3
    # around the hole (fine point 2 i on coarse point i + at): every value
    # stays finite over 6 coarse steps, and the fine solution, injected back,
    # agrees with the coarse one where the coarse grid resolves the data
    nc = (32, 32, 32)
    U, dx, x0 = inputs.z4_puncture(nc, length=8.0, ghost=3)
    prm = capi.params(ghosts=capi.SF_GHOSTS_NONE, check_finite=1)
    coarse = PatchState(capi.SF_Z4, nc, dx, 0.25 * dx[0], prm=prm)
    coarse.upload_ghosted(U)
    at, m = (8, 8, 8), (32, 32, 32)
    dxf = tuple(v / 2 for v in dx)
    x0f = tuple(x0[d] + at[d] * dx[d] for d in range(3))
    g = 3
    ax = [x0f[d] + dxf[d] * np.arange(-g, m[d] + g) for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    fine = PatchState(capi.SF_Z4, m, dxf, 0.125 * dx[0], prm=prm)
    fine.upload_ghosted(inputs.z4_puncture_at(X, Y, Z))
    pair = amr.SubcycledPair(coarse, fine, 2, at, coarse_radiative=(x0, inputs.Z4_UINF, SPEED))
    pair.step(6)
    torch.cuda.synchronize()
    assert capi.sf_get_device_status() == capi.SF_OK
    F = pair.fine.fields().cpu().numpy()
    C = pair.coarse.fields().cpu().numpy()
    assert np.all(np.isfinite(F)) and np.all(np.isfinite(C))
    # injection: coarse points under the fine patch hold the fine values
    np.testing.assert_array_equal(C[:, at[2]:at[2] + 16, at[1]:at[1] + 16, at[0]:at[0] + 16],
                                  F[:, ::2, ::2, ::2])
