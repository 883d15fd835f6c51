"""Sub-cycling in time on the GPU: Berger-Oliger without order reduction
(Sec. III.B, App. C dense output, App. D) fused with the quintic
prolongation (``sf_bor_prolong``), and the two-level loop built on it
(``amr.SubcycledPair``).

* sf_bor_prolong against the oracle: the oracle takes the coarse increments
  k_j = dt L(U^(j)) from its own right-hand side and follows App. D step by
  step at every coarse node, then prolongs; the GPU derives k_j from the
  stored stage states.  Both in FP64: agreement to 1e-12 of the data scale.
* Ratio 1: the BOR stages are then the coarse RK4 stages themselves, so a
  fine patch at the coarse resolution evolves exactly as the same box of a
  uniform run (to rounding), for the linear wave and the nonlinear CCZ4
  system.
* Ratio 2: the sub-cycled composite solution of a smooth plane wave
  converges to the exact solution at 4th order (the paper's Sec. IV.A
  result for BOR).
"""
import math

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


def _oracle_states_and_ks(system, U0, dx, dt, rk):
    """Ghosted coarse stage states and increments from the oracle."""
    U = oracle.ghosted(U0)
    Uw = U.copy()
    if rk == capi.SF_RK4:
        st = oracle.rk4_step(system, Uw, dx, dt, stages=True)
        ins = [U0, st[0], st[1], st[2]]
    else:
        st = oracle.ssprk3_step(system, Uw, dx, dt, stages=True)
        ins = [U0, st[0], st[1]]
    states = [U0] + list(st)
    ks = [oracle.ghosted(dt * oracle.rhs(system, oracle.ghosted(np.ascontiguousarray(S)), dx))
          for S in ins]
    return states, np.array(ks)


@pytest.mark.parametrize("rk", [capi.SF_RK4, capi.SF_SSPRK3])
@pytest.mark.parametrize("R", [2, 3])
def test_bor_prolong_matches_oracle(rk, R):
    n = (10, 9, 8)
    system = capi.SF_WAVE
    U0, dx = inputs.wave_plane(n, seed=1)
    U0 = U0 + 0.05 * inputs.wave_noise(n, seed=2)
    dt = 0.25 * min(dx)
    states, ks = _oracle_states_and_ks(system, U0, dx, dt, rk)
    s = 4 if rk == capi.SF_RK4 else 3
    prm = capi.params(rk=rk)
    arrs = []
    for S in states:
        st = PatchState(system, n, dx, dt, prm=prm)
        st.upload(np.ascontiguousarray(S))
        arrs.append(st)
    origin, ext = (R * 2 - 1, R + 1, R * 3), (R * 5 + 2, R * 4, R * 2 + 1)
    Ung = oracle.ghosted(np.ascontiguousarray(states[0]))
    scale = np.abs(Ung).max()
    out = torch.zeros((5, ext[2], ext[1], ext[0]), dtype=torch.float64, device="cuda")
    a0 = arrs[0]
    for r in range(R):
        want_all = oracle.bor_fine_stages(rk, Ung, ks, dt, R, r)
        for stage in range(s + 1):
            capi.sf_bor_prolong(a0.patch(a0.A, a0.A, a0.B), rk, [a.A.data_ptr() for a in arrs], 5, R, r,
                                stage, origin, ext, out.data_ptr(), ext[0], ext[0] * ext[1],
                                ext[0] * ext[1] * ext[2])
            want = oracle.prolong(np.ascontiguousarray(want_all[stage]), R, origin, ext)
            got = out.cpu().numpy()
            err = np.abs(got - want).max()
            assert err <= 1e-12 * scale, (r, stage, err)


def test_bor_prolong_rejects_bad_arguments():
    st = PatchState(capi.SF_WAVE, (8, 8, 8), (0.1,) * 3, 0.01)
    out = torch.zeros(5 * 8, dtype=torch.float64, device="cuda")
    ptrs = [st.A.data_ptr()] * 5
    p = st.patch(st.A, st.A, st.B)
    with pytest.raises(capi.SfError, match="fine step"):
        capi.sf_bor_prolong(p, capi.SF_RK4, ptrs, 5, 2, 2, 0, (4, 4, 4), (2, 2, 2), out.data_ptr(), 2, 4, 8)
    with pytest.raises(capi.SfError, match="stage"):
        capi.sf_bor_prolong(p, capi.SF_SSPRK3, ptrs, 5, 2, 0, 4, (4, 4, 4), (2, 2, 2), out.data_ptr(), 2, 4, 8)
    with pytest.raises(capi.SfError, match="NULL"):
        capi.sf_bor_prolong(p, capi.SF_RK4, ptrs[:4] + [None], 5, 2, 0, 0, (4, 4, 4), (2, 2, 2),
                            out.data_ptr(), 2, 4, 8)


def _pitch(n, pitch4):
    """Row pitch: 16-byte rows (the TMA-staged float CCZ4 kernel) or dense."""
    return (n[0] + 6 + 3) // 4 * 4 if pitch4 else None


def _pair(system, precision, nc, nf_coarse, at, R, data, dt_factor, steps, pitch4=False):
    """Run a SubcycledPair; returns (pair, coarse dx, coarse dt)."""
    U0c, dxc = data(nc)
    dtc = dt_factor * min(dxc)
    prm = capi.params()
    coarse = PatchState(system, nc, dxc, dtc, precision=precision, prm=prm,
                        x_pitch=_pitch(nc, pitch4))
    coarse.upload(U0c)
    nfine = tuple(R * v for v in nf_coarse)
    dxf = tuple(v / R for v in dxc)
    fine = PatchState(system, nfine, dxf, dtc / R, precision=precision,
                      prm=capi.params(ghosts=capi.SF_GHOSTS_NONE), x_pitch=_pitch(nfine, pitch4))
    Uf_all, _ = data(tuple(R * v for v in nc))
    sub = Uf_all[:, R * at[2]:R * at[2] + nfine[2], R * at[1]:R * at[1] + nfine[1],
                 R * at[0]:R * at[0] + nfine[0]]
    fine.upload(np.ascontiguousarray(sub))
    pair = amr.SubcycledPair(coarse, fine, R, at)
    pair.step(steps)
    torch.cuda.synchronize()
    return pair


@pytest.mark.parametrize("at", [(4, 3, 3), (2, 3, 3)])
@pytest.mark.parametrize("system,data", [
    (capi.SF_WAVE, lambda n: inputs.wave_plane(n, seed=3)),
    (capi.SF_Z4, lambda n: inputs.z4_perturbed(n, seed=3, amp=0.04)),
])
def test_ratio_one_equals_uniform_run(system, data, at):
    # at x = 2 the restriction writes inside the 3 layers whose periodic
    # images are coarse ghosts, so the step refreshes them; at x = 4 it does not
    nc, m = (16, 14, 12), (8, 7, 6)
    steps = 3
    pair = _pair(system, capi.SF_FP64, nc, m, at, 1, data, 0.2, steps)
    U0, dx = data(nc)
    whole = PatchState(system, nc, dx, 0.2 * min(dx))
    whole.upload(U0)
    whole.step(steps)
    torch.cuda.synchronize()
    W = whole.fields().cpu().numpy()
    want = W[:, at[2]:at[2] + m[2], at[1]:at[1] + m[1], at[0]:at[0] + m[0]]
    got = pair.fine.fields().cpu().numpy()
    for f in range(W.shape[0]):
        scale = max(np.abs(W[f] - np.round(W[f].mean())).max(), 1e-3)
        err = np.abs(got[f] - want[f]).max()
        assert err <= 1e-11 * scale, (f, err, scale)
    # the coarse level, fine values injected back, equals the uniform run too
    np.testing.assert_allclose(pair.coarse.fields().cpu().numpy(), W, rtol=0, atol=1e-11 * np.abs(W).max())


def test_ratio_one_equals_uniform_run_float_tma():
    # FP32-bulk CCZ4 on 16-byte rows (the TMA-staged kernel on both levels and
    # for the uniform run), ratio 1: the fine patch follows the uniform run to
    # float rounding of the 1/dx^2 stencils, accumulated over 3 steps
    data = lambda n: inputs.z4_perturbed(n, seed=3, amp=0.04)
    nc, at, m = (16, 14, 12), (4, 3, 3), (8, 7, 6)
    steps = 3
    pair = _pair(capi.SF_Z4, capi.SF_FP32_BULK_DW, nc, m, at, 1, data, 0.2, steps, pitch4=True)
    U0, dx = data(nc)
    whole = PatchState(capi.SF_Z4, nc, dx, 0.2 * min(dx), precision=capi.SF_FP32_BULK_DW,
                       x_pitch=_pitch(nc, True))
    whole.upload(U0)
    whole.step(steps)
    torch.cuda.synchronize()
    W = whole.fields().cpu().numpy()
    want = W[:, at[2]:at[2] + m[2], at[1]:at[1] + m[1], at[0]:at[0] + m[0]]
    got = pair.fine.fields().cpu().numpy()
    eps32 = float(np.finfo(np.float32).eps)
    bound = 2 * steps * 4 * 64 / 12 * eps32 * 0.2 * min(dx) / min(dx) ** 2
    assert np.abs(got - want).max() <= bound, (np.abs(got - want).max(), bound)


def test_subcycled_graph_replay_equals_steps():
    # the captured coarse step (stages, BOR ghost fills, copies, restriction
    # in one CUDA graph) advances the pair exactly as step() does
    data = lambda n: inputs.z4_perturbed(n, seed=5, amp=0.04)
    nc, at, m, R = (24, 20, 16), (6, 5, 4), (8, 6, 4), 2
    pairs = [_pair(capi.SF_Z4, capi.SF_FP32_BULK_DW, nc, m, at, R, data, 0.2, 1, pitch4=True)
             for _ in range(2)]
    pairs[0].step(2)
    pairs[1].capture(1)
    pairs[1].replay()
    pairs[1].replay()
    torch.cuda.synchronize()
    for a, b in zip((pairs[0].coarse, pairs[0].fine), (pairs[1].coarse, pairs[1].fine)):
        assert torch.equal(a.A, b.A)


def test_subcycled_two_point_layout_matches_one_point():
    # both levels on the layout of the two-point float CCZ4 kernel (rows of
    # 104 floats, one float before each row, planes of 102 rows) against the
    # same pair on 16-byte rows (the one-point TMA kernel): the two kernels
    # differ only in rounding order, so the levels agree to the float bound
    # of the stage tests, per stage taken
    data = lambda n: inputs.z4_perturbed(n, seed=7, amp=0.04)
    nc, at, m, R, steps = (32, 32, 12), (8, 8, 3), (16, 16, 6), 2, 2
    one = _pair(capi.SF_Z4, capi.SF_FP32_BULK_DW, nc, m, at, R, data, 0.2, steps, pitch4=True)
    U0c, dxc = data(nc)
    dtc = 0.2 * min(dxc)
    lay = dict(x_pitch=104, x_offset=1, plane_rows=102)
    coarse = PatchState(capi.SF_Z4, nc, dxc, dtc, precision=capi.SF_FP32_BULK_DW, **lay)
    coarse.upload(U0c)
    nfine = tuple(R * v for v in m)
    fine = PatchState(capi.SF_Z4, nfine, tuple(v / R for v in dxc), dtc / R,
                      precision=capi.SF_FP32_BULK_DW, prm=capi.params(ghosts=capi.SF_GHOSTS_NONE),
                      **lay)
    Uf_all, _ = data(tuple(R * v for v in nc))
    fine.upload(np.ascontiguousarray(Uf_all[:, R * at[2]:R * at[2] + nfine[2],
                                            R * at[1]:R * at[1] + nfine[1],
                                            R * at[0]:R * at[0] + nfine[0]]))
    two = amr.SubcycledPair(coarse, fine, R, at)
    c0 = capi.sf_launch_count()
    two.step(steps)
    torch.cuda.synchronize()
    eps32 = float(np.finfo(np.float32).eps)
    per_stage = 64 / 12 * eps32 * dtc / min(dxc) ** 2 / 1e-2
    # 4 coarse and 4 R fine stages a step, the fine ones at R times dt / dx^2
    bound = 2 * steps * 4 * (1 + R * R) * per_stage
    for a, b in ((one.coarse, two.coarse), (one.fine, two.fine)):
        x, y = a.fields().cpu().numpy(), b.fields().cpu().numpy()
        for f in range(25):
            scale = max(np.abs(x[f]).max(), 1e-2)
            assert np.abs(x[f] - y[f]).max() / scale < bound, (f, bound)
    assert capi.sf_launch_count() - c0 > 0


def test_subcycled_plane_wave_converges_at_fourth_order():
    R = 2
    errs = []
    for N in (16, 32):
        data = lambda n: inputs.wave_plane(n, k=(1, 1, 0))
        nc = (N, N, N)
        at = (N // 4, N // 4, N // 4)
        m = (N // 2, N // 2, N // 2)
        T = 0.25
        steps = int(round(T / (0.25 / N)))
        pair = _pair(capi.SF_WAVE, capi.SF_FP64, nc, m, at, R, data, 0.25, steps)
        t = steps * pair.coarse.dt
        Uf_exact, _ = inputs.wave_plane(tuple(R * v for v in nc), k=(1, 1, 0), t=t)
        fe = Uf_exact[0, R * at[2]:R * at[2] + R * m[2], R * at[1]:R * at[1] + R * m[1],
                      R * at[0]:R * at[0] + R * m[0]]
        Uc_exact, _ = inputs.wave_plane(nc, k=(1, 1, 0), t=t)
        e_f = np.abs(pair.fine.fields().cpu().numpy()[0] - fe).max()
        e_c = np.abs(pair.coarse.fields().cpu().numpy()[0] - Uc_exact[0]).max()
        errs.append(max(e_f, e_c))
    order = math.log2(errs[0] / errs[1])
    assert 3.5 < order < 4.8, (errs, order)


def test_bor_prolong_boxes_equals_single_box_calls():
    # several boxes in one launch give the same values as one call per box
    n = (10, 9, 8)
    R = 2
    U0, dx = inputs.wave_plane(n, seed=5)
    st = PatchState(capi.SF_WAVE, n, dx, 0.01)
    st.upload(U0)
    arrs = [st.A, st.B, st.C, st.D, st.A]
    for a_ in (st.B, st.C, st.D):
        a_.copy_(st.A * 1.01)
    ptrs = [a_.data_ptr() for a_ in arrs]
    specs = [((R * 2 - 1, R + 1, R * 3), (7, 5, 3)), ((0, 0, 0), (12, 2, 4)), ((3, 5, 2), (1, 1, 1)),
             ((1, 2, 3), (0, 4, 4))]
    outs_a = [torch.zeros((5,) + tuple(reversed(e)), dtype=torch.float64, device="cuda") for _, e in specs]
    outs_b = [torch.zeros_like(o) for o in outs_a]
    p = st.patch(st.A, st.A, st.B)
    boxes = []
    for (o, e), oa in zip(specs, outs_a):
        boxes.append(capi.prolong_box(o, e, oa.data_ptr(), e[0], e[0] * e[1], e[0] * e[1] * e[2]))
    capi.sf_bor_prolong_boxes(p, capi.SF_RK4, ptrs, 5, R, 1, 2, boxes)
    for (o, e), ob in zip(specs, outs_b):
        capi.sf_bor_prolong(p, capi.SF_RK4, ptrs, 5, R, 1, 2, o, e, ob.data_ptr(), e[0], e[0] * e[1],
                            e[0] * e[1] * e[2])
    torch.cuda.synchronize()
    for oa, ob in zip(outs_a, outs_b):
        assert torch.equal(oa, ob)
