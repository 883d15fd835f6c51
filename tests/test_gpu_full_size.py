"""Parity at the full sizes of the benchmarked workloads, in the launch
configurations bench.py times (the 96^3 CCZ4 patch and the 128^3 adjoint have
their own full-size tests in test_gpu_parity.py and test_gpu_adjoint.py):

* wave, 64^3 FP64, one RK4 step: every point against the oracle's step;
* MHD, 128^3 blast data (WENO5 + LLF, SSP-RK3, dt from the CFL rate), FP64
  and FP32: sampled points of the first stage against the oracle's
  right-hand side at those points;
* the batched AMR step, 512 patches {16..64}^3, wave and CCZ4 mixed,
  FP32-bulk with double-word islands, CCZ4 rows padded to 16 bytes (TMA tile
  launch + persistent launch, tuned tiles): sampled points of the first stage
  of sampled patches against the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1806_04182_gb300 import build, capi, inputs
from paper_1806_04182_gb300.state import PatchState

pytestmark = pytest.mark.gpu
TOL64 = 1e-12
EPS32 = float(np.finfo(np.float32).eps)


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    return capi.lib()


def oracle_params(prm: capi.sf_params):
    return oracle.params(sigma=prm.sigma_ko, gamma_eos=prm.gamma_eos, weno_eps=prm.weno_eps,
                         weno_q=prm.weno_q, kappa_z=prm.kappa_z, kappa_c=prm.kappa_c, eta=prm.eta,
                         g_shift=prm.g_shift, weno_variant=prm.weno_variant, slicing=prm.slicing,
                         shift_frozen=prm.shift_frozen, lopsided=prm.lopsided,
                         flux_split=prm.flux_split)


def rel(got, want, floor):
    return max(np.abs(got[f] - want[f]).max() / max(np.abs(want[f]).max(), floor)
               for f in range(want.shape[0]))


def test_wave_64cubed_fp64_step_every_point():
    n = (64, 64, 64)
    U0, dx = inputs.wave_plane(n, seed=0)
    dt = 0.25 * dx[0]
    st = PatchState(capi.SF_WAVE, n, dx, dt)
    st.upload(U0)
    st.step(1)
    got = st.fields().cpu().numpy()
    G = oracle.ghosted(U0.copy())
    oracle.rk4_step(oracle.WAVE, G, dx, dt, oracle_params(st.prm))
    assert rel(got, oracle.interior(G), 1e-3) < TOL64


def test_mhd_128cubed_fp64_first_stage_sampled():
    n = (128, 128, 128)
    U0, dx = inputs.mhd_blast(n, seed=0)
    st = PatchState(capi.SF_MHD, n, dx, 1e-3)
    st.upload(U0)
    rate = st.mhd_max_rate().item()
    st.dt = 0.3 / rate
    out = st.interior(st.stage(0)).cpu().numpy().reshape(8, -1)
    pts = inputs.observers(n, 3000, seed=5)
    r = oracle.rhs_points(oracle.MHD, oracle.ghosted(U0.copy()), dx, pts, oracle_params(st.prm))
    want = U0.reshape(8, -1)[:, pts] + st.dt * r
    assert rel(out[:, pts], want, 1e-3) < TOL64


def test_mhd_128cubed_fp32_first_stage_sampled():
    # the FP32 MHD row of the suite, same data and launch: float storage and
    # arithmetic, against the FP64 oracle with the FP32 stage bound (32 eps32
    # of each field's scale, derived at test_mhd_fp32_stages in
    # test_gpu_parity.py)
    n = (128, 128, 128)
    U0, dx = inputs.mhd_blast(n, seed=0)
    st = PatchState(capi.SF_MHD, n, dx, 1e-3, precision=capi.SF_FP32_BULK)
    st.upload(U0)
    rate = st.mhd_max_rate().item()
    dt = 0.3 / oracle.mhd_max_rate(oracle.ghosted(U0.copy()), dx, oracle_params(st.prm))
    assert rate == pytest.approx(1.0 / (dt / 0.3), rel=1e-6)
    st.dt = dt
    out = st.fields(st.stage(0)).cpu().numpy().reshape(8, -1)
    pts = inputs.observers(n, 3000, seed=5)
    r = oracle.rhs_points(oracle.MHD, oracle.ghosted(U0.copy()), dx, pts, oracle_params(st.prm))
    want = U0.reshape(8, -1)[:, pts] + dt * r
    assert rel(out[:, pts], want, 1e-3) < 32 * EPS32


def test_batch_512_patches_first_stage_sampled():
    table = inputs.amr_patch_table(512, seed=0)
    sts = []
    for q, t in enumerate(table):
        h = t["dx"]
        system = capi.SF_WAVE if t["system"] == "wave" else capi.SF_Z4
        if system == capi.SF_WAVE:
            U0, _ = inputs.wave_plane(t["n"], seed=q, length=t["n"][0] * h)
        else:
            U0, _ = inputs.z4_perturbed(t["n"], seed=q, amp=0.03)
        pitch = (t["n"][0] + 6 + 3) // 4 * 4 if system == capi.SF_Z4 else None
        st = PatchState(system, t["n"], (h, h, h), t["dt"], precision=capi.SF_FP32_BULK_DW,
                        x_pitch=pitch)
        st.upload(U0)
        st.U0 = U0
        sts.append(st)
    b = capi.sf_batch_create(capi.params(), [s_.patch(s_.B, s_.A, s_.C) for s_ in sts])
    stream = torch.cuda.Stream()
    try:
        assert capi.sf_batch_launches_per_step(b) == 12  # both TMA tile widths + persistent
        with torch.cuda.stream(stream):
            capi.sf_batch_tune(b, stream.cuda_stream)   # stage 1 on scratch only
            capi.sf_batch_substep(b, 0, stream.cuda_stream)
        stream.synchronize()
        assert capi.sf_get_device_status() == capi.SF_OK
    finally:
        capi.sf_batch_destroy(b)
    rng = np.random.default_rng(3)
    picks = list(rng.choice(len(sts), size=12, replace=False))
    assert {sts[q].system for q in picks} == {capi.SF_WAVE, capi.SF_Z4}
    for q in picks:
        st = sts[q]
        nf = st.nf
        out = st.fields(st.B).cpu().numpy().reshape(nf, -1)   # stage 0 output, offsets added back
        pts = inputs.observers(st.n, 200, seed=int(q))
        osys = oracle.Z4 if st.system == capi.SF_Z4 else oracle.WAVE
        r = oracle.rhs_points(osys, oracle.ghosted(st.U0.copy()), st.dx, pts, oracle_params(st.prm))
        want = st.U0.reshape(nf, -1)[:, pts] + 0.5 * st.dt * r
        # float rounding of the 1/dx^2 stencils of O(1) values over dt / 2, and
        # of the stored state itself, relative to the 1e-2 floor
        bound = 2 * 64 / 12 * EPS32 * 0.5 * st.dt / min(st.dx) ** 2 / 1e-2 + 4 * EPS32 / 1e-2
        assert rel(out[:, pts], want, 1e-2) < bound, (q, st.system, st.n)
