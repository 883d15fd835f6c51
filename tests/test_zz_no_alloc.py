"""sf_batch_substep_static: the batched stage for callers that cannot call
cudaMalloc (their device memory belongs to their own pool, or they must not
allocate while other work runs).  Its output must match the allocating
sf_batch_substep on the same patches, within the batch tests' tolerance, for
two full steps in a row (so the second call runs on scratch left by the first).
Collected last so that a stop-at-first-failure run has run everything else."""
import pytest
import torch

from paper_1806_04182_gb300 import build, capi, inputs
from paper_1806_04182_gb300.state import PatchState


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "needs a GPU"
    build.build()
    return capi.lib()


def states_for(table, precision):
    out = []
    for q, t in enumerate(table):
        n, h = t["n"], t["dx"]
        system = capi.SF_WAVE if t["system"] == "wave" else capi.SF_Z4
        if system == capi.SF_WAVE:
            U0, _ = inputs.wave_plane(n, seed=q, length=n[0] * h)
            U0 = 1e-2 * U0
        else:
            U0, _ = inputs.z4_perturbed(n, seed=q, amp=0.03)
        # rows kept off a multiple of 4 floats: sf_batch would send float CCZ4
        # patches with 16-byte rows to its TMA-staged kernel, and this test
        # compares the two entry points on the one persistent kernel they share
        row = n[0] + 6
        st = PatchState(system, n, (h, h, h), t["dt"], precision=precision,
                        x_pitch=row + 1 if row % 4 == 0 else row)
        st.upload(U0)
        out.append(st)
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [(capi.SF_FP64, 1e-13), (capi.SF_FP32_BULK, 0.0),
                                           (capi.SF_FP32_BULK_DW, 0.0)])
def test_static_scratch_batch_matches_allocating_batch(precision, tol):
    # Both paths launch the same compiled persistent kernel, so for FP64 they
    # agree to rounding and for FP32 bit for bit (tolerance 0).
    table = inputs.amr_patch_table(10, seed=3, lo=6, hi=21)
    a = states_for(table, precision)
    b = states_for(table, precision)
    roles = lambda sts: [st.patch(st.B, st.A, st.C) for st in sts]
    prm = capi.params()
    h = torch.cuda.current_stream().cuda_stream
    batch = capi.sf_batch_create(prm, roles(a))
    try:
        for step in range(2):
            for s in range(4):
                capi.sf_batch_substep(batch, s, h)
                capi.sf_batch_substep_static(prm, roles(b), s, h)
            torch.cuda.synchronize()
            for x, y in zip(a, b):
                ref = x.interior()
                scale = ref.abs().amax(dim=(1, 2, 3)).clamp_min(1e-3)
                err = ((y.interior() - ref).abs().amax(dim=(1, 2, 3)) / scale).max().item()
                assert err <= tol, (step, err)
    finally:
        capi.sf_batch_destroy(batch)
    assert capi.sf_get_device_status(h) == capi.SF_OK


@pytest.mark.gpu
def test_static_scratch_rejects_requests_beyond_its_maximum():
    table = inputs.amr_patch_table(65, seed=1, lo=6, hi=8)
    sts = states_for(table[:2], capi.SF_FP64)
    roles = [sts[0].patch(sts[0].B, sts[0].A, sts[0].C)] * 65
    with pytest.raises(capi.SfError, match="static scratch maximum"):
        capi.sf_batch_substep_static(capi.params(), roles, 0)
    # 3 x (4 x 32 x 24) = 9216 work items of 32x4x4 points > 8192: rejected before any launch
    big = PatchState(capi.SF_Z4, (128, 128, 96), (0.01,) * 3, 0.001, precision=capi.SF_FP32_BULK_DW)
    with pytest.raises(capi.SfError, match="static scratch maximum"):
        capi.sf_batch_substep_static(capi.params(), [big.patch(big.B, big.A, big.C)] * 3, 0)


@pytest.mark.gpu
def test_static_scratch_honours_ghosts_none():
    # SF_GHOSTS_NONE: the caller owns the ghost shells (patches that tile a
    # level), so a stage writes the interior only, like sf_batch with NONE
    table = inputs.amr_patch_table(6, seed=5, lo=6, hi=14)
    a = states_for(table, capi.SF_FP64)
    b = states_for(table, capi.SF_FP64)
    prm = capi.params(ghosts=capi.SF_GHOSTS_NONE)
    h = torch.cuda.current_stream().cuda_stream
    for st in b:
        st.B.fill_(float("nan"))
    batch = capi.sf_batch_create(prm, [st.patch(st.B, st.A, st.C) for st in a])
    try:
        capi.sf_batch_substep(batch, 0, h)
        capi.sf_batch_substep_static(prm, [st.patch(st.B, st.A, st.C) for st in b], 0, h)
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            ref = x.interior(x.B)
            scale = ref.abs().amax(dim=(1, 2, 3)).clamp_min(1e-3)
            err = ((y.interior(y.B) - ref).abs().amax(dim=(1, 2, 3)) / scale).max().item()
            assert err <= 1e-13, err
            shell = torch.ones_like(y.B, dtype=torch.bool)
            g = y.g
            shell[:, g:-g, g:-g, g:g + y.n[0]] = False
            assert torch.isnan(y.B[shell]).all()
    finally:
        capi.sf_batch_destroy(batch)
    with pytest.raises(capi.SfError, match="ghosts"):
        capi.sf_batch_substep_static(capi.params(ghosts=7), [b[0].patch(b[0].B, b[0].A, b[0].C)], 0, h)
    assert capi.sf_get_device_status(h) == capi.SF_OK
