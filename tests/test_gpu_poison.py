"""Poisoned buffers: reads of memory a stage must not read, and writes it
must make, show up as NaN.

Before one step, every array the stages write (stage scratch, RK4
accumulator) is filled with NaN, and so are the row-padding columns of the
state array, which no kernel may read or write.  After each stage its output
array must be finite on the whole ghosted box (interior and the fused
periodic ghost shell), the accumulator on the interior, and the padding must
still be NaN; the final state must equal, bit for bit, the state of the same
step run on clean buffers.  Covers the global-load, compile-time-stride and
runtime TMA-staged CCZ4 kernels (the latter with tiles overhanging the
patch), the two-point CCZ4 kernel (rows with one float before the first ghost
point, also poisoned; whole tiles with compile-time strides, and any size with
tiles overhanging the patch), the wave and MHD kernels, and the batched
dispatch.
"""
import pytest
import torch

from paper_1806_04182_gb300 import build, capi, inputs
from paper_1806_04182_gb300.state import PatchState

pytestmark = pytest.mark.gpu
NAN = float("nan")


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    return capi.lib()


def _data(system, n, q=0):
    if system == capi.SF_Z4:
        return inputs.z4_perturbed(n, seed=q, amp=0.04)
    if system == capi.SF_WAVE:
        return inputs.wave_plane(n, seed=q)
    return inputs.mhd_blast(n, seed=q)


def _box(st, arr):
    return arr[..., st.xo:st.xo + st.n[0] + 2 * st.g]


def _pad(st, arr):
    # the row padding before the first ghost point and after the last
    return torch.cat([arr[..., :st.xo], arr[..., st.xo + st.n[0] + 2 * st.g:]], dim=-1)


def _fill_pad(st, arr, v):
    arr[..., :st.xo].fill_(v)
    arr[..., st.xo + st.n[0] + 2 * st.g:].fill_(v)


def _inner(st, arr):
    g = st.g
    return arr[:, g:-g, g:-g, st.xo + g:st.xo + g + st.n[0]]


CASES = [
    # system, n, precision, pitch (None: dense + 2 padding floats), row offset
    (capi.SF_Z4, (37, 13, 5), capi.SF_FP32_BULK_DW, 44, 0),   # runtime TMA, overhanging tiles
    (capi.SF_Z4, (37, 13, 5), capi.SF_FP32_BULK_DW, 45, 0),   # global-load, runtime strides
    (capi.SF_Z4, (32, 96, 3), capi.SF_FP32_BULK_DW, 104, 0),  # TMA, compile-time strides
    (capi.SF_Z4, (32, 96, 3), capi.SF_FP32_BULK_DW, 104, 1),  # two-point kernel
    (capi.SF_Z4, (32, 96, 3), capi.SF_FP32_BULK, 104, 1),     # two-point kernel, FP64 islands
    (capi.SF_Z4, (37, 13, 5), capi.SF_FP32_BULK_DW, 48, 1),   # two-point, any size, overhanging tiles
    (capi.SF_Z4, (48, 21, 4), capi.SF_FP32_BULK_DW, 56, 1),   # two-point, any size, even width
    (capi.SF_Z4, (11, 9, 7), capi.SF_FP64, 19, 0),
    (capi.SF_WAVE, (19, 7, 6), capi.SF_FP32_BULK, 27, 0),
    (capi.SF_WAVE, (19, 7, 6), capi.SF_FP64, 26, 0),
    (capi.SF_MHD, (12, 10, 8), capi.SF_FP64, 20, 0),
]


@pytest.mark.parametrize("system,n,precision,pitch,xo", CASES)
def test_stage_writes_every_output_and_reads_no_padding(system, n, precision, pitch, xo):
    U0, dx = _data(system, n)
    dt = 0.25 * min(dx) if system != capi.SF_MHD else 1e-3
    clean = PatchState(system, n, dx, dt, precision=precision, x_pitch=pitch, x_offset=xo)
    clean.upload(U0)
    clean.step(1)
    st = PatchState(system, n, dx, dt, precision=precision, x_pitch=pitch, x_offset=xo)
    st.upload(U0)
    for arr in (st.B, st.C) + ((st.D,) if st.D is not None else ()):
        arr.fill_(NAN)
    _fill_pad(st, st.A, NAN)
    for s in range(st.nstages):
        out = st.stage(s)
        torch.cuda.synchronize()
        assert torch.isfinite(_box(st, out)).all(), ("stage", s, "left NaN in its output")
        assert torch.isnan(_pad(st, out)).all(), ("stage", s, "wrote into row padding")
        if st.D is not None and s < 3:
            assert torch.isfinite(_inner(st, st.D)).all(), ("stage", s, "accumulator")
    assert torch.equal(_box(st, st.A), _box(clean, clean.A))


def test_batch_writes_every_output_and_reads_no_padding():
    # float CCZ4 patches on 16-byte rows (TMA tiles overhanging every patch)
    # and wave patches on the persistent kernel, rows padded by one float
    table = inputs.amr_patch_table(6, seed=3, lo=6, hi=21)
    sts, clean = [], []
    for q, t in enumerate(table):
        system = capi.SF_WAVE if t["system"] == "wave" else capi.SF_Z4
        n = t["n"]
        U0, _ = _data(system, n, q)
        row = n[0] + 6
        pitch = (row + 3) // 4 * 4 if system == capi.SF_Z4 else (row + 1 if (row + 1) % 4 else row + 2)
        for lst in (sts, clean):
            s_ = PatchState(system, n, (t["dx"],) * 3, t["dt"], precision=capi.SF_FP32_BULK_DW,
                            x_pitch=pitch)
            s_.upload(U0)
            lst.append(s_)
    if all(_pad(s_, s_.A).numel() == 0 for s_ in sts):
        pytest.skip("no padding in this table")
    for s_ in sts:
        for arr in (s_.B, s_.C, s_.D):
            arr.fill_(NAN)
        _fill_pad(s_, s_.A, NAN)
    h = torch.cuda.current_stream().cuda_stream
    bp = capi.sf_batch_create(capi.params(), [s_.patch(s_.B, s_.A, s_.C) for s_ in sts])
    bc = capi.sf_batch_create(capi.params(), [s_.patch(s_.B, s_.A, s_.C) for s_ in clean])
    try:
        for stage in range(4):
            capi.sf_batch_substep(bp, stage, h)
            capi.sf_batch_substep(bc, stage, h)
        torch.cuda.synchronize()
    finally:
        capi.sf_batch_destroy(bp)
        capi.sf_batch_destroy(bc)
    for s_, c_ in zip(sts, clean):
        assert torch.isfinite(_box(s_, s_.A)).all()
        assert torch.isnan(_pad(s_, s_.A)).all()
        assert torch.equal(_box(s_, s_.A), _box(c_, c_.A))
