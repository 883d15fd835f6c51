"""Batched persistent dispatch over a mixed AMR patch table (wave and CCZ4
patches of different sizes, levels, dx and dt): the persistent kernel must give
the same states as per-patch launches of the same stage kernels, through the
plain stage calls and through the captured CUDA graph, and match the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1806_04182_gb300 import build, capi, inputs
from paper_1806_04182_gb300.state import PatchState

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    build.build()
    return capi.lib()


def make_states(table, precision, seed=0, tma_pitch=False, pair_layout=False):
    """tma_pitch: CCZ4 rows padded to a multiple of 4 floats, so that a float
    batch sends those patches to the TMA-staged kernel.  pair_layout: CCZ4
    rows of a multiple of 4 floats with one float before each row, so that a
    double-word batch sends them to the two-point kernel."""
    states = []
    for q, t in enumerate(table):
        n = t["n"]
        h = t["dx"]
        system = capi.SF_WAVE if t["system"] == "wave" else capi.SF_Z4
        if system == capi.SF_WAVE:
            U0, _ = inputs.wave_plane(n, seed=seed + q, length=n[0] * h)
            U0 = U0 * 1e-2
        else:
            U0, _ = inputs.z4_perturbed(n, seed=seed + q, amp=0.03)
        pitch, xo = None, 0
        if tma_pitch and system == capi.SF_Z4:
            pitch = (n[0] + 6 + 3) // 4 * 4
        if pair_layout and system == capi.SF_Z4:
            pitch, xo = (n[0] + 7 + 3) // 4 * 4, 1
        st = PatchState(system, n, (h, h, h), t["dt"], precision=precision, x_pitch=pitch,
                        x_offset=xo)
        st.upload(U0)
        st.U0 = U0
        states.append(st)
    return states


def batch_patches(states):
    # batch roles: u_n = A (state), u_stage = B, u_next = C, acc = D, kahan = E
    return [st.patch(st.B, st.A, st.C) for st in states]


def expected_launches_per_step(states):
    """Launches per RK4 step of a batch: one per stage for each TMA tile width
    in use (float CCZ4 patches with 16-byte rows; a patch takes the 16 x 24
    tile when that covers it with fewer tiles than 32 x 12) and one for the
    persistent kernel unless every patch is on TMA."""
    def tiles(n, tx, ty):
        return -(-n[0] // tx) * -(-n[1] // ty)
    widths, rest = set(), False
    for st in states:
        if st.system == capi.SF_Z4 and st.precision != capi.SF_FP64 and st.pitch % 4 == 0:
            widths.add(16 if tiles(st.n, 16, 24) < tiles(st.n, 32, 12) else 32)
        else:
            rest = True
    return 4 * (len(widths) + (1 if rest or not widths else 0))


def fp_bound(precision, st, steps=2):
    """FP64: summation-order rounding.  FP32: the two kernels are compiled
    separately (FMA contraction may differ), so they differ by the float
    rounding of the O(1) metric's second-derivative stencils, ~64/12 eps32
    / dx^2 per evaluation, times dt per stage, four stages per step, relative
    to the 1e-2 floor of the comparison."""
    if precision == capi.SF_FP64:
        return 1e-13
    eps32 = float(np.finfo(np.float32).eps)
    h = min(st.dx)
    return 2 * steps * 4 * 64 / 12 * eps32 * st.dt / h ** 2 / 1e-2


def small_table(npatch=10, seed=3):
    t = inputs.amr_patch_table(npatch, seed=seed, lo=6, hi=21)
    assert {p["system"] for p in t} == {"wave", "z4"}
    return t


@pytest.mark.parametrize("precision", [capi.SF_FP64, capi.SF_FP32_BULK_DW])
def test_batch_equals_per_patch_launches(precision):
    table = small_table()
    ref_states = make_states(table, precision)
    for st in ref_states:
        st.step(2)
    states = make_states(table, precision)
    b = capi.sf_batch_create(capi.params(), batch_patches(states))
    try:
        for _ in range(2):
            for s in range(4):
                capi.sf_batch_substep(b, s, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        for st, ref in zip(states, ref_states):
            a, r = st.interior(), ref.interior()
            scale = r.abs().amax(dim=(1, 2, 3)).clamp_min(1e-2)
            err = ((a - r).abs().amax(dim=(1, 2, 3)) / scale).max().item()
            assert err < fp_bound(precision, st), err
    finally:
        capi.sf_batch_destroy(b)


def test_batch_fp64_matches_oracle():
    table = small_table(6, seed=5)
    states = make_states(table, capi.SF_FP64)
    b = capi.sf_batch_create(capi.params(), batch_patches(states))
    try:
        for s in range(4):
            capi.sf_batch_substep(b, s, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
    finally:
        capi.sf_batch_destroy(b)
    for st, t in zip(states, table):
        sysid = oracle.WAVE if t["system"] == "wave" else oracle.Z4
        G = oracle.ghosted(st.U0.copy())
        oracle.rk4_step(sysid, G, st.dx, st.dt, oracle.params())
        want = oracle.interior(G)
        got = st.interior().cpu().numpy()
        for f in range(want.shape[0]):
            scale = max(np.abs(want[f]).max(), 1e-2)
            assert np.abs(got[f] - want[f]).max() <= 1e-12 * scale, (t, f)


def test_batch_graph_tune_and_capture():
    table = small_table(12, seed=7)
    states = make_states(table, capi.SF_FP32_BULK_DW)
    ref = make_states(table, capi.SF_FP32_BULK_DW)
    for st in ref:
        st.step(3)
    b = capi.sf_batch_create(capi.params(), batch_patches(states))
    stream = torch.cuda.Stream()
    try:
        with torch.cuda.stream(stream):
            capi.sf_batch_tune(b, stream.cuda_stream)  # writes scratch only
            capi.sf_batch_capture(b, stream.cuda_stream)
            for _ in range(3):
                capi.sf_batch_launch(b, stream.cuda_stream)
        stream.synchronize()
        # float CCZ4 patches whose dense rows happen to be a multiple of 4 floats
        # go to the TMA-staged kernel
        assert capi.sf_batch_launches_per_step(b) == expected_launches_per_step(states)
        for st, r in zip(states, ref):
            a, w = st.interior(), r.interior()
            scale = w.abs().amax(dim=(1, 2, 3)).clamp_min(1e-2)
            err = ((a - w).abs().amax(dim=(1, 2, 3)) / scale).max().item()
            assert err < fp_bound(capi.SF_FP32_BULK_DW, st, steps=3), err
    finally:
        capi.sf_batch_destroy(b)


def test_batch_rejects_mixed_precision_and_mhd():
    table = small_table(4)
    s64 = make_states(table[:2], capi.SF_FP64)
    s32 = make_states(table[2:], capi.SF_FP32_BULK_DW)
    with pytest.raises(capi.SfError, match="precision"):
        capi.sf_batch_create(capi.params(), batch_patches(s64 + s32))
    m = PatchState(capi.SF_MHD, (8, 8, 8), (0.1,) * 3, 0.01, prm=capi.params())
    with pytest.raises(capi.SfError):
        capi.sf_batch_create(capi.params(), [m.patch(m.B, m.A, m.C)])


# ------------------------------------------------------------------ TMA-staged CCZ4 tiles
@pytest.mark.parametrize("precision", [capi.SF_FP32_BULK_DW, capi.SF_FP32_BULK])
def test_batch_tma_tiles_equal_per_patch_launches(precision):
    # CCZ4 rows padded to 16 bytes: the batch sends those patches to the
    # TMA-staged kernel (32 x 12 x 1 tiles overhanging every patch here,
    # sizes 6..21), the wave patches to the persistent kernel; per-patch
    # launches run the global-load kernel on the same layouts.
    table = small_table(10, seed=11)
    ref_states = make_states(table, precision, tma_pitch=True)
    for st in ref_states:
        st.step(2)
    states = make_states(table, precision, tma_pitch=True)
    b = capi.sf_batch_create(capi.params(), batch_patches(states))
    try:
        assert capi.sf_batch_launches_per_step(b) == expected_launches_per_step(states)
        assert capi.sf_batch_launches_per_step(b) >= 8  # TMA tiles + persistent, 4 stages
        for _ in range(2):
            for s in range(4):
                capi.sf_batch_substep(b, s, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert capi.sf_get_device_status() == capi.SF_OK
        for st, ref in zip(states, ref_states):
            a, r = st.interior(), ref.interior()
            scale = r.abs().amax(dim=(1, 2, 3)).clamp_min(1e-2)
            err = ((a - r).abs().amax(dim=(1, 2, 3)) / scale).max().item()
            assert err < fp_bound(precision, st), err
    finally:
        capi.sf_batch_destroy(b)


def test_batch_tma_tiles_match_oracle_through_graph():
    # CCZ4 patches only (one launch per stage), sizes across the tile edges,
    # one RK4 step through the captured graph against the FP64 oracle; the
    # smooth periodic data of z4_perturbed with its own dx per patch, and the
    # float bound of the single-patch TMA test
    eps32 = float(np.finfo(np.float32).eps)
    states = []
    for q, n in enumerate(((32, 12, 4), (33, 13, 5), (7, 25, 3), (45, 11, 6))):
        U0, dx = inputs.z4_perturbed(n, seed=20 + q, amp=0.05)
        st = PatchState(capi.SF_Z4, n, dx, 0.25 * min(dx), precision=capi.SF_FP32_BULK_DW,
                        x_pitch=(n[0] + 6 + 3) // 4 * 4)
        st.upload(U0)
        st.U0 = U0
        states.append(st)
    b = capi.sf_batch_create(capi.params(), batch_patches(states))
    stream = torch.cuda.Stream()
    try:
        # (33, 13, 5) and (7, 25, 3) take the 16 x 24 tile, the others 32 x 12: two
        # launches per stage
        assert capi.sf_batch_launches_per_step(b) == expected_launches_per_step(states) == 8
        with torch.cuda.stream(stream):
            capi.sf_batch_tune(b, stream.cuda_stream)  # no persistent items: TMA widths only
            capi.sf_batch_capture(b, stream.cuda_stream)
            capi.sf_batch_launch(b, stream.cuda_stream)
        stream.synchronize()
    finally:
        capi.sf_batch_destroy(b)
    for st in states:
        G = oracle.ghosted(st.U0.copy())
        oracle.rk4_step(oracle.Z4, G, st.dx, st.dt, oracle.params())
        want = oracle.interior(G)
        got = st.fields().cpu().numpy()  # flat-space offsets added back
        bound = 4 * 64 / 12 * eps32 * st.dt / min(st.dx) ** 2 / 1e-2
        for f in range(want.shape[0]):
            e = np.abs(got[f] - want[f]).max() / max(np.abs(want[f]).max(), 1e-2)
            assert e < bound, (st.n, f, e, bound)


def test_batch_tune_measures_tma_tile_width():
    # the tuner times both TMA tile widths for every size class with TMA
    # patches and keeps one; the two widths are separate kernel instances of
    # the same per-point code, so a step after tuning equals a step before it
    # within the float bound of two separately compiled kernels
    table = small_table(12, seed=5)
    a = make_states(table, capi.SF_FP32_BULK_DW, tma_pitch=True)
    c = make_states(table, capi.SF_FP32_BULK_DW, tma_pitch=True)
    ba = capi.sf_batch_create(capi.params(), batch_patches(a))
    bc = capi.sf_batch_create(capi.params(), batch_patches(c))
    stream = torch.cuda.Stream()
    try:
        before = capi.sf_batch_tuned(bc)
        with torch.cuda.stream(stream):
            # tuning runs stage 1, which writes scratch only; reset it after
            capi.sf_batch_tune(bc, stream.cuda_stream)
        stream.synchronize()
        after = capi.sf_batch_tuned(bc)
        for name, v in after.items():
            if name.startswith("z4"):
                assert v["tma_tile_width"] in ((16, 32) if before[name]["tma_tile_width"] else (0,))
            else:
                assert v["tma_tile_width"] == 0
        h = torch.cuda.current_stream().cuda_stream
        for st in c:
            for t in (st.B, st.C, st.D):
                t.zero_()
        for b in (ba, bc):
            for s in range(4):
                capi.sf_batch_substep(b, s, h)
        torch.cuda.synchronize()
        for x, y in zip(a, c):
            r, g = x.interior(), y.interior()
            scale = r.abs().amax(dim=(1, 2, 3)).clamp_min(1e-2)
            err = ((g - r).abs().amax(dim=(1, 2, 3)) / scale).max().item()
            assert err < fp_bound(capi.SF_FP32_BULK_DW, x, steps=1), err
    finally:
        capi.sf_batch_destroy(ba)
        capi.sf_batch_destroy(bc)


# ------------------------------------------------------------------ two-point CCZ4 tiles
def test_batch_pair_tiles_equal_per_patch_launches():
    # double-word CCZ4 patches on the one-float row offset layout go to the
    # two-point kernel in 32 x 16 tiles that overhang every patch here (sizes
    # 6..21, odd ones included), the wave patches to the persistent kernel;
    # per-patch launches run the global-load kernel on the same layouts
    table = small_table(10, seed=11)
    ref_states = make_states(table, capi.SF_FP32_BULK_DW, pair_layout=True)
    for st in ref_states:
        st.step(2)
    states = make_states(table, capi.SF_FP32_BULK_DW, pair_layout=True)
    b = capi.sf_batch_create(capi.params(), batch_patches(states))
    try:
        assert capi.sf_batch_launches_per_step(b) == 8  # two-point tiles + persistent, 4 stages
        for _ in range(2):
            for s in range(4):
                capi.sf_batch_substep(b, s, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert capi.sf_get_device_status() == capi.SF_OK
        for st, ref in zip(states, ref_states):
            a, r = st.interior(), ref.interior()
            scale = r.abs().amax(dim=(1, 2, 3)).clamp_min(1e-2)
            err = ((a - r).abs().amax(dim=(1, 2, 3)) / scale).max().item()
            assert err < fp_bound(capi.SF_FP32_BULK_DW, st), err
            # the periodic ghost shell written by the tiles equals a fresh fill
            g = st.A.clone()
            st.fill_ghosts(g)
            torch.cuda.synchronize()
            assert torch.equal(g, st.A)
    finally:
        capi.sf_batch_destroy(b)


def test_batch_pair_tiles_match_oracle_through_graph():
    # sizes across the 32 x 16 tile edges, odd widths included, one RK4 step
    # through the captured graph against the FP64 oracle (float bound of the
    # single-patch TMA test)
    eps32 = float(np.finfo(np.float32).eps)
    states = []
    for q, n in enumerate(((32, 16, 4), (33, 17, 5), (7, 25, 3), (45, 11, 6), (64, 32, 3))):
        U0, dx = inputs.z4_perturbed(n, seed=40 + q, amp=0.05)
        st = PatchState(capi.SF_Z4, n, dx, 0.25 * min(dx), precision=capi.SF_FP32_BULK_DW,
                        x_pitch=(n[0] + 7 + 3) // 4 * 4, x_offset=1)
        st.upload(U0)
        st.U0 = U0
        states.append(st)
    b = capi.sf_batch_create(capi.params(), batch_patches(states))
    stream = torch.cuda.Stream()
    try:
        assert capi.sf_batch_launches_per_step(b) == 4  # one two-point launch per stage
        with torch.cuda.stream(stream):
            capi.sf_batch_tune(b, stream.cuda_stream)
            capi.sf_batch_capture(b, stream.cuda_stream)
            capi.sf_batch_launch(b, stream.cuda_stream)
        stream.synchronize()
        assert capi.sf_get_device_status() == capi.SF_OK
    finally:
        capi.sf_batch_destroy(b)
    for st in states:
        G = oracle.ghosted(st.U0.copy())
        oracle.rk4_step(oracle.Z4, G, st.dx, st.dt, oracle.params())
        want = oracle.interior(G)
        got = st.fields().cpu().numpy()
        bound = 4 * 64 / 12 * eps32 * st.dt / min(st.dx) ** 2 / 1e-2
        for f in range(want.shape[0]):
            e = np.abs(got[f] - want[f]).max() / max(np.abs(want[f]).max(), 1e-2)
            assert e < bound, (st.n, f, e, bound)


def test_batch_pair_tiles_write_every_ghost_and_no_padding():
    # scratch roles and row padding filled with NaN: after a step through the
    # two-point tiles every ghosted point of the new state is finite, the
    # padding (the float before each row, the row tails, the extra plane
    # rows) is still NaN, and the state equals a clean run bit for bit
    shapes = ((33, 17, 5), (45, 11, 6))
    def run(poison):
        states = []
        for q, n in enumerate(shapes):
            U0, dx = inputs.z4_perturbed(n, seed=60 + q, amp=0.05)
            st = PatchState(capi.SF_Z4, n, dx, 0.25 * min(dx), precision=capi.SF_FP32_BULK_DW,
                            x_pitch=(n[0] + 7 + 3) // 4 * 4 + 4, x_offset=1, plane_rows=n[1] + 8)
            if poison:
                for t in (st.A, st.B, st.C, st.D):
                    t.fill_(float("nan"))
            st.upload(U0)
            states.append(st)
        b = capi.sf_batch_create(capi.params(), batch_patches(states))
        try:
            for s in range(4):
                capi.sf_batch_substep(b, s, torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
        finally:
            capi.sf_batch_destroy(b)
        return states
    clean, dirty = run(False), run(True)
    for c_, d_ in zip(clean, dirty):
        n, xo, g = d_.n, d_.xo, d_.g
        box = d_.A[:, :, :n[1] + 2 * g, xo:xo + n[0] + 2 * g]
        assert torch.isfinite(box).all()
        assert torch.isnan(d_.A[..., 0]).all()                      # before each row
        assert torch.isnan(d_.A[..., xo + n[0] + 2 * g:]).all()     # row tails
        assert torch.isnan(d_.A[:, :, n[1] + 2 * g:, :]).all()      # extra plane rows
        assert torch.equal(box, c_.A[:, :, :n[1] + 2 * g, xo:xo + n[0] + 2 * g])
