"""Host logic of the AMR level loop, checked on the CPU: the box-copy
descriptors that amr.py builds are applied here by a plain Python reading of
the sf_box_copy contract in include/sf.h (point (x, y, z) of field f is read at
src_off + f src_sf + R (z src_sz + y src_sy + x) and written at
dst_off + f dst_sf + z dst_sz + y dst_sy + x), on arrays in host memory.

* Same-level synchronisation (Sec. III): after the halo copies, every patch of
  a periodic box split into blocks holds, ghosts included, exactly the window
  of the undecomposed box that the oracle's periodic ghost fill gives.
* The six ghost-shell slabs of a patch cover its ghost shell once.
* Injection restriction copies fine point R (i - at) into coarse point i.
* The sub-cycled pair's stage-state table lists the arrays its coarse stages
  write, in stage order, and the coarse periodic images are refreshed exactly
  when the restriction writes a point that is some ghost's source.
"""
import itertools

import numpy as np
import pytest
import torch

import oracle
from paper_1806_04182_gb300 import amr, build, capi, inputs
from paper_1806_04182_gb300.state import PatchState


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return capi.lib()


def apply_boxes(boxes, arrays):
    """sf_copy_boxes on host tensors; `arrays` maps data_ptr -> tensor."""
    for bx in boxes:
        src = arrays[bx.src].view(-1)
        dst = arrays[bx.dst].view(-1)
        R = bx.src_step
        for f in range(bx.nf):
            for z in range(bx.ext[2]):
                for y in range(bx.ext[1]):
                    x = np.arange(bx.ext[0])
                    s = bx.src_off + f * bx.src_sf + R * (z * bx.src_sz + y * bx.src_sy + x)
                    d = bx.dst_off + f * bx.dst_sf + z * bx.dst_sz + y * bx.dst_sy + x
                    dst[torch.as_tensor(d)] = src[torch.as_tensor(s)]


def cpu_state(n, prm=None, pitch=None, system=capi.SF_WAVE):
    return PatchState(system, n, (0.1, 0.1, 0.1), 0.01,
                      prm=prm or capi.params(ghosts=capi.SF_GHOSTS_NONE), device="cpu",
                      x_pitch=pitch)


@pytest.mark.parametrize("N,parts,pitch", [((12, 10, 8), (2, 2, 2), None),
                                           ((9, 8, 12), (3, 1, 2), 16),
                                           ((6, 6, 6), (1, 1, 1), None)])
def test_halo_boxes_reproduce_the_periodic_fill(N, parts, pitch):
    m = tuple(N[a] // parts[a] for a in range(3))
    U = inputs.wave_noise(N, seed=11)
    want = oracle.ghosted(U.copy())
    grid, arrays = {}, {}
    for a, b, c in itertools.product(*(range(p) for p in parts)):
        st = cpu_state(m, pitch=pitch)
        st.A.fill_(np.nan)
        sub = U[:, c * m[2]:(c + 1) * m[2], b * m[1]:(b + 1) * m[1], a * m[0]:(a + 1) * m[0]]
        st.A[:, 3:3 + m[2], 3:3 + m[1], 3:3 + m[0]] = torch.as_tensor(sub)
        grid[(a, b, c)] = st
        arrays[st.A.data_ptr()] = st.A
    boxes = amr.halo_boxes(grid, "A")
    assert len(boxes) == 26 * len(grid)
    apply_boxes(boxes, arrays)
    for (a, b, c), st in grid.items():
        got = st.A[..., :m[0] + 6].numpy()
        win = want[:, c * m[2]:c * m[2] + m[2] + 6, b * m[1]:b * m[1] + m[1] + 6,
                   a * m[0]:a * m[0] + m[0] + 6]
        np.testing.assert_array_equal(got, win)
        if pitch:  # the row padding is never written
            assert torch.isnan(st.A[..., m[0] + 6:]).all()


def test_ghost_shell_boxes_cover_the_shell_once():
    st = cpu_state((7, 5, 4))
    g = st.g
    count = np.zeros((4 + 2 * g, 5 + 2 * g, 7 + 2 * g), dtype=int)
    for lo, ext in amr.ghost_shell_boxes(st):
        count[lo[2] + g:lo[2] + g + ext[2], lo[1] + g:lo[1] + g + ext[1],
              lo[0] + g:lo[0] + g + ext[0]] += 1
    interior = np.zeros_like(count, dtype=bool)
    interior[g:-g, g:-g, g:-g] = True
    assert (count[interior] == 0).all()
    assert (count[~interior] == 1).all()


@pytest.mark.parametrize("R", [2, 3])
def test_restrict_box_injects_coincident_fine_points(R):
    coarse = cpu_state((12, 10, 9))
    fine = cpu_state((R * 4, R * 3, R * 2))
    at = (5, 4, 3)
    fine.A.copy_(torch.as_tensor(np.random.default_rng(R).normal(size=fine.shape)))
    coarse.A.zero_()
    origin, ext = (6, 4, 4), (2, 3, 1)   # inside the fine patch's coarse footprint
    bx = amr.restrict_box(fine, coarse, R, origin, ext, fine_at=at)
    apply_boxes([bx], {fine.A.data_ptr(): fine.A, coarse.A.data_ptr(): coarse.A})
    g = 3
    for i, j, k in itertools.product(*(range(o, o + e) for o, e in zip(origin, ext))):
        fi, fj, fk = (R * (v - a) for v, a in zip((i, j, k), at))
        np.testing.assert_array_equal(coarse.A[:, k + g, j + g, i + g].numpy(),
                                      fine.A[:, fk + g, fj + g, fi + g].numpy())
    assert int((coarse.A != 0).any(dim=0).sum()) == ext[0] * ext[1] * ext[2]


def test_subcycled_pair_stage_states_are_the_stage_outputs():
    prm = capi.params()
    coarse = cpu_state((16, 16, 16), prm=prm, system=capi.SF_Z4)
    fine = cpu_state((16, 16, 16), system=capi.SF_Z4)
    pair = amr.SubcycledPair(coarse, fine, 2, (4, 4, 4))
    outs = [pair._coarse_stage_patch(s).u_next for s in range(4)]
    ins = [pair._coarse_stage_patch(s).u_stage for s in range(4)]
    states = pair._states()
    # U^n aside, then U(2), U(3), U(4), U^{n+1}: each the output of the stage before
    assert states[0] == pair.S0.data_ptr()
    assert states[1:] == outs
    # every stage reads the previous stage's output; stage 0 reads U^n in A
    assert ins == [coarse.A.data_ptr()] + outs[:3]
    # no stage overwrites a state that BOR reads later, except U^n (copied to S0)
    assert len(set(outs)) == 4
    assert pair._box_S0.src == coarse.A.data_ptr() and pair._box_S0.dst == pair.S0.data_ptr()


@pytest.mark.parametrize("at,refresh", [((4, 4, 4), False), ((3, 3, 3), False),
                                        ((5, 5, 5), False), ((2, 4, 4), True),
                                        ((4, 4, 6), True)])
def test_subcycled_pair_refreshes_images_only_when_needed(at, refresh):
    # coarse 16^3, fine footprint 8^3 coarse points (at .. at + 7); the
    # images' sources are coarse points 0..2 and 13..15 along each axis
    coarse = cpu_state((16, 16, 16), prm=capi.params(), system=capi.SF_Z4)
    fine = cpu_state((16, 16, 16), system=capi.SF_Z4)
    pair = amr.SubcycledPair(coarse, fine, 2, at)
    assert pair._refresh_images is refresh
