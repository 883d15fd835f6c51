"""Host-side bookkeeping of the AMR level loop (Sec. III) over the C ABI.

A periodic box tiled by a regular grid of equal patches exchanges its ghost
shells with ``sf_copy_boxes`` (same-level synchronisation): for each patch
and each of its 26 neighbours, the neighbour's interior slab next to the
shared face, edge or corner is copied into this patch's ghost zone.  Every
copy is a box descriptor; the kernels run in libsf.so.
"""
from __future__ import annotations

import itertools

from . import capi
from .state import PatchState


def _strides(st: PatchState):
    nx, ny, nz = st.n
    g = st.g
    sy = nx + 2 * g
    sz = sy * (ny + 2 * g)
    sf = sz * (nz + 2 * g)
    return sy, sz, sf


def _off(st: PatchState, i: int, j: int, k: int) -> int:
    """Element offset of interior point (i, j, k) (may lie in the ghost zone)."""
    sy, sz, _ = _strides(st)
    g = st.g
    return (k + g) * sz + (j + g) * sy + (i + g)


def halo_boxes(grid: dict, which: str = "A") -> list:
    """Box copies that fill every patch's ghost shell from its periodic
    neighbours.  `grid` maps (a, b, c) block coordinates to PatchStates of one
    common size; `which` names the array (A, B or C) to synchronise."""
    keys = list(grid)
    px = 1 + max(k[0] for k in keys)
    py = 1 + max(k[1] for k in keys)
    pz = 1 + max(k[2] for k in keys)
    any_st = grid[keys[0]]
    n = any_st.n
    g = any_st.g
    boxes = []
    for (a, b, c), st in grid.items():
        dst = getattr(st, which)
        sy, sz, sf = _strides(st)
        for d in itertools.product((-1, 0, 1), repeat=3):
            if d == (0, 0, 0):
                continue
            nb = grid[((a + d[0]) % px, (b + d[1]) % py, (c + d[2]) % pz)]
            src = getattr(nb, which)
            lo_src, lo_dst, ext = [], [], []
            for ax in range(3):
                if d[ax] == -1:    # ghost below: neighbour's top slab
                    lo_src.append(n[ax] - g); lo_dst.append(-g); ext.append(g)
                elif d[ax] == 1:   # ghost above: neighbour's bottom slab
                    lo_src.append(0); lo_dst.append(n[ax]); ext.append(g)
                else:
                    lo_src.append(0); lo_dst.append(0); ext.append(n[ax])
            bx = capi.sf_box_copy()
            bx.src = src.data_ptr()
            bx.dst = dst.data_ptr()
            bx.src_off = _off(nb, *lo_src)
            bx.dst_off = _off(st, *lo_dst)
            bx.src_sy = bx.dst_sy = sy
            bx.src_sz = bx.dst_sz = sz
            bx.src_sf = bx.dst_sf = sf
            bx.ext[:] = ext
            bx.nf = st.nf
            bx.src_step = 1
            bx.reserved = 0
            boxes.append(bx)
    return boxes


def restrict_box(fine: PatchState, coarse: PatchState, ratio: int, coarse_origin, ext,
                 fine_array=None, coarse_array=None) -> capi.sf_box_copy:
    """Box copy injecting fine point R*i into coarse points origin..origin+ext-1
    (both patches share the origin of their interior index spaces)."""
    fa = fine.A if fine_array is None else fine_array
    ca = coarse.A if coarse_array is None else coarse_array
    fsy, fsz, fsf = _strides(fine)
    csy, csz, csf = _strides(coarse)
    bx = capi.sf_box_copy()
    bx.src = fa.data_ptr()
    bx.dst = ca.data_ptr()
    bx.src_off = _off(fine, *(ratio * o for o in coarse_origin))
    bx.dst_off = _off(coarse, *coarse_origin)
    bx.src_sy, bx.src_sz, bx.src_sf = fsy, fsz, fsf
    bx.dst_sy, bx.dst_sz, bx.dst_sf = csy, csz, csf
    bx.ext[:] = ext
    bx.nf = fine.nf
    bx.src_step = ratio
    bx.reserved = 0
    return bx
