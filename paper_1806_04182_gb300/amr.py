"""Host-side bookkeeping of the AMR level loop (Sec. III) over the C ABI.

* Same-level synchronisation: a periodic box tiled by a regular grid of equal
  patches exchanges its ghost shells with ``sf_copy_boxes``; for each patch
  and each of its 26 neighbours, the neighbour's interior slab next to the
  shared face, edge or corner is copied into this patch's ghost zone.
* A level stepped as one batch (``level_batch``): the patches of the grid
  go into one ``sf_batch`` whose every stage ends with the ghost-shell
  copies of the buffer it wrote, so a whole step of the level (stage
  kernels and synchronisation) is one captured CUDA graph.
* Restriction by injection (``restrict_box``).
* Sub-cycling in time (``SubcycledPair``): a periodic coarse patch and one
  fine patch R times finer in space and time; the fine ghost zone at every
  fine RK stage is filled by Berger-Oliger without order reduction
  (Sec. III.B, App. D) fused with the quintic prolongation
  (``sf_bor_prolong``), and the fine solution is injected back into the
  coarse level after the R fine steps.
Every copy and every interpolation runs in libsf.so; this module only builds
descriptors and orders the calls.
"""
from __future__ import annotations

import itertools

import torch

from . import capi
from .state import PatchState


def _strides(st: PatchState):
    return st.strides


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
            bx.src = nb.ptr(src)
            bx.dst = st.ptr(dst)
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


def level_batch(grid: dict) -> int:
    """One sf_batch over the patches of `grid` (as for halo_boxes; created
    with ghosts=SF_GHOSTS_NONE and one common precision and RK scheme) with
    the halo copies of each buffer role registered: u_n = A, u_stage = B,
    u_next = C.  Fill the A ghosts once (sf_copy_boxes of halo_boxes(grid,
    "A")) before the first step.  The caller destroys the batch."""
    sts = list(grid.values())
    prm = sts[0].prm
    if prm.ghosts != capi.SF_GHOSTS_NONE:
        raise ValueError("level patches need ghosts=SF_GHOSTS_NONE (their ghosts come from neighbours)")
    b = capi.sf_batch_create(prm, [st.patch(st.B, st.A, st.C) for st in sts])
    try:
        for role, name in enumerate("ABC"):
            capi.sf_batch_set_halo(b, role, halo_boxes(grid, name))
    except Exception:
        capi.sf_batch_destroy(b)
        raise
    return b


def restrict_box(fine: PatchState, coarse: PatchState, ratio: int, coarse_origin, ext,
                 fine_array=None, coarse_array=None, fine_at=(0, 0, 0)) -> capi.sf_box_copy:
    """Box copy injecting fine values into coarse points origin..origin+ext-1.
    Fine interior point 0 sits on coarse interior point `fine_at`, so coarse
    point i takes fine point R*(i - fine_at)."""
    fa = fine.A if fine_array is None else fine_array
    ca = coarse.A if coarse_array is None else coarse_array
    fsy, fsz, fsf = _strides(fine)
    csy, csz, csf = _strides(coarse)
    bx = capi.sf_box_copy()
    bx.src = fine.ptr(fa)
    bx.dst = coarse.ptr(ca)
    bx.src_off = _off(fine, *(ratio * (o - a) for o, a in zip(coarse_origin, fine_at)))
    bx.dst_off = _off(coarse, *coarse_origin)
    bx.src_sy, bx.src_sz, bx.src_sf = fsy, fsz, fsf
    bx.dst_sy, bx.dst_sz, bx.dst_sf = csy, csz, csf
    bx.ext[:] = ext
    bx.nf = fine.nf
    bx.src_step = ratio
    bx.reserved = 0
    return bx


def whole_array_box(st: PatchState, src, dst) -> capi.sf_box_copy:
    """Box copy of a complete ghosted array (all fields, ghosts included)."""
    sy, sz, sf = _strides(st)
    nx, ny, nz = st.n
    g = st.g
    bx = capi.sf_box_copy()
    bx.src = st.ptr(src)
    bx.dst = st.ptr(dst)
    bx.src_off = bx.dst_off = 0
    bx.src_sy = bx.dst_sy = sy
    bx.src_sz = bx.dst_sz = sz
    bx.src_sf = bx.dst_sf = sf
    bx.ext[:] = (nx + 2 * g, ny + 2 * g, nz + 2 * g)
    bx.nf = st.nf
    bx.src_step = 1
    bx.reserved = 0
    return bx


def ghost_shell_boxes(st: PatchState):
    """The ghost shell of a patch as six disjoint boxes (local interior
    coordinates of the lower corner, extent): z slabs over the full x-y
    extent, then y slabs, then x slabs."""
    nx, ny, nz = st.n
    g = st.g
    X, Y = nx + 2 * g, ny + 2 * g
    return [((-g, -g, -g), (X, Y, g)), ((-g, -g, nz), (X, Y, g)),
            ((-g, -g, 0), (X, g, nz)), ((-g, ny, 0), (X, g, nz)),
            ((-g, 0, 0), (g, ny, nz)), ((nx, 0, 0), (g, ny, nz))]


class SubcycledPair:
    """A coarse patch and one fine patch, `ratio` times finer in space and
    time, advanced with sub-cycling (Sec. III.B).  The coarse patch is
    periodic, or, with `coarse_radiative` = (x0, u_inf, speed), an outer box
    whose ghost shell follows the radiative condition of Sec. V (its params
    must then have ghosts = SF_GHOSTS_NONE).

    The fine patch covers coarse interior points at .. at + n_fine/ratio - 1
    and has no periodic images of its own: before each fine RK stage its
    ghost zone receives the BOR value of that stage (App. D), prolonged from
    the coarse stage states.  After the `ratio` fine steps of one coarse step
    the fine interior is injected into the coarse points it covers.

    The coarse stage states that BOR needs are the stage inputs the coarse
    substeps leave behind.  U^n, which the last coarse stage overwrites, is
    copied aside; under RK4 the third coarse stage writes U^(4) into an array
    of its own (instead of over U^(2), as a lone patch does), so U^(2) stays.
    """

    def __init__(self, coarse: PatchState, fine: PatchState, ratio: int, at,
                 coarse_radiative=None):
        if coarse.prm.rk != fine.prm.rk:
            raise ValueError("coarse and fine levels must use the same RK scheme")
        if fine.prm.ghosts != capi.SF_GHOSTS_NONE:
            raise ValueError("the fine patch must be created with ghosts=SF_GHOSTS_NONE")
        if any(v % ratio for v in fine.n):
            raise ValueError("fine patch size must be a multiple of the ratio")
        if coarse_radiative is not None and coarse.prm.ghosts != capi.SF_GHOSTS_NONE:
            raise ValueError("a radiative coarse patch needs ghosts=SF_GHOSTS_NONE")
        self.radiative = coarse_radiative
        self.coarse, self.fine, self.R = coarse, fine, int(ratio)
        self.at = tuple(int(v) for v in at)
        self.rk = coarse.prm.rk
        self.s = 4 if self.rk == capi.SF_RK4 else 3
        kw = dict(dtype=coarse.dtype, device=coarse.A.device)
        self.S0 = torch.zeros(coarse.shape, **kw)
        self.S1 = torch.zeros(coarse.shape, **kw) if self.rk == capi.SF_RK4 else None
        self._box_S0 = whole_array_box(coarse, coarse.A, self.S0)
        cext = tuple(v // ratio for v in fine.n)
        self._restrict = restrict_box(fine, coarse, ratio, self.at, cext, fine_at=self.at)
        self._shell = ghost_shell_boxes(fine)
        # the periodic images of the coarse patch change with the restriction
        # only if it writes inside the g layers next to a face (the images'
        # sources); otherwise the last coarse stage's fused ghost writes stand
        g = coarse.g
        self._refresh_images = any(a < g or a + e > n - g
                                   for a, e, n in zip(self.at, cext, coarse.n))

    def _states(self):
        c = self.coarse
        if self.rk == capi.SF_RK4:
            return [c.ptr(self.S0), c.ptr(c.B), c.ptr(c.C), c.ptr(self.S1), c.ptr(c.A)]
        return [c.ptr(self.S0), c.ptr(c.B), c.ptr(c.C), c.ptr(c.A)]

    def _coarse_stage_patch(self, s: int) -> capi.sf_patch:
        """The coarse patch's stage s; under RK4 U^(4) goes to S1."""
        c = self.coarse
        if self.rk == capi.SF_RK4 and s >= 2:
            return c.patch(self.S1, c.A, c.A) if s == 3 else c.patch(c.C, c.A, self.S1)
        return c.stage_patch(s)

    def fill_fine_ghosts(self, array, r: int, stage: int, stream=None) -> None:
        """BOR value of fine step r, fine stage `stage`, into the ghost shell
        of the fine array `array`."""
        f, c, R = self.fine, self.coarse, self.R
        h = _stream(stream)
        sy, sz, sf = _strides(f)
        es = array.element_size()
        states = self._states()
        cpatch = c.patch(c.A, c.A, c.B)
        boxes = []
        for lo, ext in self._shell:
            origin = tuple(R * a + l for a, l in zip(self.at, lo))
            ptr = f.ptr(array) + _off(f, *lo) * es
            boxes.append(capi.prolong_box(origin, ext, ptr, sy, sz, sf))
        # the six slabs of the shell in one launch
        capi.sf_bor_prolong_boxes(cpatch, self.rk, states, f.nf, R, r, stage, boxes, h)

    def step(self, nsteps: int = 1, stream=None) -> None:
        """Advance the pair by nsteps coarse steps on `stream` (default: the
        current stream).  The BOR fill of each fine stage runs on a stream of
        its own, at the same time as the fine stage before it: the fill writes
        only the ghost shell of the next stage's input, which that stage
        neither reads nor writes (it writes interior points).  A fill waits
        for the coarse stages and for the fine stage two before it, the last
        to read the ghost shell it overwrites (the stage inputs cycle
        A, B, C, B); each fine stage waits for its own fill."""
        c, f, R = self.coarse, self.fine, self.R
        main = _torch_stream(stream)
        h = main.cuda_stream
        if getattr(self, "_side", None) is None:
            self._side = torch.cuda.Stream(device=c.A.device)
        side = self._side
        for _ in range(nsteps):
            capi.sf_copy_boxes([self._box_S0], c.precision, h)
            for s in range(c.nstages):
                cp = self._coarse_stage_patch(s)
                capi.sf_substep(c.prm, cp, s, h)
                if self.radiative is not None:
                    capi.sf_radiative_substep(c.prm, cp, *self.radiative, s, h)
            side.wait_stream(main)  # the coarse stage states are complete
            done = []  # event after each fine stage, in order
            for r in range(R):
                for s in range(f.nstages):
                    if len(done) >= 2:
                        side.wait_event(done[-2])
                    self.fill_fine_ghosts(f.roles(s)[0], r, s, side.cuda_stream)
                    filled = torch.cuda.Event()
                    filled.record(side)
                    main.wait_event(filled)
                    capi.sf_substep(f.prm, f.stage_patch(s), s, h)
                    ev = torch.cuda.Event()
                    ev.record(main)
                    done.append(ev)
            capi.sf_copy_boxes([self._restrict], c.precision, h)
            if self.radiative is None and self._refresh_images:
                c.fill_ghosts(c.A, h)

    def capture(self, nsteps: int = 1) -> None:
        """Record `nsteps` coarse steps (every launch of step(), the coarse and
        fine stages, the BOR ghost fills, the stage-state copies and the
        restriction) into a CUDA graph; replay() then advances the pair by
        those steps with one graph launch, free of the per-launch host work of
        the Python driver.  Call step() at least once first, so that the
        library's one-time set-up (kernel attributes, device addresses) has
        run outside the capture.  The graph holds the current buffers and dt."""
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step(nsteps)
        self._graph = g

    def replay(self) -> None:
        """Advance by the steps recorded with capture()."""
        if getattr(self, "_graph", None) is None:
            raise RuntimeError("capture() first")
        self._graph.replay()


def _torch_stream(stream) -> torch.cuda.Stream:
    if stream is None:
        return torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return stream
    return torch.cuda.ExternalStream(stream)


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)
