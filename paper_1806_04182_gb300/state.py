"""Device buffers of one ghosted patch and its RK stepping through the C ABI.

PyTorch only allocates the device arrays and supplies the stream; every
stage runs in libsf.so.  Buffer roles (all with the layout of include/sf.h):
  A  the state U^n (updated in place by the last stage)
  B, C  stage scratch
  D  RK4 accumulator
  E  Kahan compensation (FP32_BULK only)
RK4:    stage 0: A -> B, 1: B -> C, 2: C -> B, 3: B -> A.
SSP-RK3: stage 0: A -> B, 1: B -> C, 2: C -> A.
"""
from __future__ import annotations

import json

import numpy as np
import torch

from . import capi


def _stream_handle(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


class PatchState:
    def __init__(self, system: int, n, dx, dt: float, precision: int = capi.SF_FP64,
                 prm: capi.sf_params | None = None, ghost: int = 3, device="cuda",
                 x_pitch: int | None = None, x_offset: int = 0, plane_rows: int | None = None):
        """x_pitch: row length of the ghosted arrays in elements (default
        nx + 2 ghost).  A pitch that makes every row, plane and field start
        on a 16-byte boundary (a multiple of 4 floats) lets the float CCZ4
        substep stage its stencils with TMA bulk-tensor copies.  x_offset:
        elements before the first ghosted point of each row.  With a pitch of
        a multiple of 4 floats and x_offset = 1, interior points with even x
        sit on 8-byte boundaries, which the float CCZ4 kernel that computes
        two neighbouring points per thread needs.  plane_rows: rows per plane
        (default ny + 2 ghost); that kernel's compile-time layout has planes of
        102 rows of 104 floats, so a smaller patch reaches it with
        x_pitch=104, x_offset=1, plane_rows=102."""
        self.system = system
        self.n = tuple(int(v) for v in n)
        self.dx = tuple(float(v) for v in dx)
        self.dt = float(dt)
        self.precision = precision
        self.prm = prm if prm is not None else capi.params(
            rk=capi.SF_SSPRK3 if system == capi.SF_MHD else capi.SF_RK4)
        self.g = ghost
        self.nf = capi.sf_nfields(system)
        self.dtype = torch.float64 if precision == capi.SF_FP64 else torch.float32
        nx, ny, nz = self.n
        g = ghost
        self.xo = int(x_offset)
        self.pitch = self.xo + nx + 2 * g if x_pitch is None else int(x_pitch)
        if self.xo < 0 or self.pitch < self.xo + nx + 2 * g:
            raise ValueError("x_pitch shorter than x_offset plus a ghosted row")
        self.rows = ny + 2 * g if plane_rows is None else int(plane_rows)
        if self.rows < ny + 2 * g:
            raise ValueError("plane_rows shorter than a ghosted plane")
        self.shape = (self.nf, nz + 2 * g, self.rows, self.pitch)
        kw = dict(dtype=self.dtype, device=device)
        self.A = torch.zeros(self.shape, **kw)
        self.B = torch.zeros(self.shape, **kw)
        self.C = torch.zeros(self.shape, **kw)
        self.D = torch.zeros(self.shape, **kw) if self.prm.rk == capi.SF_RK4 else None
        self.E = (torch.zeros(self.shape, **kw)
                  if precision != capi.SF_FP64 and self.prm.rk == capi.SF_RK4 else None)
        self._rate = None  # MHD: device rate of the current U^n, if known

    # ------------------------------------------------------------------ ABI
    def ptr(self, t: torch.Tensor) -> int:
        """Device address of ghosted point (0, 0, 0) of field 0 of array t."""
        return t.data_ptr() + self.xo * t.element_size()

    def patch(self, u_stage, u_n, u_next) -> capi.sf_patch:
        p = capi.sf_patch()
        p.n[:] = self.n
        p.ghost = self.g
        p.dx[:] = self.dx
        p.dt = self.dt
        p.system = self.system
        p.precision = self.precision
        p.sy, p.sz, p.sf = self.strides
        p.u_stage = self.ptr(u_stage)
        p.u_n = self.ptr(u_n)
        p.acc = self.ptr(self.D) if self.D is not None else None
        p.u_next = self.ptr(u_next)
        p.kahan = self.ptr(self.E) if self.E is not None else None
        p.cfl_rate = None
        return p

    @property
    def strides(self):
        """Element strides (y, z, field) of the ghosted arrays."""
        sy = self.pitch
        sz = sy * self.shape[2]
        return sy, sz, sz * self.shape[1]

    def roles(self, stage: int):
        if self.prm.rk == capi.SF_RK4:
            return [(self.A, self.B), (self.B, self.C), (self.C, self.B), (self.B, self.A)][stage]
        return [(self.A, self.B), (self.B, self.C), (self.C, self.A)][stage]

    def stage_patch(self, stage: int) -> capi.sf_patch:
        us, nx = self.roles(stage)
        return self.patch(us, self.A, nx)

    @property
    def nstages(self) -> int:
        return 4 if self.prm.rk == capi.SF_RK4 else 3

    # ------------------------------------------------------------------ data
    # fields stored minus their flat value 1 in the float CCZ4 arrays
    Z4_OFFSET_FIELDS = (0, 1, 4, 6, 18)

    @property
    def offset_fields(self):
        if self.system == capi.SF_Z4 and self.precision != capi.SF_FP64:
            return self.Z4_OFFSET_FIELDS
        return ()

    def upload(self, interior, stream=None) -> None:
        """Set U^n from an interior array (nf, nz, ny, nx) of field values and
        fill periodic ghosts (float CCZ4 arrays get the flat-space offset
        subtracted in double precision before rounding to float)."""
        g = self.g
        t = torch.as_tensor(np.ascontiguousarray(interior) if isinstance(interior, np.ndarray)
                            else interior).double()
        if self.offset_fields:
            t = t.clone()
            for f in self.offset_fields:
                t[f] -= 1.0
        nx, xo = self.n[0], self.xo
        ny = self.n[1]
        self.A[:, g:self.shape[1] - g, g:g + ny, xo + g:xo + g + nx].copy_(t.to(self.dtype))
        if self.E is not None:
            self.E.zero_()
        self._rate = None
        self.fill_ghosts(self.A, stream)

    def upload_ghosted(self, ghosted, stream=None) -> None:
        """Set U^n from a full ghosted array (nf, nz+2g, ny+2g, nx+2g) of field
        values, ghost points included (non-periodic patches)."""
        t = torch.as_tensor(np.ascontiguousarray(ghosted) if isinstance(ghosted, np.ndarray)
                            else ghosted).double().clone()
        for f in self.offset_fields:
            t[f] -= 1.0
        nx, ny = self.n[0] + 2 * self.g, self.n[1] + 2 * self.g
        self.A[:, :, :ny, self.xo:self.xo + nx].copy_(t.to(self.dtype))
        if self.E is not None:
            self.E.zero_()
        self._rate = None

    def step_radiative(self, nsteps: int, x0, u_inf, speed, stream=None) -> None:
        """RK steps of a non-periodic patch: the interior by sf_substep, the
        ghost shell by the radiative boundary condition (Sec. V).  The patch's
        params must have ghosts = SF_GHOSTS_NONE."""
        h = _stream_handle(stream)
        for _ in range(nsteps):
            for s in range(self.nstages):
                p = self.stage_patch(s)
                capi.sf_substep(self.prm, p, s, h)
                capi.sf_radiative_substep(self.prm, p, x0, u_inf, speed, s, h)

    def fill_ghosts(self, array: torch.Tensor, stream=None) -> None:
        capi.sf_fill_ghosts_periodic(self.patch(array, array, array), self.ptr(array), self.nf,
                                     _stream_handle(stream))

    def interior(self, array: torch.Tensor | None = None) -> torch.Tensor:
        """Interior view of the stored values (float CCZ4: with offsets)."""
        a = self.A if array is None else array
        g = self.g
        return a[:, g:self.shape[1] - g, g:g + self.n[1], self.xo + g:self.xo + g + self.n[0]]

    def fields(self, array: torch.Tensor | None = None) -> torch.Tensor:
        """Interior field values in float64 (flat-space offsets added back)."""
        v = self.interior(array).double().clone()
        for f in self.offset_fields:
            v[f] += 1.0
        return v

    # ------------------------------------------------------------------ stepping
    def stage(self, s: int, stream=None) -> torch.Tensor:
        """Run RK stage s; returns the array holding its output."""
        self._rate = None
        capi.sf_substep(self.prm, self.stage_patch(s), s, _stream_handle(stream))
        return self.roles(s)[1]

    def step(self, nsteps: int = 1, stream=None) -> None:
        self._rate = None
        h = _stream_handle(stream)
        for _ in range(nsteps):
            for s in range(self.nstages):
                capi.sf_substep(self.prm, self.stage_patch(s), s, h)

    def step_cfl(self, nsteps: int = 1, cfl: float = 0.3, stream=None) -> list[float]:
        """MHD steps with dt = cfl / rate, the rate of U^n coming from the
        previous step's last stage (the first from sf_mhd_max_rate).  Returns
        the rate used by every step (one device-to-host read per step)."""
        if self.system != capi.SF_MHD:
            raise ValueError("step_cfl is for SF_MHD patches")
        h = _stream_handle(stream)
        # the rate of the current U^n: kept from the previous call's last
        # stage, else one sf_mhd_max_rate sweep
        rate = self._rate if self._rate is not None else self.mhd_max_rate(stream=stream)
        self._rate = rate
        rates = []
        for _ in range(nsteps):
            r = rate.item()
            rates.append(r)
            self.dt = cfl / r
            for s in range(self.nstages):
                p = self.stage_patch(s)
                if s == self.nstages - 1:
                    p.cfl_rate = rate.data_ptr()
                capi.sf_substep(self.prm, p, s, h)
        return rates

    def adjoint_step(self, nsteps: int = 1, stream=None) -> None:
        """RK4 steps of the transposed wave operator on A (adjoint fields)."""
        h = _stream_handle(stream)
        for _ in range(nsteps):
            for s in range(4):
                capi.sf_adjoint_substep(self.prm, self.stage_patch(s), s, h)

    def rhs(self, array: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """(L + Q_d)(array) on the interior, shape (nf, nz, ny, nx)."""
        a = self.A if array is None else array
        nx, ny, nz = self.n
        out = torch.empty((self.nf, nz, ny, nx), dtype=self.dtype, device=a.device)
        capi.sf_rhs(self.prm, self.patch(a, a, self.B), out.data_ptr(), _stream_handle(stream))
        return out

    def diagnostics(self, array: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        a = self.A if array is None else array
        out = torch.empty(5, dtype=torch.float64, device=a.device)
        capi.sf_diagnostics(self.prm, self.patch(a, a, self.B), self.ptr(a), out.data_ptr(),
                            _stream_handle(stream))
        return out

    def mhd_max_rate(self, array: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        a = self.A if array is None else array
        out = torch.empty(1, dtype=torch.float64, device=a.device)
        capi.sf_mhd_max_rate(self.prm, self.patch(a, a, self.B), self.ptr(a), out.data_ptr(),
                             _stream_handle(stream))
        return out

    # ------------------------------------------------------------------ checkpoint
    _PRM_FIELDS = [f for f, _ in capi.sf_params._fields_]

    def save(self, path: str, step: int = 0, t: float = 0.0) -> None:
        """Write U^n (with ghosts), the Kahan compensation and the run
        metadata to `path` (.npz); `load` resumes bit for bit."""
        meta = dict(system=self.system, n=self.n, dx=self.dx, dt=self.dt,
                    precision=self.precision, ghost=self.g, step=step, t=t, pitch=self.pitch,
                    x_offset=self.xo, plane_rows=self.rows,
                    prm={f: getattr(self.prm, f) for f in self._PRM_FIELDS})
        arrays = {"A": self.A.cpu().numpy()}
        if self.E is not None:
            arrays["E"] = self.E.cpu().numpy()
        np.savez(path, meta=np.array(json.dumps(meta)), **arrays)

    @classmethod
    def load(cls, path: str, device="cuda"):
        """(state, step, t) from a file written by `save`."""
        z = np.load(path, allow_pickle=False)
        meta = json.loads(str(z["meta"]))
        st = cls(meta["system"], meta["n"], meta["dx"], meta["dt"], precision=meta["precision"],
                 prm=capi.params(**meta["prm"]), ghost=meta["ghost"], device=device,
                 x_pitch=meta.get("pitch"), x_offset=meta.get("x_offset", 0),
                 plane_rows=meta.get("plane_rows"))
        st.A.copy_(torch.from_numpy(z["A"]))
        if st.E is not None and "E" in z:
            st.E.copy_(torch.from_numpy(z["E"]))
        return st, meta["step"], meta["t"]


class HostPipeline:
    """RK steps of patch states that live in host memory, through the C-ABI
    call ``sf_step_host``.

    A state's host image is ``sf_state_span`` elements of the ghosted array
    from ghosted point (0, 0, 0) (the layout and storage convention of
    ``PatchState.A``; :meth:`image` gives that view of a device array, and
    :meth:`host_buffer` a pinned buffer of that size).  ``run(host_in,
    host_out)`` advances one RK step per entry: upload of ``host_in[k]``,
    the stages, download into ``host_out[k]``, on three streams of the
    pipeline.  With ``slots`` of 2 to 4 the copies of other steps overlap the
    stages (with 3 an upload no longer waits for the download just before
    it); a step whose input is an earlier step's output waits for that
    download, so an evolution kept in host memory (``host_in[k] is
    host_out[k - 1]``) is correct.  ``reset_kahan`` restarts the FP32-bulk
    compensation from zero at every upload (independent states); without
    it the device slot's compensation carries over (a continuing evolution,
    one slot).  ``host_out`` holds the results after :meth:`synchronize` (or
    once a stream waits on :meth:`join`).  ``interior=True`` (periodic
    patches): host images hold the interior only (``sf_interior_span``
    elements, field, z, y, x), the ghost shell rebuilt on the device.
    """

    def __init__(self, *args, slots: int = 2, interior: bool = False, **kw):
        """Arguments as for ``PatchState`` (one patch description)."""
        self.states = tuple(PatchState(*args, **kw) for _ in range(slots))
        self.interior = bool(interior)
        cur = torch.cuda.current_stream()
        self.compute = torch.cuda.Stream()
        self.up = torch.cuda.Stream()
        self.down = torch.cuda.Stream()
        for st_ in (self.compute, self.up, self.down):
            st_.wait_stream(cur)  # the buffers' zero fill
            # the caching allocator must not hand these buffers out again while
            # work queued on the pipeline's streams still uses them
            for state in self.states:
                for t in (state.A, state.B, state.C, state.D, state.E):
                    if t is not None:
                        t.record_stream(st_)
        st = self.states[0]
        self.geom = st.patch(st.A, st.A, st.B)
        self.span = (capi.sf_interior_span(self.geom) if self.interior
                     else capi.sf_state_span(self.geom))
        self.slots = [capi.sf_state(u=s_.ptr(s_.A), s1=s_.ptr(s_.B), s2=s_.ptr(s_.C),
                                    acc=s_.ptr(s_.D) if s_.D is not None else None,
                                    kahan=s_.ptr(s_.E) if s_.E is not None else None)
                      for s_ in self.states]

    @property
    def dtype(self):
        return self.states[0].dtype

    def image(self, array: torch.Tensor) -> torch.Tensor:
        """The host image of an array laid out like the pipeline's states: a
        view of span elements from ghosted (0,0,0), or (interior images) a
        dense copy of the interior."""
        if self.interior:
            return self.states[0].interior(array).contiguous().reshape(-1)
        xo = self.states[0].xo
        return array.reshape(-1)[xo:xo + self.span]

    def host_buffer(self) -> torch.Tensor:
        return torch.empty(self.span, dtype=self.dtype, pin_memory=True)

    def run(self, host_in, host_out, reset_kahan: bool = True) -> None:
        st = self.states[0]
        flags = capi.SF_HOST_RESET_KAHAN if (reset_kahan and st.E is not None) else 0
        if self.interior:
            flags |= capi.SF_HOST_INTERIOR
        capi.sf_step_host(st.prm, self.geom, self.slots, [t.data_ptr() for t in host_in],
                          [t.data_ptr() for t in host_out], flags, self.compute.cuda_stream,
                          self.up.cuda_stream, self.down.cuda_stream)

    def step(self, host_in: torch.Tensor, host_out: torch.Tensor, reset_kahan: bool = True) -> None:
        self.run([host_in], [host_out], reset_kahan)

    def join(self, stream: torch.cuda.Stream | None = None) -> None:
        """Make `stream` (default: the current one) wait for all queued work."""
        stream = stream if stream is not None else torch.cuda.current_stream()
        for st_ in (self.up, self.compute, self.down):
            stream.wait_stream(st_)

    def start(self, stream: torch.cuda.Stream | None = None) -> None:
        """Order the pipeline's streams after the work queued on `stream`."""
        stream = stream if stream is not None else torch.cuda.current_stream()
        for st_ in (self.up, self.compute, self.down):
            st_.wait_stream(stream)

    def synchronize(self) -> None:
        for st_ in (self.up, self.compute, self.down):
            st_.synchronize()
