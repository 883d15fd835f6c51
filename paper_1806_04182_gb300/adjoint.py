"""Gradient of an observer misfit of the RK4 wave evolution w.r.t. initial data.

J = 1/2 sum_{n=1..N} sum_o (phi^n(x_o) - ref[n-1, o])^2 for the first-order
wave system (Sec. IV.A) started from (phi0, Pi0, D_x phi0, D_y phi0, D_z phi0).

Forward: N RK4 steps through ``sf_substep``, keeping only a checkpoint of
the state every K steps.  Backward: for each segment, newest first, the
forward states are recomputed from the segment's checkpoint (observer
samples through ``sf_gather``), then the adjoint runs backwards through the
segment: the misfit residual of step n is injected into lambda_phi
(``sf_scatter_add``) and one RK4 step of the transposed operator
(``sf_adjoint_substep``, which applies P(dt L)^T = P(dt L^T)) maps lambda^n to
lambda^{n-1}.  Finally the initial-data map is transposed:
dJ/dphi0 = lambda_phi + sum_i D_i^T lambda_{d_i} = lambda_phi - sum_i D_i lambda_{d_i},
dJ/dPi0 = lambda_Pi.  The D_i and D_i^T of the initial map are evaluated by
``sf_rhs`` of the wave system on states holding only the relevant fields
(the RHS of d_i is -D_i Pi, the RHS of Pi is -sum_i D_i d_i, and KO of a zero
field is zero).  Every stencil, stage and adjoint step runs in libsf.so; the
observer residuals and the misfit sum (n_obs values a step) are formed with
torch.
"""
from __future__ import annotations

import torch

from . import capi
from .state import PatchState


def _rhs_of(st: PatchState, fields: dict[int, torch.Tensor]) -> torch.Tensor:
    """sf_rhs of a state whose only non-zero fields are `fields` (interior arrays)."""
    st.B.zero_()
    g = st.g
    for f, v in fields.items():
        st.B[f, g:-g, g:-g, g:-g].copy_(v)
    st.fill_ghosts(st.B)
    return st.rhs(st.B)


def _d_of(st: PatchState, phi: torch.Tensor) -> torch.Tensor:
    """(D_x phi, D_y phi, D_z phi): minus the d-rows of the RHS with phi in the Pi slot."""
    r = _rhs_of(st, {1: phi})
    return -r[2:5]


def _div_of(st: PatchState, d: torch.Tensor) -> torch.Tensor:
    """sum_i D_i d_i: minus the Pi row of the RHS with d in the d slots."""
    r = _rhs_of(st, {2: d[0], 3: d[1], 4: d[2]})
    return -r[1]


class WaveMisfit(torch.autograd.Function):
    """J(phi0, Pi0); phi0 and Pi0 are (nz, ny, nx) device tensors."""

    @staticmethod
    def forward(ctx, phi0, Pi0, obs, ref, dx, dt, nsteps, precision, checkpoint_every, prm):
        n = (phi0.shape[2], phi0.shape[1], phi0.shape[0])
        st = PatchState(capi.SF_WAVE, n, dx, dt, precision=precision, prm=prm,
                        device=phi0.device)
        d0 = _d_of(st, phi0.to(st.dtype))
        U0 = torch.stack([phi0.to(st.dtype), Pi0.to(st.dtype), d0[0], d0[1], d0[2]])
        st.upload(U0)
        K = max(1, int(checkpoint_every))
        ckpts = []
        J = torch.zeros((), dtype=torch.float64, device=phi0.device)
        vals = torch.empty(obs.numel(), dtype=st.dtype, device=phi0.device)
        p0 = st.patch(st.A, st.A, st.B)
        for s in range(nsteps):
            if s % K == 0:
                ckpts.append(st.A.clone())
            st.step(1)
            capi.sf_gather(p0, st.ptr(st.A), 0, obs.data_ptr(), obs.numel(), vals.data_ptr())
            r = vals.double() - ref[s].double()
            J = J + 0.5 * (r * r).sum()
        ctx.save_for_backward(obs, ref)
        ctx.st = st
        ctx.ckpts = ckpts
        ctx.K = K
        ctx.nsteps = nsteps
        return J

    @staticmethod
    def backward(ctx, gJ):
        obs, ref = ctx.saved_tensors
        st, ckpts, K, N = ctx.st, ctx.ckpts, ctx.K, ctx.nsteps
        fwd = PatchState(capi.SF_WAVE, st.n, st.dx, st.dt, precision=st.precision, prm=st.prm,
                         device=st.A.device)
        lam = torch.zeros_like(st.A)
        adj = PatchState(capi.SF_WAVE, st.n, st.dx, st.dt, precision=st.precision, prm=st.prm,
                         device=st.A.device)
        adj.A = lam
        p0 = fwd.patch(fwd.A, fwd.A, fwd.B)
        vals = torch.empty(obs.numel(), dtype=st.dtype, device=st.A.device)
        for seg in range(len(ckpts) - 1, -1, -1):
            s0 = seg * K
            s1 = min(N, s0 + K)
            # recompute the forward observer samples of this segment
            fwd.A.copy_(ckpts[seg])
            if fwd.E is not None:
                fwd.E.zero_()
            res = []
            for s in range(s0, s1):
                fwd.step(1)
                capi.sf_gather(p0, fwd.ptr(fwd.A), 0, obs.data_ptr(), obs.numel(),
                               vals.data_ptr())
                res.append(((vals.double() - ref[s].double()) * gJ).to(st.dtype))
            # adjoint sweep through the segment, newest step first
            for s in range(s1 - 1, s0 - 1, -1):
                capi.sf_scatter_add(p0, adj.ptr(adj.A), 0, obs.data_ptr(), obs.numel(),
                                    res[s - s0].data_ptr())
                adj.fill_ghosts(adj.A)  # the injection changed interior points only
                adj.adjoint_step(1)
        g = adj.g
        lam_i = adj.A[:, g:-g, g:-g, g:-g]
        gphi = lam_i[0] - _div_of(fwd, lam_i[2:5].contiguous())
        gPi = lam_i[1].clone()
        return gphi, gPi, None, None, None, None, None, None, None, None


def observe(phi0, Pi0, obs, dx, dt, nsteps, precision=capi.SF_FP64, prm=None):
    """phi at the observers after each of `nsteps` RK4 steps: shape (nsteps, nobs)."""
    prm = prm if prm is not None else capi.params()
    n = (phi0.shape[2], phi0.shape[1], phi0.shape[0])
    st = PatchState(capi.SF_WAVE, n, dx, dt, precision=precision, prm=prm, device=phi0.device)
    d0 = _d_of(st, phi0.to(st.dtype))
    st.upload(torch.stack([phi0.to(st.dtype), Pi0.to(st.dtype), d0[0], d0[1], d0[2]]))
    out = torch.empty((nsteps, obs.numel()), dtype=st.dtype, device=phi0.device)
    p0 = st.patch(st.A, st.A, st.B)
    for s in range(nsteps):
        st.step(1)
        capi.sf_gather(p0, st.ptr(st.A), 0, obs.data_ptr(), obs.numel(), out[s].data_ptr())
    return out


def misfit(phi0, Pi0, obs, ref, dx, dt, nsteps, precision=capi.SF_FP64, checkpoint_every=20,
           prm=None):
    """Differentiable misfit J(phi0, Pi0) (see module docstring)."""
    prm = prm if prm is not None else capi.params()
    return WaveMisfit.apply(phi0, Pi0, obs, ref, dx, dt, nsteps, precision, checkpoint_every, prm)
