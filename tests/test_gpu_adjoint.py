"""Adjoint of the RK4 wave evolution (hand-written transposed stage kernel behind
torch.autograd.Function, checkpoint every K steps with recompute) against the
oracle's discrete adjoint and against central finite differences.  The misfit
is quadratic in the initial data (linear dynamics), so central differences are
exact up to rounding for any step size.

Rounding bound, FP64 and FP32 alike.  The gradient is a sum of adjoint
responses to the observer residuals r_n = phi^n(x_o) - ref_n; the residuals
are small differences of O(1) values of phi, so the forward states' rounding
dominates: after n steps of a non-expansive scheme it is about
eps sqrt(n) max|phi_0| (independent roundings per step), which relative to
the residuals' rms gives est = eps sqrt(N) max|phi_0| / rms(r), with
rms(r) = sqrt(2 J / (N n_obs)).  The gradient is checked to 4 est against the
oracle and against central differences (to 8 est there: the difference of
two rounded misfits adds the same order again)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1806_04182_gb300 import adjoint, build, capi, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available()
    build.build()
    return capi.lib()


def setup(n, nsteps, nobs, seed=0, precision=capi.SF_FP64):
    U0, dx = inputs.wave_plane(n, seed=seed)
    dt = 0.25 * min(dx)
    obs = inputs.observers(n, nobs, seed=seed + 1)
    dev = torch.device("cuda")
    dtype = torch.float64 if precision == capi.SF_FP64 else torch.float32
    phi0 = torch.tensor(U0[0], device=dev, dtype=dtype)
    Pi0 = torch.tensor(U0[1], device=dev, dtype=dtype)
    bump = torch.tensor(1e-3 * inputs.smooth_bump(n, seed=seed + 2), device=dev, dtype=dtype)
    obs_t = torch.tensor(obs, device=dev)
    ref = adjoint.observe(phi0 + bump, Pi0, obs_t, dx, dt, nsteps, precision=precision)
    return U0, dx, dt, obs, obs_t, phi0, Pi0, ref


def rounding_estimate(precision, nsteps, nobs, J, phi0):
    eps = float(np.finfo(np.float64 if precision == capi.SF_FP64 else np.float32).eps)
    rms_r = math.sqrt(2.0 * J / (nsteps * nobs))
    return eps * math.sqrt(nsteps) * float(phi0.abs().max()) / rms_r


@pytest.mark.parametrize("precision,n,nsteps,nobs,K", [
    (capi.SF_FP64, (12, 10, 8), 10, 6, 4),
    (capi.SF_FP32_BULK, (12, 10, 8), 10, 6, 4),
    (capi.SF_FP32_BULK, (14, 12, 10), 12, 8, 5),
    (capi.SF_FP32_BULK, (32, 32, 32), 50, 16, 10)])
def test_gradient_matches_oracle_adjoint(precision, n, nsteps, nobs, K):
    U0, dx, dt, obs, obs_t, phi0, Pi0, ref = setup(n, nsteps, nobs, precision=precision)
    phi = phi0.clone().requires_grad_(True)
    Pi = Pi0.clone().requires_grad_(True)
    J = adjoint.misfit(phi, Pi, obs_t, ref, dx, dt, nsteps, precision=precision, checkpoint_every=K)
    J.backward()
    # the oracle starts from the same (for FP32: float-rounded) initial data
    # and observes against the same reference samples
    Jo, gphi_o, gPi_o = oracle.misfit_gradient(phi0.double().cpu().numpy(),
                                               Pi0.double().cpu().numpy(), dx, dt, nsteps, obs,
                                               ref.double().cpu().numpy())
    est = rounding_estimate(precision, nsteps, nobs, Jo, phi0)
    assert J.item() == pytest.approx(Jo, rel=4 * est)
    s = max(np.abs(gphi_o).max(), np.abs(gPi_o).max())
    err = max(np.abs(phi.grad.double().cpu().numpy() - gphi_o).max(),
              np.abs(Pi.grad.double().cpu().numpy() - gPi_o).max()) / s
    assert err < 4 * est, (err, est)


@pytest.mark.parametrize("K", [1, 3, 7])
def test_checkpoint_interval_does_not_change_gradient(K):
    n = (10, 9, 8)
    nsteps = 7
    U0, dx, dt, obs, obs_t, phi0, Pi0, ref = setup(n, nsteps, 5, seed=3)
    grads = []
    for k in (K, nsteps):
        phi = phi0.clone().requires_grad_(True)
        J = adjoint.misfit(phi, Pi0, obs_t, ref, dx, dt, nsteps, checkpoint_every=k)
        J.backward()
        grads.append(phi.grad.clone())
    assert torch.equal(grads[0], grads[1])


def fd_check(n, nsteps, nobs, ndir, K, precision):
    U0, dx, dt, obs, obs_t, phi0, Pi0, ref = setup(n, nsteps, nobs, seed=1, precision=precision)
    phi = phi0.clone().requires_grad_(True)
    Pi = Pi0.clone().requires_grad_(True)
    J = adjoint.misfit(phi, Pi, obs_t, ref, dx, dt, nsteps, precision=precision, checkpoint_every=K)
    J.backward()
    tol = 8 * rounding_estimate(precision, nsteps, nobs, J.item(), phi0)
    worst = 0.0
    for r in range(ndir):
        v1 = torch.tensor(inputs.normal(50 + r, phi0.numel()).reshape(phi0.shape),
                          device=phi0.device, dtype=phi0.dtype)
        v2 = torch.tensor(inputs.normal(80 + r, Pi0.numel()).reshape(Pi0.shape),
                          device=phi0.device, dtype=phi0.dtype)
        eps = 1e-3
        Jp = adjoint.misfit(phi0 + eps * v1, Pi0 + eps * v2, obs_t, ref, dx, dt, nsteps,
                            precision=precision, checkpoint_every=K).item()
        Jm = adjoint.misfit(phi0 - eps * v1, Pi0 - eps * v2, obs_t, ref, dx, dt, nsteps,
                            precision=precision, checkpoint_every=K).item()
        fd = (Jp - Jm) / (2 * eps)
        an = (phi.grad.double() * v1.double()).sum().item() + (Pi.grad.double() * v2.double()).sum().item()
        worst = max(worst, abs(an - fd) / max(abs(fd), 1e-30))
    assert worst < tol, (worst, tol)
    return worst, tol


@pytest.mark.parametrize("precision", [capi.SF_FP64, capi.SF_FP32_BULK])
def test_finite_differences_small(precision):
    fd_check((14, 12, 10), 12, 8, 4, 5, precision)


@pytest.mark.parametrize("precision", [capi.SF_FP64, capi.SF_FP32_BULK])
def test_finite_differences_full_config(precision):
    # 128^3, 200 RK4 steps, 64 observers, checkpoints every 20 steps, 16 directions
    worst, tol = fd_check((128, 128, 128), 200, 64, 16, 20, precision)
    if precision == capi.SF_FP64:
        assert tol < 1e-8  # the FP64 bound is tight: ~1e-10 here
