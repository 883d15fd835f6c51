"""Adjoint of the RK4 wave evolution (hand-written transposed stage kernel behind
torch.autograd.Function, checkpoint every K steps with recompute) against the
oracle's discrete adjoint and against central finite differences.  The misfit
is quadratic in the initial data (linear dynamics), so central differences are
exact up to rounding for any step size."""
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


def test_gradient_matches_oracle_adjoint():
    n = (12, 10, 8)
    nsteps, K = 10, 4
    U0, dx, dt, obs, obs_t, phi0, Pi0, ref = setup(n, nsteps, 6)
    phi = phi0.clone().requires_grad_(True)
    Pi = Pi0.clone().requires_grad_(True)
    J = adjoint.misfit(phi, Pi, obs_t, ref, dx, dt, nsteps, checkpoint_every=K)
    J.backward()
    Jo, gphi_o, gPi_o = oracle.misfit_gradient(U0[0], U0[1], dx, dt, nsteps, obs,
                                               ref.cpu().numpy())
    assert J.item() == pytest.approx(Jo, rel=1e-10)
    s = max(np.abs(gphi_o).max(), np.abs(gPi_o).max())
    assert np.abs(phi.grad.cpu().numpy() - gphi_o).max() < 1e-10 * s
    assert np.abs(Pi.grad.cpu().numpy() - gPi_o).max() < 1e-10 * s


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


def fd_check(n, nsteps, nobs, ndir, K, precision, rel):
    U0, dx, dt, obs, obs_t, phi0, Pi0, ref = setup(n, nsteps, nobs, seed=1, precision=precision)
    phi = phi0.clone().requires_grad_(True)
    Pi = Pi0.clone().requires_grad_(True)
    J = adjoint.misfit(phi, Pi, obs_t, ref, dx, dt, nsteps, precision=precision, checkpoint_every=K)
    J.backward()
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
    assert worst < rel, worst


def test_finite_differences_small():
    fd_check((14, 12, 10), 12, 8, 4, 5, capi.SF_FP64, 1e-7)


def test_finite_differences_full_config_fp64():
    # 128^3, 200 RK4 steps, 64 observers, checkpoints every 20 steps, 16 directions
    fd_check((128, 128, 128), 200, 64, 16, 20, capi.SF_FP64, 1e-6)
