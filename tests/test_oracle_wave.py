"""Pins of the oracle's wave system, RK drivers and adjoint (Sec. IV.A, II.C).

* A single grid Fourier mode evolves under the fully discrete scheme as
  P(dt M_k)^n with M_k the 5x5 matrix of stencil symbols and P the RK
  amplification polynomial: a closed form that catches any wrong term, sign
  or stage weight.
* 4th-order convergence to the continuum plane wave (the paper's claim, Sec. IV.A).
* Energy 1/2 sum(Pi^2 + |d|^2) never increases with sigma > 0.
* <L u, v> = <u, L^T v> for the transposed operator, and the misfit
  gradient agrees with central differences (exact for a quadratic misfit).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1806_04182_gb300 import inputs


def mode_matrix(theta, h, sigma):
    """Symbols of the semi-discrete wave operator on e^{i theta . j}."""
    dsym = [1j * (8 * math.sin(t) - math.sin(2 * t)) / (6 * hh) for t, hh in zip(theta, h)]
    q = -sigma * sum(math.sin(t / 2) ** 6 / hh for t, hh in zip(theta, h))
    M = np.zeros((5, 5), dtype=complex)
    M[0, 0] = q
    M[0, 1] = -1
    M[1, 1] = q
    for d in range(3):
        M[1, 2 + d] = -dsym[d]
        M[2 + d, 1] = -dsym[d]
        M[2 + d, 2 + d] = q
    return M


def poly_step(M, dt, order):
    Z = dt * M
    P = np.eye(5, dtype=complex)
    term = np.eye(5, dtype=complex)
    for m in range(1, order + 1):
        term = term @ Z / m
        P = P + term
    return P


def mode_data(n, kvec, amp):
    nx, ny, nz = n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = 2 * math.pi * (kvec[0] * i / nx + kvec[1] * j / ny + kvec[2] * k / nz)
    e = np.exp(1j * ph)
    return np.stack([np.real(a * e) for a in amp]), (2 * math.pi * kvec[0] / nx,
                                                    2 * math.pi * kvec[1] / ny,
                                                    2 * math.pi * kvec[2] / nz)


@pytest.mark.parametrize("rk", ["rk4", "ssprk3"])
def test_single_mode_closed_form(rk):
    n = (8, 6, 10)
    h = (0.11, 0.13, 0.07)
    sigma = 0.1
    kvec = (1, 2, 3)
    amp = np.array([0.3 + 0.2j, -0.5 + 0.1j, 0.25j, 0.4, -0.1 - 0.3j])
    U0, theta = mode_data(n, kvec, amp)
    U = oracle.ghosted(U0)
    dt = 0.02
    p = oracle.params(sigma=sigma)
    order = 4 if rk == "rk4" else 3
    S = poly_step(mode_matrix(theta, h, sigma), dt, order)
    a = amp.copy()
    for _ in range(3):
        if rk == "rk4":
            oracle.rk4_step(oracle.WAVE, U, h, dt, p)
        else:
            oracle.ssprk3_step(oracle.WAVE, U, h, dt, p)
        a = S @ a
    want, _ = mode_data(n, kvec, a)
    np.testing.assert_allclose(oracle.interior(U), want, atol=2e-14, rtol=0)


def test_ssprk3_equals_shu_osher_form():
    # App. D's k-form and the Shu-Osher convex form are the same method.
    U0, dx = inputs.wave_plane((6, 7, 5), seed=1)
    U0 = U0 + inputs.wave_noise((6, 7, 5), seed=2, amp=0.1)
    dt = 0.01
    U = oracle.ghosted(U0.copy())
    st = oracle.ssprk3_step(oracle.WAVE, U, dx, dt, stages=True)
    L = lambda V: oracle.rhs(oracle.WAVE, oracle.ghosted(V), dx)
    U1 = U0 + dt * L(U0)
    U2 = 0.75 * U0 + 0.25 * (U1 + dt * L(U1))
    U3 = U0 / 3.0 + 2.0 / 3.0 * (U2 + dt * L(U2))
    np.testing.assert_allclose(st[0], U1, atol=1e-14)
    np.testing.assert_allclose(st[1], U2, atol=1e-14)
    np.testing.assert_allclose(st[2], U3, atol=1e-14)


def test_fourth_order_convergence_to_plane_wave():
    errs = []
    for N in (12, 24):
        U0, dx = inputs.wave_plane((N, N, N), k=(1, 2, 1))
        U = oracle.ghosted(U0)
        dt = 0.25 * dx[0]
        T = 0.125
        ns = int(round(T / dt))
        for _ in range(ns):
            oracle.rk4_step(oracle.WAVE, U, dx, dt, oracle.params(sigma=0.1))
        Ue, _ = inputs.wave_plane((N, N, N), k=(1, 2, 1), t=ns * dt)
        errs.append(np.abs(oracle.interior(U) - Ue).sum() / np.abs(Ue).sum())
    order = math.log2(errs[0] / errs[1])
    assert 3.7 < order < 4.5, (errs, order)


def test_energy_non_increasing_with_dissipation():
    U0, dx = inputs.wave_plane((10, 10, 10), seed=3)
    U0 = U0 + inputs.wave_noise((10, 10, 10), seed=4, amp=0.5)
    U = oracle.ghosted(U0)
    dt = 0.25 * dx[0]
    E = [oracle.wave_energy(U, dx)]
    for _ in range(6):
        oracle.rk4_step(oracle.WAVE, U, dx, dt, oracle.params(sigma=0.1))
        E.append(oracle.wave_energy(U, dx))
    assert all(b <= a for a, b in zip(E, E[1:])), E
    assert E[-1] < E[0] * 0.999  # grid-scale noise is damped


def test_energy_loss_without_dissipation_matches_rk4_amplification():
    # A single mode with sigma = 0: the semi-discrete operator is skew, so the
    # energy changes only through |P(i w dt)|^2 per step, w = |D symbol|.
    N = 16
    U0, dx = inputs.wave_plane((N, N, N), k=(1, 1, 1))
    U = oracle.ghosted(U0)
    dt = 0.25 * dx[0]
    E0 = oracle.wave_energy(U, dx)
    steps = 4
    for _ in range(steps):
        oracle.rk4_step(oracle.WAVE, U, dx, dt, oracle.params(sigma=0.0))
    E1 = oracle.wave_energy(U, dx)
    t = 2 * math.pi / N
    w = math.sqrt(3) * (8 * math.sin(t) - math.sin(2 * t)) / (6 * dx[0])
    z = 1j * w * dt
    P = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    assert E1 / E0 == pytest.approx(abs(P) ** (2 * steps), rel=1e-12)
    assert E1 < E0


def test_adjoint_operator_is_transpose():
    n = (6, 7, 5)
    dx = (0.1, 0.12, 0.09)
    u = inputs.wave_noise(n, seed=11)
    v = inputs.wave_noise(n, seed=12)
    Lu = oracle.rhs(oracle.WAVE, oracle.ghosted(u), dx)
    LTv = oracle.rhs(oracle.WAVE_ADJ, oracle.ghosted(v), dx)
    a, b = np.sum(Lu * v), np.sum(u * LTv)
    assert a == pytest.approx(b, rel=1e-12)


def test_misfit_gradient_matches_central_differences():
    n = (8, 8, 8)
    U0, dx = inputs.wave_plane(n, seed=5)
    phi0, Pi0 = U0[0].copy(), U0[1].copy()
    dt = 0.25 * dx[0]
    nsteps = 6
    obs = inputs.observers(n, 5, seed=6)
    ref = 0.1 * inputs.uniform(7, nsteps * obs.size).reshape(nsteps, obs.size)
    J, gphi, gPi = oracle.misfit_gradient(phi0, Pi0, dx, dt, nsteps, obs, ref)
    for s in range(3):
        vphi = inputs.normal(100 + s, phi0.size).reshape(phi0.shape)
        vPi = inputs.normal(200 + s, Pi0.size).reshape(Pi0.shape)
        eps = 1e-3
        Jp = oracle.misfit_gradient(phi0 + eps * vphi, Pi0 + eps * vPi, dx, dt, nsteps, obs, ref)[0]
        Jm = oracle.misfit_gradient(phi0 - eps * vphi, Pi0 - eps * vPi, dx, dt, nsteps, obs, ref)[0]
        fd = (Jp - Jm) / (2 * eps)
        an = np.sum(gphi * vphi) + np.sum(gPi * vPi)
        assert an == pytest.approx(fd, rel=1e-8)
