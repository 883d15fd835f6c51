"""Pins of the radiative boundary condition in the oracle and of the puncture
initial data of Sec. V.

* U = U_inf everywhere: the radiative right-hand side is exactly zero.
* Quartic data: every derivative stencil the condition uses (centred,
  off-centred and fully one-sided, at both ends of every axis) is exact on
  polynomials of degree 4, so the right-hand side equals its closed form
  -v x.grad(p)/r - v p/r at every ghost point.
* An exact outgoing spherical wave U = U_inf + f(r - v t)/r satisfies the
  condition in the continuum; the discrete right-hand side converges to
  dU/dt = -v f'(r)/r at 4th order.
* The RK4 step with radiative ghosts equals the periodic step in the
  interior for data that vanish near the boundary.
* Puncture data: Bowen-York A~ is symmetric and trace-free, psi^6 A~ is
  divergence-free in flat space (the momentum constraint), chi = psi^-4 and
  alpha = psi^-2.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1806_04182_gb300 import inputs

G = 3


def _ghost_mask(n):
    m = np.ones((n[2] + 2 * G, n[1] + 2 * G, n[0] + 2 * G), dtype=bool)
    m[G:-G, G:-G, G:-G] = False
    return m


def _positions(n, dx, x0):
    ax = [x0[d] + dx[d] * np.arange(-G, n[d] + G) for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X, Y, Z


def test_constant_at_infinity_gives_zero():
    n = (6, 7, 5)
    dx, x0 = (0.3, 0.25, 0.4), (-1.0, -0.9, -1.1)
    uinf = np.array([1.0, -2.0, 0.5])
    U = np.ones((3,) + _ghost_mask(n).shape) * uinf[:, None, None, None]
    r = oracle.radiative_rhs(U, dx, x0, uinf, 1.0)
    assert np.all(r == 0.0)


def test_quartic_data_closed_form():
    n = (6, 7, 5)
    dx, x0 = (0.25, 0.5, 0.25), (-0.6, -1.7, -0.55)
    X, Y, Z = _positions(n, dx, x0)
    # p = quartic in each coordinate plus a mixed term of degree 3
    p = 0.3 * X ** 4 - 0.2 * X ** 3 + X - 0.5 * Y ** 4 + 0.7 * Y ** 2 + 0.1 * Z ** 4 - Z ** 3 \
        + 0.2 * X * Y * Z
    px = 1.2 * X ** 3 - 0.6 * X ** 2 + 1.0 + 0.2 * Y * Z
    py = -2.0 * Y ** 3 + 1.4 * Y + 0.2 * X * Z
    pz = 0.4 * Z ** 3 - 3.0 * Z ** 2 + 0.2 * X * Y
    uinf, v = 0.75, 1.3
    U = (uinf + p)[None]
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    want = -v * (X * px + Y * py + Z * pz) / r - v * p / r
    got = oracle.radiative_rhs(np.ascontiguousarray(U), dx, x0, [uinf], [v])[0]
    m = _ghost_mask(n)
    np.testing.assert_allclose(got[m], want[m], rtol=1e-11, atol=1e-11)
    assert np.all(got[~m] == 0.0)


def test_outgoing_spherical_wave_fourth_order():
    # f(s) = exp(-(s - s0)^2 / w^2); dU/dt = -v f'(r) / r at t = 0
    v, s0, w = 1.0, 2.2, 0.6
    errs = []
    for N in (16, 32):
        n = (N, N, N)
        dx, x0 = inputs.z4_puncture_box(n, 4.0)
        X, Y, Z = _positions(n, dx, x0)
        r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
        f = np.exp(-((r - s0) / w) ** 2)
        fp = -2 * (r - s0) / w ** 2 * f
        U = (0.5 + f / r)[None]
        got = oracle.radiative_rhs(np.ascontiguousarray(U), dx, x0, [0.5], [v])[0]
        want = -v * fp / r
        m = _ghost_mask(n)
        errs.append(np.abs(got[m] - want[m]).max())
    order = math.log2(errs[0] / errs[1])
    assert 3.5 < order < 4.7, (errs, order)


def test_radiative_step_equals_periodic_step_for_compact_data():
    n = (40, 40, 40)
    dx = (1 / 40,) * 3
    x0 = (-0.5 + 1 / 80,) * 3
    X, Y, Z = _positions(n, dx, x0)
    r2 = X ** 2 + Y ** 2 + Z ** 2
    # wave data supported within r < 0.1 (4 points): one RK4 step spreads it by
    # 4 stages x 3 points, which stays 3 points inside the interior
    bump = np.where(r2 < 0.01, (1 - r2 / 0.01) ** 6, 0.0)
    Ug = np.stack([bump, 0.5 * bump, 0 * bump, 0 * bump, 0 * bump])
    U1 = np.ascontiguousarray(Ug)
    U2 = U1.copy()
    dt = 0.25 * dx[0]
    oracle.rk4_step_radiative(oracle.WAVE, U1, dx, x0, 0.0, 1.0, dt)
    oracle.rk4_step(oracle.WAVE, U2, dx, dt)
    np.testing.assert_array_equal(oracle.interior(U1), oracle.interior(U2))
    assert np.all(U1[:, _ghost_mask(n)] == 0.0)


def test_radiative_step_stage_outputs():
    # the returned stages are the ghosted stage inputs: U(2) = U + (dt/2) k_1
    # with k_1 at ghost points the radiative right-hand side of U (here a
    # constant offset of the ghost shell over zero interior data)
    n = (8, 8, 8)
    dx, x0 = (0.1,) * 3, (-0.35,) * 3
    U = np.zeros((5, 14, 14, 14))
    m = _ghost_mask(n)
    U[:, m] = 0.01
    dt = 0.02
    st = oracle.rk4_step_radiative(oracle.WAVE, U.copy(), dx, x0, 0.0, 1.0, dt, stages=True)
    k1 = oracle.radiative_rhs(U, dx, x0, 0.0, 1.0)
    np.testing.assert_allclose(st[0][:, m], (U + 0.5 * dt * k1)[:, m], rtol=0, atol=1e-15)
    # the outermost corner sees only ghost values along every axis stencil
    # (fully one-sided, all 0.01): its derivative vanishes and it decays as
    # dU/dt = -v U / r
    X, Y, Z = _positions(n, dx, x0)
    r = np.sqrt(X[0, 0, 0] ** 2 + Y[0, 0, 0] ** 2 + Z[0, 0, 0] ** 2)
    assert k1[0, 0, 0, 0] == pytest.approx(-0.01 / r, rel=1e-12)


def test_puncture_data_properties():
    n = (20, 18, 16)
    U, dx, x0 = inputs.z4_puncture(n, length=6.0)
    h = inputs.z4_puncture(n, length=6.0)
    np.testing.assert_array_equal(U, h[0])
    # trace-free with respect to the flat conformal metric
    tr = U[8] + U[11] + U[13]
    assert np.abs(tr).max() < 1e-13 * np.abs(U[8:14]).max()
    # chi and alpha from psi at one point, recomputed by hand
    i, j, k = 3, 5, 7
    x = np.array([x0[0] + i * dx[0], x0[1] + j * dx[1], x0[2] + k * dx[2]])
    rA = np.linalg.norm(x - np.array([0.05, -0.03, 0.02]))
    psi = 1 + 1.0 / (2 * rA)
    assert U[0, k, j, i] == pytest.approx(psi ** -4, rel=1e-14)
    assert U[18, k, j, i] == pytest.approx(psi ** -2, rel=1e-14)
    assert U[1, k, j, i] == 1.0 and U[2, k, j, i] == 0.0


def test_bowen_york_momentum_constraint():
    # psi^6 A~_ij = A^_ij solves d_j A^_ij = 0 in flat space away from the
    # hole: 4th-order differences of the exact field converge to zero
    hole = dict(m=0.8, pos=(0.0, 0.0, 0.0), P=(0.3, -0.2, 0.1), S=(0.1, 0.25, -0.15))
    res = []
    for N in (24, 48):
        n = (N, N, N)
        U, dx, x0 = inputs.z4_puncture(n, length=4.0, holes=[hole])
        chi = U[0]
        psi6 = chi ** -1.5
        idx = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
        Ahat = np.zeros((3, 3) + chi.shape)
        for q, (a, b) in enumerate(idx):
            Ahat[a, b] = Ahat[b, a] = psi6 * U[8 + q]
        div = np.zeros((3,) + chi.shape)
        for a in range(3):
            for b in range(3):
                axis = 2 - b
                f = Ahat[a, b]
                d = (np.roll(f, 2, axis) - 8 * np.roll(f, 1, axis) + 8 * np.roll(f, -1, axis)
                     - np.roll(f, -2, axis)) / (12 * dx[b])
                div[a] += d
        # sample a shell 1 < r < 1.5 (away from the hole and from the box edge)
        ax = [x0[d] + dx[d] * np.arange(n[d]) for d in range(3)]
        Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
        sel = (r > 1.0) & (r < 1.5)
        res.append(np.abs(div[:, sel]).max() / np.abs(Ahat[:, :, sel]).max())
    order = math.log2(res[0] / res[1])
    assert order > 3.5, (res, order)
