"""Pins of the oracle's sub-cycling arithmetic: the dense output of App. C and
Berger-Oliger without order reduction (BOR) of App. D.

What fixes the expected values, independently of the formulas under test:
* theta = 0 and theta = 1 of the dense output give U^n and the oracle's own
  RK step U^{n+1} (a separate function, on a real right-hand side);
* the theta-derivatives agree with an exact 5-point difference of the
  (cubic) interpolant;
* for a forcing f(t) alone (f_U = 0) the solution is a polynomial in t: the
  interpolant of order q reproduces it exactly, and the BOR fine stages equal
  the fine RK stages built from the exact solution and f;
* with R = 1 the BOR fine stages are the coarse RK4 stages themselves, for
  any increments (an algebraic identity that every coefficient of App. D,
  including the sign of b_4's cubic term, takes part in);
* on a linear system U' = A U (f_U != 0) the BOR stage values approach the
  exact fine stage values at 4th order (RK4) as dt halves.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1806_04182_gb300 import inputs

RK4, SSP = oracle.RK4, oracle.SSPRK3


def _rk_ks(system, U, dx, dt, rk, p=None):
    """Coarse increments k_j = dt L(U^(j)) from the oracle RHS and the stage
    inputs that the oracle's own RK step produces."""
    p = p or oracle.params()
    U0 = U.copy()
    Uw = U.copy()
    if rk == RK4:
        st = oracle.rk4_step(system, Uw, dx, dt, p, stages=True)
        inputs_ = [oracle.interior(U0)] + [st[0], st[1], st[2]]
    else:
        st = oracle.ssprk3_step(system, Uw, dx, dt, p, stages=True)
        inputs_ = [oracle.interior(U0)] + [st[0], st[1]]
    ks = []
    for S in inputs_:
        G = oracle.ghosted(np.ascontiguousarray(S))
        ks.append(dt * oracle.rhs(system, G, dx, p))
    return np.array(ks), st


@pytest.mark.parametrize("rk", [RK4, SSP])
def test_dense_output_endpoints_match_rk_step(rk):
    U0, dx = inputs.wave_plane((6, 5, 4), seed=3)
    U = oracle.ghosted(U0)
    dt = 0.2 * min(dx)
    k, st = _rk_ks(oracle.WAVE, U, dx, dt, rk)
    Un = oracle.interior(U)
    np.testing.assert_array_equal(oracle.dense_output(rk, Un, k, dt, 0.0), Un)
    got = oracle.dense_output(rk, Un, k, dt, 1.0)
    want = st[-1]
    assert np.abs(got - want).max() <= 1e-14 * np.abs(want).max()


@pytest.mark.parametrize("rk", [RK4, SSP])
@pytest.mark.parametrize("theta", [0.25, 0.5, 0.75])
def test_dense_output_derivatives_are_theta_derivatives(rk, theta):
    rng = np.random.default_rng(5)
    s = 4 if rk == RK4 else 3
    Un = rng.standard_normal(7)
    k = rng.standard_normal((s, 7))
    dt = 0.5
    h = 0.125  # the interpolant is a cubic in theta: the 5-point formula is exact
    for m in (1, 2, 3):
        f = [oracle.dense_output(rk, Un, k, dt, theta + o * h, m - 1) for o in (-2, -1, 1, 2)]
        fd = (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h) / dt
        got = oracle.dense_output(rk, Un, k, dt, theta, m)
        np.testing.assert_allclose(got, fd, rtol=1e-12, atol=1e-12)


def _forcing(rk):
    """A forcing f(t) of the interpolant's degree minus one and its integral."""
    if rk == RK4:
        c = (0.7, -1.3, 2.1)        # f = c0 + c1 t + c2 t^2, U cubic
    else:
        c = (0.7, -1.3, 0.0)        # f linear, U quadratic
    f = lambda t: c[0] + c[1] * t + c[2] * t * t
    df = lambda t: c[1] + 2 * c[2] * t
    ddf = lambda t: 2 * c[2]
    U = lambda t: 0.4 + c[0] * t + c[1] * t * t / 2 + c[2] * t ** 3 / 3
    return f, df, ddf, U


@pytest.mark.parametrize("rk", [RK4, SSP])
def test_dense_output_exact_on_polynomial_solutions(rk):
    f, df, ddf, U = _forcing(rk)
    tn, dt = 0.3, 0.4
    cs = (0.0, 0.5, 0.5, 1.0) if rk == RK4 else (0.0, 1.0, 0.5)
    k = np.array([[dt * f(tn + c * dt)] for c in cs])
    Un = np.array([U(tn)])
    for th in (0.0, 0.2, 1.0 / 3.0, 0.5, 0.9, 1.0):
        t = tn + th * dt
        assert oracle.dense_output(rk, Un, k, dt, th)[0] == pytest.approx(U(t), rel=1e-14)
        assert oracle.dense_output(rk, Un, k, dt, th, 1)[0] == pytest.approx(f(t), rel=1e-13, abs=1e-13)
        assert oracle.dense_output(rk, Un, k, dt, th, 2)[0] == pytest.approx(df(t), rel=1e-12, abs=1e-12)
        if rk == RK4:
            assert oracle.dense_output(rk, Un, k, dt, th, 3)[0] == pytest.approx(ddf(t), rel=1e-11)


@pytest.mark.parametrize("rk", [RK4, SSP])
@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_bor_fine_stages_equal_fine_rk_stages_for_polynomial_forcing(rk, R):
    f, df, ddf, U = _forcing(rk)
    tn, dt = 0.3, 0.4
    cs = (0.0, 0.5, 0.5, 1.0) if rk == RK4 else (0.0, 1.0, 0.5)
    k = np.array([[dt * f(tn + c * dt)] for c in cs])
    Un = np.array([U(tn)])
    h = dt / R
    for r in range(R):
        t = tn + r * h
        got = oracle.bor_fine_stages(rk, Un, k, dt, R, r)[:, 0]
        u = U(t)
        if rk == RK4:
            k1, k2, k4 = h * f(t), h * f(t + h / 2), h * f(t + h)
            want = [u, u + k1 / 2, u + k2 / 2, u + k2, u + (k1 + 4 * k2 + k4) / 6]
        else:
            k1, k2, k3 = h * f(t), h * f(t + h), h * f(t + h / 2)
            want = [u, u + k1, u + k1 / 4 + k2 / 4, u + (k1 + k2 + 4 * k3) / 6]
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-14)
        # the end value of an exact-polynomial step is the exact solution
        assert got[-1] == pytest.approx(U(t + h), rel=1e-13)


@pytest.mark.parametrize("system", [oracle.WAVE, oracle.Z4])
def test_bor_with_ratio_one_gives_the_coarse_rk4_stages(system):
    if system == oracle.WAVE:
        U0, dx = inputs.wave_plane((6, 5, 4), seed=4)
    else:
        U0, dx = inputs.z4_perturbed((6, 5, 4), seed=4, amp=0.05)
    U = oracle.ghosted(U0)
    dt = 0.2 * min(dx)
    k, st = _rk_ks(system, U, dx, dt, RK4)
    Un = oracle.interior(U)
    got = oracle.bor_fine_stages(RK4, Un, k, dt, 1, 0)
    np.testing.assert_array_equal(got[0], Un)
    for s in range(4):
        want = st[s]
        scale = np.abs(want - Un).max()
        assert np.abs(got[s + 1] - want).max() <= 1e-12 * max(scale, 1e-300) + 1e-15 * np.abs(want).max()


def test_bor_with_ratio_one_for_random_increments():
    # the identity holds for any k_j, not only for those of a smooth problem
    rng = np.random.default_rng(11)
    Un = rng.standard_normal(9)
    k = rng.standard_normal((4, 9))
    got = oracle.bor_fine_stages(RK4, Un, k, 0.37, 1, 0)
    want = [Un, Un + k[0] / 2, Un + k[1] / 2, Un + k[2], Un + (k[0] + 2 * k[1] + 2 * k[2] + k[3]) / 6]
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def _linear_system():
    # a damped rotation plus a growing mode: U' = A U, exact U(t) = expm(A t) U0
    A = np.array([[-0.3, 2.0, 0.0], [-2.0, -0.3, 0.5], [0.0, 0.0, 0.8]])
    w, V = np.linalg.eig(A)
    Vi = np.linalg.inv(V)
    expm = lambda t: (V @ np.diag(np.exp(w * t)) @ Vi).real
    return A, expm


def _rk4_ks(A, U, dt):
    k1 = dt * A @ U
    k2 = dt * A @ (U + k1 / 2)
    k3 = dt * A @ (U + k2 / 2)
    k4 = dt * A @ (U + k3)
    return np.array([k1, k2, k3, k4])


@pytest.mark.parametrize("R", [2, 3])
def test_bor_fourth_order_on_a_linear_system(R):
    A, expm = _linear_system()
    U0 = np.array([1.0, -0.5, 0.3])
    errs = []
    for dt in (0.1, 0.05):
        k = _rk4_ks(A, U0, dt)
        h = dt / R
        e = 0.0
        for r in range(R):
            got = oracle.bor_fine_stages(RK4, U0, k, dt, R, r)
            u = expm(r * h) @ U0
            k1 = h * A @ u
            k2 = h * A @ (u + k1 / 2)
            k3 = h * A @ (u + k2 / 2)
            want = [u, u + k1 / 2, u + k2 / 2, u + k3]
            for s in range(4):
                e = max(e, np.abs(got[s] - want[s]).max())
        errs.append(e)
    order = math.log2(errs[0] / errs[1])
    assert 3.7 < order < 4.6, (errs, order)


def test_bor_rejects_bad_arguments():
    with pytest.raises(ValueError):
        oracle.bor_fine_stages(RK4, np.zeros(2), np.zeros((4, 2)), 0.1, 2, 2)
    with pytest.raises(ValueError):
        oracle.bor_fine_stages(RK4, np.zeros(2), np.zeros((4, 2)), 0.1, 0, 0)
