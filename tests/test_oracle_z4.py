"""Pins of the oracle's CCZ4 right-hand side (Sec. V) against exact solutions.

* Minkowski data: every stencil of a constant is exactly zero and ln 1 = 0,
  so the whole RHS is bitwise zero.
* Gauge wave (harmonic slicing, zero frozen shift) is an exact solution of
  the Einstein equations written from the line element of Sec. V: the
  discrete RHS approaches its exact time derivative at 4th order, and a few
  RK4 steps converge to the moving solution.
* Flat space in curvilinear coordinates x' = x + xi(x) (metric = pull-back of
  delta, K = 0): the Ricci tensor vanishes geometrically, so every RHS
  component is a pure truncation error -> 0 at 4th order.  This checks the
  Christoffel symbols and both Ricci pieces independently of the CCZ4 text.
* The same flat metric with a non-trivial lapse: d/dt Khat = -Laplacian(alpha)
  and d/dt A~_ij = -chi [nabla_i nabla_j alpha]^TF, computed here with SymPy
  from the physical metric (Laplace-Beltrami, physical Christoffels).
* Z^i / Theta coupling terms vanish on all of these; they are pinned on
  homogeneous states (test_oracle_z4_homogeneous.py) and on polynomial states
  with gradients and shift (test_oracle_z4_polynomial.py) against the damped
  covariant Z4 equations.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1806_04182_gb300 import inputs


def test_minkowski_rhs_is_bitwise_zero():
    U = oracle.ghosted(inputs.z4_minkowski((5, 6, 7)))
    for slicing in (0, 1):
        r = oracle.rhs(oracle.Z4, U, (0.1, 0.2, 0.3), oracle.params(slicing=slicing))
        assert np.all(r == 0.0)


def exact_dt(fn, n, t=0.0, h=1e-4):
    a = fn(n, t=t - 2 * h)[0]
    b = fn(n, t=t - h)[0]
    c = fn(n, t=t + h)[0]
    d = fn(n, t=t + 2 * h)[0]
    return (a - 8 * b + 8 * c - d) / (12 * h)


def test_gauge_wave_truncation_is_fourth_order():
    p = oracle.params(slicing=1, shift_frozen=1)
    errs = []
    for N in (16, 32):
        n = (N, 4, 4)
        U0, dx = inputs.z4_gauge_wave(n)
        r = oracle.rhs(oracle.Z4, oracle.ghosted(U0), dx, p)
        errs.append(np.abs(r - exact_dt(inputs.z4_gauge_wave, n)).max())
    assert errs[1] < 1e-4
    assert errs[0] / errs[1] > 14.0, errs


def test_gauge_wave_evolution_converges():
    p = oracle.params(slicing=1, shift_frozen=1, sigma=0.0)
    errs = []
    T = 0.05
    for N in (16, 32):
        n = (N, 3, 3)
        U0, dx = inputs.z4_gauge_wave(n)
        U = oracle.ghosted(U0)
        ns = int(round(T / (0.25 * dx[0])))
        dt = T / ns
        for _ in range(ns):
            oracle.rk4_step(oracle.Z4, U, dx, dt, p)
        Ue, _ = inputs.z4_gauge_wave(n, t=T)
        errs.append(np.abs(oracle.interior(U) - Ue).max())
    assert errs[0] / errs[1] > 12.0, errs


# ------------------------------------------------------------------ SymPy pins
sp = pytest.importorskip("sympy")


def curvilinear_flat(lapse_amp):
    """SymPy closed forms for flat space in coordinates x' = x + xi(x)."""
    x, y, z = sp.symbols("x y z", real=True)
    X = (x, y, z)
    tp = 2 * sp.pi
    xi = (sp.Rational(2, 100) * sp.sin(tp * y) + sp.Rational(1, 100) * sp.sin(tp * z),
          sp.Rational(15, 1000) * sp.sin(tp * z + sp.Rational(3, 10)) + sp.Rational(1, 100) * sp.cos(tp * x),
          sp.Rational(2, 100) * sp.sin(tp * x + sp.Rational(7, 10)) + sp.Rational(1, 100) * sp.sin(tp * y))
    J = sp.Matrix(3, 3, lambda a, i: (1 if a == i else 0) + sp.diff(xi[a], X[i]))
    gam = (J.T * J).applyfunc(sp.expand)
    detJ = J.det()
    detg = detJ ** 2
    chi = detg ** sp.Rational(-1, 3)
    gt = gam * chi
    igam = J.inv() * J.inv().T  # gamma^{ij} = (J^T J)^{-1}
    igt = igam / chi
    Gt = [-sum(sp.diff(igt[i, j], X[j]) for j in range(3)) for i in range(3)]
    alpha = 1 + lapse_amp * sp.sin(tp * x + sp.Rational(1, 5)) * sp.cos(tp * z)
    dal = [sp.diff(alpha, v) for v in X]
    # physical Christoffels Gamma^k_ij and nabla_i nabla_j alpha
    dgam = [[[sp.diff(gam[i, j], X[k]) for k in range(3)] for j in range(3)] for i in range(3)]
    Chr = [[[sum(igam[k, l] * (dgam[l][j][i] + dgam[l][i][j] - dgam[i][j][l]) for l in range(3)) / 2
             for j in range(3)] for i in range(3)] for k in range(3)]
    DD = sp.Matrix(3, 3, lambda i, j: sp.diff(alpha, X[i], X[j]) - sum(Chr[k][i][j] * dal[k] for k in range(3)))
    lap = sum(igam[i, j] * DD[i, j] for i in range(3) for j in range(3))
    ATF = -chi * (DD - gam * lap / 3)
    return X, dict(chi=chi, gt=gt, Gt=Gt, alpha=alpha, dKh=-lap, dAt=ATF)


def evaluate(expr, X, n, dx):
    nx, ny, nz = n
    f = sp.lambdify(X, expr, "numpy")
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v = f(i * dx[0], j * dx[1], k * dx[2])
    return np.broadcast_to(np.asarray(v, dtype=np.float64), (nz, ny, nx)).copy()


SYM = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def curvilinear_data(cf, X, n):
    dx = tuple(1.0 / m for m in n)
    U = np.zeros((25,) + (n[2], n[1], n[0]))
    U[0] = evaluate(cf["chi"], X, n, dx)
    for s, (a, b) in enumerate(SYM):
        U[1 + s] = evaluate(cf["gt"][a, b], X, n, dx)
    for a in range(3):
        U[14 + a] = evaluate(cf["Gt"][a], X, n, dx)
    U[18] = evaluate(cf["alpha"], X, n, dx)
    return U, dx


@pytest.fixture(scope="module")
def flat_forms():
    return curvilinear_flat(0), curvilinear_flat(sp.Rational(3, 100))


def test_flat_curvilinear_rhs_vanishes_at_fourth_order(flat_forms):
    X, cf = flat_forms[0]
    p = oracle.params(sigma=0.0)
    errs = []
    for N in (12, 24):
        U0, dx = curvilinear_data(cf, X, (N, N, N))
        r = oracle.rhs(oracle.Z4, oracle.ghosted(U0), dx, p)
        errs.append(np.abs(r).max())
    assert errs[0] / errs[1] > 13.0, errs


def test_lapse_second_derivatives_in_curvilinear_flat_space(flat_forms):
    X, cf = flat_forms[1]
    p = oracle.params(sigma=0.0)
    errs = []
    for N in (12, 24):
        n = (N, N, N)
        U0, dx = curvilinear_data(cf, X, n)
        r = oracle.rhs(oracle.Z4, oracle.ghosted(U0), dx, p)
        want = np.zeros_like(r)
        want[7] = evaluate(cf["dKh"], X, n, dx)
        for s, (a, b) in enumerate(SYM):
            want[8 + s] = evaluate(cf["dAt"][a, b], X, n, dx)
        assert np.abs(want[7]).max() > 0.1  # the check is not vacuous
        errs.append(np.abs(r - want).max())
    assert errs[0] / errs[1] > 13.0, errs


def test_noise_is_not_amplified():
    # Robust-stability data: grid-scale noise first redistributes into the
    # derived fields (amplitude ~ noise / (k dx) for grid modes), after which
    # the norm must not grow: KO dissipation damps it.
    n = (12, 12, 12)
    U0, dx = inputs.z4_minkowski_noise(n, seed=1, amp=1e-10)
    U = oracle.ghosted(U0)
    base = oracle.ghosted(inputs.z4_minkowski(n))
    dt = 0.25 * dx[0]
    rms = []
    for s in range(40):
        oracle.rk4_step(oracle.Z4, U, dx, dt)
        if s + 1 in (10, 40):
            rms.append(np.sqrt(np.mean(oracle.interior(U - base) ** 2)))
    assert rms[1] < rms[0] < 1e-8, rms


def test_monitors_on_exact_data():
    U, dx = inputs.z4_gauge_wave((16, 4, 4))
    m = oracle.z4_monitors(oracle.ghosted(U), dx)
    assert m[0] == 0.0          # Theta
    assert m[2] < 1e-15         # ln det gt = 0 analytically
    assert m[3] < 1e-15         # tr A~ = 0 analytically
    assert 0 < m[1] < 1e-4      # Z ~ truncation error of Gamma~


def test_lopsided_advection_converges_to_centred():
    # with a non-zero shift, one-sided and centred advection differ by the
    # stencils' truncation only: the RHS difference falls at 4th order
    errs = []
    for N in (16, 32):
        U0, dx = inputs.z4_perturbed((N, N, N), seed=9, amp=0.05)
        G = oracle.ghosted(U0)
        a = oracle.rhs(oracle.Z4, G, dx, oracle.params(lopsided=0))
        b = oracle.rhs(oracle.Z4, G, dx, oracle.params(lopsided=1))
        errs.append(np.abs(a - b).max())
    assert errs[0] > 0 and errs[0] / errs[1] > 13.0, errs


def test_bench_flop_constant_is_the_oracle_count():
    # bench.py reports the ALU roofline with the per-cell operation count of
    # the CCZ4 right-hand side; it must be the count of the counting scalar
    import bench
    U, dx = inputs.z4_perturbed((6, 6, 6), seed=1, amp=0.05)
    c = oracle.count_ops(oracle.Z4, oracle.ghosted(U), dx)
    assert c["add"] + c["mul"] + c["div"] + c["log"] == bench.FLOPS_PER_CELL_UPDATE, c
