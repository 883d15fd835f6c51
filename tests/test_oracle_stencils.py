"""Pins of the Sec. II.B.1 stencils in the oracle, against closed forms.

Each operator is checked against what the mathematics fixes, not against a
retyped copy of its coefficients: polynomial exactness up to the degree the
4th-order truncation allows (exact rational values), and the Fourier symbol
on a single grid mode.  A wrong coefficient, sign or offset fails one of them.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

G = 3
N = (6, 7, 5)
H = (0.5, 0.25, 1.0)  # exactly representable spacings


def poly_field(fn):
    """Ghosted single-field array with u = fn(x, y, z) at x = i*hx etc. (no ghost fill)."""
    nx, ny, nz = N
    U = np.zeros((1, nz + 2 * G, ny + 2 * G, nx + 2 * G))
    for k in range(-G, nz + G):
        for j in range(-G, ny + G):
            for i in range(-G, nx + G):
                x, y, z = Fraction(i) * Fraction(H[0]), Fraction(j) * Fraction(H[1]), Fraction(k) * Fraction(H[2])
                U[0, k + G, j + G, i + G] = float(fn(x, y, z))
    return U


def coord(d, i, j, k):
    return Fraction((i, j, k)[d]) * Fraction(H[d])


def test_first_derivative_exact_on_quartics():
    # D_d is 4th order: exact for every polynomial of degree <= 4.
    c = [3, -2, 5, 1, -4]
    for d in range(3):
        fn = lambda x, y, z, d=d: sum(Fraction(c[p]) * (x, y, z)[d] ** p for p in range(5)) + y * z
        dfn = lambda x, y, z, d=d: sum(Fraction(p * c[p]) * (x, y, z)[d] ** (p - 1) for p in range(1, 5)) + \
            (z if d == 1 else 0) + (y if d == 2 else 0)
        U = poly_field(fn)
        for (i, j, k) in [(0, 0, 0), (2, 3, 1), (5, 6, 4)]:
            got = oracle.stencil(oracle.D1, U, H, 0, i, j, k, d1=d)
            want = dfn(coord(0, i, j, k), coord(1, i, j, k), coord(2, i, j, k))
            assert got == pytest.approx(float(want), rel=1e-14, abs=1e-12)


def test_first_derivative_not_exact_on_quintic():
    # the truncation term -h^4/30 u^(5) must show on x^5: pins the order itself
    U = poly_field(lambda x, y, z: x ** 5)
    i = 2
    x = Fraction(i) * Fraction(H[0])
    got = oracle.stencil(oracle.D1, U, H, 0, i, 1, 1, d1=0)
    want = 5 * x ** 4 - Fraction(H[0]) ** 4 / 30 * 120
    assert got == pytest.approx(float(want), rel=1e-14)


def test_second_derivative_exact_on_quintics():
    c = [1, 2, -3, 4, -1, 2]
    for d in range(3):
        fn = lambda x, y, z, d=d: sum(Fraction(c[p]) * (x, y, z)[d] ** p for p in range(6))
        d2fn = lambda x, y, z, d=d: sum(Fraction(p * (p - 1) * c[p]) * (x, y, z)[d] ** (p - 2)
                                        for p in range(2, 6))
        U = poly_field(fn)
        for (i, j, k) in [(0, 0, 0), (3, 2, 2), (5, 6, 4)]:
            got = oracle.stencil(oracle.D2, U, H, 0, i, j, k, d1=d)
            want = d2fn(coord(0, i, j, k), coord(1, i, j, k), coord(2, i, j, k))
            assert got == pytest.approx(float(want), rel=1e-13, abs=1e-10)


def test_mixed_derivative_exact_on_products_of_quartics():
    for (d1, d2) in [(0, 1), (0, 2), (1, 2)]:
        def fn(x, y, z, d1=d1, d2=d2):
            a, b = (x, y, z)[d1], (x, y, z)[d2]
            return (a ** 4 - 2 * a ** 3 + a) * (b ** 4 + 3 * b ** 2 - b)

        def want_fn(x, y, z, d1=d1, d2=d2):
            a, b = (x, y, z)[d1], (x, y, z)[d2]
            return (4 * a ** 3 - 6 * a ** 2 + 1) * (4 * b ** 3 + 6 * b - 1)

        U = poly_field(fn)
        for (i, j, k) in [(0, 0, 0), (2, 4, 3), (5, 6, 4)]:
            got = oracle.stencil(oracle.DMIX, U, H, 0, i, j, k, d1=d1, d2=d2)
            got_swapped = oracle.stencil(oracle.DMIX, U, H, 0, i, j, k, d1=d2, d2=d1)
            want = want_fn(coord(0, i, j, k), coord(1, i, j, k), coord(2, i, j, k))
            assert got == pytest.approx(float(want), rel=1e-13, abs=1e-9)
            assert got_swapped == pytest.approx(got, rel=1e-13, abs=1e-9)


def test_ko_annihilates_quintics_and_scales_sextic():
    sigma = 0.3
    U = poly_field(lambda x, y, z: x ** 5 - 3 * y ** 4 * z + z ** 5 + x * y * z)
    assert abs(oracle.stencil(oracle.KO, U, H, 0, 2, 3, 1, sigma=sigma)) < 1e-9
    # delta^6 x^6 = 6! h^6 in each direction
    U = poly_field(lambda x, y, z: x ** 6 + y ** 6 + z ** 6)
    want = sum(sigma / (64 * h) * 720 * h ** 6 for h in H)
    got = oracle.stencil(oracle.KO, U, H, 0, 2, 3, 1, sigma=sigma)
    assert got == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("m", [1, 2, 5])
def test_fourier_symbols(m):
    # single grid mode u_j = cos(theta j) on a periodic line of n points
    n = 12
    theta = 2 * math.pi * m / n
    h = 0.1
    U = np.zeros((1, 1 + 2 * G, 1 + 2 * G, n + 2 * G))
    U[0, G, G, G:G + n] = np.cos(theta * np.arange(n))
    oracle.fill_ghosts(U, G)
    dx = (h, 1.0, 1.0)
    sigma = 0.7
    for i in range(n):
        c, s = math.cos(theta * i), math.sin(theta * i)
        # D: i(8 sin t - sin 2t)/(6h) e^{i t j}  ->  -(8 sin t - sin 2t)/(6h) sin(t i)
        d1 = -(8 * math.sin(theta) - math.sin(2 * theta)) / (6 * h) * s
        # D_xx: -(30 - 32 cos t + 2 cos 2t)/(12 h^2)
        d2 = -(30 - 32 * math.cos(theta) + 2 * math.cos(2 * theta)) / (12 * h * h) * c
        # Q_d: -sigma sin^6(t/2)/h  (y and z are constant: no contribution)
        ko = -sigma * math.sin(theta / 2) ** 6 / h * c
        assert oracle.stencil(oracle.D1, U, dx, 0, i, 0, 0, d1=0) == pytest.approx(d1, abs=1e-12)
        assert oracle.stencil(oracle.D2, U, dx, 0, i, 0, 0, d1=0) == pytest.approx(d2, abs=1e-10)
        assert oracle.stencil(oracle.KO, U, dx, 0, i, 0, 0, sigma=sigma) == pytest.approx(ko, abs=1e-12)


def test_lopsided_advection_stencils():
    # Sec. II.B.1 one-sided stencils: exact on quartics in both orientations,
    # each reads only the points on its side (i-1..i+3 for beta > 0, i-3..i+1 for
    # beta < 0), and the two mirror stencils share the leading truncation term
    # +h^4/20 u^(5) (sum of coefficient x offset^5 = 72 for both)
    c = [2, -1, 3, 1, -2]
    for d in range(3):
        fn = lambda x, y, z, d=d: sum(Fraction(c[p]) * (x, y, z)[d] ** p for p in range(5))
        dfn = lambda x, y, z, d=d: sum(Fraction(p * c[p]) * (x, y, z)[d] ** (p - 1) for p in range(1, 5))
        U = poly_field(fn)
        for sgn in (1, -1):
            for (i, j, k) in [(1, 1, 1), (3, 4, 2)]:
                got = oracle.stencil(oracle.DLOP, U, H, 0, i, j, k, d1=d, d2=sgn)
                want = dfn(coord(0, i, j, k), coord(1, i, j, k), coord(2, i, j, k))
                assert got == pytest.approx(float(want), rel=1e-13, abs=1e-11)
    # one-sidedness: a spike 2 points behind the upwind side is invisible
    U = np.zeros((1, N[2] + 2 * G, N[1] + 2 * G, N[0] + 2 * G))
    U[0, G + 2, G + 3, G + 3 - 2] = 1.0  # x offset -2 from (3, 3, 2)
    assert oracle.stencil(oracle.DLOP, U, H, 0, 3, 3, 2, d1=0, d2=1) == 0.0
    assert oracle.stencil(oracle.DLOP, U, H, 0, 3, 3, 2, d1=0, d2=-1) != 0.0
    U[...] = 0.0
    U[0, G + 2, G + 3, G + 3 + 2] = 1.0  # x offset +2
    assert oracle.stencil(oracle.DLOP, U, H, 0, 3, 3, 2, d1=0, d2=-1) == 0.0
    assert oracle.stencil(oracle.DLOP, U, H, 0, 3, 3, 2, d1=0, d2=1) != 0.0
    # 4th order: the truncation term h^4/20 * 5! is visible on x^5, equal for both
    U = poly_field(lambda x, y, z: x ** 5)
    x = Fraction(3) * Fraction(H[0])
    plus = oracle.stencil(oracle.DLOP, U, H, 0, 3, 1, 1, d1=0, d2=1) - float(5 * x ** 4)
    minus = oracle.stencil(oracle.DLOP, U, H, 0, 3, 1, 1, d1=0, d2=-1) - float(5 * x ** 4)
    assert plus == pytest.approx(H[0] ** 4 * 120 / 20, rel=1e-10)
    assert minus == pytest.approx(plus, rel=1e-10)
