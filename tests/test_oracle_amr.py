"""Pins of the oracle's prolongation and restriction (Sec. III.A).

* Quintic Lagrange interpolation is exact on every polynomial whose degree in
  each variable is at most 5, for refinement ratios 2, 3 and 4; it is not
  exact on x^6.
* For ratio 2 the fine midpoint weights are the paper's (150, -25, 3)/256
  (read off by interpolating a single coarse delta).
* Fine points that coincide with coarse points take the coarse value exactly;
  restriction by injection returns the coincident fine values.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle

G = 3


def coarse_poly(n, fn):
    U = np.zeros((1, n[2] + 2 * G, n[1] + 2 * G, n[0] + 2 * G))
    for k in range(-G, n[2] + G):
        for j in range(-G, n[1] + G):
            for i in range(-G, n[0] + G):
                U[0, k + G, j + G, i + G] = float(fn(Fraction(i), Fraction(j), Fraction(k)))
    return U


@pytest.mark.parametrize("R", [2, 3, 4])
def test_prolongation_exact_on_quintics(R):
    n = (6, 5, 6)
    fn = lambda x, y, z: (x ** 5 - 2 * x ** 3 + x) * (y ** 4 + 3 * y - 2) * (z ** 5 - z ** 2 + 1)
    U = coarse_poly(n, fn)
    origin, ext = (R * 1, R * 1 - 1, R * 2), (R + 2, R + 1, R)
    got = oracle.prolong(U, R, origin, ext)
    for k in range(ext[2]):
        for j in range(ext[1]):
            for i in range(ext[0]):
                x, y, z = (Fraction(origin[0] + i, R), Fraction(origin[1] + j, R),
                           Fraction(origin[2] + k, R))
                want = float(fn(x, y, z))
                assert got[0, k, j, i] == pytest.approx(want, rel=1e-12, abs=1e-9)


def test_prolongation_not_exact_on_sextic():
    U = coarse_poly((6, 4, 4), lambda x, y, z: x ** 6)
    got = oracle.prolong(U, 2, (5, 2, 2), (1, 1, 1))  # x = 5/2, a midpoint
    assert abs(got[0, 0, 0, 0] - 2.5 ** 6) > 1e-6


def test_midpoint_weights_are_the_papers():
    n = (8, 4, 4)
    U = np.zeros((1, n[2] + 2 * G, n[1] + 2 * G, n[0] + 2 * G))
    # delta at coarse x = 4 (y = z = 1): the fine midpoints x = 4 +- 1/2, 3/2, 5/2
    U[0, 1 + G, 1 + G, 4 + G] = 1.0
    got = oracle.prolong(U, 2, (3, 2, 2), (7, 1, 1))[0, 0, 0]  # fine x = 1.5 .. 4.5 step 0.5
    # fine 3 -> x 1.5 (delta 2.5 away), 5 -> 2.5 (1.5), 7 -> 3.5 (0.5), 9 -> 4.5 (0.5)
    assert got[0] == pytest.approx(3 / 256, abs=1e-15)
    assert got[2] == pytest.approx(-25 / 256, abs=1e-15)
    assert got[4] == pytest.approx(150 / 256, abs=1e-15)
    assert got[6] == pytest.approx(150 / 256, abs=1e-15)
    # coincident fine points (even indices) see only their own coarse value
    assert got[1] == 0.0 and got[3] == 0.0 and got[5] == 1.0


@pytest.mark.parametrize("R", [2, 3])
def test_coincident_points_and_restriction_are_injections(R):
    rng = np.random.default_rng(4)
    n = (5, 4, 6)
    U = oracle.ghosted(rng.standard_normal((2, n[2], n[1], n[0])))
    got = oracle.prolong(U, R, (0, 0, 0), (R * 4 + 1, R * 3 + 1, R * 5 + 1))
    np.testing.assert_array_equal(got[:, ::R, ::R, ::R], oracle.interior(U)[:, :6, :4, :5])
    # restriction of that fine box returns the coarse values bit for bit
    nf_ = (R * 4 + 1, R * 3 + 1, R * 5 + 1)
    Uf = np.zeros((2, nf_[2] + 2 * G, nf_[1] + 2 * G, nf_[0] + 2 * G))
    Uf[:, G:G + nf_[2], G:G + nf_[1], G:G + nf_[0]] = got
    back = oracle.restrict(Uf, R, (0, 0, 0), (5, 4, 6))
    np.testing.assert_array_equal(back, oracle.interior(U)[:, :6, :4, :5])
