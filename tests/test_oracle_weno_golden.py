"""The oracle's WENO reconstructions against the coefficients the paper prints
(Sec. II.B.2: table of c_{r,j} for k = 2 and 3, and the linear weights d_r),
read from tests/golden/weno_coefficients.txt.

* Candidate by candidate: with values of size H outside the cells of
  candidate r, every other smoothness indicator is ~H^2, so the nonlinear
  weight of candidate r is 1 to ~H^-4 (JS and Z weights alike), and unit data
  on its own cells returns the printed c_{r,j}.
* Linear weights: with epsilon far above every smoothness indicator the
  nonlinear weights reduce to d_r (resp. d~_r = d_{k-1-r} on the right), and
  unit data return sum_r d_r c_{r,.}.
"""
import os
from fractions import Fraction

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _table():
    c = {2: {}, 3: {}}
    d = {}
    with open(os.path.join(HERE, "golden", "weno_coefficients.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if not line:
                continue
            if line[0] == "d":
                d[int(line[1])] = [float(Fraction(v)) for v in line[2:]]
            else:
                c[int(line[0])][int(line[1])] = [float(Fraction(v)) for v in line[2:]]
    return c, d


C, D = _table()
H = 1.0e6


def _isolating_data(k, side, r, j):
    """w = U_{i-2..i+2}: unit value on cell j of candidate r, 0 on its other
    cells, H and -3H on the cells the candidate does not use."""
    # cells of candidate r (offsets from i): left  i-r .. i-r+k-1,
    #                                        right i-r .. i-r+k-1 as well
    cells = [-r + q for q in range(k)]
    w = [0.0] * 5
    big = [H, -3.0 * H]  # unequal, so that WENO-Z's tau = |beta_0 - beta_2| stays ~H^2
    lo, hi = (-2, 2) if k == 3 else (-1, 1)
    q = 0
    for off in range(lo, hi + 1):
        if off not in cells:
            w[off + 2] = big[q]
            q += 1
    w[cells[j] + 2] = 1.0
    return w


@pytest.mark.parametrize("variant,k", [(0, 3), (1, 3), (2, 2)])
@pytest.mark.parametrize("side", [0, 1])
def test_isolated_candidates_match_printed_table(variant, k, side):
    for r in range(k):
        row = C[k][r] if side == 0 else C[k][r - 1]
        for j in range(k):
            w = _isolating_data(k, side, r, j)
            got = oracle.weno(variant, side, w, 1e-40)
            assert got == pytest.approx(row[j], abs=1e-9), (k, side, r, j, got, row[j])


@pytest.mark.parametrize("variant,k", [(0, 3), (1, 3), (2, 2)])
@pytest.mark.parametrize("side", [0, 1])
def test_linear_weights_match_printed_d(variant, k, side):
    d = D[k] if side == 0 else list(reversed(D[k]))
    for m in range(5):
        w = [0.0] * 5
        w[m] = 1.0
        off = m - 2
        want = 0.0
        for r in range(k):
            j = off + r
            if 0 <= j < k:
                want += d[r] * (C[k][r][j] if side == 0 else C[k][r - 1][j])
        got = oracle.weno(variant, side, w, 1e30)
        assert got == pytest.approx(want, abs=1e-13), (variant, side, m, got, want)
