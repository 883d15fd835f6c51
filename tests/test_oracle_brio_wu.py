"""The Brio & Wu magnetic shock tube (Sec. IV.B.2) on the oracle's MHD path:
WENO5-JS reconstruction of the evolved fields, LLF flux, SSP-RK3, dt = 0.2 dx,
Gamma = 2, to t = 0.2 (the paper's setup, on a doubled periodic tube; see
inputs.mhd_brio_wu).  Like the paper, the accuracy is judged against a
high-resolution run of the same scheme (tests/golden/brio_wu_reference.txt,
written by tests/golden/make_brio_wu.py with 1600 points on the unit tube;
the paper uses PPM with 4000): the L1 error of rho, B_y and p falls with every
refinement of N = 100, 200, 400 points on the unit tube (the paper's
resolutions), and density and pressure stay positive with bounded overshoots.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1806_04182_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def load_reference():
    rows = [line.split() for line in open(os.path.join(HERE, "golden", "brio_wu_reference.txt"))
            if not line.startswith("#")]
    a = np.array(rows, dtype=float)
    return a[:, 0], a[:, 1], a[:, 2], a[:, 3], a[:, 4]


def run(n, gamma=2.0, t_end=0.2):
    U0, dx = inputs.mhd_brio_wu((n, 1, 1), gamma=gamma)
    G = oracle.ghosted(U0)
    dt = 0.2 * dx[0]
    for _ in range(int(round(t_end / dt))):
        oracle.ssprk3_step(oracle.MHD, G, dx, dt, oracle.params(gamma_eos=gamma))
    U = oracle.interior(G)[:, 0, 0, :]
    rho, sx, sy, sz, E, bx, by, bz = U
    vx = sx / rho
    p = (gamma - 1) * (E - 0.5 * (sx * sx + sy * sy + sz * sz) / rho - 0.5 * (bx * bx + by * by + bz * bz))
    return rho, vx, by, p


@pytest.fixture(scope="module")
def runs():
    return {n: run(n) for n in (200, 400, 800)}  # 100, 200, 400 points on the unit tube


def test_brio_wu_converges_to_high_resolution_run(runs):
    x, rho_r, vx_r, by_r, p_r = load_reference()
    m = np.arange(0, len(x), 2)              # points common to every resolution
    errs = {}
    for n, (rho, vx, by, p) in runs.items():
        idx = m * n // 400
        errs[n] = [np.abs(q[idx] - r[m]).mean() for q, r in ((rho, rho_r), (by, by_r), (p, p_r))]
    for k in range(3):
        e = [errs[n][k] for n in (200, 400, 800)]
        assert e[0] > e[1] > e[2], (k, e)
        assert e[0] / e[2] > 2.0, (k, e)


def test_brio_wu_stays_positive_and_bounded(runs):
    for n, (rho, vx, by, p) in runs.items():
        assert rho.min() > 0.1 and rho.max() < 1.1, (n, rho.min(), rho.max())
        assert p.min() > 0.05 and p.max() < 1.1, (n, p.min(), p.max())
        assert np.abs(by).max() < 1.1, n
