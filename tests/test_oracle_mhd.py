"""Pins of the oracle's ideal-MHD right-hand side (Sec. IV.B, Sec. II.B.2, App. B).

* Every property below holds for both reconstructions: of the evolved fields
  (then LLF, the paper's tests) and of the Lax-Friedrichs split fluxes.
* A uniform state has identical left/right states everywhere: RHS exactly 0.
* Conservative form: on a periodic box the flux differences telescope, so
  the cell sum of every RHS component vanishes to rounding.
* Data varying along x only: every (y, z) column gives the same RHS, which
  equals the RHS of a one-cell-thick problem.
* Rotating the axes (x <-> y with the vector components swapped) commutes
  with the operator.
* The circularly polarised Alfven wave (Sec. IV.B.1) is an exact smooth
  solution: the scheme converges to it at 5th order (the paper's WENO5 result),
  which a wrong flux term, sign, WENO weight or candidate would break.
* The CFL rate of a uniform state equals the closed-form fast speed.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1806_04182_gb300 import inputs


@pytest.mark.parametrize("split", [0, 1])
def test_uniform_state_gives_exact_zero(split):
    U = oracle.ghosted(inputs.mhd_uniform((6, 5, 7)))
    r = oracle.rhs(oracle.MHD, U, (0.1, 0.2, 0.15), oracle.params(flux_split=split))
    assert np.all(r == 0.0)


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_periodic_conservation(variant, split):
    U0, dx = inputs.mhd_blast((8, 9, 7), seed=3, radius=0.3)
    r = oracle.rhs(oracle.MHD, oracle.ghosted(U0), dx,
                   oracle.params(weno_variant=variant, flux_split=split))
    tot = r.sum(axis=(1, 2, 3))
    scale = np.abs(r).sum(axis=(1, 2, 3)) + 1e-300
    assert np.all(np.abs(tot) <= 1e-12 * scale), tot / scale


@pytest.mark.parametrize("split", [0, 1])
def test_one_dimensional_data(split):
    n1 = (16, 1, 1)
    U1, dx = inputs.mhd_alfven(n1, m=(1, 0))
    U1[:, :, :, 5:9] *= 1.05  # break the exact Alfven structure a bit
    U3 = np.repeat(np.repeat(U1, 4, axis=1), 3, axis=2)
    p = oracle.params(flux_split=split)
    r1 = oracle.rhs(oracle.MHD, oracle.ghosted(U1), (dx[0], 0.3, 0.2), p)
    r3 = oracle.rhs(oracle.MHD, oracle.ghosted(U3), (dx[0], 0.3, 0.2), p)
    for j in range(4):
        for k in range(3):
            np.testing.assert_array_equal(r3[:, j:j + 1, k:k + 1, :], r1)


@pytest.mark.parametrize("split", [0, 1])
def test_axis_permutation_equivariance(split):
    U0, dx = inputs.mhd_blast((7, 7, 6), seed=8, radius=0.35)
    h = (0.13, 0.13, 0.17)
    p = oracle.params(flux_split=split)
    r = oracle.rhs(oracle.MHD, oracle.ghosted(U0), h, p)
    # swap x and y: axes (z, y, x) -> (z, x, y), components S_x<->S_y, B_x<->B_y
    perm = [0, 2, 1, 3, 4, 6, 5, 7]
    V0 = np.ascontiguousarray(U0[perm].transpose(0, 1, 3, 2))
    rv = oracle.rhs(oracle.MHD, oracle.ghosted(V0), (h[1], h[0], h[2]), p)
    back = rv[perm].transpose(0, 1, 3, 2)
    np.testing.assert_allclose(back, r, atol=1e-13 * np.abs(r).max())


@pytest.mark.parametrize("variant,split,lo,hi", [(0, 0, 4.5, 6.0), (1, 0, 4.5, 6.0), (2, 0, 2.6, 3.6),
                                                 (0, 1, 4.5, 6.0), (2, 1, 2.6, 3.6)])
def test_alfven_wave_convergence_order(variant, split, lo, hi):
    # WENO5-JS and WENO5-Z converge at 5th order, WENO3 at 3rd (Sec. IV.B.1),
    # whether the fields or the split fluxes are reconstructed
    p = oracle.params(weno_variant=variant, weno_q=2.0, flux_split=split)
    errs = []
    for N in (16, 32):
        U0, dx = inputs.mhd_alfven((N, N, 1))
        U = oracle.ghosted(U0)
        T = 0.25
        ns = int(math.ceil(T / (dx[0] / (4 * math.sqrt(2)))))
        dt = T / ns
        for _ in range(ns):
            oracle.rk4_step(oracle.MHD, U, dx, dt, p)
        Ue, _ = inputs.mhd_alfven((N, N, 1), t=T)
        # relative L1 error of B_x (Eq. def:relative_error)
        errs.append(np.abs(oracle.interior(U)[5] - Ue[5]).sum() / np.abs(Ue[5]).sum())
    order = math.log2(errs[0] / errs[1])
    assert lo < order < hi, (errs, order)


def test_max_rate_closed_form():
    n = (4, 3, 2)
    U = oracle.ghosted(inputs.mhd_uniform(n))
    gam = 5.0 / 3.0
    rho, v, p, B = 1.3, (0.2, -0.1, 0.05), 0.7, (0.4, 0.3, -0.2)
    h = (0.1, 0.05, 0.2)
    B2 = sum(b * b for b in B)
    best = 0.0
    for d in range(3):
        a2, b2, bd2 = gam * p / rho, B2 / rho, B[d] ** 2 / rho
        cf = math.sqrt(0.5 * (a2 + b2 + math.sqrt((a2 + b2) ** 2 - 4 * a2 * bd2)))
        best = max(best, (abs(v[d]) + cf) / h[d])
    assert oracle.mhd_max_rate(U, h) == pytest.approx(best, rel=1e-14)


def test_glm_psi_decays_on_uniform_state():
    n = (4, 4, 4)
    U8 = inputs.mhd_uniform(n)
    U9 = np.concatenate([U8, 0.3 * np.ones((1,) + U8.shape[1:])])
    p = oracle.params(mhd_glm=1, ch=1.5, kappa_psi=2.0)
    r = oracle.rhs(oracle.MHD, oracle.ghosted(U9), (0.1, 0.1, 0.1), p)
    assert np.all(r[:8] == 0.0)
    np.testing.assert_allclose(r[8], -2.0 * 0.3)
