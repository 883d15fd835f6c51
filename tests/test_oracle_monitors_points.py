"""Pins of two oracle functions that the GPU checks rely on.

* ``z4_monitors`` (Sec. V names Theta, Z^i, ln det gt~ and tr A~ as the
  quantities the damping terms drive to zero).  The monitors are root mean
  squares over the interior cells of Theta, |Z| (Euclidean norm of
  Z^i = chi/2 (Gammahat^i - Gamma~^i)), ln det gt~ and gt~^{ij} A~_ij.  They
  are checked here on states where every monitor is non-zero and known in
  closed form:
    - a homogeneous conformal metric gt~ = R diag(l) R^T with a fixed
      rotation R (every entry non-zero), so det gt~ = l1 l2 l3 and, with
      A~ = R diag(m) R^T, tr A~ = sum m_i / l_i; Gamma~ = 0 exactly (every
      stencil of a constant is zero), so Z = chi/2 Gammahat; Theta and chi
      vary over the grid with known means of their squares;
    - a diagonal conformal metric varying along x with det gt~ != 1, whose
      contracted Christoffels Gamma~^i have a closed form; with Gammahat =
      Gamma~ + v for a constant v, |Z| = chi/2 |v| to 4th order in dx.
* ``rhs_points`` decodes linear interior indices itself; it must return
  exactly (bit for bit) the columns of ``rhs`` at those points, in any order.
"""
import math

import numpy as np

import oracle
from paper_1806_04182_gb300 import inputs


def rotation(a: float, b: float, c: float) -> np.ndarray:
    """Rotation by c about z, then b about y, then a about x (closed form)."""
    ca, sa, cb, sb, cc, sc = math.cos(a), math.sin(a), math.cos(b), math.sin(b), math.cos(c), math.sin(c)
    Rx = np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]])
    Ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    Rz = np.array([[cc, -sc, 0], [sc, cc, 0], [0, 0, 1]])
    return Rx @ Ry @ Rz


SYM = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def homogeneous_state(n, lam, mu, v, theta0, chi0, chi1):
    nx, ny, nz = n
    R = rotation(0.4, -0.7, 1.1)
    gt = R @ np.diag(lam) @ R.T
    At = R @ np.diag(mu) @ R.T
    U = np.zeros((25, nz, ny, nx))
    y = np.arange(ny) / ny
    x = np.arange(nx) / nx
    U[0] = (chi0 + chi1 * np.cos(2 * math.pi * y))[None, :, None]
    for q, (a, b) in enumerate(SYM):
        U[1 + q] = gt[a, b]
        U[8 + q] = At[a, b]
    for a in range(3):
        U[14 + a] = v[a]
    U[17] = (theta0 * np.sin(2 * math.pi * x))[None, None, :]
    U[18] = 1.0
    return U, gt


def test_monitors_closed_form_on_homogeneous_metric():
    n = (8, 6, 5)
    dx = (1 / 8, 1 / 6, 1 / 5)
    lam = (1.3, 0.8, 1.15)
    mu = (0.05, -0.02, 0.03)
    v = (0.3, -0.2, 0.1)
    theta0, chi0, chi1 = 0.07, 0.7, 0.2
    U, gt = homogeneous_state(n, lam, mu, v, theta0, chi0, chi1)
    assert np.all(np.abs(gt[np.triu_indices(3, 1)]) > 0.05)  # every off-diagonal entry matters
    m = oracle.z4_monitors(oracle.ghosted(U), dx)
    # mean over a full period of sin^2 or cos^2 on >= 3 equispaced points is 1/2
    rms_theta = theta0 / math.sqrt(2.0)
    rms_chi = math.sqrt(chi0 ** 2 + chi1 ** 2 / 2)
    rms_z = 0.5 * rms_chi * math.sqrt(sum(c * c for c in v))
    lndet = math.log(lam[0] * lam[1] * lam[2])
    trA = sum(a / b for a, b in zip(mu, lam))
    want = np.array([rms_theta, rms_z, abs(lndet), abs(trA)])
    assert np.all(want > 1e-3)
    np.testing.assert_allclose(m, want, rtol=1e-12, atol=0)


def test_monitors_on_metric_varying_along_x():
    # Gamma~^i from the discrete metric derivatives (the term the homogeneous
    # test cannot see).  For gt~ = diag(a(x), b(x), 1) the contracted
    # Christoffels are Gamma~^x = (a'/a - b'/b) / (2 a), Gamma~^y = Gamma~^z = 0;
    # det gt~ = a b != 1.  With Gammahat = Gamma~ + v, |Z| = chi/2 |v| up to the
    # stencils' 4th-order truncation.
    v = np.array([0.03, -0.02, 0.01])
    m_xx = 0.02
    rel = []
    for N in (32, 64):
        n = (N, 4, 5)
        dx = (1.0 / N, 1.0 / 4, 1.0 / 5)
        x = (np.arange(N) / N)[None, None, :]
        y = (np.arange(4) / 4)[None, :, None]
        ph = 2 * math.pi * x
        a = 1 + 0.1 * np.sin(ph)
        b = 1 + 0.05 * np.cos(ph)
        da = 0.2 * math.pi * np.cos(ph)
        db = -0.1 * math.pi * np.sin(ph)
        U = np.zeros((25, 5, 4, N))
        U[0] = 1 + 0.1 * np.cos(2 * math.pi * y)
        U[1] = a
        U[4] = b
        U[6] = 1.0
        U[8] = m_xx * a          # A~_xx: gt~^{ij} A~_ij = m_xx everywhere
        U[14] = (da / a - db / b) / (2 * a) + v[0]
        U[15] = v[1]
        U[16] = v[2]
        U[18] = 1.0
        m = oracle.z4_monitors(oracle.ghosted(U), dx)
        chi2 = 1 + 0.1 ** 2 / 2   # mean of chi^2 over the grid
        want_z = 0.5 * np.linalg.norm(v) * math.sqrt(chi2)
        want_lndet = math.sqrt(float(np.mean(np.log(a * b) ** 2)))
        assert m[0] == 0.0
        np.testing.assert_allclose(m[2], want_lndet, rtol=1e-12)
        np.testing.assert_allclose(m[3], m_xx, rtol=1e-12)
        rel.append(abs(m[1] - want_z) / want_z)
    assert rel[1] < 1e-5, rel
    assert rel[0] / rel[1] > 12.0, rel  # the difference is the 4th-order truncation


def test_rhs_points_equals_rhs_columns():
    n = (7, 5, 6)
    rng = np.random.default_rng(5)
    cases = [(oracle.Z4, inputs.z4_perturbed(n, seed=4, amp=0.05), oracle.params()),
             (oracle.WAVE, inputs.wave_plane(n, seed=2), oracle.params()),
             (oracle.MHD, inputs.mhd_blast(n, seed=1), oracle.params())]
    for system, (U0, dx), p in cases:
        G = oracle.ghosted(U0)
        full = oracle.rhs(system, G, dx, p)
        nf = full.shape[0]
        flat = full.reshape(nf, -1)
        pts = rng.permutation(n[0] * n[1] * n[2])
        got = oracle.rhs_points(system, G, dx, pts, p)
        assert np.array_equal(got, flat[:, pts]), system
        # a ragged subset with repeats
        sub = rng.integers(0, pts.size, size=37)
        assert np.array_equal(oracle.rhs_points(system, G, dx, sub, p), flat[:, sub])
