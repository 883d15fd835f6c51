"""Pin of the oracle's CCZ4 algebraic (non-derivative) terms, the Theta and Z
couplings included, against the covariant damped Z4 system.

On a spatially homogeneous state (every field constant) every stencil of the
discrete right-hand side is exactly zero, and so is the geometry: a constant
metric has no Christoffels and no curvature, and a constant lapse, Theta or Z
has no gradient.  What is left of the CCZ4 right-hand side (Sec. V) is pure
algebra: the products of the extrinsic curvature, Theta and the Z vector, the
damping terms and the gauge terms.

The same time derivatives follow independently from the damped Z4 equations
in 3+1 form (Bona, Ledvinka, Palenzuela & Zacek, Phys. Rev. D 67, 104005,
2003; damping as in Gundlach, Calabrese, Hinder & Martin-Garcia, Class.
Quantum Grav. 22, 3767, 2005), which on a homogeneous state reduce to

    d/dt gamma_ij = -2 alpha K_ij
    d/dt K_ij     = alpha [-2 K_ik K^k_j + (K - 2 Theta) K_ij - k1 (1 + k2) Theta gamma_ij]
    d/dt Theta    = alpha/2 [(K - 2 Theta) K - K_ij K^ij - 2 k1 (2 + k2) Theta]
    d/dt Z_i      = alpha [-2 K_i^j Z_j - k1 Z_i]

(shift advection and Lie terms vanish for constant fields).  The paper's
damping terms are those of k1 = kappa_z, k2 = 0 (its Theta equation damps
with 2 kappa_z Theta and its Khat equation carries + kappa_z Theta).  The
CCZ4 variables are functions of (gamma, K, Theta, Z): chi = det(gamma)^(-1/3),
gt = chi gamma, Khat = K - 2 Theta, At = chi (K_ij - gamma_ij K / 3),
Gammahat^i = Gammatilde^i + 2 gt^ij Z_j with Gammatilde = 0 here; their time
derivatives come from the chain rule, evaluated exactly by a complex-step
derivative along the Z4 velocity.  The gauge fields follow the paper's 1+log
slicing (d/dt alpha = -2 alpha Khat) and Gamma-driver (d/dt beta = g B,
d/dt B = d/dt Gammahat - eta B).  The conformal-constraint damping terms
(kappa_c) vanish because det gt = 1 and tr At = 0 hold exactly.
"""
import numpy as np
import pytest

import oracle

SYM = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def sym(v):
    m = np.empty((3, 3), dtype=v.dtype)
    for q, (a, b) in enumerate(SYM):
        m[a, b] = m[b, a] = v[q]
    return m


def unsym(m):
    return np.array([m[a, b] for a, b in SYM])


def z4_velocity(gam, K, theta, Z, alpha, k1, k2=0.0):
    """Time derivatives of the 3+1 Z4 variables on a homogeneous state."""
    ig = np.linalg.inv(gam)
    trK = np.trace(ig @ K)
    Kud = ig @ K                       # K^i_j
    KK = np.trace(Kud @ Kud)           # K_ij K^ij
    dgam = -2 * alpha * K
    dK = alpha * (-2 * K @ Kud + (trK - 2 * theta) * K - k1 * (1 + k2) * theta * gam)
    dtheta = alpha / 2 * ((trK - 2 * theta) * trK - KK - 2 * k1 * (2 + k2) * theta)
    dZ = alpha * (-2 * Kud.T @ Z - k1 * Z)
    return dgam, dK, dtheta, dZ


def ccz4_vars(gam, K, theta, Z):
    """(chi, gt_ij, Khat, At_ij, Gammahat^i) of a homogeneous state."""
    chi = np.linalg.det(gam) ** (-1.0 / 3.0)
    gt = chi * gam
    trK = np.trace(np.linalg.inv(gam) @ K)
    At = chi * (K - gam * trK / 3)
    Gh = 2 * np.linalg.inv(gt) @ Z
    return chi, gt, trK - 2 * theta, At, Gh


def random_state(rng):
    a = rng.normal(size=(3, 3)) * 0.15
    gam = np.eye(3) + (a + a.T) / 2
    b = rng.normal(size=(3, 3)) * 0.3
    K = (b + b.T) / 2
    return (gam, K, rng.normal() * 0.2, rng.normal(size=3) * 0.2, 0.6 + rng.random(),
            rng.normal(size=3) * 0.3, rng.normal(size=3) * 0.3)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("kz,kc", [(1.0, 1.0), (0.3, 2.0)])
def test_homogeneous_rhs_equals_damped_z4(seed, kz, kc):
    rng = np.random.default_rng(seed)
    gam, K, theta, Z, alpha, beta, B = random_state(rng)
    g_shift, eta = 0.75, 2.0
    chi, gt, Kh, At, Gh = ccz4_vars(gam, K, theta, Z)

    # exact time derivatives of the CCZ4 variables: complex step along the Z4 velocity
    dgam, dK, dtheta, dZ = z4_velocity(gam, K, theta, Z, alpha, kz)
    h = 1e-30
    c = ccz4_vars(gam + 1j * h * dgam, K + 1j * h * dK, theta + 1j * h * dtheta, Z + 1j * h * dZ)
    d_chi, d_gt, d_Kh, d_At, d_Gh = (np.imag(v) / h for v in c)
    want = np.zeros(25)
    want[0] = d_chi
    want[1:7] = unsym(d_gt)
    want[7] = d_Kh
    want[8:14] = unsym(d_At)
    want[14:17] = d_Gh
    want[17] = dtheta
    want[18] = -2 * alpha * Kh                  # 1+log slicing
    want[19:22] = g_shift * B                   # Gamma-driver
    want[22:25] = d_Gh - eta * B

    # the oracle on a constant grid
    state = np.zeros(25)
    state[0] = chi
    state[1:7] = unsym(gt)
    state[7] = Kh
    state[8:14] = unsym(At)
    state[14:17] = Gh
    state[17] = theta
    state[18] = alpha
    state[19:22] = beta
    state[22:25] = B
    U = oracle.ghosted(np.broadcast_to(state[:, None, None, None], (25, 3, 3, 3)).copy())
    p = oracle.params(kappa_z=kz, kappa_c=kc, eta=eta, g_shift=g_shift, slicing=0,
                      shift_frozen=0)
    r = oracle.rhs(oracle.Z4, U, (0.1, 0.1, 0.1), p)
    got = r[:, 1, 1, 1]
    assert np.allclose(r, got[:, None, None, None], rtol=0, atol=0)  # every point the same
    scale = max(np.abs(want).max(), 1.0)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * scale)


def test_theta_and_z_decay_at_the_damping_rates():
    # linear regime: a small homogeneous Theta or Z in flat space decays at the
    # damped-Z4 rates (2 kappa_z for Theta, kappa_z for Z), with Khat fed by
    # + kappa_z Theta: the constraint-damping property the terms exist for
    kz = 0.7
    p = oracle.params(kappa_z=kz, kappa_c=0.0, slicing=1, shift_frozen=1)
    state = np.zeros(25)
    state[0] = 1.0
    state[[1, 4, 6]] = 1.0
    state[18] = 1.0
    eps = 1e-7
    state[17] = eps                      # Theta
    state[14:17] = 2 * eps * np.array([1.0, -0.5, 0.25])   # Gammahat = 2 Z
    U = oracle.ghosted(np.broadcast_to(state[:, None, None, None], (25, 3, 3, 3)).copy())
    r = oracle.rhs(oracle.Z4, U, (0.1, 0.1, 0.1), p)[:, 1, 1, 1]
    np.testing.assert_allclose(r[17], -2 * kz * eps, rtol=1e-6)
    np.testing.assert_allclose(r[7], kz * eps, rtol=1e-6)
    np.testing.assert_allclose(r[14:17], -kz * state[14:17], rtol=1e-6)
