"""Pin of the oracle's CCZ4 right-hand side, the terms that couple Z and Theta
to gradients included, against the covariant damped Z4 system on polynomial
data.

The state: conformal metric gt = delta, constant trace-free A~ (so det gt = 1
and tr A~ = 0 hold exactly, the surface on which CCZ4 and Z4 describe the same
evolution), and chi, alpha, Theta, Khat and Gammahat^i polynomials of degree
<= 2 in x, y, z, the shift zero or quadratic too, constant B.  Every field is given on the whole
ghosted grid (the ghosts hold the same polynomials, not a periodic copy), so
the 4th-order first, second and mixed derivative stencils of Sec. II.B.1 are
exact (they are exact on polynomials of degree <= 4) and the 6th-order KO
term vanishes: the discrete right-hand side equals the continuum one up to
rounding.  The continuum one is derived here with SymPy, independently of the
CCZ4 text of Sec. V, from

  * the physical variables gamma_ij = gt_ij / chi, K = Khat + 2 Theta,
    K_ij = (A~_ij + gt_ij K / 3) / chi, Z_i = gamma_ij Z^j with
    Z^i = chi / 2 (Gammahat^i - Gammatilde^i);
  * the damped Z4 equations in 3+1 form (Bona, Ledvinka,
    Palenzuela & Zacek, Phys. Rev. D 67, 104005, 2003; damping of Gundlach et
    al., Class. Quantum Grav. 22, 3767, 2005, with k1 = kappa_z, k2 = 0):
    with d/dt replaced by d/dt - L_beta (Lie derivative along the shift):
      d/dt gamma_ij = -2 alpha K_ij
      d/dt K_ij  = -D_i D_j alpha + alpha [R_ij + D_i Z_j + D_j Z_i
                   - 2 K_ik K^k_j + (K - 2 Theta) K_ij - k1 Theta gamma_ij]
      d/dt Theta = alpha / 2 [R + 2 D_k Z^k + (K - 2 Theta) K - K_ij K^ij
                   - 2 Z^k d_k alpha / alpha - 4 k1 Theta]
      d/dt Z_i   = alpha [D_j (K_i^j - delta_i^j K) + d_i Theta
                   - 2 K_i^j Z_j - Theta d_i alpha / alpha - k1 Z_i]
  * the chain rule to the CCZ4 variables (chi = det(gamma)^(-1/3),
    gt = chi gamma, Khat = K - 2 Theta, A~ = chi (K_ij - gamma_ij K / 3),
    Gammahat^i = Gammatilde^i + 2 gt^ij Z_j with Gammatilde^i = gt^jk
    Gammatilde^i_jk, whose time derivative needs the spatial derivatives of
    d/dt gt);
  * the paper's gauge: 1+log slicing d/dt alpha = beta . d alpha - 2 alpha Khat,
    Gamma-driver d/dt beta = beta . d beta + g B, d/dt B = beta . d B - eta B +
    d/dt Gammahat - beta . d Gammahat.
"""
import numpy as np
import pytest

import oracle

sp = pytest.importorskip("sympy")


def derive(coef, X0, kz, g_shift, eta, shift):
    """Continuum CCZ4 right-hand side at X0 from the Z4 system (SymPy)."""
    x, y, z = X = sp.symbols("x y z", real=True)

    def poly(c):  # c = (c0, c1, c2, c3, c4, ...) -> c0 + c1 x + c2 y + c3 z + quadratic terms
        return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * z
                + c[6] * x * z + c[7] * y * y)

    chi = poly(coef["chi"])
    alpha = poly(coef["alpha"])
    theta = poly(coef["theta"])
    Kh = poly(coef["Kh"])
    Gh = [poly(coef["Gh"][i]) for i in range(3)]
    At = sp.Matrix(3, 3, lambda i, j: coef["At"][i][j])
    B = coef["B"]
    be = [poly(coef["beta"][i]) if shift else sp.Integer(0) for i in range(3)]
    gt = sp.eye(3)
    igt = sp.eye(3)

    # physical variables
    gam = gt / chi
    igam = igt * chi
    K = Kh + 2 * theta
    Kij = (At + gt * K / 3) / chi
    dgt = [[[sp.diff(gt[i, j], X[k]) for k in range(3)] for j in range(3)] for i in range(3)]
    Gtld_l = [[[(dgt[a][b][c] + dgt[a][c][b] - dgt[b][c][a]) / 2 for c in range(3)]
               for b in range(3)] for a in range(3)]  # Gamma~_{a bc}
    Gtld = [sum(igt[b, c] * sum(igt[i, a] * Gtld_l[a][b][c] for a in range(3))
                for b in range(3) for c in range(3)) for i in range(3)]
    Zu = [chi / 2 * (Gh[i] - Gtld[i]) for i in range(3)]  # Z^i
    Zd = [sum(gam[i, j] * Zu[j] for j in range(3)) for i in range(3)]

    # geometry of gamma
    dg = [[[sp.diff(gam[i, j], X[k]) for k in range(3)] for j in range(3)] for i in range(3)]
    Chr = [[[sum(igam[k, l] * (dg[l][i][j] + dg[l][j][i] - dg[i][j][l]) for l in range(3)) / 2
             for j in range(3)] for i in range(3)] for k in range(3)]  # Gamma^k_ij
    Ric = sp.Matrix(3, 3, lambda i, j: sum(sp.diff(Chr[k][i][j], X[k]) for k in range(3))
                    - sum(sp.diff(Chr[k][i][k], X[j]) for k in range(3))
                    + sum(Chr[k][k][l] * Chr[l][i][j] for k in range(3) for l in range(3))
                    - sum(Chr[k][j][l] * Chr[l][i][k] for k in range(3) for l in range(3)))
    Rs = sum(igam[i, j] * Ric[i, j] for i in range(3) for j in range(3))
    dal = [sp.diff(alpha, v) for v in X]
    DDal = sp.Matrix(3, 3, lambda i, j: sp.diff(alpha, X[i], X[j])
                     - sum(Chr[k][i][j] * dal[k] for k in range(3)))
    DZ = sp.Matrix(3, 3, lambda i, j: sp.diff(Zd[j], X[i]) - sum(Chr[k][i][j] * Zd[k] for k in range(3)))
    divZ = sum(sp.diff(Zu[k], X[k]) for k in range(3)) + sum(Chr[k][k][l] * Zu[l] for k in range(3)
                                                             for l in range(3))
    Kmix = Kij * igam                 # K_i^j (column j raised)
    KK = sum(Kij[i, j] * (igam * Kij * igam)[i, j] for i in range(3) for j in range(3))

    # Lie derivatives along the shift
    dbe = [[sp.diff(be[i], X[k]) for k in range(3)] for i in range(3)]  # d_k beta^i
    adv = lambda f: sum(be[k] * sp.diff(f, X[k]) for k in range(3))
    lie2 = lambda M: sp.Matrix(3, 3, lambda i, j: adv(M[i, j]) + sum(
        M[k, j] * dbe[k][i] + M[i, k] * dbe[k][j] for k in range(3)))

    # Z4 right-hand sides
    d_gam = -2 * alpha * Kij + lie2(gam)
    d_K = -DDal + alpha * (Ric + DZ + DZ.T - 2 * Kij * igam * Kij + (K - 2 * theta) * Kij
                           - kz * theta * gam) + lie2(Kij)
    d_theta = alpha / 2 * (Rs + 2 * divZ + (K - 2 * theta) * K - KK
                           - 2 * sum(Zu[k] * dal[k] for k in range(3)) / alpha - 4 * kz * theta) \
        + adv(theta)
    # D_j (K_i^j - delta_i^j K): covariant divergence of a (1,1) tensor on its upper index
    T = Kmix - sp.eye(3) * sum(igam[a, b] * Kij[a, b] for a in range(3) for b in range(3))
    divT = [sum(sp.diff(T[i, j], X[j]) for j in range(3))
            + sum(Chr[j][j][l] * T[i, l] for j in range(3) for l in range(3))
            - sum(Chr[l][j][i] * T[l, j] for j in range(3) for l in range(3)) for i in range(3)]
    d_Z = [alpha * (divT[i] + sp.diff(theta, X[i]) - 2 * sum(Kmix[i, j] * Zd[j] for j in range(3))
                    - theta * dal[i] / alpha - kz * Zd[i])
           + adv(Zd[i]) + sum(Zd[k] * dbe[k][i] for k in range(3)) for i in range(3)]

    # chain rule to the CCZ4 variables
    d_chi = -chi / 3 * sum(igam[i, j] * d_gam[i, j] for i in range(3) for j in range(3))
    d_gt = d_chi * gam + chi * d_gam
    d_Ktr = sum(igam[i, j] * d_K[i, j] for i in range(3) for j in range(3)) - sum(
        (igam * d_gam * igam)[i, j] * Kij[i, j] for i in range(3) for j in range(3))
    d_Kh = d_Ktr - 2 * d_theta
    d_At = d_chi * (Kij - gam * K / 3) + chi * (d_K - d_gam * K / 3 - gam * d_Ktr / 3)
    d_igt = -igt * d_gt * igt
    # d/dt Gammatilde^i = d/dt (gt^jk Gammatilde^i_jk), gt = delta here
    d_dgt = [[[sp.diff(d_gt[i, j], X[k]) for k in range(3)] for j in range(3)] for i in range(3)]
    d_Gtld = [sum(d_igt[b, c] * Gtld_l[i][b][c] for b in range(3) for c in range(3))
              + sum(igt[b, c] * sum(igt[i, a] * (d_dgt[a][b][c] + d_dgt[a][c][b] - d_dgt[b][c][a]) / 2
                                    for a in range(3)) for b in range(3) for c in range(3))
              + sum(igt[b, c] * sum(d_igt[i, a] * Gtld_l[a][b][c] for a in range(3))
                    for b in range(3) for c in range(3)) for i in range(3)]
    d_Gh = [d_Gtld[i] + 2 * sum(d_igt[i, j] * Zd[j] + igt[i, j] * d_Z[j] for j in range(3))
            for i in range(3)]
    sub = dict(zip(X, X0))
    ev = lambda e: float(sp.N(sp.sympify(e).subs(sub), 30))
    sym = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))
    out = np.zeros(25)
    out[0] = ev(d_chi)
    out[1:7] = [ev(d_gt[i, j]) for i, j in sym]
    out[7] = ev(d_Kh)
    out[8:14] = [ev(d_At[i, j]) for i, j in sym]
    out[14:17] = [ev(d_Gh[i]) for i in range(3)]
    out[17] = ev(d_theta)
    out[18] = ev(adv(alpha) - 2 * alpha * Kh)
    out[19:22] = [ev(adv(be[i]) + g_shift * B[i]) for i in range(3)]
    # d/dt B = beta . dB - eta B + (d/dt Gammahat - beta . d Gammahat), B constant
    out[22:25] = [out[14 + i] - ev(adv(Gh[i])) - eta * B[i] for i in range(3)]
    # the fields themselves on the grid
    fields = [chi] + [gt[i, j] for i, j in sym] + [Kh] + [At[i, j] for i, j in sym] + Gh + \
             [theta, alpha] + be + list(B)
    return out, [sp.lambdify(X, sp.sympify(f), "numpy") for f in fields]


def random_coef(rng):
    def c(base, lin, quad):
        return [base] + list(rng.normal(size=3) * lin) + list(rng.normal(size=4) * quad)
    a = rng.normal(size=(3, 3)) * 0.1
    At = (a + a.T) / 2
    At -= np.eye(3) * np.trace(At) / 3
    return dict(chi=c(1.0, 0.05, 0.02), alpha=c(1.0, 0.08, 0.03), theta=c(0.05, 0.05, 0.02),
                Kh=c(0.1, 0.05, 0.02), Gh=[c(0.0, 0.05, 0.02) for _ in range(3)],
                beta=[c(0.0, 0.06, 0.03) for _ in range(3)],
                At=At.tolist(), B=list(rng.normal(size=3) * 0.1))


@pytest.mark.parametrize("shift", [False, True])
@pytest.mark.parametrize("seed", range(3))
def test_polynomial_state_rhs_equals_damped_z4(seed, shift):
    rng = np.random.default_rng(100 + seed)
    coef = random_coef(rng)
    h, g, n = 0.25, 3, (3, 3, 3)
    kz, g_shift, eta = 0.8, 0.75, 2.0
    X0 = (1 * h, 1 * h, 1 * h)  # interior point (1, 1, 1); interior x_i = i h
    want, fns = derive(coef, X0, kz, g_shift, eta, shift)
    ax = (np.arange(n[0] + 2 * g) - g) * h
    Zg, Yg, Xg = np.meshgrid(ax, ax, ax, indexing="ij")
    U = np.zeros((25,) + Xg.shape)
    for f, fn in enumerate(fns):
        U[f] = np.broadcast_to(np.asarray(fn(Xg, Yg, Zg), dtype=float), Xg.shape)
    p = oracle.params(kappa_z=kz, kappa_c=0.0, eta=eta, g_shift=g_shift, slicing=0,
                      shift_frozen=0, sigma=0.0)
    got = oracle.rhs(oracle.Z4, U, (h, h, h), p)[:, 1, 1, 1]
    scale = max(np.abs(want).max(), 1.0)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-10 * scale)
