"""Seeded synthetic inputs shaped like the paper's test problems.

This module holds no arithmetic of the method (no stencil, flux, RHS or time
step): it only draws random numbers and evaluates closed-form initial data.
Both the CUDA path (tests, bench) and the oracle tests take their inputs from
here, so the two sides see bit-identical data.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated counter-style:
draw i of stream `seed` is mix(seed * 2^32 + i + 1) scaled by the golden
gamma; doubles take the top 53 bits; normals use Box-Muller.

All arrays are numpy float64, interior-only, shape (nf, nz, ny, nx) with x
fastest; domains are periodic, x_i = i * dx (Sec. II.A), except the puncture
boxes of Sec. V (cell-centred, non-periodic, optionally with ghost points).
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Counter-based SplitMix64: outputs offset..offset+count-1 of stream `seed`."""
    ctr = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    base = np.uint64((int(seed) << 32) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        z = (base + ctr) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller from pairs of uniforms."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * m, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:count]


def coords(n, dx):
    """Broadcastable grid coordinates x_i = i dx (z, y, x order of axes)."""
    nx, ny, nz = n
    x = np.arange(nx) * dx[0]
    y = np.arange(ny) * dx[1]
    z = np.arange(nz) * dx[2]
    return z[:, None, None], y[None, :, None], x[None, None, :]


# ------------------------------------------------------------------- wave
def wave_k(seed: int) -> tuple[int, int, int]:
    """Integer wave vector with components drawn from {1, 2, 3}."""
    u = uniform(seed, 3, offset=1000)
    return tuple(int(1 + math.floor(3.0 * v)) for v in u)


def wave_plane(n, seed: int = 0, t: float = 0.0, k=None, length: float = 1.0):
    """Right-moving plane wave on the periodic box [0, length)^3.

    phi = sin(2 pi (k.x/length - |k| t/length)); with Pi = -d phi/dt and
    d_i = d phi / dx_i this is an exact solution of the first-order wave
    system (phi, Pi, d_x, d_y, d_z).  Returns (U, dx).
    """
    if k is None:
        k = wave_k(seed)
    nx, ny, nz = n
    dx = (length / nx, length / ny, length / nz)
    Z, Y, X = coords(n, dx)
    kn = math.sqrt(k[0] ** 2 + k[1] ** 2 + k[2] ** 2)
    ph = 2.0 * math.pi * (k[0] * X + k[1] * Y + k[2] * Z - kn * t) / length
    U = np.zeros((5, nz, ny, nx))
    U[0] = np.sin(ph)
    c = np.cos(ph) * (2.0 * math.pi / length)
    U[1] = kn * c
    U[2] = k[0] * c
    U[3] = k[1] * c
    U[4] = k[2] * c
    return U, dx


def wave_noise(n, seed: int = 0, amp: float = 1.0):
    """Uniform noise in (-amp, amp) on all five wave fields (for linear-algebra tests)."""
    nx, ny, nz = n
    return amp * (2.0 * uniform(seed, 5 * nx * ny * nz).reshape(5, nz, ny, nx) - 1.0)


def observers(n, count: int, seed: int = 0) -> np.ndarray:
    """Distinct interior linear indices (k*ny + j)*nx + i of observer points."""
    nx, ny, nz = n
    tot = nx * ny * nz
    u = uniform(seed, 4 * count + 64, offset=7000)
    picks = []
    for v in u:
        c = int(v * tot)
        if c not in picks:
            picks.append(c)
        if len(picks) == count:
            break
    return np.array(picks, dtype=np.int64)


def smooth_bump(n, seed: int = 0, width: float = 0.15):
    """Periodic Gaussian bump at a seeded centre of the unit box (nz, ny, nx)."""
    nx, ny, nz = n
    dx = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    c = uniform(seed, 3, offset=9000)
    Z, Y, X = coords(n, dx)
    d2 = 0.0
    for Xd, cd in ((X, c[0]), (Y, c[1]), (Z, c[2])):
        dd = np.abs(Xd - cd)
        dd = np.minimum(dd, 1.0 - dd)
        d2 = d2 + dd * dd
    return np.exp(-d2 / (width * width))


# ------------------------------------------------------------------- MHD
def mhd_primitive_to_conserved(rho, v, p, B, gamma):
    """Conserved (rho, S, E, B) from primitives, E = rho v^2/2 + p/(Gamma-1) + B^2/2."""
    S = [rho * vi for vi in v]
    v2 = sum(vi * vi for vi in v)
    B2 = sum(Bi * Bi for Bi in B)
    E = 0.5 * rho * v2 + p / (gamma - 1.0) + 0.5 * B2
    return np.stack([rho * np.ones_like(E), S[0], S[1], S[2], E, B[0], B[1], B[2]])


def mhd_blast(n, seed: int = 0, gamma: float = 5.0 / 3.0, vrms: float = 0.1,
              radius: float = 0.1, boost: float = 10.0):
    """rho = 1, p = 0.1, B = (0.5, 0.5, 0), i.i.d. Gaussian velocity per cell
    and component with total rms vrms, pressure x boost inside a periodic
    sphere of given radius around a seeded centre.  Returns (U, dx)."""
    nx, ny, nz = n
    dx = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    shape = (nz, ny, nx)
    N = nx * ny * nz
    g = normal(seed, 3 * N).reshape(3, nz, ny, nx) * (vrms / math.sqrt(3.0))
    rho = np.ones(shape)
    p = 0.1 * np.ones(shape)
    c = uniform(seed, 3, offset=5000)
    Z, Y, X = coords(n, dx)
    d2 = np.zeros(shape)
    for Xd, cd in ((X, c[0]), (Y, c[1]), (Z, c[2])):
        dd = np.abs(Xd - cd)
        dd = np.minimum(dd, 1.0 - dd)
        d2 = d2 + dd * dd
    p = np.where(d2 < radius * radius, p * boost, p)
    B = [0.5 * np.ones(shape), 0.5 * np.ones(shape), np.zeros(shape)]
    return mhd_primitive_to_conserved(rho, [g[0], g[1], g[2]], p, B, gamma), dx


def mhd_brio_wu(n, gamma: float = 2.0):
    """Brio & Wu magnetic shock tube (Sec. IV.B.2) on a periodic domain
    [0, 2) along x, doubled so that it needs no outflow boundary: the left
    state (rho, p, B_y) = (1, 1, 1) for x <= 0.5 and x > 1.5, the right state
    (0.125, 0.1, -1) in between, B_x = 0.75, B_z = v = 0, Gamma = 2.  The jump
    at x = 0.5 is the paper's tube; the waves of the two jumps stay apart
    until t = 0.2 (fastest speed below 2).  Uniform in y and z; dx = 2 / nx
    in every direction.  Returns (U, dx)."""
    nx, ny, nz = n
    h = 2.0 / nx
    dx = (h, h, h)
    x = np.arange(nx) * h
    left = (x <= 0.5) | (x > 1.5)
    shape = (nz, ny, nx)
    rho = np.broadcast_to(np.where(left, 1.0, 0.125), shape)
    p = np.broadcast_to(np.where(left, 1.0, 0.1), shape)
    by = np.broadcast_to(np.where(left, 1.0, -1.0), shape)
    zero = np.zeros(shape)
    B = [0.75 * np.ones(shape), by.copy(), zero.copy()]
    return mhd_primitive_to_conserved(rho.copy(), [zero.copy()] * 3, p.copy(), B, gamma), dx


def mhd_alfven(n, t: float = 0.0, m=(1, 1), gamma: float = 5.0 / 3.0):
    """Circularly polarised Alfven wave (Sec. IV.B.1) on the unit box, z-invariant.

    Phase 2 pi (m.x + |m| t): rho = 1, p = 0.1, B_par = 1, B_perp = v_perp =
    0.1 sin(phase), B_z = v_z = 0.1 cos(phase).  With v = +B/sqrt(rho) the
    wave travels along -m at the Alfven speed 1.  Returns (U, dx).
    """
    nx, ny, nz = n
    dx = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    Z, Y, X = coords(n, dx)
    mn = math.hypot(m[0], m[1])
    ca, sa = m[0] / mn, m[1] / mn
    ph = 2.0 * math.pi * (m[0] * X + m[1] * Y + mn * t) + 0.0 * Z
    bperp = 0.1 * np.sin(ph)
    bz = 0.1 * np.cos(ph)
    Bx = 1.0 * ca - bperp * sa
    By = 1.0 * sa + bperp * ca
    vx = -bperp * sa
    vy = bperp * ca
    rho = np.ones_like(ph)
    p = 0.1 * np.ones_like(ph)
    return mhd_primitive_to_conserved(rho, [vx, vy, bz], p, [Bx, By, bz], gamma), dx


def mhd_uniform(n, gamma: float = 5.0 / 3.0):
    nx, ny, nz = n
    shape = (nz, ny, nx)
    one = np.ones(shape)
    return mhd_primitive_to_conserved(1.3 * one, [0.2 * one, -0.1 * one, 0.05 * one], 0.7 * one,
                                      [0.4 * one, 0.3 * one, -0.2 * one], gamma)


# ------------------------------------------------------------------- Z4
Z4_NF = 25
# field order: chi | gt_xx gt_xy gt_xz gt_yy gt_yz gt_zz | Khat | At_ij (same order) |
# Gammahat^x,y,z | Theta | alpha | beta^x,y,z | B^x,y,z
Z4_NAMES = ["chi", "gt_xx", "gt_xy", "gt_xz", "gt_yy", "gt_yz", "gt_zz", "Khat", "At_xx",
            "At_xy", "At_xz", "At_yy", "At_yz", "At_zz", "Gh_x", "Gh_y", "Gh_z", "Theta",
            "alpha", "beta_x", "beta_y", "beta_z", "B_x", "B_y", "B_z"]


def z4_minkowski(n):
    """Flat space: chi = 1, gt = delta, alpha = 1, everything else 0."""
    nx, ny, nz = n
    U = np.zeros((Z4_NF, nz, ny, nx))
    U[0] = 1.0
    U[1] = U[4] = U[6] = 1.0
    U[18] = 1.0
    return U


def z4_minkowski_noise(n, seed: int = 0, amp: float = 1e-10):
    """Minkowski plus i.i.d. uniform noise in (-amp, amp) on every field.  Returns (U, dx)."""
    nx, ny, nz = n
    U = z4_minkowski(n)
    U += amp * (2.0 * uniform(seed, U.size).reshape(U.shape) - 1.0)
    return U, (1.0 / nx, 1.0 / ny, 1.0 / nz)


def z4_gauge_wave(n, amp: float = 0.01, t: float = 0.0):
    """Gauge wave along x on the unit box: ds^2 = H(-dt^2 + dx^2) + dy^2 + dz^2,
    H = 1 - amp sin(2 pi (x - t)).  Exact for harmonic slicing with zero,
    frozen shift.  Returns (U, dx)."""
    nx, ny, nz = n
    dx = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    Z, Y, X = coords(n, dx)
    ph = 2.0 * math.pi * (X - t) + 0.0 * Y + 0.0 * Z
    H = 1.0 - amp * np.sin(ph)
    dtH = 2.0 * math.pi * amp * np.cos(ph)
    dxH = -dtH
    U = np.zeros((Z4_NF, nz, ny, nx))
    chi = H ** (-1.0 / 3.0)
    Kxx = -dtH / (2.0 * np.sqrt(H))
    trK = Kxx / H
    U[0] = chi
    U[1] = H ** (2.0 / 3.0)
    U[4] = chi
    U[6] = chi
    U[7] = trK
    U[8] = (2.0 / 3.0) * chi * Kxx
    U[11] = -(1.0 / 3.0) * chi * Kxx / H
    U[13] = U[11]
    U[14] = (2.0 / 3.0) * H ** (-5.0 / 3.0) * dxH
    U[18] = np.sqrt(H)
    return U, dx


def z4_perturbed(n, seed: int = 0, amp: float = 0.05):
    """Minkowski plus smooth periodic perturbations of every field: each field
    gets amp * sum of three Fourier modes with seeded integer wave vectors in
    {1,2}^3 and seeded phases.  Exercises every term of the right-hand side
    (non-zero shift, curvature, Theta, Z).  Returns (U, dx)."""
    nx, ny, nz = n
    dx = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    Z, Y, X = coords(n, dx)
    U = z4_minkowski(n)
    r = uniform(seed, Z4_NF * 3 * 4, offset=30000).reshape(Z4_NF, 3, 4)
    for f in range(Z4_NF):
        for m in range(3):
            kx, ky, kz = (1 + int(2 * r[f, m, q]) for q in range(3))
            ph = 2.0 * math.pi * (kx * X + ky * Y + kz * Z + r[f, m, 3])
            U[f] += amp / 3.0 * np.sin(ph)
    return U, dx


# ------------------------------------------------------------------- batches
def z4_puncture_box(n, length: float):
    """Cell-centred grid on the cube [-length/2, length/2)^3: returns
    (dx, x0) with x0 the position of point (0,0,0), so no point sits on the
    origin (or on a puncture placed at a cell corner)."""
    dx = tuple(length / v for v in n)
    x0 = tuple(-length / 2 + 0.5 * h for h in dx)
    return dx, x0


DEFAULT_HOLES = [dict(m=1.0, pos=(0.05, -0.03, 0.02), P=(0.1, 0.05, 0.0), S=(0.0, 0.0, 0.2))]


def z4_puncture_at(X, Y, Z, holes=None):
    """Puncture initial data of Sec. V at the points (X, Y, Z) (arrays of one
    shape): Brill-Lindquist conformal factor and Bowen-York curvature,
      psi = 1 + sum_A m_A / (2 r_A),  chi = psi^-4,  alpha = psi^-2,
      gt_ij = delta_ij,  Khat = Theta = 0,  Gammahat = beta = B = 0,
      At_ij = sum_A 3/(2 r_A^2 psi^6) [P_i n_j + P_j n_i - (delta_ij - n_i n_j) P.n]
            + sum_A 3/(r_A^3 psi^6) [eps_kil S^l n^k n_j + eps_kjl S^l n^k n_i],
    n = (x - x_A)/r_A.  `holes`: list of dicts with keys m, pos, P, S (default
    DEFAULT_HOLES: one spinning, boosted hole of bare mass 1 near the origin).
    Returns an array (25,) + X.shape."""
    if holes is None:
        holes = DEFAULT_HOLES
    xs = (X, Y, Z)
    psi = np.ones_like(X)
    for h in holes:
        r = np.sqrt(sum((xs[d] - h["pos"][d]) ** 2 for d in range(3)))
        psi += h["m"] / (2 * r)
    At = np.zeros((3, 3) + X.shape)
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1.0
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1.0
    for h in holes:
        rel = [xs[d] - h["pos"][d] for d in range(3)]
        r = np.sqrt(sum(c * c for c in rel))
        nv = [c / r for c in rel]
        P, S = h["P"], h["S"]
        Pn = sum(P[d] * nv[d] for d in range(3))
        for i in range(3):
            for j in range(3):
                dij = 1.0 if i == j else 0.0
                lin = P[i] * nv[j] + P[j] * nv[i] - (dij - nv[i] * nv[j]) * Pn
                spin = 0.0
                for k in range(3):
                    for l in range(3):
                        spin = spin + eps[k, i, l] * S[l] * nv[k] * nv[j] + eps[k, j, l] * S[l] * nv[k] * nv[i]
                At[i, j] += 1.5 / r ** 2 * lin + 3.0 / r ** 3 * spin
    At /= psi ** 6
    U = np.zeros((Z4_NF,) + X.shape)
    U[0] = psi ** -4
    U[1] = U[4] = U[6] = 1.0
    for q, (i, j) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        U[8 + q] = At[i, j]
    U[18] = psi ** -2
    return U


def z4_puncture(n, length: float = 8.0, holes=None, ghost: int = 0):
    """z4_puncture_at on the cell-centred box of z4_puncture_box.  With
    ghost > 0 the data also cover the ghost points (arrays (25, nz+2g,
    ny+2g, nx+2g)).  Returns (U, dx, x0), x0 = position of interior point
    (0,0,0)."""
    dx, x0 = z4_puncture_box(n, length)
    g = ghost
    ax = [x0[d] + dx[d] * np.arange(-g, n[d] + g) for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return z4_puncture_at(X, Y, Z, holes), dx, x0


# values at infinity of the CCZ4 fields (flat space) for radiative boundaries
Z4_UINF = np.array([1.0, 1, 0, 0, 1, 0, 1] + [0.0] * 11 + [1.0] + [0.0] * 6)


def amr_patch_table(npatch: int = 512, seed: int = 0, lo: int = 16, hi: int = 64):
    """Seeded patch descriptors for the batched AMR step: sizes (nx, ny, nz)
    each uniform in {lo..hi}, level in {0, 1, 2} with dx = 1/64, 1/128, 1/384
    (refinement ratios 2 then 3), dt = 0.25 dx, system 'wave' or 'z4' by coin."""
    u = uniform(seed, 5 * npatch, offset=20000).reshape(npatch, 5)
    table = []
    for r in u:
        size = tuple(int(lo + math.floor((hi - lo + 1) * v)) for v in r[:3])
        level = int(math.floor(3 * r[3]))
        h = (1.0 / 64, 1.0 / 128, 1.0 / 384)[level]
        system = "wave" if r[4] < 0.5 else "z4"
        table.append(dict(n=size, level=level, dx=h, dt=0.25 * h, system=system))
    return table
