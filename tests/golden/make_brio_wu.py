"""Writes brio_wu_reference.txt: the high-resolution run the Brio & Wu shock
tube tests compare against (Sec. IV.B.2 compares with a run of its own at
N = 4000 points on the unit tube).  Calls only the oracle and the input
generators: the FP64 CPU oracle, WENO5-JS + LLF, SSP-RK3, dt = 0.2 dx, Gamma
= 2, on the doubled periodic tube of inputs.mhd_brio_wu with 3200 points on
[0, 2) (1600 on the unit tube), run to t = 0.2.  Stored: rho, v_x, B_y and p
at the 400 points x = 2 m / 400 (m = 0..199, i.e. x in [0, 1)), which every
test resolution (200, 400, 800 on [0, 2)) contains.

    python tests/golden/make_brio_wu.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1806_04182_gb300 import inputs  # noqa: E402

NREF, NOUT, GAMMA, T = 3200, 400, 2.0, 0.2


def run(n, gamma=GAMMA, t_end=T):
    U0, dx = inputs.mhd_brio_wu((n, 1, 1), gamma=gamma)
    G = oracle.ghosted(U0)
    dt = 0.2 * dx[0]
    for _ in range(int(round(t_end / dt))):
        oracle.ssprk3_step(oracle.MHD, G, dx, dt, oracle.params(gamma_eos=gamma))
    return oracle.interior(G)[:, 0, 0, :]


def primitives(U, gamma=GAMMA):
    rho, sx, sy, sz, E, bx, by, bz = U
    vx, vy, vz = sx / rho, sy / rho, sz / rho
    p = (gamma - 1) * (E - 0.5 * rho * (vx * vx + vy * vy + vz * vz) - 0.5 * (bx * bx + by * by + bz * bz))
    return rho, vx, by, p


if __name__ == "__main__":
    U = run(NREF)
    step = NREF // NOUT
    rho, vx, by, p = (q[::step][:NOUT // 2] for q in primitives(U))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "brio_wu_reference.txt")
    with open(out, "w") as f:
        f.write("# Brio & Wu shock tube (Sec. IV.B.2) at t = 0.2: FP64 oracle, WENO5-JS + LLF,\n")
        f.write(f"# SSP-RK3, dt = 0.2 dx, Gamma = 2, {NREF} points on the doubled periodic tube [0, 2)\n")
        f.write(f"# (tests/golden/make_brio_wu.py).  Columns: x rho v_x B_y p at x = 2 m / {NOUT}.\n")
        for m in range(NOUT // 2):
            f.write(f"{2.0 * m / NOUT:.6f} {rho[m]:.12e} {vx[m]:.12e} {by[m]:.12e} {p[m]:.12e}\n")
    print("wrote", out)
