"""Writes tgv64_diagnostics.json: integral diagnostics of the oracle's
compressible Taylor-Green vortex run (Section 6: Ma = 0.1, Re = 1600, Pr =
0.72, gamma = 1.4, [0, 2 pi]^3 periodic, Navier-Stokes with WENO5-JS, HLLC,
C4 viscous and heat fluxes, TVD-RK3 at CFL 0.5) on a 64^3 grid for 500 CFL
steps, sampled every 10 steps.

Long runs are compared by integral quantities, not point values: the
volume-averaged kinetic energy
    E_k = < rho |u|^2 / 2 >
and enstrophy
    Omega = < rho |omega|^2 / 2 >,  omega = curl u
(second-order central differences on the periodic grid), both averages over
the cells of the uniform grid.  These are post-processing of a state, not
part of the scheme.

Only the oracle runs here:  python tests/golden/make_tgv64_diagnostics.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "tgv64_diagnostics.json")
N = 64
STEPS = 500
EVERY = 10


def diagnostics(U, n=N, length=2 * np.pi):
    """(E_k, Omega) of a state U[5][n][n][n] (x fastest) on the periodic
    cube of side `length`."""
    U = np.asarray(U, dtype=np.float64).reshape(5, n, n, n)
    rho = U[0]
    vel = U[1:4] / rho  # u, v, w; arrays indexed [z][y][x]
    ek = float(np.mean(0.5 * rho * (vel ** 2).sum(axis=0)))
    h = length / n

    def d(f, axis):  # d/dx_axis, axis 0 = x (array axis 2)
        a = 2 - axis
        return (np.roll(f, -1, axis=a) - np.roll(f, 1, axis=a)) / (2 * h)

    u, v, w = vel
    wx = d(w, 1) - d(v, 2)
    wy = d(u, 2) - d(w, 0)
    wz = d(v, 0) - d(u, 1)
    ens = float(np.mean(0.5 * rho * (wx * wx + wy * wy + wz * wz)))
    return ek, ens


def main():
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2203_13760_gb300 import inputs
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    case = inputs.taylor_green(N)
    c = oracle.config(**case.params())
    U = case.U.copy()
    t = 0.0
    rows = []
    for step in range(STEPS + 1):
        if step % EVERY == 0:
            ek, ens = diagnostics(U)
            rows.append({"step": step, "t": t, "kinetic_energy": ek, "enstrophy": ens})
            print(step, t, ek, ens, flush=True)
        if step == STEPS:
            break
        dt = oracle.compute_dt(c, U)
        U = oracle.rk3_step(c, U, dt)
        t += dt
    rec = {
        "source": "oracle (FP64 C++), written by tests/golden/make_tgv64_diagnostics.py",
        "citation": "Section 6 (compressible Taylor-Green vortex, Ma = 0.1, Re = 1600); Table 3 setup 'HLLC'",
        "grid": [N, N, N], "steps": STEPS, "every": EVERY, "cfl": 0.5,
        "diagnostics": "E_k = <rho |u|^2 / 2>, Omega = <rho |curl u|^2 / 2>, central differences",
        "rows": rows,
    }
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)


if __name__ == "__main__":
    main()
