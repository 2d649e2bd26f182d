"""Writes tests/golden/oracle_vcycle_factors.json from the FP64 oracle only: the residual
history of seven V-cycles (no stopping test) on the linearised system of one backward-Euler step
(eq. 14, Delta t = 1e-7 s, old state 0.99 x the state) of the benchmark's discharge family
(constant transport, -300 V, seed 0) on 257^2, 513^2, 1025^2 and 2049^2 nodes.  The oracle's
default multigrid (V(4,4) above 65^2, red-black collective Gauss-Seidel, coarse operators
rediscretised on injected states).  Its convergence factor grows with the grid at this Delta t
(the ions' drift dominates their diffusion on the coarse levels); the GPU's cycle must follow
the same history.

Run from the repository root:  python tests/golden/make_oracle_vcycle_factors.py   (about 5 minutes)
"""
import json
import os
import sys
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import discretization as disc  # noqa: E402
from oracle import multigrid as omg  # noqa: E402
from oracle.grid import Grid  # noqa: E402

SIZES = (256, 512, 1024, 2048)
DT = 1e-7
CYCLES = 7


def history(n):
    d = W.make_discharge(n, seed=0, V_cathode=-300.0)
    g = Grid(d.nr, d.nz, d.R, d.z)
    phys = disc.Physics(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p,
                        D_p=d.D_p, table=d.table, pressure_factor=d.pressure_factor)
    u = np.stack([d.ne0, d.np0, d.V0])
    F, T = disc.residual(g, u, u * 0.99, d.S_e, d.S_p, DT, phys, with_terms=True)
    tn = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
    _, h = omg.Hierarchy(g, u, DT, phys).solve(disc.to_vec(g, -F), 0.0, CYCLES, scale=tn)
    return [float(v) for v in h]


def main():
    out = {"dt": DT, "cycles": CYCLES, "workload": "make_discharge(n, seed=0, V_cathode=-300.0), old state 0.99 u",
           "histories": {}}
    for n in SIZES:
        t0 = time.time()
        out["histories"][str(n)] = history(n)
        print(n, f"{time.time() - t0:.0f} s", out["histories"][str(n)], flush=True)
    with open(os.path.join(ROOT, "tests", "golden", "oracle_vcycle_factors.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
