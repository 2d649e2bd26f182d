"""Work counts of the oracle's own steady continuation (test / baseline infrastructure).

Runs ``solver.solve_steady`` on a workload and records, per grid level, the accepted
and rejected steps, Newton iterations and V-cycles (the counts the GPU path's parity test
compares with, written to tests/golden by a script that calls only this package).
"""
from __future__ import annotations

import time

import numpy as np

from . import discretization as disc
from . import solver as so
from .grid import Grid


def steady_counts(d, tol=1e-8, opt=None):
    """(counts, wall_seconds, final_state) of solve_steady on a workloads.Discharge."""
    opt = opt or so.SolverOptions()
    g = Grid(d.nr, d.nz, d.R, d.z)
    phys = disc.Physics(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p,
                        D_p=d.D_p, table=d.table, pressure_factor=d.pressure_factor)
    u0 = np.stack([d.ne0, d.np0, d.V0])
    t0 = time.perf_counter()
    u, ok, rec_c, rec_f = so.solve_steady(g, u0, d.S_e, d.S_p, phys, tol, opt)
    wall = time.perf_counter() - t0

    def summarize(rec, n):
        acc = [r for r in rec if r[1]]
        return {"n": n, "steps": len(acc), "rejected": len(rec) - len(acc),
                "newton": int(sum(r[2] for r in rec)), "vcycles": int(sum(r[3] for r in rec))}

    counts = {"ok": bool(ok), "levels": [summarize(rec_c, d.nr // 2), summarize(rec_f, d.nr)]}
    return counts, wall, u
