"""Work counts of the oracle's own steady continuation (test / baseline infrastructure).

Runs ``solver.solve_steady`` on a workload and records, per grid level, the accepted
and rejected steps, Newton iterations and V-cycles.  A CPU-baseline timer multiplies
these counts by per-unit oracle timings measured on a bounded sample.
"""
from __future__ import annotations

import time

import numpy as np

from . import discretization as disc
from . import multigrid as mg
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


def unit_times(d, level_n, dt=1e-6, vcycles=3, opt=None):
    """Seconds per oracle work unit on the grid with level_n intervals: one Jacobian hierarchy
    build, one nonlinear residual, one V-cycle (from the workload's initial state)."""
    opt = opt or so.SolverOptions()
    step = d.nr // level_n
    g = Grid(level_n, d.nz // step, d.R, d.z[::step])
    phys = disc.Physics(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p,
                        D_p=d.D_p, table=d.table, pressure_factor=d.pressure_factor)
    u = np.stack([d.ne0, d.np0, d.V0])[:, ::step, ::step].copy()
    S_e, S_p = d.S_e[::step, ::step], d.S_p[::step, ::step]
    t0 = time.perf_counter()
    F, T = disc.residual(g, u, u, S_e, S_p, dt, phys, with_terms=True)
    t_res = time.perf_counter() - t0
    t0 = time.perf_counter()
    H = mg.Hierarchy(g, u, dt, phys, opt.coarsest, opt.nu1, opt.nu2, opt.nu_coarse_n, opt.nu_coarse1,
                     opt.nu_coarse2, opt.nu_tiny_n, opt.nu_tiny1, opt.nu_tiny2)
    t_hier = time.perf_counter() - t0
    f = -disc.to_vec(g, F)
    x = np.zeros_like(f)
    t0 = time.perf_counter()
    for _ in range(vcycles):
        x = H.vcycle(0, x, f)
        _ = f - H.levels[0].J @ x
    t_vc = (time.perf_counter() - t0) / vcycles
    return {"residual": t_res, "hierarchy": t_hier, "vcycle": t_vc}
