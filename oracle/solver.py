"""Newton-Raphson backward-Euler step, Delta-t ramp and coarse-to-fine steady continuation.

* ``step``: one implicit step k -> k+1 of eq. 7 (with eqs. 8-13), solved by
  Newton-Raphson (Sec. 2): linearise into eq. 14, solve J du = -F by multigrid,
  u += du, until every field's scale-free residual rho_f <= tol.  The step is
  rejected when Newton needs more than ``max_newton`` iterations (the paper
  observed fewer than 10), when max |dV| exceeds ``corr_limit`` (the "upper
  limit" on the Newton correction norm of Sec. 2, read as half the applied voltage
  0.5 |V_anode - V_cathode|), when
  the linear solve fails, or on non-finite values.
* ``march``: Delta t_1, then Delta t_{k+1} = n Delta t_k (n = 5) capped at dt_max;
  after a rejection go back and retry with the previous accepted Delta t, and
  halve it if that fails as well (Sec. 2 says "go back and choose
  Delta t_{k+1} = Delta t_k"; the halving is this project's addition).  Stops
  when the steady residual (time term dropped) is <= tol.
* ``solve_steady``: the "multilevel prolongation" of Sec. 2 / abstract: steady
  state on the grid coarsened by two, prolonged bilinearly to the fine grid,
  then the fine march starts with the long step dt_max.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

from . import discretization as disc
from . import multigrid as mg
from .grid import Grid


@dataclasses.dataclass
class SolverOptions:
    nu1: int = 4
    nu2: int = 4
    nu_coarse_n: int = 64     # levels with at most this many intervals per side smooth with
    nu_coarse1: int = 2       # nu_coarse1 / nu_coarse2 sweeps (0: nu1 / nu2 everywhere)
    nu_coarse2: int = 2
    nu_tiny_n: int = 8        # levels with at most this many intervals per side smooth with
    nu_tiny1: int = 1         # nu_tiny1 / nu_tiny2 sweeps (checked before nu_coarse_n)
    nu_tiny2: int = 1
    chain_from: int = 1       # continuation starts on the grid coarsened this many times
    eta: float = 1e-3               # inexact-Newton linear tolerance
    max_vcycles: int = 60
    coarsest: int = 2
    max_newton: int = 10
    corr_limit_frac: float = 0.5    # reject if max|dV| > frac * |V_anode - V_cathode|
    dt1: float = 1e-9
    dt_growth: float = 5.0
    dt_max: float = 1e-6
    max_steps: int = 400
    newton_tol: Optional[float] = None   # per-step Newton tolerance; default 0.1 * steady tol
    newton_tol_rel: float = 0.1     # > 0: a step's tolerance is max(newton_tol, this x the steady
                                    # residual at the step's start); 0: every step to newton_tol
    eta_adapt: bool = True          # relax eta when the Newton residual is near its target
    full_jacobian: bool = False     # Newton with the field dependence of mu, D in the Jacobian
    max_corrections: int = 20       # defect corrections per Newton iteration (full_jacobian)
    line_smoother: object = False   # line Gauss-Seidel instead of point red-black: True / "z"
                                    # (z-lines), "r" (r-lines), "alt" (alternating)


@dataclasses.dataclass
class StepStats:
    accepted: bool
    newton: int
    vcycles: List[int]
    rho: np.ndarray
    reason: str = ""


def forcing_term(opt: SolverOptions, rho_k: float, tol: float) -> float:
    """Linear tolerance of Newton iteration k: opt.eta, relaxed (up to 0.1) so that the linear
    residual is only driven to half the Newton target, eta_k = max(eta, min(0.1, tol / (2 rho_k)))
    (an inexact-Newton forcing term; the paper does not specify one)."""
    if not opt.eta_adapt:
        return opt.eta
    return max(opt.eta, min(0.1, 0.5 * tol / rho_k))


def full_jacobian_correct(g: Grid, x, dt, phys, H, fvec, du, eta, tn, opt: SolverOptions):
    """Newton step of the full Jacobian J_F (mu, D functions of |E|) by defect correction with
    the multigrid solver of the Picard Jacobian J_P: while
        max_f ||fvec - J_F du||_f / tn_f  >  eta * max_f ||fvec||_f / tn_f,
    solve J_P e = fvec - J_F du by V-cycles (same test, relative to the defect) and add e.
    Returns (du, V-cycles spent, converged)."""
    s = np.where(np.asarray(tn) > 0, tn, 1.0)

    def wnorm(v):
        return max(np.linalg.norm(v[k::3]) / s[k] for k in range(3))

    J = H.levels[0].J
    f0 = wnorm(fvec)
    ncyc = 0
    for _ in range(opt.max_corrections):
        r = fvec - disc.jacobian_full_apply(g, x, dt, phys, du, J)
        if wnorm(r) <= eta * f0:
            return du, ncyc, True
        e, hist = H.solve(r, eta, opt.max_vcycles, scale=tn)
        ncyc += len(hist) - 1
        if not np.isfinite(hist[-1]) or hist[-1] > eta:
            return du, ncyc, False
        du = du + e
    r = fvec - disc.jacobian_full_apply(g, x, dt, phys, du, J)
    return du, ncyc, bool(wnorm(r) <= eta * f0)


def step(g: Grid, u: np.ndarray, S_e, S_p, dt: float, phys: disc.Physics, tol: float,
         opt: SolverOptions):
    """One backward-Euler step; returns (u_new, StepStats).  u is not modified."""
    u_old = u
    x = disc.apply_dirichlet(u, phys, g)
    vcyc = []
    limit = opt.corr_limit_frac * abs(phys.V_anode - phys.V_cathode)
    for it in range(opt.max_newton + 1):
        F, T = disc.residual(g, x, u_old, S_e, S_p, dt, phys, with_terms=True)
        r = disc.rho(F, T)
        if not np.all(np.isfinite(r)):
            return u, StepStats(False, it, vcyc, r, "nonfinite")
        if r.max() <= tol:
            return x, StepStats(True, it, vcyc, r)
        if it == opt.max_newton:
            break
        H = mg.Hierarchy(g, x, dt, phys, opt.coarsest, opt.nu1, opt.nu2, opt.nu_coarse_n, opt.nu_coarse1,
                         opt.nu_coarse2, opt.nu_tiny_n, opt.nu_tiny1, opt.nu_tiny2, opt.line_smoother)
        tn = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
        eta = forcing_term(opt, r.max(), tol)
        fvec = -disc.to_vec(g, F)
        du, hist = H.solve(fvec, eta, opt.max_vcycles, scale=tn)
        vcyc.append(len(hist) - 1)
        if not np.isfinite(hist[-1]) or hist[-1] > eta:
            return u, StepStats(False, it + 1, vcyc, r, "linear solve failed")
        if opt.full_jacobian:
            du, ncyc, ok = full_jacobian_correct(g, x, dt, phys, H, fvec, du, eta, tn, opt)
            vcyc[-1] += ncyc
            if not ok:
                return u, StepStats(False, it + 1, vcyc, r, "full-Jacobian correction failed")
        d = disc.from_vec(g, du)
        if np.abs(d[2]).max() > limit:
            return u, StepStats(False, it + 1, vcyc, r, "correction limit")
        x = x + d
    return u, StepStats(False, opt.max_newton, vcyc, r, "newton cap")


def steady_rho(g: Grid, u, S_e, S_p, phys):
    F, T = disc.residual(g, u, None, S_e, S_p, None, phys, with_terms=True)
    return disc.rho(F, T)


def march(g: Grid, u, S_e, S_p, phys, tol, opt: SolverOptions, dt_start: float, log=None):
    """Time-march with the Delta-t ramp until the steady residual <= tol.

    Returns (u, converged, records) where records lists (dt, accepted, newton, vcycles, steady_rho).
    """
    dt = dt_start
    dt_prev = None
    records = []
    newton_tol = 0.1 * tol if opt.newton_tol is None else opt.newton_tol
    # Sec. 2: the time accuracy of the march does not matter for the steady state, so a step may
    # be solved only to a fraction of the steady residual it starts from
    r_start = steady_rho(g, u, S_e, S_p, phys).max() if opt.newton_tol_rel > 0 else 0.0
    for _ in range(opt.max_steps):
        u_new, st = step(g, u, S_e, S_p, dt, phys, max(newton_tol, opt.newton_tol_rel * r_start), opt)
        if st.accepted:
            u = u_new
            rs = steady_rho(g, u, S_e, S_p, phys)
            r_start = rs.max()
            records.append((dt, True, st.newton, sum(st.vcycles), rs.max()))
            if log:
                log(records[-1])
            if rs.max() <= tol:
                return u, True, records
            dt_prev = dt
            dt = min(dt * opt.dt_growth, opt.dt_max)
        else:
            records.append((dt, False, st.newton, sum(st.vcycles), np.nan))
            if log:
                log(records[-1] + (st.reason,))
            if dt_prev is not None and dt > dt_prev:
                dt = dt_prev
            else:
                dt = 0.5 * dt
                dt_prev = None if dt_prev is None else min(dt_prev, dt)
    return u, False, records


def prolong_state(gc: Grid, gf: Grid, uc: np.ndarray) -> np.ndarray:
    """Bilinear interpolation of node arrays (3, ...) from gc to the nested finer gf."""
    out = np.zeros((uc.shape[0],) + gf.shape)
    out[:, ::2, ::2] = uc
    out[:, ::2, 1::2] = 0.5 * (uc[:, :, :-1] + uc[:, :, 1:])
    w1 = (gf.z[1::2] - gc.z[:-1]) / (gc.z[1:] - gc.z[:-1])
    out[:, 1::2, :] = (1.0 - w1)[None, :, None] * out[:, 0:-1:2, :] + w1[None, :, None] * out[:, 2::2, :]
    return out


def solve_steady(g: Grid, u0, S_e, S_p, phys, tol, opt: SolverOptions, log=None):
    """Multilevel continuation (abstract and Sec. 2): steady solve on the grid coarsened
    opt.chain_from times (u0 and the sources injected, march from dt1), then on each finer grid
    the prolonged steady state marched from dt_max.  Returns (u, ok, coarse records, fine
    records); the coarse records hold every level but the finest."""
    grids, us, Se, Sp = [g], [u0], [S_e], [S_p]
    for _ in range(opt.chain_from):
        gc = grids[-1].coarse()
        us.append(mg.inject(grids[-1], us[-1]))
        Se.append(mg.inject(grids[-1], Se[-1]))
        Sp.append(mg.inject(grids[-1], Sp[-1]))
        grids.append(gc)
    k = opt.chain_from
    u = disc.apply_dirichlet(us[k], phys, grids[k])
    u, ok, rec_c = march(grids[k], u, Se[k], Sp[k], phys, tol, opt, opt.dt1, log)
    if not ok:
        return u0, False, rec_c, []
    for k in range(opt.chain_from - 1, -1, -1):
        u = disc.apply_dirichlet(prolong_state(grids[k + 1], grids[k], u), phys, grids[k])
        u, ok, rec = march(grids[k], u, Se[k], Sp[k], phys, tol, opt, opt.dt_max, log)
        if k > 0:
            rec_c = rec_c + rec
            if not ok:
                return u0, False, rec_c, []
        else:
            return u, ok, rec_c, rec
    raise AssertionError("unreachable")
