"""Pins for the oracle's Newton time step, Delta-t ramp and steady continuation (Sec. 2).

* a Newton step solved with V-cycles equals the same step solved with a direct
  dense solve of eq. 14 (single-level hierarchy);
* with mu = 0 the system is linear, so exact Newton converges in one iteration;
* the paper's run statistics: fewer than 10 Newton iterations per step;
* a steady state is a fixed point of the implicit step for any dt;
* the Delta-t ramp follows Delta t_{k+1} = 5 Delta t_k from 1 ns (the values printed
  in Sec. 2, stored under tests/golden/) and goes back to the previous Delta t after a
  forced rejection;
* the state prolongation of the continuation is exact for bilinear functions.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import discretization as disc
from oracle import multigrid as mg
from oracle import solver as so
from oracle.grid import Grid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _case(n=16, V_c=-200.0, table=False, seed=0):
    d = W.make_discharge(n, seed=seed, V_cathode=V_c, use_table=table)
    g = Grid(d.nr, d.nz, d.R, d.z)
    phys = disc.Physics(V_cathode=d.V_cathode, table=d.table)
    u = np.stack([d.ne0, d.np0, d.V0])
    return d, g, phys, u


def test_paper_printed_driver_constants():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as fh:
        pc = json.load(fh)
    opt = so.SolverOptions()
    assert opt.dt1 == pc["dt1_s"]["value"]
    assert opt.dt_growth == pc["dt_growth_n"]["value"]
    assert opt.max_newton == pc["newton_iterations_below"]["value"]


def test_mg_step_equals_direct_step():
    d, g, phys, u = _case(16)
    opt_mg = so.SolverOptions(eta=1e-13)
    opt_lu = so.SolverOptions(eta=1e-13, coarsest=10 ** 6)   # one level: dense LU
    a, sa = so.step(g, u, d.S_e, d.S_p, 1e-9, phys, 1e-12, opt_mg)
    b, sb = so.step(g, u, d.S_e, d.S_p, 1e-9, phys, 1e-12, opt_lu)
    assert sa.accepted and sb.accepted
    for f in range(3):
        assert np.abs(a[f] - b[f]).max() <= 1e-11 * np.abs(b[f]).max()


def test_linear_case_newton_converges_in_one_iteration():
    d, g, phys, u = _case(16)
    phys.mu_e = 0.0
    phys.mu_p = 0.0
    opt = so.SolverOptions(eta=1e-14, max_vcycles=200)
    _, st = so.step(g, u, d.S_e, d.S_p, 1e-8, phys, 1e-12, opt)
    assert st.accepted and st.newton == 1, st


def test_transient_33_newton_iterations_below_ten():
    d = W.transient_33()
    g = Grid(d.nr, d.nz, d.R, d.z)
    phys = disc.Physics(V_cathode=d.V_cathode)
    u = np.stack([d.ne0, d.np0, d.V0])
    opt = so.SolverOptions(eta=1e-12)
    for _ in range(3):
        u, st = so.step(g, u, d.S_e, d.S_p, 1e-9, phys, 1e-10, opt)
        assert st.accepted and st.newton < 10 and st.rho.max() <= 1e-10


def test_steady_state_is_fixed_point_of_the_step():
    d, g, phys, u = _case(16, V_c=-300.0, table=True)
    opt = so.SolverOptions(eta=1e-6)
    us, ok, rec = so.march(g, u, d.S_e, d.S_p, phys, 1e-10, opt, 1e-9)
    assert ok
    for dt in (1e-9, 1e-6, 1e-3):
        F, T = disc.residual(g, us, us, d.S_e, d.S_p, dt, phys, with_terms=True)
        assert disc.rho(F, T).max() <= 1e-9


def test_dt_ramp_and_rejection():
    d, g, phys, u = _case(8, V_c=-300.0)
    opt = so.SolverOptions(eta=1e-6, dt_max=1e-7, max_steps=6, newton_tol=1e-8)
    _, _, rec = so.march(g, u, d.S_e, d.S_p, phys, 1e-30, opt, 1e-9)
    dts = [r[0] for r in rec if r[1]]
    assert np.allclose(dts[:4], [1e-9, 5e-9, 2.5e-8, 1e-7])
    # force a rejection at the first step with a correction limit of ~0: the ramp halves dt
    opt2 = so.SolverOptions(eta=1e-6, corr_limit_frac=1e-12, max_steps=3, newton_tol=1e-8)
    _, ok, rec2 = so.march(g, u, d.S_e, d.S_p, phys, 1e-30, opt2, 1e-9)
    assert not ok and [r[1] for r in rec2] == [False] * 3
    assert np.allclose([r[0] for r in rec2], [1e-9, 5e-10, 2.5e-10])


def test_rejected_step_goes_back_to_previous_dt():
    d, g, phys, u = _case(8, V_c=-300.0)
    calls = []
    real_step = so.step

    def fake_step(g_, u_, Se, Sp, dt, ph, tol, opt):
        calls.append(dt)
        if len(calls) == 3:            # third attempt (dt = 2.5e-8) is rejected
            return u_, so.StepStats(False, 1, [1], np.zeros(3), "forced")
        return real_step(g_, u_, Se, Sp, dt, ph, tol, opt)

    so.step = fake_step
    try:
        so.march(g, u, d.S_e, d.S_p, phys, 1e-30, so.SolverOptions(eta=1e-6, max_steps=5, newton_tol=1e-8), 1e-9)
    finally:
        so.step = real_step
    assert np.allclose(calls[:5], [1e-9, 5e-9, 2.5e-8, 5e-9, 2.5e-8])


def test_prolong_state_exact_for_bilinear():
    gf = Grid(16, 16, 1e-2, W.z_nodes(16, 1e-2))
    gc = gf.coarse()
    f = lambda r, z: 1.0 - 2.0 * r / 1e-2 + 0.5 * z / 1e-2 + 3.0 * r * z / 1e-4
    rc, zc = np.meshgrid(gc.r, gc.z)
    rf, zf = np.meshgrid(gf.r, gf.z)
    out = so.prolong_state(gc, gf, np.stack([f(rc, zc)] * 3))
    assert np.allclose(out, np.stack([f(rf, zf)] * 3), rtol=1e-13, atol=1e-13)


def test_transient_33_regression_golden():
    """Regression against values written by tests/golden/make_golden.py (oracle only)."""
    with open(os.path.join(GOLDEN, "oracle_transient_33.json")) as fh:
        gold = json.load(fh)
    d = W.transient_33()
    g = Grid(d.nr, d.nz, d.R, d.z)
    phys = disc.Physics(V_cathode=d.V_cathode)
    u = np.stack([d.ne0, d.np0, d.V0])
    opt = so.SolverOptions(eta=1e-12)
    for _ in range(gold["steps"]):
        u, st = so.step(g, u, d.S_e, d.S_p, gold["dt"], phys, gold["tol"], opt)
        assert st.accepted
    for k, name in enumerate(("ne", "np", "V")):
        assert np.isclose(np.abs(u[k]).sum(), gold[name + "_l1"], rtol=1e-10)
        assert np.isclose(u[k][gold["probe_j"], gold["probe_i"]], gold[name + "_probe"], rtol=1e-10)


def _steady_problem(n, seed=0):
    d = W.make_discharge(n, seed=seed, V_cathode=-300.0)
    g = Grid(d.nr, d.nz, d.R, d.z)
    phys = disc.Physics(V_cathode=d.V_cathode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p, D_p=d.D_p)
    return d, g, phys, np.stack([d.ne0, d.np0, d.V0])


def test_chain_from_one_is_the_two_level_continuation():
    """chain_from = 1 is the printed two-level schedule: inject to N/2, march from dt1,
    prolong, march from dt_max (written out here step by step)."""
    d, g, phys, u0 = _steady_problem(16)
    opt = so.SolverOptions(eta=1e-10)
    u, ok, rc, rf = so.solve_steady(g, u0, d.S_e, d.S_p, phys, 1e-8, opt)
    assert ok
    gc = g.coarse()
    uc = disc.apply_dirichlet(mg.inject(g, u0), phys)
    uc, okc, _ = so.march(gc, uc, mg.inject(g, d.S_e), mg.inject(g, d.S_p), phys, 1e-8, opt, opt.dt1)
    uf = disc.apply_dirichlet(so.prolong_state(gc, g, uc), phys)
    uf, okf, _ = so.march(g, uf, d.S_e, d.S_p, phys, 1e-8, opt, opt.dt_max)
    assert okc and okf
    assert np.array_equal(u, uf)


@pytest.mark.parametrize("dt_max", [1e-6, 1.0])
def test_chain_reaches_the_same_steady_state(dt_max):
    """Starting the continuation two levels further down (and with the paper's uncapped ramp)
    ends on the same discrete steady state: rho <= tol on the finest grid and the state of the
    two-level schedule to the accuracy the tolerance allows."""
    d, g, phys, u0 = _steady_problem(16, seed=3)
    base, ok0, _, _ = so.solve_steady(g, u0, d.S_e, d.S_p, phys, 1e-9, so.SolverOptions(eta=1e-10))
    assert ok0
    opt = so.SolverOptions(eta=1e-10, chain_from=2, dt_max=dt_max)
    u, ok, rc, rf = so.solve_steady(g, u0, d.S_e, d.S_p, phys, 1e-9, opt)
    assert ok and len(rf) >= 1
    assert so.steady_rho(g, u, d.S_e, d.S_p, phys).max() <= 1e-9
    for q in range(3):
        assert np.abs(u[q] - base[q]).max() <= 1e-6 * np.abs(base[q]).max(), q


def test_march_step_tolerances(monkeypatch):
    """The per-step Newton tolerance of a march: 0.1 x the steady tolerance with newton_tol_rel = 0,
    and with newton_tol_rel = theta the larger of it and theta x the steady residual of the state
    the step starts from (the initial state, then each accepted step's result)."""
    d, g, phys, u0 = _steady_problem(8, seed=2)
    tol, theta = 1e-9, 0.05
    seen = []
    real_step = so.step

    def spy(g_, u_, Se, Sp, dt, phys_, ntol, opt_):
        seen.append((ntol, so.steady_rho(g_, u_, Se, Sp, phys_).max()))
        return real_step(g_, u_, Se, Sp, dt, phys_, ntol, opt_)

    monkeypatch.setattr(so, "step", spy)
    _, ok, rec = so.march(g, u0, d.S_e, d.S_p, phys, tol, so.SolverOptions(eta=1e-10, newton_tol_rel=0.0), 1e-9)
    assert ok and len(seen) == len(rec) and all(t == 0.1 * tol for t, _ in seen)
    seen.clear()
    _, ok, rec = so.march(g, u0, d.S_e, d.S_p, phys, tol, so.SolverOptions(eta=1e-10, newton_tol_rel=theta), 1e-9)
    assert ok and len(seen) == len(rec)
    for t, r_start in seen:
        assert t == max(0.1 * tol, theta * r_start)
    assert seen[0][0] > 0.1 * tol    # the first steps, far from the steady state, are solved loosely


def test_relative_step_tolerance_reaches_the_same_steady_state():
    """Loose steps far from the steady state (newton_tol_rel) end on the same discrete steady
    state as steps each solved to 0.1 x the steady tolerance, with fewer Newton iterations."""
    d, g, phys, u0 = _steady_problem(16, seed=3)
    base, ok0, rc0, rf0 = so.solve_steady(g, u0, d.S_e, d.S_p, phys, 1e-9,
                                          so.SolverOptions(eta=1e-10, newton_tol_rel=0.0))
    u, ok, rc, rf = so.solve_steady(g, u0, d.S_e, d.S_p, phys, 1e-9, so.SolverOptions(eta=1e-10, newton_tol_rel=0.1))
    assert ok0 and ok
    assert so.steady_rho(g, u, d.S_e, d.S_p, phys).max() <= 1e-9
    for q in range(3):
        assert np.abs(u[q] - base[q]).max() <= 1e-6 * np.abs(base[q]).max(), q
    newton = lambda recs: sum(r[2] for r in recs)
    assert newton(rc) + newton(rf) < newton(rc0) + newton(rf0)


def _cathode_ion_current(g, u, phys):
    _, (mez, dez, mpz, dpz) = disc.face_transport(g, u[2], phys)
    phi = disc.sg_flux(g.gz[0], mpz[0], dpz[0], 1.0, u[1][0], u[1][1], u[2][0], u[2][1])
    return -2.0 * np.pi * 1.602176634e-19 * phi.sum()


@pytest.mark.parametrize("a,b,key,rtol", [(30.0, 24.0, "a30_b24", 0.06), (10.0, 1.0, "a10_b1", 0.02)])
def test_argon_ion_current_matches_the_paper(a, b, key, rtol):
    """The paper's argon discharge (Sec. 3) on 33^2 nodes: the steady ion current into the
    cathode is the printed one (0.59 mA and 0.035 mA, two significant digits).  At steady state
    it equals e times the total ion production, nearly independent of the ion mobility the
    paper does not print (here a stand-in), so the printed currents pin the Dirichlet-wall
    discretisation, the sources and the continuation together."""
    with open(os.path.join(GOLDEN, "paper_constants.json")) as fh:
        ref = json.load(fh)["argon_ion_current_mA"][key]
    d = W.argon(32, a=a, b=b)
    g = Grid(d.nr, d.nz, d.R, d.z, wall_dirichlet=True)
    phys = disc.Physics(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p, D_p=d.D_p)
    u, ok, _, _ = so.solve_steady(g, np.stack([d.ne0, d.np0, d.V0]), d.S_e, d.S_p, phys, 1e-8, so.SolverOptions())
    assert ok
    I_mA = _cathode_ion_current(g, u, phys) * 1e3
    assert abs(I_mA - ref) <= rtol * ref, (I_mA, ref)
    # and it is the ion production, whatever the ion mobility (within the losses to the walls)
    prod = 2.0 * np.pi * 1.602176634e-19 * (g.A[1:-1, :g.ni] * d.S_p[1:-1, :g.ni]).sum() * 1e3
    assert abs(I_mA - prod) <= 0.01 * prod


def test_full_jacobian_newton_converges_quadratically():
    """f4: with the field dependence of mu(|E|), D(|E|) in the Jacobian (defect correction around
    the Picard multigrid solve), Newton from a 2 % density perturbation of a near-steady state
    needs half the iterations of the Picard iteration (2 against 4 to rho <= 1e-11 at every dt)
    and ends on the same state."""
    d = W.make_discharge(16, seed=1, V_cathode=-300.0, use_table=True)
    g = Grid(d.nr, d.nz, d.R, d.z)
    phys = disc.Physics(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p,
                        D_p=d.D_p, table=d.table, pressure_factor=d.pressure_factor)
    us, ok, _ = so.march(g, np.stack([d.ne0, d.np0, d.V0]), d.S_e, d.S_p, phys, 1e-6, so.SolverOptions(eta=1e-10),
                         1e-9)
    assert ok
    start = us * np.array([1.02, 1.02, 1.0])[:, None, None]
    for dt in (1e-7, 1e-5, 1e-3):
        up, sp_ = so.step(g, start, d.S_e, d.S_p, dt, phys, 1e-11, so.SolverOptions(eta=1e-10))
        uf, sf = so.step(g, start, d.S_e, d.S_p, dt, phys, 1e-11, so.SolverOptions(eta=1e-10, full_jacobian=True))
        assert sp_.accepted and sf.accepted
        assert sf.newton == 2 and sp_.newton >= 3, (dt, sf.newton, sp_.newton)
        for q in range(3):
            assert np.abs(uf[q] - up[q]).max() <= 1e-9 * np.abs(up[q]).max(), (dt, q)
