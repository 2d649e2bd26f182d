"""GPU (CUDA, sm_103a) parity of the C-ABI library against the FP64 CPU oracle.

Every call goes through libmg.so (include/mg.h) via the ctypes binding.  FP64
tolerances: residual rows and Jacobian products agree to 1e-12 of the row
scale (rounding order only); linear and Newton solves to 1e-10 relative
max-norm per field (both sides solved to 1e-12 or tighter).
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import discretization as disc
from oracle import multigrid as omg
from oracle import solver as osv
from oracle.grid import Grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0811_4446_gb300 import build, mg as mgmod
    build.build()
    return mgmod


def _oracle(d):
    g = Grid(d.nr, d.nz, d.R, d.z)
    phys = disc.Physics(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p,
                        D_p=d.D_p, table=d.table, pressure_factor=d.pressure_factor)
    return g, phys


def _random_state(d, rng, scale=1.0):
    shape = d.shape
    ne = 1e14 * (0.5 + rng.random(shape)) * scale
    np_ = 1e14 * (0.5 + rng.random(shape)) * scale
    V = d.V0 + 3.0 * rng.standard_normal(shape)
    u = disc.apply_dirichlet(np.stack([ne, np_, V]), disc.Physics(V_cathode=d.V_cathode))
    return u


# Measured GPU-vs-oracle agreement of the steady paths (FP64, same algorithm, same counts):
# 1e-16 .. 2e-14 relative max-norm per field on 17^2 ... 257^2, mixed 257^2 9e-13.  The contract
# tolerances below (FP64 1e-10, mixed 1e-8) therefore hold with orders of magnitude to spare.
FP64_TOL = 1e-10
MIXED_TOL = 1e-8
# GPU and oracle evaluate the scale-free residual of the same state to 1e-9 relative
# (test_residual_parity); a GPU result that met its tolerance meets the oracle's test up to that.
RHO_AGREE = 1e-9


def _assert_fields(ug, uo, tol, what=""):
    for q in range(3):
        err = np.abs(ug[q] - uo[q]).max() / np.abs(uo[q]).max()
        assert err <= tol, (what, q, err)


def _gpu_counts(st):
    """(coarse steps, coarse Newton, coarse V-cycles, all steps, rejected, Newton, V-cycles)."""
    return (st["coarse_steps"], st["coarse_newton"], st["coarse_vcycles"],
            st["steps_accepted"] + st["steps_rejected"], st["steps_rejected"], st["newton_iterations"],
            st["vcycles"])


def _oracle_counts(rec_c, rec_f):
    rr = rec_c + rec_f
    return (len(rec_c), sum(r[2] for r in rec_c), sum(r[3] for r in rec_c), len(rr),
            sum(1 for r in rr if not r[1]), sum(r[2] for r in rr), sum(r[3] for r in rr))


CASES = [(8, 8, False), (32, 32, False), (32, 32, True), (64, 16, True), (16, 64, False), (128, 128, True)]


@pytest.mark.parametrize("nr,nz,table", CASES)
@pytest.mark.parametrize("dt", [1e-9, 1e-6, 0.0])
def test_residual_parity(mg, nr, nz, table, dt):
    d = W.make_discharge(nr, nz=nz, seed=3, V_cathode=-250.0, use_table=table, pressure_factor=1.3)
    g, phys = _oracle(d)
    rng = np.random.default_rng(11)
    u = _random_state(d, rng)
    uo = _random_state(d, rng)
    s = mg.from_discharge(d)
    s.set_state(*[np.ascontiguousarray(a) for a in u])
    s.set_old_state(*[np.ascontiguousarray(a) for a in uo])
    Fg, rho_g = s.residual(dt)
    F, T = disc.residual(g, u, uo, d.S_e, d.S_p, dt if dt > 0 else None, phys, with_terms=True)
    for f in range(3):
        scale = np.abs(T[f]).max()
        assert np.abs(Fg[f] - F[f]).max() <= 1e-12 * scale, (f, np.abs(Fg[f] - F[f]).max(), scale)
    assert np.allclose(rho_g, disc.rho(F, T), rtol=1e-9, atol=1e-300)


@pytest.mark.parametrize("nr,nz,table", CASES[:5])
def test_jacobian_apply_parity(mg, nr, nz, table):
    d = W.make_discharge(nr, nz=nz, seed=5, V_cathode=-300.0, use_table=table)
    g, phys = _oracle(d)
    rng = np.random.default_rng(2)
    u = _random_state(d, rng)
    s = mg.from_discharge(d)
    s.set_state(*[np.ascontiguousarray(a) for a in u])
    for dt in (1e-9, 0.0):
        v = np.zeros((3,) + d.shape)
        v[:, 1:-1] = rng.standard_normal((3, d.nz - 1, d.nr + 1))
        v[0:2] *= 1e12
        Jg = s.jacobian_apply(dt, list(v))
        J = disc.jacobian(g, u, dt if dt > 0 else None, phys)
        Jv = disc.from_vec(g, J @ disc.to_vec(g, v))
        absJ = abs(J)
        scale = disc.from_vec(g, absJ @ np.abs(disc.to_vec(g, v)))
        for f in range(3):
            assert np.abs(Jg[f] - Jv[f]).max() <= 1e-12 * scale[f].max(), f


@pytest.mark.parametrize("state", ["zero_field", "zero_density"])
@pytest.mark.parametrize("table", [False, True])
def test_degenerate_states_parity(mg, state, table):
    """Degenerate states of the method against the oracle.  zero_field: no applied voltage and
    V = 0, so alpha = 0 on every face and the Scharfetter-Gummel weights take the Bernoulli
    series branch (B(0) = 1) everywhere; with the table, |E| = 0 lies below its range.
    zero_density: n_e = n_p = 0 under the applied field, so the fluxes, their V couplings and
    the space charge vanish.  Residual rows and Jacobian products to 1e-12 of the row scale, and
    linear solves to the FP64 (1e-10) and mixed (1e-8) bars."""
    d = W.make_discharge(32, seed=3, V_cathode=0.0 if state == "zero_field" else -300.0, use_table=table)
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    if state == "zero_field":
        assert not u[2].any()
    else:
        u[0:2] = 0.0
    uo = u * 0.99
    dt = 1e-9
    F, T = disc.residual(g, u, uo, d.S_e, d.S_p, dt, phys, with_terms=True)
    J = disc.jacobian(g, u, dt, phys)
    rng = np.random.default_rng(5)
    v = np.zeros((3,) + d.shape)
    v[:, 1:-1] = rng.standard_normal((3, d.nz - 1, d.nr + 1))
    v[0:2] *= 1e12
    Jv = disc.from_vec(g, J @ disc.to_vec(g, v))
    scale_j = disc.from_vec(g, abs(J) @ np.abs(disc.to_vec(g, v)))
    tn = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
    x, ho = omg.Hierarchy(g, u, dt, phys).solve(disc.to_vec(g, -F), 1e-12, 200, scale=tn)
    xo = disc.from_vec(g, x)
    for prec, tol in ((mg.MG_FP64, FP64_TOL), (mg.MG_MIXED, MIXED_TOL)):
        s = mg.from_discharge(d, precision=prec)
        s.set_state(*[np.ascontiguousarray(a) for a in u])
        s.set_old_state(*[np.ascontiguousarray(a) for a in uo])
        Fg, _ = s.residual(dt)
        for f in range(3):
            assert np.abs(Fg[f] - F[f]).max() <= 1e-12 * max(np.abs(T[f]).max(), 1e-300), (prec, f)
        Jg = s.jacobian_apply(dt, list(v))
        for f in range(3):
            assert np.abs(Jg[f] - Jv[f]).max() <= 1e-12 * scale_j[f].max(), (prec, f)
        xg, hg, rc = s.linear_solve(dt, list(-F), 1e-12, 200)  # the oracle's stopping residual
        assert rc == mg.MG_OK, (prec, hg)
        _assert_fields(xg, xo, tol, (state, prec))
        s.close()


@pytest.mark.parametrize("nr,nz", [(16, 16), (64, 64), (32, 16)])
def test_full_jacobian_apply_parity(mg, nr, nz):
    """f4: the full Jacobian (mu, D functions of |E|) times a random vector, FP64 GPU against
    the oracle's J_P v + transport_jv, to 1e-12 of the row scale."""
    d = W.make_discharge(nr, nz=nz, seed=5, V_cathode=-300.0, use_table=True)
    g, phys = _oracle(d)
    rng = np.random.default_rng(4)
    u = _random_state(d, rng)
    s = mg.from_discharge(d, full_jacobian=1)
    s.set_state(*[np.ascontiguousarray(a) for a in u])
    for dt in (1e-9, 0.0):
        v = np.zeros((3,) + d.shape)
        v[:, 1:-1] = rng.standard_normal((3, d.nz - 1, d.nr + 1))
        v[0:2] *= 1e12
        Jg = s.jacobian_apply(dt, list(v))
        J = disc.jacobian(g, u, dt if dt > 0 else None, phys)
        x = disc.to_vec(g, v)
        Jv = disc.from_vec(g, disc.jacobian_full_apply(g, u, dt if dt > 0 else None, phys, x, J))
        scale = disc.from_vec(g, abs(J) @ np.abs(x))
        for f in range(3):
            assert np.abs(Jg[f] - Jv[f]).max() <= 1e-12 * scale[f].max(), (dt, f)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_jacobian_newton_step_parity(mg, precision):
    """f4: one backward-Euler step with the full-Jacobian Newton (defect corrections around the
    Picard multigrid solve) from a 2 % density perturbation of a near-steady 17^2 state: the
    oracle's Newton iterations (fewer than the Picard Newton's) and state."""
    d = W.make_discharge(16, seed=1, V_cathode=-300.0, use_table=True)
    g, phys = _oracle(d)
    us, ok, _ = osv.march(g, np.stack([d.ne0, d.np0, d.V0]), d.S_e, d.S_p, phys, 1e-6,
                          osv.SolverOptions(eta=1e-10), 1e-9)
    assert ok
    start = disc.apply_dirichlet(us * np.array([1.02, 1.02, 1.0])[:, None, None], phys, g)
    prec = mg.MG_MIXED if precision == "mixed" else mg.MG_FP64
    counts = []
    for full in (0, 1):
        s = mg.from_discharge(d, precision=prec, eta=1e-10, max_vcycles=200, full_jacobian=full)
        s.set_state(*[np.ascontiguousarray(a) for a in start])
        rc, st = s.step(1e-5, 1e-11)
        assert rc == mg.MG_OK, st
        counts.append(st["newton_iterations"])
        uo, so_ = osv.step(g, start, d.S_e, d.S_p, 1e-5, phys, 1e-11,
                           osv.SolverOptions(eta=1e-10, max_vcycles=200, full_jacobian=bool(full)))
        assert so_.accepted and so_.newton == st["newton_iterations"], (full, so_.newton, st)
        ug = s.get_state()
        tolr = 1e-8 if precision == "mixed" else 1e-10
        for q in range(3):
            assert np.abs(ug[q] - uo[q]).max() <= tolr * np.abs(uo[q]).max(), (full, q)
    assert counts[1] < counts[0]


@pytest.mark.parametrize("n,table,dt", [(4, False, 1e-9), (16, False, 1e-9), (32, True, 1e-7), (64, True, 1e-6)])
def test_linear_solve_parity(mg, n, table, dt):
    d = W.make_discharge(n, seed=0, V_cathode=-300.0, use_table=table)
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    s = mg.from_discharge(d)
    s.set_old_state(*[np.ascontiguousarray(a * 0.99) for a in u])
    F, T = disc.residual(g, u, u * 0.99, d.S_e, d.S_p, dt, phys, with_terms=True)
    f = -F
    xg, hg, rc = s.linear_solve(dt, list(f), 1e-12, 200)
    assert rc == mg.MG_OK
    H = omg.Hierarchy(g, u, dt, phys)
    tn = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
    x, ho = H.solve(disc.to_vec(g, f), 1e-12, 200, scale=tn)
    xo = disc.from_vec(g, x)
    for q in range(3):
        assert np.abs(xg[q] - xo[q]).max() <= 1e-10 * np.abs(xo[q]).max(), q
    # same algorithm: the same cycle count and the same residual history
    assert abs(len(hg) - len(ho)) <= 1
    k = min(len(hg), len(ho), 6)
    assert np.allclose(hg[:k], ho[:k], rtol=1e-5, atol=1e-14)


@pytest.mark.parametrize("n,R,table,precision,line", [
    (32, 1e-2, False, "fp64", 1), (64, 1e-1, True, "fp64", 1), (32, 1e-1, False, "mixed", 1), (16, 1e-2, True, "fp64", 1),
    (32, 2e-3, False, "fp64", 2), (64, 2e-3, True, "fp64", 3), (32, 1e-3, False, "mixed", 2),
    (32, 1e-1, False, "fp64", 3), (16, 1e-2, True, "fp64", 2), (32, 1e-3, True, "mixed", 3)])
def test_line_smoother_linear_solve_parity(mg, n, R, table, precision, line):
    """f1: linear solves with zebra line smoothing on every level, z-lines (1), r-lines (2) or
    alternating lines (3; each sweep z-lines, then r-lines): block-tridiagonal line solves by
    cyclic reduction on the GPU, exact sparse line solves in the oracle.  The oracle's residual
    history cycle by cycle and its solution; where the lines follow the strong coupling (z-lines
    or alternating lines with R = 10 d, r-lines or alternating lines with R = d / 5 or d / 10)
    far fewer cycles than the point smoother.  FP64 cases with r-coupled grids take R = d / 5:
    with R = d / 10 the weighted residual's rounding floor (3e-12, both sides) keeps the solves
    from the 1e-12 the 1e-10 comparison needs."""
    d = W.make_discharge(n, seed=0, V_cathode=-300.0, use_table=table, R=R)
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    dt = 1e-7
    F, T = disc.residual(g, u, u * 0.99, d.S_e, d.S_p, dt, phys, with_terms=True)
    tn = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
    prec = mg.MG_MIXED if precision == "mixed" else mg.MG_FP64
    s = mg.from_discharge(d, precision=prec, line_smoother=line)
    s.set_old_state(*[np.ascontiguousarray(a * 0.99) for a in u])
    eta = 1e-12 if precision == "fp64" else 1e-10
    xg, hg, rc = s.linear_solve(dt, list(-F), eta, 200)
    assert rc == mg.MG_OK
    H = omg.Hierarchy(g, u, dt, phys, line={1: "z", 2: "r", 3: "alt"}[line])
    x, ho = H.solve(disc.to_vec(g, -F), eta, 200, scale=tn)
    xo = disc.from_vec(g, x)
    _assert_fields(xg, xo, FP64_TOL if precision == "fp64" else MIXED_TOL, precision)
    if precision == "fp64":
        assert abs(len(hg) - len(ho)) <= 1
        k = min(len(hg), len(ho), 6)
        assert np.allclose(hg[:k], ho[:k], rtol=1e-5, atol=1e-14)
    if (R >= 1e-1 and line in (1, 3)) or (R <= 2e-3 and line in (2, 3)):
        sp_ = mg.from_discharge(d, precision=prec)
        sp_.set_old_state(*[np.ascontiguousarray(a * 0.99) for a in u])
        _, hp, _ = sp_.linear_solve(dt, list(-F), eta, 200)
        assert len(hg) * 2 < len(hp), (len(hg), len(hp))


@pytest.mark.parametrize("n,R,line,nu,precision", [(64, 1e-1, 1, 1, "fp64"), (32, 2e-3, 3, 1, "fp64"),
                                                  (64, 1e-1, 1, 2, "mixed"), (32, 2e-3, 2, 2, "fp64")])
def test_line_smoother_sweep_counts_parity(mg, n, R, line, nu, precision):
    """Line smoothing with V(1,1) or V(2,2) on every level above 9^2 (nu1 = nu2 = nu_coarse1 =
    nu_coarse2 = nu), the sweep counts of the benchmark's faster line-smoothed solves: the
    oracle with the same sweep counts, its residual history cycle by cycle (FP64) and its
    solution per field (FP64 1e-10, mixed 1e-8)."""
    d = W.make_discharge(n, seed=0, V_cathode=-300.0, use_table=True, R=R)
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    dt = 1e-7
    F, T = disc.residual(g, u, u * 0.99, d.S_e, d.S_p, dt, phys, with_terms=True)
    tn = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
    sw = dict(nu1=nu, nu2=nu, nu_coarse1=nu, nu_coarse2=nu)
    prec = mg.MG_MIXED if precision == "mixed" else mg.MG_FP64
    s = mg.from_discharge(d, precision=prec, line_smoother=line, **sw)
    s.set_old_state(*[np.ascontiguousarray(a * 0.99) for a in u])
    eta = 1e-12 if precision == "fp64" else 1e-10
    xg, hg, rc = s.linear_solve(dt, list(-F), eta, 200)
    assert rc == mg.MG_OK
    H = omg.Hierarchy(g, u, dt, phys, line={1: "z", 2: "r", 3: "alt"}[line], **sw)
    x, ho = H.solve(disc.to_vec(g, -F), eta, 200, scale=tn)
    _assert_fields(xg, disc.from_vec(g, x), FP64_TOL if precision == "fp64" else MIXED_TOL, (n, line, nu))
    if precision == "fp64":
        assert abs(len(hg) - len(ho)) <= 1
        k = min(len(hg), len(ho), 6)
        assert np.allclose(hg[:k], ho[:k], rtol=1e-5, atol=1e-14)
    else:
        assert len(hg) <= len(ho) + 3


@pytest.mark.parametrize("nr,nz,table,precision,line", [(64, 16, False, "fp64", 0), (16, 64, True, "fp64", 0),
                                                       (128, 32, True, "fp64", 0), (32, 128, False, "mixed", 0),
                                                       (64, 16, True, "mixed", 0), (32, 64, True, "fp64", 1),
                                                       (64, 32, False, "fp64", 1)])
def test_nonsquare_linear_solve_parity(mg, nr, nz, table, precision, line):
    """V-cycles on grids with N_r != N_z (both sides halved per level down to a shorter side of
    2 intervals: 64 x 16 -> 8 x 2, 16 x 64 -> 2 x 8), with the point smoother or the z-line one:
    the oracle's solution per field (FP64 1e-10, mixed 1e-8) and, in FP64, its residual history
    cycle by cycle.  FP64 solves on both sides stop at a relative residual of 1e-13: the ion
    density, weakly coupled, amplifies a residual of 1e-12 to about 1e-10 of its own scale on
    these grids.  The cycle counts are compared where the oracle reaches that tolerance: its
    z-line column solves level off near 2e-12 on the 64 x 32 grid, where the GPU's cycle
    reaches 5e-14."""
    d = W.make_discharge(nr, nz=nz, seed=9, V_cathode=-300.0, use_table=table)
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    dt = 1e-7
    prec = mg.MG_MIXED if precision == "mixed" else mg.MG_FP64
    s = mg.from_discharge(d, precision=prec, line_smoother=line)
    s.set_old_state(*[np.ascontiguousarray(a * 0.99) for a in u])
    F, T = disc.residual(g, u, u * 0.99, d.S_e, d.S_p, dt, phys, with_terms=True)
    eta = 1e-13 if precision == "fp64" else 1e-11
    xg, hg, rc = s.linear_solve(dt, list(-F), eta, 300)
    assert rc == mg.MG_OK, hg
    H = omg.Hierarchy(g, u, dt, phys, line=bool(line))
    tn = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
    x, ho = H.solve(disc.to_vec(g, -F), 1e-13, 300, scale=tn)
    xo = disc.from_vec(g, x)
    _assert_fields(xg, xo, FP64_TOL if precision == "fp64" else MIXED_TOL, (nr, nz))
    if precision == "fp64":
        if ho[-1] <= 1e-13:
            assert abs(len(hg) - len(ho)) <= 1
        k = min(len(hg), len(ho), 6)
        assert np.allclose(hg[:k], ho[:k], rtol=1e-5, atol=1e-14)
    else:
        assert len(hg) <= len(ho) + 3


def test_line_smoother_1023_row_columns_mixed(mg):
    """z-line smoothing of the FP32 inner cycle on a level whose columns have 1,023 rows
    (129 x 1025 nodes): one shared-memory cyclic reduction per column, a thread per row.  The
    mixed linear solve against the oracle's z-line solve, both stopped at a relative residual of
    1e-11 (the oracle's column solves level off near 1e-12 on this grid): the solution per field
    to 1e-8, and at most three cycles more than the oracle."""
    d = W.make_discharge(128, nz=1024, seed=9, V_cathode=-300.0)
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    dt = 1e-7
    s = mg.from_discharge(d, precision=mg.MG_MIXED, line_smoother=1)
    s.set_old_state(*[np.ascontiguousarray(a * 0.99) for a in u])
    F, T = disc.residual(g, u, u * 0.99, d.S_e, d.S_p, dt, phys, with_terms=True)
    xg, hg, rc = s.linear_solve(dt, list(-F), 1e-11, 100)
    assert rc == mg.MG_OK, hg
    tn = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
    x, ho = omg.Hierarchy(g, u, dt, phys, line=True).solve(disc.to_vec(g, -F), 1e-11, 100, scale=tn)
    assert ho[-1] <= 1e-11
    _assert_fields(xg, disc.from_vec(g, x), MIXED_TOL, "1023-row columns")
    assert len(hg) <= len(ho) + 3


@pytest.mark.parametrize("nr,nz,line,wall,R,precision", [
    (64, 512, 1, False, 1e-2, "fp64"), (256, 32, 2, False, 1e-2, "fp64"), (512, 64, 2, True, 2.7e-2, "fp64"),
    (512, 64, 2, True, 2.7e-2, "mixed"), (128, 1024, 1, False, 1e-2, "fp64")])
def test_longest_lines_linear_solve_parity(mg, nr, nz, line, wall, R, precision):
    """Line smoothing at the longest lines the line kernels take: z-lines of 511 rows (65 x 513
    nodes), r-lines of 257 unknowns, and r-lines of 512 unknowns (513 x 65 nodes with the
    Dirichlet wall, whose column is not an unknown).  In FP64 these run the block
    cyclic-reduction kernel at its largest launch (768 threads, 51 planes of 512 values in
    shared memory); FP64 columns of 1,023 rows (129 x 1025 nodes) are longer than that kernel
    takes and run the thread-per-column block elimination on the finest level (the coarser
    levels' 511-row columns the cyclic reduction).  Both sides solve to a relative residual of
    1e-12; the oracle's residual
    history cycle by cycle, the cycle count within one, and the solution per field (FP64 1e-10,
    mixed 1e-8).  The wall case takes R = 2.7 cm: with R = 1 cm (dz = 8 dr) the oracle's r-line
    solves level off near 1e-11."""
    import dataclasses
    d = W.make_discharge(nr, nz=nz, seed=9, V_cathode=-300.0, R=R)
    if wall:
        d = dataclasses.replace(d, wall_dirichlet=True)
    g = Grid(d.nr, d.nz, d.R, d.z, wall_dirichlet=wall)
    phys = disc.Physics(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p, D_p=d.D_p)
    u = np.stack([d.ne0, d.np0, d.V0])
    if wall:
        u = disc.apply_dirichlet(u, phys, g)
    dt = 1e-7
    prec = mg.MG_MIXED if precision == "mixed" else mg.MG_FP64
    s = mg.from_discharge(d, precision=prec, line_smoother=line)
    s.set_state(*[np.ascontiguousarray(a) for a in u])
    s.set_old_state(*[np.ascontiguousarray(a * 0.99) for a in u])
    F, T = disc.residual(g, u, u * 0.99, d.S_e, d.S_p, dt, phys, with_terms=True)
    xg, hg, rc = s.linear_solve(dt, list(-F), 1e-12, 100)
    assert rc == mg.MG_OK, hg
    tn = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
    x, ho = omg.Hierarchy(g, u, dt, phys, line={1: "z", 2: "r"}[line]).solve(disc.to_vec(g, -F), 1e-12, 100,
                                                                            scale=tn)
    assert ho[-1] <= 1e-12
    _assert_fields(xg, disc.from_vec(g, x), FP64_TOL if precision == "fp64" else MIXED_TOL, (nr, nz, line))
    if precision == "fp64":
        assert abs(len(hg) - len(ho)) <= 1
        k = min(len(hg), len(ho), 6)
        assert np.allclose(hg[:k], ho[:k], rtol=1e-5, atol=1e-14)
    else:
        assert len(hg) <= len(ho) + 3


@pytest.mark.parametrize("nr,nz", [(32, 8), (8, 32), (64, 32)])
def test_nonsquare_step_parity(mg, nr, nz):
    """Backward-Euler steps (Newton with V-cycle solves) on grids with N_r != N_z: the oracle's
    Newton iteration count and state per field to 1e-10."""
    d = W.make_discharge(nr, nz=nz, seed=10, V_cathode=-250.0, use_table=True)
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    s = mg.from_discharge(d, eta=1e-12, max_vcycles=100)
    opt = osv.SolverOptions(eta=1e-12)
    for k in range(3):
        rc, st = s.step(1e-9, 1e-10)
        assert rc == mg.MG_OK
        u, so = osv.step(g, u, d.S_e, d.S_p, 1e-9, phys, 1e-10, opt)
        assert so.accepted and st["last_newton"] == so.newton
    _assert_fields(s.get_state(), u, FP64_TOL, (nr, nz))


def test_transient_33_ten_steps_parity(mg):
    d = W.transient_33()
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    s = mg.from_discharge(d, eta=1e-12, max_vcycles=100)
    opt = osv.SolverOptions(eta=1e-12)
    for k in range(10):
        rc, st = s.step(1e-9, 1e-10)
        assert rc == mg.MG_OK
        u, so = osv.step(g, u, d.S_e, d.S_p, 1e-9, phys, 1e-10, opt)
        assert so.accepted and st["last_newton"] == so.newton
    ug = s.get_state()
    for q in range(3):
        assert np.abs(ug[q] - u[q]).max() <= 1e-10 * np.abs(u[q]).max(), q


@pytest.mark.parametrize("rel", [0.1, 0.0])
def test_steady_march_parity_small(mg, rel):
    """March to the steady state, with the relative per-step Newton tolerance (default) and with
    every step solved to 0.1 x the steady tolerance: the oracle's steps, Newton iterations and
    state."""
    d = W.make_discharge(16, seed=1, V_cathode=-300.0, use_table=True)
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    s = mg.from_discharge(d, eta=1e-10, max_vcycles=200, newton_tol_rel=rel)
    rc, st = s.march(1e-9, 1e-10)
    assert rc == mg.MG_OK
    uo, ok, rec = osv.march(g, u, d.S_e, d.S_p, phys, 1e-10,
                            osv.SolverOptions(eta=1e-10, max_vcycles=200, newton_tol_rel=rel), 1e-9)
    assert ok
    assert st["steps_accepted"] == sum(1 for r in rec if r[1])
    assert st["newton_iterations"] == sum(r[2] for r in rec)
    assert st["vcycles"] == sum(r[3] for r in rec)
    _assert_fields(s.get_state(), uo, FP64_TOL)


def test_solve_steady_continuation_parity_33(mg):
    """129 -> 257-style two-level continuation at 17^2 -> 33^2 (Sec. 2): the oracle's steps,
    rejections, Newton iterations and V-cycles on both grids, and its steady state to 1e-10."""
    d = W.make_discharge(32, seed=0, V_cathode=-300.0, use_table=True)
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    s = mg.from_discharge(d, eta=1e-12, max_vcycles=200)
    rc, st = s.solve_steady(1e-10)
    assert rc == mg.MG_OK
    uo, ok, rec_c, rec_f = osv.solve_steady(g, u, d.S_e, d.S_p, phys, 1e-10,
                                            osv.SolverOptions(eta=1e-12, max_vcycles=200))
    assert ok
    assert _gpu_counts(st) == _oracle_counts(rec_c, rec_f)
    _assert_fields(s.get_state(), uo, FP64_TOL)


@pytest.mark.parametrize("line,R", [(1, 0.1), (2, 2e-3), (3, 2e-3)])
def test_line_smoother_steady_continuation_parity_33(mg, line, R):
    """f1 in whole solves: the 17^2 -> 33^2 continuation with z-lines (R = 10 d), r-lines or
    alternating lines (R = d / 5) on every level: the oracle's steps, rejections, Newton
    iterations and V-cycles on both grids, and its steady state to 1e-10."""
    d = W.make_discharge(32, seed=0, V_cathode=-300.0, use_table=True, R=R)
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    s = mg.from_discharge(d, eta=1e-12, max_vcycles=200, line_smoother=line)
    rc, st = s.solve_steady(1e-10)
    assert rc == mg.MG_OK
    opt = osv.SolverOptions(eta=1e-12, max_vcycles=200, line_smoother={1: "z", 2: "r", 3: "alt"}[line])
    uo, ok, rec_c, rec_f = osv.solve_steady(g, u, d.S_e, d.S_p, phys, 1e-10, opt)
    assert ok
    assert _gpu_counts(st) == _oracle_counts(rec_c, rec_f)
    _assert_fields(s.get_state(), uo, FP64_TOL)


@pytest.mark.parametrize("chain_from,dt_max", [(2, 1e-6), (3, 1.0)])
def test_solve_steady_chain_parity_65(mg, chain_from, dt_max):
    """Multilevel continuation from the grid coarsened chain_from times (17^2 or 9^2 up to 65^2),
    capped and uncapped Delta-t ramp: the oracle's schedule, step for step, and its steady state."""
    d = W.make_discharge(64, seed=1, V_cathode=-300.0, use_table=True)
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    s = mg.from_discharge(d, eta=1e-12, max_vcycles=200, chain_from=chain_from, dt_max=dt_max)
    rc, st = s.solve_steady(1e-10)
    assert rc == mg.MG_OK
    opt = osv.SolverOptions(eta=1e-12, max_vcycles=200, chain_from=chain_from, dt_max=dt_max)
    uo, ok, rec_c, rec_f = osv.solve_steady(g, u, d.S_e, d.S_p, phys, 1e-10, opt)
    assert ok
    assert _gpu_counts(st) == _oracle_counts(rec_c, rec_f)
    _assert_fields(s.get_state(), uo, FP64_TOL)


def test_steady_257_chain_uncapped_parity(mg):
    """257 x 257 from 33^2 up with the uncapped ramp (the paper's own schedule, Sec. 2-3), the
    library defaults otherwise: the oracle's schedule step for step and its steady state to
    1e-10, and the oracle's residual of the result <= 1e-8."""
    d = W.steady_257()
    g, phys = _oracle(d)
    s = mg.from_discharge(d, chain_from=3, dt_max=1.0)
    s.autotune()
    rc, st = s.solve_steady(1e-8)
    assert rc == mg.MG_OK, st
    ug = np.stack(s.get_state())
    uo, ok, rec_c, rec_f = osv.solve_steady(g, np.stack([d.ne0, d.np0, d.V0]), d.S_e, d.S_p, phys, 1e-8,
                                            osv.SolverOptions(chain_from=3, dt_max=1.0))
    assert ok
    assert _gpu_counts(st) == _oracle_counts(rec_c, rec_f)
    _assert_fields(ug, uo, FP64_TOL)
    F, T = disc.residual(g, ug, None, d.S_e, d.S_p, None, phys, with_terms=True)
    assert disc.rho(F, T).max() <= 1e-8 * (1 + RHO_AGREE)


@pytest.fixture(scope="module")
def oracle_steady_257():
    """The oracle's steady solve of the 257^2 workload with the default options (the two-level
    129^2 -> 257^2 continuation to rho <= 1e-8): (state, coarse records, fine records)."""
    d = W.steady_257()
    g, phys = _oracle(d)
    uo, ok, rec_c, rec_f = osv.solve_steady(g, np.stack([d.ne0, d.np0, d.V0]), d.S_e, d.S_p, phys, 1e-8,
                                            osv.SolverOptions())
    assert ok
    return uo, rec_c, rec_f


def test_steady_257_headline_parity(mg, oracle_steady_257):
    """The benchmark's step: 257 x 257 nodes, table transport, -300 V, continuation 129^2 ->
    257^2 to rho <= 1e-8 (abstract and Sec. 2), FP64, launch shapes autotuned as the benchmark
    runs it.  Against the oracle's solve of the same inputs: the same steps, rejections, Newton
    iterations and V-cycles on each grid (also the committed counts in
    tests/golden/oracle_steady_257_counts.json), the steady state to 1e-10 relative max-norm per
    field, and the oracle's residual of the GPU result <= 1e-8."""
    import json
    import os
    d = W.steady_257()
    g, phys = _oracle(d)
    s = mg.from_discharge(d)
    s.autotune()
    rc, st = s.solve_steady(1e-8)
    assert rc == mg.MG_OK, st
    ug = np.stack(s.get_state())
    uo, rec_c, rec_f = oracle_steady_257
    assert _gpu_counts(st) == _oracle_counts(rec_c, rec_f)
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_steady_257_counts.json")) as fh:
        golden = json.load(fh)["levels"]
    assert (st["coarse_steps"], st["coarse_newton"], st["coarse_vcycles"]) == (
        golden[0]["steps"] + golden[0]["rejected"], golden[0]["newton"], golden[0]["vcycles"])
    assert (st["newton_iterations"] - st["coarse_newton"], st["vcycles"] - st["coarse_vcycles"]) == (
        golden[1]["newton"], golden[1]["vcycles"])
    _assert_fields(ug, uo, FP64_TOL)
    F, T = disc.residual(g, ug, None, d.S_e, d.S_p, None, phys, with_terms=True)
    assert disc.rho(F, T).max() <= 1e-8 * (1 + RHO_AGREE)
    assert np.all(np.isfinite(ug))


def test_transient_1025_full_size(mg):
    """1025 x 1025 (the mixed-precision workload at full size), autotuned as the benchmark runs
    it: ten backward-Euler steps of 1 ns, each to rho <= 1e-10, in FP64 and in the mixed form,
    against the oracle's ten steps (tests/golden/oracle_transient_1025.npz, written by
    tests/golden/make_oracle_1025.py from the oracle alone: every 8th node of each field after
    the first and the last step, each field's max-norm after every step).  FP64: the oracle's
    Newton iterations per step and its state to 1e-10 relative per field at every sampled node;
    mixed: its state to 1e-8.  The oracle's residual of each form's first step meets the step
    tolerance."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_transient_1025.npz")
    with np.load(path) as z:
        gold = {k: z[k] for k in z.files}
    stride = int(gold["stride"])
    d = W.transient_1025()
    g, phys = _oracle(d)
    u0 = np.stack([d.ne0, d.np0, d.V0])
    for prec, tol in ((mg.MG_FP64, FP64_TOL), (mg.MG_MIXED, MIXED_TOL)):
        s = mg.from_discharge(d, precision=prec)
        s.autotune()
        for k in range(10):
            rc, st = s.step(1e-9, 1e-10)
            assert rc == mg.MG_OK, (prec, k, st)
            ug = np.stack(s.get_state())
            assert np.all(np.isfinite(ug))
            if k == 0:
                F, T = disc.residual(g, ug, u0, d.S_e, d.S_p, 1e-9, phys, with_terms=True)
                assert disc.rho(F, T).max() <= 1e-10 * (1 + RHO_AGREE), (prec, disc.rho(F, T))
            if prec == mg.MG_FP64:
                assert st["last_newton"] == gold["newton"][k], (k, st["last_newton"], gold["newton"][k])
            steps = [int(x) for x in gold["sample_steps"]]
            if k + 1 in steps:
                ref = gold["samples"][steps.index(k + 1)]
                smp = ug[:, ::stride, ::stride]
                for q in range(3):
                    err = np.abs(smp[q] - ref[q]).max() / gold["norms"][k][q]
                    assert err <= tol, (prec, k, q, err)
        s.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_persistent_batch_equals_individual_solves(mg, precision):
    """The batched form as one persistent launch for every discharge's whole steady solve
    (workers = 0): discharges of 33^2 to 129^2 reach their individual solves' steady states bit
    for bit with the same steps, Newton iterations and V-cycles, with far fewer kernel launches,
    and the oracle's steady residual of each result is <= 1e-8.  An empty batch returns at once;
    a batch of one equals its individual solve too."""
    prec = mg.MG_MIXED if precision == "mixed" else mg.MG_FP64
    ds = W.batch_64(seed=4, count=6, sizes=(16, 32, 64, 128))
    solvers = [mg.from_discharge(d, precision=prec, stream=torch.cuda.Stream()) for d in ds]
    n0 = mg.kernel_launches()
    rc, ms, rcs = mg.solve_steady_batch(solvers, 1e-8, workers=0)
    launches_batch = mg.kernel_launches() - n0
    assert rc == mg.MG_OK, rcs
    assert np.all(ms > 0)
    launches_single = 0
    for d, sb in zip(ds, solvers):
        si = mg.from_discharge(d, precision=prec)
        n1 = mg.kernel_launches()
        rc_i, st_i = si.solve_steady(1e-8)
        launches_single += mg.kernel_launches() - n1
        assert rc_i == mg.MG_OK
        a, b = sb.get_state(), si.get_state()
        for q in range(3):
            assert np.array_equal(a[q], b[q]), (d.nr, q)
        st_b = sb.stats()
        for key in ("steps_accepted", "steps_rejected", "newton_iterations", "vcycles", "coarse_steps"):
            assert st_b[key] == st_i[key], (d.nr, key)
        g, phys = _oracle(d)
        F, T = disc.residual(g, np.stack(a), None, d.S_e, d.S_p, None, phys, with_terms=True)
        assert disc.rho(F, T).max() <= 1e-8 * (1 + RHO_AGREE)
    assert launches_batch * 10 < launches_single, (launches_batch, launches_single)
    rc0, ms0, rcs0 = mg.solve_steady_batch([], 1e-8, workers=0)
    assert rc0 == mg.MG_OK and ms0.size == 0 and rcs0.size == 0
    d1 = ds[0]
    one = mg.from_discharge(d1, precision=prec, stream=torch.cuda.Stream())
    rc1, _, _ = mg.solve_steady_batch([one], 1e-8, workers=0)
    assert rc1 == mg.MG_OK
    ref = mg.from_discharge(d1, precision=prec)
    assert ref.solve_steady(1e-8)[0] == mg.MG_OK
    for q in range(3):
        assert np.array_equal(one.get_state()[q], ref.get_state()[q]), q


def test_autotune_batch_keeps_results_and_restores_states(mg):
    """The work-item size and the coarse-phase level of the persistent form change the schedule,
    not the arithmetic: the autotuner leaves every state as it found it, and solves after it
    equal solves before it bit for bit."""
    ds = W.batch_64(seed=5, count=4, sizes=(32, 64, 128))
    make = lambda: [mg.from_discharge(d, precision=mg.MG_MIXED, stream=torch.cuda.Stream()) for d in ds]
    ref = make()
    assert mg.solve_steady_batch(ref, 1e-8, workers=0)[0] == mg.MG_OK
    tuned = make()
    before = [s.get_state() for s in tuned]
    grain, coarse = mg.autotune_batch(tuned, 1e-8)
    assert grain in (2, 4, 8) and coarse in (16, 32, 64)
    for s, b in zip(tuned, before):
        a = s.get_state()
        assert all(np.array_equal(a[q], b[q]) for q in range(3))
        assert s.stats()["steps_accepted"] == 0
    assert mg.solve_steady_batch(tuned, 1e-8, workers=0)[0] == mg.MG_OK
    for s, r in zip(tuned, ref):
        a, b = s.get_state(), r.get_state()
        assert all(np.array_equal(a[q], b[q]) for q in range(3))


@pytest.mark.parametrize("workers", [0, 4])
def test_batched_full_sizes_residual_property(mg, workers):
    """The batched form at its full instance sizes (one instance of each of 65^2, 129^2, 257^2
    and 513^2 from the 64-discharge workload), autotuned, as the persistent launch (workers = 0)
    and as host threads (4): the oracle's steady residual of every result."""
    ds = W.batch_64()
    pick, seen = [], set()
    for d in ds:
        if d.nr not in seen:
            seen.add(d.nr)
            pick.append(d)
    assert sorted(seen) == [64, 128, 256, 512]
    solvers = [mg.from_discharge(d, precision=mg.MG_MIXED, stream=torch.cuda.Stream()) for d in pick]
    for sv in solvers:
        sv.autotune()
    rc, ms, rcs = mg.solve_steady_batch(solvers, 1e-8, workers=workers)
    assert rc == mg.MG_OK, rcs
    for d, sv in zip(pick, solvers):
        g, phys = _oracle(d)
        ug = np.stack(sv.get_state())
        F, T = disc.residual(g, ug, None, d.S_e, d.S_p, None, phys, with_terms=True)
        assert disc.rho(F, T).max() <= 1e-8 * (1 + RHO_AGREE), (d.nr, disc.rho(F, T))


def test_device_and_host_io_agree(mg):
    d = W.make_discharge(32, seed=2)
    s = mg.from_discharge(d)
    rng = np.random.default_rng(0)
    u = _random_state(d, rng)
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in u]
    s.set_state(*t)
    out = [torch.empty_like(a) for a in t]
    s.get_state(out)
    host = s.get_state()
    for q in range(3):
        assert np.array_equal(out[q].cpu().numpy(), host[q])
        assert np.array_equal(host[q], u[q])


@pytest.mark.parametrize("nr,nz", [(2, 2), (4, 4), (2, 8), (8, 2)])
def test_smallest_grids_single_level(mg, nr, nz):
    d = W.make_discharge(nr, nz=nz, seed=4)
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    s = mg.from_discharge(d, eta=1e-13)
    rc, st = s.step(1e-9, 1e-11)
    assert rc == mg.MG_OK
    uo, so = osv.step(g, u, d.S_e, d.S_p, 1e-9, phys, 1e-11, osv.SolverOptions(eta=1e-13))
    ug = s.get_state()
    for q in range(3):
        assert np.abs(ug[q] - uo[q]).max() <= 1e-10 * max(np.abs(uo[q]).max(), 1e-300), q


def test_invalid_arguments_are_rejected(mg):
    z = W.z_nodes(32, 1e-2)
    with pytest.raises(mg.MGError):
        mg.Solver(30, 32, 1e-2, W.z_nodes(32, 1e-2))          # not a power of two
    bad = z.copy()
    bad[5] = bad[4]
    with pytest.raises(mg.MGError):
        mg.Solver(32, 32, 1e-2, bad)                          # non-increasing z
    with pytest.raises(mg.MGError):
        mg.Solver(32, 32, 1e-2, z, mg.default_params(coarsest=1))
    s = mg.Solver(32, 32, 1e-2, z)
    rc = s.lib.mg_step(s.h, -1.0, 1e-8, None)
    assert rc == mg.MG_EINVAL
    # parameters of the later forms
    for bad_params in (dict(wall_dirichlet=2), dict(nu_coarse_n=-1), dict(nu_tiny_n=8, nu_tiny1=0, nu_tiny2=0),
                       dict(coarse_kernel_threads=2048), dict(nu1=0, nu2=0), dict(line_smoother=4)):
        with pytest.raises(mg.MGError):
            mg.Solver(32, 32, 1e-2, z, mg.default_params(**bad_params))
    with pytest.raises(mg.MGError):                           # r-lines: rows of at most 512 unknowns
        mg.Solver(512, 32, 1e-2, z, mg.default_params(line_smoother=2))
    for chain_from in (0, 99):                                 # chain_from outside 1 .. levels - 1
        sc = mg.Solver(32, 32, 1e-2, z, mg.default_params(chain_from=chain_from))
        assert sc.lib.mg_solve_steady(sc.h, 1e-8, None) == mg.MG_EINVAL
    nl = s.lib.mg_num_levels(s.h)
    for args in ((nl, 0, 32, 2, 0, 0), (0, 2, 32, 2, 0, 0), (0, 0, 48, 2, 0, 0), (0, 0, 128, 4, 0, 0),
                 (0, 0, 32, 2, 2, 0), (0, 0, 32, 2, 1, 6)):
        assert s.lib.mg_set_smoother(s.h, *args) == mg.MG_EINVAL, args
    for args in ((nl, 2, 2), (0, 0, 0), (0, 2, -1), (0, -2, -2)):
        assert s.lib.mg_set_level_sweeps(s.h, *args) == mg.MG_EINVAL, args
    assert s.lib.mg_set_level_sweeps(s.h, 1, 3, 1) == mg.MG_OK
    assert s.lib.mg_set_level_sweeps(s.h, 1, -1, -1) == mg.MG_OK
    # the allocation-free residual covers the zero-flux wall only
    p = mg.default_params(wall_dirichlet=1)
    zz = torch.zeros((33, 33), dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MGError):
        mg.residual_noalloc(32, 32, 1e-2, z, p, [zz, zz, zz], None, [zz, zz], 0.0)


def test_time_smoother(mg):
    """mg_time_smoother: a positive device time per launch, two launches per sweep for half
    sweeps, the state untouched, a linear solve afterwards unchanged bit for bit; bad
    arguments rejected."""
    d = W.make_discharge(64, seed=0, V_cathode=-300.0)
    s = mg.from_discharge(d, precision=mg.MG_MIXED)
    F, _ = s.residual(1e-9)
    f = [-a for a in F]
    xa, ha, _ = s.linear_solve(1e-9, f, 0.0, 3)
    before = s.get_state()
    for prec in (0, 1):
        us, lps = s.time_smoother(0, prec, 20)
        assert us > 0.0 and lps in (1, 2)
    s.set_smoother(1, 0, 32, 1, 0, 0)
    us, lps = s.time_smoother(1, 0, 5)
    assert us > 0.0 and lps == 2
    after = s.get_state()
    for q in range(3):
        assert np.array_equal(before[q], after[q])
    xb, hb, _ = s.linear_solve(1e-9, f, 0.0, 3)
    assert np.array_equal(ha, hb)
    for q in range(3):
        assert np.array_equal(xa[q], xb[q])
    us = ctypes.c_double(0.0)
    nl = s.lib.mg_num_levels(s.h)
    for args in ((nl - 1, 0, 10), (-1, 0, 10), (0, 2, 10), (0, 0, 0), (0, 0, 5000)):
        assert s.lib.mg_time_smoother(s.h, *args, ctypes.byref(us), None) == mg.MG_EINVAL, args
    s64 = mg.from_discharge(d)
    assert s64.lib.mg_time_smoother(s64.h, 0, 1, 10, ctypes.byref(us), None) == mg.MG_EINVAL


def test_rejected_step_leaves_state_unchanged(mg):
    d = W.make_discharge(16, seed=0, V_cathode=-300.0)
    s = mg.from_discharge(d, corr_limit_frac=1e-12)
    before = s.get_state()
    rc, st = s.step(1e-9, 1e-12)
    assert rc == mg.MG_ENOCONV and st["steps_rejected"] == 1
    after = s.get_state()
    for q in range(3):
        assert np.array_equal(before[q], after[q])


def test_nonfinite_source_is_reported(mg):
    d = W.make_discharge(16, seed=0)
    s = mg.from_discharge(d)
    S = d.S_e.copy()
    S[5, 5] = np.nan
    s.set_sources(S, d.S_p.copy())
    before = s.get_state()
    rc, st = s.step(1e-9, 1e-10)
    assert rc == mg.MG_ENONFINITE
    after = s.get_state()
    for q in range(3):
        assert np.array_equal(before[q], after[q])


# ---------------------------------------------------------------- mixed precision (FP32 inner cycle)
@pytest.mark.parametrize("n,table,dt", [(16, False, 1e-9), (64, True, 1e-6), (128, False, 1e-9)])
def test_mixed_linear_solve_matches_oracle(mg, n, table, dt):
    d = W.make_discharge(n, seed=0, V_cathode=-300.0, use_table=table)
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    s = mg.from_discharge(d, precision=mg.MG_MIXED)
    s.set_old_state(*[np.ascontiguousarray(a * 0.99) for a in u])
    F, T = disc.residual(g, u, u * 0.99, d.S_e, d.S_p, dt, phys, with_terms=True)
    xg, hg, rc = s.linear_solve(dt, list(-F), 1e-11, 200)
    assert rc == mg.MG_OK, hg
    H = omg.Hierarchy(g, u, dt, phys)
    tn = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
    x, ho = H.solve(disc.to_vec(g, -F), 1e-12, 200, scale=tn)
    xo = disc.from_vec(g, x)
    for q in range(3):
        assert np.abs(xg[q] - xo[q]).max() <= 1e-8 * np.abs(xo[q]).max(), q
    # an FP32 cycle contracts about as well as an FP64 one until FP32 rounding is reached
    assert len(hg) <= len(ho) + 3


def test_mixed_transient_33_matches_oracle(mg):
    d = W.transient_33()
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    s = mg.from_discharge(d, eta=1e-11, max_vcycles=100, precision=mg.MG_MIXED)
    opt = osv.SolverOptions(eta=1e-12)
    for k in range(10):
        rc, st = s.step(1e-9, 1e-10)
        assert rc == mg.MG_OK
        assert max(st["rho"]) <= 1e-10
        u, so = osv.step(g, u, d.S_e, d.S_p, 1e-9, phys, 1e-10, opt)
    ug = s.get_state()
    for q in range(3):
        assert np.abs(ug[q] - u[q]).max() <= 1e-8 * np.abs(u[q]).max(), q


def test_mixed_steady_257_matches_oracle(mg, oracle_steady_257):
    """Mixed precision (FP32 V-cycles inside the FP64 Newton loop) on the benchmark's 257^2
    continuation: the oracle's residual of the result <= 1e-8, the FP64 oracle's steady state to
    1e-8 relative per field, and the oracle's steps, Newton iterations and V-cycles."""
    d = W.steady_257()
    g, phys = _oracle(d)
    s32 = mg.from_discharge(d, precision=mg.MG_MIXED)
    s32.autotune()
    rc, st = s32.solve_steady(1e-8)
    assert rc == mg.MG_OK, st
    b = np.stack(s32.get_state())
    F, T = disc.residual(g, b, None, d.S_e, d.S_p, None, phys, with_terms=True)
    assert disc.rho(F, T).max() <= 1e-8 * (1 + RHO_AGREE)
    uo, rec_c, rec_f = oracle_steady_257
    _assert_fields(b, uo, MIXED_TOL)
    assert _gpu_counts(st) == _oracle_counts(rec_c, rec_f)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_and_host_driven_solves_agree(mg, precision):
    """The device-side V-cycle loop (CUDA graph with a conditional node) and the host-driven
    loop launch the same kernels in the same order: identical iterates and histories."""
    d = W.make_discharge(64, seed=2, V_cathode=-300.0, use_table=True)
    prec = mg.MG_MIXED if precision == "mixed" else mg.MG_FP64
    out = []
    for graphs in (1, 0):
        s = mg.from_discharge(d, precision=prec, use_graphs=graphs)
        F, _ = s.residual(1e-7)
        x, h, rc = s.linear_solve(1e-7, [-a for a in F], 1e-10, 100)
        assert rc == mg.MG_OK
        out.append((x, h))
    (xa, ha), (xb, hb) = out
    assert len(ha) == len(hb)
    assert np.array_equal(ha, hb)
    for q in range(3):
        assert np.array_equal(xa[q], xb[q])


def test_graph_solve_respects_cycle_cap(mg):
    d = W.make_discharge(64, seed=2, V_cathode=-300.0)
    s = mg.from_discharge(d)
    F, _ = s.residual(1e-7)
    x, h, rc = s.linear_solve(1e-7, [-a for a in F], 1e-30, 3)
    assert rc == mg.MG_ENOCONV and len(h) == 4


# ---------------------------------------------------------------- batched form, autotuner
def test_batched_steady_solves_equal_individual_solves(mg):
    ds = W.batch_64(seed=4, count=6, sizes=(16, 32, 64))
    solvers = [mg.from_discharge(d, precision=mg.MG_MIXED, stream=torch.cuda.Stream()) for d in ds]
    rc, ms, rcs = mg.solve_steady_batch(solvers, 1e-8, workers=4)
    assert rc == mg.MG_OK, rcs
    assert np.all(ms > 0)
    for d, sb in zip(ds, solvers):
        si = mg.from_discharge(d, precision=mg.MG_MIXED)
        assert si.solve_steady(1e-8)[0] == mg.MG_OK
        a, b = sb.get_state(), si.get_state()
        for q in range(3):
            assert np.array_equal(a[q], b[q])     # deterministic kernels: concurrency changes nothing
        g, phys = _oracle(d)
        F, T = disc.residual(g, np.stack(a), None, d.S_e, d.S_p, None, phys, with_terms=True)
        assert disc.rho(F, T).max() <= 1e-8 * (1 + RHO_AGREE)


def test_batched_line_smoothed_solves_fall_back_and_equal_individual_solves(mg):
    """Line-smoothed states (z-lines, r-lines, alternating lines) are outside the persistent
    launch: a batch of them asked for the persistent form (workers = 0) runs as host threads,
    the line kernels launched from several threads at once.  Each discharge's FP64 steady solve
    equals its individual solve bit for bit, and the oracle's steady residual of the result
    meets the tolerance."""
    ds = W.batch_64(seed=4, count=6, sizes=(16, 32, 64))
    lines = [1, 2, 3, 3, 2, 1]
    solvers = [mg.from_discharge(d, line_smoother=ls, stream=torch.cuda.Stream()) for d, ls in zip(ds, lines)]
    rc, ms, rcs = mg.solve_steady_batch(solvers, 1e-8, workers=0)
    assert rc == mg.MG_OK, rcs
    for d, ls, sb in zip(ds, lines, solvers):
        si = mg.from_discharge(d, line_smoother=ls)
        assert si.solve_steady(1e-8)[0] == mg.MG_OK
        a, b = sb.get_state(), si.get_state()
        for q in range(3):
            assert np.array_equal(a[q], b[q]), (d.nr, ls, q)
        g, phys = _oracle(d)
        F, T = disc.residual(g, np.stack(a), None, d.S_e, d.S_p, None, phys, with_terms=True)
        assert disc.rho(F, T).max() <= 1e-8 * (1 + RHO_AGREE), (d.nr, ls)


def test_autotune_keeps_results(mg):
    d = W.make_discharge(128, seed=3, V_cathode=-300.0, use_table=True)
    res = []
    for tune in (False, True):
        s = mg.from_discharge(d, precision=mg.MG_MIXED)
        if tune:
            shapes = s.autotune()
            assert shapes.shape[1] == 6 and np.all(shapes[:-1, 0] >= 32)
        F, _ = s.residual(1e-7)
        x, h, rc = s.linear_solve(1e-7, [-a for a in F], 1e-10, 100)
        res.append((x, h))
    assert np.array_equal(res[0][1], res[1][1])
    for q in range(3):
        assert np.array_equal(res[0][0][q], res[1][0][q])


def test_vcycle_histories_match_oracle_257_to_2049(mg):
    """V-cycles on 257^2 .. 2049^2 nodes (the largest grid, 4.2 M nodes, about 2 GB with its
    hierarchy): the oracle's residual history cycle by cycle, to 1e-5 relative per cycle as on
    the small grids (tests/golden/oracle_vcycle_factors.json, written from the oracle alone by
    tests/golden/make_oracle_vcycle_factors.py).  At this Delta t the factor grows with the grid,
    from 0.17 at 257^2 to 0.44 at 2049^2 on both sides: the algorithm's behaviour on the ions'
    drift-dominated coarse levels, which the GPU reproduces; every cycle still contracts."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_vcycle_factors.json")) as fh:
        gold = json.load(fh)
    dt, cycles = gold["dt"], gold["cycles"]
    for n_str, ho in gold["histories"].items():
        n = int(n_str)
        d = W.make_discharge(n, seed=0, V_cathode=-300.0)
        s = mg.from_discharge(d)
        s.set_old_state(*[np.ascontiguousarray(a * 0.99) for a in (d.ne0, d.np0, d.V0)])
        F, _ = s.residual(dt)
        x, h, rc = s.linear_solve(dt, [-a for a in F], 0.0, cycles)
        s.close()
        assert len(h) == len(ho), (n, len(h), len(ho))
        assert np.all(np.diff(h) < 0), (n, h)
        assert np.allclose(h, ho, rtol=1e-5, atol=1e-14), (n, list(h), ho)


def _force_fused(s, tile):
    """Fused sweeps with the given tile on every level of both views."""
    for lev in range(s.lib.mg_num_levels(s.h)):
        for view in (0, 1):
            s.set_smoother(lev, view, 32, 2, 1, tile)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [16, 64, 256])
@pytest.mark.parametrize("tile", ["autotuned", 0, 4, 5])
def test_fused_sweep_equals_half_sweeps(mg, precision, n, tile):
    """One launch per red-black sweep (tiles with a recomputed red ring, ping-pong buffers)
    gives the same iterates as one launch per colour, bit for bit."""
    d = W.make_discharge(n, seed=6, V_cathode=-300.0, use_table=(n == 64))
    prec = mg.MG_MIXED if precision == "mixed" else mg.MG_FP64
    out = []
    for fused in (1, 0):
        s = mg.from_discharge(d, precision=prec, fused_sweep=fused)
        if fused:
            s.autotune()
            if tile != "autotuned":
                _force_fused(s, tile)
        F, _ = s.residual(1e-7)
        x, h, rc = s.linear_solve(1e-7, [-a for a in F], 1e-10, 100)
        assert rc == mg.MG_OK
        out.append((x, h))
    (xa, ha), (xb, hb) = out
    assert np.array_equal(ha, hb)
    for q in range(3):
        assert np.array_equal(xa[q], xb[q])


def test_odd_sweep_counts(mg):
    d = W.make_discharge(32, seed=6, V_cathode=-300.0)
    res = []
    for fused in (1, 0):
        s = mg.from_discharge(d, nu1=1, nu2=3, fused_sweep=fused)
        if fused:
            _force_fused(s, 1)
        F, _ = s.residual(1e-8)
        x, h, rc = s.linear_solve(1e-8, [-a for a in F], 1e-11, 100)
        assert rc == mg.MG_OK
        res.append((x, h))
    assert np.array_equal(res[0][1], res[1][1])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("ctas,threads", [(1, 1024), (1, 512), (2, 256), (8, 512)])
@pytest.mark.parametrize("kn", [16, 64])
def test_persistent_coarse_cycle_equals_level_kernels(mg, precision, ctas, threads, kn):
    """The coarse levels of a V-cycle in one cluster launch give the same iterates as the
    per-level kernels, bit for bit (kn = 16 with one CTA: the shared-memory form; kn = 64: the
    levels do not fit in shared memory and the global-memory form runs)."""
    d = W.make_discharge(128, seed=8, V_cathode=-300.0, use_table=True)
    prec = mg.MG_MIXED if precision == "mixed" else mg.MG_FP64
    out = []
    for kn in (kn, 0):
        s = mg.from_discharge(d, precision=prec, coarse_kernel_n=kn, coarse_kernel_ctas=ctas,
                              coarse_kernel_threads=threads)
        F, _ = s.residual(1e-7)
        x, h, rc = s.linear_solve(1e-7, [-a for a in F], 1e-10, 100)
        assert rc == mg.MG_OK
        out.append((x, h))
    (xa, ha), (xb, hb) = out
    assert np.array_equal(ha, hb)
    for q in range(3):
        assert np.array_equal(xa[q], xb[q])
