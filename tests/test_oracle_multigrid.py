"""Pins for the oracle's multigrid solver of eq. 14 and the transfer operators.

* the V-cycle solution equals a dense direct solve of the same (equilibrated)
  Jacobian on small grids (up to 33 x 33 nodes);
* the prolongation reproduces functions bilinear in (r, z) exactly (it is the
  interpolation it claims to be), and R = P^T;
* the V-cycle convergence factor does not grow with the grid in the transient
  regime (the O(N) property Sec. 2 relies on).
"""
import numpy as np
import pytest

import workloads as W
from oracle import discretization as disc
from oracle import multigrid as mg
from oracle.grid import Grid


def _dense_reference(J, f):
    """Equilibrated dense solve (columns then rows scaled to unit max-abs entry)."""
    Jd = J.toarray()
    c = 1.0 / np.abs(Jd).max(axis=0)
    Jd = Jd * c
    r = 1.0 / np.abs(Jd).max(axis=1)
    return c * np.linalg.solve(Jd * r[:, None], r * f)


def _problem(n, dt=1e-9, table=False, V_c=-200.0, seed=0):
    d = W.make_discharge(n, seed=seed, V_cathode=V_c, use_table=table)
    g = Grid(d.nr, d.nz, d.R, d.z)
    phys = disc.Physics(V_cathode=d.V_cathode, table=d.table)
    u = np.stack([d.ne0, d.np0, d.V0])
    F, T = disc.residual(g, u, u * 0.99, d.S_e, d.S_p, dt, phys, with_terms=True)
    return g, phys, u, F, T


@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_vcycle_solution_matches_sparse_lu(n):
    g, phys, u, F, T = _problem(n)
    H = mg.Hierarchy(g, u, 1e-9, phys)
    f = -disc.to_vec(g, F)
    scale = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
    x, hist = H.solve(f, 1e-13, 60, scale=scale)
    xd = _dense_reference(H.levels[0].J, f)
    for k in range(3):
        assert np.abs(x[k::3] - xd[k::3]).max() <= 1e-9 * np.abs(xd[k::3]).max(), k


@pytest.mark.parametrize("dt", [1e-9, 1e-7])
def test_vcycle_with_table_transport_matches_sparse_lu(dt):
    g, phys, u, F, T = _problem(16, dt=dt, table=True, V_c=-300.0)
    H = mg.Hierarchy(g, u, dt, phys)
    f = -disc.to_vec(g, F)
    scale = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
    x, hist = H.solve(f, 1e-13, 100, scale=scale)
    xd = _dense_reference(H.levels[0].J, f)
    for k in range(3):
        assert np.abs(x[k::3] - xd[k::3]).max() <= 1e-9 * np.abs(xd[k::3]).max(), k


def test_prolongation_is_exact_on_bilinear_functions():
    gf = Grid(16, 16, 1e-2, W.z_nodes(16, 1e-2))
    gc = gf.coarse()
    P = mg.prolongation(gf, gc)
    f = lambda r, z: 2.0 + 3.0 * r / 1e-2 - 1.5 * z / 1e-2 + 4.0 * r * z / 1e-4
    rc, zc = np.meshgrid(gc.r, gc.z)
    rf, zf = np.meshgrid(gf.r, gf.z)
    # electrode rows are Dirichlet (zero correction): use a function vanishing there
    w = lambda r, z: f(r, z) * z * (1e-2 - z) / 1e-4
    vc = np.stack([w(rc, zc)] * 3)
    xf = P @ disc.to_vec(gc, vc)
    # the product with the z-bubble is not bilinear, so check the pure bilinear part on interior
    # rows adjacent to even rows only through linearity of P: P(a f + b g) = a Pf + b Pg
    vc1 = np.stack([f(rc, zc)] * 3)
    vc1[:, 0, :] = 0.0
    vc1[:, -1, :] = 0.0
    x1 = disc.from_vec(gf, P @ disc.to_vec(gc, vc1))
    ref = f(rf, zf)
    inner = np.zeros(gf.shape, bool)
    inner[2:-2, :] = True              # rows not interpolating toward an electrode node
    for k in range(3):
        assert np.allclose(x1[k][inner], ref[inner], rtol=1e-13, atol=1e-13)
    assert np.all(np.isfinite(xf))


def test_restriction_is_prolongation_transpose():
    gf = Grid(8, 8, 1e-2, W.z_nodes(8, 1e-2))
    gc = gf.coarse()
    P = mg.prolongation(gf, gc)
    rng = np.random.default_rng(1)
    a = rng.standard_normal(P.shape[1])
    b = rng.standard_normal(P.shape[0])
    # <P a, b> = <a, P^T b>: the restriction used in the V-cycle is P.T
    assert np.isclose((P @ a) @ b, a @ (P.T @ b), rtol=1e-13)
    # column sums on a uniform grid: an interior coarse node collects weight 4 (cell-area ratio)
    gu = Grid(8, 8, 1e-2, W.z_nodes(8, 1e-2, ratio_ref=1.0))
    cs = np.asarray(mg.prolongation(gu, gu.coarse()).sum(axis=0)).ravel()
    idc = gu.coarse().node_index()
    k = idc[2, 2]
    assert np.isclose(cs[3 * k], 4.0, rtol=1e-12)


def _factor(n, dt):
    g, phys, u, F, T = _problem(n, dt=dt)
    H = mg.Hierarchy(g, u, dt, phys)
    scale = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
    _, hist = H.solve(-disc.to_vec(g, F), 1e-10, 30, scale=scale)
    steps = hist[1:] / hist[:-1]
    return np.exp(np.mean(np.log(steps[1:])))


def test_vcycle_factor_independent_of_grid_size():
    facs = [_factor(n, 1e-9) for n in (16, 32, 64, 128)]
    assert max(facs) < 0.15, facs
    assert facs[-1] < 2.0 * facs[1] + 0.02, facs


@pytest.mark.parametrize("n", [8, 16])
def test_vcycle_with_dirichlet_wall_matches_dense_solve(n):
    """The argon case's boundary (Sec. 3): Dirichlet wall; the V-cycle still converges to the
    equilibrated dense solution of the smaller unknown set."""
    d = W.argon(n, a=30.0, b=24.0)
    g = Grid(d.nr, d.nz, d.R, d.z, wall_dirichlet=True)
    phys = disc.Physics(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p, D_p=d.D_p)
    u = np.stack([d.ne0, d.np0, d.V0])
    F, T = disc.residual(g, u, u * 0.99, d.S_e, d.S_p, 1e-9, phys, with_terms=True)
    H = mg.Hierarchy(g, u, 1e-9, phys)
    f = -disc.to_vec(g, F)
    scale = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
    x, hist = H.solve(f, 1e-13, 80, scale=scale)
    xd = _dense_reference(H.levels[0].J, f)
    for k in range(3):
        assert np.abs(x[k::3] - xd[k::3]).max() <= 1e-9 * np.abs(xd[k::3]).max(), k


def _line_case(R, n=32):
    d = W.make_discharge(n, seed=0, V_cathode=-300.0, R=R)
    g = Grid(d.nr, d.nz, d.R, d.z)
    phys = disc.Physics(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p, D_p=d.D_p)
    u = np.stack([d.ne0, d.np0, d.V0])
    F, T = disc.residual(g, u, 0.99 * u, d.S_e, d.S_p, 1e-7, phys, with_terms=True)
    tn = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
    return g, u, phys, -disc.to_vec(g, F), tn


def test_line_half_sweep_solves_its_columns():
    """f1: a zebra half sweep leaves zero residual (to rounding) in every row of the columns of
    its parity, whatever the other columns hold: each column's block-tridiagonal system is
    solved exactly."""
    g, u, phys, f, tn = _line_case(1e-2)
    lev = mg.Level(g, u, 1e-7, phys, line=True)
    rng = np.random.default_rng(0)
    for c in (0, 1):
        x = rng.standard_normal(f.shape) * np.tile([1e12, 1e12, 1.0], len(f) // 3)
        U, O, lu, JUO = lev.lines[c]
        x[U] = lu.solve(f[U] - JUO @ x[O])
        r = f - lev.J @ x
        sc = abs(lev.J) @ np.abs(x) + np.abs(f)
        assert np.abs(r[U]).max() <= 1e-13 * sc[U].max(), c
        assert np.abs(r[O]).max() > 1e-3 * sc[O].max()
    # the two parities together cover every unknown once
    assert sorted(np.concatenate([lev.lines[0][0], lev.lines[1][0]])) == list(range(len(f)))


@pytest.mark.parametrize("R", [1e-2, 1e-1])
def test_line_smoother_converges_and_resists_anisotropy(R):
    """f1: V-cycles with the z-line smoother converge to the same solution as the point
    smoother; with dr = 10 dz (R = 10 d, strong z-coupling) their convergence factor stays
    below 0.05 while the point smoother's rises above 0.2 (and above ten times the line one's)."""
    g, u, phys, f, tn = _line_case(R)
    res = {}
    for line in (False, True):
        H = mg.Hierarchy(g, u, 1e-7, phys, line=line)
        x, hist = H.solve(f, 1e-12, 100, scale=tn)
        assert hist[-1] <= (1e-12 if line else 1e-10)   # the point smoother stalls at rounding level
        fac = (hist[min(6, len(hist) - 1)] / hist[1]) ** (1.0 / (min(6, len(hist) - 1) - 1))
        res[line] = (x, fac)
    xp, xl = res[False][0], res[True][0]
    for k in range(3):
        assert np.abs(xl[k::3] - xp[k::3]).max() <= 1e-7 * np.abs(xp[k::3]).max(), k
    assert res[True][1] < 0.05
    if R >= 1e-1:
        assert res[False][1] > 0.2 and res[False][1] > 10 * res[True][1]


def test_rline_half_sweep_solves_its_rows():
    """f1, r-lines: a zebra half sweep leaves zero residual (to rounding) in every unknown of the
    rows of its parity, whatever the other rows hold (each row's block-tridiagonal system along
    r solved exactly); the two parities together cover every unknown once; alternating lines
    run the z-line half sweeps, then the r-line ones."""
    g, u, phys, f, tn = _line_case(1e-3)
    lev = mg.Level(g, u, 1e-7, phys, line="r")
    rng = np.random.default_rng(1)
    for c in (0, 1):
        x = rng.standard_normal(f.shape) * np.tile([1e12, 1e12, 1.0], len(f) // 3)
        U, O, lu, JUO = lev.lines[c]
        x[U] = lu.solve(f[U] - JUO @ x[O])
        r = f - lev.J @ x
        sc = abs(lev.J) @ np.abs(x) + np.abs(f)
        assert np.abs(r[U]).max() <= 1e-13 * sc[U].max(), c
        assert np.abs(r[O]).max() > 1e-3 * sc[O].max()
        # the rows of parity c: unknowns of the rows j with j % 2 == c (j from the cathode row 0)
        rows = (U[::3] // 3) // g.ni + 1
        assert np.all(rows % 2 == c)
    assert sorted(np.concatenate([lev.lines[0][0], lev.lines[1][0]])) == list(range(len(f)))
    alt = mg.Level(g, u, 1e-7, phys, line="alt")
    zl = mg.Level(g, u, 1e-7, phys, line=True)
    assert len(alt.lines) == 4
    for q in range(2):
        assert np.array_equal(alt.lines[q][0], zl.lines[q][0])
        assert np.array_equal(alt.lines[2 + q][0], lev.lines[q][0])


@pytest.mark.parametrize("R", [1e-3, 1e-1])
def test_line_directions_resist_anisotropy_along_their_lines(R):
    """f1: smoothing along the strongly coupled direction.  With dr = dz / 10 (R = d / 10: the
    r-faces couple 100 times more strongly) r-lines and alternating lines converge with a factor
    below 0.2 while point and z-line smoothing stall above 0.5; with dr = 10 dz (R = 10 d) z-lines
    and alternating lines stay below 0.05 while point and r-line smoothing exceed 0.2.  Every
    smoother that reaches the tolerance reaches the alternating lines' solution."""
    g, u, phys, f, tn = _line_case(R)
    res = {}
    for line in (False, "z", "r", "alt"):
        H = mg.Hierarchy(g, u, 1e-7, phys, line=line)
        x, hist = H.solve(f, 1e-11, 150, scale=tn)
        fac = (hist[min(6, len(hist) - 1)] / hist[1]) ** (1.0 / (min(6, len(hist) - 1) - 1))
        res[line] = (x, fac, hist[-1] <= 1e-11)
    if R < 1e-2:
        good, bad, good_max, bad_min = ("r", "alt"), (False, "z"), 0.2, 0.5
    else:
        good, bad, good_max, bad_min = ("z", "alt"), (False, "r"), 0.05, 0.2
    for line in good:
        assert res[line][2] and res[line][1] < good_max, (line, res[line][1])
    for line in bad:
        assert res[line][1] > bad_min, (line, res[line][1])
    xa = res["alt"][0]
    for line in (False, "z", "r"):
        if res[line][2]:
            for k in range(3):
                assert np.abs(res[line][0][k::3] - xa[k::3]).max() <= 1e-6 * np.abs(xa[k::3]).max(), (line, k)
