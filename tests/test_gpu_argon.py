"""GPU parity for the paper's own argon discharge (Sec. 3): Dirichlet walls (n = 0, V linear in
z on r = R), cathode at 0 V and anode at 255.9 V, the analytic sources with (a, b) = (30, 24) and
(10, 1), mu_e = 30 / p.  Oracle: oracle/ with Grid(..., wall_dirichlet=True).  The paper's ion
currents (0.59 mA and 0.035 mA) depend on an ion mobility it does not print; the stand-in here
does not reproduce them, so they are reported, not asserted."""
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
    from paper_0811_4446_gb300 import build, mg as m
    build.build()
    return m


def _oracle(d):
    g = Grid(d.nr, d.nz, d.R, d.z, wall_dirichlet=True)
    phys = disc.Physics(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p, D_p=d.D_p)
    return g, phys


def _random_state(d, g, phys, rng):
    ne = 1e14 * (0.5 + rng.random(d.shape))
    np_ = 1e14 * (0.5 + rng.random(d.shape))
    V = d.V0 + 3.0 * rng.standard_normal(d.shape)
    return disc.apply_dirichlet(np.stack([ne, np_, V]), phys, g)


@pytest.mark.parametrize("n", [16, 64])
@pytest.mark.parametrize("dt", [1e-9, 0.0])
def test_argon_residual_and_jacobian_parity(mg, n, dt):
    d = W.argon(n)
    g, phys = _oracle(d)
    rng = np.random.default_rng(5)
    u, uo = _random_state(d, g, phys, rng), _random_state(d, g, phys, rng)
    s = mg.from_discharge(d)
    s.set_state(*[np.ascontiguousarray(a) for a in u])
    s.set_old_state(*[np.ascontiguousarray(a) for a in uo])
    Fg, rho_g = s.residual(dt)
    F, T = disc.residual(g, u, uo, d.S_e, d.S_p, dt if dt > 0 else None, phys, with_terms=True)
    for f in range(3):
        assert np.abs(Fg[f] - F[f]).max() <= 1e-12 * np.abs(T[f]).max(), f
    assert np.allclose(rho_g, disc.rho(F, T), rtol=1e-9, atol=1e-300)
    v = rng.standard_normal((3,) + d.shape)
    v[0:2] *= 1e12
    Jg = s.jacobian_apply(dt, [np.ascontiguousarray(a) for a in v])
    J = disc.jacobian(g, u, dt if dt > 0 else None, phys)
    Jv = disc.from_vec(g, J @ disc.to_vec(g, v))
    scale = disc.from_vec(g, abs(J) @ np.abs(disc.to_vec(g, v)))
    for f in range(3):
        assert np.abs(Jg[f] - Jv[f]).max() <= 1e-12 * scale[f].max(), f


@pytest.mark.parametrize("n,dt", [(16, 1e-9), (64, 1e-7)])
def test_argon_linear_solve_parity(mg, n, dt):
    d = W.argon(n, a=10.0, b=1.0)
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    s = mg.from_discharge(d)
    s.set_old_state(*[np.ascontiguousarray(a * 0.99) for a in u])
    F, T = disc.residual(g, u, u * 0.99, d.S_e, d.S_p, dt, phys, with_terms=True)
    xg, hg, rc = s.linear_solve(dt, list(-F), 1e-12, 200)
    assert rc == mg.MG_OK
    H = omg.Hierarchy(g, u, dt, phys)
    tn = np.array([np.linalg.norm(T[k, 1:-1]) for k in range(3)])
    x, ho = H.solve(disc.to_vec(g, -F), 1e-12, 200, scale=tn)
    xo = disc.from_vec(g, x)
    for q in range(3):
        assert np.abs(xg[q] - xo[q]).max() <= 1e-10 * np.abs(xo[q]).max(), q
        assert np.all(xg[q][:, -1] == 0.0)
    assert abs(len(hg) - len(ho)) <= 1


@pytest.mark.parametrize("a,b", [(30.0, 24.0), (10.0, 1.0)])
def test_argon_steady_continuation_parity_33(mg, a, b):
    """The paper's argon discharge (Sec. 3), 17^2 -> 33^2 continuation with every linear solve to
    1e-12: the oracle's schedule step for step (steps, Newton iterations, V-cycles on both grids)
    and its steady state to 1e-10 relative max-norm per field."""
    d = W.argon(32, a=a, b=b)
    g, phys = _oracle(d)
    u = np.stack([d.ne0, d.np0, d.V0])
    s = mg.from_discharge(d, eta=1e-12, max_vcycles=200)
    rc, st = s.solve_steady(1e-10)
    assert rc == mg.MG_OK, st
    uo, ok, rec_c, rec_f = osv.solve_steady(g, u, d.S_e, d.S_p, phys, 1e-10,
                                            osv.SolverOptions(eta=1e-12, max_vcycles=200))
    assert ok
    rr = rec_c + rec_f
    assert (st["coarse_steps"], st["steps_accepted"] + st["steps_rejected"], st["newton_iterations"],
            st["vcycles"]) == (len(rec_c), len(rr), sum(r[2] for r in rr), sum(r[3] for r in rr))
    ug = s.get_state()
    for q in range(3):
        assert np.abs(ug[q] - uo[q]).max() <= 1e-10 * np.abs(uo[q]).max(), q
    assert np.all(ug[0][:, -1] == 0.0) and np.all(ug[1][:, -1] == 0.0)


def _cathode_ion_current(g, u, phys):
    """Ion current into the cathode (A): the Scharfetter-Gummel ion flux through the first row
    of z-faces (per radian, from row 0 to row 1) times -2 pi e."""
    _, (mez, dez, mpz, dpz) = disc.face_transport(g, u[2], phys)
    phi = disc.sg_flux(g.gz[0], mpz[0], dpz[0], 1.0, u[1][0], u[1][1], u[2][0], u[2][1])
    return -2.0 * np.pi * 1.602176634e-19 * phi.sum()


@pytest.mark.parametrize("a,b", [(30.0, 24.0), (10.0, 1.0)])
def test_argon_257_steady_parity(mg, a, b):
    """257 x 257 argon discharge, two-level continuation to rho <= 1e-8: the oracle's schedule
    step for step, its steady state to 1e-10 relative per field, and the oracle's residual of
    the result <= 1e-8 (GPU and oracle evaluate rho of one state to 1e-9 relative)."""
    d = W.argon(256, a=a, b=b)
    g, phys = _oracle(d)
    s = mg.from_discharge(d)
    rc, st = s.solve_steady(1e-8)
    assert rc == mg.MG_OK, st
    ug = np.stack(s.get_state())
    assert np.all(np.isfinite(ug))
    F, T = disc.residual(g, ug, None, d.S_e, d.S_p, None, phys, with_terms=True)
    assert disc.rho(F, T).max() <= 1e-8 * (1 + 1e-9)
    uo, ok, rec_c, rec_f = osv.solve_steady(g, np.stack([d.ne0, d.np0, d.V0]), d.S_e, d.S_p, phys, 1e-8,
                                            osv.SolverOptions())
    assert ok
    rr = rec_c + rec_f
    assert (st["coarse_steps"], st["steps_accepted"] + st["steps_rejected"], st["newton_iterations"],
            st["vcycles"]) == (len(rec_c), len(rr), sum(r[2] for r in rr), sum(r[3] for r in rr))
    for q in range(3):
        assert np.abs(ug[q] - uo[q]).max() <= 1e-10 * np.abs(uo[q]).max(), q
    print(f"argon a={a} b={b}: {st['steps_accepted']} steps, {st['newton_iterations']} Newton, "
          f"{st['vcycles']} V-cycles, max n_e {ug[0].max():.3e}, max n_p {ug[1].max():.3e}, "
          f"ion current to the cathode {_cathode_ion_current(g, ug, phys) * 1e3:.4f} mA")
