"""Pins for the discrete fluxes, residual and Jacobian of the oracle (eqs. 3-14).

Each check compares against something fixed by the paper or by mathematics,
not against a retyped copy of the oracle's own formula:
* SG flux: exact for 1-D constant-field constant-flux drift-diffusion, and its
  alpha -> 0 limit is the central drift-diffusion flux of eqs. 3-4 (this fixes
  the G/F pairing of eq. 9, printed there as G/G);
* Poisson rows divided by A/dr^2 reproduce the printed coefficients of eq. 12
  (interior) and eq. 13 (axis);
* the flux divergence telescopes: summed over all rows it equals the net flux
  through the electrode faces (discrete charge balance / Gauss law);
* the Jacobian matches central finite differences of the residual;
* manufactured cylindrical Poisson solution converges at second order.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import bernoulli as bn
from oracle import discretization as disc
from oracle.grid import Grid


def _grid(n, nz=None, ratio=1.05):
    nz = n if nz is None else nz
    return Grid(n, nz, 1e-2, W.z_nodes(nz, 1e-2, ratio_ref=ratio))


# ---------------------------------------------------------------- SG flux (eqs. 8-11)
@pytest.mark.parametrize("s", [-1.0, 1.0])
@pytest.mark.parametrize("E", [-3e4, -50.0, 1e-3, 2e2, 5e5])
def test_sg_flux_exact_for_constant_field(s, E):
    # phi = s mu E n - D dn/dx = phi0 has n(x) = phi0/(s mu E) + C exp(s mu E x / D)
    mu, D, h, phi0, C = 0.15, 0.0038, 3e-5, 2.5e18, 4e13
    k = s * mu * E / D
    n = lambda x: phi0 / (s * mu * E) + C * np.exp(k * x)
    VL, VR = 0.0, -E * h            # E = -(V_R - V_L)/h
    got = disc.sg_flux(1.0 / h, mu, D, s, n(0.0), n(h), VL, VR)
    assert abs(got - phi0) <= 1e-9 * abs(phi0) + 1e-12 * abs(C * D / h * max(1, np.exp(k * h))), (got, phi0)


@pytest.mark.parametrize("s", [-1.0, 1.0])
def test_sg_flux_small_alpha_limit_is_central_drift_diffusion(s):
    mu, D, h = 30.0, 60.0, 1e-4
    nL, nR = 3e15, 1e15
    errs = []
    for dV in (1e-2, 5e-3, 2.5e-3, 1.25e-3):
        VL, VR = 0.0, dV
        E = -(VR - VL) / h
        central = s * mu * E * 0.5 * (nL + nR) - D * (nR - nL) / h      # eqs. 3-4
        sg = disc.sg_flux(1.0 / h, mu, D, s, nL, nR, VL, VR)
        errs.append(abs(sg - central) / abs(central))
        # the printed G/G pairing carries no drift: for uniform n it gives zero flux
        a = -s * (mu / D) * (VR - VL)
        nu = 2e15
        gg = (D / h) * (nu * bn.G(np.array([a]))[0] - nu * bn.G(np.array([a]))[0])
        drift = s * mu * E * nu
        assert gg == 0.0 and abs(drift) > 0
        assert np.isclose(disc.sg_flux(1.0 / h, mu, D, s, nu, nu, VL, VR), drift, rtol=1e-12)
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 3.5) and np.all(ratios < 4.5), errs    # O(alpha^2)


# ---------------------------------------------------------------- Poisson rows (eqs. 12-13)
def test_poisson_rows_reproduce_eq12_and_eq13():
    g = _grid(8)
    u = np.zeros((3,) + g.shape)
    J = disc.jacobian(g, u, None, disc.Physics()).toarray()
    idx = g.node_index()
    kap = disc.E_CHARGE / disc.EPS0
    dr, dz = g.dr, g.dz
    for j in range(1, g.nz):
        dzm, dzp = dz[j - 1], dz[j]
        dzc = 0.5 * (dzm + dzp)          # the control width written delta z_{j-1/2} in eq. 12
        for i in range(0, g.nr):         # the outer wall row is the half cell (not in eq. 12)
            row = 3 * idx[j, i] + 2
            scale = g.A[j, i] / dr ** 2
            c = lambda jj, ii, f=2: J[row, 3 * idx[jj, ii] + f] / scale if idx[jj, ii] >= 0 else None
            zc = dr ** 2 * (dzm + dzp) / (dzc * dzm * dzp)
            if i == 0:     # eq. 13
                assert np.isclose(c(j, 0), -4.0 - zc, rtol=1e-13)
                assert np.isclose(c(j, 1), 4.0, rtol=1e-13)
            else:          # eq. 12
                assert np.isclose(c(j, i), -2.0 - zc, rtol=1e-13)
                assert np.isclose(c(j, i - 1), 1.0 - 1.0 / (2 * i), rtol=1e-13)
                assert np.isclose(c(j, i + 1), 1.0 + 1.0 / (2 * i), rtol=1e-13)
            if j > 1:
                assert np.isclose(c(j - 1, i), dr ** 2 / (dzc * dzm), rtol=1e-13)
            if j < g.nz - 1:
                assert np.isclose(c(j + 1, i), dr ** 2 / (dzc * dzp), rtol=1e-13)
            assert np.isclose(c(j, i, 0), -kap * dr ** 2, rtol=1e-13)
            assert np.isclose(c(j, i, 1), kap * dr ** 2, rtol=1e-13)


def _mms_error(n):
    R = d = 1e-2
    g = _grid(n)
    rr, zz = np.meshgrid(g.r, g.z)
    Vex = np.sin(np.pi * zz / d) * (1 - rr ** 2 / R ** 2) ** 2
    lap = np.sin(np.pi * zz / d) * (-8 / R ** 2 + 16 * rr ** 2 / R ** 4) \
        - (np.pi / d) ** 2 * Vex
    phys = disc.Physics(V_cathode=0.0, V_anode=0.0, mu_e=0.0, mu_p=0.0)
    u = np.zeros((3,) + g.shape)
    u[1] = -lap / disc.KAPPA                    # kappa (n_p - n_e) = -lap V
    F = disc.residual(g, u, None, 0 * rr, 0 * rr, None, phys)
    J = disc.jacobian(g, u, None, phys)
    Jvv = J[2::3, 2::3]
    V = spla.spsolve(Jvv.tocsc(), -disc.to_vec(g, F)[2::3])
    Vh = np.zeros(g.shape)
    Vh[1:-1] = V.reshape(g.nz - 1, g.nr + 1)
    return np.abs(Vh - Vex).max()


def test_manufactured_cylindrical_poisson_second_order():
    errs = [_mms_error(n) for n in (16, 32, 64, 128)]
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 3.5) and np.all(ratios < 4.6), (errs, ratios)


# ---------------------------------------------------------------- conservation
def _random_state(g, rng, V_c=-200.0):
    u = np.zeros((3,) + g.shape)
    u[0] = 1e14 * (1 + rng.random(g.shape))
    u[1] = 1e14 * (1 + rng.random(g.shape))
    rr, zz = np.meshgrid(g.r, g.z)
    u[2] = V_c * (1 - zz / g.z[-1]) + 5 * rng.standard_normal(g.shape)
    return disc.apply_dirichlet(u, disc.Physics(V_cathode=V_c))


@pytest.mark.parametrize("table", [False, True])
def test_flux_divergence_telescopes_to_electrode_flux(table):
    rng = np.random.default_rng(7)
    g = _grid(16, 32)
    phys = disc.Physics(table=W.transport_table(2) if table else None, pressure_factor=1.3)
    u = _random_state(g, rng)
    S = 1e20 * rng.random(g.shape)
    zero = np.zeros(g.shape)
    F = disc.residual(g, u, None, S, S, None, phys)
    (mer, der, mpr, dpr), (mez, dez, mpz, dpz) = disc.face_transport(g, u[2], phys)
    for fi, s, mu, D in ((0, -1.0, mez, dez), (1, 1.0, mpz, dpz)):
        n, V = u[fi], u[2]
        # flux leaving through the cathode face (j = 1/2, outward = toward -z) and the anode face
        cath = disc.sg_flux(g.gz[0], mu[0], D[0], s, n[0], n[1], V[0], V[1])
        anod = disc.sg_flux(g.gz[-1], mu[-1], D[-1], s, n[-2], n[-1], V[-2], V[-1])
        net_out = anod.sum() - cath.sum()
        lhs = (F[fi, 1:-1] + g.A[1:-1] * S[1:-1]).sum()
        assert np.isclose(lhs, net_out, rtol=1e-10, atol=1e-12 * np.abs(F[fi]).sum()), (lhs, net_out)
    # discrete Gauss law: sum of Poisson rows = electrode-face field flux + enclosed charge
    V = u[2]
    gauss = (g.gz[-1] * (V[-1] - V[-2])).sum() - (g.gz[0] * (V[1] - V[0])).sum()
    charge = (g.A[1:-1] * disc.KAPPA * (u[1, 1:-1] - u[0, 1:-1])).sum()
    assert np.isclose(F[2, 1:-1].sum(), gauss + charge, rtol=1e-10)
    del zero


def test_time_term_volume_weighting():
    # uniform change of n with no flux change: F = A dn/dt summed = total volume * dn/dt
    g = _grid(8)
    u = np.zeros((3,) + g.shape)
    u_old = u.copy()
    u[0, 1:-1] = 2.0
    phys = disc.Physics(mu_e=0.0, D_e=1e-300, mu_p=0.0, D_p=1e-300, V_cathode=0.0)
    F = disc.residual(g, u, u_old, 0 * u[0], 0 * u[0], 0.5, phys)
    vol_rows = np.pi * g.R ** 2 / (2 * np.pi) * (g.z[-1] - g.z[0] - 0.5 * (g.dz[0] + g.dz[-1]))
    assert np.isclose(F[0, 1:-1].sum(), 4.0 * vol_rows, rtol=1e-12)


# ---------------------------------------------------------------- Jacobian
@pytest.mark.parametrize("dt", [1e-9, None])
def test_jacobian_matches_finite_differences(dt):
    rng = np.random.default_rng(3)
    g = _grid(8)
    phys = disc.Physics()
    u = _random_state(g, rng)
    u_old = _random_state(g, rng)
    S = 1e20 * rng.random(g.shape)
    J = disc.jacobian(g, u, dt, phys)
    F0 = lambda x: disc.to_vec(g, disc.residual(g, x, u_old, S, S, dt, phys))
    for _ in range(4):
        v = disc.from_vec(g, rng.standard_normal(3 * g.n_nodes_unknown))
        v[0:2] *= 1e12
        eps = 1e-4
        fd = (F0(u + eps * v) - F0(u - eps * v)) / (2 * eps)
        jv = J @ disc.to_vec(g, v)
        for f in range(3):
            a, b = fd[f::3], jv[f::3]
            assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b), (f, np.linalg.norm(a - b), np.linalg.norm(b))


def test_block_structure_of_eq14():
    # 3x3 diagonal block has 7 structural nonzeros, off-diagonal blocks 5 (eq. 14)
    rng = np.random.default_rng(5)
    g = _grid(8)
    J = disc.jacobian(g, _random_state(g, rng), 1e-9, disc.Physics()).toarray()
    k = g.node_index()[4, 4]
    kn = g.node_index()[4, 5]
    diag = J[3 * k:3 * k + 3, 3 * k:3 * k + 3]
    off = J[3 * k:3 * k + 3, 3 * kn:3 * kn + 3]
    assert (diag != 0).sum() == 7 and diag[0, 1] == 0 and diag[1, 0] == 0
    assert (off != 0).sum() == 5 and off[2, 0] == 0 and off[2, 1] == 0


# ---------------------------------------------------------------- Dirichlet wall (Sec. 3)
def _wall_grid(n):
    return Grid(n, n, 1e-2, W.z_nodes(n, 1e-2), wall_dirichlet=True)


def test_dirichlet_wall_values_and_unknowns():
    """The argon case's wall (Sec. 3): n_e = n_p = 0 and V linear in z along r = R; the wall
    column carries no unknowns and no residual rows."""
    g = _wall_grid(8)
    phys = disc.Physics(V_cathode=0.0, V_anode=255.9)
    u = disc.apply_dirichlet(np.ones((3,) + g.shape), phys, g)
    assert np.all(u[0:2, :, -1] == 0.0)
    assert np.allclose(u[2, :, -1], 255.9 * (g.z - g.z[0]) / (g.z[-1] - g.z[0]), rtol=1e-15, atol=0)
    assert g.n_nodes_unknown == (g.nz - 1) * g.nr and (g.node_index()[:, -1] == -1).all()
    F = disc.residual(g, u, None, np.ones(g.shape), np.ones(g.shape), None, phys)
    assert np.all(F[:, :, -1] == 0.0)
    x = np.arange(3.0 * g.n_nodes_unknown)
    assert np.array_equal(disc.to_vec(g, disc.from_vec(g, x)), x)


def test_flux_divergence_telescopes_with_dirichlet_wall():
    """Summed over the unknown rows the flux divergence equals the flux through the electrode
    faces of the unknown columns plus the flux into the wall."""
    rng = np.random.default_rng(11)
    g = _wall_grid(16)
    phys = disc.Physics(V_cathode=0.0, V_anode=255.9)
    u = _random_state(g, rng, V_c=-255.9)
    u = disc.apply_dirichlet(u, phys, g)
    S = 1e20 * rng.random(g.shape)
    F = disc.residual(g, u, None, S, S, None, phys)
    (mer, der, mpr, dpr), (mez, dez, mpz, dpz) = disc.face_transport(g, u[2], phys)
    ni = g.ni
    for fi, s, (mr, dr_), (mz, dz_) in ((0, -1.0, (mer, der), (mez, dez)), (1, 1.0, (mpr, dpr), (mpz, dpz))):
        n, V = u[fi], u[2]
        cath = disc.sg_flux(g.gz[0, :ni], mz[0, :ni], dz_[0, :ni], s, n[0, :ni], n[1, :ni], V[0, :ni], V[1, :ni])
        anod = disc.sg_flux(g.gz[-1, :ni], mz[-1, :ni], dz_[-1, :ni], s, n[-2, :ni], n[-1, :ni], V[-2, :ni],
                            V[-1, :ni])
        wall = disc.sg_flux(g.gr[1:-1, -1], mr[1:-1, -1], dr_[1:-1, -1], s, n[1:-1, -2], n[1:-1, -1], V[1:-1, -2],
                            V[1:-1, -1])
        net_out = anod.sum() - cath.sum() + wall.sum()
        lhs = (F[fi, 1:-1, :ni] + g.A[1:-1, :ni] * S[1:-1, :ni]).sum()
        assert np.isclose(lhs, net_out, rtol=1e-10, atol=1e-12 * np.abs(F[fi]).sum()), (lhs, net_out)


@pytest.mark.parametrize("dt", [1e-9, None])
def test_jacobian_matches_finite_differences_dirichlet_wall(dt):
    rng = np.random.default_rng(4)
    g = _wall_grid(8)
    phys = disc.Physics(V_cathode=0.0, V_anode=255.9)
    u = disc.apply_dirichlet(_random_state(g, rng), phys, g)
    u_old = disc.apply_dirichlet(_random_state(g, rng), phys, g)
    S = 1e20 * rng.random(g.shape)
    J = disc.jacobian(g, u, dt, phys)
    assert J.shape == (3 * g.n_nodes_unknown,) * 2
    F0 = lambda x: disc.to_vec(g, disc.residual(g, x, u_old, S, S, dt, phys))
    for _ in range(4):
        v = disc.from_vec(g, rng.standard_normal(3 * g.n_nodes_unknown))
        v[0:2] *= 1e12
        eps = 1e-4
        fd = (F0(u + eps * v) - F0(u - eps * v)) / (2 * eps)
        jv = J @ disc.to_vec(g, v)
        for f in range(3):
            a, b = fd[f::3], jv[f::3]
            assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b), (f, np.linalg.norm(a - b), np.linalg.norm(b))


def _table_problem(seed=3):
    d = W.make_discharge(16, seed=1, V_cathode=-300.0, use_table=True)
    g = Grid(d.nr, d.nz, d.R, d.z)
    phys = disc.Physics(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p,
                        D_p=d.D_p, table=d.table, pressure_factor=d.pressure_factor)
    rng = np.random.default_rng(seed)
    u = np.stack([d.ne0 * (1 + 0.3 * rng.random(d.shape)), d.np0 * (1 + 0.3 * rng.random(d.shape)),
                  d.V0 + 5 * rng.standard_normal(d.shape)])
    return d, g, phys, disc.apply_dirichlet(u, phys, g), rng


def test_full_jacobian_matches_finite_differences():
    """f4: the full Jacobian (mu, D functions of |E|) is the residual's derivative: central
    differences of the residual along a random direction agree with J_P x + transport_jv to
    1e-8 of the row scale, while the Picard Jacobian alone misses the electron rows by > 1 %."""
    d, g, phys, u, rng = _table_problem()
    uo = 0.99 * u
    x = rng.standard_normal(3 * g.n_nodes_unknown)
    x[0::3] *= 1e12
    x[1::3] *= 1e12
    w = disc.from_vec(g, x)
    J = disc.jacobian(g, u, 1e-9, phys)
    jf = disc.jacobian_full_apply(g, u, 1e-9, phys, x, J)
    h = 1e-4
    Fp = disc.residual(g, u + h * w, uo, d.S_e, d.S_p, 1e-9, phys)
    Fm = disc.residual(g, u - h * w, uo, d.S_e, d.S_p, 1e-9, phys)
    fd = disc.to_vec(g, (Fp - Fm) / (2 * h))
    scale = abs(J) @ np.abs(x)
    for k in range(3):
        assert np.abs(fd[k::3] - jf[k::3]).max() <= 1e-8 * scale[k::3].max(), k
    assert np.abs(fd[0::3] - (J @ x)[0::3]).max() > 1e-2 * scale[0::3].max()


def test_transport_jv_vanishes_without_table():
    """Constant mobilities and diffusion coefficients: the full Jacobian is the Picard one."""
    d, g, phys, u, rng = _table_problem()
    phys0 = disc.Physics(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=30.0, D_e=60.0, mu_p=0.15, D_p=0.0038)
    w = disc.from_vec(g, rng.standard_normal(3 * g.n_nodes_unknown))
    assert not np.any(disc.transport_jv(g, u, w, phys0))


def test_table_slopes_are_the_lerp_derivative():
    """The segment slopes are the one-sided derivatives of table_lookup inside the table and
    zero beyond its ends (clamped lookup)."""
    d, g, phys, u, rng = _table_problem()
    E = d.table[:, 0]
    x = np.concatenate([np.exp(rng.uniform(np.log(E[0]), np.log(E[-1]), 200)), [0.5 * E[0], 2.0 * E[-1]]])
    h = 1e-7 * x
    up = disc.table_lookup(d.table, x + h)
    slopes = disc.table_slopes(d.table, x)
    for c in range(4):
        fd = (up[c] - disc.table_lookup(d.table, x)[c]) / h
        assert np.allclose(fd, slopes[c], rtol=1e-5, atol=1e-12 * np.abs(d.table[:, c + 1]).max() / E[0]), c


# ---------------------------------------------------------------- face |E| components (reading 7)
def _bilinear_quadratic_field(g, a=0.3e-2, b=0.7e-2, c1=2.0e5, c2=-3.0e4):
    """V = c1 r^2 (b + z) + c2 (a + r) z^2 on the grid nodes; its face differences have closed
    forms in the node coordinates alone."""
    r, z = g.r[None, :], g.z[:, None]
    return c1 * r ** 2 * (b + z) + c2 * (a + r) * z ** 2


def test_face_field_components_closed_forms():
    """E = -grad V (eq. 6) on the faces of a stretched grid for V = c1 r^2 (b+z) + c2 (a+r) z^2,
    against closed forms written from the node coordinates (no index arithmetic of the oracle):
    * r-face (i+1/2, j): E_r = -[c1 (r_i + r_{i+1})(b + z_j) + c2 z_j^2];
    * z-face (i, j+1/2): E_z = -[c1 r_i^2 + c2 (a + r_i)(z_j + z_{j+1})];
    * transverse E_z on an interior r-face: the mean of the four z-faces at columns i, i+1 and
      rows j-1/2, j+1/2, i.e. -[c1 (r_i^2 + r_{i+1}^2)/2 + c2 (a + r_{i+1/2})(z_{j-1} + 2 z_j + z_{j+1})/2];
    * transverse E_r on a z-face of an inner column: the mean of the four r-faces at rows j, j+1
      and columns i-1/2, i+1/2, i.e. -[c1 2 r_i (b + (z_j + z_{j+1})/2) + c2 (z_j^2 + z_{j+1}^2)/2];
    * zero transverse part on the electrode-row r-faces and on the axis and wall z-faces.
    A dropped term, a wrong neighbour index or a transposed average fails one of these."""
    a, b, c1, c2 = 0.3e-2, 0.7e-2, 2.0e5, -3.0e4
    g = _grid(8, 16, ratio=1.3)
    V = _bilinear_quadratic_field(g, a, b, c1, c2)
    Er, Ez_t, Ez, Er_t = disc.face_field_components(g, V)
    r, z = g.r, g.z
    rh = 0.5 * (r[:-1] + r[1:])
    ex_Er = -(c1 * (r[:-1] + r[1:])[None, :] * (b + z)[:, None] + c2 * (z ** 2)[:, None] * np.ones(g.nr)[None, :])
    ex_Ez = -(c1 * (r ** 2)[None, :] * np.ones(g.nz)[:, None] + c2 * (a + r)[None, :] * (z[:-1] + z[1:])[:, None])
    ex_Ez_t = np.zeros((g.nz + 1, g.nr))
    ex_Ez_t[1:-1] = -(c1 * 0.5 * (r[:-1] ** 2 + r[1:] ** 2)[None, :]
                      + c2 * (a + rh)[None, :] * (0.5 * (z[:-2] + 2 * z[1:-1] + z[2:]))[:, None])
    ex_Er_t = np.zeros((g.nz, g.nr + 1))
    ex_Er_t[:, 1:-1] = -(c1 * 2 * r[1:-1][None, :] * (b + 0.5 * (z[:-1] + z[1:]))[:, None]
                         + c2 * (0.5 * (z[:-1] ** 2 + z[1:] ** 2))[:, None])
    for got, ex in ((Er, ex_Er), (Ez, ex_Ez), (Ez_t, ex_Ez_t), (Er_t, ex_Er_t)):
        assert got.shape == ex.shape
        assert np.abs(got - ex).max() <= 1e-11 * np.abs(ex).max()
    # |E| combines the normal and the transverse component in quadrature
    Eabs_r, Eabs_z = disc.face_fields(g, V)
    assert np.allclose(Eabs_r, np.hypot(ex_Er, ex_Ez_t), rtol=1e-11)
    assert np.allclose(Eabs_z, np.hypot(ex_Ez, ex_Er_t), rtol=1e-11)


def test_face_field_components_hand_values():
    """A 2 x 2-interval grid (r = 0, 1, 2 mm; z = 0, 1, 3 mm) and V with node values written out;
    every face value below was computed by hand from E = -(V_R - V_L)/h."""
    g = Grid(2, 2, 2e-3, np.array([0.0, 1e-3, 3e-3]))
    V = np.array([[0.0, 1.0, 4.0],      # z = 0
                  [2.0, 2.0, 8.0],      # z = 1 mm
                  [6.0, 9.0, 3.0]])     # z = 3 mm
    Er, Ez_t, Ez, Er_t = disc.face_field_components(g, V)
    k = 1e3   # 1/mm
    assert np.allclose(Er, -k * np.array([[1.0, 3.0], [0.0, 6.0], [3.0, -6.0]]), rtol=1e-14)
    assert np.allclose(Ez, -k * np.array([[2.0, 1.0, 4.0], [2.0, 3.5, -2.5]]), rtol=1e-14)
    # transverse E_z on the middle-row r-faces: (Ez[0,i] + Ez[1,i] + Ez[0,i+1] + Ez[1,i+1]) / 4
    assert np.allclose(Ez_t, -k * np.array([[0.0, 0.0], [8.5 / 4, 6.0 / 4], [0.0, 0.0]]), rtol=1e-14)
    # transverse E_r on the middle-column z-faces: (Er[j,0] + Er[j,1] + Er[j+1,0] + Er[j+1,1]) / 4
    assert np.allclose(Er_t, -k * np.array([[0.0, 10.0 / 4, 0.0], [0.0, 3.0 / 4, 0.0]]), rtol=1e-14)


# ---------------------------------------------------------------- table lookup (reading 7)
_HAND_TABLE = np.array([[1.0, 5.0, 1.0, 0.50, 10.0],
                        [10.0, 3.0, 2.0, 0.25, 20.0],
                        [100.0, 7.0, 3.0, 1.00, 40.0]])


@pytest.mark.parametrize("E,expect", [
    (0.5, (5.0, 1.0, 0.5, 10.0)),                 # below the first node: clamped to row 0
    (1.0, (5.0, 1.0, 0.5, 10.0)),                 # at node 0
    (4.0, (13.0 / 3, 4.0 / 3, 0.5 - 0.25 / 3, 40.0 / 3)),   # a third of the way to node 1
    (10.0, (3.0, 2.0, 0.25, 20.0)),               # at node 1
    (55.0, (5.0, 2.5, 0.625, 30.0)),              # half way between nodes 1 and 2
    (100.0, (7.0, 3.0, 1.0, 40.0)),               # at the last node
    (1e3, (7.0, 3.0, 1.0, 40.0)),                 # beyond it: clamped to the last row
])
def test_table_lookup_hand_values(E, expect):
    """Linear interpolation in |E| (not in log |E|) between the bracketing rows, clamped at both
    ends: hand-computed values of a three-row table."""
    got = disc.table_lookup(_HAND_TABLE, np.array([E]))
    assert np.allclose([c[0] for c in got], expect, rtol=1e-14, atol=0)


def test_table_slopes_hand_values():
    """Segment slopes of the three-row table: (row k+1 - row k) / (E_{k+1} - E_k) inside, zero
    beyond the ends."""
    x = np.array([0.5, 4.0, 55.0, 2e3])
    s = disc.table_slopes(_HAND_TABLE, x)
    assert np.allclose(s[0], [0.0, -2.0 / 9, 4.0 / 90, 0.0], rtol=1e-14, atol=0)
    assert np.allclose(s[3], [0.0, 10.0 / 9, 20.0 / 90, 0.0], rtol=1e-14, atol=0)


def test_table_lookup_reproduces_linear_columns_on_the_log_spaced_table():
    """On the 64-row log-spaced |E| nodes, a column that is linear in |E| is reproduced exactly
    between any two nodes (interpolation in log |E|, or on the wrong segment, is not)."""
    E = W.transport_table(seed=2)[:, 0]
    tab = np.stack([E, 3.0 + 2e-4 * E, 1.0 + 0 * E, 7.0 - 1e-6 * E, 2.0 * E], axis=1)
    rng = np.random.default_rng(5)
    x = np.concatenate([np.exp(rng.uniform(np.log(E[0]), np.log(E[-1]), 500)), E])
    got = disc.table_lookup(tab, x)
    for c, ex in enumerate((3.0 + 2e-4 * x, 1.0 + 0 * x, 7.0 - 1e-6 * x, 2.0 * x)):
        assert np.allclose(got[c], ex, rtol=1e-13, atol=0), c
