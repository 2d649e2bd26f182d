"""Discrete drift-diffusion-Poisson system: fluxes, residual, Newton Jacobian.

State u = (n_e, n_p, V), array (3, N_z+1, N_r+1), SI units, n0 = 1 (the paper's
scaling n0 of eq. 12 is a pure unit choice; the oracle works in m^-3).

* Face fluxes: Scharfetter-Gummel, eqs. 8-9, with the drift parameter of
  eqs. 10-11 (s = -1 electrons, s = +1 ions).  Eq. 9 is printed with G for both
  nodes; this oracle uses G for n_{i,j} and F for n_{i,j+1}, the same pairing as
  eq. 8.  That is the only pairing whose alpha -> 0 limit is the drift-diffusion
  flux of eqs. 3-4 (pinned by a test).
* Residual rows (finite-volume integrated, i.e. eq. 7 multiplied by the control
  volume): continuity
      A (n - n^k)/dt + [sum of outward face fluxes] - A S
  and Poisson (eqs. 5, 12, 13)
      [sum over faces of g (V_nb - V)] + A (e/eps0) (n_p - n_e).
  Electrode rows j = 0, N_z are Dirichlet (n_e = n_p = 0, V = V_cathode / V_anode);
  the outer wall r = R has zero normal flux and dV/dr = 0; the axis row is the
  natural finite-volume row.
* Jacobian (eq. 14): analytic derivatives of the residual rows, 3x3 blocks in a
  five-point stencil.  With field-dependent mu(|E|), D(|E|) the transport
  coefficients are frozen at the current iterate (Picard in mu, D).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.sparse as sp

from . import bernoulli
from .grid import Grid

E_CHARGE = 1.602176634e-19
EPS0 = 8.8541878128e-12
KAPPA = E_CHARGE / EPS0          # e / eps0 of eq. 5


@dataclasses.dataclass
class Physics:
    V_cathode: float = -200.0
    V_anode: float = 0.0
    mu_e: float = 30.0
    D_e: float = 60.0
    mu_p: float = 0.15
    D_p: float = 0.0038
    table: Optional[np.ndarray] = None     # (64, 5): |E|, mu_e, D_e, mu_p, D_p
    pressure_factor: float = 1.0


def apply_dirichlet(u: np.ndarray, phys: Physics, g: Optional[Grid] = None) -> np.ndarray:
    """Electrode rows: n_e = n_p = 0, V(z=0) = V_cathode, V(z=d) = V_anode; with a grid whose
    wall is Dirichlet (Sec. 3) also the wall column: n_e = n_p = 0, V linear in z between them."""
    u = u.copy()
    u[0:2, 0, :] = 0.0
    u[0:2, -1, :] = 0.0
    u[2, 0, :] = phys.V_cathode
    u[2, -1, :] = phys.V_anode
    if g is not None and g.wall_dirichlet:
        u[0:2, :, -1] = 0.0
        u[2, :, -1] = phys.V_cathode + (phys.V_anode - phys.V_cathode) * (g.z - g.z[0]) / (g.z[-1] - g.z[0])
    return u


# --------------------------------------------------------------------------- fields
def face_field_components(g: Grid, V: np.ndarray):
    """Components of E = -grad V (eq. 6) on the faces: (Er, Ez_t) on r-faces (nz+1, nr) and
    (Ez, Er_t) on z-faces (nz, nr+1).

    The face-normal component is the two-point difference across the face; the
    transverse component is the mean of the four adjacent perpendicular face
    fields.  On the axis and the outer wall the perpendicular field is taken as
    zero (dV/dr = 0 there by symmetry).  Electrode-row r-faces get no transverse
    part (they never enter a residual row).  Linear in V.
    """
    Er = -(V[:, 1:] - V[:, :-1]) / g.dr
    Ez = -(V[1:, :] - V[:-1, :]) / g.dz[:, None]
    Ez_t = np.zeros_like(Er)
    Ez_t[1:-1, :] = 0.25 * (Ez[:-1, :-1] + Ez[1:, :-1] + Ez[:-1, 1:] + Ez[1:, 1:])
    Er_t = np.zeros_like(Ez)
    Er_t[:, 1:-1] = 0.25 * (Er[:-1, :-1] + Er[:-1, 1:] + Er[1:, :-1] + Er[1:, 1:])
    return Er, Ez_t, Ez, Er_t


def face_fields(g: Grid, V: np.ndarray):
    """|E| on r-faces (nz+1, nr) and z-faces (nz, nr+1) (see face_field_components)."""
    Er, Ez_t, Ez, Er_t = face_field_components(g, V)
    return np.sqrt(Er ** 2 + Ez_t ** 2), np.sqrt(Ez ** 2 + Er_t ** 2)


def table_lookup(table: np.ndarray, Eabs: np.ndarray):
    """Piecewise-linear interpolation in |E| between the table nodes, clamped at both ends."""
    E = table[:, 0]
    x = np.clip(Eabs, E[0], E[-1])
    k = np.clip(np.searchsorted(E, x, side="right") - 1, 0, len(E) - 2)
    t = (x - E[k]) / (E[k + 1] - E[k])
    cols = [table[k, c] + t * (table[k + 1, c] - table[k, c]) for c in range(1, 5)]
    return cols  # mu_e, D_e, mu_p, D_p


def table_slopes(table: np.ndarray, Eabs: np.ndarray):
    """d/d|E| of each interpolated column at |E|: the slope of the segment table_lookup
    interpolates on, zero where |E| lies outside the table (the lookup is clamped there)."""
    E = table[:, 0]
    inside = (Eabs >= E[0]) & (Eabs <= E[-1])
    x = np.clip(Eabs, E[0], E[-1])
    k = np.clip(np.searchsorted(E, x, side="right") - 1, 0, len(E) - 2)
    h = E[k + 1] - E[k]
    return [np.where(inside, (table[k + 1, c] - table[k, c]) / h, 0.0) for c in range(1, 5)]


def face_transport(g: Grid, V: np.ndarray, phys: Physics):
    """(mu_e, D_e, mu_p, D_p) on r-faces and z-faces; constants or table lerp, / pressure factor."""
    f = phys.pressure_factor
    if phys.table is None:
        mk = lambda shape: [np.full(shape, v / f) for v in (phys.mu_e, phys.D_e, phys.mu_p, phys.D_p)]
        return mk((g.nz + 1, g.nr)), mk((g.nz, g.nr + 1))
    Er, Ez = face_fields(g, V)
    return ([c / f for c in table_lookup(phys.table, Er)],
            [c / f for c in table_lookup(phys.table, Ez)])


# --------------------------------------------------------------------------- fluxes
def sg_flux(gfac, mu, D, s, nL, nR, VL, VR):
    """Integrated SG flux from L to R through one face (eqs. 8-11).

    alpha = -s (mu/D)(V_R - V_L);  flux = g D (n_L G(alpha) - n_R F(alpha)).
    """
    alpha = -s * (mu / D) * (VR - VL)
    return gfac * D * (nL * bernoulli.G(alpha) - nR * bernoulli.F(alpha))


def _faces(g: Grid, u: np.ndarray, phys: Physics):
    """Yield (set, gfac, mu/D per species, L-slice, R-slice) for the r- and z-face sets."""
    (mer, der, mpr, dpr), (mez, dez, mpz, dpz) = face_transport(g, u[2], phys)
    yield ("r", g.gr, (mer, der), (mpr, dpr), (slice(None), slice(0, -1)), (slice(None), slice(1, None)))
    yield ("z", g.gz, (mez, dez), (mpz, dpz), (slice(0, -1), slice(None)), (slice(1, None), slice(None)))


def residual(g: Grid, u: np.ndarray, u_old: Optional[np.ndarray], S_e, S_p, dt: Optional[float],
             phys: Physics, with_terms: bool = False):
    """Residual rows F (3, nz+1, nr+1) (zero on electrode rows); optionally T = sum |terms|.

    dt=None gives the steady residual (time term dropped).
    """
    ne, npos, V = u
    F = np.zeros_like(u)
    T = np.zeros_like(u)
    A = g.A
    if dt is not None:
        F[0] += A * (ne - u_old[0]) / dt
        F[1] += A * (npos - u_old[1]) / dt
        T[0] += A * (np.abs(ne) + np.abs(u_old[0])) / dt
        T[1] += A * (np.abs(npos) + np.abs(u_old[1])) / dt
    F[0] -= A * S_e
    F[1] -= A * S_p
    T[0] += A * np.abs(S_e)
    T[1] += A * np.abs(S_p)
    for _, gf, (mue, De), (mup, Dp), Ls, Rs in _faces(g, u, phys):
        for fi, s, mu, D in ((0, -1.0, mue, De), (1, +1.0, mup, Dp)):
            n = u[fi]
            phi = sg_flux(gf, mu, D, s, n[Ls], n[Rs], V[Ls], V[Rs])
            F[fi][Ls] += phi
            F[fi][Rs] -= phi
            T[fi][Ls] += np.abs(phi)
            T[fi][Rs] += np.abs(phi)
        psi = gf * (V[Rs] - V[Ls])
        F[2][Ls] += psi
        F[2][Rs] -= psi
        T[2][Ls] += np.abs(psi)
        T[2][Rs] += np.abs(psi)
    F[2] += A * KAPPA * (npos - ne)
    T[2] += A * KAPPA * (np.abs(npos) + np.abs(ne))
    F[:, 0, :] = 0.0
    F[:, -1, :] = 0.0
    T[:, 0, :] = 0.0
    T[:, -1, :] = 0.0
    if g.wall_dirichlet:
        F[:, :, -1] = 0.0
        T[:, :, -1] = 0.0
    return (F, T) if with_terms else F


def rho(F: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Per-field scale-free residual ||F_f||_2 / ||T_f||_2 over the unknown rows."""
    out = np.zeros(3)
    for f in range(3):
        nf = np.linalg.norm(F[f, 1:-1].ravel())
        nt = np.linalg.norm(T[f, 1:-1].ravel())
        out[f] = 0.0 if nf == 0.0 else (nf / nt if nt > 0 else np.inf)
    return out


# --------------------------------------------------------------------------- Jacobian
def face_coefficients(g: Grid, u: np.ndarray, phys: Physics):
    """Per face set and species: cG = g D G(a), cF = g D F(a), cV = d(flux)/dV_R; and g.

    d(flux)/dn_L = cG, d(flux)/dn_R = -cF, d(flux)/dV_R = cV = -d(flux)/dV_L,
    cV = -s g mu (n_L G'(a) - n_R F'(a)) (mu, D frozen).
    """
    V = u[2]
    out = {}
    for name, gf, (mue, De), (mup, Dp), Ls, Rs in _faces(g, u, phys):
        per = {"g": gf, "L": Ls, "R": Rs}
        for fi, s, mu, D in ((0, -1.0, mue, De), (1, +1.0, mup, Dp)):
            n = u[fi]
            a = -s * (mu / D) * (V[Rs] - V[Ls])
            cG = gf * D * bernoulli.G(a)
            cF = gf * D * bernoulli.F(a)
            cV = -s * gf * mu * (n[Ls] * bernoulli.dG(a) - n[Rs] * bernoulli.dF(a))
            per[fi] = (cG, cF, cV)
        out[name] = per
    return out


def jacobian(g: Grid, u: np.ndarray, dt: Optional[float], phys: Physics) -> sp.csr_matrix:
    """Sparse Jacobian dF/du over the unknowns (eq. 14), node-major ordering 3*k + field."""
    idx = g.node_index()
    rows, cols, vals = [], [], []

    def add(r_node, r_f, c_node, c_f, v):
        m = (r_node >= 0) & (c_node >= 0)
        rows.append(3 * r_node[m] + r_f)
        cols.append(3 * c_node[m] + c_f)
        vals.append(np.broadcast_to(v, r_node.shape)[m])

    A = g.A
    if dt is not None:
        add(idx, 0, idx, 0, A / dt)
        add(idx, 1, idx, 1, A / dt)
    add(idx, 2, idx, 0, -A * KAPPA)
    add(idx, 2, idx, 1, A * KAPPA)
    for name, per in face_coefficients(g, u, phys).items():
        L, R, gf = idx[per["L"]], idx[per["R"]], per["g"]
        for fi in (0, 1):
            cG, cF, cV = per[fi]
            # row L gets +flux, row R gets -flux
            add(L, fi, L, fi, cG)
            add(L, fi, R, fi, -cF)
            add(L, fi, L, 2, -cV)
            add(L, fi, R, 2, cV)
            add(R, fi, L, fi, -cG)
            add(R, fi, R, fi, cF)
            add(R, fi, L, 2, cV)
            add(R, fi, R, 2, -cV)
        add(L, 2, L, 2, -gf)
        add(L, 2, R, 2, gf)
        add(R, 2, L, 2, gf)
        add(R, 2, R, 2, -gf)
    n = 3 * g.n_nodes_unknown
    J = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return J.tocsr()


def transport_jv(g: Grid, u: np.ndarray, w: np.ndarray, phys: Physics) -> np.ndarray:
    """The part of the residual's directional derivative along w (3, nz+1, nr+1) that the
    Picard Jacobian leaves out: the flux change through mu(|E|), D(|E|) as the potential moves
    by w[2] (Sec. 2: mobilities and diffusion coefficients are functions of the local field).

    Per face and species, flux = g D (n_L G(a) - n_R F(a)) with a = -s (mu/D)(V_R - V_L)
    (eqs. 8-11), so at fixed n, V_R - V_L:
        d flux = g dD (n_L G(a) - n_R F(a)) + g D (n_L G'(a) - n_R F'(a)) da,
        da = -s (V_R - V_L) (dmu D - mu dD) / D^2,
    with dmu, dD the table slopes times d|E|, and d|E| = (E_n dE_n + E_t dE_t) / |E| from
    the field components of w[2].  Rows as in residual (L += d flux, R -= d flux); zero
    without a transport table.
    """
    out = np.zeros_like(u)
    if phys.table is None:
        return out
    V, f = u[2], phys.pressure_factor
    Er, Ezt, Ez, Ert = face_field_components(g, V)
    dEr, dEzt, dEz, dErt = face_field_components(g, w[2])
    sets = (("r", Er, Ezt, dEr, dEzt), ("z", Ez, Ert, dEz, dErt))
    for (name, gf, _, _, Ls, Rs), (_, En, Et, dEn, dEt) in zip(_faces(g, u, phys), sets):
        Em = np.sqrt(En ** 2 + Et ** 2)
        dEm = np.divide(En * dEn + Et * dEt, Em, out=np.zeros_like(Em), where=Em > 0)
        vals = [c / f for c in table_lookup(phys.table, Em)]
        slopes = [c / f for c in table_slopes(phys.table, Em)]
        dVf = V[Rs] - V[Ls]
        for fi, s, (mu, D), (smu, sD) in ((0, -1.0, vals[0:2], slopes[0:2]), (1, 1.0, vals[2:4], slopes[2:4])):
            n = u[fi]
            a = -s * (mu / D) * dVf
            dmu, dD = smu * dEm, sD * dEm
            da = -s * dVf * (dmu * D - mu * dD) / D ** 2
            dflux = (gf * dD * (n[Ls] * bernoulli.G(a) - n[Rs] * bernoulli.F(a))
                     + gf * D * (n[Ls] * bernoulli.dG(a) - n[Rs] * bernoulli.dF(a)) * da)
            out[fi][Ls] += dflux
            out[fi][Rs] -= dflux
    return out


def jacobian_full_apply(g: Grid, u: np.ndarray, dt: Optional[float], phys: Physics, x: np.ndarray,
                        J: Optional[sp.csr_matrix] = None) -> np.ndarray:
    """Full Jacobian (field dependence of mu, D included) times an unknown vector x:
    J x (Picard Jacobian, eq. 14) plus transport_jv along x."""
    J = jacobian(g, u, dt, phys) if J is None else J
    return J @ x + to_vec(g, transport_jv(g, u, from_vec(g, x), phys))


def to_vec(g: Grid, a: np.ndarray) -> np.ndarray:
    """(3, nz+1, nr+1) -> unknown vector (node-major, 3 per node)."""
    return np.ascontiguousarray(np.moveaxis(a[:, 1:-1, :g.ni], 0, -1)).reshape(-1)


def from_vec(g: Grid, x: np.ndarray) -> np.ndarray:
    """Unknown vector -> (3, nz+1, nr+1) with zeros on the Dirichlet nodes."""
    out = np.zeros((3,) + g.shape)
    out[:, 1:-1, :g.ni] = np.moveaxis(x.reshape(g.nz - 1, g.ni, 3), -1, 0)
    return out
