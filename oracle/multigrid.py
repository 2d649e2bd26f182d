"""Multigrid V-cycle for the Newton system of eq. 14 (plain FP64, sparse matrices).

Sec. 2 of the paper solves eq. 14 by "the multigrid method" of its ref. [4] and
names no component.  The components below are this project's readings:

* hierarchy: vertex-centred coarsening by two in r and z (nested node subsets),
  down to ``coarsest`` intervals per direction;
* coarse operator: the Jacobian rediscretised on the coarse grid at the state
  injected from the fine grid (u_c = u_f at the shared nodes), same dt;
* smoother: collective (3x3 point-block) Gauss-Seidel in red-black order,
  red = (i + j) even first; in a five-point stencil nodes of one colour do not
  couple, so a half sweep is an exact block solve of the colour's own rows;
  or (line=True or "z") z-line Gauss-Seidel in zebra order, even columns first: a half
  sweep solves the block-tridiagonal system of every column of one parity
  exactly, its r-neighbours (the other parity) held fixed; (line="r") r-line
  Gauss-Seidel, the same along the rows, even rows first (row index j counted from the
  cathode row 0); (line="alt") alternating lines: each sweep a z-line sweep, then an
  r-line sweep;
* prolongation P: bilinear interpolation in the node coordinates (r equidistant,
  z by distance weights), identity across the three fields; electrode rows carry 0;
* restriction R = P^T acting on the finite-volume-integrated residual;
* coarsest level: dense LU with partial pivoting of the whole (equilibrated) 3-field system;
* V(nu1, nu2) cycles (V(nu_coarse1, nu_coarse2) smoothing on the small levels) until the
  field-weighted residual norm has dropped by eta.
"""
from __future__ import annotations

from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import discretization as disc
from .grid import Grid


def prolongation(gf: Grid, gc: Grid) -> sp.csr_matrix:
    """Bilinear P mapping coarse unknowns (gc) to fine unknowns (gf)."""
    idf, idc = gf.node_index(), gc.node_index()
    rows, cols, vals = [], [], []
    for j in range(1, gf.nz):
        if j % 2 == 0:
            zw = [(j // 2, 1.0)]
        else:
            J0 = (j - 1) // 2
            w1 = (gf.z[j] - gc.z[J0]) / (gc.z[J0 + 1] - gc.z[J0])
            zw = [(J0, 1.0 - w1), (J0 + 1, w1)]
        for i in range(gf.nr + 1):
            rw = [(i // 2, 1.0)] if i % 2 == 0 else [((i - 1) // 2, 0.5), ((i + 1) // 2, 0.5)]
            for Jc, wz in zw:
                if Jc < 1 or Jc > gc.nz - 1:
                    continue
                for Ic, wr in rw:
                    if idf[j, i] < 0 or idc[Jc, Ic] < 0:
                        continue   # Dirichlet wall nodes carry no correction
                    for f in range(3):
                        rows.append(3 * idf[j, i] + f)
                        cols.append(3 * idc[Jc, Ic] + f)
                        vals.append(wz * wr)
    n_f, n_c = 3 * gf.n_nodes_unknown, 3 * gc.n_nodes_unknown
    return sp.csr_matrix((vals, (rows, cols)), shape=(n_f, n_c))


def inject(gf: Grid, a: np.ndarray) -> np.ndarray:
    """Node-array injection fine -> coarse (every other node)."""
    return a[..., ::2, ::2].copy()


class _ScaledLU:
    """Solve of an equilibrated system: A = diag(1/rs) (rs A cs) diag(1/cs)."""

    def __init__(self, lu, rs, cs):
        self.lu, self.rs, self.cs = lu, rs, cs

    def solve(self, b):
        return self.cs * self.lu.solve(self.rs * b)


class Level:
    def __init__(self, g: Grid, u: np.ndarray, dt: Optional[float], phys: disc.Physics, line=False):
        self.g = g
        if line not in (False, True, "z", "r", "alt"):
            raise ValueError("line must be False, True / 'z', 'r' or 'alt'")
        self.line = "z" if line is True else line
        self.J = disc.jacobian(g, u, dt, phys)
        nodes = np.arange(g.n_nodes_unknown)
        jj = nodes // g.ni + 1
        ii = nodes % g.ni
        self.colors = []
        for c in (0, 1):
            nc = nodes[(ii + jj) % 2 == c]
            oc = nodes[(ii + jj) % 2 != c]
            U = (3 * nc[:, None] + np.arange(3)[None, :]).ravel()
            O = (3 * oc[:, None] + np.arange(3)[None, :]).ravel()
            Jcc = self.J[U][:, U].tocoo()
            if np.any((Jcc.row // 3) != (Jcc.col // 3)):
                raise AssertionError("same-colour nodes couple: not a five-point stencil")
            blocks = np.zeros((len(nc), 3, 3))
            blocks[Jcc.row // 3, Jcc.row % 3, Jcc.col % 3] = Jcc.data
            self.colors.append((U, O, blocks, self.J[U][:, O].tocsr()))
        # line half sweeps in their order within a sweep: z-lines (columns of one parity), then
        # r-lines (rows of one parity); the unknowns of one parity's lines couple only along
        # their own line, so one sparse LU solves every line of the half sweep exactly.  The
        # line matrices are equilibrated first (every column, then every row scaled to a unit
        # max-abs entry, as in `direct`): unscaled, densities (~1e14) and potentials (~1e2) in
        # one system left the sparse LU's pivots off by up to 1e-6 of a field on lines along the
        # weakly coupled direction
        self.lines = []
        groups = {"z": [ii], "r": [jj], "alt": [ii, jj]}.get(self.line, [])
        for idx in groups:
            for c in (0, 1):
                nc = nodes[idx % 2 == c]
                oc = nodes[idx % 2 != c]
                if len(nc) == 0:
                    continue  # a level with a single line across: no line of this parity
                U = (3 * nc[:, None] + np.arange(3)[None, :]).ravel()
                O = (3 * oc[:, None] + np.arange(3)[None, :]).ravel()
                JUU = self.J[U][:, U].tocoo()
                if np.any(idx[nc[JUU.row // 3]] != idx[nc[JUU.col // 3]]):
                    raise AssertionError("lines of one parity couple: not a five-point stencil")
                A = JUU.tocsr()
                cs = 1.0 / np.asarray(abs(A).max(axis=0).todense()).ravel()
                A = A @ sp.diags(cs)
                rs = 1.0 / np.asarray(abs(A).max(axis=1).todense()).ravel()
                A = sp.diags(rs) @ A
                self.lines.append((U, O, _ScaledLU(spla.splu(A.tocsc()), rs, cs), self.J[U][:, O].tocsr()))
        self.dense = None

    def smooth(self, x: np.ndarray, f: np.ndarray, sweeps: int) -> np.ndarray:
        if self.line:
            for _ in range(sweeps):
                for U, O, lu, JUO in self.lines:
                    x[U] = lu.solve(f[U] - JUO @ x[O])
            return x
        for _ in range(sweeps):
            for U, O, blocks, JUO in self.colors:
                rhs = (f[U] - JUO @ x[O]).reshape(-1, 3, 1)
                x[U] = np.linalg.solve(blocks, rhs).reshape(-1)
        return x

    def direct(self, f: np.ndarray) -> np.ndarray:
        """Dense LU with partial pivoting of the row- and column-equilibrated matrix.

        The unscaled Jacobian mixes densities (~1e14 m^-3) and potentials (~1e2 V),
        so its condition number is ~1e28; scaling every column, then every row, to a
        unit max-abs entry (the classic equilibration) brings it to O(1e2).
        """
        if self.dense is None:
            Jd = self.J.toarray()
            c = 1.0 / np.abs(Jd).max(axis=0)
            Jd = Jd * c[None, :]
            r = 1.0 / np.abs(Jd).max(axis=1)
            self.dense = (sla.lu_factor(Jd * r[:, None]), r, c)
        lu, r, c = self.dense
        return c * sla.lu_solve(lu, r * f)


class Hierarchy:
    """Levels 0 (finest) .. L-1 built at the state u (injected downward)."""

    def __init__(self, g: Grid, u: np.ndarray, dt: Optional[float], phys: disc.Physics,
                 coarsest: int = 2, nu1: int = 4, nu2: int = 4, nu_coarse_n: int = 64,
                 nu_coarse1: int = 2, nu_coarse2: int = 2, nu_tiny_n: int = 8, nu_tiny1: int = 1,
                 nu_tiny2: int = 1, line=False):
        """Smoothing: nu1 / nu2 sweeps before / after the coarse-grid correction, except on
        levels whose larger side has at most nu_tiny_n intervals (nu_tiny1 / nu_tiny2) or else at
        most nu_coarse_n intervals (nu_coarse1 / nu_coarse2); 0 switches a tier off."""
        self.levels: List[Level] = []
        self.P: List[sp.csr_matrix] = []
        self.nus: List[tuple] = []
        while True:
            self.levels.append(Level(g, u, dt, phys, line))
            side = max(g.nr, g.nz)
            if nu_tiny_n > 0 and side <= nu_tiny_n:
                self.nus.append((nu_tiny1, nu_tiny2))
            elif nu_coarse_n > 0 and side <= nu_coarse_n:
                self.nus.append((nu_coarse1, nu_coarse2))
            else:
                self.nus.append((nu1, nu2))
            if min(g.nr, g.nz) <= coarsest or g.nr % 2 or g.nz % 2:
                break
            gc = g.coarse()
            self.P.append(prolongation(g, gc))
            u = inject(g, u)
            g = gc

    def vcycle(self, l: int, x: np.ndarray, f: np.ndarray) -> np.ndarray:
        lev = self.levels[l]
        if l == len(self.levels) - 1:
            return lev.direct(f)
        nu1, nu2 = self.nus[l]
        x = lev.smooth(x, f, nu1)
        r = f - lev.J @ x
        fc = self.P[l].T @ r
        xc = self.vcycle(l + 1, np.zeros_like(fc), fc)
        x = x + self.P[l] @ xc
        return lev.smooth(x, f, nu2)

    def solve(self, f: np.ndarray, eta: float, max_cycles: int = 100, x0: Optional[np.ndarray] = None,
              scale: Optional[np.ndarray] = None):
        """V-cycles from x0 (default 0) until  max_f ||f - Jx||_f / s_f  <=  eta * max_f ||f||_f / s_f.

        s_f is a per-field scale (the norm of the nonlinear residual's absolute terms,
        so that the test is relative to the Newton residual rho); default s_f = 1.
        Returns (x, history) with history[k] = max_f ||r_f|| / s_f after k cycles,
        normalised by its value at x = 0.
        """
        J = self.levels[0].J
        x = np.zeros_like(f) if x0 is None else x0.copy()
        s = np.ones(3) if scale is None else np.where(np.asarray(scale) > 0, scale, 1.0)

        def wnorm(r):
            return max(np.linalg.norm(r[k::3]) / s[k] for k in range(3))

        f0 = wnorm(f)
        if f0 == 0.0:
            return x, np.zeros(1)
        hist = [wnorm(f - J @ x) / f0]
        for _ in range(max_cycles):
            if hist[-1] <= eta:
                break
            x = self.vcycle(0, x, f)
            hist.append(wnorm(f - J @ x) / f0)
            if not np.isfinite(hist[-1]):
                break
        return x, np.array(hist)
