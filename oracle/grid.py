"""Axisymmetric node grid and finite-volume geometry (Sec. 2; eqs. 12-13).

Nodes: r_i = i dr (i = 0..N_r, equidistant), z_j given (j = 0..N_z, non-equidistant).
Intervals dz_j = z_{j+1} - z_j.  Everything below is "per radian" (the 2 pi of the
azimuthal integral cancels from every row).

Control volume of node (i, j), bounded by the midpoints r_{i +- 1/2}, z_{j +- 1/2}:
* radial extent  volr_i = int r dr:  dr^2/8 (axis, i = 0), i dr^2 (interior),
  (N_r - 1/4) dr^2 / 2 (outer wall, i = N_r, half cell);
* axial width    dzc_j = (dz_{j-1} + dz_j) / 2  (eq. 12 writes this width as
  delta z_{j-1/2}; it is the only reading under which eq. 12 is the standard
  non-uniform three-point Laplacian);
* volume         A_ij = volr_i dzc_j.
Face "conductances" (area / distance):
* r-face (i+1/2, j):  gr_ij = r_{i+1/2} dzc_j / dr = (i + 1/2) dzc_j
* z-face (i, j+1/2):  gz_ij = volr_i / dz_j
Dividing the finite-volume Poisson row by A_ij / dr^2 reproduces the printed
coefficients of eq. 12 (interior) and eq. 13 (axis); the tests check this.

Unknown rows are j = 1..N_z-1 (electrode rows j = 0, N_z carry Dirichlet data),
i = 0..N_r (axis row: natural finite-volume row; wall row: half cell, zero outer flux).
With wall_dirichlet (the paper's argon case, Sec. 3: n_e = n_p = 0 on the wall and V
interpolated linearly along it) the wall column i = N_r carries Dirichlet data too and the
unknowns are i = 0..N_r-1.
"""
from __future__ import annotations

import numpy as np


class Grid:
    def __init__(self, nr: int, nz: int, R: float, z: np.ndarray, wall_dirichlet: bool = False):
        z = np.asarray(z, dtype=np.float64)
        if z.shape != (nz + 1,):
            raise ValueError("z must have nz + 1 entries")
        if np.any(np.diff(z) <= 0):
            raise ValueError("z must increase strictly")
        self.nr, self.nz, self.R = int(nr), int(nz), float(R)
        self.z = z.copy()
        self.dr = self.R / self.nr
        self.r = np.arange(self.nr + 1, dtype=np.float64) * self.dr
        self.dz = np.diff(self.z)                                  # (nz,)
        dzc = np.zeros(self.nz + 1)
        dzc[1:-1] = 0.5 * (self.dz[:-1] + self.dz[1:])             # rows 1..nz-1
        self.dzc = dzc
        i = np.arange(self.nr + 1, dtype=np.float64)
        volr = i * self.dr ** 2
        volr[0] = self.dr ** 2 / 8.0
        volr[-1] = (self.nr - 0.25) * self.dr ** 2 / 2.0
        self.volr = volr                                           # (nr+1,)
        self.A = self.dzc[:, None] * self.volr[None, :]            # (nz+1, nr+1)
        # r-face conductance (i+1/2, j): (i+1/2) * dzc_j, shape (nz+1, nr)
        self.gr = (np.arange(self.nr) + 0.5)[None, :] * self.dzc[:, None]
        # z-face conductance (i, j+1/2): volr_i / dz_j, shape (nz, nr+1)
        self.gz = self.volr[None, :] / self.dz[:, None]
        self.shape = (self.nz + 1, self.nr + 1)
        self.wall_dirichlet = bool(wall_dirichlet)
        self.ni = self.nr if self.wall_dirichlet else self.nr + 1   # unknown columns
        self.n_nodes_unknown = (self.nz - 1) * self.ni

    def coarse(self) -> "Grid":
        """Vertex-centred coarsening by two in both directions (nested node subset)."""
        if self.nr % 2 or self.nz % 2:
            raise ValueError("cannot coarsen an odd grid")
        return Grid(self.nr // 2, self.nz // 2, self.R, self.z[::2], self.wall_dirichlet)

    # unknown numbering: node-major, three fields per node (n_e, n_p, V)
    def node_index(self):
        """(nz+1, nr+1) int array of unknown-node numbers (-1 on Dirichlet nodes)."""
        idx = -np.ones(self.shape, dtype=np.int64)
        idx[1:-1, :self.ni] = np.arange(self.n_nodes_unknown).reshape(self.nz - 1, self.ni)
        return idx
