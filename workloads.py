"""Seeded synthetic inputs for the axisymmetric (r, z) discharge problems.

This module only *generates inputs*: grid node coordinates, source maps,
initial states, transport tables and batch specifications.  It holds none of
the solver's arithmetic (no fluxes, no residuals, no multigrid), so both the
FP64 CPU oracle and the CUDA library can consume the same arrays.

Problem geometry follows Sec. 2 of the paper (domain [0, R] x [0, d], radial
nodes equidistant, axial nodes non-equidistant).  The axial stretching is
symmetric and geometric toward both electrodes; with N_z intervals the
per-interval ratio is q = 1.05**(32 / N_z), so that every coarser node set is
exactly the even-indexed subset of the finer one (the multigrid hierarchy and
the 128 -> 256 continuation of Sec. 2 then nest exactly).

Arrays are laid out [j, i] with j the axial (slow) index and i the radial
(fast) index, shape (N_z + 1, N_r + 1), float64, SI units (m, V, s, m^-3).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

# Physical constants (SI, CODATA 2018 exact / recommended values).
ELEMENTARY_CHARGE = 1.602176634e-19
EPSILON_0 = 8.8541878128e-12

TABLE_POINTS = 64
TABLE_EMIN = 1.0e2
TABLE_EMAX = 1.0e6


def z_nodes(nz: int, d: float, ratio_ref: float = 1.05, nz_ref: int = 32) -> np.ndarray:
    """Axial node coordinates z_0 = 0 < ... < z_nz = d.

    Interval j has length dz0 * q**j for j < nz/2 and mirrors for j >= nz/2,
    q = ratio_ref**(nz_ref / nz); dz0 is fixed by sum = d.  nz must be even.
    """
    if nz < 2 or nz % 2:
        raise ValueError("nz must be even and >= 2")
    q = ratio_ref ** (nz_ref / nz)
    half = nz // 2
    steps = q ** np.arange(half, dtype=np.float64)
    widths = np.concatenate([steps, steps[::-1]])
    widths *= d / widths.sum()
    z = np.concatenate([[0.0], np.cumsum(widths)])
    z[-1] = d
    return z


def r_nodes(nr: int, R: float) -> np.ndarray:
    return np.arange(nr + 1, dtype=np.float64) * (R / nr)


@dataclasses.dataclass
class Discharge:
    """One synthetic discharge: grid, boundary values, transport data, sources, initial state."""

    nr: int
    nz: int
    R: float
    d: float
    z: np.ndarray
    V_cathode: float
    V_anode: float
    mu_e: float
    D_e: float
    mu_p: float
    D_p: float
    pressure_factor: float
    table: Optional[np.ndarray]  # (64, 5): |E|, mu_e, D_e, mu_p, D_p  or None
    S_e: np.ndarray
    S_p: np.ndarray
    ne0: np.ndarray
    np0: np.ndarray
    V0: np.ndarray
    seed: int
    wall_dirichlet: bool = False   # the argon case: n = 0 and V linear in z on the wall r = R

    @property
    def r(self) -> np.ndarray:
        return r_nodes(self.nr, self.R)

    @property
    def shape(self):
        return (self.nz + 1, self.nr + 1)


def gaussian_bump_params(rng: np.random.Generator, R: float, d: float):
    rc = rng.uniform(0.0, 0.3 * R)
    zc = rng.uniform(0.3 * d, 0.7 * d)
    sr = rng.uniform(0.05e-2, 0.2e-2)
    sz = rng.uniform(0.05e-2, 0.2e-2)
    return rc, zc, sr, sz


def gaussian_bump(r, z, rc, zc, sr, sz, peak):
    rr, zz = np.meshgrid(r, z)
    return peak * np.exp(-((rr - rc) ** 2 / (2 * sr * sr) + (zz - zc) ** 2 / (2 * sz * sz)))


def initial_state(r, z, R, d, V_cathode, V_anode, n_peak=1.0e14):
    rr, zz = np.meshgrid(r, z)
    n = n_peak * np.exp(-rr ** 2 / (2 * (0.3 * R) ** 2) - (zz - d / 2) ** 2 / (2 * (0.2 * d) ** 2))
    n[0, :] = 0.0
    n[-1, :] = 0.0
    V = V_cathode + (V_anode - V_cathode) * (zz / d)
    V[0, :] = V_cathode
    V[-1, :] = V_anode
    return n.copy(), n.copy(), V


def transport_table(seed: int = 2) -> np.ndarray:
    """Seeded 64-entry log-spaced |E| table with columns |E|, mu_e, D_e, mu_p, D_p."""
    rng = np.random.default_rng(seed)
    k = np.arange(TABLE_POINTS, dtype=np.float64)
    E = TABLE_EMIN * 10.0 ** (4.0 * k / (TABLE_POINTS - 1))
    E[-1] = TABLE_EMAX
    xi = rng.uniform(-1.0, 1.0, TABLE_POINTS)
    xi2 = rng.uniform(-1.0, 1.0, TABLE_POINTS)
    mu_e = 30.0 * (E / 1e4) ** (-0.1) * (1.0 + 0.05 * xi)
    D_e = 2.0 * mu_e
    mu_p = 0.15 * (1.0 + E / 1e5) ** (-0.5) * (1.0 + 0.05 * xi2)
    D_p = 0.02533 * mu_p
    return np.stack([E, mu_e, D_e, mu_p, D_p], axis=1)


def make_discharge(n: int, *, seed: int = 0, V_cathode: float = -200.0, use_table: bool = False,
                   table_seed: int = 2, pressure_factor: float = 1.0, nz: Optional[int] = None,
                   R: float = 1e-2, d: float = 1e-2, source_peak: float = 1e20) -> Discharge:
    """Synthetic discharge on an (n+1) x (nz+1) node grid (nz defaults to n)."""
    nr = n
    nz = n if nz is None else nz
    if nr < 2 or (nr & (nr - 1)) or nz < 2 or (nz & (nz - 1)):
        raise ValueError("N_r and N_z must be powers of two >= 2")
    rng = np.random.default_rng(seed)
    z = z_nodes(nz, d)
    r = r_nodes(nr, R)
    rc, zc, sr, sz = gaussian_bump_params(rng, R, d)
    S = gaussian_bump(r, z, rc, zc, sr, sz, source_peak)
    ne0, np0, V0 = initial_state(r, z, R, d, V_cathode, 0.0)
    return Discharge(nr=nr, nz=nz, R=R, d=d, z=z, V_cathode=V_cathode, V_anode=0.0,
                     mu_e=30.0, D_e=60.0, mu_p=0.15, D_p=0.0038,
                     pressure_factor=pressure_factor,
                     table=transport_table(table_seed) if use_table else None,
                     S_e=S.copy(), S_p=S.copy(), ne0=ne0, np0=np0, V0=V0, seed=seed)


# --- the paper's argon discharge (Sec. 3) ----------------------------------------------
ARGON_P_TORR = 0.514           # pd = 75 Pa cm at d = 1.1 cm
ARGON_MU_P = 0.22              # stand-in ion mobility (m^2 / V s): the paper's value comes from
                               # its ref. [7] and is not printed


def argon_sources(r, z, R, L, a, b):
    """The analytic source terms of Sec. 3 (m^-3 s^-1) with the length scale L = d."""
    rr, zz = np.meshgrid(r, z)
    x = zz / L
    radial = 1.0 / (1.0 + np.exp(a * rr / R - b))
    S_p = 0.35e22 * x ** 2 * np.exp(-50.0 * x ** 8) * radial
    S_e = 1.75e22 * (x - 0.5) * np.exp(-40.0 * (x - 0.5) ** 2) * (x > 0.5) * radial
    return S_e, S_p


def argon(n: int, a: float = 30.0, b: float = 24.0) -> Discharge:
    """The glow discharge of Sec. 3 on an (n+1)^2 node grid: d = 1.1 cm, R = 2.7 cm, p = 0.514
    torr, V = 0 at z = 0 (cathode) and 255.9 V at z = d, Dirichlet walls (n = 0, V linear in z),
    mu_e = 30 / p, D_e = mu_e x 1 V, D_p = mu_p x 0.026 V (the printed "D_e" of the ion line read
    as D_p), the analytic sources with (a, b) = (30, 24) or (10, 1); z stretched as the other
    workloads; initial densities the other workloads' Gaussian, zero on the wall."""
    if n < 2 or (n & (n - 1)):
        raise ValueError("N must be a power of two >= 2")
    R, d = 2.7e-2, 1.1e-2
    z = z_nodes(n, d)
    r = r_nodes(n, R)
    S_e, S_p = argon_sources(r, z, R, d, a, b)
    ne0, np0, V0 = initial_state(r, z, R, d, 0.0, 255.9)
    ne0[:, -1] = 0.0
    np0[:, -1] = 0.0
    mu_e = 30.0 / ARGON_P_TORR
    return Discharge(nr=n, nz=n, R=R, d=d, z=z, V_cathode=0.0, V_anode=255.9,
                     mu_e=mu_e, D_e=mu_e * 1.0, mu_p=ARGON_MU_P, D_p=ARGON_MU_P * 0.026,
                     pressure_factor=1.0, table=None, S_e=S_e, S_p=S_p, ne0=ne0, np0=np0, V0=V0,
                     seed=0, wall_dirichlet=True)


# --- the five workloads -------------------------------------------------------------

def transient_33(seed: int = 0) -> Discharge:
    """33 x 33 nodes, constant transport, -200 V; 10 backward-Euler steps of 1 ns."""
    return make_discharge(32, seed=seed, V_cathode=-200.0)


def steady_257(seed: int = 0) -> Discharge:
    """257 x 257 nodes, -300 V, field-dependent transport table (seed 2); steady state."""
    return make_discharge(256, seed=seed, V_cathode=-300.0, use_table=True)


def transient_1025(seed: int = 0) -> Discharge:
    """1025 x 1025 nodes with the 33 x 33 case's physics (mixed-precision workload)."""
    return make_discharge(1024, seed=seed, V_cathode=-200.0)


def batch_64(seed: int = 4, count: int = 64, sizes=(64, 128, 256, 512)) -> List[Discharge]:
    """Independent discharges of seeded sizes, cathode voltages and pressure factors."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(sizes[rng.integers(0, len(sizes))])
        vc = float(rng.uniform(-400.0, -150.0))
        pf = float(rng.uniform(0.5, 2.0))
        out.append(make_discharge(n, seed=seed * 100003 + k, V_cathode=vc, pressure_factor=pf))
    return out


def unet_sample_params(seed: int):
    """Parameters of one learned-guess training / test instance (ranges of the batch workload)."""
    rng = np.random.default_rng(seed)
    return dict(V_cathode=float(rng.uniform(-400.0, -150.0)),
                pressure_factor=float(rng.uniform(0.5, 2.0)))
