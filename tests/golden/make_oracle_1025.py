"""Writes tests/golden/oracle_transient_1025.npz from the FP64 oracle only: ten backward-Euler
steps of 1 ns on the 1025 x 1025-node workload (the 33^2 physics: constant transport, -200 V,
Gaussian source, seed 0), each solved by Newton-Raphson with multigrid to rho <= 1e-10, the
oracle's default options (the same algorithm the library runs).

Stored: the state after the first and the last step at every 8th node in both directions
(129 x 129 per field; `sample_steps` names the steps), the exact max-norm of each field over all
nodes after every step, and per step the Newton iterations, V-cycles and final rho.  The 1025^2
oracle takes minutes per step; the stride and the two sampled steps keep the file small.

Run from the repository root:  python tests/golden/make_oracle_1025.py   (about 15 minutes)
"""
import os
import sys
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import discretization as disc  # noqa: E402
from oracle import solver as so  # noqa: E402
from oracle.grid import Grid  # noqa: E402

STRIDE = 8
STEPS = 10
SAMPLE_STEPS = (1, STEPS)
DT = 1e-9
TOL = 1e-10


def main():
    d = W.transient_1025()
    g = Grid(d.nr, d.nz, d.R, d.z)
    phys = disc.Physics(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p,
                        D_p=d.D_p, table=d.table, pressure_factor=d.pressure_factor)
    u = np.stack([d.ne0, d.np0, d.V0])
    samples, norms, newton, vcycles, rho, secs = [], [], [], [], [], []
    for k in range(STEPS):
        t0 = time.perf_counter()
        u, st = so.step(g, u, d.S_e, d.S_p, DT, phys, TOL, so.SolverOptions())
        assert st.accepted, st
        secs.append(time.perf_counter() - t0)
        if k + 1 in SAMPLE_STEPS:
            samples.append(u[:, ::STRIDE, ::STRIDE].copy())
        norms.append(np.abs(u).reshape(3, -1).max(axis=1))
        newton.append(st.newton)
        vcycles.append(list(st.vcycles))
        rho.append(st.rho)
        print(f"step {k + 1}: {st.newton} Newton, V-cycles {st.vcycles}, rho {st.rho}, {secs[-1]:.1f} s", flush=True)
    vc = np.zeros((STEPS, max(len(v) for v in vcycles)), dtype=np.int32)
    for k, v in enumerate(vcycles):
        vc[k, :len(v)] = v
    np.savez_compressed(os.path.join(ROOT, "tests", "golden", "oracle_transient_1025.npz"),
                        stride=STRIDE, dt=DT, tol=TOL, sample_steps=np.array(SAMPLE_STEPS, dtype=np.int32),
                        samples=np.stack(samples), norms=np.stack(norms),
                        newton=np.array(newton, dtype=np.int32), vcycles=vc, rho=np.stack(rho),
                        seconds=np.array(secs))


if __name__ == "__main__":
    main()
