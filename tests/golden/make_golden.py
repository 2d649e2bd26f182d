"""Writes tests/golden/oracle_transient_33.json from the FP64 oracle only.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import discretization as disc  # noqa: E402
from oracle import solver as so  # noqa: E402
from oracle.grid import Grid  # noqa: E402


def main():
    d = W.transient_33()
    g = Grid(d.nr, d.nz, d.R, d.z)
    phys = disc.Physics(V_cathode=d.V_cathode)
    u = np.stack([d.ne0, d.np0, d.V0])
    opt = so.SolverOptions(eta=1e-12)
    out = {"workload": "33x33 nodes, -200 V, seed 0, 10 steps of 1 ns, rho <= 1e-10",
           "steps": 10, "dt": 1e-9, "tol": 1e-10, "probe_j": 16, "probe_i": 3}
    for _ in range(out["steps"]):
        u, st = so.step(g, u, d.S_e, d.S_p, out["dt"], phys, out["tol"], opt)
        assert st.accepted
    for k, name in enumerate(("ne", "np", "V")):
        out[name + "_l1"] = float(np.abs(u[k]).sum())
        out[name + "_probe"] = float(u[k][out["probe_j"], out["probe_i"]])
    with open(os.path.join(ROOT, "tests", "golden", "oracle_transient_33.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
