"""Small fixed workloads for profiling runs (ncu captures of single kernels).

    python -m paper_0811_4446_gb300.cases vcycles N [CYCLES] [--mixed] [--eager]

builds the N x N-node discharge of the benchmark family (table transport for N = 256),
evaluates the Newton residual at the initial state and runs CYCLES multigrid V-cycles
(default 3) on the linearised system (eq. 14) at Delta t = 1e-6 s.  Smoother launches per
V-cycle: 4 per level on the way down, 4 per level on the way up, finest level first.
--eager launches the V-cycle kernels from the host instead of the device-side graph loop
(kernel profilers cannot attribute kernels inside graphs with conditional nodes).
"""
from __future__ import annotations

import os
import sys


def vcycles(n: int, cycles: int = 3, mixed: bool = False, eager: bool = False) -> float:
    import torch

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import workloads as W
    from . import mg

    d = W.make_discharge(n, seed=0, V_cathode=-300.0, use_table=(n == 256))
    s = mg.from_discharge(d, precision=mg.MG_MIXED if mixed else mg.MG_FP64, use_graphs=0 if eager else 1)
    F, _ = s.residual(1e-6)
    _, hist, _ = s.linear_solve(1e-6, [-a for a in F], 0.0, cycles)
    torch.cuda.synchronize()
    return float(hist[-1])


if __name__ == "__main__":
    if len(sys.argv) < 3 or sys.argv[1] != "vcycles":
        print(__doc__)
        sys.exit(2)
    N = int(sys.argv[2])
    C = int(sys.argv[3]) if len(sys.argv) > 3 and not sys.argv[3].startswith("--") else 3
    print("ok", N, vcycles(N, C, "--mixed" in sys.argv, "--eager" in sys.argv))
