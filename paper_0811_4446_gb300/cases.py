"""Small fixed workloads for profiling runs (ncu captures of single kernels).

    python -m paper_0811_4446_gb300.cases vcycles N [CYCLES] [--mixed] [--eager] [--autotune] [--half] [--line | --rline | --alt]
    python -m paper_0811_4446_gb300.cases unet B N [REPS] [--mma | --gather | --tma | --halo] [--eager]
    python -m paper_0811_4446_gb300.cases steady [--mixed] [--eager]
    python -m paper_0811_4446_gb300.cases batch COUNT [--fp64]

builds the N x N-node discharge of the benchmark family (table transport for N = 256),
evaluates the Newton residual at the initial state and runs CYCLES multigrid V-cycles
(default 3) on the linearised system (eq. 14) at Delta t = 1e-6 s.  Smoother launches per
V-cycle and level: nu1 sweeps on the way down and nu2 on the way up (one launch per fused
sweep, two per half-sweep pair, as the autotuner chose for the level), finest level first.
--eager launches the V-cycle kernels from the host instead of the device-side graph loop
(kernel profilers cannot attribute kernels inside graphs with conditional nodes).
--autotune picks the smoother launch shapes and fused / half sweeps per level as the
benchmark does (its timing launches come before the V-cycles).  The linear solve (its
residual, hierarchy set-up and V-cycles) runs inside the NVTX range "measure".  --half
smooths with two half-sweep launches per sweep on every level (no fused sweeps); --line
uses the z-line zebra smoother (on a grid with R = 10 d, dr = 10 dz, where it pays); --rline the
r-line one and --alt alternating z- and r-lines (on a grid with R = d / 5, dz = 5 dr, where r-lines
pay).

steady: one steady solve of the benchmark's 257 x 257 workload (129 -> 257 continuation,
table transport, rho <= 1e-8) after one untimed solve, autotuned as the benchmark does, inside
the NVTX range "measure"; --eager launches every kernel from the host (no graphs), so that a
kernel profiler sees each launch of the solve.

batch: the persistent batched form (one launch of the work-list kernel) on COUNT discharges of
the batched workload's family with sizes 33^2 to 129^2 (seed 4), mixed precision (--fp64: FP64),
after one untimed batch, inside the NVTX range "measure".

unet: REPS (default 2) forward passes plus one training step of the learned-guess network
on a batch of B random (N+1) x (N+1) inputs; --mma selects the mma.sync convolutions instead
of the tcgen05 ones, --gather the thread-gathered tcgen05 forward convolutions instead of the
TMA-fed ones, --tma the TMA-fed ones without the halo loads (default, --halo: with them); --eager launches kernel by
kernel instead of the per-batch-size CUDA graphs (kernel profilers cannot attribute the graphs'
launches).
"""
from __future__ import annotations

import os
import sys


def vcycles(n: int, cycles: int = 3, mixed: bool = False, eager: bool = False, autotune: bool = False,
            half: bool = False, line: int = 0) -> float:
    import torch

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import workloads as W
    from . import mg

    R = {0: 1e-2, 1: 0.1, 2: 2e-3, 3: 2e-3}[line]
    d = W.make_discharge(n, seed=0, V_cathode=-300.0, use_table=(n == 256), R=R)
    s = mg.from_discharge(d, precision=mg.MG_MIXED if mixed else mg.MG_FP64, use_graphs=0 if eager else 1,
                          fused_sweep=0 if half else 1, line_smoother=line)
    if autotune:
        s.autotune()
    F, _ = s.residual(1e-6)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("measure")  # profilers can select the launches inside this range
    _, hist, _ = s.linear_solve(1e-6, [-a for a in F], 0.0, cycles)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    return float(hist[-1])


def steady(mixed: bool = False, eager: bool = False) -> float:
    import numpy as np
    import torch

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import workloads as W
    from . import mg

    d = W.steady_257()
    s = mg.from_discharge(d, precision=mg.MG_MIXED if mixed else mg.MG_FP64, use_graphs=0 if eager else 1)
    s.autotune()
    ins = [np.ascontiguousarray(a) for a in (d.ne0, d.np0, d.V0)]
    s.set_state(*ins)
    s.solve_steady(1e-8)
    s.set_state(*ins)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("measure")
    rc, st = s.solve_steady(1e-8)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if rc != mg.MG_OK:
        raise RuntimeError(f"steady solve failed: {rc}")
    return float(st["steady_rho"])


def batch(count: int, fp64: bool = False) -> int:
    import numpy as np
    import torch

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import workloads as W
    from . import mg

    ds = W.batch_64(seed=4, count=count, sizes=(32, 64, 128))
    sv = [mg.from_discharge(d, precision=mg.MG_FP64 if fp64 else mg.MG_MIXED, stream=torch.cuda.Stream()) for d in ds]
    ins = [[np.ascontiguousarray(a) for a in (d.ne0, d.np0, d.V0)] for d in ds]
    mg.solve_steady_batch(sv, 1e-8, workers=0)
    for s, i in zip(sv, ins):
        s.set_state(*i)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("measure")
    rc, _, _ = mg.solve_steady_batch(sv, 1e-8, workers=0)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if rc != mg.MG_OK:
        raise RuntimeError(f"batched solve failed: {rc}")
    return count


def unet_case(B: int, n: int, reps: int = 2, mma: bool = False, gather: bool = False, tma: bool = False,
              eager: bool = False) -> float:
    import numpy as np
    import torch
    from . import unet

    rng = np.random.default_rng(0)
    x = torch.from_numpy(rng.standard_normal((B, n + 1, n + 1, 8)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((B, n + 1, n + 1, 3)).astype(np.float32)).cuda()
    net = unet.UNet(B, n)
    net.set_tensor_path(0 if mma else (1 if gather else (2 if tma else 3)))
    if eager:
        net.set_graphs(False)
    net.set_params(unet.init_params(0))
    ysum = 0.0
    for _ in range(reps):
        ysum += float(net.forward(x).abs().mean())
    loss = net.train_step(x, t, 1e-4)
    torch.cuda.synchronize()
    net.close()
    return float(loss) + ysum


if __name__ == "__main__":
    if len(sys.argv) >= 4 and sys.argv[1] == "unet":
        R = int(sys.argv[4]) if len(sys.argv) > 4 and not sys.argv[4].startswith("--") else 2
        print("ok", unet_case(int(sys.argv[2]), int(sys.argv[3]), R, "--mma" in sys.argv, "--gather" in sys.argv,
                                "--tma" in sys.argv, "--eager" in sys.argv))
        sys.exit(0)
    if len(sys.argv) >= 3 and sys.argv[1] == "batch":
        print("ok", batch(int(sys.argv[2]), "--fp64" in sys.argv))
        sys.exit(0)
    if len(sys.argv) >= 2 and sys.argv[1] == "steady":
        print("ok", steady("--mixed" in sys.argv, "--eager" in sys.argv))
        sys.exit(0)
    if len(sys.argv) < 3 or sys.argv[1] != "vcycles":
        print(__doc__)
        sys.exit(2)
    N = int(sys.argv[2])
    C = int(sys.argv[3]) if len(sys.argv) > 3 and not sys.argv[3].startswith("--") else 3
    print("ok", N, vcycles(N, C, "--mixed" in sys.argv, "--eager" in sys.argv, "--autotune" in sys.argv,
                           "--half" in sys.argv,
                           1 if "--line" in sys.argv else 2 if "--rline" in sys.argv else 3 if "--alt" in sys.argv else 0))
