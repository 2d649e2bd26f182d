"""Trains the learned-initial-guess network on solver-generated steady states (on the GPU).

    python -m paper_0811_4446_gb300.train_guess [--samples 2000] [--epochs 20] [--batch 16]
                                                [--n 256] [--out PATH] [--eval 8]

1. Generates `samples` steady states of the learned-guess family (seeds 1000, 1001, ...:
   cathode voltage U[-400, -150] V, pressure factor U[0.5, 2], own Gaussian source) with the
   batched mixed-precision solver (rho <= 1e-8).
2. Trains the U-Net of include/unet.h with Adam (cosine decay) on the device.
3. Writes the FP32 parameter vector to --out and evaluates time-to-1e-8 from the guess against
   the plain continuation on `eval` held-out seeds (9000, 9001, ...).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--out", default="unet_guess_257.f32")
    ap.add_argument("--eval", type=int, default=8)
    args = ap.parse_args()

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import numpy as np
    import torch
    from . import build, mg, unet

    build.build()
    report = {"samples": args.samples, "epochs": args.epochs, "batch": args.batch, "n": args.n}
    t0 = time.perf_counter()
    X, T = unet.generate(list(range(1000, 1000 + args.samples)), n=args.n)
    report["generate_s"] = time.perf_counter() - t0
    report["generated"] = int(X.shape[0])
    print(f"generated {X.shape[0]} steady states in {report['generate_s']:.1f} s", flush=True)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    del X, T
    net = unet.UNet(args.batch, args.n)
    net.set_params(unet.init_params(0))
    t0 = time.perf_counter()
    hist = unet.train(net, Xd, Td, args.epochs, args.batch, args.lr,
                      log=lambda ep, l: print(f"epoch {ep} loss {l:.5f}", flush=True))
    torch.cuda.synchronize()
    report["train_s"] = time.perf_counter() - t0
    report["loss"] = hist
    p = net.get_params()
    p.tofile(args.out)
    # held-out evaluation: guess + refine vs continuation (mixed precision both)
    net1 = unet.UNet(1, args.n)
    net1.set_params(p)
    rows = []
    for seed in range(9000, 9000 + args.eval):
        d = unet.guess_discharge(seed, args.n)
        c = mg.from_discharge(d, precision=mg.MG_MIXED)
        torch.cuda.synchronize()
        b = time.perf_counter()
        rc2, st2 = c.solve_steady(1e-8)
        torch.cuda.synchronize()
        e = time.perf_counter()
        ref = np.stack(c.get_state())
        row = {"seed": seed, "continuation_ms": 1e3 * (e - b), "cont_steps": st2["steps_accepted"]}
        y = net1.forward(unet.features(d)[None])[0]
        g = unet.state_from_output(y, d.V_cathode)
        row["guess_max_rel_err"] = [float(np.abs(g[q] - ref[q]).max() / np.abs(ref[q]).max()) for q in range(3)]
        for level in (0, 1):
            s = mg.from_discharge(d, precision=mg.MG_MIXED, guess_level=level, guess_dt_max=1e-6)
            torch.cuda.synchronize()
            a = time.perf_counter()
            y = net1.forward(unet.features(d)[None])[0]
            rc, st, fb = s.solve_steady_guess(*unet.state_from_output(y, d.V_cathode), 1e-8)
            torch.cuda.synchronize()
            t = time.perf_counter() - a
            row[f"guess_level{level}"] = {"ms": 1e3 * t, "fallback": fb, "steps": st["steps_accepted"],
                                         "rejected": st["steps_rejected"], "rc": rc}
        rows.append(row)
        print(row, flush=True)
    report["eval"] = rows
    for level in (0, 1):
        report[f"median_speedup_level{level}"] = float(np.median(
            [r["continuation_ms"] / r[f"guess_level{level}"]["ms"] for r in rows]))
    print(json.dumps(report), flush=True)


if __name__ == "__main__":
    main()
