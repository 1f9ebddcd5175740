"""Time the FP32 Riemann-state kernel in each reconstruction mode on one state (for profiling).

    python -m paper_2401_16543_gb300.recon_modes [--n 1024] [--reps 30]

On the 2D radius-2 Voronoi state (64 regions, seed 2, outflow) it times ``kfvm_reconstruct`` with the
library's own event tracing ("profile" 1), L2 flushed between calls, in: the fused learned gate
("recon" 2), the same decisions from a caller mask (the gate's own ``kfvm_gate_mask``, "recon" 3), that
mask without the positivity limiter, linear everywhere ("recon" 1) with and without the limiter,
KXRCF ("recon" 4, the mask kernel and the masked reconstruction) and WENO-AO everywhere ("recon" 0).
The differences split the headline kernel's time into gate, limiter, WENO-AO and linear parts.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def main() -> None:
    import torch

    import workloads
    from paper_2401_16543_gb300 import KFVM

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--reps", type=int, default=30)
    args = ap.parse_args()
    n = args.n
    U0 = workloads.voronoi_2d(n, k=64, seed=2, device="cuda").contiguous()
    params = np.load(os.path.join(HERE, "gate_params_2d.npy"))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def run(label, recon, positivity=1):
        g = KFVM([n, n], dims=2, radius=2, bc="outflow")
        g.set_option("precision", 32)
        g.gate_set_params(params)
        g.set_option("gate_threshold", 0.8)
        g.set_option("recon", 2)
        m = g.gate_mask(U0)
        if recon == 3:
            g.set_smooth_mask(m)
        else:
            g.set_option("recon", recon)
        g.set_option("positivity", positivity)
        faces = g.reconstruct(U0)
        torch.cuda.synchronize()
        g.set_option("profile", 1)
        g.profile_reset()
        for _ in range(args.reps):
            flush.zero_()
            g.reconstruct(U0, faces)
        torch.cuda.synchronize()
        p = g.profile()
        per = {k: v[1] / v[0] * 1e3 for k, v in p.items() if k != "shadow"}
        g.sync_status()
        print(f"{label:34s} " + "  ".join(f"{k} {v:7.1f} us" for k, v in per.items())
              + (f"   (linear cells {float(m.float().mean()):.3f})" if recon in (2, 3) else ""), flush=True)

    run("gated (recon 2)", 2)
    run("gate's mask (recon 3)", 3)
    run("gate's mask, limiter off", 3, 0)
    run("linear everywhere (recon 1)", 1)
    run("linear everywhere, limiter off", 1, 0)
    run("KXRCF (recon 4)", 4)
    run("WENO-AO everywhere (recon 0)", 0)


if __name__ == "__main__":
    main()
