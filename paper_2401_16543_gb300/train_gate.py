"""Train the smooth-cell gate on the GPU with the library's own kernels.

Training pairs come from the method itself: for every cell of a state, the
gate features (radius-2 stencil of rho and p, shape-normalised) and the label
"the cell's own WENO-AO weights keep omega_0/gamma_0 >= 1 - tau in every
linearized primitive component" (kfvm_gate_features).  States are taken along
runs of the two 2D workloads:

* the smooth translation on 64^2 cells (periodic, CFL 0.4, to t = 0.1): every step;
* the 1024^2 Voronoi state (64 regions, seed 2, outflow, CFL 0.4): every 20th
  of 200 SSP-RK3 steps.

From the pooled pairs, `--pairs` are drawn with seed 41 (the last 5% held out);
the network is trained by kfvm_gate_train_step (BF16 forward/backward on the
tensor cores, FP32 accumulation, Adam on FP32 masters; 20 epochs of batches of
2048, learning rate 1e-3 stepped down to 3.3e-4 and 1e-4: smaller batches than
the GPU could take give more steps and a better-separated (more confident)
network at the same data).  The result is written
as float32 .npy in the packing of kfvm_gate_set_params.

    python -m paper_2401_16543_gb300.train_gate --out paper_2401_16543_gb300/gate_params_2d.npy

3D (radius-3 labels; the radius-2 stencils of rho and p plus the two radius-3 shell
inputs): pairs from smooth runs on 24^3 ... 64^3 cells and two 128^3 Voronoi runs
(generate_3d), all of them used, written to gate_params_3d.npy:

    python -m paper_2401_16543_gb300.train_gate --dims 3 --radius 3 --pairs 36000000
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

DEFAULT_OUT = {2: os.path.join(HERE, "gate_params_2d.npy"), 3: os.path.join(HERE, "gate_params_3d.npy")}


def init_params(n_in: int, seed: int) -> np.ndarray:
    """He initialisation (seeded): W1 [32][n_in], b1, W2 [32][32], b2, W3 [32], b3."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / n_in), (32, n_in))
    W2 = rng.normal(0, np.sqrt(2.0 / 32), (32, 32))
    W3 = rng.normal(0, np.sqrt(1.0 / 32), 32)
    return np.concatenate([W1.ravel(), np.zeros(32), W2.ravel(), np.zeros(32), W3, [0.0]]).astype(np.float32)


def generate(tau: float, voronoi_n: int = 1024, voronoi_steps: int = 200, every: int = 20, device="cuda"):
    """Pooled (X, y) device tensors from the two workload runs."""
    import torch

    import workloads
    from paper_2401_16543_gb300 import KFVM
    Xs, ys = [], []
    # smooth translation, 64^2, periodic
    g = KFVM([64, 64], dims=2, radius=2, bc="periodic")
    g.set_option("precision", 32)
    U = workloads.sine_2d(64, device=device).contiguous()
    t = 0.0
    while t < 0.1:
        X, y = g.gate_features(U, tau)
        Xs.append(X)
        ys.append(y)
        t += g.step(U, 0.4, 0.1 - t)
    # Voronoi, outflow
    g = KFVM([voronoi_n, voronoi_n], dims=2, radius=2, bc="outflow")
    g.set_option("precision", 32)
    U = workloads.voronoi_2d(voronoi_n, k=64, seed=2, device=device).contiguous()
    for k in range(voronoi_steps + 1):
        if k % every == 0:
            X, y = g.gate_features(U, tau)
            Xs.append(X)
            ys.append(y)
        if k < voronoi_steps:
            g.step(U, 0.4)
    return torch.cat(Xs), torch.cat(ys)


def generate_3d(tau: float, n: int = 128, steps: int = 30, every: int = 6, R: int = 3, device="cuda"):
    """Pooled (X, y) from 3D runs at radius R, FP32 WENO-AO everywhere, CFL 0.4:
    the smooth translation on 24^3 ... 64^3 cells (periodic, to t = 0.05), the
    half-sine / half-Voronoi state (16 regions in x >= 1/2, seed 3, periodic) and the
    mixed state (16 regions, each smooth or constant, seed 5, outflow) on n^3 cells,
    features and labels of every `every`-th of `steps` SSP-RK3 steps."""
    import torch

    import workloads
    from paper_2401_16543_gb300 import KFVM
    Xs, ys = [], []
    # the smooth translation at several resolutions (the sine's phase step per cell changes the
    # shape of a normalised stencil); snapshots thinned so that each resolution gives ~1-2 M pairs
    for ns, every_s in ((24, 1), (32, 1), (48, 2), (64, 4)):
        g = KFVM([ns] * 3, dims=3, radius=R, bc="periodic")
        g.set_option("precision", 32)
        U = workloads.sine_3d(ns, R=R, device=device).contiguous()
        t, k = 0.0, 0
        while t < 0.05:
            if k % every_s == 0:
                X, y = g.gate_features(U, tau)
                Xs.append(X)
                ys.append(y)
            t += g.step(U, 0.4, 0.05 - t)
            k += 1
        del U, g
    for make, bc in ((lambda: workloads.half_sine_voronoi_3d(n, k=16, seed=3, R=R, device=device), "periodic"),
                     (lambda: workloads.mixed_voronoi(3, n, 16, seed=5, R=R, device=device), "outflow")):
        g = KFVM([n, n, n], dims=3, radius=R, bc=bc)
        g.set_option("precision", 32)
        U = make().contiguous()
        for k in range(steps + 1):
            if k % every == 0:
                X, y = g.gate_features(U, tau)
                Xs.append(X)
                ys.append(y)
            if k < steps:
                g.step(U, 0.4)
        del U, g
    return torch.cat(Xs), torch.cat(ys)


def train(X, y, pairs: int, epochs: int, batch: int, lr: float, seed: int = 41, init_seed: int = 0,
          log=print):
    """Train on `pairs` samples drawn with `seed`; returns (params, held-out metrics, loss history)."""
    import torch

    from paper_2401_16543_gb300 import KFVM
    gen = torch.Generator(device=X.device)
    gen.manual_seed(seed)
    idx = torch.randperm(X.shape[0], generator=gen, device=X.device)
    if pairs < idx.numel():
        idx = idx[:pairs]
    else:
        reps = (pairs + idx.numel() - 1) // idx.numel()
        idx = torch.cat([idx] * reps)[:pairs]
    n_hold = max(1, pairs // 20)
    tr, ho = idx[:-n_hold], idx[-n_hold:]
    Xtr, ytr = X[tr].contiguous(), y[tr].contiguous()
    Xho, yho = X[ho].contiguous(), y[ho].contiguous()
    dims = 2 if X.shape[1] == 26 else 3
    g = KFVM([8] * dims, dims=dims, radius=2)
    g.gate_set_params(init_params(X.shape[1], init_seed))
    loss = torch.zeros(1, dtype=torch.float32, device=X.device)
    hist = []
    for ep in range(epochs):
        # step schedule: full rate for 60% of the epochs, then 1/3, then 1/10
        lr_ep = lr if ep < 0.6 * epochs else (lr / 3 if ep < 0.9 * epochs else lr / 10)
        perm = torch.randperm(Xtr.shape[0], generator=gen, device=X.device)
        acc, nb = 0.0, 0
        for s in range(0, Xtr.shape[0], batch):
            b = perm[s:s + batch]
            g.gate_train_step(Xtr[b].contiguous(), ytr[b].contiguous(), lr_ep, loss=loss)
            if nb % 50 == 0:
                acc += float(loss.item())
            nb += 1
        hist.append(acc / max(1, (nb + 49) // 50))
        log(f"epoch {ep}: mean batch loss {hist[-1]:.5f}")
    prob = g.gate_forward(Xho)
    lab = yho > 0.5
    metrics = {"held_out": int(n_hold), "smooth_fraction_label": float(lab.float().mean().item()), "thresholds": {}}
    for th in (0.5, 0.7, 0.8, 0.9):
        pred = prob > th
        metrics["thresholds"][str(th)] = {
            "accuracy": float((pred == lab).float().mean().item()),
            "false_smooth_rate": float((pred & ~lab).float().sum().item() / max(1.0, (~lab).float().sum().item())),
            "false_weno_rate": float((~pred & lab).float().sum().item() / max(1.0, lab.float().sum().item())),
            "predicted_smooth_fraction": float(pred.float().mean().item()),
        }
    return g.gate_get_params(), metrics, hist


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, default=2, choices=(2, 3))
    ap.add_argument("--radius", type=int, default=3, help="3D only: radius of the labelling WENO-AO")
    ap.add_argument("--out", default=None)
    ap.add_argument("--pairs", type=int, default=10_000_000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=2048)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--tau", type=float, default=0.5)
    args = ap.parse_args()
    t0 = time.time()
    X, y = generate(args.tau) if args.dims == 2 else generate_3d(args.tau, R=args.radius)
    print(f"generated {X.shape[0]} pairs in {time.time() - t0:.1f} s; smooth label fraction {y.mean().item():.3f}")
    t1 = time.time()
    params, metrics, hist = train(X, y, args.pairs, args.epochs, args.batch, args.lr)
    metrics["train_seconds"] = time.time() - t1
    metrics["loss_history"] = hist
    np.save(args.out or DEFAULT_OUT[args.dims], params.astype(np.float32))
    print(json.dumps(metrics))


if __name__ == "__main__":
    main()
