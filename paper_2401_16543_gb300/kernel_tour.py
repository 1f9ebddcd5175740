"""Run every kernel of the library once on small synthetic grids (for profilers).

    python -m paper_2401_16543_gb300.kernel_tour

Launches, in order: the FP64 path (build_weights, max_rate, recon64, flux_update), the flux-only
entry (face_flux, update) and recon64 in characteristic variables on 2D 256^2; the FP32 path in 3D radius 2 (shadow, recon32<3,2>,
flux_update, and recon32<3,2> in characteristic variables) on 48^3; 3D radius 3 on 32^3 (recon33 on the FP32 pipe, recon33_tc on the tensor
cores, label33); the learned gate (features, label, forward, mask, train, adam) and the KXRCF
indicator (float64 and float32) on the 2D grid.
Every computation goes through the C ABI; results are not checked here (the tests do that).
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def main() -> None:
    import torch

    import workloads
    from paper_2401_16543_gb300 import KFVM

    dev = "cuda"
    # FP64 path, 2D radius 2
    U2 = workloads.voronoi_2d(256, k=16, seed=2, device=dev).contiguous()
    g = KFVM([256, 256], dims=2, radius=2, bc="outflow")
    g.step(U2.clone(), 0.4)
    faces = g.reconstruct(U2)
    g.flux(faces)
    # WENO-AO in characteristic variables (Sec. 3.4.1), FP64
    g.set_option("variables", 1)
    g.reconstruct(U2)
    g.set_option("variables", 0)
    # the gate on the 2D grid (features + labels, forward, training step, the mask of the gated step)
    g.set_option("precision", 32)
    g.gate_set_params(np.load(os.path.join(HERE, "gate_params_2d.npy")))
    X, y = g.gate_features(U2, 0.5)
    g.gate_forward(X[:65536].contiguous())
    g.gate_train_step(X[:16384].contiguous(), y[:16384].contiguous(), 0.0)
    g.set_option("precision", 64)
    g.set_option("recon", 2)
    g.gate_mask(U2)
    # the KXRCF troubled-cell indicator (Sec. 3.5) in both precisions
    g.kxrcf_mask(U2)
    g.set_option("precision", 32)
    g.kxrcf_mask(U2)
    g.set_option("precision", 64)
    # FP32 path, 3D radius 2
    U3 = workloads.half_sine_voronoi_3d(48, k=8, seed=3, device=dev).contiguous()
    h = KFVM([48, 48, 48], dims=3, radius=2, bc="periodic")
    h.set_option("precision", 32)
    h.step(U3.clone(), 0.4)
    h.set_option("variables", 1)
    h.reconstruct(U3)
    h.set_option("variables", 0)
    # 3D radius 3: FP32 pipe, tensor cores, labels
    V = workloads.mixed_voronoi(3, 32, 4, seed=5, R=3, device=dev).contiguous()
    t = KFVM([32, 32, 32], dims=3, radius=3, bc="outflow")
    t.set_option("precision", 32)
    t.set_option("tensor_cores", 0)
    t.reconstruct(V)
    t.set_option("tensor_cores", 1)
    t.reconstruct(V)
    t.gate_features(V, 0.5)
    torch.cuda.synchronize()
    for solver in (g, h, t):
        solver.sync_status()
    print("kernel tour done")


if __name__ == "__main__":
    main()
