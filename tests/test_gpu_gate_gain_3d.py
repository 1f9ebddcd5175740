"""What the trained 3D gate gains at radius 3 (the 512^3 workload's scheme), on small grids.

The shipped parameters (paper_2401_16543_gb300/gate_params_3d.npy, trained on the
GPU by ``train_gate.py --dims 3 --radius 3`` with radius-3 WENO-AO labels) are used
at threshold 0.8, in the mixed-precision path.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads  # noqa: E402

PARAMS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2401_16543_gb300",
                      "gate_params_3d.npy")


@pytest.fixture(scope="module")
def kfvm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(PARAMS):
        pytest.skip("no trained 3D gate parameters")
    import paper_2401_16543_gb300 as pkg
    return pkg


def _gated(kfvm, n, bc, tc=1):
    g = kfvm.KFVM([n] * 3, dims=3, radius=3, bc=bc)
    g.set_option("precision", 32)
    g.set_option("tensor_cores", tc)
    g.gate_set_params(np.load(PARAMS))
    g.set_option("gate_threshold", 0.8)
    g.set_option("recon", 2)
    return g


@pytest.mark.parametrize("tc,bound", [(0, 1.1), (1, 1.15)])
def test_smooth_translation_3d_gated_error_known_gap_within_15pct_of_fp64_weno(kfvm, tc, bound):
    """A KNOWN GAP, recorded: at radius 3 in 3D the matched-L1 target (gated mixed path's L1 density
    error within 1e-6 relative of the plain FP64 WENO-AO path's on smooth data) is NOT met.

    32^3 sine translation (periodic) to t = 0.05: the gated mixed path's L1 density error against
    the exact solution, relative to the plain FP64 WENO-AO path's.  In 3D at radius 3 the shipped
    gate sends only part of the smooth cells (about a quarter here) to the linear reconstruction:
    its training labels come from radius-3 WENO-AO weights, which call much of an evolving 3D flow
    non-smooth, and its inputs see radius 2 plus a summary of the radius-3 shell.  A field that
    mixes linear and WENO-AO cells measures 8% (FP32-pipe contraction) / 11% (tensor-core
    contraction) above the all-WENO error; this test bounds that gap at 10% / 15%.  The cause is
    the linear operator: at radius 3 in 3D the linear S0 reconstruction is not stable (von Neumann
    symbol of the oracle's weights, which an independent 40-digit solve pins: max Re lambda Delta
    = +7.5; all cells linear diverge, test_gpu_kxrcf.py), so linear cells in smooth regions lean
    on the WENO-AO cells around them and cannot bring the 2D gate's ~10x gain."""
    n, t_end = 32, 0.05
    U0 = workloads.sine_3d(n)
    ex = workloads.sine_3d_exact_density(n, t_end)
    g64 = kfvm.KFVM([n] * 3, dims=3, radius=3)
    U64 = U0.cuda()
    g64.run(U64, 0.4, t_end)
    gg = _gated(kfvm, n, "periodic", tc)
    assert gg.gate_mask(U0.cuda()).float().mean().item() > 0.0
    Ug = U0.cuda()
    gg.run(Ug, 0.4, t_end)
    e64 = np.abs(U64[0].cpu().numpy() - ex).mean()
    eg = np.abs(Ug[0].cpu().numpy() - ex).mean()
    print(f"3D gated L1 error / FP64 WENO-AO error (tensor cores {tc}): {eg / e64:.4f}")
    assert eg <= e64 * bound, (eg, e64)


def test_mixed_voronoi_3d_gated_stays_close_to_weno_everywhere(kfvm):
    """64^3 mixed smooth/constant Voronoi state (outflow), 10 steps: the gated mixed path stays
    admissible and within 2% (L1 of rho, relative) of FP64 WENO-AO everywhere, with the gate sending
    a share of the cells to the linear reconstruction (in 3D at radius 3 the WENO-AO weights of an
    evolving Voronoi state leave fewer cells smooth than in 2D)."""
    n = 64
    U0 = workloads.mixed_voronoi(3, n, 8, seed=5, R=3).cuda()
    g64 = kfvm.KFVM([n] * 3, dims=3, radius=3, bc="outflow")
    gg = _gated(kfvm, n, "outflow")
    frac = gg.gate_mask(U0).float().mean().item()
    U64, Ug = U0.clone(), U0.clone()
    for _ in range(10):
        g64.step(U64, 0.4)
        gg.step(Ug, 0.4)
    rel = ((Ug[0] - U64[0]).abs().sum() / U64[0].abs().sum()).item()
    assert rel <= 2e-2, rel
    assert frac > 0.1, frac
