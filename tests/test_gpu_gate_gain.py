"""What the trained gate gains over the method without it (WENO-AO on every cell).

The shipped parameters (paper_2401_16543_gb300/gate_params_2d.npy, trained on
the GPU by paper_2401_16543_gb300/train_gate.py) are used at the bench's
threshold 0.8.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402

PARAMS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2401_16543_gb300",
                      "gate_params_2d.npy")


@pytest.fixture(scope="module")
def kfvm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_16543_gb300 as pkg
    return pkg


def _gated(kfvm, n, bc, precision=32):
    g = kfvm.KFVM([n, n], dims=2, radius=2, bc=bc)
    g.set_option("precision", precision)
    g.gate_set_params(np.load(PARAMS))
    g.set_option("gate_threshold", 0.8)
    g.set_option("recon", 2)
    return g


def test_smooth_translation_error_not_worse_than_fp64_weno(kfvm):
    """64^2 sine translation to t = 0.1: the mixed-precision gated path's L1 density error is within
    1e-6 relative of (in fact far below) the plain FP64 WENO-AO path's, because the gate sends the
    smooth cells to the linear reconstruction whose accuracy the fixed eps = 1e-40 does not spoil."""
    n = 64
    U0 = workloads.sine_2d(n)
    ex = workloads.sine_2d_exact_density(n, 0.1)
    g64 = kfvm.KFVM([n, n], dims=2, radius=2)
    U64 = U0.cuda()
    g64.run(U64, 0.4, 0.1)
    gg = _gated(kfvm, n, "periodic")
    assert gg.gate_mask(U0.cuda()).float().mean().item() > 0.99
    Ug = U0.cuda()
    gg.run(Ug, 0.4, 0.1)
    e64 = np.abs(U64[0].cpu().numpy() - ex).mean()
    eg = np.abs(Ug[0].cpu().numpy() - ex).mean()
    assert eg <= e64 * (1 + 1e-6), (eg, e64)
    assert eg < e64 / 10, (eg, e64)
    # and the oracle agrees on the FP64 WENO error
    Ur, _, _ = oracle.Oracle([n, n], dim=2, R=2).run(U0.numpy(), 0.4, 0.1)
    assert abs(np.abs(Ur[0] - ex).mean() - e64) <= 1e-9


def test_voronoi_gated_stays_close_to_weno_everywhere(kfvm):
    """256^2 Voronoi (outflow), 40 steps: the gated mixed path stays admissible and its density stays
    within 2% (L1, relative) of the FP64 WENO-AO-everywhere result, while the gate sends most cells to
    the linear reconstruction."""
    n = 256
    U0 = workloads.voronoi_2d(n, k=64, seed=2).cuda()
    g64 = kfvm.KFVM([n, n], dims=2, radius=2, bc="outflow")
    gg = _gated(kfvm, n, "outflow")
    frac = gg.gate_mask(U0).float().mean().item()
    U64, Ug = U0.clone(), U0.clone()
    for _ in range(40):
        g64.step(U64, 0.4)
        gg.step(Ug, 0.4)
    rel = ((Ug[0] - U64[0]).abs().sum() / U64[0].abs().sum()).item()
    assert rel <= 2e-2, rel
    assert frac > 0.5, frac
