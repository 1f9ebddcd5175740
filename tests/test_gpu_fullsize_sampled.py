"""Parity at the bench's full sizes, in the configuration bench.py times, on sampled outputs.

L(U) (kfvm_rhs: Riemann states, fluxes, divergence; 3D grids above the Riemann-state buffer run in
z-slabs exactly as the timed step does) is computed on the whole workload; at 48 seeded interior cells it
is compared with the oracle's L on a crop around the cell.  L at a cell depends on the Riemann states of
the cell and its face neighbours, and those on cells within R of them, so a crop of half-width R + 1
(outflow ghosts beyond it) gives the oracle exactly the inputs of the full grid.  The gated workloads
run the gated mode on the gate's own mask (`kfvm_gate_mask` of the state, passed back with
`kfvm_set_smooth_mask`, the same kernel and launch shape as the fused gate; the fused decisions are
checked against that mask in test_gpu_gate.py), and the oracle runs its gated mode on the cropped mask.

Tolerance: the FP32 Riemann states carry 2e-5 of max |U| (test_gpu_parity32.py); L differences them
over one cell, so |dL| <= 2e-5 max|U| / h per cell.
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402

SAMPLES = 48


@pytest.fixture(scope="module")
def kfvm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_16543_gb300 as pkg
    return pkg


def _sample_cells(shape, margin, seed):
    rng = np.random.default_rng(seed)
    return [tuple(int(rng.integers(margin, s - margin)) for s in shape) for _ in range(SAMPLES)]


@pytest.mark.parametrize("name", ["voronoi2d-1024", "mixed2d-2048", "halfsine3d-256", "mixed3d-512-r3"])
def test_full_size_rhs_matches_oracle_on_sampled_cells(kfvm, name):
    W = bench._workloads()[name]
    U0 = W.make("cuda").contiguous()
    g = kfvm.KFVM(list(W.n), dims=W.dims, radius=W.R, bc=W.bc)
    g.set_option("precision", 32)
    mask = None
    if W.has_gate():
        g.gate_set_params(np.load(W.gate_path()))
        g.set_option("gate_threshold", bench.GATE_THRESHOLD)
        g.set_option("recon", 2)
        m = g.gate_mask(U0)
        g.set_smooth_mask(m)
        mask = m.cpu().numpy()
    L = g.rhs(U0)
    g.sync_status()
    half = W.R + 1
    shape = tuple(U0.shape[1:])  # (z,) y, x
    h = 1.0 / W.n[0]
    scale = float(U0.abs().max().item())
    tol = 2e-5 * scale / h
    worst = 0.0
    for cell in _sample_cells(shape, half, seed=sum(map(ord, name))):
        sl = tuple(slice(c - half, c + half + 1) for c in cell)
        crop = U0[(slice(None),) + sl].cpu().numpy()
        n_crop = [2 * half + 1] * W.dims
        box = dict(lo=[0.0] * W.dims, hi=[(2 * half + 1) * h] * W.dims)  # the full grid's cell size
        if mask is not None:
            ref = oracle.Oracle(n_crop, dim=W.dims, R=W.R, bc="outflow", recon="gated",
                                mask=np.ascontiguousarray(mask[sl]).ravel(), **box)
        else:
            ref = oracle.Oracle(n_crop, dim=W.dims, R=W.R, bc="outflow", **box)
        Lr = ref.rhs(np.ascontiguousarray(crop))
        centre = (slice(None),) + tuple([half] * W.dims)
        got = L[(slice(None),) + cell].cpu().numpy()
        worst = max(worst, float(np.abs(got - Lr[centre]).max()))
    assert worst <= tol, (worst, tol)


@pytest.mark.parametrize("name", ["voronoi2d-1024", "halfsine3d-256"])
def test_full_size_kxrcf_matches_oracle_on_sampled_cells(kfvm, name):
    """The KXRCF path as bench.py times it (FP32, "recon" 4) at full size.  At each sampled cell: the
    indicator's decision against the oracle's ratio on the crop (the indicator of a cell reads the cells
    within R + 1, all inside the crop; either decision is accepted within 1e-5 of Delta^m, the FP32 band
    of test_gpu_kxrcf.py), and L(U) against the oracle's gated L on the GPU's mask (2e-5 max|U| / h)."""
    W = bench._workloads()[name]
    U0 = W.make("cuda").contiguous()
    g = kfvm.KFVM(list(W.n), dims=W.dims, radius=W.R, bc=W.bc)
    g.set_option("precision", 32)
    g.set_option("recon", 4)
    mask = g.kxrcf_mask(U0).cpu().numpy()
    L = g.rhs(U0)
    g.sync_status()
    assert (mask == 0).any() and (mask == 1).any()
    half = W.R + 1
    shape = tuple(U0.shape[1:])
    h = 1.0 / W.n[0]
    thresh = h ** 1.5
    scale = float(U0.abs().max().item())
    tol = 2e-5 * scale / h
    worst, decided = 0.0, 0
    for cell in _sample_cells(shape, half, seed=sum(map(ord, name)) + 1):
        sl = tuple(slice(c - half, c + half + 1) for c in cell)
        crop = np.ascontiguousarray(U0[(slice(None),) + sl].cpu().numpy())
        n_crop = [2 * half + 1] * W.dims
        box = dict(lo=[0.0] * W.dims, hi=[(2 * half + 1) * h] * W.dims)
        centre = tuple([half] * W.dims)
        ratio, _ = oracle.Oracle(n_crop, dim=W.dims, R=W.R, bc="outflow", **box).kxrcf(crop)
        if abs(ratio[centre] - thresh) > 1e-5:
            assert mask[cell] == (1 if ratio[centre] < thresh else 0), (cell, ratio[centre], thresh)
            decided += 1
        ref = oracle.Oracle(n_crop, dim=W.dims, R=W.R, bc="outflow", recon="gated",
                            mask=np.ascontiguousarray(mask[sl]).ravel(), **box)
        Lr = ref.rhs(crop)
        got = L[(slice(None),) + cell].cpu().numpy()
        worst = max(worst, float(np.abs(got - Lr[(slice(None),) + centre]).max()))
    assert decided >= SAMPLES // 2
    assert worst <= tol, (worst, tol)
