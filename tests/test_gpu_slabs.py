"""3D steps in z-slabs (the Riemann-state buffer holds a few planes at a time) against whole-grid steps.

Every cell runs the same arithmetic whichever slab it falls in, so a step taken
in slabs equals the whole-grid step bit for bit; the slabbed FP64 step is also
checked against the oracle (1e-12 relative per step).  Slab sizes cover a single
plane, sizes that divide nz and ragged last slabs, periodic and outflow z ends.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402
from oracle import gate as ogate  # noqa: E402


@pytest.fixture(scope="module")
def kfvm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_16543_gb300 as pkg
    return pkg


def _state(n, seed):
    U = workloads.mixed_voronoi(3, max(n), 6, seed=seed)
    return U[:, :n[2], :n[1], :n[0]].contiguous()


def _run(kfvm, n, R, bc, precision, recon, slab, U0, steps=2, params=None):
    g = kfvm.KFVM(list(n), dims=3, radius=R, bc=bc)
    g.set_option("precision", precision)
    if params is not None:
        g.gate_set_params(params)
        g.set_option("gate_threshold", 0.5)
    g.set_option("recon", recon)
    if slab:
        g.set_option("slab_planes", slab)
    U = U0.cuda()
    dts = [g.step(U, 0.4) for _ in range(steps)]
    return U.cpu().numpy(), dts


@pytest.mark.parametrize("bc", ["periodic", "outflow"])
@pytest.mark.parametrize("precision,R", [(64, 2), (64, 3), (32, 2)])
@pytest.mark.parametrize("slab", [1, 3, 4, 7])
def test_slabbed_step_equals_whole_grid(kfvm, bc, precision, R, slab):
    # slab 7 of 8 planes would need 9 planes of Riemann states: the library lowers it to what its
    # buffer holds
    n = (11, 9, 8)
    U0 = _state(n, seed=71)
    whole, dtw = _run(kfvm, n, R, bc, precision, 0, 0, U0)
    part, dtp = _run(kfvm, n, R, bc, precision, 0, slab, U0)
    assert dtw == dtp
    assert np.array_equal(whole, part)


@pytest.mark.parametrize("precision", [64, 32])
def test_slabbed_gated_step_equals_whole_grid(kfvm, precision):
    n = (12, 10, 9)
    U0 = _state(n, seed=72)
    p = ogate.init_params(3, seed=73)
    p[-1] = 0.2
    whole, _ = _run(kfvm, n, 2, "outflow", precision, 2, 0, U0, params=p)
    part, _ = _run(kfvm, n, 2, "outflow", precision, 2, 2, U0, params=p)
    assert np.array_equal(whole, part)


@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_slabbed_step_matches_oracle(kfvm, bc):
    n = (10, 9, 7)
    U0 = _state(n, seed=74)
    U, _ = _run(kfvm, n, 2, bc, 64, 0, 2, U0, steps=1)
    Ur, _ = oracle.Oracle(list(n), dim=3, R=2, bc=bc).step(U0.numpy(), 0.4)
    assert np.abs(U - Ur).max() / np.abs(U0.numpy()).max() <= 1e-12


def test_slab_option_rejected_in_2d(kfvm):
    g = kfvm.KFVM([16, 16], dims=2, radius=2)
    with pytest.raises(kfvm.KfvmError):
        g.set_option("slab_planes", 4)
