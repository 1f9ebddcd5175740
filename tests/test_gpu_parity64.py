"""FP64 GPU path against the oracle, element by element (spec bar: 1e-12 relative per step).

Every call goes through the C ABI of libkfvm.so (via the thin binding).  Sizes
span several CTA tiles (32 x 8 in 2D, 8 x 8 x 2 in 3D) with ragged tails.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402

TOL = 1e-12


@pytest.fixture(scope="module")
def kfvm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_16543_gb300 as pkg
    return pkg


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("dim,R", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_weights_match_oracle(kfvm, dim, R):
    n = [8] * dim
    g = kfvm.KFVM(n, dims=dim, radius=R)
    w = g.weights()
    ref = oracle.flat_weights(dim, R)
    assert w.shape == ref.shape
    scale = np.maximum(1.0, np.abs(ref))
    assert np.max(np.abs(w - ref) / scale) <= 4e-16 * (10 if (dim, R) == (3, 3) else 1)


def _state(dim, n, kind, seed):
    if kind == "sine" and dim == 2:
        U = workloads.sine_2d(max(n))[:, :n[1], :n[0]]
    elif kind == "voronoi" and dim == 2:
        U = workloads.voronoi_2d(max(n), k=10, seed=seed)[:, :n[1], :n[0]]
    else:
        U = workloads.mixed_voronoi(dim, max(n), 6, seed=seed)
        U = U[:, :n[2], :n[1], :n[0]] if dim == 3 else U[:, :n[1], :n[0]]
    return U.contiguous()


CASES = [
    (2, 2, (40, 24), "outflow", "voronoi"),
    (2, 2, (37, 19), "periodic", "sine"),
    (2, 3, (45, 17), "outflow", "voronoi"),
    (3, 2, (13, 10, 7), "periodic", "mixed"),
    (3, 2, (9, 17, 5), "outflow", "mixed"),
    (3, 3, (10, 9, 6), "outflow", "mixed"),
]


@pytest.mark.parametrize("dim,R,n,bc,kind", CASES)
@pytest.mark.parametrize("recon", ["weno", "linear"])
def test_reconstruct_flux_step(kfvm, dim, R, n, bc, kind, recon):
    U0 = _state(dim, n, kind, seed=sum(n))
    ref = oracle.Oracle(list(n), dim=dim, R=R, bc=bc, recon=recon)
    g = kfvm.KFVM(list(n), dims=dim, radius=R, bc=bc)
    g.set_option("recon", 0 if recon == "weno" else 1)
    U = U0.cuda()
    # Riemann states (including the positivity limiter)
    faces = g.reconstruct(U)
    rf = ref.limit(U0.numpy(), ref.reconstruct(U0.numpy()))
    scale = np.abs(U0.numpy()).max()
    assert np.abs(faces.cpu().numpy() - rf).max() / scale <= TOL
    g.sync_status()
    # flux divergence from the oracle's own Riemann states
    dU = g.flux(torch.from_numpy(rf).cuda())
    dref = ref.flux(rf)
    assert _rel(dU.cpu().numpy(), dref) <= TOL
    # one SSP-RK3 step
    dt = g.step(U, 0.4)
    Ur, dtr = ref.step(U0.numpy(), 0.4)
    assert abs(dt - dtr) <= 1e-14 * dtr
    assert np.abs(U.cpu().numpy() - Ur).max() / scale <= TOL


def test_riemann_hll_option(kfvm):
    n = (33, 20)
    U0 = _state(2, n, "voronoi", seed=5)
    ref = oracle.Oracle(list(n), dim=2, R=2, bc="outflow", riemann="hll")
    g = kfvm.KFVM(list(n), dims=2, radius=2, bc="outflow")
    g.set_option("riemann", 1)
    U = U0.cuda()
    g.step(U, 0.4)
    Ur, _ = ref.step(U0.numpy(), 0.4)
    assert np.abs(U.cpu().numpy() - Ur).max() / np.abs(Ur).max() <= TOL


def test_positivity_off_matches(kfvm):
    n = (32, 16)
    U0 = workloads.sine_2d(32)[:, :16, :].contiguous()
    ref = oracle.Oracle([32, 16], dim=2, R=2, bc="outflow", positivity=False)
    g = kfvm.KFVM([32, 16], dims=2, radius=2, bc="outflow")
    g.set_option("positivity", 0)
    faces = g.reconstruct(U0.cuda())
    assert np.abs(faces.cpu().numpy() - ref.reconstruct(U0.numpy())).max() <= TOL * 3


def test_sine_workload_many_steps(kfvm):
    """The 2D radius-2 sine workload (64^2, periodic, CFL 0.4): 20 steps stay within 1e-12 of the oracle."""
    n = 64
    U0 = workloads.sine_2d(n)
    ref = oracle.Oracle([n, n], dim=2, R=2)
    g = kfvm.KFVM([n, n], dims=2, radius=2)
    U = U0.cuda()
    Ur = U0.numpy()
    for _ in range(20):
        g.step(U, 0.4, 0.1)
        Ur, _ = ref.step(Ur, 0.4, 0.1)
    assert np.abs(U.cpu().numpy() - Ur).max() / np.abs(Ur).max() <= 20 * TOL


def test_tiny_periodic_grids_wrap_more_than_once(kfvm):
    """Grids smaller than the stencil (periodic wrap several times) and one-cell-wide axes."""
    for n in ((3, 2), (1, 5), (4, 1)):
        U0 = workloads.mixed_voronoi(2, 8, 4, seed=3)[:, :n[1], :n[0]].contiguous()
        ref = oracle.Oracle(list(n), dim=2, R=3)
        g = kfvm.KFVM(list(n), dims=2, radius=3)
        U = U0.cuda()
        g.step(U, 0.3)
        Ur, _ = ref.step(U0.numpy(), 0.3)
        assert np.abs(U.cpu().numpy() - Ur).max() / np.abs(Ur).max() <= TOL


def test_nonphysical_input_is_reported(kfvm):
    n = (16, 16)
    U0 = workloads.voronoi_2d(16, k=4, seed=1).clone()
    U0[3, 5, 7] = -1.0  # negative energy: p < 0 in one cell
    g = kfvm.KFVM(list(n), dims=2, radius=2, bc="outflow")
    with pytest.raises(kfvm.KfvmError) as e:
        g.step(U0.cuda(), 0.4)
    assert e.value.code == 4
    # the context stays usable
    U = workloads.voronoi_2d(16, k=4, seed=1).cuda()
    g.step(U, 0.4)


def test_bench_workload_rhs_full_size(kfvm):
    """The bench workload (1024^2 Voronoi, outflow, radius 2) at full size: L(U) on every cell."""
    n = 1024
    U0 = workloads.voronoi_2d(n, k=64, seed=2)
    g = kfvm.KFVM([n, n], dims=2, radius=2, bc="outflow")
    dU = g.rhs(U0.cuda())
    ref = oracle.Oracle([n, n], dim=2, R=2, bc="outflow")
    dref = ref.rhs(U0.numpy())
    assert _rel(dU.cpu().numpy(), dref) <= TOL
