"""FP32 (mixed-precision) GPU path against the FP64 oracle.

Tolerances follow from the arithmetic (the CFL rate is formed in float32, so dt
agrees to 1e-6): the float32 shadow of the state carries a
relative rounding of 2^-24 ~ 6e-8; each Riemann-state value is a contraction
whose weights sum in absolute value to ~2-3.3 (2D, 3D radius 2), so its error
is a few 1e-7 of the state's magnitude (the S0 face rows of 3D radius 3 sum to
~70: a few 1e-6 there); the nonlinear weights and the limiter's
theta factors move by O(1e-6) relative.  Face states are checked at 2e-5 of the
state's magnitude, one SSP-RK3 step at 2e-6 (the update is dt*L with
dt*|L| ~ CFL * |U|, accumulated in float64).  The accuracy target of the
mixed path is the L1 density error on smooth data: within 1e-6 relative of
the FP64 result.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402

G = 1.4


@pytest.fixture(scope="module")
def kfvm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_16543_gb300 as pkg
    return pkg


def to_prim(f, dim):
    rho = f[:, 0]
    vel = f[:, 1:1 + dim] / rho[:, None]
    p = (G - 1) * (f[:, dim + 1] - 0.5 * rho * (vel ** 2).sum(1))
    return np.concatenate([rho[:, None], vel, p[:, None]], axis=1)


def _state(dim, n, seed):
    if dim == 2:
        U = workloads.voronoi_2d(max(n), k=10, seed=seed)[:, :n[1], :n[0]]
    else:
        U = workloads.mixed_voronoi(3, max(n), 6, seed=seed)[:, :n[2], :n[1], :n[0]]
    return U.contiguous()


CASES = [(2, 2, (40, 24), "outflow"), (2, 3, (45, 17), "outflow"), (3, 2, (13, 10, 7), "periodic"),
         (2, 2, (37, 19), "periodic"), (3, 3, (10, 9, 6), "outflow"), (3, 3, (9, 8, 7), "periodic")]


@pytest.mark.parametrize("dim,R,n,bc", CASES)
@pytest.mark.parametrize("recon", ["weno", "linear"])
def test_fp32_faces_and_step(kfvm, dim, R, n, bc, recon):
    U0 = _state(dim, n, seed=sum(n) + 1)
    ref = oracle.Oracle(list(n), dim=dim, R=R, bc=bc, recon=recon)
    g = kfvm.KFVM(list(n), dims=dim, radius=R, bc=bc)
    g.set_option("precision", 32)
    g.set_option("recon", 0 if recon == "weno" else 1)
    U = U0.cuda()
    faces = g.faces_primitive(g.reconstruct(U)).cpu().numpy().astype(np.float64)
    rf = to_prim(ref.limit(U0.numpy(), ref.reconstruct(U0.numpy())), dim).reshape(faces.shape)
    scale = np.abs(rf).max()
    err_f = np.abs(faces - rf).max() / scale
    assert err_f <= 2e-5, err_f
    g.sync_status()
    dt = g.step(U, 0.4)
    Ur, dtr = ref.step(U0.numpy(), 0.4)
    assert abs(dt - dtr) <= 1e-6 * dtr  # the mixed path forms the CFL rate in float32
    err_s = np.abs(U.cpu().numpy() - Ur).max() / np.abs(Ur).max()
    assert err_s <= 2e-6, err_s


def test_fp32_l1_density_on_smooth_translation(kfvm):
    """64^2 sine translation to t = 0.1 (75 steps): the FP32 path's density stays within 1e-6
    (relative, L1) of the FP64 oracle, and its L1 error against the exact solution matches FP64's."""
    n = 64
    U0 = workloads.sine_2d(n)
    ref = oracle.Oracle([n, n], dim=2, R=2)
    Ur, _, _ = ref.run(U0.numpy(), 0.4, 0.1)
    g = kfvm.KFVM([n, n], dims=2, radius=2)
    g.set_option("precision", 32)
    U = U0.cuda()
    t, k = g.run(U, 0.4, 0.1)
    rho = U[0].cpu().numpy()
    rel = np.abs(rho - Ur[0]).sum() / np.abs(Ur[0]).sum()
    assert rel <= 1e-6, rel
    ex = workloads.sine_2d_exact_density(n, 0.1)
    e32, e64 = np.abs(rho - ex).mean(), np.abs(Ur[0] - ex).mean()
    assert e32 <= e64 * (1 + 1e-2), (e32, e64)


def test_fp32_bench_workload_full_size(kfvm):
    """1024^2 Voronoi workload: one FP32 step against the FP64 GPU path on every cell."""
    n = 1024
    U0 = workloads.voronoi_2d(n, k=64, seed=2).cuda()
    g64 = kfvm.KFVM([n, n], dims=2, radius=2, bc="outflow")
    g32 = kfvm.KFVM([n, n], dims=2, radius=2, bc="outflow")
    g32.set_option("precision", 32)
    U64, U32 = U0.clone(), U0.clone()
    g64.step(U64, 0.4)
    g32.step(U32, 0.4)
    err = ((U32 - U64).abs().max() / U64.abs().max()).item()
    assert err <= 2e-6, err
