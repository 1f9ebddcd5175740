"""The tensor-core (tcgen05) FP32 reconstruction of 3D radius 3 against the oracle and against the
CUDA-core kernel.

The contraction runs as FP16 hi/lo split products with FP32 accumulation in TMEM (~22 bits per
product, the accuracy of the float32 contraction), so the bars are those of the FP32 path: Riemann
states within 2e-5 of the state's magnitude, one SSP-RK3 step within 2e-6; the two FP32 kernels
agree to 1e-5.  Grids cover ragged 8 x 4 x 4 tiles, both boundary kinds, more tiles than SMs (the
persistent loop), the linear and the gated modes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402
from oracle import gate as ogate  # noqa: E402

G = 1.4


@pytest.fixture(scope="module")
def kfvm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_16543_gb300 as pkg
    return pkg


def to_prim(f):
    rho = f[:, 0]
    vel = f[:, 1:4] / rho[:, None]
    p = (G - 1) * (f[:, 4] - 0.5 * rho * (vel ** 2).sum(1))
    return np.concatenate([rho[:, None], vel, p[:, None]], axis=1)


def _state(n, seed):
    return workloads.mixed_voronoi(3, max(n), 6, seed=seed, R=3)[:, :n[2], :n[1], :n[0]].contiguous()


def _solver(kfvm, n, bc, tc, recon=0):
    g = kfvm.KFVM(list(n), dims=3, radius=3, bc=bc)
    g.set_option("precision", 32)
    g.set_option("tensor_cores", tc)
    g.set_option("recon", recon)
    return g


@pytest.mark.parametrize("n,bc", [((10, 9, 6), "outflow"), ((9, 8, 7), "periodic"), ((17, 5, 9), "outflow")])
@pytest.mark.parametrize("recon", ["weno", "linear"])
def test_tc_faces_and_step_match_oracle(kfvm, n, bc, recon):
    U0 = _state(n, seed=sum(n) + 3)
    ref = oracle.Oracle(list(n), dim=3, R=3, bc=bc, recon=recon)
    g = _solver(kfvm, n, bc, 1, 0 if recon == "weno" else 1)
    U = U0.cuda()
    faces = g.faces_primitive(g.reconstruct(U)).cpu().numpy().astype(np.float64)
    rf = to_prim(ref.limit(U0.numpy(), ref.reconstruct(U0.numpy()))).reshape(faces.shape)
    err_f = np.abs(faces - rf).max() / np.abs(rf).max()
    assert err_f <= 2e-5, err_f
    g.sync_status()
    g.step(U, 0.4)
    Ur, _ = ref.step(U0.numpy(), 0.4)
    err_s = np.abs(U.cpu().numpy() - Ur).max() / np.abs(Ur).max()
    assert err_s <= 2e-6, err_s


@pytest.mark.parametrize("recon", [0, 1])
def test_tc_equals_cuda_core_kernel_on_many_tiles(kfvm, recon):
    """40 x 36 x 32 cells = 360 tiles (more than the SMs: every CTA loops over several tiles)."""
    n = (40, 36, 32)
    U0 = _state(n, seed=5).cuda()
    out = []
    for tc in (1, 0):
        g = _solver(kfvm, n, "outflow", tc, recon)
        out.append(g.faces_primitive(g.reconstruct(U0)).cpu().numpy().astype(np.float64))
        g.sync_status()
    err = np.abs(out[0] - out[1]).max() / np.abs(out[1]).max()
    assert err <= 1e-5, err


def test_tc_gated_with_a_given_mask_matches_oracle(kfvm):
    n = (12, 9, 8)
    U0 = _state(n, seed=31)
    Xr = ogate.features(U0.numpy(), 3, "outflow", R=3)
    mask = (np.abs(Xr[:, :33]).max(axis=1) < 0.99).astype(np.uint8)
    mask[::5] = 1 - mask[::5]
    ref = oracle.Oracle(list(n), dim=3, R=3, bc="outflow", recon="gated", mask=mask)
    g = _solver(kfvm, n, "outflow", 1)
    g.set_smooth_mask(torch.from_numpy(mask).cuda())
    U = U0.cuda()
    U1r, _ = ref.step(U0.numpy(), 0.4)
    g.step(U, 0.4)
    err = np.abs(U.cpu().numpy() - U1r).max() / np.abs(U1r).max()
    assert err <= 2e-6, err


def test_tc_all_linear_tiles_take_the_short_path(kfvm):
    """An all-ones mask makes every tile linear (pass 1 skipped, S0 k-steps only): the result equals
    the linear mode's."""
    n = (16, 8, 8)
    U0 = _state(n, seed=37).cuda()
    g = _solver(kfvm, n, "outflow", 1)
    g.set_smooth_mask(torch.ones(n[::-1], dtype=torch.uint8, device="cuda"))
    f_mask = g.reconstruct(U0).cpu().numpy()
    h = _solver(kfvm, n, "outflow", 1, 1)
    f_lin = h.reconstruct(U0).cpu().numpy()
    assert np.array_equal(f_mask, f_lin)


def test_bounded_wait_timeout_is_reported_and_the_context_survives(kfvm):
    """The tensor-core kernel's waits have iteration limits: the test hook makes one wait on a phase
    that nothing completes, the kernel raises the timeout flag instead of hanging, the host reads
    KFVM_ERR_TIMEOUT, and the next reconstruction is correct."""
    n = (10, 9, 6)
    U0 = _state(n, seed=41).cuda()
    g = _solver(kfvm, n, "outflow", 1)
    ref = g.faces_primitive(g.reconstruct(U0)).cpu().numpy()
    g.sync_status()
    g.set_option("timeout_probe", 1)
    g.reconstruct(U0)
    with pytest.raises(kfvm.KfvmError) as e:
        g.sync_status()
    assert e.value.code == 6  # KFVM_ERR_TIMEOUT
    again = g.faces_primitive(g.reconstruct(U0)).cpu().numpy()
    g.sync_status()
    assert np.array_equal(again, ref)
