"""WENO-AO in characteristic variables (Sec. 3.4.1, option "variables" 1) against the oracle, through
the C ABI.  FP64 path: Riemann states and one SSP-RK3 step to 1e-12 relative (2D and 3D, radius 2
and 3, both boundary kinds, ragged tiles), also under the KXRCF indicator.  FP32 path (2D at radius
2 and 3, 3D at radius 2): Riemann states within 2e-5 and one step within 2e-6 of the state's
magnitude (the FP32 bars; the characteristic transform adds dense 5 x 5 float32 products, ~1e-7
relative), WENO-AO everywhere and under a caller mask; the radius-3 3D kernels are linearized
primitive only and refuse the option with KFVM_ERR_STATE.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402


@pytest.fixture(scope="module")
def kfvm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_16543_gb300 as pkg
    return pkg


def _state(dim, n, seed):
    if dim == 2:
        U = workloads.voronoi_2d(max(n), k=10, seed=seed)[:, :n[1], :n[0]]
    else:
        U = workloads.mixed_voronoi(3, max(n), 6, seed=seed)[:, :n[2], :n[1], :n[0]]
    return U.contiguous()


CASES = [(2, 2, (40, 24), "outflow"), (2, 2, (37, 19), "periodic"), (2, 3, (45, 17), "outflow"),
         (3, 2, (13, 10, 7), "periodic"), (3, 3, (10, 9, 6), "outflow")]


@pytest.mark.parametrize("recon", ["weno", "kxrcf"])
@pytest.mark.parametrize("dim,R,n,bc", CASES)
def test_characteristic_states_and_step_match_oracle(kfvm, dim, R, n, bc, recon):
    U0 = _state(dim, n, seed=sum(n) + 5)
    ref = oracle.Oracle(list(n), dim=dim, R=R, bc=bc, recon=recon, variables="characteristic")
    g = kfvm.KFVM(list(n), dims=dim, radius=R, bc=bc)
    g.set_option("variables", 1)
    g.set_option("recon", 0 if recon == "weno" else 4)
    U = U0.cuda()
    faces = g.reconstruct(U).cpu().numpy()
    rf = ref.limit(U0.numpy(), ref.reconstruct(U0.numpy())).reshape(faces.shape)
    assert np.abs(faces - rf).max() / np.abs(rf).max() <= 1e-12
    g.sync_status()
    dt = g.step(U, 0.4)
    Ur, dtr = ref.step(U0.numpy(), 0.4)
    assert abs(dt - dtr) <= 1e-14 * dtr
    assert np.abs(U.cpu().numpy() - Ur).max() / np.abs(Ur).max() <= 1e-12


def test_characteristic_differs_from_linearized_primitive(kfvm):
    U0 = _state(2, (40, 24), seed=69).cuda()
    out = []
    for variables in (0, 1):
        g = kfvm.KFVM([40, 24], dims=2, radius=2, bc="outflow")
        g.set_option("variables", variables)
        out.append(g.reconstruct(U0).cpu().numpy())
    assert np.abs(out[0] - out[1]).max() > 1e-3


G = 1.4


def _prim(f, dim):
    rho = f[:, 0]
    vel = f[:, 1:1 + dim] / rho[:, None]
    p = (G - 1) * (f[:, dim + 1] - 0.5 * rho * (vel ** 2).sum(1))
    return np.concatenate([rho[:, None], vel, p[:, None]], axis=1)


CASES32 = [(2, 2, (40, 24), "outflow"), (2, 2, (37, 19), "periodic"), (2, 3, (45, 17), "outflow"),
           (3, 2, (13, 10, 7), "periodic"), (3, 2, (11, 9, 8), "outflow")]


@pytest.mark.parametrize("dim,R,n,bc", CASES32)
def test_fp32_characteristic_states_and_step_match_oracle(kfvm, dim, R, n, bc):
    U0 = _state(dim, n, seed=sum(n) + 9)
    ref = oracle.Oracle(list(n), dim=dim, R=R, bc=bc, variables="characteristic")
    g = kfvm.KFVM(list(n), dims=dim, radius=R, bc=bc)
    g.set_option("precision", 32)
    g.set_option("variables", 1)
    U = U0.cuda()
    faces = g.faces_primitive(g.reconstruct(U)).cpu().numpy().astype(np.float64)
    rf = _prim(ref.limit(U0.numpy(), ref.reconstruct(U0.numpy())), dim).reshape(faces.shape)
    err = np.abs(faces - rf).max() / np.abs(rf).max()
    assert err <= 2e-5, err
    g.sync_status()
    g.step(U, 0.4)
    Ur, _ = ref.step(U0.numpy(), 0.4)
    err_s = np.abs(U.cpu().numpy() - Ur).max() / np.abs(Ur).max()
    assert err_s <= 2e-6, err_s


@pytest.mark.parametrize("dim,R,n", [(2, 2, (40, 24)), (3, 2, (13, 10, 7))])
def test_fp32_characteristic_under_a_caller_mask_matches_oracle(kfvm, dim, R, n):
    """Mask-driven mode: the marked cells take the linear reconstruction (conservative variables, as on
    the FP64 path), the others WENO-AO in characteristic variables."""
    U0 = _state(dim, n, seed=sum(n) + 13)
    rng = np.random.default_rng(3)
    mask = (rng.uniform(size=int(np.prod(n))) < 0.5).astype(np.uint8)
    ref = oracle.Oracle(list(n), dim=dim, R=R, bc="outflow", recon="gated", mask=mask,
                        variables="characteristic")
    g = kfvm.KFVM(list(n), dims=dim, radius=R, bc="outflow")
    g.set_option("precision", 32)
    g.set_option("variables", 1)
    g.set_smooth_mask(torch.from_numpy(mask).cuda())
    U = U0.cuda()
    g.step(U, 0.4)
    Ur, _ = ref.step(U0.numpy(), 0.4)
    err = np.abs(U.cpu().numpy() - Ur).max() / np.abs(Ur).max()
    assert err <= 2e-6, err


def test_fp32_characteristic_differs_from_linearized_primitive(kfvm):
    U0 = _state(2, (40, 24), seed=69).cuda()
    out = []
    for variables in (0, 1):
        g = kfvm.KFVM([40, 24], dims=2, radius=2, bc="outflow")
        g.set_option("precision", 32)
        g.set_option("variables", variables)
        out.append(g.reconstruct(U0).cpu().numpy())
    assert np.abs(out[0] - out[1]).max() > 1e-3


def test_fp32_radius3_3d_refuses_characteristic_variables(kfvm):
    g = kfvm.KFVM([12, 10, 8], dims=3, radius=3, bc="outflow")
    g.set_option("precision", 32)
    g.set_option("variables", 1)
    U = _state(3, (12, 10, 8), seed=4).cuda()
    with pytest.raises(kfvm.KfvmError) as e:
        g.reconstruct(U)
    assert e.value.code == 5  # KFVM_ERR_STATE


def test_variables_option_is_checked(kfvm):
    g = kfvm.KFVM([16, 16], dims=2, radius=2, bc="outflow")
    for bad in (2.0, -1.0, 0.5):
        with pytest.raises(kfvm.KfvmError) as e:
            g.set_option("variables", bad)
        assert e.value.code == 1  # KFVM_ERR_ARG
