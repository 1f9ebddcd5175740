"""The KXRCF troubled-cell indicator (Sec. 3.5) and its gated step ("recon" 4) against the oracle.

Every call goes through the C ABI.  The indicator's decision compares a float ratio with
Delta^m, so near the threshold both sides can disagree by rounding; cells whose oracle ratio
lies within a band around Delta^m accept either decision and every other cell must match
exactly.  FP64 band: 1e-9 relative (the two sides' reconstructions differ by ~1e-15).  FP32
band: 1e-5 absolute on the ratio, from the float32 arithmetic: the float32 copy of the state
(6e-8 relative) and a contraction whose weights sum in absolute value to ~3 give states within
~2e-7 relative; the pressure recovery E - |m|^2/(2 rho) amplifies that by E/p (<= ~13 on these
inputs) and rho^-gamma adds ~2e-7, so each q carries ~2e-6 of <Q> and a jump ~4e-6: the band
keeps a 2.5x margin.  (Delta^m itself is 3e-5 at 1024^2, so the band must stay well below it.)
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402

G = 1.4
FP32_BAND = 1e-5  # absolute, on the ratio (see above)


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


def _thresh(n, m=1.5):
    return (1.0 / min(n)) ** m  # unit box: Delta = the largest cell width


# (dims, R, cells, boundary, seed): every crop holds flagged and smooth cells
CASES = [(2, 2, (40, 24), "outflow", 67), (2, 2, (37, 19), "periodic", 59), (2, 3, (45, 17), "outflow", 65),
         (3, 2, (13, 10, 7), "periodic", 33), (3, 2, (9, 17, 5), "outflow", 34), (3, 3, (10, 9, 6), "outflow", 28),
         (3, 3, (9, 8, 7), "periodic", 5)]


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("dim,R,n,bc,seed", CASES)
def test_mask_matches_oracle(kfvm, dim, R, n, bc, seed, precision):
    U0 = _state(dim, n, seed)
    ratio, want = oracle.Oracle(list(n), dim=dim, R=R, bc=bc).kxrcf(U0.numpy())
    g = kfvm.KFVM(list(n), dims=dim, radius=R, bc=bc)
    g.set_option("precision", precision)
    got = g.kxrcf_mask(U0.cuda()).cpu().numpy()
    th = _thresh(n)
    band = np.abs(ratio - th) <= (1e-9 * th if precision == 64 else FP32_BAND)
    assert (got[~band] == want[~band]).all(), np.argwhere((got != want) & ~band)[:5]
    assert set(np.unique(got)) <= {0, 1}
    assert (want == 0).any() and (want == 1).any()
    if precision == 64:
        assert not band.any()


def test_mask_on_smooth_and_constant_data(kfvm):
    """The 64^2 smooth translation flags no cell; a constant state flags none either, in both precisions."""
    for precision in (64, 32):
        g = kfvm.KFVM([64, 64], dims=2, radius=2, bc="periodic")
        g.set_option("precision", precision)
        assert g.kxrcf_mask(workloads.sine_2d(64).cuda()).all()
        c = workloads.constant_state(2, [64, 64], rho=0.3, vel=[0.5, -0.2], p=0.7).cuda()
        assert g.kxrcf_mask(c).all()


@pytest.mark.parametrize("dim,R,n,bc,seed", [CASES[0], CASES[2], CASES[3], CASES[5]])
def test_fp64_kxrcf_step_matches_oracle(kfvm, dim, R, n, bc, seed):
    """FP64 path in the KXRCF mode: Riemann states and one SSP-RK3 step (the mask recomputed at every
    stage from that stage's state) equal the oracle's to 1e-12 relative."""
    U0 = _state(dim, n, seed)
    ref = oracle.Oracle(list(n), dim=dim, R=R, bc=bc, recon="kxrcf")
    g = kfvm.KFVM(list(n), dims=dim, radius=R, bc=bc)
    g.set_option("recon", 4)
    U = U0.cuda()
    faces = g.reconstruct(U).cpu().numpy()
    rf = ref.limit(U0.numpy(), ref.reconstruct(U0.numpy())).reshape(faces.shape)
    assert np.abs(faces - rf).max() / np.abs(rf).max() <= 1e-12
    g.sync_status()
    dt = g.step(U, 0.4)
    Ur, dtr = ref.step(U0.numpy(), 0.4)
    assert abs(dt - dtr) <= 1e-14 * dtr
    assert np.abs(U.cpu().numpy() - Ur).max() / np.abs(Ur).max() <= 1e-12


@pytest.mark.parametrize("dim,R,n,bc,seed", [CASES[0], CASES[3], CASES[5], CASES[6]])
def test_fp32_kxrcf_states_match_oracle_on_its_mask(kfvm, dim, R, n, bc, seed):
    """FP32 path in the KXRCF mode: the Riemann states equal the oracle's gated reconstruction on the
    mask the FP32 indicator chose, within the FP32 path's 2e-5 of max |state|."""
    U0 = _state(dim, n, seed)
    g = kfvm.KFVM(list(n), dims=dim, radius=R, bc=bc)
    g.set_option("precision", 32)
    g.set_option("recon", 4)
    U = U0.cuda()
    mask = g.kxrcf_mask(U).cpu().numpy()
    f = g.faces_primitive(g.reconstruct(U)).cpu().numpy().astype(np.float64)
    ref = oracle.Oracle(list(n), dim=dim, R=R, bc=bc, recon="gated", mask=mask)
    rf = ref.limit(U0.numpy(), ref.reconstruct(U0.numpy()))
    rho = rf[:, 0]
    vel = rf[:, 1:1 + dim] / rho[:, None]
    p = (G - 1) * (rf[:, dim + 1] - 0.5 * rho * (vel ** 2).sum(1))
    prim = np.concatenate([rho[:, None], vel, p[:, None]], axis=1).reshape(f.shape)
    assert np.abs(f - prim).max() / np.abs(prim).max() <= 2e-5
    g.sync_status()


def test_kxrcf_slabs_equal_whole_grid(kfvm):
    """3D steps in z-slabs take the indicator of the whole grid per stage: bit-identical results."""
    n = (12, 10, 9)
    U0 = _state(3, n, seed=77)
    out = []
    for slab in (None, 3):
        g = kfvm.KFVM(list(n), dims=3, radius=2, bc="outflow")
        g.set_option("precision", 32)
        g.set_option("recon", 4)
        if slab:
            g.set_option("slab_planes", slab)
        U = U0.cuda()
        g.step(U, 0.4)
        out.append(U.cpu().numpy())
    assert np.array_equal(out[0], out[1])


def test_kxrcf_path_on_smooth_translation(kfvm):
    """64^2 sine translation to t = 0.1 (the accuracy case): the indicator flags nothing, so the KXRCF
    path is the linear path (FP64: bit for bit) and its L1 density error is below WENO-AO
    everywhere's; the FP32 KXRCF path's density stays within 1e-6 (relative L1) of the FP64 one."""
    n, t_end = 64, 0.1
    U0 = workloads.sine_2d(n)
    ex = workloads.sine_2d_exact_density(n, t_end)
    res = {}
    for name, prec, recon in [("kx64", 64, 4), ("lin64", 64, 1), ("weno64", 64, 0), ("kx32", 32, 4)]:
        g = kfvm.KFVM([n, n], dims=2, radius=2, bc="periodic")
        g.set_option("precision", prec)
        g.set_option("recon", recon)
        U = U0.cuda()
        g.run(U, 0.4, t_end)
        res[name] = U[0].cpu().numpy()
    assert np.array_equal(res["kx64"], res["lin64"])
    e = {k: np.abs(v - ex).mean() for k, v in res.items()}
    assert e["kx64"] < e["weno64"], e
    rel = np.abs(res["kx32"] - res["kx64"]).sum() / np.abs(res["kx64"]).sum()
    assert rel <= 1e-6, rel


def test_kxrcf_options_are_checked(kfvm):
    """"recon" 4 selects the KXRCF mode; "kxrcf_m" accepts 0 < m <= 16 and changes the decisions."""
    g = kfvm.KFVM([40, 24], dims=2, radius=2, bc="outflow")
    for bad in (0.0, -1.0, 17.0):
        with pytest.raises(kfvm.KfvmError) as e:
            g.set_option("kxrcf_m", bad)
        assert e.value.code == 1  # KFVM_ERR_ARG
    with pytest.raises(kfvm.KfvmError):
        g.set_option("recon", 3)  # the caller-mask mode is set by kfvm_set_smooth_mask only
    U = workloads.mixed_voronoi(2, 40, 6, seed=3)[:, :24, :40].contiguous().cuda()  # smooth and constant regions
    g.set_option("kxrcf_m", 1.5)
    m15 = g.kxrcf_mask(U).cpu().numpy()
    g.set_option("kxrcf_m", 4.0)  # a smaller threshold Delta^m flags more cells
    m40 = g.kxrcf_mask(U).cpu().numpy()
    assert (m40 <= m15).all() and m40.sum() < m15.sum()


def test_kxrcf_mixed_path_on_3d_smooth_translation(kfvm):
    """32^3 sine translation (periodic) at radius 2 -- the paper's 3D radius -- to t = 0.05: the KXRCF
    indicator flags no cell of this smooth flow, so the FP32 path takes the linear reconstruction
    everywhere, and its L1 density error against the exact solution stays at or below the plain FP64
    WENO-AO path's.  This is the "matched L1" bar E <= E_FP64 (1 + 1e-6), met in 3D with the paper's
    own indicator.  (At radius 3 in 3D the linear S0 reconstruction with SSP-RK3 is not stable at
    CFL 0.4: on the oracle the error leaves its truncation level within ~7 steps on 16^3, and later
    at smaller CFL, while WENO-AO stays stable.  The paper runs radius 3 only in 2D, so there KXRCF,
    or any gate, must keep WENO-AO on part of a smooth 3D flow.)"""
    n, t_end = 32, 0.05
    U0 = workloads.sine_3d(n, R=2)
    ex = workloads.sine_3d_exact_density(n, t_end)
    g64 = kfvm.KFVM([n] * 3, dims=3, radius=2)
    U64 = U0.cuda()
    g64.run(U64, 0.4, t_end)
    gk = kfvm.KFVM([n] * 3, dims=3, radius=2)
    gk.set_option("precision", 32)
    gk.set_option("recon", 4)
    assert gk.kxrcf_mask(U0.cuda()).all()
    Uk = U0.cuda()
    gk.run(Uk, 0.4, t_end)
    e64 = np.abs(U64[0].cpu().numpy() - ex).mean()
    ek = np.abs(Uk[0].cpu().numpy() - ex).mean()
    print(f"3D R2 KXRCF FP32 L1 error / FP64 WENO-AO error: {ek / e64:.4f}")
    assert ek <= e64 * (1 + 1e-6), (ek, e64)
