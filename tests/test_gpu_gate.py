"""The learned gate on the GPU (BF16 tensor-core MLP, FP32 accumulation) against the oracle.

Tolerances: features are float32 computations of [-1, 1]-normalised values
(1e-3); the network's operands are bf16 (8-bit mantissa, relative rounding
2^-9).  Against an oracle that rounds to bf16 at the same points, the
probabilities agree to 2e-3 and the gradients to 1e-2 per tensor (summation
order and float32 accumulation only); against exact FP64 backprop the rounding
compounds over three layers (bound 1e-1 per tensor, 1e-2 on the loss).  Gated
reconstructions driven by one mask follow the FP64 (1e-12) and FP32 (2e-6 per
step) bars of the ungated paths.
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


def _cases():
    return [("sine", workloads.sine_2d(64), "periodic"),
            ("voronoi", workloads.voronoi_2d(48, k=8, seed=5)[:, :40, :].contiguous(), "outflow")]


def _block_amplitude(U, bc, blk):
    """max over the radius-2 stencil of |v_l - v_c| / |v_c| for rho (blk 0) or p (blk 1), per cell."""
    from oracle import stencils
    rho = U[0]
    p = 0.4 * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / rho)
    v = rho if blk == 0 else p
    mode = "wrap" if bc == "periodic" else "edge"
    P = np.pad(v, 2, mode=mode)
    ny, nx = v.shape
    amp = np.zeros(v.size)
    for o in stencils.full_stencil(2, 2):
        amp = np.maximum(amp, np.abs(P[2 + o[1]:2 + o[1] + ny, 2 + o[0]:2 + o[0] + nx] - v).ravel())
    return amp / np.abs(v).ravel()


@pytest.mark.parametrize("idx", [0, 1])
def test_features_and_labels(kfvm, idx):
    name, U0, bc = _cases()[idx]
    n = list(reversed(U0.shape[1:]))
    g = kfvm.KFVM(n, dims=2, radius=2, bc=bc)
    X, y = g.gate_features(U0.cuda(), tau=0.5)
    Xg = X.cpu().numpy()
    Xr = ogate.features(U0.numpy(), 2, bc)
    # blocks whose relative variation is far above float32 rounding agree to 1e-3; blocks that are
    # flat to ~1e-7 relative hold float32 rounding noise scaled by the 1e-4 floor
    U = U0.numpy()
    for blk in range(2):
        sl = slice(13 * blk, 13 * blk + 13)
        amp = _block_amplitude(U, bc, blk)
        big = amp > 1e-4
        if big.any():
            assert np.abs(Xg[big, sl] - Xr[big, sl]).max() <= 1e-3
        if (~big).any():
            assert np.abs(Xg[~big, sl]).max() <= 0.5
    o = oracle.Oracle(n, dim=2, R=2, bc=bc)
    _, om = o.reconstruct(U0.numpy(), with_omega=True)
    amp = ogate.linprim_amplitude(U0.numpy(), 2, 2, bc)
    yr, worst = ogate.labels_from_omega(om, 2, 0.5, amp)
    # cells whose decision sits at a threshold (weights or amplitude) may fall either way in float32
    far = (np.abs(worst - 0.5) > 1e-3) & (np.abs(np.log10(np.maximum(amp[[0, -1]], 1e-30)) + 4).min(axis=0) > 0.05)
    assert np.array_equal(y.cpu().numpy()[far], yr[far])
    assert far.mean() > 0.9


def test_forward_matches_oracle(kfvm):
    g = kfvm.KFVM([16, 16], dims=2, radius=2)
    p = ogate.init_params(2, seed=11)
    p[-1] = 0.3
    g.gate_set_params(p)
    X = np.random.default_rng(12).uniform(-1, 1, (1000, 26)).astype(np.float32)
    prob = g.gate_forward(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    zq = ogate.forward(p, X, 2, quantize=True)
    z64 = ogate.forward(p, X, 2)
    sig = lambda z: 1 / (1 + np.exp(-z))  # noqa: E731
    assert np.abs(prob - sig(zq)).max() <= 2e-3
    assert np.abs(prob - sig(z64)).max() <= 3e-2


@pytest.mark.parametrize("dim", [2, 3])
def test_gradients_match_fp64_backprop(kfvm, dim):
    n_in = ogate.n_in(dim)
    g = kfvm.KFVM([8] * dim, dims=dim, radius=2)
    p = ogate.init_params(dim, seed=21)
    g.gate_set_params(p)
    rng = np.random.default_rng(22)
    X = rng.uniform(-1, 1, (777, n_in)).astype(np.float32)
    y = (rng.uniform(size=777) > 0.4).astype(np.float32)
    grads = torch.zeros(ogate.param_count(dim), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    g.gate_train_step(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), lr=0.0, loss=loss, grads=grads)
    torch.cuda.synchronize()
    gg = grads.cpu().numpy().astype(np.float64)
    # against backprop with the GPU's bf16 rounding points: only summation order and
    # float32 accumulation differ
    lq, gq = ogate.loss_and_grad(p, X, y, dim, quantize=True)
    assert abs(loss.item() - lq) <= 1e-4 * abs(lq)
    for a, b in zip(ogate.unpack(gg, dim), ogate.unpack(gq, dim)):
        a, b = np.ravel(a), np.ravel(b)
        assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b) + 1e-7
    # against exact FP64 backprop: bf16 operands (2^-9 relative rounding) compound over three layers
    lref, gref = ogate.loss_and_grad(p, X, y, dim)
    assert abs(loss.item() - lref) <= 1e-2 * abs(lref)
    for a, b in zip(ogate.unpack(gg, dim), ogate.unpack(gref, dim)):
        a, b = np.ravel(a), np.ravel(b)
        assert np.linalg.norm(a - b) <= 1e-1 * np.linalg.norm(b) + 1e-7
    # lr = 0 leaves the parameters unchanged
    assert np.array_equal(g.gate_get_params(), p)


def test_adam_step_updates_parameters(kfvm):
    g = kfvm.KFVM([8, 8], dims=2, radius=2)
    p = ogate.init_params(2, seed=31)
    g.gate_set_params(p)
    rng = np.random.default_rng(32)
    X = torch.from_numpy(rng.uniform(-1, 1, (256, 26)).astype(np.float32)).cuda()
    y = torch.from_numpy((rng.uniform(size=256) > 0.5).astype(np.float32)).cuda()
    grads = torch.zeros(ogate.param_count(2), dtype=torch.float32, device="cuda")
    g.gate_train_step(X, y, lr=1e-3, grads=grads)
    gr = grads.cpu().numpy()
    # first Adam step: m/bc1 = g, v/bc2 = g^2, so the update is lr * g / (|g| + 1e-8)
    want = p - 1e-3 * gr / (np.abs(gr) + 1e-8)
    assert np.allclose(g.gate_get_params(), want, rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("precision", [64, 32])
def test_gated_reconstruction_with_a_given_mask(kfvm, precision):
    n = (40, 24)
    U0 = workloads.voronoi_2d(48, k=10, seed=8)[:, :24, :40].contiguous()
    Xr = ogate.features(U0.numpy(), 2, "outflow")
    # a mask from the oracle's own gate features: smooth where the stencil of rho is nearly flat
    mask = (np.abs(Xr[:, :13]).max(axis=1) < 0.99).astype(np.uint8)
    mask[::7] = 1 - mask[::7]  # and some arbitrary flips, to mix linear and WENO cells inside every tile
    ref = oracle.Oracle(list(n), dim=2, R=2, bc="outflow", recon="gated", mask=mask)
    g = kfvm.KFVM(list(n), dims=2, radius=2, bc="outflow")
    g.set_option("precision", precision)
    g.set_smooth_mask(torch.from_numpy(mask).cuda())
    U = U0.cuda()
    U1r, _ = ref.step(U0.numpy(), 0.4)
    g.step(U, 0.4)
    err = np.abs(U.cpu().numpy() - U1r).max() / np.abs(U1r).max()
    assert err <= (1e-12 if precision == 64 else 2e-6), err


@pytest.mark.parametrize("precision", [64, 32])
def test_learned_mask_matches_oracle_gate(kfvm, precision):
    """The mask the gated step computes (features + tensor-core MLP) against the oracle's gate."""
    n = 64
    U0 = workloads.mixed_voronoi(2, n, 12, seed=13)
    g = kfvm.KFVM([n, n], dims=2, radius=2, bc="outflow")
    g.set_option("precision", precision)
    p = ogate.init_params(2, seed=41)
    p[-1] = 0.1
    g.gate_set_params(p)
    mask = g.gate_mask(U0.cuda()).cpu().numpy().ravel()
    Xr = ogate.features(U0.numpy(), 2, "outflow")
    pr = 1 / (1 + np.exp(-ogate.forward(p, Xr, 2, quantize=True)))
    far = np.abs(pr - 0.5) > 1e-2
    assert far.mean() > 0.9
    assert np.array_equal(mask[far] == 1, pr[far] > 0.5)


@pytest.mark.parametrize("precision", [64, 32])
def test_gated_reconstruction_3d_r3_with_a_given_mask(kfvm, precision):
    """3D, radius 3 (the float32 row-table kernel): a mixed linear/WENO mask against the oracle."""
    n = (10, 9, 6)
    U0 = workloads.mixed_voronoi(3, 10, 6, seed=17)[:, :n[2], :n[1], :n[0]].contiguous()
    Xr = ogate.features(U0.numpy(), 3, "outflow")
    mask = (np.abs(Xr[:, :33]).max(axis=1) < 0.99).astype(np.uint8)
    mask[::5] = 1 - mask[::5]
    ref = oracle.Oracle(list(n), dim=3, R=3, bc="outflow", recon="gated", mask=mask)
    g = kfvm.KFVM(list(n), dims=3, radius=3, bc="outflow")
    g.set_option("precision", precision)
    g.set_smooth_mask(torch.from_numpy(mask).cuda())
    U = U0.cuda()
    U1r, _ = ref.step(U0.numpy(), 0.4)
    g.step(U, 0.4)
    err = np.abs(U.cpu().numpy() - U1r).max() / np.abs(U1r).max()
    assert err <= (1e-12 if precision == 64 else 2e-6), err


@pytest.mark.parametrize("dim,R,n", [(2, 2, (40, 24)), (3, 2, (12, 9, 8)), (3, 3, (12, 9, 8))])
def test_fused_gate_decisions_equal_gate_mask(kfvm, dim, R, n):
    """The FP32 reconstruction's fused gate takes the decisions kfvm_gate_mask reports: its Riemann
    states equal those of a reconstruction driven by that mask, up to cells at the threshold.
    (A full step differs, since the fused gate re-decides on every stage's state.)"""
    m = max(n)
    U0 = workloads.mixed_voronoi(dim, m, 8, seed=19)
    U0 = (U0[:, :n[2], :n[1], :n[0]] if dim == 3 else U0[:, :n[1], :n[0]]).contiguous()
    g = kfvm.KFVM(list(n), dims=dim, radius=R, bc="outflow")
    g.set_option("precision", 32)
    g.gate_set_params(ogate.init_params(dim, seed=43))
    g.set_option("recon", 2)
    # threshold at the median probability, so that both branches are exercised
    X, _ = g.gate_features(U0.cuda(), 0.5)
    th = float(g.gate_forward(X).median().item())
    g.set_option("gate_threshold", min(max(th, 0.02), 0.98))
    mask = g.gate_mask(U0.cuda())
    assert 0.05 < mask.float().mean().item() < 0.95
    f2 = g.faces_primitive(g.reconstruct(U0.cuda())).cpu().numpy()
    h = kfvm.KFVM(list(n), dims=dim, radius=R, bc="outflow")
    h.set_option("precision", 32)
    h.set_smooth_mask(mask)
    f3 = h.faces_primitive(h.reconstruct(U0.cuda())).cpu().numpy()
    d = np.abs(f2 - f3).max(axis=(0, 1))
    assert (d > 0).mean() <= 0.01, (d > 0).mean()


@pytest.mark.parametrize("R", [2, 3])
def test_3d_features_with_shell_match_oracle(kfvm, R):
    """3D gate inputs, including the radius-3 shell inputs (zero at radius 2), against the oracle."""
    n = (11, 9, 8)
    U0 = workloads.mixed_voronoi(3, 11, 5, seed=23)[:, :n[2], :n[1], :n[0]].contiguous()
    g = kfvm.KFVM(list(n), dims=3, radius=R, bc="outflow")
    X, _ = g.gate_features(U0.cuda(), tau=0.5)
    Xg = X.cpu().numpy()
    Xr = ogate.features(U0.numpy(), 3, "outflow", R=R)
    assert Xg.shape == Xr.shape == (np.prod(n), 68)
    # blocks whose relative variation is far above float32 rounding agree to 1e-3 (as in 2D)
    from oracle import stencils
    U = U0.numpy()
    rho = U[0]
    p = 0.4 * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / rho)
    for blk, v in enumerate((rho, p)):
        P = np.pad(v, 2, mode="edge")
        amp = np.zeros(v.size)
        for o in stencils.full_stencil(3, 2):
            sl = P[2 + o[2]:2 + o[2] + n[2], 2 + o[1]:2 + o[1] + n[1], 2 + o[0]:2 + o[0] + n[0]]
            amp = np.maximum(amp, np.abs(sl - v).ravel())
        big = amp / np.abs(v).ravel() > 1e-4
        assert big.any()
        sl = slice(33 * blk, 33 * blk + 33)
        assert np.abs(Xg[big, sl] - Xr[big, sl]).max() <= 1e-3
        # shell input m/(m + d): float32 noise in a block that is flat to ~1e-7 moves it, so the
        # comparison covers the cells whose block varies, and (rho, formed without cancellation) all
        if R == 2:
            assert np.abs(Xg[:, 66 + blk]).max() == 0.0
        else:
            cells = slice(None) if blk == 0 else big
            assert np.abs(Xg[cells, 66 + blk] - Xr[cells, 66 + blk]).max() <= 1e-3


@pytest.mark.parametrize("R", [2, 3])
def test_3d_labels_match_oracle(kfvm, R):
    """3D training labels (float64 deltas, float32 indicators) against the oracle's FP64 labels, on the
    cells whose decision is not at a threshold."""
    n = (10, 9, 8)
    U0 = workloads.mixed_voronoi(3, 10, 5, seed=29)[:, :n[2], :n[1], :n[0]].contiguous()
    g = kfvm.KFVM(list(n), dims=3, radius=R, bc="outflow")
    _, y = g.gate_features(U0.cuda(), tau=0.5)
    o = oracle.Oracle(list(n), dim=3, R=R, bc="outflow")
    _, om = o.reconstruct(U0.numpy(), with_omega=True)
    amp = ogate.linprim_amplitude(U0.numpy(), 3, R, "outflow")
    yr, worst = ogate.labels_from_omega(om, 3, 0.5, amp)
    far = (np.abs(worst - 0.5) > 1e-3) & (np.abs(np.log10(np.maximum(amp[[0, -1]], 1e-30)) + 4).min(axis=0) > 0.05)
    assert far.mean() > 0.9
    assert np.array_equal(y.cpu().numpy()[far], yr[far])
    assert 0.05 < yr.mean() < 0.95


def test_gate_load_float32_and_bfloat16(kfvm):
    g = kfvm.KFVM([8, 8], dims=2, radius=2)
    p = ogate.init_params(2, seed=51)
    g.gate_load(p)
    assert np.array_equal(g.gate_get_params(), p)
    bits = (np.ascontiguousarray(ogate.bf16(p).astype(np.float32)).view(np.uint32) >> 16).astype(np.uint16)
    g.gate_load(bits)
    assert np.array_equal(g.gate_get_params(), ogate.bf16(p).astype(np.float32))
    with pytest.raises(kfvm.KfvmError):
        g.gate_load(p[:-1])


def test_gate_train_equals_consecutive_train_steps(kfvm):
    """kfvm_gate_train: one epoch over 5000 samples = Adam steps on batches 0-2047, 2048-4095, 4096-4999."""
    rng = np.random.default_rng(52)
    X = torch.from_numpy(rng.uniform(-1, 1, (5000, 26)).astype(np.float32)).cuda()
    y = torch.from_numpy((rng.uniform(size=5000) > 0.5).astype(np.float32)).cuda()
    p = ogate.init_params(2, seed=53)
    a = kfvm.KFVM([8, 8], dims=2, radius=2)
    a.gate_set_params(p)
    a.gate_train(X, y, epochs=1, lr=1e-3)
    b = kfvm.KFVM([8, 8], dims=2, radius=2)
    b.gate_set_params(p)
    for r0 in (0, 2048, 4096):
        r1 = min(r0 + 2048, 5000)
        b.gate_train_step(X[r0:r1].contiguous(), y[r0:r1].contiguous(), 1e-3)
    pa, pb = a.gate_get_params(), b.gate_get_params()
    # the gradients are float32 atomic sums, whose order varies between launches; Adam's first steps
    # move a parameter by ~lr * sign(gradient), so a component whose gradient is ~0 may differ by up to
    # 2 lr per step; all others agree to rounding
    d = np.abs(pa - pb)
    assert (d <= 1e-6 * np.abs(pb).max() + 1e-7).mean() >= 0.99
    assert d.max() <= 3 * 2e-3 + 1e-6
    assert np.abs(pa - p).max() > 1e-5  # the parameters moved
