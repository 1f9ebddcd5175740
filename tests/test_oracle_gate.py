"""Pins of the gate oracle (the gate has no counterpart in the paper; these pin the
definitions themselves against independent computations)."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import gate


@pytest.mark.parametrize("dim", [2, 3])
def test_quantized_backprop_is_close_to_exact(dim):
    """The bf16-rounding variant differs from exact backprop by bf16-sized amounts only."""
    rng = np.random.default_rng(5)
    p = gate.init_params(dim, seed=6).astype(np.float64)
    X = rng.uniform(-1, 1, (300, gate.n_in(dim)))
    y = (rng.uniform(size=300) > 0.5).astype(np.float64)
    l0, g0 = gate.loss_and_grad(p, X, y, dim)
    l1, g1 = gate.loss_and_grad(p, X, y, dim, quantize=True)
    assert abs(l1 - l0) < 2e-2 * l0
    assert np.linalg.norm(g1 - g0) < 0.1 * np.linalg.norm(g0)


@pytest.mark.parametrize("dim", [2, 3])
def test_backprop_matches_central_differences(dim):
    rng = np.random.default_rng(1)
    p = gate.init_params(dim, seed=3).astype(np.float64)
    X = rng.uniform(-1, 1, (40, gate.n_in(dim)))
    y = (rng.uniform(size=40) > 0.5).astype(np.float64)
    _, g = gate.loss_and_grad(p, X, y, dim)
    h = 1e-6
    idx = rng.choice(p.size, 60, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (gate.loss_and_grad(p + e, X, y, dim)[0] - gate.loss_and_grad(p - e, X, y, dim)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_constant_network_loss_closed_form():
    """All weights zero, bias b: z = b everywhere, loss = mean(softplus(b) - b y)."""
    dim = 2
    p = np.zeros(gate.param_count(dim))
    p[-1] = 0.7
    X = np.random.default_rng(2).uniform(-1, 1, (17, gate.n_in(dim)))
    y = np.array([1.0] * 10 + [0.0] * 7)
    loss, g = gate.loss_and_grad(p, X, y, dim)
    want = np.mean(np.log1p(np.exp(0.7)) - 0.7 * y)
    assert abs(loss - want) < 1e-14
    s = 1 / (1 + np.exp(-0.7))
    assert abs(g[-1] - np.mean(s - y)) < 1e-14


def test_features_shift_scale_invariant_and_zero_on_constants():
    n = 16
    U = workloads.voronoi_2d(n, k=5, seed=4).numpy()
    f = gate.features(U, 2, "outflow")
    assert f.shape == (n * n, 26)
    assert np.abs(f).max() <= 1 + 1e-12
    # scaling density and pressure (rho -> a rho, m -> a m, E -> a E scales p by a) leaves features unchanged
    f2 = gate.features(3.0 * U, 2, "outflow")
    assert np.allclose(f, f2, atol=1e-9)
    C = workloads.constant_state(2, [n, n]).numpy()
    assert np.abs(gate.features(C, 2)).max() == 0.0


def test_features_match_direct_stencil_loop():
    """Brute-force loop over cells and stencil offsets (periodic) against the vectorised definition."""
    n = 7
    U = workloads.mixed_voronoi(2, n, 3, seed=9).numpy()
    f = gate.features(U, 2, "periodic")
    s0 = oracle.stencils.full_stencil(2, 2)
    for j in range(n):
        for i in range(n):
            rho = np.array([U[0, (j + o[1]) % n, (i + o[0]) % n] for o in s0])
            E = np.array([U[3, (j + o[1]) % n, (i + o[0]) % n] for o in s0])
            m2 = np.array([U[1, (j + o[1]) % n, (i + o[0]) % n] ** 2 + U[2, (j + o[1]) % n, (i + o[0]) % n] ** 2
                           for o in s0])
            p = 0.4 * (E - 0.5 * m2 / rho)
            want = []
            c = s0.index((0, 0, 0))
            for v in (rho, p):
                d = v - v[c]
                want.append(d / max(np.abs(d).max(), 1e-4 * abs(v[c]) + 1e-30))
            assert np.allclose(f[j * n + i], np.concatenate(want), atol=1e-13)


def test_3d_shell_features_see_a_jump_three_cells_away():
    """A density jump at distance 3 from a cell is invisible to the radius-2 blocks (exactly zero)
    but sets the radius-3 shell input of rho to ~1; constant data gives zero shell inputs; the
    shell inputs are zero when the reconstruction radius is 2; a brute-force loop over the 90
    shell offsets agrees."""
    n = 10
    C = workloads.constant_state(3, [n, n, n])
    U = C.clone().numpy()
    U[:, :, :, 6:] *= 2.0  # rho, m, E doubled for x >= 6: a jump in rho (and p), velocity unchanged
    f = gate.features(U, 3, "outflow", R=3)
    assert f.shape == (n ** 3, 68) and gate.n_in(3) == 68
    assert len(gate.shell_offsets()) == 90
    cell = (5 * n + 5) * n + 3  # x = 3: the jump is 3 cells away
    assert np.abs(f[cell, :66]).max() == 0.0
    assert f[cell, 66] > 0.99 and f[cell, 67] > 0.99
    far = (5 * n + 5) * n + 1  # x = 1: 5 cells away
    assert np.abs(f[far]).max() == 0.0
    assert np.abs(gate.features(C.numpy(), 3, "outflow", R=3)).max() == 0.0
    assert np.abs(gate.features(U, 3, "outflow", R=2)[:, 66:]).max() == 0.0
    # brute force on a periodic smooth/constant mix
    m = 7
    V = workloads.mixed_voronoi(3, m, 3, seed=12).numpy()
    fv = gate.features(V, 3, "periodic", R=3)
    sh = gate.shell_offsets()
    s0 = oracle.stencils.full_stencil(3, 2)
    for k, j, i in [(0, 0, 0), (3, 5, 1), (6, 2, 4)]:
        def at(o, v):
            return V[v, (k + o[2]) % m, (j + o[1]) % m, (i + o[0]) % m]
        for blk in range(2):
            if blk == 0:
                val = lambda o: at(o, 0)  # noqa: E731
            else:
                val = lambda o: 0.4 * (at(o, 4) - 0.5 * sum(at(o, 1 + q) ** 2 for q in range(3)) / at(o, 0))  # noqa: E731
            vc = val((0, 0, 0))
            d = max(max(abs(val(o) - vc) for o in s0), 1e-4 * abs(vc) + 1e-30)
            ms = max(abs(val(o) - vc) for o in sh)
            assert abs(fv[(k * m + j) * m + i, 66 + blk] - ms / (ms + d)) <= 1e-13


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -2.5], dtype=np.float32)
    r = gate.bf16(x)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7 and goes to the even mantissa (1.0)
    assert list(r) == [1.0, 1.0, 1.0, 1.0 + 2 ** -7, -2.5]


def test_gated_oracle_reduces_to_its_two_modes():
    n = 12
    U = workloads.voronoi_2d(n, k=5, seed=6).numpy()
    ones = np.ones(n * n, dtype=np.uint8)
    zeros = np.zeros(n * n, dtype=np.uint8)
    lin = oracle.Oracle([n, n], dim=2, R=2, bc="outflow", recon="linear").reconstruct(U)
    wen = oracle.Oracle([n, n], dim=2, R=2, bc="outflow").reconstruct(U)
    g1 = oracle.Oracle([n, n], dim=2, R=2, bc="outflow", recon="gated", mask=ones).reconstruct(U)
    g0 = oracle.Oracle([n, n], dim=2, R=2, bc="outflow", recon="gated", mask=zeros).reconstruct(U)
    assert np.array_equal(g1, lin) and np.array_equal(g0, wen)


def test_amplitude_clause_marks_constant_and_tiny_variations_smooth():
    n = 12
    C = workloads.constant_state(2, [n, n]).numpy()
    amp = gate.linprim_amplitude(C, 2, 2)
    assert amp.max() == 0.0
    rng = np.random.default_rng(3)
    U = C * (1 + 1e-9 * rng.uniform(-1, 1, C.shape))
    o = oracle.Oracle([n, n], dim=2, R=2)
    _, om = o.reconstruct(U, with_omega=True)
    y, _ = gate.labels_from_omega(om, 2, 0.5, gate.linprim_amplitude(U, 2, 2))
    assert y.min() == 1.0
    # a real jump is not rescued by the clause
    V = workloads.voronoi_2d(n, k=3, seed=1).numpy()
    _, om = oracle.Oracle([n, n], dim=2, R=2, bc="outflow").reconstruct(V, with_omega=True)
    y, _ = gate.labels_from_omega(om, 2, 0.5, gate.linprim_amplitude(V, 2, 2, "outflow"))
    assert y.min() == 0.0


def test_labels_count_density_and_pressure_only():
    """The label looks at the density and pressure components of the linearized primitive variables
    (what the features describe): a velocity component whose weights say non-smooth does not change
    it, the density or the pressure component does."""
    g = oracle.stencils.linear_weights(2)
    nq, nv, ncell = len(g), 4, 3
    om = np.tile(np.asarray(g)[:, None, None], (1, nv, ncell))  # omega = gamma: smooth everywhere
    bad = np.zeros(nq)
    bad[0], bad[1] = 0.1, 0.9  # omega_0 / gamma_0 = 0.125
    om[:, 1, 0] = bad  # cell 0: u non-smooth
    om[:, 0, 1] = bad  # cell 1: rho non-smooth
    om[:, 3, 2] = bad  # cell 2: p non-smooth
    y, worst = gate.labels_from_omega(om, 2, 0.5)
    assert list(y) == [1.0, 0.0, 0.0]
    assert worst[0] == 1.0 and abs(worst[1] - 0.125) < 1e-15
