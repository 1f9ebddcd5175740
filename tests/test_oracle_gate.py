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
                want.append(d / max(np.abs(d).max(), 1e-6 * abs(v[c]) + 1e-30))
            assert np.allclose(f[j * n + i], np.concatenate(want), atol=1e-13)


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
