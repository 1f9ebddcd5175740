"""Pins of the oracle's Riemann solvers (HLLC / HLL with Batten wave speeds, Sec. 5.4)."""
import numpy as np
import pytest

import oracle

G = 1.4


def cons(rho, vel, p):
    return np.array([rho] + [rho * v for v in vel] + [p / (G - 1) + 0.5 * rho * sum(v * v for v in vel)])


def euler_flux(U, dim, d):
    rho = U[0]
    vel = U[1:1 + dim] / rho
    p = (G - 1) * (U[-1] - 0.5 * rho * vel @ vel)
    f = np.empty_like(U)
    f[0] = rho * vel[d]
    f[1:1 + dim] = rho * vel[d] * vel
    f[1 + d] += p
    f[-1] = vel[d] * (U[-1] + p)
    return f


@pytest.mark.parametrize("solver", ["hllc", "hll"])
@pytest.mark.parametrize("dim", [2, 3])
def test_consistency(solver, dim):
    """F^(u, u) = F(u) (Eq. 1 flux) for any state and direction."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        u = cons(rng.uniform(0.1, 2), list(rng.uniform(-2, 2, dim)), rng.uniform(0.1, 2))
        for d in range(dim):
            f = oracle.riemann_flux(dim, G, d, u, u, solver)
            assert np.allclose(f, euler_flux(u, dim, d), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_hllc_resolves_stationary_contact(dim):
    """HLLC keeps an isolated stationary contact exact: flux = (0, p e_d, 0)."""
    uL = cons(1.0, [0.0] * dim, 0.7)
    uR = cons(0.2, [0.0] * dim, 0.7)
    for d in range(dim):
        f = oracle.riemann_flux(dim, G, d, uL, uR, "hllc")
        want = np.zeros(dim + 2)
        want[1 + d] = 0.7
        assert np.allclose(f, want, atol=1e-14)
    # HLL smears it (a nonzero mass flux)
    f = oracle.riemann_flux(dim, G, 0, uL, uR, "hll")
    assert abs(f[0]) > 1e-3


@pytest.mark.parametrize("solver", ["hllc", "hll"])
def test_supersonic_upwinding(solver):
    uL = cons(1.0, [5.0, 0.3], 1.0)
    uR = cons(0.5, [4.0, -0.2], 0.8)
    assert np.allclose(oracle.riemann_flux(2, G, 0, uL, uR, solver), euler_flux(uL, 2, 0), rtol=1e-14)
    uL = cons(1.0, [-5.0, 0.3], 1.0)
    uR = cons(0.5, [-4.0, -0.2], 0.8)
    assert np.allclose(oracle.riemann_flux(2, G, 0, uL, uR, solver), euler_flux(uR, 2, 0), rtol=1e-14)


@pytest.mark.parametrize("solver", ["hllc", "hll"])
def test_rotational_invariance(solver):
    """The y-flux of states equals the x-flux of the same states with x and y swapped."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        uL = cons(rng.uniform(0.1, 2), list(rng.uniform(-1, 1, 2)), rng.uniform(0.1, 2))
        uR = cons(rng.uniform(0.1, 2), list(rng.uniform(-1, 1, 2)), rng.uniform(0.1, 2))
        sw = [0, 2, 1, 3]
        fy = oracle.riemann_flux(2, G, 1, uL, uR, solver)
        fx = oracle.riemann_flux(2, G, 0, uL[sw], uR[sw], solver)
        assert np.allclose(fy, fx[sw], rtol=1e-13, atol=1e-14)


def test_mirror_antisymmetry():
    """Mirroring x swaps the states and negates the normal velocity: F0 flips sign."""
    rng = np.random.default_rng(9)
    for solver in ("hllc", "hll"):
        for _ in range(20):
            uL = cons(rng.uniform(0.1, 2), list(rng.uniform(-1, 1, 2)), rng.uniform(0.1, 2))
            uR = cons(rng.uniform(0.1, 2), list(rng.uniform(-1, 1, 2)), rng.uniform(0.1, 2))
            m = np.array([1, -1, 1, 1.0])
            f = oracle.riemann_flux(2, G, 0, uL, uR, solver)
            g = oracle.riemann_flux(2, G, 0, uR * m, uL * m, solver)
            # mass, transverse momentum and energy fluxes change sign; normal momentum flux does not
            assert np.allclose(g, f * np.array([-1, 1, -1, -1]), rtol=1e-12, atol=1e-14)
