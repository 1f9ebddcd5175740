"""Pins of the oracle's WENO-AO in characteristic variables (Sec. 3.4.1).

Per direction the reference state's flux Jacobian A = dF/dU is diagonalised, A = R Lambda L, and the
reconstruction runs in W = L U with Phi^{-1} = R.  Pinned by
* L R = I, and L A R = diag(u_n - c, u_n, ..., u_n + c) with A from central finite differences of
  the Euler flux written out here (not the eigenvector formulas);
* constant data reconstructed exactly, linear data reconstructed exactly at every face point
  (all smoothness indicators equal, so the weights are the linear ones);
* the step: free stream, periodic conservation, mirror symmetry, no y dependence on x-only data, and
  the Sod problem against its exact solution, as close to it as the linearized primitive variables.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from tests.test_oracle_step import _sod_exact

G = 1.4


def _flux(U, d, dim):
    rho, m, E = U[0], U[1:1 + dim], U[dim + 1]
    p = (G - 1) * (E - 0.5 * (m @ m) / rho)
    un = m[d] / rho
    f = np.empty(dim + 2)
    f[0] = m[d]
    f[1:1 + dim] = m * un
    f[1 + d] += p
    f[dim + 1] = un * (E + p)
    return f


def _states(dim, k=6, seed=3):
    rng = np.random.default_rng(seed)
    for _ in range(k):
        rho = rng.uniform(0.2, 2.0)
        u = rng.uniform(-1.5, 1.5, dim)
        p = rng.uniform(0.1, 3.0)
        yield np.concatenate([[rho], rho * u, [p / (G - 1) + 0.5 * rho * (u @ u)]])


@pytest.mark.parametrize("dim", [2, 3])
def test_eigenvectors_diagonalise_the_flux_jacobian(dim):
    nv = dim + 2
    for U in _states(dim):
        rho, u = U[0], U[1:1 + dim] / U[0]
        p = (G - 1) * (U[-1] - 0.5 * rho * (u @ u))
        c = math.sqrt(G * p / rho)
        for d in range(dim):
            L, R = oracle.char_matrices(dim, G, U, d)
            assert np.abs(L @ R - np.eye(nv)).max() < 1e-13
            h = 1e-6
            A = np.empty((nv, nv))
            for j in range(nv):
                e = np.zeros(nv)
                e[j] = h * max(1.0, abs(U[j]))
                A[:, j] = (_flux(U + e, d, dim) - _flux(U - e, d, dim)) / (2 * e[j])
            lam = L @ A @ R
            want = np.diag([u[d] - c] + [u[d]] * (nv - 2) + [u[d] + c])
            assert np.abs(lam - want).max() < 1e-7 * max(1.0, np.abs(want).max()), (d, lam)


@pytest.mark.parametrize("dim,R", [(2, 2), (2, 3), (3, 2)])
def test_constant_and_linear_data_are_exact(dim, R):
    n = [9, 8, 7][:dim]
    o = oracle.Oracle(n, dim=dim, R=R, bc="periodic", variables="characteristic", positivity=False)
    U = workloads.constant_state(dim, n, rho=0.7, vel=[0.3, -0.6, 0.2][:dim], p=1.3).numpy()
    f = o.reconstruct(U)
    assert np.abs(f - U[None]).max() < 1e-14 * np.abs(U).max()
    # linear conservative data: cell averages equal the centre values; every face point exact
    h = R + 1  # cells whose stencils stay inside the grid
    n = [2 * h + 3, 2 * h + 2, 2 * h + 1][:dim]
    oo = oracle.Oracle(n, dim=dim, R=R, bc="outflow", variables="characteristic", positivity=False)
    axes = [np.arange(k) + 0.5 for k in n]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]  # x, y(, z) arrays of shape (z,) y, x
    coef = np.array([[1.0, 0.01, -0.02, 0.015], [0.2, 0.01, 0.005, -0.01], [-0.1, 0.004, 0.01, 0.02],
                     [0.05, -0.01, 0.02, 0.01], [3.0, 0.02, -0.03, 0.01]])[:dim + 2]
    U = np.stack([coef[v, 0] + sum(coef[v, 1 + a] * grids[a] for a in range(dim)) for v in range(dim + 2)])
    f = oo.reconstruct(np.ascontiguousarray(U))
    pts = oracle.face_points(dim, R)
    inner = (slice(None), slice(None)) + tuple(slice(h, k - h) for k in reversed(n))
    for s, x in enumerate(pts):
        want = np.stack([coef[v, 0] + sum(coef[v, 1 + a] * (grids[a] + x[a]) for a in range(dim))
                         for v in range(dim + 2)])
        assert np.abs(f[s][inner[1:]] - want[inner[1:]]).max() < 1e-12, s


def test_step_invariants():
    n = 16
    U = workloads.voronoi_2d(n, k=10, seed=31).numpy()
    o = oracle.Oracle([n, n], dim=2, R=2, bc="outflow", variables="characteristic")
    # free stream
    c = workloads.constant_state(2, [n, n], rho=0.9, vel=[0.4, -0.3], p=0.6).numpy()
    c1, _ = o.step(c, 0.4)
    assert np.abs(c1 - c).max() < 1e-14 * np.abs(c).max()
    # mirror symmetry x -> 1 - x
    Um = U[:, :, ::-1].copy()
    Um[1] *= -1
    U1, dt1 = o.step(U, 0.4)
    V1, dt2 = o.step(Um, 0.4)
    assert o.status == 0 and dt1 == dt2
    V1 = V1[:, :, ::-1]
    V1[1] *= -1
    assert np.abs(U1 - V1).max() < 1e-13
    # periodic conservation
    op = oracle.Oracle([n, n], dim=2, R=2, bc="periodic", variables="characteristic")
    P1, _ = op.step(U, 0.4)
    for v in range(4):
        assert abs(math.fsum(P1[v].ravel()) - math.fsum(U[v].ravel())) <= 1e-13 * math.fsum(np.abs(U[v]).ravel())
    # the reconstruction differs from the linearized primitive one away from smooth data
    ol = oracle.Oracle([n, n], dim=2, R=2, bc="outflow")
    assert np.abs(o.reconstruct(U) - ol.reconstruct(U)).max() > 1e-3


@pytest.mark.parametrize("R", [2, 3])
def test_sod_against_exact_solution(R):
    nx, ny = 100, 2
    x = (np.arange(nx) + 0.5) / nx
    U = np.zeros((4, ny, nx))
    U[0] = np.where(x < 0.5, 1.0, 0.125)
    U[3] = np.where(x < 0.5, 1.0, 0.1) / (G - 1)
    ex = _sod_exact(x, 0.2)
    err = {}
    for variables in ("characteristic", "linprim"):
        o = oracle.Oracle([nx, ny], dim=2, R=R, lo=[0, 0], hi=[1.0, 0.02], bc=["outflow", "periodic"],
                          variables=variables)
        V, t, k = o.run(U.copy(), 0.4, 0.2)
        err[variables] = np.abs(V[0, 0] - ex).mean()
        assert np.max(np.abs(V[:, 0] - V[:, 1])) < 1e-13
    assert err["characteristic"] < 6e-3, err
    assert err["characteristic"] <= 1.25 * err["linprim"], err


def test_y_aligned_problem_is_the_transposed_x_problem():
    """The y faces take the y direction's eigenvectors: the Sod problem along y, with x and y (and the
    momenta) swapped, gives the transposed solution to round-off."""
    nx, ny = 40, 3
    x = (np.arange(nx) + 0.5) / nx
    U = np.zeros((4, ny, nx))
    U[0] = np.where(x < 0.5, 1.0, 0.125)
    U[1] = 0.3
    U[2] = 0.2
    U[3] = np.where(x < 0.5, 1.0, 0.1) / (G - 1) + 0.5 * (0.09 + 0.04) / U[0]
    ox = oracle.Oracle([nx, ny], dim=2, R=2, lo=[0, 0], hi=[1.0, ny / nx], bc=["outflow", "periodic"],
                       variables="characteristic")
    oy = oracle.Oracle([ny, nx], dim=2, R=2, lo=[0, 0], hi=[ny / nx, 1.0], bc=["periodic", "outflow"],
                       variables="characteristic")
    V = np.ascontiguousarray(np.stack([U[0].T, U[2].T, U[1].T, U[3].T]))
    Ux, _, _ = ox.run(U, 0.4, 0.05)
    Vy, _, _ = oy.run(V, 0.4, 0.05)
    back = np.stack([Vy[0].T, Vy[2].T, Vy[1].T, Vy[3].T])
    assert np.abs(Ux - back).max() < 1e-13


def test_z_aligned_problem_is_the_permuted_x_problem():
    """3D: the Sod-like problem along z, with x and z (and their momenta) exchanged, gives the
    permuted solution of the problem along x: the z faces take the z direction's eigenvectors."""
    n, m = 16, 3
    x = (np.arange(n) + 0.5) / n
    rho = np.where(x < 0.5, 1.0, 0.125)
    p = np.where(x < 0.5, 1.0, 0.1)
    u, v, w = 0.3, 0.2, -0.1
    U = np.zeros((5, m, m, n))  # [var][z][y][x], varying along x
    U[0] = rho
    U[1] = rho * u
    U[2] = rho * v
    U[3] = rho * w
    U[4] = p / (G - 1) + 0.5 * rho * (u * u + v * v + w * w)
    ox = oracle.Oracle([n, m, m], dim=3, R=2, hi=[1.0, m / n, m / n],
                       bc=[("outflow", "outflow"), ("periodic", "periodic"), ("periodic", "periodic")],
                       variables="characteristic")
    oz = oracle.Oracle([m, m, n], dim=3, R=2, hi=[m / n, m / n, 1.0],
                       bc=[("periodic", "periodic"), ("periodic", "periodic"), ("outflow", "outflow")],
                       variables="characteristic")
    # exchange x and z: array axes (z, y, x) -> (x, y, z), momenta m_x <-> m_z
    V = np.ascontiguousarray(np.stack([U[0].transpose(2, 1, 0), U[3].transpose(2, 1, 0), U[2].transpose(2, 1, 0),
                                       U[1].transpose(2, 1, 0), U[4].transpose(2, 1, 0)]))
    Ux, _, _ = ox.run(np.ascontiguousarray(U), 0.4, 0.05)
    Vz, _, _ = oz.run(V, 0.4, 0.05)
    back = np.stack([Vz[0].transpose(2, 1, 0), Vz[3].transpose(2, 1, 0), Vz[2].transpose(2, 1, 0),
                     Vz[1].transpose(2, 1, 0), Vz[4].transpose(2, 1, 0)])
    assert np.abs(Ux - back).max() < 1e-13
