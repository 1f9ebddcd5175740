"""Pins of the oracle's reconstruction stage (Sec. 3.2-3.4, Sec. 5.3 step 2)."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import stencils

G = 1.4


def _prim_to_cons(rho, vel, p):
    return np.array([rho] + [rho * v for v in vel] + [p / (G - 1) + 0.5 * rho * sum(v * v for v in vel)])


def _cons_to_prim(U, dim):
    rho = U[0]
    vel = U[1:1 + dim] / rho
    p = (G - 1) * (U[dim + 1] - 0.5 * rho * np.sum(vel * vel))
    return np.concatenate([[rho], vel, [p]])


@pytest.mark.parametrize("dim", [2, 3])
def test_phi_is_jacobian_and_inverse(dim):
    """Phi = dV/dU and Phi^{-1} = dU/dV (appendix A), checked by central differences."""
    rng = np.random.default_rng(dim)
    ut = _prim_to_cons(rng.uniform(0.5, 2), list(rng.uniform(-1, 1, dim)), rng.uniform(0.5, 2))
    phi, phinv = oracle.phi_matrices(dim, G, ut)
    assert np.max(np.abs(phi @ phinv - np.eye(dim + 2))) < 1e-14
    h = 1e-6
    J = np.zeros_like(phi)
    for j in range(dim + 2):
        e = np.zeros(dim + 2)
        e[j] = h
        J[:, j] = (_cons_to_prim(ut + e, dim) - _cons_to_prim(ut - e, dim)) / (2 * h)
    assert np.max(np.abs(J - phi)) < 1e-8
    vt = _cons_to_prim(ut, dim)
    Ji = np.zeros_like(phi)
    for j in range(dim + 2):
        e = np.zeros(dim + 2)
        e[j] = h
        Ji[:, j] = (_prim_to_cons(vt[0] + e[0], vt[1:1 + dim] + e[1:1 + dim], vt[-1] + e[-1])
                    - _prim_to_cons(vt[0] - e[0], vt[1:1 + dim] - e[1:1 + dim], vt[-1] - e[-1])) / (2 * h)
    assert np.max(np.abs(Ji - phinv)) < 1e-8


def _grid_coords(n, dim):
    c = [(np.arange(n) + 0.5) / n for _ in range(dim)]
    return list(reversed(np.meshgrid(*reversed(c), indexing="ij")))


@pytest.mark.parametrize("dim,R", [(2, 2), (2, 3), (3, 2)])
def test_constant_data(dim, R):
    n = 8
    o = oracle.Oracle([n] * dim, dim=dim, R=R)
    U = workloads.constant_state(dim, [n] * dim, rho=0.7, p=0.4).numpy()
    faces, om = o.reconstruct(U, with_omega=True)
    assert np.max(np.abs(faces - U[None])) < 1e-14
    g = np.array(stencils.linear_weights(dim))
    assert np.max(np.abs(om - g.reshape((-1,) + (1,) * (dim + 1)))) < 1e-15


@pytest.mark.parametrize("dim,R", [(2, 2), (2, 3), (3, 2)])
def test_linear_data_recovers_linear_weights_and_exact_values(dim, R):
    """Linear data: every substencil reproduces degree 1 exactly, so all beta_q are equal,
    omega = gamma, and the WENO-AO state equals the exact point value (Eq. 19)."""
    n = 12
    h = 1.0 / n
    o = oracle.Oracle([n] * dim, dim=dim, R=R, bc="outflow")
    X = _grid_coords(n, dim)
    a = [0.3, -0.2, 0.1][:dim]
    rho = 1.0 + sum(a[k] * X[k] for k in range(dim))  # cell averages of linear data are centre values
    mx = 0.2 + 0.1 * X[0]
    U = np.stack([rho, mx] + [0.05 * X[k] for k in range(1, dim)] + [2.5 + 0.2 * X[-1]])
    faces, om = o.reconstruct(U, with_omega=True)
    gam = np.array(stencils.linear_weights(dim))
    # interior cells (outflow ghosts break linearity near the boundary)
    sl = (slice(None), slice(None)) + tuple(slice(R + 1, n - R - 1) for _ in range(dim))
    inner_om = om[sl]
    assert np.max(np.abs(inner_om - gam.reshape((-1,) + (1,) * (dim + 1)))) < 1e-9
    pts = oracle.face_points(dim, R)
    for s in range(len(pts)):
        Xs = [X[k] + pts[s, k] * h for k in range(dim)]
        want = np.stack([1.0 + sum(a[k] * Xs[k] for k in range(dim)), 0.2 + 0.1 * Xs[0]]
                        + [0.05 * Xs[k] for k in range(1, dim)] + [2.5 + 0.2 * Xs[-1]])
        got = faces[s]
        inner = (slice(None),) + tuple(slice(R + 1, n - R - 1) for _ in range(dim))
        assert np.max(np.abs(got[inner] - want[inner])) < 1e-12


def test_linear_mode_is_exact_for_cubics():
    """S0 (degree 3 at radius 2) reproduces cubic data in the unlimited mode."""
    n, dim, R = 10, 2, 2
    h = 1.0 / n
    o = oracle.Oracle([n, n], dim=dim, R=R, bc="outflow", recon="linear")
    # exact cell averages of x^3 + x y^2 + y on unit-square cells of width h
    def avg_x3(xc):
        return ((xc + h / 2) ** 4 - (xc - h / 2) ** 4) / (4 * h)

    def avg_x2(xc):
        return ((xc + h / 2) ** 3 - (xc - h / 2) ** 3) / (3 * h)

    X, Y = _grid_coords(n, 2)
    f = avg_x3(X) + X * avg_x2(Y) + Y
    U = np.stack([2 + f, 0.1 * f, -0.1 * f, 5 + f])
    faces = o.reconstruct(U)
    pts = oracle.face_points(dim, R)
    inner = slice(R, n - R)
    for s in range(len(pts)):
        xs, ys = X + pts[s, 0] * h, Y + pts[s, 1] * h
        fs = xs ** 3 + xs * ys ** 2 + ys
        assert np.max(np.abs(faces[s, 0][inner, inner] - (2 + fs)[inner, inner])) < 1e-12


def test_step_data_switches_off_crossing_substencils():
    """A jump in x kills the weights of substencils that straddle it (Sec. 3.2)."""
    n, dim, R = 16, 2, 2
    o = oracle.Oracle([n, n], dim=dim, R=R, bc="outflow")
    X, Y = _grid_coords(n, 2)
    rho = np.where(X < 0.5, 1.0, 0.125)
    p = np.where(X < 0.5, 1.0, 0.1)
    U = np.stack([rho, 0 * rho, 0 * rho, p / (G - 1)])
    _, om = o.reconstruct(U, with_omega=True)
    i = n // 2 - 1  # last cell left of the jump: S2 (x-biased, +x side) crosses it, S3 does not
    w = om[:, 0, n // 2, i]
    assert w[3] > 0.99
    assert w[0] < 1e-10 and w[2] < 1e-10
    assert abs(om.sum(0) - 1).max() < 1e-14


def test_weights_sum_to_one_on_random_data():
    n = 12
    o = oracle.Oracle([n, n], dim=2, R=2)
    U = workloads.voronoi_2d(n, k=8, seed=11).numpy()
    _, om = o.reconstruct(U, with_omega=True)
    assert abs(om.sum(0) - 1).max() < 1e-14
    assert om.min() >= 0


def _prim(f, dim):
    rho = f[:, 0]
    ke = 0.5 * sum(f[:, 1 + k] ** 2 for k in range(dim)) / rho
    return rho, (G - 1) * (f[:, dim + 1] - ke)


def test_limiter_enforces_bounds_by_uniform_contraction():
    """Sec. 4: after the limiter every Riemann state of a cell lies within the
    data-dependent bounds, and the states moved toward the cell average by one
    common factor theta in [0, 1] (Eqs. 37, 38)."""
    n, dim, kappa = 48, 2, 0.1
    o = oracle.Oracle([n, n], dim=dim, R=2, bc="outflow", kappa=kappa)
    U = workloads.voronoi_2d(n).numpy()
    raw = o.reconstruct(U)
    lim = o.limit(U, raw)
    assert o.status == 0
    rho, p = _prim(lim, dim)
    # neighbourhood bounds (3x3, clamped at the outflow edges)
    Up = np.pad(U, ((0, 0), (1, 1), (1, 1)), mode="edge")
    rb = np.stack([Up[0, 1 + j:1 + j + n, 1 + i:1 + i + n] for j in (-1, 0, 1) for i in (-1, 0, 1)])
    pb = np.stack([(G - 1) * (Up[3] - 0.5 * (Up[1] ** 2 + Up[2] ** 2) / Up[0])[1 + j:1 + j + n, 1 + i:1 + i + n]
                   for j in (-1, 0, 1) for i in (-1, 0, 1)])
    assert np.all(rho >= rb.min(0) * (1 - kappa) * (1 - 1e-14))
    assert np.all(rho <= rb.max(0) * (1 + kappa) * (1 + 1e-14))
    assert np.all(p >= pb.min(0) * (1 - kappa) * (1 - 1e-12))
    # one common contraction factor per cell
    d_raw = raw - U[None]
    d_lim = lim - U[None]
    changed = 0
    for y in range(n):
        for x in range(n):
            a, b = d_raw[:, :, y, x].ravel(), d_lim[:, :, y, x].ravel()
            th = (a @ b) / (a @ a) if a @ a > 0 else 1.0
            assert -1e-14 <= th <= 1 + 1e-14
            assert np.allclose(b, th * a, rtol=0, atol=1e-12)
            changed += th < 1 - 1e-12
    assert changed > 0


def test_limiter_inactive_on_smooth_data():
    n = 32
    o = oracle.Oracle([n, n], dim=2, R=2)
    U = workloads.sine_2d(n).numpy()
    raw = o.reconstruct(U)
    assert np.array_equal(o.limit(U, raw), raw)
