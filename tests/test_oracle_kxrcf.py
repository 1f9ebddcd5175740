"""Pins of the oracle's KXRCF troubled-cell indicator (Sec. 3.5; Sec. 5.3 step 2).

The indicator flags a cell for WENO-AO when the relative jump of the entropy
q = p / rho^gamma between its own unlimited linear reconstruction and its
neighbours' at the shared face Gauss points reaches Delta^m (m = 3/2).  Pinned by

* constant data: every jump vanishes, nothing is flagged;
* cubic data: the linear S0 reconstruction reproduces polynomials of degree
  2R - 1 = 3 exactly (Sec. 2.1), so both sides of every interior face agree at
  every Gauss point -- which fails if a point is matched with the wrong
  transverse point or side;
* a contact discontinuity: only cells whose own or neighbours' stencils reach
  across the jump can be flagged, the two cells touching it are, and the
  transposed problem gives the transposed mask;
* smooth data: the largest ratio decays like Delta^(2R) (the paper's "ideally"),
  i.e. with an observed order of about four at R = 2;
* the ratio's homogeneity: scaling (rho, m, E) by lambda leaves it unchanged;
* brute force: every ratio recomputed by physical coordinates -- each face point
  located in space, the cell across it found by position (periodic wrap,
  outflow skip), both reconstructions evaluated there through the coefficient
  form of the KFVM expansion (Eq. 10 solved at 40 digits with quadrature
  entries) -- without the oracle's point-index arithmetic.
"""
import numpy as np
import pytest

import oracle
import workloads

GAMMA = 1.4


def _poly_state_2d(nx, ny):
    """Exact cell averages of cubic conservative variables on [0, 1]^2 (positive rho and p)."""
    def avg(a, b):
        x0 = np.arange(nx) / nx
        x1 = (np.arange(nx) + 1) / nx
        y0 = np.arange(ny) / ny
        y1 = (np.arange(ny) + 1) / ny
        ix = (x1 ** (a + 1) - x0 ** (a + 1)) / (a + 1) * nx
        iy = (y1 ** (b + 1) - y0 ** (b + 1)) / (b + 1) * ny
        return np.outer(iy, ix)

    def poly(terms):
        return sum(c * avg(a, b) for c, a, b in terms)

    rho = poly([(1.5, 0, 0), (0.3, 1, 0), (-0.2, 0, 1), (0.1, 2, 1), (0.2, 0, 3)])
    mx = poly([(0.1, 0, 0), (0.2, 1, 1)])
    my = poly([(-0.1, 0, 0), (0.3, 2, 0)])
    E = poly([(3.0, 0, 0), (1.0, 3, 0), (-1.0, 0, 1), (0.5, 1, 1)])
    return np.stack([rho, mx, my, E])


def _contact(nx, ny, j, axis=0):
    """rho = 1 left of the face x_j (0.125 right of it), u = 0.3, v = -0.2, p = 1 (a contact)."""
    rho = np.where(np.arange(nx) < j, 1.0, 0.125)[None, :].repeat(ny, 0)
    u, v, p = 0.3, -0.2, 1.0
    U = np.stack([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)])
    if axis == 1:
        U = np.stack([U[0].T, U[2].T, U[1].T, U[3].T])
    return np.ascontiguousarray(U)


@pytest.mark.parametrize("bc", ["periodic", "outflow"])
@pytest.mark.parametrize("dim,R", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_constant_state_has_no_jumps(dim, R, bc):
    n = [9, 7, 6][:dim]
    U = workloads.constant_state(dim, n, rho=0.7, vel=[0.4, -0.3, 0.2][:dim], p=2.5).numpy()
    r, m = oracle.Oracle(n, dim=dim, R=R, bc=bc).kxrcf(U)
    assert r.max() <= 1e-13
    assert m.all()


@pytest.mark.parametrize("R", [2])
def test_cubic_data_has_no_interior_jumps(R):
    nx, ny = 20, 16
    U = _poly_state_2d(nx, ny)
    r, m = oracle.Oracle([nx, ny], dim=2, R=R, bc="outflow").kxrcf(U)
    h = R + 1  # cells whose own and neighbours' stencils stay inside the grid
    inner = r[h:ny - h, h:nx - h]
    assert inner.max() <= 1e-12, inner.max()
    # next to the clamped ghost cells the reconstruction is no longer exact
    assert r.max() > 1e-8


@pytest.mark.parametrize("R", [2, 3])
def test_contact_flags_only_cells_that_see_it(R):
    nx, ny, j = 24, 8, 12
    o = oracle.Oracle([nx, ny], dim=2, R=R, bc="outflow")
    r, m = o.kxrcf(_contact(nx, ny, j))
    flagged_cols = np.where((m == 0).any(axis=0))[0]
    # cell i sees the jump through its own stencil (i-R..i+R) or a neighbour's (i-1-R..i+1+R)
    assert flagged_cols.min() >= j - R - 1 and flagged_cols.max() <= j + R, flagged_cols
    assert (m[:, j - 1] == 0).all() and (m[:, j] == 0).all()
    far = np.r_[0:j - R - 1, j + R + 1:nx]
    assert r[:, far].max() <= 1e-13
    # the same problem along y: the transposed mask
    rT, mT = oracle.Oracle([ny, nx], dim=2, R=R, bc="outflow").kxrcf(_contact(nx, ny, j, axis=1))
    assert (mT == m.T).all()
    assert np.allclose(rT, r.T, rtol=1e-12, atol=1e-15)


def test_smooth_data_ratio_decays_at_design_order():
    worst = []
    for n in (16, 32, 64):
        U = workloads.sine_2d(n, R=2).numpy()
        r, m = oracle.Oracle([n, n], dim=2, R=2, bc="periodic").kxrcf(U)
        worst.append(r.max())
        if n == 64:
            assert m.all()  # every cell of the smooth translation takes the linear reconstruction
    eoc = np.log2(np.array(worst[:-1]) / np.array(worst[1:]))
    assert (eoc >= 3.5).all(), (worst, eoc)


def test_ratio_is_homogeneous_of_degree_zero():
    U = workloads.voronoi_2d(24, k=6, seed=3).numpy()
    o = oracle.Oracle([24, 24], dim=2, R=2, bc="outflow")
    r1, m1 = o.kxrcf(U)
    r2, m2 = o.kxrcf(U * 3.7)
    fin = np.isfinite(r1)
    assert (np.isfinite(r2) == fin).all()
    assert np.allclose(r1[fin], r2[fin], rtol=1e-11, atol=1e-15)
    assert (m1 == m2).all()


def test_threshold_is_delta_to_the_m():
    """Same data on a larger domain: identical ratios, decisions against the new Delta^m."""
    U = workloads.voronoi_2d(24, k=6, seed=5).numpy()
    r, _ = oracle.Oracle([24, 24], dim=2, R=2, bc="outflow").kxrcf(U)
    for L, m in [(3.0, 1.5), (1.0, 2.0), (0.05, 1.0)]:
        rL, mL = oracle.Oracle([24, 24], dim=2, R=2, bc="outflow", hi=[L, L], kxrcf_m=m).kxrcf(U)
        assert np.array_equal(rL, r)
        assert (mL == (r < (L / 24) ** m)).all()


# --------------------------------------------------------------------------
# brute force by physical coordinates, reconstructions from the coefficient form
# --------------------------------------------------------------------------
def _coefficient_form_evaluator(dim, R):
    """x -> row e(x) with e(x) . g = the S0 reconstruction at x (unit-cell coordinates) of averages g:
    Eq. 10 solved at 40 digits (kernel cell integrals by quadrature), then Eq. 2 evaluated at x."""
    mp = pytest.importorskip("mpmath")
    from oracle import stencils
    from tests.test_oracle_weights import _mp_system

    mp.mp.dps = 40
    offs = list(stencils.full_stencil(dim, R))
    mons = stencils.monomials(dim, stencils.degrees(dim, R)[0])
    A, _ = _mp_system(dim, offs, stencils.degrees(dim, R)[0], 5, [], [])
    N = len(offs)
    M = A.copy()
    for h in range(N):
        for l in range(N):
            M[h, l] = A[l, h]
    Minv = mp.inverse(M)
    cache = {}

    def row(x):
        key = tuple(round(float(v), 12) for v in x)
        if key not in cache:
            xs = [mp.mpf(v) for v in x]
            basis = [mp.exp(-sum((xs[k] - offs[l][k]) ** 2 for k in range(dim)) / 50) for l in range(N)]
            basis += [mp.fprod([xs[k] ** a[k] for k in range(dim)]) for a in mons]
            cache[key] = np.array([float(mp.fsum(basis[i] * Minv[i, l] for i in range(len(basis))))
                                   for l in range(N)])
        return cache[key]

    return offs, row


def _brute_force_ratio(U, bc, R, m_pow=1.5, hi=(1.0, 1.0)):
    ny, nx = U.shape[1:]
    dx, dy = hi[0] / nx, hi[1] / ny
    offs, row = _coefficient_form_evaluator(2, R)
    nodes = np.polynomial.legendre.leggauss(R)[0] / 2

    def ghost(i, n):
        return i % n if bc == "periodic" else min(max(i, 0), n - 1)

    def recon(ix, iy, x):
        """cell (ix, iy)'s reconstruction at the physical point x"""
        xi = ((x[0] - (ix + 0.5) * dx) / dx, (x[1] - (iy + 0.5) * dy) / dy)
        e = row(xi)
        g = np.array([[U[v, ghost(iy + o[1], ny), ghost(ix + o[0], nx)] for o in offs] for v in range(4)])
        return g @ e

    def q(u):
        p = (GAMMA - 1) * (u[3] - 0.5 * (u[1] ** 2 + u[2] ** 2) / u[0])
        return p / u[0] ** GAMMA if (u[0] > 0 and p > 0) else np.inf

    ratio = np.zeros((ny, nx))
    for iy in range(ny):
        for ix in range(nx):
            cx, cy = (ix + 0.5) * dx, (iy + 0.5) * dy
            jmax = 0.0
            for axis in (0, 1):
                for sgn in (-1, 1):
                    for t in nodes:
                        P = [cx + t * dx, cy + t * dy]
                        P[axis] = (cx, cy)[axis] + sgn * 0.5 * (dx, dy)[axis]
                        # the cell across the face, found by position just outside this cell
                        probe = list(P)
                        probe[axis] += sgn * 1e-9
                        jx, jy = int(np.floor(probe[0] / dx)), int(np.floor(probe[1] / dy))
                        if not (0 <= jx < nx and 0 <= jy < ny):
                            if bc == "outflow":
                                continue
                            # periodic: the wrapped cell, with P moved into its periodic image
                            sx = (jx // nx) * hi[0]
                            sy = (jy // ny) * hi[1]
                            jx, jy = jx % nx, jy % ny
                            Pn = (P[0] - sx, P[1] - sy)
                        else:
                            Pn = P
                        qm, qp = q(recon(ix, iy, P)), q(recon(jx, jy, Pn))
                        jmax = max(jmax, np.inf if np.isinf(qm) or np.isinf(qp) else abs(qp - qm))
            ratio[iy, ix] = jmax / q(U[:, iy, ix])
    return ratio, ratio < max(dx, dy) ** m_pow


@pytest.mark.parametrize("bc,R", [("outflow", 2), ("periodic", 2), ("outflow", 3)])
def test_ratio_matches_brute_force_by_position(bc, R):
    nx, ny = 7, 6
    U = np.ascontiguousarray(workloads.mixed_voronoi(2, 8, 4, seed=21).numpy()[:, :ny, :nx])
    o = oracle.Oracle([nx, ny], dim=2, R=R, bc=bc)
    r, m = o.kxrcf(U)
    rb, mb = _brute_force_ratio(U, bc, R)
    fin = np.isfinite(rb)
    assert (np.isfinite(r) == fin).all()
    scale = np.maximum(rb[fin], 1e-9)
    assert np.max(np.abs(r[fin] - rb[fin]) / scale) < 1e-11
    # decisions equal wherever the ratio is not within rounding of the threshold
    clear = np.abs(np.log(np.maximum(rb, 1e-300) / (1 / nx) ** 1.5)) > 1e-6
    assert (m[clear] == mb[clear]).all()
    assert (m == 0).any() and (m == 1).any()


def test_kxrcf_step_reduces_to_linear_on_smooth_data():
    """On the 64^2 smooth translation every cell is smooth: the KXRCF step is the linear step."""
    U = workloads.sine_2d(64, R=2).numpy()
    a, dta = oracle.Oracle([64, 64], dim=2, R=2, bc="periodic", recon="kxrcf").step(U, 0.4)
    b, dtb = oracle.Oracle([64, 64], dim=2, R=2, bc="periodic", recon="linear").step(U, 0.4)
    assert dta == dtb and np.array_equal(a, b)


def test_kxrcf_step_equals_gated_step_on_its_mask():
    """The KXRCF mode is the gated reconstruction driven by the indicator of each stage's state."""
    U = workloads.voronoi_2d(32, k=8, seed=9).numpy()
    o = oracle.Oracle([32, 32], dim=2, R=2, bc="outflow", recon="kxrcf")
    _, mask = o.kxrcf(U)
    assert 0 < mask.mean() < 1
    L = o.rhs(U)
    Lg = oracle.Oracle([32, 32], dim=2, R=2, bc="outflow", recon="gated", mask=mask).rhs(U)
    assert np.array_equal(L, Lg)
