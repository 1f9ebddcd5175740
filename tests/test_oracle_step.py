"""Pins of the oracle's full RHS and SSP-RK3 step against invariants and exact solutions."""
import math

import numpy as np
import pytest

import oracle
import workloads

G = 1.4


@pytest.mark.parametrize("dim,R,bc", [(2, 2, "periodic"), (2, 3, "outflow"), (3, 2, "periodic"), (3, 2, "outflow")])
def test_free_stream_preserved(dim, R, bc):
    n = [7, 6, 5][:dim]
    o = oracle.Oracle(n, dim=dim, R=R, bc=bc)
    U = workloads.constant_state(dim, n, rho=0.9, vel=[0.4, -0.3, 0.2][:dim], p=0.6).numpy()
    U1, dt = o.step(U, 0.4)
    assert o.status == 0 and dt > 0
    assert np.max(np.abs(U1 - U)) < 1e-14 * np.abs(U).max()


@pytest.mark.parametrize("dim,R", [(2, 2), (2, 3), (3, 2)])
def test_periodic_conservation(dim, R):
    n = [12, 10, 8][:dim] if dim == 2 else [8, 7, 6]
    o = oracle.Oracle(n, dim=dim, R=R)
    if dim == 2:
        U = workloads.mixed_voronoi(2, 12, 6, seed=21).numpy()[:, :10, :12]
    else:
        U = workloads.mixed_voronoi(3, 8, 5, seed=22).numpy()[:, :6, :7, :8]
    U = np.ascontiguousarray(U)
    U1, dt = o.step(U, 0.4)
    assert o.status == 0
    for v in range(dim + 2):
        drift = abs(math.fsum(U1[v].ravel()) - math.fsum(U[v].ravel()))
        assert drift <= 1e-13 * math.fsum(np.abs(U[v]).ravel()), v


@pytest.mark.parametrize("R", [2, 3])
def test_mirror_symmetry(R):
    """x -> 1-x with rho*u negated commutes with a step, to round-off (Sec. 6.6 notes
    symmetry holds only to round-off in multidimensional reconstruction)."""
    n = 16
    o = oracle.Oracle([n, n], dim=2, R=R, bc="outflow")
    U = workloads.voronoi_2d(n, k=10, seed=31).numpy()
    Um = U[:, :, ::-1].copy()
    Um[1] *= -1
    U1, dt1 = o.step(U, 0.4)
    V1, dt2 = o.step(Um, 0.4)
    assert dt1 == dt2
    V1 = V1[:, :, ::-1]
    V1[1] *= -1
    assert np.max(np.abs(U1 - V1)) < 1e-13


def _rhs_truncation(n, R, recon):
    o = oracle.Oracle([n, n], dim=2, R=R, recon=recon)
    U = workloads.sine_2d(n, R=max(R, 3)).numpy()
    L = o.rhs(U)
    h = 1.0 / n
    xc = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    damp = (math.sin(math.pi * h) / (math.pi * h)) ** 2
    drho = -0.2 * 4 * math.pi * np.cos(2 * math.pi * (X + Y)) * damp
    return max(np.abs(L[v] - drho).max() for v in range(4))


@pytest.mark.parametrize("R,order", [(2, 4), (3, 6)])
def test_design_order_of_linear_reconstruction(R, order):
    """The semi-discrete operator on the smooth translation converges at order >= 2R
    (Sec. 3.1 and Table 1): measured on 16..64 cells; exact cell-average dU/dt is known."""
    errs = [_rhs_truncation(n, R, "linear") for n in (16, 32, 64)]
    eoc = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert eoc[-1] > order - 0.3, (errs, eoc)


def test_rk3_third_order_in_time():
    n = 24
    o = oracle.Oracle([n, n], dim=2, R=2, recon="linear")
    U0 = workloads.sine_2d(n).numpy()
    ref, _, _ = o.run(U0, 0.05, 0.06)
    errs = []
    for cfl in (0.8, 0.4, 0.2):
        U, _, _ = o.run(U0, cfl, 0.06)
        errs.append(np.abs(U - ref).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 2.6, (errs, rates)


def test_sine_translation_accuracy():
    """The smooth translation to t = 0.1 on 64^2 at CFL 0.4 (the 2D radius-2 sine workload):
    error against the exact cell averages."""
    n = 64
    U0 = workloads.sine_2d(n).numpy()
    ex = workloads.sine_2d_exact_density(n, 0.1)
    lin = oracle.Oracle([n, n], dim=2, R=2, recon="linear")
    U, t, k = lin.run(U0, 0.4, 0.1)
    assert abs(t - 0.1) < 1e-15 and k == 75
    e_lin = np.abs(U[0] - ex).mean()
    assert e_lin < 2e-7
    weno = oracle.Oracle([n, n], dim=2, R=2)
    U, _, _ = weno.run(U0, 0.4, 0.1)
    e_weno = np.abs(U[0] - ex).mean()
    # fixed eps = 1e-40 costs accuracy on smooth data (Sec. 3.3 relies on the troubled-cell bypass)
    assert e_lin < e_weno < 1e-4


# ---- Sod shock tube against the exact Riemann solution (Sec. 6.2) -------------------------

def _sod_exact(x, t, x0=0.5, L=(1.0, 0.0, 1.0), Rr=(0.125, 0.0, 0.1)):
    """Exact solution of the Riemann problem (textbook: Newton on the star pressure)."""
    rL, uL, pL = L
    rR, uR, pR = Rr
    cL, cR = math.sqrt(G * pL / rL), math.sqrt(G * pR / rR)

    def fk(p, r, pk, ck):
        if p > pk:
            A, B = 2 / ((G + 1) * r), (G - 1) / (G + 1) * pk
            return (p - pk) * math.sqrt(A / (p + B)), math.sqrt(A / (p + B)) * (1 - (p - pk) / (2 * (B + p)))
        e = (G - 1) / (2 * G)
        return 2 * ck / (G - 1) * ((p / pk) ** e - 1), (p / pk) ** (-(G + 1) / (2 * G)) / (r * ck)

    p = 0.5 * (pL + pR)
    for _ in range(100):
        f1, d1 = fk(p, rL, pL, cL)
        f2, d2 = fk(p, rR, pR, cR)
        dp = (f1 + f2 + uR - uL) / (d1 + d2)
        p = max(p - dp, 1e-12)
        if abs(dp) < 1e-15 * p:
            break
    us = 0.5 * (uL + uR) + 0.5 * (fk(p, rR, pR, cR)[0] - fk(p, rL, pL, cL)[0])
    out = np.empty_like(x)
    for i, xi in enumerate(x):
        s = (xi - x0) / t
        if s < us:  # left of the contact: rarefaction (pL > p*)
            rls = rL * (p / pL) ** (1 / G)
            cls = cL * (p / pL) ** ((G - 1) / (2 * G))
            if s < uL - cL:
                out[i] = rL
            elif s > us - cls:
                out[i] = rls
            else:
                out[i] = rL * (2 / (G + 1) + (G - 1) / ((G + 1) * cL) * (uL - s)) ** (2 / (G - 1))
        else:  # right of the contact: shock (p* > pR)
            sR = uR + cR * math.sqrt((G + 1) / (2 * G) * p / pR + (G - 1) / (2 * G))
            rrs = rR * ((p / pR + (G - 1) / (G + 1)) / ((G - 1) / (G + 1) * p / pR + 1))
            out[i] = rrs if s < sR else rR
    return out


@pytest.mark.parametrize("R", [2, 3])
def test_sod_against_exact_solution(R):
    nx, ny = 100, 2
    o = oracle.Oracle([nx, ny], dim=2, R=R, lo=[0, 0], hi=[1.0, 0.02], bc=["outflow", "periodic"])
    x = (np.arange(nx) + 0.5) / nx
    rho = np.where(x < 0.5, 1.0, 0.125)
    p = np.where(x < 0.5, 1.0, 0.1)
    U = np.zeros((4, ny, nx))
    U[0] = rho
    U[3] = p / (G - 1)
    U, t, k = o.run(U, 0.4, 0.2)
    ex = _sod_exact(x, 0.2)
    err = np.abs(U[0, 0] - ex).mean()
    assert err < 6e-3, err
    assert np.max(np.abs(U[:, 0] - U[:, 1])) < 1e-13  # no y dependence develops
