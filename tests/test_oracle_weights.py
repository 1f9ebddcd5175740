"""Pins of the oracle's reconstruction and derivative vectors (Sec. 2.1, Sec. 3.3).

* polynomial reproduction with exact rational cell averages of monomials;
* an independent high-precision dense solve with mpmath, whose kernel
  integrals come from numerical quadrature and whose kernel derivatives come
  from numerical differentiation (not the oracle's erf / Hermite closed forms),
  on every stencil of 2D and 3D at radius 2 and 3;
* the coefficient form of the reconstruction (solve Eq. 10 for a and b, then
  evaluate the expansion Eq. 2 at the point) against the dot product r.g;
* mirror symmetry of the face vectors.
"""
from fractions import Fraction
from math import factorial

import numpy as np
import pytest

import oracle
from oracle import stencils

mp = pytest.importorskip("mpmath")


def _avg_mono_exact(o, a):
    val = Fraction(1)
    for ok, ak in zip(o, a):
        val *= (Fraction(2 * ok + 1, 2) ** (ak + 1) - Fraction(2 * ok - 1, 2) ** (ak + 1)) / (ak + 1)
    return val


@pytest.mark.parametrize("dim,R", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_polynomial_and_derivative_reproduction(dim, R):
    full = stencils.full_stencil(dim, R)
    pts = oracle.face_points(dim, R)
    ders = stencils.deriv_indices(dim, R)
    for (rf, rd), idx, p in zip(oracle.weights(dim, R), stencils.substencils(dim, R), stencils.degrees(dim, R)):
        offs = [full[n] for n in idx]
        for a in stencils.monomials(dim, p):
            lam = np.array([float(_avg_mono_exact(o, a)) for o in offs])
            # face points: r . lambda(x^a) = x_s^a
            want = np.prod(pts ** np.array(a), axis=1)
            scale = max(1.0, np.abs(rf).sum(1).max() * np.abs(lam).max())
            assert np.max(np.abs(rf @ lam - want)) < 2e-14 * scale
            # derivatives: d(b) . lambda(x^a) = d^b x^a at 0 = a! [a == b]
            want_d = np.array([float(np.prod([factorial(x) for x in a])) if tuple(b) == tuple(a) else 0.0
                               for b in ders])
            scale = max(1.0, np.abs(rd).sum(1).max() * np.abs(lam).max())
            assert np.max(np.abs(rd @ lam - want_d)) < 5e-14 * scale


def _mp_system(dim, offs, p, ell, pts, ders):
    """Dense saddle-point system with quadrature / numerical-derivative entries at 40 digits."""
    N = len(offs)
    mons = stencils.monomials(dim, p)
    D = len(mons)
    two_l2 = 2 * mp.mpf(ell) ** 2

    def k1(x, c):
        return mp.exp(-(x - c) ** 2 / two_l2)

    cache = {}

    def cell_int(delta):
        if delta not in cache:
            cache[delta] = mp.quad(lambda x: k1(x, 0), [delta - mp.mpf(1) / 2, delta + mp.mpf(1) / 2])
        return cache[delta]

    A = mp.zeros(N + D, N + D)
    for h in range(N):
        for l in range(N):
            q = mp.mpf(1)
            for k in range(dim):
                q *= cell_int(offs[h][k] - offs[l][k])
            A[l, h] = q  # Q^T
        for v, a in enumerate(mons):
            val = mp.mpf(_avg_mono_exact(offs[h][:dim], a[:dim]).numerator) / _avg_mono_exact(offs[h][:dim], a[:dim]).denominator
            A[h, N + v] = val
            A[N + v, h] = val
    rhs = []
    for x in pts:
        b = mp.zeros(N + D, 1)
        for l in range(N):
            b[l] = mp.exp(-sum((mp.mpf(x[k]) - offs[l][k]) ** 2 for k in range(dim)) / two_l2)
        for v, a in enumerate(mons):
            b[N + v] = mp.fprod([mp.mpf(x[k]) ** a[k] for k in range(dim)])
        rhs.append(b)
    for a in ders:
        b = mp.zeros(N + D, 1)
        for l in range(N):
            val = mp.mpf(1)
            for k in range(dim):
                val *= mp.diff(lambda t: k1(t, offs[l][k]), 0, a[k]) if a[k] else k1(0, offs[l][k])
            b[l] = val
        for v, m in enumerate(mons):
            b[N + v] = mp.mpf(int(np.prod([factorial(x) for x in a]))) if tuple(m) == tuple(a) else 0
        rhs.append(b)
    return A, rhs


def _mp_face_points(dim, R):
    """Face Gauss points recomputed in mpmath from the Legendre roots."""
    nodes = sorted(mp.polyroots(mp.taylor(lambda t: mp.legendre(R, t), 0, R)[::-1]))
    nodes = [mp.re(r) / 2 for r in nodes]
    out = []
    for d in range(dim):
        tr = [a for a in range(dim) if a != d]
        for side in (0, 1):
            for t in range(R ** (dim - 1)):
                x = [mp.mpf(0)] * 3
                x[d] = mp.mpf(1) / 2 if side else -mp.mpf(1) / 2
                x[tr[0]] = nodes[t % R]
                if dim == 3:
                    x[tr[1]] = nodes[t // R]
                out.append(x)
    return out


@pytest.mark.parametrize("dim,R", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_weights_match_independent_mpmath_solve(dim, R):
    """Every stencil of every (d, R), S0 included (3D R3: the 123-cell S0 with 56 monomials, a 179 x 179
    saddle-point system of condition ~5e17): the oracle's binary128 weights rounded to double equal a
    40-digit solve assembled independently (quadrature, numerical differentiation, Gauss points from the
    Legendre roots), factored once per stencil and applied to all F + M right-hand sides."""
    mp.mp.dps = 40
    full = stencils.full_stencil(dim, R)
    pts = _mp_face_points(dim, R)
    assert np.allclose(np.array([[float(c) for c in x] for x in pts]), oracle.face_points(dim, R), atol=1e-16)
    ders = stencils.deriv_indices(dim, R)
    W = oracle.weights(dim, R)
    subs = stencils.substencils(dim, R)
    for q in range(len(subs)):
        idx, p = subs[q], stencils.degrees(dim, R)[q]
        offs = [full[n] for n in idx]
        A, rhs = _mp_system(dim, offs, p, 5, pts, ders)
        rf, rd = W[q]
        prec = mp.mp.prec
        mp.mp.prec += 10
        try:
            LU, piv = mp.mp.LU_decomp(A.copy())
            for s, b in enumerate(rhs):
                sol = mp.mp.U_solve(LU, mp.mp.L_solve(LU, b.copy(), piv))
                r = np.array([float(sol[l]) for l in range(len(offs))])
                got = rf[s] if s < len(pts) else rd[s - len(pts)]
                assert np.max(np.abs(got - r)) <= 4e-16 * max(1.0, np.abs(r).max()), (q, s)
        finally:
            mp.mp.prec = prec


def test_coefficient_form_equals_reconstruction_vector():
    """Solve [[Q, P], [P^T, 0]] [a; b] = [g; 0] (Eq. 10) and evaluate Eq. 2 at x_s."""
    mp.mp.dps = 40
    dim, R = 2, 2
    full = stencils.full_stencil(dim, R)
    offs = list(full)
    p = stencils.degrees(dim, R)[0]
    mons = stencils.monomials(dim, p)
    pts = _mp_face_points(dim, R)
    A, _ = _mp_system(dim, offs, p, 5, pts, [])
    # A holds Q^T in its kernel block; Q is symmetric on unit cells, so transpose back explicitly
    N = len(offs)
    M = A.copy()
    for h in range(N):
        for l in range(N):
            M[h, l] = A[l, h]
    rng = np.random.default_rng(7)
    g = rng.uniform(-1, 1, N)
    rhs = mp.matrix([mp.mpf(x) for x in g] + [0] * len(mons))
    sol = mp.lu_solve(M, rhs)
    rf = oracle.weights(dim, R)[0][0]
    for s, x in enumerate(pts):
        val = mp.mpf(0)
        for l in range(N):
            val += sol[l] * mp.exp(-sum((x[k] - offs[l][k]) ** 2 for k in range(dim)) / 50)
        for v, a in enumerate(mons):
            val += sol[N + v] * mp.fprod([x[k] ** a[k] for k in range(dim)])
        assert abs(float(val) - float(rf[s] @ g)) < 1e-14


@pytest.mark.parametrize("dim,R", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_face_vectors_are_mirror_symmetric(dim, R):
    """Mirroring axis a maps face point (a, +, t) to (a, -, t) and S0 onto itself."""
    full = stencils.full_stencil(dim, R)
    pos = {o: n for n, o in enumerate(full)}
    rf = oracle.weights(dim, R)[0][0]
    nt = R ** (dim - 1)
    for a in range(dim):
        perm = [pos[tuple(-c if ax == a else c for ax, c in enumerate(o))] for o in full]
        for t in range(nt):
            lo = rf[(2 * a) * nt + t]
            hi = rf[(2 * a + 1) * nt + t]
            assert np.max(np.abs(hi[perm] - lo)) < 1e-15 * max(1, np.abs(lo).max())
