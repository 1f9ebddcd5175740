"""Stencil geometry of KFVM-WENO, written out plainly (test infrastructure only).

This module belongs to the oracle: only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg may import it.  Nothing here is shared with
the CUDA path.

Contents, each following the paper (May & Lee, "KFVM-WENO", arXiv 2401.16543):

* ``full_stencil(dim, R)``  -- the spherical stencil S0 = {o : |o|^2 <= R^2}
  (Sec. 3.1, "Stencils and substencils"), enumerated z-outer, x-fastest.
* ``substencils(dim, R)``   -- S1 (radius R-1) and the 2*dim biased substencils
  (Sec. 3.1), as ascending index lists into S0.  Cells with |j| = i belong to
  two biased substencils, exactly as the paper's "<=" conditions say.
* ``poly_degree(offsets)``  -- the largest total degree p for which the
  cell-average monomial matrix P is unisolvent (full column rank) over the
  stencil (Sec. 2.1: choose the stencil first, then the maximal p that keeps
  unisolvence).  The rank is computed EXACTLY over the rationals with
  ``fractions.Fraction`` (P's entries are rationals), so no tolerance enters.
* ``monomials(dim, p)`` / ``deriv_indices(dim, R)`` -- multi-indices with
  |alpha| <= p, and 0 < |alpha| <= R for the smoothness indicators (Eq. 22,
  p = R as chosen in Sec. 3.3).
* ``linear_weights(dim)``  -- gamma_q with gamma_hi = gamma_lo = 0.8 (Sec. 3.2).
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from itertools import product


def _offsets_in_box(dim: int, R: int):
    """All integer offsets in [-R, R]^dim, z outermost and x fastest."""
    rng = range(-R, R + 1)
    if dim == 2:
        for j in rng:
            for i in rng:
                yield (i, j, 0)
    else:
        for k in rng:
            for j in rng:
                for i in rng:
                    yield (i, j, k)


@lru_cache(maxsize=None)
def full_stencil(dim: int, R: int):
    """S0: unit cells whose centre offset o satisfies |o|^2 <= R^2 (Sec. 3.1)."""
    return tuple(o for o in _offsets_in_box(dim, R) if o[0] ** 2 + o[1] ** 2 + o[2] ** 2 <= R * R)


def _biased_conditions(dim: int):
    """Membership tests of the biased substencils S2..S_{2dim+1} (Sec. 3.1).

    2D: S2 |j|<=i, S3 |j|<=-i, S4 |i|<=j, S5 |i|<=-j.
    3D: the same with both transverse indices bounded by the biased one.
    """
    if dim == 2:
        return [
            lambda i, j, k: abs(j) <= i,
            lambda i, j, k: abs(j) <= -i,
            lambda i, j, k: abs(i) <= j,
            lambda i, j, k: abs(i) <= -j,
        ]
    return [
        lambda i, j, k: abs(j) <= i and abs(k) <= i,
        lambda i, j, k: abs(j) <= -i and abs(k) <= -i,
        lambda i, j, k: abs(i) <= j and abs(k) <= j,
        lambda i, j, k: abs(i) <= -j and abs(k) <= -j,
        lambda i, j, k: abs(i) <= k and abs(j) <= k,
        lambda i, j, k: abs(i) <= -k and abs(j) <= -k,
    ]


@lru_cache(maxsize=None)
def substencils(dim: int, R: int):
    """Index lists into S0 for q = 0..N_S (q = 0 is S0 itself)."""
    s0 = full_stencil(dim, R)
    out = [tuple(range(len(s0)))]
    out.append(tuple(n for n, (i, j, k) in enumerate(s0) if i * i + j * j + k * k <= (R - 1) ** 2))
    for cond in _biased_conditions(dim):
        out.append(tuple(n for n, o in enumerate(s0) if cond(*o)))
    return tuple(out)


@lru_cache(maxsize=None)
def monomials(dim: int, p: int):
    """Multi-indices alpha with |alpha| <= p, by total degree, then alpha_x descending."""
    out = []
    for n in range(p + 1):
        for a in product(range(n, -1, -1), repeat=dim):
            if sum(a) == n:
                out.append(tuple(a) + (0,) * (3 - dim))
    return tuple(out)


@lru_cache(maxsize=None)
def deriv_indices(dim: int, R: int):
    """Derivative multi-indices of the smoothness indicator: 0 < |alpha| <= R (Eq. 22, p = R)."""
    return monomials(dim, R)[1:]


def _cell_avg_monomial_exact(o, a):
    """lambda_h x^alpha over the unit cell centred at o: prod_k [(o+1/2)^(a+1) - (o-1/2)^(a+1)]/(a+1)."""
    val = Fraction(1)
    for ok, ak in zip(o, a):
        hi = Fraction(2 * ok + 1, 2)
        lo = Fraction(2 * ok - 1, 2)
        val *= (hi ** (ak + 1) - lo ** (ak + 1)) / (ak + 1)
    return val


def exact_rank(rows):
    """Rank of a rational matrix by fraction-exact Gaussian elimination."""
    m = [list(r) for r in rows]
    rank = 0
    ncol = len(m[0]) if m else 0
    for c in range(ncol):
        piv = next((r for r in range(rank, len(m)) if m[r][c] != 0), None)
        if piv is None:
            continue
        m[rank], m[piv] = m[piv], m[rank]
        for r in range(len(m)):
            if r != rank and m[r][c] != 0:
                f = m[r][c] / m[rank][c]
                m[r] = [x - f * y for x, y in zip(m[r], m[rank])]
        rank += 1
    return rank


def p_matrix_exact(offsets, dim: int, p: int):
    """The N x D cell-average monomial matrix P of Eq. (8), exact rationals."""
    mons = monomials(dim, p)
    return [[_cell_avg_monomial_exact(o, a) for a in mons] for o in offsets]


def poly_degree(offsets, dim: int) -> int:
    """Maximal total degree p keeping P unisolvent over the stencil (Sec. 2.1)."""
    p = 0
    while True:
        nxt = p + 1
        D = len(monomials(dim, nxt))
        if D > len(offsets):
            return p
        if exact_rank(p_matrix_exact(offsets, dim, nxt)) < D:
            return p
        p = nxt


@lru_cache(maxsize=None)
def degrees(dim: int, R: int):
    """Polynomial degree p_q of every (sub)stencil q = 0..N_S."""
    s0 = full_stencil(dim, R)
    return tuple(poly_degree([s0[n] for n in idx], dim) for idx in substencils(dim, R))


def linear_weights(dim: int):
    """gamma_q for q = 0..N_S with gamma_hi = gamma_lo = 0.8 (Sec. 3.2)."""
    ghi = glo = 0.8
    nb = 2 * dim
    return (ghi, (1 - ghi) * glo) + ((1 - ghi) * (1 - glo) / nb,) * nb


def n_face_points(dim: int, R: int) -> int:
    """Gauss-Legendre points on all 2*dim faces, R per face dimension (Sec. 5.1)."""
    return 2 * dim * R ** (dim - 1)
