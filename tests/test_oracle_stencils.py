"""Pins of the oracle's stencil geometry against the paper's printed counts and brute force."""
import itertools

import numpy as np
import pytest

from oracle import stencils
from tests.paper_values import load

PV = load()


def test_2d_sizes_match_paper_captions():
    sub = stencils.substencils(2, 2)
    assert len(stencils.full_stencil(2, 2)) == PV["2d_r2_s0"]
    assert [len(s) for s in sub[1:]] == [PV["2d_r2_sub"]] * 5
    sub = stencils.substencils(2, 3)
    assert len(stencils.full_stencil(2, 3)) == PV["2d_r3_s0"]
    assert len(sub[1]) == PV["2d_r3_s1"]
    assert [len(s) for s in sub[2:]] == [PV["2d_r3_biased"]] * 4


@pytest.mark.parametrize("dim,R", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_sets_by_brute_force(dim, R):
    """Re-derive every set with numpy masks over the box and compare as sets."""
    g = np.array(list(itertools.product(range(-R, R + 1), repeat=dim)))
    i, j = g[:, 0], g[:, 1]
    k = g[:, 2] if dim == 3 else np.zeros_like(i)
    r2 = i * i + j * j + k * k
    s0 = r2 <= R * R
    masks = [s0, s0 & (r2 <= (R - 1) ** 2)]
    if dim == 2:
        masks += [s0 & (np.abs(j) <= i), s0 & (np.abs(j) <= -i), s0 & (np.abs(i) <= j), s0 & (np.abs(i) <= -j)]
    else:
        masks += [s0 & (np.abs(j) <= i) & (np.abs(k) <= i), s0 & (np.abs(j) <= -i) & (np.abs(k) <= -i),
                  s0 & (np.abs(i) <= j) & (np.abs(k) <= j), s0 & (np.abs(i) <= -j) & (np.abs(k) <= -j),
                  s0 & (np.abs(i) <= k) & (np.abs(j) <= k), s0 & (np.abs(i) <= -k) & (np.abs(j) <= -k)]
    full = stencils.full_stencil(dim, R)
    for m, idx in zip(masks, stencils.substencils(dim, R)):
        want = {(int(a), int(b), int(c)) for a, b, c in zip(i[m], j[m], k[m])}
        got = {full[n] for n in idx}
        assert got == want
    # the central cell is in every set, and the enumeration is x-fastest
    for idx in stencils.substencils(dim, R):
        assert any(full[n] == (0, 0, 0) for n in idx)
    keys = [(o[2], o[1], o[0]) for o in full]
    assert keys == sorted(keys)


@pytest.mark.parametrize("dim,R", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_biased_substencils_are_mirror_images(dim, R):
    full = stencils.full_stencil(dim, R)
    subs = stencils.substencils(dim, R)
    for a in range(dim):
        plus = {full[n] for n in subs[2 + 2 * a]}
        minus = {full[n] for n in subs[3 + 2 * a]}
        flip = {tuple(-c if ax == a else c for ax, c in enumerate(o)) for o in plus}
        assert flip == minus


def test_full_stencil_degrees_match_paper():
    assert stencils.degrees(2, 2)[0] == PV["deg_s0_r2"]
    assert stencils.degrees(2, 3)[0] == PV["deg_s0_r3"]
    assert stencils.degrees(3, 2)[0] == PV["deg_s0_r2"]
    assert stencils.degrees(3, 3)[0] == PV["deg_s0_r3"]


def _p_float(offs, dim, p):
    """Cell-average monomials in floating point by a midpoint-free closed form (numpy)."""
    mons = stencils.monomials(dim, p)
    P = np.ones((len(offs), len(mons)))
    for h, o in enumerate(offs):
        for v, a in enumerate(mons):
            for ok, ak in zip(o[:dim], a[:dim]):
                P[h, v] *= ((ok + 0.5) ** (ak + 1) - (ok - 0.5) ** (ak + 1)) / (ak + 1)
    return P


@pytest.mark.parametrize("dim,R", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_degrees_are_maximal_unisolvent_by_svd(dim, R):
    """Independent check of the exact-rank choice with a floating SVD rank."""
    full = stencils.full_stencil(dim, R)
    for idx, p in zip(stencils.substencils(dim, R), stencils.degrees(dim, R)):
        offs = [full[n] for n in idx]
        P = _p_float(offs, dim, p)
        assert np.linalg.matrix_rank(P) == P.shape[1]
        P1 = _p_float(offs, dim, p + 1)
        assert P1.shape[1] > len(offs) or np.linalg.matrix_rank(P1) < P1.shape[1]


def test_derivative_counts_match_paper():
    assert len(stencils.deriv_indices(2, 2)) == PV["nderiv_2d_r2"]
    assert len(stencils.deriv_indices(2, 3)) == PV["nderiv_2d_r3"]
    assert len(stencils.deriv_indices(3, 2)) == PV["nderiv_3d_r2"]
    assert len(stencils.deriv_indices(3, 3)) == PV["nderiv_3d_r3"]


def test_linear_weights_match_paper():
    ghi, glo = PV["gamma_hi"], PV["gamma_lo"]
    g2 = stencils.linear_weights(2)
    assert g2[0] == ghi and abs(g2[1] - (1 - ghi) * glo) < 1e-16
    assert np.allclose(g2[2:], (1 - ghi) * (1 - glo) / 4, rtol=0, atol=1e-17)
    g3 = stencils.linear_weights(3)
    assert np.allclose(g3[2:], (1 - ghi) * (1 - glo) / 6, rtol=0, atol=1e-17)
    assert abs(sum(g2) - 1) < 1e-15 and abs(sum(g3) - 1) < 1e-15
