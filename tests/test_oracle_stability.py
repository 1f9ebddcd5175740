"""Von Neumann analysis of the linear (unlimited) S0 reconstruction, from the oracle's weights.

Scalar advection along (1, ..., 1) with unit cells, upwind face fluxes and the S0 reconstruction of
Sec. 2.1 averaged over each face's Gauss points: a Fourier mode exp(i k.x) evolves with
lambda(k) = -sum_d rho_d(k) (1 - exp(-i k_d)), rho_d(k) the mode's reconstructed value at the high
d-face.  Re(lambda) <= 0 for every k means the semi-discrete linear scheme does not amplify.

Measured (kernel length scale 5 Delta, Sec. 5.1): max over k of Re(lambda) 0 (2D R2), +0.009 (2D R3),
+0.03 (3D R2), +7.5 (3D R3); max |lambda| 3.2 / 3.9 / 5.4 / 104; the largest sum of |r_0| over a face
row 2.1 / 2.9 / 3.3 / 69.5.  The 3D radius-3 stencil's weights oscillate strongly and its linear
scheme amplifies high-frequency modes; the paper runs radius 3 only in 2D.  On the oracle, a 3D
radius-3 linear run of a smooth translation leaves its truncation-level error within a few steps
at CFL 0.4, while WENO-AO stays stable (its nonlinear weights move off the oscillating S0 values).
These tests record that characterisation.
"""
import numpy as np
import pytest

import oracle
from oracle import stencils


def _symbol(dim, R, nk=20):
    r0 = oracle.weights(dim, R)[0][0]
    offs = np.array(stencils.full_stencil(dim, R))[:, :dim]
    NT = R ** (dim - 1)
    glw = oracle.gl_weights(R)
    wt = np.array([glw[t % R] * (glw[t // R] if dim == 3 else 1.0) for t in range(NT)])
    ks = np.linspace(-np.pi, np.pi, nk, endpoint=False)
    K = np.stack([g.ravel() for g in np.meshgrid(*([ks] * dim), indexing="ij")], axis=1)
    phase = np.exp(1j * K @ offs.T)
    lam = np.zeros(len(K), dtype=complex)
    for d in range(dim):
        s_hi = np.array([(2 * d + 1) * NT + t for t in range(NT)])
        lam -= ((phase @ r0[s_hi].T) @ wt) * (1 - np.exp(-1j * K[:, d]))
    return lam, np.abs(r0).sum(1).max()


def test_symbol_is_consistent():
    """lambda(k) = -i sum_d k_d + O(|k|^(2R)) near k = 0 (exact translation of smooth modes)."""
    for dim, R in ((2, 2), (2, 3), (3, 2)):
        r0 = oracle.weights(dim, R)[0][0]
        offs = np.array(stencils.full_stencil(dim, R))[:, :dim]
        NT = R ** (dim - 1)
        glw = oracle.gl_weights(R)
        wt = np.array([glw[t % R] * (glw[t // R] if dim == 3 else 1.0) for t in range(NT)])
        for eps in (0.05, 0.1):
            k = np.full(dim, eps)
            lam = 0j
            for d in range(dim):
                s_hi = [(2 * d + 1) * NT + t for t in range(NT)]
                rho = (np.exp(1j * offs @ k) @ r0[s_hi].T) @ wt
                lam -= rho * (1 - np.exp(-1j * k[d]))
            assert abs(lam - (-1j * k.sum())) < 50 * eps ** (2 * R), (dim, R, eps, lam)


def test_2d_radius2_linear_scheme_does_not_amplify():
    lam, s = _symbol(2, 2)
    assert lam.real.max() <= 1e-12
    assert s < 2.2


@pytest.mark.parametrize("dim,R,re_max,sum_max", [(2, 3, 0.02, 3.0), (3, 2, 0.05, 3.4)])
def test_other_stencils_nearly_neutral(dim, R, re_max, sum_max):
    lam, s = _symbol(dim, R)
    assert lam.real.max() < re_max and s < sum_max


def test_3d_radius3_linear_scheme_amplifies():
    """The characterisation behind the 3D radius-3 gate's limits: large oscillating weights and an
    amplifying linear scheme (see the module docstring)."""
    lam, s = _symbol(3, 3)
    assert s > 50
    assert lam.real.max() > 1.0
    assert np.abs(lam).max() > 50
