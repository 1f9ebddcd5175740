"""Oracle of the learned smooth-cell gate (test infrastructure only).

The gate has no counterpart in the paper; it stands where the paper's
troubled-cell indicator stands (Sec. 3.5 and Sec. 5.3 step 2): cells it marks
smooth take the unlimited linear reconstruction, the others WENO-AO.  This
module states, in plain FP64 numpy, what the GPU's gate computes:

* ``features``: for each cell, the radius-2 full stencil of rho and of the
  cell-average pressure p = (gamma-1)(E - |m|^2/(2 rho)), each block as
  deviations from the central cell's value divided by
  d = max(max |deviation|, 1e-4 |central value|) (+1e-30): exactly zero on
  constant data, unchanged by a common scaling of the state; the 1e-4 floor is
  the amplitude below which the labels call a component smooth, so a variation
  that small shows as a small input (and the ~1e-7 rounding of a float32
  pressure stays below 0.01).  In 3D two more
  inputs describe the shell 4 < |o|^2 <= 9 that a radius-3 reconstruction also
  reads (the radius-2 block cannot see a jump three cells away): per block
  m / (m + d) with m = max |deviation| over the shell, in [0, 1); they are zero
  unless the reconstruction radius is 3.
* ``labels``: 1 when the density and pressure components of the linearized
  primitive variables (the two quantities the features describe) are both
  smooth by the cell's own WENO-AO weights (omega_0/gamma_0 >= 1 - tau; Eqs.
  24-25 of the paper, from the oracle's reconstruction) or vary over the
  radius-R stencil by less than 1e-4 of their scale (rho~, p~), where WENO-AO
  and the linear reconstruction cannot differ by more than that (truncation
  errors of a smooth flow stay below it, and WENO-AO weights of such noise say
  nothing about smoothness).
* ``forward`` / ``loss_and_grad``: the MLP NIN -> 32 -> 32 -> 1 (ReLU, ReLU,
  sigmoid) and the gradient of its mean binary cross-entropy by backprop.
  Parameter packing: W1 [32][NIN], b1 [32], W2 [32][32], b2 [32], W3 [32], b3.
* ``bf16``: round-to-nearest-even to bfloat16 (the GPU's operand precision).

Pinned by tests/test_oracle_gate.py: gradients against central finite
differences, the closed-form loss of a constant network, feature invariance
under shift and scale, constant data giving zero features.
"""
from __future__ import annotations

import numpy as np

from . import stencils

H = 32


def n_in(dim: int) -> int:
    return 2 * len(stencils.full_stencil(dim, 2)) + (2 if dim == 3 else 0)


def shell_offsets():
    """3D offsets with 4 < |o|^2 <= 9: the radius-3 stencil minus the radius-2 stencil."""
    inner = set(map(tuple, stencils.full_stencil(3, 2)))
    return [o for o in stencils.full_stencil(3, 3) if tuple(o) not in inner]


def param_count(dim: int) -> int:
    ni = n_in(dim)
    return H * ni + H + H * H + H + H + 1


def unpack(params, dim: int):
    ni = n_in(dim)
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * ni].reshape(H, ni); o += H * ni
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, W3, [b3]])


def init_params(dim: int, seed: int = 0) -> np.ndarray:
    """He-style initialisation from a seeded numpy generator (float32 values)."""
    ni = n_in(dim)
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / ni), (H, ni))
    W2 = rng.normal(0, np.sqrt(2.0 / H), (H, H))
    W3 = rng.normal(0, np.sqrt(1.0 / H), H)
    return pack(W1, np.zeros(H), W2, np.zeros(H), W3, 0.0).astype(np.float32)


def bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def features(U, dim: int, bc="periodic", gamma: float = 1.4, R: int = 2) -> np.ndarray:
    """Gate inputs of every cell, [ncell, NIN] (cells in x-fastest order); R is the
    reconstruction radius (3D shell inputs are computed for R = 3, zero otherwise)."""
    U = np.asarray(U, dtype=np.float64)
    if isinstance(bc, str):
        bc = [bc] * dim
    s0 = stencils.full_stencil(dim, 2)
    shape = U.shape[1:]
    mode = ["wrap" if b == "periodic" else "edge" for b in bc]
    # numpy axes are (z,) y, x: axis a of the grid is numpy axis dim-1-a
    H = 3  # halo wide enough for the 3D shell
    padded = []
    for v in range(dim + 2):
        a = U[v]
        for ax in range(dim):
            npax = dim - 1 - ax
            widths = [(0, 0)] * dim
            widths[npax] = (H, H)
            a = np.pad(a, widths, mode=mode[ax])
        padded.append(a)
    P = np.stack(padded)
    rho = P[0]
    m2 = sum(P[1 + k] ** 2 for k in range(dim))
    p = (gamma - 1.0) * (P[dim + 1] - 0.5 * m2 / rho)

    def column(field, o):
        sl = []
        for npax in range(dim):
            ax = dim - 1 - npax
            lo = H + o[ax]
            sl.append(slice(lo, lo + shape[npax]))
        return field[tuple(sl)].ravel()

    centre = [n for n, o in enumerate(s0) if o == (0, 0, 0)][0]
    out, shell = [], []
    for field in (rho, p):
        A = np.stack([column(field, o) for o in s0], axis=1)
        c = A[:, centre:centre + 1]
        dev = A - c
        scale = np.maximum(np.abs(dev).max(axis=1, keepdims=True), 1e-4 * np.abs(c) + 1e-30)
        out.append(dev / scale)
        if dim == 3:
            if R >= 3:
                Sh = np.stack([column(field, o) for o in shell_offsets()], axis=1)
                m = np.abs(Sh - c).max(axis=1, keepdims=True)
                shell.append(m / (m + scale))
            else:
                shell.append(np.zeros_like(c))
    return np.concatenate(out + shell, axis=1)


def linprim_amplitude(U, dim: int, R: int, bc="periodic", gamma: float = 1.4):
    """Per cell and linearized primitive component: max over the radius-R stencil of |Phi (U_h - U_c)|
    divided by the component's scale; [nv, ncell]."""
    U = np.asarray(U, dtype=np.float64)
    if isinstance(bc, str):
        bc = [bc] * dim
    s0 = stencils.full_stencil(dim, R)
    shape = U.shape[1:]
    mode = ["wrap" if b == "periodic" else "edge" for b in bc]
    P = []
    for v in range(dim + 2):
        a = U[v]
        for ax in range(dim):
            widths = [(0, 0)] * dim
            widths[dim - 1 - ax] = (R, R)
            a = np.pad(a, widths, mode=mode[ax])
        P.append(a)
    P = np.stack(P)
    Uc = U.reshape(dim + 2, -1)
    rho = Uc[0]
    u = Uc[1:1 + dim] / rho
    kin = 0.5 * (u ** 2).sum(0)
    p = (gamma - 1.0) * (Uc[dim + 1] - rho * kin)
    cs = np.sqrt(gamma * p / rho)
    amp = np.zeros((dim + 2, Uc.shape[1]))
    for o in s0:
        sl = []
        for npax in range(dim):
            ax = dim - 1 - npax
            sl.append(slice(R + o[ax], R + o[ax] + shape[npax]))
        dU = np.stack([P[v][tuple(sl)].ravel() for v in range(dim + 2)]) - Uc
        w = [dU[0]] + [(dU[1 + k] - u[k] * dU[0]) / rho for k in range(dim)]
        w.append((gamma - 1.0) * (kin * dU[0] - (u * dU[1:1 + dim]).sum(0) + dU[dim + 1]))
        amp = np.maximum(amp, np.abs(np.stack(w)))
    scale = np.stack([rho] + [cs] * dim + [p])
    return amp / scale


LABEL_VARS = (0, -1)  # density and pressure components of the linearized primitive variables


def labels_from_omega(omega, dim: int, tau: float, amplitude=None):
    """Labels from the oracle's weights omega [nq, nv, *grid] and (optionally) linprim_amplitude;
    returns (y, worst ratio over the components that count: density and pressure)."""
    g0 = stencils.linear_weights(dim)[0]
    ratio = (omega[0] / g0).reshape(omega.shape[1], -1)
    if amplitude is not None:
        ratio = np.where(amplitude <= 1e-4, 1.0, ratio)
    worst = ratio[list(LABEL_VARS)].min(axis=0)
    return (worst >= 1.0 - tau).astype(np.float64), worst


def forward(params, X, dim: int, quantize: bool = False):
    """Logits z [n]; with quantize=True operands are rounded to bf16 where the GPU rounds them."""
    W1, b1, W2, b2, W3, b3 = unpack(params, dim)
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    h1 = np.maximum(q(X) @ q(W1).T + b1, 0.0)
    h2 = np.maximum(q(h1) @ q(W2).T + b2, 0.0)
    return q(h2) @ q(W3) + b3


def loss_and_grad(params, X, y, dim: int, quantize: bool = False):
    """Mean binary cross-entropy of sigmoid(z) against y, and its gradient (FP64 backprop).

    With quantize=True every matrix-product operand is rounded to bf16 where the
    GPU's tensor-core kernels round it (inputs, weights, activations and the
    back-propagated dH1, dH2); sums stay FP64.
    """
    W1, b1, W2, b2, W3, b3 = unpack(params, dim)
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = X.shape[0]
    a1 = q(X) @ q(W1).T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = q(h1) @ q(W2).T + b2
    h2 = np.maximum(a2, 0.0)
    z = q(h2) @ q(W3) + b3
    loss = np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z))))
    p = 1.0 / (1.0 + np.exp(-z))
    dz = (p - y) / n
    gW3 = q(h2).T @ dz
    gb3 = dz.sum()
    dh2 = q(np.outer(dz, q(W3)) * (a2 > 0))
    gW2 = dh2.T @ q(h1)
    gb2 = dh2.sum(axis=0)
    dh1 = q((dh2 @ q(W2)) * (a1 > 0))
    gW1 = dh1.T @ q(X)
    gb1 = dh1.sum(axis=0)
    return loss, pack(gW1, gb1, gW2, gb2, gW3, gb3)
