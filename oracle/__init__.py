"""The KFVM-WENO oracle: a plain, slow, obviously correct CPU implementation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path in ``paper_2401_16543_gb300`` and neither imports the
other.  The product path never falls back to it.

Layers (each cites the paper, May & Lee, arXiv 2401.16543):

* ``oracle.stencils`` -- stencils, substencils, polynomial degrees (exact
  rational rank), multi-indices, linear weights (Sec. 3.1-3.3).
* ``kfvm_oracle.c``   -- binary128 weight solve (Sec. 2.1, Eqs. 6-18, 23) and
  the FP64 per-cell pipeline (Sec. 3-5), loaded here through ctypes.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against what the paper and the mathematics fix (printed stencil sizes,
polynomial reproduction, an independent mpmath solve, closed-form sample
problems, the exact Sod solution, invariants).  The one unpinned part is the
Riemann solver's "+" term of HLLC+, which the paper cites but does not define:
HLLC (Toro) with Batten wave speeds is used, so "parity unpinned" applies to
HLLC+ specifically.
"""
from __future__ import annotations

import ctypes
from functools import lru_cache

import numpy as np

from . import gate, stencils
from .build import build as _build

__all__ = ["Oracle", "weights", "flat_weights", "stencils", "phi_matrices", "char_matrices", "riemann_flux",
           "face_points", "gate"]

_I = ctypes.c_int
_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_PI = ctypes.POINTER(ctypes.c_int)


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", _I), ("R", _I), ("nv", _I),
        ("n", _I * 3),
        ("dx", _D * 3),
        ("bc", (_I * 2) * 3),
        ("gamma", _D), ("eps", _D),
        ("nq", _I), ("n0", _I),
        ("offs", _PI), ("sub_len", _PI), ("sub_idx", _PI),
        ("lin_w", _PD),
        ("nface", _I), ("nderiv", _I),
        ("wts", _PD), ("gl_w", _PD),
        ("recon", _I), ("riemann", _I),
        ("positivity", _I), ("kappa", _D), ("eta", _D),
        ("mask", ctypes.POINTER(ctypes.c_ubyte)),
        ("kxrcf_m", _D),
        ("vars", _I),
    ]


_libs = {}


def lib(threaded: bool = False):
    """The oracle's C library; ``threaded`` loads the OpenMP timing build of the same source (equal
    results, cell loops over all host cores), used only to time the oracle on every core."""
    if threaded not in _libs:
        L = ctypes.CDLL(_build(threaded=threaded))
        L.kfo_weights.argtypes = [_I, _I, _D, _I, _PI, _I, _PI, _I, _PI, _PD, _PD]
        L.kfo_weights.restype = _I
        L.kfo_face_points.argtypes = [_I, _I, _PD]
        L.kfo_face_points.restype = _I
        L.kfo_gl_weights.argtypes = [_I, _PD]
        L.kfo_gl_weights.restype = _I
        P = ctypes.POINTER(_Problem)
        L.kfo_reconstruct.argtypes = [P, _PD, _PD, _PD]
        L.kfo_reconstruct.restype = _I
        L.kfo_kxrcf.argtypes = [P, _PD, _PD, ctypes.POINTER(ctypes.c_ubyte)]
        L.kfo_kxrcf.restype = _I
        L.kfo_limit.argtypes = [P, _PD, _PD]
        L.kfo_limit.restype = _I
        L.kfo_flux.argtypes = [P, _PD, _PD]
        L.kfo_flux.restype = _I
        L.kfo_rhs.argtypes = [P, _PD, _PD]
        L.kfo_rhs.restype = _I
        L.kfo_max_rate.argtypes = [P, _PD]
        L.kfo_max_rate.restype = _D
        L.kfo_step.argtypes = [P, _PD, _D, _D, _PD]
        L.kfo_step.restype = _I
        L.kfo_phi.argtypes = [_I, _D, _PD, _PD, _PD]
        L.kfo_phi.restype = None
        L.kfo_char.argtypes = [_I, _D, _PD, _I, _PD, _PD]
        L.kfo_char.restype = None
        L.kfo_riemann.argtypes = [_I, _D, _I, _I, _PD, _PD, _PD]
        L.kfo_riemann.restype = _I
        _libs[threaded] = L
    return _libs[threaded]


def _pd(a):
    return a.ctypes.data_as(_PD)


def _pi(a):
    return a.ctypes.data_as(_PI)


def face_points(dim: int, R: int) -> np.ndarray:
    """Face Gauss-Legendre points (F x 3) in unit-cell coordinates (Sec. 5.1)."""
    F = stencils.n_face_points(dim, R)
    out = np.zeros((F, 3))
    lib().kfo_face_points(dim, R, _pd(out))
    return out


def gl_weights(R: int) -> np.ndarray:
    w = np.zeros(R)
    lib().kfo_gl_weights(R, _pd(w))
    return w


@lru_cache(maxsize=None)
def weights(dim: int, R: int, ell: float = 5.0):
    """Per (sub)stencil q: (rface [F, N_q], rderiv [M, N_q]) -- Eqs. (14)-(18), (23).

    ``ell`` is the kernel length scale in units of the cell width (ell/Delta,
    Sec. 3.1); the paper uses 5 throughout (Sec. 5.1).
    """
    s0 = stencils.full_stencil(dim, R)
    ders = np.ascontiguousarray(np.array(stencils.deriv_indices(dim, R), dtype=np.int32))
    F = stencils.n_face_points(dim, R)
    out = []
    for idx, p in zip(stencils.substencils(dim, R), stencils.degrees(dim, R)):
        offs = np.ascontiguousarray(np.array([s0[n] for n in idx], dtype=np.int32))
        mons = np.ascontiguousarray(np.array(stencils.monomials(dim, p), dtype=np.int32))
        rf = np.zeros((F, len(idx)))
        rd = np.zeros((len(ders), len(idx)))
        rc = lib().kfo_weights(dim, R, float(ell), len(idx), _pi(offs), len(mons), _pi(mons), len(ders), _pi(ders),
                               _pd(rf), _pd(rd))
        if rc != 0:
            raise RuntimeError(f"oracle weight solve failed (status {rc})")
        rf.setflags(write=False)
        rd.setflags(write=False)
        out.append((rf, rd))
    return tuple(out)


def flat_weights(dim: int, R: int, ell: float = 5.0) -> np.ndarray:
    """All tables concatenated: for q = 0..N_S, the F x N_q face rows then the M x N_q derivative rows."""
    return np.concatenate([np.concatenate([rf.ravel(), rd.ravel()]) for rf, rd in weights(dim, R, ell)])


def phi_matrices(dim: int, gamma: float, ut):
    """(Phi, Phi^{-1}) of the linearized primitive variables at reference state ut (appendix A)."""
    nv = dim + 2
    ut = np.ascontiguousarray(np.asarray(ut, dtype=np.float64))
    phi = np.zeros((nv, nv))
    phinv = np.zeros((nv, nv))
    lib().kfo_phi(dim, float(gamma), _pd(ut), _pd(phi), _pd(phinv))
    return phi, phinv


def char_matrices(dim: int, gamma: float, ut, dir: int):
    """(L, R) of the characteristic variables of direction dir at reference state ut (Sec. 3.4.1)."""
    nv = dim + 2
    ut = np.ascontiguousarray(np.asarray(ut, dtype=np.float64))
    L = np.zeros((nv, nv))
    R = np.zeros((nv, nv))
    lib().kfo_char(dim, float(gamma), _pd(ut), int(dir), _pd(L), _pd(R))
    return L, R


def riemann_flux(dim: int, gamma: float, dir: int, uL, uR, solver: str = "hllc") -> np.ndarray:
    nv = dim + 2
    uL = np.ascontiguousarray(np.asarray(uL, dtype=np.float64))
    uR = np.ascontiguousarray(np.asarray(uR, dtype=np.float64))
    f = np.zeros(nv)
    lib().kfo_riemann(dim, float(gamma), 0 if solver == "hllc" else 1, dir, _pd(uL), _pd(uR), _pd(f))
    return f


_BC = {"periodic": 0, "outflow": 1}


class Oracle:
    """One grid + scheme configuration.

    State arrays are float64 with shape (nv, ny, nx) in 2D and (nv, nz, ny, nx)
    in 3D, variables (rho, rho u, rho v[, rho w], E), x fastest.  ``threaded``
    makes ``step`` use the OpenMP timing build (same results on every core).
    """

    def __init__(self, n, dim: int = 2, R: int = 2, lo=None, hi=None, bc="periodic", gamma: float = 1.4,
                 ell: float = 5.0, eps: float = 1e-40, recon: str = "weno", riemann: str = "hllc",
                 positivity: bool = True, kappa: float = 0.1, eta: float = 0.0, mask=None,
                 kxrcf_m: float = 1.5, variables: str = "linprim", threaded: bool = False):
        self.dim, self.R, self.nv = dim, R, dim + 2
        self._threaded = bool(threaded)
        n = list(n) + [1] * (3 - len(n))
        lo = list(lo) if lo is not None else [0.0] * dim
        hi = list(hi) if hi is not None else [1.0] * dim
        if isinstance(bc, str):
            bc = [(bc, bc)] * dim
        bc = [(b, b) if isinstance(b, str) else tuple(b) for b in bc]
        self.n = n
        self.shape = (self.nv,) + tuple(reversed(n[:dim]))
        self.ncell = n[0] * n[1] * n[2]
        self.dx = [(hi[a] - lo[a]) / n[a] for a in range(dim)] + [1.0] * (3 - dim)
        self.gamma = gamma
        s0 = stencils.full_stencil(dim, R)
        subs = stencils.substencils(dim, R)
        self._offs = np.ascontiguousarray(np.array(s0, dtype=np.int32))
        self._sub_len = np.array([len(s) for s in subs], dtype=np.int32)
        self._sub_idx = np.ascontiguousarray(np.concatenate([np.array(s, dtype=np.int32) for s in subs]))
        self._lin_w = np.array(stencils.linear_weights(dim), dtype=np.float64)
        self._wts = np.ascontiguousarray(flat_weights(dim, R, ell))
        self._gl = np.ascontiguousarray(gl_weights(R))
        self.nface = stencils.n_face_points(dim, R)
        self.nderiv = len(stencils.deriv_indices(dim, R))
        self.nq = len(subs)
        pb = _Problem()
        pb.dim, pb.R, pb.nv = dim, R, self.nv
        for a in range(3):
            pb.n[a] = n[a]
            pb.dx[a] = self.dx[a]
            if a < dim:
                pb.bc[a][0] = _BC[bc[a][0]]
                pb.bc[a][1] = _BC[bc[a][1]]
        pb.gamma, pb.eps = gamma, eps
        pb.nq, pb.n0 = self.nq, len(s0)
        pb.offs, pb.sub_len, pb.sub_idx = _pi(self._offs), _pi(self._sub_len), _pi(self._sub_idx)
        pb.lin_w = _pd(self._lin_w)
        pb.nface, pb.nderiv = self.nface, self.nderiv
        pb.wts, pb.gl_w = _pd(self._wts), _pd(self._gl)
        pb.recon = {"weno": 0, "linear": 1, "gated": 2, "kxrcf": 3}[recon]
        pb.kxrcf_m = float(kxrcf_m)
        pb.vars = {"linprim": 0, "characteristic": 1}[variables]
        if mask is not None:
            self._mask = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).ravel())
            if self._mask.size != self.ncell:
                raise ValueError("mask needs one byte per cell")
            pb.mask = self._mask.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
        pb.riemann = {"hllc": 0, "hll": 1}[riemann]
        pb.positivity, pb.kappa, pb.eta = int(bool(positivity)), float(kappa), float(eta)
        self._pb = pb

    def _state(self, U):
        U = np.ascontiguousarray(np.asarray(U, dtype=np.float64))
        if U.shape != self.shape:
            raise ValueError(f"state shape {U.shape} != {self.shape}")
        return U

    def reconstruct(self, U, with_omega: bool = False):
        """Riemann states [F, nv, *grid]; optionally the weights omega [nq, nv, *grid]."""
        U = self._state(U)
        faces = np.zeros((self.nface, self.nv) + self.shape[1:])
        om = np.zeros((self.nq, self.nv) + self.shape[1:]) if with_omega else None
        st = lib().kfo_reconstruct(ctypes.byref(self._pb), _pd(U), _pd(faces), _pd(om) if with_omega else None)
        self.status = st
        return (faces, om) if with_omega else faces

    def kxrcf(self, U):
        """KXRCF indicator of Sec. 3.5 on the unlimited linear states of U: (ratio, mask) per cell,
        ratio = max over the cell's face points of |q+ - q-| / <Q> with q = p / rho^gamma, mask 1
        (smooth: linear reconstruction) where ratio < Delta^m, Delta the largest cell width."""
        U = self._state(U)
        ratio = np.zeros(self.shape[1:])
        mask = np.zeros(self.shape[1:], dtype=np.uint8)
        self.status = lib().kfo_kxrcf(ctypes.byref(self._pb), _pd(U), _pd(ratio),
                                      mask.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        return ratio, mask

    def limit(self, U, faces):
        """Positivity-preserving limiter of Sec. 4 applied to Riemann states [F, nv, *grid]."""
        U = self._state(U)
        faces = np.ascontiguousarray(np.asarray(faces, dtype=np.float64)).copy()
        self.status = lib().kfo_limit(ctypes.byref(self._pb), _pd(U), _pd(faces))
        return faces

    def flux(self, faces):
        faces = np.ascontiguousarray(np.asarray(faces, dtype=np.float64))
        out = np.zeros(self.shape)
        self.status = lib().kfo_flux(ctypes.byref(self._pb), _pd(faces), _pd(out))
        return out

    def rhs(self, U):
        U = self._state(U)
        out = np.zeros(self.shape)
        self.status = lib().kfo_rhs(ctypes.byref(self._pb), _pd(U), _pd(out))
        return out

    def max_rate(self, U) -> float:
        return float(lib().kfo_max_rate(ctypes.byref(self._pb), _pd(self._state(U))))

    def step(self, U, cfl: float, t_rem: float = float("inf")):
        """One SSP-RK3 step; returns (U_new, dt)."""
        U = self._state(U).copy()
        dt = _D(0.0)
        self.status = lib(self._threaded).kfo_step(ctypes.byref(self._pb), _pd(U), float(cfl), float(t_rem),
                                                   ctypes.byref(dt))
        return U, dt.value

    def run(self, U, cfl: float, t_end: float, max_steps: int = 10 ** 9):
        """Advance to t_end with SSP-RK3; returns (U, t, steps)."""
        t, k = 0.0, 0
        while t < t_end and k < max_steps:
            U, dt = self.step(U, cfl, t_end - t)
            if self.status:
                raise FloatingPointError(f"oracle step failed with status {self.status}")
            t += dt
            k += 1
        return U, t, k
