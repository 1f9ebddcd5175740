"""GB300 (sm_103a) KFVM-WENO hot path: a thin Python binding of ``libkfvm.so``.

The binding only marshals arguments to the C ABI declared in
``include/kfvm.h``: every step of the path runs in the library's CUDA kernels.
PyTorch provides device memory and streams.  There is no CPU fallback: if the
library is missing or no CUDA device is present, the compute calls raise.

Method: May & Lee, "KFVM-WENO: a high-order accurate kernel-based finite
volume method for compressible hydrodynamics", arXiv 2401.16543 (Sec. 2-5).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["KFVM", "load", "stencil_info", "measure_fma_peak", "KfvmError", "library_path"]

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "_build", "libkfvm.so")

STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "singular weight system",
          4: "non-admissible state", 5: "call out of order", 6: "device wait timed out", 7: "out of memory",
          8: "problem exceeds a fixed-size buffer"}
BC = {"periodic": 0, "outflow": 1}


class KfvmError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)} (status {code})")
        self.code = code


class _Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("bc", (ctypes.c_int * 2) * 3)]


_lib = None


def load():
    """Load libkfvm.so (built in-tree by ``paper_2401_16543_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(library_path):
        raise RuntimeError(f"libkfvm.so is not built ({library_path}); run paper_2401_16543_gb300.build.build()")
    L = ctypes.CDLL(library_path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    L.kfvm_init.argtypes = [ctypes.POINTER(P), ctypes.POINTER(_Grid), I, I, D, D]
    L.kfvm_build_weights.argtypes = [P, P]
    L.kfvm_get_weights.argtypes = [P, ctypes.POINTER(D), S]
    L.kfvm_weights_count.argtypes = [P]
    L.kfvm_weights_count.restype = S
    L.kfvm_set_option.argtypes = [P, ctypes.c_char_p, D]
    L.kfvm_reconstruct.argtypes = [P, P, P, P]
    L.kfvm_flux.argtypes = [P, P, P, P]
    L.kfvm_rhs.argtypes = [P, P, P, P]
    L.kfvm_step.argtypes = [P, P, D, D, ctypes.POINTER(D), P]
    L.kfvm_sync_status.argtypes = [P, P]
    L.kfvm_gate_param_count.argtypes = [P]
    L.kfvm_gate_param_count.restype = S
    L.kfvm_gate_set_params.argtypes = [P, ctypes.POINTER(ctypes.c_float), S]
    L.kfvm_gate_get_params.argtypes = [P, ctypes.POINTER(ctypes.c_float), S]
    L.kfvm_gate_features.argtypes = [P, P, P, P, D, P]
    L.kfvm_gate_forward.argtypes = [P, P, P, S, P]
    L.kfvm_set_smooth_mask.argtypes = [P, P, P]
    L.kfvm_gate_mask.argtypes = [P, P, P, P]
    L.kfvm_kxrcf_mask.argtypes = [P, P, P, P]
    L.kfvm_gate_train_step.argtypes = [P, P, P, S, ctypes.c_float, P, P, P]
    L.kfvm_gate_load.argtypes = [P, P, S]
    L.kfvm_gate_train.argtypes = [P, P, P, S, I, ctypes.c_float, P]
    L.kfvm_stencil_info.argtypes = [I, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]
    L.kfvm_launch_count.argtypes = [P]
    L.kfvm_launch_count.restype = ctypes.c_longlong
    L.kfvm_measure_fma_peak.argtypes = [I, ctypes.POINTER(D)]
    L.kfvm_profile_count.argtypes = []
    L.kfvm_profile_get.argtypes = [P, I, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_longlong),
                                   ctypes.POINTER(D)]
    L.kfvm_profile_reset.argtypes = [P]
    L.kfvm_destroy.argtypes = [P]
    L.kfvm_destroy.restype = None
    L.kfvm_status_string.argtypes = [I]
    L.kfvm_status_string.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(code: int, what: str):
    if code != 0:
        raise KfvmError(code, what)


def stencil_info(dims: int, radius: int):
    """Host-only: (sizes N_q, degrees p_q, F face points, M derivatives) of every (sub)stencil."""
    L = load()
    sizes = (ctypes.c_int * 8)()
    degs = (ctypes.c_int * 8)()
    F, M = ctypes.c_int(), ctypes.c_int()
    n = L.kfvm_stencil_info(dims, radius, sizes, degs, ctypes.byref(F), ctypes.byref(M))
    if n < 0:
        raise ValueError("unsupported (dims, radius)")
    return list(sizes)[:n], list(degs)[:n], F.value, M.value


def measure_fma_peak(bits: int) -> float:
    """Measured FMA throughput of the current device in flop/s (bits = 32 or 64)."""
    out = ctypes.c_double()
    _check(load().kfvm_measure_fma_peak(bits, ctypes.byref(out)), "kfvm_measure_fma_peak")
    return out.value


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class KFVM:
    """One grid + scheme on the current CUDA device.

    ``n``: cells per axis (nx, ny[, nz]); ``bc``: "periodic" / "outflow" per axis
    (or per side pairs).  State tensors are float64 CUDA tensors of shape
    (nv, ny, nx) or (nv, nz, ny, nx).
    """

    def __init__(self, n, dims: int = 2, radius: int = 2, lo=None, hi=None, bc="periodic",
                 ell_over_dx: float = 5.0, gamma: float = 1.4, build_weights: bool = True):
        self._L = load()
        self.dims, self.R, self.nv = dims, radius, dims + 2
        n = list(n)
        lo = list(lo) if lo is not None else [0.0] * dims
        hi = list(hi) if hi is not None else [1.0] * dims
        if isinstance(bc, str):
            bc = [(bc, bc)] * dims
        bc = [(b, b) if isinstance(b, str) else tuple(b) for b in bc]
        g = _Grid()
        for a in range(3):
            g.n[a] = n[a] if a < dims else 1
            g.lo[a] = lo[a] if a < dims else 0.0
            g.hi[a] = hi[a] if a < dims else 1.0
            for s in range(2):
                g.bc[a][s] = BC[bc[a][s]] if a < dims else 0
        self.shape = (self.nv,) + tuple(reversed(n[:dims]))
        self.ncell = int(np.prod(n[:dims]))
        sizes, degs, self.nface, self.nderiv = stencil_info(dims, radius)
        self.sizes, self.degrees = sizes, degs
        self._ctx = ctypes.c_void_p()
        _check(self._L.kfvm_init(ctypes.byref(self._ctx), ctypes.byref(g), dims, radius, ell_over_dx, gamma),
               "kfvm_init")
        self.precision = 64
        if build_weights:
            self.build_weights()

    def __del__(self):
        ctx = getattr(self, "_ctx", None)
        if ctx is not None and ctx.value:
            self._L.kfvm_destroy(ctx)
            self._ctx = None

    # -- set-up ------------------------------------------------------------------
    def build_weights(self, stream=None):
        _check(self._L.kfvm_build_weights(self._ctx, _stream(stream)), "kfvm_build_weights")

    def weights(self) -> np.ndarray:
        n = self._L.kfvm_weights_count(self._ctx)
        out = np.zeros(n)
        _check(self._L.kfvm_get_weights(self._ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n),
               "kfvm_get_weights")
        return out

    def set_option(self, key: str, value: float):
        _check(self._L.kfvm_set_option(self._ctx, key.encode(), float(value)), f"kfvm_set_option({key})")
        if key == "precision":
            self.precision = int(value)

    # -- hot path ----------------------------------------------------------------
    def _state(self, U):
        import torch
        if U.dtype != torch.float64 or not U.is_cuda or not U.is_contiguous() or tuple(U.shape) != self.shape:
            raise ValueError(f"state must be a contiguous float64 CUDA tensor of shape {self.shape}")
        return U

    def face_dtype(self):
        import torch
        return torch.float64 if self.precision == 64 else torch.float32

    def reconstruct(self, U, faces=None, stream=None):
        import torch
        U = self._state(U)
        if faces is None:
            faces = torch.empty((self.nface, self.nv) + self.shape[1:], dtype=self.face_dtype(), device=U.device)
        _check(self._L.kfvm_reconstruct(self._ctx, _ptr(U), _ptr(faces), _stream(stream)), "kfvm_reconstruct")
        return faces

    def faces_primitive(self, faces):
        """FP32-mode Riemann states as a [F, nv, cells] float32 tensor of (rho, u, v[, w], p)."""
        import torch
        F, n = self.nface, self.ncell
        flat = faces.reshape(-1)
        a4 = flat[:F * n * 4].reshape(F, n, 4)
        comps = [a4[..., 0], a4[..., 1], a4[..., 2]]
        if self.dims == 3:
            comps.append(flat[F * n * 4:F * n * 5].reshape(F, n))
        comps.append(a4[..., 3])
        return torch.stack(comps, dim=1)

    def flux(self, faces, dUdt=None, stream=None):
        import torch
        if dUdt is None:
            dUdt = torch.empty(self.shape, dtype=torch.float64, device=faces.device)
        _check(self._L.kfvm_flux(self._ctx, _ptr(faces), _ptr(dUdt), _stream(stream)), "kfvm_flux")
        return dUdt

    def rhs(self, U, dUdt=None, stream=None):
        import torch
        U = self._state(U)
        if dUdt is None:
            dUdt = torch.empty(self.shape, dtype=torch.float64, device=U.device)
        _check(self._L.kfvm_rhs(self._ctx, _ptr(U), _ptr(dUdt), _stream(stream)), "kfvm_rhs")
        return dUdt

    def step(self, U, cfl: float, t_remaining: float = float("inf"), sync: bool = True, stream=None):
        """One SSP-RK3 step of U in place; returns dt when sync (reads the device status), else None."""
        U = self._state(U)
        t_rem = t_remaining if np.isfinite(t_remaining) else 1e300
        if sync:
            dt = ctypes.c_double()
            _check(self._L.kfvm_step(self._ctx, _ptr(U), cfl, t_rem, ctypes.byref(dt), _stream(stream)), "kfvm_step")
            return dt.value
        _check(self._L.kfvm_step(self._ctx, _ptr(U), cfl, t_rem, None, _stream(stream)), "kfvm_step")
        return None

    def sync_status(self, stream=None):
        _check(self._L.kfvm_sync_status(self._ctx, _stream(stream)), "device status")

    def run(self, U, cfl: float, t_end: float, max_steps: int = 10 ** 9):
        """Advance U in place to t_end; returns (t, steps)."""
        t, k = 0.0, 0
        while t < t_end and k < max_steps:
            dt = self.step(U, cfl, t_end - t)
            t += dt
            k += 1
        return t, k

    @property
    def launches(self) -> int:
        return int(self._L.kfvm_launch_count(self._ctx))

    def profile(self):
        """{kernel family: (launches, device ms)} since the last reset (needs the "profile" option and a sync)."""
        out = {}
        for i in range(self._L.kfvm_profile_count()):
            name = ctypes.c_char_p()
            n = ctypes.c_longlong()
            ms = ctypes.c_double()
            _check(self._L.kfvm_profile_get(self._ctx, i, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms)),
                   "kfvm_profile_get")
            if n.value:
                out[name.value.decode()] = (int(n.value), float(ms.value))
        return out

    def profile_reset(self):
        _check(self._L.kfvm_profile_reset(self._ctx), "kfvm_profile_reset")

    # -- learned gate --------------------------------------------------------------
    @property
    def gate_param_count(self) -> int:
        return int(self._L.kfvm_gate_param_count(self._ctx))

    def gate_set_params(self, params):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        _check(self._L.kfvm_gate_set_params(self._ctx, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size),
               "kfvm_gate_set_params")

    def gate_load(self, weights):
        """Load float32 or bfloat16 (numpy uint16 bit patterns) packed parameters."""
        w = np.ascontiguousarray(weights)
        _check(self._L.kfvm_gate_load(self._ctx, w.ctypes.data_as(ctypes.c_void_p), w.nbytes), "kfvm_gate_load")

    def gate_train(self, X, y, epochs: int, lr: float, stream=None):
        """Adam epochs over (X, y) in mini-batches of 2048 (device tensors)."""
        _check(self._L.kfvm_gate_train(self._ctx, _ptr(X), _ptr(y), X.shape[0], int(epochs), float(lr),
                                       _stream(stream)), "kfvm_gate_train")

    def gate_get_params(self) -> np.ndarray:
        p = np.zeros(self.gate_param_count, dtype=np.float32)
        _check(self._L.kfvm_gate_get_params(self._ctx, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size),
               "kfvm_gate_get_params")
        return p

    def gate_features(self, U, tau: float = 0.02, stream=None):
        import torch
        U = self._state(U)
        n_in = 26 if self.dims == 2 else 68  # radius-2 blocks of rho and p (+ 3D radius-3 shell inputs)
        X = torch.empty((self.ncell, n_in), dtype=torch.float32, device=U.device)
        y = torch.empty(self.ncell, dtype=torch.float32, device=U.device)
        _check(self._L.kfvm_gate_features(self._ctx, _ptr(U), _ptr(X), _ptr(y), float(tau), _stream(stream)),
               "kfvm_gate_features")
        return X, y

    def gate_mask(self, U, stream=None):
        """The gate's smooth mask of U (uint8 per cell), as the gated step computes it."""
        import torch
        U = self._state(U)
        m = torch.empty(self.shape[1:], dtype=torch.uint8, device=U.device)
        _check(self._L.kfvm_gate_mask(self._ctx, _ptr(U), _ptr(m), _stream(stream)), "kfvm_gate_mask")
        return m

    def kxrcf_mask(self, U, stream=None):
        """The KXRCF indicator's smooth mask of U (uint8 per cell, 1 = linear), as the "recon" 4 step
        computes it: from the float32 copy of U in the FP32 mode, from U in the FP64 mode."""
        import torch
        U = self._state(U)
        m = torch.empty(self.shape[1:], dtype=torch.uint8, device=U.device)
        _check(self._L.kfvm_kxrcf_mask(self._ctx, _ptr(U), _ptr(m), _stream(stream)), "kfvm_kxrcf_mask")
        return m

    def set_smooth_mask(self, mask, stream=None):
        """Gated reconstruction driven by a caller-supplied uint8 CUDA mask (1 = linear)."""
        _check(self._L.kfvm_set_smooth_mask(self._ctx, _ptr(mask), _stream(stream)), "kfvm_set_smooth_mask")

    def gate_forward(self, X, stream=None):
        import torch
        prob = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        _check(self._L.kfvm_gate_forward(self._ctx, _ptr(X), _ptr(prob), X.shape[0], _stream(stream)),
               "kfvm_gate_forward")
        return prob

    def gate_train_step(self, X, y, lr: float, loss=None, grads=None, stream=None):
        _check(self._L.kfvm_gate_train_step(self._ctx, _ptr(X), _ptr(y), X.shape[0], float(lr),
                                            _ptr(loss) if loss is not None else None,
                                            _ptr(grads) if grads is not None else None, _stream(stream)),
               "kfvm_gate_train_step")
