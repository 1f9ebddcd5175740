"""The allocation-free entry point kfvm_flux_static against kfvm_flux.

kfvm_flux_static serves callers that must not allocate device memory (plug-ins
inside an application that owns the device-memory budget, loops that must not
call cudaMalloc/cudaFree): its scratch is one fixed device array inside the
library.  This file is named so that pytest collects it last.  It must pass
alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_16543_gb300 as p
    L = p.load()
    L.kfvm_flux_static.argtypes = [ctypes.POINTER(p._Grid), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return p


def _grid(pkg, n, bc):
    g = pkg._Grid()
    for a in range(3):
        g.n[a] = n[a] if a < len(n) else 1
        g.lo[a] = 0.0
        g.hi[a] = 1.0
        for s in range(2):
            g.bc[a][s] = pkg.BC[bc] if a < len(n) else 0
    return g


def _flux_static(pkg, grid, dims, radius, faces, dUdt, status, riemann=0):
    stream = torch.cuda.current_stream().cuda_stream
    return pkg.load().kfvm_flux_static(ctypes.byref(grid), dims, radius, 1.4, riemann,
                                       ctypes.c_void_p(faces.data_ptr()), ctypes.c_void_p(dUdt.data_ptr()),
                                       ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream))


@pytest.mark.parametrize("dims,radius,n,bc,riemann", [
    (2, 2, (96, 80), "outflow", 0),
    (3, 2, (20, 18, 12), "periodic", 0),
    (2, 3, (70, 52), "periodic", 1),       # radius 3 with HLL
    (3, 3, (14, 12, 11), "outflow", 1),
    (3, 2, (51, 51, 51), "outflow", 0),    # the largest cube the fixed array holds
])
def test_static_flux_matches_kfvm_flux_twice(pkg, dims, radius, n, bc, riemann):
    g = pkg.KFVM(list(n), dims=dims, radius=radius, bc=bc)
    g.set_option("riemann", riemann)
    grid = _grid(pkg, n, bc)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for seed in (11, 12):  # two calls in a row, on different inputs
        U0 = workloads.mixed_voronoi(dims, max(n), 8, seed=seed, R=radius)
        U0 = (U0[:, :n[2], :n[1], :n[0]] if dims == 3 else U0[:, :n[1], :n[0]]).contiguous().cuda()
        faces = g.reconstruct(U0)
        want = g.flux(faces)
        got = torch.full_like(want, float("nan"))
        assert _flux_static(pkg, grid, dims, radius, faces, got, status, riemann) == 0
        torch.cuda.synchronize()
        err = (got - want).abs().max().item() / want.abs().max().item()
        assert err <= 1e-12, err
        assert int(status.item()) == 0


@pytest.mark.parametrize("n", [(1024, 1024), (512, 512), (52, 52, 52), (51, 52, 52)])
def test_static_flux_rejects_too_large_problems(pkg, n):
    """Just beyond the fixed array (2D above 511^2, 3D above 51^3) the call fails before any launch."""
    grid = _grid(pkg, n, "outflow")
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _flux_static(pkg, grid, len(n), 2, dummy, dummy, status) == 8  # KFVM_ERR_TOO_LARGE
