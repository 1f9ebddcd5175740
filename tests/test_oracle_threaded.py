"""The OpenMP timing build of the oracle (used only to time it on every host core) computes the same
SSP-RK3 step, bit for bit, as the single-threaded checker library."""
import numpy as np
import pytest

import oracle
import workloads


@pytest.mark.parametrize("dim,R,bc", [(2, 2, "outflow"), (3, 3, "periodic")])
def test_threaded_step_equals_single_threaded(dim, R, bc):
    if dim == 2:
        U0 = workloads.voronoi_2d(24, k=9, seed=11).numpy()[:, :20, :24]
        n = [24, 20]
    else:
        U0 = workloads.mixed_voronoi(3, 8, 4, seed=12, R=3).numpy()[:, :6, :7, :8]
        n = [8, 7, 6]
    U0 = np.ascontiguousarray(U0)
    a, dta = oracle.Oracle(n, dim=dim, R=R, bc=bc).step(U0, 0.4)
    o = oracle.Oracle(n, dim=dim, R=R, bc=bc, threaded=True)
    b, dtb = o.step(U0, 0.4)
    assert o.status == 0
    assert dta == dtb
    assert np.array_equal(a, b)


def test_workload_crop_equals_corner_of_full_state():
    """The CPU baseline generates only a corner crop of the large workloads: the same cell averages as
    the corner of the full state."""
    import torch
    full = workloads.mixed_voronoi(3, 24, 12, seed=5, R=3)
    assert torch.equal(full[:, :9, :9, :9], workloads.mixed_voronoi(3, 24, 12, seed=5, R=3, crop=9))
    full = workloads.voronoi_2d(40, k=9, seed=2)
    assert torch.equal(full[:, :13, :13], workloads.voronoi_2d(40, k=9, seed=2, crop=13))
    full = workloads.half_sine_voronoi_3d(20, k=9, seed=3)
    assert torch.equal(full[:, :12, :12, :12], workloads.half_sine_voronoi_3d(20, k=9, seed=3, crop=12))
