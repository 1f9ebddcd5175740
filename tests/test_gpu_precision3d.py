"""The mixed-precision path's error against the plain FP64 path, per conserved variable, on the 3D
256^3 radius-2 workload (x < 1/2 the smooth sine advection, x >= 1/2 128 seeded Voronoi regions,
periodic, CFL 0.4): after 1, 5 and 20 SSP-RK3 steps from the same state, each path with its own dt,
the relative L1 difference of every variable stays below 1e-6 (the precision-only part of the
matched-L1 target) and the largest pointwise difference below 2e-6 of the variable's magnitude (the
one-step FP32 bar, not accumulated: the update is formed in float64)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads  # noqa: E402

NAMES = ["rho", "m_x", "m_y", "m_z", "E"]


def test_fp32_per_variable_error_against_fp64_256cubed():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_16543_gb300 as pkg
    n = 256
    U0 = workloads.half_sine_voronoi_3d(n, k=128, seed=3, device="cuda")
    g64 = pkg.KFVM([n] * 3, dims=3, radius=2, bc="periodic")
    g32 = pkg.KFVM([n] * 3, dims=3, radius=2, bc="periodic")
    g32.set_option("precision", 32)
    U64, U32 = U0.clone(), U0.clone()
    k = 0
    for target in (1, 5, 20):
        while k < target:
            g64.step(U64, 0.4)
            g32.step(U32, 0.4)
            k += 1
        row = []
        for v in range(5):
            d = (U32[v] - U64[v]).abs()
            mx = (d.max() / U64[v].abs().max()).item()
            l1 = (d.sum() / U64[v].abs().sum()).item()
            row.append(f"{NAMES[v]} {mx:.2e}/{l1:.2e}")
            assert l1 <= 1e-6, (k, NAMES[v], l1)
            assert mx <= 2e-6, (k, NAMES[v], mx)
        print(f"steps {k}: " + ", ".join(row))
