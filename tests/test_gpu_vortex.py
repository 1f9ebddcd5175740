"""Convergence on the isentropic vortex (Sec. 6.1, Table 1): one period (t = 20, the vortex returns to
its initial cells) on the periodic square [-10, 10]^2, the L1 density error against the initial
cell averages, on the GPU through the C ABI.

The paper integrates in time with an error-controlled [4S]*+ scheme; here SSP-RK3 runs at a CFL
number scaled like dx^(2R/3 - 1) from 0.4 at 32^2, so that its O(dt^3) error falls at the spatial
design order 2R and the spatial error dominates.  Expected (paper, Sec. 6.1): order >= 4 at R = 2
and >= 6 at R = 3 beyond 64^2.  The KXRCF path (the paper's configuration; it flags no cell of
this smooth flow and equals the linear path bit for bit) is checked against the paper's Table 1
(tests/golden/vortex_table1.txt): at R = 2 every L1 error within 3% and every order within 0.1;
at R = 3, where the paper's error-controlled integrator differs more from SSP-RK3, within 30%
and 0.3.  WENO-AO everywhere and the FP32 path with the learned gate are reported: the gated path
is never above WENO-AO everywhere by more than 10%, or above the FP32 floor of 5e-6 (the float32
copy of the state rounds at 6e-8 of it in each of ~6000 steps).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads  # noqa: E402
from tests.vortex_golden import table1  # noqa: E402


@pytest.fixture(scope="module")
def kfvm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    import paper_2401_16543_gb300 as pkg
    return pkg, os.path.join(os.path.dirname(pkg.__file__), "gate_params_2d.npy")


def _l1(kfvm, n, R, path):
    pkg, gate = kfvm
    g = pkg.KFVM([n, n], dims=2, radius=R, lo=[-10, -10], hi=[10, 10], bc="periodic")
    if path == "linear":
        g.set_option("recon", 1)
    elif path == "kxrcf":
        g.set_option("recon", 4)
    elif path == "gated32":
        g.set_option("precision", 32)
        g.gate_set_params(np.load(gate))
        g.set_option("gate_threshold", 0.8)
        g.set_option("recon", 2)
    U0 = workloads.isentropic_vortex(n, R)
    U = U0.cuda()
    g.run(U, 0.4 * (32 / n) ** (2 * R / 3 - 1), 20.0)
    return float((U[0] - U0[0].cuda()).abs().mean().item()), U


@pytest.mark.parametrize("R,grids,rtol,eoc_tol", [(2, (32, 64, 128, 256), 0.03, 0.1), (3, (32, 64, 128), 0.3, 0.3)])
def test_vortex_order_of_accuracy(kfvm, R, grids, rtol, eoc_tol):
    paper = table1()
    table, lin_states = {}, {}
    for path in ("linear", "kxrcf", "weno", "gated32"):
        errs = []
        for n in grids:
            e, U = _l1(kfvm, n, R, path)
            errs.append(e)
            if path == "linear":
                lin_states[n] = U.cpu()
            if path == "kxrcf":
                assert torch.equal(U.cpu(), lin_states[n])
        table[path] = np.array(errs)
    for path, e in table.items():
        eoc = np.log2(e[:-1] / e[1:])
        print(f"R={R} {path:8s} L1 " + " ".join(f"{x:.3e}" for x in e) + "  EOC " + " ".join(f"{x:.2f}" for x in eoc))
    e = table["kxrcf"]
    eoc = np.log2(e[:-1] / e[1:])
    for i, n in enumerate(grids):
        want, want_eoc = paper[(R, n)]
        assert abs(e[i] / want - 1) <= rtol, (n, e[i], want)
        if want_eoc is not None:
            assert abs(eoc[i - 1] - want_eoc) <= eoc_tol, (n, eoc[i - 1], want_eoc)
    assert (table["gated32"] <= np.maximum(1.1 * table["weno"], 5e-6)).all(), table
