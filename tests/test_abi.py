"""CPU checks of the C ABI: the library loads without a GPU, exports every entry point
declared in include/kfvm.h, and its host-side stencil logic matches the oracle."""
import os
import re

import pytest

import oracle
from oracle import stencils

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_16543_gb300 import build
    build.build()
    import paper_2401_16543_gb300 as pkg
    return pkg.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "kfvm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kfvm_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("dim,R", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_host_stencil_info_matches_oracle(lib, dim, R):
    import paper_2401_16543_gb300 as pkg
    sizes, degs, F, M = pkg.stencil_info(dim, R)
    assert sizes == [len(s) for s in stencils.substencils(dim, R)]
    assert degs == list(stencils.degrees(dim, R))
    assert F == stencils.n_face_points(dim, R)
    assert M == len(stencils.deriv_indices(dim, R))


def test_unsupported_arguments_are_rejected(lib):
    import paper_2401_16543_gb300 as pkg
    with pytest.raises(ValueError):
        pkg.stencil_info(4, 2)
    assert lib.kfvm_status_string(4) == b"non-admissible state (rho <= 0, p <= 0 or NaN)"
