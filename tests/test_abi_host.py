"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point declared in include/dwsolve.h, and rejects bad arguments
before touching the device."""
import os
import re

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dw():
    import __graft_entry__ as g
    g.build()
    from paper_0706_2298_gb300 import dwsolve
    return dwsolve


def test_header_symbols_exported(dw):
    hdr = open(os.path.join(ROOT, "include", "dwsolve.h")).read()
    declared = set(re.findall(r"^(?:int|void|size_t|long long|const char\*)\s+\*?(\w+)\(", hdr, re.M))
    assert declared, "no declarations parsed"
    L = dw.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert declared <= set(dw.exported_symbols()) | {"dw_last_error"}


def _links(L):
    from paper_0706_2298_gb300 import synth
    return synth.unit_gauge(L)


@pytest.mark.parametrize("L,bs", [((8, 8, 8, 8), (3, 4, 4, 4)),     # not a power of two
                                  ((8, 8, 8, 12), (4, 4, 4, 4)),    # odd block count (3)
                                  ((8, 8, 8, 8), (8, 8, 4, 4)),     # one block in a direction
                                  ((16, 16, 16, 16), (8, 8, 4, 4))])  # block volume above 512
def test_create_rejects_bad_blocks(dw, L, bs):
    with pytest.raises(dw.DwError) as e:
        dw.dw_create(L, 0.0, 1.0, _links(L), bs)
    assert e.value.rc == dw.DW_EINVAL


def test_create_rejects_non_su3(dw):
    L = (4, 4, 4, 4)
    U = _links(L).clone()
    U[17, 2] *= 1.001
    with pytest.raises(dw.DwError) as e:
        dw.dw_create(L, 0.0, 1.0, U, (2, 2, 2, 2))
    assert e.value.rc == dw.DW_EINVAL and "SU(3)" in str(e.value)
    U = _links(L).clone()
    U[3, 0] *= torch.exp(torch.tensor(2j * 3.14159265358979 / 3, dtype=torch.complex128)) * -1  # det -1
    with pytest.raises(dw.DwError):
        dw.dw_create(L, 0.0, 1.0, U, (2, 2, 2, 2))
