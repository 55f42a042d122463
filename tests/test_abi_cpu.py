"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every entry point declared in include/chs.h, and
rejects bad arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_00622_gb300 import build, chs
    build.build()
    return chs.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "chs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chs_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    from paper_2507_00622_gb300 import chs
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(chs.EXPORTS) == set(names)


def test_version_and_empty_error(lib):
    from paper_2507_00622_gb300 import chs
    assert "sm_103a" in chs.chs_version()


def test_create_system_validates_before_cuda(lib):
    from paper_2507_00622_gb300 import chs
    h = C.c_void_p()
    assert lib.chs_create_system(C.byref(h), 999, 2, None, 0) == chs.CHS_E_INVALID
    assert "unknown model" in chs.chs_last_error()
    assert lib.chs_create_system(C.byref(h), chs.HENON_HEILES, 3, None, 0) == chs.CHS_E_INVALID
    assert lib.chs_create_system(None, chs.HENON_HEILES, 2, None, 0) == chs.CHS_E_INVALID
    arr = (C.c_double * 2)(1.0, 2.0)
    assert lib.chs_create_system(C.byref(h), chs.FPUT, 8, arr, 2) == chs.CHS_E_INVALID
    assert h.value is None


def test_null_handle_is_rejected(lib):
    from paper_2507_00622_gb300 import chs
    prm = chs.params(0.01, 10, n_dev=2)
    e = chs.Ensemble()
    assert lib.chs_integrate_batch(None, C.byref(prm), C.byref(e), None) == chs.CHS_E_INVALID
    assert lib.chs_system_dim(None) == -1
    assert lib.chs_destroy_system(None) == chs.CHS_OK


def test_struct_layouts_match_header(lib):
    from paper_2507_00622_gb300 import chs
    # chs_params: 1 double, 2 int64, 6 int32, 4 double, 1 uint64 = 88 bytes
    assert C.sizeof(chs.Params) == 88
    assert C.sizeof(chs.Ensemble) == 72


def test_binding_refuses_host_tensors(lib):
    torch = pytest.importorskip("torch")
    from paper_2507_00622_gb300 import chs
    with pytest.raises(ValueError):
        chs._ptr(torch.zeros(4))
