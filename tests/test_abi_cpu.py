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


def test_struct_layouts_match_header(lib, tmp_path):
    """The ctypes mirrors of the ABI structs have the size and field offsets
    that a C compiler gives the header's declarations."""
    import subprocess
    from paper_2507_00622_gb300 import chs
    structs = {"chs_params": chs.Params, "chs_ensemble": chs.Ensemble,
               "chs_adaptive": chs.Adaptive}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "chs.h"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append('printf("chs_lyap_job %zu\\n", sizeof(chs_lyap_job)); return 0; }')
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)
    assert int(got["chs_lyap_job"]) == C.sizeof(chs.LyapJob)
    assert C.sizeof(chs.Params) == 112 and C.sizeof(chs.Ensemble) == 72


def test_binding_refuses_host_tensors(lib):
    torch = pytest.importorskip("torch")
    from paper_2507_00622_gb300 import chs
    with pytest.raises(ValueError):
        chs._ptr(torch.zeros(4))


def test_peak_probe_validates_before_cuda(lib):
    from paper_2507_00622_gb300 import chs
    assert lib.chs_peak_probe(0, 1, 32, 10, None, None) == chs.CHS_E_INVALID
    assert lib.chs_peak_probe(chs.PROBE_DFMA, 1, 33, 10, None, None) == chs.CHS_E_INVALID
    assert lib.chs_peak_probe(chs.PROBE_DFMA, 0, 32, 10, None, None) == chs.CHS_E_INVALID
    assert lib.chs_peak_probe(chs.PROBE_DFMA, 1, 32, 1 << 29, None, None) == chs.CHS_E_INVALID
    assert lib.chs_peak_probe(chs.PROBE_DFMA, 1, 32, 10, None, None) == chs.CHS_E_INVALID
    assert "sink" in chs.chs_last_error()
    # work per thread: 8 chains of FMA (2 flops) per iteration, iterations in groups of 4
    assert chs.chs_probe_ops_per_thread(chs.PROBE_DFMA, 1000) == 16000.0
    assert chs.chs_probe_ops_per_thread(chs.PROBE_DFMA, 1001) == 16 * 1004.0
    assert chs.chs_probe_ops_per_thread(chs.PROBE_DFMA_DEP, 1000) == 2000.0
    assert chs.chs_probe_ops_per_thread(chs.PROBE_DSQRT, 1000) == 8000.0
    # 4 FMA chains (8 flops) and 4 MMAs per warp (4 x 512 flops / 32 lanes) per iteration
    assert chs.chs_probe_ops_per_thread(chs.PROBE_DFMA_DMMA, 1000) == (8 + 64) * 1000.0
    assert lib.chs_peak_probe(7, 1, 32, 10, None, None) == chs.CHS_E_INVALID
    # m8n8k4: 512 flops per MMA and warp, 8 MMAs per iteration, per lane
    assert chs.chs_probe_ops_per_thread(chs.PROBE_DMMA, 1000) == 512 * 8 * 1000 / 32
    assert chs.chs_probe_ops_per_thread(99, 1000) == 0.0


def test_params_checks_need_no_device(lib):
    """chs_check_params validates a parameter block without a handle or a GPU:
    the clock budget must be >= 0 (0 = none), and the other fields as every
    entry point checks them."""
    from paper_2507_00622_gb300 import chs
    ok = chs.params(0.01, 100, n_dev=2, clock_budget=0)
    chs.chs_check_params(ok, chs.HENON_HEILES, 2)
    chs.chs_check_params(chs.params(0.01, 100, n_dev=2, clock_budget=1 << 40), chs.HENON_HEILES, 2)
    bad = chs.params(0.01, 100, n_dev=2, clock_budget=-1)
    with pytest.raises(chs.ChsError) as e:
        chs.chs_check_params(bad, chs.HENON_HEILES, 2)
    assert e.value.code == chs.CHS_E_INVALID and "clock_budget" in str(e.value)
    for prm, word in ((chs.params(0.0, 100), "dt"), (chs.params(0.01, -1), "n_steps"),
                      (chs.params(0.01, 10, n_dev=5), "n_dev"),
                      (chs.params(0.01, 10, block_threads=48), "block_threads")):
        with pytest.raises(chs.ChsError) as e:
            chs.chs_check_params(prm, chs.HENON_HEILES, 2)
        assert word in str(e.value)
    assert lib.chs_check_params(None, chs.HENON_HEILES, 2) == chs.CHS_E_INVALID
    # threads per orbit is a choice of the FPUT Lyapunov kernels only
    with pytest.raises(chs.ChsError) as e:
        chs.chs_check_params(chs.params(0.01, 10, threads_per_orbit=2), chs.HENON_HEILES, 2)
    assert e.value.code == chs.CHS_E_UNSUPPORTED and "threads_per_orbit" in str(e.value)


def test_static_scratch_entry_point_names_no_allocation():
    """The entry point for callers that cannot allocate device memory lives in
    csrc/chs_static.cu; nothing in that file may allocate: no cudaMalloc family
    call, no cudaFree, no graph instantiation."""
    src = open(os.path.join(ROOT, "paper_2507_00622_gb300", "csrc", "chs_static.cu")).read()
    code = re.sub(r"//[^\n]*", "", re.sub(r"/\*.*?\*/", "", src, flags=re.S))
    for name in ("cudaMalloc", "cudaMallocAsync", "cudaMallocManaged", "cudaMallocHost", "cudaHostAlloc",
                 "cudaFree", "cudaGraphInstantiate", "cudaStreamBeginCapture", "cuMemAlloc", "malloc(",
                 "new "):
        assert name not in code, name
