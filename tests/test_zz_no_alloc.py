"""chs_integrate_compacted_static: the compacted run without a caller work buffer.

Some callers of this library cannot hand it device scratch memory: their device
memory belongs to another allocator (a framework's caching allocator, or an arena
sized once at start-up) that gives out no extra buffers, or their rules forbid
any device allocation while the application runs.  For them the orbit lists of
the compacted run live in a fixed device array inside the library, and the call
allocates nothing.  This test runs that entry point through the C ABI next to the
entry point that takes a work buffer, on identical ensembles, for two calls in a
row (the second call reuses the array the first one left behind), and checks the
outputs agree within the parity tolerances used everywhere else.  It sits in a
file that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2507_00622_gb300.inputs import hh_section_box
from tests.helpers import IND_TOL, STATE_RTOL, ind_err, state_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2507_00622_gb300 import chs  # noqa: E402


def _ensemble(S, ics, st, t_end, kw):
    n = ics.shape[1]
    ens = chs.DeviceEnsemble.empty(n, 4, kw["n_dev"])
    abi = ens.abi(t_end=t_end)
    chs.chs_ensemble_init(S.h, chs.params(0.01, 1, **kw), abi, ics, st)
    return ens, abi


def _host(ens):
    return {k: getattr(ens, k).cpu().numpy() for k in ("x", "w", "ld", "dh_max", "n_exec", "status")}


def test_static_scratch_run_matches_work_buffer_run():
    E = 1.0 / 6.0
    y0, y1, p0, p1 = hh_section_box(E)
    ny, npy = 61, 67  # 4087 orbits: several blocks and a ragged tail
    ics_np, st_np = O.grid_ics(E, y0, y1, ny, p0, p1, npy)
    ics = torch.from_numpy(ics_np).cuda()
    st = torch.from_numpy(st_np).cuda()
    t_end = torch.from_numpy(np.random.default_rng(6).integers(0, 50000, ny * npy).astype(np.int64)).cuda()
    S = chs.System(chs.HENON_HEILES, 2)
    kw = dict(n_dev=3, ld_p=0.5, escape_r2=4.0, early_exit=True, seed=9)
    ref, ref_abi = _ensemble(S, ics, st, t_end, kw)
    new, new_abi = _ensemble(S, ics, st, t_end, kw)
    work = chs.compact_work(ny * npy)
    ok = st_np == 0
    step = 0
    for n_steps in (20000, 20000):
        prm = chs.params(0.01, n_steps, step0=step, **kw)
        chs.chs_integrate_compacted(S.h, prm, ref_abi, 1000, work)
        torch.cuda.synchronize()
        # the call itself takes no memory from torch's allocator (nor from any
        # other: the library side names no allocating call, tests/test_abi_cpu.py)
        held = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
        chs.chs_integrate_compacted_static(S.h, prm, new_abi, 1000)
        torch.cuda.synchronize()
        # (Python may free a tensor meanwhile: the counts may drop, never grow)
        assert torch.cuda.memory_allocated() <= held[0] and torch.cuda.memory_reserved() <= held[1]
        step += n_steps
        a, b = _host(ref), _host(new)
        np.testing.assert_array_equal(a["status"], b["status"])
        np.testing.assert_array_equal(a["n_exec"], b["n_exec"])
        assert state_rel_err(b["x"][:, ok], a["x"][:, ok]).max() <= STATE_RTOL
        assert state_rel_err(b["w"][:, ok], a["w"][:, ok]).max() <= STATE_RTOL
        assert ind_err(b["ld"][ok], a["ld"][ok]).max() <= IND_TOL
    # the run did stop orbits early and at their end steps, so the lists were compacted
    assert (a["status"] == chs.ORBIT_EARLY_CHAOTIC).sum() > 100
    assert (a["n_exec"][ok & (a["status"] == 0)] < 40000).sum() > 100


def test_static_scratch_rejects_oversized_ensembles():
    S = chs.System(chs.HENON_HEILES, 2)
    ens = chs.DeviceEnsemble.empty(8, 4, 2)
    abi = ens.abi()
    abi.n_orbits = (1 << 20) + 1  # validated before any launch
    code = chs.load().chs_integrate_compacted_static(S.h, C.byref(chs.params(0.01, 10, n_dev=2)),
                                                     C.byref(abi), 100, None)
    assert code == chs.CHS_E_SIZE
    assert "1048576" in chs.chs_last_error()


def test_static_scratch_bounds_the_chunk_count():
    """Like the work-buffer entry point, at most 100000 chunks per call."""
    S = chs.System(chs.HENON_HEILES, 2)
    ens = chs.DeviceEnsemble.empty(8, 4, 2)
    code = chs.load().chs_integrate_compacted_static(S.h, C.byref(chs.params(0.01, 100001, n_dev=2)),
                                                     C.byref(ens.abi()), 1, None)
    assert code == chs.CHS_E_SIZE
    assert "100000 chunks" in chs.chs_last_error()
