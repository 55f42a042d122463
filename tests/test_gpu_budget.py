"""The clock budget (chs_params.clock_budget): a call whose orbits run past it
stops them at the next health check with status STEP_BUDGET, without waiting or
trapping, and an ample budget changes nothing.

A budget of one clock cycle is spent before the first health check (step 10
here), so every running orbit must stop exactly there: its state, step count and
largest energy error equal those of a plain 10-step run, bit for bit.
"""
import numpy as np
import pytest

import oracle as O
from paper_2507_00622_gb300.inputs import hh_section_box, normal_mode_draws
from tests.helpers import gpu_run

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2507_00622_gb300 import chs  # noqa: E402

HH = chs.HENON_HEILES
TINY, AMPLE = 1, 1 << 62
CHECK = 10


def _grid():
    y0, y1, p0, p1 = hh_section_box(1 / 8)
    return O.grid_ics(1 / 8, y0, y1, 13, p0, p1, 11)


def _run(ics, st, budget, n_steps, **kw):
    return gpu_run(HH, 2, ics, st, dt=0.01, n_steps=n_steps, k=2, ld_p=0.5, escape_r2=4.0,
                   sample_every=CHECK, clock_budget=budget, **kw)


KEYS = ("x", "w", "ld", "dh_max", "n_exec")


@pytest.mark.parametrize("mode", ["rk4", "fp32", "dop853", "persistent", "compacted"])
def test_tiny_budget_stops_at_the_first_health_check(mode):
    ics, st = _grid()
    kw = {"rk4": {}, "fp32": dict(vec_fp32=True), "dop853": dict(integrator=chs.DOP853),
          "persistent": dict(persistent=True), "compacted": dict(compact_chunk=250)}[mode]
    out = _run(ics, st, TINY, 1000, **kw)
    ref = _run(ics, st, 0, CHECK, **kw)
    v = st == 0
    assert v.sum() > 50
    assert np.all(out["status"][v] == chs.ORBIT_STEP_BUDGET)
    assert np.all(out["status"][~v] == chs.ORBIT_FORBIDDEN)
    assert np.all(out["label"][v] == -1)
    for key in KEYS:
        np.testing.assert_array_equal(out[key][..., v], ref[key][..., v])


@pytest.mark.parametrize("mode", ["rk4", "fp32", "dop853", "persistent"])
def test_ample_budget_changes_nothing(mode):
    ics, st = _grid()
    kw = {"rk4": {}, "fp32": dict(vec_fp32=True), "dop853": dict(integrator=chs.DOP853),
          "persistent": dict(persistent=True)}[mode]
    a = _run(ics, st, AMPLE, 700, **kw)
    b = _run(ics, st, 0, 700, **kw)
    for key in KEYS + ("status", "sali", "gali", "label"):
        np.testing.assert_array_equal(a[key], b[key])


def test_tiny_budget_adaptive():
    ics, st = _grid()
    v = st == 0
    res = {}
    for budget in (TINY, 0):
        S = chs.System(HH, 2)
        n = ics.shape[1]
        ens = chs.DeviceEnsemble.empty(n, 4, 2)
        abi = ens.abi()
        kw = dict(n_dev=2, ld_p=0.5, escape_r2=4.0, sample_every=CHECK, integrator=chs.DOP853,
                  clock_budget=budget)
        chs.chs_ensemble_init(S.h, chs.params(0.01, 1, **kw), abi, torch.from_numpy(ics).cuda(),
                              torch.from_numpy(st).cuda())
        t = torch.zeros(n, dtype=torch.float64, device="cuda")
        h = torch.full((n,), 0.01, dtype=torch.float64, device="cuda")
        steps = 1000 if budget else CHECK
        chs.chs_integrate_adaptive(S.h, chs.params(0.01, steps, **kw), chs.Adaptive(100.0, 1e-9, 1e-9, 0.0),
                                   abi, t, h)
        torch.cuda.synchronize()
        res[budget] = (ens.x.cpu().numpy(), ens.n_exec.cpu().numpy(), ens.status.cpu().numpy(), t.cpu().numpy())
        S.close()
    x, ne, sts, t = res[TINY]
    assert np.all(sts[v] == chs.ORBIT_STEP_BUDGET) and np.all(ne[v] == CHECK)
    np.testing.assert_array_equal(x[:, v], res[0][0][:, v])
    np.testing.assert_array_equal(t[v], res[0][3][v])


@pytest.mark.parametrize("integ,adaptive", [(chs.RK4, False), (chs.DOP853, False), (chs.DOP853, True)])
def test_tiny_budget_fput_ensembles(integ, adaptive):
    N, n, k = 8, 37, 2
    Q, P = normal_mode_draws(5, N, n)
    ics = torch.from_numpy(O.fput_mode_ics(O.fput(N), Q, P, np.full(n, 0.1 * N))).cuda()
    out = {}
    for budget in (TINY, 0):
        S = chs.System(chs.FPUT, N, (1.0, 0.0, 1.0))
        ens = chs.DeviceEnsemble.empty(n, 2 * N, k)
        abi = ens.abi(with_ld=False)
        kw = dict(n_dev=k, sample_every=CHECK, integrator=integ, seed=3, clock_budget=budget)
        chs.chs_ensemble_init(S.h, chs.params(0.05, 1, **kw), abi, ics)
        steps = 1000 if budget else CHECK
        if adaptive:
            t = torch.zeros(n, dtype=torch.float64, device="cuda")
            h = torch.full((n,), 0.05, dtype=torch.float64, device="cuda")
            chs.chs_integrate_adaptive(S.h, chs.params(0.05, steps, **kw), chs.Adaptive(1e3, 1e-9, 1e-9, 0.0),
                                       abi, t, h)
        else:
            chs.chs_integrate_batch(S.h, chs.params(0.05, steps, **kw), abi)
        torch.cuda.synchronize()
        out[budget] = (ens.x.cpu().numpy(), ens.w.cpu().numpy(), ens.n_exec.cpu().numpy(),
                       ens.status.cpu().numpy())
        S.close()
    x, w, ne, sts = out[TINY]
    assert np.all(sts == chs.ORBIT_STEP_BUDGET) and np.all(ne == CHECK)
    np.testing.assert_array_equal(x, out[0][0])
    np.testing.assert_array_equal(w, out[0][1])


@pytest.mark.parametrize("model,N,integ,adaptive", [
    (HH, 2, chs.RK4, False), (HH, 2, chs.DOP853, False), (HH, 2, chs.DOP853, True),
    (chs.FPUT, 4, chs.RK4, False), (chs.FPUT, 8, chs.RK4, False), (chs.FPUT, 16, chs.RK4, False),
    (chs.FPUT, 64, chs.RK4, False),
    (chs.FPUT, 8, chs.DOP853, False), (chs.FPUT, 8, chs.DOP853, True), (chs.FPUT, 64, chs.DOP853, False)])
def test_tiny_budget_lyapunov(model, N, integ, adaptive):
    """Lyapunov runs stop at their first check with NaN exponents; an ample
    budget gives the exponents of a run without one."""
    n = 21
    if model == HH:
        ics, st = _grid()
        ics = np.ascontiguousarray(ics[:, st == 0][:, :n])
        sp, h = (), 0.01
    else:
        Q, P = normal_mode_draws(9, N, n)
        ics = O.fput_mode_ics(O.fput(N), Q, P, np.full(n, 0.1 * N))
        sp, h = (1.0, 0.0, 1.0), 0.05
    S = chs.System(model, N, sp)
    ics_t = torch.from_numpy(ics).cuda()
    res = {}
    for budget in (TINY, AMPLE, 0):
        lam = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
        sto = torch.empty(n, dtype=torch.int32, device="cuda")
        prm = chs.params(h, 400, qr_every=10, sample_every=CHECK, integrator=integ, clock_budget=budget)
        if adaptive:
            # t_final long enough for more than sample_every accepted steps
            chs.chs_lyapunov_adaptive(S.h, prm, chs.Adaptive(10.0 if model == HH else 5.0, 1e-9, 1e-9, 0.0),
                                      n, ics_t, None, lam, sto)
        else:
            chs.chs_lyapunov_spectrum(S.h, prm, n, ics_t, None, lam, sto)
        torch.cuda.synchronize()
        res[budget] = (lam.cpu().numpy(), sto.cpu().numpy())
    lam, sto = res[TINY]
    assert np.all(sto == chs.ORBIT_STEP_BUDGET) and np.all(np.isnan(lam))
    np.testing.assert_array_equal(res[AMPLE][0], res[0][0])
    assert np.all(res[0][1] == chs.ORBIT_OK)
    S.close()


def test_negative_budget_is_rejected():
    ics, st = _grid()
    with pytest.raises(chs.ChsError) as e:
        _run(ics, st, -5, 100)
    assert e.value.code == chs.CHS_E_INVALID
