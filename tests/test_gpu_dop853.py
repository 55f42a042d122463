"""Parity of the DOP853 kernels (the paper's DOP 8 and DOP 8(5) solvers) with
the CPU oracle, through the C ABI.

Bars as for the RK4 path: FP64 states within 1e-10 of the orbit's state norm,
indicators within 1e-8 * max(1, |ref|), integers and statuses exact.  The
adaptive runs take floating-point accept/reject decisions on both sides; they
must agree on nearly every orbit (the error estimate is a difference of
nearly equal stage sums, so its summation order moves it by ~1e-8 relative
and a decision can flip only when err sits that close to 1).
"""
import numpy as np
import pytest

import oracle as O
from paper_2507_00622_gb300.inputs import hh_section_box, uniform_vectors
from tests.helpers import IND_TOL, LABEL_AGREE, STATE_RTOL, gpu_run, ind_err, oracle_run, state_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2507_00622_gb300 import chs  # noqa: E402

HH = chs.HENON_HEILES
DP = chs.DOP853


def _grid(E, ny, npy):
    y0, y1, p0, p1 = hh_section_box(E)
    return (E, y0, y1, ny, p0, p1, npy)


# --------------------------------------------------------------------------
# fixed-step DOP853
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k,ld_p", [(0, 0.5), (1, 0.0), (2, 0.5), (4, 0.5), (4, 0.75)])
def test_fixed_step_hh_grid_matches_oracle(k, ld_p):
    """24 x 24 grid at E = 1/8 (a ragged last block of the 32-thread launch),
    h = 0.05, 400 steps (t = 20)."""
    ics, st = O.grid_ics(*_grid(1 / 8, 24, 24))
    kw = dict(dt=0.05, n_steps=400, k=k, ld_p=ld_p, escape_r2=4.0, integrator=DP, seed=3)
    g = gpu_run(HH, 2, ics, st, **kw)
    r = oracle_run(HH, 2, ics, st, **kw)
    np.testing.assert_array_equal(g["status"], r["status"])
    np.testing.assert_array_equal(g["n_exec"], r["n_exec"])
    ok = r["status"] == 0
    assert state_rel_err(g["x"][:, ok], r["x"][:, ok]).max() < STATE_RTOL
    if k:
        assert np.abs(g["w"][:, ok] - r["w"][:, ok]).max() < 1e-9
    if ld_p:
        assert ind_err(g["ld"][ok], r["ld"][ok]).max() < IND_TOL
    assert ind_err(g["dh_max"][ok], r["dh_max"][ok]).max() < 1e-12
    if k >= 2:
        assert ind_err(g["sali"][ok], r["sali"][ok]).max() < 1e-8
        np.testing.assert_array_equal(np.isnan(g["gali"]), np.isnan(r["gali"]))


def test_fixed_step_quartic_k6_matches_oracle():
    rng = np.random.default_rng(11)
    dirs = rng.standard_normal((6, 300))
    E = rng.uniform(1.0, 10.0, 300)
    ics = O.shell_ics(O.system(O.QUARTIC3, 3, eps=0.1), dirs, E)
    kw = dict(dt=0.02, n_steps=300, k=6, ld_p=0.5, sys_params=(0.1,), integrator=DP, seed=9)
    g = gpu_run(chs.QUARTIC3, 3, ics, None, **kw)
    r = oracle_run(chs.QUARTIC3, 3, ics, None, **kw)
    assert state_rel_err(g["x"], r["x"]).max() < STATE_RTOL
    assert np.abs(g["w"] - r["w"]).max() < 1e-9
    assert ind_err(g["ld"], r["ld"]).max() < IND_TOL
    big = np.abs(r["gali"]) > 1e-6
    assert ind_err(g["gali"][big], r["gali"][big]).max() < 1e-8


def test_fixed_step_early_exit_end_steps_and_compaction():
    """Early exit and uneven end steps under DOP853 match the oracle; the
    compacted graph run is bit-identical to the plain run; resuming in chunks
    is bit-identical too."""
    ics, st = O.grid_ics(*_grid(1 / 8, 20, 20))
    t_end = np.random.default_rng(2).integers(50, 8000, ics.shape[1]).astype(np.int64)
    kw = dict(dt=0.05, n_steps=8000, k=2, ld_p=0.5, escape_r2=4.0, integrator=DP, early_exit=True,
              t_end=t_end, sali_threshold=1e-6)
    a = gpu_run(HH, 2, ics, st, **kw)
    b = gpu_run(HH, 2, ics, st, compact_chunk=300, chunks=[3700, 4300], **kw)
    for key in ("x", "w", "ld", "dh_max", "n_exec", "status", "sali", "gali", "label"):
        np.testing.assert_array_equal(a[key], b[key])
    r = oracle_run(HH, 2, ics, st, **kw)
    v = st == 0
    assert (a["status"][v] == chs.ORBIT_EARLY_CHAOTIC).sum() > 20
    assert (a["status"][v] == r["status"][v]).mean() >= LABEL_AGREE
    assert (a["n_exec"][v] == r["n_exec"][v]).mean() >= 0.99
    # states of clearly regular orbits (chaotic ones diverge at these times)
    same = v & (a["n_exec"] == r["n_exec"]) & (r["status"] == 0) & (r["sali"] > 1e-2)
    assert same.sum() > 50
    assert state_rel_err(a["x"][:, same], r["x"][:, same]).max() < 1e-8


def test_static_entry_runs_dop853():
    ics, st = O.grid_ics(*_grid(1 / 8, 16, 16))
    kw = dict(dt=0.05, n_steps=500, k=2, ld_p=0.5, escape_r2=4.0, integrator=DP)
    a = gpu_run(HH, 2, ics, st, **kw)
    S = chs.System(HH, 2)
    n = ics.shape[1]
    ens = chs.DeviceEnsemble.empty(n, 4, 2)
    abi = ens.abi()
    p = chs.params(0.05, 500, n_dev=2, ld_p=0.5, escape_r2=4.0, integrator=DP)
    chs.chs_ensemble_init(S.h, p, abi, torch.from_numpy(ics).cuda(), torch.from_numpy(st).cuda())
    chs.chs_integrate_compacted_static(S.h, p, abi, 200)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ens.x.cpu().numpy(), a["x"])
    np.testing.assert_array_equal(ens.n_exec.cpu().numpy(), a["n_exec"])


def test_lyapunov_small_dop853_matches_oracle():
    ics, st = O.grid_ics(*_grid(1 / 8, 8, 8))
    prm = dict(qr_every=10, sample_every=100)
    S = chs.System(HH, 2)
    n = ics.shape[1]
    lam = torch.empty((4, n), dtype=torch.float64, device="cuda")
    sto = torch.empty(n, dtype=torch.int32, device="cuda")
    chs.chs_lyapunov_spectrum(S.h, chs.params(0.05, 400, integrator=DP, **prm), n,
                              torch.from_numpy(ics).cuda(), torch.from_numpy(st).cuda(), lam, sto)
    torch.cuda.synchronize()
    r, rs = O.lyapunov(O.henon_heiles(), O.params(0.05, 400, integrator=O.DOP853, **prm), ics, st)
    np.testing.assert_array_equal(sto.cpu().numpy(), rs)
    ok = rs == 0
    assert np.abs(lam.cpu().numpy()[:, ok] - r[:, ok]).max() < 1e-8


@pytest.mark.parametrize("N,n,steps", [(4, 37, 120), (8, 13, 120), (16, 9, 100), (32, 5, 60),
                                       (64, 3, 40)])
def test_fput_lyapunov_dop853_matches_oracle(N, n, steps):
    """FPUT chains with DOP853 (ragged orbit groups: n is not a multiple of the
    orbits per block), one orbit with a non-OK initial status."""
    from paper_2507_00622_gb300.inputs import normal_mode_draws
    Q, P = normal_mode_draws(77 + N, N, n)
    ics = O.fput_mode_ics(O.fput(N), Q, P, np.full(n, 0.1 * N))
    st = np.zeros(n, dtype=np.int32)
    st[n // 2] = chs.ORBIT_FORBIDDEN
    prm = dict(qr_every=10, sample_every=20)
    S = chs.System(chs.FPUT, N, (1.0, 0.0, 1.0))
    lam = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
    sto = torch.empty(n, dtype=torch.int32, device="cuda")
    chs.chs_lyapunov_spectrum(S.h, chs.params(0.05, steps, integrator=DP, **prm), n,
                              torch.from_numpy(ics).cuda(), torch.from_numpy(st).cuda(), lam, sto)
    torch.cuda.synchronize()
    r, rs = O.lyapunov(O.fput(N), O.params(0.05, steps, integrator=O.DOP853, **prm), ics, st)
    np.testing.assert_array_equal(sto.cpu().numpy(), rs)
    ok = rs == 0
    g = lam.cpu().numpy()
    assert np.abs(g[:, ok] - r[:, ok]).max() < 1e-8
    assert np.all(np.isnan(g[:, ~ok]))


def test_fput_lyapunov_batch_dop853_equals_separate_calls():
    from paper_2507_00622_gb300.inputs import normal_mode_draws
    jobs, outs, keep = [], [], []
    for N, integ in ((8, DP), (16, chs.RK4), (32, DP)):
        n = 40
        Q, P = normal_mode_draws(5 + N, N, n)
        ics = torch.from_numpy(O.fput_mode_ics(O.fput(N), Q, P, np.full(n, 0.1 * N))).cuda()
        S = chs.System(chs.FPUT, N, (1.0, 0.0, 1.0))
        prm = chs.params(0.05, 100, integrator=integ, qr_every=20)
        lam = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
        sto = torch.empty(n, dtype=torch.int32, device="cuda")
        lam1 = torch.empty_like(lam)
        sto1 = torch.empty_like(sto)
        chs.chs_lyapunov_spectrum(S.h, prm, n, ics, None, lam1, sto1)
        jobs.append((S.h, prm, n, ics, None, lam, sto))
        outs.append((lam, sto, lam1, sto1))
        keep.append(S)
    chs.chs_lyapunov_batch(jobs)
    torch.cuda.synchronize()
    for lam, sto, lam1, sto1 in outs:
        assert torch.equal(lam, lam1) and torch.equal(sto, sto1)


def test_dop853_argument_checks():
    S = chs.System(HH, 2)
    ens = chs.DeviceEnsemble.empty(4, 4, 2, vec_fp32=True)
    p = chs.params(0.05, 10, n_dev=2, vec_precision=chs.VEC_FP32, integrator=DP)
    with pytest.raises(chs.ChsError) as e:
        chs.chs_integrate_batch(S.h, p, ens.abi())
    assert e.value.code == chs.CHS_E_UNSUPPORTED
    with pytest.raises(chs.ChsError) as e:
        chs.chs_integrate_batch(S.h, chs.params(0.05, 10, n_dev=2, integrator=1), ens.abi())
    assert e.value.code == chs.CHS_E_INVALID
    e64 = chs.DeviceEnsemble.empty(4, 4, 2)
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    h = torch.full((4,), 0.1, dtype=torch.float64, device="cuda")
    ad = chs.Adaptive(10.0, 1e-9, 1e-9, 0.0)
    with pytest.raises(chs.ChsError) as e:
        chs.chs_integrate_adaptive(S.h, chs.params(0.05, 10, n_dev=2), ad, e64.abi(), t, h)
    assert e.value.code == chs.CHS_E_INVALID
    te = torch.full((4,), 5, dtype=torch.int64, device="cuda")
    with pytest.raises(chs.ChsError) as e:
        chs.chs_integrate_adaptive(S.h, chs.params(0.05, 10, n_dev=2, integrator=DP), ad,
                                   e64.abi(t_end=te), t, h)
    assert e.value.code == chs.CHS_E_INVALID


# --------------------------------------------------------------------------
# adaptive DOP 8(5)
# --------------------------------------------------------------------------

def _gpu_adaptive(model, n_dof, ics, st, *, k, ld_p, h_first, t_final, rtol, atol, calls,
                  sys_params=(), seed=1, escape_r2=0.0, t0=None):
    """Runs `calls` = [(n_steps, t_final), ...] of chs_integrate_adaptive."""
    S = chs.System(model, n_dof, sys_params)
    n = ics.shape[1]
    ens = chs.DeviceEnsemble.empty(n, S.d, k)
    abi = ens.abi(with_ld=ld_p > 0)
    kw = dict(n_dev=k, ld_p=ld_p, seed=seed, escape_r2=escape_r2, integrator=DP)
    chs.chs_ensemble_init(S.h, chs.params(h_first, 1, **kw), abi, torch.from_numpy(ics).cuda(),
                          None if st is None else torch.from_numpy(st).cuda())
    t = torch.zeros(n, dtype=torch.float64, device="cuda") if t0 is None else \
        torch.from_numpy(np.ascontiguousarray(t0)).cuda()
    h = torch.full((n,), h_first, dtype=torch.float64, device="cuda")
    el = torch.zeros(n, dtype=torch.float64, device="cuda")
    em = torch.zeros(n, dtype=torch.float64, device="cuda")
    nr = torch.zeros(n, dtype=torch.int64, device="cuda")
    for n_steps, tf in calls:
        chs.chs_integrate_adaptive(S.h, chs.params(h_first, n_steps, **kw),
                                   chs.Adaptive(tf, rtol, atol, 0.0), abi, t, h, el, em, nr)
    torch.cuda.synchronize()
    return dict(x=ens.x.cpu().numpy(), w=ens.w.cpu().numpy(), ld=ens.ld.cpu().numpy(),
                n_exec=ens.n_exec.cpu().numpy(), status=ens.status.cpu().numpy(),
                t=t.cpu().numpy(), h=h.cpu().numpy(), err_last=el.cpu().numpy(),
                err_max=em.cpu().numpy(), n_rej=nr.cpu().numpy(),
                dh_max=ens.dh_max.cpu().numpy())


def _oracle_adaptive(model, n_dof, ics, st, *, k, ld_p, h_first, t_final, rtol, atol,
                     sys_params=(), seed=1, escape_r2=0.0):
    from tests.helpers import oracle_system
    S = oracle_system(model, n_dof, sys_params)
    prm = O.params(h_first, 10**9, n_dev=k, ld_p=ld_p, escape_r2=escape_r2, integrator=O.DOP853)
    e = O.Ensemble(S, prm, ics, st, seed=seed)
    e.integrate_adaptive(prm, t_final, rtol, atol)
    return e


@pytest.mark.parametrize("tol,k", [(1e-10, 2), (1e-7, 4)])
def test_adaptive_hh_grid_matches_oracle(tol, k):
    ics, st = O.grid_ics(*_grid(1 / 8, 20, 20))
    kw = dict(k=k, ld_p=0.5, h_first=0.01, t_final=30.0, rtol=tol, atol=tol, escape_r2=4.0, seed=5)
    g = _gpu_adaptive(HH, 2, ics, st, calls=[(10**9, 30.0)], **kw)
    r = _oracle_adaptive(HH, 2, ics, st, **kw)
    v = st == 0
    np.testing.assert_array_equal(g["status"], r.status)
    assert np.all(g["t"][v] == 30.0)
    same = v & (g["n_exec"] == r.n_exec) & (g["n_rej"] == r.n_rej)
    assert same.sum() >= 0.99 * v.sum()
    assert state_rel_err(g["x"][:, same], r.x[:, same]).max() < STATE_RTOL
    assert np.abs(g["w"][:, same] - r.w[:, same]).max() < 1e-9
    # The LD is not in the error norm and its integrand sum_i |f_i|^(1/2) is not
    # smooth, so its quadrature error follows the step sequence closely: in the
    # oracle alone, moving the tolerance by 1e-7 relative (the step sizes by
    # ~1e-8) moves the LD by up to 4e-6 relative while the states move by 3e-14.
    # Step sizes here agree to ~1e-8, so the LD is held to 1e-5.
    assert (np.abs(g["ld"][same] - r.ld[same]) / r.ld[same]).max() < 1e-5
    # the last step is clipped to t_final; its error is tiny and mostly rounding
    # of the stage sums, so only the largest error (steps with err near 1) is
    # held tightly
    np.testing.assert_allclose(g["err_last"][same], r.err_last[same], rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(g["err_max"][same], r.err_max[same], rtol=1e-6, atol=0)
    # the next step size after the clipped last step follows err_last^(-1/8)
    m = same & (r.err_last > 1e-3)
    np.testing.assert_allclose(g["h"][m], r.h[m], rtol=1e-5, atol=0)
    assert np.all(g["err_last"][v] < 1.0)


@pytest.mark.parametrize("tol,steps", [(1e-10, 300), (1e-7, 60)])
def test_adaptive_per_step_error_on_unclipped_steps(tol, steps):
    """The error of each integration step (Sec. Functionalities) on steps that
    are never clipped: t_final lies out of reach, so every orbit stops after
    n_steps accepted steps of the controller's own choosing.  There err_last
    (the scaled error of the last accepted step) and the next step size are
    compared with the oracle where err_last > 1e-3, to 1e-6 relative on every
    orbit whose err_last the oracle itself reproduces to 1e-7 when its initial
    states move by one ulp (two such runs), and elsewhere to 4x the larger of
    that one-ulp spread and 1e-6.  (At tol = 1e-10 the one-ulp spread stays below
    3e-7 after 300 steps; at tol = 1e-7 the steps are ~10x longer and after 60 of
    them it reaches ~3e-6 on about 1 % of the orbits.  With a last step clipped
    to t_final, err_last is the error of a short step, tiny and dominated by
    rounding: test_adaptive_hh_grid_matches_oracle.)"""
    ics, st = O.grid_ics(*_grid(1 / 8, 20, 20))
    kw = dict(k=2, ld_p=0.5, h_first=0.01, t_final=1e9, rtol=tol, atol=tol, escape_r2=4.0, seed=5)
    g = _gpu_adaptive(HH, 2, ics, st, calls=[(steps, 1e9)], **kw)
    prm = O.params(0.01, steps, n_dev=2, ld_p=0.5, escape_r2=4.0, integrator=O.DOP853)
    runs = []
    rng = np.random.default_rng(0)
    for k in range(3):
        x = ics if k == 0 else np.nextafter(ics, ics + rng.choice([-1.0, 1.0], ics.shape))
        e = O.Ensemble(O.henon_heiles(), prm, x, st, seed=5)
        e.integrate_adaptive(prm, 1e9, tol, tol)
        runs.append(e)
    r = runs[0]
    v = st == 0
    np.testing.assert_array_equal(g["status"], r.status)
    assert np.all(g["n_exec"][v] == steps) and np.all(r.n_exec[v] == steps)
    same = v & (g["n_rej"] == r.n_rej) & (runs[1].n_rej == r.n_rej) & (runs[2].n_rej == r.n_rej)
    assert same.sum() >= 0.98 * v.sum()
    m = same & (r.err_last > 1e-3)
    assert m.sum() >= 0.9 * same.sum()
    for key in ("err_last", "h"):
        ref = getattr(r, key)[m]
        spread = np.maximum(*[np.abs(getattr(q, key)[m] - ref) / ref for q in runs[1:]])
        err = np.abs(g[key][m] - ref) / ref
        tight = spread <= 1e-7
        assert tight.mean() >= 0.5
        assert err[tight].max() <= 1e-6, (key, err[tight].max())
        assert err.max() <= 4.0 * max(spread.max(), 1e-6), (key, err.max(), spread.max())
    np.testing.assert_allclose(g["t"][same], r.t[same], rtol=1e-7, atol=0)


def test_adaptive_with_step_cap_matches_oracle_ld():
    """With h_max small and a loose tolerance every step is h_max (the last one
    clipped to t_final): both sides take the same step sequence, and the LD
    agrees to the fixed-step bar."""
    ics, st = O.grid_ics(*_grid(1 / 8, 16, 16))
    n = ics.shape[1]
    S = chs.System(HH, 2)
    ens = chs.DeviceEnsemble.empty(n, 4, 2)
    abi = ens.abi()
    kw = dict(n_dev=2, ld_p=0.5, escape_r2=4.0, integrator=DP)
    chs.chs_ensemble_init(S.h, chs.params(0.05, 1, **kw), abi, torch.from_numpy(ics).cuda(),
                          torch.from_numpy(st).cuda())
    t = torch.zeros(n, dtype=torch.float64, device="cuda")
    h = torch.full((n,), 0.05, dtype=torch.float64, device="cuda")
    chs.chs_integrate_adaptive(S.h, chs.params(0.05, 10**6, **kw), chs.Adaptive(20.01, 1e-3, 1e-3, 0.05),
                               abi, t, h)
    torch.cuda.synchronize()
    prm = O.params(0.05, 10**6, n_dev=2, ld_p=0.5, escape_r2=4.0, integrator=O.DOP853)
    e = O.Ensemble(O.henon_heiles(), prm, ics, st)
    e.integrate_adaptive(prm, 20.01, 1e-3, 1e-3, h_max=0.05)
    v = st == 0
    np.testing.assert_array_equal(ens.n_exec.cpu().numpy(), e.n_exec)
    assert np.all(e.n_exec[v] == 401)
    assert state_rel_err(ens.x.cpu().numpy()[:, v], e.x[:, v]).max() < STATE_RTOL
    assert ind_err(ens.ld.cpu().numpy()[v], e.ld[v]).max() < IND_TOL


def test_adaptive_resumed_in_calls_is_bit_identical():
    """A call ends only after an accepted step, so splitting a run into calls of
    a few accepted steps (and intermediate t_final values) changes nothing."""
    ics, st = O.grid_ics(*_grid(1 / 8, 12, 12))
    kw = dict(k=2, ld_p=0.5, h_first=0.02, t_final=15.0, rtol=1e-9, atol=1e-9, escape_r2=4.0)
    a = _gpu_adaptive(HH, 2, ics, st, calls=[(10**9, 15.0)], **kw)
    b = _gpu_adaptive(HH, 2, ics, st, calls=[(7, 15.0)] * 5 + [(10**9, 15.0)], **kw)
    for key in ("x", "w", "ld", "n_exec", "status", "t", "h", "err_last", "err_max", "n_rej"):
        np.testing.assert_array_equal(a[key], b[key])


def test_adaptive_quartic_and_step_fail():
    rng = np.random.default_rng(4)
    dirs = rng.standard_normal((6, 100))
    E = rng.uniform(1.0, 10.0, 100)
    ics = O.shell_ics(O.system(O.QUARTIC3, 3, eps=0.1), dirs, E)
    kw = dict(k=6, ld_p=0.5, h_first=0.05, t_final=10.0, rtol=1e-9, atol=1e-9, sys_params=(0.1,))
    g = _gpu_adaptive(chs.QUARTIC3, 3, ics, None, calls=[(10**9, 10.0)], **kw)
    r = _oracle_adaptive(chs.QUARTIC3, 3, ics, None, **kw)
    same = (g["n_exec"] == r.n_exec) & (g["n_rej"] == r.n_rej)
    assert same.mean() >= 0.99
    assert state_rel_err(g["x"][:, same], r.x[:, same]).max() < STATE_RTOL
    # orbits that start at t = 1e20 cannot take a step: STEP_FAIL, state untouched
    t0 = np.zeros(100)
    t0[::7] = 1e20
    f = _gpu_adaptive(chs.QUARTIC3, 3, ics, None, calls=[(200, 2e20)], t0=t0, **kw)
    bad = t0 > 0
    assert np.all(f["status"][bad] == chs.ORBIT_STEP_FAIL)
    np.testing.assert_array_equal(f["x"][:, bad], ics[:, bad])
    assert np.all(f["n_exec"][bad] == 0) and np.all(f["n_rej"][bad] >= 1)


# --------------------------------------------------------------------------
# Lyapunov spectra with adaptive DOP 8(5)
# --------------------------------------------------------------------------

def _gpu_lyap_adaptive(model, N, ics, st, params, T, tol, sys_params=()):
    S = chs.System(model, N, sys_params)
    n = ics.shape[1]
    lam = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
    sto = torch.empty(n, dtype=torch.int32, device="cuda")
    acc = torch.empty(n, dtype=torch.int64, device="cuda")
    rej = torch.empty(n, dtype=torch.int64, device="cuda")
    chs.chs_lyapunov_adaptive(S.h, params, chs.Adaptive(T, tol, tol, 0.0), n,
                              torch.from_numpy(np.ascontiguousarray(ics)).cuda(),
                              None if st is None else torch.from_numpy(st).cuda(), lam, sto, acc, rej)
    torch.cuda.synchronize()
    return lam.cpu().numpy(), sto.cpu().numpy(), acc.cpu().numpy(), rej.cpu().numpy()


def test_adaptive_lyapunov_hh_matches_oracle():
    ics, st = O.grid_ics(*_grid(1 / 8, 12, 12))
    prm = chs.params(0.01, 10**6, qr_every=10, integrator=DP)
    g, gs, ga, gr = _gpu_lyap_adaptive(HH, 2, ics, st, prm, 20.0, 1e-10)
    r, rs, ra, rr = O.lyapunov_adaptive(O.henon_heiles(), O.params(0.01, 10**6, qr_every=10), ics,
                                        20.0, 1e-10, 1e-10, ic_status=st)
    np.testing.assert_array_equal(gs, rs)
    ok = rs == 0
    same = ok & (ga == ra) & (gr == rr)
    assert same.sum() >= 0.99 * ok.sum()
    assert np.abs(g[:, same] - r[:, same]).max() < 1e-8
    assert np.all(np.isnan(g[:, ~ok]))


@pytest.mark.parametrize("N,n", [(4, 37), (8, 13), (16, 9), (32, 5), (64, 3)])
def test_adaptive_lyapunov_fput_matches_oracle(N, n):
    from paper_2507_00622_gb300.inputs import normal_mode_draws
    Q, P = normal_mode_draws(91 + N, N, n)
    ics = O.fput_mode_ics(O.fput(N), Q, P, np.full(n, 0.1 * N))
    st = np.zeros(n, dtype=np.int32)
    st[-1] = chs.ORBIT_FORBIDDEN
    T = 6.0 if N == 64 else 10.0
    prm = chs.params(0.05, 10**6, qr_every=10, integrator=DP)
    g, gs, ga, gr = _gpu_lyap_adaptive(chs.FPUT, N, ics, st, prm, T, 1e-9, (1.0, 0.0, 1.0))
    r, rs, ra, rr = O.lyapunov_adaptive(O.fput(N), O.params(0.05, 10**6, qr_every=10), ics, T,
                                        1e-9, 1e-9, ic_status=st)
    np.testing.assert_array_equal(gs, rs)
    ok = rs == 0
    same = ok & (ga == ra) & (gr == rr)
    assert same.sum() >= ok.sum() - 1
    assert np.abs(g[:, same] - r[:, same]).max() < 1e-8
    assert np.all(np.isnan(g[:, ~ok]))
    # a step budget shorter than the run: STEP_FAIL with NaN exponents
    g2, gs2, ga2, _ = _gpu_lyap_adaptive(chs.FPUT, N, ics, None,
                                         chs.params(0.05, 3, qr_every=10, integrator=DP), T, 1e-9,
                                         (1.0, 0.0, 1.0))
    assert np.all(gs2 == chs.ORBIT_STEP_FAIL) and np.all(ga2 == 3) and np.all(np.isnan(g2))
