"""Parity of the FPUT ensemble kernels (k <= 6 deviation vectors on FPUT-beta
chains, RK4 / DOP853 fixed steps and adaptive DOP 8(5); the FPU workload of
Sec. Examples: GALI_4 of random normal-mode orbits) with the CPU oracle,
through the C ABI.

Bars as for the other ensembles: FP64 states within 1e-10 of the orbit's
state norm, vectors within 1e-9, indicators within 1e-8 * max(1, |ref|),
statuses, step counts and labels exact.  Inputs: normal-mode initial
conditions at energy density 0.1 (seeded draws), ragged orbit counts, one
FORBIDDEN orbit.
"""
import numpy as np
import pytest

import oracle as O
from paper_2507_00622_gb300.inputs import normal_mode_draws
from tests.helpers import IND_TOL, STATE_RTOL, gpu_run, ind_err, oracle_run, state_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2507_00622_gb300 import chs  # noqa: E402

FPUT = chs.FPUT
SP = (1.0, 0.0, 1.0)
RK4, DP = chs.RK4, chs.DOP853


def _ics(N, n, seed, density=0.1):
    Q, P = normal_mode_draws(seed, N, n)
    E = density * N if np.isscalar(density) else np.asarray(density) * N
    return O.fput_mode_ics(O.fput(N), Q, P, np.broadcast_to(E, (n,)).copy())


def _compare(g, r, v, k, w_tol=1e-9):
    np.testing.assert_array_equal(g["status"], r["status"])
    np.testing.assert_array_equal(g["n_exec"], r["n_exec"])
    assert state_rel_err(g["x"][:, v], r["x"][:, v]).max() < STATE_RTOL
    if k > 0:
        assert np.abs(g["w"][:, v] - r["w"][:, v]).max() < w_tol
    assert np.abs(g["dh_max"][v] - r["dh_max"][v]).max() < 1e-12
    if k >= 2:
        assert ind_err(g["sali"][v], r["sali"][v]).max() < IND_TOL
        assert ind_err(g["gali"][:, v], r["gali"][:, v]).max() < IND_TOL
        np.testing.assert_array_equal(g["label"], r["label"])


@pytest.mark.parametrize("N,n,k,integ,steps", [
    (4, 37, 4, RK4, 200), (4, 19, 6, DP, 120), (8, 21, 6, DP, 150), (8, 17, 1, RK4, 100),
    (16, 11, 4, RK4, 150), (16, 9, 2, DP, 120), (32, 7, 4, DP, 100), (32, 5, 0, RK4, 100),
    (64, 5, 4, DP, 60), (64, 3, 6, RK4, 80)])
def test_fput_ensemble_matches_oracle(N, n, k, integ, steps):
    ics = _ics(N, n, 100 + N)
    st = np.zeros(n, dtype=np.int32)
    st[n // 3] = chs.ORBIT_FORBIDDEN
    kw = dict(dt=0.05, n_steps=steps, k=k, ld_p=0.0, sample_every=20, sys_params=SP,
              integrator=integ, seed=3)
    g = gpu_run(FPUT, N, ics, st, **kw)
    r = oracle_run(FPUT, N, ics, st, **kw)
    v = st == 0
    _compare(g, r, v, k)
    # H0 from the initial state, and the untouched FORBIDDEN orbit
    h0 = np.array([O.energy(O.fput(N), ics[:, o]) for o in range(n)])
    np.testing.assert_allclose(g["h0"][v], h0[v], rtol=1e-14)
    assert np.isnan(g["h0"][~v]).all()
    np.testing.assert_array_equal(g["x"][:, ~v], ics[:, ~v])
    if k >= 2:
        assert np.isnan(g["sali"][~v]).all() and np.isnan(g["gali"][:, ~v]).all()


def test_fput_ensemble_without_renorm_and_from_given_vectors():
    N, n, k = 8, 24, 3
    ics = _ics(N, n, 11)
    rng = np.random.default_rng(12)
    w_in = rng.standard_normal((k * 2 * N, n))
    for renorm in (False, True):
        kw = dict(dt=0.05, n_steps=80, k=k, ld_p=0.0, sample_every=40, sys_params=SP,
                  integrator=DP, renorm=renorm, w_in=w_in)
        g = gpu_run(FPUT, N, ics, None, **kw)
        r = oracle_run(FPUT, N, ics, None, **kw)
        v = np.ones(n, dtype=bool)
        scale = np.abs(r["w"]).max()
        assert np.abs(g["w"] - r["w"]).max() < 1e-9 * max(1.0, scale)
        _compare(g, r, v, k, w_tol=1e-9 * max(1.0, scale))


def test_fput_ensemble_seeded_vectors_bit_exact():
    """The seeded unit vectors (SplitMix64, normalised, again with renorm) equal
    the oracle's bit for bit, with and without renorm."""
    N, n, k = 16, 50, 4
    ics = _ics(N, n, 21)
    for renorm in (False, True):
        S = chs.System(FPUT, N, SP)
        ens = chs.DeviceEnsemble.empty(n, S.d, k)
        p = chs.params(0.05, 1, n_dev=k, ld_p=0.0, renorm=renorm, seed=99)
        chs.chs_ensemble_init(S.h, p, ens.abi(with_ld=False), torch.from_numpy(ics).cuda())
        torch.cuda.synchronize()
        e = O.Ensemble(O.fput(N), O.params(0.05, 1, n_dev=k, renorm=renorm), ics, seed=99)
        np.testing.assert_array_equal(ens.w.cpu().numpy(), e.w)
        np.testing.assert_array_equal(ens.x.cpu().numpy(), ics)
        S.close()


def test_fput_ensemble_chunks_are_bit_identical():
    N, n, k = 16, 12, 4
    ics = _ics(N, n, 31)
    kw = dict(dt=0.05, k=k, ld_p=0.0, sample_every=10, sys_params=SP, integrator=DP)
    a = gpu_run(FPUT, N, ics, None, n_steps=150, **kw)
    b = gpu_run(FPUT, N, ics, None, n_steps=150, chunks=[33, 70, 47], **kw)
    for key in ("x", "w", "dh_max", "n_exec", "status", "sali", "gali"):
        np.testing.assert_array_equal(a[key], b[key])


def test_fput_ensemble_escape_and_end_steps():
    N, n, k, steps = 8, 64, 2, 200
    ics = _ics(N, n, 41, density=np.linspace(0.05, 0.6, n))
    r2 = (ics[:N] ** 2).sum(axis=0)
    escape_r2 = float(np.median(r2)) * 1.5
    t_end = np.random.default_rng(42).integers(40, steps + 30, n).astype(np.int64)
    kw = dict(dt=0.05, n_steps=steps, k=k, ld_p=0.0, sample_every=25, sys_params=SP,
              integrator=RK4, escape_r2=escape_r2, t_end=t_end)
    g = gpu_run(FPUT, N, ics, None, **kw)
    r = oracle_run(FPUT, N, ics, None, **kw)
    v = r["status"] == 0
    _compare(g, r, np.ones(n, dtype=bool), k)
    esc = r["status"] == chs.ORBIT_ESCAPED
    assert esc.any() and v.any()
    assert (r["n_exec"][v] < steps).any()  # some orbits stopped at their t_end
    np.testing.assert_array_equal(g["label"][esc], 2)


def test_fput_ensemble_energy_drift_nonfinite_and_early_exit():
    N, n, k, steps = 16, 40, 2, 160
    ics = _ics(N, n, 51)
    # one orbit at a huge energy leaves RK4's stability region: overflow, then
    # NaN, frozen at the next health check
    big = _ics(N, 1, 52, density=1e6)
    ics[:, 5] = big[:, 0]
    base = dict(dt=0.1, n_steps=steps, k=k, ld_p=0.0, sample_every=20, sys_params=SP, integrator=RK4)
    pre = oracle_run(FPUT, N, ics, None, **base)
    ok = pre["status"] == 0
    assert pre["status"][5] == chs.ORBIT_NONFINITE
    # thresholds halfway between two neighbouring values of the plain run, far
    # from any single orbit's value in units of rounding
    dh = np.sort(pre["dh_max"][ok])
    dh_limit = float(0.5 * (dh[len(dh) // 2] + dh[len(dh) // 2 + 1]))
    g = gpu_run(FPUT, N, ics, None, dh_limit=dh_limit, **base)
    r = oracle_run(FPUT, N, ics, None, dh_limit=dh_limit, **base)
    fin = r["status"] != chs.ORBIT_NONFINITE
    np.testing.assert_array_equal(g["status"], r["status"])
    np.testing.assert_array_equal(g["n_exec"], r["n_exec"])
    assert (r["status"] == chs.ORBIT_ENERGY_DRIFT).sum() >= 5
    assert state_rel_err(g["x"][:, fin], r["x"][:, fin]).max() < STATE_RTOL
    # early exit: SALI below a (large) threshold at a health check
    sa = np.sort(pre["sali"][ok])
    thr = float(0.5 * (sa[len(sa) // 2] + sa[len(sa) // 2 + 1]))
    kw = dict(base, early_exit=True, sali_threshold=thr)
    g = gpu_run(FPUT, N, ics, None, **kw)
    r = oracle_run(FPUT, N, ics, None, **kw)
    np.testing.assert_array_equal(g["status"], r["status"])
    np.testing.assert_array_equal(g["n_exec"], r["n_exec"])
    ec = r["status"] == chs.ORBIT_EARLY_CHAOTIC
    assert ec.any()
    np.testing.assert_array_equal(g["label"][ec], 1)


def _gpu_adaptive(N, ics, *, k, h_first, t_final, tol, calls):
    S = chs.System(FPUT, N, SP)
    n = ics.shape[1]
    ens = chs.DeviceEnsemble.empty(n, S.d, k)
    abi = ens.abi(with_ld=False)
    kw = dict(n_dev=k, ld_p=0.0, integrator=DP, sample_every=10)
    chs.chs_ensemble_init(S.h, chs.params(h_first, 1, **kw), abi, torch.from_numpy(ics).cuda())
    t = torch.zeros(n, dtype=torch.float64, device="cuda")
    h = torch.full((n,), h_first, dtype=torch.float64, device="cuda")
    el = torch.zeros(n, dtype=torch.float64, device="cuda")
    em = torch.zeros(n, dtype=torch.float64, device="cuda")
    nr = torch.zeros(n, dtype=torch.int64, device="cuda")
    for n_steps, tf in calls:
        chs.chs_integrate_adaptive(S.h, chs.params(h_first, n_steps, **kw), chs.Adaptive(tf, tol, tol, 0.0),
                                   abi, t, h, el, em, nr)
    gali = torch.empty((max(k - 1, 1), n), dtype=torch.float64, device="cuda")
    if k >= 2:
        chs.chs_indicators(S.h, chs.params(h_first, 0, **kw), abi, 0, 0, None, gali, None, None)
    torch.cuda.synchronize()
    out = dict(x=ens.x.cpu().numpy(), w=ens.w.cpu().numpy(), n_exec=ens.n_exec.cpu().numpy(),
               status=ens.status.cpu().numpy(), t=t.cpu().numpy(), h=h.cpu().numpy(),
               err_max=em.cpu().numpy(), n_rej=nr.cpu().numpy(), dh_max=ens.dh_max.cpu().numpy(),
               gali=gali.cpu().numpy())
    S.close()
    return out


@pytest.mark.parametrize("N,n,k,tol", [(4, 33, 4, 1e-8), (16, 10, 4, 1e-10), (64, 3, 4, 1e-8)])
def test_fput_ensemble_adaptive_matches_oracle(N, n, k, tol):
    """Adaptive DOP 8(5), the FPU timing workload's solver (GALI_4)."""
    ics = _ics(N, n, 61 + N)
    g = _gpu_adaptive(N, ics, k=k, h_first=0.05, t_final=8.0, tol=tol, calls=[(10**9, 8.0)])
    prm = O.params(0.05, 10**9, n_dev=k, integrator=O.DOP853, sample_every=10)
    e = O.Ensemble(O.fput(N), prm, ics)
    e.integrate_adaptive(prm, 8.0, tol, tol)
    np.testing.assert_array_equal(g["status"], e.status)
    assert np.all(g["t"] == 8.0)
    same = (g["n_exec"] == e.n_exec) & (g["n_rej"] == e.n_rej)
    assert same.mean() >= 0.9
    assert state_rel_err(g["x"][:, same], e.x[:, same]).max() < STATE_RTOL
    assert np.abs(g["w"][:, same] - e.w[:, same]).max() < 1e-9
    assert np.abs(g["dh_max"][same] - e.dh_max[same]).max() < 1e-12
    # the error estimate is a sum of stage derivatives that cancels down to the
    # local error (~1e-8 of the state here), so rounding of the stage sums in a
    # different order moves it by ~1e-16 / 1e-10 relative
    np.testing.assert_allclose(g["err_max"][same], e.err_max[same], rtol=2e-5)
    _, gali, _ = e.indicators()
    assert ind_err(g["gali"][:, same], gali[:, same]).max() < IND_TOL


def test_fput_ensemble_adaptive_resumed_is_bit_identical():
    ics = _ics(8, 20, 71)
    kw = dict(k=4, h_first=0.05, t_final=6.0, tol=1e-9)
    a = _gpu_adaptive(8, ics, calls=[(10**9, 6.0)], **kw)
    b = _gpu_adaptive(8, ics, calls=[(9, 6.0)] * 4 + [(10**9, 6.0)], **kw)
    for key in a:
        np.testing.assert_array_equal(a[key], b[key])


def test_fput_ensemble_argument_checks():
    ens = chs.DeviceEnsemble.empty(4, 10, 2)
    S5 = chs.System(FPUT, 5, SP)
    with pytest.raises(chs.ChsError) as e:
        chs.chs_integrate_batch(S5.h, chs.params(0.05, 10, n_dev=2, ld_p=0.0), ens.abi(with_ld=False))
    assert e.value.code == chs.CHS_E_UNSUPPORTED
    S = chs.System(FPUT, 4, SP)
    e8 = chs.DeviceEnsemble.empty(4, 8, 2)
    with pytest.raises(chs.ChsError) as e:
        chs.chs_integrate_batch(S.h, chs.params(0.05, 10, n_dev=2, ld_p=0.5), e8.abi())
    assert e.value.code == chs.CHS_E_UNSUPPORTED
    e32 = chs.DeviceEnsemble.empty(4, 8, 2, vec_fp32=True)
    with pytest.raises(chs.ChsError) as e:
        chs.chs_integrate_batch(S.h, chs.params(0.05, 10, n_dev=2, ld_p=0.0, vec_precision=chs.VEC_FP32),
                                e32.abi(with_ld=False))
    assert e.value.code == chs.CHS_E_UNSUPPORTED
    with pytest.raises(chs.ChsError) as e:
        chs.chs_integrate_batch(S.h, chs.params(0.05, 10, n_dev=7, ld_p=0.0), e8.abi(with_ld=False))
    assert e.value.code == chs.CHS_E_INVALID
    with pytest.raises(chs.ChsError) as e:
        chs.chs_integrate_compacted(S.h, chs.params(0.05, 10, n_dev=2, ld_p=0.0), e8.abi(with_ld=False), 5,
                                    chs.compact_work(4))
    assert e.value.code == chs.CHS_E_UNSUPPORTED
    ldi = torch.empty((2, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(chs.ChsError) as e:
        chs.chs_indicators(S.h, chs.params(0.05, 0, n_dev=2, ld_p=0.0), e8.abi(with_ld=False), 2, 2,
                           None, None, ldi, None)
    assert e.value.code == chs.CHS_E_UNSUPPORTED
    S.close()
    S5.close()


@pytest.mark.parametrize("integ", [RK4, DP])
def test_fput_ensemble_linear_chain_matches_matrix_exponential(integ):
    """alpha = beta = 0: state and renormalised vectors equal expm(A t) applied to
    the start (A = [[0, I], [-K, 0]], K the fixed-end Laplacian), up to the
    integrator's error; SALI and GALI_2..4 equal those of the exact unit vectors."""
    from scipy.linalg import expm
    N, n, k, h, steps = 16, 7, 4, 0.005, 2000
    K = 2.0 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)
    A = np.block([[np.zeros((N, N)), np.eye(N)], [-K, np.zeros((N, N))]])
    Q, P = normal_mode_draws(23, N, n)
    ics = O.fput_mode_ics(O.fput(N, beta=0.0), Q, P, np.full(n, 0.2 * N))
    w0 = np.random.default_rng(24).standard_normal((k * 2 * N, n))
    g = gpu_run(FPUT, N, ics, None, dt=h, n_steps=steps, k=k, ld_p=0.0, sys_params=(1.0, 0.0, 0.0),
                integrator=integ, w_in=w0)
    Phi = expm(A * h * steps)
    d = 2 * N
    np.testing.assert_allclose(g["x"], Phi @ ics, atol=1e-8)
    U = []
    for j in range(k):
        v = Phi @ w0[j * d:(j + 1) * d]
        U.append(v / np.linalg.norm(v, axis=0))
        np.testing.assert_allclose(g["w"][j * d:(j + 1) * d], U[j], atol=1e-8)
    U = np.stack(U)
    for o in range(n):
        for m in range(2, k + 1):
            sv = np.linalg.svd(U[:m, :, o].T, compute_uv=False)
            np.testing.assert_allclose(g["gali"][m - 2, o], np.prod(sv), rtol=1e-6)
        a, b = U[0, :, o], U[1, :, o]
        np.testing.assert_allclose(g["sali"][o], min(np.linalg.norm(a + b), np.linalg.norm(a - b)),
                                   rtol=1e-6)
