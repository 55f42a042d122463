"""Mixed-length FPUT Lyapunov batches -- one CUDA graph of concurrent branches,
and one persistent kernel over a work queue -- and the autotuner."""
import json

import numpy as np
import pytest

import oracle as O
from paper_2507_00622_gb300.inputs import normal_mode_draws

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2507_00622_gb300 import autotune, chs  # noqa: E402


def _fput_job(N, n, steps, qr=10):
    S = chs.System(chs.FPUT, N, (1.0, 0.0, 1.0))
    Q, P = normal_mode_draws(500 + N, N, n)
    ics = torch.from_numpy(O.fput_mode_ics(O.fput(N), Q, P, np.full(n, 0.1 * N))).cuda()
    lam = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    return S, chs.params(0.05, steps, qr_every=qr, sample_every=100), n, ics, lam, st


def _fput_job_params(N, n, steps, sp=(1.0, 0.0, 1.0), qr=10, seed=0):
    S = chs.System(chs.FPUT, N, sp)
    Q, P = normal_mode_draws(700 + N + seed, N, max(n, 1))
    ics = torch.from_numpy(np.ascontiguousarray(
        O.fput_mode_ics(O.fput(N), Q, P, np.full(max(n, 1), 0.1 * N))[:, :n])).cuda()
    lam = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    return S, chs.params(0.05, steps, qr_every=qr, sample_every=50), n, ics, lam, st


def test_persistent_mixed_chain_batch_equals_separate_calls():
    """One persistent kernel over every chain length at once (ragged ensembles,
    an FPUT-alpha+beta job, an empty job, a chain length twice, jobs out of
    order) gives bit for bit the exponents and statuses of separate calls."""
    specs = [(8, 45, (1.0, 0.0, 1.0)), (64, 3, (1.0, 0.0, 1.0)), (4, 70, (1.0, 0.25, 1.0)),
             (16, 9, (1.0, 0.0, 1.0)), (32, 5, (1.0, 0.0, 1.0)), (4, 33, (1.0, 0.0, 1.0)),
             (16, 0, (1.0, 0.0, 1.0)), (8, 7, (1.0, 0.3, 1.0))]
    jobs = [_fput_job_params(N, n, 330, sp, qr=7, seed=i) for i, (N, n, sp) in enumerate(specs)]
    work = torch.empty(1, dtype=torch.int64, device="cuda")
    for _ in range(2):  # the queue counter is reset by every call
        chs.chs_lyapunov_batch_persistent([(S.h, prm, n, ics, None, lam, st) for S, prm, n, ics, lam, st in jobs],
                                          work)
        torch.cuda.synchronize()
    got = [(lam.cpu().numpy().copy(), st.cpu().numpy().copy()) for *_x, lam, st in jobs]
    for (S, prm, n, ics, lam, st), (gl, gs) in zip(jobs, got):
        if n == 0:
            continue
        chs.chs_lyapunov_spectrum(S.h, prm, n, ics, None, lam, st)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(gl, lam.cpu().numpy())
        np.testing.assert_array_equal(gs, st.cpu().numpy())
        assert (gs == chs.ORBIT_OK).all()


def test_persistent_batch_argument_checks():
    S, prm, n, ics, lam, st = _fput_job_params(8, 4, 10)
    work = torch.empty(1, dtype=torch.int64, device="cuda")
    job = (S.h, prm, n, ics, None, lam, st)
    with pytest.raises(chs.ChsError) as e:
        chs.chs_lyapunov_batch_persistent([job] * 17, work)
    assert e.value.code == chs.CHS_E_INVALID
    dp = chs.params(0.05, 10, qr_every=10, integrator=chs.DOP853)
    with pytest.raises(chs.ChsError) as e:
        chs.chs_lyapunov_batch_persistent([(S.h, dp, n, ics, None, lam, st)], work)
    assert e.value.code == chs.CHS_E_UNSUPPORTED
    H = chs.System(chs.HENON_HEILES, 2)
    hl = torch.empty((4, n), dtype=torch.float64, device="cuda")
    hi = torch.zeros((4, n), dtype=torch.float64, device="cuda")
    with pytest.raises(chs.ChsError) as e:
        chs.chs_lyapunov_batch_persistent([(H.h, chs.params(0.01, 10, qr_every=10), n, hi, None, hl, st)], work)
    assert e.value.code == chs.CHS_E_UNSUPPORTED
    code = chs.load().chs_lyapunov_batch_persistent(None, 1, None, 8, None)
    assert code == chs.CHS_E_INVALID


def test_mixed_chain_batch_equals_separate_calls():
    jobs = [_fput_job(N, n, 400) for N, n in ((4, 100), (8, 33), (16, 17), (32, 9), (64, 5))]
    chs.chs_lyapunov_batch([(S.h, prm, n, ics, None, lam, st) for S, prm, n, ics, lam, st in jobs])
    torch.cuda.synchronize()
    batch = [lam.clone() for *_x, lam, _st in jobs]
    for (S, prm, n, ics, lam, st), b in zip(jobs, batch):
        chs.chs_lyapunov_spectrum(S.h, prm, n, ics, None, lam, st)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(lam.cpu().numpy(), b.cpu().numpy())
        assert (st.cpu().numpy() == 0).all()


def test_qr_interval_changes_the_spectrum_only_by_rounding():
    """In exact arithmetic the accumulated ln R_ii do not depend on when the QR is
    taken; in FP64 the spectra for intervals 10 and 50 agree to rounding."""
    a = _fput_job(16, 24, 1000, qr=10)
    b = _fput_job(16, 24, 1000, qr=50)
    for S, prm, n, ics, lam, st in (a, b):
        chs.chs_lyapunov_spectrum(S.h, prm, n, ics, None, lam, st)
    torch.cuda.synchronize()
    assert np.abs(a[4].cpu().numpy() - b[4].cpu().numpy()).max() < 1e-11


def test_autotuner_caches_a_valid_choice(tmp_path, monkeypatch):
    monkeypatch.setenv("CHS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    r = autotune.tune_fput_qr(8, candidates=(10, 20, 50), n_orbits=152, steps=200)
    assert r["qr_every"] in (10, 20, 50)
    assert r["max_abs_diff_vs_ref"][str(r["qr_every"])] <= 1e-10
    c = autotune.tune_compact_chunk(side=64, steps=20000, candidates=(1000, 5000))
    assert c["chunk_steps"] in (1000, 5000)
    saved = json.load(open(tmp_path / "tune.json"))
    assert len(saved) == 2
    # a second call is served from the cache
    assert autotune.tune_fput_qr(8, candidates=(10, 20, 50), n_orbits=152, steps=200) == r
