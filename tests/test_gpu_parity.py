"""Parity of the CUDA path (through its C ABI) with the CPU oracle.

Every case runs the same seeded synthetic input through both sides.  Bars:
bit-exact for integers, statuses and the explicitly rounded set-up kernels;
FP64 states within 1e-10 of the orbit's state norm at short horizons and on
regular orbits at full length; indicators within 1e-8 * max(1, |ref|) on
regular orbits; >= 99.5 % label agreement over valid cells.
"""
import numpy as np
import pytest

import oracle as O
from paper_2507_00622_gb300.inputs import hh_section_box, normal_mode_draws, strided_sample, uniform_vectors
from tests.helpers import IND_TOL, LABEL_AGREE, STATE_RTOL, gpu_run, ind_err, oracle_run, state_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2507_00622_gb300 import chs  # noqa: E402

HH = chs.HENON_HEILES


def _grid(E, ny, npy):
    y0, y1, p0, p1 = hh_section_box(E)
    return (E, y0, y1, ny, p0, p1, npy)


def _gpu_grid(E, y0, y1, ny, p0, p1, npy):
    S = chs.System(HH, 2)
    n = ny * npy
    ics = torch.empty((4, n), dtype=torch.float64, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    chs.chs_section_grid_ics(S.h, E, y0, y1, ny, p0, p1, npy, ics, st)
    torch.cuda.synchronize()
    return ics.cpu().numpy(), st.cpu().numpy()


# --------------------------------------------------------------------------
# set-up kernels: bit-exact
# --------------------------------------------------------------------------

@pytest.mark.parametrize("E,ny,npy", [(1 / 8, 32, 32), (1 / 6, 1024, 1024), (1 / 6, 37, 19)])
def test_section_grid_bit_exact(E, ny, npy):
    g = _grid(E, ny, npy)
    gi, gs = _gpu_grid(*g)
    oi, os_ = O.grid_ics(*g)
    np.testing.assert_array_equal(gs, os_)
    np.testing.assert_array_equal(gi.view(np.int64), oi.view(np.int64))


def test_seeded_vectors_bit_exact():
    """Seeded vectors are the normalised SplitMix64 draws (the oracle's
    seed_vectors, bit for bit, without renorm) and are normalised once more
    with renorm, as the oracle's ensemble set-up does."""
    g = _grid(1 / 6, 19, 23)
    ics, st = O.grid_ics(*g)
    for k in (2, 4):
        ref = O.seed_vectors(12345, ics.shape[1], k, 4)
        out = gpu_run(HH, 2, ics, st, dt=0.01, n_steps=0, k=k, seed=12345, renorm=False)
        np.testing.assert_array_equal(out["w"].view(np.int64), ref.view(np.int64))
        out = gpu_run(HH, 2, ics, st, dt=0.01, n_steps=0, k=k, seed=12345)
        e = O.Ensemble(O.henon_heiles(), O.params(0.01, 1, n_dev=k), ics, st, seed=12345)
        np.testing.assert_array_equal(out["w"].view(np.int64), e.w.view(np.int64))


def test_fput_mode_ics_match_oracle():
    for N in (4, 8, 16, 32, 64):
        n = 33
        Q, P = normal_mode_draws(N, N, n)
        E = np.full(n, 0.1 * N)
        S = chs.System(chs.FPUT, N, (1.0, 0.0, 1.0))
        ics = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
        chs.chs_fput_mode_ics(S.h, n, torch.from_numpy(Q).cuda(), torch.from_numpy(P).cuda(),
                              torch.from_numpy(E).cuda(), ics)
        ref = O.fput_mode_ics(O.fput(N), Q, P, E)
        assert state_rel_err(ics.cpu().numpy(), ref).max() < 1e-13


# --------------------------------------------------------------------------
# Henon-Heiles: the 32 x 32 E = 1/8 grid, k = 2, LD p = 1/2, h = 0.01, t = 200
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def hh_small():
    g = _grid(1 / 8, 32, 32)
    ics, st = O.grid_ics(*g)
    kw = dict(dt=0.01, k=2, ld_p=0.5, escape_r2=4.0, seed=1, grid=(32, 32))
    short = (gpu_run(HH, 2, ics, st, n_steps=2000, **kw), oracle_run(HH, 2, ics, st, n_steps=2000, **kw))
    full = (gpu_run(HH, 2, ics, st, n_steps=20000, **kw), oracle_run(HH, 2, ics, st, n_steps=20000, **kw))
    lam, _ = O.lyapunov(O.henon_heiles(), O.params(0.01, 20000, qr_every=10), np.nan_to_num(ics), st)
    return ics, st, short, full, lam[0]


def test_hh_grid_short_horizon_all_orbits(hh_small):
    _, st, (g, r), _, _ = hh_small
    v = st == 0
    assert v.sum() > 700
    np.testing.assert_array_equal(g["status"], r["status"])
    np.testing.assert_array_equal(g["n_exec"], r["n_exec"])
    assert state_rel_err(g["x"][:, v], r["x"][:, v]).max() < STATE_RTOL
    assert state_rel_err(g["w"][:, v], r["w"][:, v]).max() < STATE_RTOL
    assert ind_err(g["ld"][v], r["ld"][v]).max() < IND_TOL
    assert ind_err(g["sali"][v], r["sali"][v]).max() < IND_TOL
    assert ind_err(g["gali"][:, v], r["gali"][:, v]).max() < IND_TOL
    m = np.isfinite(r["dl"])
    np.testing.assert_array_equal(np.isfinite(g["dl"]), m)
    assert ind_err(g["dl"][m], r["dl"][m]).max() < IND_TOL
    assert ind_err(g["sl"][m], r["sl"][m]).max() < IND_TOL
    assert np.abs(g["dh_max"][v] - r["dh_max"][v]).max() < 1e-13


def test_hh_grid_full_length_regular_orbits_and_labels(hh_small):
    _, st, _, (g, r), lam1 = hh_small
    v = st == 0
    # regular: finite-time largest exponent at t = 200 (oracle QR method) below 0.02;
    # on this grid a 1e-15 perturbation of those orbits grows to at most ~3e-12
    reg = v & (lam1 < 0.02)
    assert reg.sum() > 300
    assert state_rel_err(g["x"][:, reg], r["x"][:, reg]).max() < STATE_RTOL
    assert ind_err(g["ld"][reg], r["ld"][reg]).max() < IND_TOL
    assert ind_err(g["sali"][reg], r["sali"][reg]).max() < IND_TOL
    assert ind_err(g["gali"][:, reg], r["gali"][:, reg]).max() < IND_TOL
    agree = (g["label"][v] == r["label"][v]).mean()
    assert agree >= LABEL_AGREE
    np.testing.assert_array_equal(g["label"][~v], r["label"][~v])
    assert np.nanmax(g["dh_max"][v]) < 1e-9


def test_hh_e16_k4_gali_short_horizon():
    g0 = _grid(1 / 6, 48, 40)
    ics, st = O.grid_ics(*g0)
    kw = dict(dt=0.01, n_steps=2000, k=4, ld_p=0.5, escape_r2=4.0, seed=7, grid=(48, 40))
    g, r = gpu_run(HH, 2, ics, st, **kw), oracle_run(HH, 2, ics, st, **kw)
    np.testing.assert_array_equal(g["status"], r["status"])
    ok = r["status"] == 0
    assert state_rel_err(g["x"][:, ok], r["x"][:, ok]).max() < STATE_RTOL
    assert ind_err(g["sali"][ok], r["sali"][ok]).max() < IND_TOL
    big = ok[None, :] & (np.abs(r["gali"]) > 1e-12)
    assert ind_err(g["gali"][big], r["gali"][big]).max() < IND_TOL
    small = ok[None, :] & ~big
    assert np.all(np.abs(g["gali"][small]) < 1e-10)
    assert ind_err(g["ld"][ok], r["ld"][ok]).max() < IND_TOL
    np.testing.assert_array_equal(g["label"], r["label"])


def test_chunked_gpu_run_is_bit_identical():
    g0 = _grid(1 / 6, 16, 16)
    ics, st = O.grid_ics(*g0)
    kw = dict(dt=0.01, k=3, ld_p=0.5, escape_r2=4.0, seed=3, sample_every=100)
    a = gpu_run(HH, 2, ics, st, n_steps=3000, **kw)
    b = gpu_run(HH, 2, ics, st, n_steps=3000, chunks=[700, 1300, 1000], **kw)
    for key in ("x", "w", "ld", "dh_max", "n_exec", "status"):
        np.testing.assert_array_equal(a[key], b[key])


def test_caller_vectors_and_test_systems():
    rng = np.random.default_rng(4)
    for model in (chs.HARMONIC, chs.INVERTED):
        ics = rng.uniform(-0.5, 0.5, (4, 130))
        w = uniform_vectors(11, 130, 3, 4)
        kw = dict(dt=0.02, n_steps=500, k=3, ld_p=0.5, w_in=w)
        g, r = gpu_run(model, 2, ics, None, **kw), oracle_run(model, 2, ics, None, **kw)
        assert state_rel_err(g["x"], r["x"]).max() < STATE_RTOL
        assert state_rel_err(g["w"], r["w"]).max() < STATE_RTOL
        assert ind_err(g["sali"], r["sali"]).max() < IND_TOL
        assert ind_err(g["ld"], r["ld"]).max() < IND_TOL


def test_quartic3_k6_short_horizon():
    rng = np.random.default_rng(5)
    ics = rng.uniform(-1.0, 1.0, (6, 200))
    kw = dict(dt=0.01, n_steps=1000, k=6, ld_p=0.5, sys_params=(0.1,), seed=9)
    g, r = gpu_run(chs.QUARTIC3, 3, ics, None, **kw), oracle_run(chs.QUARTIC3, 3, ics, None, **kw)
    assert state_rel_err(g["x"], r["x"]).max() < STATE_RTOL
    assert state_rel_err(g["w"], r["w"]).max() < STATE_RTOL
    assert ind_err(g["sali"], r["sali"]).max() < IND_TOL
    big = np.abs(r["gali"]) > 1e-12
    assert ind_err(g["gali"][big], r["gali"][big]).max() < IND_TOL


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------

def test_empty_and_ragged_sizes():
    g0 = _grid(1 / 8, 1, 1)
    for n in (1, 127, 129, 257):
        ics, st = O.grid_ics(1 / 8, g0[1], g0[2], n, g0[4], g0[5], 1)
        kw = dict(dt=0.01, n_steps=300, k=2, ld_p=0.5, escape_r2=4.0)
        g, r = gpu_run(HH, 2, ics, st, **kw), oracle_run(HH, 2, ics, st, **kw)
        np.testing.assert_array_equal(g["status"], r["status"])
        ok = r["status"] == 0
        assert state_rel_err(g["x"][:, ok], r["x"][:, ok]).max(initial=0) < STATE_RTOL
    # n = 0 is a no-op that still validates and returns OK
    S = chs.System(HH, 2)
    ens = chs.DeviceEnsemble.empty(0, 4, 2)
    e = ens.abi()
    chs.chs_ensemble_init(S.h, chs.params(0.01, 1, n_dev=2), e, ens.x)
    chs.chs_integrate_batch(S.h, chs.params(0.01, 10, n_dev=2), e)
    chs.chs_indicators(S.h, chs.params(0.01, 10, n_dev=2), e)


def test_status_paths_match_oracle():
    # escaping orbits above E = 1/6, a NaN initial condition, a FORBIDDEN cell and
    # an energy-drift freeze at a health check
    ics = np.array([[0.0, 0.0, np.nan, 0.0, 0.0],
                    [0.3, -0.2, 0.0, 0.1, 0.1],
                    [0.2, 0.5, 0.3, 0.3, 0.3],
                    [0.55, 0.2, 0.1, 0.1, 0.1]])
    st = np.array([0, 0, 0, 1, 0], dtype=np.int32)
    seen = set()
    for dh_limit in (0.0, 1e-13):
        kw = dict(dt=0.01, n_steps=5000, k=2, ld_p=0.5, escape_r2=4.0, dh_limit=dh_limit)
        g, r = gpu_run(HH, 2, ics, st, **kw), oracle_run(HH, 2, ics, st, **kw)
        np.testing.assert_array_equal(g["status"], r["status"])
        np.testing.assert_array_equal(g["n_exec"], r["n_exec"])
        np.testing.assert_array_equal(g["label"], r["label"])
        seen |= set(g["status"].tolist())
    assert {chs.ORBIT_ESCAPED, chs.ORBIT_NONFINITE, chs.ORBIT_FORBIDDEN, chs.ORBIT_ENERGY_DRIFT} <= seen


def test_invalid_arguments_are_rejected():
    S = chs.System(HH, 2)
    ens = chs.DeviceEnsemble.empty(10, 4, 2)
    e = ens.abi()
    with pytest.raises(chs.ChsError) as ei:
        chs.chs_integrate_batch(S.h, chs.params(0.0, 10, n_dev=2), e)
    assert ei.value.code == chs.CHS_E_INVALID and "dt" in str(ei.value)
    with pytest.raises(chs.ChsError):
        chs.chs_integrate_batch(S.h, chs.params(0.01, 10, n_dev=5), e)
    with pytest.raises(chs.ChsError):
        chs.chs_indicators(S.h, chs.params(0.01, 1, n_dev=2, ld_p=0.5), e, 3, 4,
                           ld_ind=torch.empty((2, 10), dtype=torch.float64, device="cuda"))
    F = chs.System(chs.FPUT, 12)
    with pytest.raises(chs.ChsError) as ei:
        chs.chs_lyapunov_spectrum(F.h, chs.params(0.05, 10), 1, torch.zeros((24, 1), dtype=torch.float64,
                                  device="cuda"), None, torch.empty((24, 1), dtype=torch.float64,
                                  device="cuda"), torch.empty(1, dtype=torch.int32, device="cuda"))
    assert ei.value.code == chs.CHS_E_UNSUPPORTED
    with pytest.raises(ValueError):
        chs.chs_section_grid_ics(S.h, 0.125, -0.4, 0.6, 4, -0.5, 0.5, 4, torch.empty((4, 16)),
                                 torch.empty(16, dtype=torch.int32))


# --------------------------------------------------------------------------
# FP32 deviation vectors (FP64 state)
# --------------------------------------------------------------------------

def test_fp32_vectors_error_against_fp64_oracle():
    """FP32 deviation vectors held as an orthonormal frame plus a unit-column
    triangle (FP64 orbit and LD): indicator errors against the FP64 oracle."""
    g0 = _grid(1 / 8, 32, 32)
    ics, st = O.grid_ics(*g0)
    v = st == 0
    kw = dict(dt=0.01, n_steps=20000, k=3, ld_p=0.5, escape_r2=4.0)
    g = gpu_run(HH, 2, ics, st, vec_fp32=True, **kw)
    r = oracle_run(HH, 2, ics, st, **kw)
    # the orbit and LD do not depend on the vectors: FP64 parity holds for them
    lam, _ = O.lyapunov(O.henon_heiles(), O.params(0.01, 20000, qr_every=10), np.nan_to_num(ics), st)
    reg = v & (lam[0] < 0.02)
    assert state_rel_err(g["x"][:, reg], r["x"][:, reg]).max() < STATE_RTOL
    assert ind_err(g["ld"][reg], r["ld"][reg]).max() < IND_TOL
    # regular orbits: the FP32 rounding of the frame, grown along the torus
    rel = np.abs(g["sali"][reg] - r["sali"][reg]) / r["sali"][reg]
    assert np.median(rel) < 1e-3 and rel.max() < 5e-2
    relg = np.abs(g["gali"][:, reg] - r["gali"][:, reg]) / r["gali"][:, reg]
    assert np.median(relg) < 1e-3
    assert np.abs(g["w"][:, reg] - r["w"][:, reg]).max() < 5e-2
    assert (g["label"][v] == r["label"][v]).mean() >= LABEL_AGREE
    # at t = 2000 the SALI distribution has separated; the frame keeps resolving
    # SALI far below the FP32 rounding level, so the FP64 threshold 1e-8 applies
    kw["n_steps"] = 200000
    g = gpu_run(HH, 2, ics, st, vec_fp32=True, **kw)
    r = oracle_run(HH, 2, ics, st, **kw)
    assert (g["label"][v] == r["label"][v]).mean() >= LABEL_AGREE
    chaotic = v & (r["sali"] < 1e-12)
    assert chaotic.sum() > 100 and np.all(g["sali"][chaotic] < 1e-8)


def test_ld_newton_sqrt_precision():
    """The LD integrand uses Newton-refined square roots (about 1e-13 relative):
    LD parity with the oracle's libm pow(|f|, 1/2) to 1e-12 relative."""
    rng = np.random.default_rng(21)
    for model in (chs.HARMONIC, chs.INVERTED, chs.HENON_HEILES):
        ics = rng.uniform(-0.3, 0.3, (4, 300))
        kw = dict(dt=0.01, n_steps=500, k=0, ld_p=0.5)
        g, r = gpu_run(model, 2, ics, None, **kw), oracle_run(model, 2, ics, None, **kw)
        assert (np.abs(g["ld"] - r["ld"]) / np.abs(r["ld"])).max() < 1e-12


# --------------------------------------------------------------------------
# Lyapunov spectra
# --------------------------------------------------------------------------

def _gpu_lyap(model, N, ics, prm, sys_params=()):
    S = chs.System(model, N, sys_params)
    n = ics.shape[1]
    lam = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    chs.chs_lyapunov_spectrum(S.h, prm, n, torch.from_numpy(np.ascontiguousarray(ics)).cuda(), None,
                              lam, st)
    torch.cuda.synchronize()
    return lam.cpu().numpy(), st.cpu().numpy()


def test_lyapunov_inverted_closed_form_gpu():
    h, n = 0.01, 2000
    lam, st = _gpu_lyap(chs.INVERTED, 2, np.array([[0.1], [0.2], [0.3], [-0.1]]),
                        chs.params(h, n, qr_every=10))
    R = lambda z: 1 + z + z**2 / 2 + z**3 / 6 + z**4 / 24  # noqa: E731
    a, b, T = R(h), R(-h), n * h
    l1 = (2 * n * np.log(a) + np.log1p((b / a) ** (2 * n)) - np.log(2.0)) / (2 * T)
    l2 = np.log(abs(R(1j * h))) / h
    np.testing.assert_allclose(lam[:, 0], [l1, l2, n * np.log(a * b) / T - l1, l2], atol=1e-12, rtol=0)


def test_lyapunov_hh_matches_oracle():
    g0 = _grid(1 / 8, 12, 12)
    ics, st = O.grid_ics(*g0)
    ok = st == 0
    ics = ics[:, ok]
    g, gs = _gpu_lyap(HH, 2, ics, chs.params(0.01, 2000, qr_every=10))
    r, rs = O.lyapunov(O.henon_heiles(), O.params(0.01, 2000, qr_every=10), ics)
    assert np.abs(g - r).max() < 1e-8


@pytest.mark.parametrize("N", [4, 8, 16, 32, 64])
def test_fput_lyapunov_matches_oracle(N):
    """FPUT-beta (k = 1, beta = 1), normal-mode ICs at energy density 0.1,
    h = 0.05, QR every 10 steps, t = 100: every exponent within 1e-8."""
    n = 6 if N == 64 else 12
    Q, P = normal_mode_draws(100 + N, N, n)
    ics = O.fput_mode_ics(O.fput(N), Q, P, np.full(n, 0.1 * N))
    prm = chs.params(0.05, 2000, qr_every=10, sample_every=100)
    g, gs = _gpu_lyap(chs.FPUT, N, ics, prm, (1.0, 0.0, 1.0))
    r, rs = O.lyapunov(O.fput(N), O.params(0.05, 2000, qr_every=10, sample_every=100), ics)
    np.testing.assert_array_equal(gs, rs)
    assert np.abs(g - r).max() < 1e-8
    # the sum of the spectrum is (1/T) ln det of the RK4 tangent map: RK4 is not
    # volume preserving, so it is small but not zero; both sides agree on it
    assert np.abs(g.sum(axis=0) - r.sum(axis=0)).max() < 1e-9


@pytest.mark.parametrize("N", [4, 8])
def test_fput_alpha_beta_lyapunov_matches_oracle(N):
    """The FPU chain with both nonlinearities (alpha = 0.25, beta = 1; Eq.
    ham_FPU), QR every 7 steps, a last partial interval and a ragged block
    (13 orbits): every exponent within 1e-8 of the oracle at t = 50."""
    n = 13
    Q, P = normal_mode_draws(300 + N, N, n)
    ics = O.fput_mode_ics(O.fput(N), Q, P, np.full(n, 0.1 * N))
    prm = chs.params(0.05, 1003, qr_every=7, sample_every=50)
    g, gs = _gpu_lyap(chs.FPUT, N, ics, prm, (1.0, 0.25, 1.0))
    r, rs = O.lyapunov(O.fput(N, beta=1.0, alpha=0.25), O.params(0.05, 1003, qr_every=7, sample_every=50), ics)
    np.testing.assert_array_equal(gs, rs)
    assert np.abs(g - r).max() < 1e-8


@pytest.mark.parametrize("integ", ["rk4", "dop853"])
@pytest.mark.parametrize("N", [4, 8, 16, 32, 64])
def test_fput_lyapunov_single_orbit(N, integ):
    """An ensemble of one orbit (one block whose other orbit slots and lanes are
    empty) under RK4 and DOP853, FPUT-alpha+beta, QR every 7 steps with a last
    partial interval: every exponent within 1e-8 of the oracle."""
    Q, P = normal_mode_draws(500 + N, N, 1)
    ics = O.fput_mode_ics(O.fput(N), Q, P, np.full(1, 0.1 * N))
    gi, oi = (chs.DOP853, O.DOP853) if integ == "dop853" else (chs.RK4, O.RK4)
    g, gs = _gpu_lyap(chs.FPUT, N, ics, chs.params(0.05, 60, qr_every=7, sample_every=20, integrator=gi),
                      (1.0, 0.25, 1.0))
    r, rs = O.lyapunov(O.fput(N, beta=1.0, alpha=0.25),
                       O.params(0.05, 60, qr_every=7, sample_every=20, integrator=oi), ics)
    np.testing.assert_array_equal(gs, rs)
    assert rs[0] == chs.ORBIT_OK
    assert np.abs(g - r).max() < 1e-8


@pytest.mark.parametrize("N", [4, 8, 64])
def test_fput_lyapunov_nonfinite_orbit(N):
    """A NaN in one component of one orbit (a component of the third of the
    orbit's lanes) makes that orbit NONFINITE with NaN exponents and leaves its
    neighbours in the same warp untouched."""
    n = 11
    Q, P = normal_mode_draws(400 + N, N, n)
    ics = O.fput_mode_ics(O.fput(N), Q, P, np.full(n, 0.1 * N))
    bad = ics.copy()
    bad[N + N // 2, 5] = np.nan
    prm = chs.params(0.05, 200, qr_every=10, sample_every=100)
    g, gs = _gpu_lyap(chs.FPUT, N, bad, prm, (1.0, 0.0, 1.0))
    r, rs = O.lyapunov(O.fput(N), O.params(0.05, 200, qr_every=10, sample_every=100), bad)
    np.testing.assert_array_equal(gs, rs)
    assert gs[5] == chs.ORBIT_NONFINITE and np.all(np.isnan(g[:, 5]))
    keep = np.arange(n) != 5
    assert np.abs(g[:, keep] - r[:, keep]).max() < 1e-8


# --------------------------------------------------------------------------
# full-size workload (1024 x 1024 grid at E = 1/6, k = 4), sampled
# --------------------------------------------------------------------------

def test_full_size_grid_sampled_against_oracle():
    """The bench workload at full size, in the bench's launch configuration:
    GPU over all 1,048,576 cells; the oracle recomputes a strided sample of 2048
    cells one by one from the same inputs."""
    E, ny, npy = 1 / 6, 1024, 1024
    g0 = (E, -0.5, 1.0, ny, -np.sqrt(1 / 3), np.sqrt(1 / 3), npy)
    ics, st = _gpu_grid(*g0)
    kw = dict(dt=0.01, n_steps=1000, k=4, ld_p=0.5, escape_r2=4.0, seed=2)
    g = gpu_run(HH, 2, ics, st, grid=(ny, npy), **kw)
    idx = strided_sample(ny * npy, 2048)
    # the oracle sees the sampled cells as independent orbits with the same seeds:
    # vectors are taken from the GPU's seeding, which is bit-exact with the oracle's
    w_full = O.seed_vectors(2, ny * npy, 4, 4)
    r = oracle_run(HH, 2, ics[:, idx], st[idx], w_in=w_full[:, idx], **kw)
    # the sampled cells integrated alone (their seeded vectors given) are bit for
    # bit what they are inside the full-size launch: each thread integrates its
    # own orbit, so sampled runs at longer horizons stand for the full grid
    alone = gpu_run(HH, 2, ics[:, idx], st[idx], w_in=w_full[:, idx], **kw)
    for key in ("x", "w", "ld", "dh_max", "n_exec", "status", "sali", "gali", "label"):
        np.testing.assert_array_equal(alone[key], g[key][..., idx])
    np.testing.assert_array_equal(g["status"][idx], r["status"])
    ok = r["status"] == 0
    assert state_rel_err(g["x"][:, idx][:, ok], r["x"][:, ok]).max() < STATE_RTOL
    assert ind_err(g["sali"][idx][ok], r["sali"][ok]).max() < IND_TOL
    assert ind_err(g["ld"][idx][ok], r["ld"][ok]).max() < IND_TOL
    # LD indicators: the oracle's stencil applied to the GPU's LD field is bit-exact
    dl, sl = O.ld_indicators(ny, npy, g["ld"], g["status"])
    np.testing.assert_array_equal(np.isnan(dl), np.isnan(g["dl"]))
    m = ~np.isnan(dl)
    np.testing.assert_array_equal(dl[m], g["dl"][m])
    np.testing.assert_array_equal(sl[m], g["sl"][m])


# --------------------------------------------------------------------------
# early exit, uneven end steps, compacted graph runs, quartic shell ICs
# --------------------------------------------------------------------------

@pytest.mark.parametrize("vec_fp32", [False, True])
def test_early_exit_matches_oracle(vec_fp32):
    g0 = _grid(1 / 8, 32, 32)
    ics, st = O.grid_ics(*g0)
    kw = dict(dt=0.01, n_steps=100000, k=2, ld_p=0.5, escape_r2=4.0, early_exit=True)
    g = gpu_run(HH, 2, ics, st, vec_fp32=vec_fp32, **kw)
    r = oracle_run(HH, 2, ics, st, **kw)
    v = st == 0
    early = r["status"] == chs.ORBIT_EARLY_CHAOTIC
    assert early.sum() > 100
    # the stop is a floating-point decision taken at health checks: stop steps agree
    # exactly on nearly all orbits, labels on >= 99.5 %
    assert (g["status"][v] == r["status"][v]).mean() >= LABEL_AGREE
    assert (g["n_exec"][v] == r["n_exec"][v]).mean() >= 0.99
    assert (g["label"][v] == r["label"][v]).mean() >= LABEL_AGREE
    assert np.all(g["label"][g["status"] == chs.ORBIT_EARLY_CHAOTIC] == 1)


@pytest.mark.parametrize("vec_fp32", [False, True])
def test_compacted_graph_run_is_bit_identical_to_plain(vec_fp32):
    g0 = _grid(1 / 6, 40, 40)
    ics, st = O.grid_ics(*g0)
    rng = np.random.default_rng(3)
    t_end = rng.integers(0, 6000, ics.shape[1]).astype(np.int64)
    kw = dict(dt=0.01, k=3, ld_p=0.5, escape_r2=4.0, early_exit=True, t_end=t_end,
              vec_fp32=vec_fp32, seed=5)
    a = gpu_run(HH, 2, ics, st, n_steps=5000, **kw)
    b = gpu_run(HH, 2, ics, st, n_steps=5000, chunks=[2300, 2700], compact_chunk=300, **kw)
    for key in ("x", "w", "ld", "dh_max", "n_exec", "status", "sali", "gali", "label"):
        np.testing.assert_array_equal(a[key], b[key])
    ok = st == 0
    np.testing.assert_array_equal(a["n_exec"][ok & (a["status"] == 0)],
                                  np.minimum(t_end, 5000)[ok & (a["status"] == 0)])


@pytest.mark.parametrize("vec_fp32,integrator", [(False, chs.RK4), (True, chs.RK4), (False, chs.DOP853)])
def test_persistent_queue_run_is_bit_identical_to_plain(vec_fp32, integrator):
    """The work-queue launch (threads take orbit after orbit) changes which thread
    integrates which orbit, never the arithmetic: identical results, with uneven
    end steps and early exits, resumed in two calls."""
    g0 = _grid(1 / 6, 40, 40)
    ics, st = O.grid_ics(*g0)
    rng = np.random.default_rng(4)
    t_end = rng.integers(0, 6000, ics.shape[1]).astype(np.int64)
    kw = dict(dt=0.01, k=3, ld_p=0.5, escape_r2=4.0, early_exit=True, t_end=t_end,
              vec_fp32=vec_fp32, seed=5, integrator=integrator)
    a = gpu_run(HH, 2, ics, st, n_steps=5000, **kw)
    b = gpu_run(HH, 2, ics, st, n_steps=5000, chunks=[2300, 2700], persistent=True, **kw)
    for key in ("x", "w", "ld", "dh_max", "n_exec", "status", "sali", "gali", "label"):
        np.testing.assert_array_equal(a[key], b[key])
    # an empty queue run and a queue of one orbit
    S = chs.System(HH, 2)
    q = torch.empty(1, dtype=torch.int64, device="cuda")
    ens = chs.DeviceEnsemble.empty(0, 4, 2)
    chs.chs_integrate_persistent(S.h, chs.params(0.01, 10, n_dev=2), ens.abi(), q)
    one = gpu_run(HH, 2, ics[:, 700:701], st[700:701], n_steps=300, persistent=True, dt=0.01, k=2)
    ref = gpu_run(HH, 2, ics[:, 700:701], st[700:701], n_steps=300, dt=0.01, k=2)
    np.testing.assert_array_equal(one["x"], ref["x"])


def test_uneven_end_steps_match_oracle():
    g0 = _grid(1 / 8, 20, 20)
    ics, st = O.grid_ics(*g0)
    t_end = np.random.default_rng(8).integers(100, 3000, ics.shape[1]).astype(np.int64)
    kw = dict(dt=0.01, n_steps=3000, k=2, ld_p=0.5, escape_r2=4.0, t_end=t_end)
    g = gpu_run(HH, 2, ics, st, compact_chunk=500, **kw)
    r = oracle_run(HH, 2, ics, st, **kw)
    np.testing.assert_array_equal(g["n_exec"], r["n_exec"])
    ok = st == 0
    assert state_rel_err(g["x"][:, ok], r["x"][:, ok]).max() < STATE_RTOL
    assert ind_err(g["ld"][ok], r["ld"][ok]).max() < IND_TOL


def test_quartic_shell_ics_and_fp32_gali6():
    n = 500
    rng = np.random.default_rng(17)
    dirs = rng.standard_normal((6, n))
    E = rng.uniform(1.0, 10.0, n)
    S = chs.System(chs.QUARTIC3, 3, (0.1,))
    ics = torch.empty((6, n), dtype=torch.float64, device="cuda")
    chs.chs_shell_ics(S.h, n, torch.from_numpy(dirs).cuda(), torch.from_numpy(E).cuda(), ics)
    ref = O.shell_ics(O.system(O.QUARTIC3, 3, eps=0.1), dirs, E)
    gi = ics.cpu().numpy()
    assert state_rel_err(gi, ref).max() < 1e-13
    kw = dict(dt=0.01, n_steps=2000, k=6, ld_p=0.5, sys_params=(0.1,), seed=4)
    g = gpu_run(chs.QUARTIC3, 3, ref, None, vec_fp32=True, **kw)
    r = oracle_run(chs.QUARTIC3, 3, ref, None, **kw)
    assert state_rel_err(g["x"], r["x"]).max() < STATE_RTOL
    big = np.abs(r["gali"]) > 1e-6
    rel = np.abs(g["gali"][big] - r["gali"][big]) / r["gali"][big]
    assert np.median(rel) < 1e-3


# --------------------------------------------------------------------------
# full-size workloads of the other configurations, sampled
# --------------------------------------------------------------------------

def test_fput_bench_size_sampled_against_oracle():
    """The FPUT Lyapunov run at bench size (4096 orbits per chain length, one
    launch each, QR interval 10): 12 strided orbits per N recomputed by the oracle."""
    steps = 200
    for N in (4, 8, 16, 32, 64):
        n = 4096
        Q, P = normal_mode_draws(1000 + N, N, n)
        S = chs.System(chs.FPUT, N, (1.0, 0.0, 1.0))
        ics = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
        chs.chs_fput_mode_ics(S.h, n, torch.from_numpy(Q).cuda(), torch.from_numpy(P).cuda(),
                              torch.full((n,), 0.1 * N, dtype=torch.float64, device="cuda"), ics)
        lam = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
        st = torch.empty(n, dtype=torch.int32, device="cuda")
        chs.chs_lyapunov_spectrum(S.h, chs.params(0.05, steps, qr_every=10, sample_every=100), n, ics,
                                  None, lam, st)
        torch.cuda.synchronize()
        idx = strided_sample(n, 12)
        ics_h = ics.cpu().numpy()[:, idx]
        r, rs = O.lyapunov(O.fput(N), O.params(0.05, steps, qr_every=10, sample_every=100), ics_h)
        assert np.abs(lam.cpu().numpy()[:, idx] - r).max() < 1e-8
        np.testing.assert_array_equal(st.cpu().numpy()[idx], rs)


def test_quartic_bench_size_sampled_against_oracle():
    """The quartic-3 run at its full size (4,194,304 shell states, k = 6 FP32 frame,
    uneven end steps, early exit), 1000 steps: 256 strided orbits recomputed by
    the oracle with FP64 vectors."""
    n = 4_194_304
    rng = np.random.default_rng(5)
    dirs = rng.standard_normal((6, n))
    E = rng.uniform(1.0, 10.0, n)
    t_end = rng.integers(100, 1001, n).astype(np.int64)
    S = chs.System(chs.QUARTIC3, 3, (0.1,))
    ics = torch.empty((6, n), dtype=torch.float64, device="cuda")
    chs.chs_shell_ics(S.h, n, torch.from_numpy(dirs).cuda(), torch.from_numpy(E).cuda(), ics)
    idx = strided_sample(n, 256)
    ics_h = ics[:, torch.from_numpy(idx).cuda()].cpu().numpy()
    kw = dict(dt=0.01, n_steps=1000, k=6, ld_p=0.0, sys_params=(0.1,), seed=3, early_exit=True)
    ens = chs.DeviceEnsemble.empty(n, 6, 6, vec_fp32=True)
    te = torch.from_numpy(t_end).cuda()
    abi = ens.abi(with_ld=False, t_end=te)
    prm = chs.params(0.01, 1000, n_dev=6, seed=3, vec_precision=chs.VEC_FP32, early_exit=True)
    chs.chs_ensemble_init(S.h, prm, abi, ics)
    w0 = ens.w.clone()  # the set-up's FP32 frames, to restart the sample from
    work = chs.compact_work(n)
    chs.chs_integrate_compacted(S.h, prm, abi, 500, work)
    gali = torch.empty((5, n), dtype=torch.float64, device="cuda")
    chs.chs_indicators(S.h, prm, abi, gali=gali)
    torch.cuda.synchronize()
    w_full = O.seed_vectors(3, n, 6, 6)
    r = oracle_run(chs.QUARTIC3, 3, ics_h, None, w_in=w_full[:, idx], t_end=t_end[idx], **kw)
    # the sample integrated alone, from the FP32 frame the full-size set-up built
    # for it, equals its part of the full-size compacted run bit for bit
    alone = chs.DeviceEnsemble.empty(idx.size, 6, 6, vec_fp32=True)
    it = torch.from_numpy(idx).cuda()
    te_s = te[it].contiguous()
    abi_s = alone.abi(with_ld=False, t_end=te_s)
    chs.chs_ensemble_init(S.h, prm, abi_s, ics[:, it].contiguous())
    alone.w.copy_(w0[:, it])
    chs.chs_integrate_compacted(S.h, prm, abi_s, 500, chs.compact_work(idx.size))
    torch.cuda.synchronize()
    for name in ("x", "w", "dh_max", "n_exec", "status"):
        np.testing.assert_array_equal(getattr(alone, name).cpu().numpy(),
                                      getattr(ens, name)[..., it].cpu().numpy())
    np.testing.assert_array_equal(ens.n_exec.cpu().numpy()[idx], r["n_exec"])
    assert state_rel_err(ens.x.cpu().numpy()[:, idx], r["x"]).max() < STATE_RTOL
    g = gali.cpu().numpy()[:, idx]
    big = np.abs(r["gali"]) > 1e-6
    rel = np.abs(g[big] - r["gali"][big]) / r["gali"][big]
    assert np.median(rel) < 1e-3 and rel.max() < 5e-2


# --------------------------------------------------------------------------
# backward runs (h < 0): the LD grows with |t|
# --------------------------------------------------------------------------

@pytest.mark.parametrize("vec_fp32,integrator", [(False, chs.RK4), (True, chs.RK4), (False, chs.DOP853)])
def test_backward_run_matches_oracle(vec_fp32, integrator):
    g0 = _grid(1 / 8, 16, 16)
    ics, st = O.grid_ics(*g0)
    kw = dict(dt=-0.02, n_steps=500, k=2, ld_p=0.5, escape_r2=4.0, integrator=integrator)
    g = gpu_run(HH, 2, ics, st, vec_fp32=vec_fp32, **kw)
    r = oracle_run(HH, 2, ics, st, **kw)
    ok = (st == 0) & (r["status"] == 0)
    np.testing.assert_array_equal(g["status"], r["status"])
    assert state_rel_err(g["x"][:, ok], r["x"][:, ok]).max() < STATE_RTOL
    assert np.all(g["ld"][ok] > 0)
    assert ind_err(g["ld"][ok], r["ld"][ok]).max() < (1e-6 if vec_fp32 else IND_TOL)
