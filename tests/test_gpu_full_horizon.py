"""Parity of the headline workloads with the CPU oracle at their full length.

The shorter parity tests stop at t = 20 .. 200; here each workload runs to its
own end time, through the C ABI in the launch configuration the bench times:
  - the Henon-Heiles section grid at E = 1/6 (1024 x 1024 cells, k = 4 vectors,
    LD p = 1/2, RK4 h = 0.01, 1000-step calls) to t = 1e4, with FP64 and with
    FP32 deviation vectors (Sec. Functionalities; Sec. Examples, Henon-Heiles);
  - the FPUT-beta Lyapunov spectra, N = 4 .. 64, QR every 10 steps, to t = 1e4
    (Sec. Examples, FPU chain);
  - the coupled quartic oscillators with uneven end times t_end in [1e3, 1e4],
    early exit and FP32 vectors.
The oracle recomputes strided samples of each workload from the same inputs.
The FP32 grid run covers the whole grid; the FP64 grid run and the quartic run
integrate their samples alone, which gives bit for bit the results those orbits
have inside the full-size launch (each thread integrates its own orbit; checked
at the bench's chunk length in tests/test_gpu_parity.py).

Bars.  Labels (regular / chaotic / escaped) agree on >= 99.5 % of a sample.
At t = 1e4 the short-horizon tolerances of the other parity tests (states
within 1e-10, indicators within 1e-8 on regular orbits) lie below what FP64
itself reproduces: the oracle run a second time from initial states moved by one ulp
drifts from its first run by up to ~6e-10 in the state and ~4e-7 in SALI on
regular orbits of the E = 1/8 grid (the phase along a torus drifts with every
rounding difference, at a rate growing with t).  So each test runs the oracle
twice -- from the initial states and from the states moved by one ulp -- and
holds the GPU to the oracle's own reproducibility on the regular orbits (oracle
SALI > 1e-2 at the end, where a chaotic orbit would need lambda_1 < 2.3e-4,
SALI ~ exp(-2 lambda_1 t)):
  - states: the largest and the median error (relative to the orbit's state
    norm) at most 4x those of the one-ulp run, and never required below 1e-10;
  - SALI, GALI_k (values >= 1e-12; below that they sit at the vectors' rounding
    floor) and the LD, each against 1e-8 * max(1, |ref|): no more orbits past
    that bar than twice the one-ulp run's count plus 2, and the largest error at
    most 4x the one-ulp run's largest plus 1e-8;
  - FP32 vectors: labels and the orbit (FP64) as above, the LD within 1e-6, and
    the errors of SALI and GALI against the FP64 oracle reported (printed) with
    an order-of-magnitude bar: on regular orbits the FP32 frame's rounding
    accumulates under the shear of the torus to ~10 % at t = 1e4;
  - Lyapunov exponents: lambda_1 at t = 1e4 of a chaotic chain moves by 5 - 40 %
    under a 1e-14 change of its initial state (the oracle against itself,
    tests/golden/make_fput_lyapunov_t1e4.py), so the 5 % bar applies to the mean
    of lambda_1 over each chain length's sample; orbits whose lambda_1 the oracle
    reproduces under that change (regular ones) are held to 1e-8 each;
  - quartic runs with early exit: a chaotic orbit's stop step is as sensitive to
    rounding as its state, so statuses (which decide the labels) are compared,
    and the step counts of the orbits that run to their end.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2507_00622_gb300.inputs import normal_mode_draws, strided_sample
from tests.helpers import IND_TOL, LABEL_AGREE, STATE_RTOL, gpu_run, ind_err, oracle_run, state_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2507_00622_gb300 import chs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
HH = chs.HENON_HEILES

# Henon-Heiles grid run at E = 1/6
E16, SIDE, K = 1.0 / 6.0, 1024, 4
STEPS, CHUNK = 1_000_000, 1000
GRID_KW = dict(dt=0.01, k=K, ld_p=0.5, escape_r2=4.0, seed=2)
N_SAMPLE = 1024
REGULAR_SALI = 1e-2
GALI_FLOOR = 1e-12


def _grid_box():
    return (E16, -0.5, 1.0, SIDE, -np.sqrt(1.0 / 3.0), np.sqrt(1.0 / 3.0), SIDE)


def _one_ulp(ics, seed=0):
    """The initial states moved by one ulp each, in seeded random directions."""
    rng = np.random.default_rng(seed)
    return np.nextafter(ics, ics + rng.choice([-1.0, 1.0], ics.shape))


def _oracle_pair(ics, st, **kw):
    """The oracle from the initial states, and again from the states moved by one
    ulp (same vectors): the second run shows how far two FP64 computations that
    round differently drift apart on each orbit."""
    return oracle_run(HH, 2, ics, st, **kw), oracle_run(HH, 2, _one_ulp(ics), st, **kw)


def _check_states(g, r, rp, sel):
    """States on the orbits `sel` against the oracle's one-ulp reproducibility."""
    eg = state_rel_err(g["x"][:, sel], r["x"][:, sel])
    ep = state_rel_err(rp["x"][:, sel], r["x"][:, sel])
    assert eg.max() <= max(STATE_RTOL, 4.0 * ep.max()), (eg.max(), ep.max())
    assert np.median(eg) <= max(STATE_RTOL, 4.0 * np.median(ep)), (np.median(eg), np.median(ep))


def _check_indicators(g, r, rp, sel):
    """SALI, GALI_k (values >= 1e-12) and the LD on the orbits `sel` against
    1e-8 * max(1, |ref|), relative to the oracle's one-ulp reproducibility."""
    pairs = [(g["sali"][sel], rp["sali"][sel], r["sali"][sel]), (g["ld"][sel], rp["ld"][sel], r["ld"][sel])]
    big = np.abs(r["gali"][:, sel]) >= GALI_FLOOR
    pairs.append((g["gali"][:, sel][big], rp["gali"][:, sel][big], r["gali"][:, sel][big]))
    for gv, pv, rv in pairs:
        eg, ep = ind_err(gv, rv), ind_err(pv, rv)
        assert (eg > IND_TOL).sum() <= 2 * (ep > IND_TOL).sum() + 2, ((eg > IND_TOL).sum(), (ep > IND_TOL).sum())
        assert eg.max() <= 4.0 * ep.max() + IND_TOL, (eg.max(), ep.max())


@pytest.fixture(scope="module")
def grid_e16_oracle():
    """A strided sample of the valid cells of the 1024 x 1024 grid at E = 1/6,
    integrated by the oracle to t = 1e4 from the grid's initial states and the
    device-seeded vectors of those cells (both bit-exact with the GPU's set-up),
    and again from the states moved by one ulp."""
    ics, st = O.grid_ics(*_grid_box())
    valid = np.where(st == 0)[0]
    idx = valid[strided_sample(valid.size, N_SAMPLE)]
    w = O.seed_vectors(GRID_KW["seed"], SIDE * SIDE, K, 4)[:, idx]
    ref, ref_ulp = _oracle_pair(ics[:, idx], st[idx], w_in=w, n_steps=STEPS, **GRID_KW)
    return ics, st, idx, w, ref, ref_ulp


def _check_grid_against_oracle(g, r, rp, fp32: bool, min_regular: int):
    """Labels on the whole sample; states and indicators on its regular orbits
    (at least min_regular of them, so that the check is never vacuous)."""
    agree = float((g["label"] == r["label"]).mean())
    assert agree >= LABEL_AGREE, agree
    reg = (r["status"] == chs.ORBIT_OK) & (r["sali"] > REGULAR_SALI)
    assert reg.sum() >= min_regular, reg.sum()
    np.testing.assert_array_equal(g["status"][reg], r["status"][reg])
    np.testing.assert_array_equal(g["n_exec"][reg], r["n_exec"][reg])
    _check_states(g, r, rp, reg)
    if not fp32:
        _check_indicators(g, r, rp, reg)
    else:
        _fp32_indicator_errors("grid", g, r, reg)
        # the LD is accumulated in FP64 from an integrand summed in FP32 (each of
        # its ~1e6 x 4 terms rounded to ~6e-8 relative, unbiased)
        assert (np.abs(g["ld"][reg] - r["ld"][reg]) / r["ld"][reg]).max() < 1e-6
    return agree, int(reg.sum())


def _fp32_indicator_errors(what, g, r, reg):
    """Errors of the FP32-vector indicators against the FP64 oracle on regular
    orbits, printed for the record.  On a torus the tangent flow neither damps
    nor amplifies directions exponentially but shears them, so the frame's FP32
    rounding accumulates over the run (median relative error < 1e-3 at t = 200,
    tests/test_gpu_parity.py, but of order 10 % at t = 1e4).  Regular-orbit SALI
    and GALI values sit decades above the label thresholds, so the labels do not
    move; the bar is the order of magnitude: median |log10(gpu / oracle)| < 0.3."""
    out = {}
    big = np.abs(r["gali"][:, reg]) > 1e-6
    for name, gv, rv in (("SALI", g["sali"][reg], r["sali"][reg]),
                         ("GALI", g["gali"][:, reg][big], r["gali"][:, reg][big])):
        rel = np.abs(gv - rv) / np.abs(rv)
        dlog = np.abs(np.log10(np.maximum(np.abs(gv), 1e-300) / np.abs(rv)))
        out[name] = (np.median(rel), np.quantile(rel, 0.9), rel.max(), np.median(dlog))
        print(f"{what} FP32 vectors, {name} on {int(reg.sum())} regular orbits: relative error median "
              f"{out[name][0]:.3g}, 90th percentile {out[name][1]:.3g}, max {out[name][2]:.3g}; "
              f"median |log10 ratio| {out[name][3]:.3g}")
        assert out[name][3] < 0.3, (name, out[name])
    return out


def test_grid_e16_full_horizon_fp64(grid_e16_oracle):
    """FP64 vectors: the sampled cells in 1000-step calls to t = 1e4."""
    ics, st, idx, w, r, rp = grid_e16_oracle
    g = gpu_run(HH, 2, ics[:, idx], st[idx], w_in=w, n_steps=STEPS, chunks=[CHUNK] * (STEPS // CHUNK),
                **GRID_KW)
    # E = 1/6 is the escape energy and most of the section is chaotic: the oracle
    # finds 30 of the 1024 sampled cells regular at t = 1e4, 20 of them with
    # SALI > 1e-2 (labels are checked on all 1024)
    _check_grid_against_oracle(g, r, rp, fp32=False, min_regular=15)
    assert np.nanmax(g["dh_max"][r["status"] == chs.ORBIT_OK]) < 1e-7


def test_grid_e16_full_horizon_fp32_vectors_full_grid(grid_e16_oracle):
    """FP32 vectors (FP64 orbit, energy check and LD): the whole 1024 x 1024 grid
    as the bench runs it -- grid set-up, device-seeded vectors, 1000-step calls
    to t = 1e4, indicators and LD indicators -- compared with the FP64 oracle on
    the sampled cells."""
    ics, st, idx, _w, r, rp = grid_e16_oracle
    n = SIDE * SIDE
    S = chs.System(HH, 2)
    ics_t = torch.empty((4, n), dtype=torch.float64, device="cuda")
    st_t = torch.empty(n, dtype=torch.int32, device="cuda")
    chs.chs_section_grid_ics(S.h, *_grid_box(), ics_t, st_t)
    kw = dict(n_dev=K, ld_p=0.5, escape_r2=4.0, seed=GRID_KW["seed"], vec_precision=chs.VEC_FP32)
    ens = chs.DeviceEnsemble.empty(n, 4, K, vec_fp32=True)
    abi = ens.abi()
    chs.chs_ensemble_init(S.h, chs.params(0.01, 1, **kw), abi, ics_t, st_t)
    for c in range(STEPS // CHUNK):
        chs.chs_integrate_batch(S.h, chs.params(0.01, CHUNK, step0=c * CHUNK, **kw), abi)
    sali = torch.empty(n, dtype=torch.float64, device="cuda")
    gali = torch.empty((K - 1, n), dtype=torch.float64, device="cuda")
    label = torch.empty(n, dtype=torch.int8, device="cuda")
    ldi = torch.empty((2, n), dtype=torch.float64, device="cuda")
    chs.chs_indicators(S.h, chs.params(0.01, 0, **kw), abi, SIDE, SIDE, sali, gali, ldi, label)
    torch.cuda.synchronize()
    it = torch.from_numpy(idx).cuda()
    g = {"x": ens.x[:, it].cpu().numpy(), "ld": ens.ld[it].cpu().numpy(),
         "status": ens.status[it].cpu().numpy(), "n_exec": ens.n_exec[it].cpu().numpy(),
         "sali": sali[it].cpu().numpy(), "gali": gali[:, it].cpu().numpy(),
         "label": label[it].cpu().numpy()}
    # the grid set-up is the oracle's, bit for bit, and every valid cell ran
    np.testing.assert_array_equal(st_t.cpu().numpy(), st)
    _check_grid_against_oracle(g, r, rp, fp32=True, min_regular=15)
    # whole-grid sanity: every valid cell has a label, FORBIDDEN cells have none
    lab = label.cpu().numpy()
    assert np.all(np.isin(lab[st == 0], (0, 1, 2))) and np.all(lab[st != 0] == -1)
    # the LD indicators of the full field are the oracle's stencil of the GPU's LD field
    dl, sl = O.ld_indicators(SIDE, SIDE, ens.ld.cpu().numpy(), ens.status.cpu().numpy())
    gdl = ldi[0].cpu().numpy()
    np.testing.assert_array_equal(np.isnan(dl), np.isnan(gdl))
    m = ~np.isnan(dl)
    np.testing.assert_array_equal(dl[m], gdl[m])
    S.close()


# --------------------------------------------------------------------------
# Henon-Heiles grid at E = 1/8 (the classification workload's geometry), k = 2
# --------------------------------------------------------------------------

E18_KW = dict(dt=0.01, k=2, ld_p=0.5, escape_r2=4.0, seed=1)


@pytest.fixture(scope="module")
def grid_e18_oracle():
    """A strided sample of the valid cells of the 1024 x 1024 section grid at
    E = 1/8, integrated by the oracle to t = 1e4 (FP64 vectors, every orbit to
    the end, labels from the final SALI); vectors seeded for the sample."""
    from paper_2507_00622_gb300.inputs import hh_section_box

    E = 1.0 / 8.0
    y0, y1, p0, p1 = hh_section_box(E)
    ics, st = O.grid_ics(E, y0, y1, SIDE, p0, p1, SIDE)
    valid = np.where(st == 0)[0]
    idx = valid[strided_sample(valid.size, N_SAMPLE)]
    ref, ref_ulp = _oracle_pair(ics[:, idx], st[idx], n_steps=STEPS, **E18_KW)
    return ics[:, idx], st[idx], ref, ref_ulp


def test_grid_e18_full_horizon_plain_form(grid_e18_oracle):
    """The plain form of the classification (FP64 vectors, every orbit to t =
    1e4, 100,000-step calls) against the oracle."""
    ics, st, r, rp = grid_e18_oracle
    g = gpu_run(HH, 2, ics, st, n_steps=STEPS, chunks=[100_000] * (STEPS // 100_000), **E18_KW)
    _check_grid_against_oracle(g, r, rp, fp32=False, min_regular=200)


def test_grid_e18_full_horizon_fast_form(grid_e18_oracle):
    """The fast form of the classification (FP32 vector frame, early exit once
    SALI < 1e-8, compacted 2000-step chunks to t = 1e4) against the oracle's
    plain labels."""
    ics, st, r, rp = grid_e18_oracle
    g = gpu_run(HH, 2, ics, st, n_steps=STEPS, vec_fp32=True, early_exit=True,
                t_end=np.full(ics.shape[1], STEPS, dtype=np.int64), compact_chunk=2000, **E18_KW)
    agree = float((g["label"] == r["label"]).mean())
    assert agree >= LABEL_AGREE, agree
    early = g["status"] == chs.ORBIT_EARLY_CHAOTIC
    assert early.sum() > 100
    reg = (r["status"] == chs.ORBIT_OK) & (r["sali"] > REGULAR_SALI)
    _check_states(g, r, rp, reg)


# --------------------------------------------------------------------------
# FPUT-beta Lyapunov spectra to t = 1e4 against the oracle's stored values
# --------------------------------------------------------------------------

def _fput_golden():
    with open(os.path.join(HERE, "golden", "fput_lyapunov_t1e4.json")) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def fput_t1e4():
    """Every chain length's sample (the draws the golden file names, initial
    states from the oracle's normal-mode map) integrated on the GPU to t = 1e4
    with QR every 10 steps, all chain lengths in one batched launch."""
    gold = _fput_golden()
    wl = gold["workload"]
    jobs, keep = [], []
    for key, rec in gold["chains"].items():
        N = int(key)
        idx = np.asarray(rec["draw_index"])
        Q, P = normal_mode_draws(1000 + N, N, wl["draws_per_N"])
        ics = O.fput_mode_ics(O.fput(N), Q[:, idx], P[:, idx], np.full(idx.size, wl["energy_density"] * N))
        S = chs.System(chs.FPUT, N, (1.0, 0.0, wl["beta"]))
        lam = torch.empty((2 * N, idx.size), dtype=torch.float64, device="cuda")
        st = torch.empty(idx.size, dtype=torch.int32, device="cuda")
        prm = chs.params(wl["dt"], wl["n_steps"], qr_every=wl["qr_every"], sample_every=100)
        ics_t = torch.from_numpy(ics).cuda()
        jobs.append((S.h, prm, idx.size, ics_t, None, lam, st))
        keep.append((N, S, ics_t, lam, st, rec))
    chs.chs_lyapunov_batch(jobs)
    torch.cuda.synchronize()
    out = {N: (lam.cpu().numpy(), st.cpu().numpy(), rec) for N, S, _i, lam, st, rec in keep}
    for _N, S, *_r in keep:
        S.close()
    return out


@pytest.mark.parametrize("N", [4, 8, 16, 32, 64])
def test_fput_lyapunov_t1e4_against_oracle(fput_t1e4, N):
    lam, st, rec = fput_t1e4[N]
    np.testing.assert_array_equal(st, rec["status"])
    l1 = lam[0]
    ref = np.asarray(rec["lambda1"])
    # the sample mean of lambda_1 within 5 %
    assert abs(l1.mean() / ref.mean() - 1.0) < 0.05, (l1.mean(), ref.mean())
    # orbits whose lambda_1 the oracle reproduces under a 1e-14 change of the
    # initial state (regular ones) agree orbit by orbit
    if "lambda1_perturbed_1e-14" in rec:
        pert = np.asarray(rec["lambda1_perturbed_1e-14"])
        reg = np.abs(pert - ref) <= 1e-9 * np.abs(ref)
        if N == 4:
            assert reg.sum() >= ref.size // 2
        if reg.any():
            assert ind_err(l1[reg], ref[reg]).max() < IND_TOL
    # a Hamiltonian spectrum comes in pairs lambda_i ~ -lambda_{2N+1-i}; with RK4
    # (not volume preserving) the pair sums are small and the GPU's sample means
    # equal the oracle's to well within lambda_1's own spread
    mean = lam.mean(axis=1)
    ref_mean = np.asarray(rec["mean_spectrum"])
    pair = mean + mean[::-1]
    ref_pair = ref_mean + ref_mean[::-1]
    assert np.abs(pair - ref_pair).max() < 0.05 * ref.mean()


# --------------------------------------------------------------------------
# coupled quartic oscillators: uneven end times t_end in [1e3, 1e4], early exit
# --------------------------------------------------------------------------

def test_quartic_full_horizon_labels():
    """A strided sample of the 4,194,304 shell states of the quartic run (eps =
    0.1, E ~ U[1, 10], k = 6 vectors, end steps ~ U[1e5, 1e6] at h = 0.01, early
    exit once SALI < 1e-8), integrated to each orbit's end: the GPU with FP32
    vectors in compacted 500-step chunks, the oracle with FP64 vectors, both
    from the vectors seeded for the sample (seed 3, sample-local indices)."""
    n_all, m = 4_194_304, 2048
    rng = np.random.default_rng(5)
    dirs = rng.standard_normal((6, n_all))
    E = rng.uniform(1.0, 10.0, n_all)
    t_end = rng.integers(100_000, 1_000_001, n_all).astype(np.int64)
    idx = strided_sample(n_all, m)
    ics = O.shell_ics(O.system(O.QUARTIC3, 3, eps=0.1), dirs[:, idx], E[idx])
    te = t_end[idx]
    kw = dict(dt=0.01, n_steps=1_000_000, k=6, ld_p=0.0, sys_params=(0.1,), seed=3, early_exit=True,
              t_end=te)
    g = gpu_run(chs.QUARTIC3, 3, ics, None, vec_fp32=True, compact_chunk=500, **kw)
    r = oracle_run(chs.QUARTIC3, 3, ics, None, **kw)
    rp = oracle_run(chs.QUARTIC3, 3, _one_ulp(ics), None, **kw)
    early = r["status"] == chs.ORBIT_EARLY_CHAOTIC
    assert early.sum() > m // 4
    agree = float((g["label"] == r["label"]).mean())
    assert agree >= LABEL_AGREE, agree
    # statuses decide the labels; a chaotic orbit's stop step moves with rounding
    # (the oracle's one-ulp run stops some chaotic orbits at other checks too),
    # the orbits that run to their end run all of their steps
    assert float((g["status"] == r["status"]).mean()) >= LABEL_AGREE
    ran = (g["status"] == chs.ORBIT_OK) & (r["status"] == chs.ORBIT_OK)
    np.testing.assert_array_equal(g["n_exec"][ran], te[ran])
    np.testing.assert_array_equal(r["n_exec"][ran], te[ran])
    # orbits that ran to their end and are regular: the orbit (FP64 on both sides)
    # against the oracle's one-ulp reproducibility; GALI_2..6 of the FP32 frame
    # against the FP64 oracle
    reg = ran & (rp["status"] == chs.ORBIT_OK) & (r["sali"] > REGULAR_SALI)
    assert reg.sum() >= 50, reg.sum()
    _check_states(g, r, rp, reg)
    _fp32_indicator_errors("quartic", g, r, reg)
