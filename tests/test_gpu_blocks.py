"""Block size (chs_params.block_threads) of the RK4 kernels that offer the choice:
results are bit-identical for every block size, invalid sizes are refused, and
the autotuner picks one of the candidates and caches it."""
import json

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

KEYS = ("x", "w", "ld", "dh_max", "n_exec", "status", "sali", "gali", "label")


def _grid_ics(ny=37, npy=29):
    y0, y1, p0, p1 = hh_section_box(1 / 6)
    return O.grid_ics(1 / 6, y0, y1, ny, p0, p1, npy)


@pytest.mark.parametrize("vec_fp32,persistent", [(False, False), (True, False), (False, True)])
def test_integrate_block_size_is_bit_identical(vec_fp32, persistent):
    ics, st = _grid_ics()
    kw = dict(dt=0.01, n_steps=300, k=4, ld_p=0.5, escape_r2=4.0, vec_fp32=vec_fp32,
              persistent=persistent, early_exit=persistent, sali_threshold=1e-3)
    ref = gpu_run(chs.HENON_HEILES, 2, ics, st, **kw)
    for b in (32, 64, 128):
        out = gpu_run(chs.HENON_HEILES, 2, ics, st, block_threads=b, **kw)
        for key in KEYS:
            np.testing.assert_array_equal(out[key], ref[key])


def test_fput_lyapunov_block_size_is_bit_identical():
    for N in (4, 8, 16, 32, 64):
        n = 45
        Q, P = normal_mode_draws(7 + N, N, n)
        ics = torch.from_numpy(O.fput_mode_ics(O.fput(N), Q, P, np.full(n, 0.1 * N))).cuda()
        S = chs.System(chs.FPUT, N, (1.0, 0.0, 1.0))
        outs = []
        for b in [0] + [b for b in (32, 64, 128) if b >= 2 * N] + ([256] if N == 64 else []):
            lam = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
            sto = torch.empty(n, dtype=torch.int32, device="cuda")
            chs.chs_lyapunov_spectrum(S.h, chs.params(0.05, 60, qr_every=10, block_threads=b), n, ics, None,
                                      lam, sto)
            outs.append((lam.cpu().numpy(), sto.cpu().numpy()))
        for lam, sto in outs[1:]:
            np.testing.assert_array_equal(lam, outs[0][0])
            np.testing.assert_array_equal(sto, outs[0][1])
        S.close()


@pytest.mark.parametrize("N,lanes", [(4, (1, 2, 4)), (8, (2, 4, 8))])
def test_fput_lyapunov_lanes_per_orbit_is_bit_identical(N, lanes):
    """The short chains' kernel with 1, 2 or 4 lanes per orbit (N = 4) or 2, 4
    or 8 (N = 8), at every block size, FPUT-beta and FPUT-alpha+beta, a ragged last
    block and a health check: identical exponents and statuses."""
    n = 45
    Q, P = normal_mode_draws(17 + N, N, n)
    ics = torch.from_numpy(O.fput_mode_ics(O.fput(N), Q, P, np.full(n, 0.1 * N))).cuda()
    for sp in ((1.0, 0.0, 1.0), (1.0, 0.25, 1.0)):
        S = chs.System(chs.FPUT, N, sp)
        outs = []
        for L in (0,) + lanes:
            for b in (0, 32, 64, 128):
                lam = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
                sto = torch.empty(n, dtype=torch.int32, device="cuda")
                chs.chs_lyapunov_spectrum(S.h, chs.params(0.05, 130, qr_every=7, sample_every=20, block_threads=b,
                                                          threads_per_orbit=L), n, ics, None, lam, sto)
                outs.append((lam.cpu().numpy(), sto.cpu().numpy()))
        for lam, sto in outs[1:]:
            np.testing.assert_array_equal(lam, outs[0][0])
            np.testing.assert_array_equal(sto, outs[0][1])
        S.close()


def test_fput_n64_two_threads_per_vector_is_bit_identical():
    """N = 64 with 256 threads per orbit (two per deviation vector) against the
    128-thread body: FPUT-alpha+beta, QR every 7 steps with a last partial
    interval, health checks, and one orbit made NONFINITE: identical exponents
    and statuses."""
    N, n = 64, 7
    Q, P = normal_mode_draws(640, N, n)
    ics = O.fput_mode_ics(O.fput(N), Q, P, np.full(n, 0.1 * N))
    ics[N + 3, 4] = np.nan
    ics = torch.from_numpy(ics).cuda()
    for sp in ((1.0, 0.0, 1.0), (1.0, 0.25, 1.0)):
        S = chs.System(chs.FPUT, N, sp)
        outs = []
        for b in (0, 256, 128):
            lam = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
            sto = torch.empty(n, dtype=torch.int32, device="cuda")
            chs.chs_lyapunov_spectrum(S.h, chs.params(0.05, 130, qr_every=7, sample_every=20, block_threads=b),
                                      n, ics, None, lam, sto)
            outs.append((lam.cpu().numpy(), sto.cpu().numpy()))
        assert outs[0][1][4] == chs.ORBIT_NONFINITE and (outs[0][1] == chs.ORBIT_OK).sum() == n - 1
        for lam, sto in outs[1:]:
            np.testing.assert_array_equal(lam, outs[0][0])
            np.testing.assert_array_equal(sto, outs[0][1])
        S.close()


def test_fput_block_256_only_at_n64():
    for N, integ in ((32, chs.RK4), (32, chs.DOP853), (16, chs.RK4)):
        S = chs.System(chs.FPUT, N, (1.0, 0.0, 1.0))
        ics = torch.zeros((2 * N, 2), dtype=torch.float64, device="cuda")
        lam = torch.empty((2 * N, 2), dtype=torch.float64, device="cuda")
        sto = torch.empty(2, dtype=torch.int32, device="cuda")
        with pytest.raises(chs.ChsError) as e:
            chs.chs_lyapunov_spectrum(S.h, chs.params(0.05, 10, qr_every=10, block_threads=256, integrator=integ),
                                      2, ics, None, lam, sto)
        assert e.value.code == chs.CHS_E_INVALID
        S.close()


def test_fput_dop853_n64_two_threads_per_vector_is_bit_identical():
    """DOP853 at N = 64 with 256 threads per orbit (the default) against the
    128-thread form: FPUT-alpha+beta, QR every 7 steps with a last partial
    interval, health checks, one orbit made NONFINITE: identical exponents and
    statuses."""
    N, n = 64, 5
    Q, P = normal_mode_draws(641, N, n)
    ics = O.fput_mode_ics(O.fput(N), Q, P, np.full(n, 0.1 * N))
    ics[3, 2] = np.nan
    ics = torch.from_numpy(ics).cuda()
    for sp in ((1.0, 0.0, 1.0), (1.0, 0.25, 1.0)):
        S = chs.System(chs.FPUT, N, sp)
        outs = []
        for b in (0, 256, 128):
            lam = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
            sto = torch.empty(n, dtype=torch.int32, device="cuda")
            chs.chs_lyapunov_spectrum(S.h, chs.params(0.05, 45, qr_every=7, sample_every=20, block_threads=b,
                                                      integrator=chs.DOP853), n, ics, None, lam, sto)
            outs.append((lam.cpu().numpy(), sto.cpu().numpy()))
        assert outs[0][1][2] == chs.ORBIT_NONFINITE and (outs[0][1] == chs.ORBIT_OK).sum() == n - 1
        for lam, sto in outs[1:]:
            np.testing.assert_array_equal(lam, outs[0][0])
            np.testing.assert_array_equal(sto, outs[0][1])
        S.close()


def test_fput_lanes_argument_checks():
    S = chs.System(chs.FPUT, 8, (1.0, 0.0, 1.0))
    ics = torch.zeros((16, 4), dtype=torch.float64, device="cuda")
    lam = torch.empty((16, 4), dtype=torch.float64, device="cuda")
    sto = torch.empty(4, dtype=torch.int32, device="cuda")
    for L in (1, 3, 16):
        with pytest.raises(chs.ChsError) as e:
            chs.chs_lyapunov_spectrum(S.h, chs.params(0.05, 10, qr_every=10, threads_per_orbit=L), 4, ics, None,
                                      lam, sto)
        assert e.value.code == chs.CHS_E_UNSUPPORTED
    with pytest.raises(chs.ChsError):
        chs.chs_lyapunov_spectrum(S.h, chs.params(0.05, 10, qr_every=10, threads_per_orbit=2,
                                                  integrator=chs.DOP853), 4, ics, None, lam, sto)
    H = chs.System(chs.FPUT, 16, (1.0, 0.0, 1.0))
    with pytest.raises(chs.ChsError):
        chs.chs_lyapunov_spectrum(H.h, chs.params(0.05, 10, qr_every=10, threads_per_orbit=4), 0, None, None,
                                  None, None)


def test_fput_lanes_autotuner_picks_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("CHS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_2507_00622_gb300 import autotune
    r = autotune.tune_fput_lanes(4, n_orbits=1024, steps=40)
    assert r["threads_per_orbit"] in (1, 2, 4) and r["block_threads"] in (32, 64, 128)
    assert len(r["seconds"]) == 9
    assert autotune.tune_fput_lanes(4, n_orbits=1024, steps=40) == r


def test_block_threads_argument_checks():
    S = chs.System(chs.HENON_HEILES, 2)
    ens = chs.DeviceEnsemble.empty(8, 4, 2)
    with pytest.raises(chs.ChsError) as e:
        chs.chs_integrate_batch(S.h, chs.params(0.01, 5, n_dev=2, block_threads=48), ens.abi())
    assert e.value.code == chs.CHS_E_INVALID
    F = chs.System(chs.FPUT, 32, (1.0, 0.0, 1.0))
    ics = torch.zeros((64, 4), dtype=torch.float64, device="cuda")
    lam = torch.empty((64, 4), dtype=torch.float64, device="cuda")
    sto = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(chs.ChsError) as e:
        chs.chs_lyapunov_spectrum(F.h, chs.params(0.05, 5, block_threads=32), 4, ics, None, lam, sto)
    assert e.value.code == chs.CHS_E_INVALID
    S.close()
    F.close()


def test_block_autotuner_picks_and_caches(tmp_path, monkeypatch):
    from paper_2507_00622_gb300 import autotune
    monkeypatch.setenv("CHS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    r = autotune.tune_block_integrate(k=2, side=64, steps=20)
    assert r["block_threads"] in (32, 64, 128) and set(r["seconds"]) == {"32", "64", "128"}
    f = autotune.tune_fput_block(16, n_orbits=256, steps=20)
    assert f["block_threads"] in (32, 64, 128)
    f32 = autotune.tune_fput_block(32, n_orbits=128, steps=20)
    assert set(f32["seconds"]) == {"64", "128"}
    cache = json.loads((tmp_path / "tune.json").read_text())
    assert len(cache) == 3
    assert autotune.tune_fput_block(16, n_orbits=256, steps=20) == f  # served from the cache
