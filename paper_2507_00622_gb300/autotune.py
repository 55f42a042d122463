"""Autotuner for launch-level parameters, with a JSON cache keyed by the GPU and
the workload.  Every candidate runs through the C ABI on a sample of the workload;
the choice is cached and reused.

Tuned parameters:
- qr_every of the FPUT Lyapunov run.  The QR steps only re-orthonormalise the
  vectors: the accumulated sum of ln R_ii equals the log-diagonal of the R factor
  of the whole propagator product, whatever the interval, so the spectrum changes
  only by rounding.  A longer interval lets the columns drift towards the fastest
  direction (cond(W) ~ exp((lambda_max - lambda_min) q h)), which the
  Gram-Schmidt step must undo.  The tuner keeps the fastest candidate whose
  spectrum matches the reference interval's to `tol` on the sample.
- chunk_steps of compacted runs (chs_integrate_compacted): the fastest candidate
  on a sample grid; short chunks drop finished orbits sooner, long chunks launch
  less often.
- block_threads (threads per block) of the one-orbit-per-thread RK4 integrate
  kernels and of the RK4 FPUT Lyapunov kernel (orbits per block = threads / 2N):
  the fastest of 32, 64 and 128 on a sample.  Results do not depend on the block
  size, so no accuracy guard is needed.  Orbits per thread stay at one in the
  one-orbit-per-thread kernels: a thread holds its orbit's whole joint state in
  registers (168 for Henon-Heiles with four vectors and the LD), and the kernels
  are bound by the FP64 pipe, which a second interleaved orbit per thread could
  not feed any faster.
- threads_per_orbit and block_threads together of the FPUT Lyapunov kernel of
  the short chains (N = 4: 1, 2 or 4 lanes per orbit; N = 8: 2, 4 or 8): fewer lanes
  per orbit do less redundant bond work and exchange less, more lanes give an
  ensemble more warps to spread over the SMs' sub-partitions; the best choice
  depends on the ensemble size.  Results do not depend on either.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np
import torch

from . import chs
from .inputs import hh_section_box, normal_mode_draws


def cache_path() -> str:
    return os.environ.get("CHS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "chs_autotune.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value: dict) -> None:
    d = _load()
    d[key] = value
    os.makedirs(os.path.dirname(cache_path()), exist_ok=True)
    tmp = cache_path() + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1)
    os.replace(tmp, cache_path())


def _gpu() -> str:
    return torch.cuda.get_device_name(torch.cuda.current_device())


def tune_fput_qr(N: int, candidates=(10, 20, 50, 100, 200, 500), reference: int = 10, tol: float = 1e-10,
                 n_orbits: int = 1216, steps: int = 2000, dt: float = 0.05, refresh: bool = False,
                 integrator: str = "rk4") -> dict:
    """Pick qr_every for the FPUT-beta chain of N sites (energy density 0.1) under
    the given integrator ("rk4" or "dop853")."""
    key = f"fput_qr|{_gpu()}|N={N}|ref={reference}|cand={','.join(map(str, candidates))}|tol={tol}"
    if integrator != "rk4":
        key += f"|{integrator}"
    integ = chs.DOP853 if integrator == "dop853" else chs.RK4
    if not refresh:
        hit = _load().get(key)
        if hit:
            return hit
    S = chs.System(chs.FPUT, N, (1.0, 0.0, 1.0))
    Q, P = normal_mode_draws(4242 + N, N, n_orbits)
    ics = torch.empty((2 * N, n_orbits), dtype=torch.float64, device="cuda")
    chs.chs_fput_mode_ics(S.h, n_orbits, torch.from_numpy(Q).cuda(), torch.from_numpy(P).cuda(),
                          torch.full((n_orbits,), 0.1 * N, dtype=torch.float64, device="cuda"), ics)
    lam = {q: torch.empty((2 * N, n_orbits), dtype=torch.float64, device="cuda") for q in candidates}
    st = torch.empty(n_orbits, dtype=torch.int32, device="cuda")
    times = {}
    for q in candidates:
        prm = chs.params(dt, steps, qr_every=q, sample_every=100, integrator=integ)
        chs.chs_lyapunov_spectrum(S.h, prm, n_orbits, ics, None, lam[q], st)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        chs.chs_lyapunov_spectrum(S.h, prm, n_orbits, ics, None, lam[q], st)
        torch.cuda.synchronize()
        times[q] = time.perf_counter() - t0
    ref = lam[reference].cpu().numpy()
    errs = {q: float(np.abs(lam[q].cpu().numpy() - ref).max()) for q in candidates}
    ok = [q for q in candidates if errs[q] <= tol]
    best = min(ok, key=lambda q: times[q])
    out = {"qr_every": int(best), "seconds": {str(q): times[q] for q in candidates},
           "max_abs_diff_vs_ref": {str(q): errs[q] for q in candidates}, "n_orbits": n_orbits,
           "steps": steps}
    _store(key, out)
    return out


def tune_compact_chunk(E: float = 0.125, side: int = 256, steps: int = 100_000, k: int = 2,
                       candidates=(500, 1000, 2000, 5000, 10000), refresh: bool = False) -> dict:
    """Pick chunk_steps for compacted Henon-Heiles grid runs (FP32 frame, early exit)."""
    key = f"compact_chunk|{_gpu()}|E={E}|side={side}|k={k}|cand={','.join(map(str, candidates))}"
    if not refresh:
        hit = _load().get(key)
        if hit:
            return hit
    S = chs.System(chs.HENON_HEILES, 2)
    y0, y1, p0, p1 = hh_section_box(E)
    n = side * side
    ics = torch.empty((4, n), dtype=torch.float64, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    chs.chs_section_grid_ics(S.h, E, y0, y1, side, p0, p1, side, ics, st)
    kw = dict(n_dev=k, ld_p=0.5, escape_r2=4.0, vec_precision=chs.VEC_FP32, early_exit=True)
    work = chs.compact_work(n)
    times = {}
    for c in candidates:
        best = None
        for _ in range(2):
            ens = chs.DeviceEnsemble.empty(n, 4, k, vec_fp32=True)
            abi = ens.abi()
            chs.chs_ensemble_init(S.h, chs.params(0.01, 1, **kw), abi, ics, st)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            chs.chs_integrate_compacted(S.h, chs.params(0.01, steps, **kw), abi, c, work)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        times[c] = best
    choice = min(candidates, key=lambda c: times[c])
    out = {"chunk_steps": int(choice), "seconds": {str(c): times[c] for c in candidates},
           "side": side, "steps": steps}
    _store(key, out)
    return out


def _best_time(fn, reps: int = 2) -> float:
    best = None
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return best


def tune_block_integrate(k: int = 4, ld: bool = True, vec_fp32: bool = False, side: int = 512,
                         steps: int = 200, candidates=(32, 64, 128), refresh: bool = False) -> dict:
    """Pick block_threads of chs_integrate_batch on a Henon-Heiles grid at E = 1/6
    (k vectors, LD p = 1/2 when `ld`)."""
    key = (f"block_integrate|{_gpu()}|k={k}|ld={int(ld)}|fp32={int(vec_fp32)}|side={side}"
           f"|cand={','.join(map(str, candidates))}")
    if not refresh:
        hit = _load().get(key)
        if hit:
            return hit
    E = 1.0 / 6.0
    S = chs.System(chs.HENON_HEILES, 2)
    y0, y1, p0, p1 = hh_section_box(E)
    n = side * side
    ics = torch.empty((4, n), dtype=torch.float64, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    chs.chs_section_grid_ics(S.h, E, y0, y1, side, p0, p1, side, ics, st)
    vp = chs.VEC_FP32 if vec_fp32 else chs.VEC_FP64
    kw = dict(n_dev=k, ld_p=0.5 if ld else 0.0, escape_r2=4.0, vec_precision=vp)
    ens = chs.DeviceEnsemble.empty(n, 4, k, vec_fp32=vec_fp32)
    abi = ens.abi(with_ld=ld)
    chs.chs_ensemble_init(S.h, chs.params(0.01, 1, **kw), abi, ics, st)
    times = {}
    step = 0
    for b in candidates:
        def run():
            nonlocal step
            chs.chs_integrate_batch(S.h, chs.params(0.01, steps, step0=step, block_threads=b, **kw), abi)
            step += steps
        run()  # warm-up
        times[b] = _best_time(run)
    choice = min(candidates, key=lambda b: times[b])
    out = {"block_threads": int(choice), "seconds": {str(b): times[b] for b in candidates},
           "side": side, "steps": steps}
    _store(key, out)
    return out


def tune_fput_block(N: int, qr_every: int = 10, n_orbits: int = 4096, steps: int = 200,
                    refresh: bool = False) -> dict:
    """Pick block_threads of the RK4 FPUT Lyapunov kernel for chains of N sites
    (every multiple of 2N among 32, 64, 128; at N = 64 also 256, two threads per
    vector)."""
    cands = [b for b in (32, 64, 128) if b >= 2 * N] + ([256] if N == 64 else [])
    key = f"block_fput|{_gpu()}|N={N}|qr={qr_every}|n={n_orbits}|cand={','.join(map(str, cands))}"
    if not refresh:
        hit = _load().get(key)
        if hit:
            return hit
    S = chs.System(chs.FPUT, N, (1.0, 0.0, 1.0))
    Q, P = normal_mode_draws(4343 + N, N, n_orbits)
    ics = torch.empty((2 * N, n_orbits), dtype=torch.float64, device="cuda")
    chs.chs_fput_mode_ics(S.h, n_orbits, torch.from_numpy(Q).cuda(), torch.from_numpy(P).cuda(),
                          torch.full((n_orbits,), 0.1 * N, dtype=torch.float64, device="cuda"), ics)
    lam = torch.empty((2 * N, n_orbits), dtype=torch.float64, device="cuda")
    st = torch.empty(n_orbits, dtype=torch.int32, device="cuda")
    times = {}
    for b in cands:
        prm = chs.params(0.05, steps, qr_every=qr_every, sample_every=100, block_threads=b)
        run = lambda: chs.chs_lyapunov_spectrum(S.h, prm, n_orbits, ics, None, lam, st)  # noqa: E731
        run()  # warm-up
        times[b] = _best_time(run)
    choice = min(cands, key=lambda b: times[b])
    out = {"block_threads": int(choice), "seconds": {str(b): times[b] for b in cands},
           "n_orbits": n_orbits, "steps": steps}
    _store(key, out)
    return out


def tune_fput_lanes(N: int, qr_every: int = 10, n_orbits: int = 4096, steps: int = 200,
                    refresh: bool = False) -> dict:
    """Pick threads_per_orbit and block_threads of the RK4 FPUT Lyapunov kernel of
    the short chains (N = 4: 1, 2, 4 lanes per orbit; N = 8: 2, 4, 8) on an ensemble
    of n_orbits, measuring every pair with the block sizes 32, 64 and 128."""
    lanes = {4: (1, 2, 4), 8: (2, 4, 8)}[N]
    blocks = (32, 64, 128)
    key = f"lanes_fput|{_gpu()}|N={N}|qr={qr_every}|n={n_orbits}"
    if not refresh:
        hit = _load().get(key)
        if hit:
            return hit
    S = chs.System(chs.FPUT, N, (1.0, 0.0, 1.0))
    Q, P = normal_mode_draws(4444 + N, N, n_orbits)
    ics = torch.empty((2 * N, n_orbits), dtype=torch.float64, device="cuda")
    chs.chs_fput_mode_ics(S.h, n_orbits, torch.from_numpy(Q).cuda(), torch.from_numpy(P).cuda(),
                          torch.full((n_orbits,), 0.1 * N, dtype=torch.float64, device="cuda"), ics)
    lam = torch.empty((2 * N, n_orbits), dtype=torch.float64, device="cuda")
    st = torch.empty(n_orbits, dtype=torch.int32, device="cuda")
    times = {}
    for L in lanes:
        for b in blocks:
            prm = chs.params(0.05, steps, qr_every=qr_every, sample_every=100, block_threads=b,
                             threads_per_orbit=L)
            run = lambda: chs.chs_lyapunov_spectrum(S.h, prm, n_orbits, ics, None, lam, st)  # noqa: E731
            run()  # warm-up
            times[(L, b)] = _best_time(run)
    L, b = min(times, key=times.get)
    out = {"threads_per_orbit": int(L), "block_threads": int(b),
           "seconds": {f"{k[0]}x{k[1]}": v for k, v in times.items()}, "n_orbits": n_orbits, "steps": steps}
    _store(key, out)
    return out
