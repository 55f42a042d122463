"""Throughput bench of the chaos-indicator hot path on GB300.

Workload (the Henon-Heiles grid run): E = 1/6, 1024 x 1024 cell-centred grid of
(y, p_y) on the x = 0 section, p_x >= 0 from the energy, FP64 classic RK4 with
h = 0.01, k = 4 deviation vectors renormalised every step, LD (p = 1/2), SALI,
GALI_2..4, LD indicators and labels.  One bench step advances the whole grid by
`--chunk` RK4 steps (continuing the same run from the previous step, so the
timed steps cover a window of the t = 1e4 integration) and then evaluates every
indicator on the new state: each step runs every stage of the hot path.

Prints one JSON line (rank 0).  Beside the headline, the line carries the other
configurations, each with its roofline and CPU baseline (skip with --no-extra):
the same grid with FP32 deviation vectors (`fp32_vectors`), the FPUT-beta
Lyapunov spectra for N = 4 .. 64 at QR every 10 steps and at the tuned interval
(`fput_lyapunov_qr10`, `fput_lyapunov_qr_tuned`), the coupled quartic
oscillators (`quartic`), and the time to classify the 1024 x 1024 grid at
E = 1/8 by the plain and the fast forms (`classify`; --classify-side 0 skips it).
`--impl reference` times the CPU oracle on a bounded sample of the same workload
instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("orbit-steps/sec and % FP64 roofline; time-to-classified-grid vs plain at "
          "≥99.5% agreement")
UNIT = "orbit-steps/s"
E_GRID = 1.0 / 6.0
DT = 0.01
K_DEV = 4
SM_COUNT = 152
FP64_FLOP_PER_CLK_SM = 4  # 2 DFMA lanes per SM per clock (measured 1.20 TFLOP/s at ~1.99 GHz)


# DRAM traffic of one k_integrate<HenonHeiles,4,LD> launch over the 1024 x 1024 grid
# (dram__bytes_read.sum + dram__bytes_write.sum from one ncu capture; a launch reads
# and writes the ensemble state once whatever its step count), valid while the
# kernel sources hash to the recorded value.
TRAFFIC_SOURCES = ("k_small.cu", "rk4_common.cuh", "fastmath.cuh", "systems.cuh", "chs_internal.cuh")
TRAFFIC_RECORD = {"sha256_16": "dc5c5bf95608332b", "bytes_per_launch": 146702848.0 + 78981888.0,
                  "n_side": 1024}


def recorded_traffic(n_side: int, vec_fp32: bool):
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2507_00622_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if vec_fp32 or n_side != TRAFFIC_RECORD["n_side"] or h.hexdigest()[:16] != TRAFFIC_RECORD["sha256_16"]:
        return None
    return TRAFFIC_RECORD["bytes_per_launch"]


def grid_box(E: float):
    """Energy-allowed (y, p_y) box of the x = 0 section at E = 1/6."""
    return -0.5, 1.0, -float(np.sqrt(2 * E)), float(np.sqrt(2 * E))


def flops_per_orbit_step(k: int, ld: bool, vec_fp32: bool) -> tuple[int, int]:
    """Algorithmic flops of one RK4 step of the Henon-Heiles joint system
    (FMA = 2, sqrt and rsqrt = 1), as (FP64 flops, FP32 flops).
    Orbit (FP64): per stage f and Hess V 10, LD 7 (4 sqrt + 3 add); stage
      inputs 2 per component (3 stages); accumulation 7 per component of
      (x, L); escape test 3.
    FP64 vectors (direct RK4, as the oracle computes them): variational 6 per
      vector and stage, stage inputs 2 per component (3 stages), accumulation
      7 per component, renormalisation 12 per vector.
    FP32 frame: propagator blocks 104, application 32 per vector, Gram-Schmidt
      16 per vector pair and 13 per vector, triangle update and normalisation
      74 (for k = 4); the LD integrand (7 per stage) is summed in FP32 there, and
      the stage Hessians (3 of the 10 per stage) are formed in FP32."""
    xs = 4 * (10 + (7 if ld else 0)) + 3 * 2 * 4 + 7 * (4 + (1 if ld else 0)) + 3
    if vec_fp32:
        tri = sum(2 * (j - i + 1) for j in range(k) for i in range(j + 1))
        nr = k * (k + 1) // 2
        vs = 104 + 32 * k + 16 * k * (k - 1) // 2 + 13 * k + tri + 2 * nr + k + nr
        moved = (4 * 7 if ld else 0) + 4 * 3
        return xs - moved, vs + moved
    vs = 4 * 6 * k + 3 * 2 * 4 * k + 7 * 4 * k + 12 * k
    return xs + vs, 0


def dp_flops_per_orbit_step(k: int, ld: bool) -> int:
    """Algorithmic FP64 flops of one DOP853 step of the Henon-Heiles joint system,
    counted like the RK4 figure (FMA = 2, sqrt and rsqrt = 1).  The tableau has
    50 nonzero a_sj over the 11 stage inputs and 8 nonzero b_s.
    Orbit: per stage f and Hess V 10 (12 stages); LD 7 at the 8 stages with
      b_s != 0; stage inputs 2 per nonzero a_sj plus 2 for x + h * sum, per
      component; accumulation 17 per component of (x, L) (7 FMA + 1 mul for
      sum_s b_s K_s, then x + h * sum); escape test 3.
    Vectors: variational 6 per stage, stage inputs as for the orbit,
      accumulation 17 per component, renormalisation 12."""
    inputs = (50 * 2 + 11 * 2) * 4
    xs = 12 * 10 + (8 * 7 if ld else 0) + inputs + 17 * (4 + (1 if ld else 0)) + 3
    vs = 12 * 6 + inputs + 17 * 4 + 12
    return xs + k * vs


def fp64_peak_tflops(sm_mhz: float) -> float:
    """The formula FP64 peak: 152 SMs x 2 DFMA lanes per clock x 2 flops."""
    return SM_COUNT * FP64_FLOP_PER_CLK_SM * sm_mhz * 1e6 / 1e12


def probe_rate(kind: int, n_blocks: int, n_threads: int, n_iter: int, reps: int = 5) -> dict:
    """Best-of-reps rate of one pipe probe (chs_peak_probe), timed with CUDA
    events on the launching stream after one untimed launch: operations per
    second (flops for the FMA and MMA probes, square roots for the sqrt probe)."""
    import torch

    from paper_2507_00622_gb300 import chs

    sink = torch.empty(n_blocks * n_threads, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    chs.chs_peak_probe(kind, n_blocks, n_threads, n_iter, sink, stream)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        chs.chs_peak_probe(kind, n_blocks, n_threads, n_iter, sink, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    ops = chs.chs_probe_ops_per_thread(kind, n_iter) * n_blocks * n_threads
    return {"ops_per_s": ops / (best / 1e3), "ms": best, "blocks": n_blocks, "threads": n_threads,
            "n_iter": n_iter}


def measured_fp64_peak(sm_count: int) -> dict:
    """The FP64 FMA peak measured by the DFMA probe (8 independent chains per
    thread, 32 warps per SM), with the SM clock sampled while it ran."""
    from paper_2507_00622_gb300 import chs

    clocks = ClockSampler(None)
    clocks.start()
    r = probe_rate(chs.PROBE_DFMA, sm_count * 4, 256, 1 << 17)
    clk = clocks.stop()
    return {"tflops": r["ops_per_s"] / 1e12, "sm_mhz": clk["sm_mhz"], "ms": r["ms"],
            "probe": f"DFMA, {sm_count * 4} x 256 threads x 8 chains x {r['n_iter']} iterations, best of 5"}


def measured_fp32_peak(sm_count: int) -> dict:
    """The FP32 FMA peak measured by the FFMA probe (8 independent chains per
    thread, 32 warps per SM), with the SM clock sampled while it ran."""
    from paper_2507_00622_gb300 import chs

    clocks = ClockSampler(None)
    clocks.start()
    r = probe_rate(chs.PROBE_FFMA, sm_count * 4, 256, 1 << 21)
    clk = clocks.stop()
    return {"tflops": r["ops_per_s"] / 1e12, "sm_mhz": clk["sm_mhz"],
            "probe": f"FFMA, {sm_count * 4} x 256 threads x 8 chains x {r['n_iter']} iterations, best of 5"}


def grid_fp32_result(steps: int, warmup: int, chunk: int, fp64_peak: dict, n_side: int = 1024) -> dict:
    """The Henon-Heiles grid run with FP32 deviation vectors (the second run of
    the E = 1/6 workload): the same grid, k = 4, LD, RK4 h = 0.01, `chunk` steps
    per bench step plus the indicators; orbit-steps/s and the roofline fractions
    of the integrate kernel on the FP64 pipe (orbit, energy, LD) and on the FP32
    pipe (the vector frame) against the measured peaks."""
    import torch

    from paper_2507_00622_gb300 import chs

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f32_peak = measured_fp32_peak(sms)
    n = n_side * n_side
    y0, y1, p0, p1 = grid_box(E_GRID)
    S = chs.System(chs.HENON_HEILES, 2)
    ics = torch.empty((4, n), dtype=torch.float64, device="cuda")
    ic_st = torch.empty(n, dtype=torch.int32, device="cuda")
    chs.chs_section_grid_ics(S.h, E_GRID, y0, y1, n_side, p0, p1, n_side, ics, ic_st)
    kw = dict(n_dev=K_DEV, ld_p=0.5, escape_r2=4.0, sample_every=100, seed=1, vec_precision=chs.VEC_FP32)
    ens = chs.DeviceEnsemble.empty(n, 4, K_DEV, True)
    abi = ens.abi()
    chs.chs_ensemble_init(S.h, chs.params(DT, 1, **kw), abi, ics, ic_st)
    sali = torch.empty(n, dtype=torch.float64, device="cuda")
    gali = torch.empty((K_DEV - 1, n), dtype=torch.float64, device="cuda")
    label = torch.empty(n, dtype=torch.int8, device="cuda")
    ldi = torch.empty((2, n), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    step = 0
    kev = []

    def one(timed):
        nonlocal step
        prm = chs.params(DT, chunk, step0=step, **kw)
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record(stream)
        chs.chs_integrate_batch(S.h, prm, abi, stream)
        ev[1].record(stream)
        chs.chs_indicators(S.h, prm, abi, n_side, n_side, sali, gali, ldi, label, stream)
        if timed:
            kev.append(ev)
        step += chunk

    for _ in range(warmup):
        one(False)
    torch.cuda.synchronize()
    e0 = int(ens.n_exec.sum())
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        one(True)
    t1.record(stream)
    torch.cuda.synchronize()
    total_ms = t0.elapsed_time(t1)
    kern_ms = float(np.mean([a.elapsed_time(b) for a, b in kev]))
    done = int(ens.n_exec.sum()) - e0
    f64, f32 = flops_per_orbit_step(K_DEV, True, True)
    per_launch = done / steps
    a64 = f64 * per_launch / (kern_ms / 1e3) / 1e12
    a32 = f32 * per_launch / (kern_ms / 1e3) / 1e12
    S.close()
    return {"workload": f"henon_heiles_E1/6_grid{n_side}x{n_side}_k4_sali_gali2-4_ld_rk4_fp32vectors",
            "value": done / (total_ms / 1e3), "unit": UNIT, "steps": steps, "warmup": warmup,
            "steps_per_bench_step": chunk, "ms_per_step": total_ms / steps, "dtype": "f64 orbit + f32 frame",
            "roofline": {"kernel": "k_integrate_f32<HenonHeiles,4,LD>", "kernel_ms_avg": kern_ms,
                         "flops_per_orbit_step": {"fp64": f64, "fp32": f32},
                         "fp64": {"achieved": a64, "peak": fp64_peak["tflops"], "frac": a64 / fp64_peak["tflops"],
                                  "unit": "TFLOP/s"},
                         "fp32": {"achieved": a32, "peak": f32_peak["tflops"], "frac": a32 / f32_peak["tflops"],
                                  "unit": "TFLOP/s", "peak_basis": "measured: " + f32_peak["probe"]}},
            "cpu_baseline_note": "the oracle integrates FP64 vectors only: the headline line's cpu_baseline "
                                 "is this workload's CPU baseline too"}


def shard_rows(ny: int, rank: int, world: int) -> tuple[int, int, int, int]:
    """Weak scaling: every rank owns `ny` grid rows of a (world * ny)-row grid.
    Returns (first_row, n_rows, halo_lo, halo_hi) of the slab it integrates,
    with one extra row on each side that has a neighbour rank, so the LD
    stencil of every owned cell is complete without any exchange."""
    lo = rank * ny
    halo_lo = 1 if rank > 0 else 0
    halo_hi = 1 if rank < world - 1 else 0
    return lo - halo_lo, ny + halo_lo + halo_hi, halo_lo, halo_hi


def slab_bounds(y0: float, y1: float, ny: int, rank: int, world: int):
    """y-range, row count and owned-row slice of rank's slab of the (world*ny)-row grid."""
    dyg = (y1 - y0) / (ny * world)
    first, rows, hlo, hhi = shard_rows(ny, rank, world)
    return y0 + first * dyg, y0 + (first + rows) * dyg, rows, hlo


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.proc = None
        self.uuid = uuid

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_oracle_sample(chunk: int, budget_s: float, n_sample: int = 4096, ny: int = 1024,
                      integrator: str = "rk4"):
    """The oracle as it stands on the host cores: a strided sample of valid cells of
    the same grid, integrated chunk by chunk until `budget_s` of CPU time."""
    import oracle as O
    from paper_2507_00622_gb300.inputs import strided_sample

    y0, y1, p0, p1 = grid_box(E_GRID)
    ics, st = O.grid_ics(E_GRID, y0, y1, ny, p0, p1, ny)
    valid = np.where(st == 0)[0]
    idx = valid[strided_sample(valid.size, n_sample)]
    kw = dict(n_dev=K_DEV, ld_p=0.5, escape_r2=4.0, sample_every=100,
              integrator=O.DOP853 if integrator == "dop853" else O.RK4)
    w = O.seed_vectors(1, ics.shape[1], K_DEV, 4)[:, idx]
    ens = O.Ensemble(O.henon_heiles(), O.params(DT, 1, **kw), ics[:, idx], st[idx], w_in=w)
    done, step, t0 = 0, 0, time.perf_counter()
    while True:
        before = int(ens.n_exec.sum())
        ens.integrate(O.params(DT, chunk, step0=step, **kw))
        ens.indicators()
        O.ld_indicators(1, idx.size, ens.ld, ens.status)
        done += int(ens.n_exec.sum()) - before
        step += chunk
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": done / el, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
            "sample": f"{idx.size} strided valid cells of the 1024x1024 E=1/6 grid, k=4, LD, "
                      f"{step} {integrator.upper()} steps from t=0 ({done} orbit-steps in {el:.1f} s)"}


def cpu_fput_sample(Ns, chunk: int, qr: dict, budget_s: float, integrator: str = "rk4",
                    n_sample: int = 64):
    """The oracle on the host cores for the FPUT Lyapunov workload: n_sample
    orbits per chain length (the bench's first draws), each chain length given
    an equal share of budget_s, integrated chunk by chunk (fresh runs of `chunk`
    steps from the initial conditions) until its share is spent; the rate is
    that of the bench's mix (equal orbit-steps per chain length)."""
    import oracle as O
    from paper_2507_00622_gb300.inputs import normal_mode_draws

    inv_rate, parts = 0.0, []
    for N in Ns:
        Q, P = normal_mode_draws(1000 + N, N, n_sample)
        ics = O.fput_mode_ics(O.fput(N), Q, P, np.full(n_sample, 0.1 * N))
        prm = O.params(0.05, chunk, qr_every=qr[N], sample_every=100,
                       integrator=O.DOP853 if integrator == "dop853" else O.RK4)
        t0 = time.perf_counter()
        runs = 0
        while True:
            O.lyapunov(O.fput(N), prm, ics)
            runs += 1
            if time.perf_counter() - t0 >= budget_s / len(Ns):
                break
        el = time.perf_counter() - t0
        inv_rate += el / (runs * n_sample * chunk)
        parts.append(f"N={N}: {runs} x {n_sample} orbits x {chunk} steps in {el:.1f} s")
    # the bench's mix: the same number of orbit-steps for every chain length
    return {"value": len(Ns) / inv_rate, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
            "sample": "; ".join(parts) + " (rate of an equal mix of orbit-steps per N)"}


def cpu_quartic_sample(chunk: int, budget_s: float, n_sample: int = 16384):
    """The oracle on the host cores for the quartic-3 workload: a strided sample of
    the bench's shell states with FP64 vectors (the oracle's precision), k = 6,
    early exit, their own end steps, integrated chunk by chunk until budget_s."""
    import oracle as O
    from paper_2507_00622_gb300.inputs import strided_sample

    n = 4_194_304
    rng = np.random.default_rng(5)
    dirs = rng.standard_normal((6, n))
    E = rng.uniform(1.0, 10.0, n)
    t_end = rng.integers(100_000, 1_000_001, n).astype(np.int64)
    idx = strided_sample(n, n_sample)
    sysd = O.system(O.QUARTIC3, 3, eps=0.1)
    ics = O.shell_ics(sysd, dirs[:, idx], E[idx])
    kw = dict(n_dev=6, ld_p=0.0, sample_every=100, early_exit=True)
    ens = O.Ensemble(sysd, O.params(0.01, 1, **kw), ics, seed=3)
    done, step, t0 = 0, 0, time.perf_counter()
    while True:
        before = int(ens.n_exec.sum())
        ens.integrate(O.params(0.01, chunk, step0=step, **kw), t_end=t_end[idx])
        ens.indicators()
        done += int(ens.n_exec.sum()) - before
        step += chunk
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": done / el, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
            "sample": f"{n_sample} strided shell states, k = 6 FP64 vectors, {step} RK4 steps "
                      f"({done} orbit-steps in {el:.1f} s)"}


def run_peaks(args):
    """Pipe peaks on this GPU (chs_peak_probe, CUDA events, best of 5): FP64 FMA,
    FP32 FMA, FP64 sqrt and FP64 mma.sync m8n8k4 at 32 warps per SM; the FP64 FMA
    rate against warps per SM (one warp per block, 8 independent chains per
    thread); and the dependent FP64 FMA latency (one chain, one warp per SM)."""
    import torch

    from paper_2507_00622_gb300 import build as cuda_build
    from paper_2507_00622_gb300 import chs

    cuda_build.build()
    chs.load()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clocks = ClockSampler(None)
    clocks.start()
    time.sleep(0.3)
    full = {"dfma": probe_rate(chs.PROBE_DFMA, sms * 4, 256, 1 << 17),
            "ffma": probe_rate(chs.PROBE_FFMA, sms * 4, 256, 1 << 21),
            "dsqrt": probe_rate(chs.PROBE_DSQRT, sms * 4, 256, 1 << 12),
            "dmma": probe_rate(chs.PROBE_DMMA, sms * 4, 256, 1 << 14),
            "dfma_dmma": probe_rate(chs.PROBE_DFMA_DMMA, sms * 4, 256, 1 << 15)}
    sweep = []
    for w in (1, 2, 3, 4, 6, 8, 12, 16, 32):
        r = probe_rate(chs.PROBE_DFMA, sms * w, 32, max(4096, (1 << 20) // w))
        sweep.append({"warps_per_sm": w, "tflops": r["ops_per_s"] / 1e12, "ms": r["ms"]})
    dep = probe_rate(chs.PROBE_DFMA_DEP, sms, 32, 1 << 18)
    dep4 = probe_rate(chs.PROBE_DFMA_DEP, sms * 4, 32, 1 << 18)
    clk = clocks.stop()
    mhz = clk["sm_mhz"] or 2070.0
    line = {"workload": "pipe_peaks", "sms": sms, "clocks": clk,
            "fp64_fma_tflops": full["dfma"]["ops_per_s"] / 1e12,
            "fp32_fma_tflops": full["ffma"]["ops_per_s"] / 1e12,
            "fp64_sqrt_per_s": full["dsqrt"]["ops_per_s"],
            "fp64_mma_m8n8k4_tflops": full["dmma"]["ops_per_s"] / 1e12,
            # FMA and MMA interleaved in one kernel: the sum stays at either's rate
            # when the two share the FP64 pipe
            "fp64_fma_plus_mma_tflops": full["dfma_dmma"]["ops_per_s"] / 1e12,
            "fp64_formula_tflops": fp64_peak_tflops(mhz),
            "fp64_fma_lanes_per_sm_per_clock": full["dfma"]["ops_per_s"] / 2 / (sms * mhz * 1e6),
            "fp64_vs_warps_per_sm": sweep,
            "fp64_dependent_fma_cycles": {
                "1_warp_per_sm": dep["ms"] * 1e-3 * mhz * 1e6 / dep["n_iter"],
                "4_warps_per_sm": dep4["ms"] * 1e-3 * mhz * 1e6 / dep4["n_iter"]},
            "probes": full}
    print(json.dumps(line))
    return 0


def run_mlp(args):
    """The surrogate's kernels on 1,048,576 orbits (the 1024 x 1024 grid): the
    fused forward pass (chs_mlp_forward) and the decision (chs_surrogate_decide:
    features, forward, status update), timed with CUDA events (best of 5 after a
    warm-up), with their multiply-add rate against the measured FP32 FMA peak
    (the perceptron runs on the FP32 pipe with BF16 operands)."""
    import torch

    from paper_2507_00622_gb300 import build as cuda_build
    from paper_2507_00622_gb300 import chs
    from paper_2507_00622_gb300 import surrogate as SG

    cuda_build.build()
    chs.load()
    n = 1 << 20
    rng = np.random.default_rng(11)
    sur = SG.Surrogate.load()
    X = torch.from_numpy(rng.standard_normal((12, n)).astype(np.float32)).cuda()
    Y = torch.empty((2, n), dtype=torch.float32, device="cuda")
    series = torch.from_numpy(10.0 ** rng.uniform(-12, 0, (10, n))).cuda()
    ld = torch.from_numpy(rng.uniform(400.0, 700.0, n)).cuda()
    E = torch.full((n,), 0.125, dtype=torch.float64, device="cuda")
    status = torch.zeros(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def best(fn):
        fn()
        torch.cuda.synchronize()
        t = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            t.append(a.elapsed_time(b))
        return min(t)

    fwd_ms = best(lambda: chs.chs_mlp_forward(sur.params, X, n, Y))

    def decide():
        status.zero_()
        chs.chs_surrogate_decide(sur.params, series, 10, ld, 500.0, E, 0.98, n, status)

    dec_ms = best(decide)
    macs = 12 * 128 + 128 * 128 + 128 * 128 + 128 * 2  # per orbit
    f32 = measured_fp32_peak(torch.cuda.get_device_properties(0).multi_processor_count)
    tf = 2.0 * macs * n / (fwd_ms / 1e3) / 1e12
    print(json.dumps({"workload": "surrogate_mlp_12-128-128-128-2_bf16", "n_orbits": n,
                      "forward_ms": fwd_ms, "decide_ms": dec_ms, "macs_per_orbit": macs,
                      "forward_tflops": tf, "fp32_fma_peak_tflops": f32["tflops"],
                      "frac_of_fp32_peak": tf / f32["tflops"]}))
    return 0


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle as O
    O.build()
    t_all = []
    res = None
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_sample(args.chunk, 0.0, n_sample=args.ref_sample, integrator=args.integrator)
        if i >= args.warmup:
            t_all.append(r["value"])
            res = r
    value = float(np.mean(t_all))
    ms = 1e3 * args.ref_sample * args.chunk / value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "henon_heiles_E1/6_grid1024x1024_k4_sali_gali2-4_ld_" + args.integrator,
                       "sample_per_step": f"{args.ref_sample} strided valid cells x {args.chunk} steps"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": res["cores"], "kind": "oracle",
                             "sample": res["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import torch

    from paper_2507_00622_gb300 import build as cuda_build
    from paper_2507_00622_gb300 import chs

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if rank == 0:
        cuda_build.build()
    if world > 1:
        dist.barrier()
    chs.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    ny = npy = args.n_side
    y0, y1, p0, p1 = grid_box(E_GRID)
    sy0, sy1, rows, hlo = slab_bounds(y0, y1, ny, rank, world)
    n = rows * npy
    own = slice(hlo * npy, (hlo + ny) * npy)
    vec_fp32 = args.vec == "fp32"
    vp = chs.VEC_FP32 if vec_fp32 else chs.VEC_FP64
    S = chs.System(chs.HENON_HEILES, 2)
    ics = torch.empty((4, n), dtype=torch.float64, device=dev)
    ic_st = torch.empty(n, dtype=torch.int32, device=dev)
    chs.chs_section_grid_ics(S.h, E_GRID, sy0, sy1, rows, p0, p1, npy, ics, ic_st)
    dop = args.integrator == "dop853"
    if dop and vec_fp32:
        raise SystemExit("DOP853 runs with FP64 deviation vectors only")
    block = 0
    if not dop and args.block == "auto":
        from paper_2507_00622_gb300 import autotune
        block = autotune.tune_block_integrate(k=K_DEV, ld=True, vec_fp32=vec_fp32)["block_threads"]
    elif not dop:
        block = int(args.block)
    kw = dict(n_dev=K_DEV, ld_p=0.5, escape_r2=4.0, sample_every=100, seed=1 + rank,
              vec_precision=vp, sali_threshold=1e-8, integrator=chs.DOP853 if dop else chs.RK4,
              block_threads=block)
    ens = chs.DeviceEnsemble.empty(n, 4, K_DEV, vec_fp32, device=dev)
    abi = ens.abi()
    chs.chs_ensemble_init(S.h, chs.params(DT, 1, **kw), abi, ics, ic_st)
    sali = torch.empty(n, dtype=torch.float64, device=dev)
    gali = torch.empty((K_DEV - 1, n), dtype=torch.float64, device=dev)
    label = torch.empty(n, dtype=torch.int8, device=dev)
    ldi = torch.empty((2, n), dtype=torch.float64, device=dev)
    step = 0

    def one_step(ev=None):
        nonlocal step
        prm = chs.params(DT, args.chunk, step0=step, **kw)
        if ev is not None:
            ev[0].record(stream)
        chs.chs_integrate_batch(S.h, prm, abi, stream)
        if ev is not None:
            ev[1].record(stream)
        chs.chs_indicators(S.h, prm, abi, rows, npy, sali, gali, ldi, label, stream)
        step += args.chunk

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    exec0 = int(ens.n_exec[own].sum())
    t_window0 = step * DT

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid).replace("GPU-", "")
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.5)
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    for i in range(args.steps):
        one_step(kev[i])
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = t0.elapsed_time(t1)
    kern_ms = float(np.mean([a.elapsed_time(b) for a, b in kev]))
    exec1 = int(ens.n_exec[own].sum())
    orbit_steps = exec1 - exec0
    t_window1 = step * DT

    # end to end through the C ABI from pinned host buffers: every step uploads the
    # whole ensemble state, integrates, evaluates the indicators and reads back the
    # state and every indicator
    host = {k: getattr(ens, k).cpu().pin_memory() for k in ("x", "w", "ld", "h0", "dh_max", "n_exec",
                                                             "status")}
    outs = [sali, gali, label, ldi]
    host_out = [t.cpu().pin_memory() for t in outs]
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = h2d + sum(t.numel() * t.element_size() for t in host_out)
    e2e_steps = max(1, args.e2e_steps)
    e_exec0 = int(host["n_exec"][own].sum())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        for k, t in host.items():
            getattr(ens, k).copy_(t, non_blocking=True)
        one_step()
        for k, t in host.items():
            t.copy_(getattr(ens, k), non_blocking=True)
        for src, dst in zip(outs, host_out):
            dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - w0
    e_orbit_steps = int(host["n_exec"][own].sum()) - e_exec0

    if world > 1:
        t = torch.tensor([total_ms, e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        c = torch.tensor([orbit_steps, e_orbit_steps], dtype=torch.int64, device=dev)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        total_ms, e2e_s = float(t[0]), float(t[1])
        orbit_steps, e_orbit_steps = int(c[0]), int(c[1])

    if rank == 0:
        value = orbit_steps / (total_ms / 1e3)
        if dop:
            f64, f32 = dp_flops_per_orbit_step(K_DEV, True), 0
        else:
            f64, f32 = flops_per_orbit_step(K_DEV, True, vec_fp32)
        per_launch_steps = (exec1 - exec0) / args.steps
        achieved = f64 * per_launch_steps / (kern_ms / 1e3) / 1e12
        peak_mhz = clk["sm_max_mhz"] or 2070.0
        formula = fp64_peak_tflops(peak_mhz)
        mp = measured_fp64_peak(torch.cuda.get_device_properties(local).multi_processor_count)
        # the probe's rate at the clock the timed region ran at
        scale = (clk["sm_mhz"] / mp["sm_mhz"]) if (clk["sm_mhz"] and mp["sm_mhz"]) else 1.0
        peak = mp["tflops"] * scale
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if not vec_fp32 else "f64+f32",
            "data": "synthetic",
            "config": {"workload": "henon_heiles_E1/6_grid1024x1024_k4_sali_gali2-4_ld_"
                                   + ("dop853" if dop else "rk4"),
                       "grid_per_gpu": [ny, npy], "n_orbits_per_gpu": ny * npy, "dt": DT,
                       "integrator": "DOP853 (fixed step)" if dop else "RK4",
                       "steps_per_bench_step": args.chunk,
                       "block_threads": None if dop else (block or 128),
                       "t_window": [t_window0, t_window1], "t_end_of_full_run": 1e4,
                       "deviation_vectors": f"{K_DEV} x {'fp32' if vec_fp32 else 'fp64'}",
                       "l2": "inputs larger than L2: ensemble state %.0f MB per GPU" %
                             (h2d / 1e6),
                       "parallelism": f"orbit-range shards x{world}, no data-path collective"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": None if dop or block not in (0, 128) else recorded_traffic(ny, vec_fp32),
                         "kernel": "k_integrate_dp<HenonHeiles,4,LD>" if dop else
                                   "k_integrate<HenonHeiles,4,LD>",
                         "flops_per_orbit_step": {"fp64": f64, "fp32": f32},
                         "flops_basis": "algorithmic count of the method as the oracle computes it "
                                        "(direct stage-wise RK4 on orbit, vectors and LD; FMA = 2, "
                                        "sqrt = 1); the RK4 kernel executes the vectors by the "
                                        "equivalent one-step propagator and fewer FP64 instructions",
                         "peak_basis": f"measured: FP64 FMA probe {mp['tflops']:.4f} TFLOP/s at "
                                       f"{mp['sm_mhz']} MHz, scaled to the timed region's median "
                                       f"{clk['sm_mhz']} MHz (x{scale:.4f}); {mp['probe']}",
                         "peak_formula": formula,
                         "peak_formula_basis": f"152 SMs x 2 DFMA/clk x 2 flop x {peak_mhz:.0f} MHz",
                         "frac_of_formula": achieved / formula,
                         "kernel_ms_avg": kern_ms},
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                       "reasons": clk["reasons"]},
            "e2e": {"value": e_orbit_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d * world,
                    "d2h_bytes_per_step": d2h * world},
            "gpu_launches": 3 * args.steps,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_oracle_sample(args.chunk, args.cpu_budget,
                                                     integrator=args.integrator)
        if world == 1 and not args.no_extra:
            # the other configurations, each with its own roofline and CPU baseline
            line["fp32_vectors"] = grid_fp32_result(3, 2, args.chunk, mp)
            fa = argparse.Namespace(**vars(args))
            fa.chunk, fa.steps, fa.warmup, fa.integrator, fa.block, fa.fput_batch = 200, 3, 2, "rk4", "0", False
            fa.cpu_budget = min(args.cpu_budget, 6.0)
            fa.qr_every = "10"
            line["fput_lyapunov_qr10"] = fput_result(fa)
            fa.qr_every = "auto"
            line["fput_lyapunov_qr_tuned"] = fput_result(fa)
            qa = argparse.Namespace(**vars(args))
            qa.chunk, qa.steps, qa.warmup, qa.persistent = 1000, 3, 2, False
            line["quartic"] = quartic_result(qa)
        if world == 1 and args.classify_side > 0:
            c = classify_result(args.classify_side, 1_000_000)
            line["classify"] = {
                "what": c["metric"], "config": c["config"], "plain_s": c["plain"]["seconds"],
                "fast_s": c["fast"]["seconds"], "fast_speedup": c["fast"]["speedup"],
                "fast_agreement": c["fast"]["agreement"]}
            if "fast_surrogate" in c:
                fs = c["fast_surrogate"]
                line["classify"].update(surrogate_s=fs["seconds"], surrogate_speedup=fs["speedup"],
                                        surrogate_agreement=fs["agreement"],
                                        surrogate_judge_sample=fs["judge_sample"],
                                        surrogate_judge_agreement=fs["judge_agreement"],
                                        surrogate_confidence=fs["confidence"],
                                        surrogate_second_decision=fs["second_decision"])
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# Flops of one RK4 step of a quartic-3 orbit with k = 6 FP32 frame vectors
# (FMA = 2): FP64 -- the orbit's four stages (RHS ~12 each), stage inputs and
# accumulation over 6 components, energy and escape checks amortised (~170);
# FP32 -- the stage Hessians (12 per stage), the 6 x 6 propagator applied to 6
# frame vectors, Gram-Schmidt of the frame and the triangle update (~930).
QUARTIC_FLOPS = (170, 930)


def fput_flops_per_orbit_step(N: int, qr_every: int = 10) -> int:
    """Algorithmic FP64 flops of one step of the FPUT Lyapunov run (FMA = 2):
    propagation of the 2N vectors by the banded one-step RK4 propagator, 36 N^2
    FMA; its rows, ~60 N; the orbit's RK4, ~50 N; modified Gram-Schmidt of the
    2N x 2N matrix, (2N)^2 (2N + 1) FMA every qr_every steps."""
    d = 2 * N
    return 72 * N * N + 60 * N + 50 * N + (2 * d * d * (d + 1)) // qr_every


def fput_dp_flops_per_orbit_step(N: int, qr_every: int = 10) -> int:
    """Algorithmic FP64 flops of one DOP853 step of the FPUT Lyapunov run (FMA = 2):
    per column of W and row pair (q_i, p_i), stage inputs 2 x (2 per nonzero a_sj
    + 2) = 244, the tridiagonal J_s w 5 per stage (60), the 8 weighted sums 32 and
    the update 4: 340 per (column, row pair), 680 N^2 in all; the orbit's stages
    ~120 per component (240 N); modified Gram-Schmidt as for RK4."""
    d = 2 * N
    return 680 * N * N + 240 * N + (2 * d * d * (d + 1)) // qr_every


def run_fput(args):
    """FPUT-beta Lyapunov spectra (k = 1, beta = 1, h = 0.05, QR every 10 steps):
    4096 normal-mode orbits at energy density 0.1 per chain length; one bench
    step integrates every chain length for --chunk steps."""
    from paper_2507_00622_gb300 import build as cuda_build
    from paper_2507_00622_gb300 import chs

    cuda_build.build()
    chs.load()
    print(json.dumps(fput_result(args)))
    return 0


def fput_result(args) -> dict:
    """The FPUT Lyapunov line (see run_fput) as a dict."""
    import torch

    from paper_2507_00622_gb300 import chs
    from paper_2507_00622_gb300.inputs import normal_mode_draws

    Ns = [int(v) for v in args.fput_n.split(",")]
    n = args.fput_orbits
    runs = []
    for N in Ns:
        S = chs.System(chs.FPUT, N, (1.0, 0.0, 1.0))
        Q, P = normal_mode_draws(1000 + N, N, n)
        ics = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
        chs.chs_fput_mode_ics(S.h, n, torch.from_numpy(Q).cuda(), torch.from_numpy(P).cuda(),
                              torch.full((n,), 0.1 * N, dtype=torch.float64, device="cuda"), ics)
        lam = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
        st = torch.empty(n, dtype=torch.int32, device="cuda")
        runs.append((N, S, ics, lam, st))
    qr = {}
    for N in Ns:
        if args.qr_every == "auto":
            from paper_2507_00622_gb300 import autotune
            qr[N] = autotune.tune_fput_qr(N, integrator=args.integrator)["qr_every"]
        else:
            qr[N] = int(args.qr_every)
    dop = args.integrator == "dop853"
    blk, lanes, tuned = {}, {}, {}
    for N in Ns:
        lanes[N] = 0
        if dop:
            blk[N] = 0  # the DOP853 kernel keeps its own block shape
        elif args.block == "auto" and N in (4, 8):
            from paper_2507_00622_gb300 import autotune
            t = autotune.tune_fput_lanes(N, qr_every=qr[N], n_orbits=n)
            blk[N], lanes[N] = t["block_threads"], t["threads_per_orbit"]
            tuned[N] = t
        elif args.block == "auto":
            from paper_2507_00622_gb300 import autotune
            t = autotune.tune_fput_block(N, qr_every=qr[N])
            blk[N] = t["block_threads"]
            tuned[N] = t
        else:
            blk[N] = int(args.block)
    prms = {N: chs.params(0.05, args.chunk, qr_every=qr[N], sample_every=100,
                          integrator=chs.DOP853 if dop else chs.RK4, block_threads=blk[N],
                          threads_per_orbit=lanes[N]) for N in Ns}
    flops = fput_dp_flops_per_orbit_step if dop else fput_flops_per_orbit_step
    stream = torch.cuda.current_stream()

    work = torch.empty(1, dtype=torch.int64, device="cuda")
    persistent = getattr(args, "fput_persistent", False)

    def step(evs=None):
        if persistent:
            # every chain length in one persistent kernel over a work queue
            chs.chs_lyapunov_batch_persistent([(S.h, prms[N], n, ics, None, lam, st) for N, S, ics, lam, st in runs],
                                              work)
            return
        if args.fput_batch:
            # every chain length in one CUDA graph with concurrent branches
            chs.chs_lyapunov_batch([(S.h, prms[N], n, ics, None, lam, st) for N, S, ics, lam, st in runs])
            return
        for i, (N, S, ics, lam, st) in enumerate(runs):
            if evs is not None:
                evs[i][0].record(stream)
            chs.chs_lyapunov_spectrum(S.h, prms[N], n, ics, None, lam, st)
            if evs is not None:
                evs[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in runs] for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        step(evs[i])
    t1.record(stream)
    torch.cuda.synchronize()
    total_ms = t0.elapsed_time(t1)
    mp = measured_fp64_peak(torch.cuda.get_device_properties(0).multi_processor_count)
    per_n = {}
    for j, (N, *_rest) in enumerate(runs):
        if args.fput_batch or persistent:
            per_n[str(N)] = {"qr_every": qr[N]}
            continue
        ms = float(np.mean([evs[i][j][0].elapsed_time(evs[i][j][1]) for i in range(args.steps)]))
        os_ = n * args.chunk / (ms / 1e3)
        tf = flops(N, qr[N]) * os_ / 1e12
        per_n[str(N)] = {"orbit_steps_per_s": os_, "kernel_ms": ms, "fp64_tflops": tf,
                         "frac_of_fp64_peak": tf / mp["tflops"],
                         "frac_of_fp64_formula": tf / fp64_peak_tflops(2070.0), "qr_every": qr[N],
                         "block_threads": blk[N] or None, "threads_per_orbit": lanes[N] or None}
        if N in tuned:  # the tuner's timings (s per run; "lanes x block" or block)
            per_n[str(N)]["tuner"] = {"seconds": tuned[N]["seconds"], "steps": tuned[N]["steps"],
                                      "n_orbits": tuned[N]["n_orbits"]}
    value = len(runs) * n * args.chunk * args.steps / (total_ms / 1e3)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "fput_beta_lyapunov_h0.05" + ("_dop853" if dop else ""),
                       "N": Ns, "integrator": "DOP853 (fixed step)" if dop else "RK4",
                       "orbits_per_N": n, "steps_per_bench_step": args.chunk,
                       "qr_every": args.qr_every,
                       "launch": "one persistent kernel over a work queue" if persistent else
                                 ("one CUDA graph, concurrent branches" if args.fput_batch else "one launch per N")},
            "per_N": per_n,
            "fp64_peak": {"measured_tflops": mp["tflops"], "sm_mhz": mp["sm_mhz"],
                          "probe": mp["probe"], "formula_tflops": fp64_peak_tflops(2070.0)},
            **({} if args.no_cpu_baseline else
               {"cpu_baseline": cpu_fput_sample(Ns, args.chunk, qr, args.cpu_budget,
                                                args.integrator)})}


def fput_ens_flops_per_step(N: int, k: int) -> int:
    """Algorithmic FP64 flops of one accepted DOP853 step of an FPUT ensemble
    orbit with k deviation vectors (FMA = 2): 340 per (vector, row pair) as in
    fput_dp_flops_per_orbit_step, the orbit's stages ~240 N, the error norm ~12 N."""
    return 340 * k * N + 252 * N


def cpu_fput_gali_sample(Ns, n_orbits: int, tol: float, budget_s: float, n_sample: int = 16,
                         t_sample: float = 50.0):
    """The oracle on the host cores for the FPU GALI_4 workload: n_sample of the
    bench's orbits per chain length, adaptive DOP 8(5) at the bench's tolerance
    from t = 0 to t_sample (repeated while the chain length's share of budget_s
    lasts); the rate is that of the bench's mix (orbit-steps of every chain
    length in the proportion the GPU run took them)."""
    import oracle as O
    from paper_2507_00622_gb300.inputs import normal_mode_draws

    parts, rates = [], {}
    for N in Ns:
        Q, P = normal_mode_draws(2000 + N, N, n_orbits)
        ics = O.fput_mode_ics(O.fput(N), Q[:, :n_sample], P[:, :n_sample], np.full(n_sample, 0.1 * N))
        prm = O.params(0.05, 10**9, n_dev=4, sample_every=100, integrator=O.DOP853)
        t0 = time.perf_counter()
        done = 0
        while True:
            e = O.Ensemble(O.fput(N), prm, ics, seed=7)
            e.integrate_adaptive(prm, t_sample, tol, tol)
            e.indicators()
            done += int(e.n_exec.sum())
            if time.perf_counter() - t0 >= budget_s / len(Ns):
                break
        el = time.perf_counter() - t0
        rates[N] = done / el
        parts.append(f"N={N}: {done} orbit-steps of {n_sample} orbits to t={t_sample:g} in {el:.1f} s")
    return rates, {"cores": O.max_threads(), "kind": "oracle", "sample": "; ".join(parts)}


def run_fput_gali(args):
    """The FPU timing experiment of Sec. Examples: for every chain length N, 1e3
    random normal-mode orbits (energy density 0.1) with k = 4 deviation vectors
    integrated by adaptive DOP 8(5) (atol = rtol = --gali-tol) from t = 0 to
    tau = --gali-tau, then GALI_2..4.  One bench step is the whole experiment
    (set-up, integration and indicators for every N); per-N times by CUDA events."""
    import torch

    from paper_2507_00622_gb300 import build as cuda_build
    from paper_2507_00622_gb300 import chs
    from paper_2507_00622_gb300.inputs import normal_mode_draws

    cuda_build.build()
    chs.load()
    Ns = [int(v) for v in args.fput_n.split(",")]
    n, k, tau, tol = args.gali_orbits, 4, args.gali_tau, args.gali_tol
    runs = []
    for N in Ns:
        S = chs.System(chs.FPUT, N, (1.0, 0.0, 1.0))
        Q, P = normal_mode_draws(2000 + N, N, n)
        ics = torch.empty((2 * N, n), dtype=torch.float64, device="cuda")
        chs.chs_fput_mode_ics(S.h, n, torch.from_numpy(Q).cuda(), torch.from_numpy(P).cuda(),
                              torch.full((n,), 0.1 * N, dtype=torch.float64, device="cuda"), ics)
        ens = chs.DeviceEnsemble.empty(n, 2 * N, k)
        t = torch.empty(n, dtype=torch.float64, device="cuda")
        h = torch.empty(n, dtype=torch.float64, device="cuda")
        nr = torch.zeros(n, dtype=torch.int64, device="cuda")
        gali = torch.empty((k - 1, n), dtype=torch.float64, device="cuda")
        runs.append((N, S, ics, ens, t, h, nr, gali))
    kw = dict(n_dev=k, ld_p=0.0, sample_every=100, integrator=chs.DOP853, seed=7)
    ad = chs.Adaptive(tau, tol, tol, 0.0)
    stream = torch.cuda.current_stream()

    def one(N, S, ics, ens, t, h, nr, gali):
        abi = ens.abi(with_ld=False)
        chs.chs_ensemble_init(S.h, chs.params(0.05, 1, **kw), abi, ics)
        t.zero_()
        h.fill_(0.05)
        nr.zero_()
        chs.chs_integrate_adaptive(S.h, chs.params(0.05, 10**9, **kw), ad, abi, t, h, None, None, nr)
        chs.chs_indicators(S.h, chs.params(0.05, 0, **kw), abi, 0, 0, None, gali, None, None)

    for _ in range(args.warmup):
        for r in runs:
            one(*r)
    torch.cuda.synchronize()
    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in runs] for _ in range(args.steps)]
    clocks = ClockSampler(None)
    clocks.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        for j, r in enumerate(runs):
            evs[i][j][0].record(stream)
            one(*r)
            evs[i][j][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = t0.elapsed_time(t1)
    per_n, steps_by_n = {}, {}
    total_steps = 0
    for j, (N, S, ics, ens, t, h, nr, gali) in enumerate(runs):
        ms = float(np.mean([evs[i][j][0].elapsed_time(evs[i][j][1]) for i in range(args.steps)]))
        acc = int(ens.n_exec.sum())
        rej = int(nr.sum())
        st = ens.status.cpu().numpy()
        g4 = gali[k - 2].cpu().numpy()
        steps_by_n[N] = acc
        total_steps += acc
        tf = (acc * fput_ens_flops_per_step(N, k) + rej * 252 * N) / (ms / 1e3) / 1e12
        per_n[str(N)] = {"s_per_run": ms / 1e3, "us_per_orbit": 1e3 * ms / n,
                         "accepted_steps_per_orbit": acc / n, "rejected_per_orbit": rej / n,
                         "orbit_steps_per_s": acc / (ms / 1e3), "fp64_tflops": tf,
                         "frac_of_fp64_peak": tf / fp64_peak_tflops(clk["sm_mhz"] or 2070.0),
                         "max_dH": float(ens.dh_max.max().item()),
                         "status_ok": int((st == 0).sum()),
                         "gali4_median": float(np.median(g4[st == 0])) if (st == 0).any() else None}
    value = total_steps * args.steps / (total_ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "fpu_gali4_adaptive_dop853", "N": Ns, "orbits_per_N": n,
                       "k": k, "tau": tau, "atol": tol, "rtol": tol, "energy_density": 0.1,
                       "bench_step": "init + adaptive integration to tau + GALI_2..4, every N"},
            "clocks": clk, "per_N": per_n}
    if not args.no_cpu_baseline:
        rates, meta = cpu_fput_gali_sample(Ns, n, tol, args.cpu_budget)
        # the GPU run's mix of orbit-steps over the chain lengths
        inv = sum(steps_by_n[N] / total_steps / rates[N] for N in Ns)
        line["cpu_baseline"] = {"value": 1.0 / inv, "unit": UNIT, **meta}
    print(json.dumps(line))
    return 0


def classify_result(n_side: int, final_steps: int, confidence=None) -> dict:
    """Time to classify a Henon-Heiles section grid (E = 1/8, final t = steps * 0.01)
    by the plain form (FP64 vectors, every orbit to the end) and by the fast form
    (FP32 vector frame, early exit, compacted CUDA-graph chunks, and the trained
    surrogate when its weights are present), with the label agreement.  The
    surrogate form's time includes its judge: a 2 % random sample of the orbits
    the surrogate stopped, re-integrated by the plain form to the final time
    beside the rest of the fast form, whose labels give the surrogate's error."""
    from paper_2507_00622_gb300 import chs
    from paper_2507_00622_gb300 import classify as CL
    from paper_2507_00622_gb300 import surrogate as SG

    g = CL.GridSpec(E=1.0 / 8.0, n_side=n_side, n_steps=final_steps)
    plain = CL.run_plain(g)
    fast = CL.run_fast(g)
    valid = plain.status != chs.ORBIT_FORBIDDEN
    out = {"metric": "time-to-classified-grid vs plain at >=99.5% agreement", "unit": "s",
           "config": {"workload": f"henon_heiles_E1/8_grid{n_side}x{n_side}_k2_ld",
                      "final_t": final_steps * 0.01, "valid_cells": int(valid.sum())},
           "plain": {"seconds": plain.seconds, "orbit_steps": plain.orbit_steps, "dtype": "f64"},
           "fast": {"seconds": fast.seconds, "orbit_steps": fast.orbit_steps, "dtype": "f64 orbit + f32 frame",
                    "speedup": plain.seconds / fast.seconds,
                    "agreement": CL.agreement(plain, fast, plain.status)}}
    if os.path.exists(SG.WEIGHTS):
        import json as _json
        with np.load(SG.WEIGHTS) as z:
            meta = _json.loads(str(z["meta"]))
        sur = SG.Surrogate.load()
        sur2 = SG.Surrogate.load_second()
        conf = float(confidence or meta.get("confidence", 0.999))
        conf2 = float(meta.get("confidence2", 0.999))
        fs = CL.run_fast(g, surrogate=sur, confidence=conf, judge_fraction=0.02, surrogate2=sur2,
                         confidence2=conf2)
        # the judge: a 2 % random sample of the orbits the surrogate stopped,
        # re-integrated by the plain form to the final time on a second stream
        # beside the rest of the fast form; its cost is inside the surrogate
        # form's time
        judge = fs.extra.get("judge_cells", np.zeros(0, dtype=np.int64))
        jl = fs.extra.get("judge_label")
        out["fast_surrogate"] = {
            "seconds": fs.seconds, "orbit_steps": fs.orbit_steps, "confidence": conf,
            "speedup": plain.seconds / fs.seconds, "agreement": CL.agreement(plain, fs, plain.status),
            "stopped_by_surrogate": int(fs.extra["surrogate_stopped"]),
            "second_decision": None if sur2 is None else {
                "t": SG.DT * SG.DECIDE2_STEP, "confidence": conf2,
                "stopped": int(fs.extra["surrogate2_stopped"])},
            "judge": "plain FP64 re-integration to the final time of a random 2 % of the orbits "
                     "the surrogate stopped (at either decision), on a second stream from the first "
                     "decision on",
            "judge_sample": int(judge.size),
            "judge_orbit_steps": int(fs.extra.get("judge_orbit_steps", 0)),
            "judge_agreement": float(np.mean(fs.label[judge] == jl)) if judge.size else None,
            "judge_vs_full_plain_run": float(np.mean(jl == plain.label[judge])) if judge.size else None,
            "training": meta}
    return out


def run_classify(args):
    from paper_2507_00622_gb300 import build as cuda_build
    from paper_2507_00622_gb300 import chs

    cuda_build.build()
    chs.load()
    print(json.dumps(classify_result(args.n_side, args.final_steps, args.confidence)))
    return 0


def run_quartic(args):
    """The coupled quartic oscillator run: 4,194,304 states on energy shells
    E ~ U[1, 10] (random directions), eps = 0.1, k = 6 FP32 frame vectors (GALI_2..6),
    per-orbit end times t_end ~ U[1e3, 1e4] with early exit, compacted CUDA-graph
    chunks.  One bench step advances every live orbit by --chunk steps and
    evaluates SALI and GALI_2..6."""
    from paper_2507_00622_gb300 import build as cuda_build
    from paper_2507_00622_gb300 import chs

    cuda_build.build()
    chs.load()
    print(json.dumps(quartic_result(args)))
    return 0


def quartic_result(args) -> dict:
    """The quartic line (see run_quartic) as a dict."""
    import torch

    from paper_2507_00622_gb300 import chs

    n = args.quartic_orbits
    rng = np.random.default_rng(5)
    dirs = torch.from_numpy(rng.standard_normal((6, n))).cuda()
    E = torch.from_numpy(rng.uniform(1.0, 10.0, n)).cuda()
    t_end = torch.from_numpy(rng.integers(100_000, 1_000_001, n).astype(np.int64)).cuda()
    S = chs.System(chs.QUARTIC3, 3, (0.1,))
    ics = torch.empty((6, n), dtype=torch.float64, device="cuda")
    chs.chs_shell_ics(S.h, n, dirs, E, ics)
    del dirs
    k = 6
    kw = dict(n_dev=k, escape_r2=0.0, seed=3, vec_precision=chs.VEC_FP32, early_exit=True)
    ens = chs.DeviceEnsemble.empty(n, 6, k, vec_fp32=True)
    abi = ens.abi(with_ld=False, t_end=t_end)
    chs.chs_ensemble_init(S.h, chs.params(0.01, 1, **kw), abi, ics)
    work = chs.compact_work(n)
    sali = torch.empty(n, dtype=torch.float64, device="cuda")
    gali = torch.empty((k - 1, n), dtype=torch.float64, device="cuda")
    step = 0
    stream = torch.cuda.current_stream()

    queue = torch.empty(1, dtype=torch.int64, device="cuda")

    def one():
        nonlocal step
        if args.persistent:
            chs.chs_integrate_persistent(S.h, chs.params(0.01, args.chunk, step0=step, **kw), abi, queue)
        else:
            chs.chs_integrate_compacted(S.h, chs.params(0.01, args.chunk, step0=step, **kw), abi, 500, work)
        chs.chs_indicators(S.h, chs.params(0.01, 0, **kw), abi, sali=sali, gali=gali)
        step += args.chunk

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    e0 = int(ens.n_exec.sum())
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        one()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    done = int(ens.n_exec.sum()) - e0
    st = ens.status.cpu().numpy()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    p64, p32 = measured_fp64_peak(sms), measured_fp32_peak(sms)
    rate = done / (ms / 1e3)
    f64, f32 = QUARTIC_FLOPS
    return {"metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": 1,
            "roofline": {"bound": "alu", "unit": "TFLOP/s", "window": "whole bench step (integrate + indicators)",
                         "flops_per_orbit_step": {"fp64": f64, "fp32": f32},
                         "flops_basis": "estimate: orbit RHS and RK4 on FP64, the k = 6 frame's propagator, "
                                        "Gram-Schmidt and triangle update on FP32",
                         "fp64": {"achieved": f64 * rate / 1e12, "peak": p64["tflops"],
                                  "frac": f64 * rate / 1e12 / p64["tflops"]},
                         "fp32": {"achieved": f32 * rate / 1e12, "peak": p32["tflops"],
                                  "frac": f32 * rate / 1e12 / p32["tflops"]}},
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 orbit + f32 frame", "data": "synthetic",
            "config": {"workload": "quartic3_eps0.1_shellE1-10_k6_fp32frame_gali2-6",
                       "n_orbits": n, "rk4_steps_per_bench_step": args.chunk,
                       "launch": "persistent work queue" if args.persistent
                                 else "compacted 500-step chunks (CUDA graph)",
                       "t_window": [args.warmup * args.chunk * 0.01, step * 0.01],
                       "early_exited": int((st == chs.ORBIT_EARLY_CHAOTIC).sum())},
            **({} if args.no_cpu_baseline else
               {"cpu_baseline": cpu_quartic_sample(100, args.cpu_budget)})}


def run_integrators(args):
    """Cost of accuracy, RK4 against the paper's DOP853: the 256 x 256 grid at
    E = 1/6 (k = 4, LD) integrated to t = 100 by classic RK4 at two fixed steps,
    DOP853 at two fixed steps and adaptive DOP 8(5) at three tolerances; every
    final state is compared with DOP853 at h = 0.0025 on the orbits that are
    regular by that reference (SALI > 1e-2; chaotic orbits amplify any
    difference by exp(lambda t)).  Prints one JSON line: per method the kernel
    time, orbit-steps, and the median and maximum relative state error."""
    import torch

    from paper_2507_00622_gb300 import build as cuda_build
    from paper_2507_00622_gb300 import chs

    cuda_build.build()
    chs.load()
    side, T, k = 256, 100.0, 4
    n = side * side
    y0, y1, p0, p1 = grid_box(E_GRID)
    S = chs.System(chs.HENON_HEILES, 2)
    ics = torch.empty((4, n), dtype=torch.float64, device="cuda")
    ic_st = torch.empty(n, dtype=torch.int32, device="cuda")
    chs.chs_section_grid_ics(S.h, E_GRID, y0, y1, side, p0, p1, side, ics, ic_st)
    stream = torch.cuda.current_stream()

    def run(integ, h=None, tol=None):
        kw = dict(n_dev=k, ld_p=0.5, escape_r2=4.0, sample_every=100, integrator=integ)
        ens = chs.DeviceEnsemble.empty(n, 4, k)
        abi = ens.abi()
        chs.chs_ensemble_init(S.h, chs.params(h or 0.01, 1, **kw), abi, ics, ic_st)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if tol is None:
            steps = int(round(T / h))
            prm = chs.params(h, steps, **kw)
            torch.cuda.synchronize()
            ev0.record(stream)
            chs.chs_integrate_batch(S.h, prm, abi, stream)
            ev1.record(stream)
        else:
            t = torch.zeros(n, dtype=torch.float64, device="cuda")
            hs = torch.full((n,), 0.01, dtype=torch.float64, device="cuda")
            rej = torch.zeros(n, dtype=torch.int64, device="cuda")
            prm = chs.params(0.01, 10**8, **kw)
            torch.cuda.synchronize()
            ev0.record(stream)
            chs.chs_integrate_adaptive(S.h, prm, chs.Adaptive(T, tol, tol, 0.0), abi, t, hs, None, None, rej,
                                       stream)
            ev1.record(stream)
        torch.cuda.synchronize()
        sali = torch.empty(n, dtype=torch.float64, device="cuda")
        chs.chs_indicators(S.h, chs.params(0.01, 0, **kw), abi, sali=sali)
        torch.cuda.synchronize()
        return dict(ms=ev0.elapsed_time(ev1), x=ens.x.cpu().numpy(), st=ens.status.cpu().numpy(),
                    steps=int(ens.n_exec.sum()), sali=sali.cpu().numpy())

    ref = run(chs.DOP853, h=0.0025)
    keep = (ref["st"] == 0) & (ref["sali"] > 1e-2)
    scale = np.abs(ref["x"][:, keep]).max(axis=0)
    out = {}
    for name, integ, h, tol in (("rk4_h0.01", chs.RK4, 0.01, None), ("rk4_h0.005", chs.RK4, 0.005, None),
                                ("dop853_h0.1", chs.DOP853, 0.1, None), ("dop853_h0.05", chs.DOP853, 0.05, None),
                                ("dop853_adaptive_tol1e-8", chs.DOP853, None, 1e-8),
                                ("dop853_adaptive_tol1e-10", chs.DOP853, None, 1e-10),
                                ("dop853_adaptive_tol1e-12", chs.DOP853, None, 1e-12)):
        r = run(integ, h=h, tol=tol)
        ok = keep & (r["st"] == 0)
        err = (np.abs(r["x"][:, ok] - ref["x"][:, ok]).max(axis=0) / scale[ok[keep]])
        out[name] = {"kernel_ms": r["ms"], "orbit_steps": r["steps"],
                     "median_rel_err": float(np.median(err)), "max_rel_err": float(err.max()),
                     "orbits_compared": int(ok.sum())}
    print(json.dumps({"workload": f"henon_heiles_E1/6_grid{side}x{side}_k4_ld_to_t{T:g}",
                      "reference": "DOP853 h = 0.0025", "regular_orbits": int(keep.sum()),
                      "methods": out}))
    return 0


def run_saturation(args):
    """GPU saturation curve of the paper's Henon-Heiles experiment (Sec. Examples:
    time per initial condition against the number of initial conditions, SALI
    with 2 deviation vectors): section grids at E = 1/8 of 2^10 ... 2^20 cells,
    --chunk steps of the chosen integrator (h = 0.01; DOP853 at the same step),
    or with --sat-tol > 0 adaptive DOP 8(5) at atol = rtol = --sat-tol over the
    same time span (--chunk x 0.01), plus SALI, timed with CUDA events; one JSON
    line with the curve."""
    import torch

    from paper_2507_00622_gb300 import build as cuda_build
    from paper_2507_00622_gb300 import chs

    cuda_build.build()
    chs.load()
    from paper_2507_00622_gb300.inputs import hh_section_box

    E = 1.0 / 8.0
    y0, y1, p0, p1 = hh_section_box(E)
    S = chs.System(chs.HENON_HEILES, 2)
    adaptive = args.sat_tol > 0.0
    integ = chs.DOP853 if (args.integrator == "dop853" or adaptive) else chs.RK4
    # health checks (and so max |H - H0|) every 100 fixed steps, every 10 accepted adaptive ones
    kw = dict(n_dev=2, ld_p=0.5, escape_r2=4.0, sample_every=10 if adaptive else 100, integrator=integ)
    t_span = args.chunk * 0.01
    stream = torch.cuda.current_stream()
    curve = []
    for e in range(10, 21, 2):
        side = 1 << (e // 2)
        n = side * side
        ics = torch.empty((4, n), dtype=torch.float64, device="cuda")
        st = torch.empty(n, dtype=torch.int32, device="cuda")
        chs.chs_section_grid_ics(S.h, E, y0, y1, side, p0, p1, side, ics, st)
        ens = chs.DeviceEnsemble.empty(n, 4, 2)
        abi = ens.abi()
        sali = torch.empty(n, dtype=torch.float64, device="cuda")
        tt = torch.zeros(n, dtype=torch.float64, device="cuda")
        hh = torch.zeros(n, dtype=torch.float64, device="cuda")
        times = []
        for rep in range(1 + max(1, args.steps)):
            chs.chs_ensemble_init(S.h, chs.params(0.01, 1, **kw), abi, ics, st)
            tt.zero_()
            hh.fill_(0.01)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            if adaptive:
                chs.chs_integrate_adaptive(S.h, chs.params(0.01, 10**9, **kw),
                                           chs.Adaptive(t_span, args.sat_tol, args.sat_tol, 0.0), abi, tt, hh,
                                           stream=stream)
            else:
                chs.chs_integrate_batch(S.h, chs.params(0.01, args.chunk, **kw), abi, stream)
            chs.chs_indicators(S.h, chs.params(0.01, 0, **kw), abi, sali=sali, stream=stream)
            ev1.record(stream)
            torch.cuda.synchronize()
            if rep:
                times.append(ev0.elapsed_time(ev1))
        ms = float(np.median(times))
        valid = int((st == 0).sum())
        steps_done = int(ens.n_exec.sum())
        curve.append({"n_ics": n, "valid": valid, "ms": ms, "us_per_ic": 1e3 * ms / valid,
                      "orbit_steps_per_s": steps_done / (ms / 1e3),
                      "steps_per_ic": steps_done / valid, "max_dH": float(ens.dh_max[st == 0].max())})
    print(json.dumps({"workload": "henon_heiles_E1/8_saturation_sali_k2_ld",
                      "integrator": ("DOP 8(5) adaptive, atol = rtol = %g" % args.sat_tol) if adaptive
                                    else args.integrator,
                      "t_span": t_span, "steps": None if adaptive else args.chunk, "dt": 0.01,
                      "curve": curve}))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--chunk", type=int, default=1000, help="RK4 steps per bench step")
    ap.add_argument("--n-side", type=int, default=1024, help="grid side per GPU")
    ap.add_argument("--vec", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--integrator", choices=["rk4", "dop853"], default="rk4",
                    help="grid workload: classic RK4 or the paper's DOP853 at the same fixed step")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="grid line only: skip the FP32-vector, FPUT and quartic keys")
    ap.add_argument("--ref-sample", type=int, default=4096)
    ap.add_argument("--workload", choices=["grid", "fput", "classify", "quartic", "integrators",
                                           "saturation", "fput_gali", "peaks", "mlp"], default="grid")
    ap.add_argument("--quartic-orbits", type=int, default=4_194_304)
    ap.add_argument("--persistent", action="store_true",
                    help="quartic workload: one persistent work-queue launch per bench step")
    ap.add_argument("--final-steps", type=int, default=1_000_000)
    ap.add_argument("--confidence", type=float, default=None)
    ap.add_argument("--classify-side", type=int, default=1024,
                    help="grid side of the time-to-classified-grid measurement added to the "
                         "throughput line (0 = skip)")
    ap.add_argument("--fput-n", default="4,8,16,32,64")
    ap.add_argument("--fput-orbits", type=int, default=4096)
    ap.add_argument("--qr-every", default="10", help="QR interval of the FPUT run, or 'auto' (autotuner)")
    ap.add_argument("--fput-batch", action="store_true", help="all chain lengths in one CUDA graph")
    ap.add_argument("--fput-persistent", action="store_true",
                    help="all chain lengths in one persistent kernel (RK4)")
    ap.add_argument("--block", default="0", choices=["0", "32", "64", "128", "auto"],
                    help="threads per block of the RK4 kernels (grid: integrate kernel; fput: "
                         "Lyapunov kernel); 0 = library default, auto = autotuner")
    ap.add_argument("--sat-tol", type=float, default=0.0,
                    help="saturation: adaptive DOP 8(5) at this atol = rtol (0: fixed steps)")
    ap.add_argument("--gali-orbits", type=int, default=1000, help="fput_gali: orbits per chain length")
    ap.add_argument("--gali-tau", type=float, default=1000.0, help="fput_gali: integration time")
    ap.add_argument("--gali-tol", type=float, default=1e-8, help="fput_gali: atol = rtol")
    args = ap.parse_args()
    if args.workload == "fput":
        return run_fput(args)
    if args.workload == "classify":
        return run_classify(args)
    if args.workload == "integrators":
        return run_integrators(args)
    if args.workload == "saturation":
        return run_saturation(args)
    if args.workload == "quartic":
        return run_quartic(args)
    if args.workload == "fput_gali":
        return run_fput_gali(args)
    if args.workload == "peaks":
        return run_peaks(args)
    if args.workload == "mlp":
        return run_mlp(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
