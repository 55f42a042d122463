"""Classifying a Henon-Heiles section grid as regular or chaotic (labels from SALI
at a final time), in two forms that call only the C ABI:

- plain: FP64 deviation vectors renormalised every step, every orbit integrated to
  the final step, labels from the final SALI;
- fast: FP32 vector frame (FP64 orbit), early exit once SALI < threshold, the run
  compacted over live orbits every chunk (CUDA graph), and optionally a surrogate
  that, at a decision time, stops the orbits whose final label it predicts with
  confidence.

Both forms use the same grid, seeds and threshold, so their labels can be
compared orbit by orbit.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import chs


@dataclass
class GridSpec:
    E: float = 1.0 / 8.0
    n_side: int = 1024
    box: tuple[float, float, float, float] | None = None  # (y0, y1, py0, py1)
    dt: float = 0.01
    n_steps: int = 1_000_000          # final time 1e4
    k: int = 2
    seed: int = 1
    sali_threshold: float = 1e-8

    def bounds(self):
        if self.box is not None:
            return self.box
        from .inputs import hh_section_box
        return hh_section_box(self.E)


@dataclass
class RunResult:
    label: np.ndarray
    status: np.ndarray
    n_exec: np.ndarray
    seconds: float
    orbit_steps: int
    extra: dict = field(default_factory=dict)


def _grid(S, g: GridSpec):
    y0, y1, p0, p1 = g.bounds()
    n = g.n_side * g.n_side
    ics = torch.empty((4, n), dtype=torch.float64, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    chs.chs_section_grid_ics(S.h, g.E, y0, y1, g.n_side, p0, p1, g.n_side, ics, st)
    return ics, st


def run_plain(g: GridSpec, chunk: int = 100_000) -> RunResult:
    """FP64 vectors, every orbit to the final step, labels from the final SALI."""
    S = chs.System(chs.HENON_HEILES, 2)
    ics, st = _grid(S, g)
    n = ics.shape[1]
    kw = dict(n_dev=g.k, ld_p=0.5, escape_r2=4.0, seed=g.seed, sali_threshold=g.sali_threshold)
    ens = chs.DeviceEnsemble.empty(n, 4, g.k)
    abi = ens.abi()
    chs.chs_ensemble_init(S.h, chs.params(g.dt, 1, **kw), abi, ics, st)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step = 0
    while step < g.n_steps:
        c = min(chunk, g.n_steps - step)
        chs.chs_integrate_batch(S.h, chs.params(g.dt, c, step0=step, **kw), abi)
        step += c
    label = torch.empty(n, dtype=torch.int8, device="cuda")
    chs.chs_indicators(S.h, chs.params(g.dt, 0, **kw), abi, label=label,
                       sali=torch.empty(n, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    n_exec = ens.n_exec.cpu().numpy()
    return RunResult(label.cpu().numpy(), ens.status.cpu().numpy(), n_exec, sec, int(n_exec.sum()))


def start_plain_cells(g: GridSpec, ics, st, cells: np.ndarray, stream=None) -> dict:
    """Launches the plain form (FP64 vectors seeded for that set, every orbit to
    the final step, labels from the final SALI) on the grid cells `cells`, taking
    their initial states from the grid arrays ics / st, asynchronously on
    `stream` (default: the current stream).  It carries no LD: the LD never acts
    on the orbit or its vectors, and the labels need SALI only, so they are those
    of the full plain run.  Returns the device tensors, valid once that stream
    has finished."""
    stream = stream or torch.cuda.current_stream()
    with torch.cuda.stream(stream):
        S = chs.System(chs.HENON_HEILES, 2)
        idx = torch.from_numpy(np.ascontiguousarray(cells, dtype=np.int64)).cuda()
        ics_c = ics[:, idx].contiguous()
        st_c = st[idx].contiguous()
        n = ics_c.shape[1]
        kw = dict(n_dev=g.k, ld_p=0.0, escape_r2=4.0, seed=g.seed, sali_threshold=g.sali_threshold)
        ens = chs.DeviceEnsemble.empty(n, 4, g.k)
        abi = ens.abi(with_ld=False)
        chs.chs_ensemble_init(S.h, chs.params(g.dt, 1, **kw), abi, ics_c, st_c)
        step, chunk = 0, 100_000
        while step < g.n_steps:
            c = min(chunk, g.n_steps - step)
            chs.chs_integrate_batch(S.h, chs.params(g.dt, c, step0=step, **kw), abi)
            step += c
        label = torch.empty(n, dtype=torch.int8, device="cuda")
        sali = torch.empty(n, dtype=torch.float64, device="cuda")
        chs.chs_indicators(S.h, chs.params(g.dt, 0, **kw), abi, label=label, sali=sali)
    return {"system": S, "ensemble": ens, "label": label, "sali": sali, "ics": ics_c, "status_in": st_c}


def run_plain_cells(g: GridSpec, cells: np.ndarray) -> RunResult:
    """The plain form on the grid cells `cells` only, timed."""
    S = chs.System(chs.HENON_HEILES, 2)
    ics, st = _grid(S, g)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = start_plain_cells(g, ics, st, cells)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    n_exec = r["ensemble"].n_exec.cpu().numpy()
    return RunResult(r["label"].cpu().numpy(), r["ensemble"].status.cpu().numpy(), n_exec, sec,
                     int(n_exec.sum()))


def run_fast(g: GridSpec, chunk: int = 2000, surrogate=None, confidence: float = 0.999,
             judge_fraction: float = 0.0, judge_seed: int = 0) -> RunResult:
    """FP32 frame, early exit, compacted graph chunks; with a surrogate, the orbits
    still running at the decision time (t = 500) whose final label it predicts
    with probability >= confidence stop there and keep that label.

    With judge_fraction > 0 the plain form is the judge of the surrogate's
    error: right after the decision a seeded random sample of that fraction of
    the orbits the surrogate stopped is re-integrated by the plain form to the
    final time, on a second stream beside the rest of the fast form.  The wall
    time includes it; extra["judge_cells"] / extra["judge_label"] hold the sample
    and its plain labels.  (Starting the judge at t = 0 on a random sample of
    all cells measured slower: its orbits then share the SMs with the whole
    fast form, not only with its undecided tail.)"""
    from . import surrogate as sg
    S = chs.System(chs.HENON_HEILES, 2)
    ics, st = _grid(S, g)
    n = ics.shape[1]
    E = torch.full((n,), g.E, dtype=torch.float64, device="cuda")
    on_decision = None
    if surrogate is not None and judge_fraction > 0.0:
        side = torch.cuda.Stream()

        def on_decision(status_dec, status):
            stopped = torch.nonzero((status_dec == chs.ORBIT_OK) & (status != chs.ORBIT_OK)).squeeze(1)
            stopped = stopped.cpu().numpy()
            if stopped.size == 0:
                return None
            rng = np.random.default_rng(judge_seed)
            cells = np.sort(rng.choice(stopped, max(1, int(judge_fraction * stopped.size)), replace=False))
            side.wait_stream(torch.cuda.current_stream())
            return cells, start_plain_cells(g, ics, st, cells, side)

    run = sg.run_sampled(ics, st, k=g.k, seed=g.seed, final_step=g.n_steps, chunk=chunk,
                         surrogate=surrogate, E=E, confidence=confidence, on_decision=on_decision)
    status = run["status"].cpu().numpy()
    n_exec = run["n_exec"].cpu().numpy()
    extra = {"surrogate_stopped": int(np.sum(status == chs.ORBIT_PREDICTED_REGULAR))
             + int(np.sum((status == chs.ORBIT_EARLY_CHAOTIC) & (n_exec == sg.DECIDE_STEP)))}
    steps = int(n_exec.sum())
    if run["on_decision"] is not None:
        cells, jr = run["on_decision"]
        jn = jr["ensemble"].n_exec.cpu().numpy()
        extra.update(judge_cells=cells, judge_label=jr["label"].cpu().numpy(), judge_orbit_steps=int(jn.sum()),
                     judge_sampled=int(cells.size))
        steps += int(jn.sum())
    return RunResult(run["label"].cpu().numpy(), status, n_exec, run["seconds"], steps, extra)


def agreement(a: RunResult, b: RunResult, status_ref: np.ndarray) -> float:
    """Label agreement over the valid (non-FORBIDDEN) cells."""
    v = status_ref != chs.ORBIT_FORBIDDEN
    return float((a.label[v] == b.label[v]).mean())
