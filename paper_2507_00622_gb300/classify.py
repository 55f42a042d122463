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
             judge_fraction: float = 0.0, judge_seed: int = 0, surrogate2=None,
             confidence2: float = 0.999) -> RunResult:
    """FP32 frame, early exit, compacted graph chunks; with a surrogate, the orbits
    still running at the decision time (t = 500) whose final label it predicts
    with probability >= confidence stop there and keep that label; with a second
    surrogate the orbits still running at t = 2000 get a second decision.

    With judge_fraction > 0 the plain form is the judge of the surrogates'
    error: right after the first decision a seeded random sample of that
    fraction of the orbits the surrogate stopped, and (with a second surrogate)
    of that fraction of the orbits still undecided, is re-integrated by the
    plain form to the final time, on a second stream beside the rest of the
    fast form.  The undecided orbits of the sample that the second surrogate
    stops at t = 2000 are a random sample of its decisions, judged with the
    first ones: starting them at the first decision keeps the judge's run, one
    orbit's 1e6 FP64 steps long, inside the first one's time.  The wall time
    includes the judge; extra["judge_cells"] / extra["judge_label"] hold the
    judged orbits and their plain labels.  (Starting the judge at t = 0 on a
    random sample of all cells measured slower: its orbits then share the SMs
    with the whole fast form, not only with its undecided tail.)"""
    from . import surrogate as sg
    S = chs.System(chs.HENON_HEILES, 2)
    ics, st = _grid(S, g)
    n = ics.shape[1]
    E = torch.full((n,), g.E, dtype=torch.float64, device="cuda")
    on_decision = on_decision2 = None
    if surrogate is not None and judge_fraction > 0.0:
        side = torch.cuda.Stream()

        def on_decision(status_dec, status):
            ok_dec = status_dec == chs.ORBIT_OK
            stopped = torch.nonzero(ok_dec & (status != chs.ORBIT_OK)).squeeze(1).cpu().numpy()
            rng = np.random.default_rng(judge_seed)
            pick = [rng.choice(stopped, max(1, int(judge_fraction * stopped.size)), replace=False)
                    if stopped.size else np.zeros(0, dtype=np.int64)]
            later = np.zeros(0, dtype=np.int64)
            if surrogate2 is not None:
                undecided = torch.nonzero(status == chs.ORBIT_OK).squeeze(1).cpu().numpy()
                if undecided.size:
                    later = np.sort(rng.choice(undecided, max(1, int(judge_fraction * undecided.size)),
                                               replace=False))
                pick.append(later)
            cells = np.unique(np.concatenate(pick))
            if cells.size == 0:
                return None
            side.wait_stream(torch.cuda.current_stream())
            return cells, start_plain_cells(g, ics, st, cells, side), np.sort(pick[0]), later

        if surrogate2 is not None:
            def on_decision2(status_dec2, status):
                # the orbits the second surrogate stopped (on the device, read after the run)
                return (status_dec2 == chs.ORBIT_OK) & (status != chs.ORBIT_OK)

    run = sg.run_sampled(ics, st, k=g.k, seed=g.seed, final_step=g.n_steps, chunk=chunk,
                         surrogate=surrogate, E=E, confidence=confidence, on_decision=on_decision,
                         surrogate2=surrogate2, confidence2=confidence2, on_decision2=on_decision2)
    status = run["status"].cpu().numpy()
    n_exec = run["n_exec"].cpu().numpy()
    by_net = (status == chs.ORBIT_PREDICTED_REGULAR) | ((status == chs.ORBIT_EARLY_CHAOTIC)
                                                       & ((n_exec == sg.DECIDE_STEP) | (n_exec == sg.DECIDE2_STEP)))
    extra = {"surrogate_stopped": int(np.sum(by_net & (n_exec == sg.DECIDE_STEP))),
             "surrogate2_stopped": int(np.sum(by_net & (n_exec == sg.DECIDE2_STEP))) if surrogate2 is not None else 0}
    steps = int(n_exec.sum())
    if run["on_decision"] is not None:
        cells, jr, first, later = run["on_decision"]
        judged = first
        if surrogate2 is not None and later.size:
            stopped2 = run["on_decision2"].cpu().numpy()
            judged = np.unique(np.concatenate([first, later[stopped2[later]]]))
        jl_all = jr["label"].cpu().numpy()
        pos = np.searchsorted(cells, judged)
        jn = jr["ensemble"].n_exec.cpu().numpy()
        extra.update(judge_cells=judged, judge_label=jl_all[pos], judge_orbit_steps=int(jn.sum()),
                     judge_sampled=int(judged.size), judge_run=int(cells.size))
        steps += int(jn.sum())
    return RunResult(run["label"].cpu().numpy(), status, n_exec, run["seconds"], steps, extra)


def agreement(a: RunResult, b: RunResult, status_ref: np.ndarray) -> float:
    """Label agreement over the valid (non-FORBIDDEN) cells."""
    v = status_ref != chs.ORBIT_FORBIDDEN
    return float((a.label[v] == b.label[v]).mean())
