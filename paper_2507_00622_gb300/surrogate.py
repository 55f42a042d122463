"""Early-stop surrogate for grid classification (the learned part of the path).

The method itself produces the training data: Henon-Heiles section grids at
energies spread over [0.10, 0.166] are integrated by the library (FP32 vector
frame, FP64 orbit, early exit, compacted chunks) to the final time; SALI is
sampled every 50 time units up to the decision time t = 500 and the LD is read
at t = 500.  The perceptron (include/chs.h, "Early-stop surrogate") learns the
final label (chaotic when the final SALI < 1e-8) from those early features and
is trained on the GPU by the library's own forward, backward and Adam kernels.
During a classification run it stops, at t = 500, the orbits whose final label
it predicts with the chosen confidence; the others are integrated to the end.

Usage (GPU):  python -m paper_2507_00622_gb300.surrogate --out <weights.npz>
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

from . import chs
from .inputs import hh_section_box, mlp_init

DT = 0.01
SAMPLE_EVERY = 5_000        # SALI samples every 50 time units
N_SAMPLES = 10              # ... up to the decision time t = 500
DECIDE_STEP = SAMPLE_EVERY * N_SAMPLES
SAMPLE2_EVERY = 20_000      # second decision: SALI samples every 200 time units
DECIDE2_STEP = SAMPLE2_EVERY * N_SAMPLES  # ... up to t = 2000
FINAL_STEP = 1_000_000      # final time 1e4


def _first_series_row(step: int) -> int:
    """Row of the first decision's series sampled at `step`, or -1."""
    if step <= DECIDE_STEP and step % SAMPLE_EVERY == 0:
        return step // SAMPLE_EVERY - 1
    return -1
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "surrogate_weights.npz")


def grid_ics(energies, side: int):
    """Cell-centred x = 0 section grids (side x side) at each energy, stacked:
    ics [4][n], status [n], E [n] on the device."""
    S = chs.System(chs.HENON_HEILES, 2)
    m = side * side
    n = m * len(energies)
    ics = torch.empty((4, n), dtype=torch.float64, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    E = torch.empty(n, dtype=torch.float64, device="cuda")
    tmp = torch.empty((4, m), dtype=torch.float64, device="cuda")
    tst = torch.empty(m, dtype=torch.int32, device="cuda")
    for i, e in enumerate(energies):
        y0, y1, p0, p1 = hh_section_box(float(e))
        chs.chs_section_grid_ics(S.h, float(e), y0, y1, side, p0, p1, side, tmp, tst)
        ics[:, i * m:(i + 1) * m].copy_(tmp)
        st[i * m:(i + 1) * m].copy_(tst)
        E[i * m:(i + 1) * m] = float(e)
    return ics, st, E


def run_sampled(ics, st, k: int = 2, seed: int = 1, final_step: int = FINAL_STEP, chunk: int = 2000,
                surrogate=None, E=None, confidence: float = 0.999, on_decision=None, second: bool = False,
                surrogate2=None, confidence2: float = 0.999, on_decision2=None):
    """Fast-form run with SALI samples up to the decision step.  Returns a dict of
    device tensors: series [10][n], ld_dec, status_dec (at the decision step),
    sali, label (final), n_exec, and the wall time (to the end of all device
    work, whatever stream it runs on).  on_decision(status_dec, status), when
    given, is called right after the surrogate's decision, before the run
    continues; its return value comes back as "on_decision".

    With `second` (or a second surrogate), when the run ends after t = 2000, it
    goes on sampling SALI every 200 time units to a second decision at t = 2000
    (the samples at t = 200 and 400 are those of the first series): series2,
    ld_dec2 and status_dec2 come back as well, surrogate2 decides there for the
    orbits still running, and on_decision2 is called as on_decision is."""
    S = chs.System(chs.HENON_HEILES, 2)
    n = ics.shape[1]
    kw = dict(n_dev=k, ld_p=0.5, escape_r2=4.0, seed=seed, sali_threshold=1e-8,
              vec_precision=chs.VEC_FP32, early_exit=True)
    ens = chs.DeviceEnsemble.empty(n, 4, k, vec_fp32=True)
    t_end = torch.full((n,), final_step, dtype=torch.int64, device="cuda")
    abi = ens.abi(t_end=t_end)
    work = chs.compact_work(n)
    series = torch.empty((N_SAMPLES, n), dtype=torch.float64, device="cuda")
    sali = torch.empty(n, dtype=torch.float64, device="cuda")
    label = torch.empty(n, dtype=torch.int8, device="cuda")
    chs.chs_ensemble_init(S.h, chs.params(DT, 1, **kw), abi, ics, st)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step = 0
    for i in range(N_SAMPLES):
        chs.chs_integrate_compacted(S.h, chs.params(DT, SAMPLE_EVERY, step0=step, **kw), abi, chunk, work)
        step += SAMPLE_EVERY
        chs.chs_indicators(S.h, chs.params(DT, 0, **kw), abi, sali=series[i])
    ld_dec = ens.ld.clone()
    status_dec = ens.status.clone()
    if surrogate is not None:
        surrogate.decide(series, ens.ld, ens.status, E, DT * DECIDE_STEP, confidence)
    side = on_decision(status_dec, ens.status) if on_decision is not None else None
    series2 = ld_dec2 = status_dec2 = side2 = None
    if (second or surrogate2 is not None) and final_step > DECIDE2_STEP:
        series2 = torch.empty((N_SAMPLES, n), dtype=torch.float64, device="cuda")
        for i in range(N_SAMPLES):
            target = (i + 1) * SAMPLE2_EVERY
            row = _first_series_row(target)
            if row >= 0:
                series2[i].copy_(series[row])
                continue
            chs.chs_integrate_compacted(S.h, chs.params(DT, target - step, step0=step, **kw), abi, chunk, work)
            step = target
            chs.chs_indicators(S.h, chs.params(DT, 0, **kw), abi, sali=series2[i])
        ld_dec2 = ens.ld.clone()
        status_dec2 = ens.status.clone()
        if surrogate2 is not None:
            surrogate2.decide(series2, ens.ld, ens.status, E, DT * DECIDE2_STEP, confidence2)
        side2 = on_decision2(status_dec2, ens.status) if on_decision2 is not None else None
    if final_step > step:
        chs.chs_integrate_compacted(S.h, chs.params(DT, final_step - step, step0=step, **kw), abi, chunk, work)
    chs.chs_indicators(S.h, chs.params(DT, 0, **kw), abi, sali=sali, label=label)
    torch.cuda.synchronize()  # the whole device: every stream's work is done
    sec = time.perf_counter() - t0
    return dict(series=series, ld_dec=ld_dec, status_dec=status_dec, sali=sali, label=label,
                status=ens.status, n_exec=ens.n_exec, seconds=sec, on_decision=side,
                series2=series2, ld_dec2=ld_dec2, status_dec2=status_dec2, on_decision2=side2)


def make_dataset(run, E, second: bool = False, among=None):
    """Features (library kernel) and targets of the orbits still running at the
    decision step (the second one with `second`) whose final label is regular
    (0) or chaotic (1), restricted to the orbits where the boolean device mask
    `among` is set when it is given.  Returns X, label, target and the orbits'
    indices."""
    n = E.shape[0]
    X = torch.empty((12, n), dtype=torch.float32, device="cuda")
    series, ld, status, t = ((run["series2"], run["ld_dec2"], run["status_dec2"], DT * DECIDE2_STEP) if second
                             else (run["series"], run["ld_dec"], run["status_dec"], DT * DECIDE_STEP))
    chs.chs_mlp_features(series, N_SAMPLES, ld, t, E, n, X)
    lab = run["label"].long()
    keep = (status == chs.ORBIT_OK) & ((lab == 0) | (lab == 1))
    if among is not None:
        keep &= among
    target = torch.log10(torch.clamp(run["sali"], min=1e-20)).float() / 8.0
    idx = torch.nonzero(keep).squeeze(1)
    return X[:, idx].contiguous(), lab[idx].float().contiguous(), target[idx].contiguous(), idx


class Surrogate:
    """BF16 perceptron parameters on the device and the decision call."""

    def __init__(self, params_fp32: np.ndarray):
        self.master = torch.from_numpy(np.asarray(params_fp32, dtype=np.float32)).cuda()
        self.params = self.master.to(torch.bfloat16)

    @classmethod
    def load(cls, path: str = WEIGHTS) -> "Surrogate":
        with np.load(path) as z:
            return cls(z["params"])

    @classmethod
    def load_second(cls, path: str = WEIGHTS) -> "Surrogate | None":
        """The second decision's network (t = 2000), if the file holds one."""
        with np.load(path) as z:
            return cls(z["params2"]) if "params2" in z.files else None

    def save(self, path: str = WEIGHTS, meta: dict | None = None, second: "Surrogate | None" = None):
        arrays = dict(params=self.master.cpu().numpy(), meta=json.dumps(meta or {}))
        if second is not None:
            arrays["params2"] = second.master.cpu().numpy()
        np.savez(path, **arrays)

    def decide(self, series, ld, status, E, t_decide: float, confidence: float) -> None:
        n = status.shape[0]
        chs.chs_surrogate_decide(self.params, series, N_SAMPLES, ld, t_decide, E, confidence, n, status)

    def probabilities(self, X) -> np.ndarray:
        n = X.shape[1]
        Y = torch.empty((2, n), dtype=torch.float32, device="cuda")
        chs.chs_mlp_forward(self.params, X, n, Y)
        return torch.sigmoid(Y[0]).cpu().numpy()


def train(X, label, target, *, epochs: int = 40, batch: int = 4096, lr: float = 2e-3,
          w_reg: float = 0.25, seed: int = 0, log=print) -> Surrogate:
    """Adam training with the library's kernels on mini-batches (the shuffling is
    index bookkeeping in torch; every arithmetic step is a library kernel)."""
    P = chs.chs_mlp_param_count()
    net = Surrogate(mlp_init(seed))
    m = torch.zeros(P, device="cuda")
    v = torch.zeros(P, device="cuda")
    n = X.shape[1]
    Y = torch.empty((2, batch), device="cuda")
    act = torch.empty((3, 128, batch), dtype=torch.bfloat16, device="cuda")
    dY = torch.empty((2, batch), device="cuda")
    loss = torch.empty(1, device="cuda")
    delta = torch.empty((3, 128, batch), device="cuda")
    G = torch.empty(P, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=gen)
        tot, cnt = 0.0, 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb = X[:, idx].contiguous()
            lb = label[idx].contiguous()
            tb = target[idx].contiguous()
            chs.chs_mlp_forward(net.params, xb, batch, Y, act)
            chs.chs_mlp_loss_grad(Y, lb, tb, batch, w_reg, dY, loss)
            chs.chs_mlp_backward(net.params, xb, act, dY, batch, delta, G)
            step += 1
            lr_t = lr * (0.5 * (1 + np.cos(np.pi * step / (epochs * (n // batch)))))
            chs.chs_mlp_adam(net.master, m, v, G, max(lr_t, 1e-5), 0.9, 0.999, 1e-8, step, net.params)
            tot += loss.item() if (b0 // batch) % 20 == 0 else 0.0
            cnt += 1 if (b0 // batch) % 20 == 0 else 0
        if log and (ep % 5 == 0 or ep == epochs - 1):
            log(f"epoch {ep}: loss {tot / max(cnt, 1):.4f}")
    return net


CONFIDENCES = (0.9, 0.92, 0.94, 0.95, 0.96, 0.97, 0.98, 0.99, 0.995, 0.998, 0.999, 0.9995, 0.9999)


def confidence_table(prob: np.ndarray, label: np.ndarray) -> dict:
    """Per candidate confidence c: the fraction of samples decided (p >= c or
    p <= 1 - c) and the fraction decided wrongly, both over all samples."""
    pred = prob >= 0.5
    out = {}
    for c in CONFIDENCES:
        dec = (prob >= c) | (prob <= 1 - c)
        out[str(c)] = (float(dec.mean()), float(np.mean(dec & (pred != (label > 0.5)))))
    return out


def choose_confidence(prob: np.ndarray, label: np.ndarray, max_error: float) -> tuple[float, float, float]:
    """Smallest confidence c whose confident decisions (p >= c or p <= 1 - c) err
    on at most max_error of all samples; returns (c, decided fraction, error fraction)."""
    table = confidence_table(prob, label)
    for c in CONFIDENCES:
        frac, err = table[str(c)]
        if err <= max_error:
            return c, frac, err
    return 0.9999, 0.0, 0.0


def _fit(X, label, target, epochs: int, max_error: float, seed: int = 0):
    """Train on 90 % of the orbits, choose the confidence on the held-out 10 %."""
    n = X.shape[1]
    rng = np.random.default_rng(seed)
    order = torch.from_numpy(rng.permutation(n)).cuda()
    nv = n // 10
    val, tr = order[:nv], order[nv:]
    t1 = time.perf_counter()
    net = train(X[:, tr].contiguous(), label[tr].contiguous(), target[tr].contiguous(), epochs=epochs)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    pv = net.probabilities(X[:, val].contiguous())
    lv = label[val].cpu().numpy()
    conf, frac, err = choose_confidence(pv, lv, max_error)
    meta = dict(train_orbits=int(n - nv), val_orbits=int(nv), val_accuracy=float(np.mean((pv >= 0.5) == (lv > 0.5))),
                confidence=conf, val_decided_fraction=frac, val_error_fraction=err, max_error=max_error,
                val_by_confidence=confidence_table(pv, lv), epochs=epochs, training_seconds=t_train,
                chaotic_fraction=float(np.mean(label.cpu().numpy())))
    return net, meta


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--energies", type=int, default=96)
    ap.add_argument("--side", type=int, default=128)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--final-step", type=int, default=FINAL_STEP)
    # The classification allows 0.5 % of a grid's valid cells to disagree with the
    # plain form; about two thirds of the cells are still running at the decision,
    # so wrong confident decisions on 0.3 % of those orbits use ~0.2 % of the cells,
    # leaving the rest of the allowance to the fast form's own disagreement and to
    # the difference between the validation energies and a grid's.
    ap.add_argument("--max-error", type=float, default=0.003)
    # The second decision (t = 2000) sees only the orbits the first one left
    # undecided, about a seventh of a grid's valid cells: wrong decisions on
    # 0.5 % of them cost ~0.07 % of the cells.
    ap.add_argument("--max-error2", type=float, default=0.005)
    ap.add_argument("--no-second", action="store_true", help="train the first decision's network only")
    args = ap.parse_args()
    torch.cuda.set_device(0)
    from . import build as cuda_build
    cuda_build.build()
    chs.load()
    energies = 0.10 + (np.arange(args.energies) + 0.5) * (0.166 - 0.10) / args.energies
    ics, st, E = grid_ics(energies, args.side)
    t0 = time.perf_counter()
    run = run_sampled(ics, st, final_step=args.final_step, second=not args.no_second)
    t_gen = time.perf_counter() - t0
    X, label, target, idx = make_dataset(run, E)
    net, meta = _fit(X, label, target, args.epochs, args.max_error)
    meta.update(generation_seconds=t_gen, energies=[float(energies[0]), float(energies[-1])],
                grid_side=args.side, final_step=args.final_step, decide_step=DECIDE_STEP)
    net2 = None
    if not args.no_second:
        # the orbits the first network leaves undecided at its confidence are the
        # second network's data, as they are its inputs in a classification run
        p1 = net.probabilities(X)
        undecided = (p1 < meta["confidence"]) & (p1 > 1.0 - meta["confidence"])
        among = torch.zeros(E.shape[0], dtype=torch.bool, device="cuda")
        among[idx[torch.from_numpy(undecided).cuda()]] = True
        X2, label2, target2, _ = make_dataset(run, E, second=True, among=among)
        net2, meta2 = _fit(X2, label2, target2, args.epochs, args.max_error2, seed=1)
        meta2.update(decide_step=DECIDE2_STEP)
        meta["second"] = meta2
        meta["confidence2"] = meta2["confidence"]
    net.save(args.out, meta, second=net2)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
