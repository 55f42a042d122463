"""Writes fput_lyapunov_t1e4.json: Lyapunov spectra of FPUT-beta chains at
t = 1e4 computed by the CPU oracle alone.

Workload: the FPUT-beta Lyapunov run (beta = 1, fixed ends, h = 0.05, QR every
10 steps, 200,000 RK4 steps, i.e. t = 1e4), orbits drawn as random normal modes
at energy density 0.1.  For every chain length N the orbits are a strided
sample of the 4096 seeded draws the bench integrates (normal_mode_draws(1000 + N,
N, 4096)); their initial states come from the oracle's normal-mode map.

Stored per N: the sampled draw indices, lambda_1 of every sampled orbit, the
sample mean of every exponent, and, for the short chains (N <= 8), lambda_1 of
the same orbits started from states perturbed by 1e-14 relative: the spread
between the two says which orbits are regular (lambda_1 reproducible to
rounding) and how far a chaotic orbit's finite-time lambda_1 moves under a
rounding-size change of its path.

The N = 64 chains take about six minutes of one core per orbit.  Run from the
repository root:
    python tests/golden/make_fput_lyapunov_t1e4.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2507_00622_gb300.inputs import normal_mode_draws, strided_sample  # noqa: E402

N_ALL = 4096
STEPS = 200_000
DT = 0.05
QR_EVERY = 10
SAMPLE = {4: 32, 8: 128, 16: 128, 32: 64, 64: 24}
PERTURBED = (4, 8)


def sample_ics(N: int, m: int):
    """Oracle initial states of the m strided draws of chain length N (and their indices)."""
    Q, P = normal_mode_draws(1000 + N, N, N_ALL)
    idx = strided_sample(N_ALL, m)
    ics = O.fput_mode_ics(O.fput(N), Q[:, idx], P[:, idx], np.full(m, 0.1 * N))
    return idx, ics


def main():
    out = {"source": "tests/golden/make_fput_lyapunov_t1e4.py (CPU oracle)",
           "workload": {"model": "FPUT-beta, fixed ends", "beta": 1.0, "energy_density": 0.1,
                        "dt": DT, "n_steps": STEPS, "qr_every": QR_EVERY, "draws_per_N": N_ALL,
                        "draw_seed": "1000 + N"},
           "chains": {}}
    prm = O.params(DT, STEPS, qr_every=QR_EVERY, sample_every=100)
    for N, m in SAMPLE.items():
        t0 = time.perf_counter()
        idx, ics = sample_ics(N, m)
        lam, st = O.lyapunov(O.fput(N), prm, ics)
        rec = {"draw_index": [int(i) for i in idx], "status": [int(s) for s in st],
               "lambda1": [float(v) for v in lam[0]],
               "mean_spectrum": [float(v) for v in lam.mean(axis=1)]}
        if N in PERTURBED:
            rng = np.random.default_rng(N)
            pert = ics * (1.0 + 1e-14 * rng.standard_normal(ics.shape))
            lam_p, _ = O.lyapunov(O.fput(N), prm, pert)
            rec["lambda1_perturbed_1e-14"] = [float(v) for v in lam_p[0]]
        out["chains"][str(N)] = rec
        print(f"N={N}: {m} orbits in {time.perf_counter() - t0:.0f} s, "
              f"mean lambda_1 {lam[0].mean():.5g}", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fput_lyapunov_t1e4.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
