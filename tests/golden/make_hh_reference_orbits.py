"""Writes hh_reference_orbits.json: one regular and one chaotic Henon-Heiles
orbit at E = 1/8 on the x = 0 section, picked by the CPU oracle alone.

A 16 x 16 cell-centred grid is integrated with RK4 (h = 0.01) to t = 1000 with
two deviation vectors, and the largest Lyapunov exponent of every valid cell is
estimated by the oracle's QR method over the same time.  The chaotic pick is
the cell with the largest exponent among those whose SALI fell below 1e-12;
the regular pick is the cell with the smallest exponent.  Run from the repository root:
    python tests/golden/make_hh_reference_orbits.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2507_00622_gb300.inputs import hh_section_box  # noqa: E402


def main():
    E = 1.0 / 8.0
    y0, y1, p0, p1 = hh_section_box(E)
    n = 16
    ics, st = O.grid_ics(E, y0, y1, n, p0, p1, n)
    S = O.henon_heiles()
    prm = O.params(0.01, 100000, n_dev=2)
    ens = O.Ensemble(S, prm, ics, st, seed=1)
    ens.integrate(prm)
    sali, _, _ = ens.indicators()
    valid = np.where(st == 0)[0]
    lam, _ = O.lyapunov(S, O.params(0.01, 100000, qr_every=10), ics[:, valid])
    l1 = lam[0]
    cand = np.where(sali[valid] < 1e-12)[0]
    ci = cand[np.argmax(l1[cand])]
    chaotic = (int(valid[ci]), float(l1[ci]))
    ri = int(np.argmin(l1))
    regular = int(valid[ri])
    out = {
        "source": "tests/golden/make_hh_reference_orbits.py (CPU oracle, RK4 h=0.01, t=1000)",
        "chaotic": {"E": E, "y": float(ics[1, chaotic[0]]), "py": float(ics[3, chaotic[0]]),
                    "sali_t1000": float(sali[chaotic[0]]), "lambda1_t1000": chaotic[1]},
        "regular": {"E": E, "y": float(ics[1, regular]), "py": float(ics[3, regular]),
                    "sali_t1000": float(sali[regular]), "lambda1_t1000": float(l1[ri])},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hh_reference_orbits.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
