"""The algorithmic flop counts behind bench.py's roofline figures (CPU only).

The roofline's `achieved` is algorithmic flops per orbit-step times the rate,
so the counts are pinned here: the DOP853 figure's tableau facts against the
oracle's tableau, and the published per-step totals of the RK4, FP32-frame,
DOP853, FPUT and FPUT-ensemble workloads against their formulas.
"""
import numpy as np

import bench
import oracle as O


def test_dop853_tableau_facts_used_by_the_count():
    a, b, e5, b3 = O.dop853_tableau()
    a = np.asarray(a)
    # the count takes 50 nonzero a_sj over the 11 stage inputs and 8 nonzero b_s
    assert int((a[1:12] != 0).sum()) == 50
    assert int((np.asarray(b) != 0).sum()) == 8


def test_published_per_step_totals():
    assert bench.flops_per_orbit_step(4, True, False) == (482, 0)
    assert bench.flops_per_orbit_step(4, True, True) == (90, 494)
    assert bench.dp_flops_per_orbit_step(4, True) == 3312
    # the DOP853 count grows by one vector's share per vector
    per_vector = bench.dp_flops_per_orbit_step(4, True) - bench.dp_flops_per_orbit_step(3, True)
    assert per_vector == 12 * 6 + (50 * 2 + 11 * 2) * 4 + 17 * 4 + 12


def test_fput_counts_scale_with_the_chain():
    for N in (4, 8, 16, 32, 64):
        d = 2 * N
        qr = 2 * d * d * (d + 1)
        assert bench.fput_flops_per_orbit_step(N, 10) == 72 * N * N + 110 * N + qr // 10
        assert bench.fput_dp_flops_per_orbit_step(N, 10) == 680 * N * N + 240 * N + qr // 10
        assert bench.fput_ens_flops_per_step(N, 4) == (340 * 4 + 252) * N


def test_fp64_peak_from_unit_counts():
    # 152 SMs x 2 DFMA lanes per clock x 2 flops x 2070 MHz
    assert abs(bench.fp64_peak_tflops(2070.0) - 1.25856) < 1e-12
