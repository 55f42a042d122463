"""Seeded synthetic inputs shared by the CUDA path's tests, the bench and the oracle.

This module holds no arithmetic of the method itself: it only draws random
numbers (numpy ``default_rng``) and computes the extent of the initial-condition
grid, so that both sides of a parity test receive identical inputs.  The
method's own steps (grid placement, normal-mode transform, energy scaling,
vector normalisation) are done separately by the CUDA library and the oracle.
"""
from __future__ import annotations

import numpy as np


def hh_section_box(E: float) -> tuple[float, float, float, float]:
    """Bounding box (y0, y1, py0, py1) of the energy-allowed region of the
    Henon-Heiles x = 0 section at energy E: |p_y| <= sqrt(2E) and y between the
    two real roots of y^2/2 - y^3/3 = E that bracket the origin."""
    roots = np.roots([-1.0 / 3.0, 0.5, 0.0, -E])
    real = np.sort(roots[np.abs(roots.imag) < 1e-9].real)
    lo = real[real < 0].max()
    hi = real[real > 0].min()
    pmax = float(np.sqrt(2.0 * E))
    return float(lo), float(hi), -pmax, pmax


def uniform_vectors(seed: int, n: int, k: int, d: int) -> np.ndarray:
    """k deviation vectors per orbit with components uniform in [-1, 1), not
    normalised; layout [k*d, n] (vector j occupies rows j*d .. j*d+d-1)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(k * d, n))


def normal_mode_draws(seed: int, N: int, n: int) -> tuple[np.ndarray, np.ndarray]:
    """Standard-normal normal-mode amplitudes (Q_m, P_m), each of shape [N, n]."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N, n)), rng.standard_normal((N, n))


def strided_sample(n: int, count: int) -> np.ndarray:
    """`count` orbit indices spread evenly over range(n)."""
    count = min(count, n)
    return np.unique(np.linspace(0, n - 1, count).round().astype(np.int64))


MLP_SHAPES = [((128, 12), True), ((128,), False), ((128, 128), True), ((128,), False),
              ((128, 128), True), ((128,), False), ((2, 128), True), ((2,), False)]


def mlp_init(seed: int) -> np.ndarray:
    """Initial perceptron parameters (flat, the layout of the surrogate): weights
    uniform in +-sqrt(6 / fan_in), biases zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for shape, is_w in MLP_SHAPES:
        if is_w:
            lim = np.sqrt(6.0 / shape[1])
            parts.append(rng.uniform(-lim, lim, shape).ravel())
        else:
            parts.append(np.zeros(shape))
    return np.concatenate(parts)
