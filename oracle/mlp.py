"""Plain numpy (FP64) oracle of the early-stop surrogate perceptron (test
infrastructure only).

The network: 12 features -> 128 -> 128 -> 128 (ReLU) -> 2 outputs, parameters in
one flat array (row-major out x in): W1[128][12] b1 W2[128][128] b2 W3[128][128] b3
W4[2][128] b4.  Features of an orbit at decision time t from S SALI samples and
the LD: f_i = log10(max(SALI_i, 1e-20)) / 8, f_10 = LD / t - 1,
f_11 = (E - 0.133) / 0.033.  Loss: mean over the batch of BCE(sigmoid(y0), label)
+ w_reg (y1 - target)^2.

`bf16_acts=True` rounds every hidden activation to bfloat16 as the GPU kernels
store them, so that GPU and oracle can be compared tightly; the arithmetic is
otherwise exact FP64 and follows the definitions above step by step.
"""
from __future__ import annotations

import numpy as np

F, H, O, S_MAX = 12, 128, 2, 10
SHAPES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
          ("W4", (O, H)), ("b4", (O,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p: np.ndarray) -> dict:
    out, i = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(p[i:i + k], dtype=np.float64).reshape(shape)
        i += k
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (round to nearest, ties to even) and return as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def features(series: np.ndarray, ld: np.ndarray, t: float, E) -> np.ndarray:
    """E: the orbits' energies (array [n] or one scalar)."""
    S, n = series.shape
    X = np.empty((F, n))
    for i in range(S_MAX):
        s = series[i] if i < S else np.full(n, 1e-20)
        s = np.where(np.isfinite(s) & (s > 1e-20), s, 1e-20)
        X[i] = np.log10(s) / 8.0
    X[10] = ld / t - 1.0
    X[11] = (np.broadcast_to(np.asarray(E, dtype=np.float64), (n,)) - 0.133) / 0.033
    return X


def forward(p: np.ndarray, X: np.ndarray, bf16_acts: bool = False):
    w = unpack(p)
    r = bf16 if bf16_acts else (lambda v: v)
    a1 = r(np.maximum(w["W1"] @ X + w["b1"][:, None], 0.0))
    a2 = r(np.maximum(w["W2"] @ a1 + w["b2"][:, None], 0.0))
    a3 = r(np.maximum(w["W3"] @ a2 + w["b3"][:, None], 0.0))
    Y = w["W4"] @ a3 + w["b4"][:, None]
    return Y, (a1, a2, a3)


def loss_grad(Y: np.ndarray, label: np.ndarray, target: np.ndarray, w_reg: float):
    n = Y.shape[1]
    y0, y1 = Y[0], Y[1]
    p = 1.0 / (1.0 + np.exp(-y0))
    bce = np.maximum(y0, 0.0) - y0 * label + np.log1p(np.exp(-np.abs(y0)))
    L = float(np.mean(bce + w_reg * (y1 - target) ** 2))
    dY = np.stack([(p - label) / n, 2.0 * w_reg * (y1 - target) / n])
    return L, dY


def backward(p: np.ndarray, X: np.ndarray, acts, dY: np.ndarray) -> np.ndarray:
    """Gradients of the loss w.r.t. the flat parameters, given dL/dY."""
    w = unpack(p)
    a1, a2, a3 = acts
    g = {}
    g["W4"] = dY @ a3.T
    g["b4"] = dY.sum(axis=1)
    d3 = (w["W4"].T @ dY) * (a3 > 0)
    g["W3"] = d3 @ a2.T
    g["b3"] = d3.sum(axis=1)
    d2 = (w["W3"].T @ d3) * (a2 > 0)
    g["W2"] = d2 @ a1.T
    g["b2"] = d2.sum(axis=1)
    d1 = (w["W2"].T @ d2) * (a1 > 0)
    g["W1"] = d1 @ X.T
    g["b1"] = d1.sum(axis=1)
    return pack(g)


def adam(W, m, v, g, lr, b1, b2, eps, step):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    W = W - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
    return W, m, v
