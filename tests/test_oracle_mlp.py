"""Pins of the perceptron oracle (oracle/mlp.py) to facts outside it: finite
differences of its own loss, closed forms of a network with a zero last layer,
the library's bfloat16 rounding, and the first Adam step."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2507_00622_gb300.inputs import mlp_init


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((M.F, n))
    label = (rng.uniform(size=n) < 0.5).astype(float)
    target = rng.standard_normal(n)
    return X, label, target


def test_backward_matches_finite_differences():
    p = mlp_init(3)
    X, label, target = _batch(7, 1)
    Y, acts = M.forward(p, X)
    _, dY = M.loss_grad(Y, label, target, 0.3)
    g = M.backward(p, X, acts, dY)
    rng = np.random.default_rng(0)
    idx = rng.choice(M.N_PARAMS, 60, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = 1e-6
        Lp = M.loss_grad(M.forward(p + e, X)[0], label, target, 0.3)[0]
        Lm = M.loss_grad(M.forward(p - e, X)[0], label, target, 0.3)[0]
        fd = (Lp - Lm) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_zero_last_layer_closed_form():
    p = mlp_init(5)
    w = M.unpack(p)
    w["W4"][:] = 0.0
    w["b4"][:] = [0.7, -0.2]
    p = M.pack(w)
    X, label, target = _batch(11, 2)
    Y, acts = M.forward(p, X)
    assert np.all(Y[0] == 0.7) and np.all(Y[1] == -0.2)
    L, dY = M.loss_grad(Y, label, target, 0.5)
    sig = 1.0 / (1.0 + np.exp(-0.7))
    ref = np.mean(-label * np.log(sig) - (1 - label) * np.log(1 - sig) + 0.5 * (-0.2 - target) ** 2)
    assert abs(L - ref) < 1e-12
    g = M.unpack(M.backward(p, X, acts, dY))
    np.testing.assert_allclose(g["b4"], [np.mean(sig - label), np.mean(2 * 0.5 * (-0.2 - target))], atol=1e-14)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert np.all(g[name] == 0.0)


def test_bf16_rounding_matches_library():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(9).standard_normal(10000) * 10.0 ** np.random.default_rng(1).uniform(-5, 5, 10000)
    x = np.concatenate([x, [1.0, 1.0 + 2.0**-8, 1.0 + 3 * 2.0**-9, -2.5, 0.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.bf16(x), ref)


def test_features_of_known_samples():
    series = np.array([[1e-8, 0.0, 1.0, np.nan]] * 10)
    X = M.features(series, np.array([30.0, 20.0, 10.0, 10.0]), 10.0, 0.133)
    np.testing.assert_allclose(X[0], [-1.0, -2.5, 0.0, -2.5])
    np.testing.assert_allclose(X[10], [2.0, 1.0, 0.0, 0.0])
    assert np.all(X[11] == 0.0)


def test_first_adam_step_is_a_signed_step():
    rng = np.random.default_rng(4)
    W = rng.standard_normal(100)
    g = rng.standard_normal(100)
    W1, m, v = M.adam(W, np.zeros(100), np.zeros(100), g, 1e-3, 0.9, 0.999, 1e-12, 1)
    np.testing.assert_allclose(W1, W - 1e-3 * np.sign(g), atol=1e-12)
