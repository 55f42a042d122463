"""The surrogate perceptron's CUDA kernels (through the C ABI) against the numpy
FP64 oracle in oracle/mlp.py: forward pass, loss gradient, backward pass
(parameter gradients), Adam, features and the decision kernel."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2507_00622_gb300.inputs import mlp_init

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2507_00622_gb300 import chs  # noqa: E402


def _params(seed):
    p = M.bf16(mlp_init(seed))  # the BF16 weights both sides use
    pb = torch.from_numpy(p.astype(np.float32)).to(torch.bfloat16).cuda()
    return p, pb


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((M.F, n)).astype(np.float32)
    label = (rng.uniform(size=n) < 0.5).astype(np.float32)
    target = rng.standard_normal(n).astype(np.float32)
    return X, label, target


def test_param_count():
    assert chs.chs_mlp_param_count() == M.N_PARAMS == 34946


@pytest.mark.parametrize("n", [1, 63, 64, 1000, 4099])
def test_forward_matches_oracle(n):
    p, pb = _params(1)
    X, _, _ = _batch(n, 2)
    Y = torch.empty((2, n), dtype=torch.float32, device="cuda")
    act = torch.empty((3, 128, n), dtype=torch.bfloat16, device="cuda")
    chs.chs_mlp_forward(pb, torch.from_numpy(X).cuda(), n, Y, act)
    torch.cuda.synchronize()
    Yr, acts = M.forward(p, X.astype(np.float64), bf16_acts=True)
    # FP32 accumulation vs FP64 with the same BF16 weights and activation rounding;
    # a rounding boundary crossed by an activation shifts it by one BF16 ulp
    err = np.abs(Y.cpu().numpy() - Yr) / (1.0 + np.abs(Yr))
    assert np.median(err) < 1e-5 and err.max() < 2e-2
    a = act.float().cpu().numpy()
    assert np.mean(np.abs(a - np.stack(acts))) < 1e-3


def test_backward_gradients_match_oracle():
    n = 4096
    p, pb = _params(7)
    X, label, target = _batch(n, 3)
    Xd = torch.from_numpy(X).cuda()
    Y = torch.empty((2, n), dtype=torch.float32, device="cuda")
    act = torch.empty((3, 128, n), dtype=torch.bfloat16, device="cuda")
    dY = torch.empty((2, n), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    delta = torch.empty((3, 128, n), dtype=torch.float32, device="cuda")
    G = torch.empty(M.N_PARAMS, dtype=torch.float32, device="cuda")
    chs.chs_mlp_forward(pb, Xd, n, Y, act)
    chs.chs_mlp_loss_grad(Y, torch.from_numpy(label).cuda(), torch.from_numpy(target).cuda(), n, 0.25,
                          dY, loss)
    chs.chs_mlp_backward(pb, Xd, act, dY, n, delta, G)
    torch.cuda.synchronize()
    Yr, acts = M.forward(p, X.astype(np.float64), bf16_acts=True)
    Lr, dYr = M.loss_grad(Yr, label.astype(np.float64), target.astype(np.float64), 0.25)
    assert abs(loss.item() - Lr) < 1e-4 * max(1.0, Lr)
    # dY follows the outputs, which a BF16 activation rounding boundary can shift
    err = np.abs(dY.cpu().numpy() - dYr) / (np.abs(dYr) + 1e-12)
    assert np.median(err) < 1e-5 and err.max() < 1e-2
    gr = M.backward(p, X.astype(np.float64), acts, dYr)
    g = G.cpu().numpy()
    # per-tensor relative L2 error (BF16 activations on both sides, FP32 vs FP64 sums)
    i = 0
    for name, shape in M.SHAPES:
        k = int(np.prod(shape))
        a, b = g[i:i + k], gr[i:i + k]
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-9, name
        i += k


def test_adam_matches_oracle():
    P = M.N_PARAMS
    rng = np.random.default_rng(5)
    W = rng.standard_normal(P).astype(np.float32)
    m = np.zeros(P, np.float32)
    v = np.zeros(P, np.float32)
    Wd, md, vd = (torch.from_numpy(a.copy()).cuda() for a in (W, m, v))
    Wb = torch.empty(P, dtype=torch.bfloat16, device="cuda")
    Wo, mo, vo = W.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for step in range(1, 4):
        g = rng.standard_normal(P).astype(np.float32)
        chs.chs_mlp_adam(Wd, md, vd, torch.from_numpy(g).cuda(), 1e-3, 0.9, 0.999, 1e-8, step, Wb)
        Wo, mo, vo = M.adam(Wo, mo, vo, g.astype(np.float64), 1e-3, 0.9, 0.999, 1e-8, step)
    torch.cuda.synchronize()
    np.testing.assert_allclose(Wd.cpu().numpy(), Wo, rtol=1e-6, atol=1e-6)
    np.testing.assert_array_equal(Wb.float().cpu().numpy(), M.bf16(Wd.cpu().numpy()))


def test_features_and_decision_match_oracle():
    n = 777
    rng = np.random.default_rng(11)
    series = 10.0 ** rng.uniform(-18, 0, (10, n))
    series[:, :5] = 0.0
    ld = rng.uniform(5.0, 15.0, n) * 5.0
    X = torch.empty((12, n), dtype=torch.float32, device="cuda")
    sd, ldd = torch.from_numpy(series).cuda(), torch.from_numpy(ld).cuda()
    Ed = torch.full((n,), 0.125, dtype=torch.float64, device="cuda")
    chs.chs_mlp_features(sd, 10, ldd, 5.0, Ed, n, X)
    Xr = M.features(series, ld, 5.0, 0.125)
    np.testing.assert_allclose(X.cpu().numpy(), Xr, rtol=1e-6, atol=1e-6)
    p, pb = _params(2)
    status = torch.zeros(n, dtype=torch.int32, device="cuda")
    status[:3] = chs.ORBIT_ESCAPED
    prob = torch.empty(n, dtype=torch.float32, device="cuda")
    chs.chs_surrogate_decide(pb, sd, 10, ldd, 5.0, Ed, 0.8, n, status, prob)
    torch.cuda.synchronize()
    Yr, _ = M.forward(p, Xr, bf16_acts=True)
    pr = 1.0 / (1.0 + np.exp(-Yr[0]))
    np.testing.assert_allclose(prob.cpu().numpy(), pr, atol=5e-3)
    st = status.cpu().numpy()
    assert np.all(st[:3] == chs.ORBIT_ESCAPED)
    sure = np.abs(pr[3:] - 0.5) > 0.31  # away from the 0.8 / 0.2 boundaries
    exp = np.where(pr[3:] >= 0.8, chs.ORBIT_EARLY_CHAOTIC,
                   np.where(pr[3:] <= 0.2, chs.ORBIT_PREDICTED_REGULAR, chs.ORBIT_OK))
    np.testing.assert_array_equal(st[3:][sure], exp[sure])


def test_training_reduces_loss_on_a_separable_task():
    n = 8192
    rng = np.random.default_rng(21)
    X = rng.standard_normal((12, n)).astype(np.float32)
    label = (X[0] + 0.5 * X[3] > 0).astype(np.float32)
    target = (X[1] * 0.5).astype(np.float32)
    P = M.N_PARAMS
    master = torch.from_numpy(mlp_init(9).astype(np.float32)).cuda()
    pb = master.to(torch.bfloat16)
    m = torch.zeros(P, device="cuda")
    v = torch.zeros(P, device="cuda")
    Xd, ld, td = (torch.from_numpy(a).cuda() for a in (X, label, target))
    Y = torch.empty((2, n), device="cuda")
    act = torch.empty((3, 128, n), dtype=torch.bfloat16, device="cuda")
    dY = torch.empty((2, n), device="cuda")
    loss = torch.empty(1, device="cuda")
    delta = torch.empty((3, 128, n), device="cuda")
    G = torch.empty(P, device="cuda")
    losses = []
    for step in range(1, 201):
        chs.chs_mlp_forward(pb, Xd, n, Y, act)
        chs.chs_mlp_loss_grad(Y, ld, td, n, 0.5, dY, loss)
        chs.chs_mlp_backward(pb, Xd, act, dY, n, delta, G)
        chs.chs_mlp_adam(master, m, v, G, 3e-3, 0.9, 0.999, 1e-8, step, pb)
        losses.append(loss.item())
    assert losses[-1] < 0.2 * losses[0]
    pred = (Y[0].cpu().numpy() > 0).astype(np.float32)
    assert (pred == label).mean() > 0.97
