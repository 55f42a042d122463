"""The surrogate pipeline at small scale: the method generates labelled data, the
library's kernels train the perceptron on the GPU, and the trained network stops
confidently classified orbits at the decision time.  The test measures what the
network gains over the run without it (orbit-steps saved) and what it costs in
label agreement."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2507_00622_gb300 import chs  # noqa: E402
from paper_2507_00622_gb300 import surrogate as SG  # noqa: E402


def test_surrogate_trains_and_saves_integration():
    final = 200_000  # t = 2000
    energies = 0.10 + (np.arange(12) + 0.5) * 0.066 / 12
    ics, st, E = SG.grid_ics(energies, 40)
    run = SG.run_sampled(ics, st, final_step=final)
    X, label, target = SG.make_dataset(run, E)
    n = X.shape[1]
    assert n > 5000 and 0.1 < float(label.mean()) < 0.9
    perm = torch.from_numpy(np.random.default_rng(1).permutation(n)).cuda()
    val, tr = perm[: n // 5], perm[n // 5:]
    net = SG.train(X[:, tr].contiguous(), label[tr].contiguous(), target[tr].contiguous(),
                   epochs=25, batch=512, lr=3e-3, log=None)
    pv = net.probabilities(X[:, val].contiguous())
    lv = label[val].cpu().numpy()
    assert np.mean((pv >= 0.5) == (lv > 0.5)) > 0.85
    # the trained network in a run over a grid it has not seen (E = 0.13)
    ics2, st2, E2 = SG.grid_ics([0.13], 48)
    base = SG.run_sampled(ics2, st2, final_step=final)
    conf = 0.95
    with_net = SG.run_sampled(ics2, st2, final_step=final, surrogate=net, E=E2, confidence=conf)
    v = st2.cpu().numpy() == 0
    lb, ln = base["label"].cpu().numpy(), with_net["label"].cpu().numpy()
    stopped = (with_net["status"].cpu().numpy() == chs.ORBIT_PREDICTED_REGULAR)
    saved = 1.0 - with_net["n_exec"].sum().item() / base["n_exec"].sum().item()
    print(f"stopped {stopped.sum()} of {v.sum()}, orbit-steps saved {saved:.3f}, "
          f"agreement {np.mean(lb[v] == ln[v]):.4f}")
    assert stopped.sum() > 0 and saved > 0.1
    assert np.mean(lb[v] == ln[v]) > 0.95
