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
    X, label, target, _ = SG.make_dataset(run, E)
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


def test_second_decision_plumbing():
    """The two-decision run: the second series reuses the first one's samples at
    t = 200 and 400 and samples the rest itself; a second network decides at
    t = 2000 for the orbits still running (here the first network again, the
    plumbing being under test), and the judge's sample covers both decisions."""
    energies = [0.12, 0.14]
    ics, st, E = SG.grid_ics(energies, 32)
    final = 300_000  # t = 3000
    run = SG.run_sampled(ics, st, final_step=final, second=True)
    s1, s2 = run["series"].cpu().numpy(), run["series2"].cpu().numpy()
    np.testing.assert_array_equal(s2[0], s1[3])
    np.testing.assert_array_equal(s2[1], s1[7])
    assert run["status_dec2"] is not None and run["ld_dec2"] is not None
    X2, l2, t2, idx2 = SG.make_dataset(run, E, second=True)
    assert X2.shape[0] == 12 and X2.shape[1] == idx2.numel() > 0
    # running at t = 2000 implies running at t = 500
    assert bool(torch.all(run["status_dec"][idx2] == chs.ORBIT_OK))
    net = SG.Surrogate.load()
    two = SG.run_sampled(ics, st, final_step=final, surrogate=net, E=E, confidence=0.95,
                         surrogate2=net, confidence2=0.95)
    ne = two["n_exec"].cpu().numpy()
    sts = two["status"].cpu().numpy()
    stopped2 = np.isin(sts, (chs.ORBIT_PREDICTED_REGULAR, chs.ORBIT_EARLY_CHAOTIC)) & (ne == SG.DECIDE2_STEP)
    assert stopped2.sum() > 0
    # every orbit stopped at the second decision was running at the first
    assert np.all(two["status_dec"].cpu().numpy()[stopped2] == chs.ORBIT_OK)



def test_two_decision_classification_and_its_judge():
    """classify.run_fast with both decisions and the judge on a small grid: the
    judged orbits are orbits the networks stopped, their plain labels come from
    the judge's own run, and the labels of the fast form stay within a few
    percent of the plain form's."""
    from paper_2507_00622_gb300 import classify as CL
    g = CL.GridSpec(E=1.0 / 8.0, n_side=64, n_steps=300_000)
    net = SG.Surrogate.load()
    plain = CL.run_plain(g)
    fs = CL.run_fast(g, surrogate=net, confidence=0.95, judge_fraction=0.1, surrogate2=net, confidence2=0.95)
    cells, jl = fs.extra["judge_cells"], fs.extra["judge_label"]
    assert cells.size == jl.size > 0 and np.all(np.diff(cells) > 0)
    assert fs.extra["judge_run"] >= cells.size
    by_net = np.isin(fs.status[cells], (chs.ORBIT_PREDICTED_REGULAR, chs.ORBIT_EARLY_CHAOTIC))
    assert np.all(by_net)
    # the judge integrates the plain form (its vectors seeded for its own set,
    # so an orbit at the threshold may differ): its labels are the full plain run's
    assert np.mean(jl == plain.label[cells]) > 0.98
    assert CL.agreement(plain, fs, plain.status) > 0.95
