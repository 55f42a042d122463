"""Host logic of the surrogate's decision threshold (CPU only): the table of
decided and wrongly decided fractions per candidate confidence, and the choice
of the smallest confidence within an error budget."""
import numpy as np

from paper_2507_00622_gb300 import surrogate as SG


def _samples():
    # 10 samples: probabilities of "chaotic" and the true labels
    prob = np.array([0.999, 0.97, 0.93, 0.6, 0.4, 0.05, 0.001, 0.96, 0.02, 0.91])
    label = np.array([1, 1, 0, 1, 0, 0, 0, 0, 1, 1], dtype=np.float32)
    return prob, label


def test_confidence_table_counts_decided_and_wrong_over_all_samples():
    prob, label = _samples()
    t = SG.confidence_table(prob, label)
    # c = 0.9: decided = p >= 0.9 or p <= 0.1 -> 0.999 0.97 0.93 0.05 0.001 0.96 0.02 0.91 (8);
    # wrong among them: 0.93 (label 0), 0.96 (label 0), 0.02 (label 1) -> 3
    assert t["0.9"] == (0.8, 0.3)
    # c = 0.95: 0.999 0.97 0.05 0.001 0.96 0.02 (6); wrong: 0.96, 0.02
    assert t["0.95"] == (0.6, 0.2)
    # c = 0.98: 0.999 0.001 0.02 (3); wrong: 0.02
    assert t["0.98"] == (0.3, 0.1)
    # c = 0.999: 0.999 0.001 (2, p >= c and p <= 1 - c inclusive); none wrong
    assert t["0.999"] == (0.2, 0.0)
    # the fractions never grow with the confidence
    fr = [t[str(c)] for c in SG.CONFIDENCES]
    assert all(a[0] >= b[0] and a[1] >= b[1] for a, b in zip(fr, fr[1:]))


def test_choose_confidence_takes_the_smallest_within_budget():
    prob, label = _samples()
    assert SG.choose_confidence(prob, label, 0.3) == (0.9, 0.8, 0.3)
    # 0.92 still decides 0.93 (wrong); 0.94 does not
    assert SG.choose_confidence(prob, label, 0.25) == (0.94, 0.6, 0.2)
    # 0.97 and 0.98 still decide 0.02 (wrong); 0.99 decides 0.999 and 0.001 only
    assert SG.choose_confidence(prob, label, 0.05) == (0.99, 0.2, 0.0)
    # nothing within a negative budget: the largest confidence, nothing decided
    assert SG.choose_confidence(prob, label, -1.0) == (0.9999, 0.0, 0.0)
