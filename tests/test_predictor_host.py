"""Host logic of the learned part on the CPU: the product's label rule against the oracle's
brute-force definition."""
import numpy as np

from oracle import mlp_oracle as M


def test_labels_at_rule_accuracy_against_the_oracle_definition():
    """The product's Lagrangian label rule against the oracle's brute-force definition on
    tables of per-block errors like the method's (256x per slice, spread scales)."""
    from paper_2601_08077_gb300 import predictor
    rng = np.random.default_rng(3)
    worse = 0
    for trial in range(40):
        nblk = int(rng.integers(2, 5))
        scale = 10.0 ** rng.uniform(-6, 0, size=nblk)
        err = scale[:, None] * 256.0 ** -np.arange(1, 9)[None, :] * rng.uniform(0.5, 2.0, size=(nblk, 8))
        err[:, 6:] = np.maximum(err[:, 6:], 1e-17)       # the FP64 rounding floor
        for s_rule in (3, 5):
            got = predictor.labels_at_rule_accuracy(err, s_rule)
            opt = M.labels_at_rule_accuracy(err, s_rule)
            budget = err[:, s_rule - 1].sum()
            assert err[np.arange(nblk), got - 1].sum() <= budget
            w_got = sum(predictor.pairs(int(s)) for s in got)
            w_opt = sum(predictor.pairs(int(s)) for s in opt)
            assert w_opt <= w_got <= nblk * predictor.pairs(s_rule)
            worse += w_got > w_opt
    assert worse <= 8
