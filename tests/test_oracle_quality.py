"""Pins of the oracle's segmentation-quality metrics (Section 4.2.1): worked
examples counted by hand, and properties that hold for any prediction."""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "quality_worked.json")


def test_worked_examples():
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        conf, met = oracle.quality(np.array(c["pred"]), np.array(c["truth"]), c["L"])
        assert conf.tolist() == c["confusion"], c["note"]
        want = np.array([[n / d for n, d in row] for row in c["metrics"]])
        assert np.array_equal(met, want), c["note"]


def test_identity_and_complement():
    rng = np.random.default_rng(5)
    truth = rng.integers(0, 2, size=(17, 23)).astype(np.uint8)
    conf, met = oracle.quality(truth, truth, 2)
    assert conf[0, 1] == 0 and conf[1, 0] == 0
    assert np.all(met[:, :3] == 1.0) and np.array_equal(met[:, 3], met[:, 4])
    conf, met = oracle.quality(1 - truth, truth, 2)
    assert conf[0, 0] == 0 and conf[1, 1] == 0
    assert np.all(met[:, :3] == 0.0)


def test_counts_and_fractions():
    rng = np.random.default_rng(11)
    for L in (1, 2, 3, 5):
        truth = rng.integers(0, L, size=(31, 7)).astype(np.uint8)
        pred = rng.integers(0, L, size=(31, 7)).astype(np.uint8)
        conf, met = oracle.quality(pred, truth, L)
        n = truth.size
        assert conf.sum() == n
        for l in range(L):
            assert conf[l, :].sum() == (truth == l).sum()
            assert conf[:, l].sum() == (pred == l).sum()
            assert met[l, 3] == (pred == l).sum() / n and met[l, 4] == (truth == l).sum() / n
            agree = ((pred == l) == (truth == l)).sum()
            assert met[l, 2] == agree / n
        if L == 2:  # one-against-the-rest accuracy is the same for both labels
            assert met[0, 2] == met[1, 2] == (pred == truth).sum() / n


def test_absent_label_is_nan_and_bad_label_rejected():
    truth = np.array([0, 1, 1, 0], np.uint8)
    pred = np.array([1, 1, 0, 0], np.uint8)
    conf, met = oracle.quality(pred, truth, 3)
    assert np.isnan(met[2, 0]) and np.isnan(met[2, 1]) and met[2, 2] == 1.0 and met[2, 3] == 0.0
    with pytest.raises(RuntimeError):
        oracle.quality(np.array([0, 2], np.uint8), np.array([0, 1], np.uint8), 2)
