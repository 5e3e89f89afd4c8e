"""The selector trainer's host logic without a GPU: cost-sensitive targets,
and the second level's configuration table (each entry a valid SLICED
choice, equal to the committed data set's)."""
import os

import numpy as np
import pytest

import paper_1511_02494_gb300 as sp
from paper_1511_02494_gb300 import train_selector as ts
from paper_1511_02494_gb300.build import build

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1511_02494_gb300", "data")


def test_soft_targets_weigh_variants_by_their_slowdown():
    t = np.array([[1.0, 1.05, 2.0, 1.0], [3.0, 1.5, 1.5, 6.0]])
    for beta in (2.0, 8.0, 16.0):
        q = ts.soft_targets(t, beta)
        assert q.dtype == np.float32 and np.allclose(q.sum(1), 1.0)
        r = t / t.min(1, keepdims=True)
        expect = r ** -beta / (r ** -beta).sum(1, keepdims=True)
        np.testing.assert_allclose(q, expect, rtol=1e-6)
        # the fastest keep the most weight, ties equally; slower never more
        assert q[0, 0] == q[0, 3] and q[0, 0] > q[0, 1] > q[0, 2]
    # beta = inf: the best variants only, ties shared
    q = ts.soft_targets(t, np.inf)
    np.testing.assert_allclose(q, [[0.5, 0, 0, 0.5], [0, 0.5, 0.5, 0]])


def test_second_level_configurations_are_valid_sliced_choices():
    build()
    k = len(ts.SLICED_CONFIGS)
    assert ts.SLICED_CONFIGS[0] == (0, 0, 0)  # the structural rules
    assert len(set(ts.SLICED_CONFIGS)) == k
    g = np.random.default_rng(0)
    params = (g.standard_normal(64 * 16 + 64 + 64 * 64 + 64 + k * 64 + k) * 0.1).astype(np.float32)
    m = sp.spmv_model_create(64, 64, k, np.zeros(16, np.float32), np.ones(16, np.float32), params,
                             [sp.VARIANT_IDS["sliced"]] * k, 0.0)
    sp.spmv_model_set_launch(m, np.array(ts.SLICED_CONFIGS, np.int32))  # validated by the library
    s = np.load(os.path.join(DATA, "sliced_dataset.npz"))
    assert np.array_equal(s["configs"], np.array(ts.SLICED_CONFIGS, np.int32))
    assert s["times"].shape == (2000, k) and np.all(s["times"] > 0)


def test_margin_curve_applies_the_rule_below_the_margin():
    # three matrices, two variants; the rule always names variant 1
    times = np.array([[1.0, 2.0], [4.0, 1.0], [1.0, 1.0]])
    logits = np.array([[3.0, 0.0], [0.5, 0.0], [0.0, 0.1]], np.float32)  # margins 3, 0.5, 0.1
    rule = np.array([1, 1, 1])
    c = ts.margin_curve(times, logits, rule, [0.0, 0.2, 1.0, 5.0])
    assert [e["fallback_rate"] for e in c] == [0.0, 1 / 3, 2 / 3, 1.0]
    # mu 0: picks 0, 0, 1 -> slowdowns 1, 4, 1; mu 1: the second takes the rule -> 1, 1, 1
    assert c[0]["slowdown"] == pytest.approx(4 ** (1 / 3))
    assert c[2]["slowdown"] == pytest.approx(1.0)
    assert c[3]["slowdown"] == pytest.approx(2 ** (1 / 3))
