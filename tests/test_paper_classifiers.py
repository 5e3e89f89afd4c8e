"""The paper's feature classifiers (Section 3.2.2: CART decision tree,
Gaussian naive Bayes) as comparators for the learned selector, on the
committed training set (CPU, scikit-learn)."""
import json
import os

import numpy as np
import pytest

pytest.importorskip("sklearn")

from paper_1511_02494_gb300 import classifiers  # noqa: E402
from paper_1511_02494_gb300.build import build  # noqa: E402


@pytest.fixture(scope="module")
def report():
    build()
    return classifiers.evaluate()


def test_report_is_reproducible(report):
    with open(os.path.join(classifiers.DATA, "classifier_report.json")) as f:
        stored = json.load(f)
    for name, pol in report["policies"].items():
        for k, v in pol.items():
            assert v == pytest.approx(stored["policies"][name][k], rel=1e-9), (name, k)


def test_classifiers_learn_the_rule_and_the_network_selects_best(report):
    P = report["policies"]
    counts = np.array(list(report["class_counts_test"].values()))
    majority = counts.max() / counts.sum()
    # the paper's set-up: features predict the profiling class well above chance
    assert P["decision_tree_class"]["class_accuracy"] > majority + 0.1
    assert P["naive_bayes_class"]["class_accuracy"] > majority
    # selecting through classes cannot beat the rule it imitates by much, and
    # the network selects closer to the exhaustive best than every comparator
    best_net = P["learned_selector"]["slowdown_vs_best"]
    for name, pol in P.items():
        if name != "learned_selector":
            assert best_net <= pol["slowdown_vs_best"] + 1e-12, name
