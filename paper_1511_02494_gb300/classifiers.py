"""The paper's feature-based classifiers as comparators for the learned
selector (Section 3.2.2): a CART decision tree and Gaussian naive Bayes,
trained with scikit-learn on the CPU from the committed training set.

Two set-ups, both on the 80/20 split by seed used for the network:

* as in the paper: the 14 Table 1 features (the first 14 entries of the
  feature vector) predict the bottleneck class that the profiling rule
  (Section 3.2.1) assigns from the stored probe speedups; the predicted
  class then selects its variant through the class -> variant table.  The
  class accuracy is the figure the paper's Tables 3 and 4 report.
* the same classifiers predicting the fastest variant directly from the
  16-entry vector (the network's input and labels).

For every policy the report gives the geometric-mean slowdown of its
choices against the exhaustive best, beside the network's and the rule's.

    python -m paper_1511_02494_gb300.classifiers [--data DIR]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
CLASSES = ("CML", "MB", "IMB", "CMP")


def _geomean(a):
    return float(np.exp(np.mean(np.log(a))))


def rule_classes(prof: np.ndarray) -> np.ndarray:
    """Class of each stored probe triple under the library's rule."""
    import paper_1511_02494_gb300 as sp
    out = []
    for s_noxmiss, s_inflate, s_balance in prof:
        p = sp.Profile()
        p.s_noxmiss, p.s_inflate, p.s_balance = float(s_noxmiss), float(s_inflate), float(s_balance)
        out.append(sp.spmv_classify_profile(p))
    return np.array(out, np.int64)


def evaluate(data_dir: str = DATA) -> dict:
    from sklearn.naive_bayes import GaussianNB
    from sklearn.tree import DecisionTreeClassifier
    import paper_1511_02494_gb300 as sp

    d = np.load(os.path.join(data_dir, "selector_dataset.npz"))
    seeds, vec, times = d["seed"], d["vec"].astype(np.float64), d["times"]
    tr, te = np.where(seeds % 5 != 0)[0], np.where(seeds % 5 == 0)[0]
    best = times.min(1)
    cls = rule_classes(d["prof"])
    variant_of_class = np.array([sp.spmv_class_variant(c) for c in range(4)])
    labels = times.argmin(1)

    def slowdown(idx, pick):
        return _geomean(times[idx, pick] / best[idx])

    report = {"matrices": {"train": int(len(tr)), "test": int(len(te))},
              "class_counts_test": {CLASSES[c]: int((cls[te] == c).sum()) for c in range(4)},
              "policies": {}}
    models = {"decision_tree": lambda: DecisionTreeClassifier(random_state=0),
              "naive_bayes": lambda: GaussianNB()}
    for name, make in models.items():
        # the paper's set-up: Table 1 features -> rule class -> variant
        m = make().fit(vec[tr, :14], cls[tr])
        pc = m.predict(vec[te, :14])
        report["policies"][f"{name}_class"] = {
            "class_accuracy": float(np.mean(pc == cls[te])),
            "slowdown_vs_best": slowdown(te, variant_of_class[pc]),
        }
        # the network's set-up: 16 features -> fastest variant
        m = make().fit(vec[tr], labels[tr])
        pv = m.predict(vec[te])
        report["policies"][f"{name}_variant"] = {
            "variant_accuracy": float(np.mean(pv == labels[te])),
            "slowdown_vs_best": slowdown(te, pv),
        }
    report["policies"]["profiling_rule"] = {"slowdown_vs_best": slowdown(te, variant_of_class[cls[te]])}
    with open(os.path.join(data_dir, "selector_report.json")) as f:
        net = json.load(f)["test"]
    report["policies"]["learned_selector"] = {
        "variant_accuracy": 1.0 - net["misselection_mlp"],
        "slowdown_vs_best": net["slowdown_vs_best_geomean"]["mlp_with_fallback"]}
    return report


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--data", default=DATA)
    args = ap.parse_args()
    rep = evaluate(args.data)
    with open(os.path.join(args.data, "classifier_report.json"), "w") as f:
        json.dump(rep, f, indent=1)
    print(json.dumps(rep, indent=1))


if __name__ == "__main__":
    main()
