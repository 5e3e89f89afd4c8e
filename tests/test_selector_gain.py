"""What the learned selector gains over the method without it, on the
committed training set (GB300 timings of every variant on 2000 seeded
matrices) and the committed model: on the held-out fifth of the matrices
(seed % 5 == 0) the network's choice -- computed here with the oracle's
forward pass -- is compared with the exhaustive best, with the paper's
profiling rule (Section 3.2.1) and with the best single fixed variant.  CPU
only."""
import os

import numpy as np
import pytest

import oracle
import paper_1511_02494_gb300 as sp
from paper_1511_02494_gb300.build import build

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1511_02494_gb300", "data")


def _read_model(path):
    raw = open(path, "rb").read()
    assert raw[:8] == b"SPMVMLP1"
    h1, h2, k = np.frombuffer(raw, np.int32, 3, 8)
    f = np.frombuffer(raw, np.float32, offset=20)
    mean, istd = f[:16], f[16:32]
    o = 32
    P = {"mean": mean, "istd": istd}
    for name, shape in (("W1", (h1, 16)), ("b1", (h1,)), ("W2", (h2, h1)), ("b2", (h2,)),
                        ("W3", (k, h2)), ("b3", (k,))):
        n = int(np.prod(shape))
        P[name] = f[o:o + n].reshape(shape)
        o += n
    variants = np.frombuffer(raw, np.int32, k, 20 + 4 * o)
    return P, variants, int(k)


@pytest.fixture(scope="module")
def data():
    d = np.load(os.path.join(DATA, "selector_dataset.npz"))
    P, variants, k = _read_model(os.path.join(DATA, "selector_mlp.bin"))
    return d, P, variants, k


def _geomean(a):
    return float(np.exp(np.mean(np.log(a))))


def test_dataset_shape(data):
    d, P, variants, k = data
    assert d["seed"].size == 2000 and d["times"].shape == (2000, k) and k <= len(sp.VARIANTS)
    assert np.array_equal(np.sort(d["seed"]), np.arange(2000))
    assert np.all(d["times"] > 0)


def test_learned_selector_beats_the_profiling_rule_on_held_out_matrices(data):
    d, P, variants, k = data
    test = np.where(d["seed"] % 5 == 0)[0]
    times = d["times"][test]
    best = times.min(1)
    logits = oracle.mlp_forward_f32(P, d["vec"][test])
    pick = variants[logits.argmax(1)]
    t_mlp = times[np.arange(len(test)), pick]
    t_rule = times[np.arange(len(test)), d["rule_variant"][test]]
    fixed = min(_geomean(times[:, v] / best) for v in range(k))
    slow_mlp, slow_rule = _geomean(t_mlp / best), _geomean(t_rule / best)
    # within 5 % of the exhaustive best, and better than the rule and any
    # single fixed variant
    assert slow_mlp <= 1.05
    assert slow_mlp < slow_rule
    assert slow_mlp < fixed
    # the features it needs cost far fewer plain SpMVs than the profiling runs
    plain = times[:, 0]
    feat = np.median(d["features_ms"][test] / plain)
    prof = np.median(d["profile_ms"][test] / plain)
    assert feat < 20 and feat < prof / 5


def test_library_logits_equal_oracle_on_the_dataset(data):
    build()
    d, P, variants, k = data
    m = sp.spmv_model_load(os.path.join(DATA, "selector_mlp.bin"))
    ref = oracle.mlp_forward_f32(P, d["vec"][:300])
    for i in range(300):
        assert np.array_equal(sp.spmv_model_logits(m, d["vec"][i], k), ref[i])


def test_class_variant_table_is_the_per_class_best_on_training_data(data):
    """The profiling rule's class -> variant table is calibrated: for each
    class the rule names on the training matrices, the mapped variant has the
    lowest geometric-mean slowdown against the exhaustive best."""
    d, P, variants, k = data
    tr = np.where(d["seed"] % 5 != 0)[0]
    times = d["times"][tr]
    best = times.min(1)
    cls = np.array([oracle.profile_class(*p) for p in d["prof"][tr]])
    for c in range(4):
        m = cls == c
        if m.sum() < 20:
            continue
        slow = [_geomean(times[m, v] / best[m]) for v in range(k)]
        assert oracle.class_variant(c) == int(np.argmin(slow)), (c, slow)
