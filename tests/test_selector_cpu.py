"""Learned selector without a GPU: model files, the host forward pass against
the oracle's fixed-order fmaf chain (bit for bit), and the margin fallback to
the profiling rule (Section 3.2.1)."""
import os

import numpy as np
import pytest

import oracle
import paper_1511_02494_gb300 as sp
from paper_1511_02494_gb300 import _abi
from paper_1511_02494_gb300.build import build


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build()
    sp.lib()


def _params(h1=64, h2=64, k=7, seed=0):
    g = np.random.default_rng(seed)
    return {"mean": g.standard_normal(16).astype(np.float32),
            "istd": (0.5 + g.random(16)).astype(np.float32),
            "W1": (g.standard_normal((h1, 16)) * 0.3).astype(np.float32),
            "b1": (g.standard_normal(h1) * 0.1).astype(np.float32),
            "W2": (g.standard_normal((h2, h1)) * 0.15).astype(np.float32),
            "b2": (g.standard_normal(h2) * 0.1).astype(np.float32),
            "W3": (g.standard_normal((k, h2)) * 0.15).astype(np.float32),
            "b3": (g.standard_normal(k) * 0.1).astype(np.float32)}


def _packed(P):
    return np.concatenate([P[n].reshape(-1) for n in ("W1", "b1", "W2", "b2", "W3", "b3")])


def _model(P, margin=0.0, variants=None):
    k = P["W3"].shape[0]
    variants = list(range(k)) if variants is None else variants
    return sp.spmv_model_create(P["W1"].shape[0], P["W2"].shape[0], k, P["mean"], P["istd"],
                                _packed(P), variants, margin)


def test_host_logits_bit_exact_with_oracle():
    for seed in range(3):
        P = _params(seed=seed)
        m = _model(P)
        v = np.random.default_rng(seed + 10).standard_normal((50, 16)).astype(np.float32) * 3
        ref = oracle.mlp_forward_f32(P, v)
        for s in range(50):
            assert np.array_equal(sp.spmv_model_logits(m, v[s], 7), ref[s])


def test_model_file_roundtrip_and_corruption(tmp_path):
    P = _params(32, 16, 5, seed=4)
    m = _model(P, margin=0.25, variants=[0, 1, 3, 4, 6])
    path = tmp_path / "m.bin"
    sp.spmv_model_save(m, path)
    m2 = sp.spmv_model_load(path)
    v = np.random.default_rng(1).standard_normal(16).astype(np.float32)
    assert np.array_equal(sp.spmv_model_logits(m, v, 5), sp.spmv_model_logits(m2, v, 5))
    raw = path.read_bytes()
    for bad in (raw[:-3], raw + b"x", b"XXXXXXXX" + raw[8:], raw[:20]):
        path.write_bytes(bad)
        with pytest.raises(sp.SpmvError) as e:
            sp.spmv_model_load(path)
        assert e.value.status == 7
    with pytest.raises(sp.SpmvError) as e:
        sp.spmv_model_load(tmp_path / "missing.bin")
    assert e.value.status == 7


def test_model_create_rejects_bad_models():
    P = _params(8, 8, 3)
    with pytest.raises(sp.SpmvError):
        _model(P, variants=[0, 1, 9])
    P["W2"][0, 0] = np.nan
    with pytest.raises(sp.SpmvError):
        _model(P)


def test_select_model_margin_fallback_matches_oracle():
    P = _params(seed=7)
    g = np.random.default_rng(3)
    t = sp.spmv_default_thresholds()
    tau = (t.tau_noxmiss, t.tau_inflate, t.tau_balance)
    table = [sp.spmv_class_variant(c) for c in range(4)]
    for margin_thr in (0.0, 0.5, 100.0):
        m = _model(P, margin=margin_thr, variants=[6, 5, 4, 3, 2, 1, 0])
        for _ in range(40):
            f = _abi.Features()
            vec = (g.standard_normal(16) * 2).astype(np.float32)
            for i in range(16):
                f.vec[i] = float(vec[i])
            prof = _abi.Profile()
            prof.s_noxmiss, prof.s_inflate, prof.s_balance = 0.8 + g.random(3) * 3
            ch = sp.spmv_select_model(f, m, prof)
            logits = oracle.mlp_forward_f32(P, vec)[0]
            best, margin = oracle.argmax(logits)
            assert ch.margin == np.float32(margin)
            if margin < margin_thr:
                cls = oracle.profile_class(prof.s_noxmiss, prof.s_inflate, prof.s_balance, tau)
                assert ch.used_fallback == 1 and ch.variant == oracle.class_variant(cls, table)
            else:
                assert ch.used_fallback == 0 and ch.variant == [6, 5, 4, 3, 2, 1, 0][best]
            ch2 = sp.spmv_select_model(f, m)  # no profile: never falls back
            assert ch2.used_fallback == 0 and ch2.variant == [6, 5, 4, 3, 2, 1, 0][best]


_LAUNCH = np.array([[0, 0, 0], [1, 1, 1024], [4, 1, 1024], [1, 4096, 32], [4, 4096, 32]], np.int32)


def test_second_level_model_file_and_launch_table(tmp_path):
    """A model with a launch table (the second level of selection) is saved
    as SPMVMLP2, loads back with its table, and its choice carries the
    launch parameters of the output the oracle's forward ranks first."""
    P = _params(32, 32, 5, seed=11)
    sl = sp.VARIANT_IDS["sliced"]
    m = _model(P, variants=[sl] * 5)
    sp.spmv_model_set_launch(m, _LAUNCH)
    path = tmp_path / "sub.bin"
    sp.spmv_model_save(m, path)
    assert path.read_bytes()[:8] == b"SPMVMLP2"
    m2 = sp.spmv_model_load(path)
    g = np.random.default_rng(12)
    for _ in range(30):
        f = _abi.Features()
        vec = (g.standard_normal(16) * 2).astype(np.float32)
        for i in range(16):
            f.vec[i] = float(vec[i])
        best, _ = oracle.argmax(oracle.mlp_forward_f32(P, vec)[0])
        for mm in (m, m2):
            ch = sp.spmv_select_model(f, mm)
            assert ch.variant == sl
            assert [ch.threads_per_row, ch.block_nnz, ch.items_per_warp] == _LAUNCH[best].tolist()
    # a truncated table is a corrupt file; a plain model still saves as version 1
    (tmp_path / "cut.bin").write_bytes(path.read_bytes()[:-4])
    with pytest.raises(sp.SpmvError):
        sp.spmv_model_load(tmp_path / "cut.bin")
    sp.spmv_model_save(_model(P), tmp_path / "v1.bin")
    assert (tmp_path / "v1.bin").read_bytes()[:8] == b"SPMVMLP1"


def test_second_level_rejects_invalid_launch_parameters():
    P = _params(16, 16, 5, seed=13)
    bad = _LAUNCH.copy()
    bad[2] = [3, 1, 1024]  # three slices per warp: not a SLICED choice
    m = _model(P, variants=[sp.VARIANT_IDS["sliced"]] * 5)
    with pytest.raises(sp.SpmvError):
        sp.spmv_model_set_launch(m, bad)
    m = _model(P, variants=[sp.VARIANT_IDS["subwarp"]] * 5)
    with pytest.raises(sp.SpmvError):  # items_per_warp 7: not a valid choice
        sp.spmv_model_set_launch(m, np.array([[0, 0, 7]] * 5, np.int32))


def test_refined_selection_applies_the_second_level_to_its_variant():
    """Two levels: the first model's choice, then, when it names SLICED, the
    second model's launch parameters; another variant keeps none."""
    sl, sw = sp.VARIANT_IDS["sliced"], sp.VARIANT_IDS["subwarp"]
    P1, P2 = _params(16, 16, 2, seed=21), _params(16, 16, 5, seed=22)
    first = _model(P1, variants=[sl, sw])
    sub = _model(P2, variants=[sl] * 5)
    sp.spmv_model_set_launch(sub, _LAUNCH)
    g = np.random.default_rng(23)
    seen = set()
    for _ in range(60):
        f = _abi.Features()
        vec = (g.standard_normal(16) * 2).astype(np.float32)
        for i in range(16):
            f.vec[i] = float(vec[i])
        b1, _ = oracle.argmax(oracle.mlp_forward_f32(P1, vec)[0])
        b2, _ = oracle.argmax(oracle.mlp_forward_f32(P2, vec)[0])
        ch = sp.spmv_select_model_refined(f, first, sub)
        assert ch.variant == [sl, sw][b1]
        got = [ch.threads_per_row, ch.block_nnz, ch.items_per_warp]
        assert got == (_LAUNCH[b2].tolist() if b1 == 0 else [0, 0, 0])
        assert sp.spmv_select_model_refined(f, first, None).variant == ch.variant
        seen.add(b1)
    assert seen == {0, 1}
