"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(hand-derived worked examples, closed forms, invariants, exact arithmetic and
brute force), never against the oracle's own formulas.  CPU only."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import synth


def _exact_row_sums(A, x):
    """Exact rational y_i = sum val_j * x_colj (every double is a rational)."""
    rp, ci, v = A.rowptr.numpy(), A.colind.numpy(), A.val.numpy()
    xs = [Fraction(float(t)) for t in np.asarray(x)]
    out = []
    for i in range(A.n_rows):
        s = Fraction(0)
        for j in range(rp[i], rp[i + 1]):
            s += Fraction(float(v[j])) * xs[ci[j]]
        out.append(s)
    return out


# --------------------------------------------------------------- SpMV (Alg. 1)
def test_spmv_matches_dense_brute_force():
    for seed in range(5):
        A = synth.random_csr(23, 17, 9, seed=seed)
        x = synth.uniform_vector(17, seed + 100)
        D = np.zeros((23, 17))
        rp, ci, v = A.rowptr.numpy(), A.colind.numpy(), A.val.numpy()
        for i in range(23):
            for j in range(rp[i], rp[i + 1]):
                D[i, ci[j]] = v[j]
        y = oracle.spmv(A, x)
        exact = _exact_row_sums(A, x)
        _, scale = oracle.spmv_ref(A, x)
        for i in range(23):
            # sequential FP64 sum of k terms: |err| <= k * u * sum|a x| (first order)
            k = rp[i + 1] - rp[i]
            assert abs(Fraction(y[i]) - exact[i]) <= Fraction(k * 2.0 ** -52 * scale[i] + 1e-300)
        np.testing.assert_allclose(y, D @ x.numpy(), rtol=0, atol=1e-13)


def test_spmv_integer_valued_is_exact_against_dense():
    g = np.random.default_rng(3)
    D = g.integers(-5, 6, size=(40, 31)).astype(np.float64)
    D[g.random((40, 31)) < 0.6] = 0.0
    D[7] = 0.0  # an empty row
    A = synth.dense_to_csr(torch.from_numpy(D))
    x = g.integers(-9, 10, size=31).astype(np.float64)
    y = oracle.spmv(A, x)
    assert np.array_equal(y, D @ x)
    assert y[7] == 0.0


def test_spmv_identity_and_permutation_exact():
    n = 257
    x = synth.uniform_vector(n, 1).numpy()
    I = synth.dense_to_csr(torch.eye(n, dtype=torch.float64))
    assert np.array_equal(oracle.spmv(I, x), x)
    perm = np.random.default_rng(5).permutation(n)
    P = np.zeros((n, n))
    P[np.arange(n), perm] = 1.0
    assert np.array_equal(oracle.spmv(synth.dense_to_csr(torch.from_numpy(P)), x), x[perm])


def test_spmv_laplacian_closed_forms():
    A = synth.laplacian_2d_5pt(64, 64)
    # A 1 = 4 - (number of neighbours): 0 inside, 1 on an edge, 2 at a corner
    y = oracle.spmv(A, np.ones(4096))
    gy, gx = np.divmod(np.arange(4096), 64)
    missing = (gy == 0).astype(int) + (gy == 63) + (gx == 0) + (gx == 63)
    assert np.array_equal(y, missing.astype(np.float64))
    # linear field a*gx + b*gy + c is annihilated at interior points
    f = (3 * gx - 5 * gy + 7).astype(np.float64)
    y = oracle.spmv(A, f)
    inner = (gy > 0) & (gy < 63) & (gx > 0) & (gx < 63)
    assert np.all(y[inner] == 0.0)


def test_spmv_empty_matrix_and_rows():
    A = synth.random_csr(0, 5, 3)
    assert oracle.spmv(A, np.ones(5)).size == 0
    A = synth.random_csr(50, 40, 0, seed=1)  # all rows empty
    assert np.all(oracle.spmv(A, np.ones(40)) == 0.0)


def test_spmv_ref_is_within_one_ulp_of_exact():
    A = synth.random_csr(30, 30, 30, seed=7, empty_frac=0.0)
    # cancellation-heavy values
    A.val = torch.from_numpy(np.random.default_rng(7).standard_normal(A.nnz) * 1e8)
    # x = 1: every product is exact, so the compensated sum is within one ulp
    ones = np.ones(30)
    y1, s1 = oracle.spmv_ref(A, ones)
    exact1 = _exact_row_sums(A, ones)
    for i in range(30):
        assert abs(Fraction(y1[i]) - exact1[i]) <= Fraction(math.ulp(abs(y1[i])))
        assert s1[i] == pytest.approx(float(np.abs(A.val.numpy()[A.rowptr[i]:A.rowptr[i + 1]]).sum()))
    # general x: each product adds at most u |p| of rounding before the sum
    x = synth.uniform_vector(30, 8)
    y, scale = oracle.spmv_ref(A, x)
    exact = _exact_row_sums(A, x)
    for i in range(30):
        bound = Fraction(math.ulp(abs(y[i]))) + Fraction(2.0 ** -52) * Fraction(scale[i])
        assert abs(Fraction(y[i]) - exact[i]) <= bound
    # the subset form agrees with the full form
    rows = np.array([29, 0, 13], np.int64)
    ys, ss = oracle.spmv_ref(A, x, rows)
    assert np.array_equal(ys, y[rows]) and np.array_equal(ss, scale[rows])


def test_spmv_lowp_equals_fp64_on_representable_values():
    A = synth.random_csr(60, 50, 12, seed=2)
    # values with 8 significant bits are exact in bfloat16 and float32
    g = np.random.default_rng(2)
    A.val = torch.from_numpy(g.integers(-128, 128, A.nnz).astype(np.float64) / 64.0)
    x = synth.uniform_vector(50, 3)
    ref = oracle.spmv(A, x)
    assert np.array_equal(oracle.spmv_lowp(A, x, 1, oracle.round_f32(A.val)), ref)
    assert np.array_equal(oracle.spmv_lowp(A, x, 2, oracle.round_bf16(A.val)), ref)


def test_spmv_lowp32_exact_on_small_integers_and_bounded_otherwise():
    A = synth.random_csr(80, 60, 20, seed=4)
    g = np.random.default_rng(4)
    # values and x with few bits: every float operation is exact
    A.val = torch.from_numpy(g.integers(-16, 17, A.nnz).astype(np.float64))
    x = g.integers(-16, 17, 60).astype(np.float64)
    assert np.array_equal(oracle.spmv_lowp32(A, x, 1, oracle.round_f32(A.val)), oracle.spmv(A, x))
    # general values: within the FP32 rounding bound of the float-valued product
    A.val = torch.from_numpy(g.standard_normal(A.nnz))
    xr = synth.uniform_vector(60, 6)
    low = oracle.round_bf16(A.val)
    exact = oracle.spmv_lowp(A, oracle.round_f32(xr).astype(np.float64), 2, low)
    _, scale = oracle.spmv_ref(A, xr)
    k = np.diff(A.rowptr.numpy())
    got = oracle.spmv_lowp32(A, xr, 2, low)
    assert np.all(np.abs(got - exact) <= (k + 1) * 2.0 ** -23 * scale * 1.01 + 1e-300)


# --------------------------------------------------------------- rounding
def test_bf16_rounding_golden(golden_dir):
    d = json.load(open(os.path.join(golden_dir, "bf16_rounding.json")))
    for c in d["cases"]:
        v = Fraction(0)
        for e in c["pow2"]:
            if isinstance(e, str):
                v -= Fraction(2) ** int(e[1:])
            else:
                v += Fraction(2) ** e
        if c.get("neg"):
            v = -v
        got = int(oracle.round_bf16(np.array([float(v)]))[0])
        assert got == int(c["bits"], 16), (c, hex(got))


def _bf16_value(bits):
    """Exact value of a finite bfloat16 bit pattern."""
    s = -1 if bits & 0x8000 else 1
    e = (bits >> 7) & 0xFF
    f = bits & 0x7F
    if e == 0:
        return s * Fraction(f) * Fraction(2) ** -133
    return s * (1 + Fraction(f, 128)) * Fraction(2) ** (e - 127)


def test_bf16_rounding_brute_force_nearest_even():
    """For random doubles across the range, the result is the nearest
    bfloat16 by exact arithmetic, ties to the even fraction."""
    g = np.random.default_rng(11)
    vals = np.concatenate([g.standard_normal(300) * 2.0 ** g.integers(-140, 120, 300),
                           g.uniform(-1, 1, 100)])
    got = oracle.round_bf16(vals)
    for v, b in zip(vals, got):
        b = int(b)
        fv = Fraction(float(v))
        mag = abs(fv)
        # candidates: the result and its neighbours
        cand = [(c, _bf16_value(c)) for c in {b & 0x7FFF, max((b & 0x7FFF) - 1, 0), (b & 0x7FFF) + 1}
                if ((c >> 7) & 0xFF) != 0xFF]
        best = min(abs(_bf16_value(c) - mag) for c, _ in cand)
        assert abs(_bf16_value(b & 0x7FFF) - mag) == best
        ties = [c for c, val in cand if abs(val - mag) == best]
        if len(ties) > 1:
            assert (b & 1) == 0
        assert (b >> 15) == (1 if v < 0 else 0)


def test_f32_rounding_matches_numpy_cast():
    v = np.random.default_rng(4).standard_normal(1000) * 1e3
    assert np.array_equal(oracle.round_f32(v), v.astype(np.float32))


# --------------------------------------------------------------- Table 1 features
def test_features_tiny_worked_example(golden_dir):
    d = json.load(open(os.path.join(golden_dir, "features_tiny_4x4.json")))
    D = np.zeros((4, 4))
    for i, r in enumerate(d["rows"]):
        D[i, r] = 1.0
    A = synth.dense_to_csr(torch.from_numpy(D))
    for lb, misses in d["misses_sum_by_line_bytes"].items():
        f = oracle.features(A, line_bytes=int(lb), l2_bytes=1 << 20)
        assert f["misses_sum"] == misses
    f = oracle.features(A, line_bytes=64, l2_bytes=1 << 20)
    for k in ("nnz_sum", "nnz_sumsq", "nnz_min", "nnz_max", "bw_min", "bw_max", "bw_sum",
              "bw_sumsq", "ngroups_sum"):
        assert f[k] == d[k], k
    assert f["nnz_avg"] == d["nnz_avg"]
    assert f["nnz_sd"] == pytest.approx(math.sqrt(d["nnz_sd_sq"]), rel=1e-15)
    pr = d["per_row"]
    q = [(n << 32) // m for n, m in pr["disp"]]
    assert f["disp_sum"] == sum(q)
    assert f["disp_avg"] == pytest.approx(sum(Fraction(n, m) for n, m in pr["disp"]) / 4, rel=1e-9)
    cq = [(n << 32) // m for n, m in pr["clust"]]
    assert f["clust_sum"] == sum(cq)
    assert f["clustering"] == pytest.approx(float(sum(Fraction(n, m) for n, m in pr["clust"]) / 4),
                                            rel=1e-9)
    assert f["size"] == 1.0 and f["density"] == 7 / 16


def test_features_laplacian_64_golden(golden_dir):
    d = json.load(open(os.path.join(golden_dir, "features_laplacian2d_64.json")))
    A = synth.laplacian_2d_5pt(64, 64)
    f = oracle.features(A, line_bytes=128, l2_bytes=126 << 20)
    for k in ("nnz_sum", "nnz_sumsq", "nnz_min", "nnz_max", "bw_sum", "bw_sumsq", "bw_min",
              "bw_max", "ngroups_sum", "misses_sum"):
        assert f[k] == d[k], k
    assert f["density"] == d["density"] and f["nnz_avg"] == d["nnz_avg"]
    assert f["miss_ratio"] == d["miss_ratio"]
    assert sum(t["count"] for t in d["row_types"]) == d["n"]
    # per-row fixed-point sums from the hand-derived row classes
    disp = sum(t["count"] * ((t["nnz"] << 32) // (t["bw"] + 1)) for t in d["row_types"])
    clust = sum(t["count"] * ((t["ngroups"] << 32) // t["nnz"]) for t in d["row_types"])
    assert f["disp_sum"] == disp and f["clust_sum"] == clust
    exact_clust = sum(Fraction(t["count"] * t["ngroups"], t["nnz"]) for t in d["row_types"]) / 4096
    assert f["clustering"] == pytest.approx(float(exact_clust), abs=4096 * 2.0 ** -32)
    f64 = oracle.features(A, line_bytes=64, l2_bytes=0)
    assert f64["misses_sum"] == d["misses_sum"] and f64["size"] == 0.0


@pytest.mark.parametrize("n", [4, 8, 13])
def test_features_27pt_stencil_closed_forms(n):
    A = synth.stencil_27pt(n, seed=0)
    f = oracle.features(A, line_bytes=128, l2_bytes=0)
    assert f["nnz"] == (3 * n - 2) ** 3
    assert (f["nnz_min"], f["nnz_max"]) == (8, 27)
    assert f["bw_max"] == 2 * (n * n + n + 1) and f["bw_min"] == n * n + n + 1
    # each row of the stencil has 9 groups (one per (dz,dy) pair present)
    per_row = (3 - (np.arange(n) == 0) - (np.arange(n) == n - 1))
    groups = int(np.sum(np.multiply.outer(per_row, per_row)) * n)  # pairs (z, y) present x rows in x
    assert f["ngroups_sum"] == groups


def test_features_empty_and_degenerate():
    f = oracle.features(synth.random_csr(0, 0, 0), 128, 0)
    assert f["nnz"] == 0 and f["nnz_min"] == 0 and f["nnz_avg"] == 0.0
    A = synth.random_csr(10, 10, 0, seed=0)
    f = oracle.features(A, 128, 1 << 20)
    assert f["nnz_max"] == 0 and f["misses_sum"] == 0 and f["clustering"] == 0.0
    # a single full dense row: one group, disp 1
    A = synth.dense_to_csr(torch.ones(1, 300, dtype=torch.float64))
    f = oracle.features(A, 128, 1 << 20)
    assert f["ngroups_sum"] == 1 and f["disp_sum"] == 1 << 32 and f["bw_max"] == 299


def test_features_invariants_random():
    for seed in range(4):
        A = synth.random_csr(200, 500, 40, seed=seed)
        f = oracle.features(A, 64, 1 << 30)
        lens = (A.rowptr[1:] - A.rowptr[:-1]).numpy()
        assert f["nnz_sum"] == A.nnz == int(lens.sum())
        assert f["nnz_sumsq"] == int((lens.astype(np.int64) ** 2).sum())
        assert f["nnz_sd"] == pytest.approx(float(np.std(lens)), rel=1e-12)
        # misses and groups never exceed nnz; every nonempty row has >= 1 of each
        nonempty = int((lens > 0).sum())
        assert nonempty <= f["ngroups_sum"] <= A.nnz and nonempty <= f["misses_sum"] <= A.nnz
        # shifting all columns by a constant changes nothing
        B = synth.HostCSR(A.n_rows, A.n_cols + 3, A.rowptr, A.colind + 3, A.val)
        g = oracle.features(B, 64, 1 << 30)
        for k in ("bw_sum", "ngroups_sum", "misses_sum", "disp_sum", "clust_sum"):
            assert f[k] == g[k]


def test_feature_vector_definition():
    A = synth.laplacian_2d_5pt(64, 64)
    f = oracle.features(A, 128, 1 << 30)
    v = f["vec"]
    assert v.dtype == np.float32 and v.shape == (16,)
    assert v[0] == 1.0 and v[14] == np.float32(math.log2(4097.0))
    assert v[2] == np.float32(2.0)  # log2(1 + 3)


# --------------------------------------------------------------- profile rule
def test_profile_rule_golden(golden_dir):
    d = json.load(open(os.path.join(golden_dir, "profile_rule_cases.json")))
    for c in d["cases"]:
        got = oracle.profile_class(*c["s"], tau=tuple(d["tau"]))
        assert d["classes"][got] == c["class"], c


def test_profile_rule_nan_never_selected():
    tau = (1.1, 1.1, 1.1)
    assert oracle.profile_class(float("nan"), 1.0, 1.0, tau) == oracle.CMP
    assert oracle.profile_class(float("nan"), 2.0, 1.0, tau) == oracle.MB


def test_profile_rule_needs_explicit_thresholds():
    # the paper prints no threshold values, so the oracle holds none
    with pytest.raises(TypeError):
        oracle.profile_class(2.0, 1.0, 1.0)
    # the same speedups classify differently under different thresholds
    assert oracle.profile_class(1.3, 1.2, 1.0, (1.25, 1.5, 3.0)) == oracle.CML
    assert oracle.profile_class(1.3, 1.2, 1.0, (1.4, 1.1, 3.0)) == oracle.MB
    assert oracle.profile_class(1.3, 1.2, 1.0, (1.4, 1.5, 3.0)) == oracle.CMP


def test_class_to_variant_default_is_table2():
    # Table 2 (Section 3.3): CML -> software prefetching of x, MB -> delta
    # coding of column indices, IMB -> dynamic scheduling, CMP -> unrolling
    # with vectorisation; in the library's variant names
    names = ("scalar", "subwarp", "stream", "merge", "dynamic", "latency", "compressed", "sliced")
    got = [names[oracle.class_variant(c)] for c in range(4)]
    assert got == ["latency", "compressed", "dynamic", "subwarp"]
    assert oracle.class_variant(4) == -1 and oracle.class_variant(-1) == -1


def test_class_to_variant_follows_the_given_table():
    table = (3, 0, 7, 2)
    assert [oracle.class_variant(c, table) for c in range(4)] == list(table)
    assert oracle.class_variant(5, table) == -1


# --------------------------------------------------------------- partitions
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_static_partition_is_smallest_row_reaching_target(seed):
    A = synth.zipf_rows(3000, 3000, 1.5, 800, seed=seed)
    rp = A.rowptr.numpy().astype(np.int64)
    for W in (1, 7, 64, 5000):
        b = oracle.static_partition(A, W)
        targets = (np.arange(W) * A.nnz) // W
        assert np.array_equal(b[:-1], np.searchsorted(rp, targets, side="left"))
        assert b[-1] == A.n_rows and np.all(np.diff(b) >= 0)


def _csr_lengths(lengths):
    rp = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int32)
    n = int(rp[-1])
    ci = np.concatenate([np.arange(L) for L in lengths]).astype(np.int32) if n else np.zeros(0, np.int32)
    return synth.HostCSR(len(lengths), max(max(lengths, default=1), 1), torch.from_numpy(rp),
                         torch.from_numpy(ci), torch.ones(n, dtype=torch.float64))


def test_sliced_segments_hand_example():
    """Row lengths 3, 5000, 1, 2048, 2049, 0 with cap 2 and segments of 2048:
    long rows 0, 1, 3, 4 (ascending); segments 1, 3, 1, 2 -> offsets 0, 1, 4,
    5, 7; row 1 = [3, 2051), [2051, 4099), [4099, 5003); row 4 starts at
    7052: [7052, 9100), [9100, 9101); single-segment rows 0 and 3 write y
    themselves; rows with several segments are list entries 1 and 3."""
    A = _csr_lengths([3, 5000, 1, 2048, 2049, 0])
    lst, off, be, srow, fix, sfix = oracle.sliced_segments(A, cap=2, seg=2048)
    assert list(lst) == [0, 1, 3, 4] and list(off) == [0, 1, 4, 5, 7]
    assert be.tolist() == [[0, 3], [3, 2051], [2051, 4099], [4099, 5003], [5004, 7052],
                           [7052, 9100], [9100, 9101]]
    assert list(srow) == [0, -1, -1, -1, 3, -1, -1]
    assert list(fix) == [1, 3] and list(sfix) == [-1, 0, 0, 0, -1, 1, 1]


@pytest.mark.parametrize("cap,seg", [(32, 2048), (1024, 2048), (0, 256)])
def test_sliced_segments_cover_each_long_row(cap, seg):
    A = synth.zipf_rows(4000, 4000, 1.3, 3500, seed=2)
    lst, off, be, srow, fix, sfix = oracle.sliced_segments(A, cap, seg)
    rp = A.rowptr.numpy().astype(np.int64)
    lens = np.diff(rp)
    assert np.array_equal(lst, np.flatnonzero(lens > cap))
    for q, r in enumerate(lst):
        segs = be[off[q]:off[q + 1]]
        assert segs[0, 0] == rp[r] and segs[-1, 1] == rp[r + 1]
        assert np.all(segs[1:, 0] == segs[:-1, 1]) and np.all(segs[:, 1] - segs[:, 0] <= seg)
        assert np.all(segs[:, 1] > segs[:, 0])
        single = off[q + 1] - off[q] == 1
        assert np.all(srow[off[q]:off[q + 1]] == (r if single else -1))
        if not single:
            t = int(np.flatnonzero(fix == q)[0])
            assert np.all(sfix[off[q]:off[q + 1]] == t)
    assert len(fix) == int(np.sum(np.diff(off) > 1))


def test_dyn_tiers_hand_example():
    """lim_s 4, segments of 100: lengths 4 -> none; 5 and 64 -> m1; 65 and
    100 -> m2; 101 -> long, 2 segments; 250 -> long, 3 segments."""
    A = _csr_lengths([4, 5, 64, 65, 100, 101, 0, 250])
    m1, m2, lr, sc = oracle.dyn_tiers(A, lim_s=4, seg=100)
    assert list(m1) == [1, 2] and list(m2) == [3, 4]
    assert list(lr) == [5, 7] and list(sc) == [2, 3]


def test_dyn_tiers_partition_the_rows():
    A = synth.zipf_rows(5000, 5000, 1.4, 3000, seed=3)
    lens = np.diff(A.rowptr.numpy().astype(np.int64))
    m1, m2, lr, sc = oracle.dyn_tiers(A, lim_s=16, seg=512)
    assert np.array_equal(m1, np.flatnonzero((lens > 16) & (lens <= 64)))
    assert np.array_equal(m2, np.flatnonzero((lens > 64) & (lens <= 512)))
    assert np.array_equal(lr, np.flatnonzero(lens > 512))
    assert np.array_equal(sc, -(-lens[lr] // 512))


def test_row_blocks_cover_rows_by_window():
    A = synth.zipf_rows(2000, 2000, 1.6, 700, seed=4)
    rp = A.rowptr.numpy().astype(np.int64)
    for B in (64, 256, 1024):
        R = oracle.row_blocks(A, B)
        nb = -(-A.nnz // B)
        assert R.size == nb + 1 and R[0] == 0 and R[-1] == A.n_rows
        assert np.array_equal(R[:-1], np.searchsorted(rp, np.arange(nb) * B, side="left"))


def _merge_coords_by_sorting(rp, items):
    """Merge path by explicit sort of all items: row end i has key
    (rowptr[i+1], 0, i), nonzero j has key (j, 1, j)."""
    n = rp.size - 1
    nnz = int(rp[-1])
    keys = [(int(rp[i + 1]), 0, i) for i in range(n)] + [(j, 1, j) for j in range(nnz)]
    keys.sort()
    is_row = np.array([k[1] == 0 for k in keys], dtype=np.int64)
    rows_before = np.concatenate([[0], np.cumsum(is_row)])
    total = n + nnz
    parts = max(1, -(-total // items))
    d = np.minimum(np.arange(parts + 1) * items, total)
    return rows_before[d], d - rows_before[d]


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_merge_path_matches_sorted_merge(seed):
    A = synth.random_csr(150, 90, 30, seed=seed, empty_frac=0.3)
    rp = A.rowptr.numpy().astype(np.int64)
    for items in (1, 5, 32, 224, 10 ** 6):
        rs, ns = oracle.merge_path(A, items)
        er, en = _merge_coords_by_sorting(rp, items)
        assert np.array_equal(rs, er) and np.array_equal(ns, en)


def test_compress_u16_decodes_and_flags_wide_rows():
    A = synth.random_csr(300, 200_000, 6, seed=9)
    base, off, wide = oracle.compress_u16(A)
    rp, ci = A.rowptr.numpy(), A.colind.numpy()
    n_wide = 0
    for i in range(A.n_rows):
        b, e = rp[i], rp[i + 1]
        if b == e:
            assert base[i] == 0
            continue
        if ci[e - 1] - ci[b] >= 65536:
            n_wide += 1
            assert base[i] == -1
        else:
            assert np.array_equal(base[i] + off[b:e].astype(np.int64), ci[b:e])
    assert wide == n_wide > 0


# --------------------------------------------------------------- MLP
def _params(h1=64, h2=64, k=7, seed=0, scale=0.3):
    g = np.random.default_rng(seed)
    return {"mean": g.standard_normal(16).astype(np.float32),
            "istd": (0.5 + g.random(16)).astype(np.float32),
            "W1": (g.standard_normal((h1, 16)) * scale).astype(np.float32),
            "b1": (g.standard_normal(h1) * 0.1).astype(np.float32),
            "W2": (g.standard_normal((h2, h1)) * scale / 2).astype(np.float32),
            "b2": (g.standard_normal(h2) * 0.1).astype(np.float32),
            "W3": (g.standard_normal((k, h2)) * scale / 2).astype(np.float32),
            "b3": (g.standard_normal(k) * 0.1).astype(np.float32)}


def test_mlp_forward_exact_on_dyadic_network():
    """Small dyadic weights make every float op exact: the result is the exact
    real-arithmetic network output."""
    g = np.random.default_rng(1)
    P = {k: (np.round(v * 8) / 8).astype(np.float32) for k, v in _params(8, 8, 4, 1).items()}
    P["istd"] = np.ones(16, np.float32)
    v = (g.integers(-8, 8, (5, 16)) / 4).astype(np.float32)
    got = oracle.mlp_forward_f32(P, v)
    z = v.astype(np.float64) - P["mean"]
    a1 = np.maximum(z @ P["W1"].T.astype(np.float64) + P["b1"], 0)
    a2 = np.maximum(a1 @ P["W2"].T.astype(np.float64) + P["b2"], 0)
    assert np.array_equal(got.astype(np.float64), a2 @ P["W3"].T.astype(np.float64) + P["b3"])


def test_mlp_forward_close_to_fp64():
    P = _params()
    v = np.random.default_rng(2).standard_normal((20, 16)).astype(np.float32)
    got = oracle.mlp_forward_f32(P, v)
    z = (v - P["mean"]).astype(np.float64) * P["istd"]
    a1 = np.maximum(z @ P["W1"].T.astype(np.float64) + P["b1"], 0)
    a2 = np.maximum(a1 @ P["W2"].T.astype(np.float64) + P["b2"], 0)
    ref = a2 @ P["W3"].T.astype(np.float64) + P["b3"]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-4)


def test_argmax_ties_to_lowest_and_margin():
    assert oracle.argmax(np.array([1, 3, 3, 2], np.float32)) == (1, 0.0)
    assert oracle.argmax(np.array([5, 1, 2], np.float32)) == (0, 3.0)


def test_mlp_gradients_match_finite_differences():
    P = _params(16, 12, 5, 3)
    g = np.random.default_rng(5)
    z = g.standard_normal((9, 16))
    lab = g.integers(0, 5, 9).astype(np.int32)
    P64 = {k: v.astype(np.float64) for k, v in P.items()}
    loss, G = oracle.mlp_loss_grad_f64(P64, z, lab)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = P64[name].reshape(-1)
        for idx in g.choice(flat.size, min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = oracle.mlp_loss_grad_f64(P64, z, lab)
            flat[idx] = old - h
            lm, _ = oracle.mlp_loss_grad_f64(P64, z, lab)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert G[name].reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-8), name
    # loss of uniform logits is log K
    Z = {k: np.zeros_like(v) for k, v in P64.items()}
    l0, _ = oracle.mlp_loss_grad_f64(Z, z, lab)
    assert l0 == pytest.approx(math.log(5), rel=1e-15)


def test_mlp_soft_target_gradients_match_finite_differences():
    P = _params(16, 10, 6, 4)
    g = np.random.default_rng(8)
    z = g.standard_normal((7, 16))
    q = g.random((7, 6))
    q[:3] /= q[:3].sum(1, keepdims=True)  # distributions and unnormalised weights
    P64 = {k: v.astype(np.float64) for k, v in P.items()}
    loss, G = oracle.mlp_loss_grad_soft_f64(P64, z, q)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = P64[name].reshape(-1)
        for idx in g.choice(flat.size, min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = oracle.mlp_loss_grad_soft_f64(P64, z, q)
            flat[idx] = old - h
            lm, _ = oracle.mlp_loss_grad_soft_f64(P64, z, q)
            flat[idx] = old
            assert G[name].reshape(-1)[idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-8)


def test_mlp_soft_targets_closed_forms():
    """All-zero network: every logit is 0, p = 1/K, so the loss is
    log K * mean(sum q) and dL/db3 = mean(sum(q)/K - q).  One-hot targets
    reproduce the integer-label loss and gradient."""
    P = _params(16, 8, 5, 6)
    Z = {k: np.zeros_like(v, dtype=np.float64) for k, v in P.items()}
    g = np.random.default_rng(9)
    z = g.standard_normal((11, 16))
    q = g.random((11, 5))
    loss, G = oracle.mlp_loss_grad_soft_f64(Z, z, q)
    S = q.sum(1)
    assert loss == pytest.approx(math.log(5) * S.mean(), rel=1e-14)
    np.testing.assert_allclose(G["b3"], (S[:, None] / 5 - q).mean(0), rtol=1e-13, atol=1e-16)
    assert np.all(G["W1"] == 0) and np.all(G["W2"] == 0)
    P64 = {k: v.astype(np.float64) for k, v in P.items()}
    lab = g.integers(0, 5, 11).astype(np.int32)
    l1, G1 = oracle.mlp_loss_grad_f64(P64, z, lab)
    l2, G2 = oracle.mlp_loss_grad_soft_f64(P64, z, np.eye(5)[lab])
    assert l1 == l2
    for n_ in G1:
        assert np.array_equal(G1[n_], G2[n_])


# --------------------------------------------------------------- sliced layout
def _csr_from_lengths(lengths, n_cols=100, seed=0):
    g = np.random.default_rng(seed)
    rp = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int32)
    cols = np.concatenate([np.sort(g.choice(n_cols, l, replace=False)) for l in lengths]
                          or [np.zeros(0)]).astype(np.int32)
    vals = g.standard_normal(int(rp[-1]))
    return synth.HostCSR(len(lengths), n_cols, torch.from_numpy(rp), torch.from_numpy(cols),
                         torch.from_numpy(vals), "lengths")


def test_sliced_layout_hand_example():
    """Five rows of lengths 1, 3, 0, 5, 2 with windows of 4 rows and long
    rows above 4 nonzeros, worked by hand: window 0 holds rows 0-3 with key
    lengths 1, 3, 0, 0 (row 3 is long) -> order 1, 0, 2, 3; window 1 holds row
    4.  One slice of 32 positions; its length is 3 (row 1)."""
    A = _csr_from_lengths([1, 3, 0, 5, 2])
    perm, rowlen, slen, sptr, n_long = oracle.sliced_layout(A, sigma=4, cap=4)
    assert perm.tolist() == [1, 0, 2, 3, 4]
    assert rowlen.tolist() == [3, 1, 0, -1, 2] + [-1] * 27
    assert slen.tolist() == [3] and sptr.tolist() == [0, 96] and n_long == 1
    col, val = oracle.sliced_fill(A, perm, rowlen, sptr)
    ci = A.colind.numpy()
    # position 0 holds row 1 (elements 1..3 of colind), position 4 row 4
    assert [col[32 * k + 0] for k in range(3)] == ci[1:4].tolist()
    assert [col[32 * k + 4] for k in range(2)] == ci[9:11].tolist()
    assert col[32 * 1 + 1] == 0 and val[32 * 1 + 1] == 0.0  # padding of row 0
    # four elements of a row side by side: the slice holds 32 x 4 slots;
    # element k of position p at 128 (k // 4) + 4 p + k % 4
    _, _, slen4, sptr4, _ = oracle.sliced_layout(A, sigma=4, cap=4, vec=4)
    assert slen4.tolist() == [3] and sptr4.tolist() == [0, 128]
    col4, _ = oracle.sliced_fill(A, perm, rowlen, sptr4, vec=4)
    assert col4[0:3].tolist() == ci[1:4].tolist() and col4[3] == 0
    assert col4[16:18].tolist() == ci[9:11].tolist()
    # sigma = 1: identity order
    perm1, rowlen1, slen1, _, _ = oracle.sliced_layout(A, sigma=1, cap=4)
    assert perm1.tolist() == [0, 1, 2, 3, 4] and rowlen1[:5].tolist() == [1, 3, 0, -1, 2]
    assert slen1.tolist() == [3]


@pytest.mark.parametrize("vec", [1, 2, 4])
@pytest.mark.parametrize("sigma,cap", [(1, 1000), (32, 1000), (256, 40), (64, 7)])
def test_sliced_layout_against_numpy_sort_and_reconstruction(sigma, cap, vec):
    g = np.random.default_rng(sigma + cap)
    lengths = np.minimum(g.zipf(1.6, 1000), 60)
    lengths[g.integers(0, 1000, 30)] = 0
    A = _csr_from_lengths(lengths.tolist(), n_cols=200, seed=3)
    perm, rowlen, slen, sptr, n_long = oracle.sliced_layout(A, sigma=sigma, cap=cap, vec=vec)
    key = np.where(lengths > cap, 0, lengths)
    expect = np.arange(1000)
    if sigma > 1:
        expect = np.concatenate([w + np.argsort(-key[w:w + sigma], kind="stable")
                                 for w in range(0, 1000, sigma)])
    assert np.array_equal(perm, expect)
    assert n_long == int((lengths > cap).sum())
    full = np.full(32 * len(slen), -1)
    full[:1000] = np.where(lengths[perm] > cap, -1, lengths[perm])
    assert np.array_equal(rowlen, full)
    assert np.array_equal(slen, np.maximum(full.reshape(-1, 32).max(1), 0))
    padded = (slen + vec - 1) // vec * vec
    assert np.array_equal(sptr, np.concatenate([[0], np.cumsum(32 * padded)]))
    # the slices hold exactly the short rows' elements
    col, val = oracle.sliced_fill(A, perm, rowlen, sptr, vec=vec)
    rp, ci, va = A.rowptr.numpy(), A.colind.numpy(), A.val.numpy()
    for p in range(1000):
        r, s, l = perm[p], p // 32, p % 32
        if rowlen[p] < 0:
            continue
        k = np.arange(rowlen[p])
        idx = sptr[s] + 32 * vec * (k // vec) + vec * l + k % vec
        assert np.array_equal(col[idx], ci[rp[r]:rp[r + 1]])
        assert np.array_equal(val[idx], va[rp[r]:rp[r + 1]])
    assert np.count_nonzero(val) == np.count_nonzero(va[np.repeat(lengths <= cap, lengths)])


def _csr_rows(rows, n_cols):
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    ci = np.array([c for r in rows for c in r], np.int32)
    va = np.arange(1, len(ci) + 1, dtype=np.float64)
    return synth.HostCSR(len(rows), n_cols, torch.from_numpy(rp), torch.from_numpy(ci),
                         torch.from_numpy(va), "rows")


def test_sliced_diag_hand_example():
    """Rows {0, 2}, {1}, {0, 1, 300} in order, one slice of length 3, element
    k of position p at slot 32 k + p: offsets column - row are 0, 2 (row 0),
    0 (row 1), -2, -1, 298 (row 2); the largest is 298, so 16-bit offsets.
    Without column 300 the largest is 2: 8-bit offsets."""
    A = _csr_rows([[0, 2], [1], [0, 1, 300]], 400)
    perm, rowlen, slen, sptr, _ = oracle.sliced_layout(A, sigma=1, cap=1024)
    d, reach, nb = oracle.sliced_diag(A, perm, rowlen, sptr)
    expect = np.zeros(96, np.int32)
    expect[[0, 32]] = [0, 2]
    expect[1] = 0
    expect[[2, 34, 66]] = [-2, -1, 298]
    assert np.array_equal(d, expect) and reach == 298 and nb == 2
    B = _csr_rows([[0, 2], [1], [0, 1]], 400)
    perm, rowlen, slen, sptr, _ = oracle.sliced_layout(B, sigma=1, cap=1024)
    assert oracle.sliced_diag(B, perm, rowlen, sptr)[1:] == (2, 1)
    # the width rule at its boundaries
    assert [oracle.sliced_index_bytes(r) for r in (0, 127, 128, 32767, 32768, 1 << 30)] == [1, 1, 2, 2, 4, 4]


@pytest.mark.parametrize("sigma,cap", [(1, 1000), (64, 20)])
def test_sliced_diag_decodes_to_the_columns(sigma, cap):
    """row + offset gives back every column in the slices (rows sorted or
    not, long rows left out), padding holds 0, and the reach is the largest
    |column - row| over the rows in the slices."""
    g = np.random.default_rng(5 + sigma)
    lengths = np.minimum(g.zipf(1.7, 500), 30)
    lengths[:4] = [0, 1, 31, 2]
    A = _csr_from_lengths(lengths.tolist(), n_cols=700, seed=6)
    perm, rowlen, slen, sptr, _ = oracle.sliced_layout(A, sigma=sigma, cap=cap)
    col, _ = oracle.sliced_fill(A, perm, rowlen, sptr)
    d, reach, nb = oracle.sliced_diag(A, perm, rowlen, sptr)
    rows = np.full(len(d), 0, np.int64)
    real = np.zeros(len(d), bool)
    far = 0
    rp, ci = A.rowptr.numpy(), A.colind.numpy()
    for p in range(A.n_rows):
        if rowlen[p] <= 0:
            continue
        k = np.arange(rowlen[p])
        idx = sptr[p // 32] + 32 * k + p % 32
        rows[idx] = perm[p]
        real[idx] = True
        far = max(far, int(np.abs(ci[rp[perm[p]]:rp[perm[p] + 1]].astype(np.int64) - perm[p]).max()))
    assert np.array_equal((rows + d)[real], col[real].astype(np.int64))
    assert not d[~real].any()
    assert reach == far and nb == (1 if far <= 127 else 2 if far <= 32767 else 4)


def test_sliced_delta_and_panel_hand_example():
    """Rows {3, 4, 300}, {}, {70000, 70001, 200000} in order, one slice of
    length 3, element k of position p at slot 32 k + p.
    Delta coding (O24): bases 3, 0, 70000; deltas 0, 1, 296 (row 0) and
    0, 1, 129999 (row 2); the largest, 129999, needs more than 16 bits.
    Panels of 65536 columns (O25): row 0 lies in panel 0 (offsets 3, 4, 300,
    steps 0, 0, 0); row 2: 70000 = 65536 + 4464 (panel 1, step 1), 70001
    (offset 4465, step 0), 200000 = 3 * 65536 + 3392 (step 2); largest step 2."""
    A = _csr_rows([[3, 4, 300], [], [70000, 70001, 200000]], 300000)
    perm, rowlen, slen, sptr, _ = oracle.sliced_layout(A, sigma=1, cap=1024)
    base, d, big, nb = oracle.sliced_delta(A, perm, rowlen, sptr)
    expect = np.zeros(96, np.int32)
    expect[[32, 64]] = [1, 296]
    expect[[34, 66]] = [1, 129999]
    assert np.array_equal(d, expect)
    assert list(base[:3]) == [3, 0, 70000] and not base[3:].any()
    assert big == 129999 and nb == 0
    lo, st, big_step = oracle.sliced_panel(A, perm, rowlen, sptr)
    e_lo = np.zeros(96, np.uint16)
    e_st = np.zeros(96, np.int32)
    e_lo[[0, 32, 64]] = [3, 4, 300]
    e_lo[[2, 34, 66]] = [4464, 4465, 3392]
    e_st[[2, 34, 66]] = [1, 0, 2]
    assert np.array_equal(lo, e_lo) and np.array_equal(st, e_st) and big_step == 2
    # without column 200000 the largest delta is 296: 16-bit deltas
    B = _csr_rows([[3, 4, 300], [], [70000, 70001]], 300000)
    perm, rowlen, slen, sptr, _ = oracle.sliced_layout(B, sigma=1, cap=1024)
    assert oracle.sliced_delta(B, perm, rowlen, sptr)[2:] == (296, 2)
    # the width rule ("8 or 16 bits, never both") at its boundaries
    assert [oracle.delta_bytes(v) for v in (0, 1, 255, 256, 65535, 65536, 1 << 30)] == [1, 1, 1, 2, 2, 0, 0]


@pytest.mark.parametrize("sigma,cap,n_cols", [(1, 1000, 700), (64, 20, 700), (1, 1000, 3_000_000)])
def test_sliced_delta_and_panel_decode_to_the_columns(sigma, cap, n_cols):
    """A running sum of the deltas from the row base, and panel * 65536 +
    offset with the panel a running sum of the steps, give back every column
    in the slices (rows sorted or not, long rows left out); padding holds 0;
    the reported largest delta and step are the largest over the rows."""
    g = np.random.default_rng(11 + sigma)
    lengths = np.minimum(g.zipf(1.7, 400), 30)
    lengths[:4] = [0, 1, 30, 2]
    A = _csr_from_lengths(lengths.tolist(), n_cols=n_cols, seed=7)
    perm, rowlen, slen, sptr, _ = oracle.sliced_layout(A, sigma=sigma, cap=cap)
    col, _ = oracle.sliced_fill(A, perm, rowlen, sptr)
    base, d, big, nb = oracle.sliced_delta(A, perm, rowlen, sptr)
    lo, st, big_step = oracle.sliced_panel(A, perm, rowlen, sptr)
    real = np.zeros(len(d), bool)
    want_big = want_step = 0
    rp, ci = A.rowptr.numpy(), A.colind.numpy().astype(np.int64)
    for p in range(A.n_rows):
        if rowlen[p] <= 0:
            assert base[p] == 0
            continue
        idx = sptr[p // 32] + 32 * np.arange(rowlen[p]) + p % 32
        real[idx] = True
        cols = ci[rp[perm[p]]:rp[perm[p] + 1]]
        assert d[idx[0]] == 0 and base[p] == cols[0]
        assert np.array_equal(base[p] + np.cumsum(d[idx]), cols)
        assert np.array_equal(np.cumsum(st[idx]) * 65536 + lo[idx], cols)
        assert np.array_equal(col[idx], cols)
        want_big = max(want_big, int(np.diff(cols).max(initial=0)))
        want_step = max(want_step, int(np.diff(np.concatenate([[0], cols // 65536])).max()))
    assert not d[~real].any() and not st[~real].any() and not lo[~real].any()
    assert big == want_big and big_step == want_step
    assert nb == (1 if big <= 255 else 2 if big <= 65535 else 0)


@pytest.mark.parametrize("vec", [1, 4])
def test_sliced_offsets_decode_to_the_columns(vec):
    """base + offset gives back every column of every row in the slices,
    padding and rows outside the slices hold 0, and the span is the largest
    last - first column of a row in the slices."""
    g = np.random.default_rng(17)
    lengths = np.minimum(g.zipf(1.7, 300), 40)
    lengths[:5] = [0, 1, 3, 41, 2]
    A = _csr_from_lengths(lengths.tolist(), n_cols=5000, seed=4)
    perm, rowlen, slen, sptr, _ = oracle.sliced_layout(A, sigma=64, cap=40, vec=vec)
    col, _ = oracle.sliced_fill(A, perm, rowlen, sptr, vec=vec)
    base, off, span = oracle.sliced_offsets(A, perm, rowlen, sptr, vec=vec)
    rp, ci = A.rowptr.numpy(), A.colind.numpy()
    spans = []
    for p in range(32 * len(slen)):
        if p >= A.n_rows or rowlen[p] <= 0:
            assert base[p] == 0
            continue
        s, l = p // 32, p % 32
        k = np.arange(rowlen[p])
        idx = sptr[s] + 32 * vec * (k // vec) + vec * l + k % vec
        assert np.array_equal(base[p] + off[idx].astype(np.int64), col[idx])
        r = perm[p]
        assert base[p] == ci[rp[r]]
        spans.append(ci[rp[r + 1] - 1] - ci[rp[r]])
    assert span == max(spans)
    real = np.zeros(len(off), bool)
    for p in range(A.n_rows):
        if rowlen[p] > 0:
            k = np.arange(rowlen[p])
            real[sptr[p // 32] + 32 * vec * (k // vec) + vec * (p % 32) + k % vec] = True
    assert np.all(off[~real] == 0)


# --------------------------------------------------------------- CG
def test_cg_solves_small_spd_exactly_in_n_steps():
    g = np.random.default_rng(0)
    n = 12
    M = g.standard_normal((n, n))
    D = M @ M.T + n * np.eye(n)
    A = synth.dense_to_csr(torch.from_numpy(D))
    b = g.standard_normal(n)
    x, resid = oracle.cg(A, b, np.zeros(n), n)
    np.testing.assert_allclose(x, np.linalg.solve(D, b), rtol=1e-10, atol=1e-12)
    assert resid[0] == pytest.approx(np.linalg.norm(b), rel=1e-15)
    assert resid[n] < 1e-9 * resid[0]


def test_cg_lowp_with_representable_values_equals_fp64():
    A = synth.laplacian_3d_7pt(6)
    b = synth.uniform_vector(A.n_rows, 2).numpy()
    x64, r64 = oracle.cg(A, b, np.zeros(A.n_rows), 40)
    x2, r2 = oracle.cg(A, b, np.zeros(A.n_rows), 40, vkind=2, lowval=oracle.round_bf16(A.val))
    assert np.array_equal(x64, x2) and np.array_equal(r64, r2)

def test_cg_refinement_converges_to_the_fp64_solution():
    """With BF16 values and the residual recomputed in FP64 (search restarted
    from it) every k iterations, x converges to the solution of the FP64
    system (dense solve), which plain BF16 CG cannot reach."""
    A = synth.variable_coeff_laplacian_3d(6, seed=1)
    b = synth.uniform_vector(A.n_rows, 2).numpy()
    D = np.zeros((A.n_rows, A.n_rows))
    rp, ci, v = A.rowptr.numpy(), A.colind.numpy(), A.val.numpy()
    for i in range(A.n_rows):
        D[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    xs = np.linalg.solve(D, b)
    low = oracle.round_bf16(A.val)
    for k in (5, 10, 25):
        x, _ = oracle.cg(A, b, np.zeros(A.n_rows), 200, vkind=2, lowval=low, refine=k)
        np.testing.assert_allclose(x, xs, rtol=1e-10, atol=1e-12)
    xn, _ = oracle.cg(A, b, np.zeros(A.n_rows), 200, vkind=2, lowval=low, refine=0)
    assert np.max(np.abs(xn - xs)) > 1e-5 * np.max(np.abs(xs))


# ----------------------------------------------------------------- Adam
def _adam_run(p0, grads, lr, b1, b2, eps, wd):
    """Steps of the oracle's Adam from m = v = 0 with the bias corrections
    c1 = 1 - b1^t, c2 = 1 - b2^t of step t."""
    p = np.asarray(p0, np.float32)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t, g in enumerate(grads, 1):
        p, m, v = oracle.adam_f32(p, np.asarray(g, np.float32), m, v, lr, b1, b2, eps, wd,
                                  np.float32(1 - b1 ** t), np.float32(1 - b2 ** t))
    return p, m, v


def test_adam_first_step_is_lr_whatever_the_gradient_scale():
    """With bias correction, the first step divides m_hat = g by
    sqrt(v_hat) = |g|: every coordinate moves by lr against the sign of its
    gradient, whatever the gradient's size (eps small against |g|)."""
    g = np.array([1e-3, -0.5, 2.0, -7e2, 3e4], np.float32)
    p0 = np.zeros(g.size, np.float32)
    p1, _, _ = _adam_run(p0, [g], lr=1e-2, b1=0.9, b2=0.999, eps=1e-12, wd=0.0)
    np.testing.assert_allclose(p0 - p1, 1e-2 * np.sign(g), rtol=1e-5)


def test_adam_constant_gradient_moves_lr_every_step():
    """A constant gradient keeps m_hat = g and v_hat = g^2 at every step t
    (the bias corrections undo the zero start), so t steps move t * lr;
    a wrong correction would shrink or grow the early steps."""
    g = np.array([0.25, -3.0], np.float32)
    p0 = np.zeros(2, np.float32)
    p, _, _ = _adam_run(p0, [g] * 10, lr=1e-3, b1=0.9, b2=0.999, eps=1e-12, wd=0.0)
    np.testing.assert_allclose(p0 - p, 10 * 1e-3 * np.sign(g), rtol=1e-4)


def test_adam_is_scale_invariant_bit_for_bit():
    """With eps = 0, scaling every gradient by a power of two scales m by it
    and v by its square exactly, so sqrt(v) scales back and the parameters
    follow the same trajectory bit for bit."""
    rng = np.random.default_rng(5)
    grads = [rng.standard_normal(16).astype(np.float32) for _ in range(6)]
    p0 = rng.standard_normal(16).astype(np.float32)
    a, _, _ = _adam_run(p0, grads, 3e-3, 0.9, 0.999, 0.0, 1e-2)
    b, _, _ = _adam_run(p0, [np.float32(64.0) * g for g in grads], 3e-3, 0.9, 0.999, 0.0, 1e-2)
    assert np.array_equal(a, b)


def test_adam_weight_decay_is_decoupled():
    """A zero gradient leaves m = v = 0 and the update is the decay alone:
    p <- p - lr * wd * p (decoupled from the gradient; an L2 term added to
    the gradient would instead be normalised to a step of about lr)."""
    p0 = np.array([2.0, -0.5, 8.0], np.float32)
    p1, m, v = _adam_run(p0, [np.zeros(3, np.float32)], lr=0.1, b1=0.9, b2=0.999, eps=1e-8, wd=0.05)
    assert not m.any() and not v.any()
    np.testing.assert_allclose(p1, p0 * (1 - 0.1 * 0.05), rtol=1e-6)
