"""Property tests of the oracle on random tiny CSR matrices (hypothesis,
derandomized): the product against a dense matrix-vector product computed
independently, Table 1's integer aggregates against per-row definitions
written out with numpy, and the sliced layout's reconstruction.  Shapes
include empty rows, single-nonzero rows, a full row, one row, no nonzeros
and rectangular matrices.  CPU only."""
import numpy as np
import pytest
import torch

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


@st.composite
def tiny_integer_csr(draw):
    n = draw(st.integers(1, 12))
    m = draw(st.integers(1, 12))
    density = draw(st.sampled_from([0.0, 0.15, 0.5, 1.0]))
    seed = draw(st.integers(0, 2**31 - 1))
    g = np.random.default_rng(seed)
    D = g.integers(-9, 10, size=(n, m)).astype(np.float64)
    D[g.random((n, m)) >= density] = 0.0
    if draw(st.booleans()) and m > 0:
        D[g.integers(0, n)] = g.integers(1, 9, m)  # one full row
    x = g.integers(-20, 21, m).astype(np.float64)
    return D, x


SETTINGS = settings(max_examples=150, deadline=None, derandomize=True)


@SETTINGS
@given(tiny_integer_csr())
def test_spmv_equals_dense_product_exactly(case):
    D, x = case
    A = synth.dense_to_csr(torch.from_numpy(D))
    # integer data: every partial sum is exact, so the sums agree bit for bit
    assert np.array_equal(oracle.spmv(A, torch.from_numpy(x)), D @ x)
    ref, scale = oracle.spmv_ref(A, torch.from_numpy(x))
    assert np.array_equal(ref, D @ x) and np.array_equal(scale, np.abs(D) @ np.abs(x))


@SETTINGS
@given(tiny_integer_csr(), st.sampled_from([8, 16, 64, 128]))
def test_table1_aggregates_equal_their_row_definitions(case, line_bytes):
    D, _ = case
    A = synth.dense_to_csr(torch.from_numpy(D))
    f = oracle.features(A, line_bytes=line_bytes)
    L = line_bytes // 8
    nnz, bw, groups, misses = [], [], [], []
    for row in D:
        c = np.nonzero(row)[0]
        nnz.append(len(c))
        bw.append(int(c[-1] - c[0]) if len(c) > 1 else 0)
        groups.append(0 if len(c) == 0 else 1 + int(np.sum(np.diff(c) != 1)))
        misses.append(0 if len(c) == 0 else 1 + int(np.sum(np.diff(c) > L)))
    assert (f["nnz_min"], f["nnz_max"], f["nnz_sum"]) == (min(nnz), max(nnz), sum(nnz))
    assert f["nnz_sumsq"] == sum(v * v for v in nnz)
    assert (f["bw_min"], f["bw_max"], f["bw_sum"]) == (min(bw), max(bw), sum(bw))
    assert f["bw_sumsq"] == sum(v * v for v in bw)
    assert f["ngroups_sum"] == sum(groups) and f["misses_sum"] == sum(misses)
    # fixed-point ratios: floor(2^32 * nnz / span) and floor(2^32 * groups / nnz), 0 for empty rows
    disp = sum((n_ << 32) // (b_ + 1) for n_, b_ in zip(nnz, bw) if n_)
    clust = sum((g_ << 32) // n_ for g_, n_ in zip(groups, nnz) if n_)
    assert f["disp_sum"] == disp and f["clust_sum"] == clust


@SETTINGS
@given(tiny_integer_csr(), st.sampled_from([1, 32, 64]), st.sampled_from([1, 2, 3, 1024]),
       st.sampled_from([1, 4]))
def test_sliced_layout_holds_every_short_row(case, sigma, cap, vec):
    D, _ = case
    A = synth.dense_to_csr(torch.from_numpy(D))
    perm, rowlen, slen, sptr, n_long = oracle.sliced_layout(A, sigma, cap, vec=vec)
    col, val = oracle.sliced_fill(A, perm, rowlen, sptr, vec=vec)
    assert sorted(perm.tolist()) == list(range(A.n_rows))
    lens = (D != 0).sum(1)
    assert n_long == int((lens > cap).sum())
    for p in range(A.n_rows):
        r = perm[p]
        c = np.nonzero(D[r])[0]
        if len(c) > cap:
            assert rowlen[p] == -1
            continue
        assert rowlen[p] == len(c)
        k = np.arange(len(c))
        idx = sptr[p // 32] + 32 * vec * (k // vec) + vec * (p % 32) + k % vec
        assert np.array_equal(col[idx], c) and np.array_equal(val[idx], D[r, c])
