"""The CPU restatement of Table 2's optimizations (Section 3.3) and of the
paper's multithreaded baseline (Section 3.2.1), a baseline the benchmark
reports beside the GPU: every form against the oracle within 1e-12 *
sum_j |a_ij x_j| per row, and its delta coding decoded back to the columns.
CPU only."""
import numpy as np
import pytest
import torch

import baseline
import oracle
import synth


def _mats():
    yield synth.laplacian_2d_5pt(64, 64)
    yield synth.random_csr(1000, 700, 40, seed=3, empty_frac=0.3)
    yield synth.zipf_rows(5000, 5000, 1.5, 3000, seed=1)
    yield synth.short_rows(3001, 8, seed=2)
    yield synth.stencil_27pt(10, seed=4)
    yield synth.random_csr(300, 200_000, 50, seed=5)       # wide rows: some stay 32-bit
    yield synth.random_csr(1, 50, 50, seed=7, empty_frac=0.0)
    yield synth.random_csr(777, 100, 0, seed=8)            # no nonzeros
    yield synth.random_csr(0, 10, 3)                        # no rows


MATS = list(_mats())


@pytest.mark.parametrize("form", baseline.FORMS)
@pytest.mark.parametrize("k", range(len(MATS)))
def test_every_form_matches_the_oracle(form, k):
    A = MATS[k]
    x = synth.uniform_vector(A.n_cols, 4)
    M = baseline.Matrix(A)
    y = baseline.spmv(form, M, x)
    y_ref, scale = oracle.spmv_ref(A, x)
    assert np.all(np.abs(y - y_ref) <= 1e-12 * scale)
    assert np.all(y[scale == 0] == 0.0)


@pytest.mark.parametrize("k", range(len(MATS)))
def test_delta_coding_decodes_to_the_columns(k):
    A = MATS[k]
    M = baseline.Matrix(A)
    base, coded, raw, width = M.prepare_delta()
    d = raw.view(np.uint8 if width == 1 else np.uint16)
    rp, ci = M.rowptr.astype(np.int64), M.colind
    lim = 255 if width == 1 else 65535
    for i in range(A.n_rows):
        cols = ci[rp[i]:rp[i + 1]]
        fits = cols.size > 0 and (np.diff(cols).max(initial=0) <= lim)
        assert bool(coded[i]) == fits
        if fits:
            assert base[i] == cols[0] and d[rp[i]] == 0
            assert np.array_equal(base[i] + np.cumsum(d[rp[i]:rp[i + 1]]), cols)


def test_delta_width_takes_the_fewer_bytes():
    # gaps of 1..8: every row fits 8 bits -> 8-bit; gaps near 300: 16-bit
    assert baseline.Matrix(synth.short_rows(2000, 8, seed=1)).prepare_delta()[3] == 1
    rows = [list(range(0, 3000, 300)) for _ in range(50)]
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    A = synth.HostCSR(50, 3000, torch.from_numpy(rp), torch.from_numpy(np.concatenate(rows).astype(np.int32)),
                      torch.ones(int(rp[-1]), dtype=torch.float64))
    assert baseline.Matrix(A).prepare_delta()[3] == 2


def test_threads_and_class_forms():
    assert baseline.threads() >= 1
    assert set(baseline.CLASS_FORM) == {"CML", "MB", "IMB", "CMP"}
    assert set(baseline.CLASS_FORM.values()) <= set(baseline.FORMS)
    with pytest.raises(ValueError):
        baseline.spmv("nope", baseline.Matrix(MATS[0]), np.zeros(MATS[0].n_cols))
