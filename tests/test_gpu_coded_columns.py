"""Table 2's delta coding of column indices (Section 3.3) in the FP64 sliced
layout, and the column-blocked form for wide rows (readings O24, O25).

Through the C ABI: the prepared arrays (row bases, deltas; panel offsets
and steps) bit-exact against the oracle's orc_sliced_delta /
orc_sliced_panel on the oracle's layout, the width rule (8-bit deltas, else
16-bit, else panels, else 32-bit columns), and y against the oracle's product
within 1e-12 * sum_j |a_ij x_j| (bit-exact for integer values), with and
without long rows (which run in the same launch as the slices).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1511_02494_gb300 as sp
import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1511_02494_gb300.build import build
    build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _export(P, which, n, dtype):
    out = torch.empty(n, dtype=dtype)
    sp.spmv_prepared_export(P, which, out)
    return out.numpy()


def _wide_far(n_rows=3000, n_cols=1 << 25, per_row=5, seed=3):
    # rows whose first column lies beyond 256 panels: no coding applies
    A = synth.random_csr(n_rows, n_cols, per_row, seed=seed, empty_frac=0.1)
    return A


def _mats():
    yield "short_rows", synth.short_rows(20_000, 8, seed=2), 1, 1           # gaps <= 16: 8-bit deltas
    yield "laplacian64", synth.laplacian_2d_5pt(64, 64), 1, 1               # gaps 1, 63: 8-bit
    yield "stencil27_n20", synth.stencil_27pt(20, seed=4), 1, 2             # gaps up to 362: 16-bit
    yield "random_cols", synth.random_columns(40_000, 3_000_000, 16, seed=5), 1, 3  # wide: panels
    yield "zipf", synth.zipf_rows(30_000, 30_000, 1.5, 20_000, seed=1), 1, 2
    yield "empty_rows", synth.random_csr(1000, 700, 40, seed=3, empty_frac=0.3), 1, 2
    yield "panels_asked", synth.stencil_27pt(12, seed=6), 2, 3              # panels when asked for
    yield "far_columns", _wide_far(), 1, 4                                  # neither applies


MATS = list(_mats())


@pytest.mark.parametrize("sigma,cap", [(1, 1024), (4096, 32)])
@pytest.mark.parametrize("name,A,coding,nbytes", MATS, ids=[m[0] for m in MATS])
def test_coded_columns_bit_exact_and_y_within_tolerance(sigma, cap, name, A, coding, nbytes):
    dA = sp.DeviceCSR.from_host(A)
    P = sp.spmv_prepare(dA, sp.make_choice("sliced", block_nnz=sigma, items_per_warp=cap,
                                           index_coding=coding))
    info = P.info()
    perm, rowlen, slen, sptr, n_long = oracle.sliced_layout(A, sigma, cap)
    S = (A.n_rows + 31) // 32
    tot = int(sptr[-1])
    base, d, big, db = oracle.sliced_delta(A, perm, rowlen, sptr)
    lo, st, big_step = oracle.sliced_panel(A, perm, rowlen, sptr)
    if coding == 1 and db:
        want = (1, db)
    elif big_step <= 255:
        want = (2, 3)
    else:
        want = (0, 4)
    assert (info.index_coding, info.index_bytes) == want, (name, big, big_step)
    if sigma == 1 and cap == 1024:
        assert info.index_bytes == nbytes  # the expected form for this matrix
    assert info.n_long_rows == n_long and info.launches == 1
    assert info.threads_per_row == 1 or info.index_coding == 0
    if info.index_coding == 1:
        dt = torch.uint8 if info.index_bytes == 1 else torch.int16
        got = _export(P, sp.EXPORT_SLICE_DELTA, tot, dt)
        assert np.array_equal(got.astype(np.int64) & (0xFF if dt == torch.uint8 else 0xFFFF), d)
        assert np.array_equal(_export(P, sp.EXPORT_SLICE_ROWBASE, 32 * S, torch.int32), base)
    elif info.index_coding == 2:
        got_lo = _export(P, sp.EXPORT_SLICE_PANEL_LO, tot, torch.int16).astype(np.int64) & 0xFFFF
        assert np.array_equal(got_lo, lo.astype(np.int64))
        assert np.array_equal(_export(P, sp.EXPORT_SLICE_PANEL_STEP, tot, torch.uint8), st)
    x = synth.uniform_vector(A.n_cols, 5)
    y = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    sp.spmv(P, x.cuda(), y)
    torch.cuda.synchronize()
    y_ref, scale = oracle.spmv_ref(A, x)
    yy = y.cpu().numpy()
    assert np.all(np.abs(yy - y_ref) <= RTOL * scale)
    assert np.all(yy[scale == 0] == 0.0)
    P.free()


@pytest.mark.parametrize("coding", [1, 2])
def test_coded_columns_integer_values_exact(coding):
    A = synth.zipf_rows(20_000, 200_000, 1.4, 15_000, seed=7)
    g = np.random.default_rng(1)
    A.val = torch.from_numpy(g.integers(-3, 4, A.nnz).astype(np.float64))
    x = torch.from_numpy(g.integers(-2, 3, A.n_cols).astype(np.float64))
    dA = sp.DeviceCSR.from_host(A)
    for sigma, cap in ((1, 1024), (4096, 32)):
        P = sp.spmv_prepare(dA, sp.make_choice("sliced", block_nnz=sigma, items_per_warp=cap,
                                               index_coding=coding))
        assert P.info().index_coding != 0
        y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        for _ in range(2):
            sp.spmv(P, x.cuda(), y)
            torch.cuda.synchronize()
            assert np.array_equal(y.cpu().numpy(), oracle.spmv(A, x))
        P.free()


def test_coded_columns_choice_validation():
    A = sp.DeviceCSR.from_host(synth.laplacian_2d_5pt(16, 16))
    for bad in (dict(index_coding=3), dict(index_coding=-1), dict(index_coding=1, index_bytes=2),
                dict(index_coding=1, threads_per_row=4), dict(index_coding=1, value_type=sp.VAL_BF16)):
        with pytest.raises(sp.SpmvError):
            sp.spmv_prepare(A, sp.make_choice("sliced", **bad))
    with pytest.raises(sp.SpmvError):
        sp.spmv_prepare(A, sp.make_choice("compressed", index_coding=1))


def test_coded_columns_in_cg_and_batch_fall_back_to_their_own_forms():
    # CG takes the separate SpMV + dot path, the batch lays the matrix out anew
    A = synth.variable_coeff_laplacian_3d(12, seed=0)
    dA = sp.DeviceCSR.from_host(A)
    P = sp.spmv_prepare(dA, sp.make_choice("sliced", index_coding=1))
    assert P.info().index_coding == 1
    b = synth.uniform_vector(A.n_rows, 1)
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    sp.spmv_cg(P, b.cuda(), x, 30)
    torch.cuda.synchronize()
    xr, _ = oracle.cg(A, b, np.zeros(A.n_rows), 30)
    assert np.allclose(x.cpu().numpy(), xr, rtol=1e-9, atol=1e-9 * np.abs(xr).max())
    B = sp.spmv_batch_create_sliced([P])
    xs = [synth.uniform_vector(A.n_cols, 2).cuda()]
    ys = [torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")]
    sp.spmv_batch_bind(B, xs, ys)
    sp.spmv_batch_run(B)
    torch.cuda.synchronize()
    y_ref, scale = oracle.spmv_ref(A, xs[0].cpu())
    assert np.all(np.abs(ys[0].cpu().numpy() - y_ref) <= RTOL * scale)
    B.free()
    P.free()
