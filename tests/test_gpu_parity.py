"""GPU parity of the CUDA library against the CPU oracle, through the C ABI.

Floating point: |y_gpu - y_ref| <= 1e-12 * sum_j |a_ij x_j| per row (rows whose
scale is 0 must be exactly 0); integer-valued, identity and permutation
inputs must match bit for bit.  Integer work (features, prepared arrays,
selections) must be bit-exact.
"""
import os

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
    sp.lib()


def _assert_close(y_gpu, A, x, rows=None, rtol=RTOL):
    y_ref, scale = oracle.spmv_ref(A, x, rows)
    y = y_gpu.detach().cpu().numpy()
    if rows is not None:
        y = y[np.asarray(rows)]
    err = np.abs(y - y_ref)
    bad = err > rtol * scale
    assert not bad.any(), (f"{int(bad.sum())} rows off; worst row {int(np.argmax(err - rtol * scale))}"
                           f" err {err.max():.3e}")
    assert np.all(y[scale == 0] == 0.0)


def _run(A, choice, x=None, reps=1):
    dA = sp.DeviceCSR.from_host(A)
    if x is None:
        x = synth.uniform_vector(A.n_cols, 1)
    dx = x.cuda()
    dy = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    P = sp.spmv_prepare(dA, choice)
    outs = []
    for _ in range(reps):
        dy.fill_(float("nan"))
        sp.spmv(P, dx, dy)
        torch.cuda.synchronize()
        outs.append(dy.clone())
    P.free()
    return outs if reps > 1 else outs[0], x


CHOICES = [
    ("scalar", {}),
    ("subwarp", {"threads_per_row": 1}), ("subwarp", {"threads_per_row": 2}),
    ("subwarp", {"threads_per_row": 4}), ("subwarp", {"threads_per_row": 8}),
    ("subwarp", {"threads_per_row": 16}), ("subwarp", {"threads_per_row": 32}),
    ("subwarp", {}),
    ("stream", {"block_nnz": 64}), ("stream", {"block_nnz": 256}), ("stream", {}),
    ("stream", {"block_nnz": 1024}), ("stream", {"block_nnz": 8192}),
    ("merge", {"block_nnz": 1024}), ("merge", {"block_nnz": 2048}), ("merge", {}),
    ("dynamic", {"threads_per_row": 1}), ("dynamic", {"threads_per_row": 8}), ("dynamic", {}),
    ("dynamic", {"threads_per_row": 32, "block_nnz": 256}), ("dynamic", {"block_nnz": 256}),
    ("latency", {"threads_per_row": 1}), ("latency", {"threads_per_row": 4}), ("latency", {}),
    ("latency", {"threads_per_row": 32}),
    ("compressed", {}), ("compressed", {"threads_per_row": 1}),
    ("compressed", {"threads_per_row": 32}),
    ("sliced", {}), ("sliced", {"block_nnz": 1}), ("sliced", {"block_nnz": 32}),
    ("sliced", {"block_nnz": 4096}), ("sliced", {"block_nnz": 4096, "items_per_warp": 32}),
    ("sliced", {"items_per_warp": 1}), ("sliced", {"threads_per_row": 1}),
    ("sliced", {"threads_per_row": 2}), ("sliced", {"threads_per_row": 4}),
    ("sliced", {"threads_per_row": 4, "block_nnz": 256, "items_per_warp": 8}),
    ("sliced", {"index_bytes": 1}), ("sliced", {"index_bytes": 2}),
    ("sliced", {"index_bytes": 1, "threads_per_row": 4}), ("sliced", {"index_bytes": 1, "threads_per_row": 2}),
]


def _matrices():
    yield "laplacian64", synth.laplacian_2d_5pt(64, 64)
    yield "random_empty_rows", synth.random_csr(1000, 700, 40, seed=3, empty_frac=0.3)
    yield "zipf_long_rows", synth.zipf_rows(5000, 5000, 1.5, 3000, seed=1)
    yield "short_rows", synth.short_rows(3001, 8, seed=2)
    yield "stencil27_n10", synth.stencil_27pt(10, seed=4)
    yield "one_dense_row", synth.dense_to_csr(torch.cat([torch.rand(1, 9000, dtype=torch.float64) + 0.1,
                                                         torch.zeros(3, 9000, dtype=torch.float64)]))
    yield "rectangular_wide", synth.random_csr(300, 200_000, 50, seed=5)
    yield "rectangular_tall", synth.random_csr(5000, 17, 9, seed=6)
    yield "single_row", synth.random_csr(1, 50, 50, seed=7, empty_frac=0.0)
    yield "all_empty", synth.random_csr(777, 100, 0, seed=8)


MATS = list(_matrices())


@pytest.mark.parametrize("variant,params", CHOICES, ids=[f"{v}{p}" for v, p in CHOICES])
@pytest.mark.parametrize("name,A", MATS, ids=[m[0] for m in MATS])
def test_spmv_variant_parity(variant, params, name, A):
    y, x = _run(A, sp.make_choice(variant, **params))
    _assert_close(y, A, x)


@pytest.mark.parametrize("variant,params", CHOICES, ids=[f"{v}{p}" for v, p in CHOICES])
def test_spmv_bit_exact_on_integer_inputs(variant, params):
    g = np.random.default_rng(0)
    D = g.integers(-7, 8, size=(600, 450)).astype(np.float64)
    D[g.random(D.shape) < 0.9] = 0.0
    D[5] = 0.0
    A = synth.dense_to_csr(torch.from_numpy(D))
    x = torch.from_numpy(g.integers(-20, 21, 450).astype(np.float64))
    y, _ = _run(A, sp.make_choice(variant, **params), x)
    assert np.array_equal(y.cpu().numpy(), oracle.spmv(A, x))


@pytest.mark.parametrize("variant", sp.VARIANTS)
def test_identity_and_permutation_bit_exact(variant):
    n = 4099
    x = synth.uniform_vector(n, 11)
    I = synth.HostCSR(n, n, torch.arange(n + 1, dtype=torch.int32),
                      torch.arange(n, dtype=torch.int32), torch.ones(n, dtype=torch.float64))
    y, _ = _run(I, sp.make_choice(variant), x)
    assert torch.equal(y.cpu(), x)
    perm = torch.randperm(n, generator=torch.Generator().manual_seed(2))
    P = synth.HostCSR(n, n, torch.arange(n + 1, dtype=torch.int32),
                      perm.to(torch.int32), torch.ones(n, dtype=torch.float64))
    y, _ = _run(P, sp.make_choice(variant), x)
    assert torch.equal(y.cpu(), x[perm])


@pytest.mark.parametrize("variant", ["dynamic", "merge", "stream", "latency", "sliced"])
def test_repeated_launches_identical(variant):
    """Back-to-back launches (counter reset, carry reuse, the per-row ticket of
    SLICED's rows with several segments) give the same y."""
    A = synth.zipf_rows(20000, 20000, 1.6, 5000, seed=9)
    outs, x = _run(A, sp.make_choice(variant), reps=4)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    _assert_close(outs[0], A, x)


def test_sliced_rows_of_many_segments_summed_in_order():
    # rows of up to 60 segments of 2048 nonzeros, each row's segments summed
    # in order by the warp finishing last: integer values give the exact sum,
    # and repeated launches give the same bits
    A = synth.zipf_rows(3000, 200_000, 1.2, 120_000, seed=12)
    g = np.random.default_rng(3)
    A.val = torch.from_numpy(g.integers(-3, 4, A.nnz).astype(np.float64))
    x = torch.from_numpy(g.integers(-2, 3, A.n_cols).astype(np.float64))
    outs, _ = _run(A, sp.make_choice("sliced", block_nnz=4096, items_per_warp=32), x, reps=3)
    for o in outs:
        assert np.array_equal(o.cpu().numpy(), oracle.spmv(A, x))


def test_merge_long_row_spans_many_parts():
    A = synth.zipf_rows(3000, 60000, 1.3, 40000, seed=10)
    y, x = _run(A, sp.make_choice("merge", items_per_warp=32))
    _assert_close(y, A, x)


def test_empty_matrix_all_variants():
    A = synth.random_csr(0, 10, 3)
    dA = sp.DeviceCSR.from_host(A)
    for v in sp.VARIANTS:
        P = sp.spmv_prepare(dA, sp.make_choice(v))
        sp.spmv(P, torch.zeros(10, dtype=torch.float64, device="cuda"),
                torch.zeros(0, dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        P.free()


def test_rows_without_columns_all_variants():
    """n_cols = 0: every row is empty, so y = 0 for every variant and
    launch shape (the SLICED layout is uniform with rows of length 0)."""
    A = synth.HostCSR(100, 0, torch.zeros(101, dtype=torch.int32), torch.zeros(0, dtype=torch.int32),
                      torch.zeros(0, dtype=torch.float64), "no_columns")
    dA = sp.DeviceCSR.from_host(A)
    x = torch.zeros(1, dtype=torch.float64, device="cuda")  # a valid pointer, never read
    for v, params in CHOICES:
        P = sp.spmv_prepare(dA, sp.make_choice(v, **params))
        y = torch.full((100,), float("nan"), dtype=torch.float64, device="cuda")
        sp.spmv(P, x, y)
        torch.cuda.synchronize()
        assert torch.equal(y, torch.zeros_like(y)), (v, params)
        if v == "sliced" and not params:
            assert P.info().uniform_len == 0
        P.free()


# ----------------------------------------------------------------- features
def _features_match(A, line_bytes=128):
    dA = sp.DeviceCSR.from_host(A)
    g = sp.spmv_features(dA, line_bytes).as_dict()
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    o = oracle.features(A, line_bytes=line_bytes, l2_bytes=l2)
    for k, v in o.items():
        if k == "vec":
            assert np.array_equal(np.array(g["vec"], np.float32), v), (k, g["vec"], v)
        else:
            assert g[k] == v, (k, g[k], v)


@pytest.mark.parametrize("name,A", MATS, ids=[m[0] for m in MATS])
def test_features_bit_exact(name, A):
    _features_match(A, 128)
    _features_match(A, 64)


def test_features_bit_exact_config1_laplacian():
    A = synth.laplacian_2d_5pt(64, 64)
    _features_match(A)
    f = sp.spmv_features(sp.DeviceCSR.from_host(A)).as_dict()
    assert f["misses_sum"] == 12160 and f["nnz_sumsq"] == 100104


def test_features_empty_matrix():
    _features_match(synth.random_csr(0, 0, 0))


def _bad_csr(kind):
    rp = torch.tensor([0, 2, 3, 5], dtype=torch.int32)
    ci = torch.tensor([0, 2, 1, 0, 3], dtype=torch.int32)
    if kind == "rowptr0":
        rp = torch.tensor([1, 2, 3, 5], dtype=torch.int32)
    elif kind == "decreasing":
        rp = torch.tensor([0, 3, 2, 5], dtype=torch.int32)
    elif kind == "beyond_nnz":
        rp = torch.tensor([0, 2, 9, 5], dtype=torch.int32)
    elif kind == "col_range":
        ci = torch.tensor([0, 2, 1, 0, 4], dtype=torch.int32)
    elif kind == "negative_col":
        ci = torch.tensor([0, 2, -1, 0, 3], dtype=torch.int32)
    elif kind == "unsorted":
        ci = torch.tensor([2, 0, 1, 0, 3], dtype=torch.int32)
    elif kind == "duplicate":
        ci = torch.tensor([0, 2, 1, 3, 3], dtype=torch.int32)
    return synth.HostCSR(3, 4, rp, ci, torch.ones(5, dtype=torch.float64))


@pytest.mark.parametrize("kind", ["rowptr0", "decreasing", "beyond_nnz", "col_range",
                                  "negative_col", "unsorted", "duplicate"])
def test_invalid_csr_rejected(kind):
    dA = sp.DeviceCSR.from_host(_bad_csr(kind))
    for call in (lambda: sp.spmv_validate(dA), lambda: sp.spmv_features(dA),
                 lambda: sp.spmv_prepare(dA, sp.make_choice("merge"))):
        with pytest.raises(sp.SpmvError) as e:
            call()
        assert e.value.status == 2
    sp.spmv_validate(sp.DeviceCSR.from_host(_bad_csr("ok")))


def _unaligned(A):
    """The same matrix with every array starting 4 or 8 bytes past a 16-byte
    boundary, which rules out the bulk-copy kernels."""
    def shifted(t, pad):
        buf = torch.zeros(t.numel() + pad, dtype=t.dtype, device="cuda")
        v = buf[pad:]
        v.copy_(t.to("cuda"))
        return v
    return sp.DeviceCSR(A.n_rows, A.n_cols, shifted(A.rowptr, 1), shifted(A.colind, 1),
                        shifted(A.val, 1))


@pytest.mark.parametrize("name,A", MATS, ids=[m[0] for m in MATS])
def test_merge_unaligned_fallback_parity(name, A):
    dU = _unaligned(A)
    if A.nnz:
        assert dU.colind.data_ptr() % 16 != 0
    x = synth.uniform_vector(A.n_cols, 1)
    for items in (32, 256):
        P = sp.spmv_prepare(dU, sp.make_choice("merge", items_per_warp=items))
        if A.nnz:
            assert P.info().bulk_copy == 0
        y = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
        sp.spmv(P, x.cuda(), y)
        torch.cuda.synchronize()
        _assert_close(y, A, x)


@pytest.mark.parametrize("name,A", MATS, ids=[m[0] for m in MATS])
def test_stream_unaligned_fallback_parity(name, A):
    dU = _unaligned(A)
    x = synth.uniform_vector(A.n_cols, 1)
    P = sp.spmv_prepare(dU, sp.make_choice("stream", block_nnz=1024))
    if A.nnz:
        assert P.info().bulk_copy == 0
    y = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    sp.spmv(P, x.cuda(), y)
    torch.cuda.synchronize()
    _assert_close(y, A, x)


@pytest.mark.parametrize("variant", ["stream", "merge"])
@pytest.mark.parametrize("name,A", MATS, ids=[m[0] for m in MATS])
def test_pipelined_kernels_report_no_timeout(variant, name, A):
    dA = sp.DeviceCSR.from_host(A)
    for tile in (1024, 2048):
        P = sp.spmv_prepare(dA, sp.make_choice(variant, block_nnz=tile))
        assert P.info().bulk_copy == (1 if A.nnz else P.info().bulk_copy)
        y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        x = synth.uniform_vector(A.n_cols, 2)
        for _ in range(3):
            sp.spmv(P, x.cuda(), y)
        sp.spmv_prepared_status(P)
        _assert_close(y, A, x)


# ----------------------------------------------------------------- prepared arrays
def _export(P, which, n, dtype):
    t = torch.empty(n, dtype=dtype)
    sp.spmv_prepared_export(P, which, t)
    return t.numpy()


@pytest.mark.parametrize("sigma,cap", [(1, 1024), (32, 1024), (256, 1024), (1, 8), (4096, 32)])
@pytest.mark.parametrize("name,A", MATS, ids=[m[0] for m in MATS])
def test_sliced_layout_bit_exact(sigma, cap, name, A):
    """The SLICED prepared arrays equal the oracle's sliced layout, for the
    default row-length cap (1024) and chosen ones."""
    dA = sp.DeviceCSR.from_host(A)
    P = sp.spmv_prepare(dA, sp.make_choice("sliced", block_nnz=sigma, index_bytes=4,
                                           items_per_warp=0 if cap == 1024 else cap))
    perm, rowlen, slen, sptr, n_long = oracle.sliced_layout(A, sigma, cap)
    S = (A.n_rows + 31) // 32
    info = P.info()
    assert info.n_blocks == S and info.block_nnz == sigma and info.items_per_warp == cap
    # slices and long-row segments run in one launch
    assert info.launches == (0 if A.n_rows == 0 else 1) and info.n_long_rows == n_long
    if S == 0:
        return
    assert np.array_equal(_export(P, sp.EXPORT_SLICE_ROWLEN, 32 * S, torch.int32), rowlen)
    assert np.array_equal(_export(P, sp.EXPORT_SLICE_LEN, S, torch.int32), slen)
    assert np.array_equal(_export(P, sp.EXPORT_SLICE_PTR, S + 1, torch.int64), sptr)
    if sigma > 1:
        assert np.array_equal(_export(P, sp.EXPORT_SLICE_PERM, A.n_rows, torch.int32), perm)
    else:
        with pytest.raises(sp.SpmvError):
            _export(P, sp.EXPORT_SLICE_PERM, A.n_rows, torch.int32)
    col, val = oracle.sliced_fill(A, perm, rowlen, sptr)
    tot = int(sptr[-1])
    assert info.index_bytes == 4
    if tot:
        assert np.array_equal(_export(P, sp.EXPORT_SLICE_COL, tot, torch.int32), col)
        assert np.array_equal(_export(P, sp.EXPORT_SLICE_VAL, tot, torch.float64), val)
        with pytest.raises(sp.SpmvError):
            _export(P, sp.EXPORT_SLICE_DIAG, tot, torch.int16)
    # the narrowest column form the rows allow (Table 2's 8/16-bit
    # compression of column indices, reading O23)
    d, reach, nb = oracle.sliced_diag(A, perm, rowlen, sptr)
    Q = sp.spmv_prepare(dA, sp.make_choice("sliced", block_nnz=sigma, index_bytes=1,
                                           items_per_warp=0 if cap == 1024 else cap))
    assert Q.info().index_bytes == nb
    # by default the narrowest form only where every row has one length and
    # the rows stay in order (no slice header), else 32-bit columns
    lens = np.diff(A.rowptr.numpy())
    uniform = A.n_rows > 0 and sigma == 1 and n_long == 0 and lens.min() == lens.max()
    D = sp.spmv_prepare(dA, sp.make_choice("sliced", block_nnz=sigma,
                                           items_per_warp=0 if cap == 1024 else cap))
    assert D.info().index_bytes == (nb if uniform else 4)
    if tot and nb < 4:
        got = _export(Q, sp.EXPORT_SLICE_DIAG, tot, torch.int8 if nb == 1 else torch.int16)
        assert np.array_equal(got.astype(np.int32), d)
        with pytest.raises(sp.SpmvError):
            _export(Q, sp.EXPORT_SLICE_COL, tot, torch.int32)


@pytest.mark.parametrize("vt", [sp.VAL_F32, sp.VAL_BF16])
@pytest.mark.parametrize("sigma", [1, 256])
@pytest.mark.parametrize("name,A", MATS, ids=[m[0] for m in MATS])
def test_sliced_low_precision_layout_bit_exact(vt, sigma, name, A):
    """Values rounded as the oracle rounds them; 16-bit offsets from each
    row's first column when every row in the slices spans < 65536 columns."""
    dA = sp.DeviceCSR.from_host(A)
    P = sp.spmv_prepare(dA, sp.make_choice("sliced", block_nnz=sigma, value_type=vt))
    assert P.info().accumulate == sp.ACC_F32
    # low-precision slices keep four elements of a row side by side
    perm, rowlen, slen, sptr, n_long = oracle.sliced_layout(A, sigma, 1024, vec=4)
    S, tot = (A.n_rows + 31) // 32, int(sptr[-1])
    if tot == 0:
        return
    assert np.array_equal(_export(P, sp.EXPORT_SLICE_PTR, S + 1, torch.int64), sptr)
    col, val = oracle.sliced_fill(A, perm, rowlen, sptr, vec=4)
    if vt == sp.VAL_F32:
        got = _export(P, sp.EXPORT_SLICE_VAL, tot, torch.float32)
        assert np.array_equal(got, oracle.round_f32(val))
    else:
        got = _export(P, sp.EXPORT_SLICE_VAL, tot, torch.int16).view(np.uint16)
        assert np.array_equal(got, oracle.round_bf16(val))
    base, off, span = oracle.sliced_offsets(A, perm, rowlen, sptr, vec=4)
    if span < 65536:
        assert np.array_equal(_export(P, sp.EXPORT_SLICE_OFF16, tot, torch.int16).view(np.uint16), off)
        assert np.array_equal(_export(P, sp.EXPORT_SLICE_ROWBASE, 32 * S, torch.int32), base)
        with pytest.raises(sp.SpmvError):
            _export(P, sp.EXPORT_SLICE_COL, tot, torch.int32)
    else:
        assert np.array_equal(_export(P, sp.EXPORT_SLICE_COL, tot, torch.int32), col)


@pytest.mark.parametrize("ipw", [0, 16])
@pytest.mark.parametrize("vt,vkind", [(sp.VAL_F32, 1), (sp.VAL_BF16, 2)])
@pytest.mark.parametrize("name,A", MATS, ids=[m[0] for m in MATS])
def test_sliced_low_precision_parity(vt, vkind, ipw, name, A):
    """FP32 accumulation: rows in slices are summed in row order with fmaf,
    bit for bit the oracle's FP32 form; long rows (segments + shuffle tree)
    within the FP32 bound.  FP64 accumulation: within the FP64 bound.  The
    row-length cap is chosen (ipw = 0) or set."""
    lowval = oracle.round_f32(A.val) if vkind == 1 else oracle.round_bf16(A.val)
    x = synth.uniform_vector(A.n_cols, 5)
    choice = sp.make_choice("sliced", value_type=vt, items_per_warp=ipw)
    cap = sp.spmv_prepare(sp.DeviceCSR.from_host(A), choice).info().items_per_warp
    assert cap == (ipw or cap) and cap in (ipw, 32, 1024)
    y32, _ = _run(A, choice, x)
    ref32 = oracle.spmv_lowp32(A, x, vkind, lowval)
    lens = (A.rowptr[1:] - A.rowptr[:-1]).numpy()
    short = lens <= cap
    got = y32.cpu().numpy()
    assert np.array_equal(got[short], ref32[short])
    if (~short).any():
        bound = _lowp32_bound(A, x, lowval, vkind)
        assert np.all(np.abs(got - ref32)[~short] <= bound[~short])
    y64, _ = _run(A, sp.make_choice("sliced", value_type=vt, accumulate=sp.ACC_F64,
                                    items_per_warp=ipw), x)
    ref64 = oracle.spmv_lowp(A, x, vkind, lowval)
    _, scale = oracle.spmv_ref(A, x)
    assert np.all(np.abs(y64.cpu().numpy() - ref64) <= RTOL * scale * 1.01)


@pytest.mark.parametrize("reach,nb", [(127, 1), (128, 2), (-128, 2), (32767, 2), (32768, 4), (-32768, 4)])
def test_sliced_index_width_at_its_boundaries(reach, nb):
    """The diagonal plus one element at column row + reach in row 40000:
    8-bit offsets up to 127, 16-bit up to 32767, then 32-bit columns; the
    product is bit-exact with the oracle on integer data whatever the width."""
    n = 80_000
    r0 = 40_000
    rows = [[i] for i in range(n)]
    rows[r0] = sorted([r0, r0 + reach])
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    ci = np.array([c for r in rows for c in r], np.int32)
    g = np.random.default_rng(abs(reach))
    va = g.integers(-9, 10, len(ci)).astype(np.float64)
    A = synth.HostCSR(n, n, torch.from_numpy(rp), torch.from_numpy(ci), torch.from_numpy(va), "diag")
    x = torch.from_numpy(g.integers(-20, 21, n).astype(np.float64))
    dA = sp.DeviceCSR.from_host(A)
    for R in (0, 1, 2):
        P = sp.spmv_prepare(dA, sp.make_choice("sliced", threads_per_row=R, index_bytes=1))
        assert P.info().index_bytes == nb
        assert sp.spmv_prepare(dA, sp.make_choice("sliced", index_bytes=2)).info().index_bytes == max(nb, 2)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        sp.spmv(P, x.cuda(), y)
        assert np.array_equal(y.cpu().numpy(), oracle.spmv(A, x))


UNIFORM = [("random_cols_16", synth.random_columns(70_001, 70_001, 16, seed=11)),
           ("random_cols_37", synth.random_columns(2049, 5000, 37, seed=14)),
           ("random_cols_1", synth.random_columns(3000, 50, 1, seed=13)),
           ("short_rows", synth.short_rows(50_001, 8, seed=12)),
           ("all_empty", synth.random_csr(777, 100, 0, seed=8))]


@pytest.mark.parametrize("tpr", [0, 1, 2, 4])
@pytest.mark.parametrize("nb", [4, 1])
@pytest.mark.parametrize("name,A", UNIFORM, ids=[m[0] for m in UNIFORM])
def test_sliced_uniform_rows_bit_exact(name, A, nb, tpr):
    """Rows all of one length, kept in order: the slice starts are implied
    by the length and no header is read.  The same rows laid out in sorted
    windows of 32 (read through the slice header) give the same bits, y is
    within the bound of the oracle's, and bit-exact with it on integer data."""
    x = synth.uniform_vector(A.n_cols, 3)
    lens = np.diff(A.rowptr.numpy())
    dA = sp.DeviceCSR.from_host(A)
    for sigma, want in ((1, int(lens[0])), (32, -1)):
        info = sp.spmv_prepare(dA, sp.make_choice("sliced", block_nnz=sigma, index_bytes=nb,
                                                  threads_per_row=tpr)).info()
        assert info.uniform_len == want
    ys = [_run(A, sp.make_choice("sliced", block_nnz=sigma, index_bytes=nb, threads_per_row=tpr), x)[0]
          for sigma in (1, 32)]
    assert torch.equal(ys[0], ys[1])
    _assert_close(ys[0], A, x)
    g = np.random.default_rng(A.nnz)
    vi = torch.from_numpy(g.integers(-9, 10, A.nnz).astype(np.float64))
    Ai = synth.HostCSR(A.n_rows, A.n_cols, A.rowptr, A.colind, vi, A.name)
    xi = torch.from_numpy(g.integers(-20, 21, A.n_cols).astype(np.float64))
    y, _ = _run(Ai, sp.make_choice("sliced", block_nnz=1, index_bytes=nb, threads_per_row=tpr), xi)
    assert np.array_equal(y.cpu().numpy(), oracle.spmv(Ai, xi))


def test_sliced_auto_window_and_long_rows():
    # regular rows: kept in order, one slice per warp; Zipf rows: sorted in
    # windows of 4096 and every row above 32 nonzeros computed from CSR
    L = synth.laplacian_2d_5pt(100, 100)
    info = sp.spmv_prepare(sp.DeviceCSR.from_host(L), sp.make_choice("sliced")).info()
    assert info.block_nnz == 1 and info.items_per_warp == 1024 and info.threads_per_row == 1
    Z = synth.zipf_rows(60_000, 60_000, 1.4, 20_000, seed=9)
    P = sp.spmv_prepare(sp.DeviceCSR.from_host(Z), sp.make_choice("sliced"))
    assert P.info().block_nnz == 4096 and P.info().items_per_warp == 32 and P.info().launches == 1
    # a chosen cap is kept
    P = sp.spmv_prepare(sp.DeviceCSR.from_host(Z), sp.make_choice("sliced", items_per_warp=512))
    assert P.info().block_nnz == 4096 and P.info().items_per_warp == 512
    # rows of two nonzeros: four slices per warp (FP64), one with FP32 values
    S = synth.short_rows(50_000)
    assert sp.spmv_prepare(sp.DeviceCSR.from_host(S), sp.make_choice("sliced")).info().threads_per_row == 4
    assert sp.spmv_prepare(sp.DeviceCSR.from_host(S), sp.make_choice(
        "sliced", value_type=sp.VAL_F32)).info().threads_per_row == 1
    for bad in (3, 8, 32):
        with pytest.raises(sp.SpmvError):
            sp.spmv_prepare(sp.DeviceCSR.from_host(S), sp.make_choice("sliced", threads_per_row=bad))
    for bad in (dict(variant="sliced", index_bytes=3), dict(variant="compressed", index_bytes=2),
                dict(variant="sliced", index_bytes=1, value_type=sp.VAL_F32)):
        with pytest.raises(sp.SpmvError):
            sp.spmv_prepare(sp.DeviceCSR.from_host(S), sp.make_choice(**bad))
    y, x = _run(Z, sp.make_choice("sliced"))
    _assert_close(y, Z, x)
    for bad in (2, 16, 8192):
        with pytest.raises(sp.SpmvError):
            sp.spmv_prepare(sp.DeviceCSR.from_host(L), sp.make_choice("sliced", block_nnz=bad))
    for bad in (-1, 65537):
        with pytest.raises(sp.SpmvError):
            sp.spmv_prepare(sp.DeviceCSR.from_host(L), sp.make_choice("sliced", items_per_warp=bad))
    # a cap of 32 sends every Zipf row above 32 nonzeros to the segments
    P = sp.spmv_prepare(sp.DeviceCSR.from_host(Z), sp.make_choice("sliced", block_nnz=4096,
                                                                   items_per_warp=32))
    assert P.info().items_per_warp == 32 and P.info().launches == 1
    y, x = _run(Z, sp.make_choice("sliced", block_nnz=4096, items_per_warp=32))
    _assert_close(y, Z, x)


@pytest.mark.parametrize("name,A", MATS[:6], ids=[m[0] for m in MATS[:6]])
def test_prepared_arrays_bit_exact(name, A):
    dA = sp.DeviceCSR.from_host(A)
    for B in (64, 1024):
        P = sp.spmv_prepare(dA, sp.make_choice("stream", block_nnz=B))
        n = P.info().n_blocks
        assert np.array_equal(_export(P, sp.EXPORT_ROW_BLOCKS, n + 1, torch.int32),
                              oracle.row_blocks(A, B))
    for tile in (1024, 2048):
        P = sp.spmv_prepare(dA, sp.make_choice("merge", block_nnz=tile))
        info = P.info()
        assert info.bulk_copy == 1 and info.tile_items == tile
        rs, ns = oracle.merge_path(A, tile)
        assert np.array_equal(_export(P, sp.EXPORT_MERGE_ROWS, info.n_blocks + 1, torch.int32), rs)
        assert np.array_equal(_export(P, sp.EXPORT_MERGE_NZ, info.n_blocks + 1, torch.int32), ns)
    for items in (32, 256, 512):
        dU = _unaligned(A)
        P = sp.spmv_prepare(dU, sp.make_choice("merge", items_per_warp=items))
        assert P.info().bulk_copy == 0 and P.info().tile_items == items
        n = P.info().n_blocks
        rs, ns = oracle.merge_path(A, items)
        assert np.array_equal(_export(P, sp.EXPORT_MERGE_ROWS, n + 1, torch.int32), rs)
        assert np.array_equal(_export(P, sp.EXPORT_MERGE_NZ, n + 1, torch.int32), ns)
    P = sp.spmv_prepare(dA, sp.make_choice("compressed"))
    base, off, wide = oracle.compress_u16(A)
    assert P.info().n_wide_rows == wide
    assert np.array_equal(_export(P, sp.EXPORT_ROWBASE, A.n_rows, torch.int32), base)
    if wide < A.n_rows and A.nnz:
        got = _export(P, sp.EXPORT_OFFSETS, A.nnz, torch.int16).view(np.uint16)
        assert np.array_equal(got, off)


def test_compressed_value_rounding_bit_exact():
    A = synth.random_csr(2000, 3000, 30, seed=12)
    # include values that straddle bfloat16 ties
    A.val = torch.from_numpy(np.random.default_rng(1).standard_normal(A.nnz) * 3.0)
    A.val[:4] = torch.tensor([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -40, 2.0 ** -134],
                             dtype=torch.float64)
    dA = sp.DeviceCSR.from_host(A)
    P = sp.spmv_prepare(dA, sp.make_choice("compressed", value_type=sp.VAL_BF16))
    got = _export(P, sp.EXPORT_VALUES, A.nnz, torch.int16).view(np.uint16)
    assert np.array_equal(got, oracle.round_bf16(A.val))
    P = sp.spmv_prepare(dA, sp.make_choice("compressed", value_type=sp.VAL_F32))
    got = _export(P, sp.EXPORT_VALUES, A.nnz, torch.float32)
    assert np.array_equal(got, oracle.round_f32(A.val))


@pytest.mark.parametrize("vt", [sp.VAL_F32, sp.VAL_BF16])
@pytest.mark.parametrize("name,A", [MATS[0], MATS[2], MATS[6]], ids=["laplacian", "zipf", "wide"])
def test_compressed_low_precision_parity(vt, name, A):
    """FP64 accumulation of the rounded values: within the FP64 bound."""
    lowval = oracle.round_f32(A.val) if vt == sp.VAL_F32 else oracle.round_bf16(A.val)
    P_choice = sp.make_choice("compressed", value_type=vt, accumulate=sp.ACC_F64)
    y, x = _run(A, P_choice)
    ref = oracle.spmv_lowp(A, x, 1 if vt == sp.VAL_F32 else 2, lowval)
    _, scale = oracle.spmv_ref(A, x)
    err = np.abs(y.cpu().numpy() - ref)
    assert np.all(err <= RTOL * scale * 1.01)


def _lowp32_bound(A, x, lowval, vkind):
    """Two FP32 sums of the same rounded products in different orders
    differ by at most 2 * gamma_(n+5) * sum |a_j x_j| with u = 2^-24
    (n = row length; the 5 covers the lane-shuffle levels)."""
    rp = A.rowptr.numpy().astype(np.int64)
    a = np.abs(lowval.astype(np.float64) if vkind == 1
               else (lowval.astype(np.uint32) << 16).view(np.float32).astype(np.float64))
    xf = np.abs(x.cpu().numpy().astype(np.float32).astype(np.float64))
    prod = a * xf[A.colind.numpy()]
    s = np.add.reduceat(np.concatenate([prod, [0.0]]), np.minimum(rp[:-1], A.nnz))
    s[rp[1:] == rp[:-1]] = 0.0
    n = (rp[1:] - rp[:-1]).astype(np.float64) + 5
    u = 2.0 ** -24
    return 2 * (n * u / (1 - n * u)) * s


@pytest.mark.parametrize("vt", [sp.VAL_F32, sp.VAL_BF16])
@pytest.mark.parametrize("tpr", [0, 1, 8, 32])
@pytest.mark.parametrize("name,A", [MATS[0], MATS[2], MATS[6]], ids=["laplacian", "zipf", "wide"])
def test_compressed_fp32_accumulation_parity(vt, tpr, name, A):
    """FP32 accumulation (the default for FP32/BF16 values) against the
    oracle's FP32 form: same rounded x and values, FP32 fused multiply-adds,
    equal up to summation order."""
    vkind = 1 if vt == sp.VAL_F32 else 2
    lowval = oracle.round_f32(A.val) if vkind == 1 else oracle.round_bf16(A.val)
    dA = sp.DeviceCSR.from_host(A)
    P = sp.spmv_prepare(dA, sp.make_choice("compressed", value_type=vt, threads_per_row=tpr))
    assert P.info().accumulate == sp.ACC_F32
    x = synth.uniform_vector(A.n_cols, 11).cuda()
    y = torch.full((A.n_rows,), np.nan, dtype=torch.float64, device="cuda")
    sp.spmv(P, x, y)
    sp.spmv(P, x, y)  # the FP32 copy of x is rewritten each call
    ref = oracle.spmv_lowp32(A, x.cpu(), vkind, lowval)
    err = np.abs(y.cpu().numpy() - ref)
    bound = _lowp32_bound(A, x, lowval, vkind)
    assert np.all(err <= bound), float(np.max(err - bound))
    # outputs are FP32 values widened to FP64
    yn = y.cpu().numpy()
    assert np.array_equal(yn, yn.astype(np.float32).astype(np.float64))


def test_compressed_fp32_accumulation_exact_on_small_integers():
    A = synth.random_csr(3000, 2000, 12, seed=21)
    g = np.random.default_rng(4)
    A.val = torch.from_numpy(g.integers(-8, 9, A.nnz).astype(np.float64))
    x = torch.from_numpy(g.integers(-16, 17, A.n_cols).astype(np.float64))
    dA = sp.DeviceCSR.from_host(A)
    for vt, vkind in ((sp.VAL_F32, 1), (sp.VAL_BF16, 2)):
        lowval = oracle.round_f32(A.val) if vkind == 1 else oracle.round_bf16(A.val)
        P = sp.spmv_prepare(dA, sp.make_choice("compressed", value_type=vt))
        y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        sp.spmv(P, x.cuda(), y)
        assert np.array_equal(y.cpu().numpy(), oracle.spmv_lowp32(A, x, vkind, lowval))
        assert np.array_equal(y.cpu().numpy(), oracle.spmv(A, x))


def test_accumulate_choice_validation():
    A = synth.laplacian_2d_5pt(20)
    dA = sp.DeviceCSR.from_host(A)
    assert sp.spmv_prepare(dA, sp.make_choice("compressed")).info().accumulate == sp.ACC_F64
    assert sp.spmv_prepare(dA, sp.make_choice("compressed", value_type=sp.VAL_F32,
                                              accumulate=sp.ACC_F64)).info().accumulate == sp.ACC_F64
    for bad in (sp.make_choice("compressed", accumulate=sp.ACC_F32),
                sp.make_choice("subwarp", accumulate=sp.ACC_F32),
                sp.make_choice("compressed", value_type=sp.VAL_BF16, accumulate=3)):
        with pytest.raises(sp.SpmvError):
            sp.spmv_prepare(dA, bad)


def test_gather_probe_sum_and_launch_counts():
    A = synth.random_csr(50_000, 70_000, 9, seed=31)
    g = np.random.default_rng(2)
    x = torch.from_numpy(g.integers(-4, 5, A.n_cols).astype(np.float64))
    dA = sp.DeviceCSR.from_host(A)
    out = torch.empty(1, dtype=torch.int64, device="cuda")
    sp.spmv_gather_probe(dA, x.cuda(), out)
    bits = x.numpy().view(np.uint64)[A.colind.numpy()]
    with np.errstate(over="ignore"):
        expect = np.add.reduce(bits, dtype=np.uint64)
    assert np.uint64(out.cpu().numpy().view(np.uint64)[0]) == expect
    expect = {"scalar": 1, "subwarp": 1, "latency": 1, "merge": 2}
    for v, n in expect.items():
        assert sp.spmv_prepare(dA, sp.make_choice(v)).info().launches == n
    assert sp.spmv_prepare(dA, sp.make_choice("compressed")).info().launches == 1
    assert sp.spmv_prepare(dA, sp.make_choice("compressed", value_type=sp.VAL_BF16)).info().launches == 2
    Z = synth.zipf_rows(20_000, 20_000, 1.5, 10_000, seed=1)
    dZ = sp.DeviceCSR.from_host(Z)
    P = sp.spmv_prepare(dZ, sp.make_choice("dynamic", block_nnz=256))
    assert P.info().launches == 1  # long rows summed by the warp finishing their last segment


# ----------------------------------------------------------------- profile + select
def test_profile_runs_and_selection_consistent():
    A = synth.zipf_rows(200_000, 200_000, 1.5, 50_000, seed=3)
    dA = sp.DeviceCSR.from_host(A)
    x = synth.uniform_vector(A.n_cols, 0).cuda()
    p = sp.spmv_profile(dA, x, reps=3)
    d = p.as_dict()
    for k in ("t_base_ms", "t_noxmiss_ms", "t_inflate_ms", "t_span_ms", "t_worker_mean_ms"):
        assert d[k] > 0 and np.isfinite(d[k]), k
    assert d["s_noxmiss"] == d["t_base_ms"] / d["t_noxmiss_ms"]
    assert d["s_inflate"] == d["t_inflate_ms"] / d["t_base_ms"]
    assert d["t_span_ms"] >= d["t_worker_mean_ms"]
    ch = sp.spmv_select(profile=p)
    t = sp.spmv_default_thresholds()
    cls = oracle.profile_class(d["s_noxmiss"], d["s_inflate"], d["s_balance"],
                               tau=(t.tau_noxmiss, t.tau_inflate, t.tau_balance))
    assert ch.cls == cls and ch.variant == oracle.class_variant(cls, [sp.spmv_class_variant(c) for c in range(4)])
    # one giant row among short ones: the balance probe must see the imbalance
    assert d["s_balance"] > 2.0


def test_spmv_host_end_to_end():
    A = synth.stencil_27pt(12, seed=1)
    dA = sp.DeviceCSR.from_host(A)
    P = sp.spmv_prepare(dA, sp.make_choice("stream"))
    x = synth.uniform_vector(A.n_cols, 5).pin_memory()
    y = torch.empty(A.n_rows, dtype=torch.float64).pin_memory()
    for _ in range(2):
        sp.spmv_host(P, x, y)
        _assert_close(y, A, x)


def test_spmv_host_async_on_several_streams():
    """Matrices issued with spmv_host_async on separate streams, each y
    valid after its stream is synchronised."""
    mats = [synth.stencil_27pt(14, seed=3), synth.random_csr(20_000, 15_000, 12, seed=4),
            synth.short_rows(30_000, 8, seed=5)]
    variants = ["sliced", "subwarp", "compressed"]
    preps = [sp.spmv_prepare(sp.DeviceCSR.from_host(A), sp.make_choice(v)) for A, v in zip(mats, variants)]
    xs = [synth.uniform_vector(A.n_cols, 20 + i).pin_memory() for i, A in enumerate(mats)]
    ys = [torch.full((A.n_rows,), float("nan"), dtype=torch.float64).pin_memory() for A in mats]
    streams = [torch.cuda.Stream() for _ in mats]
    for _ in range(2):
        for P, x, y, s in zip(preps, xs, ys, streams):
            sp.spmv_host_async(P, x, y, stream=s)
        for s in streams:
            s.synchronize()
        for A, x, y in zip(mats, xs, ys):
            _assert_close(y, A, x)


# ----------------------------------------------------------------- full size
@pytest.fixture(scope="module")
def four_class():
    return synth.four_class_set()


def test_latency_persisting_carve_out_released():
    """LATENCY with an x over half the L2 raises the persisting-L2 carve-out
    while an object needs it; freeing the last such object puts it back, so
    that later kernels get the whole L2 (stale persisting lines measured
    6-20 % slower SLICED and DYNAMIC launches)."""
    import ctypes
    cu = ctypes.CDLL("libcuda.so.1")

    def limit():
        v = ctypes.c_size_t()
        assert cu.cuCtxGetLimit(ctypes.byref(v), 6) == 0  # CU_LIMIT_PERSISTING_L2_CACHE_SIZE
        return v.value

    torch.cuda.synchronize()
    before = limit()
    l2 = getattr(torch.cuda.get_device_properties(0), "L2_cache_size", 128 << 20)
    A = synth.random_columns(4096, l2 // 8 + 4096, 8, seed=21)  # x of more than the whole L2
    dA = sp.DeviceCSR.from_host(A)
    P = sp.spmv_prepare(dA, sp.make_choice("latency"))
    raised = limit()
    assert raised >= before
    x = synth.uniform_vector(A.n_cols, 4)
    y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
    sp.spmv(P, x.cuda(), y)
    torch.cuda.synchronize()
    _assert_close(y, A, x)
    Q = sp.spmv_prepare(dA, sp.make_choice("latency"))  # a second user
    P.free()
    assert limit() == raised
    Q.free()
    assert limit() == before


def _sample_rows(A, k=3000, seed=0):
    g = np.random.default_rng(seed)
    lens = (A.rowptr[1:] - A.rowptr[:-1]).numpy()
    rows = np.concatenate([[0, A.n_rows - 1, int(np.argmax(lens))], g.integers(0, A.n_rows, k)])
    return np.unique(rows)


FULL_CHOICES = [("scalar", {}), ("subwarp", {}), ("stream", {}), ("merge", {}), ("dynamic", {}),
                ("latency", {}), ("compressed", {}), ("sliced", {}), ("sliced", {"threads_per_row": 2})]


@pytest.mark.parametrize("variant,params", FULL_CHOICES, ids=[v for v, _ in FULL_CHOICES])
def test_full_size_sampled_parity(four_class, variant, params):
    """The four-class matrices at full size (2.1M-8.4M rows, 17M-67M nonzeros)
    in the launch configuration the benchmark times; rows sampled."""
    for A in four_class:
        y, x = _run(A, sp.make_choice(variant, **params))
        _assert_close(y, A, x, rows=_sample_rows(A))


def test_full_size_selected_configuration_parity(four_class):
    """Each four-class matrix at full size with the choice the benchmark
    makes: Table 1 features, the committed selector's two levels, prepare,
    one SpMV; rows sampled."""
    data = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_1511_02494_gb300", "data")
    model = sp.spmv_model_load(os.path.join(data, "selector_mlp.bin"))
    sub = sp.spmv_model_load(os.path.join(data, "selector_sliced_mlp.bin"))
    for A in four_class:
        dA = sp.DeviceCSR.from_host(A)
        ch = sp.spmv_select_model_refined(sp.spmv_features(dA), model, sub)
        y, x = _run(A, ch)
        _assert_close(y, A, x, rows=_sample_rows(A))


def test_full_size_features_bit_exact(four_class):
    for A in four_class:
        _features_match(A)


def test_prepared_free_releases_every_array():
    # narrow (int16) stored columns and long-row segment tables are owned
    # arrays too: repeated prepare/free must not lose device memory
    cases = [(synth.stencil_27pt(40, seed=1), dict(index_bytes=2)),
             (synth.zipf_rows(50_000, 50_000, 1.5, 20_000, seed=2), dict(block_nnz=4096, items_per_warp=32)),
             (synth.stencil_27pt(40, seed=1), dict(value_type=sp.VAL_BF16))]
    dev = [(sp.DeviceCSR.from_host(A), kw) for A, kw in cases]
    for dA, kw in dev:  # warm-up: scratch kept per thread is allocated once
        sp.spmv_prepare(dA, sp.make_choice("sliced", **kw)).free()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(20):
        for dA, kw in dev:
            sp.spmv_prepare(dA, sp.make_choice("sliced", **kw)).free()
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] < (16 << 20)
