"""Index tables that two variants prepare, against the oracle, through the
C ABI (spmv_prepared_export):

* DYNAMIC's row tiers (Table 2's IMB optimization with rows split by
  length).  The lists are filled with atomics, so a prepare fixes each
  list's set of rows, not their order: the sets are compared with the
  oracle's orc_dyn_tiers, and the segment offsets are checked for the order
  the prepare produced (a running sum of ceil(len / segment)).
* SLICED's long-row segment table (reading O22): the long rows (ascending),
  segment offsets and bounds, single-segment rows, the rows summed from
  partials; bit-exact against orc_sliced_segments.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1511_02494_gb300 as sp
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1511_02494_gb300.build import build
    build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _export(P, which, n, dtype):
    out = torch.empty(n, dtype=dtype)
    sp.spmv_prepared_export(P, which, out)
    return out.numpy()


def _mats():
    yield "zipf_long_rows", synth.zipf_rows(5000, 5000, 1.5, 3000, seed=1)
    yield "zipf_200k", synth.zipf_rows(200_000, 200_000, 1.5, 50_000, seed=3)
    yield "random_empty_rows", synth.random_csr(1000, 700, 40, seed=3, empty_frac=0.3)
    yield "short_rows", synth.short_rows(3001, 8, seed=2)
    yield "one_dense_row", synth.dense_to_csr(torch.cat([torch.rand(1, 9000, dtype=torch.float64) + 0.1,
                                                         torch.zeros(3, 9000, dtype=torch.float64)]))
    yield "stencil27_n10", synth.stencil_27pt(10, seed=4)


MATS = list(_mats())


@pytest.mark.parametrize("kw", [{}, {"threads_per_row": 1}, {"threads_per_row": 8},
                                {"threads_per_row": 32, "block_nnz": 256}, {"block_nnz": 256}])
@pytest.mark.parametrize("name,A", MATS, ids=[m[0] for m in MATS])
def test_dynamic_tiers_match_oracle(name, A, kw):
    dA = sp.DeviceCSR.from_host(A)
    P = sp.spmv_prepare(dA, sp.make_choice("dynamic", **kw))
    info = P.info()
    T, seg = info.threads_per_row, info.block_nnz
    m1, m2, lr, sc = oracle.dyn_tiers(A, min(16 * T, seg), seg)
    g1 = _export(P, sp.EXPORT_DYN_M1, len(m1), torch.int32)
    g2 = _export(P, sp.EXPORT_DYN_M2, len(m2), torch.int32)
    gl = _export(P, sp.EXPORT_DYN_LONG, len(lr), torch.int32)
    assert np.array_equal(np.sort(g1), m1) and np.array_equal(np.sort(g2), m2)
    assert np.array_equal(np.sort(gl), lr)
    if len(lr):
        off = _export(P, sp.EXPORT_DYN_SEG_OFF, len(lr) + 1, torch.int32)
        lens = np.diff(A.rowptr.numpy().astype(np.int64))[gl]
        assert off[0] == 0 and np.array_equal(np.diff(off), -(-lens // seg))
    P.free()


@pytest.mark.parametrize("sigma,cap", [(1, 1024), (4096, 32), (1, 8)])
@pytest.mark.parametrize("vt", [sp.VAL_F64, sp.VAL_BF16])
@pytest.mark.parametrize("name,A", MATS, ids=[m[0] for m in MATS])
def test_sliced_segment_table_bit_exact(name, A, sigma, cap, vt):
    dA = sp.DeviceCSR.from_host(A)
    P = sp.spmv_prepare(dA, sp.make_choice("sliced", block_nnz=sigma, items_per_warp=cap, value_type=vt))
    lst, off, be, srow, fix, sfix = oracle.sliced_segments(A, cap, 2048)
    assert P.info().n_long_rows == len(lst)
    if len(lst) == 0:
        return
    ns = len(srow)
    assert np.array_equal(_export(P, sp.EXPORT_SLICE_LONG, len(lst), torch.int32), lst)
    assert np.array_equal(_export(P, sp.EXPORT_SLICE_SEG_OFF, len(lst) + 1, torch.int32), off)
    assert np.array_equal(_export(P, sp.EXPORT_SLICE_SEG_BOUNDS, 2 * ns, torch.int64), be.reshape(-1))
    assert np.array_equal(_export(P, sp.EXPORT_SLICE_SEG_ROW, ns, torch.int32), srow)
    assert np.array_equal(_export(P, sp.EXPORT_SLICE_FIX, len(fix), torch.int32), fix)
    if vt == sp.VAL_F64:
        assert np.array_equal(_export(P, sp.EXPORT_SLICE_SEG_FIX, ns, torch.int32), sfix)
    P.free()
