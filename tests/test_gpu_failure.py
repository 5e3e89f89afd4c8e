"""Failure detection without a GPU fault: the bounded device wait of the
pipelined kernels gives up by itself, reports a timeout status, and the
context stays usable."""
import time

import numpy as np
import pytest
import torch

import oracle
import paper_1511_02494_gb300 as sp
import synth

pytestmark = pytest.mark.gpu


def _name(e):
    return sp.STATUS_NAMES[e.value.status]


def test_bounded_wait_completes_when_the_arrival_comes():
    sp.spmv_wait_check(50_000_000, arrive=True)


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    t0 = time.perf_counter()
    with pytest.raises(sp.SpmvError) as e:
        sp.spmv_wait_check(5_000_000, arrive=False)   # nothing arrives: 5 ms limit
    assert _name(e) == "SPMV_ERR_TIMEOUT"
    assert time.perf_counter() - t0 < 5.0
    # the device still runs the library's kernels, and a later check passes
    A = synth.laplacian_2d_5pt(64, 64)
    x = synth.uniform_vector(A.n_cols, 3)
    dA = sp.DeviceCSR.from_host(A)
    y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
    for v in ("stream", "merge", "sliced"):
        P = sp.spmv_prepare(dA, sp.make_choice(v))
        sp.spmv(P, x.cuda(), y)
        sp.spmv_prepared_status(P)
        ref, scale = oracle.spmv_ref(A, x)
        assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-12 * scale)
    sp.spmv_wait_check(50_000_000, arrive=True)


@pytest.mark.parametrize("limit", [0, -1, 3_000_000_000])
def test_bounded_wait_check_rejects_bad_limits(limit):
    with pytest.raises(sp.SpmvError) as e:
        sp.spmv_wait_check(limit, arrive=False)
    assert _name(e) == "SPMV_ERR_INVALID_ARG"


def _fixup(kind, carry_row, carry_val, status, y):
    n_parts = len(carry_row)
    cr = torch.tensor(carry_row, dtype=torch.int32, device="cuda")
    cv = torch.tensor(carry_val, dtype=torch.float64, device="cuda")
    st = torch.tensor([status], dtype=torch.int32, device="cuda")
    yd = torch.tensor(y, dtype=torch.float64, device="cuda")
    assert cr.numel() == n_parts
    sp.spmv_fixup_check(kind, cr, cv, st, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("kind", [0, 1])
def test_fixup_skips_out_of_range_carry_rows(kind):
    # parts 1-2 carry row 3, part 5 row 7; -5, 10 and 99999 lie outside the
    # 10 rows (left by an earlier, larger matrix) and must be ignored
    rows = [-5, 3, 3, 99999, -1, 7, 10]
    vals = [100.0, 0.5, 0.25, 100.0, 100.0, 2.0, 100.0]
    y0 = np.arange(10, dtype=np.float64)
    y = _fixup(kind, rows, vals, 0, y0)
    want = y0.copy()
    want[3] += 0.75
    want[7] += 2.0
    assert np.array_equal(y, want)


@pytest.mark.parametrize("kind", [0, 1])
def test_fixup_does_nothing_after_a_timeout(kind):
    # a bounded wait gave up (status set): the carries may be stale, y is left alone
    rows = [0, 0, 99999, -3, 4]
    y0 = np.linspace(-1.0, 1.0, 5)
    y = _fixup(kind, rows, [1.0] * 5, 1, y0)
    assert np.array_equal(y, y0)


def test_fixup_check_rejects_bad_arguments():
    lib = sp.lib()
    assert lib.spmv_fixup_check(2, 1, 1, None, None, None, None, None) == 1
    assert lib.spmv_fixup_check(0, -1, 1, None, None, None, None, None) == 1
    assert lib.spmv_fixup_check(0, 3, 1, None, None, None, None, None) == 1
