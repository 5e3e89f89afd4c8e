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
