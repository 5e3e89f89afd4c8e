"""The no-allocation entry point, spmv_stream_noalloc.

It serves callers that must not allocate device memory (a solver loop that
may never stall the device on cudaMalloc/cudaFree, or a program that commits
all device memory through its own allocator up front): its scratch is a fixed
static device array instead of prepared buffers.  Here it is called through
the C ABI, on two calls in a row, and compared with the oracle's product
(within the parity tolerance of the other GPU tests) and with the existing
entry point (spmv on a STREAM-prepared matrix).  The scratch is shared by
every call and keeps the last call's contents, so the cases also run a small
matrix right after a large one and a matrix with rows but no nonzeros.  The
file name makes pytest collect it last.
"""
import ctypes as C

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


def _matrices():
    return [synth.laplacian_2d_5pt(64, 64), synth.zipf_rows(20000, 20000, 1.5, 9000, seed=3),
            synth.stencil_27pt(24, seed=5), synth.random_csr(3000, 500, 40, seed=6, empty_frac=0.3),
            synth.random_csr(3000, 500, 0, seed=7)]


def _noalloc(lib, dA, x, n_rows):
    y = torch.full((n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.spmv_stream_noalloc(C.byref(dA.desc), C.c_void_p(x.data_ptr()),
                                 C.c_void_p(y.data_ptr()), stream)
    assert st == 0, lib.spmv_last_error().decode()
    assert lib.spmv_stream_noalloc_status(stream) == 0, lib.spmv_last_error().decode()
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("k", range(5))
def test_noalloc_matches_oracle_and_existing_entry_point_twice(k):
    A = _matrices()[k]
    dA = sp.DeviceCSR.from_host(A)
    P = sp.spmv_prepare(dA, sp.make_choice("stream", block_nnz=2048))
    lib = sp.lib()
    for call in range(2):
        x = synth.uniform_vector(A.n_cols, 9 + call).cuda()
        y_ref, scale = oracle.spmv_ref(A, x.cpu())
        y_st = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
        sp.spmv(P, x, y_st)
        a = _noalloc(lib, dA, x, A.n_rows)
        b = y_st.cpu().numpy()
        assert np.all(np.abs(a - y_ref) <= RTOL * scale), call
        assert np.all(np.abs(a - b) <= RTOL * scale), call
        assert np.all(a[scale == 0] == 0.0)
    P.free()


def test_noalloc_small_matrix_after_a_large_one():
    # the large call leaves its window starts and carried rows in the shared
    # scratch; the small call right after must not pick any of them up
    lib = sp.lib()
    big = synth.zipf_rows(60000, 60000, 1.4, 40000, seed=8)
    small = synth.random_csr(700, 300, 30, seed=9, empty_frac=0.2)
    for A in (big, small, big, small):
        dA = sp.DeviceCSR.from_host(A)
        x = synth.uniform_vector(A.n_cols, 4).cuda()
        y_ref, scale = oracle.spmv_ref(A, x.cpu())
        y = _noalloc(lib, dA, x, A.n_rows)
        assert np.all(np.abs(y - y_ref) <= RTOL * scale)


def test_noalloc_rejects_oversized_and_unaligned():
    lib = sp.lib()
    A = synth.laplacian_2d_5pt(8, 8)
    dA = sp.DeviceCSR.from_host(A)
    x = torch.zeros(A.n_cols, dtype=torch.float64, device="cuda")
    y = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    big = sp.CSR(A.n_rows, A.n_cols, 65536 * 2048 + 1, dA.desc.rowptr, dA.desc.colind, dA.desc.val)
    assert lib.spmv_stream_noalloc(C.byref(big), C.c_void_p(x.data_ptr()),
                                   C.c_void_p(y.data_ptr()), None) == 3
    assert "134217728" in lib.spmv_last_error().decode()
    buf = torch.zeros(A.nnz + 1, dtype=torch.float64, device="cuda")
    odd = sp.CSR(A.n_rows, A.n_cols, A.nnz, dA.desc.rowptr, dA.desc.colind,
                 C.c_void_p(buf.data_ptr() + 8))
    assert lib.spmv_stream_noalloc(C.byref(odd), C.c_void_p(x.data_ptr()),
                                   C.c_void_p(y.data_ptr()), None) == 3
