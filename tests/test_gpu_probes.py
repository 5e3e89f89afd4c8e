"""GPU parity of the profiling runs (Section 3.2.1) against the CPU oracle.

spmv_profile only times its probes; spmv_profile_outputs returns what each
computes, on the same kernels and set-up.  Checked here, through the C ABI:
  * the baseline's static equal-nonzero partition, bit-exact against
    oracle.static_partition, for the worker count spmv_profile uses and for
    counts below and far above the number of rows;
  * the baseline's y against the oracle within 1e-12 * sum_j |a_ij x_j|;
  * the inflate (64-bit indices) and balance (time-stamped) runs bit-identical
    to the baseline, since they change only the index width or add stamps;
  * the noxmiss run against the oracle's product with every column index 0,
    y_i = x[0] * sum_j a_ij, within 1e-12 * sum_j |a_ij x[0]|.
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
    sp.lib()


class _Host:
    def __init__(self, n_rows, n_cols, rowptr, colind, val):
        self.n_rows, self.n_cols = n_rows, n_cols
        self.rowptr, self.colind, self.val = rowptr, colind, val
        self.nnz = int(colind.numel())


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
    yield "zipf_200k", synth.zipf_rows(200_000, 200_000, 1.5, 50_000, seed=3)


MATS = list(_matrices())


def _outputs(A, x, W):
    dA = sp.DeviceCSR.from_host(A)
    dx = x.cuda()
    n = A.n_rows
    ys = [torch.full((n,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(4)]
    wb = W if W > 0 else sp.spmv_profile(dA, dx, reps=1).n_workers
    bounds = torch.full((wb + 1,), -7, dtype=torch.int64, device="cuda")
    sp.spmv_profile_outputs(dA, dx, W, bounds, *ys)
    torch.cuda.synchronize()
    return wb, bounds.cpu().numpy(), [y.cpu().numpy() for y in ys]


@pytest.mark.parametrize("name,A", MATS, ids=[m[0] for m in MATS])
def test_probe_outputs_match_oracle(name, A):
    x = synth.uniform_vector(A.n_cols, 11)
    W, bounds, (yb, yn, yi, ys) = _outputs(A, x, 0)
    assert np.array_equal(bounds, oracle.static_partition(A, W))
    y_ref, scale = oracle.spmv_ref(A, x)
    assert np.all(np.abs(yb - y_ref) <= RTOL * scale), name
    assert np.all(yb[scale == 0] == 0.0)
    assert np.array_equal(yi, yb) and np.array_equal(ys, yb)
    Z = _Host(A.n_rows, A.n_cols, A.rowptr, torch.zeros_like(A.colind), A.val)
    z_ref, z_scale = oracle.spmv_ref(Z, x)
    assert np.all(np.abs(yn - z_ref) <= RTOL * z_scale), name
    # the closed form of the noxmiss product: x[0] times the row sums
    rs = np.add.reduceat(np.append(A.val.numpy(), 0.0), A.rowptr.numpy()[:-1].astype(np.int64))
    rs[np.diff(A.rowptr.numpy()) == 0] = 0.0
    assert np.allclose(yn, float(x[0]) * rs, rtol=1e-12, atol=1e-12 * np.abs(A.val.numpy()).sum())


@pytest.mark.parametrize("W", [1, 7, 64, 4999, 100_000])
def test_probe_partition_any_worker_count(W):
    A = synth.zipf_rows(5000, 5000, 1.5, 3000, seed=1)
    x = synth.uniform_vector(A.n_cols, 2)
    _, bounds, (yb, _, _, _) = _outputs(A, x, W)
    b = oracle.static_partition(A, W)
    assert np.array_equal(bounds, b)
    # every row is in exactly one worker's range, so y is complete for any W
    y_ref, scale = oracle.spmv_ref(A, x)
    assert np.all(np.abs(yb - y_ref) <= RTOL * scale)


def test_probe_outputs_reject_empty_and_bad_counts():
    A = synth.random_csr(100, 100, 0, seed=1)
    dA = sp.DeviceCSR.from_host(A)
    x = torch.zeros(100, dtype=torch.float64, device="cuda")
    with pytest.raises(sp.SpmvError) as e:
        sp.spmv_profile_outputs(dA, x, 0)
    assert e.value.status == 3
    B = sp.DeviceCSR.from_host(synth.laplacian_2d_5pt(8, 8))
    with pytest.raises(sp.SpmvError) as e:
        sp.spmv_profile_outputs(B, torch.zeros(64, dtype=torch.float64, device="cuda"), -1)
    assert e.value.status == 1
