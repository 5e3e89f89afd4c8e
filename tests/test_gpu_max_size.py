"""The library at its size limit: 2,147,483,600 nonzeros (the largest even
count below 2^31 - 1, the int32 index limit), 1,073,741,800 rows of two.
Row i < N - 1 holds columns {i, i + 1}; the last row holds {0, N - 1}.

* Table 1 features (Section 3.2.2) against their closed forms: every
  aggregate of this matrix follows from the two row kinds, so the GPU's
  exact integer sums (64- and 128-bit) are checked bit for bit.
* y of the plain CSR kernel and of SLICED (whose slice storage here holds
  2^31 slots, so slot indices pass 32 bits; every row has two nonzeros, so
  it is the header-free kernel) on sampled rows -- the first,
  the last and 4096 random ones -- against the oracle's product of those rows,
  within 1e-12 * sum_j |a_ij x_j|.
About 80 GB of device memory; the arrays are built on the device in chunks.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1511_02494_gb300 as sp
import synth

pytestmark = pytest.mark.gpu
N = 1_073_741_800
NNZ = 2 * N
CHUNK = 1 << 26


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1511_02494_gb300.build import build
    build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.fixture(scope="module")
def big():
    dev = "cuda"
    rowptr = torch.arange(0, NNZ + 1, 2, dtype=torch.int32, device=dev)
    colind = torch.empty(NNZ, dtype=torch.int32, device=dev)
    val = torch.empty(NNZ, dtype=torch.float64, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(12)
    for a in range(0, N, CHUNK):
        b = min(N, a + CHUNK)
        r = torch.arange(a, b, dtype=torch.int64, device=dev)
        colind[2 * a:2 * b] = torch.stack([r, r + 1], 1).reshape(-1).to(torch.int32)
        val[2 * a:2 * b] = torch.rand(2 * (b - a), generator=g, dtype=torch.float64, device=dev) * 2 - 1
        del r
    colind[NNZ - 2] = 0
    colind[NNZ - 1] = N - 1
    x = synth.uniform_vector(N, 5, device=dev)
    A = sp.DeviceCSR(N, N, rowptr, colind, val)
    yield A, x
    del A, rowptr, colind, val, x
    torch.cuda.empty_cache()


def test_features_at_the_size_limit(big):
    A, _ = big
    f = sp.spmv_features(A).as_dict()
    n = N
    q_last = (1 << 33) // n          # disp of the last row: floor(2^32 * 2 / n)
    assert f["nnz"] == NNZ and f["nnz_min"] == 2 and f["nnz_max"] == 2
    assert f["nnz_sum"] == 2 * n and f["nnz_sumsq"] == 4 * n
    assert f["bw_min"] == 1 and f["bw_max"] == n - 1
    assert f["bw_sum"] == 2 * (n - 1) and f["bw_sumsq"] == (n - 1) + (n - 1) ** 2
    assert f["ngroups_sum"] == n + 1 and f["misses_sum"] == n + 1
    assert f["disp_sum"] == (n - 1) * (1 << 32) + q_last
    assert f["disp_sumsq"] == (n - 1) * (1 << 64) + q_last * q_last
    assert f["clust_sum"] == (n - 1) * (1 << 31) + (1 << 32)


def _sample_reference(A, x, rows):
    rp = A.rowptr[torch.from_numpy(rows).cuda()].to(torch.int64)
    idx = torch.stack([rp, rp + 1], 1).reshape(-1)
    cols = A.colind[idx].cpu().numpy().astype(np.int64)
    vals = A.val[idx].cpu()
    uniq, inv = np.unique(cols, return_inverse=True)
    xs = x[torch.from_numpy(uniq).cuda()].cpu()
    S = synth.HostCSR(len(rows), len(uniq), torch.arange(0, 2 * len(rows) + 1, 2, dtype=torch.int32),
                      torch.from_numpy(inv.astype(np.int32)), vals)
    return oracle.spmv_ref(S, xs)


@pytest.mark.parametrize("variant", ["scalar", "sliced"])
def test_spmv_at_the_size_limit(big, variant):
    A, x = big
    rows = np.unique(np.concatenate([[0, 1, N - 2, N - 1],
                                     np.random.default_rng(3).integers(0, N, 4096)])).astype(np.int64)
    y_ref, scale = _sample_reference(A, x, rows)
    P = sp.spmv_prepare(A, sp.make_choice(variant))
    info = P.info()
    if variant == "sliced":
        # every row has two nonzeros: the header-free kernel, whose slot
        # index 64 s + 32 k + lane passes 2^31; the last row's reach keeps
        # 32-bit columns
        assert info.n_blocks == (N + 31) // 32 and info.n_long_rows == 0
        assert info.uniform_len == 2 and info.index_bytes == 4
    y = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
    sp.spmv(P, x, y)
    torch.cuda.synchronize()
    got = y[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.all(np.abs(got - y_ref) <= 1e-12 * scale)
    assert not torch.isnan(y).any()
    P.free()
    del y
    torch.cuda.empty_cache()
