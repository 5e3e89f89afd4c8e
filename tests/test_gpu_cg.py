"""Conjugate gradients on the GPU against the oracle's CG (same algorithm,
same arithmetic up to summation order): FP64 throughout, and a low-precision
inner SpMV (FP32 / BF16 values, FP64 accumulation) with FP64 residual
recomputation; FP32 accumulation is checked against the FP64 solve's
accuracy instead."""
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
    assert torch.cuda.is_available()


def _run(A, b, iters, inner, refine=0, graph=False, exact="subwarp"):
    dA = sp.DeviceCSR.from_host(A)
    Pi = sp.spmv_prepare(dA, inner)
    Pe = sp.spmv_prepare(dA, sp.make_choice(exact))
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    res = torch.empty(iters + 1, dtype=torch.float64, device="cuda")
    sp.spmv_cg(Pi, b.cuda(), x, iters, refine, A_exact=Pe, resid=res, use_graph=graph)
    torch.cuda.synchronize()
    return x.cpu().numpy(), res.cpu().numpy()


def _close(x, r, xo, ro):
    assert np.max(np.abs(x - xo)) <= 1e-9 * np.max(np.abs(xo))
    assert np.all(np.abs(r - ro) <= 1e-6 * ro + 1e-12 * ro[0])


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("variant", ["subwarp", "compressed", "dynamic", "stream", "sliced", "sliced_i8"])
def test_cg_fp64_matches_oracle(variant, graph):
    A = synth.variable_coeff_laplacian_3d(14, seed=1)
    b = synth.uniform_vector(A.n_rows, 3)
    # sliced_i8: the fused kernel with column offsets from the row index
    # (this matrix's rows reach 196 columns from the diagonal: 16 bits)
    ch = sp.make_choice("sliced", index_bytes=1) if variant == "sliced_i8" else sp.make_choice(variant)
    x, r = _run(A, b, 60, ch, graph=graph)
    xo, ro = oracle.cg(A, b, np.zeros(A.n_rows), 60)
    _close(x, r, xo, ro)
    assert r[-1] < 1e-6 * r[0]


def _periodic_laplacian(n: int, shift: float, seed: int):
    """2-D five-point operator on an n x n torus with a diagonal of 4 + shift
    and random off-diagonal weights in [-1, -0.5], symmetrised: SPD, and
    every row has five nonzeros (the uniform sliced layout)."""
    g = np.random.default_rng(seed)
    N = n * n
    idx = lambda i, j: (i % n) * n + (j % n)
    w_right = -g.uniform(0.5, 1.0, N)
    w_down = -g.uniform(0.5, 1.0, N)
    rows = []
    for i in range(n):
        for j in range(n):
            r = idx(i, j)
            e = {r: 4.0 + shift,
                 idx(i, j + 1): w_right[r], idx(i, j - 1): w_right[idx(i, j - 1)],
                 idx(i + 1, j): w_down[r], idx(i - 1, j): w_down[idx(i - 1, j)]}
            rows.append(sorted(e.items()))
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    ci = np.array([c for r in rows for c, _ in r], np.int32)
    va = np.array([v for r in rows for _, v in r], np.float64)
    return synth.HostCSR(N, N, torch.from_numpy(rp), torch.from_numpy(ci), torch.from_numpy(va),
                         f"torus_{n}")


@pytest.mark.parametrize("graph", [False, True])
def test_cg_rows_of_one_length(graph):
    """Every row of the torus operator has five nonzeros: SLICED's default
    form stores its columns as int16 offsets from the row, and the CG loop
    (fused SpMV and dot) runs on that form; it agrees with the oracle."""
    A = _periodic_laplacian(24, 0.5, seed=7)
    P = sp.spmv_prepare(sp.DeviceCSR.from_host(A), sp.make_choice("sliced"))
    assert P.info().index_bytes == 2 and P.info().block_nnz == 1
    b = synth.uniform_vector(A.n_rows, 5)
    x, r = _run(A, b, 40, sp.make_choice("sliced"), graph=graph)
    xo, ro = oracle.cg(A, b, np.zeros(A.n_rows), 40)
    _close(x, r, xo, ro)
    assert r[-1] < 1e-6 * r[0]


@pytest.mark.parametrize("vt,vkind", [(sp.VAL_F32, 1), (sp.VAL_BF16, 2)])
@pytest.mark.parametrize("refine", [0, 10])
def test_cg_low_precision_inner_matches_oracle(vt, vkind, refine):
    A = synth.variable_coeff_laplacian_3d(12, seed=2)
    b = synth.uniform_vector(A.n_rows, 4)
    low = oracle.round_f32(A.val) if vkind == 1 else oracle.round_bf16(A.val)
    for variant in ("compressed", "sliced"):
        x, r = _run(A, b, 50, sp.make_choice(variant, value_type=vt, accumulate=sp.ACC_F64),
                    refine=refine)
        xo, ro = oracle.cg(A, b, np.zeros(A.n_rows), 50, vkind=vkind, lowval=low, refine=refine)
        _close(x, r, xo, ro)


def test_cg_refinement_recovers_fp64_accuracy():
    """With BF16 values the recursive residual drifts from the true one;
    recomputing it in FP64 every 10 iterations brings the true residual of
    the BF16-inner solve down to the FP64 solve's level."""
    A = synth.variable_coeff_laplacian_3d(16, seed=3)
    b = synth.uniform_vector(A.n_rows, 5)
    x64, _ = _run(A, b, 120, sp.make_choice("subwarp"))
    xr, _ = _run(A, b, 120, sp.make_choice("compressed", value_type=sp.VAL_BF16), refine=10)
    xn, _ = _run(A, b, 120, sp.make_choice("compressed", value_type=sp.VAL_BF16), refine=0)

    def true_res(x):
        return np.linalg.norm(b.numpy() - oracle.spmv(A, x)) / np.linalg.norm(b.numpy())

    assert true_res(x64) < 1e-9
    assert true_res(xr) < 1e-8
    assert true_res(xn) > 10 * true_res(xr)


@pytest.mark.parametrize("vt", [sp.VAL_F32, sp.VAL_BF16])
@pytest.mark.parametrize("graph", [False, True])
def test_cg_fp32_accumulation_with_refinement_reaches_fp64_accuracy(vt, graph):
    """The all-FP32 inner SpMV (FP32 x copy, FP32 sums) loses about 1e-7
    relative accuracy per product; FP64 residual recomputation every 10
    iterations still drives the true residual to the FP64 solve's level."""
    A = synth.variable_coeff_laplacian_3d(16, seed=3)
    b = synth.uniform_vector(A.n_rows, 5)
    x, _ = _run(A, b, 150, sp.make_choice("compressed", value_type=vt), refine=10, graph=graph)
    xn, _ = _run(A, b, 150, sp.make_choice("compressed", value_type=vt), refine=0)
    # the fused SLICED path (p's FP32 copy written by the p update)
    xs, _ = _run(A, b, 150, sp.make_choice("sliced", value_type=vt), refine=10, graph=graph,
                 exact="sliced")
    res_s = np.linalg.norm(b.numpy() - oracle.spmv(A, xs)) / np.linalg.norm(b.numpy())
    assert res_s < 1e-8
    res = np.linalg.norm(b.numpy() - oracle.spmv(A, x)) / np.linalg.norm(b.numpy())
    res_n = np.linalg.norm(b.numpy() - oracle.spmv(A, xn)) / np.linalg.norm(b.numpy())
    assert res < 1e-8
    assert res_n > 10 * res


def _laplacian_with_full_row(m=40, eps=1e-3):
    """SPD: the 2-D Laplacian on an m x m grid plus a weak coupling of row
    and column 0 to every other unknown (a row above 1024 nonzeros), with the
    diagonal raised to keep it dominant; conditioned like the Laplacian."""
    L = synth.laplacian_2d_5pt(m, m)
    n = L.n_rows
    rp, ci, v = L.rowptr.numpy(), L.colind.numpy(), L.val.numpy()
    entries = {}
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            entries[(i, int(ci[k]))] = float(v[k])
    for j in range(1, n):
        entries[(0, j)] = entries.get((0, j), 0.0) - eps
        entries[(j, 0)] = entries.get((j, 0), 0.0) - eps
        entries[(j, j)] += eps
    entries[(0, 0)] += eps * (n - 1)
    keys = sorted(entries)
    r = np.array([k[0] for k in keys]); c = np.array([k[1] for k in keys])
    vals = np.array([entries[k] for k in keys])
    rpn = np.zeros(n + 1, np.int64)
    np.add.at(rpn, r + 1, 1)
    return synth.HostCSR(n, n, torch.from_numpy(np.cumsum(rpn).astype(np.int32)),
                         torch.from_numpy(c.astype(np.int32)), torch.from_numpy(vals), "lap_full_row")


@pytest.mark.parametrize("vt", [None, sp.VAL_BF16])
def test_cg_sliced_with_a_long_row_takes_the_unfused_path(vt):
    A = _laplacian_with_full_row()
    b = synth.uniform_vector(A.n_rows, 9)
    ch = sp.make_choice("sliced") if vt is None else sp.make_choice("sliced", value_type=vt,
                                                                     accumulate=sp.ACC_F64)
    dA = sp.DeviceCSR.from_host(A)
    assert sp.spmv_prepare(dA, ch).info().n_long_rows >= 1  # long-row segments present
    x, r = _run(A, b, 40, ch, refine=10 if vt else 0)
    low = None if vt is None else oracle.round_bf16(A.val)
    xo, ro = oracle.cg(A, b, np.zeros(A.n_rows), 40, vkind=0 if vt is None else 2, lowval=low,
                       refine=10 if vt else 0)
    _close(x, r, xo, ro)
