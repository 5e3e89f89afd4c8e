"""Batched persistent SpMV against the oracle, plain and graph launches,
before and after autotuning."""
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
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def batch_case():
    mats = synth.batch_matrices(48, seed=1, lo=1e3, hi=2e4)
    mats.append(synth.random_csr(0, 5, 2))          # an empty matrix
    mats.append(synth.random_csr(700, 300, 0, seed=2))  # rows all empty
    dev = [sp.DeviceCSR.from_host(A) for A in mats]
    xs = [synth.uniform_vector(A.n_cols, 10 + i).cuda() for i, A in enumerate(mats)]
    ys = [torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda") for A in mats]
    return mats, dev, xs, ys


def _check(mats, xs, ys):
    for A, x, y in zip(mats, xs, ys):
        ref, scale = oracle.spmv_ref(A, x.cpu())
        got = y.cpu().numpy()
        assert np.all(np.abs(got - ref) <= RTOL * scale), A.name
        assert np.all(got[scale == 0] == 0.0)


def test_batch_matches_oracle_plain_graph_and_autotuned(batch_case):
    mats, dev, xs, ys = batch_case
    B = sp.spmv_batch_create(dev)
    sp.spmv_batch_bind(B, xs, ys)
    sp.spmv_batch_run(B)
    torch.cuda.synchronize()
    _check(mats, xs, ys)
    for y in ys:
        y.fill_(float("nan"))
    for _ in range(3):
        sp.spmv_batch_run(B, use_graph=True)
    torch.cuda.synchronize()
    _check(mats, xs, ys)
    first = [y.clone() for y in ys]
    sp.spmv_batch_autotune(B, reps=2)
    t, r = sp.spmv_batch_config(B)
    assert set(t.tolist()) <= {1, 2, 4, 8, 16, 32}
    passes = r // (32 // t)
    assert np.all(r == passes * (32 // t))
    assert set(passes.tolist()) <= {2, 4, 8, 16, 32}
    for y in ys:
        y.fill_(float("nan"))
    sp.spmv_batch_run(B, use_graph=True)
    torch.cuda.synchronize()
    _check(mats, xs, ys)
    B.free()


def test_batch_explicit_shapes(batch_case):
    mats, dev, xs, ys = batch_case
    n = len(mats)
    for T in (1, 4, 32):
        B = sp.spmv_batch_create(dev, threads_per_row=[T] * n, rows_per_item=[37] * n)
        sp.spmv_batch_bind(B, xs, ys)
        for y in ys:
            y.fill_(float("nan"))
        sp.spmv_batch_run(B)
        torch.cuda.synchronize()
        _check(mats, xs, ys)
        B.free()
    with pytest.raises(sp.SpmvError):
        sp.spmv_batch_create(dev, threads_per_row=[3] * n)


def test_batch_of_prepared_matrices(batch_case):
    """Each matrix in the persistent form of its own variant (SLICED as its
    slices; MERGE, DYNAMIC and BF16 SLICED as a sliced form the batch
    prepares; the others as CSR rows), and every matrix in the sliced layout
    (spmv_batch_create_sliced)."""
    mats, dev, xs, ys = batch_case
    extra = [synth.zipf_rows(20_000, 20_000, 1.4, 5_000, seed=11), synth.stencil_27pt(12, seed=2)]
    mats = list(mats) + extra
    dev = list(dev) + [sp.DeviceCSR.from_host(A) for A in extra]
    xs = list(xs) + [synth.uniform_vector(A.n_cols, 77 + i).cuda() for i, A in enumerate(extra)]
    ys = [torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda") for A in mats]
    kinds = ["sliced", "subwarp", "dynamic", ("sliced", 256), "latency", "compressed",
             ("sliced", 0, 1), ("sliced", 0, 0, sp.VAL_BF16)]
    preps = []
    for i, dA in enumerate(dev):
        k = kinds[i % len(kinds)]
        if isinstance(k, tuple):
            k = tuple(k) + (0, 0, 0)[len(k) - 1:]
            ch = sp.make_choice(k[0], block_nnz=k[1], index_bytes=k[2], value_type=k[3] or sp.VAL_F64)
        else:
            ch = sp.make_choice(k)
        preps.append(sp.spmv_prepare(dA, ch))
    # a SLICED matrix with 8- or 16-bit column offsets, and one with BF16
    # values (run by the batch in its FP64 form)
    assert any(P.info().index_bytes < 4 for P in preps)
    assert any(P.info().value_type == sp.VAL_BF16 for P in preps)
    for create in (sp.spmv_batch_create_prepared, sp.spmv_batch_create_sliced):
        B = create(preps)
        sp.spmv_batch_bind(B, xs, ys)
        sp.spmv_batch_run(B)
        torch.cuda.synchronize()
        _check(mats, xs, ys)
        for y in ys:
            y.fill_(float("nan"))
        sp.spmv_batch_run(B, use_graph=True)
        torch.cuda.synchronize()
        _check(mats, xs, ys)
        sp.spmv_batch_autotune(B, reps=2)
        t, r = sp.spmv_batch_config(B)
        # sliced matrices (all of them in the sliced batch) take one lane a row
        sl = [i for i, P in enumerate(preps)
              if create is sp.spmv_batch_create_sliced or
              P.info().variant in (sp.VARIANT_IDS["sliced"], sp.VARIANT_IDS["dynamic"])]
        assert sl and all(t[i] == 1 and r[i] % 32 == 0 for i in sl)
        for y in ys:
            y.fill_(float("nan"))
        sp.spmv_batch_run(B, use_graph=True)
        torch.cuda.synchronize()
        _check(mats, xs, ys)
        B.free()


@pytest.mark.parametrize("form", ["prepared", "sliced"])
def test_batch_with_rows_of_many_segments(form):
    # a row of 120,000 nonzeros (59 segments) and other long rows beside
    # small matrices: one work item per segment, each row of several
    # segments summed by the warp that finishes its last one; integer values
    # give exact sums, and repeated runs (tickets back at 0) the same bits,
    # equal to the single-matrix SLICED kernel's
    g = np.random.default_rng(4)
    Z = synth.zipf_rows(30_000, 200_000, 1.3, 120_000, seed=5)
    Z.val = torch.from_numpy(g.integers(-3, 4, Z.nnz).astype(np.float64))
    mats = [Z, synth.laplacian_2d_5pt(40, 40), synth.zipf_rows(5000, 5000, 1.5, 4000, seed=6)]
    dev = [sp.DeviceCSR.from_host(A) for A in mats]
    preps = [sp.spmv_prepare(dev[0], sp.make_choice("sliced", block_nnz=4096, items_per_warp=32)),
             sp.spmv_prepare(dev[1], sp.make_choice("subwarp")),
             sp.spmv_prepare(dev[2], sp.make_choice("sliced"))]
    assert preps[0].info().n_long_rows > 0
    xs = [torch.from_numpy(g.integers(-2, 3, mats[0].n_cols).astype(np.float64)).cuda()] + \
        [synth.uniform_vector(A.n_cols, 3 + i).cuda() for i, A in enumerate(mats[1:])]
    ys = [torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda") for A in mats]
    B = sp.spmv_batch_create_prepared(preps) if form == "prepared" else sp.spmv_batch_create_sliced(preps)
    sp.spmv_batch_bind(B, xs, ys)
    y_single = torch.empty_like(ys[0])
    sp.spmv(preps[0], xs[0], y_single)
    for use_graph in (False, False, True, True):
        for y in ys:
            y.fill_(float("nan"))
        sp.spmv_batch_run(B, use_graph=use_graph)
        torch.cuda.synchronize()
        assert np.array_equal(ys[0].cpu().numpy(), oracle.spmv(mats[0], xs[0].cpu()))
        assert torch.equal(ys[0], y_single)
        _check(mats, xs, ys)
    B.free()
    for P in preps:
        P.free()
