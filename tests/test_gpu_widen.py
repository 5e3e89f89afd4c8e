"""FP64 accumulation of FP32 / BF16 values (the compressed MB variants).

The kernels widen each stored value to FP64 with integer operations instead
of the FP64 conversion instruction.  These tests run one nonzero per row, so
each y_i is the single rounded product widen(v_i) * x_c, and compare it bit
for bit with the oracle's FP64-accumulate product (Table 2 compression read
as O20 with FP64 sums): every one of the 2^16 BF16 bit patterns (zeros,
subnormals, Inf and NaN included; NaN only needs to stay NaN), and FP32 edge
patterns plus random ones.
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


def _one_per_row(vals, n_cols=256):
    n = len(vals)
    return synth.HostCSR(n, n_cols, torch.arange(n + 1, dtype=torch.int32),
                         (torch.arange(n, dtype=torch.int32) % n_cols).contiguous(),
                         torch.from_numpy(np.ascontiguousarray(vals, dtype=np.float64)))


def _bf16_all():
    return (np.arange(1 << 16, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


def _f32_patterns():
    edges = np.array([0x00000000, 0x80000000, 0x00000001, 0x80000001, 0x00000002, 0x00400000,
                      0x007fffff, 0x807fffff, 0x00800000, 0x80800000, 0x00800001, 0x3f800000,
                      0xbf800000, 0x3f800001, 0x7f7fffff, 0xff7fffff, 0x7f800000, 0xff800000,
                      0x7fc00000, 0x7f800001, 0x33800000, 0x4b000000], dtype=np.uint32)
    g = np.random.default_rng(5)
    rnd = g.integers(0, 1 << 32, size=200_000, dtype=np.uint64).astype(np.uint32)
    sub = g.integers(1, 1 << 23, size=20_000, dtype=np.uint64).astype(np.uint32)  # subnormals
    sub |= (g.integers(0, 2, size=sub.size, dtype=np.uint64).astype(np.uint32) << 31)
    return np.concatenate([edges, rnd, sub]).view(np.float32).astype(np.float64)


def _check(vals, vt, choice):
    A = _one_per_row(vals)
    x = synth.uniform_vector(A.n_cols, 3)
    x[7] = 1.0
    x[8] = -0.0
    dA = sp.DeviceCSR.from_host(A)
    P = sp.spmv_prepare(dA, choice)
    assert P.info().accumulate == sp.ACC_F64
    y = torch.full((A.n_rows,), 12345.0, dtype=torch.float64, device="cuda")
    sp.spmv(P, x.cuda(), y)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    vkind = 1 if vt == sp.VAL_F32 else 2
    low = oracle.round_f32(A.val) if vt == sp.VAL_F32 else oracle.round_bf16(A.val)
    ref = oracle.spmv_lowp(A, x, vkind, low)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    bad = np.flatnonzero(got[~nan].view(np.uint64) != ref[~nan].view(np.uint64))
    assert bad.size == 0, (bad[:5], got[~nan][bad[:5]], ref[~nan][bad[:5]])
    P.free()


@pytest.mark.parametrize("variant", ["sliced", "compressed"])
def test_widen_every_bf16_pattern(variant):
    _check(_bf16_all(), sp.VAL_BF16,
           sp.make_choice(variant, value_type=sp.VAL_BF16, accumulate=sp.ACC_F64))


@pytest.mark.parametrize("variant", ["sliced", "compressed"])
def test_widen_fp32_edges_and_random_patterns(variant):
    _check(_f32_patterns(), sp.VAL_F32,
           sp.make_choice(variant, value_type=sp.VAL_F32, accumulate=sp.ACC_F64))
