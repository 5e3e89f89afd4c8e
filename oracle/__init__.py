"""CPU oracle for the SpMV optimization-selection method (arXiv 1511.02494).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the library under
``paper_1511_02494_gb300`` never does.  It shares no code with the CUDA path.

The arithmetic lives in ``oracle.c`` (plain sequential C, FP64, compiled with
``-ffp-contract=off``); this module only builds it with gcc, loads it with
ctypes and marshals numpy arrays.  Each wrapper names the passage of the paper
it follows.

Parity status per function (what pins it is in ``tests/test_oracle_pins.py``):
every function below is pinned.  The oracle holds no value measured on a GPU:
the profile rule's thresholds, which the paper never prints ("empirically
set", Section 3.2.1), and the class -> variant table are inputs of
``profile_class`` and ``class_variant`` (the latter defaults to the paper's
Table 2); the library's calibrated values are passed in by the tests.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (host architecture)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Features(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("n_rows", "n_cols", "nnz", "line_bytes", "l2_bytes",
                                         "working_set_bytes", "nnz_min", "nnz_max")] + \
        [(n, C.c_uint64) for n in ("nnz_sum", "nnz_sumsq_lo", "nnz_sumsq_hi")] + \
        [(n, C.c_int64) for n in ("bw_min", "bw_max")] + \
        [(n, C.c_uint64) for n in ("bw_sum", "bw_sumsq_lo", "bw_sumsq_hi", "disp_sum",
                                   "disp_sumsq_lo", "disp_sumsq_hi", "clust_sum",
                                   "ngroups_sum", "misses_sum")] + \
        [(n, C.c_double) for n in ("size", "density", "nnz_avg", "nnz_sd", "bw_avg", "bw_sd",
                                   "disp_avg", "disp_sd", "clustering", "miss_ratio")] + \
        [("vec", C.c_float * 16)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "vec"}
        for s in ("nnz_sumsq", "bw_sumsq", "disp_sumsq"):
            d[s] = (d.pop(s + "_hi") << 64) | d.pop(s + "_lo")
        d["vec"] = np.array(list(self.vec), dtype=np.float32)
        return d


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.c_void_p
            i64, i32 = C.c_int64, C.c_int32
            sig = {
                "orc_spmv": (None, [i64, P, P, P, P, P]),
                "orc_spmv_ref": (None, [i64, P, P, P, P, i64, P, P, P]),
                "orc_spmv_lowp": (None, [i64, P, P, i32, P, P, P]),
                "orc_spmv_lowp32": (None, [i64, P, P, i32, P, P, P]),
                "orc_round_bf16": (C.c_uint16, [C.c_double]),
                "orc_round_bf16_array": (None, [i64, P, P]),
                "orc_round_f32_array": (None, [i64, P, P]),
                "orc_features": (None, [i64, i64, P, P, i64, i64, C.POINTER(Features)]),
                "orc_profile_class": (i32, [C.c_double] * 6),
                "orc_class_variant": (i32, [i32, P]),
                "orc_static_partition": (None, [i64, P, i64, P]),
                "orc_dyn_tiers": (None, [i64, P, i32, i32, P, P, P, P, P]),
                "orc_sliced_segments": (i64, [i64, P, i32, i32, P, P, P, P, P, P, P]),
                "orc_row_blocks": (None, [i64, P, i64, i64, P]),
                "orc_merge_path": (None, [i64, P, i64, i64, P, P]),
                "orc_compress_u16": (i64, [i64, P, P, P, P]),
                "orc_mlp_forward_f32": (None, [i32, i32, i32] + [P] * 10),
                "orc_argmax": (i32, [i32, P, P]),
                "orc_mlp_loss_grad_f64": (C.c_double, [i32, i32, i32, i32] + [P] * 14),
                "orc_mlp_loss_grad_soft_f64": (C.c_double, [i32, i32, i32, i32] + [P] * 14),
                "orc_sliced_layout": (i64, [i64, P, i32, i32, i32, P, P, P, P]),
                "orc_sliced_fill": (None, [i64, P, P, P, P, P, P, i32, P, P]),
                "orc_sliced_offsets": (i64, [i64, P, P, P, P, P, i32, P, P]),
                "orc_sliced_diag": (i64, [i64, P, P, P, P, P, P]),
                "orc_sliced_index_bytes": (i32, [i64]),
                "orc_sliced_delta": (i64, [i64, P, P, P, P, P, P, P]),
                "orc_delta_bytes": (i32, [i64]),
                "orc_sliced_panel": (i64, [i64, P, P, P, P, P, P, P]),
                "orc_cg": (None, [i64, P, P, P, i32, P, i32, P, P, i32, P, P, P, P]),
                "orc_adam_f32": (None, [i64, P, P, P, P] + [C.c_float] * 7),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _np(a, dtype):
    """Contiguous numpy view/copy of a torch tensor or array."""
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _csr(A):
    return (_np(A.rowptr, np.int32), _np(A.colind, np.int32), _np(A.val, np.float64))


def spmv(A, x) -> np.ndarray:
    """Algorithm 1 (Section 2), sequential FP64: y = A x."""
    rp, ci, v = _csr(A)
    x = _np(x, np.float64)
    y = np.empty(A.n_rows, np.float64)
    _load().orc_spmv(A.n_rows, _p(rp), _p(ci), _p(v), _p(x), _p(y))
    return y


def spmv_ref(A, x, rows=None):
    """Compensated y and the per-row scale sum_j |a_ij x_j| (Algorithm 1),
    for all rows or the listed ones."""
    rp, ci, v = _csr(A)
    x = _np(x, np.float64)
    if rows is None:
        n, r = A.n_rows, None
    else:
        r = _np(rows, np.int64)
        n = r.size
    y = np.empty(n, np.float64)
    s = np.empty(n, np.float64)
    _load().orc_spmv_ref(A.n_rows, _p(rp), _p(ci), _p(v), _p(x), n,
                         _p(r) if r is not None else None, _p(y), _p(s))
    return y, s


def spmv_lowp(A, x, vkind: int, lowval) -> np.ndarray:
    """y = A x with float32 (vkind=1) or bfloat16-bit (vkind=2) stored values,
    FP64 accumulation (compressed-value MB variant, Section 3.3)."""
    rp, ci, _ = _csr(A)
    x = _np(x, np.float64)
    lv = _np(lowval, np.float32 if vkind == 1 else np.uint16)
    y = np.empty(A.n_rows, np.float64)
    _load().orc_spmv_lowp(A.n_rows, _p(rp), _p(ci), vkind, _p(lv), _p(x), _p(y))
    return y


def spmv_lowp32(A, x, vkind: int, lowval) -> np.ndarray:
    """y = A x in FP32 arithmetic: float32 (vkind=1) or bfloat16-bit
    (vkind=2) values, x rounded to float, fmaf accumulation per row."""
    rp, ci, _ = _csr(A)
    x = _np(x, np.float64)
    lv = _np(lowval, np.float32 if vkind == 1 else np.uint16)
    y = np.empty(A.n_rows, np.float64)
    _load().orc_spmv_lowp32(A.n_rows, _p(rp), _p(ci), vkind, _p(lv), _p(x), _p(y))
    return y


def round_bf16(v) -> np.ndarray:
    """Round-to-nearest-even double -> bfloat16 bit patterns (uint16)."""
    v = _np(v, np.float64).reshape(-1)
    out = np.empty(v.size, np.uint16)
    _load().orc_round_bf16_array(v.size, _p(v), _p(out))
    return out


def round_f32(v) -> np.ndarray:
    v = _np(v, np.float64).reshape(-1)
    out = np.empty(v.size, np.float32)
    _load().orc_round_f32_array(v.size, _p(v), _p(out))
    return out


def features(A, line_bytes: int = 128, l2_bytes: int = 0) -> dict:
    """Table 1 (Section 3.2.2) features with the exact integer aggregates."""
    rp, ci, _ = _csr(A)
    f = Features()
    _load().orc_features(A.n_rows, A.n_cols, _p(rp), _p(ci), line_bytes, l2_bytes, C.byref(f))
    return f.as_dict()


CML, MB, IMB, CMP = 0, 1, 2, 3


# Table 2 (Section 3.3), class -> optimization, in the library's variant ids:
# CML -> latency (software prefetch), MB -> compressed (delta-coded indices),
# IMB -> dynamic (dynamic schedule), CMP -> sub-warp (unrolled, vectorised rows)
TABLE2 = (5, 6, 4, 1)


def profile_class(s_noxmiss, s_inflate, s_balance, tau) -> int:
    """Section 3.2.1 profiling-based classification rule (readings O9-O12).
    tau = (tau_noxmiss, tau_inflate, tau_balance) must be given: the paper
    sets its thresholds empirically and prints none."""
    t = tuple(float(v) for v in tau)
    if len(t) != 3:
        raise ValueError("tau needs three thresholds")
    return int(_load().orc_profile_class(s_noxmiss, s_inflate, s_balance, *t))


def class_variant(cls: int, table=None) -> int:
    """Variant serving a class: table[cls] (4 variant ids, indexed by class),
    or the paper's Table 2 (TABLE2) when table is None."""
    if table is None:
        return int(_load().orc_class_variant(cls, None))
    m = np.ascontiguousarray(np.asarray(table, dtype=np.int32).reshape(4))
    return int(_load().orc_class_variant(cls, _p(m)))


def static_partition(A, n_workers: int) -> np.ndarray:
    """Section 3.2.1 default partition: equal-nonzero contiguous row ranges."""
    rp = _np(A.rowptr, np.int32)
    out = np.empty(n_workers + 1, np.int64)
    _load().orc_static_partition(A.n_rows, _p(rp), n_workers, _p(out))
    return out


def dyn_tiers(A, lim_s: int, seg: int):
    """Tiers of the dynamic-schedule variant (Table 2, IMB): the rows with
    lim_s < len <= 64, with 64 < len <= seg, with len > seg (ascending), and
    the segment count of each long row."""
    rp = _np(A.rowptr, np.int32)
    n = max(A.n_rows, 1)
    m1, m2, lr, sc = (np.empty(n, np.int32) for _ in range(4))
    cnt = np.zeros(3, np.int64)
    _load().orc_dyn_tiers(A.n_rows, _p(rp), lim_s, seg, _p(m1), _p(m2), _p(lr), _p(sc), _p(cnt))
    a, b, c = (int(v) for v in cnt)
    return m1[:a], m2[:b], lr[:c], sc[:c]


def sliced_segments(A, cap: int, seg: int = 2048):
    """Long rows of the sliced layout and their segment table: list, seg_off,
    seg_be (n_seg x 2), seg_row, fix, seg_fix."""
    rp = _np(A.rowptr, np.int32)
    lens = np.diff(rp.astype(np.int64))
    n_long = int((lens > cap).sum())
    n_seg_max = int(((lens[lens > cap] + seg - 1) // seg).sum())
    lst = np.empty(max(n_long, 1), np.int32)
    off = np.empty(n_long + 1, np.int32)
    be = np.empty(max(2 * n_seg_max, 2), np.int64)
    srow = np.empty(max(n_seg_max, 1), np.int32)
    fix = np.empty(max(n_long, 1), np.int32)
    sfix = np.empty(max(n_seg_max, 1), np.int32)
    nf = C.c_int64()
    ns = int(_load().orc_sliced_segments(A.n_rows, _p(rp), cap, seg, _p(lst), _p(off), _p(be), _p(srow),
                                         _p(fix), _p(sfix), C.byref(nf)))
    return (lst[:n_long], off, be[:2 * ns].reshape(ns, 2), srow[:ns], fix[:nf.value], sfix[:ns])


def row_blocks(A, block_nnz: int) -> np.ndarray:
    rp = _np(A.rowptr, np.int32)
    nb = max(1, -(-A.nnz // block_nnz))
    out = np.empty(nb + 1, np.int32)
    _load().orc_row_blocks(A.n_rows, _p(rp), block_nnz, nb, _p(out))
    return out


def merge_path(A, items: int):
    """Merge-path start coordinates (row, nonzero) of every part."""
    rp = _np(A.rowptr, np.int32)
    total = A.n_rows + A.nnz
    parts = max(1, -(-total // items))
    rs = np.empty(parts + 1, np.int32)
    ns = np.empty(parts + 1, np.int32)
    _load().orc_merge_path(A.n_rows, _p(rp), items, parts, _p(rs), _p(ns))
    return rs, ns


def compress_u16(A):
    """16-bit column offsets from each row's first column (reading O13)."""
    rp, ci, _ = _csr(A)
    base = np.empty(A.n_rows, np.int32)
    off = np.empty(A.nnz, np.uint16)
    wide = _load().orc_compress_u16(A.n_rows, _p(rp), _p(ci), _p(base), _p(off))
    return base, off, int(wide)


def sliced_layout(A, sigma: int, cap: int, vec: int = 1):
    """Sliced layout (32 rows per slice, column-major inside a slice): the
    position -> row permutation, per-position row length (-1: long row or
    past the end), slice lengths and slice starts, and the long-row count."""
    rp, _, _ = _csr(A)
    S = (A.n_rows + 31) // 32
    perm = np.empty(max(A.n_rows, 1), np.int32)
    rowlen = np.empty(max(32 * S, 1), np.int32)
    slen = np.empty(max(S, 1), np.int32)
    sptr = np.empty(S + 1, np.int64)
    n_long = _load().orc_sliced_layout(A.n_rows, _p(rp), sigma, cap, vec, _p(perm), _p(rowlen),
                                       _p(slen), _p(sptr))
    return perm[:A.n_rows], rowlen[:32 * S], slen[:S], sptr, int(n_long)


def sliced_fill(A, perm, rowlen, sptr, vec: int = 1):
    """Column-major slice contents (columns and values, zero padding)."""
    rp, ci, va = _csr(A)
    tot = int(sptr[-1])
    col = np.empty(max(tot, 1), np.int32)
    val = np.empty(max(tot, 1), np.float64)
    perm = _np(perm, np.int32)
    rowlen = _np(rowlen, np.int32)
    sptr = _np(sptr, np.int64)
    _load().orc_sliced_fill(A.n_rows, _p(rp), _p(ci), _p(va), _p(perm), _p(rowlen), _p(sptr),
                            vec, _p(col), _p(val))
    return col[:tot], val[:tot]


def sliced_offsets(A, perm, rowlen, sptr, vec: int = 1):
    """16-bit offsets of the sliced layout: per-position row base (first
    column) and col - base per slot; returns (rowbase, off, largest span)."""
    rp, ci, _ = _csr(A)
    S = (A.n_rows + 31) // 32
    tot = int(sptr[-1])
    base = np.empty(max(32 * S, 1), np.int32)
    off = np.empty(max(tot, 1), np.uint16)
    perm = _np(perm, np.int32)
    rowlen = _np(rowlen, np.int32)
    sptr = _np(sptr, np.int64)
    span = _load().orc_sliced_offsets(A.n_rows, _p(rp), _p(ci), _p(perm), _p(rowlen), _p(sptr),
                                      vec, _p(base), _p(off))
    return base[:32 * S], off[:tot], int(span)


def sliced_diag(A, perm, rowlen, sptr):
    """Offsets column - row of the FP64 sliced layout (0 in padding), the
    largest |offset| over the rows in the slices, and the bytes per stored
    index that largest offset allows (1, 2 or 4)."""
    rp, ci, _ = _csr(A)
    tot = int(sptr[-1])
    d = np.empty(max(tot, 1), np.int32)
    perm = _np(perm, np.int32)
    rowlen = _np(rowlen, np.int32)
    sptr = _np(sptr, np.int64)
    reach = int(_load().orc_sliced_diag(A.n_rows, _p(rp), _p(ci), _p(perm), _p(rowlen), _p(sptr), _p(d)))
    return d[:tot], reach, int(_load().orc_sliced_index_bytes(reach))


def sliced_delta(A, perm, rowlen, sptr):
    """Table 2's delta coding on the FP64 sliced layout (reading O24): the
    per-position row base (first column), the delta from the previous column
    at each slot (0 for first elements and padding), the largest delta, and
    the bytes per delta that largest delta allows (1, 2, or 0 = none)."""
    rp, ci, _ = _csr(A)
    S = (A.n_rows + 31) // 32
    tot = int(sptr[-1])
    base = np.empty(max(32 * S, 1), np.int32)
    d = np.empty(max(tot, 1), np.int32)
    perm = _np(perm, np.int32)
    rowlen = _np(rowlen, np.int32)
    sptr = _np(sptr, np.int64)
    big = int(_load().orc_sliced_delta(A.n_rows, _p(rp), _p(ci), _p(perm), _p(rowlen), _p(sptr),
                                       _p(base), _p(d)))
    return base[:32 * S], d[:tot], big, int(_load().orc_delta_bytes(big))


def delta_bytes(largest: int) -> int:
    return int(_load().orc_delta_bytes(int(largest)))


def sliced_panel(A, perm, rowlen, sptr):
    """Column-blocked form of the FP64 sliced layout (reading O25): the
    offset inside each element's 65536-column panel, the panel step from the
    previous element, and the largest step (the form needs it <= 255)."""
    rp, ci, _ = _csr(A)
    tot = int(sptr[-1])
    lo = np.empty(max(tot, 1), np.uint16)
    st = np.empty(max(tot, 1), np.int32)
    perm = _np(perm, np.int32)
    rowlen = _np(rowlen, np.int32)
    sptr = _np(sptr, np.int64)
    big = int(_load().orc_sliced_panel(A.n_rows, _p(rp), _p(ci), _p(perm), _p(rowlen), _p(sptr),
                                       _p(lo), _p(st)))
    return lo[:tot], st[:tot], big


def sliced_index_bytes(reach: int) -> int:
    return int(_load().orc_sliced_index_bytes(int(reach)))


def mlp_forward_f32(params: dict, v) -> np.ndarray:
    """Fixed-order fmaf forward of the 16-H1-H2-K selector network."""
    W1 = _np(params["W1"], np.float32); W2 = _np(params["W2"], np.float32)
    W3 = _np(params["W3"], np.float32)
    h1, h2, k = W1.shape[0], W2.shape[0], W3.shape[0]
    v = _np(v, np.float32).reshape(-1, 16)
    out = np.empty((v.shape[0], k), np.float32)
    args = [_np(params[n], np.float32) for n in ("mean", "istd", "W1", "b1", "W2", "b2", "W3", "b3")]
    for s in range(v.shape[0]):
        row = np.ascontiguousarray(v[s])
        res = np.empty(k, np.float32)
        _load().orc_mlp_forward_f32(h1, h2, k, *[_p(a) for a in args], _p(row), _p(res))
        out[s] = res
    return out


def argmax(logits) -> tuple[int, float]:
    lg = _np(logits, np.float32)
    m = C.c_float()
    b = _load().orc_argmax(lg.size, _p(lg), C.byref(m))
    return int(b), float(m.value)


def mlp_loss_grad_f64(params: dict, z, labels):
    """FP64 mean softmax cross-entropy and its gradients (backpropagation)."""
    P64 = {n: _np(params[n], np.float64) for n in ("W1", "b1", "W2", "b2", "W3", "b3")}
    h1, h2, k = P64["W1"].shape[0], P64["W2"].shape[0], P64["W3"].shape[0]
    z = _np(z, np.float64).reshape(-1, 16)
    lab = _np(labels, np.int32)
    G = {n: np.empty_like(a) for n, a in P64.items()}
    loss = _load().orc_mlp_loss_grad_f64(
        h1, h2, k, z.shape[0], *[_p(P64[n]) for n in ("W1", "b1", "W2", "b2", "W3", "b3")],
        _p(z), _p(lab), *[_p(G[n]) for n in ("W1", "b1", "W2", "b2", "W3", "b3")])
    return float(loss), G


def mlp_loss_grad_soft_f64(params: dict, z, q):
    """FP64 mean cross-entropy against per-sample target distributions
    q (batch x K) and its gradients."""
    P64 = {n: _np(params[n], np.float64) for n in ("W1", "b1", "W2", "b2", "W3", "b3")}
    h1, h2, k = P64["W1"].shape[0], P64["W2"].shape[0], P64["W3"].shape[0]
    z = _np(z, np.float64).reshape(-1, 16)
    q = _np(q, np.float64).reshape(z.shape[0], k)
    G = {n: np.empty_like(a) for n, a in P64.items()}
    loss = _load().orc_mlp_loss_grad_soft_f64(
        h1, h2, k, z.shape[0], *[_p(P64[n]) for n in ("W1", "b1", "W2", "b2", "W3", "b3")],
        _p(z), _p(q), *[_p(G[n]) for n in ("W1", "b1", "W2", "b2", "W3", "b3")])
    return float(loss), G


def adam_f32(p, g, m, v, lr, b1, b2, eps, wd, c1, c2):
    """One float Adam step (operations rounded as written); returns new
    (p, m, v)."""
    p = _np(p, np.float32).copy(); m = _np(m, np.float32).copy(); v = _np(v, np.float32).copy()
    g = _np(g, np.float32)
    _load().orc_adam_f32(p.size, _p(p), _p(g), _p(m), _p(v), lr, b1, b2, eps, wd, c1, c2)
    return p, m, v


def cg(A, b, x0, iters: int, vkind: int = 0, lowval=None, refine: int = 0):
    """Conjugate gradients in FP64 (optionally low-precision inner SpMV with
    FP64 residual recomputation every `refine` iterations)."""
    rp, ci, v = _csr(A)
    n = A.n_rows
    bb = _np(b, np.float64)
    x = _np(x0, np.float64).copy()
    lv = None
    if vkind:
        lv = _np(lowval, np.float32 if vkind == 1 else np.uint16)
    resid = np.empty(iters + 1, np.float64)
    r, p, q = (np.empty(n, np.float64) for _ in range(3))
    _load().orc_cg(n, _p(rp), _p(ci), _p(v), vkind, _p(lv) if lv is not None else None,
                   refine, _p(bb), _p(x), iters, _p(resid), _p(r), _p(p), _p(q))
    return x, resid
