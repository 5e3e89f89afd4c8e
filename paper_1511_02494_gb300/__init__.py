"""GB300 SpMV optimization selection (arXiv 1511.02494) -- Python binding.

A thin ctypes layer over the C ABI of ``include/spmv.h`` (library
``libspmv_gb300.so``, built by :mod:`paper_1511_02494_gb300.build`).  The
functions keep the C names; they only marshal arguments: every step of the
computation runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  There is no CPU fallback: if the library is not built or
no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from ._abi import (  # noqa: F401  (re-exported)
    Choice, CSR, Features, PreparedInfo, Profile, Thresholds,
    SPMV_OK, STATUS_NAMES, VARIANTS, VARIANT_IDS, CLASSES, VAL_F64, VAL_F32, VAL_BF16,
    EXPORT_ROW_BLOCKS, EXPORT_MERGE_ROWS, EXPORT_MERGE_NZ, EXPORT_ROWBASE, EXPORT_OFFSETS,
    EXPORT_VALUES, EXPORT_SLICE_PERM, EXPORT_SLICE_ROWLEN, EXPORT_SLICE_LEN, EXPORT_SLICE_PTR,
    EXPORT_SLICE_COL, EXPORT_SLICE_VAL, EXPORT_SLICE_OFF16, EXPORT_SLICE_ROWBASE, EXPORT_SLICE_DIAG,
    EXPORT_SLICE_DELTA, EXPORT_SLICE_PANEL_LO, EXPORT_SLICE_PANEL_STEP,
    EXPORT_DYN_M1, EXPORT_DYN_M2, EXPORT_DYN_LONG, EXPORT_DYN_SEG_OFF, EXPORT_SLICE_LONG,
    EXPORT_SLICE_SEG_OFF, EXPORT_SLICE_SEG_BOUNDS, EXPORT_SLICE_SEG_ROW, EXPORT_SLICE_FIX,
    EXPORT_SLICE_SEG_FIX,
    declare,
)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspmv_gb300.so")
_lock = threading.Lock()
_lib = None


class SpmvError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"CUDA library {LIB_PATH} is not built; run "
                    "`python -m paper_1511_02494_gb300.build` (needs nvcc)")
            _lib = declare(C.CDLL(LIB_PATH))
    return _lib


def _check(status: int):
    if status != SPMV_OK:
        msg = lib().spmv_last_error()
        raise SpmvError(status, msg.decode() if msg else "")


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


class DeviceCSR:
    """A CSR matrix on the GPU (torch tensors) plus its ABI descriptor."""

    def __init__(self, n_rows, n_cols, rowptr, colind, val):
        import torch
        for t, dt in ((rowptr, torch.int32), (colind, torch.int32), (val, torch.float64)):
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                raise ValueError("DeviceCSR needs contiguous CUDA int32/int32/float64 tensors")
        self.n_rows, self.n_cols = int(n_rows), int(n_cols)
        self.rowptr, self.colind, self.val = rowptr, colind, val
        self.desc = CSR(self.n_rows, self.n_cols, int(colind.numel()),
                        _ptr(rowptr), _ptr(colind), _ptr(val))

    @property
    def nnz(self):
        return int(self.colind.numel())

    @classmethod
    def from_host(cls, A, device="cuda"):
        """From any object with n_rows, n_cols, rowptr, colind, val tensors."""
        return cls(A.n_rows, A.n_cols, A.rowptr.to(device).contiguous(),
                   A.colind.to(device).contiguous(), A.val.to(device).contiguous())


def _desc(A):
    return A.desc if isinstance(A, DeviceCSR) else DeviceCSR.from_host(A).desc


def spmv_status_str(status: int) -> str:
    return lib().spmv_status_str(status).decode()


def spmv_last_error() -> str:
    return lib().spmv_last_error().decode()


def spmv_validate(A: DeviceCSR, stream=None) -> None:
    """Raises SpmvError(SPMV_ERR_INVALID_CSR) when A breaks a CSR rule."""
    _check(lib().spmv_validate(C.byref(A.desc), _stream(stream)))


def spmv_features(A: DeviceCSR, line_bytes: int = 128, stream=None) -> Features:
    """Table 1 structural features (Section 3.2.2) computed on the GPU."""
    out = Features()
    _check(lib().spmv_features(C.byref(A.desc), line_bytes, C.byref(out), _stream(stream)))
    return out


def spmv_profile(A: DeviceCSR, x, reps: int = 5, stream=None) -> Profile:
    """Profiling runs of Section 3.2.1 (baseline, noxmiss, inflate, balance)."""
    out = Profile()
    _check(lib().spmv_profile(C.byref(A.desc), _ptr(x), reps, C.byref(out), _stream(stream)))
    return out


def spmv_profile_outputs(A: DeviceCSR, x, n_workers: int, bounds=None, y_base=None,
                         y_noxmiss=None, y_inflate=None, y_balance=None, stream=None) -> None:
    """What the profiling runs compute: the static partition (int64 CUDA
    tensor [n_workers + 1]) and one product per probe (float64 CUDA tensors
    [n_rows]); any may be None.  n_workers 0 = spmv_profile's count."""
    _check(lib().spmv_profile_outputs(C.byref(A.desc), _ptr(x), int(n_workers), _ptr(bounds),
                                      _ptr(y_base), _ptr(y_noxmiss), _ptr(y_inflate),
                                      _ptr(y_balance), _stream(stream)))


def spmv_wait_check(limit_ns: int, arrive: bool, stream=None) -> None:
    """Bounded-wait self-test; raises SpmvError (TIMEOUT) when nothing arrives."""
    _check(lib().spmv_wait_check(int(limit_ns), 1 if arrive else 0, _stream(stream)))


def spmv_fixup_check(kind: int, carry_row, carry_val, status, y, stream=None) -> None:
    """Carry fix-up self-test (kind 0 STREAM, 1 MERGE) on device tensors:
    carry_row int32 [n_parts], carry_val float64 [n_parts], status int32 [1],
    y float64 [n_rows] (updated in place)."""
    _check(lib().spmv_fixup_check(int(kind), int(carry_row.numel()), int(y.numel()),
                                  _ptr(carry_row), _ptr(carry_val), _ptr(status), _ptr(y),
                                  _stream(stream)))


def spmv_gather_probe(A: DeviceCSR, x, out, stream=None) -> None:
    """out (device, one int64 / uint64) = sum modulo 2^64 of the bit patterns
    of x over A's column indices; its time is the cost of A's gathers of x
    alone."""
    _check(lib().spmv_gather_probe(C.byref(A.desc), _ptr(x), _ptr(out), _stream(stream)))


def spmv_default_thresholds() -> Thresholds:
    return lib().spmv_default_thresholds()


def spmv_classify_profile(profile: Profile, thresholds: Thresholds | None = None) -> int:
    cls = C.c_int32()
    _check(lib().spmv_classify_profile(C.byref(profile),
                                       C.byref(thresholds) if thresholds else None, C.byref(cls)))
    return cls.value


def spmv_class_variant(cls: int) -> int:
    return int(lib().spmv_class_variant(cls))


def spmv_class_choice(cls: int) -> Choice:
    """The class's calibrated choice (variant and launch configuration)."""
    out = Choice()
    _check(lib().spmv_class_choice(int(cls), C.byref(out)))
    return out


def spmv_select(features: Features | None = None, profile: Profile | None = None,
                thresholds: Thresholds | None = None) -> Choice:
    out = Choice()
    _check(lib().spmv_select(C.byref(features) if features else None,
                             C.byref(profile) if profile else None,
                             C.byref(thresholds) if thresholds else None, C.byref(out)))
    return out


ACC_DEFAULT, ACC_F64, ACC_F32 = 0, 1, 2


def make_choice(variant, threads_per_row=0, block_nnz=0, items_per_warp=0,
                value_type=VAL_F64, accumulate=ACC_DEFAULT, index_bytes=0, index_coding=0) -> Choice:
    v = VARIANT_IDS[variant] if isinstance(variant, str) else int(variant)
    c = Choice()
    c.variant, c.cls = v, -1
    c.threads_per_row, c.block_nnz, c.items_per_warp = threads_per_row, block_nnz, items_per_warp
    c.value_type = value_type
    c.accumulate = accumulate
    c.index_bytes = index_bytes
    c.index_coding = index_coding
    return c


class Prepared:
    """Owner of an spmv_prepared_t; keeps the matrix tensors alive."""

    def __init__(self, handle, A: DeviceCSR):
        self.handle, self.A = handle, A

    def info(self) -> PreparedInfo:
        return spmv_prepared_info(self)

    def free(self):
        if self.handle:
            lib().spmv_prepared_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def spmv_prepare(A: DeviceCSR, choice: Choice, trusted: bool = False, stream=None) -> Prepared:
    h = C.c_void_p()
    _check(lib().spmv_prepare(C.byref(A.desc), C.byref(choice), int(trusted), C.byref(h),
                              _stream(stream)))
    return Prepared(h, A)


def spmv(P: Prepared, x, y, stream=None) -> None:
    """y = A x on the GPU (asynchronous on the stream)."""
    _check(lib().spmv(P.handle, _ptr(x), _ptr(y), _stream(stream)))


def spmv_host(P: Prepared, x_host, y_host, stream=None) -> None:
    """y_host = A x_host with host (ideally pinned) float64 tensors."""
    _check(lib().spmv_host(P.handle, _ptr(x_host), _ptr(y_host), _stream(stream)))


def spmv_host_async(P: Prepared, x_host, y_host, stream=None) -> None:
    """As spmv_host, enqueued on `stream` without waiting: y_host is valid
    after the stream is synchronised (pinned tensors for overlap)."""
    _check(lib().spmv_host_async(P.handle, _ptr(x_host), _ptr(y_host), _stream(stream)))


def spmv_prepared_info(P: Prepared) -> PreparedInfo:
    out = PreparedInfo()
    _check(lib().spmv_prepared_info(P.handle, C.byref(out)))
    return out


def spmv_prepared_export(P: Prepared, which: int, out_tensor, stream=None) -> None:
    """Copies an owned array of P into a host tensor of exactly its size."""
    nbytes = out_tensor.numel() * out_tensor.element_size()
    _check(lib().spmv_prepared_export(P.handle, which, _ptr(out_tensor), nbytes, _stream(stream)))


def spmv_prepared_status(P: Prepared, stream=None) -> None:
    """Raises SpmvError(SPMV_ERR_TIMEOUT) if a bounded device wait of an
    earlier spmv on P gave up."""
    _check(lib().spmv_prepared_status(P.handle, _stream(stream)))


def spmv_stream_noalloc(A: DeviceCSR, x, y, stream=None) -> None:
    """y = A x with the pipelined STREAM kernel and no device allocation
    (scratch in a fixed static device array; see include/spmv.h)."""
    _check(lib().spmv_stream_noalloc(C.byref(A.desc), _ptr(x), _ptr(y), _stream(stream)))


def spmv_stream_noalloc_status(stream=None) -> None:
    """Raises SpmvError (TIMEOUT) when the last spmv_stream_noalloc call on
    this device gave up a bounded wait; synchronizes the stream."""
    _check(lib().spmv_stream_noalloc_status(_stream(stream)))


def spmv_cg(A_inner: Prepared, b, x, iters: int, refine_every: int = 0,
            A_exact: Prepared | None = None, resid=None, use_graph: bool = False,
            stream=None) -> None:
    """Conjugate gradients on the device (x holds x0 on entry)."""
    _check(lib().spmv_cg(A_inner.handle, A_exact.handle if A_exact else None, _ptr(b), _ptr(x),
                         int(iters), int(refine_every), _ptr(resid), int(use_graph),
                         _stream(stream)))


class Batch:
    """Owner of an spmv_batch_t; keeps its matrices and vectors alive."""

    def __init__(self, handle, mats):
        self.handle, self.mats, self.vecs = handle, mats, None

    def free(self):
        if self.handle:
            lib().spmv_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def spmv_batch_create(mats, threads_per_row=None, rows_per_item=None, stream=None) -> Batch:
    import numpy as np
    n = len(mats)
    arr = (CSR * max(n, 1))(*[m.desc for m in mats])
    tp = None if threads_per_row is None else np.ascontiguousarray(threads_per_row, np.int32)
    rp = None if rows_per_item is None else np.ascontiguousarray(rows_per_item, np.int32)
    h = C.c_void_p()
    _check(lib().spmv_batch_create(arr, n, tp.ctypes.data_as(C.c_void_p) if tp is not None else None,
                                   rp.ctypes.data_as(C.c_void_p) if rp is not None else None,
                                   C.byref(h), _stream(stream)))
    return Batch(h, list(mats))


def _prepared_array(preps):
    n = len(preps)
    return (C.c_void_p * max(n, 1))(*[P.handle.value if isinstance(P.handle, C.c_void_p) else P.handle
                                      for P in preps]), n


def spmv_batch_create_prepared(preps, stream=None) -> Batch:
    """A batch whose matrices run in the persistent form of their own
    prepared variant."""
    arr, n = _prepared_array(preps)
    h = C.c_void_p()
    _check(lib().spmv_batch_create_prepared(arr, n, C.byref(h), _stream(stream)))
    return Batch(h, list(preps))


def spmv_batch_create_sliced(preps, stream=None) -> Batch:
    """A batch whose matrices all run in the sliced layout."""
    arr, n = _prepared_array(preps)
    h = C.c_void_p()
    _check(lib().spmv_batch_create_sliced(arr, n, C.byref(h), _stream(stream)))
    return Batch(h, list(preps))


def spmv_batch_bind(B: Batch, xs, ys, stream=None) -> None:
    n = len(B.mats)
    xa = (C.c_void_p * max(n, 1))(*[x.data_ptr() for x in xs])
    ya = (C.c_void_p * max(n, 1))(*[y.data_ptr() for y in ys])
    B.vecs = (list(xs), list(ys))
    _check(lib().spmv_batch_bind(B.handle, xa, ya, _stream(stream)))


def spmv_batch_run(B: Batch, use_graph: bool = False, stream=None) -> None:
    _check(lib().spmv_batch_run(B.handle, int(use_graph), _stream(stream)))


def spmv_batch_autotune(B: Batch, reps: int = 3, stream=None) -> None:
    _check(lib().spmv_batch_autotune(B.handle, int(reps), _stream(stream)))


def spmv_batch_config(B: Batch):
    import numpy as np
    n = len(B.mats)
    t = np.zeros(max(n, 1), np.int32)
    r = np.zeros(max(n, 1), np.int32)
    _check(lib().spmv_batch_config(B.handle, t.ctypes.data_as(C.c_void_p), r.ctypes.data_as(C.c_void_p)))
    return t[:n], r[:n]


def spmv_batch_free(B: Batch) -> None:
    B.free()


class Model:
    """Owner of an spmv_model_t (the learned selector)."""

    def __init__(self, handle):
        self.handle = handle

    def free(self):
        if self.handle:
            lib().spmv_model_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _fptr(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(C.c_void_p)


def spmv_model_create(h1, h2, k, mean, istd, params, variants, min_margin=0.0) -> Model:
    import numpy as np
    mean, pm = _fptr(mean)
    istd, pi = _fptr(istd)
    params, pp = _fptr(params)
    variants = np.ascontiguousarray(variants, dtype=np.int32)
    h = C.c_void_p()
    _check(lib().spmv_model_create(h1, h2, k, pm, pi, pp, variants.ctypes.data_as(C.c_void_p),
                                   float(min_margin), C.byref(h)))
    return Model(h)


def spmv_model_load(path: str) -> Model:
    h = C.c_void_p()
    _check(lib().spmv_model_load(str(path).encode(), C.byref(h)))
    return Model(h)


def spmv_model_save(m: Model, path: str) -> None:
    _check(lib().spmv_model_save(m.handle, str(path).encode()))


def spmv_model_free(m: Model) -> None:
    m.free()


def spmv_model_set_launch(m: Model, launch) -> None:
    import numpy as np
    launch = np.ascontiguousarray(launch, dtype=np.int32)
    _check(lib().spmv_model_set_launch(m.handle, launch.ctypes.data_as(C.c_void_p)))


def spmv_select_model_refined(features: Features, model: Model, sub: Model | None = None,
                              profile: Profile | None = None,
                              thresholds: Thresholds | None = None) -> Choice:
    out = Choice()
    _check(lib().spmv_select_model_refined(C.byref(features), model.handle,
                                           sub.handle if sub is not None else None,
                                           C.byref(profile) if profile else None,
                                           C.byref(thresholds) if thresholds else None, C.byref(out)))
    return out


def spmv_model_logits(m: Model, vec16, k: int):
    import numpy as np
    v, pv = _fptr(vec16)
    out = np.empty(k, np.float32)
    _check(lib().spmv_model_logits(m.handle, pv, out.ctypes.data_as(C.c_void_p)))
    return out


def spmv_select_model(features: Features, model: Model, profile: Profile | None = None,
                      thresholds: Thresholds | None = None) -> Choice:
    out = Choice()
    _check(lib().spmv_select_model(C.byref(features), model.handle,
                                   C.byref(profile) if profile else None,
                                   C.byref(thresholds) if thresholds else None, C.byref(out)))
    return out


def spmv_mlp_forward(params, mean, istd, h1, h2, k, v, logits, stream=None) -> None:
    _check(lib().spmv_mlp_forward(_ptr(params), _ptr(mean), _ptr(istd), h1, h2, k, _ptr(v),
                                  int(v.shape[0]), _ptr(logits), _stream(stream)))


def spmv_mlp_loss_grad(params, h1, h2, k, z, labels, grad, loss, stream=None) -> None:
    _check(lib().spmv_mlp_loss_grad(_ptr(params), h1, h2, k, _ptr(z), _ptr(labels),
                                    int(z.shape[0]), _ptr(grad), _ptr(loss), _stream(stream)))


def spmv_mlp_loss_grad_soft(params, h1, h2, k, z, q, grad, loss, stream=None) -> None:
    """Cross-entropy against per-sample target distributions q ([n][k] float32)."""
    _check(lib().spmv_mlp_loss_grad_soft(_ptr(params), h1, h2, k, _ptr(z), _ptr(q),
                                         int(z.shape[0]), _ptr(grad), _ptr(loss), _stream(stream)))


def spmv_mlp_adam(params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                  weight_decay=0.0, stream=None) -> None:
    _check(lib().spmv_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(params.numel()),
                               int(step), float(lr), float(beta1), float(beta2), float(eps),
                               float(weight_decay), _stream(stream)))


def spmv_prepared_free(P: Prepared) -> None:
    P.free()
