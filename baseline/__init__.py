"""CPU restatement of the paper's Table 2 optimizations (Section 3.3) and its
unoptimized multithreaded baseline (Section 3.2.1), for the host cores.

BASELINE ONLY: the benchmark reports it beside the GPU path and the
one-core oracle; the CUDA library never imports it, and it is not the
oracle.  The arithmetic is in ``cpu_table2.c`` (C + OpenMP); this module
builds it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpu_table2.c")
_LIB = os.path.join(_HERE, "libcpu_table2.so")
_lock = threading.Lock()
_lib = None

FORMS = ("base", "prefetch", "delta", "dynamic", "simd")
# Table 2: the optimization each class receives
CLASS_FORM = {"CML": "prefetch", "MB": "delta", "IMB": "dynamic", "CMP": "simd"}


def build(force: bool = False) -> str:
    """Compile cpu_table2.c with gcc and OpenMP (without OpenMP if the
    compiler lacks it: one thread)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O3", "-fPIC", "-shared", "-o", tmp, _SRC]
        if subprocess.run(base[:2] + ["-fopenmp"] + base[2:], capture_output=True).returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
            lib.t2_threads.restype = i32
            lib.t2_threads.argtypes = []
            lib.t2_delta_prepare.restype = i32
            lib.t2_delta_prepare.argtypes = [i64, P, P, P, P, P]
            lib.t2_spmv.restype = i32
            lib.t2_spmv.argtypes = [i32, i64, P, P, P, P, P, P, P, P, i32, i32, i32]
            _lib = lib
    return _lib


def _np(a, dtype):
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def threads() -> int:
    """Threads the OpenMP forms run on."""
    return int(_load().t2_threads())


class Matrix:
    """Host CSR arrays (numpy) with the delta-coded copy built on demand."""

    def __init__(self, A):
        self.n_rows = int(A.n_rows)
        self.rowptr = _np(A.rowptr, np.int32)
        self.colind = _np(A.colind, np.int32)
        self.val = _np(A.val, np.float64)
        self.delta = None

    def prepare_delta(self):
        if self.delta is None:
            base = np.empty(max(self.n_rows, 1), np.int32)
            coded = np.empty(max(self.n_rows, 1), np.uint8)
            raw = np.empty(max(2 * self.colind.size, 1), np.uint8)
            width = int(_load().t2_delta_prepare(self.n_rows, _p(self.rowptr), _p(self.colind),
                                                 _p(base), _p(coded), _p(raw)))
            self.delta = (base, coded, raw, width)
        return self.delta

    def bytes_streamed(self, form: str) -> int:
        """Index bytes an SpMV of this form reads, plus values, rowptr, x and y
        (x read once): the minimum traffic of the form."""
        nnz, n = self.colind.size, self.n_rows
        idx = 4 * nnz
        if form == "delta":
            base, coded, _, width = self.prepare_delta()
            lens = np.diff(self.rowptr.astype(np.int64))
            coded_nnz = int(lens[coded[:n].astype(bool)].sum())
            idx = width * coded_nnz + 4 * (nnz - coded_nnz) + 5 * n
        return idx + 8 * nnz + 4 * (n + 1) + 8 * n + 8 * n


def spmv(form: str, M: Matrix, x, y=None, pref_dist: int = 0, dyn_chunk: int = 0) -> np.ndarray:
    """y = A x with one of FORMS."""
    x = _np(x, np.float64)
    if y is None:
        y = np.empty(M.n_rows, np.float64)
    base = coded = raw = None
    width = 0
    if form == "delta":
        base, coded, raw, width = M.prepare_delta()
    rc = _load().t2_spmv(FORMS.index(form), M.n_rows, _p(M.rowptr), _p(M.colind), _p(M.val), _p(x),
                         _p(y), _p(base), _p(coded), _p(raw), width, pref_dist, dyn_chunk)
    if rc != 0:
        raise ValueError(f"unknown form {form}")
    return y
