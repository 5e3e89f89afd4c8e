"""ctypes mirror of include/spmv.h: structures, enums and function signatures."""
from __future__ import annotations

import ctypes as C

SPMV_OK = 0
STATUS_NAMES = {0: "SPMV_OK", 1: "SPMV_ERR_INVALID_ARG", 2: "SPMV_ERR_INVALID_CSR",
                3: "SPMV_ERR_UNSUPPORTED", 4: "SPMV_ERR_NOMEM", 5: "SPMV_ERR_CUDA",
                6: "SPMV_ERR_TIMEOUT", 7: "SPMV_ERR_MODEL"}
VARIANTS = ("scalar", "subwarp", "stream", "merge", "dynamic", "latency", "compressed", "sliced")
VARIANT_IDS = {n: i for i, n in enumerate(VARIANTS)}
CLASSES = ("CML", "MB", "IMB", "CMP")
VAL_F64, VAL_F32, VAL_BF16 = 0, 1, 2
(EXPORT_ROW_BLOCKS, EXPORT_MERGE_ROWS, EXPORT_MERGE_NZ, EXPORT_ROWBASE, EXPORT_OFFSETS,
 EXPORT_VALUES, EXPORT_SLICE_PERM, EXPORT_SLICE_ROWLEN, EXPORT_SLICE_LEN, EXPORT_SLICE_PTR,
 EXPORT_SLICE_COL, EXPORT_SLICE_VAL, EXPORT_SLICE_OFF16, EXPORT_SLICE_ROWBASE,
 EXPORT_SLICE_DIAG, EXPORT_SLICE_DELTA, EXPORT_SLICE_PANEL_LO, EXPORT_SLICE_PANEL_STEP,
 EXPORT_DYN_M1, EXPORT_DYN_M2, EXPORT_DYN_LONG, EXPORT_DYN_SEG_OFF, EXPORT_SLICE_LONG,
 EXPORT_SLICE_SEG_OFF, EXPORT_SLICE_SEG_BOUNDS, EXPORT_SLICE_SEG_ROW, EXPORT_SLICE_FIX,
 EXPORT_SLICE_SEG_FIX) = range(28)


class CSR(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_cols", C.c_int64), ("nnz", C.c_int64),
                ("rowptr", C.c_void_p), ("colind", C.c_void_p), ("val", C.c_void_p)]


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
        d["vec"] = list(self.vec)
        return d


class Profile(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("t_base_ms", "t_noxmiss_ms", "t_inflate_ms",
                                          "t_span_ms", "t_worker_mean_ms", "s_noxmiss",
                                          "s_inflate", "s_balance", "total_ms")] + \
        [("n_workers", C.c_int32), ("reps", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Thresholds(C.Structure):
    _fields_ = [("tau_noxmiss", C.c_double), ("tau_inflate", C.c_double),
                ("tau_balance", C.c_double)]


class Choice(C.Structure):
    _fields_ = [("variant", C.c_int32), ("cls", C.c_int32), ("threads_per_row", C.c_int32),
                ("block_nnz", C.c_int32), ("items_per_warp", C.c_int32),
                ("value_type", C.c_int32), ("margin", C.c_float), ("used_fallback", C.c_int32),
                ("source", C.c_int32), ("accumulate", C.c_int32), ("index_bytes", C.c_int32),
                ("index_coding", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PreparedInfo(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("variant", "threads_per_row", "block_nnz",
                                         "items_per_warp", "value_type")] + \
        [(n, C.c_int64) for n in ("n_rows", "n_cols", "nnz", "n_blocks", "n_wide_rows",
                                  "owned_bytes", "min_bytes")] + \
        [("tile_items", C.c_int32), ("bulk_copy", C.c_int32), ("accumulate", C.c_int32),
         ("launches", C.c_int32), ("index_bytes", C.c_int32), ("n_long_rows", C.c_int64),
         ("index_coding", C.c_int32), ("uniform_len", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def declare(lib):
    """Sets restype/argtypes of every exported function."""
    P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "spmv_status_str": (C.c_char_p, [I32]),
        "spmv_last_error": (C.c_char_p, []),
        "spmv_validate": (I32, [C.POINTER(CSR), P]),
        "spmv_features": (I32, [C.POINTER(CSR), I32, C.POINTER(Features), P]),
        "spmv_profile": (I32, [C.POINTER(CSR), P, I32, C.POINTER(Profile), P]),
        "spmv_gather_probe": (I32, [C.POINTER(CSR), P, P, P]),
        "spmv_profile_outputs": (I32, [C.POINTER(CSR), P, I64, P, P, P, P, P, P]),
        "spmv_fixup_check": (I32, [I32, I64, I64, P, P, P, P, P]),
        "spmv_stream_noalloc_status": (I32, [P]),
        "spmv_wait_check": (I32, [C.c_int64, I32, P]),
        "spmv_default_thresholds": (Thresholds, []),
        "spmv_classify_profile": (I32, [C.POINTER(Profile), C.POINTER(Thresholds), C.POINTER(I32)]),
        "spmv_class_variant": (I32, [I32]),
        "spmv_class_choice": (I32, [I32, C.POINTER(Choice)]),
        "spmv_select": (I32, [C.POINTER(Features), C.POINTER(Profile), C.POINTER(Thresholds),
                              C.POINTER(Choice)]),
        "spmv_prepare": (I32, [C.POINTER(CSR), C.POINTER(Choice), I32, C.POINTER(P), P]),
        "spmv": (I32, [P, P, P, P]),
        "spmv_host": (I32, [P, P, P, P]),
        "spmv_host_async": (I32, [P, P, P, P]),
        "spmv_prepared_info": (I32, [P, C.POINTER(PreparedInfo)]),
        "spmv_prepared_export": (I32, [P, I32, P, I64, P]),
        "spmv_prepared_status": (I32, [P, P]),
        "spmv_stream_noalloc": (I32, [C.POINTER(CSR), P, P, P]),
        "spmv_cg": (I32, [P, P, P, P, I32, I32, P, I32, P]),
        "spmv_batch_create": (I32, [C.POINTER(CSR), I32, P, P, C.POINTER(P), P]),
        "spmv_batch_create_prepared": (I32, [P, I32, P, P]),
        "spmv_batch_create_sliced": (I32, [P, I32, P, P]),
        "spmv_batch_bind": (I32, [P, P, P, P]),
        "spmv_batch_run": (I32, [P, I32, P]),
        "spmv_batch_autotune": (I32, [P, I32, P]),
        "spmv_batch_config": (I32, [P, P, P]),
        "spmv_batch_free": (None, [P]),
        "spmv_model_create": (I32, [I32, I32, I32, P, P, P, P, C.c_float, C.POINTER(P)]),
        "spmv_model_save": (I32, [P, C.c_char_p]),
        "spmv_model_load": (I32, [C.c_char_p, C.POINTER(P)]),
        "spmv_model_free": (None, [P]),
        "spmv_model_set_launch": (I32, [P, P]),
        "spmv_select_model_refined": (I32, [C.POINTER(Features), P, P, C.POINTER(Profile),
                                            C.POINTER(Thresholds), C.POINTER(Choice)]),
        "spmv_model_logits": (I32, [P, P, P]),
        "spmv_select_model": (I32, [C.POINTER(Features), P, C.POINTER(Profile),
                                    C.POINTER(Thresholds), C.POINTER(Choice)]),
        "spmv_mlp_forward": (I32, [P, P, P, I32, I32, I32, P, I32, P, P]),
        "spmv_mlp_loss_grad": (I32, [P, I32, I32, I32, P, P, I32, P, P, P]),
        "spmv_mlp_loss_grad_soft": (I32, [P, I32, I32, I32, P, P, I32, P, P, P]),
        "spmv_mlp_adam": (I32, [P, P, P, P, I64, I32, C.c_float, C.c_float, C.c_float,
                                C.c_float, C.c_float, P]),
        "spmv_prepared_free": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib
