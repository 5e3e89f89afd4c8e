/*
 * spmv.h -- C ABI of the GB300 SpMV optimization-selection library.
 *
 * The library implements the method of Elafrou, Goumas and Koziris, "A
 * lightweight optimization selection method for Sparse Matrix-Vector
 * Multiplication" (arXiv 1511.02494) for one NVIDIA GB300 (sm_103a):
 *
 *   spmv_features(A)          structural features of Table 1 (Section 3.2.2)
 *   spmv_profile(A, x)        the profiling runs of Section 3.2.1
 *                             (baseline, noxmiss, inflate, balance)
 *   spmv_select(f | profile)  bottleneck class (Section 3.1) and the variant
 *                             that tackles it (Section 3.3, Table 2)
 *   spmv_prepare(A, choice)   any format conversion the variant needs
 *   spmv(P, x, y)             y = A x (Algorithm 1) with the chosen variant
 *
 * Conventions shared by every entry point:
 *   - Matrices are CSR with 0-based int32 row pointers and column indices and
 *     FP64 values; rowptr[0] = 0, rowptr[n_rows] = nnz, rowptr non-decreasing,
 *     column indices in [0, n_cols) and strictly increasing within a row.
 *   - Pointers inside spmv_csr_t and the x / y vectors are DEVICE pointers on
 *     the current CUDA device, borrowed: the caller owns them and keeps them
 *     alive while any call or prepared object uses them.  Host pointers are
 *     named *_host.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Kernels
 *     are launched on it; calls that return host results synchronize it.
 *   - Every call returns an spmv_status; nothing throws across the ABI.  On
 *     failure spmv_last_error() gives a message for the calling thread.
 *   - No call falls back to the CPU: without a usable GPU calls fail with
 *     SPMV_ERR_CUDA.
 */
#ifndef PAPER_1511_02494_GB300_SPMV_H
#define PAPER_1511_02494_GB300_SPMV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *spmv_stream_t; /* identical to cudaStream_t */

typedef enum {
    SPMV_OK = 0,
    SPMV_ERR_INVALID_ARG = 1,  /* NULL pointer, negative size, bad option */
    SPMV_ERR_INVALID_CSR = 2,  /* the matrix breaks a CSR rule above      */
    SPMV_ERR_UNSUPPORTED = 3,  /* variant/option not applicable to A       */
    SPMV_ERR_NOMEM = 4,        /* device or host allocation failed         */
    SPMV_ERR_CUDA = 5,         /* a CUDA runtime call or launch failed     */
    SPMV_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up       */
    SPMV_ERR_MODEL = 7         /* selector model missing, corrupt or bad   */
} spmv_status;

/* SpMV variants.  Each attacks one bottleneck class of Section 3.1 the way
 * Table 2's optimizations do on a CPU: LATENCY the latency of x misses
 * (CML), COMPRESSED the bytes streamed (MB), DYNAMIC the imbalance (IMB),
 * SUBWARP the per-row overhead of short rows (CMP).  SLICED is a GPU format
 * with no counterpart in Table 2: 32-row slices whose k-th elements are
 * stored next to each other, one lane per row and no reduction across lanes
 * (rows above a length cap are computed from CSR by one warp each); its
 * prepare step adapts the layout to the row lengths (a length sort and a low
 * cap when rows are uneven, four slices per warp when all are short).  The
 * class -> variant table used by the profiling rule (spmv_class_variant) is
 * calibrated on GB300 like the thresholds -- for each class the variant with
 * the lowest geometric-mean slowdown on the training matrices, which is
 * SLICED for all four classes.  SCALAR is the unoptimized
 * CSR kernel (one thread per row, Algorithm 1 as written) against which
 * speedups are reported. */
typedef enum {
    SPMV_V0_SCALAR = 0,     /* one thread per row                                */
    SPMV_V1_SUBWARP = 1,    /* T lanes per row (T = 1..32), shuffle reduction    */
    SPMV_V2_STREAM = 2,     /* windows of B nonzeros staged through shared memory */
    SPMV_V3_MERGE = 3,      /* merge-path split of rows + nonzeros per CTA tile  */
    SPMV_V4_DYNAMIC = 4,    /* rows tiered by length, long rows split, dynamic queue */
    SPMV_V5_LATENCY = 5,    /* gathers of x issued ahead, x kept in L2           */
    SPMV_V6_COMPRESSED = 6, /* 16-bit column offsets, FP64/FP32/BF16 values      */
    SPMV_V7_SLICED = 7,     /* 32-row slices stored column-major, a lane per row */
    SPMV_NUM_VARIANTS = 8
} spmv_variant;

/* Bottleneck classes of Section 3.1. */
typedef enum {
    SPMV_CLASS_CML = 0, /* cache-miss latency on x        */
    SPMV_CLASS_MB = 1,  /* memory bandwidth               */
    SPMV_CLASS_IMB = 2, /* thread/workload imbalance      */
    SPMV_CLASS_CMP = 3  /* computation / short rows       */
} spmv_class;

/* Storage type of the values of the COMPRESSED variant (x, y and the
 * accumulation are always FP64). */
typedef enum { SPMV_VAL_F64 = 0, SPMV_VAL_F32 = 1, SPMV_VAL_BF16 = 2 } spmv_value_type;

/* A CSR matrix; all pointers are device pointers, borrowed. */
typedef struct {
    int64_t n_rows, n_cols, nnz;
    const int32_t *rowptr; /* [n_rows + 1] */
    const int32_t *colind; /* [nnz]        */
    const double *val;     /* [nnz]        */
} spmv_csr_t;

/* Structural features, Table 1 (Section 3.2.2).  The integer aggregates are
 * exact; the doubles are computed from them on the host:
 *   nnz_i   = nonzeros of row i
 *   bw_i    = last column - first column of row i (0 when nnz_i <= 1)
 *   span_i  = bw_i + 1 (the "distance" of disp_i)
 *   disp_i  = nnz_i / span_i, kept as q = floor(2^32 disp_i)
 *   clust_i = ngroups_i / nnz_i, kept as q = floor(2^32 clust_i); ngroups_i
 *             counts maximal runs of consecutive columns
 *   misses_i = 1 + #{j > first : 8 (c_j - c_{j-1}) > line_bytes}
 * Empty rows count with every per-row quantity 0.  Averages divide by n_rows;
 * deviations are population deviations, sqrt(N S2 - S1^2) / N.
 * 128-bit sums are split into _lo / _hi 64-bit words.
 * vec[16] is the selector input: size, log2 density, log2(1+v) of nnz_min,
 * nnz_max, nnz_avg, nnz_sd, bw_min, bw_max, bw_avg, bw_sd, then disp_avg,
 * disp_sd, clustering, log2(1 + miss_ratio), log2(1 + n_rows),
 * log2(1 + nnz), each rounded to float. */
typedef struct {
    int64_t n_rows, n_cols, nnz, line_bytes, l2_bytes, working_set_bytes;
    int64_t nnz_min, nnz_max;
    uint64_t nnz_sum, nnz_sumsq_lo, nnz_sumsq_hi;
    int64_t bw_min, bw_max;
    uint64_t bw_sum, bw_sumsq_lo, bw_sumsq_hi;
    uint64_t disp_sum, disp_sumsq_lo, disp_sumsq_hi;
    uint64_t clust_sum;
    uint64_t ngroups_sum, misses_sum;
    double size, density, nnz_avg, nnz_sd, bw_avg, bw_sd;
    double disp_avg, disp_sd, clustering, miss_ratio;
    float vec[16];
} spmv_features_t;

/* Result of the profiling runs of Section 3.2.1.  All runs use the baseline
 * kernel: static 1-D row partition with equal nonzeros per worker (a warp),
 * each worker walking its rows.
 *   t_base_ms      median time of the baseline
 *   t_noxmiss_ms   median time with every column index replaced by 0
 *   t_inflate_ms   median time with 64-bit rowptr and colind
 *   t_span_ms      balance run: last worker end - first worker start
 *   t_worker_mean_ms  balance run: arithmetic mean of worker durations
 *   s_noxmiss = t_base / t_noxmiss, s_inflate = t_inflate / t_base,
 *   s_balance = t_span / t_worker_mean
 *   total_ms       wall time of the whole spmv_profile call */
typedef struct {
    double t_base_ms, t_noxmiss_ms, t_inflate_ms, t_span_ms, t_worker_mean_ms;
    double s_noxmiss, s_inflate, s_balance;
    double total_ms;
    int32_t n_workers, reps;
} spmv_profile_t;

/* Thresholds of the profiling rule (Section 3.2.1); a probe's speedup must be
 * strictly greater than its threshold.  The paper does not print its values;
 * spmv_default_thresholds() gives this library's calibrated defaults. */
typedef struct {
    double tau_noxmiss, tau_inflate, tau_balance;
} spmv_thresholds_t;

/* A variant and its launch parameters.  Zero parameters mean "choose".
 *   threads_per_row : SUBWARP / LATENCY / COMPRESSED / DYNAMIC (short rows) lanes
 *                     per row (1..32, power of 2)
 *   threads_per_row : SLICED with FP64 values: slices per warp, 1, 2 or 4 (a
 *                     lane sums one row of each); 0 = 4 when no slice is
 *                     longer than four elements, else 1
 *   block_nnz       : STREAM nonzeros per window (64..8192, power of 2; default
 *                     2048).  With 1024 or 2048 and 16-byte-aligned arrays the
 *                     pipelined bulk-copy kernel runs; otherwise a kernel that
 *                     stages each row block with plain loads
 *   block_nnz       : MERGE merge-path items (row ends + nonzeros) per CTA tile of
 *                     the pipelined kernel, 1024, 1536 or 2048 (default 2048)
 *   items_per_warp  : MERGE items per warp of the warp-level kernel used instead
 *                     when rowptr, colind or val is not 16-byte aligned
 *                     (32 k, k in {1, 2, 4, 6, 7, 8, 12, 16})
 *   items_per_warp  : SLICED row-length cap, 1..65536 (0 = 1024): rows with
 *                     more nonzeros are left out of the slices and computed
 *                     from CSR in segments of 2048 nonzeros, one warp each.
 *                     A lane's chain of FMAs is at most this long, so a low
 *                     cap with a wide sort window suits power-law row lengths
 *   block_nnz       : DYNAMIC nonzeros per segment of a long row (power of two,
 *                     256..2^20; default 2048)
 *   block_nnz       : SLICED window of the length sort: 1 = rows in order, or a
 *                     power of two in 32..4096 (rows sorted by length, longest
 *                     first, inside windows of that many rows); 0 = rows in
 *                     order unless that pads the slices by more than 25 %,
 *                     then 4096 with a row-length cap of 32 (unless
 *                     items_per_warp sets the cap)
 *   value_type      : COMPRESSED and SLICED value storage (spmv_value_type);
 *                     SLICED with FP32/BF16 values stores 16-bit column
 *                     offsets from each row's first column when every row in
 *                     its slices spans fewer than 65536 columns
 *   accumulate      : COMPRESSED and SLICED arithmetic.  FP32 (the default for FP32/BF16
 *                     values) rounds x to an FP32 copy owned by the prepared
 *                     object once per call and sums in FP32 (no FP64
 *                     instruction per nonzero; relative error ~1e-7 against
 *                     the same values in FP64); spmv calls on one such object
 *                     must not overlap.  FP64 converts each value and sums in
 *                     FP64.
 * Filled by spmv_select: cls (or -1), margin (model logit gap, or 0),
 * used_fallback (1 when the model deferred to the profile rule), source
 * (0 explicit, 1 profile rule, 2 model). */
typedef struct {
    int32_t variant;
    int32_t cls;
    int32_t threads_per_row;
    int32_t block_nnz;
    int32_t items_per_warp;
    int32_t value_type;
    float margin;
    int32_t used_fallback;
    int32_t source;
    int32_t accumulate;  /* COMPRESSED: 0 by value type (FP64 values -> FP64,
                            FP32/BF16 values -> FP32), 1 FP64, 2 FP32 */
    int32_t index_bytes; /* SLICED with FP64 values: narrowest stored column
                            allowed -- 4: 32-bit columns; 2 or 1: the
                            column minus the row index in int16 or int8 when
                            every row in the slices stays that close to its
                            diagonal (else the next wider form); 0: as 1 when
                            every row has the same length and the rows stay
                            in order (no slice header is read there, and the
                            narrower index stream shortens the launch), else
                            as 4 (with a header to read, the 32-bit form is
                            as fast or faster on GB300). */
    int32_t index_coding; /* SLICED with FP64 values: 0 = as index_bytes says;
                            1 = Table 2's delta coding (Section 3.3): each
                            column stored as its difference from the
                            previous column of its row, the row's first
                            column as a 32-bit base per position, in 8 bits
                            when every delta in the slices' rows is at most
                            255, else in 16 bits when at most 65535 (one
                            width per matrix); when neither fits, as 2;
                            2 = column-blocked: each column as its 16-bit
                            offset inside a panel of 65536 columns plus an
                            8-bit step from the previous element's panel,
                            when every step is at most 255; else 32-bit
                            columns.  Coded columns run one slice per warp
                            (threads_per_row 0 or 1). */
} spmv_choice_t;

/* A matrix prepared for one variant (opaque).  It borrows A's arrays and owns
 * whatever the variant built from them. */
typedef struct spmv_prepared spmv_prepared_t;

/* What a prepared object holds (for inspection and tests). */
typedef struct {
    int32_t variant, threads_per_row, block_nnz, items_per_warp, value_type;
    int64_t n_rows, n_cols, nnz;
    int64_t n_blocks;      /* STREAM windows / MERGE tiles / DYNAMIC work items /
                              SLICED slices */
    int64_t n_wide_rows;   /* COMPRESSED rows that kept 32-bit columns          */
    int64_t owned_bytes;   /* device bytes owned by the object                  */
    int64_t min_bytes;     /* minimum traffic of one spmv() with this format    */
    int32_t tile_items;    /* MERGE: merge-path items per tile as prepared      */
    int32_t bulk_copy;     /* 1 when the pipelined bulk-copy kernel is used     */
    int32_t accumulate;    /* 1 FP64, 2 FP32 (COMPRESSED with FP32 accumulation) */
    int32_t launches;      /* kernels one spmv call launches (0 when n_rows = 0) */
    int32_t index_bytes;   /* SLICED with FP64 values: bytes per stored column,
                              4 (the column), 2 or 1 (column - row, int16 or
                              int8, or with index_coding 1 the delta), 3
                              (index_coding 2: 16-bit panel offset + 8-bit
                              step); 4 for the other variants                 */
    int64_t n_long_rows;   /* SLICED: rows above the length cap, computed from
                              CSR in segments; 0 for the other variants       */
    int32_t index_coding;  /* SLICED with FP64 values: the column coding in
                              use, 0, 1 (deltas) or 2 (panels), as in
                              spmv_choice_t; 0 for the other variants         */
    int32_t uniform_len;   /* SLICED with FP64 values and uncoded columns: the
                              length every row has, when they all have one,
                              the rows stay in order and none is long (the
                              kernel then reads no slice header); else -1    */
} spmv_prepared_info_t;

/* Arrays a prepared object can export (spmv_prepared_export). */
typedef enum {
    SPMV_EXPORT_ROW_BLOCKS = 0, /* STREAM: int32 [n_blocks + 1] first row of each block */
    SPMV_EXPORT_MERGE_ROWS = 1, /* MERGE: int32 [n_blocks + 1] start row of each part   */
    SPMV_EXPORT_MERGE_NZ = 2,   /* MERGE: int32 [n_blocks + 1] start nonzero of a part  */
    SPMV_EXPORT_ROWBASE = 3,    /* COMPRESSED: int32 [n_rows] first column, -1 = wide   */
    SPMV_EXPORT_OFFSETS = 4,    /* COMPRESSED: uint16 [nnz] column - rowbase            */
    SPMV_EXPORT_VALUES = 5,     /* COMPRESSED: [nnz] values in value_type               */
    SPMV_EXPORT_SLICE_PERM = 6, /* SLICED, rows sorted: int32 [n_rows] position -> row  */
    SPMV_EXPORT_SLICE_ROWLEN = 7, /* SLICED: int32 [32 S] row length per position, -1 =
                                   long row (computed from CSR) or past the last row   */
    SPMV_EXPORT_SLICE_LEN = 8,  /* SLICED: int32 [S] slice length (longest row in it)   */
    SPMV_EXPORT_SLICE_PTR = 9,  /* SLICED: int64 [S + 1] first slot of each slice; with
                                   FP64 values element k of position 32 s + l is at
                                   slot ptr[s] + 32 k + l, with FP32/BF16 values at
                                   ptr[s] + 128 (k / 4) + 4 l + k % 4 (slices padded
                                   to a multiple of 4 elements per row)                */
    SPMV_EXPORT_SLICE_COL = 10, /* SLICED: int32 [slice_ptr[S]] columns, column-major
                                   (absent with 16-bit offsets and with index_bytes
                                   2 or 1)                                           */
    SPMV_EXPORT_SLICE_VAL = 11, /* SLICED: [slice_ptr[S]] values in value_type          */
    SPMV_EXPORT_SLICE_OFF16 = 12, /* SLICED, 16-bit offsets: uint16 [slice_ptr[S]]
                                   column - row base                                   */
    SPMV_EXPORT_SLICE_ROWBASE = 13, /* SLICED, 16-bit offsets (FP32/BF16 values) or
                                   deltas (index_coding 1): int32 [32 S] first column
                                   of each position's row (0 where none)               */
    SPMV_EXPORT_SLICE_DIAG = 14,  /* SLICED, FP64 values, index_bytes 2 or 1: int16 or
                                     int8 [slice_ptr[S]] column - row, column-major
                                     like SLICE_COL, 0 in padding                  */
    SPMV_EXPORT_SLICE_DELTA = 15, /* SLICED, index_coding 1: uint8 or uint16
                                     (index_bytes) [slice_ptr[S]] column - previous
                                     column of the row, 0 for a row's first element
                                     and in padding, column-major like SLICE_COL   */
    SPMV_EXPORT_SLICE_PANEL_LO = 16,   /* SLICED, index_coding 2: uint16 [slice_ptr[S]]
                                     column mod 65536, 0 in padding                */
    SPMV_EXPORT_SLICE_PANEL_STEP = 17, /* SLICED, index_coding 2: uint8 [slice_ptr[S]]
                                     panel (column / 65536) minus the previous
                                     element's panel (0 before a row's first
                                     element), 0 in padding                        */
    SPMV_EXPORT_DYN_M1 = 18,      /* DYNAMIC: int32 [n_m1] rows with lim_s < len <= 64,
                                     lim_s = min(16 threads_per_row, block_nnz), in
                                     the order a prepare found them (atomics: the
                                     set is fixed, the order is not)               */
    SPMV_EXPORT_DYN_M2 = 19,      /* DYNAMIC: int32 [n_m2] rows with 64 < len <= block_nnz */
    SPMV_EXPORT_DYN_LONG = 20,    /* DYNAMIC: int32 [n_long] rows with len > block_nnz  */
    SPMV_EXPORT_DYN_SEG_OFF = 21, /* DYNAMIC: int32 [n_long + 1] first segment of each
                                     long row (in DYN_LONG's order): the running sum of
                                     ceil(len / block_nnz)                         */
    SPMV_EXPORT_SLICE_LONG = 22,  /* SLICED: int32 [n_long_rows] rows above the cap,
                                     ascending                                     */
    SPMV_EXPORT_SLICE_SEG_OFF = 23,    /* SLICED: int32 [n_long_rows + 1] first segment
                                     of each long row (segments of 2048 nonzeros)  */
    SPMV_EXPORT_SLICE_SEG_BOUNDS = 24, /* SLICED: int64 [2 n_seg] CSR begin and end of
                                     each segment                                  */
    SPMV_EXPORT_SLICE_SEG_ROW = 25,    /* SLICED: int32 [n_seg] the segment's row when it
                                     is its row's only segment, else -1            */
    SPMV_EXPORT_SLICE_FIX = 26,   /* SLICED: int32 [n_fix] long-row list indices of the
                                     rows with several segments                    */
    SPMV_EXPORT_SLICE_SEG_FIX = 27     /* SLICED, FP64 values: int32 [n_seg] index in
                                     SLICE_FIX of the segment's row, -1 for a row's
                                     only segment                                  */
} spmv_export;

/* ---- status ---------------------------------------------------------- */
const char *spmv_status_str(spmv_status s);
/* Message of the last failed call on this thread ("" if none). */
const char *spmv_last_error(void);

/* ---- validation -------------------------------------------------------- */
/* Checks every CSR rule above on the device.  SPMV_ERR_INVALID_CSR when one
 * fails; no device access ever leaves the arrays' declared extents. */
spmv_status spmv_validate(const spmv_csr_t *A, spmv_stream_t stream);

/* ---- Table 1 features (Section 3.2.2) ------------------------------------- */
/* One pass over rowptr and colind (validating A on the way); fills *out
 * (host) and synchronizes `stream`.  line_bytes: cache line assumed by the
 * miss count (0 = 128, the GB300 L2 line).  size compares the working set
 * with the device's L2 capacity. */
spmv_status spmv_features(const spmv_csr_t *A, int32_t line_bytes, spmv_features_t *out,
                          spmv_stream_t stream);

/* ---- profiling runs (Section 3.2.1) ---------------------------------------- */
/* Runs the baseline and the noxmiss, inflate and balance probes on A with the
 * input vector x (device, n_cols), `reps` timed runs each (0 = 5) after one
 * warm-up, and fills *out (host).  Allocates and frees its own temporary
 * device buffers (a zeroed colind and 64-bit index copies: 4 nnz +
 * 8 (n_rows + 1 + nnz) bytes).  Synchronizes `stream`. */
spmv_status spmv_profile(const spmv_csr_t *A, const double *x, int32_t reps,
                         spmv_profile_t *out, spmv_stream_t stream);

/* The products and the partition of the profiling runs, which spmv_profile
 * only times (Section 3.2.1 defines each run by what it changes in the
 * baseline SpMV; this call returns what each computes, so that it can be
 * checked).  One untimed run of each requested probe, on the kernels and the
 * set-up spmv_profile uses:
 *   bounds     device int64 [n_workers + 1] or NULL: the baseline's static
 *              partition, bounds[w] = smallest row i with
 *              rowptr[i] >= floor(w * nnz / n_workers), bounds[n_workers] =
 *              n_rows (worker w walks rows bounds[w] .. bounds[w+1] - 1)
 *   y_base     device [n_rows] or NULL: the baseline's y = A x
 *   y_noxmiss  device [n_rows] or NULL: the same with every column index 0,
 *              i.e. y_i = x[0] * sum_j a_ij (summed in the baseline's order)
 *   y_inflate  device [n_rows] or NULL: the baseline with 64-bit rowptr and
 *              colind (the same arithmetic in the same order as y_base)
 *   y_balance  device [n_rows] or NULL: the baseline with the per-worker
 *              time stamps (the same arithmetic as y_base)
 * n_workers: 0 = the count spmv_profile uses (spmv_profile_t.n_workers),
 * else 1 .. 2^26.  Validates A; allocates (stream-ordered) and frees the
 * probes' temporary buffers as spmv_profile does.  Synchronizes `stream`.
 * SPMV_ERR_UNSUPPORTED for a matrix without rows or nonzeros. */
spmv_status spmv_profile_outputs(const spmv_csr_t *A, const double *x, int64_t n_workers,
                                 int64_t *bounds, double *y_base, double *y_noxmiss,
                                 double *y_inflate, double *y_balance, spmv_stream_t stream);

/* Gather probe (a measurement aid in the spirit of the probes above, with no
 * counterpart in the paper): *sum (device, one uint64) = the sum modulo 2^64
 * of the 64-bit patterns of x[colind[j]] over every nonzero, read in storage
 * order with as many independent gathers in flight as the GPU keeps and no
 * floating-point arithmetic.  Its duration is the cost of A's accesses to x
 * alone in CSR order: a reference for matrices whose columns have no
 * locality, whose SpMV time it approaches.  A's indices are not validated
 * (they must lie in [0, n_cols)).  Allocates (stream-ordered) a small
 * scratch.  Asynchronous. */
spmv_status spmv_gather_probe(const spmv_csr_t *A, const double *x, uint64_t *sum,
                              spmv_stream_t stream);

/* Self-test of failure detection without a GPU fault: one warp waits on a
 * shared-memory mbarrier with the bounded wait (a %globaltimer limit) that the
 * STREAM and MERGE pipelines use.  arrive != 0: the barrier's one arrival is
 * made first and the call returns SPMV_OK; arrive == 0: nothing arrives, the
 * wait gives up after limit_ns (1..2e9 nanoseconds) and the call returns
 * SPMV_ERR_TIMEOUT with the device context intact.  Synchronizes `stream`. */
spmv_status spmv_wait_check(int64_t limit_ns, int32_t arrive, spmv_stream_t stream);

/* Self-test of the carry fix-ups that follow the pipelined kernels (a test
 * aid; the paper has no counterpart).  Runs the STREAM (kind 0) or MERGE
 * (kind 1) fix-up alone on caller-filled device arrays: carry_row int32
 * [n_parts] (the row of each part's carried partial sum, -1 = none; the
 * parts carrying one row are consecutive), carry_val [n_parts], status (one
 * uint32) and y [n_rows].  It adds each row's carries to y[row] in part
 * order, skips entries outside [0, n_rows), and leaves y untouched when
 * *status != 0: after a bounded wait gave up, the parts the kernel skipped
 * hold carry rows of an earlier call.  Asynchronous on `stream`. */
spmv_status spmv_fixup_check(int32_t kind, int64_t n_parts, int64_t n_rows,
                             const int32_t *carry_row, const double *carry_val,
                             const uint32_t *status, double *y, spmv_stream_t stream);

/* ---- selection (Sections 3.1-3.3) ----------------------------------------- */
spmv_thresholds_t spmv_default_thresholds(void);

/* Class of a profile by the rule of Section 3.2.1: probe speedups examined
 * from the largest down (ties in the order CML, MB, IMB); the first above its
 * threshold names the class; none -> CMP.  th may be NULL (defaults). */
spmv_status spmv_classify_profile(const spmv_profile_t *p, const spmv_thresholds_t *th,
                                  int32_t *cls);

/* Variant that tackles a class (see spmv_variant). */
int32_t spmv_class_variant(int32_t cls);

/* The whole choice for a class (Table 2 on GB300): the class's variant and
 * the launch configuration calibrated for the class (source 1, cls set).
 * All four classes take SLICED.  CML and CMP take its structural rules, MB
 * rows in order with one slice per warp, and IMB a length sort in windows
 * of 4096 with a row cap of 32.  The table was calibrated on the training
 * matrices, among the second level's configurations and delta-coded
 * layouts.  spmv_select and the fallback of spmv_select_model return this
 * choice.  SPMV_ERR_INVALID_ARG for an unknown class. */
spmv_status spmv_class_choice(int32_t cls, spmv_choice_t *out);

/* Chooses a variant.  With a profile (p != NULL) and no model, the profile
 * rule decides (spmv_class_choice of the rule's class).  Host-only; does not touch the GPU.  f may be NULL when p is
 * given.  SPMV_ERR_INVALID_ARG when p holds a NaN or non-positive speedup. */
spmv_status spmv_select(const spmv_features_t *f, const spmv_profile_t *p,
                        const spmv_thresholds_t *th, spmv_choice_t *out);

/* ---- learned selector ----------------------------------------------------------- */
/* The paper's feature-based classifier (Section 3.2.2) maps Table 1 features
 * to a class with a decision tree or naive Bayes.  This library instead maps
 * spmv_features_t.vec to a variant with a 16 -> h1 -> h2 -> k ReLU network
 * (FP32) trained on the GPU (spmv_mlp_loss_grad, spmv_mlp_adam), with the
 * profiling rule of Section 3.2.1 as its fallback when the top two logits are
 * closer than the model's min_margin.
 * params packs row-major W1[h1][16], b1[h1], W2[h2][h1], b2[h2], W3[k][h2],
 * b3[k]; inputs are standardised z = (v - mean) * istd; every dot product is
 * an fmaf chain from the bias over inputs in ascending order, identical on
 * host and device, so logits are reproducible bit for bit. */
typedef struct spmv_model spmv_model_t;

/* Copies the given host arrays into a new model.  variants[o] is the variant
 * of output o.  SPMV_ERR_MODEL for a bad shape (hidden widths 1..256,
 * 2 <= k <= 32), an unknown variant or a non-finite parameter. */
spmv_status spmv_model_create(int32_t h1, int32_t h2, int32_t k, const float *mean16,
                              const float *istd16, const float *params,
                              const int32_t *variants, float min_margin,
                              spmv_model_t **out);
/* Binary model file: "SPMVMLP1", int32 h1 h2 k, float mean[16] istd[16],
 * params, int32 variants[k], float min_margin.  Load fails with
 * SPMV_ERR_MODEL on a missing, truncated, oversized or corrupt file. */
spmv_status spmv_model_save(const spmv_model_t *m, const char *path);
spmv_status spmv_model_load(const char *path, spmv_model_t **out);
void spmv_model_free(spmv_model_t *m);

/* Attaches launch parameters to each output of m (host [k][3]: for output o,
 * threads_per_row, block_nnz, items_per_warp of the output's variant, each
 * as in spmv_choice_t), making m a second-level model that chooses among one
 * variant's launch configurations.  SPMV_ERR_MODEL when a triple is not a
 * valid choice for its variant.  spmv_model_save then writes the file as
 * "SPMVMLP2" with the int32 table appended; spmv_model_load reads both. */
spmv_status spmv_model_set_launch(spmv_model_t *m, const int32_t *launch);

/* Logits of one host 16-vector (host computation, k outputs). */
spmv_status spmv_model_logits(const spmv_model_t *m, const float *vec16, float *logits);

/* Variant for the features f: argmax of the logits (ties to the lower
 * output), margin = best - second logit; when m carries launch parameters
 * (spmv_model_set_launch) the choice takes the chosen output's.  When
 * margin < min_margin and a profile p is given, the profiling rule decides
 * instead (used_fallback = 1, source = 1, the class's choice from
 * spmv_class_choice); otherwise source = 2.  Host-only; th may be NULL. */
spmv_status spmv_select_model(const spmv_features_t *f, const spmv_model_t *m,
                              const spmv_profile_t *p, const spmv_thresholds_t *th,
                              spmv_choice_t *out);

/* Two levels (the multi-level selection the paper proposes as future work):
 * spmv_select_model with m, then, when every output of sub names the variant
 * chosen, sub's forward on the same features picks that variant's launch
 * parameters (threads_per_row, block_nnz, items_per_warp of the choice).
 * sub may be NULL (first level only).  A choice from a model with launch
 * parameters carries them; a profile fallback keeps its class's choice
 * (spmv_class_choice) and is not refined.  Host-only. */
spmv_status spmv_select_model_refined(const spmv_features_t *f, const spmv_model_t *m,
                                      const spmv_model_t *sub, const spmv_profile_t *p,
                                      const spmv_thresholds_t *th, spmv_choice_t *out);

/* Device forward for n host-layout 16-vectors v (device, [n][16]) into
 * logits (device, [n][k]); params, mean16, istd16 are device arrays.
 * Asynchronous on `stream`. */
spmv_status spmv_mlp_forward(const float *params, const float *mean16, const float *istd16,
                             int32_t h1, int32_t h2, int32_t k, const float *v, int32_t n,
                             float *logits, spmv_stream_t stream);

/* Mean softmax cross-entropy of the network on standardised inputs z
 * (device, [n][16]) with labels (device int32, [n], in [0, k)), and its
 * gradient with respect to params (device, packed as params).  loss: device,
 * 1 float.  Deterministic (fixed summation order).  Hidden widths <= 128.
 * Allocates (stream-ordered) and frees its own scratch.  Asynchronous. */
spmv_status spmv_mlp_loss_grad(const float *params, int32_t h1, int32_t h2, int32_t k,
                               const float *z, const int32_t *labels, int32_t n, float *grad,
                               float *loss, spmv_stream_t stream);

/* The same loss against a target distribution per sample: q (device,
 * [n][k] float) replaces the labels; loss = mean over samples of
 * -sum_o q_o log softmax(logits)_o.  With q = exp(-beta * log(t_o / t_best))
 * normalised (t_o: measured time of variant o) the loss is cost-sensitive:
 * a slightly slower variant is a small error, a much slower one a large one.
 * Rows of q need not sum to 1 (the gradient is exact for any non-negative
 * weights).  Otherwise as spmv_mlp_loss_grad. */
spmv_status spmv_mlp_loss_grad_soft(const float *params, int32_t h1, int32_t h2, int32_t k,
                                    const float *z, const float *q, int32_t n, float *grad,
                                    float *loss, spmv_stream_t stream);

/* One Adam step on n device floats (step counts from 1):
 *   m = b1 m + (1-b1) g,  v = b2 v + (1-b2) g^2,
 *   p -= lr (m/c1 / (sqrt(v/c2) + eps) + weight_decay p),
 * c1 = 1 - b1^step, c2 = 1 - b2^step, every operation rounded to float. */
spmv_status spmv_mlp_adam(float *params, const float *grad, float *m, float *v, int64_t n,
                          int32_t step, float lr, float beta1, float beta2, float eps,
                          float weight_decay, spmv_stream_t stream);

/* ---- prepare / run ---------------------------------------------------------- */
/* Builds the prepared form of A for c->variant (validating A first unless
 * `trusted` is non-zero), allocating device memory it owns.  Runs on
 * `stream` and synchronizes it.  On failure *out is NULL. */
spmv_status spmv_prepare(const spmv_csr_t *A, const spmv_choice_t *c, int32_t trusted,
                         spmv_prepared_t **out, spmv_stream_t stream);

/* y = A x (Algorithm 1, FP64 accumulation).  x: device [n_cols], y: device
 * [n_rows]; x and y must not overlap.  Asynchronous on `stream`; does not
 * allocate.  A prepared object holds per-call device state (STREAM and
 * MERGE carries, DYNAMIC's work counter and partial sums, SLICED's long-row
 * partials and per-row tickets, FP32 copies of x), so calls on one object
 * must not overlap on the GPU (same stream, or ordered by events); calls on
 * different objects may run concurrently.  The tickets return to 0 at the
 * end of every call that completes. */
spmv_status spmv(const spmv_prepared_t *P, const double *x, double *y, spmv_stream_t stream);

/* End-to-end form of spmv for host vectors: copies x_host [n_cols] to the
 * device, runs spmv, copies y back to y_host [n_rows] and synchronizes
 * `stream`.  Page-locked host buffers give full copy bandwidth.  The device
 * staging vectors are allocated on the first call and owned by P. */
spmv_status spmv_host(spmv_prepared_t *P, const double *x_host, double *y_host,
                      spmv_stream_t stream);

/* spmv_host without the final synchronisation: the copy of x, the SpMV and
 * the copy of y are enqueued on `stream`, and y_host is valid once the
 * stream has been synchronised.  With page-locked x_host and y_host the
 * copies are asynchronous, so calls on different prepared objects issued on
 * different streams overlap: one matrix's upload, another's SpMV and a
 * third's download run at once.  Calls on one prepared object must not
 * overlap (they share its staging buffers). */
spmv_status spmv_host_async(spmv_prepared_t *P, const double *x_host, double *y_host,
                            spmv_stream_t stream);

spmv_status spmv_prepared_info(const spmv_prepared_t *P, spmv_prepared_info_t *info);

/* Copies one owned array of P (see spmv_export) into host memory dst of
 * `bytes` bytes (must equal the array's size; a mismatch fails with
 * SPMV_ERR_INVALID_ARG and a message giving the size).  An empty array is
 * exported with bytes = 0, and dst may then be NULL.  Synchronizes
 * `stream`. */
spmv_status spmv_prepared_export(const spmv_prepared_t *P, int32_t which, void *dst,
                                 int64_t bytes, spmv_stream_t stream);

/* SPMV_ERR_TIMEOUT when a bounded device-side wait of an earlier spmv() on P
 * gave up (that call's y is then incomplete), else SPMV_OK; clears the flag.
 * Synchronizes `stream`. */
spmv_status spmv_prepared_status(const spmv_prepared_t *P, spmv_stream_t stream);

/* ---- batched SpMV -------------------------------------------------------------- */
/* Many matrices of uneven size in one persistent launch.  Each matrix has a
 * launch shape: lanes per row T (power of two, 1..32) and rows per work item
 * (default 8 * 32 / T); the work list is every matrix's row chunks, taken by
 * persistent warps from one atomic counter.  Matrices are borrowed (device
 * CSR, assumed valid); the batch owns its work list and descriptor table. */
typedef struct spmv_batch spmv_batch_t;

/* threads_per_row / rows_per_item: host [count] or NULL (T from the mean row
 * length, rows per item 8 * 32 / T).  Synchronizes `stream`. */
spmv_status spmv_batch_create(const spmv_csr_t *mats, int32_t count,
                              const int32_t *threads_per_row, const int32_t *rows_per_item,
                              spmv_batch_t **out, spmv_stream_t stream);
/* A batch of prepared matrices (borrowed; they must outlive the batch), each
 * run in the persistent form of its own variant inside the one launch: a
 * SLICED matrix with FP64 values as work items of 4 slices, and its long
 * rows as one item per segment of 2048 nonzeros (the segments of rows that
 * span several queued first, then per matrix its slices and its rows of one
 * segment; a row of several segments is summed by the warp
 * that finishes its last one, with the prepared object's per-row tickets,
 * so a batch run must not overlap spmv calls on the same prepared
 * objects); a MERGE or DYNAMIC matrix (imbalance class), or a SLICED
 * one with FP32/BF16 values (the batch sums FP64), as the sliced form with
 * the automatic layout, which the batch prepares and owns (CSR rows would
 * make a warp run as many DFMAs as its longest row); any other variant as
 * CSR row items with its prepared lanes per row.  Synchronizes `stream`. */
spmv_status spmv_batch_create_prepared(const spmv_prepared_t *const *P, int32_t count,
                                       spmv_batch_t **out, spmv_stream_t stream);
/* The same batch with every matrix in the sliced layout: a matrix prepared
 * as SLICED with FP64 values runs its own layout, any other the sliced form
 * with the automatic layout (prepared and owned by the batch).  Inside the
 * shared launch the FP64 pipe is the common bottleneck, and slices spend one
 * DFMA per element with no reductions: on a batch of 512 uneven matrices
 * this ran 1.2x faster than each matrix's own variant. */
spmv_status spmv_batch_create_sliced(const spmv_prepared_t *const *P, int32_t count,
                                     spmv_batch_t **out, spmv_stream_t stream);
/* Sets the vectors: x[m], y[m] are device pointers (host arrays of count
 * pointers).  Must precede spmv_batch_run; synchronizes `stream`. */
spmv_status spmv_batch_bind(spmv_batch_t *B, const double *const *x, double *const *y,
                            spmv_stream_t stream);
/* y[m] = A[m] x[m] for every matrix in one kernel launch.  use_graph != 0:
 * the launch is captured once into a CUDA graph (on the first such call) and
 * the graph is launched on `stream` from then on.  Asynchronous. */
spmv_status spmv_batch_run(spmv_batch_t *B, int32_t use_graph, spmv_stream_t stream);
/* Tunes the launch shapes for the throughput of the whole batch: matrices
 * are grouped by the binary order of their mean row length (SLICED matrices
 * apart, with one lane per row and only the slices per item tuned); coordinate
 * descent over the groups (most nonzeros first, two sweeps) tries lanes per
 * row T in {1, 2, ..., 32}, then rows per item in {2, 4, ..., 32} passes of
 * 32/T rows, timing the whole batch launch (median of reps, 0 = 3) and
 * keeping a change only when it is more than 1 % faster.  Runs the batch
 * (y is overwritten).  Needs a bound batch; invalidates a captured graph.
 * Synchronizes `stream`. */
spmv_status spmv_batch_autotune(spmv_batch_t *B, int32_t reps, spmv_stream_t stream);
/* Current launch shapes (host arrays of count entries; either may be NULL). */
spmv_status spmv_batch_config(const spmv_batch_t *B, int32_t *threads_per_row,
                              int32_t *rows_per_item);
void spmv_batch_free(spmv_batch_t *B);

/* ---- iterative solver ---------------------------------------------------------- */
/* Conjugate gradients for a symmetric positive definite A, the kind of
 * iterative solver in which SpMV's selection cost is amortised (Section 1).
 * A_inner: prepared matrix used for q = A p every iteration (for instance
 * COMPRESSED with FP32 or BF16 values).  A_exact: prepared FP64 form used for
 * r0 = b - A x0 and, every refine_every iterations (> 0), to recompute the
 * residual r = b - A x in FP64, after which the search direction restarts
 * from it (p = r); NULL means A_inner.  Vectors, dot products
 * and scalars are FP64.  b: device [n]; x: device [n], x0 on entry, the
 * iterate on return; resid: device [iters + 1] receiving ||r_t||_2, or NULL.
 * Runs `iters` iterations without a convergence test (no host sync inside the
 * loop); use_graph != 0 captures the whole loop into a CUDA graph and
 * launches it.  Allocates its work vectors (3n doubles) stream-ordered.
 * Asynchronous on `stream`; dot products are deterministic. */
spmv_status spmv_cg(const spmv_prepared_t *A_inner, const spmv_prepared_t *A_exact,
                    const double *b, double *x, int32_t iters, int32_t refine_every,
                    double *resid, int32_t use_graph, spmv_stream_t stream);

/* ---- no-allocation entry point ---------------------------------------------- */
/* The paper has no counterpart of this call; it exists for callers that must
 * not allocate device memory: an iterative solver's inner loop that may never
 * stall the device (cudaMalloc and cudaFree synchronize it), or a host program
 * that commits all device memory through its own allocator at start-up.
 *
 * y = A x with the pipelined STREAM kernel (windows of 2048 nonzeros),
 * asynchronous on `stream`.  It calls no cudaMalloc, cudaFree or allocating
 * routine: its scratch (window starts, carried partial rows, a status word;
 * about 1 MB) is a file-scope __device__ array that every GPU which loads the
 * library keeps until the process exits.
 *   - A: device CSR, assumed valid (this call does not validate it; use
 *     spmv_validate once).  rowptr, colind and val must be 16-byte aligned,
 *     else SPMV_ERR_UNSUPPORTED.  At most 134,217,728 nonzeros (65,536
 *     windows), else SPMV_ERR_UNSUPPORTED before any device work.
 *   - x: device [n_cols], y: device [n_rows], not overlapping.
 *   - The first call on each device looks up the scratch's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call shares the one scratch array and leaves its contents there;
 *     calls whose kernels overlap on the GPU (other streams, other host
 *     threads) race on it and must be serialized by the caller.
 *   - Bounded device waits that give up leave y incomplete (the carry
 *     fix-up then adds nothing); this call never synchronizes, so it does
 *     not report them: spmv_stream_noalloc_status does. */
spmv_status spmv_stream_noalloc(const spmv_csr_t *A, const double *x, double *y,
                                spmv_stream_t stream);

/* Whether the last spmv_stream_noalloc call on the current device finished:
 * SPMV_ERR_TIMEOUT when one of its bounded device waits gave up (its y is
 * then incomplete), else SPMV_OK (also when no call has run).  Reads the
 * scratch's status word into a host variable with cudaMemcpyAsync on
 * `stream` -- the stream of that call -- and synchronizes it; it allocates
 * nothing.  The next spmv_stream_noalloc call clears the word. */
spmv_status spmv_stream_noalloc_status(spmv_stream_t stream);

/* Releases everything P owns (device sync first).  NULL is ignored.  A
 * LATENCY object whose x exceeds half the L2 raised this process's
 * persisting-L2 carve-out when it was prepared; freeing the last such object
 * on the device releases the persisting lines and puts the carve-out back, so
 * that the kernels that run afterwards have the whole L2 again. */
void spmv_prepared_free(spmv_prepared_t *P);

#ifdef __cplusplus
}
#endif

#endif /* PAPER_1511_02494_GB300_SPMV_H */
