/*
 * CPU restatement of the paper's four class-specific SpMV optimizations
 * (Section 3.3, Table 2) and of its unoptimized multithreaded baseline
 * (Section 3.2.1's default partitioning), in C with OpenMP, for the host
 * cores of the GPU machine.
 *
 * BASELINE ONLY.  This is neither the product (the CUDA library) nor the
 * oracle (the plain sequential checker): it exists so that the benchmark can
 * report the paper's own CPU method, on the same matrices, beside the GPU.
 * The CUDA library never loads it.  Portable C: no intrinsics, no inline
 * assembly; __builtin_prefetch and OpenMP pragmas only.
 *
 * Every form computes y = A x with FP64 values and accumulation:
 *   T2_BASE      static 1-D row partition, equal nonzeros per thread
 *                (each thread's first row found by a binary search on
 *                rowptr), plain inner loop;
 *   T2_PREFETCH  CML: the baseline plus one software prefetch of x per
 *                element, pref_dist elements ahead (one cache line of FP64
 *                values by default);
 *   T2_DELTA     MB: column indices delta-coded, 8 or 16 bits per matrix
 *                (never both), in every row whose deltas fit that width; a
 *                row that does not fit keeps its 32-bit columns
 *                (t2_delta_prepare);
 *   T2_DYNAMIC   IMB: rows handed out by OpenMP's dynamic schedule in
 *                chunks of dyn_chunk rows;
 *   T2_SIMD      CMP: the inner loop unrolled by four with four independent
 *                partial sums (the scalar form of a four-wide vector loop:
 *                portable code built without -march, so the compiler emits
 *                no gather instructions).
 * The summation order differs between forms (partial sums, chunks), so
 * results agree with the sequential product to rounding, not bit for bit.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { T2_BASE = 0, T2_PREFETCH = 1, T2_DELTA = 2, T2_DYNAMIC = 3, T2_SIMD = 4 };

int32_t t2_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* first row of thread t under the equal-nonzero partition into nt parts:
 * the smallest row i with rowptr[i] >= floor(t * nnz / nt)                 */
static int64_t part_start(int64_t n_rows, const int32_t *rowptr, int64_t t, int64_t nt)
{
    int64_t target = t * (int64_t)rowptr[n_rows] / nt;
    int64_t lo = 0, hi = n_rows;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (rowptr[mid] < target) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static double row_plain(int64_t b, int64_t e, const int32_t *ci, const double *v, const double *x)
{
    double s = 0.0;
    for (int64_t j = b; j < e; ++j) s += v[j] * x[ci[j]];
    return s;
}

static double row_prefetch(int64_t b, int64_t e, int64_t nnz, const int32_t *ci, const double *v,
                           const double *x, int32_t dist)
{
    double s = 0.0;
    for (int64_t j = b; j < e; ++j) {
        if (j + dist < nnz) __builtin_prefetch(&x[ci[j + dist]], 0, 3);
        s += v[j] * x[ci[j]];
    }
    return s;
}

static double row_simd(int64_t b, int64_t e, const int32_t *ci, const double *v, const double *x)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int64_t j = b;
    for (; j + 3 < e; j += 4) {
        s0 += v[j] * x[ci[j]];
        s1 += v[j + 1] * x[ci[j + 1]];
        s2 += v[j + 2] * x[ci[j + 2]];
        s3 += v[j + 3] * x[ci[j + 3]];
    }
    for (; j < e; ++j) s0 += v[j] * x[ci[j]];
    return (s0 + s1) + (s2 + s3);
}

/* Delta-coded columns (T2_DELTA).  width 1 or 2 bytes.  For a coded row
 * (coded[i] = 1) element j holds column_j - column_{j-1} at delta[j] (the
 * row's first element 0, its column in base[i]); an uncoded row keeps its
 * columns in ci.  The width is the one of 8 and 16 bits under which the
 * matrix's column indices take fewer bytes (8 bits on a tie).  Returns the width; fills the
 * caller's arrays base[n_rows], coded[n_rows], delta[nnz * width].         */
int32_t t2_delta_prepare(int64_t n_rows, const int32_t *rowptr, const int32_t *ci, int32_t *base,
                         uint8_t *coded, void *delta)
{
    int64_t fit8 = 0, fit16 = 0;
#pragma omp parallel for reduction(+ : fit8, fit16) schedule(static)
    for (int64_t i = 0; i < n_rows; ++i) {
        int64_t big = 0;
        for (int64_t j = rowptr[i] + 1; j < rowptr[i + 1]; ++j)
            if (ci[j] - ci[j - 1] > big) big = ci[j] - ci[j - 1];
        int64_t len = rowptr[i + 1] - rowptr[i];
        if (big <= 255) fit8 += len;
        if (big <= 65535) fit16 += len;
    }
    const int64_t nnz = n_rows > 0 ? rowptr[n_rows] : 0;
    const int64_t bytes8 = fit8 + 4 * (nnz - fit8), bytes16 = 2 * fit16 + 4 * (nnz - fit16);
    const int32_t width = bytes8 <= bytes16 ? 1 : 2;
    const int64_t lim = width == 1 ? 255 : 65535;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_rows; ++i) {
        int64_t b = rowptr[i], e = rowptr[i + 1], big = 0;
        for (int64_t j = b + 1; j < e; ++j)
            if (ci[j] - ci[j - 1] > big) big = ci[j] - ci[j - 1];
        coded[i] = (uint8_t)(e > b && big <= lim);
        base[i] = e > b ? ci[b] : 0;
        for (int64_t j = b; j < e; ++j) {
            int32_t d = (j == b || !coded[i]) ? 0 : ci[j] - ci[j - 1];
            if (width == 1) ((uint8_t *)delta)[j] = (uint8_t)d;
            else ((uint16_t *)delta)[j] = (uint16_t)d;
        }
    }
    return width;
}

static double row_delta(int64_t i, int64_t b, int64_t e, const int32_t *ci, const int32_t *base,
                        const uint8_t *coded, const void *delta, int32_t width, const double *v,
                        const double *x)
{
    if (!coded[i]) return row_plain(b, e, ci, v, x);
    double s = 0.0;
    int32_t c = base[i];
    if (width == 1) {
        const uint8_t *d = (const uint8_t *)delta;
        for (int64_t j = b; j < e; ++j) {
            c += d[j];
            s += v[j] * x[c];
        }
    } else {
        const uint16_t *d = (const uint16_t *)delta;
        for (int64_t j = b; j < e; ++j) {
            c += d[j];
            s += v[j] * x[c];
        }
    }
    return s;
}

/* y = A x in form `which`.  base / coded / delta / width: from
 * t2_delta_prepare (T2_DELTA only, else may be NULL / 0).  pref_dist: the
 * prefetch distance in elements (0 = 8).  dyn_chunk: rows per dynamic chunk
 * (0 = 64).  Returns 0, or -1 for an unknown form.                          */
int32_t t2_spmv(int32_t which, int64_t n_rows, const int32_t *rowptr, const int32_t *ci,
                const double *v, const double *x, double *y, const int32_t *base,
                const uint8_t *coded, const void *delta, int32_t width, int32_t pref_dist,
                int32_t dyn_chunk)
{
    if (which < T2_BASE || which > T2_SIMD) return -1;
    const int64_t nnz = n_rows > 0 ? rowptr[n_rows] : 0;
    const int32_t dist = pref_dist > 0 ? pref_dist : 8;
    const int32_t chunk = dyn_chunk > 0 ? dyn_chunk : 64;
    if (which == T2_DYNAMIC) {
#pragma omp parallel for schedule(dynamic, chunk)
        for (int64_t i = 0; i < n_rows; ++i) y[i] = row_plain(rowptr[i], rowptr[i + 1], ci, v, x);
        return 0;
    }
#pragma omp parallel
    {
        int64_t t = 0, nt = 1;
#ifdef _OPENMP
        t = omp_get_thread_num();
        nt = omp_get_num_threads();
#endif
        const int64_t r0 = part_start(n_rows, rowptr, t, nt);
        const int64_t r1 = t + 1 == nt ? n_rows : part_start(n_rows, rowptr, t + 1, nt);
        for (int64_t i = r0; i < r1; ++i) {
            const int64_t b = rowptr[i], e = rowptr[i + 1];
            double s;
            switch (which) {
                case T2_PREFETCH: s = row_prefetch(b, e, nnz, ci, v, x, dist); break;
                case T2_DELTA: s = row_delta(i, b, e, ci, base, coded, delta, width, v, x); break;
                case T2_SIMD: s = row_simd(b, e, ci, v, x); break;
                default: s = row_plain(b, e, ci, v, x);
            }
            y[i] = s;
        }
    }
    return 0;
}
