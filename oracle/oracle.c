/*
 * CPU oracle for the SpMV optimization-selection method of Elafrou, Goumas and
 * Koziris, "A lightweight optimization selection method for Sparse
 * Matrix-Vector Multiplication" (arXiv 1511.02494).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, sequential
 * restatement of what the method computes, used to check the CUDA library.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header or table with the CUDA library.
 *
 * Compiled with -O2 -ffp-contract=off: every floating-point operation below
 * is rounded as written (no fused multiply-add unless fmaf is called).
 *
 * Readings of the paper where it is silent or garbled (numbered O1..O23; the
 * ones that concern a single function are stated beside it):
 *   O1  Algorithm 1 writes an assignment over an inclusive, 1-based range; the
 *       product is read as y_i = sum over the half-open 0-based range
 *       [rowptr_i, rowptr_{i+1}), with y_i = 0 for an empty row.
 *   O2  bw_i = last column - first column of row i; 0 when nnz_i <= 1.
 *   O3  distance_i in disp_i = nnz_i / distance_i is span_i = bw_i + 1.
 *   O4  ngroups_i counts maximal runs of consecutive column indices.
 *   O5  element j (not the first of its row) is a miss when
 *       8 * (c_j - c_{j-1}) > line_bytes; the first element of a non-empty
 *       row always counts as a miss.
 *   O6  miss_ratio is the literal Table 1 formula (1/N) * sum misses_i.
 *   O7  standard deviations are population (1/N) deviations.
 *   O8  size = 1 when bytes(rowptr, colind, val, x, y) <= LLC (here: L2) bytes.
 *   O9-O12 profile rule: speedups sorted descending (ties broken in the
 *       fixed order CML, MB, IMB); the first one strictly above its threshold
 *       names the class; none above -> CMP.  s_inflate = T_inflate / T_base.
 *   O15 empty rows take part in the row statistics with nnz = bw = 0 and
 *       disp = clust = 0.
 *   O23 Table 2's delta coding of column indices (8 or 16 bits) takes, for
 *       the FP64 sliced layout, the offset of each column from its row's
 *       index: 8 bits when every |column - row| in the slices is at most 127,
 *       16 bits when at most 32767.
 *   O24 Table 2's delta coding proper: each column minus the previous
 *       column of its row, the row's first column kept whole; one width per
 *       matrix ("never both"), 8 bits when every delta is at most 255, else
 *       16 bits when at most 65535, else not applicable.
 *   O25 for rows whose deltas exceed 16 bits, a column-blocked form: a
 *       16-bit offset inside a panel of 65536 columns and an 8-bit step
 *       between the panels of consecutive elements.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (Section 2): y = A x over CSR, sequential FP64 accumulation in
 * column order, reading O1.                                                  */
void orc_spmv(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
              const double *val, const double *x, double *y)
{
    for (int64_t i = 0; i < n_rows; ++i) {
        double s = 0.0;
        for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j)
            s = s + val[j] * x[colind[j]];
        y[i] = s;
    }
}

/* Neumaier-compensated row sums (the reference of record for tolerances) and
 * the per-row scale sum_j |a_ij x_j| that the tolerance is relative to.
 * Only the listed rows are computed (all rows when rows == NULL).            */
void orc_spmv_ref(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                  const double *val, const double *x, int64_t n_sel,
                  const int64_t *rows, double *y, double *scale)
{
    int64_t n = rows ? n_sel : n_rows;
    for (int64_t k = 0; k < n; ++k) {
        int64_t i = rows ? rows[k] : k;
        double s = 0.0, c = 0.0, a = 0.0;
        for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) {
            double p = val[j] * x[colind[j]];
            double t = s + p;
            if (fabs(s) >= fabs(p)) c += (s - t) + p;
            else                    c += (p - t) + s;
            s = t;
            a += fabs(p);
        }
        y[k] = s + c;
        scale[k] = a;
    }
}

/* Low-precision stored values, FP64 accumulation (the compressed-value
 * variant of the MB class, Section 3.3 / Table 2).  vkind: 1 = float32,
 * 2 = bfloat16 bit patterns.                                                  */
static double bf16_to_double(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

void orc_spmv_lowp(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                   int32_t vkind, const void *val, const double *x, double *y)
{
    for (int64_t i = 0; i < n_rows; ++i) {
        double s = 0.0;
        for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) {
            double a = vkind == 1 ? (double)((const float *)val)[j]
                                  : bf16_to_double(((const uint16_t *)val)[j]);
            s = s + a * x[colind[j]];
        }
        y[i] = s;
    }
}

/* The same product with FP32 arithmetic: x rounded to float once, every
 * product accumulated by fmaf in column order, the row sum rounded to double
 * (the compressed variant's FP32-accumulation mode).                          */
void orc_spmv_lowp32(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                     int32_t vkind, const void *val, const double *x, double *y)
{
    for (int64_t i = 0; i < n_rows; ++i) {
        float s = 0.0f;
        for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) {
            float a = vkind == 1 ? ((const float *)val)[j]
                                 : (float)bf16_to_double(((const uint16_t *)val)[j]);
            s = fmaf(a, (float)x[colind[j]], s);
        }
        y[i] = (double)s;
    }
}

/* IEEE round-to-nearest-even of a double to bfloat16 (8 significant bits,
 * float32 exponent range), done in one rounding step: scale by a power of two
 * so that one bfloat16 quantum becomes 1, round with nearbyint (ties to even
 * in the default rounding mode), scale back.                                 */
uint16_t orc_round_bf16(double v)
{
    if (isnan(v)) return 0x7FC0;
    double a = fabs(v);
    uint32_t sign = signbit(v) ? 0x8000u : 0u;
    double q;
    if (a == 0.0) {
        q = 0.0;
    } else {
        int e;
        frexp(a, &e);           /* a = m 2^e, m in [0.5, 1): leading bit 2^(e-1) */
        int qexp = e - 8;       /* quantum for 8 significant bits */
        if (qexp < -133) qexp = -133;   /* subnormal bfloat16 quantum 2^-133 */
        q = ldexp(nearbyint(ldexp(a, -qexp)), qexp);
    }
    /* largest finite bfloat16: (2 - 2^-7) 2^127 */
    if (q > ldexp(255.0, 120) || isinf(a)) return (uint16_t)(sign | 0x7F80u);
    float f = (float)q;         /* exact: q has <= 8 significant bits */
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)(sign | ((u >> 16) & 0x7FFFu));
}

void orc_round_bf16_array(int64_t n, const double *v, uint16_t *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_round_bf16(v[i]);
}

void orc_round_f32_array(int64_t n, const double *v, float *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = (float)v[i];
}

/* ------------------------------------------------------------------------ */
/* Table 1 (Section 3.2.2): structural features, as exact integer aggregates
 * first, then the double formulas.                                           */
typedef struct {
    int64_t n_rows, n_cols, nnz, line_bytes, l2_bytes, working_set_bytes;
    int64_t nnz_min, nnz_max;
    uint64_t nnz_sum, nnz_sumsq_lo, nnz_sumsq_hi;
    int64_t bw_min, bw_max;
    uint64_t bw_sum, bw_sumsq_lo, bw_sumsq_hi;
    uint64_t disp_sum, disp_sumsq_lo, disp_sumsq_hi; /* q = floor(2^32 nnz_i/span_i) */
    uint64_t clust_sum;                              /* q = floor(2^32 ngroups_i/nnz_i) */
    uint64_t ngroups_sum, misses_sum;
    double size, density, nnz_avg, nnz_sd, bw_avg, bw_sd;
    double disp_avg, disp_sd, clustering, miss_ratio;
    float vec[16];
} orc_features_t;

/* population sd from exact integer sums: sqrt(N*S2 - S1^2) / N */
static double sd_from_sums(uint64_t n, uint64_t s1, u128 s2)
{
    u128 num = (u128)n * s2 - (u128)s1 * (u128)s1;
    return sqrt((double)num) / (double)n;
}

static float lg1p(double v) { return (float)log2(1.0 + v); }

void orc_features(int64_t n_rows, int64_t n_cols, const int32_t *rowptr,
                  const int32_t *colind, int64_t line_bytes, int64_t l2_bytes,
                  orc_features_t *o)
{
    memset(o, 0, sizeof(*o));
    int64_t nnz = n_rows > 0 ? rowptr[n_rows] : 0;
    o->n_rows = n_rows; o->n_cols = n_cols; o->nnz = nnz;
    o->line_bytes = line_bytes; o->l2_bytes = l2_bytes;
    o->working_set_bytes = 4 * (n_rows + 1) + 12 * nnz + 8 * n_cols + 8 * n_rows;

    u128 nnz_s2 = 0, bw_s2 = 0, disp_s2 = 0;
    o->nnz_min = INT64_MAX; o->bw_min = INT64_MAX;
    o->nnz_max = 0; o->bw_max = 0;
    for (int64_t i = 0; i < n_rows; ++i) {
        int64_t b = rowptr[i], e = rowptr[i + 1];
        int64_t nz = e - b;
        int64_t bw = 0, ngroups = 0, misses = 0;
        uint64_t dq = 0, cq = 0;
        if (nz > 0) {
            bw = (int64_t)colind[e - 1] - (int64_t)colind[b];       /* O2 */
            ngroups = 1; misses = 1;                                /* O4, O5 */
            for (int64_t j = b + 1; j < e; ++j) {
                int64_t d = (int64_t)colind[j] - (int64_t)colind[j - 1];
                if (d != 1) ngroups += 1;
                if (8 * d > line_bytes) misses += 1;
            }
            int64_t span = bw + 1;                                  /* O3 */
            dq = (uint64_t)((((u128)nz) << 32) / (u128)span);
            cq = (uint64_t)((((u128)ngroups) << 32) / (u128)nz);
        }
        if (nz < o->nnz_min) o->nnz_min = nz;
        if (nz > o->nnz_max) o->nnz_max = nz;
        if (bw < o->bw_min) o->bw_min = bw;
        if (bw > o->bw_max) o->bw_max = bw;
        o->nnz_sum += (uint64_t)nz;  nnz_s2 += (u128)nz * (u128)nz;
        o->bw_sum += (uint64_t)bw;   bw_s2 += (u128)bw * (u128)bw;
        o->disp_sum += dq;           disp_s2 += (u128)dq * (u128)dq;
        o->clust_sum += cq;
        o->ngroups_sum += (uint64_t)ngroups;
        o->misses_sum += (uint64_t)misses;
    }
    if (n_rows == 0) { o->nnz_min = 0; o->bw_min = 0; }
    o->nnz_sumsq_lo = (uint64_t)nnz_s2;  o->nnz_sumsq_hi = (uint64_t)(nnz_s2 >> 64);
    o->bw_sumsq_lo = (uint64_t)bw_s2;    o->bw_sumsq_hi = (uint64_t)(bw_s2 >> 64);
    o->disp_sumsq_lo = (uint64_t)disp_s2; o->disp_sumsq_hi = (uint64_t)(disp_s2 >> 64);

    o->size = o->working_set_bytes <= l2_bytes ? 1.0 : 0.0;        /* O8 */
    if (n_rows > 0 && n_cols > 0)
        o->density = (double)nnz / ((double)n_rows * (double)n_cols);
    if (n_rows > 0) {
        const double q32 = 1.0 / 4294967296.0;
        double N = (double)n_rows;
        o->nnz_avg = (double)o->nnz_sum / N;
        o->nnz_sd = sd_from_sums((uint64_t)n_rows, o->nnz_sum, nnz_s2);
        o->bw_avg = (double)o->bw_sum / N;
        o->bw_sd = sd_from_sums((uint64_t)n_rows, o->bw_sum, bw_s2);
        o->disp_avg = ((double)o->disp_sum / N) * q32;
        o->disp_sd = sd_from_sums((uint64_t)n_rows, o->disp_sum, disp_s2) * q32;
        o->clustering = ((double)o->clust_sum / N) * q32;
        o->miss_ratio = (double)o->misses_sum / N;
    }
    /* the 16-entry model input: the 14 Table 1 features (heavy-tailed counts
     * on a log2(1+v) scale) plus log2 N and log2(1+NNZ)                       */
    double dens = o->density > 0x1p-64 ? o->density : 0x1p-64;
    o->vec[0] = (float)o->size;
    o->vec[1] = (float)log2(dens);
    o->vec[2] = lg1p((double)o->nnz_min);
    o->vec[3] = lg1p((double)o->nnz_max);
    o->vec[4] = lg1p(o->nnz_avg);
    o->vec[5] = lg1p(o->nnz_sd);
    o->vec[6] = lg1p((double)o->bw_min);
    o->vec[7] = lg1p((double)o->bw_max);
    o->vec[8] = lg1p(o->bw_avg);
    o->vec[9] = lg1p(o->bw_sd);
    o->vec[10] = (float)o->disp_avg;
    o->vec[11] = (float)o->disp_sd;
    o->vec[12] = (float)o->clustering;
    o->vec[13] = lg1p(o->miss_ratio);
    o->vec[14] = lg1p((double)n_rows);
    o->vec[15] = lg1p((double)nnz);
}

/* ------------------------------------------------------------------------ */
/* Section 3.2.1 profiling-based classifier, readings O9-O12.
 * Classes in the fixed tie order: 0 CML, 1 MB, 2 IMB; 3 CMP when no probe's
 * speedup is strictly above its threshold.  NaN counts as -infinity.  The
 * thresholds are inputs: the paper sets them empirically and prints none.    */
int32_t orc_profile_class(double s_noxmiss, double s_inflate, double s_balance,
                          double tau_noxmiss, double tau_inflate, double tau_balance)
{
    double s[3] = {s_noxmiss, s_inflate, s_balance};
    double tau[3] = {tau_noxmiss, tau_inflate, tau_balance};
    int used[3] = {0, 0, 0};
    for (int rank = 0; rank < 3; ++rank) {
        int best = -1;
        for (int c = 0; c < 3; ++c) {
            if (used[c]) continue;
            double v = isnan(s[c]) ? -INFINITY : s[c];
            double bv = best < 0 ? 0.0 : (isnan(s[best]) ? -INFINITY : s[best]);
            if (best < 0 || v > bv) best = c;   /* strict: ties keep the lower class */
        }
        used[best] = 1;
        if (!isnan(s[best]) && s[best] > tau[best]) return best;
    }
    return 3;
}

/* Table 2: the optimization assigned to each class, as a variant id of the
 * library's enumeration (0 scalar, 1 sub-warp, 2 stream, 3 merge-path,
 * 4 dynamic, 5 latency, 6 compressed, 7 sliced).  map (4 entries, indexed by
 * class) is an input: the paper fixes the classes but its optimizations are
 * CPU techniques, so which GPU variant serves a class is a choice of the
 * caller.  map == NULL takes the paper's own Table 2 row by row:
 *   CML -> software prefetching of x      -> latency (5)
 *   MB  -> delta-coded column indices     -> compressed (6)
 *   IMB -> dynamic / auto scheduling      -> dynamic (4)
 *   CMP -> inner-loop unrolling + SIMD    -> sub-warp (1)
 * An unknown class gives -1.                                                 */
int32_t orc_class_variant(int32_t cls, const int32_t *map)
{
    static const int32_t table2[4] = {5, 6, 4, 1};
    const int32_t *m = map ? map : table2;
    return (cls >= 0 && cls < 4) ? m[cls] : -1;
}

/* ------------------------------------------------------------------------ */
/* Section 3.2.1 default partitioning for the balance benchmark: static 1-D
 * row partition with (as near as possible) equal nonzeros per worker.
 * bounds[w] = smallest row i with rowptr[i] >= floor(w * NNZ / W);
 * bounds[W] = N.  Linear scan.                                               */
void orc_static_partition(int64_t n_rows, const int32_t *rowptr, int64_t n_workers,
                          int64_t *bounds)
{
    int64_t nnz = n_rows > 0 ? rowptr[n_rows] : 0;
    int64_t i = 0;
    for (int64_t w = 0; w < n_workers; ++w) {
        int64_t target = (w * nnz) / n_workers;
        while (i < n_rows && rowptr[i] < target) ++i;
        bounds[w] = i;
    }
    bounds[n_workers] = n_rows;
}

/* Tiers of the dynamic-schedule variant (Table 2's IMB optimization with
 * the rows split by length): rows with lim_s < len <= 64 (m1), with
 * 64 < len <= seg (m2) and with len > seg (lrow), each list in ascending row
 * order; a row of lrow is cut into seg_count = ceil(len / seg) segments.
 * counts[0..2] = the three list lengths.  Rows of at most lim_s nonzeros
 * are in no list (they run in contiguous chunks).                           */
void orc_dyn_tiers(int64_t n_rows, const int32_t *rowptr, int32_t lim_s, int32_t seg,
                   int32_t *m1, int32_t *m2, int32_t *lrow, int32_t *seg_count, int64_t *counts)
{
    int64_t a = 0, b = 0, c = 0;
    for (int64_t i = 0; i < n_rows; ++i) {
        int64_t len = rowptr[i + 1] - rowptr[i];
        if (len <= lim_s) continue;
        if (len <= 64) m1[a++] = (int32_t)i;
        else if (len <= seg) m2[b++] = (int32_t)i;
        else {
            seg_count[c] = (int32_t)((len + seg - 1) / seg);
            lrow[c++] = (int32_t)i;
        }
    }
    counts[0] = a;
    counts[1] = b;
    counts[2] = c;
}

/* Long rows of the sliced layout (reading O22: rows above the cap are left
 * out of the slices and computed from CSR): the rows longer than cap in
 * ascending order (list); each cut into segments of seg nonzeros, seg_off
 * the exclusive running count of segments per long row; per segment its CSR
 * bounds seg_be[2j], seg_be[2j+1]; seg_row[j] its row when it is its row's
 * only segment, else -1; fix the list indices of the rows with several
 * segments (n_fix of them) and seg_fix[j] the index in fix of segment j's
 * row, else -1.  Returns the number of segments.                            */
int64_t orc_sliced_segments(int64_t n_rows, const int32_t *rowptr, int32_t cap, int32_t seg,
                            int32_t *list, int32_t *seg_off, int64_t *seg_be, int32_t *seg_row,
                            int32_t *fix, int32_t *seg_fix, int64_t *n_fix)
{
    int64_t q = 0, j = 0, t = 0;
    seg_off[0] = 0;
    for (int64_t i = 0; i < n_rows; ++i) {
        int64_t b = rowptr[i], e = rowptr[i + 1];
        if (e - b <= cap) continue;
        int64_t k = (e - b + seg - 1) / seg;
        list[q] = (int32_t)i;
        for (int64_t s = 0; s < k; ++s, ++j) {
            seg_be[2 * j] = b + s * seg;
            seg_be[2 * j + 1] = b + (s + 1) * seg < e ? b + (s + 1) * seg : e;
            seg_row[j] = k == 1 ? (int32_t)i : -1;
            seg_fix[j] = k == 1 ? -1 : (int32_t)t;
        }
        if (k > 1) fix[t++] = (int32_t)q;
        seg_off[++q] = (int32_t)j;
    }
    *n_fix = t;
    return j;
}

/* Row blocks for the staged (stream) variant: block k owns the rows whose
 * first nonzero index lies in the window [k B, (k+1) B):
 * R_k = smallest i with rowptr[i] >= k B, R_{n_blocks} = N.  Linear scan.   */
void orc_row_blocks(int64_t n_rows, const int32_t *rowptr, int64_t block_nnz,
                    int64_t n_blocks, int32_t *out)
{
    int64_t i = 0;
    for (int64_t k = 0; k < n_blocks; ++k) {
        int64_t target = k * block_nnz;
        while (i < n_rows && rowptr[i] < target) ++i;
        out[k] = (int32_t)i;
    }
    out[n_blocks] = (int32_t)n_rows;
}

/* Merge-path coordinates for the balanced variant: the path merges the row
 * ends rowptr[1..N] with the nonzero indices 0..NNZ-1; one step consumes the
 * end of row i when all of its nonzeros have been consumed
 * (rowptr[i+1] <= j), otherwise nonzero j.  Part p starts at diagonal
 * d = min(p * items, N + NNZ).  Brute-force walk.                            */
void orc_merge_path(int64_t n_rows, const int32_t *rowptr, int64_t items,
                    int64_t n_parts, int32_t *row_start, int32_t *nz_start)
{
    int64_t nnz = n_rows > 0 ? rowptr[n_rows] : 0;
    int64_t total = n_rows + nnz;
    int64_t i = 0, j = 0, d = 0;
    for (int64_t p = 0; p <= n_parts; ++p) {
        int64_t target = p * items < total ? p * items : total;
        while (d < target) {
            if (i < n_rows && (j >= nnz || rowptr[i + 1] <= j)) ++i;
            else ++j;
            ++d;
        }
        row_start[p] = (int32_t)i;
        nz_start[p] = (int32_t)j;
    }
}

/* MB-class compression (Section 3.3, Table 2: column-index compression),
 * GPU reading O13: each row stores its first column in rowbase and every
 * column as a 16-bit offset from it when bw_i < 65536.  Wider rows keep
 * their 32-bit columns and get rowbase = -1.  Empty rows: rowbase = 0.
 * Returns the number of wide rows.                                           */
int64_t orc_compress_u16(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                         int32_t *rowbase, uint16_t *off)
{
    int64_t wide = 0;
    for (int64_t i = 0; i < n_rows; ++i) {
        int64_t b = rowptr[i], e = rowptr[i + 1];
        if (e == b) { rowbase[i] = 0; continue; }
        int64_t first = colind[b];
        if ((int64_t)colind[e - 1] - first >= 65536) {
            rowbase[i] = -1;
            ++wide;
            for (int64_t j = b; j < e; ++j) off[j] = 0;
        } else {
            rowbase[i] = (int32_t)first;
            for (int64_t j = b; j < e; ++j) off[j] = (uint16_t)(colind[j] - first);
        }
    }
    return wide;
}

/* ------------------------------------------------------------------------ */
/* Sliced layout of the SLICED variant (a GPU format for the MB and CML
 * classes: 32 rows per slice, elements stored column-major inside a slice so
 * that one lane per row reads coalesced).
 *   positions: rows in order when sigma == 1; otherwise, inside each window
 *   of sigma consecutive rows, rows sorted by key length descending, ties by
 *   row index ascending, where a row longer than `cap` has key length 0.
 *   rowlen[p]: length of the row at position p, -1 for a long row (> cap) or
 *   a position past the last row (positions run to 32 * S, S = ceil(N/32)).
 *   slice_len[s] = max(0, max rowlen over positions 32s .. 32s+31).
 *   slice_ptr[0] = 0, slice_ptr[s+1] = slice_ptr[s] + 32 * slice_len[s]
 *   rounded up to a multiple of vec.
 * With vec elements of a row side by side (vec = 1, 2 or 4), the element k
 * of the row at position p = 32s + l lives at
 * slice_ptr[s] + 32 vec floor(k / vec) + vec l + (k mod vec)
 * (for vec = 1: slice_ptr[s] + 32 k + l).  Returns the number of long rows.  */
static const int32_t *g_sort_rowptr;
static int32_t g_sort_cap;

static int32_t key_len(int64_t i)
{
    int64_t len = g_sort_rowptr[i + 1] - g_sort_rowptr[i];
    return len > g_sort_cap ? 0 : (int32_t)len;
}

static int cmp_rows(const void *a, const void *b)
{
    int32_t ra = *(const int32_t *)a, rb = *(const int32_t *)b;
    int32_t la = key_len(ra), lb = key_len(rb);
    if (la != lb) return la > lb ? -1 : 1;
    return ra < rb ? -1 : (ra > rb ? 1 : 0);
}

int64_t orc_sliced_layout(int64_t n_rows, const int32_t *rowptr, int32_t sigma, int32_t cap,
                          int32_t vec, int32_t *perm, int32_t *rowlen, int32_t *slice_len,
                          int64_t *slice_ptr)
{
    int64_t n_slices = (n_rows + 31) / 32, n_long = 0;
    for (int64_t i = 0; i < n_rows; ++i) perm[i] = (int32_t)i;
    if (sigma > 1) {
        g_sort_rowptr = rowptr;
        g_sort_cap = cap;
        for (int64_t w = 0; w < n_rows; w += sigma) {
            int64_t cnt = n_rows - w < sigma ? n_rows - w : sigma;
            qsort(perm + w, (size_t)cnt, sizeof(int32_t), cmp_rows);
        }
    }
    for (int64_t p = 0; p < 32 * n_slices; ++p) {
        if (p >= n_rows) { rowlen[p] = -1; continue; }
        int64_t r = perm[p];
        int64_t len = rowptr[r + 1] - rowptr[r];
        if (len > cap) { rowlen[p] = -1; ++n_long; }
        else rowlen[p] = (int32_t)len;
    }
    slice_ptr[0] = 0;
    for (int64_t s = 0; s < n_slices; ++s) {
        int32_t m = 0;
        for (int64_t l = 0; l < 32; ++l)
            if (rowlen[32 * s + l] > m) m = rowlen[32 * s + l];
        slice_len[s] = m;
        slice_ptr[s + 1] = slice_ptr[s] + 32 * (int64_t)((m + vec - 1) / vec * vec);
    }
    return n_long;
}

/* Column-major slice contents: col/val at slice_ptr[s] + 32 k + l for k <
 * rowlen[32s + l]; every other slot is 0.                                     */
static int64_t slot_of(const int64_t *slice_ptr, int64_t p, int64_t k, int32_t vec)
{
    return slice_ptr[p / 32] + 32 * vec * (k / vec) + vec * (p % 32) + k % vec;
}

void orc_sliced_fill(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                     const double *val, const int32_t *perm, const int32_t *rowlen,
                     const int64_t *slice_ptr, int32_t vec, int32_t *col_out, double *val_out)
{
    int64_t n_slices = (n_rows + 31) / 32;
    int64_t tot = slice_ptr[n_slices];
    for (int64_t q = 0; q < tot; ++q) { col_out[q] = 0; val_out[q] = 0.0; }
    for (int64_t p = 0; p < n_rows; ++p) {
        if (rowlen[p] < 0) continue;
        int64_t b = rowptr[perm[p]];
        for (int64_t k = 0; k < rowlen[p]; ++k) {
            col_out[slot_of(slice_ptr, p, k, vec)] = colind[b + k];
            val_out[slot_of(slice_ptr, p, k, vec)] = val[b + k];
        }
    }
}

/* 16-bit form of the sliced layout's columns (reading O13 on slices): the
 * row at position p has base rowbase_pos[p] = its first column (0 for an
 * empty row, a long row or a position past the last row), and every slot of
 * it holds col - base; padding slots hold 0.  Returns the largest span
 * (last - first column) over the rows in slices; offsets are meaningful only
 * when it is below 65536.                                                     */
/* Column offsets from the row index for the FP64 sliced layout (reading
 * O23): d = column - row at every element's slot (vec = 1 placement), 0 in
 * padding, and the largest |d| over the rows in the slices.  The library
 * keeps d in 8 bits when that largest |d| is at most 127, in 16 bits when at
 * most 32767, and 32-bit columns otherwise (orc_sliced_index_bytes).          */
int64_t orc_sliced_diag(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                        const int32_t *perm, const int32_t *rowlen, const int64_t *slice_ptr,
                        int32_t *d_out)
{
    int64_t n_slices = (n_rows + 31) / 32, reach = 0;
    int64_t tot = slice_ptr[n_slices];
    for (int64_t q = 0; q < tot; ++q) d_out[q] = 0;
    for (int64_t p = 0; p < 32 * n_slices; ++p) {
        if (p >= n_rows || rowlen[p] <= 0) continue;
        int64_t r = perm[p], b = rowptr[r];
        for (int64_t k = 0; k < rowlen[p]; ++k) {
            int64_t d = (int64_t)colind[b + k] - r;
            d_out[slot_of(slice_ptr, p, k, 1)] = (int32_t)d;
            if (d > reach) reach = d;
            if (-d > reach) reach = -d;
        }
    }
    return reach;
}

int32_t orc_sliced_index_bytes(int64_t reach)
{
    return reach <= 127 ? 1 : (reach <= 32767 ? 2 : 4);
}

/* Table 2's delta coding of column indices for the FP64 sliced layout
 * (reading O24): every column of a row is kept as its difference from the
 * previous column of the same row, and the row's first column as an
 * absolute base at its position.  d_out: the delta at each element's slot
 * (vec = 1 placement), 0 for a row's first element and in padding;
 * rowbase_pos: the first column per position, 0 where no row sits in the
 * slices.  Returns the largest delta over the rows in the slices (0 when no
 * row has two elements).                                                     */
int64_t orc_sliced_delta(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                         const int32_t *perm, const int32_t *rowlen, const int64_t *slice_ptr,
                         int32_t *rowbase_pos, int32_t *d_out)
{
    int64_t n_slices = (n_rows + 31) / 32, largest = 0;
    int64_t tot = slice_ptr[n_slices];
    for (int64_t q = 0; q < tot; ++q) d_out[q] = 0;
    for (int64_t p = 0; p < 32 * n_slices; ++p) {
        rowbase_pos[p] = 0;
        if (p >= n_rows || rowlen[p] <= 0) continue;
        int64_t b = rowptr[perm[p]];
        rowbase_pos[p] = colind[b];
        for (int64_t k = 1; k < rowlen[p]; ++k) {
            int64_t d = (int64_t)colind[b + k] - colind[b + k - 1];
            d_out[slot_of(slice_ptr, p, k, 1)] = (int32_t)d;
            if (d > largest) largest = d;
        }
    }
    return largest;
}

/* Section 3.3's delta width, one width only (8 or 16 bits, not a mix), per
 * matrix: 1 byte when every delta is at most 255, 2 when at most 65535, 0
 * when some delta needs more (the delta coding does not apply).               */
int32_t orc_delta_bytes(int64_t largest_delta)
{
    return largest_delta <= 255 ? 1 : (largest_delta <= 65535 ? 2 : 0);
}

/* Column-blocked form of the FP64 sliced layout's columns, for rows whose
 * deltas do not fit 16 bits (reading O25): the column space is cut into
 * panels of 65536 columns; each element keeps its offset inside its panel
 * (column mod 65536) and the step from the previous element's panel to its
 * own (the first element's from panel 0).  lo_out and step_out at each
 * element's slot, 0 in padding.  Returns the largest step over the rows in
 * the slices; the form applies when it is at most 255 (8 bits).             */
int64_t orc_sliced_panel(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                         const int32_t *perm, const int32_t *rowlen, const int64_t *slice_ptr,
                         uint16_t *lo_out, int32_t *step_out)
{
    int64_t n_slices = (n_rows + 31) / 32, largest = 0;
    int64_t tot = slice_ptr[n_slices];
    for (int64_t q = 0; q < tot; ++q) {
        lo_out[q] = 0;
        step_out[q] = 0;
    }
    for (int64_t p = 0; p < 32 * n_slices; ++p) {
        if (p >= n_rows || rowlen[p] <= 0) continue;
        int64_t b = rowptr[perm[p]], panel = 0;
        for (int64_t k = 0; k < rowlen[p]; ++k) {
            int64_t c = colind[b + k];
            int64_t step = c / 65536 - panel;
            panel = c / 65536;
            lo_out[slot_of(slice_ptr, p, k, 1)] = (uint16_t)(c % 65536);
            step_out[slot_of(slice_ptr, p, k, 1)] = (int32_t)step;
            if (step > largest) largest = step;
        }
    }
    return largest;
}

int64_t orc_sliced_offsets(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                           const int32_t *perm, const int32_t *rowlen, const int64_t *slice_ptr,
                           int32_t vec, int32_t *rowbase_pos, uint16_t *off_out)
{
    int64_t n_slices = (n_rows + 31) / 32, span = 0;
    int64_t tot = slice_ptr[n_slices];
    for (int64_t q = 0; q < tot; ++q) off_out[q] = 0;
    for (int64_t p = 0; p < 32 * n_slices; ++p) {
        rowbase_pos[p] = 0;
        if (p >= n_rows || rowlen[p] <= 0) continue;
        int64_t b = rowptr[perm[p]], len = rowlen[p];
        int64_t first = colind[b];
        rowbase_pos[p] = (int32_t)first;
        if (colind[b + len - 1] - first > span) span = colind[b + len - 1] - first;
        for (int64_t k = 0; k < len; ++k)
            off_out[slot_of(slice_ptr, p, k, vec)] = (uint16_t)(colind[b + k] - first);
    }
    return span;
}

/* ------------------------------------------------------------------------ */
/* Learned selector: fully connected 16 -> H1 -> H2 -> K network with ReLU.
 * Input standardisation z_k = (v_k - mean_k) * istd_k, each product and
 * difference rounded to float.  Every dot product is a chain of fmaf calls
 * starting from the bias, inputs in ascending order; that fixed order makes
 * the logits reproducible bit for bit.  Weights are row-major [out][in].     */
void orc_mlp_forward_f32(int32_t h1, int32_t h2, int32_t k,
                         const float *mean, const float *istd,
                         const float *W1, const float *b1, const float *W2, const float *b2,
                         const float *W3, const float *b3, const float *v, float *logits)
{
    float z[16], a1[256], a2[256];
    for (int i = 0; i < 16; ++i) z[i] = (v[i] - mean[i]) * istd[i];
    for (int o = 0; o < h1; ++o) {
        float acc = b1[o];
        for (int i = 0; i < 16; ++i) acc = fmaf(W1[o * 16 + i], z[i], acc);
        a1[o] = acc > 0.0f ? acc : 0.0f;
    }
    for (int o = 0; o < h2; ++o) {
        float acc = b2[o];
        for (int i = 0; i < h1; ++i) acc = fmaf(W2[o * h1 + i], a1[i], acc);
        a2[o] = acc > 0.0f ? acc : 0.0f;
    }
    for (int o = 0; o < k; ++o) {
        float acc = b3[o];
        for (int i = 0; i < h2; ++i) acc = fmaf(W3[o * h2 + i], a2[i], acc);
        logits[o] = acc;
    }
}

/* argmax with ties to the lowest index; margin = best - second best logit. */
int32_t orc_argmax(int32_t k, const float *logits, float *margin)
{
    int32_t b = 0;
    for (int32_t o = 1; o < k; ++o) if (logits[o] > logits[b]) b = o;
    float second = -INFINITY;
    for (int32_t o = 0; o < k; ++o) if (o != b && logits[o] > second) second = logits[o];
    *margin = k > 1 ? logits[b] - second : INFINITY;
    return b;
}

/* FP64 forward + backward of the mean softmax cross-entropy over a batch,
 * given standardized inputs z[B][16] and labels.  Gradients are written to
 * g* (same layouts as the weights); returns the loss.  Textbook
 * backpropagation, written out loop by loop.                                  */
/* Shared by the hard-label and soft-target forms: with q == NULL the target
 * of sample s is the one-hot vector of label[s]; otherwise it is the row
 * q[s*k .. s*k+k-1].  Loss per sample: -sum_o q_o log p_o with p = softmax
 * of the logits; its derivative with respect to logit o is p_o * S - q_o,
 * S = sum_o q_o (S = 1 for a distribution). */
static double mlp_loss_grad(int32_t h1, int32_t h2, int32_t k, int32_t batch,
                            const double *W1, const double *b1, const double *W2,
                            const double *b2, const double *W3, const double *b3,
                            const double *z, const int32_t *label, const double *q,
                            double *gW1, double *gb1, double *gW2, double *gb2,
                            double *gW3, double *gb3)
{
    memset(gW1, 0, sizeof(double) * h1 * 16); memset(gb1, 0, sizeof(double) * h1);
    memset(gW2, 0, sizeof(double) * h2 * h1); memset(gb2, 0, sizeof(double) * h2);
    memset(gW3, 0, sizeof(double) * k * h2);  memset(gb3, 0, sizeof(double) * k);
    double loss = 0.0;
    double a1[256], a2[256], p[256], d1[256], d2[256];
    for (int32_t s = 0; s < batch; ++s) {
        const double *x = z + (int64_t)s * 16;
        for (int o = 0; o < h1; ++o) {
            double acc = b1[o];
            for (int i = 0; i < 16; ++i) acc += W1[o * 16 + i] * x[i];
            a1[o] = acc > 0 ? acc : 0;
        }
        for (int o = 0; o < h2; ++o) {
            double acc = b2[o];
            for (int i = 0; i < h1; ++i) acc += W2[o * h1 + i] * a1[i];
            a2[o] = acc > 0 ? acc : 0;
        }
        double mx = -INFINITY;
        for (int o = 0; o < k; ++o) {
            double acc = b3[o];
            for (int i = 0; i < h2; ++i) acc += W3[o * h2 + i] * a2[i];
            p[o] = acc;
            if (acc > mx) mx = acc;
        }
        double den = 0.0;
        for (int o = 0; o < k; ++o) den += exp(p[o] - mx);
        const double lse = mx + log(den);  /* log sum_o exp(logit_o) */
        double tq[256], S = 0.0;
        for (int o = 0; o < k; ++o) {
            tq[o] = q ? q[(int64_t)s * k + o] : (o == label[s] ? 1.0 : 0.0);
            S += tq[o];
        }
        for (int o = 0; o < k; ++o) loss += -tq[o] * (p[o] - lse);  /* log p_o = logit_o - lse */
        /* dL/dlogit = (p S - q) / B */
        for (int o = 0; o < k; ++o) p[o] = (exp(p[o] - lse) * S - tq[o]) / batch;
        for (int i = 0; i < h2; ++i) d2[i] = 0.0;
        for (int o = 0; o < k; ++o) {
            gb3[o] += p[o];
            for (int i = 0; i < h2; ++i) { gW3[o * h2 + i] += p[o] * a2[i]; d2[i] += W3[o * h2 + i] * p[o]; }
        }
        for (int i = 0; i < h2; ++i) if (a2[i] <= 0) d2[i] = 0.0;
        for (int i = 0; i < h1; ++i) d1[i] = 0.0;
        for (int o = 0; o < h2; ++o) {
            gb2[o] += d2[o];
            for (int i = 0; i < h1; ++i) { gW2[o * h1 + i] += d2[o] * a1[i]; d1[i] += W2[o * h1 + i] * d2[o]; }
        }
        for (int i = 0; i < h1; ++i) if (a1[i] <= 0) d1[i] = 0.0;
        for (int o = 0; o < h1; ++o) {
            gb1[o] += d1[o];
            for (int i = 0; i < 16; ++i) gW1[o * 16 + i] += d1[o] * x[i];
        }
    }
    return loss / batch;
}

/* Mean softmax cross-entropy over a batch with integer labels and its
 * gradient by backpropagation, in FP64. */
double orc_mlp_loss_grad_f64(int32_t h1, int32_t h2, int32_t k, int32_t batch,
                             const double *W1, const double *b1, const double *W2,
                             const double *b2, const double *W3, const double *b3,
                             const double *z, const int32_t *label,
                             double *gW1, double *gb1, double *gW2, double *gb2,
                             double *gW3, double *gb3)
{
    return mlp_loss_grad(h1, h2, k, batch, W1, b1, W2, b2, W3, b3, z, label, NULL,
                         gW1, gb1, gW2, gb2, gW3, gb3);
}

/* The same with a target distribution per sample (q: batch x k, row-major):
 * cross-entropy against soft targets, used to make training cost-sensitive. */
double orc_mlp_loss_grad_soft_f64(int32_t h1, int32_t h2, int32_t k, int32_t batch,
                                  const double *W1, const double *b1, const double *W2,
                                  const double *b2, const double *W3, const double *b3,
                                  const double *z, const double *q,
                                  double *gW1, double *gb1, double *gW2, double *gb2,
                                  double *gW3, double *gb3)
{
    return mlp_loss_grad(h1, h2, k, batch, W1, b1, W2, b2, W3, b3, z, NULL, q,
                         gW1, gb1, gW2, gb2, gW3, gb3);
}

/* One Adam step in float, each operation rounded as written:
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;
 *   p = p - lr (m / c1 / (sqrt(v / c2) + eps) + wd p),  c1 = 1 - b1^t, c2 = 1 - b2^t
 * with c1, c2 given (computed once per step by the caller).                 */
void orc_adam_f32(int64_t n, float *p, const float *g, float *m, float *v, float lr, float b1,
                  float b2, float eps, float wd, float c1, float c2)
{
    for (int64_t i = 0; i < n; ++i) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.0f - b1) * gi;
        float vi = b2 * v[i] + (1.0f - b2) * (gi * gi);
        m[i] = mi;
        v[i] = vi;
        float mh = mi / c1, vh = vi / c2;
        p[i] = p[i] - lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
    }
}

/* ------------------------------------------------------------------------ */
/* Conjugate gradients (Hestenes-Stiefel), the iterative solver the paper's
 * SpMV serves (Section 1), in FP64 with sequential dot products.  When
 * vkind != 0 the inner product A p uses the low-precision stored values
 * lowval (1 = float32, 2 = bfloat16) and, every `refine` iterations (> 0),
 * the residual is recomputed as r = b - A x with the FP64 values and the
 * search direction restarts from it (p = r).
 * resid[t] = ||r_t||_2 after iteration t (t = 0 is the initial residual).
 * x holds x0 on entry.  Work arrays r, p, q have n entries each.             */
static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = s + a[i] * b[i];
    return s;
}

void orc_cg(int64_t n, const int32_t *rowptr, const int32_t *colind, const double *val,
            int32_t vkind, const void *lowval, int32_t refine,
            const double *b, double *x, int32_t iters, double *resid,
            double *r, double *p, double *q)
{
    orc_spmv(n, rowptr, colind, val, x, q);
    for (int64_t i = 0; i < n; ++i) { r[i] = b[i] - q[i]; p[i] = r[i]; }
    double rs = dot(n, r, r);
    resid[0] = sqrt(rs);
    for (int32_t t = 1; t <= iters; ++t) {
        if (vkind == 0) orc_spmv(n, rowptr, colind, val, p, q);
        else orc_spmv_lowp(n, rowptr, colind, vkind, lowval, p, q);
        double pq = dot(n, p, q);
        double alpha = rs / pq;
        for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
        int restart = vkind != 0 && refine > 0 && t % refine == 0;
        if (restart) {
            orc_spmv(n, rowptr, colind, val, x, q);
            for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
        } else {
            for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
        }
        double rs_new = dot(n, r, r);
        /* after the residual is recomputed the search restarts from it */
        double beta = restart ? 0.0 : rs_new / rs;
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rs = rs_new;
        resid[t] = sqrt(rs);
    }
}
