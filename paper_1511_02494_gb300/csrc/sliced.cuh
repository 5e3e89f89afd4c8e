// Device side of the sliced layout (SLICED variant), shared by its kernels,
// the batched kernel and the fused CG kernel.
//
// One 32-row slice: lane l sums the row at position p = 32 s + l, element k
// of which sits at slot slice_ptr[s] + 32 k + l, as one FMA chain in row
// order; loads and FMAs past the row's length are predicated off.
// rowlen[p] < 0 marks a position without a row (a long row computed
// elsewhere, or past the last row): *row is then -1.
#pragma once

#include <cuda_bf16.h>

#include "rowdot.cuh"

namespace spmvlib {
namespace dev {

// FP64 values.  The column of a slot is stored as CT: int (the column
// itself), or int16_t / int8_t (the column minus the row index: Table 2's
// 8- and 16-bit compression of column indices, decoded with one add).
template <typename CT>
__device__ __forceinline__ int column_of(CT stored, int row)
{
    if constexpr (sizeof(CT) == 4) return (int)stored;
    else return row + (int)stored;
}

template <int U, typename CT = int>
__device__ __forceinline__ double slice_value(int64_t s, int lane, const int* __restrict__ rowlen,
                                              const int* __restrict__ slice_len,
                                              const int64_t* __restrict__ slice_ptr,
                                              const int* __restrict__ perm,
                                              const CT* __restrict__ col,
                                              const double* __restrict__ val,
                                              const double* __restrict__ x, int* row)
{
    const int64_t p = s * 32 + lane;
    const int len = rowlen[p];
    const int L = slice_len[s];
    const int64_t q0 = slice_ptr[s] + lane;
    const CT* __restrict__ cp = col + q0;       // element k at cp[32 k]
    const double* __restrict__ vp = val + q0;
    // offsets from the row index need the row before the gathers; 32-bit
    // columns look it up after the loop, off the loads' critical path
    int r = -1;
    if constexpr (sizeof(CT) != 4) r = len >= 0 ? (perm ? perm[p] : (int)p) : -1;
    double acc = 0.0;
    for (int k = 0; k < L; k += U) {
        int c[U];
        double a[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = k + u < len;
            c[u] = ok ? column_of(__ldcs(cp + (k + u) * 32), r) : 0;
            a[u] = ok ? __ldcs(vp + (k + u) * 32) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) xv[u] = k + u < len ? ldx(x + c[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k + u < len) acc = fma(a[u], xv[u], acc);
    }
    if constexpr (sizeof(CT) == 4) r = len >= 0 ? (perm ? perm[p] : (int)p) : -1;
    *row = r;
    return acc;
}

template <int U, typename CT = int>
__device__ __forceinline__ void slice_rows(int64_t s, int lane, const int* __restrict__ rowlen,
                                           const int* __restrict__ slice_len,
                                           const int64_t* __restrict__ slice_ptr,
                                           const int* __restrict__ perm,
                                           const CT* __restrict__ col,
                                           const double* __restrict__ val,
                                           const double* __restrict__ x, double* __restrict__ y)
{
    int row;
    const double v = slice_value<U, CT>(s, lane, rowlen, slice_len, slice_ptr, perm, col, val, x, &row);
    if (row >= 0) y[row] = v;
}

// R consecutive slices s0 .. s0 + R - 1 at once: the lane sums one row of
// each (the same FMA chain per row as slice_value), with U elements of every
// row in flight, so a warp overlaps the R slices' load latencies.  Slices
// past n_slices are skipped.
template <int U, int R, typename CT = int>
__device__ __forceinline__ void slice_rows_multi(int64_t s0, int64_t n_slices, int lane,
                                                 const int* __restrict__ rowlen,
                                                 const int* __restrict__ slice_len,
                                                 const int64_t* __restrict__ slice_ptr,
                                                 const int* __restrict__ perm,
                                                 const CT* __restrict__ col,
                                                 const double* __restrict__ val,
                                                 const double* __restrict__ x, double* __restrict__ y)
{
    int len[R], row[R];
    int64_t q0[R];
    double acc[R];
    int L = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t s = s0 + r;
        const bool in = s < n_slices;
        const int64_t p = s * 32 + lane;
        len[r] = in ? rowlen[p] : -1;
        q0[r] = in ? slice_ptr[s] + lane : 0;
        L = max(L, in ? slice_len[s] : 0);
        row[r] = len[r] >= 0 ? (perm ? perm[p] : (int)p) : -1;
        acc[r] = 0.0;
    }
    for (int k = 0; k < L; k += U) {
        int c[R][U];
        double a[R][U], xv[R][U];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = k + u < len[r];
                c[r][u] = ok ? column_of(__ldcs(col + q0[r] + (k + u) * 32), row[r]) : 0;
                a[r][u] = ok ? __ldcs(val + q0[r] + (k + u) * 32) : 0.0;
            }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int u = 0; u < U; ++u) xv[r][u] = k + u < len[r] ? ldx(x + c[r][u]) : 0.0;
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (k + u < len[r]) acc[r] = fma(a[r][u], xv[r][u], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (row[r] >= 0) y[row[r]] = acc[r];
}

// Slices s0 .. s0 + R - 1 of a layout whose rows all have length L, in
// order, none long (an ELLPACK matrix): slice s starts at 32 L s and holds
// rows 32 s .. 32 s + 31, so no slice header (row lengths, slice length and
// start) is read -- one dependent round trip less per slice.  The lane sums
// one row of each slice with the same FMA chain as slice_value, U elements
// of every row in flight; slices at or past s_end and rows at or past n_rows
// are skipped.
template <int U, int R, typename CT = int>
__device__ __forceinline__ void uniform_rows(int64_t s0, int64_t s_end, int64_t n_rows, int L, int lane,
                                             const CT* __restrict__ col, const double* __restrict__ val,
                                             const double* __restrict__ x, double* __restrict__ y)
{
    int64_t q0[R];
    int row[R];
    bool in[R];
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t p = (s0 + r) * 32 + lane;
        in[r] = s0 + r < s_end && p < n_rows;
        row[r] = in[r] ? (int)p : 0;
        q0[r] = (s0 + r) * 32 * (int64_t)L + lane;
        acc[r] = 0.0;
    }
    for (int k = 0; k < L; k += U) {
        int c[R][U];
        double a[R][U], xv[R][U];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = in[r] && k + u < L;
                c[r][u] = ok ? column_of(__ldcs(col + q0[r] + (int64_t)(k + u) * 32), row[r]) : 0;
                a[r][u] = ok ? __ldcs(val + q0[r] + (int64_t)(k + u) * 32) : 0.0;
            }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int u = 0; u < U; ++u) xv[r][u] = in[r] && k + u < L ? ldx(x + c[r][u]) : 0.0;
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (in[r] && k + u < L) acc[r] = fma(a[r][u], xv[r][u], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (in[r]) y[row[r]] = acc[r];
}

// FP64 values with coded columns.  A lane walks its row in order, so a
// column is decoded from the one before it with integer operations:
//   MODE 1, Table 2's delta coding: cs (DT = uint8_t or uint16_t) holds the
//     column minus the previous column of the row (0 for the row's first
//     element), rowbase[p] the row's first column;
//   MODE 2, the column-blocked form: cs (uint16_t) holds the column modulo
//     65536, step the step from the previous element's 65536-column panel
//     (the first element's from panel 0).
// Otherwise as slice_value: U elements of the row in flight, one DFMA chain.
template <int U, int MODE, typename DT>
__device__ __forceinline__ double slice_value_coded(int64_t s, int lane, const int* __restrict__ rowlen,
                                                    const int* __restrict__ slice_len,
                                                    const int64_t* __restrict__ slice_ptr,
                                                    const int* __restrict__ perm,
                                                    const DT* __restrict__ cs,
                                                    const uint8_t* __restrict__ step,
                                                    const int* __restrict__ rowbase,
                                                    const double* __restrict__ val,
                                                    const double* __restrict__ x, int* row)
{
    const int64_t p = s * 32 + lane;
    const int len = rowlen[p];
    const int L = slice_len[s];
    const int64_t q0 = slice_ptr[s] + lane;
    const DT* __restrict__ dp = cs + q0;
    const double* __restrict__ vp = val + q0;
    int c = 0;  // MODE 1: the running column; MODE 2: the running panel << 16
    if constexpr (MODE == 1) c = rowbase[p];
    double acc = 0.0;
    for (int k = 0; k < L; k += U) {
        int cc[U];
        double a[U], xv[U];
        int lo[U], hi[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = k + u < len;
            lo[u] = ok ? (int)__ldcs(dp + (k + u) * 32) : 0;
            if constexpr (MODE == 2) hi[u] = ok ? (int)__ldcs(step + q0 + (k + u) * 32) : 0;
            a[u] = ok ? __ldcs(vp + (k + u) * 32) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if constexpr (MODE == 1) {
                c += lo[u];
                cc[u] = c;
            } else {
                c += hi[u] << 16;
                cc[u] = c | lo[u];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) xv[u] = k + u < len ? ldx(x + cc[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k + u < len) acc = fma(a[u], xv[u], acc);
    }
    *row = len >= 0 ? (perm ? perm[p] : (int)p) : -1;
    return acc;
}

// FP32 or BF16 values, 32-bit columns or 16-bit offsets from rowbase[p],
// with four elements of a row side by side: element k of the row at
// position p = 32 s + l sits at slot slice_ptr[s] + 128 (k / 4) + 4 l + k % 4,
// so one lane loads four offsets (8 bytes) and four values (8 or 16 bytes)
// per instruction.  ACC32: x32 is the FP32 copy of x; fmaf chain in row
// order, one widening per row.  Otherwise each value is widened to FP64 with
// integer operations (widen_f32, no FP64 instruction) and summed with DFMAs.  Padded slots are loaded with their group but never
// multiplied.
__device__ __forceinline__ void load4(const __nv_bfloat16* p, float* a) {
    const uint2 v = __ldcs(reinterpret_cast<const uint2*>(p));
    a[0] = __uint_as_float(v.x << 16);
    a[1] = __uint_as_float(v.x & 0xffff0000u);
    a[2] = __uint_as_float(v.y << 16);
    a[3] = __uint_as_float(v.y & 0xffff0000u);
}
__device__ __forceinline__ void load4(const float* p, float* a) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
}

template <int G, typename VT, bool OFF16, bool ACC32>
__device__ __forceinline__ double slice_value_lp(int64_t s, int lane, const int* __restrict__ rowlen,
                                                 const int* __restrict__ slice_len,
                                                 const int64_t* __restrict__ slice_ptr,
                                                 const int* __restrict__ perm,
                                                 const int* __restrict__ col,
                                                 const uint16_t* __restrict__ off,
                                                 const int* __restrict__ rowbase,
                                                 const VT* __restrict__ val,
                                                 const double* __restrict__ x,
                                                 const float* __restrict__ x32, int* row)
{
    const int64_t p = s * 32 + lane;
    const int len = rowlen[p];
    const int L = slice_len[s];
    const int64_t q0 = slice_ptr[s] + 4 * lane;   // group g of the row at q0 + 128 g
    const int base = OFF16 ? rowbase[p] : 0;
    float acc32 = 0.f;
    double acc64 = 0.0;
    for (int k = 0; k < L; k += 4 * G) {
        int c[G][4];
        float a[G][4];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int kg = k + 4 * g;
            const int64_t q = q0 + (int64_t)(kg >> 2) * 128;
            if (kg < len) {
                if (OFF16) {
                    const uint2 o = __ldcs(reinterpret_cast<const uint2*>(off + q));
                    c[g][0] = base + (int)(o.x & 0xffffu);
                    c[g][1] = base + (int)(o.x >> 16);
                    c[g][2] = base + (int)(o.y & 0xffffu);
                    c[g][3] = base + (int)(o.y >> 16);
                } else {
                    const int4 o = __ldcs(reinterpret_cast<const int4*>(col + q));
                    c[g][0] = o.x; c[g][1] = o.y; c[g][2] = o.z; c[g][3] = o.w;
                }
                load4(val + q, a[g]);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) { c[g][u] = 0; a[g][u] = 0.f; }
            }
        }
        if (ACC32) {
            float xv[G][4];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int u = 0; u < 4; ++u) xv[g][u] = k + 4 * g + u < len ? __ldg(x32 + c[g][u]) : 0.f;
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (k + 4 * g + u < len) acc32 = fmaf(a[g][u], xv[g][u], acc32);
        } else {
            double xv[G][4];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int u = 0; u < 4; ++u) xv[g][u] = k + 4 * g + u < len ? ldx(x + c[g][u]) : 0.0;
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (k + 4 * g + u < len) acc64 = fma(widen_f32(a[g][u]), xv[g][u], acc64);
        }
    }
    *row = len >= 0 ? (perm ? perm[p] : (int)p) : -1;
    return ACC32 ? (double)acc32 : acc64;
}

}  // namespace dev
}  // namespace spmvlib
