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

// FP64 values and 32-bit columns
template <int U>
__device__ __forceinline__ double slice_value(int64_t s, int lane, const int* __restrict__ rowlen,
                                              const int* __restrict__ slice_len,
                                              const int64_t* __restrict__ slice_ptr,
                                              const int* __restrict__ perm,
                                              const int* __restrict__ col,
                                              const double* __restrict__ val,
                                              const double* __restrict__ x, int* row)
{
    const int64_t p = s * 32 + lane;
    const int len = rowlen[p];
    const int L = slice_len[s];
    const int64_t q0 = slice_ptr[s] + lane;
    const int* __restrict__ cp = col + q0;      // element k at cp[32 k] (k < 1025)
    const double* __restrict__ vp = val + q0;
    double acc = 0.0;
    for (int k = 0; k < L; k += U) {
        int c[U];
        double a[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = k + u < len;
            c[u] = ok ? __ldcs(cp + (k + u) * 32) : 0;
            a[u] = ok ? __ldcs(vp + (k + u) * 32) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) xv[u] = k + u < len ? ldx(x + c[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k + u < len) acc = fma(a[u], xv[u], acc);
    }
    *row = len >= 0 ? (perm ? perm[p] : (int)p) : -1;
    return acc;
}

template <int U>
__device__ __forceinline__ void slice_rows(int64_t s, int lane, const int* __restrict__ rowlen,
                                           const int* __restrict__ slice_len,
                                           const int64_t* __restrict__ slice_ptr,
                                           const int* __restrict__ perm,
                                           const int* __restrict__ col,
                                           const double* __restrict__ val,
                                           const double* __restrict__ x, double* __restrict__ y)
{
    int row;
    const double v = slice_value<U>(s, lane, rowlen, slice_len, slice_ptr, perm, col, val, x, &row);
    if (row >= 0) y[row] = v;
}

// FP32 or BF16 values, 32-bit columns or 16-bit offsets from rowbase[p].
// ACC32: x32 is the FP32 copy of x; fmaf chain, one widening per row.
// Otherwise each value is widened to FP64 and summed with DFMAs.
template <int U, typename VT, bool OFF16, bool ACC32>
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
    const int64_t q0 = slice_ptr[s] + lane;
    const int base = OFF16 ? rowbase[p] : 0;
    const VT* __restrict__ vp = val + q0;
    float acc32 = 0.f;
    double acc64 = 0.0;
    for (int k = 0; k < L; k += U) {
        int c[U];
        float a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = k + u < len;
            if (OFF16) c[u] = ok ? base + (int)__ldcs(off + q0 + (k + u) * 32) : 0;
            else c[u] = ok ? __ldcs(col + q0 + (k + u) * 32) : 0;
            a[u] = ok ? ldval32(vp + (k + u) * 32) : 0.f;  // exact widening of FP32 / BF16
        }
        if (ACC32) {
            float xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) xv[u] = k + u < len ? __ldg(x32 + c[u]) : 0.f;
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (k + u < len) acc32 = fmaf(a[u], xv[u], acc32);
        } else {
            double xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) xv[u] = k + u < len ? ldx(x + c[u]) : 0.0;
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (k + u < len) acc64 = fma((double)a[u], xv[u], acc64);
        }
    }
    *row = len >= 0 ? (perm ? perm[p] : (int)p) : -1;
    return ACC32 ? (double)acc32 : acc64;
}

}  // namespace dev
}  // namespace spmvlib
