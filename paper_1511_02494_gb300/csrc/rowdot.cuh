// Device building blocks shared by the SpMV kernels: cache-hinted loads and
// the per-row dot product of a group of T lanes with U independent loads in
// flight per lane.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace spmvlib {
namespace dev {

constexpr unsigned FULL = 0xffffffffu;

// x is gathered through the read-only (non-coherent) path; arrays that are
// streamed once are loaded evict-first so they do not push x out of L2.
__device__ __forceinline__ double ldx(const double* p) { return __ldg(p); }
__device__ __forceinline__ int ldcs(const int* p) { return __ldcs(p); }
__device__ __forceinline__ long long ldcs(const long long* p) { return __ldcs(p); }
__device__ __forceinline__ int64_t ldcs(const int64_t* p) {
    return (int64_t)__ldcs(reinterpret_cast<const long long*>(p));
}
__device__ __forceinline__ double ldcs(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ldcs(const float* p) { return __ldcs(p); }
__device__ __forceinline__ unsigned short ldcs(const unsigned short* p) { return __ldcs(p); }

// Exact FP32 -> FP64 widening in integer arithmetic.  The conversion
// instruction runs on the FP64 pipe, this GPU's scarce unit (about two FP64
// operations per clock per SM), so widening each FP32 or BF16 value with it
// costs as much as the DFMA the value feeds.  The same double is assembled
// from the float's bits with a few integer operations instead:
//   exponent e in 1..254: sign, exponent e - 127 + 1023, the 23 mantissa
//     bits at the top of the 52 (high word (e + 896) << 20 | m >> 3, low
//     word m << 29);
//   e = 255 (Inf, NaN): exponent 2047, the mantissa shifted the same way;
//   zero: the zero of the same sign;
//   subnormal (e = 0, m != 0): m 2^-149, renormalised from its leading one
//     at bit p: exponent p + 874, mantissa m << (52 - p) without that bit.
// A BF16 value is the FP32 value with the bits b << 16.
__device__ __forceinline__ double widen_f32_bits(uint32_t f)
{
    const uint32_t sign = f & 0x80000000u;
    const uint32_t mag = f & 0x7fffffffu;
    uint32_t hi = sign | ((mag >> 3) + 0x38000000u);
    const uint32_t lo = f << 29;
    if (mag >= 0x7f800000u) hi += 0x38000000u;
    if (mag < 0x00800000u) {
        if (mag == 0u) return __hiloint2double((int)sign, 0);
        const int p = 31 - __clz((int)mag);
        const uint64_t bits = ((uint64_t)sign << 32) | ((uint64_t)(p + 874) << 52) |
                              (((uint64_t)mag << (52 - p)) & 0x000fffffffffffffull);
        return __longlong_as_double((long long)bits);
    }
    return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double widen_f32(float a) { return widen_f32_bits(__float_as_uint(a)); }

__device__ __forceinline__ double ldval(const double* p) { return __ldcs(p); }
__device__ __forceinline__ double ldval(const float* p) { return widen_f32(__ldcs(p)); }
__device__ __forceinline__ double ldval(const __nv_bfloat16* p) {
    const unsigned short b = __ldcs(reinterpret_cast<const unsigned short*>(p));
    return widen_f32_bits(((uint32_t)b) << 16);
}

__device__ __forceinline__ double group_sum(double s, int width) {
    for (int o = width >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    return s;
}

// Column of element j: plain index array, or 16-bit offset from a row base.
template <typename IT>
struct ColPlain {
    const IT* ci;
    __device__ __forceinline__ int64_t operator()(int64_t j) const { return (int64_t)ldcs(ci + j); }
};
struct ColOff16 {
    const unsigned short* off;
    int64_t base;
    __device__ __forceinline__ int64_t operator()(int64_t j) const {
        return base + (int64_t)ldcs(off + j);
    }
};

// Partial dot product of row [b, e) for lane `lane` of a group of T lanes:
// lane handles j = b + lane + k T.
//
// FP64 is the scarce resource on this GPU (about 2 DFMA per clock per SM), so
// the loop spends exactly one DFMA per element and nothing else in FP64: one
// accumulator, no per-lane partial sums to combine.  Memory parallelism comes
// from the loads instead: each pass issues U column and U value loads, then
// U gathers of x, before its U chained DFMAs.  The remainder (< U elements
// per lane) issues its loads together and runs only as many DFMAs as the
// longest lane of the warp needs.  Every lane of the warp must call this
// (the remainder uses warp votes).
template <int T, int U, typename COL, typename VT>
__device__ __forceinline__ double row_partial(int64_t b, int64_t e, int lane, const COL& col,
                                              const VT* __restrict__ v,
                                              const double* __restrict__ x)
{
    double acc = 0.0;
    int64_t j = b + lane;
    for (; j + (int64_t)(U - 1) * T < e; j += (int64_t)U * T) {
        int64_t c[U];
        double a[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) { c[u] = col(j + u * T); a[u] = ldval(v + j + u * T); }
#pragma unroll
        for (int u = 0; u < U; ++u) xv[u] = ldx(x + c[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) acc = fma(a[u], xv[u], acc);
    }
    const int rem = j < e ? (int)((e - j + T - 1) / T) : 0;  // 0 <= rem < U
    int64_t c[U];
    double a[U], xv[U];
#pragma unroll
    for (int u = 0; u < U - 1; ++u) {
        const bool ok = u < rem;
        c[u] = ok ? col(j + u * T) : 0;
        a[u] = ok ? ldval(v + j + u * T) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U - 1; ++u) xv[u] = u < rem ? ldx(x + c[u]) : 0.0;
#pragma unroll
    for (int u = 0; u < U - 1; ++u)
        if (__any_sync(FULL, u < rem)) acc = u < rem ? fma(a[u], xv[u], acc) : acc;
    return acc;
}

// FP32 form for low-precision values: x comes from an FP32 copy, products
// and sums are FP32 FMAs (the FP32 pipe is ~60x wider than FP64's on this
// GPU), so the row costs no FP64 instruction at all.
__device__ __forceinline__ float ldval32(const float* p) { return __ldcs(p); }
__device__ __forceinline__ float ldval32(const __nv_bfloat16* p) {
    const unsigned short b = __ldcs(reinterpret_cast<const unsigned short*>(p));
    return __uint_as_float(((unsigned)b) << 16);
}

template <int T, int U, typename COL, typename VT>
__device__ __forceinline__ float row_partial32(int64_t b, int64_t e, int lane, const COL& col,
                                               const VT* __restrict__ v,
                                               const float* __restrict__ x)
{
    float acc = 0.f;
    int64_t j = b + lane;
    for (; j + (int64_t)(U - 1) * T < e; j += (int64_t)U * T) {
        int64_t c[U];
        float a[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) { c[u] = col(j + u * T); a[u] = ldval32(v + j + u * T); }
#pragma unroll
        for (int u = 0; u < U; ++u) xv[u] = __ldg(x + c[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) acc = fmaf(a[u], xv[u], acc);
    }
    for (; j < e; j += T) acc = fmaf(ldval32(v + j), __ldg(x + col(j)), acc);
    return acc;
}

__device__ __forceinline__ float group_sum32(float s, int width) {
    for (int o = width >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    return s;
}

}  // namespace dev
}  // namespace spmvlib
