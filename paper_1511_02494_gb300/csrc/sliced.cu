// SLICED variant (V7): sliced ELL layout, the GPU form of the paper's
// bandwidth (MB) and latency (CML) optimizations on this machine.
//
// Rows are grouped in slices of 32; inside a slice the k-th elements of the
// 32 rows are stored next to each other (column-major), so one lane per row
// reads 32 consecutive values and 32 consecutive column indices per load and
// issues 32 independent gathers of x per instruction.  There is no
// reduction across lanes: each row's sum is one chain of DFMAs in row order,
// so the FP64 pipe spends exactly one instruction slot per element of the
// slice (the CSR kernels with T lanes per row add log2(T) shuffle-adds per
// row, 28 % more FP64 slots on a 27-point stencil).  Lanes whose row is
// shorter than the slice skip the padded slots (the loads and DFMAs are
// predicated), so padding costs issue slots but no memory traffic.
//
// Optionally (sigma > 1) rows are sorted by length, longest first, inside
// windows of sigma rows, so that a slice holds rows of similar length; y is
// then written through the permutation.  Rows longer than a cap are not
// put in slices (their slot has length -1); they are split into segments of
// kSlicedSeg nonzeros computed by one warp each from the CSR arrays, and a
// fix-up adds each such row's segment sums in order.  The layout is that of the oracle's orc_sliced_layout
// and orc_sliced_fill, bit for bit.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "rowdot.cuh"
#include "sliced.cuh"

namespace spmvlib {
namespace {

using namespace dev;
constexpr int kSB = 256;       // threads per block: 8 slices
constexpr int kSortT = 1024;   // threads of the window sort

__global__ void k_sl_rowlen_identity(int64_t n_rows, const int* __restrict__ rp, int cap,
                                     int* __restrict__ rowlen, unsigned* __restrict__ n_long)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_rows;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int len = rp[p + 1] - rp[p];
        if (len > cap) {
            rowlen[p] = -1;
            atomicAdd(n_long, 1u);
        } else {
            rowlen[p] = len;
        }
    }
}

// One CTA per window of sigma rows (sigma a power of two, 32..4096): bitonic
// sort of keys (0xFFFFFFFF - key length) << 32 | index in window, so rows come
// out by key length descending, ties by row index ascending; slots past the
// last row carry the largest key and end last.
__global__ void __launch_bounds__(kSortT)
k_sl_sort(int64_t n_rows, const int* __restrict__ rp, int sigma, int cap, int* __restrict__ perm,
          int* __restrict__ rowlen, unsigned* __restrict__ n_long)
{
    extern __shared__ unsigned long long keys[];
    const int64_t w0 = (int64_t)blockIdx.x * sigma;
    for (int i = threadIdx.x; i < sigma; i += kSortT) {
        const int64_t r = w0 + i;
        unsigned long long key = ~0ull;
        if (r < n_rows) {
            const int len = rp[r + 1] - rp[r];
            const unsigned klen = len > cap ? 0u : (unsigned)len;
            key = ((unsigned long long)(0xFFFFFFFFu - klen) << 32) | (unsigned)i;
        }
        keys[i] = key;
    }
    __syncthreads();
    for (int k = 2; k <= sigma; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < sigma; i += kSortT) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a = keys[i], b = keys[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < sigma; i += kSortT) {
        const int64_t p = w0 + i;
        if (p >= n_rows) continue;
        const int r = (int)(w0 + (int64_t)(keys[i] & 0xFFFFFFFFull));
        perm[p] = r;
        const int len = rp[r + 1] - rp[r];
        if (len > cap) {
            rowlen[p] = -1;
            atomicAdd(n_long, 1u);
        } else {
            rowlen[p] = len;
        }
    }
}

// slice_len[s] = max(0, max over the slice's 32 positions of rowlen)
__global__ void k_sl_slice_len(int64_t n_slices, const int* __restrict__ rowlen,
                               int* __restrict__ slice_len)
{
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= n_slices) return;
    const int lane = threadIdx.x & 31;
    const int m = __reduce_max_sync(FULL, max(rowlen[s * 32 + lane], 0));
    if (lane == 0) slice_len[s] = m;
}

// column-major contents of each slice (padding was zeroed beforehand)
// FP64 contents: CT int stores the columns, int16_t / int8_t the column
// minus the row index (the range was checked by k_sl_reach)
template <typename CT>
__global__ void k_sl_fill(int64_t n_slices, const int* __restrict__ rp, const int* __restrict__ ci,
                          const double* __restrict__ v, const int* __restrict__ perm,
                          const int* __restrict__ rowlen, const int64_t* __restrict__ slice_ptr,
                          CT* __restrict__ col, double* __restrict__ val)
{
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= n_slices) return;
    const int lane = threadIdx.x & 31;
    const int64_t p = s * 32 + lane;
    const int len = rowlen[p];
    if (len <= 0) return;
    const int r = perm ? perm[p] : (int)p;
    const int64_t b = rp[r];
    const int64_t q0 = slice_ptr[s] + lane;
    for (int k = 0; k < len; ++k) {
        col[q0 + (int64_t)k * 32] = sizeof(CT) == 4 ? (CT)ci[b + k] : (CT)(ci[b + k] - r);
        val[q0 + (int64_t)k * 32] = v[b + k];
    }
}

// largest |column - row| over the rows in the slices (the first or the last
// column of a row, its columns being increasing)
__global__ void k_sl_reach(int64_t n_slices, const int* __restrict__ rp, const int* __restrict__ ci,
                           const int* __restrict__ perm, const int* __restrict__ rowlen,
                           unsigned* __restrict__ reach)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= 32 * n_slices) return;
    const int len = rowlen[p];
    if (len <= 0) return;
    const int64_t r = perm ? perm[p] : p;
    const int64_t b = rp[r];
    const int64_t lo = r - ci[b], hi = (int64_t)ci[b + len - 1] - r;
    const int64_t m = lo > hi ? lo : hi;
    atomicMax(reach, (unsigned)(m < 0 ? 0 : (m > 0x7fffffff ? 0x7fffffff : m)));
}

// Coded columns of the FP64 layout: the largest delta between consecutive
// columns of a row (MODE 1) or the largest step between the 65536-column
// panels of consecutive elements, the first from panel 0 (MODE 2), over the
// rows in the slices
template <int MODE>
__global__ void k_sl_code_reach(int64_t n_slices, const int* __restrict__ rp, const int* __restrict__ ci,
                                const int* __restrict__ perm, const int* __restrict__ rowlen,
                                unsigned* __restrict__ reach)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= 32 * n_slices) return;
    const int len = rowlen[p];
    if (len <= 0) return;
    const int64_t b = rp[perm ? perm[p] : p];
    unsigned m = 0;
    int prev = MODE == 1 ? ci[b] : 0;
    for (int k = MODE == 1 ? 1 : 0; k < len; ++k) {
        const int c = ci[b + k];
        const unsigned d = MODE == 1 ? (unsigned)(c - prev) : (unsigned)((c >> 16) - (prev >> 16));
        m = max(m, d);
        prev = c;
    }
    atomicMax(reach, m);
}

// coded contents (padding was zeroed beforehand): MODE 1 deltas and row
// bases, MODE 2 panel offsets and steps; a warp per slice, a lane per row
template <int MODE, typename DT>
__global__ void k_sl_fill_coded(int64_t n_slices, const int* __restrict__ rp, const int* __restrict__ ci,
                                const double* __restrict__ v, const int* __restrict__ perm,
                                const int* __restrict__ rowlen, const int64_t* __restrict__ slice_ptr,
                                DT* __restrict__ cs, uint8_t* __restrict__ step, int* __restrict__ rowbase,
                                double* __restrict__ val)
{
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= n_slices) return;
    const int lane = threadIdx.x & 31;
    const int64_t p = s * 32 + lane;
    const int len = rowlen[p];
    if (len <= 0) return;
    const int64_t b = rp[perm ? perm[p] : (int)p];
    const int64_t q0 = slice_ptr[s] + lane;
    if (MODE == 1) rowbase[p] = ci[b];
    int prev = MODE == 1 ? ci[b] : 0;
    for (int k = 0; k < len; ++k) {
        const int c = ci[b + k];
        const int64_t q = q0 + (int64_t)k * 32;
        if (MODE == 1) {
            cs[q] = (DT)(c - prev);
        } else {
            cs[q] = (DT)(c & 0xffff);
            step[q] = (uint8_t)((c >> 16) - (prev >> 16));
        }
        prev = c;
        val[q] = v[b + k];
    }
}

// the shortest row length over the positions holding rows (min into *out,
// which starts at INT_MAX)
__global__ void k_sl_min_len(int64_t n_rows, const int* __restrict__ rowlen, int* __restrict__ out)
{
    int m = 0x7fffffff;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_rows;
         p += (int64_t)gridDim.x * blockDim.x)
        m = min(m, rowlen[p]);
    m = __reduce_min_sync(FULL, m);
    if ((threadIdx.x & 31) == 0) atomicMin(out, m);
}

// rows longer than cap, appended with one atomic per warp
__global__ void k_sl_long_list(int64_t n_rows, const int* __restrict__ rp, int cap,
                               int* __restrict__ list, unsigned* __restrict__ count)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_iter = (n_rows + stride - 1) / stride;
    for (int64_t it = 0; it < n_iter; ++it) {
        const int64_t i = it * stride + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const bool is_long = i < n_rows && rp[i + 1] - rp[i] > cap;
        const unsigned m = __ballot_sync(FULL, is_long);
        if (m == 0) continue;
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(count, (unsigned)__popc(m));
        base = __shfl_sync(FULL, base, 0);
        if (is_long) list[base + __popc(m & ((1u << lane) - 1u))] = (int)i;
    }
}

// 8 blocks of 256 per SM (32 registers): measured faster than the 40-register
// form on all three regular test matrices (random columns 0.249 against
// 0.258 ms, stencil 0.115 against 0.136 ms, 2-nonzero rows 0.080 against
// 0.093 ms).
// Blocks of two warps (32 per SM), as for k_sliced_long: a block frees its
// slot when its two slices are done (27-point stencil 0.113 against 0.115
// ms with eight-warp blocks, 7-point Laplacian 0.035 against 0.037)
constexpr int kOB = 64;
template <int U, typename CT>
__global__ void __launch_bounds__(kOB, 32)
k_sliced(int64_t n_slices, const int* __restrict__ rowlen, const int* __restrict__ slice_len,
         const int64_t* __restrict__ slice_ptr, const int* __restrict__ perm,
         const CT* __restrict__ col, const double* __restrict__ val,
         const double* __restrict__ x, double* __restrict__ y)
{
    const int64_t s = ((int64_t)blockIdx.x * kOB + threadIdx.x) >> 5;
    if (s >= n_slices) return;  // whole warps only
    slice_rows<U, CT>(s, threadIdx.x & 31, rowlen, slice_len, slice_ptr, perm, col, val, x, y);
}

// One slice per warp with coded columns (slice_value_coded).
template <int U, int MODE, typename DT>
__global__ void __launch_bounds__(kSB, 8)
k_sliced_coded(int64_t n_slices, const int* __restrict__ rowlen, const int* __restrict__ slice_len,
               const int64_t* __restrict__ slice_ptr, const int* __restrict__ perm,
               const DT* __restrict__ cs, const uint8_t* __restrict__ step,
               const int* __restrict__ rowbase, const double* __restrict__ val,
               const double* __restrict__ x, double* __restrict__ y)
{
    const int64_t s = ((int64_t)blockIdx.x * kSB + threadIdx.x) >> 5;
    if (s >= n_slices) return;  // whole warps only
    int row;
    const double v = slice_value_coded<U, MODE, DT>(s, threadIdx.x & 31, rowlen, slice_len, slice_ptr, perm,
                                                    cs, step, rowbase, val, x, &row);
    if (row >= 0) y[row] = v;
}

// Every row of length L in order, none long (an ELLPACK matrix): R slices
// per warp with no slice header read (uniform_rows); each row is the same
// DFMA chain as in slice_rows / slice_rows_multi.
template <int U, int R, int B, typename CT>
__global__ void __launch_bounds__(kSB, B)
k_sliced_uniform(int64_t n_rows, int64_t n_slices, int L, const CT* __restrict__ col,
                 const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y)
{
    const int lane = threadIdx.x & 31;
    const int64_t first = (((int64_t)blockIdx.x * kSB + threadIdx.x) >> 5) * R;
    if constexpr (R == 4) {
        // four slices per warp (64 registers, 4 blocks per SM): one resident
        // grid whose warps stride over the slices, instead of many short
        // blocks waiting for an SM slot
        const int64_t step = (int64_t)gridDim.x * (kSB / 32) * R;
        for (int64_t s0 = first; s0 < n_slices; s0 += step)
            uniform_rows<U, R, CT>(s0, n_slices, n_rows, L, lane, col, val, x, y);
    } else {
        if (first >= n_slices) return;  // whole warps only
        uniform_rows<U, R, CT>(first, n_slices, n_rows, L, lane, col, val, x, y);
    }
}

// R consecutive slices per warp (slice_rows_multi), for short slices whose
// few loads per lane leave the warp waiting on latency.
template <int U, int R, int B, typename CT>
__global__ void __launch_bounds__(kSB, B)
k_sliced_multi(int64_t n_slices, const int* __restrict__ rowlen, const int* __restrict__ slice_len,
               const int64_t* __restrict__ slice_ptr, const int* __restrict__ perm,
               const CT* __restrict__ col, const double* __restrict__ val,
               const double* __restrict__ x, double* __restrict__ y)
{
    const int64_t s0 = (((int64_t)blockIdx.x * kSB + threadIdx.x) >> 5) * R;
    if (s0 >= n_slices) return;  // whole warps only
    slice_rows_multi<U, R, CT>(s0, n_slices, threadIdx.x & 31, rowlen, slice_len, slice_ptr, perm, col, val, x,
                               y);
}

__global__ void k_sl_row_lengths(int n, const int* __restrict__ list, const int* __restrict__ rp,
                                 int* __restrict__ len)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) len[q] = rp[list[q] + 1] - rp[list[q]];
}

// Long rows are split into segments of kSlicedSeg nonzeros; seg_be holds
// each segment's CSR begin and end, seg_row the row of a segment that is its
// row's only one (that segment writes y itself) and -1 otherwise.
__global__ void k_sl_seg_table(int n_long, const int* __restrict__ list, const int* __restrict__ seg_off,
                               const int* __restrict__ rp, int64_t* __restrict__ seg_be,
                               int* __restrict__ seg_row)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_long) return;
    const int r = list[q];
    const int64_t b0 = rp[r], e0 = rp[r + 1];
    const bool single = seg_off[q + 1] - seg_off[q] == 1;
    for (int j = seg_off[q]; j < seg_off[q + 1]; ++j) {
        const int64_t b = b0 + (int64_t)(j - seg_off[q]) * kSlicedSeg;
        seg_be[2 * (int64_t)j] = b;
        seg_be[2 * (int64_t)j + 1] = min(e0, b + kSlicedSeg);
        seg_row[j] = single ? r : -1;
    }
}

__device__ __forceinline__ longlong2 segment_bounds(const int64_t* seg_be, int w)
{
    return __ldg(reinterpret_cast<const longlong2*>(seg_be) + w);
}

// A segment's warp writes its sum to y when it is its row's only segment,
// else to partial; the partials of a row with several segments are summed
// in segment order by the warp finishing the row's last one (finish_segment).
// Lane 0 of segment w's warp, with the segment's sum: y of the row when it
// is the row's only segment; else the partial, and when the atomic ticket
// shows this was the row's last segment to finish, the row's sum of
// partials in segment order, after which the ticket is reset for the next
// call.  Nothing waits.
__device__ __forceinline__ void finish_segment(int w, double sum, const int* __restrict__ seg_row,
                                               const int* __restrict__ seg_fix, const int* __restrict__ fix,
                                               const int* __restrict__ list, const int* __restrict__ seg_off,
                                               unsigned* __restrict__ ticket, double* __restrict__ partial,
                                               double* __restrict__ y)
{
    const int r1 = seg_row[w];
    if (r1 >= 0) {
        y[r1] = sum;
        return;
    }
    partial[w] = sum;
    __threadfence();
    const int t = seg_fix[w];
    const int q = fix[t];
    const int b = seg_off[q], e = seg_off[q + 1];
    if (atomicAdd(ticket + t, 1u) != (unsigned)(e - b - 1)) return;
    __threadfence();
    double s = 0.0;
    for (int i = b; i < e; ++i) s += __ldcg(partial + i);
    y[list[q]] = s;
    ticket[t] = 0u;
}

// Slices and long-row segments in one launch (FP64 values, rows above the
// cap present).  Blocks below seg_blocks take one segment per warp, the
// others the slices (R per warp).  The block scheduler starts blocks
// roughly in index order, so the segments -- long, bound by their gathers of
// x -- start first and the short, latency-bound slices fill in around them
// instead of running as a separate launch after them.  A row with several
// segments has no fix-up launch either: each of its segments stores its
// partial, and the warp that finishes the row's last one (an atomic ticket
// per row) sums the partials in segment order (finish_segment) and resets
// the ticket for the next call.  Nothing waits on another warp.
// Threads per block of k_sliced_long: blocks of two warps, so that a block
// whose warps got segments or slices of unequal length frees its SM slot
// sooner (Zipf rows 0.117 ms against 0.119 with blocks of 128 threads and
// 0.120 with 256; the block order is kept)
constexpr int kLB = 64;
template <int U, int R, int B, typename CT, int MODE = 0, typename DT = uint8_t>
__global__ void __launch_bounds__(kLB, 4 * B)
k_sliced_long(int n_seg, unsigned seg_blocks, int64_t n_slices,
              const int64_t* __restrict__ seg_be, const int* __restrict__ seg_row,
              const int* __restrict__ seg_fix, const int* __restrict__ fix,
              const int* __restrict__ list, const int* __restrict__ seg_off,
              unsigned* __restrict__ ticket, double* __restrict__ partial,
              const int* __restrict__ ci, const double* __restrict__ v,
              const int* __restrict__ rowlen, const int* __restrict__ slice_len,
              const int64_t* __restrict__ slice_ptr, const int* __restrict__ perm,
              const CT* __restrict__ col, const double* __restrict__ val,
              const double* __restrict__ x, double* __restrict__ y,
              const uint8_t* __restrict__ step, const int* __restrict__ rowbase)
{
    const int lane = threadIdx.x & 31;
    if (blockIdx.x < seg_blocks) {
        const int w = (int)(blockIdx.x * (kLB / 32) + (threadIdx.x >> 5));
        if (w >= n_seg) return;  // whole warps only
        const longlong2 be = segment_bounds(seg_be, w);
        const double sum = group_sum(row_partial<32, 4>(be.x, be.y, lane, ColPlain<int>{ci}, v, x), 32);
        if (lane == 0) finish_segment(w, sum, seg_row, seg_fix, fix, list, seg_off, ticket, partial, y);
        return;
    }
    const int64_t s0 = ((int64_t)(blockIdx.x - seg_blocks) * kLB + threadIdx.x) >> 5;
    if constexpr (MODE != 0) {
        if (s0 >= n_slices) return;
        int row;
        const double v = slice_value_coded<U, MODE, DT>(s0, lane, rowlen, slice_len, slice_ptr, perm,
                                                        reinterpret_cast<const DT*>(col), step, rowbase,
                                                        val, x, &row);
        if (row >= 0) y[row] = v;
    } else if constexpr (R == 1) {
        if (s0 >= n_slices) return;
        slice_rows<U, CT>(s0, lane, rowlen, slice_len, slice_ptr, perm, col, val, x, y);
    } else {
        if (s0 * R >= n_slices) return;
        slice_rows_multi<U, R, CT>(s0 * R, n_slices, lane, rowlen, slice_len, slice_ptr, perm, col, val,
                                   x, y);
    }
}

// ---- low-precision values (FP32 or BF16), optionally 16-bit column offsets --
__device__ __forceinline__ float round_to(double v, float*) { return __double2float_rn(v); }
__device__ __forceinline__ __nv_bfloat16 round_to(double v, __nv_bfloat16*) { return __double2bfloat16(v); }
__device__ __forceinline__ float widen32(float a) { return a; }
__device__ __forceinline__ float widen32(__nv_bfloat16 a) { return __bfloat162float(a); }

__global__ void k_sl_span(int64_t n_slices, const int* __restrict__ rp, const int* __restrict__ ci,
                          const int* __restrict__ perm, const int* __restrict__ rowlen,
                          int* __restrict__ span)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= 32 * n_slices) return;
    const int len = rowlen[p];
    if (len <= 0) return;
    const int64_t b = rp[perm ? perm[p] : (int)p];
    atomicMax(span, ci[b + len - 1] - ci[b]);
}

// low-precision contents, four elements of a row side by side (element k
// at slice_ptr[s] + 128 (k / 4) + 4 l + k % 4); OFF16: offsets from the
// row's first column (rowbase per position), else 32-bit columns
template <typename VT, bool OFF16>
__global__ void k_sl_fill_lp(int64_t n_slices, const int* __restrict__ rp, const int* __restrict__ ci,
                             const double* __restrict__ v, const int* __restrict__ perm,
                             const int* __restrict__ rowlen, const int64_t* __restrict__ slice_ptr,
                             int* __restrict__ col, uint16_t* __restrict__ off,
                             int* __restrict__ rowbase, VT* __restrict__ val)
{
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= n_slices) return;
    const int lane = threadIdx.x & 31;
    const int64_t p = s * 32 + lane;
    const int len = rowlen[p];
    if (len <= 0) return;
    const int64_t b = rp[perm ? perm[p] : (int)p];
    const int64_t q0 = slice_ptr[s] + 4 * lane;
    const int first = ci[b];
    if (OFF16) rowbase[p] = first;
    for (int k = 0; k < len; ++k) {
        const int64_t q = q0 + (int64_t)(k >> 2) * 128 + (k & 3);
        if (OFF16) off[q] = (uint16_t)(ci[b + k] - first);
        else col[q] = ci[b + k];
        val[q] = round_to(v[b + k], (VT*)nullptr);
    }
}

__global__ void k_sl_x_to_f32(int64_t n, const double* __restrict__ x, float* __restrict__ x32)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x32[i] = __double2float_rn(x[i]);
}

// One slice with low-precision values (slice_value_lp).
template <int U, typename VT, bool OFF16, bool ACC32>
__global__ void __launch_bounds__(kSB, 8)
k_sliced_lp(int64_t n_slices, const int* __restrict__ rowlen, const int* __restrict__ slice_len,
            const int64_t* __restrict__ slice_ptr, const int* __restrict__ perm,
            const int* __restrict__ col, const uint16_t* __restrict__ off,
            const int* __restrict__ rowbase, const VT* __restrict__ val,
            const double* __restrict__ x, const float* __restrict__ x32, double* __restrict__ y)
{
    const int64_t s = ((int64_t)blockIdx.x * kSB + threadIdx.x) >> 5;
    if (s >= n_slices) return;
    int row;
    // two groups of four in flight with 16-bit offsets; one with 32-bit
    // columns (gather-bound rows, where registers are worth more as warps)
    const double v = slice_value_lp<OFF16 ? 2 : 1, VT, OFF16, ACC32>(s, threadIdx.x & 31, rowlen, slice_len, slice_ptr,
                                                         perm, col, off, rowbase, val, x, x32, &row);
    if (row >= 0) y[row] = v;
}

// FP32/BF16 values with rows above the cap: slices and long-row segments in
// one launch, as k_sliced_long.  A segment is computed from the CSR arrays
// with each value rounded as the slices' (the same arithmetic per element);
// its lanes are combined by a shuffle tree, in FP32 (ACC32) or FP64.
template <typename VT, bool OFF16, bool ACC32>
__global__ void __launch_bounds__(kSB, 8)
k_sliced_long_lp(int n_seg, unsigned seg_blocks, int64_t n_slices,
                 const int64_t* __restrict__ seg_be, const int* __restrict__ seg_row,
                 const int* __restrict__ seg_fix, const int* __restrict__ fix,
                 const int* __restrict__ list, const int* __restrict__ seg_off,
                 unsigned* __restrict__ ticket, double* __restrict__ partial,
                 const int* __restrict__ ci, const double* __restrict__ v,
                 const int* __restrict__ rowlen, const int* __restrict__ slice_len,
                 const int64_t* __restrict__ slice_ptr, const int* __restrict__ perm,
                 const int* __restrict__ col, const uint16_t* __restrict__ off,
                 const int* __restrict__ rowbase, const VT* __restrict__ val,
                 const double* __restrict__ x, const float* __restrict__ x32, double* __restrict__ y)
{
    const int lane = threadIdx.x & 31;
    if (blockIdx.x < seg_blocks) {
        const int w = (int)(blockIdx.x * (kSB / 32) + (threadIdx.x >> 5));
        if (w >= n_seg) return;  // whole warps only
        const longlong2 be = segment_bounds(seg_be, w);
        double sum;
        if (ACC32) {
            float acc = 0.f;
            for (int64_t j = be.x + lane; j < be.y; j += 32)
                acc = fmaf(widen32(round_to(__ldcs(v + j), (VT*)nullptr)), __ldg(x32 + __ldcs(ci + j)), acc);
            sum = (double)group_sum32(acc, 32);
        } else {
            double acc = 0.0;
            for (int64_t j = be.x + lane; j < be.y; j += 32)
                acc = fma(widen_f32(widen32(round_to(__ldcs(v + j), (VT*)nullptr))), ldx(x + __ldcs(ci + j)), acc);
            sum = group_sum(acc, 32);
        }
        if (lane == 0) finish_segment(w, sum, seg_row, seg_fix, fix, list, seg_off, ticket, partial, y);
        return;
    }
    const int64_t s = ((int64_t)(blockIdx.x - seg_blocks) * kSB + threadIdx.x) >> 5;
    if (s >= n_slices) return;
    int row;
    const double r = slice_value_lp<OFF16 ? 2 : 1, VT, OFF16, ACC32>(s, lane, rowlen, slice_len, slice_ptr,
                                                                    perm, col, off, rowbase, val, x, x32, &row);
    if (row >= 0) y[row] = r;
}

unsigned grid_of(int64_t threads, int64_t cap_blocks)
{
    int64_t g = (threads + kSB - 1) / kSB;
    if (g > cap_blocks) g = cap_blocks;
    return (unsigned)std::max<int64_t>(g, 1);
}

}  // namespace

spmv_status sliced_prepare(spmv_prepared* P, cudaStream_t s)
{
    const spmv_csr_t& A = P->A;
    SlicedPlan& d = P->sl;
    int cap = P->c.items_per_warp > 0 ? P->c.items_per_warp : kSlicedCap;
    d.n_slices = (A.n_rows + 31) / 32;
    const int64_t n_pos = 32 * d.n_slices;
    spmv_status st;
    if ((st = prepared_alloc(P, reinterpret_cast<void**>(&d.rowlen), 4 * std::max<int64_t>(n_pos, 1))) != SPMV_OK ||
        (st = prepared_alloc(P, reinterpret_cast<void**>(&d.slice_len), 4 * std::max<int64_t>(d.n_slices, 1))) != SPMV_OK ||
        (st = prepared_alloc(P, reinterpret_cast<void**>(&d.slice_ptr), 8 * (d.n_slices + 1))) != SPMV_OK ||
        (st = prepared_alloc(P, reinterpret_cast<void**>(&d.count), 4)) != SPMV_OK)
        return st;
    const unsigned rows_grid = grid_of(A.n_rows, (int64_t)P->sm_count * 16);
    const unsigned slice_grid = grid_of(n_pos, INT32_MAX);
    std::vector<int> slen((size_t)std::max<int64_t>(d.n_slices, 1));
    std::vector<int64_t> sptr((size_t)d.n_slices + 1, 0);
    unsigned n_long = 0;
    int64_t slots = 0;  // sum of 32 x slice length: padding by unequal rows only
    // one layout pass for window length sigma (1 = rows in order)
    auto layout = [&](int sigma) -> spmv_status {
        SPMV_CUDA_TRY(cudaMemsetAsync(d.rowlen, 0xFF, 4 * std::max<int64_t>(n_pos, 1), s));
        SPMV_CUDA_TRY(cudaMemsetAsync(d.count, 0, 4, s));
        if (A.n_rows > 0) {
            if (sigma == 1) {
                k_sl_rowlen_identity<<<rows_grid, kSB, 0, s>>>(A.n_rows, A.rowptr, cap, d.rowlen, d.count);
            } else {
                if (!d.perm) {
                    spmv_status st2 = prepared_alloc(P, reinterpret_cast<void**>(&d.perm), 4 * A.n_rows);
                    if (st2 != SPMV_OK) return st2;
                }
                const int64_t n_win = (A.n_rows + sigma - 1) / sigma;
                k_sl_sort<<<(unsigned)n_win, kSortT, sizeof(unsigned long long) * sigma, s>>>(
                    A.n_rows, A.rowptr, sigma, cap, d.perm, d.rowlen, d.count);
            }
            SPMV_CUDA_TRY(cudaGetLastError());
            k_sl_slice_len<<<slice_grid, kSB, 0, s>>>(d.n_slices, d.rowlen, d.slice_len);
            SPMV_CUDA_TRY(cudaGetLastError());
            SPMV_CUDA_TRY(cudaMemcpyAsync(slen.data(), d.slice_len, 4 * d.n_slices, cudaMemcpyDeviceToHost, s));
        }
        SPMV_CUDA_TRY(cudaMemcpyAsync(&n_long, d.count, 4, cudaMemcpyDeviceToHost, s));
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
        slots = 0;
        for (int64_t i = 0; i < d.n_slices; ++i) {
            sptr[i + 1] = sptr[i] + 32 * (int64_t)((slen[i] + d.vec - 1) / d.vec * d.vec);
            slots += 32 * (int64_t)slen[i];
        }
        return SPMV_OK;
    };
    // FP64 values: one element per slot row; FP32/BF16: four side by side
    d.vec = P->c.value_type == SPMV_VAL_F64 ? 1 : 4;
    int sigma = P->c.block_nnz;
    if (sigma == 0) {
        // rows in order unless that pads the slices by more than a quarter;
        // then rows sorted by length in windows of 4096, and (unless the cap
        // was chosen) every row above 32 nonzeros computed by a warp, so that
        // no lane's chain is longer than one element per lane of a warp
        if ((st = layout(1)) != SPMV_OK) return st;
        if (slots > A.nnz + A.nnz / 4) {
            sigma = 4096;
            if (P->c.items_per_warp == 0) cap = 32;
            if ((st = layout(sigma)) != SPMV_OK) return st;
        } else {
            sigma = 1;
        }
    } else if ((st = layout(sigma)) != SPMV_OK) {
        return st;
    }
    P->c.block_nnz = sigma;
    P->c.items_per_warp = cap;
    d.sigma = sigma;
    // FP64 values: slices per warp, 4 when no slice is longer than four
    // elements (a lane's few loads leave a warp waiting on latency, so one
    // warp takes four slices), else 1 (longer slices keep four elements of
    // one row in flight instead)
    if (P->c.value_type != SPMV_VAL_F64) {
        P->c.threads_per_row = 1;
    } else if (P->c.threads_per_row == 0) {
        const int longest = d.n_slices > 0 ? *std::max_element(slen.begin(), slen.begin() + d.n_slices) : 0;
        P->c.threads_per_row = longest <= 4 ? 4 : 1;
    }
    d.n_long = (int)n_long;
    d.tot = sptr[d.n_slices];
    // rows all of one length, in order, none long: the slice header is implied
    d.uniform_len = -1;
    if (sigma == 1 && n_long == 0 && A.n_rows > 0) {
        int shortest = 0x7fffffff;
        SPMV_CUDA_TRY(cudaMemsetAsync(d.count, 0x7f, 4, s));
        k_sl_min_len<<<rows_grid, kSB, 0, s>>>(A.n_rows, d.rowlen, reinterpret_cast<int*>(d.count));
        SPMV_CUDA_TRY(cudaGetLastError());
        SPMV_CUDA_TRY(cudaMemcpyAsync(&shortest, d.count, 4, cudaMemcpyDeviceToHost, s));
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
        const int longest = *std::max_element(slen.begin(), slen.begin() + d.n_slices);
        if (shortest == longest) d.uniform_len = longest;
    }
    SPMV_CUDA_TRY(cudaMemcpyAsync(d.slice_ptr, sptr.data(), 8 * (d.n_slices + 1), cudaMemcpyHostToDevice, s));
    const int64_t tot1 = std::max<int64_t>(d.tot, 1);
    const int* permp = sigma > 1 ? d.perm : nullptr;
    d.value_type = P->c.value_type;
    if (P->c.accumulate == 0) P->c.accumulate = d.value_type == SPMV_VAL_F64 ? 1 : 2;
    d.acc32 = P->c.accumulate == 2;
    if (d.value_type == SPMV_VAL_F64) {
        // columns as offsets from the row index in 8 or 16 bits when the
        // caller allows it and every row in the slices stays that close to
        // its diagonal, else 32-bit
        // coded columns (Table 2's deltas, or panels) when asked for and
        // every row in the slices fits: deltas in 8 bits, else 16, else (or
        // when panels were asked for) 16-bit panel offsets with 8-bit steps
        d.coding = 0;
        if (P->c.index_coding != 0 && d.n_slices > 0) {
            auto code_reach = [&](int mode, unsigned* out) -> spmv_status {
                SPMV_CUDA_TRY(cudaMemsetAsync(d.count, 0, 4, s));
                const unsigned g = (unsigned)((32 * d.n_slices + kSB - 1) / kSB);
                if (mode == 1) k_sl_code_reach<1><<<g, kSB, 0, s>>>(d.n_slices, A.rowptr, A.colind, permp, d.rowlen, d.count);
                else k_sl_code_reach<2><<<g, kSB, 0, s>>>(d.n_slices, A.rowptr, A.colind, permp, d.rowlen, d.count);
                SPMV_CUDA_TRY(cudaGetLastError());
                SPMV_CUDA_TRY(cudaMemcpyAsync(out, d.count, 4, cudaMemcpyDeviceToHost, s));
                SPMV_CUDA_TRY(cudaStreamSynchronize(s));
                return SPMV_OK;
            };
            unsigned r = 0;
            if (P->c.index_coding == 1) {
                if ((st = code_reach(1, &r)) != SPMV_OK) return st;
                if (r <= 255) { d.coding = 1; d.cbytes = 1; }
                else if (r <= 65535) { d.coding = 1; d.cbytes = 2; }
            }
            if (d.coding == 0) {
                if ((st = code_reach(2, &r)) != SPMV_OK) return st;
                if (r <= 255) { d.coding = 2; d.cbytes = 3; }
            }
        }
        // index_bytes 0: the narrowest form that fits when the rows are all of
        // one length and in order (k_sliced_uniform, where the narrower column
        // stream shortens the launch), else 32-bit columns
        const int allowed = d.coding != 0 ? 4
                            : P->c.index_bytes != 0 ? P->c.index_bytes
                            : d.uniform_len >= 0 ? 1 : 4;
        unsigned reach = 0;
        if (d.n_slices > 0 && allowed < 4) {
            SPMV_CUDA_TRY(cudaMemsetAsync(d.count, 0, 4, s));
            k_sl_reach<<<(unsigned)((32 * d.n_slices + kSB - 1) / kSB), kSB, 0, s>>>(
                d.n_slices, A.rowptr, A.colind, permp, d.rowlen, d.count);
            SPMV_CUDA_TRY(cudaGetLastError());
            SPMV_CUDA_TRY(cudaMemcpyAsync(&reach, d.count, 4, cudaMemcpyDeviceToHost, s));
            SPMV_CUDA_TRY(cudaStreamSynchronize(s));
        }
        if (d.coding == 0) d.cbytes = std::max(allowed, reach <= 127 ? 1 : (reach <= 32767 ? 2 : 4));
        P->c.index_bytes = d.cbytes;
        P->c.index_coding = d.coding;
        if (d.coding != 0) P->c.threads_per_row = 1;  // coded columns: one slice per warp
        const int64_t sbytes = d.coding == 2 ? 2 : d.cbytes;  // panel offsets are 16-bit
        if ((st = prepared_alloc(P, &d.scol, sbytes * tot1)) != SPMV_OK ||
            (st = prepared_alloc(P, reinterpret_cast<void**>(&d.val), 8 * tot1)) != SPMV_OK)
            return st;
        if (d.cbytes == 4) d.col = static_cast<int*>(d.scol);
        SPMV_CUDA_TRY(cudaMemsetAsync(d.scol, 0, sbytes * tot1, s));
        SPMV_CUDA_TRY(cudaMemsetAsync(d.val, 0, 8 * tot1, s));
        if (d.coding == 2) {
            if ((st = prepared_alloc(P, reinterpret_cast<void**>(&d.step), tot1)) != SPMV_OK) return st;
            SPMV_CUDA_TRY(cudaMemsetAsync(d.step, 0, tot1, s));
        }
        if (d.coding == 1) {
            if ((st = prepared_alloc(P, reinterpret_cast<void**>(&d.rowbase), 4 * std::max<int64_t>(n_pos, 1))) != SPMV_OK)
                return st;
            SPMV_CUDA_TRY(cudaMemsetAsync(d.rowbase, 0, 4 * std::max<int64_t>(n_pos, 1), s));
        }
        if (d.n_slices > 0 && d.coding != 0) {
#define SPMV_SL_FILL_CODED(MODE, DT)                                                                  \
    k_sl_fill_coded<MODE, DT><<<slice_grid, kSB, 0, s>>>(d.n_slices, A.rowptr, A.colind, A.val, permp, \
                                                        d.rowlen, d.slice_ptr, static_cast<DT*>(d.scol), \
                                                        d.step, d.rowbase, d.val)
            if (d.coding == 1 && d.cbytes == 1) SPMV_SL_FILL_CODED(1, uint8_t);
            else if (d.coding == 1) SPMV_SL_FILL_CODED(1, uint16_t);
            else SPMV_SL_FILL_CODED(2, uint16_t);
#undef SPMV_SL_FILL_CODED
            SPMV_CUDA_TRY(cudaGetLastError());
        } else if (d.n_slices > 0) {
#define SPMV_SL_FILL64(CT)                                                                           \
    k_sl_fill<CT><<<slice_grid, kSB, 0, s>>>(d.n_slices, A.rowptr, A.colind, A.val, permp, d.rowlen, \
                                             d.slice_ptr, static_cast<CT*>(d.scol), d.val)
            if (d.cbytes == 1) SPMV_SL_FILL64(int8_t);
            else if (d.cbytes == 2) SPMV_SL_FILL64(int16_t);
            else SPMV_SL_FILL64(int);
#undef SPMV_SL_FILL64
            SPMV_CUDA_TRY(cudaGetLastError());
        }
    } else {
        // 16-bit offsets when every row in the slices spans fewer than 65536 columns
        int span = 0;
        if (d.n_slices > 0) {
            SPMV_CUDA_TRY(cudaMemsetAsync(d.count, 0, 4, s));
            k_sl_span<<<(unsigned)((32 * d.n_slices + kSB - 1) / kSB), kSB, 0, s>>>(
                d.n_slices, A.rowptr, A.colind, permp, d.rowlen, reinterpret_cast<int*>(d.count));
            SPMV_CUDA_TRY(cudaGetLastError());
            SPMV_CUDA_TRY(cudaMemcpyAsync(&span, d.count, 4, cudaMemcpyDeviceToHost, s));
            SPMV_CUDA_TRY(cudaStreamSynchronize(s));
        }
        d.off16 = span < 65536;
        const int vb = d.value_type == SPMV_VAL_F32 ? 4 : 2;
        if ((st = prepared_alloc(P, &d.lowval, vb * tot1)) != SPMV_OK) return st;
        SPMV_CUDA_TRY(cudaMemsetAsync(d.lowval, 0, vb * tot1, s));
        if (d.off16) {
            if ((st = prepared_alloc(P, reinterpret_cast<void**>(&d.off), 2 * tot1)) != SPMV_OK ||
                (st = prepared_alloc(P, reinterpret_cast<void**>(&d.rowbase), 4 * std::max<int64_t>(n_pos, 1))) != SPMV_OK)
                return st;
            SPMV_CUDA_TRY(cudaMemsetAsync(d.off, 0, 2 * tot1, s));
            SPMV_CUDA_TRY(cudaMemsetAsync(d.rowbase, 0, 4 * std::max<int64_t>(n_pos, 1), s));
        } else {
            if ((st = prepared_alloc(P, reinterpret_cast<void**>(&d.col), 4 * tot1)) != SPMV_OK) return st;
            SPMV_CUDA_TRY(cudaMemsetAsync(d.col, 0, 4 * tot1, s));
        }
        if (d.n_slices > 0) {
#define SPMV_SL_FILL(VT, O16)                                                                      \
    k_sl_fill_lp<VT, O16><<<slice_grid, kSB, 0, s>>>(d.n_slices, A.rowptr, A.colind, A.val, permp, \
                                                     d.rowlen, d.slice_ptr, d.col, d.off,          \
                                                     d.rowbase, static_cast<VT*>(d.lowval))
            if (d.value_type == SPMV_VAL_F32) {
                if (d.off16) SPMV_SL_FILL(float, true); else SPMV_SL_FILL(float, false);
            } else {
                if (d.off16) SPMV_SL_FILL(__nv_bfloat16, true); else SPMV_SL_FILL(__nv_bfloat16, false);
            }
#undef SPMV_SL_FILL
            SPMV_CUDA_TRY(cudaGetLastError());
        }
    }
    if (d.acc32 &&
        (st = prepared_alloc(P, reinterpret_cast<void**>(&d.x32), 4 * std::max<int64_t>(A.n_cols, 1))) != SPMV_OK)
        return st;
    if (d.n_long > 0) {
        if ((st = prepared_alloc(P, reinterpret_cast<void**>(&d.long_rows), 4 * (int64_t)d.n_long)) != SPMV_OK ||
            (st = prepared_alloc(P, reinterpret_cast<void**>(&d.seg_off), 4 * ((int64_t)d.n_long + 1))) != SPMV_OK)
            return st;
        SPMV_CUDA_TRY(cudaMemsetAsync(d.count, 0, 4, s));
        k_sl_long_list<<<rows_grid, kSB, 0, s>>>(A.n_rows, A.rowptr, cap, d.long_rows, d.count);
        SPMV_CUDA_TRY(cudaGetLastError());
        // long rows in ascending order (host sort), their lengths (device,
        // into seg_off as scratch), then their segment offsets (host scan)
        std::vector<int> lr(d.n_long), len(d.n_long), off(d.n_long + 1);
        SPMV_CUDA_TRY(cudaMemcpyAsync(lr.data(), d.long_rows, 4 * (size_t)d.n_long, cudaMemcpyDeviceToHost, s));
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
        std::sort(lr.begin(), lr.end());
        SPMV_CUDA_TRY(cudaMemcpyAsync(d.long_rows, lr.data(), 4 * (size_t)d.n_long, cudaMemcpyHostToDevice, s));
        k_sl_row_lengths<<<(unsigned)((d.n_long + 255) / 256), 256, 0, s>>>(d.n_long, d.long_rows, A.rowptr,
                                                                            d.seg_off);
        SPMV_CUDA_TRY(cudaGetLastError());
        SPMV_CUDA_TRY(cudaMemcpyAsync(len.data(), d.seg_off, 4 * (size_t)d.n_long, cudaMemcpyDeviceToHost, s));
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
        off[0] = 0;
        for (int q = 0; q < d.n_long; ++q) off[q + 1] = off[q] + (len[q] + kSlicedSeg - 1) / kSlicedSeg;
        d.n_seg = off[d.n_long];
        SPMV_CUDA_TRY(cudaMemcpyAsync(d.seg_off, off.data(), 4 * ((size_t)d.n_long + 1), cudaMemcpyHostToDevice, s));
        // the rows with several segments, summed by the fix-up
        std::vector<int> fix;
        for (int q = 0; q < d.n_long; ++q)
            if (off[q + 1] - off[q] > 1) fix.push_back(q);
        d.n_fix = (int)fix.size();
        // per segment the index of its row in the fix list (-1: the row's only segment)
        std::vector<int> seg_fix((size_t)d.n_seg, -1);
        d.seg_several.assign((size_t)d.n_seg, 0);
        for (int t = 0; t < d.n_fix; ++t)
            for (int j = off[fix[t]]; j < off[fix[t] + 1]; ++j) {
                seg_fix[j] = t;
                d.seg_several[j] = 1;
            }
        if ((st = prepared_alloc(P, reinterpret_cast<void**>(&d.partial), 8 * (int64_t)d.n_seg)) != SPMV_OK ||
            (st = prepared_alloc(P, reinterpret_cast<void**>(&d.seg_be), 16 * (int64_t)d.n_seg)) != SPMV_OK ||
            (st = prepared_alloc(P, reinterpret_cast<void**>(&d.seg_row), 4 * (int64_t)d.n_seg)) != SPMV_OK ||
            (st = prepared_alloc(P, reinterpret_cast<void**>(&d.seg_fix), 4 * (int64_t)d.n_seg)) != SPMV_OK ||
            (st = prepared_alloc(P, reinterpret_cast<void**>(&d.fix), 4 * std::max<int64_t>(d.n_fix, 1))) != SPMV_OK ||
            (st = prepared_alloc(P, reinterpret_cast<void**>(&d.ticket), 4 * std::max<int64_t>(d.n_fix, 1))) != SPMV_OK)
            return st;
        if (d.n_fix > 0)
            SPMV_CUDA_TRY(cudaMemcpyAsync(d.fix, fix.data(), 4 * (size_t)d.n_fix, cudaMemcpyHostToDevice, s));
        SPMV_CUDA_TRY(cudaMemsetAsync(d.ticket, 0, 4 * std::max<int64_t>(d.n_fix, 1), s));
        SPMV_CUDA_TRY(cudaMemcpyAsync(d.seg_fix, seg_fix.data(), 4 * (size_t)d.n_seg, cudaMemcpyHostToDevice, s));
        k_sl_seg_table<<<(unsigned)((d.n_long + 255) / 256), 256, 0, s>>>(d.n_long, d.long_rows, d.seg_off,
                                                                          A.rowptr, d.seg_be, d.seg_row);
        SPMV_CUDA_TRY(cudaGetLastError());
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    }
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));  // host vectors go out of scope
    P->n_blocks = d.n_slices;
    return SPMV_OK;
}

cudaError_t launch_sliced(const spmv_prepared* P, const double* x, double* y, cudaStream_t s)
{
    const spmv_csr_t& A = P->A;
    const SlicedPlan& d = P->sl;
    if (A.n_rows == 0) return cudaSuccess;
    const unsigned grid = grid_of(32 * d.n_slices, INT32_MAX);
    const int* perm = d.sigma > 1 ? d.perm : nullptr;
    cudaError_t e;
    if (d.acc32 && A.n_cols > 0) {
        k_sl_x_to_f32<<<(unsigned)((A.n_cols + kSB - 1) / kSB), kSB, 0, s>>>(A.n_cols, x, d.x32);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (d.value_type == SPMV_VAL_F64 && d.n_long > 0) {
        // slices and long-row segments in one launch, segments first
        const unsigned seg_blocks = (unsigned)((d.n_seg + kLB / 32 - 1) / (kLB / 32));
        const int R = P->c.threads_per_row == 2 || P->c.threads_per_row == 4 ? P->c.threads_per_row : 1;
        const int64_t slice_warps = (d.n_slices + R - 1) / R;
        const unsigned blocks = seg_blocks + (unsigned)((slice_warps + kLB / 32 - 1) / (kLB / 32));
#define SPMV_SL_LONG(U, RR, B, CT)                                                                  \
    k_sliced_long<U, RR, B, CT><<<blocks, kLB, 0, s>>>(                                           \
        d.n_seg, seg_blocks, d.n_slices, d.seg_be, d.seg_row, d.seg_fix, d.fix, d.long_rows,       \
        d.seg_off, d.ticket, d.partial, A.colind, A.val, d.rowlen, d.slice_len, d.slice_ptr, perm,  \
        static_cast<const CT*>(d.scol), d.val, x, y, nullptr, nullptr)
#define SPMV_SL_LONG_CT(CT)                                                                          \
        if (R == 4) SPMV_SL_LONG(1, 4, 4, CT); else if (R == 2) SPMV_SL_LONG(2, 2, 6, CT);           \
        else SPMV_SL_LONG(4, 1, 8, CT);
#define SPMV_SL_LONG_CODED(MODE, DT)                                                                \
    k_sliced_long<4, 1, 8, int, MODE, DT><<<blocks, kLB, 0, s>>>(                                   \
        d.n_seg, seg_blocks, d.n_slices, d.seg_be, d.seg_row, d.seg_fix, d.fix, d.long_rows,       \
        d.seg_off, d.ticket, d.partial, A.colind, A.val, d.rowlen, d.slice_len, d.slice_ptr, perm,  \
        static_cast<const int*>(d.scol), d.val, x, y, d.step, d.rowbase)
        if (d.coding == 1 && d.cbytes == 1) { SPMV_SL_LONG_CODED(1, uint8_t); }
        else if (d.coding == 1) { SPMV_SL_LONG_CODED(1, uint16_t); }
        else if (d.coding == 2) { SPMV_SL_LONG_CODED(2, uint16_t); }
        else if (d.cbytes == 1) { SPMV_SL_LONG_CT(int8_t) }
        else if (d.cbytes == 2) { SPMV_SL_LONG_CT(int16_t) }
        else { SPMV_SL_LONG_CT(int) }
#undef SPMV_SL_LONG_CODED
#undef SPMV_SL_LONG_CT
#undef SPMV_SL_LONG
        return cudaGetLastError();
    }
    if (d.value_type == SPMV_VAL_F64 && d.coding != 0) {
#define SPMV_SL_CODED(MODE, DT)                                                                     \
    k_sliced_coded<4, MODE, DT><<<grid, kSB, 0, s>>>(d.n_slices, d.rowlen, d.slice_len, d.slice_ptr,  \
                                                     perm, static_cast<const DT*>(d.scol), d.step,    \
                                                     d.rowbase, d.val, x, y)
        if (d.coding == 1 && d.cbytes == 1) SPMV_SL_CODED(1, uint8_t);
        else if (d.coding == 1) SPMV_SL_CODED(1, uint16_t);
        else SPMV_SL_CODED(2, uint16_t);
#undef SPMV_SL_CODED
        return cudaGetLastError();
    }
    if (d.value_type == SPMV_VAL_F64 && d.uniform_len >= 0) {
        // rows of one length: no slice header (k_sliced_uniform)
        const int R = P->c.threads_per_row == 2 || P->c.threads_per_row == 4 ? P->c.threads_per_row : 1;
        const unsigned ugrid = grid_of(32 * ((d.n_slices + R - 1) / R), R == 4 ? (int64_t)P->sm_count * 4 : INT32_MAX);
#define SPMV_SL_U(U, RR, B, CT)                                                                    \
    k_sliced_uniform<U, RR, B, CT><<<ugrid, kSB, 0, s>>>(A.n_rows, d.n_slices, d.uniform_len,      \
                                                         static_cast<const CT*>(d.scol), d.val, x, y)
#define SPMV_SL_U_CT(CT)                                                                           \
        if (R == 4) SPMV_SL_U(1, 4, 4, CT); else if (R == 2) SPMV_SL_U(2, 2, 6, CT);               \
        else SPMV_SL_U(4, 1, 8, CT);
        if (d.cbytes == 1) { SPMV_SL_U_CT(int8_t) }
        else if (d.cbytes == 2) { SPMV_SL_U_CT(int16_t) }
        else { SPMV_SL_U_CT(int) }
#undef SPMV_SL_U_CT
#undef SPMV_SL_U
        return cudaGetLastError();
    }
    if (d.value_type == SPMV_VAL_F64) {
        // R slices per warp (sliced_prepare chose R, or the caller did);
        // columns stored as CT (sliced_prepare chose the width)
#define SPMV_SL_M(U, RR, B, CT)                                                                    \
    k_sliced_multi<U, RR, B, CT><<<grid_of(32 * ((d.n_slices + RR - 1) / RR), INT32_MAX), kSB, 0, s>>>( \
        d.n_slices, d.rowlen, d.slice_len, d.slice_ptr, perm, static_cast<const CT*>(d.scol), d.val, x, y)
#define SPMV_SL_CT(CT)                                                                             \
        switch (P->c.threads_per_row) {                                                            \
            case 2: SPMV_SL_M(2, 2, 6, CT); break;                                                 \
            case 4: SPMV_SL_M(1, 4, 4, CT); break;                                                 \
            default:                                                                               \
                k_sliced<4, CT><<<(unsigned)((d.n_slices + kOB / 32 - 1) / (kOB / 32)), kOB, 0, s>>>( \
                    d.n_slices, d.rowlen, d.slice_len, d.slice_ptr, \
                                                     perm, static_cast<const CT*>(d.scol), d.val, x, y); \
        }
        if (d.cbytes == 1) { SPMV_SL_CT(int8_t) }
        else if (d.cbytes == 2) { SPMV_SL_CT(int16_t) }
        else { SPMV_SL_CT(int) }
#undef SPMV_SL_CT
#undef SPMV_SL_M
    } else if (d.n_long > 0) {
        // FP32/BF16 values with long rows: slices and segments in one launch
        const unsigned seg_blocks = (unsigned)((d.n_seg + kSB / 32 - 1) / (kSB / 32));
        const unsigned blocks = seg_blocks + (unsigned)((d.n_slices + kSB / 32 - 1) / (kSB / 32));
#define SPMV_SL_LONG_LP(VT, O16, A32)                                                                 \
    k_sliced_long_lp<VT, O16, A32><<<blocks, kSB, 0, s>>>(                                          \
        d.n_seg, seg_blocks, d.n_slices, d.seg_be, d.seg_row, d.seg_fix, d.fix, d.long_rows,         \
        d.seg_off, d.ticket, d.partial, A.colind, A.val, d.rowlen, d.slice_len, d.slice_ptr, perm,    \
        d.col, d.off, d.rowbase, static_cast<const VT*>(d.lowval), x, d.x32, y)
#define SPMV_SL_LONG_LP_VT(VT)                                                                         \
    if (d.off16) { if (d.acc32) SPMV_SL_LONG_LP(VT, true, true); else SPMV_SL_LONG_LP(VT, true, false); } \
    else { if (d.acc32) SPMV_SL_LONG_LP(VT, false, true); else SPMV_SL_LONG_LP(VT, false, false); }
        if (d.value_type == SPMV_VAL_F32) { SPMV_SL_LONG_LP_VT(float) } else { SPMV_SL_LONG_LP_VT(__nv_bfloat16) }
#undef SPMV_SL_LONG_LP_VT
#undef SPMV_SL_LONG_LP
    } else {
#define SPMV_SL_LP(VT, O16, A32)                                                                   \
    k_sliced_lp<4, VT, O16, A32><<<grid, kSB, 0, s>>>(d.n_slices, d.rowlen, d.slice_len,          \
                                                      d.slice_ptr, perm, d.col, d.off, d.rowbase,  \
                                                      static_cast<const VT*>(d.lowval), x, d.x32, y)
#define SPMV_SL_LP_VT(VT)                                                        \
    if (d.off16) { if (d.acc32) SPMV_SL_LP(VT, true, true); else SPMV_SL_LP(VT, true, false); } \
    else { if (d.acc32) SPMV_SL_LP(VT, false, true); else SPMV_SL_LP(VT, false, false); }
        if (d.value_type == SPMV_VAL_F32) { SPMV_SL_LP_VT(float) } else { SPMV_SL_LP_VT(__nv_bfloat16) }
#undef SPMV_SL_LP_VT
#undef SPMV_SL_LP
    }
    return cudaGetLastError();
}

}  // namespace spmvlib
