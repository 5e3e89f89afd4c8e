// SpMV variants y = A x over CSR (Algorithm 1, Section 2), one per bottleneck
// class of Section 3.1, plus the preprocessing kernels some of them need.
//
// Every kernel writes every y[i] (empty rows get 0), accumulates in FP64 and
// never reads outside the arrays' extents for a CSR that passed validation.
// Loads of the streamed arrays (rowptr, colind, val) bypass L1 allocation
// where they are touched once; gathers of x go through the read-only
// (non-coherent) path.
#include <cuda_bf16.h>

#include "common.cuh"
#include "rowdot.cuh"

namespace spmvlib {
namespace {

using namespace dev;
constexpr int kBlock = 256;

__device__ __forceinline__ double warp_sum(double s, int width) { return group_sum(s, width); }
__device__ __forceinline__ double ldg_x(const double* p) { return ldx(p); }
template <typename P>
__device__ __forceinline__ auto ld_cs(const P* p) { return ldcs(p); }

// ------------------------------------------------------------------------
// V0 SCALAR: one thread per row, Algorithm 1 as written.  The unoptimized
// CSR kernel that speedups are measured against.
__global__ void __launch_bounds__(kBlock)
k_scalar(int64_t n_rows, const int* __restrict__ rp, const int* __restrict__ ci,
         const double* __restrict__ v, const double* __restrict__ x, double* __restrict__ y)
{
    int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (i >= n_rows) return;
    int b = rp[i], e = rp[i + 1];
    double s = 0.0;
    for (int j = b; j < e; ++j) s += v[j] * x[ci[j]];
    y[i] = s;
}

// ------------------------------------------------------------------------
// V1 SUBWARP: T lanes per row (CMP class: short-row loop overhead and
// vectorisation, Table 2 "unrolling + vectorization").  Each lane keeps two
// independent partial sums; the T partials are combined by shuffles.
template <int T>
__global__ void __launch_bounds__(kBlock)
k_subwarp(int64_t n_rows, const int* __restrict__ rp, const int* __restrict__ ci,
          const double* __restrict__ v, const double* __restrict__ x, double* __restrict__ y)
{
    const int64_t row = (int64_t)blockIdx.x * (kBlock / T) + threadIdx.x / T;
    const int lane = threadIdx.x & (T - 1);
    int64_t b = 0, e = 0;
    if (row < n_rows) { b = rp[row]; e = rp[row + 1]; }
    const double s = group_sum(row_partial<T, 4>(b, e, lane, ColPlain<int>{ci}, v, x), T);
    if (lane == 0 && row < n_rows) y[row] = s;
}

// ------------------------------------------------------------------------
// V2 STREAM: row blocks.  Block k owns the rows whose first nonzero lies in
// the window [k B, (k+1) B).  The CTA stages the products val*x of the whole
// block in shared memory with coalesced loads, then reduces each row from
// shared memory with a power-of-two group of threads per row.  A block whose
// nonzeros exceed the staging capacity (it holds a row longer than B) is
// reduced row by row by the whole CTA straight from global memory.

// R_k = smallest i with rowptr[i] >= k B (k < n_blocks), R_n_blocks = n_rows.
__global__ void k_row_blocks(int64_t n_rows, const int* __restrict__ rp, int64_t block_nnz,
                             int64_t n_blocks, int32_t* __restrict__ out)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n_blocks) return;
    if (k == n_blocks) { out[k] = (int32_t)n_rows; return; }
    int64_t target = k * block_nnz;
    int64_t lo = 0, hi = n_rows;  // answer in [0, n_rows]
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)rp[mid] < target) lo = mid + 1; else hi = mid;
    }
    out[k] = (int32_t)lo;
}

__device__ __forceinline__ double block_sum(double s, double* red) {
    s = warp_sum(s, 32);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = lane < (kBlock / 32) ? red[lane] : 0.0;
        t = warp_sum(t, 32);
    }
    return t;  // valid in thread 0
}

__global__ void __launch_bounds__(kBlock)
k_stream(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
         const double* __restrict__ x, double* __restrict__ y, const int32_t* __restrict__ blocks,
         int cap)
{
    extern __shared__ double prod[];
    __shared__ double red[kBlock / 32];
    const int64_t k = blockIdx.x;
    const int r0 = blocks[k], r1 = blocks[k + 1];
    if (r0 == r1) return;
    const int nz0 = rp[r0], nz1 = rp[r1];
    const int cnt = nz1 - nz0;
    const int nrows = r1 - r0;
    if (cnt <= cap) {
        for (int t0 = threadIdx.x; t0 < cnt; t0 += 4 * kBlock) {
            int c[4];
            double a[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = t0 + u * kBlock;
                c[u] = t < cnt ? ld_cs(ci + nz0 + t) : 0;
                a[u] = t < cnt ? ld_cs(v + nz0 + t) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = t0 + u * kBlock;
                if (t < cnt) prod[t] = a[u] * ldg_x(x + c[u]);
            }
        }
        __syncthreads();
        if (nrows >= kBlock) {
            for (int r = threadIdx.x; r < nrows; r += kBlock) {
                const int b = rp[r0 + r] - nz0, e = rp[r0 + r + 1] - nz0;
                double s = 0.0;
                for (int j = b; j < e; ++j) s += prod[j];
                y[r0 + r] = s;
            }
        } else {
            int T = 1;
            while (T < 32 && nrows * (T * 2) <= kBlock) T *= 2;
            const int g = threadIdx.x / T, lane = threadIdx.x & (T - 1);
            double s = 0.0;
            int b = 0, e = 0;
            if (g < nrows) { b = rp[r0 + g] - nz0; e = rp[r0 + g + 1] - nz0; }
            for (int j = b + lane; j < e; j += T) s += prod[j];
            s = warp_sum(s, T);
            if (lane == 0 && g < nrows) y[r0 + g] = s;
        }
    } else {
        for (int r = r0; r < r1; ++r) {
            const double p = row_partial<kBlock, 4>(rp[r], rp[r + 1], threadIdx.x,
                                                    ColPlain<int>{ci}, v, x);
            const double s = block_sum(p, red);
            if (threadIdx.x == 0) y[r] = s;
        }
    }
}

// ------------------------------------------------------------------------
// V3 MERGE: merge-path split (IMB class; the GPU counterpart of balancing
// the work of Table 2's dynamic scheduling).  The path merges the row ends
// rowptr[1..N] with the nonzero indices; every warp gets the same number of
// path items (rows + nonzeros), so a long row is shared by many warps and
// many short rows by one.  Part p starts at diagonal p * ITEMS.

__global__ void k_merge_coords(int64_t n_rows, int64_t nnz, const int* __restrict__ rp,
                               int64_t items, int64_t n_parts, int32_t* __restrict__ mrow,
                               int32_t* __restrict__ mnz)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p > n_parts) return;
    const int64_t total = n_rows + nnz;
    const int64_t d = p * items < total ? p * items : total;
    // number i of row ends among the first d path items: the path takes the
    // end of row i before nonzero j exactly when rowptr[i+1] <= j.
    int64_t lo = d - nnz > 0 ? d - nnz : 0;
    int64_t hi = d < n_rows ? d : n_rows;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)rp[mid + 1] <= d - mid - 1) lo = mid + 1; else hi = mid;
    }
    mrow[p] = (int32_t)lo;
    mnz[p] = (int32_t)(d - lo);
}

constexpr int kMergeWarps = 4;

template <int IPT>
__global__ void __launch_bounds__(kMergeWarps * 32)
k_merge(int64_t n_parts, const int* __restrict__ rp, const int* __restrict__ ci,
        const double* __restrict__ v, const double* __restrict__ x, double* __restrict__ y,
        const int32_t* __restrict__ mrow, const int32_t* __restrict__ mnz,
        int32_t* __restrict__ carry_row, double* __restrict__ carry_val)
{
    constexpr int ITEMS = 32 * IPT;
    __shared__ double s_prod[kMergeWarps][ITEMS];
    __shared__ int s_end[kMergeWarps][ITEMS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * kMergeWarps + w;
    if (p >= n_parts) return;  // uniform per warp
    const int r0 = mrow[p], r1 = mrow[p + 1];
    const int n0 = mnz[p], n1 = mnz[p + 1];
    const int nr = r1 - r0, nn = n1 - n0;
    {
        int c[IPT];
        double a[IPT];
#pragma unroll
        for (int u = 0; u < IPT; ++u) {
            const int k = lane + 32 * u;
            c[u] = k < nn ? ld_cs(ci + n0 + k) : 0;
            a[u] = k < nn ? ld_cs(v + n0 + k) : 0.0;
            if (k < nr) s_end[w][k] = ld_cs(rp + r0 + 1 + k);
        }
#pragma unroll
        for (int u = 0; u < IPT; ++u) {
            const int k = lane + 32 * u;
            if (k < nn) s_prod[w][k] = a[u] * ldg_x(x + c[u]);
        }
    }
    __syncwarp();

    const int total = nr + nn;
    const int d = min(lane * IPT, total);
    const int dend = min(d + IPT, total);
    int lo = max(0, d - nn), hi = min(d, nr);
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (s_end[w][mid] <= n0 + d - mid - 1) lo = mid + 1; else hi = mid;
    }
    int i = lo, j = d - lo;
    double run = 0.0, first_val = 0.0;
    int first_row = -1;
    for (int t = d; t < dend; ++t) {
        if (i < nr && s_end[w][i] <= n0 + j) {
            if (first_row < 0) { first_row = i; first_val = run; }
            else y[r0 + i] = run;
            run = 0.0;
            ++i;
        } else {
            run += s_prod[w][j];
            ++j;
        }
    }
    // segmented inclusive scan over lanes: a lane that ended a row starts a
    // new segment with its own trailing partial sum
    double val = run;
    int flag = first_row >= 0;
    for (int o = 1; o < 32; o <<= 1) {
        double vu = __shfl_up_sync(FULL_MASK, val, o);
        int fu = __shfl_up_sync(FULL_MASK, flag, o);
        if (lane >= o) {
            if (!flag) val += vu;
            flag |= fu;
        }
    }
    double cin = __shfl_up_sync(FULL_MASK, val, 1);
    if (lane == 0) cin = 0.0;
    if (first_row >= 0) y[r0 + first_row] = first_val + cin;
    if (lane == 31) { carry_row[p] = r1; carry_val[p] = val; }
}

// Adds each part's trailing partial sum to its row, summing the parts of one
// row in part order (deterministic).  carry_row is non-decreasing.
__global__ void k_merge_fixup(int64_t n_parts, int64_t n_rows, const int32_t* __restrict__ carry_row,
                              const double* __restrict__ carry_val, double* __restrict__ y)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_parts) return;
    const int r = carry_row[p];
    if (r < 0 || r >= n_rows) return;
    if (p > 0 && carry_row[p - 1] == r) return;
    double s = 0.0;
    for (int64_t q = p; q < n_parts && carry_row[q] == r; ++q) s += carry_val[q];
    y[r] += s;
}

// ------------------------------------------------------------------------
// V5 LATENCY: for matrices bound by the latency of irregular x accesses (CML
// class; Table 2 software prefetching of x).  On this GPU latency is hidden
// by residency rather than by depth: each lane batches four column loads,
// then four gathers of x, then the values, and the kernel is held to 32
// registers so that 64 warps per SM (8 blocks of 256) keep their gathers in
// flight together.  A deeper batch of eight costs eight registers and a
// quarter of the resident warps and measured slower (0.325 against 0.306 ms
// on 4M x 16 random columns).  x is read through the non-coherent path; when
// x exceeds half the L2 the launch marks (up to the persisting limit of) x as
// persisting in L2.  Smaller x stays resident by itself, and persisting lines
// left behind would shrink the L2 of the kernels that run next.
template <int T>
__global__ void __launch_bounds__(kBlock, 8)
k_latency(int64_t n_rows, const int* __restrict__ rp, const int* __restrict__ ci,
          const double* __restrict__ v, const double* __restrict__ x, double* __restrict__ y)
{
    const int64_t row = (int64_t)blockIdx.x * (kBlock / T) + threadIdx.x / T;
    const int lane = threadIdx.x & (T - 1);
    int64_t b = 0, e = 0;
    if (row < n_rows) { b = rp[row]; e = rp[row + 1]; }
    const double s = group_sum(row_partial<T, 4>(b, e, lane, ColPlain<int>{ci}, v, x), T);
    if (lane == 0 && row < n_rows) y[row] = s;
}

// ------------------------------------------------------------------------
// V6 COMPRESSED (MB class; Table 2 column-index compression): each row keeps
// its first column in rowbase and its columns as 16-bit offsets from it;
// rows spanning 65536 columns or more keep their 32-bit columns (rowbase -1)
// and read them from the original colind.  Values are stored as FP64, FP32
// or BF16; the accumulation is FP64.

__global__ void k_compress_rows(int64_t n_rows, const int* __restrict__ rp,
                                const int* __restrict__ ci, int32_t* __restrict__ rowbase,
                                unsigned long long* __restrict__ n_wide)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    const int b = rp[i], e = rp[i + 1];
    int base = 0;
    if (e > b) {
        const int first = ci[b], last = ci[e - 1];
        if ((int64_t)last - first >= 65536) {
            base = -1;
            atomicAdd(n_wide, 1ull);
        } else {
            base = first;
        }
    }
    rowbase[i] = base;
}

__global__ void k_compress_offsets(int64_t n_rows, const int* __restrict__ rp,
                                   const int* __restrict__ ci, const int32_t* __restrict__ rowbase,
                                   uint16_t* __restrict__ off)
{
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n_rows) return;
    const int b = rp[row], e = rp[row + 1];
    const int base = rowbase[row];
    for (int j = b + lane; j < e; j += 32)
        off[j] = base < 0 ? (uint16_t)0 : (uint16_t)(ci[j] - base);
}

__global__ void k_cast_values(int64_t n, const double* __restrict__ v, int value_type,
                              void* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (value_type == SPMV_VAL_F32)
        static_cast<float*>(out)[i] = __double2float_rn(v[i]);
    else
        static_cast<__nv_bfloat16*>(out)[i] = __double2bfloat16(v[i]);
}

template <int T, typename VT, bool ALL_WIDE>
__global__ void __launch_bounds__(kBlock)
k_compressed(int64_t n_rows, const int* __restrict__ rp, const int32_t* __restrict__ rowbase,
             const uint16_t* __restrict__ off, const int* __restrict__ ci,
             const VT* __restrict__ v, const double* __restrict__ x, double* __restrict__ y)
{
    const int64_t row = (int64_t)blockIdx.x * (kBlock / T) + threadIdx.x / T;
    const int lane = threadIdx.x & (T - 1);
    int64_t b = 0, e = 0;
    int base = -1;
    if (row < n_rows) {
        b = rp[row];
        e = rp[row + 1];
        if (!ALL_WIDE) base = rowbase[row];
    }
    double p;
    if (ALL_WIDE || base < 0)
        p = row_partial<T, 4>(b, e, lane, ColPlain<int>{ci}, v, x);
    else
        p = row_partial<T, 4>(b, e, lane, ColOff16{off, base}, v, x);
    const double s = group_sum(p, T);
    if (lane == 0 && row < n_rows) y[row] = s;
}

// FP32-accumulation form of the compressed variant
__global__ void k_x_to_f32(int64_t n, const double* __restrict__ x, float* __restrict__ x32)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x32[i] = __double2float_rn(x[i]);
}

template <int T, typename VT, bool ALL_WIDE>
__global__ void __launch_bounds__(kBlock)
k_compressed32(int64_t n_rows, const int* __restrict__ rp, const int32_t* __restrict__ rowbase,
               const uint16_t* __restrict__ off, const int* __restrict__ ci,
               const VT* __restrict__ v, const float* __restrict__ x32, double* __restrict__ y)
{
    const int64_t row = (int64_t)blockIdx.x * (kBlock / T) + threadIdx.x / T;
    const int lane = threadIdx.x & (T - 1);
    int64_t b = 0, e = 0;
    int base = -1;
    if (row < n_rows) {
        b = rp[row];
        e = rp[row + 1];
        if (!ALL_WIDE) base = rowbase[row];
    }
    float p;
    if (ALL_WIDE || base < 0)
        p = row_partial32<T, 4>(b, e, lane, ColPlain<int>{ci}, v, x32);
    else
        p = row_partial32<T, 4>(b, e, lane, ColOff16{off, base}, v, x32);
    const float s = group_sum32(p, T);
    if (lane == 0 && row < n_rows) y[row] = (double)s;
}

inline unsigned grid_for(int64_t threads) {
    return (unsigned)((threads + kBlock - 1) / kBlock);
}

}  // namespace

// ============================================================================
// launchers

cudaError_t launch_scalar(const spmv_csr_t& A, const double* x, double* y, cudaStream_t s)
{
    if (A.n_rows == 0) return cudaSuccess;
    k_scalar<<<grid_for(A.n_rows), kBlock, 0, s>>>(A.n_rows, A.rowptr, A.colind, A.val, x, y);
    return cudaGetLastError();
}

#define SPMV_DISPATCH_T(T, KERNEL, GRID, SMEM, STREAM, ...)                       \
    switch (T) {                                                                  \
        case 1: KERNEL<1><<<GRID, kBlock, SMEM, STREAM>>>(__VA_ARGS__); break;    \
        case 2: KERNEL<2><<<GRID, kBlock, SMEM, STREAM>>>(__VA_ARGS__); break;    \
        case 4: KERNEL<4><<<GRID, kBlock, SMEM, STREAM>>>(__VA_ARGS__); break;    \
        case 8: KERNEL<8><<<GRID, kBlock, SMEM, STREAM>>>(__VA_ARGS__); break;    \
        case 16: KERNEL<16><<<GRID, kBlock, SMEM, STREAM>>>(__VA_ARGS__); break;  \
        case 32: KERNEL<32><<<GRID, kBlock, SMEM, STREAM>>>(__VA_ARGS__); break;  \
        default: return cudaErrorInvalidValue;                                    \
    }

cudaError_t launch_subwarp(const spmv_csr_t& A, int T, const double* x, double* y, cudaStream_t s)
{
    if (A.n_rows == 0) return cudaSuccess;
    const unsigned grid = grid_for(A.n_rows * (int64_t)T);
    SPMV_DISPATCH_T(T, k_subwarp, grid, 0, s, A.n_rows, A.rowptr, A.colind, A.val, x, y);
    return cudaGetLastError();
}

cudaError_t launch_row_blocks(const spmv_csr_t& A, int64_t block_nnz, int64_t n_blocks,
                              int32_t* blocks, cudaStream_t s)
{
    k_row_blocks<<<grid_for(n_blocks + 1), kBlock, 0, s>>>(A.n_rows, A.rowptr, block_nnz,
                                                            n_blocks, blocks);
    return cudaGetLastError();
}

cudaError_t launch_stream(const spmv_csr_t& A, const int32_t* blocks, int64_t n_blocks,
                          int block_nnz, const double* x, double* y, cudaStream_t s)
{
    if (A.n_rows == 0) return cudaSuccess;
    const int cap = 2 * block_nnz;
    const size_t smem = (size_t)cap * sizeof(double);
    // the largest window (8192 -> 128 KB) is enabled once per device
    static LaunchCache cache;
    int per_sm = 0;
    cudaError_t e = cached_occupancy(cache, k_stream, kBlock, 2 * 8192 * sizeof(double), &per_sm);
    if (e != cudaSuccess) return e;
    k_stream<<<(unsigned)n_blocks, kBlock, smem, s>>>(A.rowptr, A.colind, A.val, x, y, blocks, cap);
    return cudaGetLastError();
}

cudaError_t launch_merge_coords(const spmv_csr_t& A, int items, int64_t n_parts, int32_t* mrow,
                                int32_t* mnz, cudaStream_t s)
{
    k_merge_coords<<<grid_for(n_parts + 1), kBlock, 0, s>>>(A.n_rows, A.nnz, A.rowptr, items,
                                                             n_parts, mrow, mnz);
    return cudaGetLastError();
}

cudaError_t launch_merge(const spmv_csr_t& A, int items, const int32_t* mrow, const int32_t* mnz,
                         int64_t n_parts, int32_t* carry_row, double* carry_val,
                         const double* x, double* y, cudaStream_t s)
{
    if (A.n_rows == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((n_parts + kMergeWarps - 1) / kMergeWarps);
    const int ipt = items / 32;
#define SPMV_MERGE_CASE(K)                                                                   \
    case K:                                                                                  \
        k_merge<K><<<grid, kMergeWarps * 32, 0, s>>>(n_parts, A.rowptr, A.colind, A.val, x, y, \
                                                     mrow, mnz, carry_row, carry_val);       \
        break;
    switch (ipt) {
        SPMV_MERGE_CASE(1) SPMV_MERGE_CASE(2) SPMV_MERGE_CASE(4) SPMV_MERGE_CASE(6)
        SPMV_MERGE_CASE(7) SPMV_MERGE_CASE(8) SPMV_MERGE_CASE(12) SPMV_MERGE_CASE(16)
        default: return cudaErrorInvalidValue;
    }
#undef SPMV_MERGE_CASE
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_merge_fixup<<<grid_for(n_parts), kBlock, 0, s>>>(n_parts, A.n_rows, carry_row, carry_val, y);
    return cudaGetLastError();
}

cudaError_t launch_latency(const spmv_csr_t& A, int T, const double* x, double* y,
                           int l2_window_bytes, cudaStream_t s)
{
    if (A.n_rows == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid_for(A.n_rows * (int64_t)T));
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    cfg.attrs = attr;
    cfg.numAttrs = 0;
    if (l2_window_bytes > 0) {
        const size_t xbytes = (size_t)A.n_cols * sizeof(double);
        const size_t win = xbytes < (size_t)l2_window_bytes ? xbytes : (size_t)l2_window_bytes;
        attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[0].val.accessPolicyWindow.base_ptr = const_cast<double*>(x);
        attr[0].val.accessPolicyWindow.num_bytes = win;
        attr[0].val.accessPolicyWindow.hitRatio = 1.0f;
        attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        cfg.numAttrs = 1;
    }
    const int64_t n = A.n_rows;
    switch (T) {
        case 1: return cudaLaunchKernelEx(&cfg, k_latency<1>, n, A.rowptr, A.colind, A.val, x, y);
        case 2: return cudaLaunchKernelEx(&cfg, k_latency<2>, n, A.rowptr, A.colind, A.val, x, y);
        case 4: return cudaLaunchKernelEx(&cfg, k_latency<4>, n, A.rowptr, A.colind, A.val, x, y);
        case 8: return cudaLaunchKernelEx(&cfg, k_latency<8>, n, A.rowptr, A.colind, A.val, x, y);
        case 16: return cudaLaunchKernelEx(&cfg, k_latency<16>, n, A.rowptr, A.colind, A.val, x, y);
        case 32: return cudaLaunchKernelEx(&cfg, k_latency<32>, n, A.rowptr, A.colind, A.val, x, y);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_compress(const spmv_csr_t& A, int32_t* rowbase, uint16_t* off16,
                            unsigned long long* n_wide, int value_type, void* lowval,
                            cudaStream_t s)
{
    if (A.n_rows > 0) {
        k_compress_rows<<<grid_for(A.n_rows), kBlock, 0, s>>>(A.n_rows, A.rowptr, A.colind,
                                                              rowbase, n_wide);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (off16) {
            k_compress_offsets<<<grid_for(A.n_rows * 32), kBlock, 0, s>>>(A.n_rows, A.rowptr,
                                                                           A.colind, rowbase, off16);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    if (lowval && A.nnz > 0) {
        k_cast_values<<<grid_for(A.nnz), kBlock, 0, s>>>(A.nnz, A.val, value_type, lowval);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

cudaError_t launch_compressed(const spmv_csr_t& A, int T, int value_type, const int32_t* rowbase,
                              const uint16_t* off16, const void* lowval, bool all_wide,
                              const double* x, double* y, cudaStream_t s)
{
    if (A.n_rows == 0) return cudaSuccess;
    const unsigned grid = grid_for(A.n_rows * (int64_t)T);
    const int64_t n = A.n_rows;
#define SPMV_CMP_LAUNCH(TT, VT, AW)                                                           \
    k_compressed<TT, VT, AW><<<grid, kBlock, 0, s>>>(n, A.rowptr, rowbase, off16, A.colind,   \
                                                     static_cast<const VT*>(vp), x, y)
#define SPMV_CMP_T(VT, AW)                                   \
    switch (T) {                                             \
        case 1: SPMV_CMP_LAUNCH(1, VT, AW); break;           \
        case 2: SPMV_CMP_LAUNCH(2, VT, AW); break;           \
        case 4: SPMV_CMP_LAUNCH(4, VT, AW); break;           \
        case 8: SPMV_CMP_LAUNCH(8, VT, AW); break;           \
        case 16: SPMV_CMP_LAUNCH(16, VT, AW); break;         \
        case 32: SPMV_CMP_LAUNCH(32, VT, AW); break;         \
        default: return cudaErrorInvalidValue;               \
    }
    const void* vp = value_type == SPMV_VAL_F64 ? static_cast<const void*>(A.val) : lowval;
    if (value_type == SPMV_VAL_F64) {
        if (all_wide) { SPMV_CMP_T(double, true) } else { SPMV_CMP_T(double, false) }
    } else if (value_type == SPMV_VAL_F32) {
        if (all_wide) { SPMV_CMP_T(float, true) } else { SPMV_CMP_T(float, false) }
    } else {
        if (all_wide) { SPMV_CMP_T(__nv_bfloat16, true) } else { SPMV_CMP_T(__nv_bfloat16, false) }
    }
#undef SPMV_CMP_T
#undef SPMV_CMP_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_compressed32(const spmv_csr_t& A, int T, int value_type, const int32_t* rowbase,
                                const uint16_t* off16, const void* lowval, bool all_wide,
                                const double* x, float* x32, double* y, cudaStream_t s)
{
    if (A.n_rows == 0) return cudaSuccess;
    if (A.n_cols > 0) {
        k_x_to_f32<<<grid_for(A.n_cols), kBlock, 0, s>>>(A.n_cols, x, x32);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const unsigned grid = grid_for(A.n_rows * (int64_t)T);
    const int64_t n = A.n_rows;
#define SPMV_C32_LAUNCH(TT, VT, AW)                                                            \
    k_compressed32<TT, VT, AW><<<grid, kBlock, 0, s>>>(n, A.rowptr, rowbase, off16, A.colind,  \
                                                       static_cast<const VT*>(lowval), x32, y)
#define SPMV_C32_T(VT, AW)                                   \
    switch (T) {                                             \
        case 1: SPMV_C32_LAUNCH(1, VT, AW); break;           \
        case 2: SPMV_C32_LAUNCH(2, VT, AW); break;           \
        case 4: SPMV_C32_LAUNCH(4, VT, AW); break;           \
        case 8: SPMV_C32_LAUNCH(8, VT, AW); break;           \
        case 16: SPMV_C32_LAUNCH(16, VT, AW); break;         \
        case 32: SPMV_C32_LAUNCH(32, VT, AW); break;         \
        default: return cudaErrorInvalidValue;               \
    }
    if (value_type == SPMV_VAL_F32) {
        if (all_wide) { SPMV_C32_T(float, true) } else { SPMV_C32_T(float, false) }
    } else if (value_type == SPMV_VAL_BF16) {
        if (all_wide) { SPMV_C32_T(__nv_bfloat16, true) } else { SPMV_C32_T(__nv_bfloat16, false) }
    } else {
        return cudaErrorInvalidValue;
    }
#undef SPMV_C32_T
#undef SPMV_C32_LAUNCH
    return cudaGetLastError();
}

}  // namespace spmvlib
