// Structural features of Table 1 (Section 3.2.2) and CSR validation, in one
// pass over rowptr and colind.
//
// Per row i (empty rows contribute zeros):
//   nnz_i, bw_i = last - first column (0 when nnz_i <= 1), span_i = bw_i + 1,
//   ngroups_i = maximal runs of consecutive columns,
//   misses_i  = 1 + #{j > first : 8 (c_j - c_{j-1}) > line_bytes},
//   disp q_i  = floor(2^32 nnz_i / span_i), clust q_i = floor(2^32 ngroups_i / nnz_i).
// The aggregates (min, max, sums, sums of squares) are integers; integer
// addition is associative, so global atomics give exact, order-independent
// totals.  128-bit sums are kept as (lo, hi) words with explicit carries.
// The doubles of Table 1 are derived on the host from these integers.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace spmvlib {
namespace {

typedef unsigned long long u64;
typedef unsigned __int128 u128;

// Device accumulators; every field starts at 0.  Minima are kept as the
// maximum of the bitwise complement so that 0 is the identity.
struct FeatAcc {
    u64 nnz_min_c, nnz_max, nnz_sum, nnz_sumsq;
    u64 bw_min_c, bw_max, bw_sum, bw_sq_lo, bw_sq_hi;
    u64 disp_sum, disp_sq_lo, disp_sq_hi, clust_sum;
    u64 ngroups_sum, misses_sum;
    u64 err;
    u64 n_long;  // rows of kShortCap < nnz <= kChunk (front of the list)
    u64 n_huge;  // rows of nnz > kChunk (back of the list, chunked)
};

__device__ __forceinline__ u64 shfl_u64(u64 v, int o) {
    return __shfl_xor_sync(FULL_MASK, v, o);
}

__device__ __forceinline__ void atomic_add_u128(u64* lo, u64* hi, u128 v) {
    const u64 vlo = (u64)v, vhi = (u64)(v >> 64);
    if (vlo) {
        const u64 old = atomicAdd(lo, vlo);
        if (old + vlo < old) atomicAdd(hi, 1ull);  // carry out of the low word
    }
    if (vhi) atomicAdd(hi, vhi);
}

__device__ __forceinline__ u128 warp_sum_u128(u128 v) {
    u64 lo = (u64)v, hi = (u64)(v >> 64);
    for (int o = 16; o > 0; o >>= 1) {
        const u64 lo2 = shfl_u64(lo, o), hi2 = shfl_u64(hi, o);
        const u64 nlo = lo + lo2;
        hi = hi + hi2 + (nlo < lo ? 1ull : 0ull);
        lo = nlo;
    }
    return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ u64 warp_sum_u64(u64 v) {
    for (int o = 16; o > 0; o >>= 1) v += shfl_u64(v, o);
    return v;
}
__device__ __forceinline__ u64 warp_max_u64(u64 v) {
    for (int o = 16; o > 0; o >>= 1) { u64 t = shfl_u64(v, o); v = t > v ? t : v; }
    return v;
}

constexpr int kFields = 16;  // FeatAcc words reduced per block (err excluded)

// floor(a 2^32 / b) for 0 <= a <= b < 2^31, exactly, without a 64-bit
// integer division and without 64-bit conversions (which run on the FP64
// pipe): an FP32 estimate of the quotient (a / b < 1, so it fits 32 bits),
// then the integer remainder a 2^32 - q b, converted to FP32 from two 32-bit
// halves, gives a correction, and the remainder is brought into [0, b).  The
// first estimate is within about 2^9 of the quotient, so |remainder| < 2^41
// and the second within one; the final steps run at most once (capped at
// four).  Arguments outside that range come only from rows the pass flags as
// invalid (columns not strictly increasing or out of range), whose results
// are discarded: they give 0.
__device__ __forceinline__ u64 fixq32(u64 a, u64 b)
{
    if (a == 0 || b == 0 || b >= (1ull << 31) || a > b) return 0;
    if (a == b) return 1ull << 32;
    const unsigned a32 = (unsigned)a, b32 = (unsigned)b;
    const float rb = __frcp_rn(__uint2float_rn(b32));
    int64_t q = (int64_t)__float2uint_rz(__fmul_rn(__fmul_rn(__uint2float_rn(a32), rb), 4294967296.0f));
    int64_t rem = (int64_t)(((u64)a32 << 32) - (u64)q * b32);
    const float rf = __fmaf_rn(__int2float_rn((int)(rem >> 20)), 1048576.0f,
                               __uint2float_rn((unsigned)(rem & 0xFFFFF)));
    const int c = __float2int_rd(__fmul_rn(rf, rb));
    q += c;
    rem -= (int64_t)c * b32;
    for (int i = 0; i < 4 && rem < 0; ++i) { --q; rem += b32; }
    for (int i = 0; i < 4 && rem >= (int64_t)b32; ++i) { ++q; rem -= b32; }
    return (u64)q;
}

// Per-thread partial aggregates of the rows a thread finalizes.
struct RowAgg {
    u64 nnz_min_c = 0, nnz_max = 0, nnz_sum = 0, nnz_sq = 0;
    u64 bw_min_c = 0, bw_max = 0, bw_sum = 0, disp_sum = 0, clust_sum = 0, ng_sum = 0, ms_sum = 0;
    u128 bw_sq = 0, disp_sq = 0;

    // one row: nz nonzeros, columns first..last, ng / ms counted over its
    // elements after the first (the first element adds one to each)
    __device__ __forceinline__ void add(u64 nz, int64_t first, int64_t last, u64 ng, u64 ms) {
        u64 bw = 0, dq = 0, cq = 0;
        if (nz > 0) {
            bw = (u64)(last - first);
            ng += 1;
            ms += 1;
            dq = fixq32(nz, bw + 1);
            cq = fixq32(ng, nz);
        }
        nnz_min_c = max(nnz_min_c, ~nz);
        nnz_max = max(nnz_max, nz);
        nnz_sum += nz;
        nnz_sq += nz * nz;
        bw_min_c = max(bw_min_c, ~bw);
        bw_max = max(bw_max, bw);
        bw_sum += bw;
        bw_sq += (u128)bw * bw;
        disp_sum += dq;
        disp_sq += (u128)dq * dq;
        clust_sum += cq;
        ng_sum += ng;
        ms_sum += ms;
    }
};

// Warp reduction, then block reduction, then one set of atomics per block.
template <bool FEATURES>
__device__ void flush_block(RowAgg& r, u64 err, u64 (*s_red)[kFields], u64* s_err, FeatAcc* acc)
{
    for (int o = 16; o > 0; o >>= 1) err |= shfl_u64(err, o);
    const int w = threadIdx.x >> 5;
    if (FEATURES) {
        r.nnz_min_c = warp_max_u64(r.nnz_min_c);
        r.nnz_max = warp_max_u64(r.nnz_max);
        r.nnz_sum = warp_sum_u64(r.nnz_sum);
        r.nnz_sq = warp_sum_u64(r.nnz_sq);
        r.bw_min_c = warp_max_u64(r.bw_min_c);
        r.bw_max = warp_max_u64(r.bw_max);
        r.bw_sum = warp_sum_u64(r.bw_sum);
        r.bw_sq = warp_sum_u128(r.bw_sq);
        r.disp_sum = warp_sum_u64(r.disp_sum);
        r.disp_sq = warp_sum_u128(r.disp_sq);
        r.clust_sum = warp_sum_u64(r.clust_sum);
        r.ng_sum = warp_sum_u64(r.ng_sum);
        r.ms_sum = warp_sum_u64(r.ms_sum);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        if (err) atomicOr(s_err, err);
        u64* t = s_red[w];
        t[0] = r.nnz_min_c; t[1] = r.nnz_max; t[2] = r.nnz_sum; t[3] = r.nnz_sq;
        t[4] = r.bw_min_c; t[5] = r.bw_max; t[6] = r.bw_sum;
        t[7] = (u64)r.bw_sq; t[8] = (u64)(r.bw_sq >> 64);
        t[9] = r.disp_sum; t[10] = (u64)r.disp_sq; t[11] = (u64)(r.disp_sq >> 64);
        t[12] = r.clust_sum; t[13] = r.ng_sum; t[14] = r.ms_sum; t[15] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        if (*s_err) atomicOr(&acc->err, *s_err);
        if (FEATURES) {
            u64 t[kFields] = {0};
            u128 bsq = 0, dsq = 0;
            for (int k = 0; k < nw; ++k) {
                const u64* q = s_red[k];
                t[0] = max(t[0], q[0]); t[1] = max(t[1], q[1]); t[2] += q[2]; t[3] += q[3];
                t[4] = max(t[4], q[4]); t[5] = max(t[5], q[5]); t[6] += q[6];
                bsq += ((u128)q[8] << 64) | q[7];
                t[9] += q[9];
                dsq += ((u128)q[11] << 64) | q[10];
                t[12] += q[12]; t[13] += q[13]; t[14] += q[14];
            }
            if (t[0]) atomicMax(&acc->nnz_min_c, t[0]);
            if (t[1]) atomicMax(&acc->nnz_max, t[1]);
            if (t[2]) atomicAdd(&acc->nnz_sum, t[2]);
            if (t[3]) atomicAdd(&acc->nnz_sumsq, t[3]);
            if (t[4]) atomicMax(&acc->bw_min_c, t[4]);
            if (t[5]) atomicMax(&acc->bw_max, t[5]);
            if (t[6]) atomicAdd(&acc->bw_sum, t[6]);
            atomic_add_u128(&acc->bw_sq_lo, &acc->bw_sq_hi, bsq);
            if (t[9]) atomicAdd(&acc->disp_sum, t[9]);
            atomic_add_u128(&acc->disp_sq_lo, &acc->disp_sq_hi, dsq);
            if (t[12]) atomicAdd(&acc->clust_sum, t[12]);
            if (t[13]) atomicAdd(&acc->ngroups_sum, t[13]);
            if (t[14]) atomicAdd(&acc->misses_sum, t[14]);
        }
    }
}

// The per-element tests in 32-bit integers.  Columns of a valid matrix lie
// in [0, n_cols) with n_cols < 2^31, so the unsigned compare (unsigned)c >=
// n_cols is c < 0 || c >= n_cols, and the difference of two columns, taken
// modulo 2^32, is exact; a row with an invalid column or order sets an error
// bit and the call returns an error, so its counts are never used.  A gap d
// moves more than a line of line_bytes when 8 d > line_bytes, that is when
// d > floor(line_bytes / 8) (d an integer).
struct ColTest {
    unsigned n_cols;
    int lb8;  // floor(line_bytes / 8)
};

// Elements [j0, e) of a row starting at b, every `step`-th one, U at a time:
// ng counts columns that do not follow their predecessor by one, ms those
// more than a line away from it; bad collects CSR violations.
template <int U>
__device__ __forceinline__ void count_elements(int64_t b, int64_t j0, int64_t e, int step,
                                               const int* __restrict__ ci, ColTest t, u64& ng, u64& ms,
                                               u64& bad)
{
    unsigned g = 0, m = 0;  // at most kChunk / 32 elements a lane per call
    for (; j0 < e; j0 += (int64_t)U * step) {
        int c[U], cp[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t j = j0 + u * step;
            c[u] = j < e ? ci[j] : 0;
            cp[u] = (j < e && j > b) ? ci[j - 1] : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t j = j0 + u * step;
            if (j < e) {
                if ((unsigned)c[u] >= t.n_cols) bad |= 8;
                if (j > b) {
                    const int d = (int)((unsigned)c[u] - (unsigned)cp[u]);
                    if (d <= 0) bad |= 16;
                    g += (d != 1);
                    m += (d > t.lb8);
                }
            }
        }
    }
    ng += g;
    ms += m;
}

// Rows of at most kShortCap nonzeros: a lane per row, warps taking tiles of
// 32 consecutive rows.  Each lane walks its row in order, four loads in
// flight, keeping the previous column in a register, so every element is
// loaded once and the per-row arithmetic (two 64-bit divisions, 128-bit
// squares) runs on all 32 lanes.  Longer rows are listed for the chunked
// kernels below.  Held to 64 registers (4 blocks of 256 per SM; a few bytes
// of the per-row aggregates spill): 0.126 ms on the 27-point stencil
// against 0.148 ms at 80 registers and 3 blocks.
constexpr int64_t kShortCap = 64;
constexpr int64_t kChunk = 4096;

template <bool FEATURES>
__global__ void __launch_bounds__(256, 4)
k_feature_pass(int64_t n_rows, int64_t n_cols, int64_t nnz, const int* __restrict__ rp,
               const int* __restrict__ ci, int64_t line_bytes, int* __restrict__ long_rows,
               int64_t max_long, FeatAcc* __restrict__ acc)
{
    constexpr int U = 4;
    __shared__ u64 s_red[8][kFields];
    __shared__ u64 s_err;
    const int lane = threadIdx.x & 31;
    RowAgg r;
    u64 err = 0;
    if (threadIdx.x == 0) s_err = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (rp[0] != 0) err |= 1;
        if ((int64_t)rp[n_rows] != nnz) err |= 2;
    }
    const int64_t n_tiles = (n_rows + 31) / 32;
    const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x / 32);
    const ColTest t{(unsigned)n_cols, (int)(line_bytes >> 3)};
    for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; tile < n_tiles;
         tile += n_warps) {
        const int64_t row = tile * 32 + lane;
        int64_t b = 0, nz = 0;
        bool is_long = false, row_ok = false;
        if (row < n_rows) {
            b = rp[row];
            const int64_t e = rp[row + 1];
            if (b < 0 || e < b || e > nnz) { err |= 4; b = 0; }
            else if (e - b > kShortCap) is_long = true;
            else { nz = e - b; row_ok = true; }
        }
        unsigned ng = 0, ms = 0;
        int first = 0, prev = 0;
        const int nzi = (int)nz;  // at most kShortCap
        if (nzi > 0) {
            first = prev = ci[b];
            if ((unsigned)first >= t.n_cols) err |= 8;
        }
        for (int k = 1; k < nzi; k += U) {
            int c[U];
#pragma unroll
            for (int u = 0; u < U; ++u) c[u] = k + u < nzi ? ci[b + k + u] : 0;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (k + u < nzi) {
                    if ((unsigned)c[u] >= t.n_cols) err |= 8;
                    const int d = (int)((unsigned)c[u] - (unsigned)prev);
                    if (d <= 0) err |= 16;
                    ng += (d != 1);
                    ms += (d > t.lb8);
                    prev = c[u];
                }
            }
        }
        if (FEATURES && row_ok) r.add((u64)nz, first, prev, ng, ms);
        // long rows: up to kChunk nonzeros to the front of the list (a warp
        // each), longer ones to the back (chunked)
        const bool huge = is_long && rp[row + 1] - rp[row] > kChunk;
        const unsigned mm = __ballot_sync(FULL_MASK, is_long && !huge);
        const unsigned mh = __ballot_sync(FULL_MASK, huge);
        if (mm | mh) {
            u64 bm = 0, bh = 0;
            if (lane == 0) {
                if (mm) bm = atomicAdd(&acc->n_long, (u64)__popc(mm));
                if (mh) bh = atomicAdd(&acc->n_huge, (u64)__popc(mh));
            }
            bm = __shfl_sync(FULL_MASK, bm, 0);
            bh = __shfl_sync(FULL_MASK, bh, 0);
            const unsigned lt = (1u << lane) - 1u;
            // overlapping rows (a rowptr that is not monotone) can list more
            // rows than the buffer holds; the error flag is set for them
            if (is_long && !huge) {
                const u64 pos = bm + __popc(mm & lt);
                if (pos < (u64)max_long) long_rows[pos] = (int)row;
                else err |= 4;
            }
            if (huge) {
                const u64 pos = bh + __popc(mh & lt);
                if (pos < (u64)max_long) long_rows[max_long - 1 - pos] = (int)row;
                else err |= 4;
            }
        }
    }
    flush_block<FEATURES>(r, err, s_red, &s_err, acc);
}

// Exclusive scan of the huge rows' chunk counts (one block, a contiguous
// segment per thread): chunk_off[q] is the first chunk of huge row q (list
// entry max_long - 1 - q), chunk_off[n_huge] their total.  Also zeroes the
// per-row totals, the tickets and the work counter of the chunk kernel.
__global__ void __launch_bounds__(1024)
k_chunk_offsets(const int* __restrict__ long_rows, int64_t max_long, const int* __restrict__ rp,
                int* __restrict__ chunk_off, u64* __restrict__ ng, u64* __restrict__ ms,
                unsigned* __restrict__ done, unsigned* __restrict__ next,
                const FeatAcc* __restrict__ acc)
{
    __shared__ int part[1024];
    const int64_t nh = min((int64_t)acc->n_huge, max_long);
    const int n = (int)nh;
    for (int q = threadIdx.x; q < n; q += 1024) { ng[q] = 0; ms[q] = 0; done[q] = 0; }
    if (threadIdx.x == 0) *next = 0;
    const int per = (n + 1023) / 1024;
    const int q0 = min(n, (int)threadIdx.x * per), q1 = min(n, q0 + per);
    int local = 0;
    for (int q = q0; q < q1; ++q) {
        const int row = long_rows[max_long - 1 - q];
        local += (int)((rp[row + 1] - rp[row] + kChunk - 1) / kChunk);
    }
    part[threadIdx.x] = local;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int t = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    int run = part[threadIdx.x] - local;
    for (int q = q0; q < q1; ++q) {
        chunk_off[q] = run;
        const int row = long_rows[max_long - 1 - q];
        run += (int)((rp[row + 1] - rp[row] + kChunk - 1) / kChunk);
    }
    if (threadIdx.x == 1023) chunk_off[n] = part[1023];
}

// Chunks of kChunk nonzeros of the long rows: persistent warps take chunks
// from an atomic counter, add the chunk's counts to the row's totals, and the
// warp that completes a row's last chunk (a ticket per row) adds the row to
// its aggregates.  Integer sums: the result does not depend on the order.
struct LongScratch {
    u64* ng;          // [max_long]
    u64* ms;          // [max_long]
    unsigned* done;   // [max_long] chunks finished
    unsigned* next;   // work counter
};

template <bool FEATURES>
__global__ void __launch_bounds__(256)
k_feature_chunks(const int* __restrict__ long_rows, int64_t max_long, const int* __restrict__ chunk_off,
                 int64_t n_cols, const int* __restrict__ rp, const int* __restrict__ ci,
                 int64_t line_bytes, LongScratch w, FeatAcc* __restrict__ acc)
{
    __shared__ u64 s_red[8][kFields];
    __shared__ u64 s_err;
    if (threadIdx.x == 0) s_err = 0;
    const int lane = threadIdx.x & 31;
    const int n_mid = (int)min((int64_t)acc->n_long, max_long);
    const int n_huge = (int)min((int64_t)acc->n_huge, max_long);
    const int total = n_mid + (n_huge > 0 ? chunk_off[n_huge] : 0);
    RowAgg r;
    u64 bad = 0;
    const ColTest t{(unsigned)n_cols, (int)(line_bytes >> 3)};
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(w.next, 1u);
        it = __shfl_sync(FULL_MASK, it, 0);
        if (it >= total) break;
        if (it < n_mid) {
            // a row of at most kChunk nonzeros: the whole row by this warp
            const int row = long_rows[it];
            const int64_t b = rp[row], e = rp[row + 1];
            u64 ng = 0, ms = 0;
            count_elements<4>(b, b + lane, e, 32, ci, t, ng, ms, bad);
            ng = warp_sum_u64(ng);
            ms = warp_sum_u64(ms);
            if (FEATURES && lane == 0) r.add((u64)(e - b), (int64_t)ci[b], (int64_t)ci[e - 1], ng, ms);
            continue;
        }
        const int ic = it - n_mid;
        int lo = 0, hi = n_huge - 1;  // the huge row whose chunks include ic
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (chunk_off[mid] <= ic) lo = mid; else hi = mid - 1;
        }
        const int row = long_rows[max_long - 1 - lo];
        const int64_t b = rp[row], e = rp[row + 1];
        const int64_t c0 = b + (int64_t)(ic - chunk_off[lo]) * kChunk;
        const int64_t c1 = min(e, c0 + kChunk);
        u64 ng = 0, ms = 0;
        count_elements<4>(b, c0 + lane, c1, 32, ci, t, ng, ms, bad);
        ng = warp_sum_u64(ng);
        ms = warp_sum_u64(ms);
        if (lane == 0) {
            atomicAdd(&w.ng[lo], ng);
            atomicAdd(&w.ms[lo], ms);
            __threadfence();
            const unsigned n_chunks = (unsigned)(chunk_off[lo + 1] - chunk_off[lo]);
            if (atomicAdd(&w.done[lo], 1u) == n_chunks - 1) {
                __threadfence();
                const u64 tng = atomicAdd(&w.ng[lo], 0ull), tms = atomicAdd(&w.ms[lo], 0ull);
                if (FEATURES) r.add((u64)(e - b), (int64_t)ci[b], (int64_t)ci[e - 1], tng, tms);
            }
        }
    }
    flush_block<FEATURES>(r, bad, s_red, &s_err, acc);
}

double sd_from_sums(u64 n, u64 s1, u128 s2)
{
    const u128 num = (u128)n * s2 - (u128)s1 * (u128)s1;
    return sqrt((double)num) / (double)n;
}

float lg1p(double v) { return (float)log2(1.0 + v); }

// pinned host staging for the accumulator readback, one per host thread
thread_local FeatAcc* t_host_acc = nullptr;
thread_local FeatAcc* t_dev_acc = nullptr;
thread_local int t_dev_acc_device = -1;
// device scratch of the long-row kernels, per host thread; grows, never shrinks
thread_local void* t_scratch = nullptr;
thread_local size_t t_scratch_bytes = 0;
thread_local int t_scratch_device = -1;

}  // namespace

int auto_threads_per_row(double mean_nnz)
{
    int T = 1;
    while (T < 32 && T < mean_nnz) T *= 2;
    return T;
}

spmv_status run_feature_pass(const spmv_csr_t* A, int32_t line_bytes, spmv_features_t* out,
                             cudaStream_t s)
{
    spmv_status st = check_csr_args(A);
    if (st != SPMV_OK) return st;
    DeviceInfo dev;
    st = current_device(&dev);
    if (st != SPMV_OK) return st;
    if (line_bytes <= 0) line_bytes = 128;

    if (!t_host_acc) {
        void* p = nullptr;
        if (cudaMallocHost(&p, sizeof(FeatAcc)) != cudaSuccess)
            return fail(SPMV_ERR_NOMEM, "cudaMallocHost for the feature readback failed");
        t_host_acc = static_cast<FeatAcc*>(p);
    }
    // one device accumulator per host thread and device, kept for reuse
    if (t_dev_acc_device != dev.device || !t_dev_acc) {
        void* p = nullptr;
        SPMV_CUDA_TRY(cudaMalloc(&p, sizeof(FeatAcc)));
        t_dev_acc = static_cast<FeatAcc*>(p);
        t_dev_acc_device = dev.device;
    }
    FeatAcc* acc = t_dev_acc;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(FeatAcc), s);
    if (e == cudaSuccess && A->n_rows > 0) {
        // scratch: per-long-row totals and tickets, the work counter, the
        // long-row list and the chunk offsets
        const int64_t max_long = std::min<int64_t>(A->n_rows, A->nnz / (kShortCap + 1) + 1);
        const size_t bytes = sizeof(u64) * 2 * (size_t)max_long + sizeof(unsigned) * (size_t)(max_long + 1) +
                             sizeof(int) * (size_t)(2 * max_long + 1) + 64;
        if (t_scratch_device != dev.device || t_scratch_bytes < bytes) {
            if (t_scratch) cudaFree(t_scratch);
            t_scratch = nullptr;
            t_scratch_bytes = 0;
            e = cudaMalloc(&t_scratch, bytes);
            if (e == cudaSuccess) { t_scratch_bytes = bytes; t_scratch_device = dev.device; }
        }
        u64* ng = static_cast<u64*>(t_scratch);
        u64* ms = ng + max_long;
        unsigned* done = reinterpret_cast<unsigned*>(ms + max_long);
        unsigned* next = done + max_long;
        int* long_rows = reinterpret_cast<int*>(next + 1);
        int* chunk_off = long_rows + max_long;
        int64_t blocks = ((A->n_rows + 31) / 32 * 32 + 255) / 256;
        const int64_t lim = (int64_t)dev.sm_count * 16;
        if (blocks > lim) blocks = lim;
        if (blocks < 1) blocks = 1;
        const unsigned cgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(max_long, (int64_t)dev.sm_count * 2));
        LongScratch w{ng, ms, done, next};
        if (e == cudaSuccess) {
            if (out)
                k_feature_pass<true><<<(unsigned)blocks, 256, 0, s>>>(A->n_rows, A->n_cols, A->nnz, A->rowptr,
                                                                      A->colind, line_bytes, long_rows, max_long, acc);
            else
                k_feature_pass<false><<<(unsigned)blocks, 256, 0, s>>>(A->n_rows, A->n_cols, A->nnz, A->rowptr,
                                                                       A->colind, line_bytes, long_rows, max_long, acc);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            k_chunk_offsets<<<1, 1024, 0, s>>>(long_rows, max_long, A->rowptr, chunk_off, ng, ms, done,
                                               next, acc);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            if (out)
                k_feature_chunks<true><<<cgrid, 256, 0, s>>>(long_rows, max_long, chunk_off, A->n_cols, A->rowptr,
                                                             A->colind, line_bytes, w, acc);
            else
                k_feature_chunks<false><<<cgrid, 256, 0, s>>>(long_rows, max_long, chunk_off, A->n_cols, A->rowptr,
                                                              A->colind, line_bytes, w, acc);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(t_host_acc, acc, sizeof(FeatAcc),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "feature pass");

    const FeatAcc& h = *t_host_acc;
    u64 err = h.err;
    if (A->n_rows == 0 && A->nnz != 0) err |= 2;
    if (err) {
        std::string m = "invalid CSR:";
        if (err & 1) m += " rowptr[0] != 0;";
        if (err & 2) m += " rowptr[n_rows] != nnz;";
        if (err & 4) m += " rowptr decreasing or out of [0, nnz];";
        if (err & 8) m += " column index out of [0, n_cols);";
        if (err & 16) m += " columns not strictly increasing within a row;";
        return fail(SPMV_ERR_INVALID_CSR, m);
    }
    if (!out) return SPMV_OK;

    spmv_features_t f = {};
    const int64_t N = A->n_rows, M = A->n_cols, NNZ = A->nnz;
    f.n_rows = N; f.n_cols = M; f.nnz = NNZ;
    f.line_bytes = line_bytes;
    f.l2_bytes = dev.l2_bytes;
    f.working_set_bytes = 4 * (N + 1) + 12 * NNZ + 8 * M + 8 * N;
    f.nnz_min = N > 0 ? (int64_t)~h.nnz_min_c : 0;
    f.nnz_max = (int64_t)h.nnz_max;
    f.nnz_sum = h.nnz_sum;
    f.nnz_sumsq_lo = h.nnz_sumsq;
    f.nnz_sumsq_hi = 0;
    f.bw_min = N > 0 ? (int64_t)~h.bw_min_c : 0;
    f.bw_max = (int64_t)h.bw_max;
    f.bw_sum = h.bw_sum;
    f.bw_sumsq_lo = h.bw_sq_lo;
    f.bw_sumsq_hi = h.bw_sq_hi;
    f.disp_sum = h.disp_sum;
    f.disp_sumsq_lo = h.disp_sq_lo;
    f.disp_sumsq_hi = h.disp_sq_hi;
    f.clust_sum = h.clust_sum;
    f.ngroups_sum = h.ngroups_sum;
    f.misses_sum = h.misses_sum;

    f.size = f.working_set_bytes <= f.l2_bytes ? 1.0 : 0.0;
    if (N > 0 && M > 0) f.density = (double)NNZ / ((double)N * (double)M);
    if (N > 0) {
        const double q32 = 1.0 / 4294967296.0;
        const double dn = (double)N;
        const u128 bw_s2 = ((u128)f.bw_sumsq_hi << 64) | f.bw_sumsq_lo;
        const u128 dq_s2 = ((u128)f.disp_sumsq_hi << 64) | f.disp_sumsq_lo;
        f.nnz_avg = (double)f.nnz_sum / dn;
        f.nnz_sd = sd_from_sums((u64)N, f.nnz_sum, (u128)f.nnz_sumsq_lo);
        f.bw_avg = (double)f.bw_sum / dn;
        f.bw_sd = sd_from_sums((u64)N, f.bw_sum, bw_s2);
        f.disp_avg = ((double)f.disp_sum / dn) * q32;
        f.disp_sd = sd_from_sums((u64)N, f.disp_sum, dq_s2) * q32;
        f.clustering = ((double)f.clust_sum / dn) * q32;
        f.miss_ratio = (double)f.misses_sum / dn;
    }
    const double dens = f.density > 0x1p-64 ? f.density : 0x1p-64;
    f.vec[0] = (float)f.size;
    f.vec[1] = (float)log2(dens);
    f.vec[2] = lg1p((double)f.nnz_min);
    f.vec[3] = lg1p((double)f.nnz_max);
    f.vec[4] = lg1p(f.nnz_avg);
    f.vec[5] = lg1p(f.nnz_sd);
    f.vec[6] = lg1p((double)f.bw_min);
    f.vec[7] = lg1p((double)f.bw_max);
    f.vec[8] = lg1p(f.bw_avg);
    f.vec[9] = lg1p(f.bw_sd);
    f.vec[10] = (float)f.disp_avg;
    f.vec[11] = (float)f.disp_sd;
    f.vec[12] = (float)f.clustering;
    f.vec[13] = lg1p(f.miss_ratio);
    f.vec[14] = lg1p((double)N);
    f.vec[15] = lg1p((double)NNZ);
    *out = f;
    return SPMV_OK;
}

}  // namespace spmvlib
