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

// Sub-warp of T lanes per row; a grid-stride loop over row groups.  Each lane
// examines elements j = b + lane + k T, four per pass, comparing each column
// with its predecessor in the row.
template <int T, bool FEATURES>
__global__ void __launch_bounds__(256)
k_feature_pass(int64_t n_rows, int64_t n_cols, int64_t nnz, const int* __restrict__ rp,
               const int* __restrict__ ci, int64_t line_bytes, FeatAcc* __restrict__ acc)
{
    constexpr int U = 4;
    __shared__ u64 s_red[8][kFields];
    __shared__ u64 s_err;
    const int lane = threadIdx.x & (T - 1);
    const int64_t groups_total = (int64_t)gridDim.x * (blockDim.x / T);
    u64 nnz_min_c = 0, nnz_max = 0, nnz_sum = 0, nnz_sq = 0;
    u64 bw_min_c = 0, bw_max = 0, bw_sum = 0, disp_sum = 0, clust_sum = 0, ng_sum = 0, ms_sum = 0;
    u128 bw_sq = 0, disp_sq = 0;
    u64 err = 0;
    if (threadIdx.x == 0) s_err = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (rp[0] != 0) err |= 1;
        if ((int64_t)rp[n_rows] != nnz) err |= 2;
    }
    const int64_t g0 = (int64_t)blockIdx.x * (blockDim.x / T) + threadIdx.x / T;
    const int64_t n_iter = (n_rows + groups_total - 1) / groups_total;
    for (int64_t it = 0; it < n_iter; ++it) {
        const int64_t row = g0 + it * groups_total;
        int64_t b = 0, e = 0;
        bool ok = row < n_rows;
        if (ok) {
            b = rp[row];
            e = rp[row + 1];
            if (b < 0 || e < b || e > nnz) { err |= 4; ok = false; b = e = 0; }
        }
        u64 ng = 0, ms = 0, bad = 0;
        for (int64_t j0 = b + lane; j0 < e; j0 += (int64_t)U * T) {
            int64_t c[U], cp[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t j = j0 + u * T;
                c[u] = j < e ? (int64_t)ci[j] : 0;
                cp[u] = (j < e && j > b) ? (int64_t)ci[j - 1] : 0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t j = j0 + u * T;
                if (j < e) {
                    if (c[u] < 0 || c[u] >= n_cols) bad |= 8;
                    if (j > b) {
                        const int64_t d = c[u] - cp[u];
                        if (d <= 0) bad |= 16;
                        ng += (d != 1);
                        ms += (8 * d > line_bytes);
                    }
                }
            }
        }
        for (int o = T >> 1; o > 0; o >>= 1) {
            ng += __shfl_xor_sync(FULL_MASK, ng, o);
            ms += __shfl_xor_sync(FULL_MASK, ms, o);
            bad |= __shfl_xor_sync(FULL_MASK, bad, o);
        }
        err |= bad;
        if (FEATURES && ok && lane == 0) {
            const u64 nz = (u64)(e - b);
            u64 bw = 0, dq = 0, cq = 0;
            if (nz > 0) {
                bw = (u64)((int64_t)ci[e - 1] - (int64_t)ci[b]);
                ng += 1;
                ms += 1;
                dq = (nz << 32) / (bw + 1);
                cq = (ng << 32) / nz;
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
    }
    // warp reduction, then block reduction, then one set of atomics per block
    for (int o = 16; o > 0; o >>= 1) err |= shfl_u64(err, o);
    const int w = threadIdx.x >> 5;
    if (FEATURES) {
        nnz_min_c = warp_max_u64(nnz_min_c);
        nnz_max = warp_max_u64(nnz_max);
        nnz_sum = warp_sum_u64(nnz_sum);
        nnz_sq = warp_sum_u64(nnz_sq);
        bw_min_c = warp_max_u64(bw_min_c);
        bw_max = warp_max_u64(bw_max);
        bw_sum = warp_sum_u64(bw_sum);
        bw_sq = warp_sum_u128(bw_sq);
        disp_sum = warp_sum_u64(disp_sum);
        disp_sq = warp_sum_u128(disp_sq);
        clust_sum = warp_sum_u64(clust_sum);
        ng_sum = warp_sum_u64(ng_sum);
        ms_sum = warp_sum_u64(ms_sum);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        if (err) atomicOr(&s_err, err);
        u64* r = s_red[w];
        r[0] = nnz_min_c; r[1] = nnz_max; r[2] = nnz_sum; r[3] = nnz_sq;
        r[4] = bw_min_c; r[5] = bw_max; r[6] = bw_sum;
        r[7] = (u64)bw_sq; r[8] = (u64)(bw_sq >> 64);
        r[9] = disp_sum; r[10] = (u64)disp_sq; r[11] = (u64)(disp_sq >> 64);
        r[12] = clust_sum; r[13] = ng_sum; r[14] = ms_sum; r[15] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        if (s_err) atomicOr(&acc->err, s_err);
        if (FEATURES) {
            u64 t[kFields] = {0};
            u128 bsq = 0, dsq = 0;
            for (int k = 0; k < nw; ++k) {
                const u64* r = s_red[k];
                t[0] = max(t[0], r[0]); t[1] = max(t[1], r[1]); t[2] += r[2]; t[3] += r[3];
                t[4] = max(t[4], r[4]); t[5] = max(t[5], r[5]); t[6] += r[6];
                bsq += ((u128)r[8] << 64) | r[7];
                t[9] += r[9];
                dsq += ((u128)r[11] << 64) | r[10];
                t[12] += r[12]; t[13] += r[13]; t[14] += r[14];
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

template <bool F>
cudaError_t launch_pass(int T, unsigned grid, cudaStream_t s, const spmv_csr_t* A,
                        int64_t line_bytes, FeatAcc* acc)
{
    switch (T) {
#define SPMV_FP_CASE(TT)                                                                 \
    case TT:                                                                             \
        k_feature_pass<TT, F><<<grid, 256, 0, s>>>(A->n_rows, A->n_cols, A->nnz, A->rowptr, \
                                                   A->colind, line_bytes, acc);          \
        break;
        SPMV_FP_CASE(1) SPMV_FP_CASE(2) SPMV_FP_CASE(4) SPMV_FP_CASE(8) SPMV_FP_CASE(16)
        SPMV_FP_CASE(32)
#undef SPMV_FP_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
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
        const int T = auto_threads_per_row((double)A->nnz / (double)A->n_rows / 4.0);
        int64_t blocks = (A->n_rows * T + 255) / 256;
        const int64_t cap = (int64_t)dev.sm_count * 16;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        e = out ? launch_pass<true>(T, (unsigned)blocks, s, A, line_bytes, acc)
                : launch_pass<false>(T, (unsigned)blocks, s, A, line_bytes, acc);
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
