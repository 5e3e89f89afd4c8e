// DYNAMIC variant (IMB class; Table 2's dynamic scheduling, on the GPU with
// work splitting).  Rows are put in tiers by length at prepare time:
//   S  len <= lim_s            contiguous chunks of rows, T_s lanes per row
//   M1 lim_s < len <= 64       compact list, 8 lanes per row
//   M2 64 < len <= seg         compact list, a warp per row
//   L  len > seg               split into segments of `seg` nonzeros, a warp
//                              per segment; the warp that finishes a row's
//                              last segment (an atomic ticket per row) sums
//                              its partials in segment order (deterministic)
// Persistent warps take items from one atomic counter, longest work first
// (L segments, M2, M1, then S chunks); the last warp to finish resets the
// counter.  Every tier spends one DFMA per nonzero plus log2(lanes) shuffle
// adds per row or segment.  Lists are filled with atomics, so their order
// may vary between prepares; each row's value does not.
#include <algorithm>

#include "common.cuh"
#include "rowdot.cuh"

namespace spmvlib {
namespace {

using namespace dev;
constexpr int kDB = 256;
constexpr int kM1Lim = 64;

// row-length histogram: bucket 0 holds empty rows, bucket b >= 1 holds
// 2^(b-1) < len <= 2^b, except that length 1 also lands in bucket 1
__global__ void k_len_hist(int64_t n_rows, const int* __restrict__ rp, unsigned long long* hist)
{
    __shared__ unsigned long long h[33];
    if (threadIdx.x < 33) h[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rows;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int len = rp[i + 1] - rp[i];
        const int b = len <= 1 ? len : 32 - __clz(len - 1);
        atomicAdd(&h[b], 1ull);
    }
    __syncthreads();
    if (threadIdx.x < 33 && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

struct Lists {
    int* m1; int* m2; int* lrow;
    unsigned* count;  // [0] m1, [1] m2, [2] long
};

__global__ void k_classify(int64_t n_rows, const int* __restrict__ rp, int lim_s, int seg, Lists L)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rows;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int len = rp[i + 1] - rp[i];
        if (len <= lim_s) continue;
        if (len <= kM1Lim) L.m1[atomicAdd(&L.count[0], 1u)] = (int)i;
        else if (len <= seg) L.m2[atomicAdd(&L.count[1], 1u)] = (int)i;
        else L.lrow[atomicAdd(&L.count[2], 1u)] = (int)i;
    }
}

// exclusive scan of segment counts of the long rows (one CTA)
__global__ void k_seg_offsets(int n_long, const int* __restrict__ lrow, const int* __restrict__ rp,
                              int seg, int* __restrict__ seg_off)
{
    __shared__ int part[1024];
    int carry = 0;
    for (int base = 0; base < n_long; base += 1024) {
        const int p = base + threadIdx.x;
        int c = 0;
        if (p < n_long) {
            const int r = lrow[p];
            c = (rp[r + 1] - rp[r] + seg - 1) / seg;
        }
        part[threadIdx.x] = c;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int t = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (p < n_long) seg_off[p] = carry + part[threadIdx.x] - c;
        carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) seg_off[n_long] = carry;
}

struct DynArgs {
    int64_t n_rows;
    const int* rp; const int* ci; const double* v; const double* x; double* y;
    const int* m1; const int* m2; const int* lrow; const int* seg_off;
    int n_m1, n_m2, n_long, n_seg, seg, lim_s, chunk_rows;
    double* partial;
    unsigned* counter;
    unsigned* ticket;
};

template <int TS>
__global__ void __launch_bounds__(kDB) k_dyn(DynArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t n_chunks = (a.n_rows + a.chunk_rows - 1) / a.chunk_rows;
    const int64_t n_m1_items = (a.n_m1 + 3) / 4;
    const int64_t i_m2 = a.n_seg, i_m1 = i_m2 + a.n_m2, i_s = i_m1 + n_m1_items;
    const int64_t total = i_s + n_chunks;
    const unsigned total_warps = gridDim.x * (kDB / 32);
    const ColPlain<int> col{a.ci};
    for (;;) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(a.counter, 1u);
        it = __shfl_sync(FULL, it, 0);
        if ((int64_t)it >= total) break;
        if ((int64_t)it < i_m2) {
            // segment of a long row: find its row by binary search over seg_off
            int lo = 0, hi = a.n_long - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.seg_off[mid] <= (int)it) lo = mid; else hi = mid - 1;
            }
            const int r = a.lrow[lo];
            const int64_t b = (int64_t)a.rp[r] + (int64_t)((int)it - a.seg_off[lo]) * a.seg;
            const int64_t e = min((int64_t)a.rp[r + 1], b + a.seg);
            const double s = group_sum(row_partial<32, 8>(b, e, lane, col, a.v, a.x), 32);
            if (lane == 0) {
                // the row's last segment to finish sums its partials in
                // segment order and resets the row's ticket (nothing waits)
                a.partial[it] = s;
                __threadfence();
                const int sb = a.seg_off[lo], se = a.seg_off[lo + 1];
                if (atomicAdd(a.ticket + lo, 1u) == (unsigned)(se - sb - 1)) {
                    __threadfence();
                    double t = 0.0;
                    for (int i = sb; i < se; ++i) t += __ldcg(a.partial + i);
                    a.y[r] = t;
                    a.ticket[lo] = 0u;
                }
            }
        } else if ((int64_t)it < i_m1) {
            const int r = a.m2[it - i_m2];
            const double s = group_sum(row_partial<32, 4>(a.rp[r], a.rp[r + 1], lane, col, a.v, a.x), 32);
            if (lane == 0) a.y[r] = s;
        } else if ((int64_t)it < i_s) {
            const int q = (int)(it - i_m1) * 4 + (lane >> 3);
            int64_t b = 0, e = 0;
            int r = -1;
            if (q < a.n_m1) { r = a.m1[q]; b = a.rp[r]; e = a.rp[r + 1]; }
            const double s = group_sum(row_partial<8, 4>(b, e, lane & 7, col, a.v, a.x), 8);
            if ((lane & 7) == 0 && r >= 0) a.y[r] = s;
        } else {
            const int64_t rbeg = (int64_t)(it - i_s) * a.chunk_rows;
            const int64_t rend = min(rbeg + a.chunk_rows, a.n_rows);
            for (int64_t r0 = rbeg; r0 < rend; r0 += 32 / TS) {
                const int64_t row = r0 + lane / TS;
                int64_t b = 0, e = 0;
                bool mine = false;
                if (row < rend) {
                    b = a.rp[row];
                    e = a.rp[row + 1];
                    mine = e - b <= a.lim_s;
                    if (!mine) b = e = 0;
                }
                const double s = group_sum(row_partial<TS, 4>(b, e, lane & (TS - 1), col, a.v, a.x), TS);
                if ((lane & (TS - 1)) == 0 && mine) a.y[row] = s;
            }
        }
    }
    if (lane == 0) {
        __threadfence();
        const unsigned done = atomicAdd(a.counter + 1, 1u);
        if (done == total_warps - 1) {
            a.counter[0] = 0u;
            a.counter[1] = 0u;
        }
    }
}

template <int TS>
cudaError_t launch_dyn_t(const DynArgs& a, int sm_count, cudaStream_t s)
{
    static LaunchCache cache;
    int per_sm = 0;
    cudaError_t e = cached_occupancy(cache, k_dyn<TS>, kDB, 0, &per_sm);
    if (e != cudaSuccess) return e;
    k_dyn<TS><<<(unsigned)(sm_count * per_sm), kDB, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Builds the tiers.  When threads_per_row is 0 it is chosen from the
// row-length histogram and written back into P->c.
spmv_status dyn_prepare(spmv_prepared* P, cudaStream_t s)
{
    const spmv_csr_t& A = P->A;
    DynPlan& d = P->dyn;
    if (d.seg <= 0) d.seg = 2048;
    // 1. row-length histogram -> lanes per short row
    unsigned long long* dh = nullptr;
    unsigned long long hh[33] = {0};
    SPMV_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&dh), sizeof(hh), s));
    cudaError_t e = cudaMemsetAsync(dh, 0, sizeof(hh), s);
    const unsigned grid = (unsigned)std::min<int64_t>((A.n_rows + 255) / 256, (int64_t)P->sm_count * 8);
    if (e == cudaSuccess && A.n_rows > 0) {
        k_len_hist<<<grid, 256, 0, s>>>(A.n_rows, A.rowptr, dh);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hh, dh, sizeof(hh), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(dh, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "row-length histogram");
    if (P->c.threads_per_row == 0) {
        // upper edge of the median row's length bucket / 8, as a power of two in 1..32
        unsigned long long acc = 0;
        int med = 0;
        for (int b = 0; b <= 32; ++b) {
            acc += hh[b];
            if (2 * acc >= (unsigned long long)A.n_rows) { med = b >= 31 ? (1 << 30) : (1 << b); break; }
        }
        P->c.threads_per_row = auto_threads_per_row(med / 8.0);
    }
    const int ts = P->c.threads_per_row;
    d.lim_s = std::min(16 * ts, d.seg);
    d.chunk_rows = 8 * (32 / ts);
    // 2. tier lists (capacities bounded by nnz / (tier minimum length))
    const int64_t cap_m1 = std::min<int64_t>(A.n_rows, A.nnz / (d.lim_s + 1) + 1);
    const int64_t cap_m2 = std::min<int64_t>(A.n_rows, A.nnz / (kM1Lim + 1) + 1);
    const int64_t cap_l = std::min<int64_t>(A.n_rows, A.nnz / (d.seg + 1) + 1);
    spmv_status st;
    if ((st = prepared_alloc(P, reinterpret_cast<void**>(&d.m1), 4 * cap_m1)) != SPMV_OK) return st;
    if ((st = prepared_alloc(P, reinterpret_cast<void**>(&d.m2), 4 * cap_m2)) != SPMV_OK) return st;
    if ((st = prepared_alloc(P, reinterpret_cast<void**>(&d.lrow), 4 * cap_l)) != SPMV_OK) return st;
    if ((st = prepared_alloc(P, reinterpret_cast<void**>(&d.seg_off), 4 * (cap_l + 1))) != SPMV_OK) return st;
    // counter words: [0] work items taken, [1] warps done, [2..4] list sizes
    if ((st = prepared_alloc(P, reinterpret_cast<void**>(&P->counter), 4 * 8)) != SPMV_OK) return st;
    SPMV_CUDA_TRY(cudaMemsetAsync(P->counter, 0, 32, s));
    unsigned* cnt = P->counter + 2;
    Lists L{d.m1, d.m2, d.lrow, cnt};
    if (A.n_rows > 0) {
        k_classify<<<grid, 256, 0, s>>>(A.n_rows, A.rowptr, d.lim_s, d.seg, L);
        SPMV_CUDA_TRY(cudaGetLastError());
    }
    unsigned hc[3] = {0, 0, 0};
    SPMV_CUDA_TRY(cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    d.n_m1 = (int)hc[0];
    d.n_m2 = (int)hc[1];
    d.n_long = (int)hc[2];
    // 3. long-row segments
    d.n_seg = 0;
    if (d.n_long > 0) {
        k_seg_offsets<<<1, 1024, 0, s>>>(d.n_long, d.lrow, A.rowptr, d.seg, d.seg_off);
        SPMV_CUDA_TRY(cudaGetLastError());
        int ns = 0;
        SPMV_CUDA_TRY(cudaMemcpyAsync(&ns, d.seg_off + d.n_long, 4, cudaMemcpyDeviceToHost, s));
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
        d.n_seg = ns;
        if ((st = prepared_alloc(P, reinterpret_cast<void**>(&d.partial), 8 * (int64_t)ns)) != SPMV_OK ||
            (st = prepared_alloc(P, reinterpret_cast<void**>(&d.ticket), 4 * (int64_t)d.n_long)) != SPMV_OK)
            return st;
        SPMV_CUDA_TRY(cudaMemsetAsync(d.ticket, 0, 4 * (size_t)d.n_long, s));
    }
    P->n_blocks = d.n_seg + d.n_m2 + (d.n_m1 + 3) / 4 + (A.n_rows + d.chunk_rows - 1) / d.chunk_rows;
    return SPMV_OK;
}

cudaError_t launch_dyn(const spmv_prepared* P, const double* x, double* y, cudaStream_t s)
{
    const spmv_csr_t& A = P->A;
    if (A.n_rows == 0) return cudaSuccess;
    const DynPlan& d = P->dyn;
    DynArgs a{A.n_rows, A.rowptr, A.colind, A.val, x, y, d.m1, d.m2, d.lrow, d.seg_off,
              d.n_m1, d.n_m2, d.n_long, d.n_seg, d.seg, d.lim_s, d.chunk_rows, d.partial, P->counter,
              d.ticket};
    cudaError_t e;
    switch (P->c.threads_per_row) {
        case 1: e = launch_dyn_t<1>(a, P->sm_count, s); break;
        case 2: e = launch_dyn_t<2>(a, P->sm_count, s); break;
        case 4: e = launch_dyn_t<4>(a, P->sm_count, s); break;
        case 8: e = launch_dyn_t<8>(a, P->sm_count, s); break;
        case 16: e = launch_dyn_t<16>(a, P->sm_count, s); break;
        case 32: e = launch_dyn_t<32>(a, P->sm_count, s); break;
        default: return cudaErrorInvalidValue;
    }
    return e;
}

}  // namespace spmvlib
