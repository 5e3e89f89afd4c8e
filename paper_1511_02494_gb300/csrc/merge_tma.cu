// MERGE variant, pipelined form (IMB class; also the most even split for any
// matrix): merge-path tiles of 256 * IPT items (row ends + nonzeros), each
// CTA of a persistent grid walking its tiles in a 3-stage shared-memory ring.
//
// Per tile the CTA's thread 0 issues bulk asynchronous copies (the TMA
// engine's cp.async.bulk) of the tile's values, column indices and row ends
// into the next free stage, counted on that stage's mbarrier; the few
// elements outside the 16-byte-aligned bulk ranges are loaded by plain loads.
// While later tiles stream in, the CTA
//   1. gathers x for the ready stage and overwrites each value with val * x,
//   2. walks its thread's IPT merge-path items from shared memory,
//   3. joins the threads' partial rows with a CTA-wide segmented scan,
// writing every row that ends in the tile and the tile's trailing partial
// row (carry) for k_merge_fixup.  Waits are bounded (2 s); on timeout the
// kernel records SPMV_ERR_TIMEOUT in *status and returns.
#include "common.cuh"
#include "ptx.cuh"
#include "rowdot.cuh"

namespace spmvlib {
namespace {

constexpr int kThreads = 256;
constexpr uint64_t kWaitLimitNs = 2000000000ull;

template <int IPT, int STAGES>
struct __align__(16) TileSmem {
    static constexpr int ITEMS = kThreads * IPT;
    // a bulk range may extend one 16-byte unit past each end of the wanted
    // range: up to 1 extra double or 3 extra ints at either end
    double v[STAGES][ITEMS + 2];  // values, then products
    int ci[STAGES][ITEMS + 8];    // column indices
    int re[STAGES][ITEMS + 8];    // row ends rowptr[r0+1 .. r1]
    int meta[STAGES][4];          // r0, r1, n0, n1
    uint64_t bar[STAGES];
    double wsum[kThreads / 32];
    int wflag[kThreads / 32];
};

// Elements [a, b) of an array of `len` elements of `esz` bytes are wanted in
// shared memory.  The bulk copy covers [lo, hi): lo rounded down and hi
// rounded up to 16 bytes, except that hi is rounded down when rounding up
// would pass the end of the array; [hi, b) is then left to plain loads.
struct Span { int lo, hi; };
__device__ __forceinline__ Span bulk_span(int a, int b, int len, int per16) {
    const int lo = a & ~(per16 - 1);
    int hi = (b + per16 - 1) & ~(per16 - 1);
    if (hi > len) hi = b & ~(per16 - 1);
    if (hi < lo) hi = lo;
    return {lo, hi};
}

template <int IPT, int STAGES>
__global__ void __launch_bounds__(kThreads, IPT == 8 ? 2 : 3)
k_merge_tma(int64_t n_tiles, int nnz, int n_rows, const int* __restrict__ rp,
            const int* __restrict__ ci, const double* __restrict__ v,
            const double* __restrict__ x, double* __restrict__ y,
            const int32_t* __restrict__ mrow, const int32_t* __restrict__ mnz,
            int32_t* __restrict__ carry_row, double* __restrict__ carry_val,
            unsigned* __restrict__ status)
{
    using S = TileSmem<IPT, STAGES>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S& sm = *reinterpret_cast<S*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t G = gridDim.x;
    const int64_t my_tiles = n_tiles > (int64_t)blockIdx.x ? (n_tiles - 1 - blockIdx.x) / G + 1 : 0;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) ptx::mbar_init(&sm.bar[s], 1);
        ptx::fence_mbar_init();
    }
    // thread 0's prefetched metadata of the next tile to issue
    int nx0 = 0, nx1 = 0, nx2 = 0, nx3 = 0;
    auto fetch_meta = [&](int64_t i) {
        if (i < my_tiles) {
            const int64_t t = (int64_t)blockIdx.x + i * G;
            nx0 = mrow[t]; nx1 = mrow[t + 1]; nx2 = mnz[t]; nx3 = mnz[t + 1];
        }
    };
    // Thread 0 only: stage tile i (metadata prefetched in nx*), prefetch i+1.
    auto issue = [&](int64_t i) {
        if (i >= my_tiles) return;
        const int s = (int)(i % STAGES);
        const int r0 = nx0, r1 = nx1, n0 = nx2, n1 = nx3;
        fetch_meta(i + 1);
        sm.meta[s][0] = r0; sm.meta[s][1] = r1; sm.meta[s][2] = n0; sm.meta[s][3] = n1;
        const Span sv = bulk_span(n0, n1, nnz, 2), sc = bulk_span(n0, n1, nnz, 4);
        const Span se = bulk_span(r0 + 1, r1 + 1, n_rows + 1, 4);
        // rare: elements past the last 16-byte boundary of an array
        for (int k = sv.hi; k < n1; ++k) sm.v[s][k - sv.lo] = v[k];
        for (int k = sc.hi; k < n1; ++k) sm.ci[s][k - sc.lo] = ci[k];
        for (int k = se.hi > r0 + 1 ? se.hi : r0 + 1; k <= r1; ++k) sm.re[s][k - se.lo] = rp[k];
        ptx::fence_proxy_async_smem();
        const uint32_t bv = (uint32_t)(sv.hi - sv.lo) * 8u, bc = (uint32_t)(sc.hi - sc.lo) * 4u;
        const uint32_t be = (uint32_t)(se.hi - se.lo) * 4u;
        ptx::mbar_arrive_expect_tx(&sm.bar[s], bv + bc + be);
        if (bv) ptx::bulk_g2s(&sm.v[s][0], v + sv.lo, bv, &sm.bar[s]);
        if (bc) ptx::bulk_g2s(&sm.ci[s][0], ci + sc.lo, bc, &sm.bar[s]);
        if (be) ptx::bulk_g2s(&sm.re[s][0], rp + se.lo, be, &sm.bar[s]);
    };
    // views of stage s for the tile whose metadata it holds
    struct View { int r0, r1, n0, n1; double* vs; const int* cs; const int* es; };
    auto view = [&](int s) {
        View q;
        q.r0 = sm.meta[s][0]; q.r1 = sm.meta[s][1]; q.n0 = sm.meta[s][2]; q.n1 = sm.meta[s][3];
        const Span sv = bulk_span(q.n0, q.n1, nnz, 2), sc = bulk_span(q.n0, q.n1, nnz, 4);
        const Span se = bulk_span(q.r0 + 1, q.r1 + 1, n_rows + 1, 4);
        q.vs = &sm.v[s][q.n0 - sv.lo];
        q.cs = &sm.ci[s][q.n0 - sc.lo];
        q.es = &sm.re[s][q.r0 + 1 - se.lo];
        return q;
    };
    uint32_t parity = 0;
    bool failed = false;
    auto wait_stage = [&](int s) {
        if (!ptx::wait_bounded(&sm.bar[s], (parity >> s) & 1u, kWaitLimitNs)) failed = true;
        parity ^= 1u << s;
    };

    if (tid == 0) {
        fetch_meta(0);
        for (int i = 0; i < STAGES - 1; ++i) issue(i);
    }
    __syncthreads();
    // products of tile 0
    int c[IPT];
    double a[IPT], xv[IPT];
    if (my_tiles > 0) {
        wait_stage(0);
        const View q = view(0);
        const int nn = q.n1 - q.n0;
#pragma unroll
        for (int u = 0; u < IPT; ++u) {
            const int k = tid + u * kThreads;
            if (k < nn) q.vs[k] = q.vs[k] * dev::ldx(x + q.cs[k]);
        }
    }
    if (__syncthreads_or(failed)) {
        if (tid == 0) atomicOr(status, 1u);
        return;
    }

    for (int64_t i = 0; i < my_tiles; ++i) {
        if (tid == 0) issue(i + STAGES - 1);
        const int s = (int)(i % STAGES), sn = (int)((i + 1) % STAGES);
        const bool has_next = i + 1 < my_tiles;
        // gathers of the next tile, in flight during this tile's walk
        int nn_next = 0;
        View qn;
        if (has_next) {
            wait_stage(sn);
            qn = view(sn);
            nn_next = qn.n1 - qn.n0;
#pragma unroll
            for (int u = 0; u < IPT; ++u) {
                const int k = tid + u * kThreads;
                c[u] = k < nn_next ? qn.cs[k] : 0;
                a[u] = k < nn_next ? qn.vs[k] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < IPT; ++u) xv[u] = dev::ldx(x + c[u]);
        }
        // this thread's IPT consecutive merge-path items of tile i
        const View q = view(s);
        const int nr = q.r1 - q.r0, nn = q.n1 - q.n0, total = nr + nn;
        const int d = min(tid * IPT, total), dend = min(d + IPT, total);
        int lo = max(0, d - nn), hi = min(d, nr);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (q.es[mid] <= q.n0 + d - mid - 1) lo = mid + 1; else hi = mid;
        }
        int ri = lo, nj = d - lo;
        double run = 0.0, first_val = 0.0;
        int first_row = -1;
        for (int k = d; k < dend; ++k) {
            if (ri < nr && q.es[ri] <= q.n0 + nj) {
                if (first_row < 0) { first_row = ri; first_val = run; }
                else y[q.r0 + ri] = run;
                run = 0.0;
                ++ri;
            } else {
                run += q.vs[nj];
                ++nj;
            }
        }
        // CTA segmented scan: a thread that ended a row starts a new segment
        double val = run;
        int flag = first_row >= 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double vu = __shfl_up_sync(dev::FULL, val, o);
            const int fu = __shfl_up_sync(dev::FULL, flag, o);
            if (lane >= o) {
                if (!flag) val += vu;
                flag |= fu;
            }
        }
        if (lane == 31) { sm.wsum[w] = val; sm.wflag[w] = flag; }
        if (__syncthreads_or(failed)) {
            if (tid == 0) {
                atomicOr(status, 1u);
                for (int qq = 0; qq < STAGES; ++qq)
                    ptx::wait_bounded(&sm.bar[qq], (parity >> qq) & 1u, kWaitLimitNs / 8);
            }
            __syncthreads();
            return;
        }
        double pv = 0.0;
        for (int qq = 0; qq < w; ++qq) pv = sm.wflag[qq] ? sm.wsum[qq] : pv + sm.wsum[qq];
        double ex_v = __shfl_up_sync(dev::FULL, val, 1);
        int ex_f = __shfl_up_sync(dev::FULL, flag, 1);
        if (lane == 0) { ex_v = 0.0; ex_f = 0; }
        const double cin = ex_f ? ex_v : pv + ex_v;
        if (first_row >= 0) y[q.r0 + first_row] = first_val + cin;
        if (tid == kThreads - 1) {
            const int64_t t = (int64_t)blockIdx.x + i * G;
            carry_row[t] = q.r1;
            carry_val[t] = flag ? val : pv + val;
        }
        // products of the next tile
        if (has_next) {
#pragma unroll
            for (int u = 0; u < IPT; ++u) {
                const int k = tid + u * kThreads;
                if (k < nn_next) qn.vs[k] = a[u] * xv[u];
            }
        }
        __syncthreads();
    }
}

// Adds each tile's trailing partial row to that row, summing the tiles of one
// row in tile order (deterministic).  carry_row is non-decreasing.
// Adds each tile's carry to its row in tile order.  As in k_window_fixup:
// nothing when a bounded wait of the tile kernel gave up (*status != 0,
// carry_row then holds entries of an earlier call), and no entry outside
// [0, n_rows) is used.
__global__ void k_tile_fixup(int64_t n_tiles, int64_t n_rows, const int32_t* __restrict__ carry_row,
                             const double* __restrict__ carry_val,
                             const unsigned* __restrict__ status, double* __restrict__ y)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_tiles || (status && *status != 0u)) return;
    const int r = carry_row[p];
    if (r < 0 || r >= n_rows) return;
    if (p > 0 && carry_row[p - 1] == r) return;
    double s = 0.0;
    for (int64_t q = p; q < n_tiles && carry_row[q] == r; ++q) s += carry_val[q];
    y[r] += s;
}

template <int IPT, int STAGES>
cudaError_t launch_tma_cfg(const spmv_csr_t& A, const int32_t* mrow, const int32_t* mnz,
                           int64_t n_tiles, int32_t* carry_row, double* carry_val,
                           unsigned* status, int sm_count, const double* x, double* y,
                           cudaStream_t s)
{
    static LaunchCache cache;
    const size_t smem = sizeof(TileSmem<IPT, STAGES>);
    int per_sm = 0;
    cudaError_t e = cached_occupancy(cache, k_merge_tma<IPT, STAGES>, kThreads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)sm_count * per_sm;
    if (grid > n_tiles) grid = n_tiles;
    k_merge_tma<IPT, STAGES><<<(unsigned)grid, kThreads, smem, s>>>(
        n_tiles, (int)A.nnz, (int)A.n_rows, A.rowptr, A.colind, A.val, x, y, mrow, mnz, carry_row,
        carry_val, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tile_fixup<<<(unsigned)((n_tiles + 255) / 256), 256, 0, s>>>(n_tiles, A.n_rows, carry_row,
                                                                  carry_val, status, y);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tile_fixup(int64_t n_tiles, int64_t n_rows, const int32_t* carry_row,
                              const double* carry_val, const unsigned* status, double* y,
                              cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    k_tile_fixup<<<(unsigned)((n_tiles + 255) / 256), 256, 0, s>>>(n_tiles, n_rows, carry_row,
                                                                  carry_val, status, y);
    return cudaGetLastError();
}

bool tma_aligned(const spmv_csr_t& A)
{
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    return al(A.rowptr) && (A.nnz == 0 || (al(A.colind) && al(A.val)));
}

cudaError_t launch_merge_tma(const spmv_csr_t& A, int tile_items, const int32_t* mrow,
                             const int32_t* mnz, int64_t n_tiles, int32_t* carry_row,
                             double* carry_val, unsigned* status, int sm_count, const double* x,
                             double* y, cudaStream_t s)
{
    if (A.n_rows == 0) return cudaSuccess;
    // tile_items selects (items per thread, stages): 1024 -> (4, 4),
    // 1536 -> (6, 3), 2048 -> (8, 3)
    switch (tile_items) {
        case 1024:
            return launch_tma_cfg<4, 4>(A, mrow, mnz, n_tiles, carry_row, carry_val, status,
                                        sm_count, x, y, s);
        case 1536:
            return launch_tma_cfg<6, 3>(A, mrow, mnz, n_tiles, carry_row, carry_val, status,
                                        sm_count, x, y, s);
        case 2048:
            return launch_tma_cfg<8, 3>(A, mrow, mnz, n_tiles, carry_row, carry_val, status,
                                        sm_count, x, y, s);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace spmvlib
