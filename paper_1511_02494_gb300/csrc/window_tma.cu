// STREAM variant, pipelined: fixed windows of B nonzeros.
//
// Window k covers the nonzeros [kB, (k+1)B).  It owns the rows that start in
// it (R_k <= r < R_{k+1}, R_k = first row with rowptr >= kB) and, when the
// row before R_k reaches into the window, computes that row's partial sum as
// the window's carry.  Every row is written once by its owner; carries are
// added in window order by k_window_fixup (deterministic, no float atomics).
//
// Persistent CTAs walk their windows through a ring of shared-memory stages
// filled by bulk asynchronous copies (cp.async.bulk, completed on an mbarrier
// per stage).  Windows start on multiples of B, so the value and column
// copies are 16-byte aligned and the same size for every window but the
// last.  Per window the CTA
//   1. gathers x[col] of all B nonzeros into shared memory (8 independent
//      loads per thread, no floating point),
//   2. reduces each row from shared memory with exactly one DFMA per
//      nonzero, T lanes per row, T chosen per window to minimise the warp
//      FP64 instructions (DFMAs of the longest lane + log2 T shuffle adds).
// FP64 throughput is about 2 DFMA per clock per SM on this GPU, within a
// factor of 1.2 of what HBM needs to stream the matrix, so the kernel spends
// no FP64 instruction beyond that.  Waits are bounded (2 s); on timeout the
// kernel sets *status and returns.
#include "common.cuh"
#include "ptx.cuh"
#include "rowdot.cuh"

namespace spmvlib {
namespace {

constexpr int kWT = 256;
constexpr uint64_t kWinWaitNs = 2000000000ull;

template <int B, int STAGES>
struct __align__(16) WinSmem {
    static constexpr int RP_CAP = B / 2 + 72;  // staged rowptr entries (multiple of 4)
    double v[STAGES][B];
    int ci[STAGES][B];
    int rp[STAGES][RP_CAP];
    int meta[STAGES][4];  // R_k, R_{k+1}, first staged rowptr index, rowptr staged (1/0)
    uint64_t bar[STAGES];
    double xg[B];
    double red[kWT / 32];
};

struct Span { int lo, hi; };
__device__ __forceinline__ Span rp_span(int a, int b, int len) {
    const int lo = a & ~3;
    int hi = (b + 3) & ~3;
    if (hi > len) hi = b & ~3;
    if (hi < lo) hi = lo;
    return {lo, hi};
}

template <int B, int STAGES>
__global__ void __launch_bounds__(kWT, B == 1024 ? 3 : 2)
k_window(int64_t n_win, int nnz, int n_rows, const int* __restrict__ rp,
         const int* __restrict__ ci, const double* __restrict__ v, const double* __restrict__ x,
         double* __restrict__ y, const int32_t* __restrict__ blocks,
         int32_t* __restrict__ carry_row, double* __restrict__ carry_val,
         unsigned* __restrict__ status)
{
    using S = WinSmem<B, STAGES>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S& sm = *reinterpret_cast<S*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t G = gridDim.x;
    const int64_t my = n_win > (int64_t)blockIdx.x ? (n_win - 1 - blockIdx.x) / G + 1 : 0;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) ptx::mbar_init(&sm.bar[s], 1);
        ptx::fence_mbar_init();
    }
    int nR0 = 0, nR1 = 0;  // thread 0: prefetched R_k, R_{k+1} of the next window to issue
    auto fetch = [&](int64_t i) {
        if (i < my) {
            const int64_t k = (int64_t)blockIdx.x + i * G;
            nR0 = blocks[k];
            nR1 = blocks[k + 1];
        }
    };
    auto issue = [&](int64_t i) {
        if (i >= my) return;
        const int s = (int)(i % STAGES);
        const int64_t k = (int64_t)blockIdx.x + i * G;
        const int R0 = nR0, R1 = nR1;
        fetch(i + 1);
        const int base = (int)(k * B);
        const int cnt = min(B, nnz - base);
        const int fv = cnt & ~1, fc = cnt & ~3;
        for (int t = fv; t < cnt; ++t) sm.v[s][t] = v[base + t];  // last window only
        for (int t = fc; t < cnt; ++t) sm.ci[s][t] = ci[base + t];
        const Span sp = rp_span(R0, R1 + 1, n_rows + 1);
        const bool staged = (R1 + 1 - sp.lo) + 3 <= S::RP_CAP;
        if (staged)
            for (int r = (sp.hi > R0 ? sp.hi : R0); r <= R1; ++r) sm.rp[s][r - sp.lo] = rp[r];
        sm.meta[s][0] = R0;
        sm.meta[s][1] = R1;
        sm.meta[s][2] = sp.lo;
        sm.meta[s][3] = staged ? 1 : 0;
        ptx::fence_proxy_async_smem();
        const uint32_t bv = (uint32_t)fv * 8u, bc = (uint32_t)fc * 4u;
        const uint32_t br = staged ? (uint32_t)(sp.hi - sp.lo) * 4u : 0u;
        ptx::mbar_arrive_expect_tx(&sm.bar[s], bv + bc + br);
        if (bv) ptx::bulk_g2s(&sm.v[s][0], v + base, bv, &sm.bar[s]);
        if (bc) ptx::bulk_g2s(&sm.ci[s][0], ci + base, bc, &sm.bar[s]);
        if (br) ptx::bulk_g2s(&sm.rp[s][0], rp + sp.lo, br, &sm.bar[s]);
    };

    __syncthreads();
    if (tid == 0) {
        fetch(0);
        for (int i = 0; i < STAGES - 1; ++i) issue(i);
    }
    uint32_t parity = 0;
    for (int64_t i = 0; i < my; ++i) {
        if (tid == 0) issue(i + STAGES - 1);
        const int s = (int)(i % STAGES);
        const bool ok = ptx::wait_bounded(&sm.bar[s], (parity >> s) & 1u, kWinWaitNs);
        parity ^= 1u << s;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(status, 1u);
                for (int q = 0; q < STAGES; ++q)
                    ptx::wait_bounded(&sm.bar[q], (parity >> q) & 1u, kWinWaitNs / 8);
            }
            __syncthreads();
            return;
        }
        const int64_t k = (int64_t)blockIdx.x + i * G;
        const int base = (int)(k * B);
        const int cnt = min(B, nnz - base);
        const int R0 = sm.meta[s][0], R1 = sm.meta[s][1], rplo = sm.meta[s][2];
        const bool staged = sm.meta[s][3] != 0;
        const double* vs = sm.v[s];

        // 1. gather x of the window's nonzeros
        {
            constexpr int PER = B / kWT;
            int c[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int t = tid + u * kWT;
                c[u] = t < cnt ? sm.ci[s][t] : 0;
            }
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int t = tid + u * kWT;
                if (t < cnt) sm.xg[t] = dev::ldx(x + c[u]);
            }
        }
        __syncthreads();

        // 2. rows: item 0 is the carry row when the row before R0 reaches in
        auto rpv = [&](int r) -> int { return staged ? sm.rp[s][r - rplo] : rp[r]; };
        const int first_owned = rpv(R0);
        const int has_carry = (k > 0 && first_owned > base) ? 1 : 0;
        const int n_items = has_carry + (R1 - R0);
        if (tid == 0 && !has_carry) carry_row[k] = -1;
        // local [lo, hi) of item it
        auto item_range = [&](int it, int& lo, int& hi, int& row) {
            if (has_carry && it == 0) {
                row = R0 - 1;
                lo = 0;
                hi = min(first_owned, base + cnt) - base;
            } else {
                row = R0 + it - has_carry;
                lo = rpv(row) - base;
                hi = min(rpv(row + 1), base + cnt) - base;
            }
        };
        if (n_items == 1 && cnt > kWT) {
            // a single row covers the window: the whole CTA reduces it
            int lo, hi, row;
            item_range(0, lo, hi, row);
            double acc = 0.0;
#pragma unroll 4
            for (int j = lo + tid; j < hi; j += kWT) acc = fma(vs[j], sm.xg[j], acc);
            acc = dev::group_sum(acc, 32);
            if (lane == 0) sm.red[wid] = acc;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int q = 0; q < kWT / 32; ++q) t += sm.red[q];
                if (has_carry) { carry_row[k] = row; carry_val[k] = t; }
                else y[row] = t;
            }
        } else if (n_items > 0) {
            // lanes per row minimising warp FP64 instructions
            const int avg = (cnt + n_items - 1) / n_items;
            int T = 1, best = 0x7fffffff;
            for (int t = 1, lg = 0; t <= 32; t <<= 1, ++lg) {
                const int cost = ((n_items * t + 31) >> 5) * ((avg + t - 1) / t + lg);
                if (cost < best) { best = cost; T = t; }
            }
            const int groups = kWT / T, g = tid / T, gl = tid & (T - 1);
            for (int it0 = 0; it0 < n_items; it0 += groups) {
                const int it = it0 + g;
                int lo = 0, hi = 0, row = 0;
                if (it < n_items) item_range(it, lo, hi, row);
                double acc = 0.0;
#pragma unroll 4
                for (int j = lo + gl; j < hi; j += T) acc = fma(vs[j], sm.xg[j], acc);
                for (int o = T >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(dev::FULL, acc, o);
                if (gl == 0 && it < n_items) {
                    if (has_carry && it == 0) { carry_row[k] = row; carry_val[k] = acc; }
                    else y[row] = acc;
                }
            }
        }
        __syncthreads();
    }
}

// Adds each window's carry to its row, summing the windows of one row in
// window order.  Windows without a carry hold -1; the windows carrying one
// row are consecutive.  When a bounded wait of the window kernel gave up
// (*status != 0) the windows it skipped never wrote their carry_row entry,
// which then holds whatever an earlier call left: the fix-up does nothing
// (that call's y is incomplete and reported so).  Entries outside
// [0, n_rows) are skipped as well, so no store leaves y.
__global__ void k_window_fixup(int64_t n_win, int64_t n_rows, const int32_t* __restrict__ carry_row,
                               const double* __restrict__ carry_val,
                               const unsigned* __restrict__ status, double* __restrict__ y)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_win || *status != 0u) return;
    const int r = carry_row[p];
    if (r < 0 || r >= n_rows) return;
    if (p > 0 && carry_row[p - 1] == r) return;
    double s = 0.0;
    for (int64_t q = p; q < n_win && carry_row[q] == r; ++q) s += carry_val[q];
    y[r] += s;
}

template <int B, int STAGES>
cudaError_t launch_win_cfg(const spmv_csr_t& A, const int32_t* blocks, int64_t n_win,
                           int32_t* carry_row, double* carry_val, unsigned* status,
                           int sm_count, const double* x, double* y, cudaStream_t s)
{
    static LaunchCache cache;
    const size_t smem = sizeof(WinSmem<B, STAGES>);
    int per_sm = 0;
    cudaError_t e = cached_occupancy(cache, k_window<B, STAGES>, kWT, smem, &per_sm);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)sm_count * per_sm;
    if (grid > n_win) grid = n_win;
    k_window<B, STAGES><<<(unsigned)grid, kWT, smem, s>>>(n_win, (int)A.nnz, (int)A.n_rows,
                                                          A.rowptr, A.colind, A.val, x, y, blocks,
                                                          carry_row, carry_val, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_window_fixup<<<(unsigned)((n_win + 255) / 256), 256, 0, s>>>(n_win, A.n_rows, carry_row,
                                                                   carry_val, status, y);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_window_fixup(int64_t n_win, int64_t n_rows, const int32_t* carry_row,
                                const double* carry_val, const unsigned* status, double* y,
                                cudaStream_t s)
{
    if (n_win <= 0) return cudaSuccess;
    k_window_fixup<<<(unsigned)((n_win + 255) / 256), 256, 0, s>>>(n_win, n_rows, carry_row,
                                                                   carry_val, status, y);
    return cudaGetLastError();
}

cudaError_t launch_window(const spmv_csr_t& A, int block_nnz, const int32_t* blocks, int64_t n_win,
                          int32_t* carry_row, double* carry_val, unsigned* status, int sm_count,
                          const double* x, double* y, cudaStream_t s)
{
    if (A.n_rows == 0) return cudaSuccess;
    switch (block_nnz) {
        case 1024:
            return launch_win_cfg<1024, 4>(A, blocks, n_win, carry_row, carry_val, status, sm_count,
                                           x, y, s);
        case 2048:
            return launch_win_cfg<2048, 3>(A, blocks, n_win, carry_row, carry_val, status, sm_count,
                                           x, y, s);
        default:
            return cudaErrorInvalidValue;
    }
}

namespace {

// Self-test of the bounded wait the pipelined kernels use: one warp waits on
// a shared-memory mbarrier that expects one arrival.  arrive != 0: thread 0
// arrives first and the wait completes; arrive == 0: nothing arrives, the
// wait gives up after limit_ns and thread 0 records the timeout.  No copy is
// in flight, so the kernel simply returns.
__global__ void k_wait_check(uint64_t limit_ns, int arrive, unsigned* __restrict__ status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0) ptx::mbar_arrive(&bar);
    const bool done = ptx::wait_bounded(&bar, 0u, limit_ns);
    if (!done && threadIdx.x == 0) *status = 1u;
}

}  // namespace
}  // namespace spmvlib

using namespace spmvlib;

extern "C" spmv_status spmv_wait_check(int64_t limit_ns, int32_t arrive, spmv_stream_t stream)
{
    clear_error();
    if (limit_ns <= 0 || limit_ns > 2000000000ll)
        return fail(SPMV_ERR_INVALID_ARG, "spmv_wait_check: limit_ns must be in 1..2e9");
    DeviceInfo dev;
    spmv_status st = current_device(&dev);
    if (st != SPMV_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned* d = nullptr;
    unsigned h = 0;
    SPMV_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d), sizeof(unsigned), s));
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
        k_wait_check<<<1, 32, 0, s>>>((uint64_t)limit_ns, arrive ? 1 : 0, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    const cudaError_t ef = cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = ef;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "spmv_wait_check");
    if (h) return fail(SPMV_ERR_TIMEOUT, "spmv_wait_check: the bounded wait gave up, as the test asks");
    return SPMV_OK;
}

extern "C" spmv_status spmv_fixup_check(int32_t kind, int64_t n_parts, int64_t n_rows,
                                        const int32_t* carry_row, const double* carry_val,
                                        const uint32_t* status, double* y, spmv_stream_t stream)
{
    clear_error();
    if (kind != 0 && kind != 1)
        return fail(SPMV_ERR_INVALID_ARG, "spmv_fixup_check: kind must be 0 (STREAM) or 1 (MERGE)");
    if (n_parts < 0 || n_rows < 0 || n_rows > INT32_MAX)
        return fail(SPMV_ERR_INVALID_ARG, "spmv_fixup_check: bad size");
    if (n_parts > 0 && (!carry_row || !carry_val || !status || (n_rows > 0 && !y)))
        return fail(SPMV_ERR_INVALID_ARG, "spmv_fixup_check: NULL argument");
    DeviceInfo dev;
    spmv_status st = current_device(&dev);
    if (st != SPMV_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const unsigned* stw = reinterpret_cast<const unsigned*>(status);
    SPMV_CUDA_TRY(kind == 0 ? launch_window_fixup(n_parts, n_rows, carry_row, carry_val, stw, y, s)
                            : launch_tile_fixup(n_parts, n_rows, carry_row, carry_val, stw, y, s));
    return SPMV_OK;
}
