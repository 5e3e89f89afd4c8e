// Profiling runs of the profiling-based classifier (Section 3.2.1).
//
// The baseline is CSR SpMV under the paper's default partitioning: a static
// 1-D row partition with (as nearly as possible) equal nonzeros per worker.
// On the GPU a worker is one warp; the number of workers is the number of
// warps the device keeps resident at once, so every worker runs from the
// start of the launch.  A worker walks its rows in order, 32/T rows at a
// time, each row by a group of T lanes (T from the mean row length).
//   noxmiss: the same kernel with every column index replaced by 0, which
//            removes the irregular accesses to x;
//   inflate: the same kernel with 64-bit rowptr and colind, which enlarges
//            the working set;
//   balance: the same kernel recording each worker's start and end time
//            (%globaltimer); the metric is the launch span over the mean
//            worker duration, i.e. what balancing the load could reclaim.
#include <algorithm>
#include <chrono>
#include <vector>

#include "common.cuh"
#include "rowdot.cuh"

namespace spmvlib {
namespace {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounds[w] = smallest row i with rowptr[i] >= floor(w * nnz / W); bounds[W] = N.
__global__ void k_static_bounds(int64_t n_rows, int64_t nnz, const int* __restrict__ rp,
                                int64_t n_workers, int64_t* __restrict__ bounds)
{
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w > n_workers) return;
    if (w == n_workers) { bounds[w] = n_rows; return; }
    const int64_t target = (w * nnz) / n_workers;
    int64_t lo = 0, hi = n_rows;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)rp[mid] < target) lo = mid + 1; else hi = mid;
    }
    bounds[w] = lo;
}

template <typename IT>
__global__ void k_widen(int64_t n, const int* __restrict__ in, IT* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (IT)in[i];
}

template <typename IT, bool STAMP, int T>
__global__ void __launch_bounds__(256)
k_base(int64_t n_workers, const int64_t* __restrict__ bounds, const IT* __restrict__ rp,
       const IT* __restrict__ ci, const double* __restrict__ v, const double* __restrict__ x,
       double* __restrict__ y, unsigned long long* __restrict__ stamps)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_workers) return;
    unsigned long long t0 = 0;
    if (STAMP) t0 = global_ns();
    const int64_t rb = bounds[w], re = bounds[w + 1];
    for (int64_t r0 = rb; r0 < re; r0 += 32 / T) {
        const int64_t row = r0 + lane / T;
        int64_t b = 0, e = 0;
        if (row < re) { b = (int64_t)rp[row]; e = (int64_t)rp[row + 1]; }
        const double s = dev::group_sum(
            dev::row_partial<T, 4>(b, e, lane & (T - 1), dev::ColPlain<IT>{ci}, v, x), T);
        if ((lane & (T - 1)) == 0 && row < re) y[row] = s;
    }
    if (STAMP && lane == 0) {
        const unsigned long long t1 = global_ns();
        stamps[2 * w] = t0;
        stamps[2 * w + 1] = t1;
    }
}

template <typename IT, bool STAMP>
cudaError_t launch_base(int T, int64_t n_workers, const int64_t* bounds, const IT* rp,
                        const IT* ci, const double* v, const double* x, double* y,
                        unsigned long long* st, cudaStream_t s)
{
    const unsigned grid = (unsigned)((n_workers * 32 + 255) / 256);
    switch (T) {
#define SPMV_BASE_CASE(TT) \
    case TT: k_base<IT, STAMP, TT><<<grid, 256, 0, s>>>(n_workers, bounds, rp, ci, v, x, y, st); break;
        SPMV_BASE_CASE(1) SPMV_BASE_CASE(2) SPMV_BASE_CASE(4) SPMV_BASE_CASE(8)
        SPMV_BASE_CASE(16) SPMV_BASE_CASE(32)
#undef SPMV_BASE_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

double median(std::vector<double> v)
{
    std::sort(v.begin(), v.end());
    const size_t n = v.size();
    return n % 2 ? v[n / 2] : 0.5 * (v[n / 2 - 1] + v[n / 2]);
}

struct DevBuf {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    ~DevBuf() { if (p) cudaFreeAsync(p, s); }
};

// Gather probe: a checksum of x over A's column indices in storage order --
// the 64-bit bit patterns of x[colind[j]] added modulo 2^64 -- with U
// independent gathers in flight per thread and no floating-point work (an
// FP64 add per element would cost as much FP64 issue as the SpMV's DFMA).
// Its time is the cost of A's x accesses alone in CSR storage order.
constexpr int kGT = 256;

template <int U>
__global__ void __launch_bounds__(kGT)
k_gather_probe(int64_t nnz, const int* __restrict__ ci, const double* __restrict__ x,
               unsigned long long* __restrict__ part)
{
    __shared__ unsigned long long red[kGT / 32];
    const int64_t stride = (int64_t)gridDim.x * kGT;
    int64_t i = (int64_t)blockIdx.x * kGT + threadIdx.x;
    unsigned long long acc = 0;
    const unsigned long long* xb = reinterpret_cast<const unsigned long long*>(x);
    for (; i + (U - 1) * stride < nnz; i += U * stride) {
        int c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) c[u] = __ldcs(ci + i + u * stride);
        unsigned long long v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = __ldg(xb + c[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) acc += v[u];
    }
    for (; i < nnz; i += stride) acc += __ldg(xb + __ldcs(ci + i));
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < kGT / 32; ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

__global__ void k_sum_parts(int n, const unsigned long long* __restrict__ part,
                            unsigned long long* __restrict__ out)
{
    unsigned long long s = 0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s;
}

}  // namespace

}  // namespace spmvlib

using namespace spmvlib;

extern "C" spmv_status spmv_gather_probe(const spmv_csr_t* A, const double* x, uint64_t* sum,
                                         spmv_stream_t stream)
{
    clear_error();
    if (!A || !x || !sum) return fail(SPMV_ERR_INVALID_ARG, "spmv_gather_probe: NULL argument");
    if (A->nnz < 0 || (A->nnz > 0 && !A->colind))
        return fail(SPMV_ERR_INVALID_ARG, "spmv_gather_probe: bad matrix");
    DeviceInfo dev;
    spmv_status st = current_device(&dev);
    if (st != SPMV_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int grid = dev.sm_count * 8;
    unsigned long long* part = nullptr;
    SPMV_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&part), sizeof(unsigned long long) * grid, s));
    k_gather_probe<4><<<grid, kGT, 0, s>>>(A->nnz, A->colind, x, part);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_sum_parts<<<1, 1, 0, s>>>(grid, part, reinterpret_cast<unsigned long long*>(sum));
        e = cudaGetLastError();
    }
    cudaError_t ef = cudaFreeAsync(part, s);
    if (e == cudaSuccess) e = ef;
    if (e != cudaSuccess) return cuda_fail(e, "spmv_gather_probe");
    return SPMV_OK;
}

namespace spmvlib {
namespace {

// The probes' shared set-up: the static equal-nonzero partition over W
// workers, the zeroed column indices (noxmiss) and the 64-bit index copies
// (inflate), all stream-ordered buffers released with the object.
struct Probes {
    int64_t W = 0;
    int T = 1;
    DevBuf b_bounds, b_zero, b_rp64, b_ci64, b_st;
    int64_t* bounds = nullptr;
    int* zero_ci = nullptr;
    int64_t* rp64 = nullptr;
    int64_t* ci64 = nullptr;
    unsigned long long* stamps = nullptr;

    spmv_status setup(const spmv_csr_t* A, int64_t n_workers, cudaStream_t s)
    {
        W = n_workers;
        const int64_t N = A->n_rows, NNZ = A->nnz;
        T = auto_threads_per_row((double)NNZ / (double)N / 4.0);
        b_bounds.s = b_zero.s = b_rp64.s = b_ci64.s = b_st.s = s;
        SPMV_CUDA_TRY(cudaMallocAsync(&b_bounds.p, sizeof(int64_t) * (W + 1), s));
        SPMV_CUDA_TRY(cudaMallocAsync(&b_zero.p, sizeof(int) * NNZ, s));
        SPMV_CUDA_TRY(cudaMallocAsync(&b_rp64.p, sizeof(int64_t) * (N + 1), s));
        SPMV_CUDA_TRY(cudaMallocAsync(&b_ci64.p, sizeof(int64_t) * NNZ, s));
        SPMV_CUDA_TRY(cudaMallocAsync(&b_st.p, sizeof(unsigned long long) * 2 * W, s));
        bounds = static_cast<int64_t*>(b_bounds.p);
        zero_ci = static_cast<int*>(b_zero.p);
        rp64 = static_cast<int64_t*>(b_rp64.p);
        ci64 = static_cast<int64_t*>(b_ci64.p);
        stamps = static_cast<unsigned long long*>(b_st.p);
        k_static_bounds<<<(unsigned)((W + 1 + 255) / 256), 256, 0, s>>>(N, NNZ, A->rowptr, W, bounds);
        SPMV_CUDA_TRY(cudaGetLastError());
        SPMV_CUDA_TRY(cudaMemsetAsync(zero_ci, 0, sizeof(int) * NNZ, s));
        k_widen<int64_t><<<(unsigned)((N + 1 + 255) / 256), 256, 0, s>>>(N + 1, A->rowptr, rp64);
        SPMV_CUDA_TRY(cudaGetLastError());
        k_widen<int64_t><<<(unsigned)((NNZ + 255) / 256), 256, 0, s>>>(NNZ, A->colind, ci64);
        SPMV_CUDA_TRY(cudaGetLastError());
        return SPMV_OK;
    }

    // One run of probe `which`: 0 baseline, 1 noxmiss, 2 inflate, 3 balance
    // (the baseline recording each worker's start and end time).
    cudaError_t run(int which, const spmv_csr_t* A, const double* x, double* y, cudaStream_t s) const
    {
        switch (which) {
            case 0: return launch_base<int, false>(T, W, bounds, A->rowptr, A->colind, A->val, x, y, nullptr, s);
            case 1: return launch_base<int, false>(T, W, bounds, A->rowptr, zero_ci, A->val, x, y, nullptr, s);
            case 2: return launch_base<int64_t, false>(T, W, bounds, rp64, ci64, A->val, x, y, nullptr, s);
            case 3: return launch_base<int, true>(T, W, bounds, A->rowptr, A->colind, A->val, x, y, stamps, s);
            default: return cudaErrorInvalidValue;
        }
    }
};

// Workers of the probes: as many warps as the device keeps resident.
spmv_status default_workers(const DeviceInfo& dev, int64_t* W)
{
    int per_sm = 0;
    SPMV_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_base<int, false, 4>, 256, 0));
    if (per_sm < 1) per_sm = 1;
    *W = (int64_t)dev.sm_count * per_sm * 8;
    return SPMV_OK;
}

spmv_status probe_args(const spmv_csr_t* A, const double* x, const char* who)
{
    if (!x) return fail(SPMV_ERR_INVALID_ARG, std::string(who) + ": NULL argument");
    spmv_status st = check_csr_args(A);
    if (st != SPMV_OK) return st;
    if (A->n_rows == 0 || A->nnz == 0)
        return fail(SPMV_ERR_UNSUPPORTED, std::string(who) + ": empty matrix has nothing to profile");
    return SPMV_OK;
}

}  // namespace
}  // namespace spmvlib

extern "C" spmv_status spmv_profile(const spmv_csr_t* A, const double* x, int32_t reps,
                                    spmv_profile_t* out, spmv_stream_t stream)
{
    clear_error();
    const auto wall0 = std::chrono::steady_clock::now();
    if (!out) return fail(SPMV_ERR_INVALID_ARG, "spmv_profile: NULL argument");
    spmv_status st = probe_args(A, x, "spmv_profile");
    if (st != SPMV_OK) return st;
    if (reps <= 0) reps = 5;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceInfo dev;
    st = current_device(&dev);
    if (st != SPMV_OK) return st;
    st = run_feature_pass(A, 128, nullptr, s);  // validation only
    if (st != SPMV_OK) return st;

    int64_t W = 0;
    if ((st = default_workers(dev, &W)) != SPMV_OK) return st;
    Probes pr;
    if ((st = pr.setup(A, W, s)) != SPMV_OK) return st;
    DevBuf b_y;
    b_y.s = s;
    SPMV_CUDA_TRY(cudaMallocAsync(&b_y.p, sizeof(double) * A->n_rows, s));
    double* y = static_cast<double*>(b_y.p);

    cudaEvent_t e0, e1;
    SPMV_CUDA_TRY(cudaEventCreate(&e0));
    SPMV_CUDA_TRY(cudaEventCreate(&e1));
    auto time_runs = [&](int which, double* ms_out) -> cudaError_t {
        std::vector<double> t;
        for (int r = 0; r <= reps; ++r) {
            cudaError_t e = cudaEventRecord(e0, s);
            if (e != cudaSuccess) return e;
            if ((e = pr.run(which, A, x, y, s)) != cudaSuccess) return e;
            if ((e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
            float ms = 0.f;
            if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return e;
            if (r > 0) t.push_back(ms);  // the first run is the warm-up
        }
        *ms_out = median(t);
        return cudaSuccess;
    };
    spmv_profile_t p = {};
    cudaError_t e = time_runs(0, &p.t_base_ms);
    if (e == cudaSuccess) e = time_runs(1, &p.t_noxmiss_ms);
    if (e == cudaSuccess) e = time_runs(2, &p.t_inflate_ms);
    std::vector<unsigned long long> h(2 * W);
    if (e == cudaSuccess) e = pr.run(3, A, x, y, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), pr.stamps, sizeof(unsigned long long) * 2 * W,
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "spmv_profile runs");

    unsigned long long tmin = ~0ull, tmax = 0;
    double sum = 0.0;
    for (int64_t w = 0; w < W; ++w) {
        tmin = std::min(tmin, h[2 * w]);
        tmax = std::max(tmax, h[2 * w + 1]);
        sum += (double)(h[2 * w + 1] - h[2 * w]);
    }
    p.t_span_ms = (double)(tmax - tmin) * 1e-6;
    p.t_worker_mean_ms = sum / (double)W * 1e-6;
    p.s_noxmiss = p.t_base_ms / p.t_noxmiss_ms;
    p.s_inflate = p.t_inflate_ms / p.t_base_ms;
    p.s_balance = p.t_worker_mean_ms > 0 ? p.t_span_ms / p.t_worker_mean_ms : 1.0;
    p.n_workers = (int32_t)W;
    p.reps = reps;
    // buffers are released (stream-ordered) by the DevBuf destructors; the
    // wall time includes everything up to here
    p.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    *out = p;
    return SPMV_OK;
}

extern "C" spmv_status spmv_profile_outputs(const spmv_csr_t* A, const double* x, int64_t n_workers,
                                            int64_t* bounds, double* y_base, double* y_noxmiss,
                                            double* y_inflate, double* y_balance,
                                            spmv_stream_t stream)
{
    clear_error();
    spmv_status st = probe_args(A, x, "spmv_profile_outputs");
    if (st != SPMV_OK) return st;
    if (n_workers < 0 || n_workers > ((int64_t)1 << 26))
        return fail(SPMV_ERR_INVALID_ARG, "spmv_profile_outputs: n_workers must be in 0..2^26");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceInfo dev;
    if ((st = current_device(&dev)) != SPMV_OK) return st;
    if ((st = run_feature_pass(A, 128, nullptr, s)) != SPMV_OK) return st;  // validation only
    int64_t W = n_workers;
    if (W == 0 && (st = default_workers(dev, &W)) != SPMV_OK) return st;
    Probes pr;
    if ((st = pr.setup(A, W, s)) != SPMV_OK) return st;
    double* ys[4] = {y_base, y_noxmiss, y_inflate, y_balance};
    for (int which = 0; which < 4; ++which)
        if (ys[which]) SPMV_CUDA_TRY(pr.run(which, A, x, ys[which], s));
    if (bounds)
        SPMV_CUDA_TRY(cudaMemcpyAsync(bounds, pr.bounds, sizeof(int64_t) * (W + 1),
                                      cudaMemcpyDeviceToDevice, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    return SPMV_OK;
}
