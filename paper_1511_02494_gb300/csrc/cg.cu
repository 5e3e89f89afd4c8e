// Conjugate gradients around the library's SpMV (Section 1 names iterative
// solvers as the setting in which SpMV's selection overhead is amortised).
//
// Every iteration: q = A p (the inner prepared SpMV, e.g. COMPRESSED with
// FP32 or BF16 values), alpha = rs / (p.q), x += alpha p, r -= alpha q,
// rs' = r.r, beta = rs'/rs, p = r + beta p.  Every `refine` iterations the
// residual is instead recomputed in FP64 as r = b - A x with the exact
// prepared SpMV and the search direction restarts from it (p = r): iterative
// refinement with CG sweeps on the low-precision operator.  Vectors,
// dot products and scalars are FP64 and stay on the device: there is no host
// synchronisation inside the loop, so the loop can run from a CUDA graph.
//
// Dot products are deterministic: each block writes its partial sum, and the
// last block to finish (an atomic ticket, no waiting) adds the partials in
// block order and updates the scalars.
#include <math.h>

#include "common.cuh"

namespace spmvlib {
namespace {

constexpr int kCT = 256;

struct CgState {
    double rs, rs_new, pq, alpha, beta;
    unsigned ticket;
    unsigned pad;
};

__device__ __forceinline__ double block_reduce(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = lane < kCT / 32 ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

// Called by every thread of every block after its partial is stored by
// thread 0.  Returns true in exactly one block (the last), whose threads then
// see every partial.
__device__ __forceinline__ bool last_block(unsigned* ticket)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    return last;
}

__device__ __forceinline__ double sum_partials(const double* part, double* red)
{
    double v = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kCT) v += part[i];
    return block_reduce(v, red);
}

enum Finish { kAlpha = 0, kBeta = 1, kInit = 2, kRestart = 3 };

// FINISH == kAlpha: pq = p.q, alpha = rs / pq
template <int FINISH>
__global__ void __launch_bounds__(kCT)
k_dot_pq(int64_t n, const double* __restrict__ p, const double* __restrict__ q,
         double* __restrict__ part, CgState* st)
{
    __shared__ double red[kCT / 32];
    double v = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kCT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kCT)
        v = fma(p[i], q[i], v);
    v = block_reduce(v, red);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
    if (!last_block(&st->ticket)) return;
    const double s = sum_partials(part, red);
    if (threadIdx.x == 0) {
        st->pq = s;
        st->alpha = st->rs / s;
        st->ticket = 0;
    }
}

// x += alpha p and then either r -= alpha q (RECOMPUTE = false) or
// r = b - q where q holds A x (RECOMPUTE = true); rs' = r.r; the last block
// sets beta = rs'/rs (0 after a recomputation: the search restarts from the
// new residual), rs = rs' and records sqrt(rs') in resid[t].
template <bool UPDATE_X, bool RECOMPUTE, int FINISH>
__global__ void __launch_bounds__(kCT)
k_update(int64_t n, double* __restrict__ x, const double* __restrict__ p, double* __restrict__ r,
         const double* __restrict__ q, const double* __restrict__ b, double* __restrict__ part,
         CgState* st, double* __restrict__ resid, int t)
{
    __shared__ double red[kCT / 32];
    const double alpha = st->alpha;
    double v = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kCT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kCT) {
        if (UPDATE_X) x[i] = fma(alpha, p[i], x[i]);
        double ri;
        if (RECOMPUTE) ri = b[i] - q[i];
        else ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        v = fma(ri, ri, v);
    }
    v = block_reduce(v, red);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
    if (!last_block(&st->ticket)) return;
    const double s = sum_partials(part, red);
    if (threadIdx.x == 0) {
        if (FINISH == kInit) {
            st->rs = s;
        } else if (FINISH == kRestart) {
            st->beta = 0.0;  // the search restarts from the recomputed residual
            st->rs = s;
        } else {
            st->beta = s / st->rs;
            st->rs = s;
        }
        if (resid) resid[t] = sqrt(s);
        st->ticket = 0;
    }
}

// x += alpha p only (the refinement step recomputes r from the new x)
__global__ void __launch_bounds__(kCT)
k_axpy_x(int64_t n, double* __restrict__ x, const double* __restrict__ p, const CgState* st)
{
    const double alpha = st->alpha;
    for (int64_t i = (int64_t)blockIdx.x * kCT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kCT)
        x[i] = fma(alpha, p[i], x[i]);
}

// p = r + beta p  (INIT: p = r)
template <bool INIT>
__global__ void __launch_bounds__(kCT)
k_update_p(int64_t n, double* __restrict__ p, const double* __restrict__ r, const CgState* st)
{
    const double beta = INIT ? 0.0 : st->beta;
    for (int64_t i = (int64_t)blockIdx.x * kCT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kCT)
        p[i] = INIT ? r[i] : fma(beta, p[i], r[i]);
}

struct CgBufs {
    double *r = nullptr, *p = nullptr, *q = nullptr, *part = nullptr;
    CgState* st = nullptr;
};

spmv_status enqueue_cg(const spmv_prepared* Pi, const spmv_prepared* Pe, const double* b,
                       double* x, int iters, int refine, double* resid, const CgBufs& w,
                       unsigned grid, cudaStream_t s)
{
    const int64_t n = Pi->A.n_rows;
    spmv_status st;
    // r0 = b - A x0 (exact), p0 = r0
    if ((st = spmv(Pe, x, w.q, reinterpret_cast<spmv_stream_t>(s))) != SPMV_OK) return st;
    k_update<false, true, kInit><<<grid, kCT, 0, s>>>(n, x, w.p, w.r, w.q, b, w.part, w.st, resid, 0);
    k_update_p<true><<<grid, kCT, 0, s>>>(n, w.p, w.r, w.st);
    for (int t = 1; t <= iters; ++t) {
        if ((st = spmv(Pi, w.p, w.q, reinterpret_cast<spmv_stream_t>(s))) != SPMV_OK) return st;
        k_dot_pq<kAlpha><<<grid, kCT, 0, s>>>(n, w.p, w.q, w.part, w.st);
        if (refine > 0 && t % refine == 0) {
            k_axpy_x<<<grid, kCT, 0, s>>>(n, x, w.p, w.st);
            if ((st = spmv(Pe, x, w.q, reinterpret_cast<spmv_stream_t>(s))) != SPMV_OK) return st;
            k_update<false, true, kRestart><<<grid, kCT, 0, s>>>(n, x, w.p, w.r, w.q, b, w.part,
                                                                 w.st, resid, t);
        } else {
            k_update<true, false, kBeta><<<grid, kCT, 0, s>>>(n, x, w.p, w.r, w.q, b, w.part,
                                                              w.st, resid, t);
        }
        k_update_p<false><<<grid, kCT, 0, s>>>(n, w.p, w.r, w.st);
    }
    SPMV_CUDA_TRY(cudaGetLastError());
    return SPMV_OK;
}

}  // namespace
}  // namespace spmvlib

using namespace spmvlib;

extern "C" spmv_status spmv_cg(const spmv_prepared_t* A_inner, const spmv_prepared_t* A_exact,
                               const double* b, double* x, int32_t iters, int32_t refine_every,
                               double* resid, int32_t use_graph, spmv_stream_t stream)
{
    clear_error();
    if (!A_inner || !b || !x || iters < 0 || refine_every < 0)
        return fail(SPMV_ERR_INVALID_ARG, "spmv_cg: bad argument");
    const spmv_prepared* Pi = A_inner;
    const spmv_prepared* Pe = A_exact ? A_exact : A_inner;
    if (Pi->A.n_rows != Pi->A.n_cols || Pe->A.n_rows != Pi->A.n_rows || Pe->A.n_cols != Pi->A.n_cols)
        return fail(SPMV_ERR_INVALID_ARG, "spmv_cg: square matrices of equal size required");
    const int64_t n = Pi->A.n_rows;
    if (n == 0) return SPMV_OK;
    DeviceInfo dev;
    spmv_status st = current_device(&dev);
    if (st != SPMV_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int64_t g = (n + kCT - 1) / kCT;
    if (g > (int64_t)dev.sm_count * 4) g = (int64_t)dev.sm_count * 4;
    const unsigned grid = (unsigned)g;
    CgBufs w;
    SPMV_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&w.r), 8 * n, s));
    SPMV_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&w.p), 8 * n, s));
    SPMV_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&w.q), 8 * n, s));
    SPMV_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&w.part), 8 * (size_t)grid, s));
    SPMV_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&w.st), sizeof(CgState), s));
    SPMV_CUDA_TRY(cudaMemsetAsync(w.st, 0, sizeof(CgState), s));
    if (use_graph) {
        // capture on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured), then launch on the caller's
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaStream_t cs = nullptr;
        SPMV_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            st = enqueue_cg(Pi, Pe, b, x, iters, refine_every, resid, w, grid, cs);
            e = cudaStreamEndCapture(cs, &graph);
        }
        cudaStreamDestroy(cs);
        if (st != SPMV_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "spmv_cg graph");
    } else {
        st = enqueue_cg(Pi, Pe, b, x, iters, refine_every, resid, w, grid, s);
        if (st != SPMV_OK) return st;
    }
    cudaFreeAsync(w.r, s);
    cudaFreeAsync(w.p, s);
    cudaFreeAsync(w.q, s);
    cudaFreeAsync(w.part, s);
    cudaFreeAsync(w.st, s);
    SPMV_CUDA_TRY(cudaGetLastError());
    return SPMV_OK;
}
