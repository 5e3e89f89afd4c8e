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
//
// With a SLICED inner matrix without long rows (none above its cap) q = A p and p.q
// are one kernel, and when that matrix sums in FP32 the p update also writes
// p's FP32 copy, so no separate conversion of p runs per iteration.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "sliced.cuh"

namespace spmvlib {
namespace {

constexpr int kCT = 256;
// The vector kernels give each thread kUnr elements kCT apart per pass of
// the grid-stride loop and load all of them before any arithmetic, so a
// thread keeps several independent loads of every vector in flight.
constexpr int kUnr = 4;

__device__ __forceinline__ int64_t first_index() { return (int64_t)blockIdx.x * kCT * kUnr + threadIdx.x; }
__device__ __forceinline__ int64_t grid_step() { return (int64_t)gridDim.x * kCT * kUnr; }

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
    for (int64_t i0 = first_index(); i0 < n; i0 += grid_step()) {
        double pv[kUnr], qv[kUnr];
#pragma unroll
        for (int u = 0; u < kUnr; ++u) {
            const int64_t i = i0 + u * kCT;
            pv[u] = i < n ? p[i] : 0.0;
            qv[u] = i < n ? q[i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kUnr; ++u) v = fma(pv[u], qv[u], v);
    }
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
    for (int64_t i0 = first_index(); i0 < n; i0 += grid_step()) {
        double xv[kUnr], pv[kUnr], rv[kUnr], qv[kUnr];
#pragma unroll
        for (int u = 0; u < kUnr; ++u) {
            const int64_t i = i0 + u * kCT;
            const bool ok = i < n;
            if (UPDATE_X) {
                xv[u] = ok ? x[i] : 0.0;
                pv[u] = ok ? p[i] : 0.0;
            }
            rv[u] = ok ? (RECOMPUTE ? b[i] : r[i]) : 0.0;
            qv[u] = ok ? q[i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kUnr; ++u) {
            const int64_t i = i0 + u * kCT;
            if (i < n) {
                if (UPDATE_X) x[i] = fma(alpha, pv[u], xv[u]);
                const double ri = RECOMPUTE ? rv[u] - qv[u] : fma(-alpha, qv[u], rv[u]);
                r[i] = ri;
                v = fma(ri, ri, v);
            }
        }
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
    for (int64_t i0 = first_index(); i0 < n; i0 += grid_step()) {
        double xv[kUnr], pv[kUnr];
#pragma unroll
        for (int u = 0; u < kUnr; ++u) {
            const int64_t i = i0 + u * kCT;
            xv[u] = i < n ? x[i] : 0.0;
            pv[u] = i < n ? p[i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kUnr; ++u)
            if (i0 + u * kCT < n) x[i0 + u * kCT] = fma(alpha, pv[u], xv[u]);
    }
}

// p = r + beta p  (INIT: p = r); with p32, also its FP32 copy for a
// low-precision inner SpMV that sums in FP32 (the same rounding its own
// conversion of x would apply)
template <bool INIT>
__global__ void __launch_bounds__(kCT)
k_update_p(int64_t n, double* __restrict__ p, const double* __restrict__ r, const CgState* st,
           float* __restrict__ p32)
{
    const double beta = INIT ? 0.0 : st->beta;
    for (int64_t i0 = first_index(); i0 < n; i0 += grid_step()) {
        double pv[kUnr], rv[kUnr];
#pragma unroll
        for (int u = 0; u < kUnr; ++u) {
            const int64_t i = i0 + u * kCT;
            rv[u] = i < n ? r[i] : 0.0;
            pv[u] = !INIT && i < n ? p[i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kUnr; ++u) {
            const int64_t i = i0 + u * kCT;
            if (i < n) {
                const double v = INIT ? rv[u] : fma(beta, pv[u], rv[u]);
                p[i] = v;
                if (p32) p32[i] = __double2float_rn(v);
            }
        }
    }
}

// Fused q = A p and p.q for a SLICED inner matrix without long rows: each
// lane computes its row's q_i (dev::slice_value / slice_value_lp, the same
// arithmetic as the SLICED kernels) and adds p_i q_i to its block's partial;
// the last block sums the partials in block order and sets pq and alpha.
// Resident blocks per SM of the fused kernel: FP64 values fit 8 (32
// registers, two elements in flight per lane); the low-precision bodies need
// 40 registers, so 6.
template <typename VT>
constexpr int dot_blocks() { return sizeof(VT) == 8 ? 8 : 6; }
constexpr int kDotU = 2;

struct SlArgs {
    int64_t n_slices;
    const int* rowlen; const int* slice_len; const int64_t* slice_ptr; const int* perm;
    const int* col; const double* val; const uint16_t* off; const int* rowbase; const void* lowval;
    const void* scol;  // FP64 values: stored columns (int, or int16/int8 offsets from the row)
};

template <typename VT, bool OFF16, bool ACC32, typename CT = int>
__global__ void __launch_bounds__(kCT, dot_blocks<VT>())
k_sliced_dot(SlArgs a, const double* __restrict__ p, const float* __restrict__ p32,
             double* __restrict__ q, double* __restrict__ part, CgState* st)
{
    __shared__ double red[kCT / 32];
    const int lane = threadIdx.x & 31;
    const int64_t n_warps = (int64_t)gridDim.x * (kCT / 32);
    double contrib = 0.0;
    // grid-stride over slices (a few blocks per SM): few partials, few tickets
    for (int64_t s = ((int64_t)blockIdx.x * kCT + threadIdx.x) >> 5; s < a.n_slices; s += n_warps) {
        int row;
        double v;
        if constexpr (sizeof(VT) == 8)
            v = dev::slice_value<kDotU, CT>(s, lane, a.rowlen, a.slice_len, a.slice_ptr, a.perm,
                                            static_cast<const CT*>(a.scol), a.val, p, &row);
        else
            v = dev::slice_value_lp<OFF16 ? 2 : 1, VT, OFF16, ACC32>(s, lane, a.rowlen, a.slice_len, a.slice_ptr, a.perm,
                                                         a.col, a.off, a.rowbase,
                                                         static_cast<const VT*>(a.lowval), p, p32, &row);
        if (row >= 0) {
            q[row] = v;
            contrib = fma(p[row], v, contrib);
        }
    }
    contrib = block_reduce(contrib, red);
    if (threadIdx.x == 0) part[blockIdx.x] = contrib;
    if (!last_block(&st->ticket)) return;
    const double sum = sum_partials(part, red);
    if (threadIdx.x == 0) {
        st->pq = sum;
        st->alpha = st->rs / sum;
        st->ticket = 0;
    }
}

bool fusable(const spmv_prepared* P)
{
    return P->c.variant == SPMV_V7_SLICED && P->sl.n_long == 0 && P->sl.coding == 0 && P->A.n_rows > 0;
}

unsigned sliced_dot_grid(const spmv_prepared* P)
{
    const int64_t need = (32 * P->sl.n_slices + kCT - 1) / kCT;
    const int per_sm = P->sl.value_type == SPMV_VAL_F64 ? dot_blocks<double>() : dot_blocks<float>();
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)P->sm_count * per_sm));
}

cudaError_t launch_sliced_dot(const spmv_prepared* P, const double* p, double* q, double* part,
                              CgState* st, cudaStream_t s)
{
    const SlicedPlan& d = P->sl;
    SlArgs a{d.n_slices, d.rowlen, d.slice_len, d.slice_ptr, d.sigma > 1 ? d.perm : nullptr,
             d.col, d.val, d.off, d.rowbase, d.lowval, d.scol};
    const unsigned grid = sliced_dot_grid(P);
    if (d.value_type == SPMV_VAL_F64) {
        if (d.cbytes == 1)
            k_sliced_dot<double, false, false, int8_t><<<grid, kCT, 0, s>>>(a, p, nullptr, q, part, st);
        else if (d.cbytes == 2)
            k_sliced_dot<double, false, false, int16_t><<<grid, kCT, 0, s>>>(a, p, nullptr, q, part, st);
        else
            k_sliced_dot<double, false, false, int><<<grid, kCT, 0, s>>>(a, p, nullptr, q, part, st);
    } else {
#define SPMV_CG_SL(VT, O16, A32) k_sliced_dot<VT, O16, A32><<<grid, kCT, 0, s>>>(a, p, d.x32, q, part, st)
#define SPMV_CG_SL_VT(VT)                                                                  \
    if (d.off16) { if (d.acc32) SPMV_CG_SL(VT, true, true); else SPMV_CG_SL(VT, true, false); } \
    else { if (d.acc32) SPMV_CG_SL(VT, false, true); else SPMV_CG_SL(VT, false, false); }
        if (d.value_type == SPMV_VAL_F32) { SPMV_CG_SL_VT(float) } else { SPMV_CG_SL_VT(__nv_bfloat16) }
#undef SPMV_CG_SL_VT
#undef SPMV_CG_SL
    }
    return cudaGetLastError();
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
    // a SLICED inner matrix takes the fused q = A p, p.q kernel; when it sums
    // in FP32, p's FP32 copy is written by the p update
    const bool fused = fusable(Pi);
    float* p32 = fused && Pi->sl.acc32 ? Pi->sl.x32 : nullptr;
    // r0 = b - A x0 (exact), p0 = r0
    if ((st = spmv(Pe, x, w.q, reinterpret_cast<spmv_stream_t>(s))) != SPMV_OK) return st;
    k_update<false, true, kInit><<<grid, kCT, 0, s>>>(n, x, w.p, w.r, w.q, b, w.part, w.st, resid, 0);
    k_update_p<true><<<grid, kCT, 0, s>>>(n, w.p, w.r, w.st, p32);
    for (int t = 1; t <= iters; ++t) {
        if (fused) {
            SPMV_CUDA_TRY(launch_sliced_dot(Pi, w.p, w.q, w.part, w.st, s));
        } else {
            if ((st = spmv(Pi, w.p, w.q, reinterpret_cast<spmv_stream_t>(s))) != SPMV_OK) return st;
            k_dot_pq<kAlpha><<<grid, kCT, 0, s>>>(n, w.p, w.q, w.part, w.st);
        }
        if (refine > 0 && t % refine == 0) {
            k_axpy_x<<<grid, kCT, 0, s>>>(n, x, w.p, w.st);
            if ((st = spmv(Pe, x, w.q, reinterpret_cast<spmv_stream_t>(s))) != SPMV_OK) return st;
            k_update<false, true, kRestart><<<grid, kCT, 0, s>>>(n, x, w.p, w.r, w.q, b, w.part,
                                                                 w.st, resid, t);
        } else {
            k_update<true, false, kBeta><<<grid, kCT, 0, s>>>(n, x, w.p, w.r, w.q, b, w.part,
                                                              w.st, resid, t);
        }
        k_update_p<false><<<grid, kCT, 0, s>>>(n, w.p, w.r, w.st, p32);
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
    int64_t g = (n + kCT * kUnr - 1) / (kCT * kUnr);
    if (g > (int64_t)dev.sm_count * 4) g = (int64_t)dev.sm_count * 4;
    const unsigned grid = (unsigned)g;
    CgBufs w;
    SPMV_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&w.r), 8 * n, s));
    SPMV_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&w.p), 8 * n, s));
    SPMV_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&w.q), 8 * n, s));
    const size_t n_part = std::max<size_t>(grid, fusable(Pi) ? sliced_dot_grid(Pi) : 0);
    SPMV_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&w.part), 8 * n_part, s));
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
