// Batched SpMV: many matrices of uneven size in one persistent launch.
//
// A batch holds, per matrix, its CSR arrays, its bound x and y and its
// launch shape (lanes per row T, rows per work item).  The work list is the
// concatenation of every matrix's row chunks; persistent warps take items
// from one atomic counter (the last warp resets it), so small and large
// matrices share the GPU without one launch per matrix.  An item of matrix m
// covers rows_per_item[m] consecutive rows, 32/T rows at a time, each row by T
// lanes with one DFMA per nonzero (row_partial).  A run is a single kernel
// launch with no host work, so it can be replayed from a CUDA graph.
//
// Autotuning (spmv_batch_autotune) tunes for the throughput of the whole
// batch: matrices are grouped by the binary order of their mean row length,
// and coordinate descent over the groups (largest first) tries every T in
// {1, ..., 32} and then rows per item in {2, 4, 8, 16, 32} passes of 32/T
// rows, timing the whole persistent launch each time, keeping a change only
// when it is more than 1 % faster.  Timing one matrix alone would measure
// launch overhead and tail effects, not its share of a full launch.  Without
// autotuning T comes from the mean row length.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "rowdot.cuh"
#include "sliced.cuh"

struct BatchMat {
    const int* rp;
    const int* ci;
    const double* v;
    const double* x;
    double* y;
    int64_t n_rows;
    // sliced layout (matrices prepared as SLICED), else null
    const int* rowlen;
    const int* slice_len;
    const int64_t* slice_ptr;
    const int* perm;
    const void* scol;  // stored columns: int, or int16 / int8 offsets from the row
    const double* sval;
    const int* long_rows;
    int32_t scb;       // bytes per stored column (4, 2 or 1)
    // long rows' segment table of the sliced form (see SlicedPlan)
    const int64_t* seg_be;
    const int* seg_row;
    const int* seg_fix;
    const int* fix;
    const int* seg_off;
    unsigned* ticket;
    double* partial;
};

// lg 0..5: rows [r0, r1) with 2^lg lanes per row; kSliceItem: slices
// [r0, r1) of a sliced matrix; kSegItem: segment r0 of its long rows
// (at most 2048 nonzeros; a row of several segments is summed by the warp
// that finishes its last one, as in the single-matrix kernel)
constexpr int32_t kSliceItem = 8, kSegItem = 10;
struct BatchItem {
    int32_t m, r0, r1, lg;
};

struct spmv_batch {
    int device = -1;
    int sm_count = 0;
    std::vector<spmv_csr_t> mats;
    std::vector<int32_t> tpr, rpi;   // lanes per row, rows per item
    std::vector<const spmv_prepared*> preps;  // SLICED matrices' prepared objects, else null
    std::vector<spmv_prepared*> owned;        // sliced forms the batch prepared itself
    std::vector<const double*> xs;
    std::vector<double*> ys;
    BatchMat* d_mats = nullptr;
    BatchItem* d_items = nullptr;
    int64_t n_items = 0;
    unsigned* d_counter = nullptr;
    bool bound = false;
    cudaGraphExec_t graph = nullptr;
};

namespace spmvlib {
namespace {

using namespace dev;
constexpr int kBT = 256;

template <int T>
__device__ __forceinline__ void batch_rows(const BatchMat& M, int r0, int r1, int lane)
{
    const ColPlain<int> col{M.ci};
    for (int base = r0; base < r1; base += 32 / T) {
        const int row = base + lane / T;
        int64_t b = 0, e = 0;
        if (row < r1) { b = M.rp[row]; e = M.rp[row + 1]; }
        const double s = group_sum(row_partial<T, 4>(b, e, lane & (T - 1), col, M.v, M.x), T);
        if ((lane & (T - 1)) == 0 && row < r1) M.y[row] = s;
    }
}

__global__ void __launch_bounds__(kBT, 6)
k_batch(const BatchMat* __restrict__ mats, const BatchItem* __restrict__ items, int64_t n_items,
        unsigned* __restrict__ counter)
{
    const int lane = threadIdx.x & 31;
    const unsigned total_warps = gridDim.x * (kBT / 32);
    for (;;) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(counter, 1u);
        it = __shfl_sync(FULL, it, 0);
        if ((int64_t)it >= n_items) break;
        const BatchItem I = items[it];
        const BatchMat M = mats[I.m];
        switch (I.lg) {
            case kSliceItem:
                for (int s = I.r0; s < I.r1; ++s) {
                    if (M.scb == 1)
                        slice_rows<4, int8_t>(s, lane, M.rowlen, M.slice_len, M.slice_ptr, M.perm,
                                              static_cast<const int8_t*>(M.scol), M.sval, M.x, M.y);
                    else if (M.scb == 2)
                        slice_rows<4, int16_t>(s, lane, M.rowlen, M.slice_len, M.slice_ptr, M.perm,
                                               static_cast<const int16_t*>(M.scol), M.sval, M.x, M.y);
                    else
                        slice_rows<4, int>(s, lane, M.rowlen, M.slice_len, M.slice_ptr, M.perm,
                                           static_cast<const int*>(M.scol), M.sval, M.x, M.y);
                }
                break;
            case kSegItem: {
                const int j = I.r0;
                const int64_t b = M.seg_be[2 * (int64_t)j], e = M.seg_be[2 * (int64_t)j + 1];
                const double sum = group_sum(row_partial<32, 8>(b, e, lane, ColPlain<int>{M.ci}, M.v, M.x), 32);
                if (lane == 0) {
                    const int r1 = M.seg_row[j];
                    if (r1 >= 0) {
                        M.y[r1] = sum;
                    } else {
                        M.partial[j] = sum;
                        __threadfence();
                        const int t = M.seg_fix[j];
                        const int q = M.fix[t];
                        const int sb = M.seg_off[q], se = M.seg_off[q + 1];
                        if (atomicAdd(M.ticket + t, 1u) == (unsigned)(se - sb - 1)) {
                            __threadfence();
                            double s = 0.0;
                            for (int i = sb; i < se; ++i) s += __ldcg(M.partial + i);
                            M.y[M.long_rows[q]] = s;
                            M.ticket[t] = 0u;
                        }
                    }
                }
                break;
            }
            case 0: batch_rows<1>(M, I.r0, I.r1, lane); break;
            case 1: batch_rows<2>(M, I.r0, I.r1, lane); break;
            case 2: batch_rows<4>(M, I.r0, I.r1, lane); break;
            case 3: batch_rows<8>(M, I.r0, I.r1, lane); break;
            case 4: batch_rows<16>(M, I.r0, I.r1, lane); break;
            default: batch_rows<32>(M, I.r0, I.r1, lane); break;
        }
    }
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(counter + 1, 1u) == total_warps - 1) {
            counter[0] = 0u;
            counter[1] = 0u;
        }
    }
}

int lg2(int t)
{
    int l = 0;
    while ((1 << l) < t) ++l;
    return l;
}

std::vector<BatchItem> make_items(const spmv_batch* B, const std::vector<int32_t>& tpr,
                                  const std::vector<int32_t>& rpi)
{
    std::vector<BatchItem> items;
    // the segments of rows that span several (the longest work, a row of
    // up to 2^31 nonzeros) of every sliced matrix first; then per matrix its
    // slices or row chunks, and the rows of a single segment
    for (size_t m = 0; m < B->mats.size(); ++m)
        if (const spmv_prepared* P = B->preps[m])
            for (int j = 0; j < P->sl.n_seg; ++j)
                if (P->sl.seg_several[j]) items.push_back({(int32_t)m, j, j + 1, kSegItem});
    for (size_t m = 0; m < B->mats.size(); ++m) {
        const spmv_prepared* P = B->preps[m];
        if (P) {
            // rows per item / 32 slices per item
            const int ns = (int)P->sl.n_slices;
            const int k = std::max(1, rpi[m] / 32);
            for (int s0 = 0; s0 < ns; s0 += k) items.push_back({(int32_t)m, s0, std::min(ns, s0 + k), kSliceItem});
            for (int j = 0; j < P->sl.n_seg; ++j)
                if (!P->sl.seg_several[j]) items.push_back({(int32_t)m, j, j + 1, kSegItem});
            continue;
        }
        const int n = (int)B->mats[m].n_rows;
        const int r = rpi[m];
        for (int r0 = 0; r0 < n; r0 += r) items.push_back({(int32_t)m, r0, std::min(n, r0 + r), lg2(tpr[m])});
    }
    return items;
}

spmv_status build_items(spmv_batch* B, cudaStream_t s)
{
    std::vector<BatchItem> items = make_items(B, B->tpr, B->rpi);
    if (B->d_items) cudaFree(B->d_items);
    B->d_items = nullptr;
    B->n_items = (int64_t)items.size();
    if (items.empty()) return SPMV_OK;
    SPMV_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&B->d_items), sizeof(BatchItem) * items.size()));
    SPMV_CUDA_TRY(cudaMemcpyAsync(B->d_items, items.data(), sizeof(BatchItem) * items.size(),
                                  cudaMemcpyHostToDevice, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    if (B->graph) { cudaGraphExecDestroy(B->graph); B->graph = nullptr; }
    return SPMV_OK;
}

spmv_status finish_create(spmv_batch* B, int32_t count, cudaStream_t s, spmv_batch_t** out)
{
    B->xs.assign(count, nullptr);
    B->ys.assign(count, nullptr);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&B->d_counter), 8);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_counter, 0, 8, s);
    if (e == cudaSuccess && count > 0)
        e = cudaMalloc(reinterpret_cast<void**>(&B->d_mats), sizeof(BatchMat) * count);
    if (e != cudaSuccess) { spmv_batch_free(B); return cuda_fail(e, "spmv_batch_create"); }
    spmv_status st = build_items(B, s);
    if (st != SPMV_OK) { spmv_batch_free(B); return st; }
    *out = B;
    return SPMV_OK;
}

cudaError_t launch_batch(const spmv_batch* B, const BatchMat* mats, const BatchItem* items,
                         int64_t n_items, cudaStream_t s)
{
    if (n_items == 0) return cudaSuccess;
    static LaunchCache cache;
    int per_sm = 0;
    cudaError_t e = cached_occupancy(cache, k_batch, kBT, 0, &per_sm);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)B->sm_count * per_sm;
    const int64_t need = (n_items + kBT / 32 - 1) / (kBT / 32);
    if (grid > need) grid = need;
    k_batch<<<(unsigned)grid, kBT, 0, s>>>(mats, items, n_items, B->d_counter);
    return cudaGetLastError();
}

}  // namespace
}  // namespace spmvlib

using namespace spmvlib;

extern "C" {

spmv_status spmv_batch_create(const spmv_csr_t* mats, int32_t count, const int32_t* threads_per_row,
                              const int32_t* rows_per_item, spmv_batch_t** out,
                              spmv_stream_t stream)
{
    clear_error();
    if (!out || count < 0 || (count > 0 && !mats))
        return fail(SPMV_ERR_INVALID_ARG, "spmv_batch_create: bad argument");
    *out = nullptr;
    DeviceInfo dev;
    spmv_status st = current_device(&dev);
    if (st != SPMV_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    spmv_batch* B = new (std::nothrow) spmv_batch();
    if (!B) return fail(SPMV_ERR_NOMEM, "host allocation failed");
    B->device = dev.device;
    B->sm_count = dev.sm_count;
    for (int m = 0; m < count; ++m) {
        if ((st = check_csr_args(&mats[m])) != SPMV_OK) { spmv_batch_free(B); return st; }
        const int t = threads_per_row ? threads_per_row[m] : 0;
        if (t != 0 && (t < 1 || t > 32 || (t & (t - 1)))) {
            spmv_batch_free(B);
            return fail(SPMV_ERR_INVALID_ARG, "threads_per_row must be a power of two in 1..32");
        }
        const double mean = mats[m].n_rows ? (double)mats[m].nnz / (double)mats[m].n_rows : 1.0;
        const int T = t ? t : auto_threads_per_row(mean / 7.0);
        const int r = rows_per_item && rows_per_item[m] > 0 ? rows_per_item[m] : 8 * (32 / T);
        B->mats.push_back(mats[m]);
        B->tpr.push_back(T);
        B->rpi.push_back(r);
        B->preps.push_back(nullptr);
    }
    return finish_create(B, count, s, out);
}

}  // extern "C"

namespace {

// all_sliced: every matrix in the sliced layout; otherwise each matrix in
// the persistent form of its own variant
spmv_status create_from_prepared(const spmv_prepared_t* const* P, int32_t count, bool all_sliced,
                                 spmv_batch_t** out, spmv_stream_t stream)
{
    clear_error();
    if (!out || count < 0 || (count > 0 && !P))
        return fail(SPMV_ERR_INVALID_ARG, "spmv_batch_create_prepared: bad argument");
    *out = nullptr;
    DeviceInfo dev;
    spmv_status st = current_device(&dev);
    if (st != SPMV_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    spmv_batch* B = new (std::nothrow) spmv_batch();
    if (!B) return fail(SPMV_ERR_NOMEM, "host allocation failed");
    B->device = dev.device;
    B->sm_count = dev.sm_count;
    for (int m = 0; m < count; ++m) {
        const spmv_prepared* Pm = P[m];
        if (!Pm) { spmv_batch_free(B); return fail(SPMV_ERR_INVALID_ARG, "NULL prepared matrix"); }
        if (Pm->device != dev.device) {
            spmv_batch_free(B);
            return fail(SPMV_ERR_INVALID_ARG, "prepared on another device");
        }
        const spmv_csr_t& A = Pm->A;
        // The sliced form the batch prepares and owns (automatic layout):
        // all_sliced -- for every matrix not prepared as FP64 SLICED (inside
        // the one launch the matrices share the FP64 pipe, and slices spend
        // one DFMA per element with no reductions); otherwise for the
        // imbalance variants (MERGE, DYNAMIC: as CSR rows a warp would run as
        // many DFMAs as its longest row) and for SLICED with FP32/BF16 values
        // (the batch sums FP64).  The other variants run as CSR rows of their
        // prepared lanes.
        // (a SLICED matrix with coded columns, a form the batch kernel does
        // not decode, is laid out anew like one with FP32/BF16 values)
        const bool coded = Pm->c.variant == SPMV_V7_SLICED && Pm->sl.coding != 0;
        const bool own_sliced = all_sliced
            ? (Pm->c.variant != SPMV_V7_SLICED || Pm->c.value_type != SPMV_VAL_F64 || coded)
            : (Pm->c.variant == SPMV_V3_MERGE || Pm->c.variant == SPMV_V4_DYNAMIC ||
               (Pm->c.variant == SPMV_V7_SLICED && (Pm->c.value_type != SPMV_VAL_F64 || coded)));
        if (own_sliced) {
            spmv_choice_t c{};
            c.variant = SPMV_V7_SLICED;
            c.cls = -1;
            c.block_nnz = 0;
            spmv_prepared* Q = nullptr;
            st = spmv_prepare(&A, &c, 1, &Q, stream);
            if (st != SPMV_OK) { spmv_batch_free(B); return st; }
            B->owned.push_back(Q);
            Pm = Q;
        }
        const bool sliced = Pm->c.variant == SPMV_V7_SLICED;
        const double mean = A.n_rows ? (double)A.nnz / (double)A.n_rows : 1.0;
        const int t = Pm->c.threads_per_row;
        const int T = sliced ? 1 : (t >= 1 && t <= 32 && !(t & (t - 1)) ? t : auto_threads_per_row(mean / 7.0));
        B->mats.push_back(A);
        B->tpr.push_back(T);
        B->rpi.push_back(sliced ? 4 * 32 : 8 * (32 / T));
        B->preps.push_back(sliced ? Pm : nullptr);
    }
    return finish_create(B, count, s, out);
}

}  // namespace

extern "C" {

spmv_status spmv_batch_create_prepared(const spmv_prepared_t* const* P, int32_t count,
                                       spmv_batch_t** out, spmv_stream_t stream)
{
    return create_from_prepared(P, count, false, out, stream);
}

spmv_status spmv_batch_create_sliced(const spmv_prepared_t* const* P, int32_t count,
                                     spmv_batch_t** out, spmv_stream_t stream)
{
    return create_from_prepared(P, count, true, out, stream);
}

spmv_status spmv_batch_bind(spmv_batch_t* B, const double* const* x, double* const* y,
                            spmv_stream_t stream)
{
    clear_error();
    if (!B || (!B->mats.empty() && (!x || !y)))
        return fail(SPMV_ERR_INVALID_ARG, "spmv_batch_bind: NULL argument");
    std::vector<BatchMat> h(B->mats.size());
    for (size_t m = 0; m < B->mats.size(); ++m) {
        const spmv_csr_t& A = B->mats[m];
        h[m] = {A.rowptr, A.colind, A.val, x[m], y[m], A.n_rows,
                nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 4,
                nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        if (const spmv_prepared* P = B->preps[m]) {
            const SlicedPlan& d = P->sl;
            h[m].rowlen = d.rowlen;
            h[m].slice_len = d.slice_len;
            h[m].slice_ptr = d.slice_ptr;
            h[m].perm = d.sigma > 1 ? d.perm : nullptr;
            h[m].scol = d.scol;
            h[m].scb = d.cbytes;
            h[m].sval = d.val;
            h[m].long_rows = d.long_rows;
            h[m].seg_be = d.seg_be;
            h[m].seg_row = d.seg_row;
            h[m].seg_fix = d.seg_fix;
            h[m].fix = d.fix;
            h[m].seg_off = d.seg_off;
            h[m].ticket = d.ticket;
            h[m].partial = d.partial;
        }
        B->xs[m] = x[m];
        B->ys[m] = y[m];
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!h.empty()) {
        SPMV_CUDA_TRY(cudaMemcpyAsync(B->d_mats, h.data(), sizeof(BatchMat) * h.size(),
                                      cudaMemcpyHostToDevice, s));
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    }
    B->bound = true;
    return SPMV_OK;
}

spmv_status spmv_batch_run(spmv_batch_t* B, int32_t use_graph, spmv_stream_t stream)
{
    if (!B) return fail(SPMV_ERR_INVALID_ARG, "spmv_batch_run: NULL batch");
    if (!B->bound) return fail(SPMV_ERR_INVALID_ARG, "spmv_batch_run: call spmv_batch_bind first");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!use_graph) {
        cudaError_t e = launch_batch(B, B->d_mats, B->d_items, B->n_items, s);
        return e == cudaSuccess ? SPMV_OK : cuda_fail(e, "spmv_batch_run");
    }
    if (!B->graph) {
        // capture once on a private stream, replay on any stream afterwards
        cudaStream_t cs;
        SPMV_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t el = launch_batch(B, B->d_mats, B->d_items, B->n_items, cs);
            e = cudaStreamEndCapture(cs, &g);
            if (e == cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            B->graph = nullptr;
            return cuda_fail(e, "spmv_batch_run graph capture");
        }
    }
    SPMV_CUDA_TRY(cudaGraphLaunch(B->graph, s));
    return SPMV_OK;
}

spmv_status spmv_batch_autotune(spmv_batch_t* B, int32_t reps, spmv_stream_t stream)
{
    clear_error();
    if (!B || !B->bound) return fail(SPMV_ERR_INVALID_ARG, "spmv_batch_autotune: bind first");
    if (reps <= 0) reps = 3;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t count = B->mats.size();
    // groups: binary order of the mean row length
    std::vector<int> group(count, 0);
    std::vector<int64_t> group_nnz(64, 0);
    for (size_t m = 0; m < count; ++m) {
        const spmv_csr_t& A = B->mats[m];
        const double mean = A.n_rows ? (double)A.nnz / (double)A.n_rows : 0.0;
        int g = 0;
        while (g < 31 && (double)(2 << g) <= mean) ++g;
        if (B->preps[m]) g += 32;  // sliced matrices: their own groups, one lane per row
        group[m] = g;
        group_nnz[g] += A.nnz;
    }
    std::vector<int> order;
    for (int g = 0; g < 64; ++g)
        if (group_nnz[g] > 0) order.push_back(g);
    std::sort(order.begin(), order.end(), [&](int a, int b_) { return group_nnz[a] > group_nnz[b_]; });

    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BatchItem* d_tmp = nullptr;
    size_t cap = 0;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // median time of `reps` launches of the whole batch with shapes (tpr, rpi)
    auto eval = [&](const std::vector<int32_t>& tpr, const std::vector<int32_t>& rpi, float* ms) {
        std::vector<BatchItem> items = make_items(B, tpr, rpi);
        if (items.size() > cap) {
            if (d_tmp) cudaFreeAsync(d_tmp, s);
            d_tmp = nullptr;
            cap = items.size();
            e = cudaMallocAsync(reinterpret_cast<void**>(&d_tmp), sizeof(BatchItem) * cap, s);
        }
        if (e == cudaSuccess && !items.empty())
            e = cudaMemcpyAsync(d_tmp, items.data(), sizeof(BatchItem) * items.size(),
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = launch_batch(B, B->d_mats, d_tmp, (int64_t)items.size(), s);  // warm-up
        std::vector<float> t;
        for (int k = 0; k < reps && e == cudaSuccess; ++k) {
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = launch_batch(B, B->d_mats, d_tmp, (int64_t)items.size(), s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float v = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&v, e0, e1);
            t.push_back(v);
        }
        if (e != cudaSuccess || t.empty()) { *ms = 1e30f; return; }
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
    };
    std::vector<int32_t> tpr = B->tpr, rpi = B->rpi;
    float best = 0.f;
    eval(tpr, rpi, &best);
    auto set_group = [&](std::vector<int32_t>& tv, std::vector<int32_t>& rv, int g, int T, int passes) {
        for (size_t m = 0; m < count; ++m)
            if (group[m] == g) { tv[m] = T; rv[m] = passes * (32 / T); }
    };
    for (int sweep = 0; sweep < 2 && e == cudaSuccess; ++sweep) {
        for (int g : order) {
            // lanes per row with 8 passes per item, then passes per item at that T
            int gm = -1;
            for (size_t m = 0; m < count; ++m) if (group[m] == g) { gm = (int)m; break; }
            int bestT = tpr[gm], bestP = std::max(1, rpi[gm] / (32 / tpr[gm]));
            for (int T = 1; T <= (g >= 32 ? 1 : 32) && e == cudaSuccess; T <<= 1) {
                std::vector<int32_t> tv = tpr, rv = rpi;
                set_group(tv, rv, g, T, bestP);
                float ms;
                eval(tv, rv, &ms);
                if (ms < 0.99f * best) { best = ms; bestT = T; tpr = tv; rpi = rv; }
            }
            for (int passes = 2; passes <= 32 && e == cudaSuccess; passes <<= 1) {
                std::vector<int32_t> tv = tpr, rv = rpi;
                set_group(tv, rv, g, bestT, passes);
                float ms;
                eval(tv, rv, &ms);
                if (ms < 0.99f * best) { best = ms; bestP = passes; tpr = tv; rpi = rv; }
            }
        }
    }
    if (d_tmp) cudaFreeAsync(d_tmp, s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "spmv_batch_autotune");
    B->tpr = tpr;
    B->rpi = rpi;
    return build_items(B, s);
}

spmv_status spmv_batch_config(const spmv_batch_t* B, int32_t* threads_per_row, int32_t* rows_per_item)
{
    clear_error();
    if (!B) return fail(SPMV_ERR_INVALID_ARG, "spmv_batch_config: NULL batch");
    for (size_t m = 0; m < B->mats.size(); ++m) {
        if (threads_per_row) threads_per_row[m] = B->tpr[m];
        if (rows_per_item) rows_per_item[m] = B->rpi[m];
    }
    return SPMV_OK;
}

void spmv_batch_free(spmv_batch_t* B)
{
    if (!B) return;
    cudaDeviceSynchronize();
    if (B->graph) cudaGraphExecDestroy(B->graph);
    if (B->d_items) cudaFree(B->d_items);
    if (B->d_mats) cudaFree(B->d_mats);
    if (B->d_counter) cudaFree(B->d_counter);
    for (spmv_prepared* Q : B->owned) spmv_prepared_free(Q);
    delete B;
}

}  // extern "C"
