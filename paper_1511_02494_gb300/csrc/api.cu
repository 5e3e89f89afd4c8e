// C ABI entry points: status and errors, validation, features, selection,
// prepare / run / free.  See include/spmv.h for the contract of each call.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "common.cuh"

namespace spmvlib {

namespace {
thread_local std::string t_last_error;
constexpr int kMaxDevices = 64;
DeviceInfo g_dev[kMaxDevices];
std::mutex g_dev_mu;

// LATENCY's persisting-L2 carve-out (cudaLimitPersistingL2CacheSize, a limit
// of this process's context): raised by the first prepared object that keeps
// x persisting, and put back, with every persisting line released, when the
// last such object on the device is freed.  Persisting lines left behind
// shrink the L2 of every kernel that runs afterwards (measured: SLICED and
// DYNAMIC 6-20 % slower on matrices of over 10^6 rows timed after LATENCY
// had run on a large one).
std::mutex g_persist_mu;
int g_persist_users[kMaxDevices] = {};
size_t g_persist_saved[kMaxDevices] = {};

// Raises the carve-out of device d (current) to at least want bytes and
// counts a user; false (nothing changed) where the limit cannot be set.
bool persist_acquire(int d, int64_t want)
{
    std::lock_guard<std::mutex> lk(g_persist_mu);
    size_t cur = 0;
    if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess ||
        ((int64_t)cur < want && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)want) != cudaSuccess)) {
        cudaGetLastError();
        return false;
    }
    if (g_persist_users[d]++ == 0) g_persist_saved[d] = cur;
    return true;
}

// One user of device d fewer; the last one releases the persisting lines and
// puts the carve-out back (with no kernel of the object in flight).
void persist_release(int d)
{
    std::lock_guard<std::mutex> lk(g_persist_mu);
    if (g_persist_users[d] == 0 || --g_persist_users[d] > 0) return;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) { cudaGetLastError(); return; }
    if (cur != d && cudaSetDevice(d) != cudaSuccess) { cudaGetLastError(); return; }
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, g_persist_saved[d]);
    cudaGetLastError();
    if (cur != d) cudaSetDevice(cur);
}
}  // namespace

void set_error(const std::string& msg) { t_last_error = msg; }
void clear_error() { t_last_error.clear(); }
const char* last_error_cstr() { return t_last_error.c_str(); }

spmv_status fail(spmv_status s, const std::string& msg)
{
    t_last_error = msg;
    return s;
}

spmv_status cuda_fail(cudaError_t e, const char* what)
{
    t_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return SPMV_ERR_CUDA;
}

spmv_status current_device(DeviceInfo* out)
{
    int d = -1;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (d < 0 || d >= kMaxDevices) return fail(SPMV_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (g_dev[d].device != d) {
        DeviceInfo di;
        di.device = d;
        if ((e = cudaDeviceGetAttribute(&di.sm_count, cudaDevAttrMultiProcessorCount, d)) != cudaSuccess)
            return cuda_fail(e, "cudaDeviceGetAttribute(SM count)");
        if ((e = cudaDeviceGetAttribute(&di.l2_bytes, cudaDevAttrL2CacheSize, d)) != cudaSuccess)
            return cuda_fail(e, "cudaDeviceGetAttribute(L2 size)");
        if ((e = cudaDeviceGetAttribute(&di.max_persist_l2, cudaDevAttrMaxPersistingL2CacheSize, d)) != cudaSuccess)
            return cuda_fail(e, "cudaDeviceGetAttribute(persisting L2)");
        if ((e = cudaDeviceGetAttribute(&di.max_window, cudaDevAttrMaxAccessPolicyWindowSize, d)) != cudaSuccess)
            return cuda_fail(e, "cudaDeviceGetAttribute(access window)");
        g_dev[d] = di;
    }
    *out = g_dev[d];
    return SPMV_OK;
}

spmv_status check_csr_args(const spmv_csr_t* A)
{
    if (!A) return fail(SPMV_ERR_INVALID_ARG, "NULL matrix");
    if (A->n_rows < 0 || A->n_cols < 0 || A->nnz < 0)
        return fail(SPMV_ERR_INVALID_ARG, "negative matrix size");
    if (A->n_rows >= INT32_MAX || A->n_cols >= INT32_MAX || A->nnz >= INT32_MAX)
        return fail(SPMV_ERR_UNSUPPORTED, "sizes must fit 32-bit indices");
    if (!A->rowptr) return fail(SPMV_ERR_INVALID_ARG, "NULL rowptr");
    if (A->nnz > 0 && (!A->colind || !A->val))
        return fail(SPMV_ERR_INVALID_ARG, "NULL colind or val");
    if (A->nnz > 0 && A->n_cols == 0)
        return fail(SPMV_ERR_INVALID_CSR, "nonzeros in a matrix without columns");
    return SPMV_OK;
}

spmv_status prepared_alloc(spmv_prepared* P, void** p, int64_t bytes)
{
    *p = nullptr;
    if (bytes <= 0) return SPMV_OK;
    cudaError_t e = cudaMalloc(p, (size_t)bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        *p = nullptr;
        return fail(SPMV_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    P->owned.push_back(*p);
    P->owned_bytes += bytes;
    return SPMV_OK;
}

}  // namespace spmvlib

using namespace spmvlib;

namespace {

bool is_pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

bool merge_items_ok(int items)
{
    if (items <= 0 || items % 32) return false;
    switch (items / 32) {
        case 1: case 2: case 4: case 6: case 7: case 8: case 12: case 16: return true;
        default: return false;
    }
}

template <typename T>
spmv_status dev_alloc(spmv_prepared_t* P, T** p, int64_t count)
{
    *p = nullptr;
    if (count <= 0) return SPMV_OK;
    const size_t bytes = sizeof(T) * (size_t)count;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        *p = nullptr;
        return fail(SPMV_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    P->owned.push_back(*p);
    P->owned_bytes += (int64_t)bytes;
    return SPMV_OK;
}

// Frees every device allocation the object made (each one registered itself
// in P->owned when it was made), whatever the variant.
void release(spmv_prepared_t* P)
{
    for (void* p : P->owned)
        if (p) cudaFree(p);
    P->owned.clear();
    if (P->persist_held) {
        persist_release(P->device);
        P->persist_held = false;
    }
}

int32_t launches_of(const spmv_prepared_t* P)
{
    if (P->A.n_rows == 0) return 0;
    switch (P->c.variant) {
        case SPMV_V2_STREAM: return P->bulk ? 2 : 1;               // windows + carry fix-up
        case SPMV_V3_MERGE: return 2;                              // tiles + carry fix-up
        case SPMV_V4_DYNAMIC: return 1;                            // long rows summed by their last warp
        case SPMV_V7_SLICED:
            // slices and long rows in one launch; with FP32 accumulation the
            // conversion of x to FP32 before it
            return 1 + (P->sl.acc32 && P->A.n_cols > 0 ? 1 : 0);
        case SPMV_V6_COMPRESSED: return P->c.accumulate == 2 && P->A.n_cols > 0 ? 2 : 1;  // + x to FP32
        default: return 1;
    }
}

int64_t min_bytes_of(const spmv_prepared_t* P)
{
    const spmv_csr_t& A = P->A;
    const int64_t vec = 8 * A.n_cols + 8 * A.n_rows + 4 * (A.n_rows + 1);
    if (P->c.variant == SPMV_V7_SLICED) {
        // elements once, a row length per position, slice length and start,
        // the permutation when rows are sorted, the long rows' list and
        // segment offsets, per segment its bounds and row and a partial
        const SlicedPlan& d = P->sl;
        const int vb = d.value_type == SPMV_VAL_F64 ? 8 : d.value_type == SPMV_VAL_F32 ? 4 : 2;
        const int cb = d.value_type == SPMV_VAL_F64 ? d.cbytes : (d.off16 ? 2 : 4);
        return (int64_t)(vb + cb) * A.nnz + 128 * d.n_slices * (d.off16 || d.coding == 1 ? 2 : 1) +
               12 * d.n_slices +
               (d.sigma > 1 ? 4 * A.n_rows : 0) + 12 * (int64_t)d.n_long + 36 * (int64_t)d.n_seg +
               8 * A.n_cols + (d.acc32 ? 8 * A.n_cols : 0) + 8 * A.n_rows;
    }
    if (P->c.variant != SPMV_V6_COMPRESSED) return 12 * A.nnz + vec;
    const int vb = P->c.value_type == SPMV_VAL_F64 ? 8 : P->c.value_type == SPMV_VAL_F32 ? 4 : 2;
    // FP32 accumulation: x converted once (8 + 4 bytes per column), then read as float
    const int64_t xconv = P->c.accumulate == 2 ? 4 * A.n_cols + 4 * A.n_cols : 0;
    if (P->off16 == nullptr) return (int64_t)(vb + 4) * A.nnz + vec + xconv;  // every row wide
    // 2-byte offsets + a 4-byte rowbase per row (wide rows' 4-byte columns
    // counted at 2 bytes here: a lower bound for mixed matrices)
    return (int64_t)(vb + 2) * A.nnz + 4 * A.n_rows + vec + xconv;
}

spmv_status prepare_impl(spmv_prepared_t* P, cudaStream_t s)
{
    const spmv_csr_t& A = P->A;
    spmv_choice_t& c = P->c;
    const double mean = A.n_rows ? (double)A.nnz / (double)A.n_rows : 1.0;
    spmv_status st;
    switch (c.variant) {
        case SPMV_V0_SCALAR:
            c.threads_per_row = 1;
            return SPMV_OK;
        case SPMV_V1_SUBWARP:
            if (c.threads_per_row == 0) c.threads_per_row = auto_threads_per_row(mean / 7.0);
            return SPMV_OK;
        case SPMV_V2_STREAM: {
            if (c.block_nnz == 0) c.block_nnz = 2048;
            P->n_blocks = A.nnz > 0 ? (A.nnz + c.block_nnz - 1) / c.block_nnz : 1;
            P->bulk = tma_aligned(A) && (c.block_nnz == 1024 || c.block_nnz == 2048);
            if ((st = dev_alloc(P, &P->blocks, P->n_blocks + 1)) != SPMV_OK) return st;
            if (P->bulk) {
                if ((st = dev_alloc(P, &P->carry_row, P->n_blocks)) != SPMV_OK) return st;
                if ((st = dev_alloc(P, &P->carry_val, P->n_blocks)) != SPMV_OK) return st;
                if ((st = dev_alloc(P, &P->status, 1)) != SPMV_OK) return st;
                SPMV_CUDA_TRY(cudaMemsetAsync(P->status, 0, sizeof(unsigned), s));
            }
            SPMV_CUDA_TRY(launch_row_blocks(A, c.block_nnz, P->n_blocks, P->blocks, s));
            return SPMV_OK;
        }
        case SPMV_V3_MERGE: {
            if (c.items_per_warp == 0) c.items_per_warp = 256;
            if (c.block_nnz == 0) c.block_nnz = 2048;
            P->bulk = tma_aligned(A);
            P->tile_items = P->bulk ? c.block_nnz : c.items_per_warp;
            if ((st = dev_alloc(P, &P->status, 1)) != SPMV_OK) return st;
            SPMV_CUDA_TRY(cudaMemsetAsync(P->status, 0, sizeof(unsigned), s));
            const int64_t total = A.n_rows + A.nnz;
            P->n_blocks = total > 0 ? (total + P->tile_items - 1) / P->tile_items : 1;
            if ((st = dev_alloc(P, &P->blocks, P->n_blocks + 1)) != SPMV_OK) return st;
            if ((st = dev_alloc(P, &P->merge_nz, P->n_blocks + 1)) != SPMV_OK) return st;
            if ((st = dev_alloc(P, &P->carry_row, P->n_blocks)) != SPMV_OK) return st;
            if ((st = dev_alloc(P, &P->carry_val, P->n_blocks)) != SPMV_OK) return st;
            SPMV_CUDA_TRY(launch_merge_coords(A, P->tile_items, P->n_blocks, P->blocks,
                                              P->merge_nz, s));
            return SPMV_OK;
        }
        case SPMV_V4_DYNAMIC: {
            if (c.block_nnz == 0) c.block_nnz = 2048;  // nonzeros per long-row segment
            P->dyn.seg = c.block_nnz;
            return dyn_prepare(P, s);
        }
        case SPMV_V5_LATENCY: {
            if (c.threads_per_row == 0) c.threads_per_row = auto_threads_per_row(mean / 7.0);
            DeviceInfo dev;
            if ((st = current_device(&dev)) != SPMV_OK) return st;
            // x of up to half the L2 stays resident without help (streamed
            // arrays are loaded evict-first); a persisting window would only
            // take L2 away from the kernels that run next
            const int64_t xbytes = 8 * A.n_cols;
            int64_t want = xbytes < dev.max_persist_l2 ? xbytes : dev.max_persist_l2;
            if (2 * xbytes <= (int64_t)dev.l2_bytes) want = 0;
            if (want > dev.max_window) want = dev.max_window;
            // the persisting-L2 carve-out is a limit of this process's context,
            // held while the object lives; where it cannot be set the variant
            // runs without the window
            if (want > 0) {
                if (persist_acquire(dev.device, want)) P->persist_held = true;
                else want = 0;
            }
            P->l2_window_bytes = (int)(want > 0 ? want : 0);
            return SPMV_OK;
        }
        case SPMV_V6_COMPRESSED: {
            if (c.threads_per_row == 0) c.threads_per_row = auto_threads_per_row(mean / 7.0);
            if (c.accumulate == 0) c.accumulate = c.value_type == SPMV_VAL_F64 ? 1 : 2;
            if (c.accumulate == 2 && (st = dev_alloc(P, &P->x32, std::max<int64_t>(A.n_cols, 1))) != SPMV_OK)
                return st;
            if ((st = dev_alloc(P, &P->rowbase, A.n_rows)) != SPMV_OK) return st;
            unsigned long long* d_wide = nullptr;
            SPMV_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d_wide), 8, s));
            cudaError_t e = cudaMemsetAsync(d_wide, 0, 8, s);
            if (e == cudaSuccess)
                e = launch_compress(A, P->rowbase, nullptr, d_wide, c.value_type, nullptr, s);
            unsigned long long h_wide = 0;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&h_wide, d_wide, 8, cudaMemcpyDeviceToHost, s);
            cudaFreeAsync(d_wide, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "compress rows");
            P->n_wide = (int64_t)h_wide;
            if (P->n_wide < A.n_rows && A.nnz > 0) {
                if ((st = dev_alloc(P, &P->off16, A.nnz)) != SPMV_OK) return st;
            }
            if (c.value_type != SPMV_VAL_F64 && A.nnz > 0) {
                uint16_t* lv16 = nullptr;
                float* lv32 = nullptr;
                if (c.value_type == SPMV_VAL_F32) {
                    if ((st = dev_alloc(P, &lv32, A.nnz)) != SPMV_OK) return st;
                    P->lowval = lv32;
                } else {
                    if ((st = dev_alloc(P, &lv16, A.nnz)) != SPMV_OK) return st;
                    P->lowval = lv16;
                }
            }
            // offsets and value casts (rowbase is recomputed identically)
            unsigned long long* d_w2 = nullptr;
            SPMV_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d_w2), 8, s));
            e = cudaMemsetAsync(d_w2, 0, 8, s);
            if (e == cudaSuccess)
                e = launch_compress(A, P->rowbase, P->off16, d_w2, c.value_type, P->lowval, s);
            cudaFreeAsync(d_w2, s);
            if (e != cudaSuccess) return cuda_fail(e, "compress offsets/values");
            return SPMV_OK;
        }
        case SPMV_V7_SLICED:
            return sliced_prepare(P, s);
        default:
            return fail(SPMV_ERR_INVALID_ARG, "unknown variant");
    }
}

}  // namespace

namespace spmvlib {

spmv_status check_choice(const spmv_choice_t* c)
{
    if (c->variant < 0 || c->variant >= SPMV_NUM_VARIANTS)
        return fail(SPMV_ERR_INVALID_ARG, "variant out of range");
    if (c->threads_per_row != 0 && !is_pow2_in(c->threads_per_row, 1, 32))
        return fail(SPMV_ERR_INVALID_ARG, "threads_per_row must be a power of two in 1..32");
    if (c->variant == SPMV_V2_STREAM && c->block_nnz != 0 && !is_pow2_in(c->block_nnz, 64, 8192))
        return fail(SPMV_ERR_INVALID_ARG, "block_nnz must be a power of two in 64..8192");
    if (c->variant == SPMV_V7_SLICED && c->block_nnz != 0 && c->block_nnz != 1 &&
        !is_pow2_in(c->block_nnz, 32, 4096))
        return fail(SPMV_ERR_INVALID_ARG, "SLICED sort window (block_nnz) must be 1 or a power of two in 32..4096");
    if (c->variant == SPMV_V4_DYNAMIC && c->block_nnz != 0 && !is_pow2_in(c->block_nnz, 256, 1 << 20))
        return fail(SPMV_ERR_INVALID_ARG, "DYNAMIC segment length must be a power of two in 256..2^20");
    if (c->variant == SPMV_V3_MERGE && c->block_nnz != 0 && c->block_nnz != 1024 &&
        c->block_nnz != 1536 && c->block_nnz != 2048)
        return fail(SPMV_ERR_INVALID_ARG, "MERGE tile items (block_nnz) must be 1024, 1536 or 2048");
    if (c->variant == SPMV_V7_SLICED) {
        if (c->threads_per_row != 0 && c->threads_per_row != 1 && c->threads_per_row != 2 &&
            c->threads_per_row != 4)
            return fail(SPMV_ERR_INVALID_ARG, "SLICED slices per warp (threads_per_row) must be 0, 1, 2 or 4");
        if (c->items_per_warp < 0 || c->items_per_warp > kSlicedCapMax)
            return fail(SPMV_ERR_INVALID_ARG, "SLICED row-length cap (items_per_warp) must be in 0..65536");
    } else if (c->items_per_warp != 0 && !merge_items_ok(c->items_per_warp)) {
        return fail(SPMV_ERR_INVALID_ARG, "items_per_warp must be 32*k, k in {1,2,4,6,7,8,12,16}");
    }
    if (c->value_type < SPMV_VAL_F64 || c->value_type > SPMV_VAL_BF16)
        return fail(SPMV_ERR_INVALID_ARG, "value_type out of range");
    const bool lowp_ok = c->variant == SPMV_V6_COMPRESSED || c->variant == SPMV_V7_SLICED;
    if (c->value_type != SPMV_VAL_F64 && !lowp_ok)
        return fail(SPMV_ERR_UNSUPPORTED, "low-precision values only in the COMPRESSED and SLICED variants");
    if (c->index_bytes != 0 && c->index_bytes != 1 && c->index_bytes != 2 && c->index_bytes != 4)
        return fail(SPMV_ERR_INVALID_ARG, "index_bytes must be 0, 1, 2 or 4");
    if (c->index_bytes != 0 && c->index_bytes != 4 &&
        (c->variant != SPMV_V7_SLICED || c->value_type != SPMV_VAL_F64))
        return fail(SPMV_ERR_UNSUPPORTED, "narrow column indices only in SLICED with FP64 values");
    if (c->index_coding < 0 || c->index_coding > 2)
        return fail(SPMV_ERR_INVALID_ARG, "index_coding must be 0, 1 (deltas) or 2 (column panels)");
    if (c->index_coding != 0 && (c->variant != SPMV_V7_SLICED || c->value_type != SPMV_VAL_F64))
        return fail(SPMV_ERR_UNSUPPORTED, "coded column indices only in SLICED with FP64 values");
    if (c->index_coding != 0 && (c->index_bytes == 1 || c->index_bytes == 2))
        return fail(SPMV_ERR_INVALID_ARG, "index_coding replaces the row offsets of index_bytes 1 or 2");
    if (c->index_coding != 0 && c->threads_per_row > 1)
        return fail(SPMV_ERR_UNSUPPORTED, "coded column indices run one slice per warp (threads_per_row 0 or 1)");
    if (c->accumulate < 0 || c->accumulate > 2)
        return fail(SPMV_ERR_INVALID_ARG, "accumulate must be 0 (by value type), 1 (FP64) or 2 (FP32)");
    if (c->accumulate == 2 && (!lowp_ok || c->value_type == SPMV_VAL_F64))
        return fail(SPMV_ERR_UNSUPPORTED, "FP32 accumulation needs COMPRESSED or SLICED with FP32 or BF16 values");
    return SPMV_OK;
}

}  // namespace spmvlib

namespace {

spmv_status run_impl(const spmv_prepared_t* P, const double* x, double* y, cudaStream_t s)
{
    const spmv_csr_t& A = P->A;
    const spmv_choice_t& c = P->c;
    cudaError_t e = cudaSuccess;
    switch (c.variant) {
        case SPMV_V0_SCALAR: e = launch_scalar(A, x, y, s); break;
        case SPMV_V1_SUBWARP: e = launch_subwarp(A, c.threads_per_row, x, y, s); break;
        case SPMV_V2_STREAM:
            if (P->bulk)
                e = launch_window(A, c.block_nnz, P->blocks, P->n_blocks, P->carry_row, P->carry_val,
                                  P->status, P->sm_count, x, y, s);
            else
                e = launch_stream(A, P->blocks, P->n_blocks, c.block_nnz, x, y, s);
            break;
        case SPMV_V3_MERGE:
            if (P->bulk)
                e = launch_merge_tma(A, P->tile_items, P->blocks, P->merge_nz, P->n_blocks,
                                     P->carry_row, P->carry_val, P->status, P->sm_count, x, y, s);
            else
                e = launch_merge(A, c.items_per_warp, P->blocks, P->merge_nz, P->n_blocks,
                                 P->carry_row, P->carry_val, x, y, s);
            break;
        case SPMV_V4_DYNAMIC: e = launch_dyn(P, x, y, s); break;
        case SPMV_V7_SLICED: e = launch_sliced(P, x, y, s); break;
        case SPMV_V5_LATENCY:
            e = launch_latency(A, c.threads_per_row, x, y, P->l2_window_bytes, s);
            break;
        case SPMV_V6_COMPRESSED:
            if (c.accumulate == 2)
                e = launch_compressed32(A, c.threads_per_row, c.value_type, P->rowbase, P->off16,
                                        P->lowval, P->off16 == nullptr, x, P->x32, y, s);
            else
                e = launch_compressed(A, c.threads_per_row, c.value_type, P->rowbase, P->off16,
                                      P->lowval, P->off16 == nullptr, x, y, s);
            break;
        default: return fail(SPMV_ERR_INVALID_ARG, "unknown variant");
    }
    if (e != cudaSuccess) return cuda_fail(e, "spmv launch");
    return SPMV_OK;
}

}  // namespace

extern "C" {

const char* spmv_status_str(spmv_status s)
{
    switch (s) {
        case SPMV_OK: return "SPMV_OK";
        case SPMV_ERR_INVALID_ARG: return "SPMV_ERR_INVALID_ARG";
        case SPMV_ERR_INVALID_CSR: return "SPMV_ERR_INVALID_CSR";
        case SPMV_ERR_UNSUPPORTED: return "SPMV_ERR_UNSUPPORTED";
        case SPMV_ERR_NOMEM: return "SPMV_ERR_NOMEM";
        case SPMV_ERR_CUDA: return "SPMV_ERR_CUDA";
        case SPMV_ERR_TIMEOUT: return "SPMV_ERR_TIMEOUT";
        case SPMV_ERR_MODEL: return "SPMV_ERR_MODEL";
    }
    return "SPMV_ERR_UNKNOWN";
}

const char* spmv_last_error(void) { return last_error_cstr(); }

spmv_status spmv_validate(const spmv_csr_t* A, spmv_stream_t stream)
{
    clear_error();
    return run_feature_pass(A, 128, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

spmv_status spmv_features(const spmv_csr_t* A, int32_t line_bytes, spmv_features_t* out,
                          spmv_stream_t stream)
{
    clear_error();
    if (!out) return fail(SPMV_ERR_INVALID_ARG, "spmv_features: NULL output");
    if (line_bytes < 0) return fail(SPMV_ERR_INVALID_ARG, "spmv_features: negative line size");
    return run_feature_pass(A, line_bytes, out, reinterpret_cast<cudaStream_t>(stream));
}

spmv_thresholds_t spmv_default_thresholds(void)
{
    spmv_thresholds_t t;
    // calibrated on GB300 with the four generator families: balanced matrices
    // show span/mean near 1.8 and x vectors that fit the L2 give noxmiss
    // speedups below 1.2
    t.tau_noxmiss = 1.15;
    t.tau_inflate = 1.25;
    t.tau_balance = 3.0;
    return t;
}

spmv_status spmv_classify_profile(const spmv_profile_t* p, const spmv_thresholds_t* th,
                                  int32_t* cls)
{
    clear_error();
    if (!p || !cls) return fail(SPMV_ERR_INVALID_ARG, "spmv_classify_profile: NULL argument");
    const double s[3] = {p->s_noxmiss, p->s_inflate, p->s_balance};
    for (double v : s)
        if (!(v > 0.0) || !isfinite(v))
            return fail(SPMV_ERR_INVALID_ARG, "profile speedups must be finite and positive");
    const spmv_thresholds_t t = th ? *th : spmv_default_thresholds();
    const double tau[3] = {t.tau_noxmiss, t.tau_inflate, t.tau_balance};
    // examine the probes from the largest speedup down; equal speedups keep
    // the order CML, MB, IMB
    int order[3] = {0, 1, 2};
    for (int a = 1; a < 3; ++a)
        for (int b = a; b > 0 && s[order[b]] > s[order[b - 1]]; --b) {
            int tmp = order[b];
            order[b] = order[b - 1];
            order[b - 1] = tmp;
        }
    for (int k = 0; k < 3; ++k)
        if (s[order[k]] > tau[order[k]]) { *cls = order[k]; return SPMV_OK; }
    *cls = SPMV_CLASS_CMP;
    return SPMV_OK;
}

int32_t spmv_class_variant(int32_t cls)
{
    switch (cls) {
        // calibrated on GB300: per class, the variant with the lowest
        // geometric-mean slowdown against the exhaustive best on the training
        // matrices (CML 1.03, MB 1.00, IMB 1.01, CMP 1.03).  SLICED wins every
        // class because its prepare step adapts the layout to the row lengths
        // (length sort and row cap for imbalance, four slices per warp for
        // short rows); DYNAMIC is next for IMB (1.52)
        case SPMV_CLASS_CML: return SPMV_V7_SLICED;
        case SPMV_CLASS_MB: return SPMV_V7_SLICED;
        case SPMV_CLASS_IMB: return SPMV_V7_SLICED;
        case SPMV_CLASS_CMP: return SPMV_V7_SLICED;
        default: return -1;
    }
}

spmv_status spmv_class_choice(int32_t cls, spmv_choice_t* out)
{
    clear_error();
    if (!out) return fail(SPMV_ERR_INVALID_ARG, "spmv_class_choice: NULL output");
    if (cls < 0 || cls > 3) return fail(SPMV_ERR_INVALID_ARG, "spmv_class_choice: unknown class");
    // calibrated on GB300 like the variant table: per class, the SLICED form
    // (among the second level's launch configurations and delta-coded
    // layouts) with the lowest geometric-mean slowdown on the training
    // matrices the rule puts in that class.  {slices per warp, sort window,
    // row cap, index coding}; 0 = the prepare step's structural rule.
    static const int32_t form[4][4] = {
        {0, 0, 0, 0},      // CML: the structural rules (1.052)
        {1, 1, 1024, 0},   // MB: rows in order, one slice per warp (1.022)
        {1, 4096, 32, 0},  // IMB: length sort in windows of 4096, cap 32 (1.011)
        {0, 0, 0, 0},      // CMP: the structural rules (1.053)
    };
    spmv_choice_t c = {};
    c.cls = cls;
    c.variant = spmv_class_variant(cls);
    c.threads_per_row = form[cls][0];
    c.block_nnz = form[cls][1];
    c.items_per_warp = form[cls][2];
    c.index_coding = form[cls][3];
    c.value_type = SPMV_VAL_F64;
    c.source = 1;
    *out = c;
    return SPMV_OK;
}

spmv_status spmv_select(const spmv_features_t* f, const spmv_profile_t* p,
                        const spmv_thresholds_t* th, spmv_choice_t* out)
{
    clear_error();
    (void)f;
    if (!out) return fail(SPMV_ERR_INVALID_ARG, "spmv_select: NULL output");
    if (!p)
        return fail(SPMV_ERR_MODEL, "spmv_select: selection from features alone needs a model "
                                    "(spmv_select_model)");
    int32_t cls = -1;
    spmv_status st = spmv_classify_profile(p, th, &cls);
    if (st != SPMV_OK) return st;
    return spmv_class_choice(cls, out);
}

spmv_status spmv_prepare(const spmv_csr_t* A, const spmv_choice_t* c, int32_t trusted,
                         spmv_prepared_t** out, spmv_stream_t stream)
{
    clear_error();
    if (!out) return fail(SPMV_ERR_INVALID_ARG, "spmv_prepare: NULL output");
    *out = nullptr;
    if (!c) return fail(SPMV_ERR_INVALID_ARG, "spmv_prepare: NULL choice");
    spmv_status st = check_csr_args(A);
    if (st != SPMV_OK) return st;
    if ((st = check_choice(c)) != SPMV_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!trusted) {
        st = run_feature_pass(A, 128, nullptr, s);
        if (st != SPMV_OK) return st;
    }
    DeviceInfo dev;
    if ((st = current_device(&dev)) != SPMV_OK) return st;
    spmv_prepared_t* P = new (std::nothrow) spmv_prepared_t();
    if (!P) return fail(SPMV_ERR_NOMEM, "host allocation failed");
    P->A = *A;
    P->c = *c;
    P->device = dev.device;
    P->sm_count = dev.sm_count;
    st = prepare_impl(P, s);
    if (st == SPMV_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "spmv_prepare");
    }
    if (st == SPMV_OK && A->n_rows > 0) {
        // configure the variant's kernels now (one SpMV into scratch vectors),
        // so that later launches, including captured ones, make no
        // configuration call
        double *xs = nullptr, *ys = nullptr;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&xs), 8 * std::max<int64_t>(A->n_cols, 1), s);
        if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&ys), 8 * A->n_rows, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(xs, 0, 8 * std::max<int64_t>(A->n_cols, 1), s);
        if (e == cudaSuccess) {
            spmv_status rs = run_impl(P, xs, ys, s);
            if (rs != SPMV_OK) st = rs;
        }
        if (xs) cudaFreeAsync(xs, s);
        if (ys) cudaFreeAsync(ys, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess && st == SPMV_OK) st = cuda_fail(e, "spmv_prepare configure");
        if (st == SPMV_OK && P->status) {
            // the configuring run may not leave a timeout flag behind
            cudaMemsetAsync(P->status, 0, sizeof(unsigned), s);
            cudaStreamSynchronize(s);
        }
    }
    if (st != SPMV_OK) {
        cudaStreamSynchronize(s);
        release(P);
        delete P;
        return st;
    }
    *out = P;
    return SPMV_OK;
}

spmv_status spmv(const spmv_prepared_t* P, const double* x, double* y, spmv_stream_t stream)
{
    if (!P || (!x && P->A.n_cols > 0) || (!y && P->A.n_rows > 0))
        return fail(SPMV_ERR_INVALID_ARG, "spmv: NULL argument");
    return run_impl(P, x, y, reinterpret_cast<cudaStream_t>(stream));
}

spmv_status spmv_host(spmv_prepared_t* P, const double* x_host, double* y_host,
                      spmv_stream_t stream)
{
    spmv_status st = spmv_host_async(P, x_host, y_host, stream);
    if (st != SPMV_OK) return st;
    SPMV_CUDA_TRY(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
    return SPMV_OK;
}

spmv_status spmv_host_async(spmv_prepared_t* P, const double* x_host, double* y_host,
                            spmv_stream_t stream)
{
    clear_error();
    if (!P || (!x_host && P->A.n_cols > 0) || (!y_host && P->A.n_rows > 0))
        return fail(SPMV_ERR_INVALID_ARG, "spmv_host: NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    spmv_status st;
    if (!P->x_stage && P->A.n_cols > 0 && (st = dev_alloc(P, &P->x_stage, P->A.n_cols)) != SPMV_OK)
        return st;
    if (!P->y_stage && P->A.n_rows > 0 && (st = dev_alloc(P, &P->y_stage, P->A.n_rows)) != SPMV_OK)
        return st;
    if (P->A.n_cols > 0)
        SPMV_CUDA_TRY(cudaMemcpyAsync(P->x_stage, x_host, 8 * P->A.n_cols, cudaMemcpyHostToDevice, s));
    st = run_impl(P, P->x_stage, P->y_stage, s);
    if (st != SPMV_OK) return st;
    if (P->A.n_rows > 0)
        SPMV_CUDA_TRY(cudaMemcpyAsync(y_host, P->y_stage, 8 * P->A.n_rows, cudaMemcpyDeviceToHost, s));
    return SPMV_OK;
}

spmv_status spmv_prepared_info(const spmv_prepared_t* P, spmv_prepared_info_t* info)
{
    clear_error();
    if (!P || !info) return fail(SPMV_ERR_INVALID_ARG, "spmv_prepared_info: NULL argument");
    spmv_prepared_info_t i = {};
    i.variant = P->c.variant;
    i.threads_per_row = P->c.threads_per_row;
    i.block_nnz = P->c.block_nnz;
    i.items_per_warp = P->c.items_per_warp;
    i.value_type = P->c.value_type;
    i.n_rows = P->A.n_rows;
    i.n_cols = P->A.n_cols;
    i.nnz = P->A.nnz;
    i.n_blocks = P->n_blocks;
    i.n_wide_rows = P->n_wide;
    i.owned_bytes = P->owned_bytes;
    i.min_bytes = min_bytes_of(P);
    i.tile_items = P->tile_items;
    i.bulk_copy = P->bulk ? 1 : 0;
    i.accumulate = P->c.variant == SPMV_V6_COMPRESSED || P->c.variant == SPMV_V7_SLICED ? P->c.accumulate : 1;
    i.launches = launches_of(P);
    i.index_bytes = P->c.variant == SPMV_V7_SLICED && P->sl.value_type == SPMV_VAL_F64 ? P->sl.cbytes : 4;
    i.n_long_rows = P->c.variant == SPMV_V7_SLICED ? P->sl.n_long : 0;
    i.index_coding = P->c.variant == SPMV_V7_SLICED && P->sl.value_type == SPMV_VAL_F64 ? P->sl.coding : 0;
    i.uniform_len = P->c.variant == SPMV_V7_SLICED && P->sl.value_type == SPMV_VAL_F64 && P->sl.coding == 0
                        ? P->sl.uniform_len : -1;
    *info = i;
    return SPMV_OK;
}

spmv_status spmv_prepared_export(const spmv_prepared_t* P, int32_t which, void* dst,
                                 int64_t bytes, spmv_stream_t stream)
{
    clear_error();
    if (!P || (!dst && bytes != 0)) return fail(SPMV_ERR_INVALID_ARG, "spmv_prepared_export: NULL argument");
    const void* src = nullptr;
    int64_t size = 0;
    const int v = P->c.variant;
    switch (which) {
        case SPMV_EXPORT_ROW_BLOCKS:
            if (v == SPMV_V2_STREAM) { src = P->blocks; size = 4 * (P->n_blocks + 1); }
            break;
        case SPMV_EXPORT_MERGE_ROWS:
            if (v == SPMV_V3_MERGE) { src = P->blocks; size = 4 * (P->n_blocks + 1); }
            break;
        case SPMV_EXPORT_MERGE_NZ:
            if (v == SPMV_V3_MERGE) { src = P->merge_nz; size = 4 * (P->n_blocks + 1); }
            break;
        case SPMV_EXPORT_ROWBASE:
            if (v == SPMV_V6_COMPRESSED) { src = P->rowbase; size = 4 * P->A.n_rows; }
            break;
        case SPMV_EXPORT_OFFSETS:
            if (v == SPMV_V6_COMPRESSED && P->off16) { src = P->off16; size = 2 * P->A.nnz; }
            break;
        case SPMV_EXPORT_VALUES:
            if (v == SPMV_V6_COMPRESSED) {
                if (P->c.value_type == SPMV_VAL_F64) { src = P->A.val; size = 8 * P->A.nnz; }
                else { src = P->lowval; size = (P->c.value_type == SPMV_VAL_F32 ? 4 : 2) * P->A.nnz; }
            }
            break;
        case SPMV_EXPORT_SLICE_PERM:
            if (v == SPMV_V7_SLICED && P->sl.sigma > 1) { src = P->sl.perm; size = 4 * P->A.n_rows; }
            break;
        case SPMV_EXPORT_SLICE_ROWLEN:
            if (v == SPMV_V7_SLICED) { src = P->sl.rowlen; size = 4 * 32 * P->sl.n_slices; }
            break;
        case SPMV_EXPORT_SLICE_LEN:
            if (v == SPMV_V7_SLICED) { src = P->sl.slice_len; size = 4 * P->sl.n_slices; }
            break;
        case SPMV_EXPORT_SLICE_PTR:
            if (v == SPMV_V7_SLICED) { src = P->sl.slice_ptr; size = 8 * (P->sl.n_slices + 1); }
            break;
        case SPMV_EXPORT_SLICE_COL:
            if (v == SPMV_V7_SLICED && !P->sl.off16) { src = P->sl.col; size = 4 * P->sl.tot; }
            break;
        case SPMV_EXPORT_SLICE_VAL:
            if (v == SPMV_V7_SLICED) {
                const int t = P->sl.value_type;
                src = t == SPMV_VAL_F64 ? (const void*)P->sl.val : P->sl.lowval;
                size = (t == SPMV_VAL_F64 ? 8 : t == SPMV_VAL_F32 ? 4 : 2) * P->sl.tot;
            }
            break;
        case SPMV_EXPORT_SLICE_OFF16:
            if (v == SPMV_V7_SLICED && P->sl.off16) { src = P->sl.off; size = 2 * P->sl.tot; }
            break;
        case SPMV_EXPORT_SLICE_ROWBASE:
            if (v == SPMV_V7_SLICED && (P->sl.off16 || P->sl.coding == 1)) {
                src = P->sl.rowbase;
                size = 4 * 32 * P->sl.n_slices;
            }
            break;
        case SPMV_EXPORT_SLICE_DELTA:
            if (v == SPMV_V7_SLICED && P->sl.coding == 1) {
                src = P->sl.scol;
                size = (int64_t)P->sl.cbytes * P->sl.tot;
            }
            break;
        case SPMV_EXPORT_SLICE_PANEL_LO:
            if (v == SPMV_V7_SLICED && P->sl.coding == 2) { src = P->sl.scol; size = 2 * P->sl.tot; }
            break;
        case SPMV_EXPORT_SLICE_PANEL_STEP:
            if (v == SPMV_V7_SLICED && P->sl.coding == 2) { src = P->sl.step; size = P->sl.tot; }
            break;
        case SPMV_EXPORT_DYN_M1:
            if (v == SPMV_V4_DYNAMIC) { src = P->dyn.m1; size = 4 * (int64_t)P->dyn.n_m1; }
            break;
        case SPMV_EXPORT_DYN_M2:
            if (v == SPMV_V4_DYNAMIC) { src = P->dyn.m2; size = 4 * (int64_t)P->dyn.n_m2; }
            break;
        case SPMV_EXPORT_DYN_LONG:
            if (v == SPMV_V4_DYNAMIC) { src = P->dyn.lrow; size = 4 * (int64_t)P->dyn.n_long; }
            break;
        case SPMV_EXPORT_DYN_SEG_OFF:
            if (v == SPMV_V4_DYNAMIC && P->dyn.n_long > 0) {
                src = P->dyn.seg_off;
                size = 4 * ((int64_t)P->dyn.n_long + 1);
            }
            break;
        case SPMV_EXPORT_SLICE_LONG:
            if (v == SPMV_V7_SLICED) { src = P->sl.long_rows; size = 4 * (int64_t)P->sl.n_long; }
            break;
        case SPMV_EXPORT_SLICE_SEG_OFF:
            if (v == SPMV_V7_SLICED && P->sl.n_long > 0) {
                src = P->sl.seg_off;
                size = 4 * ((int64_t)P->sl.n_long + 1);
            }
            break;
        case SPMV_EXPORT_SLICE_SEG_BOUNDS:
            if (v == SPMV_V7_SLICED) { src = P->sl.seg_be; size = 16 * (int64_t)P->sl.n_seg; }
            break;
        case SPMV_EXPORT_SLICE_SEG_ROW:
            if (v == SPMV_V7_SLICED) { src = P->sl.seg_row; size = 4 * (int64_t)P->sl.n_seg; }
            break;
        case SPMV_EXPORT_SLICE_FIX:
            if (v == SPMV_V7_SLICED) { src = P->sl.fix; size = 4 * (int64_t)P->sl.n_fix; }
            break;
        case SPMV_EXPORT_SLICE_SEG_FIX:
            if (v == SPMV_V7_SLICED) { src = P->sl.seg_fix; size = 4 * (int64_t)P->sl.n_seg; }
            break;
        case SPMV_EXPORT_SLICE_DIAG:
            if (v == SPMV_V7_SLICED && P->sl.value_type == SPMV_VAL_F64 && P->sl.cbytes < 4 &&
                P->sl.coding == 0) {
                src = P->sl.scol;
                size = (int64_t)P->sl.cbytes * P->sl.tot;
            }
            break;
        default:
            return fail(SPMV_ERR_INVALID_ARG, "unknown export");
    }
    if (size == 0 && src && bytes == 0) return SPMV_OK;  // an empty array
    if (!src && size == 0 && which == SPMV_EXPORT_OFFSETS && v == SPMV_V6_COMPRESSED)
        return fail(SPMV_ERR_UNSUPPORTED, "every row is wide: no 16-bit offsets were built");
    if (!src && size != 0) return fail(SPMV_ERR_UNSUPPORTED, "array not held");
    if (size == 0 && !src) return fail(SPMV_ERR_UNSUPPORTED, "this variant does not hold that array");
    if (bytes != size) return fail(SPMV_ERR_INVALID_ARG, "size mismatch: need " + std::to_string(size));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    SPMV_CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)size, cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    return SPMV_OK;
}

spmv_status spmv_prepared_status(const spmv_prepared_t* P, spmv_stream_t stream)
{
    clear_error();
    if (!P) return fail(SPMV_ERR_INVALID_ARG, "spmv_prepared_status: NULL argument");
    if (!P->status) return SPMV_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned h = 0;
    SPMV_CUDA_TRY(cudaMemcpyAsync(&h, P->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaMemsetAsync(P->status, 0, sizeof(unsigned), s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) return fail(SPMV_ERR_TIMEOUT, "a bounded device wait gave up during an earlier spmv");
    return SPMV_OK;
}

void spmv_prepared_free(spmv_prepared_t* P)
{
    if (!P) return;
    cudaDeviceSynchronize();
    release(P);
    delete P;
}

}  // extern "C"
