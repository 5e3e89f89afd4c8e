// spmv_stream_noalloc: y = A x with the pipelined STREAM kernel, for callers
// that must not allocate device memory.
//
// Who needs it: code that runs where a device allocation is not allowed or
// not wanted -- an iterative solver's inner loop that must never stall the
// device (cudaMalloc/cudaFree synchronize it), or a host application that
// commits all device memory through its own allocator at start-up and
// forbids allocations after that.  spmv_prepare allocates the prepared
// arrays; this entry point instead keeps its scratch (window starts, carried
// partial rows, a status word) in one file-scope __device__ array of fixed
// size, which every GPU that loads the library holds until the process exits.
#include <mutex>

#include "common.cuh"

namespace spmvlib {
namespace {

constexpr int kNaWindow = 2048;                      // nonzeros per window
constexpr int64_t kNaMaxWindows = 65536;             // 134,217,728 nonzeros at most

struct NoAllocScratch {
    double carry_val[kNaMaxWindows];   // partial sum carried by each window
    int32_t blocks[kNaMaxWindows + 1]; // first row owned by each window
    int32_t carry_row[kNaMaxWindows];  // row of that partial, -1 when none
    unsigned status;                   // bounded-wait timeout flag
};

// The scratch itself.  In host code this name is only a host-side stand-in:
// its device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kNaMaxDevices = 64;
NoAllocScratch* g_na_addr[kNaMaxDevices] = {};
std::mutex g_na_mu;

}  // namespace
}  // namespace spmvlib

using namespace spmvlib;

extern "C" spmv_status spmv_stream_noalloc(const spmv_csr_t* A, const double* x, double* y,
                                           spmv_stream_t stream)
{
    clear_error();
    spmv_status st = check_csr_args(A);
    if (st != SPMV_OK) return st;
    if ((!x && A->n_cols > 0) || (!y && A->n_rows > 0))
        return fail(SPMV_ERR_INVALID_ARG, "spmv_stream_noalloc: NULL vector");
    const int64_t n_win = A->nnz > 0 ? (A->nnz + kNaWindow - 1) / kNaWindow : 1;
    if (n_win > kNaMaxWindows)
        return fail(SPMV_ERR_UNSUPPORTED,
                    "spmv_stream_noalloc: at most 134217728 nonzeros fit its static scratch (got " +
                        std::to_string(A->nnz) + ")");
    if (!tma_aligned(*A))
        return fail(SPMV_ERR_UNSUPPORTED,
                    "spmv_stream_noalloc: rowptr, colind and val must be 16-byte aligned");
    if (A->n_rows == 0) return SPMV_OK;
    DeviceInfo dev;
    if ((st = current_device(&dev)) != SPMV_OK) return st;
    NoAllocScratch* scratch = nullptr;
    {
        // set-up on the first call on each device, with that device current
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (dev.device >= kNaMaxDevices)
            return fail(SPMV_ERR_UNSUPPORTED, "spmv_stream_noalloc: device ordinal too large");
        if (!g_na_addr[dev.device]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
            g_na_addr[dev.device] = static_cast<NoAllocScratch*>(p);
        }
        scratch = g_na_addr[dev.device];
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the status word must start at zero; blocks and carry_row are rewritten
    // in full by every call
    SPMV_CUDA_TRY(cudaMemsetAsync(&scratch->status, 0, sizeof(unsigned), s));
    SPMV_CUDA_TRY(launch_row_blocks(*A, kNaWindow, n_win, scratch->blocks, s));
    SPMV_CUDA_TRY(launch_window(*A, kNaWindow, scratch->blocks, n_win, scratch->carry_row,
                                scratch->carry_val, &scratch->status, dev.sm_count, x, y, s));
    return SPMV_OK;
}

extern "C" spmv_status spmv_stream_noalloc_status(spmv_stream_t stream)
{
    clear_error();
    DeviceInfo dev;
    spmv_status st = current_device(&dev);
    if (st != SPMV_OK) return st;
    NoAllocScratch* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (dev.device < kNaMaxDevices) scratch = g_na_addr[dev.device];
    }
    if (!scratch) return SPMV_OK;  // no call has run on this device
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned h = 0;
    SPMV_CUDA_TRY(cudaMemcpyAsync(&h, &scratch->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) return fail(SPMV_ERR_TIMEOUT, "spmv_stream_noalloc: a bounded device wait gave up; y is incomplete");
    return SPMV_OK;
}
