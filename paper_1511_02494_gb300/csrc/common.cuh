// Internal declarations shared by the library's translation units.
// Not part of the public ABI (that is include/spmv.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "spmv.h"

namespace spmvlib {

constexpr unsigned FULL_MASK = 0xffffffffu;

// ---- error reporting ------------------------------------------------------
void set_error(const std::string& msg);
void clear_error();
const char* last_error_cstr();
spmv_status fail(spmv_status s, const std::string& msg);
spmv_status cuda_fail(cudaError_t e, const char* what);

#define SPMV_CUDA_TRY(expr)                                        \
    do {                                                           \
        cudaError_t _e = (expr);                                   \
        if (_e != cudaSuccess) return ::spmvlib::cuda_fail(_e, #expr); \
    } while (0)

// ---- device facts ------------------------------------------------------------
struct DeviceInfo {
    int device = -1;
    int sm_count = 0;
    int l2_bytes = 0;
    int max_persist_l2 = 0;
    int max_window = 0;
};
// Facts of the current device (queried once per device).
spmv_status current_device(DeviceInfo* out);

// ---- matrix checks on the host side of the ABI ----------------------------------
spmv_status check_csr_args(const spmv_csr_t* A);
spmv_status check_choice(const spmv_choice_t* c);

// ---- the prepared object ----------------------------------------------------------
}  // namespace spmvlib

// DYNAMIC variant plan (dynamic.cu)
struct DynPlan {
    int seg = 0, lim_s = 0, chunk_rows = 0;
    int n_m1 = 0, n_m2 = 0, n_long = 0, n_seg = 0;
    int* m1 = nullptr;       // rows with lim_s < len <= 64
    int* m2 = nullptr;       // rows with 64 < len <= seg
    int* lrow = nullptr;     // rows longer than seg
    int* seg_off = nullptr;  // first segment of each long row, [n_long + 1]
    double* partial = nullptr;  // one partial sum per segment
    unsigned* ticket = nullptr; // [n_long] segments of the row finished in this call (0 between calls)
};

// SLICED (V7): rows longer than the plan's cap (kSlicedCap unless chosen)
// are computed from CSR in segments of kSlicedSeg nonzeros, one warp each
constexpr int kSlicedCap = 1024;
constexpr int kSlicedCapMax = 1 << 16;
constexpr int kSlicedSeg = 2048;

struct SlicedPlan {
    int64_t n_slices = 0, tot = 0;
    int sigma = 1, n_long = 0;
    int uniform_len = -1;        // >= 0: every row has this many nonzeros, rows in order, none long
    int* rowlen = nullptr;       // [32 n_slices] row length per position, -1: long or absent
    int* slice_len = nullptr;    // [n_slices]
    int64_t* slice_ptr = nullptr;  // [n_slices + 1] element offset of each slice
    int* perm = nullptr;         // [n_rows] position -> row (sigma > 1 only)
    int* col = nullptr;          // [tot] column-major slice contents (32-bit columns)
    void* scol = nullptr;        // FP64 values: [tot] stored columns, cbytes each
    int cbytes = 4;              // bytes per stored column: 4 columns; 2 / 1 column - row (coding 0)
                                 // or delta (coding 1); 3 panel offset + step (coding 2)
    int coding = 0;              // FP64 columns: 0 columns / row offsets, 1 deltas, 2 panels
    uint8_t* step = nullptr;     // [tot] coding 2: panel step from the previous element
    double* val = nullptr;       // [tot]
    int* long_rows = nullptr;    // [n_long], ascending
    int* seg_off = nullptr;      // [n_long + 1] first segment of each long row
    double* partial = nullptr;   // [n_seg] segment sums
    int64_t* seg_be = nullptr;   // [2 n_seg] CSR begin and end of each segment
    int* seg_row = nullptr;      // [n_seg] row of a segment that is its row's only one, else -1
    int* fix = nullptr;          // [n_fix] long rows (list indices) with several segments
    int* seg_fix = nullptr;      // [n_seg] index in fix of the segment's row, -1 for a single segment
    unsigned* ticket = nullptr;  // [n_fix] segments of the row finished in this call (0 between calls)
    std::vector<uint8_t> seg_several;  // host, [n_seg]: 1 when the segment's row has several
    int n_fix = 0;
    int n_seg = 0;
    // low-precision values (FP32 / BF16), optionally 16-bit column offsets
    int value_type = 0;
    int vec = 1;                 // elements of a row side by side: 1 (FP64) or 4 (FP32/BF16)
    bool acc32 = false, off16 = false;
    void* lowval = nullptr;      // [tot] values in value_type
    uint16_t* off = nullptr;     // [tot] column - rowbase (off16)
    int* rowbase = nullptr;      // [32 n_slices] first column of each position's row (off16)
    float* x32 = nullptr;        // FP32 copy of x (acc32)
    unsigned* count = nullptr;   // scratch counter
};

struct spmv_prepared {
    spmv_csr_t A{};
    spmv_choice_t c{};
    int device = -1;
    int64_t n_blocks = 0;          // STREAM blocks / MERGE parts / DYNAMIC chunks
    int32_t* blocks = nullptr;     // STREAM row blocks, MERGE start rows
    int32_t* merge_nz = nullptr;   // MERGE start nonzeros
    int32_t* carry_row = nullptr;  // MERGE per-part carry row
    double* carry_val = nullptr;   // MERGE per-part carry value
    unsigned int* counter = nullptr;  // DYNAMIC work counter
    int32_t* rowbase = nullptr;    // COMPRESSED
    uint16_t* off16 = nullptr;     // COMPRESSED
    void* lowval = nullptr;        // COMPRESSED values (F32/BF16), or NULL for F64
    int64_t n_wide = 0;
    double* x_stage = nullptr;     // spmv_host staging
    double* y_stage = nullptr;
    int64_t owned_bytes = 0;
    int sm_count = 0;
    int l2_window_bytes = 0;       // LATENCY: bytes of x kept persisting in L2
    bool persist_held = false;     // LATENCY: counted among the persisting-L2 users
    int tile_items = 0;            // MERGE: path items per tile (CTA or warp)
    bool bulk = false;             // STREAM / MERGE: pipelined bulk-copy kernel in use
    unsigned* status = nullptr;    // device status word (bounded-wait timeouts)
    DynPlan dyn;
    float* x32 = nullptr;          // COMPRESSED with FP32 accumulation: FP32 copy of x
    SlicedPlan sl;
    std::vector<void*> owned;      // every device allocation above, freed by release()
};

namespace spmvlib {

// ---- kernel launchers (spmv_kernels.cu) -------------------------------------------
cudaError_t launch_scalar(const spmv_csr_t& A, const double* x, double* y, cudaStream_t s);
cudaError_t launch_subwarp(const spmv_csr_t& A, int T, const double* x, double* y,
                           cudaStream_t s);
cudaError_t launch_row_blocks(const spmv_csr_t& A, int64_t block_nnz, int64_t n_blocks,
                              int32_t* blocks, cudaStream_t s);
cudaError_t launch_stream(const spmv_csr_t& A, const int32_t* blocks, int64_t n_blocks,
                          int block_nnz, const double* x, double* y, cudaStream_t s);
cudaError_t launch_merge_coords(const spmv_csr_t& A, int items, int64_t n_parts,
                                int32_t* mrow, int32_t* mnz, cudaStream_t s);
cudaError_t launch_merge(const spmv_csr_t& A, int items, const int32_t* mrow,
                         const int32_t* mnz, int64_t n_parts, int32_t* carry_row,
                         double* carry_val, const double* x, double* y, cudaStream_t s);
bool tma_aligned(const spmv_csr_t& A);
cudaError_t launch_merge_tma(const spmv_csr_t& A, int tile_items, const int32_t* mrow,
                             const int32_t* mnz, int64_t n_tiles, int32_t* carry_row,
                             double* carry_val, unsigned* status, int sm_count, const double* x,
                             double* y, cudaStream_t s);
cudaError_t launch_window(const spmv_csr_t& A, int block_nnz, const int32_t* blocks, int64_t n_win,
                          int32_t* carry_row, double* carry_val, unsigned* status, int sm_count,
                          const double* x, double* y, cudaStream_t s);
// The carry fix-ups of the two pipelined kernels on their own (they run
// inside launch_window / launch_merge_tma; exported for the fix-up self-test)
cudaError_t launch_window_fixup(int64_t n_win, int64_t n_rows, const int32_t* carry_row,
                                const double* carry_val, const unsigned* status, double* y,
                                cudaStream_t s);
cudaError_t launch_tile_fixup(int64_t n_tiles, int64_t n_rows, const int32_t* carry_row,
                              const double* carry_val, const unsigned* status, double* y,
                              cudaStream_t s);
spmv_status prepared_alloc(spmv_prepared* P, void** p, int64_t bytes);
spmv_status dyn_prepare(spmv_prepared* P, cudaStream_t s);
cudaError_t launch_dyn(const spmv_prepared* P, const double* x, double* y, cudaStream_t s);
spmv_status sliced_prepare(spmv_prepared* P, cudaStream_t s);
cudaError_t launch_sliced(const spmv_prepared* P, const double* x, double* y, cudaStream_t s);
cudaError_t launch_latency(const spmv_csr_t& A, int T, const double* x, double* y,
                           int l2_window_bytes, cudaStream_t s);
cudaError_t launch_compress(const spmv_csr_t& A, int32_t* rowbase, uint16_t* off16,
                            unsigned long long* n_wide, int value_type, void* lowval,
                            cudaStream_t s);
cudaError_t launch_compressed32(const spmv_csr_t& A, int T, int value_type, const int32_t* rowbase,
                                const uint16_t* off16, const void* lowval, bool all_wide,
                                const double* x, float* x32, double* y, cudaStream_t s);
cudaError_t launch_compressed(const spmv_csr_t& A, int T, int value_type,
                              const int32_t* rowbase, const uint16_t* off16,
                              const void* lowval, bool all_wide, const double* x, double* y,
                              cudaStream_t s);

// ---- features / validation (features.cu) --------------------------------------------
// Per-row pass; when `features_out` is NULL only validates.  err bits:
// 1 rowptr[0] != 0, 2 rowptr[n] != nnz, 4 rowptr decreasing / out of range,
// 8 column out of range, 16 columns not strictly increasing.
spmv_status run_feature_pass(const spmv_csr_t* A, int32_t line_bytes,
                             spmv_features_t* features_out, cudaStream_t s);

// Default lanes per row for a mean row length.
int auto_threads_per_row(double mean_nnz);

// Per-device cache of a kernel's launch configuration (dynamic shared memory
// attribute set, resident blocks per SM), filled outside any stream capture
// by the variant's configure step at prepare time so that later launches --
// including launches captured into a CUDA graph -- make no other API call.
struct LaunchCache {
    int per_sm[64] = {};
};
template <typename K>
cudaError_t cached_occupancy(LaunchCache& c, K kernel, int threads, size_t smem, int* per_sm)
{
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    if (d < 0 || d >= 64) return cudaErrorInvalidDevice;
    if (c.per_sm[d] == 0) {
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem);
        if (e != cudaSuccess) return e;
        c.per_sm[d] = n > 0 ? n : -1;
    }
    *per_sm = c.per_sm[d];
    return *per_sm > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

}  // namespace spmvlib
