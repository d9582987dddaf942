// Internal helpers shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/bbl.h"

namespace bbl {

constexpr int kWarp = 32;
constexpr int kSellC = 32;     // rows per SELL slice
constexpr int kMaxB = 16;      // largest block size
constexpr int kKronMaxK = 30;  // coupling terms of a Kronecker-factored operator
constexpr int kKronMaxFactors = 2 + 2 * kKronMaxK;

// ------------------------------------------------------------------ errors
bbl_status set_error(bbl_status s, const char* fmt, ...);
void clear_error();

#define BBL_CUDA(call)                                                                 \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            if (e_ == cudaErrorMemoryAllocation)                                       \
                return ::bbl::set_error(BBL_ERR_OOM, "%s: %s (%s:%d)", #call,          \
                                        cudaGetErrorString(e_), __FILE__, __LINE__);   \
            return ::bbl::set_error(BBL_ERR_CUDA, "%s: %s (%s:%d)", #call,             \
                                    cudaGetErrorString(e_), __FILE__, __LINE__);       \
        }                                                                              \
    } while (0)

#define BBL_TRY(expr)                                                                  \
    do {                                                                               \
        bbl_status s_ = (expr);                                                        \
        if (s_ != BBL_OK) return s_;                                                   \
    } while (0)

// Every kernel launch is followed by BBL_LAUNCH_CHECK(), which also counts it.
void count_launch();
#define BBL_LAUNCH_CHECK()            \
    do {                              \
        ::bbl::count_launch();        \
        BBL_CUDA(cudaGetLastError()); \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Internal block type of the polish stage: float-float pairs (df32.cuh), 8 bytes.
constexpr int kDF32 = 2;

inline size_t dtype_size(int dt) { return (dt == BBL_FP64 || dt == kDF32) ? 8 : 4; }

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Is p device-accessible memory the kernels may read directly?
bool is_device_pointer(const void* p);

// Frees the workspace cache's idle buffers on the current device (see
// PoolBuf); true if there were any.
bool pool_free_idle_current_device();

// ------------------------------------------------------------------ device buffers
// Owning device allocation; frees on destruction.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    // workspace growth: at least doubles, so that a buffer sized by a
    // growing basis is reallocated (cudaFree synchronises the device) a
    // logarithmic number of times
    bbl_status grow(size_t need) {
        if (bytes >= need) return BBL_OK;
        return alloc(need > 2 * bytes ? need : 2 * bytes);
    }
    bbl_status alloc(size_t nbytes) {
        release();
        if (nbytes == 0) nbytes = 16;
        cudaError_t e = cudaMalloc(&p, nbytes);
        if (e == cudaErrorMemoryAllocation && pool_free_idle_current_device()) {  // cached bases back, once more
            (void)cudaGetLastError();
            e = cudaMalloc(&p, nbytes);
        }
        if (e != cudaSuccess) {
            p = nullptr;
            (void)cudaGetLastError();
            return set_error(BBL_ERR_OOM, "cudaMalloc(%zu bytes): %s", nbytes, cudaGetErrorString(e));
        }
        bytes = nbytes;
        return BBL_OK;
    }
    template <typename T>
    T* as() const { return static_cast<T*>(p); }
};

// Large scratch kept across calls (the Lanczos bases): release() hands the
// allocation to a per-device idle list with an event recorded on the stream
// it was used on; alloc() takes the smallest idle allocation of this device
// that is large enough but at most 1/16 larger, and makes its own stream
// wait on that event, so reuse is ordered on the GPU without a host
// synchronisation.  When cudaMalloc (here or in DevBuf) runs out of memory
// the idle allocations of the device are freed and it is tried once more;
// at most kPoolIdleMax allocations per device stay idle (the oldest goes).
// bbl_workspace_release() frees every idle allocation.
struct PoolBuf {
    void* p = nullptr;
    size_t bytes = 0;  // capacity
    cudaStream_t st = nullptr;
    int dev = 0;
    PoolBuf() = default;
    PoolBuf(const PoolBuf&) = delete;
    PoolBuf& operator=(const PoolBuf&) = delete;
    ~PoolBuf() { release(); }
    bbl_status alloc(size_t nbytes, cudaStream_t stream);
    void release();
    template <typename T>
    T* as() const { return static_cast<T*>(p); }
};
// bytes held idle for device dev (counted as free when sizing a basis)
size_t pool_idle_bytes(int dev);

// Pinned host staging buffer.
struct HostBuf {
    void* p = nullptr;
    HostBuf() = default;
    HostBuf(const HostBuf&) = delete;
    HostBuf& operator=(const HostBuf&) = delete;
    ~HostBuf() { if (p) cudaFreeHost(p); }
    bbl_status alloc(size_t nbytes) {
        if (p) cudaFreeHost(p);
        p = nullptr;
        cudaError_t e = cudaMallocHost(&p, nbytes ? nbytes : 16);
        if (e != cudaSuccess) {
            p = nullptr;
            (void)cudaGetLastError();
            return set_error(BBL_ERR_OOM, "cudaMallocHost(%zu): %s", nbytes, cudaGetErrorString(e));
        }
        return BBL_OK;
    }
    template <typename T>
    T* as() const { return static_cast<T*>(p); }
};

}  // namespace bbl

// ------------------------------------------------------------------ the matrix object
struct bbl_matrix {
    int64_t n = 0, nnz = 0;
    int fmt = BBL_CSR;
    int storage = BBL_FP64;
    double norm_inf = 0.0;
    // CSR (always kept unless SELL-only FP32 without keep flag; see matrix.cu)
    bbl::DevBuf row_ptr;   // int64 [n+1]
    bbl::DevBuf col;       // int32 [nnz]
    bbl::DevBuf val;       // storage type [nnz]
    bbl::DevBuf val64;     // FP64 copy of the values (FP32 storage with keep_fp64)
    bool has_csr = false;
    // SELL-C-sigma
    int sell_sigma = 0;
    int spmm_lanes = 0;    // CSR lanes per row from the autotuner (0 = built-in rule)
    int64_t nslices = 0, padded_nnz = 0;
    bbl::DevBuf slice_ptr; // int64 [nslices+1], element offsets
    bbl::DevBuf sell_col;  // int32 [padded_nnz]
    bbl::DevBuf sell_val;  // storage type [padded_nnz]
    bbl::DevBuf sell_len;  // int32 [nslices*32] row lengths (0 past n)
    bbl::DevBuf perm;      // int32 [nslices*32] original row of each slot (-1 past n)
    // diagonal, FP64 [n]
    bbl::DevBuf diag;
    // Kronecker-factored operator (fmt == BBL_KRON): H = Hp (x) I + I (x) Hn +
    // sum_k Cp_k (x) Cn_k kept as its factors (Hp, Hn, Cp_0, Cn_0, ...),
    // packed: factor f's row pointers (int32) start at kf_ptr_off[f], its
    // columns (int32) and values (FP32 and FP64 copies) at kf_nz_off[f]
    int64_t kron_nP = 0, kron_nN = 0;
    int kron_K = 0;
    int kron_prow_cap = 0;  // most entries of one row p over Hp and all Cp_k
    int kron_row_cap = 0;   // power of two >= the most term contributions of one row of H
    bbl::DevBuf kf_ptr, kf_col, kf_val32, kf_val64;
    // tiled format (fmt == BBL_TILED, tiled.cu): row blocks and column tiles of
    // `tile` rows (<= 1024); per (row block, column tile) pair with entries:
    // the tile id (int32), its first entry (int64), tile + 1 row offsets
    // (uint16, row-major prefix sums); entries as the column within the tile
    // (uint16) and the value (storage type), slot-major per 64-row slice
    int tile = 0;
    int64_t t_nrb = 0, t_npairs = 0;
    bbl::DevBuf t_pair_ptr, t_pair_tile, t_pair_base, t_off, t_lcol, t_val;
    int64_t kf_ptr_off[bbl::kKronMaxFactors] = {};
    int64_t kf_nz_off[bbl::kKronMaxFactors] = {};
    int64_t device_bytes() const {
        return (int64_t)(row_ptr.bytes + col.bytes + val.bytes + val64.bytes + slice_ptr.bytes + sell_col.bytes +
                         sell_val.bytes + sell_len.bytes + perm.bytes + diag.bytes + kf_ptr.bytes + kf_col.bytes +
                         kf_val32.bytes + kf_val64.bytes + t_pair_ptr.bytes + t_pair_tile.bytes +
                         t_pair_base.bytes + t_off.bytes + t_lcol.bytes + t_val.bytes);
    }
};

namespace bbl {
// spmm.cu
bbl_status spmm_dispatch(const bbl_matrix* A, int b, const void* V, void* W, bool f64_arith, cudaStream_t st,
                         int rows_per_warp_hint = 0);
// W = H V with float-float blocks V, W (n x b pairs) and FP32 matrix values
bbl_status spmm_df32(const bbl_matrix* A, int b, const void* V, void* W, cudaStream_t st);
// rows [r0, r1) of W = H V in FP64 arithmetic from the CSR copy (other rows of W untouched)
bbl_status spmm_rows_f64(const bbl_matrix* A, int b, const double* V, double* W, int64_t r0, int64_t r1,
                         cudaStream_t st);
// Algorithmic bytes of one SpMM with b columns: the stored matrix (values of
// sv bytes, int32 columns, int64 row pointers) read once, V read once and W
// written once (sx bytes per block element); a factored matrix stores no
// entries, so only the factors (int32 columns and row pointers, FP32 and
// FP64 values) and the two blocks count.
inline double spmm_alg_bytes(const bbl_matrix* A, int b, double sv, double sx) {
    const double blocks = 2.0 * (double)A->n * b * sx;
    if (A->fmt == BBL_KRON) return (double)(A->kf_ptr.bytes + A->kf_col.bytes + A->kf_val32.bytes) + blocks;
    // tiled: 16-bit columns and the values, the pair tables and row offsets
    if (A->fmt == BBL_TILED)
        return (double)A->nnz * (sv + 2.0) + (double)A->t_npairs * (12.0 + 2.0 * (A->tile + 1)) + blocks;
    return (double)A->nnz * (sv + 4.0) + (double)(A->n + 1) * 8.0 + blocks;
}
// kron.cu: W = H V from the factors of a BBL_KRON matrix; dt = element type
// of V and W (BBL_FP32, BBL_FP64 or kDF32)
bbl_status kron_spmm(const bbl_matrix* A, int b, int dt, const void* V, void* W, cudaStream_t st);
// tiled.cu: the tiled copy of A's CSR (tile rows per row block / columns per
// tile), and W = H V from it (dt as in kron_spmm; b a multiple of 16 bytes of
// blocks: tiled_supports)
bbl_status tiled_build(bbl_matrix* A, int T, cudaStream_t st);
bbl_status tiled_spmm(const bbl_matrix* A, int b, int dt, const void* V, void* W, cudaStream_t st);
inline bool tiled_supports(const bbl_matrix* A, int b, int dt) {
    const int es = (dt == BBL_FP32) ? 4 : 8;
    const int vec = 16 / es;
    return A->fmt == BBL_TILED && A->tile > 0 && A->tile <= 1024 && b % vec == 0 &&
           2 * (int64_t)A->tile * vec * es <= 200 * 1024;
}
// the principal submatrix H[S,S] of a BBL_KRON matrix as CSR (FP64 values):
// S device int32 [k] ascending rows, pos device int32 [n] (position in S or
// -1); row_ptr (int64 [k+1]), col, val allocated here
bbl_status kron_submatrix(const bbl_matrix* A, int64_t k, const int* S, const int* pos, DevBuf& row_ptr,
                          DevBuf& col, DevBuf& val, int64_t* nnz, cudaStream_t st);
// block.cu
struct BlockWork;  // scratch for Gram/reorth/CholQR2
bbl_status gram(int64_t n, int b, int nblocks, int dtype, const void* Q, const void* W, double* C,
                DevBuf& partials, cudaStream_t st);
bbl_status update(int64_t n, int b, int nblocks, int dtype, const void* Q, const double* C, void* W,
                  cudaStream_t st);
// first-pass Gram C ~= Q16^T W from the FP16 copy Q16 of an FP32 basis (b = 8)
bbl_status gram_half(int64_t n, int nblocks, const void* Q16, const float* W, double* C, DevBuf& partials,
                     cudaStream_t st);
// W -= Q C (b = 8, FP32) with blocks 0 .. nblocks - nnew - 1 read from the
// FP16 copy Q16 (tensor cores, their coefficients rounded to FP16 after a
// power-of-two scaling) and the nnew newest from the FP32 basis Q (FMA);
// work is grown as needed
bbl_status update_half_old(int64_t n, int nblocks, int nnew, const void* Q16, const float* Q, const double* C,
                           float* W, DevBuf& work, cudaStream_t st);
// float-float W -= Q C (b = 8) with blocks 0 .. nblocks - nnew - 1 read from
// the FP32 copy Q32 (FP32 products and sums) and the nnew newest from the
// float-float basis Q
bbl_status update_df32_f32old(int64_t n, int nblocks, int nnew, const float* Q32, const void* Q, const double* C,
                             void* W, cudaStream_t st);
// FP16 copy (round to nearest) of count FP32 values
bbl_status to_half(int64_t count, const float* in, void* out, cudaStream_t st);
// out[e] = sum over the nparts parts of partial[p * count + e], in a fixed order
void reduce_partials(int64_t count, int nparts, const double* partial, double* out, cudaStream_t st);
// SMs the persistent Gram kernels use (the rest stay free for the Ritz solve)
int gram_worker_sms();
// cgs.cu: W -= Q C1 (written over W) and C2 = Q^T W (the updated W) in one
// read of the FP32 basis, on the tensor cores (b = 8, nblocks <=
// 128: update_gram_tc_supports); work is grown as needed
bool update_gram_tc_supports(int nblocks);
bbl_status update_gram_tc(int64_t n, int nblocks, const float* Q, const double* C1, float* W, double* C2,
                          DevBuf& work, cudaStream_t st);
bbl_status ritz_vectors(int64_t n, int b, int nblocks, int dtype, const void* Q, int k, const double* S,
                        double* X, cudaStream_t st);
bbl_status cholqr2_dev(int64_t n, int b, int dtype, void* W, double* B, double defl_abs2, int* d_ndefl,
                       int* d_deflmask, DevBuf& partials, DevBuf& small, cudaStream_t st);
// ritz.cu
bbl_status ritz_dev(int m, int p, int nev, const double* Tband, double* theta, double* S, DevBuf& work,
                    cudaStream_t st, const double* warm = nullptr, int warm_count = 0);
// rng.cu
bbl_status fill_normal(int64_t n, int b, uint64_t seed, uint64_t offset, double* P, cudaStream_t st);
bbl_status fill_uniform_cols(int64_t n, int b, int dtype, uint64_t seed, uint64_t offset, const int* mask,
                             void* Z, cudaStream_t st);
}  // namespace bbl
