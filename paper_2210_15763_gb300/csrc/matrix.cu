// bbl_matrix: device copy of H in CSR and optionally SELL-C-sigma, with
// structure validation, ||H||_inf and diag(H) computed at creation.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace bbl {
namespace {

// Copies `bytes` from host or device memory to device memory on `st`.
// Large pageable host copies go through two pinned staging buffers.
bbl_status copy_to_device(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    if (bytes == 0) return BBL_OK;
    if (is_device_pointer(src) || bytes <= (8u << 20)) {
        BBL_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
        return BBL_OK;
    }
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, src) == cudaSuccess && at.type == cudaMemoryTypeHost) {
        BBL_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));  // already pinned
        return BBL_OK;
    }
    (void)cudaGetLastError();
    const size_t chunk = 64u << 20;
    HostBuf stage[2];
    BBL_TRY(stage[0].alloc(chunk));
    BBL_TRY(stage[1].alloc(chunk));
    cudaEvent_t ev[2];
    BBL_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    BBL_CUDA(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    bool used[2] = {false, false};
    size_t off = 0;
    int k = 0;
    bbl_status rc = BBL_OK;
    while (off < bytes) {
        const size_t len = std::min(chunk, bytes - off);
        if (used[k] && cudaEventSynchronize(ev[k]) != cudaSuccess) {
            rc = set_error(BBL_ERR_CUDA, "copy_to_device: event sync failed");
            break;
        }
        std::memcpy(stage[k].p, static_cast<const char*>(src) + off, len);
        if (cudaMemcpyAsync(static_cast<char*>(dst) + off, stage[k].p, len, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaEventRecord(ev[k], st) != cudaSuccess) {
            rc = set_error(BBL_ERR_CUDA, "copy_to_device: async copy failed");
            break;
        }
        used[k] = true;
        off += len;
        k ^= 1;
    }
    cudaStreamSynchronize(st);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    return rc;
}

__global__ void f64_to_f32_kernel(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}
__global__ void f32_to_f64_kernel(int64_t n, const float* __restrict__ in, double* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

// Flags: bit0 row_ptr not monotone / wrong ends, bit1 column out of range,
// bit2 columns not strictly increasing, bit3 non-finite value.
template <typename T>
__global__ void validate_kernel(int64_t n, int64_t nnz, const int64_t* __restrict__ rp, const int* __restrict__ ci,
                                const T* __restrict__ va, int* flags) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const int64_t s = rp[row], e = rp[row + 1];
    int f = 0;
    if (lane == 0 && (e < s || s < 0 || e > nnz || (row == 0 && s != 0) || (row == n - 1 && e != nnz))) f |= 1;
    if (!(f & 1)) {
        for (int64_t k = s + lane; k < e; k += 32) {
            const int c = ci[k];
            if (c < 0 || c >= n) f |= 2;
            if (k > s && ci[k - 1] >= c) f |= 4;
            const double v = (double)va[k];
            if (!isfinite(v)) f |= 8;
        }
    }
    if (f) atomicOr(flags, f);
}

// Exact symmetry check: for every stored (i, j, v) the entry (j, i) exists with value v.
template <typename T>
__global__ void symmetry_kernel(int64_t n, const int64_t* __restrict__ rp, const int* __restrict__ ci,
                                const T* __restrict__ va, int* flags) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    int bad = 0;
    for (int64_t k = rp[row] + lane; k < rp[row + 1]; k += 32) {
        const int j = ci[k];
        int64_t lo = rp[j], hi = rp[j + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (ci[mid] < row) lo = mid + 1; else hi = mid;
        }
        if (lo >= rp[j + 1] || ci[lo] != row || va[lo] != va[k]) bad = 1;
    }
    if (bad) atomicOr(flags, 16);
}

// diag(H) (FP64) and the per-row absolute sums, reduced to max via the
// order-preserving bit pattern of non-negative doubles.
template <typename T>
__global__ void diag_norm_kernel(int64_t n, const int64_t* __restrict__ rp, const int* __restrict__ ci,
                                 const T* __restrict__ va, double* __restrict__ diag,
                                 unsigned long long* __restrict__ norm_bits) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double s = 0.0, d = 0.0;
    for (int64_t k = rp[row] + lane; k < rp[row + 1]; k += 32) {
        const double v = (double)va[k];
        s += fabs(v);
        if (ci[k] == row) d = v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, off);
        d += __shfl_xor_sync(0xffffffffu, d, off);
    }
    if (lane == 0) {
        diag[row] = d;
        atomicMax(norm_bits, (unsigned long long)__double_as_longlong(s));
    }
}

// SELL-C-sigma: sort the rows of each sigma-window by decreasing length
// (stable: equal lengths keep index order), one block per window.
__global__ void sell_sort_kernel(int64_t n, int sigma, const int64_t* __restrict__ rp, int* __restrict__ perm,
                                 int* __restrict__ slen) {
    extern __shared__ unsigned long long keys[];  // (len << 32 | (sigma-1-local)) descending == len desc, idx asc
    const int64_t w0 = (int64_t)blockIdx.x * sigma;
    int P = 1;
    while (P < sigma) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int64_t r = w0 + i;
        unsigned long long key = 0;  // padding sorts last
        if (i < sigma && r < n) {
            const unsigned long long len = (unsigned long long)(rp[r + 1] - rp[r]);
            key = ((len + 1ull) << 32) | (unsigned long long)(0xffffffffu - (unsigned)i);
        }
        keys[i] = key;
    }
    __syncthreads();
    // bitonic sort, descending
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool desc = ((i & k) == 0);
                    const unsigned long long a = keys[i], b = keys[ixj];
                    if (desc ? (a < b) : (a > b)) {
                        keys[i] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < sigma; i += blockDim.x) {
        const int64_t slot = w0 + i;
        const unsigned long long key = keys[i];
        if (key == 0) {
            perm[slot] = -1;
            slen[slot] = 0;
        } else {
            const int local = (int)(0xffffffffu - (unsigned)(key & 0xffffffffull));
            perm[slot] = (int)(w0 + local);
            slen[slot] = (int)((key >> 32) - 1ull);
        }
    }
}

__global__ void sell_width_kernel(int64_t nslices, const int* __restrict__ slen, int64_t* __restrict__ width) {
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (s >= nslices) return;
    int w = slen[s * 32 + lane];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, off));
    if (lane == 0) width[s] = w;
}

template <typename T>
__global__ void sell_fill_kernel(int64_t nslices, const int64_t* __restrict__ rp, const int* __restrict__ ci,
                                 const T* __restrict__ va, const int64_t* __restrict__ sp, const int* __restrict__ perm,
                                 const int* __restrict__ slen, int* __restrict__ sc, T* __restrict__ sv) {
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (s >= nslices) return;
    const int64_t slot = s * 32 + lane;
    const int row = perm[slot];
    const int len = slen[slot];
    const int width = (int)((sp[s + 1] - sp[s]) / 32);
    const int64_t src = row >= 0 ? rp[row] : 0;
    const int pad_col = row >= 0 ? row : 0;
    for (int k = 0; k < width; ++k) {
        const int64_t dst = sp[s] + (int64_t)k * 32 + lane;
        if (k < len) {
            sc[dst] = ci[src + k];
            sv[dst] = va[src + k];
        } else {
            sc[dst] = pad_col;
            sv[dst] = T(0);
        }
    }
}

template <typename T>
bbl_status sell_build(bbl_matrix* A, const T* val, cudaStream_t st) {
    const int sigma = A->sell_sigma;
    A->nslices = ceil_div(A->n, kSellC);
    const int64_t slots = A->nslices * kSellC;
    const int64_t nwin = ceil_div(slots, sigma);
    BBL_TRY(A->perm.alloc(sizeof(int) * nwin * sigma));
    BBL_TRY(A->sell_len.alloc(sizeof(int) * nwin * sigma));
    int P = 1;
    while (P < sigma) P <<= 1;
    sell_sort_kernel<<<(unsigned)nwin, 256, sizeof(unsigned long long) * P, st>>>(
        A->n, sigma, A->row_ptr.as<int64_t>(), A->perm.as<int>(), A->sell_len.as<int>());
    BBL_LAUNCH_CHECK();
    DevBuf width;
    BBL_TRY(width.alloc(sizeof(int64_t) * A->nslices));
    sell_width_kernel<<<(unsigned)ceil_div(A->nslices * 32, 256), 256, 0, st>>>(A->nslices, A->sell_len.as<int>(),
                                                                                width.as<int64_t>());
    BBL_LAUNCH_CHECK();
    std::vector<int64_t> w(A->nslices), sp(A->nslices + 1);
    BBL_CUDA(cudaMemcpyAsync(w.data(), width.p, sizeof(int64_t) * A->nslices, cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    sp[0] = 0;
    for (int64_t s = 0; s < A->nslices; ++s) sp[s + 1] = sp[s] + w[s] * kSellC;
    A->padded_nnz = sp[A->nslices];
    BBL_TRY(A->slice_ptr.alloc(sizeof(int64_t) * (A->nslices + 1)));
    BBL_CUDA(cudaMemcpyAsync(A->slice_ptr.p, sp.data(), sizeof(int64_t) * (A->nslices + 1), cudaMemcpyHostToDevice, st));
    BBL_TRY(A->sell_col.alloc(sizeof(int) * A->padded_nnz));
    BBL_TRY(A->sell_val.alloc(sizeof(T) * A->padded_nnz));
    sell_fill_kernel<T><<<(unsigned)ceil_div(A->nslices * 32, 256), 256, 0, st>>>(
        A->nslices, A->row_ptr.as<int64_t>(), A->col.as<int>(), val, A->slice_ptr.as<int64_t>(), A->perm.as<int>(),
        A->sell_len.as<int>(), A->sell_col.as<int>(), A->sell_val.as<T>());
    BBL_LAUNCH_CHECK();
    BBL_CUDA(cudaStreamSynchronize(st));
    return BBL_OK;
}

template <typename T>
bbl_status analyse(bbl_matrix* A, const T* val, int check_symmetry, cudaStream_t st) {
    DevBuf flags;
    BBL_TRY(flags.alloc(sizeof(int) * 2 + sizeof(unsigned long long)));
    BBL_CUDA(cudaMemsetAsync(flags.p, 0, flags.bytes, st));
    int* d_flags = flags.as<int>();
    unsigned long long* d_norm = reinterpret_cast<unsigned long long*>(flags.as<char>() + 8);
    const unsigned blocks = (unsigned)ceil_div(A->n * 32, 256);
    validate_kernel<T><<<blocks, 256, 0, st>>>(A->n, A->nnz, A->row_ptr.as<int64_t>(), A->col.as<int>(), val, d_flags);
    BBL_LAUNCH_CHECK();
    int h_flags = 0;
    BBL_CUDA(cudaMemcpyAsync(&h_flags, d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    if (h_flags)
        return set_error(BBL_ERR_INVALID_ARG,
                         "matrix_create: invalid CSR (flags 0x%x: 1=row_ptr, 2=column range, 4=unsorted/duplicate "
                         "columns, 8=non-finite value)",
                         h_flags);
    if (check_symmetry) {
        symmetry_kernel<T><<<blocks, 256, 0, st>>>(A->n, A->row_ptr.as<int64_t>(), A->col.as<int>(), val, d_flags);
        BBL_LAUNCH_CHECK();
        BBL_CUDA(cudaMemcpyAsync(&h_flags, d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
        BBL_CUDA(cudaStreamSynchronize(st));
        if (h_flags) return set_error(BBL_ERR_NOT_SYMMETRIC, "matrix_create: H is not exactly symmetric");
    }
    BBL_TRY(A->diag.alloc(sizeof(double) * A->n));
    diag_norm_kernel<T><<<blocks, 256, 0, st>>>(A->n, A->row_ptr.as<int64_t>(), A->col.as<int>(), val,
                                                A->diag.as<double>(), d_norm);
    BBL_LAUNCH_CHECK();
    unsigned long long bits = 0;
    BBL_CUDA(cudaMemcpyAsync(&bits, d_norm, sizeof(bits), cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    double nrm;
    std::memcpy(&nrm, &bits, sizeof(nrm));
    A->norm_inf = nrm;
    return BBL_OK;
}

}  // namespace
}  // namespace bbl

extern "C" {

bbl_status bbl_matrix_create(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col, const void* val,
                             bbl_dtype val_dtype, bbl_dtype storage, bbl_format fmt, int sell_sigma, int keep_fp64,
                             int check_symmetry, void* stream, bbl_matrix** out) {
    using namespace bbl;
    if (!out) return set_error(BBL_ERR_INVALID_ARG, "matrix_create: out is NULL");
    *out = nullptr;
    if (n < 1 || n >= (int64_t(1) << 31)) return set_error(BBL_ERR_INVALID_ARG, "matrix_create: n=%lld", (long long)n);
    if (nnz < 0) return set_error(BBL_ERR_INVALID_ARG, "matrix_create: nnz < 0");
    if (!row_ptr || (nnz > 0 && (!col || !val)))
        return set_error(BBL_ERR_INVALID_ARG, "matrix_create: NULL array");
    if ((val_dtype != BBL_FP64 && val_dtype != BBL_FP32) || (storage != BBL_FP64 && storage != BBL_FP32))
        return set_error(BBL_ERR_INVALID_ARG, "matrix_create: bad dtype");
    if (fmt != BBL_CSR && fmt != BBL_SELL && fmt != BBL_TILED)
        return set_error(BBL_ERR_INVALID_ARG, "matrix_create: bad format");
    const int tile = fmt == BBL_TILED ? (sell_sigma > 0 ? sell_sigma : 1024) : 0;
    if (fmt == BBL_TILED && (tile < 16 || tile > 1024))
        return set_error(BBL_ERR_INVALID_ARG, "matrix_create: tile %d outside 16..1024", tile);
    if (fmt == BBL_TILED) sell_sigma = 0;
    if (sell_sigma == 0) sell_sigma = kSellC;
    if (fmt == BBL_SELL && (sell_sigma < kSellC || sell_sigma % kSellC || sell_sigma > 4096))
        return set_error(BBL_ERR_INVALID_ARG, "matrix_create: sell_sigma must be a multiple of 32 in 32..4096");
    cudaStream_t st = as_stream(stream);
    // host-side check of the row pointer ends (cheap, before any launch)
    int64_t rp0 = 0, rpn = 0;
    if (is_device_pointer(row_ptr)) {
        BBL_CUDA(cudaMemcpyAsync(&rp0, row_ptr, 8, cudaMemcpyDeviceToHost, st));
        BBL_CUDA(cudaMemcpyAsync(&rpn, row_ptr + n, 8, cudaMemcpyDeviceToHost, st));
        BBL_CUDA(cudaStreamSynchronize(st));
    } else {
        rp0 = row_ptr[0];
        rpn = row_ptr[n];
    }
    if (rp0 != 0 || rpn != nnz)
        return set_error(BBL_ERR_INVALID_ARG, "matrix_create: row_ptr[0]=%lld, row_ptr[n]=%lld, nnz=%lld",
                         (long long)rp0, (long long)rpn, (long long)nnz);

    bbl_matrix* A = new bbl_matrix();
    A->n = n;
    A->nnz = nnz;
    A->fmt = fmt;
    A->storage = storage;
    A->sell_sigma = sell_sigma;
    auto fail = [&](bbl_status s) {
        delete A;
        return s;
    };
    bbl_status s;
    if ((s = A->row_ptr.alloc(sizeof(int64_t) * (n + 1))) != BBL_OK) return fail(s);
    if ((s = A->col.alloc(sizeof(int) * nnz)) != BBL_OK) return fail(s);
    if ((s = A->val.alloc(dtype_size(storage) * nnz)) != BBL_OK) return fail(s);
    if ((s = copy_to_device(A->row_ptr.p, row_ptr, sizeof(int64_t) * (n + 1), st)) != BBL_OK) return fail(s);
    if ((s = copy_to_device(A->col.p, col, sizeof(int) * nnz, st)) != BBL_OK) return fail(s);
    const unsigned cgrid = 152 * 8;
    if (val_dtype == storage) {
        if ((s = copy_to_device(A->val.p, val, dtype_size(storage) * nnz, st)) != BBL_OK) return fail(s);
    } else {
        DevBuf tmp;
        if ((s = tmp.alloc(dtype_size(val_dtype) * nnz)) != BBL_OK) return fail(s);
        if ((s = copy_to_device(tmp.p, val, dtype_size(val_dtype) * nnz, st)) != BBL_OK) return fail(s);
        if (val_dtype == BBL_FP64)
            f64_to_f32_kernel<<<cgrid, 256, 0, st>>>(nnz, tmp.as<double>(), A->val.as<float>());
        else
            f32_to_f64_kernel<<<cgrid, 256, 0, st>>>(nnz, tmp.as<float>(), A->val.as<double>());
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
            return fail(set_error(BBL_ERR_CUDA, "matrix_create: value conversion failed"));
    }
    A->has_csr = true;
    if (storage == BBL_FP64) s = analyse<double>(A, A->val.as<double>(), check_symmetry, st);
    else s = analyse<float>(A, A->val.as<float>(), check_symmetry, st);
    if (s != BBL_OK) return fail(s);
    if (storage == BBL_FP32 && keep_fp64) {
        if ((s = A->val64.alloc(sizeof(double) * nnz)) != BBL_OK) return fail(s);
        if (val_dtype == BBL_FP64) {
            if ((s = copy_to_device(A->val64.p, val, sizeof(double) * nnz, st)) != BBL_OK) return fail(s);
        } else {
            f32_to_f64_kernel<<<cgrid, 256, 0, st>>>(nnz, A->val.as<float>(), A->val64.as<double>());
            if (cudaGetLastError() != cudaSuccess) return fail(set_error(BBL_ERR_CUDA, "matrix_create: widen failed"));
        }
    }
    if (fmt == BBL_SELL) {
        if (storage == BBL_FP64) s = sell_build<double>(A, A->val.as<double>(), st);
        else s = sell_build<float>(A, A->val.as<float>(), st);
        if (s != BBL_OK) return fail(s);
    }
    if (fmt == BBL_TILED && (s = tiled_build(A, tile, st)) != BBL_OK) return fail(s);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(set_error(BBL_ERR_CUDA, "matrix_create: sync failed"));
    *out = A;
    return BBL_OK;
}

void bbl_matrix_destroy(bbl_matrix* A) {
    if (A) {
        cudaDeviceSynchronize();
        delete A;
    }
}

bbl_status bbl_matrix_info(const bbl_matrix* A, int64_t* n, int64_t* nnz, double* norm_inf, int64_t* device_bytes,
                           int* fmt, int* storage, int64_t* padded_nnz) {
    if (!A) return bbl::set_error(BBL_ERR_INVALID_ARG, "matrix_info: NULL matrix");
    if (n) *n = A->n;
    if (nnz) *nnz = A->nnz;
    if (norm_inf) *norm_inf = A->norm_inf;
    if (device_bytes) *device_bytes = A->device_bytes();
    if (fmt) *fmt = A->fmt;
    if (storage) *storage = A->storage;
    if (padded_nnz) *padded_nnz = A->fmt == BBL_SELL ? A->padded_nnz : A->nnz;
    return BBL_OK;
}

// diag(H) into a caller device buffer (FP64 [n]).
bbl_status bbl_matrix_set_spmm_lanes(bbl_matrix* A, int lanes_per_row) {
    if (!A || lanes_per_row < 0 || lanes_per_row > 32 || (lanes_per_row & (lanes_per_row - 1)))
        return bbl::set_error(BBL_ERR_INVALID_ARG, "matrix_set_spmm_lanes: 0 or a power of two <= 32");
    A->spmm_lanes = lanes_per_row;
    return BBL_OK;
}

bbl_status bbl_matrix_diagonal(const bbl_matrix* A, double* d, void* stream) {
    if (!A || !d) return bbl::set_error(BBL_ERR_INVALID_ARG, "matrix_diagonal: NULL argument");
    BBL_CUDA(cudaMemcpyAsync(d, A->diag.p, sizeof(double) * A->n, cudaMemcpyDefault, bbl::as_stream(stream)));
    return BBL_OK;
}

}  // extern "C"
