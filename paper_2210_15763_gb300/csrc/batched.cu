// Batched form: many independent, uneven-size block Lanczos solves advanced
// in lock-step by ONE graph launch.
//
// The problems are stacked row-wise into one block-diagonal matrix (segment
// s = rows [off[s], off[s+1])).  One block iteration is a fixed sequence of
// kernels over all segments at once (the block-diagonal SpMM, segmented
// Gram-Schmidt, segmented CholQR2, batched Ritz solves, per-segment
// convergence test); the iteration index and basis size live in device
// memory, so the sequence is captured once into the body of a CUDA graph
// "while" node whose condition a control kernel sets from the number of
// segments still running.  The whole batched solve is then a single
// cudaGraphLaunch: no host round trip per iteration.  Segments that converge
// are switched off (their Gram-Schmidt, CholQR2 and Ritz work is skipped);
// each segment runs its Ritz solve and test only on the blocks its own
// adaptive schedule picks.
//
// Storage: FP32 or FP64 blocks as the matrix; coefficients, Gram matrices,
// T and the final residuals in FP64 (no polish stage: each segment stops at
// its estimate ||B_j s_i[last b]|| <= tol * ||H_s||_inf).
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "common.cuh"

namespace bbl {
bbl_status gram_seg(int64_t n, int b, int m_max, const int* d_m, int dtype, const void* Q, const void* W,
                    const int64_t* chunks, int nchunks, const int* seg_chunk_ptr, int nseg, const int* active,
                    double* partial, double* C, cudaStream_t st);
bbl_status apply_seg(int64_t n, int b, int kc, const int* ms, int ms_stride, int dtype, const void* Q, const double* C,
                     int64_t cstride, void* W, bool sub, bool f64_out, const int64_t* ctas, int nctas, const int* active,
                     cudaStream_t st);
bbl_status chol_seg(int b, int nseg, const double* G, const double* thresh2, int relative, double* R, double* Rinv,
                    int* ndefl, int* mask, int* status, const int* active, cudaStream_t st);
bbl_status trmul_seg(int b, int nseg, const double* R2, const double* R1, double* B, const int* active, cudaStream_t st);
size_t ritz_seg_workspace_doubles(int m_max, int p, int nev);
int gram_seg_chunk_rows(int b, int dtype);
bbl_status ritz_dev_batched(int m_max, int p, int nev, int nseg, const double* Tb, int64_t sT, double* theta,
                            int64_t sTh, double* width, double* S, int64_t sS, double* ws, double* tmp, const int* d_m,
                            const int* active, cudaStream_t st);
bbl_status fill_normal(int64_t n, int b, uint64_t seed, uint64_t offset, double* P, cudaStream_t st);
}  // namespace bbl

struct bbl_batch {
    int nseg = 0;
    int64_t n_tot = 0;
    bbl_matrix* A = nullptr;
    std::vector<int64_t> off;
    bbl::DevBuf d_off, d_norm;   // int64 [nseg+1], FP64 [nseg]
    std::vector<double> norm;
    int spmm_lanes = 0;          // CSR lanes per row chosen by the autotuner (0 = built-in rule)
    ~bbl_batch() { bbl_matrix_destroy(A); }
};

namespace bbl {
namespace {

// per-segment ||H_s||_inf: row |.| sums, max per segment (non-negative doubles order as their bits)
template <typename T>
__global__ void seg_norm_kernel(int64_t n, int nseg, const int64_t* __restrict__ off, const int64_t* __restrict__ rp,
                                const int* __restrict__ ci, const T* __restrict__ va, unsigned long long* __restrict__ out,
                                int* __restrict__ bad) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    int lo = 0, hi = nseg;  // segment: off[s] <= row < off[s+1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (off[mid] <= row) lo = mid; else hi = mid;
    }
    double s = 0.0;
    int outside = 0;
    for (int64_t k = rp[row] + lane; k < rp[row + 1]; k += 32) {
        s += fabs((double)va[k]);
        const int c = ci[k];
        if (c < off[lo] || c >= off[lo + 1]) outside = 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        outside |= __shfl_xor_sync(0xffffffffu, outside, o);
    }
    if (lane == 0) {
        atomicMax(out + lo, (unsigned long long)__double_as_longlong(s));
        if (outside) atomicOr(bad, 1);
    }
}

template <typename TI, typename TO>
__global__ void convert_kernel(int64_t count, const TI* __restrict__ in, TO* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (TO)in[e];
}

// copy block src (n x b) into basis slot (*d_j + shift) and/or a fixed buffer
template <typename T>
__global__ void copy_slot_kernel(int64_t count, const int* __restrict__ d_j, int shift, const T* __restrict__ src,
                                 T* __restrict__ basis, T* __restrict__ fixed) {
    const int64_t slot = (int64_t)(*d_j + shift);
    T* dst = basis + slot * count;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        const T v = src[e];
        dst[e] = v;
        if (fixed) fixed[e] = v;
    }
}

// A_j = sym(C1[s][j-block]) and B_j into segment s's band (rows_alloc rows, b+1 columns)
__global__ void fill_AB_seg_kernel(int b, int m_max, int rows_alloc, const int* __restrict__ d_j,
                                   const int* __restrict__ active, const double* __restrict__ C1,
                                   const double* __restrict__ Bj, double* __restrict__ Tb, int which) {
    const int s = blockIdx.x;
    if (active && !active[s]) return;
    const int j = *d_j;
    const int e = threadIdx.x;
    if (e >= b * b) return;
    const int r = e / b, c = e % b;
    double* T = Tb + (int64_t)s * rows_alloc * (b + 1);
    if (which == 0) {
        if (c > r) return;
        const double* C = C1 + (int64_t)s * m_max * b;
        const int jb = j * b;
        T[(int64_t)(jb + r) * (b + 1) + (r - c)] = 0.5 * (C[(int64_t)(jb + r) * b + c] + C[(int64_t)(jb + c) * b + r]);
    } else {
        if (c < r) return;
        const int row = (j + 1) * b + r;
        if (row < rows_alloc) T[(int64_t)row * (b + 1) + (b + r - c)] = Bj[(int64_t)s * b * b + r * b + c];
    }
}

// which segments test convergence at block j: with every > 0 each every-th
// block, else (adaptive) from block next_chk[s] on; always on a breakdown
// and at the last block
__global__ void due_seg_kernel(int nseg, int J_max, int every, const int* __restrict__ d_j,
                               const int* __restrict__ active, const int* __restrict__ ndefl,
                               const int* __restrict__ next_chk, int* __restrict__ due) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const int j = *d_j;
    const bool sched = every > 0 ? ((j + 1) % every == 0) : (j >= next_chk[s]);
    due[s] = (active[s] && (sched || ndefl[s] > 0 || j + 1 >= J_max)) ? 1 : 0;
}

// per due segment: estimates, convergence / deflation decisions, and the
// next test block: rho = max_i est_i / (tol ||H_s||) and its decay per block
// since the previous test predict the blocks left; the next test is at half
// that distance, 1 to 8 blocks ahead (one block until two tests exist)
__global__ void converge_seg_kernel(int b, int nev, int nseg, int m_max, int rows_alloc, int J_max,
                                    const int* __restrict__ d_j, const double* __restrict__ Tb,
                                    const double* __restrict__ S, const double* __restrict__ norm, double tol,
                                    const int* __restrict__ ndefl, const int* __restrict__ due,
                                    int* __restrict__ active, int* __restrict__ final_j, int* __restrict__ status,
                                    double* __restrict__ est_out, int* __restrict__ next_chk, int* __restrict__ jprev,
                                    double* __restrict__ lprev) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg || !due[s]) return;
    const int j = *d_j;
    const int m = (j + 1) * b;
    const int k = min(nev, m);
    const double* T = Tb + (int64_t)s * rows_alloc * (b + 1);
    const double* Ss = S + (int64_t)s * m_max * nev;
    bool done = (k == nev);
    double rho = 0.0;
    for (int i = 0; i < k; ++i) {
        double s2 = 0.0;
        for (int r = 0; r < b; ++r) {
            double t = 0.0;
            for (int c = r; c < b; ++c) t += T[(int64_t)(m + r) * (b + 1) + (b + r - c)] * Ss[(int64_t)(m - b + c) * nev + i];
            s2 += t * t;
        }
        const double e = sqrt(s2);
        est_out[(int64_t)s * nev + i] = e;
        done = done && (e <= tol * norm[s]);
        rho = fmax(rho, e / (tol * norm[s]));
    }
    final_j[s] = j;
    if (done) {
        active[s] = 0;
        status[s] = BBL_OK;
    } else if (ndefl[s] > 0) {
        active[s] = 0;  // breakdown: keep the pairs of this block (a smaller invariant space)
        status[s] = BBL_ERR_NUMERICAL;
    } else if (j + 1 >= J_max) {
        status[s] = BBL_ERR_NOT_CONVERGED;
    }
    const double l = log(fmax(rho, 1e-300));
    int step = 1;
    if (jprev[s] >= 0 && j > jprev[s] && l < lprev[s] && l > 0.0) {
        const double blocks = l / ((lprev[s] - l) / (double)(j - jprev[s]));
        step = (int)fmin(8.0, fmax(1.0, floor(0.5 * blocks)));
    }
    jprev[s] = j;
    lprev[s] = l;
    next_chk[s] = j + step;
}

// advances the iteration and sets the while-node condition
__global__ void control_kernel(int nseg, int b, int J_max, int* __restrict__ d_j, int* __restrict__ d_m,
                               int* __restrict__ active, cudaGraphConditionalHandle handle, int in_graph,
                               int* __restrict__ iters) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int live = 0;
    for (int s = 0; s < nseg; ++s) live += active[s];
    const int j = *d_j;
    *iters = j + 1;
    if (live > 0 && j + 1 < J_max) {
        *d_j = j + 1;
        *d_m = (j + 2) * b;
        if (in_graph) cudaGraphSetConditional(handle, 1);
    } else {
        for (int s = 0; s < nseg; ++s) active[s] = 0;
        if (in_graph) cudaGraphSetConditional(handle, 0);
    }
}

// per-CTA partial sums of (Y - X diag(theta_s))^2 per column for one segment's rows
__global__ void resid_seg_kernel(int k, const int64_t* __restrict__ ctas, const double* __restrict__ Y,
                                 const double* __restrict__ X, const double* __restrict__ theta, int ldth,
                                 double* __restrict__ partial) {
    __shared__ double red[256];
    const int64_t s = ctas[3 * blockIdx.x];
    const int64_t r = ctas[3 * blockIdx.x + 1] + threadIdx.x;
    const bool in = r < ctas[3 * blockIdx.x + 2];
    for (int i = 0; i < k; ++i) {
        double d = 0.0;
        if (in) d = Y[r * k + i] - theta[s * ldth + i] * X[r * k + i];
        red[threadIdx.x] = d * d;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * k + i] = red[0];
        __syncthreads();
    }
}

}  // namespace
}  // namespace bbl

extern "C" {

bbl_status bbl_batch_create(int count, const int64_t* offsets, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                            const void* val, bbl_dtype val_dtype, bbl_dtype storage, bbl_format fmt, int sell_sigma,
                            void* stream, bbl_batch** out) {
    using namespace bbl;
    if (!out || count < 1 || !offsets) return set_error(BBL_ERR_INVALID_ARG, "batch_create: bad arguments");
    *out = nullptr;
    for (int s = 0; s < count; ++s)
        if (offsets[s + 1] <= offsets[s]) return set_error(BBL_ERR_INVALID_ARG, "batch_create: empty or unsorted segment %d", s);
    if (offsets[0] != 0) return set_error(BBL_ERR_INVALID_ARG, "batch_create: offsets[0] must be 0");
    cudaStream_t st = as_stream(stream);
    bbl_batch* Bt = new bbl_batch();
    Bt->nseg = count;
    Bt->n_tot = offsets[count];
    Bt->off.assign(offsets, offsets + count + 1);
    bbl_status s = bbl_matrix_create(Bt->n_tot, nnz, row_ptr, col, val, val_dtype, storage, fmt, sell_sigma, 0, 0,
                                     stream, &Bt->A);
    if (s != BBL_OK) {
        delete Bt;
        return s;
    }
    if ((s = Bt->d_off.alloc(sizeof(int64_t) * (count + 1))) != BBL_OK ||
        (s = Bt->d_norm.alloc(sizeof(double) * count + sizeof(int))) != BBL_OK) {
        delete Bt;
        return s;
    }
    cudaMemcpyAsync(Bt->d_off.p, offsets, sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(Bt->d_norm.p, 0, Bt->d_norm.bytes, st);
    int* bad = reinterpret_cast<int*>(Bt->d_norm.as<double>() + count);
    const unsigned blocks = (unsigned)ceil_div(Bt->n_tot * 32, 256);
    auto nb = reinterpret_cast<unsigned long long*>(Bt->d_norm.p);
    if (storage == BBL_FP64)
        seg_norm_kernel<double><<<blocks, 256, 0, st>>>(Bt->n_tot, count, Bt->d_off.as<int64_t>(), Bt->A->row_ptr.as<int64_t>(),
                                                        Bt->A->col.as<int>(), Bt->A->val.as<double>(), nb, bad);
    else
        seg_norm_kernel<float><<<blocks, 256, 0, st>>>(Bt->n_tot, count, Bt->d_off.as<int64_t>(), Bt->A->row_ptr.as<int64_t>(),
                                                       Bt->A->col.as<int>(), Bt->A->val.as<float>(), nb, bad);
    count_launch();
    std::vector<double> nrm(count);
    int hbad = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(nrm.data(), Bt->d_norm.p, sizeof(double) * count, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        delete Bt;
        return set_error(BBL_ERR_CUDA, "batch_create: segment norms failed");
    }
    if (hbad) {
        delete Bt;
        return set_error(BBL_ERR_INVALID_ARG, "batch_create: an entry couples two segments (not block diagonal)");
    }
    Bt->norm = nrm;
    BBL_CUDA(cudaMemcpyAsync(Bt->d_norm.p, nrm.data(), sizeof(double) * count, cudaMemcpyHostToDevice, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    *out = Bt;
    return BBL_OK;
}

void bbl_batch_destroy(bbl_batch* Bt) {
    if (Bt) {
        cudaDeviceSynchronize();
        delete Bt;
    }
}

bbl_status bbl_batch_matrix(bbl_batch* Bt, bbl_matrix** A) {
    if (!Bt || !A) return bbl::set_error(BBL_ERR_INVALID_ARG, "batch_matrix: NULL argument");
    *A = Bt->A;
    return BBL_OK;
}

bbl_status bbl_batch_set_schedule(bbl_batch* Bt, int lanes_per_row) {
    if (!Bt || lanes_per_row < 0 || lanes_per_row > 32 || (lanes_per_row & (lanes_per_row - 1)))
        return bbl::set_error(BBL_ERR_INVALID_ARG, "batch_set_schedule: lanes_per_row must be 0 or a power of two <= 32");
    Bt->spmm_lanes = lanes_per_row;
    return BBL_OK;
}

}  // extern "C"

namespace bbl {
namespace {

struct BatchStageOut {
    std::vector<int> fin, status;         // per segment: last block, status
    std::vector<double> theta, resid;     // nseg x nev
    float t_loop = 0.f;
    int launches = 0;                     // kernels in one captured iteration
};

// One lock-step block Lanczos run over the segments flagged in init_active
// (all when NULL).  dtype: block storage (the matrix's, or FP64 for the
// polish with FP64 arithmetic on FP32 values, f64_spmm); pivot: device FP64
// n x b, or NULL for the random pivot.  X: device FP64 n x nev, the Ritz
// vectors of the segments that ran; out: their Ritz values, true FP64
// residuals, last block and status.
bbl_status batch_stage(bbl_batch* Bt, int nev, int b, const bbl_options& o, int use_graph, int dtype, bool f64_spmm,
                       const double* pivot, const int* init_active, double* X_out, BatchStageOut& bout) {
    const int nseg = Bt->nseg;
    const int64_t n = Bt->n_tot;
    const size_t sz = dtype_size(dtype);
    int64_t nmin = Bt->off[1] - Bt->off[0];
    for (int s = 1; s < nseg; ++s) nmin = std::min(nmin, Bt->off[s + 1] - Bt->off[s]);
    int J_max = std::max(1, o.max_vectors / b);
    J_max = (int)std::min<int64_t>(J_max, nmin / b);  // no segment may exhaust its space
    if (J_max < 1 || (int64_t)nev > nmin) return set_error(BBL_ERR_INVALID_ARG, "batch_solve: a segment is smaller than nev/b");
    const int m_max = J_max * b;
    const int rows_alloc = m_max + b;
    cudaStream_t st = as_stream(o.stream);
    cudaStream_t cap = nullptr;
    if (!st) {
        BBL_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        st = cap;
    }
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() {
            if (s) cudaStreamDestroy(s);
        }
    } sg{cap};
    // ---- work tables (host) ----
    // Gram chunks: the row-contiguous kernel's tile (R rows) where it exists
    const int rows_tile = gram_seg_chunk_rows(b, dtype);
    const int64_t rpc = rows_tile > 0 ? (int64_t)rows_tile : std::max<int64_t>(256, ((n / 600) + 63) / 64 * 64);
    std::vector<int64_t> chunks, ctas;
    std::vector<int> chunk_ptr(nseg + 1, 0);
    for (int s = 0; s < nseg; ++s) {
        chunk_ptr[s] = (int)(chunks.size() / 3);
        for (int64_t r = Bt->off[s]; r < Bt->off[s + 1]; r += rpc) {
            chunks.push_back(s);
            chunks.push_back(r);
            chunks.push_back(std::min(r + rpc, Bt->off[s + 1]));
        }
        for (int64_t r = Bt->off[s]; r < Bt->off[s + 1]; r += 256) {
            ctas.push_back(s);
            ctas.push_back(r);
            ctas.push_back(std::min<int64_t>(r + 256, Bt->off[s + 1]));
        }
    }
    chunk_ptr[nseg] = (int)(chunks.size() / 3);
    const int nchunks = (int)(chunks.size() / 3), nctas = (int)(ctas.size() / 3);
    // ---- device buffers ----
    PoolBuf basis;
    DevBuf d_chunks, d_ctas, d_chunk_ptr, Vfix, Wfix, C1, C2, G, R1, R1i, R2, R2i, Bj, partial, Tb, theta, width,
        S, est, ws, tmp, ints, thr, X, Y, rpart, piv, lprev;
    BBL_TRY(d_chunks.alloc(sizeof(int64_t) * chunks.size()));
    BBL_TRY(d_ctas.alloc(sizeof(int64_t) * ctas.size()));
    BBL_TRY(d_chunk_ptr.alloc(sizeof(int) * (nseg + 1)));
    BBL_TRY(basis.alloc((size_t)(J_max + 1) * n * b * sz, st));
    BBL_TRY(Vfix.alloc((size_t)n * b * sz));
    BBL_TRY(Wfix.alloc((size_t)n * b * sz));
    BBL_TRY(C1.alloc(sizeof(double) * (size_t)nseg * m_max * b));
    BBL_TRY(C2.alloc(sizeof(double) * (size_t)nseg * m_max * b));
    const size_t bb = sizeof(double) * (size_t)nseg * b * b;
    BBL_TRY(G.alloc(bb));
    BBL_TRY(R1.alloc(bb));
    BBL_TRY(R1i.alloc(bb));
    BBL_TRY(R2.alloc(bb));
    BBL_TRY(R2i.alloc(bb));
    BBL_TRY(Bj.alloc(bb));
    // per chunk: up to 8 slots of m x b when m < 8b (row shares), else one
    BBL_TRY(partial.alloc(sizeof(double) * (size_t)nchunks * std::max(m_max, 8 * b) * b));
    BBL_TRY(Tb.alloc(sizeof(double) * (size_t)nseg * rows_alloc * (b + 1)));
    BBL_TRY(theta.alloc(sizeof(double) * (size_t)nseg * nev));
    BBL_TRY(width.alloc(sizeof(double) * (size_t)nseg * nev));
    BBL_TRY(S.alloc(sizeof(double) * (size_t)nseg * m_max * nev));
    BBL_TRY(est.alloc(sizeof(double) * (size_t)nseg * nev));
    BBL_TRY(ws.alloc(sizeof(double) * (size_t)nseg * ritz_seg_workspace_doubles(m_max, b, nev)));
    BBL_TRY(tmp.alloc(sizeof(double) * (size_t)nseg * m_max * nev));
    // ints: d_j, d_m, d_b, iters, then per segment: active, final_j, status, ndefl, mask[b], ms, due, next_chk,
    // jprev
    BBL_TRY(ints.alloc(sizeof(int) * (8 + (size_t)nseg * (8 + b))));
    BBL_TRY(lprev.alloc(sizeof(double) * nseg));
    BBL_TRY(thr.alloc(sizeof(double) * nseg * 2));
    int* d_j = ints.as<int>();
    int* d_m = d_j + 1;
    int* d_b = d_j + 2;
    int* d_iters = d_j + 3;
    int* active = d_j + 8;
    int* final_j = active + nseg;
    int* seg_status = final_j + nseg;
    int* ndefl = seg_status + nseg;
    int* mask = ndefl + nseg;
    int* ms = mask + (size_t)nseg * b;
    int* due = ms + nseg;
    int* next_chk = due + nseg;
    int* jprev = next_chk + nseg;
    BBL_CUDA(cudaMemcpyAsync(d_chunks.p, chunks.data(), sizeof(int64_t) * chunks.size(), cudaMemcpyHostToDevice, st));
    BBL_CUDA(cudaMemcpyAsync(d_ctas.p, ctas.data(), sizeof(int64_t) * ctas.size(), cudaMemcpyHostToDevice, st));
    BBL_CUDA(cudaMemcpyAsync(d_chunk_ptr.p, chunk_ptr.data(), sizeof(int) * (nseg + 1), cudaMemcpyHostToDevice, st));
    BBL_CUDA(cudaMemsetAsync(Tb.p, 0, Tb.bytes, st));
    BBL_CUDA(cudaMemsetAsync(ints.p, 0, ints.bytes, st));
    {
        std::vector<int> h(8 + (size_t)nseg * (8 + b), 0);
        h[0] = 0;
        h[1] = b;
        h[2] = b;
        for (int s = 0; s < nseg; ++s) h[8 + s] = init_active ? (init_active[s] != 0) : 1;  // active
        for (int s = 0; s < nseg; ++s) h[8 + 2 * nseg + s] = BBL_ERR_NOT_CONVERGED;
        for (int s = 0; s < nseg; ++s) h[8 + (size_t)nseg * (7 + b) + s] = -1;  // jprev: no test yet
        BBL_CUDA(cudaMemcpyAsync(ints.p, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice, st));
        const double dt = o.defl_tol > 0 ? o.defl_tol : (dtype == BBL_FP64 ? 1e-10 : 1e-6);
        std::vector<double> th(2 * nseg);
        for (int s = 0; s < nseg; ++s) {
            th[s] = (dt * Bt->norm[s]) * (dt * Bt->norm[s]);  // deflation thresholds (pass 1)
            th[nseg + s] = 1e-6;                                // pass 2 (normalised columns)
        }
        BBL_CUDA(cudaMemcpyAsync(thr.p, th.data(), sizeof(double) * th.size(), cudaMemcpyHostToDevice, st));
    }
    // ---- pivot: given, or random N(0,1) per row (splitmix64); orthonormalised per segment ----
    BBL_TRY(piv.alloc(sizeof(double) * (size_t)n * b));
    if (pivot) BBL_CUDA(cudaMemcpyAsync(piv.p, pivot, sizeof(double) * (size_t)n * b, cudaMemcpyDeviceToDevice, st));
    else BBL_TRY(fill_normal(n, b, o.seed, 0, piv.as<double>(), st));
    char* bp = basis.as<char>();
    const unsigned cg = 152 * 8;
    if (dtype == BBL_FP64)
        BBL_CUDA(cudaMemcpyAsync(Vfix.p, piv.p, sizeof(double) * n * b, cudaMemcpyDeviceToDevice, st));
    else {
        convert_kernel<double, float><<<cg, 256, 0, st>>>(n * b, piv.as<double>(), Vfix.as<float>());
        BBL_LAUNCH_CHECK();
    }
    const int64_t* CH = d_chunks.as<int64_t>();
    const int64_t* CT = d_ctas.as<int64_t>();
    const int* CP = d_chunk_ptr.as<int>();
    auto cholqr2_seg = [&](void* Wb, bool with_B, const int* act, int* nd) -> bbl_status {
        // m = b for the self Gram: d_b holds b
        BBL_TRY(gram_seg(n, b, b, d_b, dtype, Wb, Wb, CH, nchunks, CP, nseg, act, partial.as<double>(), G.as<double>(),
                         st));
        BBL_TRY(chol_seg(b, nseg, G.as<double>(), thr.as<double>(), 0, R1.as<double>(), R1i.as<double>(), nd, mask,
                         nullptr, act, st));
        BBL_TRY(apply_seg(n, b, b, d_b, 0, dtype, Wb, R1i.as<double>(), (int64_t)b * b, Wb, false, false, CT, nctas, act,
                          st));
        BBL_TRY(gram_seg(n, b, b, d_b, dtype, Wb, Wb, CH, nchunks, CP, nseg, act, partial.as<double>(), G.as<double>(),
                         st));
        BBL_TRY(chol_seg(b, nseg, G.as<double>(), thr.as<double>() + nseg, 0, R2.as<double>(), R2i.as<double>(), nullptr,
                         nullptr, nullptr, act, st));
        BBL_TRY(apply_seg(n, b, b, d_b, 0, dtype, Wb, R2i.as<double>(), (int64_t)b * b, Wb, false, false, CT, nctas, act,
                          st));
        if (with_B) BBL_TRY(trmul_seg(b, nseg, R2.as<double>(), R1.as<double>(), Bj.as<double>(), act, st));
        return BBL_OK;
    };
    // orthonormalise the pivot (relative threshold), store as block 0
    {
        std::vector<double> th(nseg, 1e-20);
        DevBuf thr0;
        BBL_TRY(thr0.alloc(sizeof(double) * nseg));
        BBL_CUDA(cudaMemcpyAsync(thr0.p, th.data(), sizeof(double) * nseg, cudaMemcpyHostToDevice, st));
        BBL_TRY(gram_seg(n, b, b, d_b, dtype, Vfix.p, Vfix.p, CH, nchunks, CP, nseg, active, partial.as<double>(),
                         G.as<double>(), st));
        BBL_TRY(chol_seg(b, nseg, G.as<double>(), thr0.as<double>(), 1, R1.as<double>(), R1i.as<double>(), nullptr,
                         nullptr, nullptr, active, st));
        BBL_TRY(apply_seg(n, b, b, d_b, 0, dtype, Vfix.p, R1i.as<double>(), (int64_t)b * b, Vfix.p, false, false, CT,
                          nctas, active, st));
        BBL_TRY(gram_seg(n, b, b, d_b, dtype, Vfix.p, Vfix.p, CH, nchunks, CP, nseg, active, partial.as<double>(),
                         G.as<double>(), st));
        BBL_TRY(chol_seg(b, nseg, G.as<double>(), thr.as<double>() + nseg, 0, R2.as<double>(), R2i.as<double>(), nullptr,
                         nullptr, nullptr, active, st));
        BBL_TRY(apply_seg(n, b, b, d_b, 0, dtype, Vfix.p, R2i.as<double>(), (int64_t)b * b, Vfix.p, false, false, CT,
                          nctas, active, st));
        BBL_CUDA(cudaMemcpyAsync(bp, Vfix.p, (size_t)n * b * sz, cudaMemcpyDeviceToDevice, st));
        BBL_CUDA(cudaStreamSynchronize(st));
    }
    // ---- one block iteration (all segments), reading j and m from device memory ----
    cudaGraphConditionalHandle handle = 0;
    // a run over a subset of the problems (the polish) multiplies only their
    // rows: maximal runs of consecutive flagged segments
    std::vector<std::pair<int64_t, int64_t>> row_runs;
    if (init_active && f64_spmm && Bt->A->has_csr) {
        for (int s = 0; s < nseg; ++s) {
            if (!init_active[s]) continue;
            if (!row_runs.empty() && row_runs.back().second == Bt->off[s]) row_runs.back().second = Bt->off[s + 1];
            else row_runs.push_back({Bt->off[s], Bt->off[s + 1]});
        }
    }
    auto iteration = [&]() -> bbl_status {
        if (!row_runs.empty()) {
            for (const auto& rr : row_runs)
                BBL_TRY(spmm_rows_f64(Bt->A, b, Vfix.as<double>(), Wfix.as<double>(), rr.first, rr.second, st));
        } else {
            BBL_TRY(spmm_dispatch(Bt->A, b, Vfix.p, Wfix.p, f64_spmm, st, Bt->spmm_lanes));
        }
        BBL_TRY(gram_seg(n, b, m_max, d_m, dtype, basis.p, Wfix.p, CH, nchunks, CP, nseg, active, partial.as<double>(),
                         C1.as<double>(), st));
        BBL_TRY(apply_seg(n, b, b, d_m, 0, dtype, basis.p, C1.as<double>(), (int64_t)m_max * b, Wfix.p, true, false, CT,
                          nctas, active, st));
        fill_AB_seg_kernel<<<nseg, 256, 0, st>>>(b, m_max, rows_alloc, d_j, active, C1.as<double>(), Bj.as<double>(),
                                                  Tb.as<double>(), 0);
        BBL_LAUNCH_CHECK();
        BBL_TRY(gram_seg(n, b, m_max, d_m, dtype, basis.p, Wfix.p, CH, nchunks, CP, nseg, active, partial.as<double>(),
                         C2.as<double>(), st));
        BBL_TRY(apply_seg(n, b, b, d_m, 0, dtype, basis.p, C2.as<double>(), (int64_t)m_max * b, Wfix.p, true, false, CT,
                          nctas, active, st));
        BBL_TRY(cholqr2_seg(Wfix.p, true, active, ndefl));
        fill_AB_seg_kernel<<<nseg, 256, 0, st>>>(b, m_max, rows_alloc, d_j, active, C1.as<double>(), Bj.as<double>(),
                                                  Tb.as<double>(), 1);
        BBL_LAUNCH_CHECK();
        if (dtype == BBL_FP64)
            copy_slot_kernel<double><<<cg, 256, 0, st>>>(n * b, d_j, 1, Wfix.as<double>(), basis.as<double>(),
                                                         Vfix.as<double>());
        else
            copy_slot_kernel<float><<<cg, 256, 0, st>>>(n * b, d_j, 1, Wfix.as<float>(), basis.as<float>(),
                                                        Vfix.as<float>());
        BBL_LAUNCH_CHECK();
        due_seg_kernel<<<(unsigned)ceil_div(nseg, 256), 256, 0, st>>>(nseg, J_max, std::max(0, o.check_every), d_j,
                                                                       active, ndefl, next_chk, due);
        BBL_LAUNCH_CHECK();
        BBL_TRY(ritz_dev_batched(m_max, b, nev, nseg, Tb.as<double>(), (int64_t)rows_alloc * (b + 1), theta.as<double>(),
                                 nev, width.as<double>(), S.as<double>(), (int64_t)m_max * nev, ws.as<double>(),
                                 tmp.as<double>(), d_m, due, st));
        converge_seg_kernel<<<(unsigned)ceil_div(nseg, 64), 64, 0, st>>>(
            b, nev, nseg, m_max, rows_alloc, J_max, d_j, Tb.as<double>(), S.as<double>(), Bt->d_norm.as<double>(), o.tol,
            ndefl, due, active, final_j, seg_status, est.as<double>(), next_chk, jprev, lprev.as<double>());
        BBL_LAUNCH_CHECK();
        control_kernel<<<1, 32, 0, st>>>(nseg, b, J_max, d_j, d_m, active, handle, use_graph ? 1 : 0, d_iters);
        BBL_LAUNCH_CHECK();
        return BBL_OK;
    };
    cudaEvent_t e0, e1;
    BBL_CUDA(cudaEventCreate(&e0));
    BBL_CUDA(cudaEventCreate(&e1));
    BBL_CUDA(cudaEventRecord(e0, st));
    int launches_in_graph = 0;
    if (use_graph) {
        cudaGraph_t graph = nullptr;
        BBL_CUDA(cudaGraphCreate(&graph, 0));
        BBL_CUDA(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        BBL_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        BBL_CUDA(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        const uint64_t l0 = bbl_kernel_launches();
        bbl_status sc = iteration();
        launches_in_graph = (int)(bbl_kernel_launches() - l0);
        cudaGraph_t captured = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(st, &captured);
        if (sc != BBL_OK) {
            cudaGraphDestroy(graph);
            return sc;
        }
        if (ec != cudaSuccess) {
            cudaGraphDestroy(graph);
            return set_error(BBL_ERR_CUDA, "batch_solve: capture failed: %s", cudaGetErrorString(ec));
        }
        cudaGraphExec_t exec = nullptr;
        cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        if (ei != cudaSuccess) {
            cudaGraphDestroy(graph);
            return set_error(BBL_ERR_CUDA, "batch_solve: instantiate failed: %s", cudaGetErrorString(ei));
        }
        BBL_CUDA(cudaEventRecord(e0, st));
        BBL_CUDA(cudaGraphLaunch(exec, st));
        BBL_CUDA(cudaEventRecord(e1, st));
        BBL_CUDA(cudaStreamSynchronize(st));
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
    } else {
        // the same sequence driven from the host, one block at a time
        for (int it = 0; it < J_max; ++it) {
            BBL_TRY(iteration());
            int h[2];
            BBL_CUDA(cudaMemcpyAsync(h, d_j, sizeof(int), cudaMemcpyDeviceToHost, st));
            BBL_CUDA(cudaMemcpyAsync(h + 1, d_iters, sizeof(int), cudaMemcpyDeviceToHost, st));
            BBL_CUDA(cudaStreamSynchronize(st));
            if (h[0] != it + 1) break;  // the control kernel did not advance: done
        }
        BBL_CUDA(cudaEventRecord(e1, st));
        BBL_CUDA(cudaStreamSynchronize(st));
    }
    float t_loop = 0.f;
    cudaEventElapsedTime(&t_loop, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // ---- results: per-segment Ritz vectors X_s = Q_s S_s and FP64 residuals ----
    bout.fin.assign(nseg, 0);
    bout.status.assign(nseg, 0);
    BBL_CUDA(cudaMemcpyAsync(bout.fin.data(), final_j, sizeof(int) * nseg, cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaMemcpyAsync(bout.status.data(), seg_status, sizeof(int) * nseg, cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    std::vector<int> hms(nseg), ran(nseg, 1);
    for (int s = 0; s < nseg; ++s) {
        hms[s] = (bout.fin[s] + 1) * b;
        if (init_active) ran[s] = init_active[s] != 0;
    }
    BBL_CUDA(cudaMemcpyAsync(ms, hms.data(), sizeof(int) * nseg, cudaMemcpyHostToDevice, st));
    BBL_CUDA(cudaMemcpyAsync(active, ran.data(), sizeof(int) * nseg, cudaMemcpyHostToDevice, st));
    BBL_CUDA(cudaMemsetAsync(X_out, 0, sizeof(double) * (size_t)n * nev, st));
    BBL_TRY(Y.alloc(sizeof(double) * (size_t)n * nev));
    BBL_TRY(apply_seg(n, b, nev, ms, 1, dtype, basis.p, S.as<double>(), (int64_t)m_max * nev, X_out, false, true, CT,
                      nctas, active, st));
    BBL_TRY(spmm_dispatch(Bt->A, nev, X_out, Y.p, true, st, 0));
    BBL_TRY(rpart.alloc(sizeof(double) * (size_t)nctas * nev));
    resid_seg_kernel<<<nctas, 256, 0, st>>>(nev, CT, Y.as<double>(), X_out, theta.as<double>(), nev,
                                            rpart.as<double>());
    BBL_LAUNCH_CHECK();
    std::vector<double> hp((size_t)nctas * nev);
    bout.theta.assign((size_t)nseg * nev, 0.0);
    BBL_CUDA(cudaMemcpyAsync(hp.data(), rpart.p, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaMemcpyAsync(bout.theta.data(), theta.p, sizeof(double) * bout.theta.size(), cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    std::vector<double> r2((size_t)nseg * nev, 0.0);
    for (int c = 0; c < nctas; ++c) {
        const int sg = (int)ctas[3 * (size_t)c];
        for (int i = 0; i < nev; ++i) r2[(size_t)sg * nev + i] += hp[(size_t)c * nev + i];
    }
    bout.resid.assign((size_t)nseg * nev, 0.0);
    for (size_t e = 0; e < r2.size(); ++e) bout.resid[e] = std::sqrt(r2[e]);
    bout.t_loop = t_loop;
    bout.launches = launches_in_graph;
    return BBL_OK;
}

}  // namespace
}  // namespace bbl

extern "C" {

bbl_status bbl_batch_solve(bbl_batch* Bt, int nev, int b, const bbl_options* opt, int use_graph, double* evals,
                           double* resid, int* iters, int* status, bbl_stats* stats) {
    using namespace bbl;
    if (!Bt || !evals || b < 1 || b > kMaxB || nev < 1 || nev > kMaxB)
        return set_error(BBL_ERR_INVALID_ARG, "batch_solve: bad arguments");
    if (b != 1 && b != 2 && b != 4 && b != 8 && b != 16)
        return set_error(BBL_ERR_UNSUPPORTED, "batch_solve: b must be 1, 2, 4, 8 or 16");
    bbl_options o;
    if (opt) o = *opt;
    else bbl_options_default(&o);
    const int nseg = Bt->nseg;
    const int64_t n = Bt->n_tot;
    const int storage = Bt->A->storage;
    DevBuf X;
    BBL_TRY(X.alloc(sizeof(double) * (size_t)n * nev));
    BatchStageOut s1, s2;
    BBL_TRY(batch_stage(Bt, nev, b, o, use_graph, storage, false, nullptr, nullptr, X.as<double>(), s1));
    std::vector<int> polished(nseg, 0), piters(nseg, 0);
    const bool pow2 = nev == 1 || nev == 2 || nev == 4 || nev == 8 || nev == 16;
    if (storage == BBL_FP32 && o.polish && pow2) {
        // polish: the segments whose FP64 residuals miss tol go on from their
        // FP32 Ritz vectors (block size nev) with FP64 blocks and FP64
        // arithmetic on the FP32 values, in one more lock-step run
        int need = 0;
        for (int s = 0; s < nseg; ++s) {
            for (int i = 0; i < nev; ++i)
                if (!(s1.resid[(size_t)s * nev + i] <= o.tol * Bt->norm[s])) polished[s] = 1;
            need += polished[s];
        }
        if (need > 0) {
            DevBuf X2;
            BBL_TRY(X2.alloc(sizeof(double) * (size_t)n * nev));
            bbl_options o2 = o;
            o2.check_every = 0;
            BBL_TRY(batch_stage(Bt, nev, nev, o2, use_graph, BBL_FP64, true, X.as<double>(), polished.data(),
                                X2.as<double>(), s2));
            for (int s = 0; s < nseg; ++s) {
                if (!polished[s]) continue;
                for (int i = 0; i < nev; ++i) {
                    s1.theta[(size_t)s * nev + i] = s2.theta[(size_t)s * nev + i];
                    s1.resid[(size_t)s * nev + i] = s2.resid[(size_t)s * nev + i];
                }
                s1.status[s] = s2.status[s];
                piters[s] = s2.fin[s] + 1;
            }
        }
    }
    int nconv = 0, maxit = 0, maxp = 0;
    for (int s = 0; s < nseg; ++s) {
        bool ok = s1.status[s] == BBL_OK;
        for (int i = 0; i < nev; ++i) {
            evals[(size_t)s * nev + i] = s1.theta[(size_t)s * nev + i];
            if (resid) resid[(size_t)s * nev + i] = s1.resid[(size_t)s * nev + i];
            // a segment counts as converged when its true FP64 residuals meet tol
            ok = ok && s1.resid[(size_t)s * nev + i] <= o.tol * Bt->norm[s] * (1.0 + 1e-6);
        }
        if (!ok && s1.status[s] == BBL_OK) s1.status[s] = BBL_ERR_NOT_CONVERGED;
        if (iters) iters[s] = s1.fin[s] + 1 + piters[s];
        if (status) status[s] = s1.status[s];
        nconv += s1.status[s] == BBL_OK;
        maxit = std::max(maxit, s1.fin[s] + 1);
        maxp = std::max(maxp, piters[s]);
    }
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->iters = maxit;
        stats->vec_equiv_iters = maxit * b;
        stats->polish_iters = maxp;
        stats->converged = nconv;
        stats->t_total_ms = s1.t_loop + s2.t_loop;
        stats->graph_kernels = s1.launches;
    }
    return nconv == nseg ? BBL_OK : BBL_ERR_NOT_CONVERGED;
}

}  // extern "C"
