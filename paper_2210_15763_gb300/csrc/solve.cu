// bbl_solve: host orchestration of the block Lanczos iteration (Sec. II.B).
//
// Per block iteration j (all device work on the caller's stream, one small
// device->host read of the Ritz report per checked iteration):
//   S1  W = H V_j                                   (spmm.cu)
//   S2  C1 = Q^T W, W -= Q C1;  A_j = sym(C1[j]);    (block.cu; Q = [V_0..V_j])
//       C2 = Q^T W, W -= Q C2                       (second Gram-Schmidt pass)
//       (float-float blocks: C1 from FP32 copies of Q and W, A_j = sym(C1[j] + C2[j]))
//   S3  V_{j+1} R2 R1 = W (CholQR2), B_j = R2 R1     (block.cu)
//   S4  T_j (Eq. 12) -> theta, S; estimates ||B_j S[last b, i]||   (ritz.cu)
// then X = Q S and the FP64 residuals ||H x_i - theta_i x_i||.
//
// The first Gram-Schmidt pass subsumes the paper's subtraction of V_n A_n
// and V_{n-1} B_{n-1}^T (Eq. 8 with the Eq. 6 term): its coefficients for
// blocks j and j-1 are exactly those in exact arithmetic.
//
// Mixed precision (FP32 storage): stage 1 runs the same loop on FP32
// blocks with FP32 SpMM and FP64 coefficients / Gram / T / residual, to
// stage1_tol; stage 2 ("polish") restarts block Lanczos from the stage-1
// Ritz vectors -- the bootstrapping idea of Sec. II.B applied across
// precisions -- until the FP64 residuals meet tol.  The polish keeps its
// blocks as float-float pairs (about 48 bits, products on the FP32 pipes;
// df32.cuh) with FP64 coefficients, Gram and T, or in plain FP64 (polish = 2).
// The residuals that decide convergence are always FP64 SpMM products.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "df32.cuh"

namespace bbl {

size_t ritz_workspace_bytes(int m, int p, int nev);

namespace {

template <typename TI, typename TO>
__global__ void convert_kernel(int64_t count, const TI* __restrict__ in, TO* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (TO)in[e];
}

// A_j = sym(C1[j-block] + C2[j-block]) into the lower band of T: both
// Gram-Schmidt passes' own-block coefficients
__global__ void fill_A2_kernel(int j, int b, const double* __restrict__ C1, const double* __restrict__ C2,
                               double* __restrict__ Tb) {
    const int e = threadIdx.x;
    if (e >= b * b) return;
    const int r = e / b, c = e % b;
    if (c > r) return;
    const int jb = j * b;
    const int64_t rc = (int64_t)(jb + r) * b + c, cr = (int64_t)(jb + c) * b + r;
    const double v = 0.5 * ((C1[rc] + C2[rc]) + (C1[cr] + C2[cr]));
    Tb[(int64_t)(jb + r) * (b + 1) + (r - c)] = v;
}

// the high FP32 parts of float-float values
__global__ void df32_hi_kernel(int64_t count, const df32* __restrict__ in, float* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = in[e].hi;
}

// B_j (upper triangular) into block (j+1, j) of T
__global__ void fill_B_kernel(int j, int b, int rows_alloc, const double* __restrict__ Bj, double* __restrict__ Tb) {
    const int e = threadIdx.x;
    if (e >= b * b) return;
    const int r = e / b, c = e % b;
    if (c < r) return;
    const int row = (j + 1) * b + r;
    if (row >= rows_alloc) return;
    Tb[(int64_t)row * (b + 1) + (b + r - c)] = Bj[r * b + c];
}

// est_i = || B_j S[m-b .. m-1, i] ||_2 with B_j read from rows m..m+b-1 of
// the band (upper triangular: B_j[r][c] at d = b + r - c, c >= r)
__global__ void estimate_kernel(int m, int b, int k, const double* __restrict__ Tb, const double* __restrict__ S,
                                double* __restrict__ est) {
    const int i = threadIdx.x;
    if (i >= k) return;
    double s2 = 0.0;
    for (int r = 0; r < b; ++r) {
        double t = 0.0;
        for (int c = r; c < b; ++c) t += Tb[(int64_t)(m + r) * (b + 1) + (b + r - c)] * S[(int64_t)(m - b + c) * k + i];
        s2 += t * t;
    }
    est[i] = sqrt(s2);
}

// Z[:, c] -> W[:, c] for masked columns
template <typename T>
__global__ void merge_cols_kernel(int64_t n, int b, const int* __restrict__ mask, const T* __restrict__ Z,
                                  T* __restrict__ W) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * b; e += (int64_t)gridDim.x * blockDim.x)
        if (mask[e % b]) W[e] = Z[e];
}

// per-CTA partial sums of (Y - X diag(theta))^2 per column, k <= 16
__global__ void resid_partial_kernel(int64_t n, int k, const double* __restrict__ Y, const double* __restrict__ X,
                                     const double* __restrict__ theta, double* __restrict__ partial) {
    __shared__ double red[256];
    for (int i = 0; i < k; ++i) {
        double s = 0.0;
        const double th = theta[i];
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
            const double d = Y[r * k + i] - th * X[r * k + i];
            s += d * d;
        }
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[blockIdx.x * k + i] = red[0];
        __syncthreads();
    }
}

// per-CTA (max |x|, first index) per column
__global__ void colmax_partial_kernel(int64_t n, int k, const double* __restrict__ X, double* __restrict__ pv,
                                      int64_t* __restrict__ pi) {
    __shared__ double bv[256];
    __shared__ int64_t bi[256];
    for (int i = 0; i < k; ++i) {
        double best = -1.0;
        int64_t idx = 0;
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
            const double v = fabs(X[r * k + i]);
            if (v > best) {
                best = v;
                idx = r;
            }
        }
        bv[threadIdx.x] = best;
        bi[threadIdx.x] = idx;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) {
                if (bv[threadIdx.x + w] > bv[threadIdx.x] ||
                    (bv[threadIdx.x + w] == bv[threadIdx.x] && bi[threadIdx.x + w] < bi[threadIdx.x])) {
                    bv[threadIdx.x] = bv[threadIdx.x + w];
                    bi[threadIdx.x] = bi[threadIdx.x + w];
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            pv[blockIdx.x * k + i] = bv[0];
            pi[blockIdx.x * k + i] = bi[0];
        }
        __syncthreads();
    }
}

__global__ void scale_cols_kernel(int64_t n, int k, const double* __restrict__ sgn, double* __restrict__ X) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x)
        X[e] *= sgn[e % k];
}

constexpr int kRedBlocks = 304;

// ------------------------------------------------------------------ thick restart
// When the basis Q of J blocks is full: H Q = Q T + V_{J+1} B_J E_J^T.  The
// k lowest Ritz pairs (theta, S) of T give X = Q S_k with
// H X = X diag(theta) + V_{J+1} C, C = B_J E_J^T S_k (b x k): in the basis
// [X, V_{J+1}] the projection is an arrowhead.  A small block Lanczos on
// diag(theta) started from C^T turns X into blocks Y_1..Y_r (r = k/b) whose
// projection is block tridiagonal with the coupling to V_{J+1} on the last
// one only; ordering them Y_r, ..., Y_1, V_{J+1} keeps T banded, so the
// Lanczos recurrence and the banded Ritz solve go on unchanged.  Each block
// of the small Lanczos is normalised "QL"-style (the QR of its columns in
// reverse order), which makes every coupling block of the reversed order
// upper triangular, as the band storage wants.
constexpr int kRestartMaxK = 16;

// One CTA.  theta[k], S (m x k row-major): the k lowest Ritz pairs of the
// band Tb (m rows; B_J in rows m..m+b-1).  Out: G (m x k row-major), the
// coordinates of the new blocks in Q (block t = columns t*b..t*b+b-1), and
// band rows 0..k+b-1 of the restarted T (the diagonal block of V_{J+1},
// rows k..k+b-1, is left zero for the next Gram-Schmidt pass to fill).
// status: bit 0 set if a value is not finite.
__global__ void __launch_bounds__(256) restart_kernel(int m, int b, int k, const double* __restrict__ theta,
                                                      const double* __restrict__ S, double* __restrict__ Tb,
                                                      double* __restrict__ G, int* __restrict__ status) {
    __shared__ double th[kRestartMaxK];
    __shared__ double C[kMaxB * kRestartMaxK];          // b x k
    __shared__ double Z[kRestartMaxK * kRestartMaxK];   // column c of the new basis at Z[c * k + i]
    __shared__ double M[kRestartMaxK * kRestartMaxK];   // Z^T diag(theta) Z
    __shared__ double U[kMaxB * kMaxB];                 // C times the last new block (b x b)
    const int t = threadIdx.x;
    const int r = k / b;
    if (t < k) th[t] = theta[t];
    // C[x][i] = sum_{c >= x} B_J[x][c] S[m - b + c][i]; B_J[x][c] at band row m + x, d = b + x - c
    for (int e = t; e < b * k; e += blockDim.x) {
        const int x = e / k, i = e % k;
        double s = 0.0;
        for (int c = x; c < b; ++c) s += Tb[(int64_t)(m + x) * (b + 1) + (b + x - c)] * S[(int64_t)(m - b + c) * k + i];
        C[e] = s;
    }
    __syncthreads();
    if (t == 0) {
        // Q columns of the small Lanczos in creation order; block i (0-based)
        // holds columns i*b .. i*b+b-1 of Qc, already in reversed ("QL") order
        double Qc[kRestartMaxK * kRestartMaxK];
        int nz = 0;
        for (int blk = 0; blk < r; ++blk) {
            double Wc[kMaxB * kRestartMaxK];  // b columns of length k, reversed column order
            for (int c = 0; c < b; ++c)
                for (int i = 0; i < k; ++i) {
                    const int src = b - 1 - c;
                    Wc[c * k + i] = blk == 0 ? C[src * k + i] : th[i] * Qc[((blk - 1) * b + src) * k + i];
                }
            for (int c = 0; c < b; ++c) {
                double* v = Wc + c * k;
                double orig = 0.0;
                for (int i = 0; i < k; ++i) orig += v[i] * v[i];
                orig = sqrt(orig);
                for (int pass = 0; pass < 2; ++pass)
                    for (int l = 0; l < nz; ++l) {
                        double dt = 0.0;
                        for (int i = 0; i < k; ++i) dt += Qc[l * k + i] * v[i];
                        for (int i = 0; i < k; ++i) v[i] -= dt * Qc[l * k + i];
                    }
                double nrm = 0.0;
                for (int i = 0; i < k; ++i) nrm += v[i] * v[i];
                nrm = sqrt(nrm);
                if (!(orig > 0.0) || !(nrm > 1e-10 * orig)) {
                    // dependent: the first unit vector left with half its length
                    // after two passes against the columns so far
                    for (int u = 0; u < k; ++u) {
                        for (int i = 0; i < k; ++i) v[i] = (i == u) ? 1.0 : 0.0;
                        for (int pass = 0; pass < 2; ++pass)
                            for (int l = 0; l < nz; ++l) {
                                double dt = 0.0;
                                for (int i = 0; i < k; ++i) dt += Qc[l * k + i] * v[i];
                                for (int i = 0; i < k; ++i) v[i] -= dt * Qc[l * k + i];
                            }
                        nrm = 0.0;
                        for (int i = 0; i < k; ++i) nrm += v[i] * v[i];
                        nrm = sqrt(nrm);
                        if (nrm > 0.5) break;
                    }
                }
                for (int i = 0; i < k; ++i) Qc[nz * k + i] = v[i] / nrm;
                ++nz;
            }
            // un-reverse: block blk's columns in natural order
            for (int c = 0; c < b / 2; ++c)
                for (int i = 0; i < k; ++i) {
                    const double a = Qc[(blk * b + c) * k + i];
                    Qc[(blk * b + c) * k + i] = Qc[(blk * b + b - 1 - c) * k + i];
                    Qc[(blk * b + b - 1 - c) * k + i] = a;
                }
        }
        // new block t = small-Lanczos block r - 1 - t (the one coupled to V_{J+1} last)
        for (int tt = 0; tt < r; ++tt)
            for (int c = 0; c < b; ++c)
                for (int i = 0; i < k; ++i) Z[(tt * b + c) * k + i] = Qc[((r - 1 - tt) * b + c) * k + i];
    }
    __syncthreads();
    for (int e = t; e < k * k; e += blockDim.x) {
        const int x = e / k, y = e % k;
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += Z[x * k + i] * th[i] * Z[y * k + i];
        M[e] = s;
    }
    for (int e = t; e < b * b; e += blockDim.x) {
        const int x = e / b, y = e % b;
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += C[x * k + i] * Z[((r - 1) * b + y) * k + i];
        U[e] = s;
    }
    __syncthreads();
    for (int64_t e = t; e < (int64_t)m * k; e += blockDim.x) {
        const int64_t row = e / k;
        const int col = (int)(e % k);
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += S[row * k + i] * Z[col * k + i];
        G[e] = s;
        if (!isfinite(s)) atomicOr(status, 1);
    }
    for (int e = t; e < (k + b) * (b + 1); e += blockDim.x) {
        const int row = e / (b + 1), d = e % (b + 1);
        const int col = row - d;
        double v = 0.0;
        if (col >= 0) {
            if (row < k) v = M[row * k + col];
            else if (col < k) v = U[(row - k) * b + (col - (r - 1) * b)];
        }
        Tb[e] = v;
    }
}

// the kept vectors Y (n x k FP64, row-major) into basis blocks 0..k/b-1
template <typename T>
__global__ void restart_store_kernel(int64_t n, int b, int k, const double* __restrict__ Y, T* __restrict__ basis) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k;
        const int c = (int)(e % k);
        basis[(int64_t)(c / b) * n * b + i * b + (c % b)] = T(Y[e]);
    }
}

struct Timer {
    cudaEvent_t ev[6] = {};
    bool ok = false;
    bbl_status init() {
        for (auto& e : ev) BBL_CUDA(cudaEventCreate(&e));
        ok = true;
        return BBL_OK;
    }
    ~Timer() {
        if (ok)
            for (auto& e : ev) cudaEventDestroy(e);
    }
    float ms(int a, int b) const {
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[a], ev[b]);
        return t;
    }
};

struct StageOut {
    std::vector<double> theta, est;
    int iters = 0, deflations = 0, nev_eff = 0, spmm_calls = 0, ritz_solves = 0;
    bool converged = false;
    double t_spmm = 0, t_reorth = 0, t_chol = 0, t_ritz = 0, t_other = 0;
    double spmm_bytes = 0, reorth_bytes = 0;
    double t_gram = 0, gram_bytes = 0;  // the first Gram-Schmidt pass's Gram (kernel + partial reduction)
    int gram_calls = 0;
    int restarts = 0;
};

// Normalise columns of X (FP64, n x k) to the sign convention and compute the
// true residuals ||H x_i - theta_i x_i||_2 (FP64 SpMM).  quick (FP32 matrix
// values only): the product H X in float-float arithmetic instead, for the
// residuals that only decide whether the polish runs.
bbl_status finish_vectors(const bbl_matrix* A, int k, double* X, const double* theta_dev, double* resid_host,
                          DevBuf& scratch, cudaStream_t st, bool quick = false) {
    const int64_t n = A->n;
    quick = quick && A->storage == BBL_FP32;
    const size_t nk2 = ((size_t)n * k + 1) & ~size_t(1);  // 16-byte aligned sub-buffers
    const size_t need = sizeof(double) * nk2 * (quick ? 3 : 1) +
                        (sizeof(double) * 2 + sizeof(int64_t)) * kRedBlocks * k + 256;
    if (scratch.bytes < need) BBL_TRY(scratch.alloc(need));
    double* Y = scratch.as<double>();
    double* pv = Y + nk2 * (quick ? 3 : 1);
    int64_t* pi = reinterpret_cast<int64_t*>(pv + (size_t)kRedBlocks * k);
    double* pr = reinterpret_cast<double*>(pi + (size_t)kRedBlocks * k);
    colmax_partial_kernel<<<kRedBlocks, 256, 0, st>>>(n, k, X, pv, pi);
    BBL_LAUNCH_CHECK();
    std::vector<double> hv((size_t)kRedBlocks * k);
    std::vector<int64_t> hi((size_t)kRedBlocks * k);
    BBL_CUDA(cudaMemcpyAsync(hv.data(), pv, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaMemcpyAsync(hi.data(), pi, sizeof(int64_t) * hi.size(), cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    std::vector<double> sgn(k, 1.0);
    for (int i = 0; i < k; ++i) {
        double best = -1.0;
        int64_t idx = 0;
        for (int blk = 0; blk < kRedBlocks; ++blk) {
            const double v = hv[(size_t)blk * k + i];
            const int64_t j = hi[(size_t)blk * k + i];
            if (v > best || (v == best && j < idx)) {
                best = v;
                idx = j;
            }
        }
        double xv = 0.0;
        BBL_CUDA(cudaMemcpy(&xv, X + idx * k + i, sizeof(double), cudaMemcpyDeviceToHost));
        if (xv < 0.0) sgn[i] = -1.0;
    }
    BBL_CUDA(cudaMemcpyAsync(pv, sgn.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
    scale_cols_kernel<<<kRedBlocks, 256, 0, st>>>(n, k, pv, X);
    BBL_LAUNCH_CHECK();
    if (resid_host) {
        if (quick) {
            df32* Xd = reinterpret_cast<df32*>(Y + nk2);
            df32* Yd = reinterpret_cast<df32*>(Y + 2 * nk2);
            convert_kernel<double, df32><<<152 * 8, 256, 0, st>>>(n * k, X, Xd);
            BBL_LAUNCH_CHECK();
            BBL_TRY(spmm_df32(A, k, Xd, Yd, st));
            convert_kernel<df32, double><<<152 * 8, 256, 0, st>>>(n * k, Yd, Y);
            BBL_LAUNCH_CHECK();
        } else {
            BBL_TRY(spmm_dispatch(A, k, X, Y, true, st));
        }
        resid_partial_kernel<<<kRedBlocks, 256, 0, st>>>(n, k, Y, X, theta_dev, pr);
        BBL_LAUNCH_CHECK();
        std::vector<double> hp((size_t)kRedBlocks * k);
        BBL_CUDA(cudaMemcpyAsync(hp.data(), pr, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
        BBL_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < k; ++i) {
            double s = 0.0;
            for (int blk = 0; blk < kRedBlocks; ++blk) s += hp[(size_t)blk * k + i];
            resid_host[i] = std::sqrt(s);
        }
    }
    return BBL_OK;
}

// When to run the Ritz solve (the convergence test of Sec. II.B).  every > 0:
// after every `every`-th block.  every == 0: adaptive.  The residual
// estimates of block Lanczos fall roughly geometrically; from the last two
// tests, rho = max_i est_i / (tol ||H||) and its per-block decay give a
// predicted number of blocks to convergence, and the next test is placed at
// half of it (1..8 blocks ahead), so a run stops at most a few blocks after
// the first block that passes.  Until two decreasing tests exist, every
// block is tested.
struct CheckPlan {
    int every = 1;
    int next = 0;
    int n_pts = 0;
    int j_prev = -1;
    double l_prev = 0.0;
    bool want(int j) const { return every > 0 ? ((j + 1) % every == 0) : (j >= next); }
    void report(int jj, double rho) {
        if (every > 0) return;
        const double l = std::log(std::max(rho, 1e-300));
        int step = 1;
        if (n_pts > 0 && jj > j_prev && l < l_prev && l > 0.0) {
            const double rate = (l_prev - l) / (double)(jj - j_prev);
            const double blocks = l / rate;
            step = (int)std::min(8.0, std::max(1.0, std::floor(0.5 * blocks)));
        }
        j_prev = jj;
        l_prev = l;
        ++n_pts;
        next = jj + step;
    }
};

// One block Lanczos run from an FP64 device pivot (n x b).  dtype: storage of
// the blocks; f64_spmm: FP64 arithmetic in the SpMM.  On return X (device
// FP64 n x nev_eff) holds the Ritz vectors, theta_dev the Ritz values.
bbl_status lanczos_stage(const bbl_matrix* A, int nev, int b, const double* pivot_dev, int dtype, bool f64_spmm,
                         double tol, const bbl_options& o, cudaStream_t st, double* X, double* theta_dev,
                         StageOut& out, int keep = 0) {
    const int64_t n = A->n;
    const size_t s = dtype_size(dtype);
    const double nrm = A->norm_inf > 0 ? A->norm_inf : 1.0;
    int J_max = std::max(1, o.max_vectors / b);
    // FP32 blocks, b = 8: the first Gram-Schmidt pass reads an FP16 copy of the basis
    const bool half1 = dtype == BBL_FP32 && b == 8 && o.half_first_pass != 0;
    // FP32 blocks, b = 8: the first update and the second Gram share one read of the basis
    const bool fuse_on = dtype == BBL_FP32 && b == 8 && o.fused_update_gram != 0;
    // b = 8 with a narrower copy of the basis kept (FP16 for FP32 blocks, FP32
    // for float-float blocks): both updates read the blocks older than the
    // two newest from it (not after a thick restart, whose kept blocks carry
    // large coefficients)
    const bool half_upd = (half1 || (dtype == kDF32 && b == 8)) && o.narrow_old_updates != 0 && keep == 0;
    {
        size_t freeb = 0, totalb = 0;
        BBL_CUDA(cudaMemGetInfo(&freeb, &totalb));
        int dev = 0;
        BBL_CUDA(cudaGetDevice(&dev));
        freeb += pool_idle_bytes(dev);  // cached bases are available to this call
        // float-float blocks also keep an FP32 copy (first Gram-Schmidt pass)
        const size_t per_block = (size_t)n * b * (s + (dtype == kDF32 ? sizeof(float) : 0) + (half1 ? 2 : 0));
        const size_t reserve = (size_t)(2ull << 30) + 8 * (size_t)n * b * 8;
        if (freeb > reserve) {
            const int fit = (int)std::min<size_t>((freeb - reserve) / per_block, (size_t)1 << 30);
            J_max = std::max(1, std::min(J_max, fit));
        }
    }
    const int m_max = J_max * b;
    if (nev > m_max) return set_error(BBL_ERR_INVALID_ARG, "solve: nev=%d exceeds the basis capacity %d", nev, m_max);
    // thick restart: keep/b blocks of kept Ritz vectors + the newest block
    const bool restart_on = keep > 0;
    const int r_keep = restart_on ? keep / b : 0;
    if (restart_on && (keep % b != 0 || keep < nev || keep > kRestartMaxK || r_keep + 2 > J_max))
        return set_error(BBL_ERR_INVALID_ARG,
                         "solve: restart_keep=%d must be a multiple of b=%d, >= nev=%d, <= %d, with room for %d more "
                         "blocks (basis capacity %d blocks)", keep, b, nev, kRestartMaxK, 2, J_max);
    const int max_total = restart_on ? (o.max_blocks > 0 ? o.max_blocks : 10000) : J_max;
    DevBuf Z, coeff, partials, small, Tb, S, rwork, flags, bj, hwork;
    PoolBuf basis;
    // float-float blocks: FP32 copies of the basis (high parts) and of W for
    // the first Gram-Schmidt pass, whose coefficients only need to remove the
    // bulk (the second pass, in float-float, takes out the rest; A_j then
    // sums both passes' own-block coefficients)
    PoolBuf shadow;
    DevBuf whi;
    BBL_TRY(basis.alloc((size_t)J_max * n * b * s, st));
    if (half1) BBL_TRY(shadow.alloc((size_t)J_max * n * b * 2, st));
    if (dtype == kDF32) {
        BBL_TRY(shadow.alloc((size_t)J_max * n * b * sizeof(float), st));
        BBL_TRY(whi.alloc((size_t)n * b * sizeof(float)));
    }
    BBL_TRY(Z.alloc((size_t)n * b * s));
    BBL_TRY(coeff.alloc(sizeof(double) * 2 * (size_t)m_max * b));
    const int t_rows = m_max + b;
    BBL_TRY(Tb.alloc(sizeof(double) * (size_t)t_rows * (b + 1)));
    BBL_TRY(S.alloc(sizeof(double) * (size_t)m_max * nev));
    BBL_TRY(rwork.alloc(ritz_workspace_bytes(m_max, b, nev) + 1024));
    BBL_TRY(bj.alloc(sizeof(double) * kMaxB * kMaxB));
    BBL_TRY(flags.alloc(sizeof(int) * (4 + 2 * kMaxB) + sizeof(double) * 2 * 64));
    BBL_TRY(small.alloc(sizeof(double) * 8 * kMaxB * kMaxB + sizeof(int) * 4 * kMaxB));
    BBL_CUDA(cudaMemsetAsync(Tb.p, 0, Tb.bytes, st));
    BBL_CUDA(cudaMemsetAsync(flags.p, 0, flags.bytes, st));
    BBL_CUDA(cudaMemsetAsync(small.p, 0, small.bytes, st));
    int* d_ndefl = flags.as<int>();          // [0] cumulative deflations
    int* d_mask = d_ndefl + 4;               // [b] deflation mask of the last CholQR2
    int* d_mask2 = d_mask + kMaxB;
    double* d_est = reinterpret_cast<double*>(flags.as<char>() + sizeof(int) * (4 + 2 * kMaxB));
    HostBuf report;
    BBL_TRY(report.alloc(sizeof(double) * 128 + sizeof(int) * 8));
    double* h_theta = report.as<double>();
    double* h_est = h_theta + 64;
    int* h_ndefl = reinterpret_cast<int*>(h_est + 64);

    auto blockp = [&](int j) -> char* { return basis.as<char>() + (size_t)j * n * b * s; };
    const unsigned cg = 152 * 8;
    // pivot -> block 0 in storage precision, orthonormalised (relative deflation)
    if (dtype == BBL_FP64)
        BBL_CUDA(cudaMemcpyAsync(blockp(0), pivot_dev, sizeof(double) * n * b, cudaMemcpyDeviceToDevice, st));
    else if (dtype == kDF32)
        convert_kernel<double, df32><<<cg, 256, 0, st>>>(n * b, pivot_dev, reinterpret_cast<df32*>(blockp(0)));
    else
        convert_kernel<double, float><<<cg, 256, 0, st>>>(n * b, pivot_dev, reinterpret_cast<float*>(blockp(0)));
    BBL_LAUNCH_CHECK();
    const double defl_tol = o.defl_tol > 0 ? o.defl_tol : (dtype == BBL_FP32 ? 1e-6 : 1e-10);
    const double thresh2 = (defl_tol * nrm) * (defl_tol * nrm);
    uint64_t defl_counter = 0;
    bool exhausted = false;
    auto replace_deflated = [&](int nb_basis, char* Wn, const int* mask_dev) -> bbl_status {
        // random columns where mask is set, orthogonalised against the basis
        // and the current block, then orthonormalised among themselves
        BBL_TRY(fill_uniform_cols(n, b, dtype, o.seed ^ 0x5DEECE66Dull, (defl_counter++) * (uint64_t)n * kMaxB, mask_dev,
                                  Z.p, st));
        for (int pass = 0; pass < 2; ++pass) {
            if (nb_basis > 0) {
                BBL_TRY(gram(n, b, nb_basis, dtype, basis.p, Z.p, coeff.as<double>(), partials, st));
                BBL_TRY(update(n, b, nb_basis, dtype, basis.p, coeff.as<double>(), Z.p, st));
            }
            BBL_TRY(gram(n, b, 1, dtype, Wn, Z.p, coeff.as<double>(), partials, st));
            BBL_TRY(update(n, b, 1, dtype, Wn, coeff.as<double>(), Z.p, st));
        }
        BBL_TRY(cholqr2_dev(n, b, dtype, Z.p, nullptr, -1e-20, nullptr, d_mask2, partials, small, st));
        // a replacement that is itself dependent means the Krylov space has
        // exhausted the whole space: the current Ritz pairs are exact
        int hm[2 * kMaxB];
        BBL_CUDA(cudaMemcpyAsync(hm, mask_dev, sizeof(int) * b, cudaMemcpyDeviceToHost, st));
        BBL_CUDA(cudaMemcpyAsync(hm + kMaxB, d_mask2, sizeof(int) * b, cudaMemcpyDeviceToHost, st));
        BBL_CUDA(cudaStreamSynchronize(st));
        for (int c = 0; c < b; ++c)
            if (hm[c] && hm[kMaxB + c]) exhausted = true;
        if (dtype == BBL_FP64)
            merge_cols_kernel<double><<<cg, 256, 0, st>>>(n, b, mask_dev, Z.as<double>(), reinterpret_cast<double*>(Wn));
        else if (dtype == kDF32)
            merge_cols_kernel<df32><<<cg, 256, 0, st>>>(n, b, mask_dev, Z.as<df32>(), reinterpret_cast<df32*>(Wn));
        else
            merge_cols_kernel<float><<<cg, 256, 0, st>>>(n, b, mask_dev, Z.as<float>(), reinterpret_cast<float*>(Wn));
        BBL_LAUNCH_CHECK();
        return BBL_OK;
    };
    BBL_TRY(cholqr2_dev(n, b, dtype, blockp(0), nullptr, -1e-20, d_ndefl + 1, d_mask, partials, small, st));
    BBL_CUDA(cudaMemcpyAsync(h_ndefl, d_ndefl + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    if (h_ndefl[0] > 0) BBL_TRY(replace_deflated(0, blockp(0), d_mask));
    auto shadow_block = [&](int jb) -> bbl_status {
        if (jb >= J_max) return BBL_OK;
        if (half1)
            return to_half(n * b, reinterpret_cast<const float*>(blockp(jb)), shadow.as<char>() + (size_t)jb * n * b * 2,
                           st);
        if (dtype != kDF32) return BBL_OK;
        df32_hi_kernel<<<cg, 256, 0, st>>>(n * b, reinterpret_cast<const df32*>(blockp(jb)),
                                           shadow.as<float>() + (size_t)jb * n * b);
        BBL_LAUNCH_CHECK();
        return BBL_OK;
    };
    BBL_TRY(shadow_block(0));
    auto narrow_update = [&](int nbk, const double* Cc, char* Wp) -> bbl_status {
        if (dtype == kDF32) return update_df32_f32old(n, nbk, 2, shadow.as<float>(), basis.p, Cc, Wp, st);
        return update_half_old(n, nbk, 2, shadow.p, basis.as<float>(), Cc, reinterpret_cast<float*>(Wp), hwork, st);
    };

    // The Ritz solve of T_j runs on a side stream while the main stream goes
    // on with block j+1 (whose SpMM does not need it); the host checks the
    // result of T_j after enqueuing block j+1.  When T_j has converged, block
    // j+1 was speculative and is not used.
    Timer tms[2];  // block tb uses tms[tb & 1]: its times are read one block later
    BBL_TRY(tms[0].init());
    BBL_TRY(tms[1].init());
    // ritz_overlap = 0: the Ritz solve runs on the caller's stream right after
    // its block and is read at once (no speculative block, no concurrency)
    const bool serial = o.ritz_overlap == 0;
    cudaStream_t side = nullptr;
    if (serial) side = st;
    else BBL_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    struct SideGuard {
        cudaStream_t s;
        cudaEvent_t e[7];
        ~SideGuard() {
            if (s) {
                cudaStreamSynchronize(s);
                cudaStreamDestroy(s);
            }
            for (auto& x : e)
                if (x) cudaEventDestroy(x);
        }
    } guard{serial ? nullptr : side, {}};
    for (int q = 0; q < 7; ++q) BBL_CUDA(cudaEventCreate(&guard.e[q]));
    cudaEvent_t* ev_main = guard.e;       // [2] main-stream block done
    cudaEvent_t* ev_r0 = guard.e + 2;     // [2] Ritz start
    cudaEvent_t* ev_r1 = guard.e + 4;     // [2] Ritz done (report in host memory)
    cudaEvent_t ev_defl = guard.e[6];     // deflation count of the last CholQR2 in host memory
    DevBuf theta2, S2, est2;
    BBL_TRY(theta2.alloc(sizeof(double) * 2 * 64));
    BBL_TRY(S2.alloc(sizeof(double) * 2 * (size_t)m_max * nev));
    BBL_TRY(est2.alloc(sizeof(double) * 2 * 64));
    DevBuf rwork2;
    BBL_TRY(rwork2.alloc(ritz_workspace_bytes(m_max, b, nev) + 1024));
    DevBuf* rw[2] = {&rwork, &rwork2};
    std::vector<double> prev_theta;
    int last_defl = 0;
    out.converged = false;
    int pending = -1;      // block whose Ritz report is in flight
    int warm_k = 0;        // Ritz values available from the previous solve
    int final_j = -1;      // block whose Ritz pairs are returned
    int final_k = 0;
    CheckPlan plan;
    plan.every = (o.check_every > 0 || o.criterion == 1) ? std::max(1, o.check_every) : 0;
    auto launch_ritz = [&](int jj, int tt) -> bbl_status {
        const int m = (jj + 1) * b;
        const int k = std::min(nev, m);
        const int slot = tt & 1;
        BBL_CUDA(cudaStreamWaitEvent(side, ev_main[slot], 0));
        BBL_CUDA(cudaEventRecord(ev_r0[slot], side));
        double* th = theta2.as<double>() + 64 * slot;
        double* Sd = S2.as<double>() + (size_t)slot * m_max * nev;
        double* es = est2.as<double>() + 64 * slot;
        // warm start from the previous Ritz solve on this stream (other slot)
        const double* warm = warm_k > 0 ? theta2.as<double>() + 64 * (slot ^ 1) : nullptr;
        BBL_TRY(ritz_dev(m, b, k, Tb.as<double>(), th, Sd, *rw[slot], side, warm, warm_k));
        warm_k = k;
        // B_jj sits in rows (jj+1)b.. of the band: the estimate reads it there
        estimate_kernel<<<1, 64, 0, side>>>(m, b, k, Tb.as<double>(), Sd, es);
        BBL_LAUNCH_CHECK();
        BBL_CUDA(cudaMemcpyAsync(h_theta + 32 * slot, th, sizeof(double) * k, cudaMemcpyDeviceToHost, side));
        BBL_CUDA(cudaMemcpyAsync(h_est + 32 * slot, es, sizeof(double) * k, cudaMemcpyDeviceToHost, side));
        BBL_CUDA(cudaEventRecord(ev_r1[slot], side));
        return BBL_OK;
    };
    // waits for the report of block jj (basis position; tt: its index over
    // all restarts); returns 1 when converged
    int final_t = -1;
    auto check_ritz = [&](int jj, int tt, bool* done) -> bbl_status {
        const int m = (jj + 1) * b;
        const int k = std::min(nev, m);
        const int slot = tt & 1;
        BBL_CUDA(cudaEventSynchronize(ev_r1[slot]));
        out.t_ritz += [&] { float t = 0.f; cudaEventElapsedTime(&t, ev_r0[slot], ev_r1[slot]); return (double)t; }();
        const double* ht = h_theta + 32 * slot;
        const double* he = h_est + 32 * slot;
        for (int i = 0; i < k; ++i)
            if (!std::isfinite(ht[i]) || !std::isfinite(he[i]))
                return set_error(BBL_ERR_NUMERICAL, "solve: non-finite Ritz value at block %d", jj);
        out.theta.assign(ht, ht + k);
        out.est.assign(he, he + k);
        *done = false;
        ++out.ritz_solves;
        if (k == nev) {
            double rho = 0.0;
            for (int i = 0; i < nev; ++i) rho = std::max(rho, he[i] / (tol * nrm));
            plan.report(tt, rho);
            if (o.criterion == 1) {
                if (prev_theta.size() == (size_t)nev) {
                    double ss = 0.0;
                    for (int i = 0; i < nev; ++i) ss += (ht[i] - prev_theta[i]) * (ht[i] - prev_theta[i]);
                    *done = std::sqrt(ss / nev) < o.rms_tol;
                }
            } else {
                *done = true;
                for (int i = 0; i < nev; ++i) *done = *done && (he[i] <= tol * nrm);
            }
        }
        prev_theta.assign(ht, ht + k);
        final_j = jj;
        final_t = tt;
        final_k = k;
        return BBL_OK;
    };
    // thick restart at the full block jf (its report checked, not converged;
    // V_{J+1} normalised in Wn): blocks 0..r_keep-1 <- Q G, block r_keep <- Wn,
    // band rows 0..keep+b-1 rebuilt
    DevBuf th_r, S_r, G_r, Y_r, st_r;
    auto thick_restart = [&](int jf, const char* Wn) -> bbl_status {
        const int m = (jf + 1) * b;
        if (!th_r.p) {
            BBL_TRY(th_r.alloc(sizeof(double) * 64));
            BBL_TRY(S_r.alloc(sizeof(double) * (size_t)m_max * keep));
            BBL_TRY(G_r.alloc(sizeof(double) * (size_t)m_max * keep));
            BBL_TRY(Y_r.alloc(sizeof(double) * (size_t)n * keep));
            BBL_TRY(st_r.alloc(sizeof(int) * 4));
        }
        BBL_CUDA(cudaStreamSynchronize(side));
        BBL_CUDA(cudaMemsetAsync(st_r.p, 0, sizeof(int) * 4, st));
        BBL_TRY(ritz_dev(m, b, keep, Tb.as<double>(), th_r.as<double>(), S_r.as<double>(), rwork, st));
        restart_kernel<<<1, 256, 0, st>>>(m, b, keep, th_r.as<double>(), S_r.as<double>(), Tb.as<double>(),
                                          G_r.as<double>(), st_r.as<int>());
        BBL_LAUNCH_CHECK();
        BBL_TRY(ritz_vectors(n, b, jf + 1, dtype, basis.p, keep, G_r.as<double>(), Y_r.as<double>(), st));
        if (dtype == BBL_FP64)
            restart_store_kernel<double><<<cg, 256, 0, st>>>(n, b, keep, Y_r.as<double>(), basis.as<double>());
        else if (dtype == kDF32)
            restart_store_kernel<df32><<<cg, 256, 0, st>>>(n, b, keep, Y_r.as<double>(), basis.as<df32>());
        else
            restart_store_kernel<float><<<cg, 256, 0, st>>>(n, b, keep, Y_r.as<double>(), basis.as<float>());
        BBL_LAUNCH_CHECK();
        BBL_CUDA(cudaMemcpyAsync(blockp(r_keep), Wn, (size_t)n * b * s, cudaMemcpyDeviceToDevice, st));
        for (int q = 0; q <= r_keep; ++q) BBL_TRY(shadow_block(q));
        int hs = 0;
        BBL_CUDA(cudaMemcpyAsync(&hs, st_r.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        BBL_CUDA(cudaStreamSynchronize(st));
        if (hs) return set_error(BBL_ERR_NUMERICAL, "solve: non-finite values in the thick restart");
        ++out.restarts;
        return BBL_OK;
    };
    int j = 0;        // basis position of the current block
    int tb = 0;       // its index over all restarts (SpMM calls so far)
    int pending_t = -1;
    bool stop = false;
    // W = H V_j is formed directly in the next basis slot (or Z when the
    // basis is full) and turned into V_{j+1} there (Gram-Schmidt only reads
    // blocks 0..j)
    auto spmm_block = [&](int jj, Timer& t) -> bbl_status {
        char* Wo = (jj + 1 < J_max) ? blockp(jj + 1) : Z.as<char>();
        BBL_CUDA(cudaEventRecord(t.ev[0], st));
        if (dtype == kDF32) return spmm_df32(A, b, blockp(jj), Wo, st);
        return spmm_dispatch(A, b, blockp(jj), Wo, f64_spmm, st);
    };
    // waits for the deflation count of block tb's CholQR2 and adds its phase times
    auto block_done = [&](Timer& t) -> bbl_status {
        BBL_CUDA(cudaEventSynchronize(ev_defl));
        out.t_spmm += t.ms(0, 1);
        out.t_reorth += t.ms(1, 2);
        out.t_chol += t.ms(2, 3);
        out.t_gram += t.ms(4, 5);
        return BBL_OK;
    };
    bool spmm_ahead = false;  // the current block's SpMM is already enqueued
    while (!stop) {
        Timer& tm = tms[tb & 1];
        char* Wn = (j + 1 < J_max) ? blockp(j + 1) : Z.as<char>();
        if (!spmm_ahead) BBL_TRY(spmm_block(j, tm));
        spmm_ahead = false;
        // ritz_overlap = 2: the Gram-Schmidt passes wait for the Ritz solve in
        // flight, which then shares the GPU with this SpMM only (the wait is
        // counted in the SpMM phase)
        if (o.ritz_overlap == 2 && pending >= 0) BBL_CUDA(cudaStreamWaitEvent(st, ev_r1[pending_t & 1], 0));
        BBL_CUDA(cudaEventRecord(tm.ev[1], st));
        double* C1 = coeff.as<double>();
        double* C2 = C1 + (size_t)m_max * b;
        const bool fused2 = fuse_on && update_gram_tc_supports(j + 1);
        BBL_CUDA(cudaEventRecord(tm.ev[4], st));
        if (dtype == kDF32) {
            df32_hi_kernel<<<cg, 256, 0, st>>>(n * b, reinterpret_cast<const df32*>(Wn), whi.as<float>());
            BBL_LAUNCH_CHECK();
            BBL_TRY(gram(n, b, j + 1, BBL_FP32, shadow.p, whi.p, C1, partials, st));
        } else if (half1) {
            BBL_TRY(gram_half(n, j + 1, shadow.p, reinterpret_cast<const float*>(Wn), C1, partials, st));
        } else {
            BBL_TRY(gram(n, b, j + 1, dtype, basis.p, Wn, C1, partials, st));
        }
        BBL_CUDA(cudaEventRecord(tm.ev[5], st));
        if (fused2) {
            // first update and second Gram in one read of the basis (tensor cores)
            BBL_TRY(update_gram_tc(n, j + 1, basis.as<float>(), C1, reinterpret_cast<float*>(Wn), C2, partials, st));
        } else {
            if (half_upd)
                BBL_TRY(narrow_update(j + 1, C1, Wn));
            else
                BBL_TRY(update(n, b, j + 1, dtype, basis.p, C1, Wn, st));
            BBL_TRY(gram(n, b, j + 1, dtype, basis.p, Wn, C2, partials, st));
        }
        if (half_upd)
            BBL_TRY(narrow_update(j + 1, C2, Wn));
        else
            BBL_TRY(update(n, b, j + 1, dtype, basis.p, C2, Wn, st));
        // A_j = sym(C1 + C2)[j-block]: the second pass's own-block coefficients
        // are the rounding (or, from a cheaper first pass, the approximation)
        // the first left in A_j
        fill_A2_kernel<<<1, 256, 0, st>>>(j, b, C1, C2, Tb.as<double>());
        BBL_LAUNCH_CHECK();
        BBL_CUDA(cudaEventRecord(tm.ev[2], st));
        BBL_TRY(cholqr2_dev(n, b, dtype, Wn, bj.as<double>(), thresh2, d_ndefl, d_mask, partials, small, st));
        fill_B_kernel<<<1, 256, 0, st>>>(j, b, t_rows, bj.as<double>(), Tb.as<double>());
        BBL_LAUNCH_CHECK();
        BBL_CUDA(cudaEventRecord(tm.ev[3], st));
        BBL_CUDA(cudaEventRecord(ev_main[tb & 1], st));
        BBL_CUDA(cudaMemcpyAsync(h_ndefl, d_ndefl, sizeof(int), cudaMemcpyDeviceToHost, st));
        BBL_CUDA(cudaEventRecord(ev_defl, st));
        out.gram_bytes += half1 ? (double)n * (j + 1) * b * 2.0 + (double)n * b * 4.0
                                : ((double)n * (j + 1) * b + (double)n * b) * (double)s;
        ++out.gram_calls;
        {
            const int m = (j + 1) * b;
            const double sx = (double)s;
            const double sv = (A->storage == BBL_FP64 || (dtype != kDF32 && f64_spmm && A->val64.p)) ? 8.0 : 4.0;
            out.spmm_bytes += spmm_alg_bytes(A, b, sv, sx);
            // two passes of Gram + update; an FP16 first-pass Gram reads 2 bytes per basis
            // element, and the fused first update + second Gram reads the basis once
            // an update with the blocks older than the two newest from the FP16 copy
            const double upd = (half_upd && j >= 2) ? 0.5 * (double)(j - 1) / (j + 1) + 2.0 / (j + 1) : 1.0;
            out.reorth_bytes += ((half1 ? 0.5 : 1.0) + (fused2 ? 1.0 : 1.0 + upd) + upd) * (double)n * m * sx +
                                6.0 * (double)n * b * sx;
        }
        out.spmm_calls = tb + 1;
        const bool full = (j == J_max - 1);
        const bool last = (tb == max_total - 1) || (full && !restart_on);
        const bool want = plan.want(tb) || last || full || (j + 1) * b < nev;
        if (want) {
            // a new Ritz solve may reuse the buffers of block j-2 only: the one of block j-1 is pending
            BBL_TRY(launch_ritz(j, tb));
        }
        if (serial && want) {  // read this block's report now
            pending = j;
            pending_t = tb;
        }
        if (pending >= 0) {
            bool done = false;
            BBL_TRY(check_ritz(pending, pending_t, &done));
            pending = -1;
            if (done) {
                out.converged = true;
                stop = true;
                BBL_TRY(block_done(tm));
                break;
            }
        }
        if (want && !serial) {
            pending = j;
            pending_t = tb;
        }
        if (last) {
            BBL_TRY(block_done(tm));
            break;
        }
        // The next block's SpMM is enqueued before the host reads this
        // block's deflation count, so that the GPU does not idle while the
        // host decides; a deflation (rare) replaces columns of V_{j+1}, and
        // the product is then formed again.
        const bool ahead = !full;
        if (ahead) {
            BBL_TRY(shadow_block(j + 1));
            BBL_TRY(spmm_block(j + 1, tms[(tb + 1) & 1]));
        }
        BBL_TRY(block_done(tm));
        spmm_ahead = ahead;
        if (h_ndefl[0] > last_defl) {
            BBL_TRY(replace_deflated(j + 1, Wn, d_mask));
            last_defl = h_ndefl[0];
            if (exhausted) break;  // no direction left to extend the basis with
            if (ahead) BBL_TRY(shadow_block(j + 1));
            spmm_ahead = false;
        }
        if (full) {
            // the basis is full: this block's report decides between stopping
            // and a thick restart
            if (pending >= 0) {  // (in line, ritz_overlap = 0, it was read above)
                bool done = false;
                BBL_TRY(check_ritz(pending, pending_t, &done));
                pending = -1;
                if (done) {
                    out.converged = true;
                    break;
                }
            }
            BBL_TRY(thick_restart(j, Wn));
            j = r_keep;
            ++tb;
            continue;
        }
        ++j;
        ++tb;
    }
    if (pending >= 0 && !stop) {
        bool done = false;
        BBL_TRY(check_ritz(pending, pending_t, &done));
        out.converged = done;
    }
    BBL_CUDA(cudaStreamSynchronize(side));
    out.deflations = last_defl;
    if (final_j < 0) return set_error(BBL_ERR_NUMERICAL, "solve: no Ritz solve completed");
    out.iters = final_t + 1;
    out.nev_eff = final_k;
    const int slot = final_t & 1;
    BBL_CUDA(cudaMemcpyAsync(theta_dev, theta2.as<double>() + 64 * slot, sizeof(double) * final_k,
                             cudaMemcpyDeviceToDevice, st));
    // Ritz vectors X = Q S (k columns) from the blocks of the returned T
    Timer& tf = tms[0];
    BBL_CUDA(cudaEventRecord(tf.ev[0], st));
    BBL_TRY(ritz_vectors(n, b, final_j + 1, dtype, basis.p, final_k, S2.as<double>() + (size_t)slot * m_max * nev, X,
                         st));
    BBL_CUDA(cudaEventRecord(tf.ev[1], st));
    BBL_CUDA(cudaStreamSynchronize(st));
    out.t_other += tf.ms(0, 1);
    return BBL_OK;
}

bbl_status solve_impl(const bbl_matrix* A, int nev, int b, const double* pivot, const bbl_options* opt, double* evals,
                      double* evecs, double* resid, bbl_stats* stats) {
    if (!A) return set_error(BBL_ERR_INVALID_ARG, "solve: matrix is NULL");
    if (b < 1 || b > kMaxB) return set_error(BBL_ERR_INVALID_ARG, "solve: b=%d outside 1..16", b);
    if (nev < 1 || nev > kMaxB) return set_error(BBL_ERR_INVALID_ARG, "solve: nev=%d outside 1..16", nev);
    if (!evals) return set_error(BBL_ERR_INVALID_ARG, "solve: evals is NULL");
    bbl_options o;
    if (opt) o = *opt;
    else bbl_options_default(&o);
    if (!(o.tol > 0) || o.max_vectors < b) return set_error(BBL_ERR_INVALID_ARG, "solve: bad tol / max_vectors");
    if (o.storage != A->storage)
        return set_error(BBL_ERR_INVALID_ARG, "solve: options.storage (%d) must match the matrix storage (%d)", o.storage,
                         A->storage);
    if (o.criterion != 0 && o.criterion != 1) return set_error(BBL_ERR_INVALID_ARG, "solve: bad criterion");
    if (o.ritz_overlap < 0 || o.ritz_overlap > 2) return set_error(BBL_ERR_INVALID_ARG, "solve: ritz_overlap must be 0, 1 or 2");
    cudaStream_t st = as_stream(o.stream);
    const int64_t n = A->n;
    if (nev > n || b > n) return set_error(BBL_ERR_INVALID_ARG, "solve: nev or b larger than n");
    cudaEvent_t t0, t1;
    BBL_CUDA(cudaEventCreate(&t0));
    BBL_CUDA(cudaEventCreate(&t1));
    BBL_CUDA(cudaEventRecord(t0, st));
    DevBuf piv, X, theta, scratch;
    BBL_TRY(piv.alloc(sizeof(double) * n * std::max(b, nev)));
    if (pivot) {
        BBL_CUDA(cudaMemcpyAsync(piv.p, pivot, sizeof(double) * n * b, cudaMemcpyDefault, st));
    } else {
        BBL_TRY(fill_normal(n, b, o.seed, 0, piv.as<double>(), st));
    }
    BBL_TRY(X.alloc(sizeof(double) * n * nev));
    BBL_TRY(theta.alloc(sizeof(double) * 64));
    StageOut s1, s2;
    const bool mixed = A->storage == BBL_FP32;
    bbl_status rc = BBL_OK;
    std::vector<double> res(nev, 0.0);
    if (!mixed) {
        BBL_TRY(lanczos_stage(A, nev, b, piv.as<double>(), BBL_FP64, false, o.tol, o, st, X.as<double>(),
                              theta.as<double>(), s1, o.restart_keep));
    } else {
        const double t1tol = o.polish ? std::max(o.tol, o.stage1_tol) : o.tol;
        BBL_TRY(lanczos_stage(A, nev, b, piv.as<double>(), BBL_FP32, false, t1tol, o, st, X.as<double>(),
                              theta.as<double>(), s1, o.restart_keep));
    }
    int k = s1.nev_eff;
    // before a polish the stage-1 residuals only decide whether it runs
    BBL_TRY(finish_vectors(A, k, X.as<double>(), theta.as<double>(), res.data(), scratch, st, mixed && o.polish));
    const double nrm = A->norm_inf > 0 ? A->norm_inf : 1.0;
    bool ok = s1.converged && k == nev;
    if (mixed && o.polish) {
        bool need = false;
        for (int i = 0; i < k; ++i) need = need || !(res[i] <= o.tol * nrm);
        if (need || k < nev) {
            // stage 2: FP64 block Lanczos from the FP32 Ritz vectors (block size nev)
            BBL_CUDA(cudaMemcpyAsync(piv.p, X.p, sizeof(double) * n * k, cudaMemcpyDeviceToDevice, st));
            bbl_options o2 = o;
            o2.criterion = 0;
            // polish 1: float-float blocks and products (FP32 pipes, ~48-bit);
            // polish 2: FP64 blocks and FP64 arithmetic
            const int pdt = o.polish == 2 ? BBL_FP64 : kDF32;
            // the polish's block size is k: its restart keeps a multiple of k
            const int keep2 = o.restart_keep > 0 ? std::min(kRestartMaxK, (int)ceil_div(o.restart_keep, k) * k) : 0;
            BBL_TRY(lanczos_stage(A, nev, k, piv.as<double>(), pdt, true, o.tol, o2, st, X.as<double>(),
                                  theta.as<double>(), s2, keep2));
            k = s2.nev_eff;
            BBL_TRY(finish_vectors(A, k, X.as<double>(), theta.as<double>(), res.data(), scratch, st));
            ok = s2.converged && k == nev;
        } else {
            // no polish needed: report FP64 residuals
            BBL_TRY(finish_vectors(A, k, X.as<double>(), theta.as<double>(), res.data(), scratch, st));
            ok = true;
        }
    }
    std::vector<double> th(k);
    BBL_CUDA(cudaMemcpyAsync(th.data(), theta.p, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    if (evecs) BBL_CUDA(cudaMemcpyAsync(evecs, X.p, sizeof(double) * n * k, cudaMemcpyDefault, st));
    BBL_CUDA(cudaEventRecord(t1, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < k; ++i) evals[i] = th[i];
    if (resid)
        for (int i = 0; i < k; ++i) resid[i] = res[i];
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->iters = s1.iters;
        stats->vec_equiv_iters = s1.iters * b;
        stats->polish_iters = s2.iters;
        stats->deflations = s1.deflations + s2.deflations;
        stats->converged = ok ? 1 : 0;
        stats->t_spmm_ms = s1.t_spmm + s2.t_spmm;
        stats->t_reorth_ms = s1.t_reorth + s2.t_reorth;
        stats->t_cholqr_ms = s1.t_chol + s2.t_chol;
        stats->t_ritz_ms = s1.t_ritz + s2.t_ritz;
        stats->t_other_ms = s1.t_other + s2.t_other;
        float tt = 0.f;
        cudaEventElapsedTime(&tt, t0, t1);
        stats->t_total_ms = tt;
        const double sv = mixed ? 4.0 : 8.0;
        stats->spmm_bytes = spmm_alg_bytes(A, b, sv, sv);
        stats->spmm_gbs = s1.t_spmm > 0 ? s1.spmm_bytes / (s1.t_spmm * 1e-3) / 1e9 : 0.0;
        stats->ns_per_op = s1.t_spmm > 0 ? s1.t_spmm * 1e6 / ((double)A->nnz * b * s1.spmm_calls) : 0.0;
        stats->spmm_bytes_total = s1.spmm_bytes + s2.spmm_bytes;
        stats->reorth_bytes_total = s1.reorth_bytes + s2.reorth_bytes;
        stats->ritz_solves = s1.ritz_solves + s2.ritz_solves;
        stats->gram_calls = s1.gram_calls;
        stats->t_gram_ms = s1.t_gram;
        stats->gram_bytes_total = s1.gram_bytes;
        stats->spmm_calls = s1.spmm_calls;
        stats->restarts = s1.restarts + s2.restarts;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (!ok) {
        set_error(BBL_ERR_NOT_CONVERGED, "solve: basis full before convergence (%d blocks)", s1.iters);
        rc = BBL_ERR_NOT_CONVERGED;
    }
    return rc;
}

}  // namespace
}  // namespace bbl

extern "C" bbl_status bbl_solve(const bbl_matrix* A, int nev, int b, const double* pivot, const bbl_options* opt,
                                double* evals, double* evecs, double* resid, bbl_stats* stats) {
    return bbl::solve_impl(A, nev, b, pivot, opt, evals, evecs, resid, stats);
}

namespace bbl {
namespace {
// dense symmetric b x b (row-major) -> lower band storage with p = b - 1
__global__ void dense_to_band_kernel(int b, const double* __restrict__ G, double* __restrict__ Tb) {
    const int e = threadIdx.x;
    if (e >= b * b) return;
    const int r = e / b, c = e % b;
    if (c > r) return;
    Tb[r * b + (r - c)] = 0.5 * (G[r * b + c] + G[c * b + r]);
}
}  // namespace
}  // namespace bbl

// Rayleigh-Ritz on the span of a pivot block: Q = orth(P), T = Q^T H Q,
// theta, S = eig(T), residuals ||H Q s_i - theta_i Q s_i||_2 (FP64).
extern "C" bbl_status bbl_pivot_rr_residual(const bbl_matrix* A, int b, const double* P, double* theta_out,
                                            double* resid_out, void* stream) {
    using namespace bbl;
    if (!A || !P || !theta_out || !resid_out || b < 1 || b > kMaxB || b > A->n)
        return set_error(BBL_ERR_INVALID_ARG, "pivot_rr_residual: bad arguments");
    cudaStream_t st = as_stream(stream);
    const int64_t n = A->n;
    DevBuf Q, W, G, Tb, th, S, X, Y, partials, small, rwork, scratch;
    BBL_TRY(Q.alloc(sizeof(double) * n * b));
    BBL_TRY(W.alloc(sizeof(double) * n * b));
    BBL_TRY(X.alloc(sizeof(double) * n * b));
    BBL_TRY(Y.alloc(sizeof(double) * n * b));
    BBL_TRY(G.alloc(sizeof(double) * b * b));
    BBL_TRY(Tb.alloc(sizeof(double) * b * b));
    BBL_TRY(th.alloc(sizeof(double) * 64));
    BBL_TRY(S.alloc(sizeof(double) * b * b));
    BBL_TRY(small.alloc(sizeof(double) * 8 * kMaxB * kMaxB + sizeof(int) * 4 * kMaxB));
    BBL_CUDA(cudaMemsetAsync(small.p, 0, small.bytes, st));
    BBL_CUDA(cudaMemsetAsync(Tb.p, 0, Tb.bytes, st));
    BBL_CUDA(cudaMemcpyAsync(Q.p, P, sizeof(double) * n * b, cudaMemcpyDefault, st));
    BBL_TRY(cholqr2_dev(n, b, BBL_FP64, Q.p, nullptr, -1e-20, nullptr, nullptr, partials, small, st));
    BBL_TRY(spmm_dispatch(A, b, Q.p, W.p, true, st));
    BBL_TRY(gram(n, b, 1, BBL_FP64, Q.p, W.p, G.as<double>(), partials, st));
    dense_to_band_kernel<<<1, 256, 0, st>>>(b, G.as<double>(), Tb.as<double>());
    BBL_LAUNCH_CHECK();
    BBL_TRY(ritz_dev(b, b - 1, b, Tb.as<double>(), th.as<double>(), S.as<double>(), rwork, st));
    BBL_TRY(ritz_vectors(n, b, 1, BBL_FP64, Q.p, b, S.as<double>(), X.as<double>(), st));
    BBL_TRY(ritz_vectors(n, b, 1, BBL_FP64, W.p, b, S.as<double>(), Y.as<double>(), st));
    const size_t need = sizeof(double) * (size_t)kRedBlocks * b;
    BBL_TRY(scratch.alloc(need));
    resid_partial_kernel<<<kRedBlocks, 256, 0, st>>>(n, b, Y.as<double>(), X.as<double>(), th.as<double>(),
                                                      scratch.as<double>());
    BBL_LAUNCH_CHECK();
    std::vector<double> hp((size_t)kRedBlocks * b);
    BBL_CUDA(cudaMemcpyAsync(hp.data(), scratch.p, need, cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaMemcpyAsync(theta_out, th.p, sizeof(double) * b, cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < b; ++i) {
        double s = 0.0;
        for (int blk = 0; blk < kRedBlocks; ++blk) s += hp[(size_t)blk * b + i];
        resid_out[i] = std::sqrt(s);
    }
    return BBL_OK;
}

// C = Q16^T W, b = 8: the FP16 first-pass Gram of the FP32 stage on its own.
extern "C" bbl_status bbl_block_gram_f16(int64_t n, int nblocks, const void* basis16, const float* W, double* C,
                                         void* stream) {
    using namespace bbl;
    if (n < 1 || nblocks < 1 || !basis16 || !W || !C) return set_error(BBL_ERR_INVALID_ARG, "block_gram_f16: bad arguments");
    if (!aligned16(basis16) || !aligned16(W))
        return set_error(BBL_ERR_INVALID_ARG, "block_gram_f16: pointers must be 16-byte aligned");
    cudaStream_t st = as_stream(stream);
    DevBuf partials;
    BBL_TRY(gram_half(n, nblocks, basis16, W, C, partials, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    return BBL_OK;
}

// W -= Q C1, then C2 = Q^T W (the updated W), b = 8, FP32: the fused first
// update and second Gram of the FP32 stage on its own.
extern "C" bbl_status bbl_block_update_gram(int64_t n, int nblocks, const float* basis, const double* C1, float* W,
                                            double* C2, void* stream) {
    using namespace bbl;
    if (n < 1 || nblocks < 1 || !basis || !C1 || !W || !C2)
        return set_error(BBL_ERR_INVALID_ARG, "block_update_gram: bad arguments");
    if (!aligned16(basis) || !aligned16(W))
        return set_error(BBL_ERR_INVALID_ARG, "block_update_gram: pointers must be 16-byte aligned");
    if (!update_gram_tc_supports(nblocks))
        return set_error(BBL_ERR_UNSUPPORTED, "block_update_gram: %d blocks (at most 128)", nblocks);
    cudaStream_t st = as_stream(stream);
    DevBuf work;
    BBL_TRY(update_gram_tc(n, nblocks, basis, C1, W, C2, work, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    return BBL_OK;
}

// W -= Q C with the blocks older than the nnew newest read from the FP16 copy
// (b = 8, FP32): the FP32 stage's first-pass update on its own.
extern "C" bbl_status bbl_block_update_f16old(int64_t n, int nblocks, int nnew, const void* basis16,
                                              const float* basis, const double* C, float* W, void* stream) {
    using namespace bbl;
    if (n < 1 || nblocks < 1 || nnew < 0 || !basis16 || !basis || !C || !W)
        return set_error(BBL_ERR_INVALID_ARG, "block_update_f16old: bad arguments");
    if (!aligned16(basis16) || !aligned16(basis) || !aligned16(W))
        return set_error(BBL_ERR_INVALID_ARG, "block_update_f16old: pointers must be 16-byte aligned");
    cudaStream_t st = as_stream(stream);
    DevBuf work;
    BBL_TRY(update_half_old(n, nblocks, nnew, basis16, basis, C, W, work, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    return BBL_OK;
}

// C = Q^T W without modifying W (FP64 coefficients), Q as in bbl_block_reorth.
extern "C" bbl_status bbl_block_gram(int64_t n, int b, int nblocks, bbl_dtype dtype, const void* basis, const void* W,
                                     double* C, void* stream) {
    using namespace bbl;
    if (n < 1 || b < 1 || b > kMaxB || nblocks < 1 || !basis || !W || !C)
        return set_error(BBL_ERR_INVALID_ARG, "block_gram: bad arguments");
    if (dtype != BBL_FP64 && dtype != BBL_FP32) return set_error(BBL_ERR_INVALID_ARG, "block_gram: bad dtype");
    if (!aligned16(basis) || !aligned16(W)) return set_error(BBL_ERR_INVALID_ARG, "block_gram: pointers must be 16-byte aligned");
    cudaStream_t st = as_stream(stream);
    DevBuf partials;
    BBL_TRY(gram(n, b, nblocks, dtype, basis, W, C, partials, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    return BBL_OK;
}
