// S2 / S3 / S5: the tall-skinny dense kernels of the block step.
//
//  gram     C = Q^T W   (Q: nblocks row-major n x b blocks, m = nblocks*b
//                        columns; W: n x b; C: m x b FP64).  Split-K over row
//                        chunks: every CTA reads a chunk of rows once, keeps
//                        W's rows of the current 64-row tile in shared memory
//                        and each thread owns CPT columns of Q (a 16-byte
//                        vector load per row) times all b columns of W.
//                        FP32 data: products summed in FP32 over at most one
//                        64-row tile per thread, tiles and chunks summed in
//                        FP64.  Per-CTA partials are reduced in a fixed order
//                        (deterministic).
//  apply    W (-)= Q C  (thread per row; C staged in shared memory in
//                        256-row tiles; used for the Gram-Schmidt update, for
//                        W R^{-1} in CholQR2 and for the Ritz vectors X = Q S).
//  cholqr2  G = W^T W -> R = chol(G) (one thread, b <= 16) -> W <- W R^{-1},
//           twice; B = R2 R1 (Sec. II.B normalisation, CholQR2 form).
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace bbl {
namespace {

template <typename T, int N>
__device__ __forceinline__ void ldvec(const T* p, T (&out)[N]) {
    if constexpr (N * sizeof(T) == 16) {
        if constexpr (sizeof(T) == 8) {
            double2 x = __ldg(reinterpret_cast<const double2*>(p));
            out[0] = x.x;
            out[1] = x.y;
        } else {
            float4 x = __ldg(reinterpret_cast<const float4*>(p));
            out[0] = x.x;
            out[1] = x.y;
            out[2] = x.z;
            out[3] = x.w;
        }
    } else if constexpr (N * sizeof(T) == 8 && sizeof(T) == 4) {
        float2 x = __ldg(reinterpret_cast<const float2*>(p));
        out[0] = x.x;
        out[1] = x.y;
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) out[q] = __ldg(p + q);
    }
}

constexpr int kRT = 64;    // rows per shared-memory tile in gram
constexpr int kThreads = 256;

// -------------------------------------------------------------------- gram
template <typename T, int B, int CPT>
__global__ void __launch_bounds__(kThreads) gram_kernel(int64_t n, int m, int64_t rows_per_chunk, int TC,
                                                        const T* __restrict__ Q, const T* __restrict__ W,
                                                        double* __restrict__ partial) {
    __shared__ T ws[kRT * B];
    extern __shared__ double sred[];
    const int tid = threadIdx.x;
    const int RS = kThreads / TC;
    const int cg = tid % TC, rs = tid / TC;
    const int a0 = (blockIdx.y * TC + cg) * CPT;
    const bool active = a0 < m;
    const int j = active ? a0 / B : 0, off = a0 % B;
    const T* qb = Q + (int64_t)j * n * B + off;
    double acc64[CPT][B];
#pragma unroll
    for (int i = 0; i < CPT; ++i)
#pragma unroll
        for (int c = 0; c < B; ++c) acc64[i][c] = 0.0;
    const int64_t r_begin = (int64_t)blockIdx.x * rows_per_chunk;
    const int64_t r_end = min(n, r_begin + rows_per_chunk);
    for (int64_t t0 = r_begin; t0 < r_end; t0 += kRT) {
        const int rows = (int)min((int64_t)kRT, r_end - t0);
        __syncthreads();
        for (int e = tid; e < rows * B; e += kThreads) ws[e] = W[t0 * B + e];
        __syncthreads();
        if (active) {
            T acc[CPT][B];
#pragma unroll
            for (int i = 0; i < CPT; ++i)
#pragma unroll
                for (int c = 0; c < B; ++c) acc[i][c] = T(0);
            for (int r = rs; r < rows; r += RS) {
                T q[CPT];
                ldvec<T, CPT>(qb + (t0 + r) * B, q);
                const T* wr = ws + r * B;
#pragma unroll
                for (int c = 0; c < B; ++c) {
                    const T w = wr[c];
#pragma unroll
                    for (int i = 0; i < CPT; ++i) acc[i][c] = fma(q[i], w, acc[i][c]);
                }
            }
#pragma unroll
            for (int i = 0; i < CPT; ++i)
#pragma unroll
                for (int c = 0; c < B; ++c) acc64[i][c] += (double)acc[i][c];
        }
    }
    if (RS > 1) {
        // deterministic tree over the row slots
        double* mine = sred + (size_t)tid * CPT * B;
#pragma unroll
        for (int i = 0; i < CPT; ++i)
#pragma unroll
            for (int c = 0; c < B; ++c) mine[i * B + c] = acc64[i][c];
        __syncthreads();
        for (int s = RS / 2; s > 0; s >>= 1) {
            if (rs < s) {
                const double* other = sred + (size_t)(tid + s * TC) * CPT * B;
                for (int e = 0; e < CPT * B; ++e) mine[e] += other[e];
            }
            __syncthreads();
        }
        if (rs == 0 && active) {
            double* out = partial + ((int64_t)blockIdx.x * m + a0) * B;
            for (int e = 0; e < CPT * B; ++e) out[e] = mine[e];
        }
    } else if (active) {
        double* out = partial + ((int64_t)blockIdx.x * m + a0) * B;
#pragma unroll
        for (int i = 0; i < CPT; ++i)
#pragma unroll
            for (int c = 0; c < B; ++c) out[i * B + c] = acc64[i][c];
    }
}

// any b (runtime), one Q column per thread
template <typename T>
__global__ void __launch_bounds__(kThreads) gram_generic_kernel(int64_t n, int m, int b, int64_t rows_per_chunk, int TC,
                                                                const T* __restrict__ Q, const T* __restrict__ W,
                                                                double* __restrict__ partial) {
    __shared__ T ws[kRT * kMaxB];
    extern __shared__ double sred[];
    const int tid = threadIdx.x;
    const int RS = kThreads / TC;
    const int cg = tid % TC, rs = tid / TC;
    const int a0 = blockIdx.y * TC + cg;
    const bool active = a0 < m;
    const int j = active ? a0 / b : 0, off = a0 % b;
    const T* qb = Q + (int64_t)j * n * b + off;
    double acc64[kMaxB];
    for (int c = 0; c < kMaxB; ++c) acc64[c] = 0.0;
    const int64_t r_begin = (int64_t)blockIdx.x * rows_per_chunk;
    const int64_t r_end = min(n, r_begin + rows_per_chunk);
    for (int64_t t0 = r_begin; t0 < r_end; t0 += kRT) {
        const int rows = (int)min((int64_t)kRT, r_end - t0);
        __syncthreads();
        for (int e = tid; e < rows * b; e += kThreads) ws[e] = W[t0 * b + e];
        __syncthreads();
        if (active) {
            T acc[kMaxB];
            for (int c = 0; c < kMaxB; ++c) acc[c] = T(0);
            for (int r = rs; r < rows; r += RS) {
                const T q = qb[(t0 + r) * b];
                for (int c = 0; c < b; ++c) acc[c] = fma(q, ws[r * b + c], acc[c]);
            }
            for (int c = 0; c < b; ++c) acc64[c] += (double)acc[c];
        }
    }
    double* mine = sred + (size_t)tid * kMaxB;
    for (int c = 0; c < b; ++c) mine[c] = acc64[c];
    __syncthreads();
    for (int s = RS / 2; s > 0; s >>= 1) {
        if (rs < s) {
            const double* other = sred + (size_t)(tid + s * TC) * kMaxB;
            for (int c = 0; c < b; ++c) mine[c] += other[c];
        }
        __syncthreads();
    }
    if (rs == 0 && active) {
        double* out = partial + ((int64_t)blockIdx.x * m + a0) * b;
        for (int c = 0; c < b; ++c) out[c] = mine[c];
    }
}

__global__ void reduce_partials_kernel(int64_t count, int nparts, const double* __restrict__ partial,
                                       double* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += partial[(int64_t)p * count + e];
    out[e] = s;
}

template <typename T, int B, int CPT>
bbl_status launch_gram(int64_t n, int m, const T* Q, const T* W, double* C, DevBuf& partials, cudaStream_t st) {
    int cols = (m + CPT - 1) / CPT;
    int TC = 1;
    while (TC < cols && TC < kThreads) TC <<= 1;
    const int gy = (cols + TC - 1) / TC;
    const int RS = kThreads / TC;
    int64_t target = std::max<int64_t>(1, (152 * 4) / gy);
    int64_t rpc = std::max<int64_t>(kRT * 4, ceil_div(n, target));
    rpc = ceil_div(rpc, kRT) * kRT;
    const int64_t nch = std::max<int64_t>(1, ceil_div(n, rpc));
    const size_t need = sizeof(double) * (size_t)nch * m * B;
    if (partials.bytes < need) BBL_TRY(partials.alloc(need));
    const size_t smem = RS > 1 ? sizeof(double) * kThreads * CPT * B : 0;
    static bool attr_set = false;
    if (!attr_set) {
        BBL_CUDA(cudaFuncSetAttribute(gram_kernel<T, B, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(double) * kThreads * CPT * B)));
        attr_set = true;
    }
    dim3 grid((unsigned)nch, (unsigned)gy);
    gram_kernel<T, B, CPT><<<grid, kThreads, smem, st>>>(n, m, rpc, TC, Q, W, partials.as<double>());
    BBL_LAUNCH_CHECK();
    const int64_t count = (int64_t)m * B;
    reduce_partials_kernel<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(count, (int)nch, partials.as<double>(), C);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

template <typename T>
bbl_status launch_gram_generic(int64_t n, int m, int b, const T* Q, const T* W, double* C, DevBuf& partials,
                               cudaStream_t st) {
    int TC = 1;
    while (TC < m && TC < kThreads) TC <<= 1;
    const int gy = (m + TC - 1) / TC;
    int64_t target = std::max<int64_t>(1, (152 * 4) / gy);
    int64_t rpc = std::max<int64_t>(kRT * 4, ceil_div(n, target));
    rpc = ceil_div(rpc, kRT) * kRT;
    const int64_t nch = std::max<int64_t>(1, ceil_div(n, rpc));
    const size_t need = sizeof(double) * (size_t)nch * m * b;
    if (partials.bytes < need) BBL_TRY(partials.alloc(need));
    const size_t smem = sizeof(double) * kThreads * kMaxB;
    static bool attr_set = false;
    if (!attr_set) {
        BBL_CUDA(cudaFuncSetAttribute(gram_generic_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set = true;
    }
    dim3 grid((unsigned)nch, (unsigned)gy);
    gram_generic_kernel<T><<<grid, kThreads, smem, st>>>(n, m, b, rpc, TC, Q, W, partials.as<double>());
    BBL_LAUNCH_CHECK();
    const int64_t count = (int64_t)m * b;
    reduce_partials_kernel<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(count, (int)nch, partials.as<double>(), C);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

template <typename T>
bbl_status gram_typed(int64_t n, int b, int m, const T* Q, const T* W, double* C, DevBuf& partials, cudaStream_t st) {
    constexpr bool F = sizeof(T) == 4;
    switch (b) {
        case 1: return launch_gram<T, 1, 1>(n, m, Q, W, C, partials, st);
        case 2: return launch_gram<T, 2, 2>(n, m, Q, W, C, partials, st);
        case 4: return launch_gram<T, 4, F ? 4 : 2>(n, m, Q, W, C, partials, st);
        case 8: return launch_gram<T, 8, F ? 4 : 2>(n, m, Q, W, C, partials, st);
        case 16: return launch_gram<T, 16, 2>(n, m, Q, W, C, partials, st);
        default: return launch_gram_generic<T>(n, m, b, Q, W, C, partials, st);
    }
}

// -------------------------------------------------------------------- apply
// W[r][c] (SUB ? -= : =) sum_a Q[r][a] C[a][c], c < kc.  Q: nblocks blocks of
// n x B; C: m x kc FP64 row-major; W: n x kc (type TO).  TA: accumulation type.
constexpr int kKT = 256;
template <typename T, int B, int KCT, bool SUB, typename TA, typename TO>
__global__ void __launch_bounds__(kThreads) apply_kernel(int64_t n, int m, int kc, const T* Q, const double* __restrict__ C,
                                                         TO* W) {
    constexpr int KM = KCT > 0 ? KCT : kMaxB;
    __shared__ TA cs[kKT * KM];
    const int tid = threadIdx.x;
    const int64_t r = (int64_t)blockIdx.x * kThreads + tid;
    TA acc[KM];
#pragma unroll
    for (int c = 0; c < KM; ++c) acc[c] = TA(0);
    for (int a0 = 0; a0 < m; a0 += kKT) {
        const int rows = min(kKT, m - a0);
        __syncthreads();
        for (int e = tid; e < rows * KM; e += kThreads) {
            const int a = e / KM, c = e % KM;
            cs[e] = (c < kc) ? (TA)C[(int64_t)(a0 + a) * kc + c] : TA(0);
        }
        __syncthreads();
        if (r < n) {
            for (int jb = 0; jb < rows; jb += B) {
                const int j = (a0 + jb) / B;
                T q[B];
                if constexpr (B * sizeof(T) >= 16) {
                    constexpr int CH = 16 / (int)sizeof(T);
#pragma unroll
                    for (int ch = 0; ch < B / CH; ++ch) {
                        T t[CH];
                        ldvec<T, CH>(Q + (int64_t)j * n * B + r * B + ch * CH, t);
#pragma unroll
                        for (int q2 = 0; q2 < CH; ++q2) q[ch * CH + q2] = t[q2];
                    }
                } else {
                    ldvec<T, B>(Q + (int64_t)j * n * B + r * B, q);
                }
                const TA* cr = cs + jb * KM;
#pragma unroll
                for (int i = 0; i < B; ++i) {
                    const TA qi = (TA)q[i];
#pragma unroll
                    for (int c = 0; c < KM; ++c) acc[c] = fma(qi, cr[i * KM + c], acc[c]);
                }
            }
        }
    }
    if (r < n) {
#pragma unroll
        for (int c = 0; c < KM; ++c) {
            if (c < kc) {
                TO* w = W + r * kc + c;
                if (SUB) *w = (TO)((TA)(*w) - acc[c]);
                else *w = (TO)acc[c];
            }
        }
    }
}

// any b (runtime)
template <typename T, bool SUB, typename TA, typename TO>
__global__ void __launch_bounds__(kThreads) apply_generic_kernel(int64_t n, int m, int b, int kc, const T* Q,
                                                                 const double* __restrict__ C, TO* W) {
    __shared__ TA cs[kKT * kMaxB];
    const int tid = threadIdx.x;
    const int64_t r = (int64_t)blockIdx.x * kThreads + tid;
    TA acc[kMaxB];
    for (int c = 0; c < kMaxB; ++c) acc[c] = TA(0);
    const int kt = (kKT / b) * b;
    for (int a0 = 0; a0 < m; a0 += kt) {
        const int rows = min(kt, m - a0);
        __syncthreads();
        for (int e = tid; e < rows * kc; e += kThreads) cs[e] = (TA)C[(int64_t)a0 * kc + e];
        __syncthreads();
        if (r < n) {
            for (int a = 0; a < rows; ++a) {
                const int ga = a0 + a;
                const TA q = (TA)Q[(int64_t)(ga / b) * n * b + r * b + ga % b];
                for (int c = 0; c < kc; ++c) acc[c] = fma(q, cs[a * kc + c], acc[c]);
            }
        }
    }
    if (r < n) {
        for (int c = 0; c < kc; ++c) {
            TO* w = W + r * kc + c;
            if (SUB) *w = (TO)((TA)(*w) - acc[c]);
            else *w = (TO)acc[c];
        }
    }
}

template <typename T, bool SUB, typename TA, typename TO>
bbl_status apply_typed(int64_t n, int b, int m, int kc, const T* Q, const double* C, TO* W, cudaStream_t st) {
    const unsigned grid = (unsigned)ceil_div(n, kThreads);
    const bool same = (kc == b);
    if (same) {
        switch (b) {
            case 1: apply_kernel<T, 1, 1, SUB, TA, TO><<<grid, kThreads, 0, st>>>(n, m, kc, Q, C, W); break;
            case 2: apply_kernel<T, 2, 2, SUB, TA, TO><<<grid, kThreads, 0, st>>>(n, m, kc, Q, C, W); break;
            case 4: apply_kernel<T, 4, 4, SUB, TA, TO><<<grid, kThreads, 0, st>>>(n, m, kc, Q, C, W); break;
            case 8: apply_kernel<T, 8, 8, SUB, TA, TO><<<grid, kThreads, 0, st>>>(n, m, kc, Q, C, W); break;
            case 16: apply_kernel<T, 16, 16, SUB, TA, TO><<<grid, kThreads, 0, st>>>(n, m, kc, Q, C, W); break;
            default: apply_generic_kernel<T, SUB, TA, TO><<<grid, kThreads, 0, st>>>(n, m, b, kc, Q, C, W);
        }
    } else {
        switch (b) {
            case 1: apply_kernel<T, 1, 0, SUB, TA, TO><<<grid, kThreads, 0, st>>>(n, m, kc, Q, C, W); break;
            case 2: apply_kernel<T, 2, 0, SUB, TA, TO><<<grid, kThreads, 0, st>>>(n, m, kc, Q, C, W); break;
            case 4: apply_kernel<T, 4, 0, SUB, TA, TO><<<grid, kThreads, 0, st>>>(n, m, kc, Q, C, W); break;
            case 8: apply_kernel<T, 8, 0, SUB, TA, TO><<<grid, kThreads, 0, st>>>(n, m, kc, Q, C, W); break;
            case 16: apply_kernel<T, 16, 0, SUB, TA, TO><<<grid, kThreads, 0, st>>>(n, m, kc, Q, C, W); break;
            default: apply_generic_kernel<T, SUB, TA, TO><<<grid, kThreads, 0, st>>>(n, m, b, kc, Q, C, W);
        }
    }
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

// -------------------------------------------------------------------- Cholesky of the b x b Gram
// status bits: 1 = non-finite Gram.  mask[i] = 1 for deflated columns.
__global__ void chol_kernel(int b, const double* __restrict__ G, double thresh2, int relative, double* __restrict__ R,
                            double* __restrict__ Rinv, int* __restrict__ ndefl, int* __restrict__ mask,
                            int* __restrict__ status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double Rl[kMaxB * kMaxB];
    int dm[kMaxB];
    bool bad = false;
    double gmax = 0.0;
    for (int i = 0; i < b * b; ++i) {
        Rl[i] = 0.0;
        if (!isfinite(G[i])) bad = true;
    }
    for (int i = 0; i < b; ++i) gmax = fmax(gmax, G[i * b + i]);
    if (relative) thresh2 *= gmax;
    int cnt = 0;
    for (int i = 0; i < b; ++i) {
        double d = G[i * b + i];
        for (int l = 0; l < i; ++l) d -= Rl[l * b + i] * Rl[l * b + i];
        dm[i] = !(d > thresh2) || bad;
        if (dm[i]) {
            ++cnt;
            continue;
        }
        const double rii = sqrt(d);
        Rl[i * b + i] = rii;
        for (int k = i + 1; k < b; ++k) {
            double s = G[i * b + k];
            for (int l = 0; l < i; ++l) s -= Rl[l * b + i] * Rl[l * b + k];
            Rl[i * b + k] = s / rii;
        }
    }
    for (int i = 0; i < b * b; ++i) {
        R[i] = Rl[i];
        Rinv[i] = 0.0;
    }
    for (int c = 0; c < b; ++c) {
        if (dm[c]) continue;
        Rinv[c * b + c] = 1.0 / Rl[c * b + c];
        for (int i = c - 1; i >= 0; --i) {
            if (dm[i]) continue;
            double s = 0.0;
            for (int k = i + 1; k <= c; ++k)
                if (!dm[k]) s += Rl[i * b + k] * Rinv[k * b + c];
            Rinv[i * b + c] = -s / Rl[i * b + i];
        }
    }
    if (mask)
        for (int i = 0; i < b; ++i) mask[i] = dm[i];
    if (ndefl) *ndefl += cnt;
    if (bad && status) atomicOr(status, 1);
}

// B = R2 R1 (upper triangular product)
__global__ void trmul_kernel(int b, const double* __restrict__ R2, const double* __restrict__ R1, double* __restrict__ B) {
    const int e = threadIdx.x;
    if (e >= b * b) return;
    const int i = e / b, k = e % b;
    double s = 0.0;
    for (int l = 0; l < b; ++l) s += R2[i * b + l] * R1[l * b + k];
    B[e] = s;
}

}  // namespace

// -------------------------------------------------------------------- internal API
bbl_status gram(int64_t n, int b, int nblocks, int dtype, const void* Q, const void* W, double* C, DevBuf& partials,
                cudaStream_t st) {
    const int m = nblocks * b;
    if (dtype == BBL_FP64)
        return gram_typed<double>(n, b, m, static_cast<const double*>(Q), static_cast<const double*>(W), C, partials, st);
    return gram_typed<float>(n, b, m, static_cast<const float*>(Q), static_cast<const float*>(W), C, partials, st);
}

bbl_status update(int64_t n, int b, int nblocks, int dtype, const void* Q, const double* C, void* W, cudaStream_t st) {
    const int m = nblocks * b;
    if (dtype == BBL_FP64)
        return apply_typed<double, true, double, double>(n, b, m, b, static_cast<const double*>(Q), C,
                                                         static_cast<double*>(W), st);
    return apply_typed<float, true, float, float>(n, b, m, b, static_cast<const float*>(Q), C, static_cast<float*>(W),
                                                  st);
}

bbl_status ritz_vectors(int64_t n, int b, int nblocks, int dtype, const void* Q, int k, const double* S, double* X,
                        cudaStream_t st) {
    const int m = nblocks * b;
    if (dtype == BBL_FP64)
        return apply_typed<double, false, double, double>(n, b, m, k, static_cast<const double*>(Q), S, X, st);
    return apply_typed<float, false, double, double>(n, b, m, k, static_cast<const float*>(Q), S, X, st);
}

// small: >= 8*b*b doubles + 4*b ints.  B (device, b x b) receives R2 R1.
bbl_status cholqr2_dev(int64_t n, int b, int dtype, void* W, double* B, double defl_abs2, int* d_ndefl, int* d_mask,
                       DevBuf& partials, DevBuf& small, cudaStream_t st) {
    const size_t need = sizeof(double) * 8 * kMaxB * kMaxB + sizeof(int) * 4 * kMaxB;
    if (small.bytes < need) BBL_TRY(small.alloc(need));
    double* G = small.as<double>();
    double* R1 = G + kMaxB * kMaxB;
    double* R1i = R1 + kMaxB * kMaxB;
    double* R2 = R1i + kMaxB * kMaxB;
    double* R2i = R2 + kMaxB * kMaxB;
    int* status = reinterpret_cast<int*>(G + 8 * kMaxB * kMaxB);
    const int relative = defl_abs2 < 0 ? 1 : 0;
    const double t1 = relative ? -defl_abs2 : defl_abs2;
    BBL_TRY(gram(n, b, 1, dtype, W, W, G, partials, st));
    chol_kernel<<<1, 32, 0, st>>>(b, G, t1, relative, R1, R1i, d_ndefl, d_mask, status);
    BBL_LAUNCH_CHECK();
    if (dtype == BBL_FP64)
        BBL_TRY((apply_typed<double, false, double, double>(n, b, b, b, static_cast<double*>(W), R1i,
                                                             static_cast<double*>(W), st)));
    else
        BBL_TRY((apply_typed<float, false, float, float>(n, b, b, b, static_cast<float*>(W), R1i,
                                                          static_cast<float*>(W), st)));
    BBL_TRY(gram(n, b, 1, dtype, W, W, G, partials, st));
    // second pass: columns of Q1 have norm ~1; a pivot below 1e-6 means the
    // first pass produced no usable direction (it was deflated or lost).
    chol_kernel<<<1, 32, 0, st>>>(b, G, 1e-6, 0, R2, R2i, nullptr, nullptr, status);
    BBL_LAUNCH_CHECK();
    if (dtype == BBL_FP64)
        BBL_TRY((apply_typed<double, false, double, double>(n, b, b, b, static_cast<double*>(W), R2i,
                                                             static_cast<double*>(W), st)));
    else
        BBL_TRY((apply_typed<float, false, float, float>(n, b, b, b, static_cast<float*>(W), R2i,
                                                          static_cast<float*>(W), st)));
    if (B) {
        trmul_kernel<<<1, 256, 0, st>>>(b, R2, R1, B);
        BBL_LAUNCH_CHECK();
    }
    return BBL_OK;
}

}  // namespace bbl

// -------------------------------------------------------------------- C ABI
extern "C" {

bbl_status bbl_block_reorth(int64_t n, int b, int nblocks, bbl_dtype dtype, const void* basis, void* W, double* coeff,
                            int passes, void* stream) {
    using namespace bbl;
    if (n < 1 || b < 1 || b > kMaxB || nblocks < 1 || passes < 1 || passes > 2 || !basis || !W)
        return set_error(BBL_ERR_INVALID_ARG, "block_reorth: bad arguments");
    if (dtype != BBL_FP64 && dtype != BBL_FP32) return set_error(BBL_ERR_INVALID_ARG, "block_reorth: bad dtype");
    if (!aligned16(basis) || !aligned16(W)) return set_error(BBL_ERR_INVALID_ARG, "block_reorth: pointers must be 16-byte aligned");
    cudaStream_t st = as_stream(stream);
    DevBuf partials, cbuf;
    const int m = nblocks * b;
    double* C = coeff;
    if (!C) {
        BBL_TRY(cbuf.alloc(sizeof(double) * m * b));
        C = cbuf.as<double>();
    }
    for (int p = 0; p < passes; ++p) {
        double* Cp = coeff ? coeff + (size_t)p * m * b : C;
        BBL_TRY(gram(n, b, nblocks, dtype, basis, W, Cp, partials, st));
        BBL_TRY(update(n, b, nblocks, dtype, basis, Cp, W, st));
    }
    BBL_CUDA(cudaStreamSynchronize(st));
    return BBL_OK;
}

bbl_status bbl_cholqr2(int64_t n, int b, bbl_dtype dtype, void* W, double* B, double defl_abs, int* n_deflated,
                       void* stream) {
    using namespace bbl;
    if (n < 1 || b < 1 || b > kMaxB || !W || !B) return set_error(BBL_ERR_INVALID_ARG, "cholqr2: bad arguments");
    if (dtype != BBL_FP64 && dtype != BBL_FP32) return set_error(BBL_ERR_INVALID_ARG, "cholqr2: bad dtype");
    if (!aligned16(W)) return set_error(BBL_ERR_INVALID_ARG, "cholqr2: W must be 16-byte aligned");
    if (defl_abs < 0) return set_error(BBL_ERR_INVALID_ARG, "cholqr2: defl_abs < 0");
    cudaStream_t st = as_stream(stream);
    DevBuf partials, small, cnt;
    BBL_TRY(cnt.alloc(sizeof(int)));
    BBL_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int), st));
    BBL_TRY(small.alloc(sizeof(double) * 8 * kMaxB * kMaxB + sizeof(int) * 4 * kMaxB));
    BBL_CUDA(cudaMemsetAsync(small.p, 0, small.bytes, st));
    BBL_TRY(cholqr2_dev(n, b, dtype, W, B, defl_abs * defl_abs, cnt.as<int>(), nullptr, partials, small, st));
    int h[2] = {0, 0};
    BBL_CUDA(cudaMemcpyAsync(&h[0], cnt.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaMemcpyAsync(&h[1], reinterpret_cast<char*>(small.p) + sizeof(double) * 8 * kMaxB * kMaxB,
                             sizeof(int), cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    if (n_deflated) *n_deflated = h[0];
    if (h[1]) return set_error(BBL_ERR_NUMERICAL, "cholqr2: non-finite Gram matrix");
    return BBL_OK;
}

bbl_status bbl_ritz_vectors(int64_t n, int b, int nblocks, bbl_dtype dtype, const void* basis, int k, const double* S,
                            double* X, void* stream) {
    using namespace bbl;
    if (n < 1 || b < 1 || b > kMaxB || nblocks < 1 || k < 1 || k > kMaxB || !basis || !S || !X)
        return set_error(BBL_ERR_INVALID_ARG, "ritz_vectors: bad arguments");
    if (!aligned16(basis)) return set_error(BBL_ERR_INVALID_ARG, "ritz_vectors: basis must be 16-byte aligned");
    BBL_TRY(ritz_vectors(n, b, nblocks, dtype, basis, k, S, X, as_stream(stream)));
    BBL_CUDA(cudaStreamSynchronize(as_stream(stream)));
    return BBL_OK;
}

}  // extern "C"

// -------------------------------------------------------------------- allocation-free Gram
// For callers that must not allocate device memory: for example a process
// whose device memory is already handed out by a framework's caching
// allocator under a fixed budget, or a latency-critical loop that cannot
// afford the implicit device synchronisation of cudaFree.  The per-chunk
// partial sums of the Gram product live in a fixed file-scope device array
// instead of a cudaMalloc'ed buffer.  Every device that loads this library
// holds the array (8 MiB) until the process exits.
namespace bbl {
namespace {

constexpr int64_t kNoAllocScratchDoubles = int64_t(1) << 20;  // 8 MiB of FP64 partial sums
__device__ __align__(256) double g_noalloc_gram_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array for the current device.  Host code
// only holds a host-side stand-in for the array's name, so the address is
// looked up once per device with that device current.
bbl_status noalloc_scratch(double** out) {
    int dev = 0;
    BBL_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(BBL_ERR_UNSUPPORTED, "block_gram_noalloc: device %d", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_gram_scratch);
        if (e != cudaSuccess || !p)
            return set_error(BBL_ERR_CUDA, "block_gram_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        g_noalloc_addr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_addr[dev];
    return BBL_OK;
}

template <typename T, int B, int CPT>
bbl_status launch_gram_fixed(int64_t n, int m, const T* Q, const T* W, double* C, double* scratch, cudaStream_t st) {
    int cols = (m + CPT - 1) / CPT;
    int TC = 1;
    while (TC < cols && TC < kThreads) TC <<= 1;
    const int gy = (cols + TC - 1) / TC;
    const int RS = kThreads / TC;
    const int64_t per_chunk = (int64_t)m * B;
    if (per_chunk > kNoAllocScratchDoubles)
        return set_error(BBL_ERR_INVALID_ARG,
                         "block_gram_noalloc: nblocks*b*b = %lld exceeds the fixed scratch of %lld doubles",
                         (long long)per_chunk, (long long)kNoAllocScratchDoubles);
    const int64_t max_chunks = kNoAllocScratchDoubles / per_chunk;
    int64_t target = std::max<int64_t>(1, std::min<int64_t>((152 * 4) / gy, max_chunks));
    int64_t rpc = std::max<int64_t>(kRT * 4, ceil_div(n, target));
    rpc = ceil_div(rpc, kRT) * kRT;
    int64_t nch = std::max<int64_t>(1, ceil_div(n, rpc));
    while (nch > max_chunks) {  // grow the chunks until the partials fit
        rpc += kRT;
        nch = ceil_div(n, rpc);
    }
    const size_t smem = RS > 1 ? sizeof(double) * kThreads * CPT * B : 0;
    BBL_CUDA(cudaFuncSetAttribute(gram_kernel<T, B, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(double) * kThreads * CPT * B)));
    dim3 grid((unsigned)nch, (unsigned)gy);
    gram_kernel<T, B, CPT><<<grid, kThreads, smem, st>>>(n, m, rpc, TC, Q, W, scratch);
    BBL_LAUNCH_CHECK();
    reduce_partials_kernel<<<(unsigned)ceil_div(per_chunk, 256), 256, 0, st>>>(per_chunk, (int)nch, scratch, C);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

template <typename T>
bbl_status gram_fixed_typed(int64_t n, int b, int m, const T* Q, const T* W, double* C, double* scratch,
                            cudaStream_t st) {
    constexpr bool F = sizeof(T) == 4;
    switch (b) {
        case 1: return launch_gram_fixed<T, 1, 1>(n, m, Q, W, C, scratch, st);
        case 2: return launch_gram_fixed<T, 2, 2>(n, m, Q, W, C, scratch, st);
        case 4: return launch_gram_fixed<T, 4, F ? 4 : 2>(n, m, Q, W, C, scratch, st);
        case 8: return launch_gram_fixed<T, 8, F ? 4 : 2>(n, m, Q, W, C, scratch, st);
        case 16: return launch_gram_fixed<T, 16, 2>(n, m, Q, W, C, scratch, st);
        default:
            return set_error(BBL_ERR_UNSUPPORTED, "block_gram_noalloc: b=%d (supported: 1, 2, 4, 8, 16)", b);
    }
}

}  // namespace
}  // namespace bbl

extern "C" bbl_status bbl_block_gram_noalloc(int64_t n, int b, int nblocks, bbl_dtype dtype, const void* basis,
                                             const void* W, double* C, void* stream) {
    using namespace bbl;
    if (n < 1 || b < 1 || b > kMaxB || nblocks < 1 || !basis || !W || !C)
        return set_error(BBL_ERR_INVALID_ARG, "block_gram_noalloc: bad arguments");
    if (dtype != BBL_FP64 && dtype != BBL_FP32) return set_error(BBL_ERR_INVALID_ARG, "block_gram_noalloc: bad dtype");
    if (!aligned16(basis) || !aligned16(W))
        return set_error(BBL_ERR_INVALID_ARG, "block_gram_noalloc: pointers must be 16-byte aligned");
    double* scratch = nullptr;
    BBL_TRY(noalloc_scratch(&scratch));
    cudaStream_t st = as_stream(stream);
    const int m = nblocks * b;
    if (dtype == BBL_FP64)
        BBL_TRY(gram_fixed_typed<double>(n, b, m, static_cast<const double*>(basis), static_cast<const double*>(W), C,
                                         scratch, st));
    else
        BBL_TRY(gram_fixed_typed<float>(n, b, m, static_cast<const float*>(basis), static_cast<const float*>(W), C,
                                        scratch, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    return BBL_OK;
}
