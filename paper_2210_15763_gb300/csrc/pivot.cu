// S6: bootstrapped pivot (Sec. II.B "bootstrap", Sec. III).
//
// The paper builds its pivot from approximate lowest eigenvectors computed in
// a truncated model space and projected into the full space.  For matrices
// without a physics basis the truncated space is the set S of the trunc_dim
// rows with the smallest diagonal entries (ties: lower index first):
//   1. threshold search on the order-preserving 64-bit key of H_ii
//      (bisection over the key range, one counting pass per bit);
//   2. stable compaction of S and of the position map pos[i] (device);
//   3. extraction of the principal submatrix H[S,S] as CSR (device);
//   4. its lowest b eigenpairs by this library's own block Lanczos (FP64);
//   5. zero-padded embedding into the n x b pivot.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace bbl {
namespace {

__device__ __forceinline__ unsigned long long order_key(double x) {
    unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void count_below_kernel(int64_t n, const double* __restrict__ d, unsigned long long t,
                                   unsigned long long* __restrict__ cnt) {
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += (order_key(d[i]) < t);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(cnt, c);
}

// flags: 1 if key < t, or key == t and among the first `need_eq` equal keys
// (decided in a second pass with the scan of the equality flags).
__global__ void flag_kernel(int64_t n, const double* __restrict__ d, unsigned long long t, int mode,
                            int* __restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = order_key(d[i]);
        flag[i] = mode == 0 ? (k < t) : (k == t);
    }
}

constexpr int kScanBlock = 1024;

__global__ void block_sum_kernel(int64_t n, const int* __restrict__ flag, int64_t* __restrict__ bsum) {
    __shared__ int64_t red[256];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    int64_t s = 0;
    for (int e = threadIdx.x; e < kScanBlock; e += 256)
        if (base + e < n) s += flag[base + e];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = red[0];
}

// exclusive scan inside each block (sequential per block, 1024 elements) given block offsets
__global__ void block_scan_kernel(int64_t n, const int* __restrict__ flag, const int64_t* __restrict__ boff,
                                  int64_t* __restrict__ pos) {
    __shared__ int64_t s[kScanBlock];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    for (int e = threadIdx.x; e < kScanBlock; e += blockDim.x) s[e] = (base + e < n) ? flag[base + e] : 0;
    __syncthreads();
    // Hillis-Steele inclusive scan
    for (int off = 1; off < kScanBlock; off <<= 1) {
        int64_t v[kScanBlock / 256];
        for (int q = 0; q < kScanBlock / 256; ++q) {
            const int e = threadIdx.x + q * 256;
            v[q] = s[e] + (e >= off ? s[e - off] : 0);
        }
        __syncthreads();
        for (int q = 0; q < kScanBlock / 256; ++q) s[threadIdx.x + q * 256] = v[q];
        __syncthreads();
    }
    for (int e = threadIdx.x; e < kScanBlock; e += blockDim.x)
        if (base + e < n) pos[base + e] = boff[blockIdx.x] + s[e] - ((base + e < n) ? flag[base + e] : 0);
}

// exclusive prefix positions of a 0/1 flag array (device), returns the total
bbl_status scan_flags(int64_t n, const int* flag, int64_t* pos, cudaStream_t st, int64_t* total) {
    const int64_t nb = ceil_div(n, kScanBlock);
    DevBuf bsum;
    BBL_TRY(bsum.alloc(sizeof(int64_t) * (nb + 1)));
    block_sum_kernel<<<(unsigned)nb, 256, 0, st>>>(n, flag, bsum.as<int64_t>());
    BBL_LAUNCH_CHECK();
    std::vector<int64_t> h(nb + 1);
    BBL_CUDA(cudaMemcpyAsync(h.data(), bsum.p, sizeof(int64_t) * nb, cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    int64_t acc = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t t = h[b];
        h[b] = acc;
        acc += t;
    }
    BBL_CUDA(cudaMemcpyAsync(bsum.p, h.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, st));
    block_scan_kernel<<<(unsigned)nb, 256, 0, st>>>(n, flag, bsum.as<int64_t>(), pos);
    BBL_LAUNCH_CHECK();
    BBL_CUDA(cudaStreamSynchronize(st));
    *total = acc;
    return BBL_OK;
}

// sel[i] = flag_lt[i] || (flag_eq[i] && rank_eq[i] < need)
__global__ void select_kernel(int64_t n, const int* __restrict__ flt, const int* __restrict__ feq,
                              const int64_t* __restrict__ req, int64_t need, int* __restrict__ sel) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        sel[i] = flt[i] || (feq[i] && req[i] < need);
}

__global__ void compact_kernel(int64_t n, const int* __restrict__ sel, const int64_t* __restrict__ spos,
                               int* __restrict__ S, int* __restrict__ pos) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (sel[i]) {
            S[spos[i]] = (int)i;
            pos[i] = (int)spos[i];
        } else {
            pos[i] = -1;
        }
    }
}

__global__ void sub_rowlen_kernel(int64_t k, const int* __restrict__ S, const int* __restrict__ pos,
                                  const int64_t* __restrict__ rp, const int* __restrict__ ci, int64_t* __restrict__ len) {
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (s >= k) return;
    const int row = S[s];
    int64_t c = 0;
    for (int64_t e = rp[row] + lane; e < rp[row + 1]; e += 32) c += (pos[ci[e]] >= 0);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if (lane == 0) len[s] = c;
}

template <typename T>
__global__ void sub_fill_kernel(int64_t k, const int* __restrict__ S, const int* __restrict__ pos,
                                const int64_t* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ va,
                                const int64_t* __restrict__ srp, int* __restrict__ sci, double* __restrict__ sva) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= k) return;
    const int row = S[s];
    int64_t o = srp[s];
    for (int64_t e = rp[row]; e < rp[row + 1]; ++e) {
        const int p = pos[ci[e]];
        if (p >= 0) {
            sci[o] = p;
            sva[o] = (double)va[e];
            ++o;
        }
    }
}

__global__ void embed_kernel(int64_t k, int b, int kcols, const int* __restrict__ S, const double* __restrict__ Y,
                             double* __restrict__ P) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < k * kcols;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = e / kcols;
        const int c = (int)(e % kcols);
        P[(int64_t)S[s] * b + c] = Y[e];
    }
}

__global__ void unit_embed_kernel(int64_t k, int b, const int* __restrict__ S, double* __restrict__ P) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s < k) P[(int64_t)S[s] * b + s] = 1.0;
}

__global__ void copy_cols_kernel(int64_t n, int b, int c0, const double* __restrict__ R, double* __restrict__ P) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * (b - c0); e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / (b - c0);
        const int c = c0 + (int)(e % (b - c0));
        P[i * b + c] = R[i * b + c];
    }
}

}  // namespace
}  // namespace bbl

extern "C" bbl_status bbl_pivot_bootstrap(const bbl_matrix* A, int64_t trunc_dim, int b, double sub_tol, uint64_t seed,
                                          double* P, void* stream) {
    using namespace bbl;
    if (!A || !P || b < 1 || b > kMaxB || trunc_dim < 1 || !(sub_tol > 0))
        return set_error(BBL_ERR_INVALID_ARG, "pivot_bootstrap: bad arguments");
    if (!A->has_csr && A->fmt != BBL_KRON)
        return set_error(BBL_ERR_UNSUPPORTED, "pivot_bootstrap: needs the CSR copy of H");
    cudaStream_t st = as_stream(stream);
    const int64_t n = A->n;
    const int64_t k = std::min(trunc_dim, n);
    const unsigned grid = 152 * 8;
    // 1. threshold: smallest key t with count(key < t) >= k  ->  kth key = t - 1
    DevBuf cnt;
    BBL_TRY(cnt.alloc(sizeof(unsigned long long)));
    auto count_below = [&](unsigned long long t, unsigned long long* out) -> bbl_status {
        BBL_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), st));
        count_below_kernel<<<grid, 256, 0, st>>>(n, A->diag.as<double>(), t, cnt.as<unsigned long long>());
        BBL_LAUNCH_CHECK();
        BBL_CUDA(cudaMemcpyAsync(out, cnt.p, sizeof(*out), cudaMemcpyDeviceToHost, st));
        BBL_CUDA(cudaStreamSynchronize(st));
        return BBL_OK;
    };
    // binary search for the k-th smallest key value kth: count(key < kth) < k <= count(key <= kth)
    unsigned long long lo = 0, hi = ~0ull;  // invariant: count(< lo) < k, count(< hi) >= k (or hi = max)
    while (hi - lo > 1) {
        const unsigned long long mid = lo + (hi - lo) / 2;
        unsigned long long c = 0;
        BBL_TRY(count_below(mid, &c));
        if (c >= (unsigned long long)k) hi = mid;
        else lo = mid;
    }
    const unsigned long long kth = lo;  // count(< kth) < k and count(< kth + 1) >= k
    unsigned long long nless = 0;
    BBL_TRY(count_below(kth, &nless));
    const int64_t need_eq = k - (int64_t)nless;
    // 2. flags, ranks, compaction
    DevBuf flt, feq, req, sel, spos, Sidx, pos;
    BBL_TRY(flt.alloc(sizeof(int) * n));
    BBL_TRY(feq.alloc(sizeof(int) * n));
    BBL_TRY(req.alloc(sizeof(int64_t) * n));
    BBL_TRY(sel.alloc(sizeof(int) * n));
    BBL_TRY(spos.alloc(sizeof(int64_t) * n));
    BBL_TRY(Sidx.alloc(sizeof(int) * k));
    BBL_TRY(pos.alloc(sizeof(int) * n));
    flag_kernel<<<grid, 256, 0, st>>>(n, A->diag.as<double>(), kth, 0, flt.as<int>());
    flag_kernel<<<grid, 256, 0, st>>>(n, A->diag.as<double>(), kth, 1, feq.as<int>());
    BBL_LAUNCH_CHECK();
    int64_t tot = 0;
    BBL_TRY(scan_flags(n, feq.as<int>(), req.as<int64_t>(), st, &tot));
    select_kernel<<<grid, 256, 0, st>>>(n, flt.as<int>(), feq.as<int>(), req.as<int64_t>(), need_eq, sel.as<int>());
    BBL_LAUNCH_CHECK();
    BBL_TRY(scan_flags(n, sel.as<int>(), spos.as<int64_t>(), st, &tot));
    if (tot != k) return set_error(BBL_ERR_NUMERICAL, "pivot_bootstrap: selected %lld of %lld rows", (long long)tot, (long long)k);
    compact_kernel<<<grid, 256, 0, st>>>(n, sel.as<int>(), spos.as<int64_t>(), Sidx.as<int>(), pos.as<int>());
    BBL_LAUNCH_CHECK();
    BBL_CUDA(cudaMemsetAsync(P, 0, sizeof(double) * n * b, st));
    const int kc = (int)std::min<int64_t>(k, b);
    if (k <= b) {
        // the truncated space is spanned by the unit vectors of S
        unit_embed_kernel<<<(unsigned)ceil_div(k, 256), 256, 0, st>>>(k, b, Sidx.as<int>(), P);
        BBL_LAUNCH_CHECK();
    } else {
        // 3. H[S,S] as CSR (of a factored matrix: from its expanded rows)
        DevBuf len, srp, sci, sva;
        int64_t acc = 0;
        if (A->fmt == BBL_KRON) {
            BBL_TRY(kron_submatrix(A, k, Sidx.as<int>(), pos.as<int>(), srp, sci, sva, &acc, st));
        } else {
        BBL_TRY(len.alloc(sizeof(int64_t) * (k + 1)));
        sub_rowlen_kernel<<<(unsigned)ceil_div(k * 32, 256), 256, 0, st>>>(k, Sidx.as<int>(), pos.as<int>(),
                                                                           A->row_ptr.as<int64_t>(), A->col.as<int>(),
                                                                           len.as<int64_t>());
        BBL_LAUNCH_CHECK();
        std::vector<int64_t> h(k + 1);
        BBL_CUDA(cudaMemcpyAsync(h.data(), len.p, sizeof(int64_t) * k, cudaMemcpyDeviceToHost, st));
        BBL_CUDA(cudaStreamSynchronize(st));
        for (int64_t s = 0; s < k; ++s) {
            const int64_t t = h[s];
            h[s] = acc;
            acc += t;
        }
        h[k] = acc;
        BBL_TRY(srp.alloc(sizeof(int64_t) * (k + 1)));
        BBL_TRY(sci.alloc(sizeof(int) * std::max<int64_t>(acc, 1)));
        BBL_TRY(sva.alloc(sizeof(double) * std::max<int64_t>(acc, 1)));
        BBL_CUDA(cudaMemcpyAsync(srp.p, h.data(), sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice, st));
        if (A->storage == BBL_FP64)
            sub_fill_kernel<double><<<(unsigned)ceil_div(k, 256), 256, 0, st>>>(
                k, Sidx.as<int>(), pos.as<int>(), A->row_ptr.as<int64_t>(), A->col.as<int>(), A->val.as<double>(),
                srp.as<int64_t>(), sci.as<int>(), sva.as<double>());
        else
            sub_fill_kernel<float><<<(unsigned)ceil_div(k, 256), 256, 0, st>>>(
                k, Sidx.as<int>(), pos.as<int>(), A->row_ptr.as<int64_t>(), A->col.as<int>(), A->val.as<float>(),
                srp.as<int64_t>(), sci.as<int>(), sva.as<double>());
        BBL_LAUNCH_CHECK();
        BBL_CUDA(cudaStreamSynchronize(st));
        }
        // 4. lowest b eigenpairs of H[S,S]: a sub-solve to sub_tol >= 1e-5 from
        // FP32 values runs in FP32 storage without the polish (its tolerance is
        // far above the FP32 stage's floor, and FP64 arithmetic runs at 1/64 of
        // the FP32 rate), tighter ones in FP64
        const bool sub32 = A->storage == BBL_FP32 && sub_tol >= 1e-5;
        bbl_matrix* sub = nullptr;
        BBL_TRY(bbl_matrix_create(k, acc, srp.as<int64_t>(), sci.as<int>(), sva.p, BBL_FP64, sub32 ? BBL_FP32 : BBL_FP64,
                                  BBL_CSR, 0, 0, 0, stream, &sub));
        bbl_options o;
        bbl_options_default(&o);
        o.tol = sub_tol;
        o.seed = seed;
        o.stream = stream;
        o.storage = sub32 ? BBL_FP32 : BBL_FP64;
        o.polish = 0;
        // a truncated space is small: its blocks take tens of microseconds, so
        // a Ritz solve beside them would only let the run overshoot its test
        o.ritz_overlap = 0;
        const int bs = (int)std::min<int64_t>(b, k);
        o.max_vectors = (int)std::min<int64_t>((k / bs) * bs, 2000);
        DevBuf Y;
        std::vector<double> ev(bs), rs(bs);
        bbl_status s = Y.alloc(sizeof(double) * k * bs);
        if (s == BBL_OK) s = bbl_solve(sub, bs, bs, nullptr, &o, ev.data(), Y.as<double>(), rs.data(), nullptr);
        bbl_matrix_destroy(sub);
        if (s != BBL_OK && s != BBL_ERR_NOT_CONVERGED) return s;
        clear_error();
        // 5. embed
        embed_kernel<<<grid, 256, 0, st>>>(k, b, bs, Sidx.as<int>(), Y.as<double>(), P);
        BBL_LAUNCH_CHECK();
    }
    if (kc < b) {
        // more columns than the truncated space holds: random columns
        DevBuf R;
        BBL_TRY(R.alloc(sizeof(double) * n * b));
        BBL_TRY(fill_normal(n, b, seed, 0, R.as<double>(), st));
        copy_cols_kernel<<<grid, 256, 0, st>>>(n, b, kc, R.as<double>(), P);
        BBL_LAUNCH_CHECK();
    }
    BBL_CUDA(cudaStreamSynchronize(st));
    return BBL_OK;
}
