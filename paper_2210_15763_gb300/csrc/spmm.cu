// S1: sparse matrix x dense block, W = H V (Sec. II.B, Eq. 3).
//
// Blocks are n x b row-major, so each stored nonzero H_ij reads the b
// contiguous values V[j, 0:b] (the paper's "loop over a innermost" with the
// vector index contiguous, Eqs. 3-5), here as 16-byte vector loads.
//
//  * CSR: a group of G lanes per row (G = 32 for long rows: a warp per row).
//    Inside a group, LPN = b*sizeof(T)/16 lanes share one nonzero (each loads
//    16 bytes of V[j, :]) and G/LPN nonzeros are in flight per step; the
//    partial sums are combined with xor shuffles at the end of the row.
//  * SELL-C-sigma (C = 32): a warp per slice of 32 rows, one lane per row,
//    column-major slices so that the index/value loads of a warp are one
//    coalesced 128-byte (FP32) transaction per step.
//
// Template parameters: TM = stored value type, TX = vector type (and the
// accumulation type).  FP64 storage uses <double, double>; the
// mixed-precision form uses <float, float>; its FP64 residual product uses
// <float, double>.
#include <type_traits>

#include "common.cuh"
#include "df32.cuh"

namespace bbl {
namespace {

template <typename TX, int B>
struct VecLayout {
    static constexpr int bytes = B * (int)sizeof(TX);
    static constexpr int LPN = bytes >= 16 ? bytes / 16 : 1;  // lanes per nonzero
    static constexpr int VEC = B / LPN;                       // values per lane
};

template <typename T, int N>
struct alignas(N * sizeof(T) >= 16 ? 16 : N * sizeof(T)) Pack {
    T v[N];
};

// type of the matrix value in the product: float-float blocks multiply by the
// FP32 value itself
template <typename TM, typename TX>
using HType = std::conditional_t<is_df32<TX>::value, float, TX>;

template <typename T, int N>
__device__ __forceinline__ void load_pack(const T* __restrict__ p, T (&out)[N]) {
    if constexpr (is_df32<T>::value) {
        if constexpr (N % 2 == 0) {
#pragma unroll
            for (int q = 0; q < N; q += 2) {
                const float4 x = __ldg(reinterpret_cast<const float4*>(p + q));
                out[q] = df32(x.x, x.y);
                out[q + 1] = df32(x.z, x.w);
            }
        } else {
#pragma unroll
            for (int q = 0; q < N; ++q) {
                const float2 x = __ldg(reinterpret_cast<const float2*>(p + q));
                out[q] = df32(x.x, x.y);
            }
        }
    } else if constexpr (N * sizeof(T) == 16) {
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

template <typename T, int N>
__device__ __forceinline__ void store_pack(T* p, const T (&v)[N]) {
    if constexpr (is_df32<T>::value) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            const df32 r = dfm::renorm(v[q].hi, v[q].lo);
            *reinterpret_cast<float2*>(p + q) = make_float2(r.hi, r.lo);
        }
    } else if constexpr (N * sizeof(T) == 16) {
        if constexpr (sizeof(T) == 8) {
            *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
        } else {
            *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) p[q] = v[q];
    }
}

// CSR, G lanes per row (G a power of two, LPN <= G <= 32).
template <typename TM, typename TX, int B, int G>
__global__ void __launch_bounds__(256) spmm_csr_kernel(int64_t n, const int64_t* __restrict__ rp,
                                                       const int* __restrict__ ci, const TM* __restrict__ va,
                                                       const TX* __restrict__ V, TX* __restrict__ W) {
    using L = VecLayout<TX, B>;
    constexpr int LPN = L::LPN, VEC = L::VEC, NPS = G / LPN;
    static_assert(G >= LPN && (G & (G - 1)) == 0 && G <= 32, "group size");
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    if (row >= n) return;  // the whole group leaves together
    const int sub = gl % LPN;
    const int slot = gl / LPN;
    const int64_t s = rp[row], e = rp[row + 1];
    TX acc[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[q] = TX(0);
#pragma unroll 4
    for (int64_t k = s + slot; k < e; k += NPS) {
        const int c = __ldg(ci + k);
        const HType<TM, TX> h = (HType<TM, TX>)__ldg(va + k);
        TX v[VEC];
        load_pack<TX, VEC>(V + (int64_t)c * B + sub * VEC, v);
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc[q] = fma(h, v[q], acc[q]);
    }
#pragma unroll
    for (int off = LPN; off < G; off <<= 1) {
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc[q] += shfl_xor_any(gmask, acc[q], off);
    }
    if (slot == 0) store_pack<TX, VEC>(W + row * B + sub * VEC, acc);
}

// CSR, any b in 1..16 (runtime), a warp per row, scalar loads.
template <typename TM, typename TX>
__global__ void __launch_bounds__(256) spmm_csr_generic(int64_t n, int b, const int64_t* __restrict__ rp,
                                                        const int* __restrict__ ci, const TM* __restrict__ va,
                                                        const TX* __restrict__ V, TX* __restrict__ W) {
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (row >= n) return;
    TX acc[kMaxB];
#pragma unroll
    for (int q = 0; q < kMaxB; ++q) acc[q] = TX(0);
    for (int64_t k = rp[row] + lane; k < rp[row + 1]; k += 32) {
        const int c = ci[k];
        const HType<TM, TX> h = (HType<TM, TX>)va[k];
#pragma unroll
        for (int q = 0; q < kMaxB; ++q)
            if (q < b) acc[q] = fma(h, V[(int64_t)c * b + q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < kMaxB; ++q) {
        TX x = acc[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += shfl_xor_any(0xffffffffu, x, off);
        acc[q] = x;
    }
    if (lane < b) {
        TX out = acc[0];
#pragma unroll
        for (int q = 1; q < kMaxB; ++q)
            if (q == lane) out = acc[q];
        if constexpr (is_df32<TX>::value) W[row * b + lane] = dfm::renorm(out.hi, out.lo);
        else W[row * b + lane] = out;
    }
}

// SELL-C-sigma: LPR = b*sizeof(TX)/16 lanes share a row (each loads 16
// bytes of the gathered row of V, so one warp load covers whole rows and the
// L1 serves one line per nonzero), a warp covers 32/LPR rows of a slice and
// LPR warps cover the 32-row slice.  The index and value loads of a warp are
// consecutive (lanes of a row read the same word).  Output row = perm[slot].
template <typename TM, typename TX, int B>
__global__ void __launch_bounds__(256) spmm_sell_kernel(int64_t nslices, const int64_t* __restrict__ sp,
                                                        const int* __restrict__ sc, const TM* __restrict__ sv,
                                                        const int* __restrict__ slen, const int* __restrict__ perm,
                                                        const TX* __restrict__ V, TX* __restrict__ W) {
    using L = VecLayout<TX, B>;
    constexpr int LPR = L::LPN, VEC = L::VEC;
    constexpr int RPP = 32 / LPR;  // rows per warp pass
    static_assert(LPR >= 1 && LPR <= 32 && (32 % LPR) == 0, "sell lane groups");
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int64_t s = gw / LPR;
    if (s >= nslices) return;
    const int r = (int)(gw % LPR) * RPP + lane / LPR;  // row within the slice
    const int part = lane % LPR;
    const int64_t slot = s * kSellC + r;
    const int len = slen[slot];
    const int64_t base = sp[s] + r;
    TX acc[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[q] = TX(0);
    // Each nonzero is a dependent pair of loads (column index, then the
    // gathered row of V).  Batches of U nonzeros: the gathers of a batch are
    // issued together, and the index/value loads of the next batch are issued
    // before this batch's products, so the two latencies overlap.
    constexpr int U = 8;
    int k = 0;
    int cn[U];
    HType<TM, TX> hn[U];
    if (U <= len) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            cn[u] = __ldg(sc + base + (int64_t)u * kSellC);
            hn[u] = (HType<TM, TX>)__ldg(sv + base + (int64_t)u * kSellC);
        }
    }
    for (; k + U <= len; k += U) {
        int c[U];
        HType<TM, TX> h[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            c[u] = cn[u];
            h[u] = hn[u];
        }
        TX v[U][VEC];
#pragma unroll
        for (int u = 0; u < U; ++u) load_pack<TX, VEC>(V + (int64_t)c[u] * B + part * VEC, v[u]);
        if (k + 2 * U <= len) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                cn[u] = __ldg(sc + base + (int64_t)(k + U + u) * kSellC);
                hn[u] = (HType<TM, TX>)__ldg(sv + base + (int64_t)(k + U + u) * kSellC);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < VEC; ++q) acc[q] = fma(h[u], v[u][q], acc[q]);
    }
    for (; k < len; ++k) {
        const int c = __ldg(sc + base + (int64_t)k * kSellC);
        const HType<TM, TX> h = (HType<TM, TX>)__ldg(sv + base + (int64_t)k * kSellC);
        TX v[VEC];
        load_pack<TX, VEC>(V + (int64_t)c * B + part * VEC, v);
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc[q] = fma(h, v[q], acc[q]);
    }
    const int row = perm[slot];
    if (row >= 0) store_pack<TX, VEC>(W + (int64_t)row * B + part * VEC, acc);
}

template <typename TM, typename TX>
__global__ void __launch_bounds__(256) spmm_sell_generic(int64_t nslices, int b, const int64_t* __restrict__ sp,
                                                         const int* __restrict__ sc, const TM* __restrict__ sv,
                                                         const int* __restrict__ slen, const int* __restrict__ perm,
                                                         const TX* __restrict__ V, TX* __restrict__ W) {
    const int lane = threadIdx.x & 31;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (s >= nslices) return;
    const int64_t slot = s * kSellC + lane;
    const int len = slen[slot];
    const int64_t base = sp[s] + lane;
    TX acc[kMaxB];
#pragma unroll
    for (int q = 0; q < kMaxB; ++q) acc[q] = TX(0);
    for (int k = 0; k < len; ++k) {
        const int c = sc[base + (int64_t)k * kSellC];
        const HType<TM, TX> h = (HType<TM, TX>)sv[base + (int64_t)k * kSellC];
#pragma unroll
        for (int q = 0; q < kMaxB; ++q)
            if (q < b) acc[q] = fma(h, V[(int64_t)c * b + q], acc[q]);
    }
    const int row = perm[slot];
    if (row >= 0) {
#pragma unroll
        for (int q = 0; q < kMaxB; ++q)
            if (q < b) {
                if constexpr (is_df32<TX>::value) W[(int64_t)row * b + q] = dfm::renorm(acc[q].hi, acc[q].lo);
                else W[(int64_t)row * b + q] = acc[q];
            }
    }
}

// rows [r0, r0 + nr) of the CSR matrix (the whole matrix: r0 = 0, nr = n)
struct CsrRows {
    int64_t nr;
    const int64_t* rp;  // row pointers from row r0
    const int* ci;
    int64_t r0;
};

template <typename TM, typename TX, int B, int G>
void launch_csr(const CsrRows& R, const TM* val, const TX* V, TX* W, cudaStream_t st) {
    const int64_t threads = R.nr * G;
    const int64_t blocks = ceil_div(threads, 256);
    spmm_csr_kernel<TM, TX, B, G><<<(unsigned)blocks, 256, 0, st>>>(R.nr, R.rp, R.ci, val, V, W + R.r0 * B);
}

template <typename TM, typename TX, int B>
void launch_csr_g(const CsrRows& R, const TM* val, const TX* V, TX* W, int G, cudaStream_t st) {
    constexpr int LPN = VecLayout<TX, B>::LPN;
    if (G < LPN) G = LPN;
    switch (G) {
        case 1: if constexpr (LPN <= 1) { launch_csr<TM, TX, B, 1>(R, val, V, W, st); return; } break;
        case 2: if constexpr (LPN <= 2) { launch_csr<TM, TX, B, 2>(R, val, V, W, st); return; } break;
        case 4: if constexpr (LPN <= 4) { launch_csr<TM, TX, B, 4>(R, val, V, W, st); return; } break;
        case 8: if constexpr (LPN <= 8) { launch_csr<TM, TX, B, 8>(R, val, V, W, st); return; } break;
        case 16: launch_csr<TM, TX, B, 16>(R, val, V, W, st); return;
        default: break;
    }
    launch_csr<TM, TX, B, 32>(R, val, V, W, st);
}

// Lanes per row: about the average row length / 2, clamped to [LPN, 32].
int default_group(const bbl_matrix* A) {
    const double avg = A->n ? (double)A->nnz / (double)A->n : 0.0;
    if (avg >= 48) return 32;
    if (avg >= 24) return 16;
    if (avg >= 12) return 8;
    if (avg >= 6) return 4;
    return 2;
}

template <typename TM, typename TX>
bbl_status spmm_typed(const bbl_matrix* A, int b, const TM* csr_val, const TM* sell_val, const TX* V, TX* W,
                      cudaStream_t st, int G, int64_t r0 = 0, int64_t r1 = -1) {
    if (G <= 0) G = A->spmm_lanes > 0 ? A->spmm_lanes : default_group(A);
    const bool pow2 = (b == 1 || b == 2 || b == 4 || b == 8 || b == 16);
    const bool ranged = r1 >= 0;  // rows [r0, r1) only, from the CSR copy
    if (r1 < 0) r1 = A->n;
    if (A->fmt == BBL_SELL && sell_val && !ranged) {
        const int64_t blocks = ceil_div(A->nslices * 32, 256);
        auto sp = A->slice_ptr.as<int64_t>();
        auto sc = A->sell_col.as<int>();
        auto sl = A->sell_len.as<int>();
        auto pm = A->perm.as<int>();
        auto sell_blocks = [&](int lpr) { return (unsigned)ceil_div(A->nslices * 32 * lpr, 256); };
        switch (pow2 ? b : 0) {
            case 1: spmm_sell_kernel<TM, TX, 1><<<sell_blocks(VecLayout<TX, 1>::LPN), 256, 0, st>>>(A->nslices, sp, sc, sell_val, sl, pm, V, W); break;
            case 2: spmm_sell_kernel<TM, TX, 2><<<sell_blocks(VecLayout<TX, 2>::LPN), 256, 0, st>>>(A->nslices, sp, sc, sell_val, sl, pm, V, W); break;
            case 4: spmm_sell_kernel<TM, TX, 4><<<sell_blocks(VecLayout<TX, 4>::LPN), 256, 0, st>>>(A->nslices, sp, sc, sell_val, sl, pm, V, W); break;
            case 8: spmm_sell_kernel<TM, TX, 8><<<sell_blocks(VecLayout<TX, 8>::LPN), 256, 0, st>>>(A->nslices, sp, sc, sell_val, sl, pm, V, W); break;
            case 16: spmm_sell_kernel<TM, TX, 16><<<sell_blocks(VecLayout<TX, 16>::LPN), 256, 0, st>>>(A->nslices, sp, sc, sell_val, sl, pm, V, W); break;
            default:
                spmm_sell_generic<TM, TX><<<(unsigned)blocks, 256, 0, st>>>(A->nslices, b, sp, sc, sell_val, sl, pm, V, W);
        }
        BBL_LAUNCH_CHECK();
        return BBL_OK;
    }
    if (!A->has_csr || !csr_val) return set_error(BBL_ERR_UNSUPPORTED, "spmm: matrix holds no CSR values of this type");
    const CsrRows R{r1 - r0, A->row_ptr.as<int64_t>() + r0, A->col.as<int>(), r0};
    if (R.nr <= 0) return BBL_OK;
    switch (pow2 ? b : 0) {
        case 1: launch_csr_g<TM, TX, 1>(R, csr_val, V, W, G, st); break;
        case 2: launch_csr_g<TM, TX, 2>(R, csr_val, V, W, G, st); break;
        case 4: launch_csr_g<TM, TX, 4>(R, csr_val, V, W, G, st); break;
        case 8: launch_csr_g<TM, TX, 8>(R, csr_val, V, W, G, st); break;
        case 16: launch_csr_g<TM, TX, 16>(R, csr_val, V, W, G, st); break;
        default: {
            const int64_t blocks = ceil_div(R.nr * 32, 256);
            spmm_csr_generic<TM, TX><<<(unsigned)blocks, 256, 0, st>>>(R.nr, b, R.rp, R.ci, csr_val, V, W + r0 * b);
        }
    }
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

}  // namespace

bbl_status spmm_dispatch(const bbl_matrix* A, int b, const void* V, void* W, bool f64_arith, cudaStream_t st,
                         int G) {
    if (A->fmt == BBL_KRON) return kron_spmm(A, b, (f64_arith || A->storage == BBL_FP64) ? BBL_FP64 : BBL_FP32, V, W, st);
    {
        const int dt = (f64_arith || A->storage == BBL_FP64) ? BBL_FP64 : BBL_FP32;
        if (G <= 0 && tiled_supports(A, b, dt)) return tiled_spmm(A, b, dt, V, W, st);
    }
    if (A->storage == BBL_FP64) {
        return spmm_typed<double, double>(A, b, A->has_csr ? A->val.as<double>() : nullptr,
                                          A->fmt == BBL_SELL ? A->sell_val.as<double>() : nullptr,
                                          static_cast<const double*>(V), static_cast<double*>(W), st, G);
    }
    if (!f64_arith) {
        return spmm_typed<float, float>(A, b, A->has_csr ? A->val.as<float>() : nullptr,
                                        A->fmt == BBL_SELL ? A->sell_val.as<float>() : nullptr,
                                        static_cast<const float*>(V), static_cast<float*>(W), st, G);
    }
    if (A->val64.p && A->has_csr) {
        // FP64 arithmetic on the FP64 copy of the values (CSR)
        return spmm_typed<double, double>(A, b, A->val64.as<double>(), nullptr, static_cast<const double*>(V),
                                          static_cast<double*>(W), st, G);
    }
    // FP64 arithmetic on FP32-stored values (exact: the values are FP32 numbers)
    return spmm_typed<float, double>(A, b, A->has_csr ? A->val.as<float>() : nullptr,
                                     A->fmt == BBL_SELL ? A->sell_val.as<float>() : nullptr,
                                     static_cast<const double*>(V), static_cast<double*>(W), st, G);
}

bbl_status spmm_rows_f64(const bbl_matrix* A, int b, const double* V, double* W, int64_t r0, int64_t r1,
                         cudaStream_t st) {
    if (A->fmt == BBL_KRON || !A->has_csr)
        return set_error(BBL_ERR_UNSUPPORTED, "spmm: a row range needs the CSR copy of the matrix");
    if (r0 < 0 || r1 > A->n || r0 > r1) return set_error(BBL_ERR_INVALID_ARG, "spmm: bad row range");
    if (A->storage == BBL_FP64)
        return spmm_typed<double, double>(A, b, A->val.as<double>(), nullptr, V, W, st, 0, r0, r1);
    return spmm_typed<float, double>(A, b, A->val.as<float>(), nullptr, V, W, st, 0, r0, r1);
}

bbl_status spmm_df32(const bbl_matrix* A, int b, const void* V, void* W, cudaStream_t st) {
    if (A->storage != BBL_FP32)
        return set_error(BBL_ERR_UNSUPPORTED, "spmm: float-float blocks need FP32 matrix values");
    if (A->fmt == BBL_KRON) return kron_spmm(A, b, kDF32, V, W, st);
    if (tiled_supports(A, b, kDF32)) return tiled_spmm(A, b, kDF32, V, W, st);
    return spmm_typed<float, df32>(A, b, A->has_csr ? A->val.as<float>() : nullptr,
                                   A->fmt == BBL_SELL ? A->sell_val.as<float>() : nullptr, static_cast<const df32*>(V),
                                   static_cast<df32*>(W), st, 0);
}

}  // namespace bbl

extern "C" {

static bbl_status check_spmm_args(const bbl_matrix* A, int b, const void* V, const void* W) {
    if (!A) return bbl::set_error(BBL_ERR_INVALID_ARG, "spmm: matrix is NULL");
    if (b < 1 || b > bbl::kMaxB) return bbl::set_error(BBL_ERR_INVALID_ARG, "spmm: b=%d outside 1..16", b);
    if (!V || !W) return bbl::set_error(BBL_ERR_INVALID_ARG, "spmm: V or W is NULL");
    if (!bbl::aligned16(V) || !bbl::aligned16(W))
        return bbl::set_error(BBL_ERR_INVALID_ARG, "spmm: V and W must be 16-byte aligned");
    if (V == W) return bbl::set_error(BBL_ERR_INVALID_ARG, "spmm: V and W must not alias");
    return BBL_OK;
}

bbl_status bbl_spmm(const bbl_matrix* A, int b, const void* V, void* W, void* stream) {
    BBL_TRY(check_spmm_args(A, b, V, W));
    return bbl::spmm_dispatch(A, b, V, W, false, bbl::as_stream(stream));
}

bbl_status bbl_spmm_f64(const bbl_matrix* A, int b, const double* V, double* W, void* stream) {
    BBL_TRY(check_spmm_args(A, b, V, W));
    return bbl::spmm_dispatch(A, b, V, W, true, bbl::as_stream(stream));
}

// Test / autotuning hook: CSR SpMM with an explicit number of lanes per row.
bbl_status bbl_spmm_group(const bbl_matrix* A, int b, const void* V, void* W, int lanes_per_row, void* stream) {
    BBL_TRY(check_spmm_args(A, b, V, W));
    if (lanes_per_row < 1 || lanes_per_row > 32 || (lanes_per_row & (lanes_per_row - 1)))
        return bbl::set_error(BBL_ERR_INVALID_ARG, "spmm: lanes_per_row must be a power of two in 1..32");
    return bbl::spmm_dispatch(A, b, V, W, false, bbl::as_stream(stream), lanes_per_row);
}

}  // extern "C"
