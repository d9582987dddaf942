// Kronecker-factored operator: W = H V without storing H (Sec. I, Sec. III.A,
// Appendix A: the matrix elements are rebuilt on the fly from factors, and
// the rebuilding is shared by the b vectors of a block, Eq. 3 with the
// vector index innermost).
//
// H = Hp (x) I_nN + I_nP (x) Hn + sum_k Cp_k (x) Cn_k, with row r = p*nN + q.
// With V viewed as nP slabs V[p'] of nN x b (row-major, contiguous), output
// slab p is
//
//   W[p] = sum_{p'} Hp[p,p'] V[p']  +  Hn V[p]  +  sum_k Cn_k U_k,
//   U_k  = sum_{p'} Cp_k[p,p'] V[p'],
//
// so every coupling term costs two short sparse products instead of the
// c_p*c_n stored entries per row of its expansion.  One CTA forms one output
// slab (or a group of its columns): the p-row combinations (Hp, Cp_k) are
// streaming, coalesced reads of whole slabs (V, 64 MB at n = 2e6, b = 8 in
// FP32, stays in L2), and the n-factor products (Hn, Cn_k) gather rows of a
// slab staged in shared memory.  Only V and W touch HBM.
//
// The same file builds what the rest of the library needs from such a
// matrix: diag(H), ||H||_inf and the number of nonzeros of the expansion (for
// the convergence scale and the throughput figures), and the principal
// submatrix H[S,S] of the bootstrapped pivot.  Those walk the expanded rows:
// one warp per row writes the row's term contributions (column, term) to
// shared memory, sorts them by (column, term) with a bitonic network and
// sums equal columns in term order (Hp, Hn, Cp_0 Cn_0, ...), in FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "df32.cuh"

namespace bbl {
namespace {

// Factors as the kernels see them (passed by value).
struct KronDesc {
    int nP, nN, K;
    int ptr_off[kKronMaxFactors];  // factor f: row pointers at ptr + ptr_off[f]
    int nz_off[kKronMaxFactors];   // columns / values at col / v + nz_off[f]
    const int* ptr;
    const int* col;
    const float* v32;
    const double* v64;
};

// factor index of Hp, Hn, Cp_k, Cn_k
__host__ __device__ constexpr int fHp() { return 0; }
__host__ __device__ constexpr int fHn() { return 1; }
__host__ __device__ constexpr int fCp(int k) { return 2 + 2 * k; }
__host__ __device__ constexpr int fCn(int k) { return 3 + 2 * k; }

KronDesc make_desc(const bbl_matrix* A) {
    KronDesc d{};
    d.nP = (int)A->kron_nP;
    d.nN = (int)A->kron_nN;
    d.K = A->kron_K;
    for (int f = 0; f < 2 + 2 * A->kron_K; ++f) {
        d.ptr_off[f] = (int)A->kf_ptr_off[f];
        d.nz_off[f] = (int)A->kf_nz_off[f];
    }
    d.ptr = A->kf_ptr.as<int>();
    d.col = A->kf_col.as<int>();
    d.v32 = A->kf_val32.as<float>();
    d.v64 = A->kf_val64.as<double>();
    return d;
}

// ------------------------------------------------------------------ expanded rows
// Term t of row (p, q): t = 0 is Hp row p times the unit entry (q, q);
// t = 1 the unit entry (p, p) times Hn row q; t = 2 + k is Cp_k row p times
// Cn_k row q.  Lane t of a warp describes term t (at most 32 terms).
struct TermRow {
    int a0 = 0, la = 0, b0 = 0, lb = 0;  // entry ranges in the packed factors (la = 0: empty term)
    int fa = -1, fb = -1;                // factor indices (-1: unit entry)
};

__device__ __forceinline__ TermRow term_row(const KronDesc& d, int t, int p, int q) {
    TermRow r;
    if (t == 0) {
        r.fa = fHp();
        r.a0 = d.ptr[d.ptr_off[r.fa] + p];
        r.la = d.ptr[d.ptr_off[r.fa] + p + 1] - r.a0;
        r.lb = 1;
    } else if (t == 1) {
        r.fb = fHn();
        r.la = 1;
        r.b0 = d.ptr[d.ptr_off[r.fb] + q];
        r.lb = d.ptr[d.ptr_off[r.fb] + q + 1] - r.b0;
    } else {
        const int k = t - 2;
        r.fa = fCp(k);
        r.fb = fCn(k);
        r.a0 = d.ptr[d.ptr_off[r.fa] + p];
        r.la = d.ptr[d.ptr_off[r.fa] + p + 1] - r.a0;
        r.b0 = d.ptr[d.ptr_off[r.fb] + q];
        r.lb = d.ptr[d.ptr_off[r.fb] + q + 1] - r.b0;
    }
    return r;
}

// Number of term contributions of each row; the largest over all rows.
__global__ void kron_rowcount_kernel(KronDesc d, int64_t n, int* __restrict__ maxlen) {
    int best = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(r / d.nN), q = (int)(r % d.nN);
        int c = 0;
        for (int t = 0; t < 2 + d.K; ++t) {
            const TermRow tr = term_row(d, t, p, q);
            c += tr.la * tr.lb;
        }
        best = max(best, c);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, off));
    if ((threadIdx.x & 31) == 0) atomicMax(maxlen, best);
}

constexpr int kRowThreads = 128;  // 4 warps, one expanded row each at a time
constexpr long long kKeyPad = 0x7fffffffffffffffll;

// Writes the contributions of row (p, q) as keys col * 64 + t and FP64
// values into keys[0..total), pads to a power of two >= 32 and sorts; returns
// total (or -1 if it exceeds cap).  Whole warp.
__device__ int expand_sorted_row(const KronDesc& d, int p, int q, long long* keys, double* vals, int cap, int lane) {
    const int nt = 2 + d.K;
    TermRow mine;
    if (lane < nt) mine = term_row(d, lane, p, q);
    const int sz = mine.la * mine.lb;
    int incl = sz;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total > cap) return -1;
    const int excl = incl - sz;
    for (int t = 0; t < nt; ++t) {
        const int la = __shfl_sync(0xffffffffu, mine.la, t), lb = __shfl_sync(0xffffffffu, mine.lb, t);
        const int a0 = __shfl_sync(0xffffffffu, mine.a0, t), b0 = __shfl_sync(0xffffffffu, mine.b0, t);
        const int fa = __shfl_sync(0xffffffffu, mine.fa, t), fb = __shfl_sync(0xffffffffu, mine.fb, t);
        const int off = __shfl_sync(0xffffffffu, excl, t);
        for (int j = lane; j < la * lb; j += 32) {
            const int ia = j / lb, ib = j - ia * lb;
            int ca = p, cb = q;
            double va = 1.0, vb = 1.0;
            if (fa >= 0) {
                ca = d.col[d.nz_off[fa] + a0 + ia];
                va = d.v64[d.nz_off[fa] + a0 + ia];
            }
            if (fb >= 0) {
                cb = d.col[d.nz_off[fb] + b0 + ib];
                vb = d.v64[d.nz_off[fb] + b0 + ib];
            }
            const long long colh = (long long)ca * d.nN + cb;
            keys[off + j] = colh * 64 + t;
            vals[off + j] = va * vb;
        }
    }
    int m = 32;
    while (m < total) m <<= 1;
    for (int j = total + lane; j < m; j += 32) {
        keys[j] = kKeyPad;
        vals[j] = 0.0;
    }
    __syncwarp();
    for (int k = 2; k <= m; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < m; i += 32) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const long long ki = keys[i], kx = keys[ixj];
                    if ((ki > kx) == up) {
                        keys[i] = kx;
                        keys[ixj] = ki;
                        const double t = vals[i];
                        vals[i] = vals[ixj];
                        vals[ixj] = t;
                    }
                }
            }
            __syncwarp();
        }
    }
    return total;
}

// Sum of the run of equal columns that starts at i (term order).
__device__ __forceinline__ double run_sum(const long long* keys, const double* vals, int i, int total) {
    const long long c = keys[i] >> 6;
    double s = vals[i];
    for (int j = i + 1; j < total && (keys[j] >> 6) == c; ++j) s += vals[j];
    return s;
}

// diag(H), the largest absolute row sum and the number of nonzeros of the
// expansion (merged entries; an exactly cancelling sum still counts).
__global__ void __launch_bounds__(kRowThreads) kron_norm_kernel(KronDesc d, int64_t n, int cap,
                                                                double* __restrict__ diag,
                                                                unsigned long long* __restrict__ norm_bits,
                                                                unsigned long long* __restrict__ nnz, int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long* keys = reinterpret_cast<long long*>(smem) + (int64_t)warp * cap;
    double* vals = reinterpret_cast<double*>(reinterpret_cast<long long*>(smem) + (int64_t)(kRowThreads / 32) * cap) +
                   (int64_t)warp * cap;
    double best = 0.0;
    unsigned long long count = 0;
    for (int64_t r = (int64_t)blockIdx.x * (kRowThreads / 32) + warp; r < n; r += (int64_t)gridDim.x * (kRowThreads / 32)) {
        const int p = (int)(r / d.nN), q = (int)(r % d.nN);
        const int total = expand_sorted_row(d, p, q, keys, vals, cap, lane);
        if (total < 0) {
            if (lane == 0) atomicOr(err, 1);
            __syncwarp();
            continue;
        }
        double abs_sum = 0.0, dg = 0.0;
        int heads = 0;
        for (int i = lane; i < total; i += 32) {
            if (i == 0 || (keys[i] >> 6) != (keys[i - 1] >> 6)) {
                const double s = run_sum(keys, vals, i, total);
                abs_sum += fabs(s);
                ++heads;
                if ((keys[i] >> 6) == r) dg = s;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            abs_sum += __shfl_xor_sync(0xffffffffu, abs_sum, off);
            dg += __shfl_xor_sync(0xffffffffu, dg, off);
            heads += __shfl_xor_sync(0xffffffffu, heads, off);
        }
        if (lane == 0) diag[r] = dg;
        best = fmax(best, abs_sum);
        count += (unsigned long long)heads;
        __syncwarp();
    }
    if (lane == 0) {
        atomicMax(norm_bits, (unsigned long long)__double_as_longlong(best));  // non-negative: order-preserving
        atomicAdd(nnz, count);
    }
}

// Rows S[s] of H restricted to the columns in S (pos[col] >= 0): MODE 0
// counts the entries of each row (len[s]); MODE 1 writes them (columns
// renumbered by pos, ascending) from row_ptr[s].
template <int MODE>
__global__ void __launch_bounds__(kRowThreads) kron_sub_kernel(KronDesc d, int64_t k, const int* __restrict__ S,
                                                               const int* __restrict__ pos, int cap,
                                                               int64_t* __restrict__ len, const int64_t* __restrict__ rp,
                                                               int* __restrict__ sci, double* __restrict__ sva,
                                                               int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long* keys = reinterpret_cast<long long*>(smem) + (int64_t)warp * cap;
    double* vals = reinterpret_cast<double*>(reinterpret_cast<long long*>(smem) + (int64_t)(kRowThreads / 32) * cap) +
                   (int64_t)warp * cap;
    for (int64_t s = (int64_t)blockIdx.x * (kRowThreads / 32) + warp; s < k; s += (int64_t)gridDim.x * (kRowThreads / 32)) {
        const int r = S[s];
        const int p = r / d.nN, q = r % d.nN;
        const int total = expand_sorted_row(d, p, q, keys, vals, cap, lane);
        if (total < 0) {
            if (lane == 0) atomicOr(err, 1);
            __syncwarp();
            continue;
        }
        int64_t out = MODE == 1 ? rp[s] : 0;
        for (int i0 = 0; i0 < total; i0 += 32) {
            const int i = i0 + lane;
            bool keep = false;
            int c = -1;
            if (i < total && (i == 0 || (keys[i] >> 6) != (keys[i - 1] >> 6))) {
                c = pos[(int)(keys[i] >> 6)];
                keep = c >= 0;
            }
            const unsigned ball = __ballot_sync(0xffffffffu, keep);
            if (MODE == 1 && keep) {
                const int64_t o = out + __popc(ball & ((1u << lane) - 1u));
                sci[o] = c;
                sva[o] = run_sum(keys, vals, i, total);
            }
            out += __popc(ball);
        }
        if (MODE == 0 && lane == 0) len[s] = out;
        __syncwarp();
    }
}

size_t row_smem(int cap) { return (size_t)(kRowThreads / 32) * cap * (sizeof(long long) + sizeof(double)); }

// ------------------------------------------------------------------ SpMM
// threads of a SpMM CTA: 512 (two CTAs per SM) or, for tiles of more than
// 2048 chunks, 1024 (one CTA per SM); at most 64 registers a thread
constexpr int kKronThreads = 512;
constexpr int kKronThreadsWide = 1024;

template <typename T>
struct KronVal {  // factor value type in the products
    using type = T;
};
template <>
struct KronVal<df32> {
    using type = float;
};

template <typename T>
__device__ __forceinline__ typename KronVal<T>::type kron_val(const KronDesc& d, int idx);
template <>
__device__ __forceinline__ float kron_val<float>(const KronDesc& d, int idx) { return __ldg(d.v32 + idx); }
template <>
__device__ __forceinline__ float kron_val<df32>(const KronDesc& d, int idx) { return __ldg(d.v32 + idx); }
template <>
__device__ __forceinline__ double kron_val<double>(const KronDesc& d, int idx) { return __ldg(d.v64 + idx); }

template <typename T, int N>
struct KVec {
    T v[N];
};

// 16-byte (or narrower) vector access of N consecutive elements
template <typename T, int N>
__device__ __forceinline__ void kload(const T* p, T (&o)[N]) {
    if constexpr (is_df32<T>::value) {
        if constexpr (N == 2) {
            const float4 x = *reinterpret_cast<const float4*>(p);
            o[0] = df32(x.x, x.y);
            o[1] = df32(x.z, x.w);
        } else {
            const float2 x = *reinterpret_cast<const float2*>(p);
            o[0] = df32(x.x, x.y);
        }
    } else if constexpr (sizeof(T) * N == 16) {
        if constexpr (sizeof(T) == 4) {
            const float4 x = *reinterpret_cast<const float4*>(p);
            o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
        } else {
            const double2 x = *reinterpret_cast<const double2*>(p);
            o[0] = x.x; o[1] = x.y;
        }
    } else if constexpr (sizeof(T) == 4 && N == 2) {
        const float2 x = *reinterpret_cast<const float2*>(p);
        o[0] = x.x; o[1] = x.y;
    } else {
#pragma unroll
        for (int v = 0; v < N; ++v) o[v] = p[v];
    }
}

template <typename T, int N>
__device__ __forceinline__ void kstore(T* p, const T (&o)[N]) {
    if constexpr (is_df32<T>::value) {
#pragma unroll
        for (int v = 0; v < N; ++v) {
            const df32 r = dfm::renorm(o[v].hi, o[v].lo);
            *reinterpret_cast<float2*>(p + v) = make_float2(r.hi, r.lo);
        }
    } else if constexpr (sizeof(T) * N == 16) {
        if constexpr (sizeof(T) == 4) *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
        else *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    } else if constexpr (sizeof(T) == 4 && N == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
    } else {
#pragma unroll
        for (int v = 0; v < N; ++v) p[v] = o[v];
    }
}

template <typename T>
__device__ __forceinline__ T kfma(typename KronVal<T>::type h, T v, T c) {
    if constexpr (is_df32<T>::value) return dfm::fma(h, v, c);
    else return fma(h, v, c);
}

template <typename T, int CB>
struct KronShape {
    static constexpr int VEC = CB < (int)(16 / sizeof(T)) ? CB : (int)(16 / sizeof(T));  // elements per chunk
    static constexpr int CPR = CB / VEC;                                                 // chunks per row
};

// One CTA: output slab p = blockIdx.x, columns [c0, c0 + CB) with c0 =
// blockIdx.y * CB.  Thread t owns the chunks ch = t + i * NT
// (i < IPT) of the slab's nN x CB tile: row q = ch / CPR, columns
// c0 + (ch % CPR) * VEC + [0, VEC).  Shared memory: the staged tile S
// (nN x CB elements) and the table of row p of Hp and of every Cp_k.
// With NT = 512, two CTAs per SM (at most 64 registers a thread), so that
// one CTA's streaming phase overlaps the other's gathers.
template <typename T, int CB, int IPT, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) kron_spmm_kernel(KronDesc d, int b, const T* __restrict__ V,
                                                                  T* __restrict__ W) {
    using H = typename KronVal<T>::type;
    using Sh = KronShape<T, CB>;
    constexpr int VEC = Sh::VEC, CPR = Sh::CPR;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nN = d.nN;
    T* S = reinterpret_cast<T*>(smem);
    int* tstart = reinterpret_cast<int*>(S + (int64_t)nN * CB);  // K + 2 offsets into the table
    int* tcol = tstart + 32;
    const int p = blockIdx.x;
    const int c0 = blockIdx.y * CB;
    const int nch = nN * CPR;
    const int64_t slab = (int64_t)nN * b;
    // table of row p of Hp (entry 0) and Cp_k (entry k + 1)
    const int nf = 1 + d.K;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int len = 0;
        if (lane < nf) {
            const int f = lane == 0 ? fHp() : fCp(lane - 1);
            len = d.ptr[d.ptr_off[f] + p + 1] - d.ptr[d.ptr_off[f] + p];
        }
        int incl = len;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane < nf) tstart[lane] = incl - len;
        if (lane == nf - 1) tstart[nf] = incl;
    }
    __syncthreads();
    // the values follow the tstart[nf] columns, 16-byte aligned
    H* tval = reinterpret_cast<H*>((reinterpret_cast<uintptr_t>(tcol + tstart[nf]) + 15) & ~uintptr_t(15));
    for (int f = threadIdx.x >> 5; f < nf; f += NT / 32) {
        const int fi = f == 0 ? fHp() : fCp(f - 1);
        const int a0 = d.ptr[d.ptr_off[fi] + p];
        const int la = d.ptr[d.ptr_off[fi] + p + 1] - a0;
        for (int e = threadIdx.x & 31; e < la; e += 32) {
            tcol[tstart[f] + e] = d.col[d.nz_off[fi] + a0 + e];
            tval[tstart[f] + e] = kron_val<T>(d, d.nz_off[fi] + a0 + e);
        }
    }
    __syncthreads();

    // chunk i of this thread: row, offset in a slab, offset in the tile
    auto row_of = [&](int i) { return (int)((threadIdx.x + i * NT) / CPR); };
    auto live = [&](int i) { return (int)threadIdx.x + i * NT < nch; };
    auto goff = [&](int i) {
        const int ch = threadIdx.x + i * NT;
        return (int64_t)(ch / CPR) * b + c0 + (ch % CPR) * VEC;
    };
    auto soff = [&](int i) {
        const int ch = threadIdx.x + i * NT;
        return (ch / CPR) * CB + (ch % CPR) * VEC;
    };

    T acc[IPT][VEC];
#pragma unroll
    for (int i = 0; i < IPT; ++i)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[i][v] = T(0.0f);

    // streaming combination sum_e tval[e] V[tcol[e]] of table entries [e0, e1)
    auto stream = [&](int e0, int e1, T (&out)[IPT][VEC]) {
        for (int e = e0; e < e1; ++e) {
            const H a = tval[e];
            const T* Vs = V + (int64_t)tcol[e] * slab;
#pragma unroll
            for (int i = 0; i < IPT; ++i) {
                if (!live(i)) continue;
                T x[VEC];
                kload<T, VEC>(Vs + goff(i), x);
#pragma unroll
                for (int v = 0; v < VEC; ++v) out[i][v] = kfma<T>(a, x[v], out[i][v]);
            }
        }
    };

    // gathers of an n-factor (Hn or Cn_k) from the staged tile into acc
    auto gather = [&](int fb) {
        const int* bp = d.ptr + d.ptr_off[fb];
        const int* bc = d.col + d.nz_off[fb];
        const int vo = d.nz_off[fb];
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            if (!live(i)) continue;
            const int q = row_of(i);
            const int cofs = soff(i) - q * CB;
            const int f0 = __ldg(bp + q), f1 = __ldg(bp + q + 1);
            for (int f = f0; f < f1; ++f) {
                const int qc = __ldg(bc + f);
                const H h = kron_val<T>(d, vo + f);
                T x[VEC];
                kload<T, VEC>(S + qc * CB + cofs, x);
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[i][v] = kfma<T>(h, x[v], acc[i][v]);
            }
        }
    };

    // (a) Hp (x) I: streaming combination of the slabs p' of row p of Hp
    stream(tstart[0], tstart[1], acc);

    // (b) I (x) Hn: stage V[p], gather
    {
        const T* Vs = V + (int64_t)p * slab;
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            if (!live(i)) continue;
            T x[VEC];
            kload<T, VEC>(Vs + goff(i), x);
            kstore<T, VEC>(S + soff(i), x);
        }
    }
    __syncthreads();
    gather(fHn());
    __syncthreads();

    // (c) Cp_k (x) Cn_k: U_k = sum_{p'} Cp_k[p,p'] V[p'] into the tile, then Cn_k U_k
    for (int k = 0; k < d.K; ++k) {
        const int e0 = tstart[k + 1], e1 = tstart[k + 2];
        if (e0 == e1) continue;  // the same for the whole CTA
        T u[IPT][VEC];
#pragma unroll
        for (int i = 0; i < IPT; ++i)
#pragma unroll
            for (int v = 0; v < VEC; ++v) u[i][v] = T(0.0f);
        stream(e0, e1, u);
#pragma unroll
        for (int i = 0; i < IPT; ++i)
            if (live(i)) kstore<T, VEC>(S + soff(i), u[i]);
        __syncthreads();
        gather(fCn(k));
        __syncthreads();
    }

    T* Ws = W + (int64_t)p * slab;
#pragma unroll
    for (int i = 0; i < IPT; ++i)
        if (live(i)) kstore<T, VEC>(Ws + goff(i), acc[i]);
}

// 16-byte asynchronous global -> shared copy (cp.async), its group commit and wait
__device__ __forceinline__ void kcp16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void kcommit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void kwait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kPipeStages = 2;  // slabs in the per-thread ring

// The same product with the slab stream prefetched: the slabs a CTA reads
// form one sequence over all terms -- row p of Hp, then V[p] itself (for
// Hn), then row p of each Cp_k -- and each thread copies its chunks of the
// next slab into its own shared-memory ring with cp.async while it
// accumulates the current one, so the stream runs on through the barriers
// and the n-factor gathers (only a thread's own copies are read back by it,
// so the ring needs no barrier).  The n-factor gathers load the row
// pointers of the next factor ahead and the columns and values of up to 4
// entries of a row at once.  Chunks are 16 bytes (VEC * sizeof(T) == 16).
template <typename T, int CB, int IPT, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) kron_pipe_kernel(KronDesc d, int b, const T* __restrict__ V,
                                                                  T* __restrict__ W) {
    using H = typename KronVal<T>::type;
    using Sh = KronShape<T, CB>;
    constexpr int VEC = Sh::VEC, CPR = Sh::CPR;
    static_assert(VEC * sizeof(T) == 16, "16-byte chunks");
    constexpr int NS = kPipeStages;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nN = d.nN;
    T* ring = reinterpret_cast<T*>(smem);                                // NS x IPT x NT chunks
    T* S = ring + (size_t)NS * IPT * NT * VEC;                          // nN x CB tile
    int* tstart = reinterpret_cast<int*>(S + (int64_t)nN * CB);          // segment starts (K + 3)
    int* tcol = tstart + 40;
    const int p = blockIdx.x;
    const int c0 = blockIdx.y * CB;
    const int nch = nN * CPR;
    const int64_t slab = (int64_t)nN * b;
    // segments: 0 = row p of Hp, 1 = V[p] itself, 2 + k = row p of Cp_k
    const int nseg = 2 + d.K;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int len = 0;
        if (lane < nseg) {
            if (lane == 1) {
                len = 1;
            } else {
                const int f = lane == 0 ? fHp() : fCp(lane - 2);
                len = d.ptr[d.ptr_off[f] + p + 1] - d.ptr[d.ptr_off[f] + p];
            }
        }
        int incl = len;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane < nseg) tstart[lane] = incl - len;
        if (lane == nseg - 1) tstart[nseg] = incl;
    }
    __syncthreads();
    H* tval = reinterpret_cast<H*>((reinterpret_cast<uintptr_t>(tcol + tstart[nseg]) + 15) & ~uintptr_t(15));
    for (int sg = threadIdx.x >> 5; sg < nseg; sg += NT / 32) {
        const int lane = threadIdx.x & 31;
        if (sg == 1) {
            if (lane == 0) {
                tcol[tstart[1]] = p;
                tval[tstart[1]] = H(1.0f);
            }
            continue;
        }
        const int fi = sg == 0 ? fHp() : fCp(sg - 2);
        const int a0 = d.ptr[d.ptr_off[fi] + p];
        const int la = d.ptr[d.ptr_off[fi] + p + 1] - a0;
        for (int e = lane; e < la; e += 32) {
            tcol[tstart[sg] + e] = d.col[d.nz_off[fi] + a0 + e];
            tval[tstart[sg] + e] = kron_val<T>(d, d.nz_off[fi] + a0 + e);
        }
    }
    __syncthreads();
    const int J = tstart[nseg];  // slabs streamed

    auto live = [&](int i) { return (int)threadIdx.x + i * NT < nch; };
    auto goff = [&](int i) {
        const int ch = threadIdx.x + i * NT;
        return (int64_t)(ch / CPR) * b + c0 + (ch % CPR) * VEC;
    };
    auto soff = [&](int i) {
        const int ch = threadIdx.x + i * NT;
        return (ch / CPR) * CB + (ch % CPR) * VEC;
    };
    auto slot = [&](int j, int i) { return ring + ((size_t)((j % NS) * IPT + i) * NT + threadIdx.x) * VEC; };
    auto issue = [&](int j) {
        if (j < J) {
            const T* Vs = V + (int64_t)tcol[j] * slab;
#pragma unroll
            for (int i = 0; i < IPT; ++i)
                if (live(i)) kcp16(slot(j, i), Vs + goff(i));
        }
        kcommit();  // an empty group past the end keeps the count uniform
    };

    T acc[IPT][VEC];
#pragma unroll
    for (int i = 0; i < IPT; ++i)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[i][v] = T(0.0f);
    // row pointers of an n-factor for this thread's rows
    int f0[IPT], f1[IPT];
    auto load_rows = [&](int fb) {
        const int* bp = d.ptr + d.ptr_off[fb];
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const int q = live(i) ? (int)((threadIdx.x + i * NT) / CPR) : 0;
            f0[i] = __ldg(bp + q);
            f1[i] = live(i) ? __ldg(bp + q + 1) : f0[i];
        }
    };
    auto gather = [&](int fb) {
        const int* bc = d.col + d.nz_off[fb];
        const int vo = d.nz_off[fb];
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const int cofs = soff(i) % CB;
            for (int f = f0[i]; f < f1[i]; f += 4) {
                int qc[4];
                H h[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool ok = f + u < f1[i];
                    qc[u] = ok ? __ldg(bc + f + u) : 0;
                    h[u] = ok ? kron_val<T>(d, vo + f + u) : H(0.0f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (f + u < f1[i]) {
                        T x[VEC];
                        kload<T, VEC>(S + qc[u] * CB + cofs, x);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[i][v] = kfma<T>(h[u], x[v], acc[i][v]);
                    }
                }
            }
        }
    };

    issue(0);
    int j = 0;
    for (int sg = 0; sg < nseg; ++sg) {
        const int fb = sg == 0 ? -1 : (sg == 1 ? fHn() : fCn(sg - 2));
        if (fb >= 0) load_rows(fb);  // in flight during the stream
        T u[IPT][VEC];
#pragma unroll
        for (int i = 0; i < IPT; ++i)
#pragma unroll
            for (int v = 0; v < VEC; ++v) u[i][v] = T(0.0f);
        for (; j < tstart[sg + 1]; ++j) {
            issue(j + 1);
            kwait<1>();  // slab j has landed (the one just issued may be in flight)
            const H a = tval[j];
#pragma unroll
            for (int i = 0; i < IPT; ++i) {
                if (!live(i)) continue;
                T x[VEC];
                kload<T, VEC>(slot(j, i), x);
#pragma unroll
                for (int v = 0; v < VEC; ++v) u[i][v] = kfma<T>(a, x[v], u[i][v]);
            }
        }
        if (sg == 0) {
#pragma unroll
            for (int i = 0; i < IPT; ++i)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[i][v] = acc[i][v] + u[i][v];
            continue;
        }
        __syncthreads();  // every thread is done with the previous gather: the tile is free
#pragma unroll
        for (int i = 0; i < IPT; ++i)
            if (live(i)) kstore<T, VEC>(S + soff(i), u[i]);
        __syncthreads();
        gather(fb);
    }
    kwait<0>();
    T* Ws = W + (int64_t)p * slab;
#pragma unroll
    for (int i = 0; i < IPT; ++i)
        if (live(i)) kstore<T, VEC>(Ws + goff(i), acc[i]);
}

// Shared memory of one CTA: the tile, 32 table offsets, the table's columns
// and (16-byte aligned) values.
template <typename T>
size_t kron_smem(const bbl_matrix* A, int CB) {
    using H = typename KronVal<T>::type;
    const size_t tile = (size_t)A->kron_nN * CB * sizeof(T);
    const size_t tab = 32 * sizeof(int) + (size_t)A->kron_prow_cap * sizeof(int) + 16 +
                       (size_t)A->kron_prow_cap * sizeof(H);
    return tile + tab;
}

constexpr size_t kKronSmemMax = 200 * 1024;

// the prefetching kernel's shared memory: ring + tile + segment table (one more entry)
template <typename T>
size_t kron_pipe_smem(const bbl_matrix* A, int CB, int IPT, int NT) {
    using H = typename KronVal<T>::type;
    const size_t ring = (size_t)kPipeStages * IPT * NT * 16;
    const size_t tile = (size_t)A->kron_nN * CB * sizeof(T);
    const size_t tab = 40 * sizeof(int) + (size_t)(A->kron_prow_cap + 1) * sizeof(int) + 16 +
                       (size_t)(A->kron_prow_cap + 1) * sizeof(H);
    return ring + tile + tab;
}

template <typename T, int CB, int IPT, int NT>
bbl_status launch_kron_pipe(const bbl_matrix* A, int b, const T* V, T* W, size_t smem, cudaStream_t st) {
    auto kern = kron_pipe_kernel<T, CB, IPT, NT>;
    static bool attr = false;
    if (!attr) {
        BBL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kKronSmemMax));
        attr = true;
    }
    dim3 grid((unsigned)A->kron_nP, (unsigned)(b / CB));
    kern<<<grid, NT, smem, st>>>(make_desc(A), b, V, W);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

template <typename T, int CB, int IPT, int NT>
bbl_status launch_kron_t(const bbl_matrix* A, int b, const T* V, T* W, size_t smem, cudaStream_t st) {
    // 16-byte chunks: the prefetching kernel when its ring fits as well
    if constexpr (CB * sizeof(T) >= 16 && CB <= 16) {
        const size_t ps = kron_pipe_smem<T>(A, CB, IPT, NT);
        if (ps <= kKronSmemMax && A->kron_K + 3 <= 40) return launch_kron_pipe<T, CB, IPT, NT>(A, b, V, W, ps, st);
    }
    auto kern = kron_spmm_kernel<T, CB, IPT, NT>;
    static bool attr = false;
    if (!attr) {
        BBL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kKronSmemMax));
        attr = true;
    }
    dim3 grid((unsigned)A->kron_nP, (unsigned)(b / CB));
    kern<<<grid, NT, smem, st>>>(make_desc(A), b, V, W);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

// nch chunks: 512 threads with 1, 2 or 4 chunks each, else 1024 with 4
template <typename T, int CB>
bbl_status launch_kron_cb(const bbl_matrix* A, int b, const T* V, T* W, int64_t nch, size_t smem, cudaStream_t st) {
    if (nch <= kKronThreads) return launch_kron_t<T, CB, 1, kKronThreads>(A, b, V, W, smem, st);
    if (nch <= 2 * kKronThreads) return launch_kron_t<T, CB, 2, kKronThreads>(A, b, V, W, smem, st);
    if (nch <= 4 * kKronThreads) return launch_kron_t<T, CB, 4, kKronThreads>(A, b, V, W, smem, st);
    return launch_kron_t<T, CB, 4, kKronThreadsWide>(A, b, V, W, smem, st);
}

// Column group: the widest power of two CB <= 16 dividing b whose tile
// fits (at most 4 chunks per thread and kKronSmemMax bytes of shared
// memory), but no wider than 32 bytes of a row when that keeps 2 chunks per
// thread: a CTA then reads whole 32-byte sectors of each row and two CTAs
// fit an SM.
template <typename T>
bbl_status kron_spmm_typed(const bbl_matrix* A, int b, const T* V, T* W, cudaStream_t st) {
    const int sector_cb = std::max<int>(1, 32 / (int)sizeof(T));
    auto chunks = [&](int CB) { return A->kron_nN * (CB / std::min<int>(CB, (int)(16 / sizeof(T)))); };
    for (int CB = 16; CB >= 1; CB >>= 1) {
        if (b % CB) continue;
        const int64_t nch = chunks(CB);
        const size_t smem = kron_smem<T>(A, CB);
        if (nch > 4 * kKronThreadsWide || smem > kKronSmemMax) continue;
        // prefer a 32-byte column group that keeps 512 threads per CTA
        if (CB > sector_cb && b % sector_cb == 0 && chunks(sector_cb) <= 4 * kKronThreads) continue;
        switch (CB) {
            case 16: return launch_kron_cb<T, 16>(A, b, V, W, nch, smem, st);
            case 8: return launch_kron_cb<T, 8>(A, b, V, W, nch, smem, st);
            case 4: return launch_kron_cb<T, 4>(A, b, V, W, nch, smem, st);
            case 2: return launch_kron_cb<T, 2>(A, b, V, W, nch, smem, st);
            default: return launch_kron_cb<T, 1>(A, b, V, W, nch, smem, st);
        }
    }
    return set_error(BBL_ERR_UNSUPPORTED, "kron spmm: nN = %lld is too large for one shared-memory tile",
                     (long long)A->kron_nN);
}

// Host copy of an int32 / FP64 array given in host or device memory.
template <typename X>
bbl_status fetch(std::vector<X>& out, const void* src, size_t count) {
    out.resize(count);
    if (count == 0) return BBL_OK;
    BBL_CUDA(cudaMemcpy(out.data(), src, sizeof(X) * count, cudaMemcpyDefault));
    return BBL_OK;
}

}  // namespace

bbl_status kron_spmm(const bbl_matrix* A, int b, int dt, const void* V, void* W, cudaStream_t st) {
    if (dt == BBL_FP32) {
        if (A->storage != BBL_FP32) return set_error(BBL_ERR_UNSUPPORTED, "kron spmm: FP32 blocks need FP32 storage");
        return kron_spmm_typed<float>(A, b, static_cast<const float*>(V), static_cast<float*>(W), st);
    }
    if (dt == kDF32) {
        if (A->storage != BBL_FP32)
            return set_error(BBL_ERR_UNSUPPORTED, "kron spmm: float-float blocks need FP32 factor values");
        return kron_spmm_typed<df32>(A, b, static_cast<const df32*>(V), static_cast<df32*>(W), st);
    }
    return kron_spmm_typed<double>(A, b, static_cast<const double*>(V), static_cast<double*>(W), st);
}

bbl_status kron_submatrix(const bbl_matrix* A, int64_t k, const int* S, const int* pos, DevBuf& row_ptr, DevBuf& col,
                          DevBuf& val, int64_t* nnz, cudaStream_t st) {
    const KronDesc d = make_desc(A);
    const int cap = A->kron_row_cap;
    const size_t smem = row_smem(cap);
    DevBuf len, err;
    BBL_TRY(len.alloc(sizeof(int64_t) * (k + 1)));
    BBL_TRY(err.alloc(sizeof(int)));
    BBL_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    const unsigned grid = (unsigned)std::min<int64_t>(152 * 16, std::max<int64_t>(1, ceil_div(k, kRowThreads / 32)));
    kron_sub_kernel<0><<<grid, kRowThreads, smem, st>>>(d, k, S, pos, cap, len.as<int64_t>(), nullptr, nullptr, nullptr,
                                                        err.as<int>());
    BBL_LAUNCH_CHECK();
    std::vector<int64_t> h(k + 1);
    int herr = 0;
    BBL_CUDA(cudaMemcpyAsync(h.data(), len.p, sizeof(int64_t) * k, cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    if (herr) return set_error(BBL_ERR_NUMERICAL, "kron submatrix: a row has more contributions than counted");
    int64_t acc = 0;
    for (int64_t s = 0; s < k; ++s) {
        const int64_t t = h[s];
        h[s] = acc;
        acc += t;
    }
    h[k] = acc;
    BBL_TRY(row_ptr.alloc(sizeof(int64_t) * (k + 1)));
    BBL_TRY(col.alloc(sizeof(int) * std::max<int64_t>(acc, 1)));
    BBL_TRY(val.alloc(sizeof(double) * std::max<int64_t>(acc, 1)));
    BBL_CUDA(cudaMemcpyAsync(row_ptr.p, h.data(), sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice, st));
    kron_sub_kernel<1><<<grid, kRowThreads, smem, st>>>(d, k, S, pos, cap, nullptr, row_ptr.as<int64_t>(),
                                                        col.as<int>(), val.as<double>(), err.as<int>());
    BBL_LAUNCH_CHECK();
    BBL_CUDA(cudaStreamSynchronize(st));
    *nnz = acc;
    return BBL_OK;
}

}  // namespace bbl

extern "C" bbl_status bbl_matrix_create_kron(int64_t nP, int64_t nN, int K, const int32_t* fptr, const int32_t* fcol,
                                             const double* fval, const int64_t* ptr_off, const int64_t* nz_off,
                                             bbl_dtype storage, int check_symmetry, void* stream, bbl_matrix** out) {
    using namespace bbl;
    if (!out) return set_error(BBL_ERR_INVALID_ARG, "matrix_create_kron: out is NULL");
    *out = nullptr;
    if (nP < 1 || nN < 1 || K < 0 || K > kKronMaxK || !fptr || !fcol || !fval || !ptr_off || !nz_off)
        return set_error(BBL_ERR_INVALID_ARG, "matrix_create_kron: bad arguments (K in 0..%d)", kKronMaxK);
    if (nP * nN >= (int64_t(1) << 31) || nP * nN * 64 >= (int64_t(1) << 62))
        return set_error(BBL_ERR_INVALID_ARG, "matrix_create_kron: n = nP*nN must be below 2^31");
    if (storage != BBL_FP64 && storage != BBL_FP32) return set_error(BBL_ERR_INVALID_ARG, "matrix_create_kron: bad storage");
    const int nf = 2 + 2 * K;
    // host copies of the (small) factors: validation and packing
    std::vector<int64_t> po(ptr_off, ptr_off + nf), zo(nz_off, nz_off + nf);
    int64_t ptr_len = 0, nz_len = 0;
    for (int f = 0; f < nf; ++f) {
        const int64_t N = (f == 1 || (f >= 2 && f % 2 == 1)) ? nN : nP;
        if (po[f] < 0 || zo[f] < 0) return set_error(BBL_ERR_INVALID_ARG, "matrix_create_kron: negative offset");
        ptr_len = std::max(ptr_len, po[f] + N + 1);
    }
    std::vector<int32_t> hp;
    BBL_TRY(fetch(hp, fptr, (size_t)ptr_len));
    for (int f = 0; f < nf; ++f) {
        const int64_t N = (f == 1 || (f >= 2 && f % 2 == 1)) ? nN : nP;
        const int32_t* rp = hp.data() + po[f];
        if (rp[0] != 0) return set_error(BBL_ERR_INVALID_ARG, "matrix_create_kron: factor %d: row_ptr[0] != 0", f);
        for (int64_t i = 0; i < N; ++i)
            if (rp[i + 1] < rp[i] || rp[i + 1] - rp[i] > N)
                return set_error(BBL_ERR_INVALID_ARG, "matrix_create_kron: factor %d: bad row_ptr", f);
        nz_len = std::max<int64_t>(nz_len, zo[f] + rp[N]);
    }
    if (ptr_len >= (int64_t(1) << 31) || nz_len >= (int64_t(1) << 31))
        return set_error(BBL_ERR_INVALID_ARG, "matrix_create_kron: factors too large");
    std::vector<int32_t> hc;
    std::vector<double> hv;
    BBL_TRY(fetch(hc, fcol, (size_t)nz_len));
    BBL_TRY(fetch(hv, fval, (size_t)nz_len));
    int prow_cap = 0;
    std::vector<int> prow(nP, 0);
    for (int f = 0; f < nf; ++f) {
        const bool pfac = !(f == 1 || (f >= 2 && f % 2 == 1));
        const int64_t N = pfac ? nP : nN;
        const int32_t* rp = hp.data() + po[f];
        for (int64_t i = 0; i < N; ++i) {
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
                const int32_t c = hc[zo[f] + e];
                if (c < 0 || c >= N || (e > rp[i] && hc[zo[f] + e - 1] >= c))
                    return set_error(BBL_ERR_INVALID_ARG,
                                     "matrix_create_kron: factor %d row %lld: columns must increase within [0, N)", f,
                                     (long long)i);
                const double v = hv[zo[f] + e];
                if (!std::isfinite(v)) return set_error(BBL_ERR_INVALID_ARG, "matrix_create_kron: non-finite value");
                if (check_symmetry) {  // (c, i) must hold the same value
                    const int32_t* cb = hc.data() + zo[f] + rp[c];
                    const int32_t* ce = hc.data() + zo[f] + rp[c + 1];
                    const int32_t* it = std::lower_bound(cb, ce, (int32_t)i);
                    if (it == ce || *it != i || hv[it - hc.data()] != v)
                        return set_error(BBL_ERR_NOT_SYMMETRIC, "matrix_create_kron: factor %d is not symmetric", f);
                }
            }
        }
        if (pfac)
            for (int64_t i = 0; i < nP; ++i) prow[i] += rp[i + 1] - rp[i];
    }
    for (int64_t i = 0; i < nP; ++i) prow_cap = std::max(prow_cap, prow[i]);
    std::vector<float> h32(nz_len);
    std::vector<double> h64(nz_len);
    for (int64_t e = 0; e < nz_len; ++e) {
        h32[e] = (float)hv[e];
        // FP32 storage: the operator's factors are the FP32 values
        h64[e] = storage == BBL_FP32 ? (double)h32[e] : hv[e];
    }
    bbl_matrix* A = new bbl_matrix();
    auto fail = [&](bbl_status s) {
        delete A;
        return s;
    };
    cudaStream_t st = as_stream(stream);
    A->n = nP * nN;
    A->fmt = BBL_KRON;
    A->storage = storage;
    A->kron_nP = nP;
    A->kron_nN = nN;
    A->kron_K = K;
    A->kron_prow_cap = prow_cap;
    for (int f = 0; f < nf; ++f) {
        A->kf_ptr_off[f] = po[f];
        A->kf_nz_off[f] = zo[f];
    }
    bbl_status s;
    if ((s = A->kf_ptr.alloc(sizeof(int32_t) * ptr_len)) != BBL_OK) return fail(s);
    if ((s = A->kf_col.alloc(sizeof(int32_t) * std::max<int64_t>(nz_len, 1))) != BBL_OK) return fail(s);
    if ((s = A->kf_val32.alloc(sizeof(float) * std::max<int64_t>(nz_len, 1))) != BBL_OK) return fail(s);
    if ((s = A->kf_val64.alloc(sizeof(double) * std::max<int64_t>(nz_len, 1))) != BBL_OK) return fail(s);
    if ((s = A->diag.alloc(sizeof(double) * A->n)) != BBL_OK) return fail(s);
    if (cudaMemcpyAsync(A->kf_ptr.p, hp.data(), sizeof(int32_t) * ptr_len, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(A->kf_col.p, hc.data(), sizeof(int32_t) * nz_len, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(A->kf_val32.p, h32.data(), sizeof(float) * nz_len, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(A->kf_val64.p, h64.data(), sizeof(double) * nz_len, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(set_error(BBL_ERR_CUDA, "matrix_create_kron: upload failed"));
    // the expansion: contributions per row (bound), then diag, ||H||_inf, nnz
    const KronDesc d = make_desc(A);
    DevBuf scratch;
    if ((s = scratch.alloc(64)) != BBL_OK) return fail(s);
    if (cudaMemsetAsync(scratch.p, 0, 64, st) != cudaSuccess) return fail(set_error(BBL_ERR_CUDA, "memset"));
    int* d_max = reinterpret_cast<int*>(scratch.as<char>());
    int* d_err = reinterpret_cast<int*>(scratch.as<char>() + 4);
    unsigned long long* d_norm = reinterpret_cast<unsigned long long*>(scratch.as<char>() + 16);
    unsigned long long* d_nnz = reinterpret_cast<unsigned long long*>(scratch.as<char>() + 24);
    kron_rowcount_kernel<<<152 * 8, 256, 0, st>>>(d, A->n, d_max);
    if (cudaGetLastError() != cudaSuccess) return fail(set_error(BBL_ERR_CUDA, "matrix_create_kron: launch failed"));
    count_launch();
    int maxlen = 0;
    if (cudaMemcpyAsync(&maxlen, d_max, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(set_error(BBL_ERR_CUDA, "matrix_create_kron: row count failed"));
    int cap = 32;
    while (cap < maxlen) cap <<= 1;
    if (row_smem(cap) > 200 * 1024)
        return fail(set_error(BBL_ERR_UNSUPPORTED, "matrix_create_kron: a row of H has %d contributions (limit %d)",
                              maxlen, (int)(200 * 1024 / row_smem(1))));
    A->kron_row_cap = cap;
    if (cudaFuncSetAttribute(kron_norm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess ||
        cudaFuncSetAttribute(kron_sub_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess ||
        cudaFuncSetAttribute(kron_sub_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
        return fail(set_error(BBL_ERR_CUDA, "matrix_create_kron: shared memory attribute"));
    const unsigned grid = (unsigned)std::min<int64_t>(152 * 16, ceil_div(A->n, kRowThreads / 32));
    kron_norm_kernel<<<grid, kRowThreads, row_smem(cap), st>>>(d, A->n, cap, A->diag.as<double>(), d_norm, d_nnz, d_err);
    if (cudaGetLastError() != cudaSuccess) return fail(set_error(BBL_ERR_CUDA, "matrix_create_kron: launch failed"));
    count_launch();
    unsigned long long hres[2] = {0, 0};
    int herr = 0;
    if (cudaMemcpyAsync(hres, d_norm, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(set_error(BBL_ERR_CUDA, "matrix_create_kron: expansion failed"));
    if (herr) return fail(set_error(BBL_ERR_NUMERICAL, "matrix_create_kron: a row has more contributions than counted"));
    double nrm;
    std::memcpy(&nrm, &hres[0], sizeof(double));
    A->norm_inf = nrm;
    A->nnz = (int64_t)hres[1];
    A->padded_nnz = A->nnz;
    *out = A;
    return BBL_OK;
}
