// Tiled stored format (BBL_TILED): W = H V with the gathered rows of V served
// from shared memory (Sec. II.B, Eq. 3: each stored element H_ij reads the b
// contiguous values V[j, :]).
//
// Rows are grouped into row blocks of T rows (T <= 1024) and columns into
// column tiles of T columns.  For each row block the stored entries are
// grouped by column tile ("pairs" (row block, tile) with at least one
// entry): a 16-bit column within the tile and the value per entry, and per
// row a 16-bit offset into the pair's segment.  Inside a pair the rows come
// in slices of 64; one warp owns a slice, lane l rows l and 32 + l, and the
// slice's entries are stored slot-major ("jagged diagonal"): slot s holds,
// in lane order, the s-th entry of every lane whose two rows have more than
// s entries in the pair (row l's entries, then row 32 + l's).  The active
// lanes of a slot read consecutive entries, so every load of the entry
// stream is coalesced, and a lane finds its entry from a warp ballot.
//
// One CTA forms the W rows of one row block (or a group of its columns): it
// walks the block's pairs, copies the pair's T x CB tile of V into shared
// memory with cp.async (two buffers: the next tile lands while the current
// one is used), and each lane multiplies its rows' entries of the pair by
// rows of the staged tile, accumulating in registers.  The 16-byte chunks
// of a tile row are XOR-swizzled by the row index so that the first chunks
// of rows that differ in their low bits fall in all eight bank groups.  The
// stored entries stream from HBM once (6 bytes per nonzero in FP32: 2 + 4);
// the tiles of V come from L2.  The L1 serves about one gathered 32-byte
// row per cycle when rows of V are fetched straight from global memory;
// from shared memory the same gathers take several rows per cycle.  The
// format helps when the rows of a block touch few column tiles (a
// block-structured sparsity such as the proton x neutron factorised
// matrices); the CSR copy is kept for the rest of the library.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "df32.cuh"

namespace bbl {
namespace {

constexpr int kTileHistThreads = 256;

// Column tiles touched by the rows of row block rb: a shared-memory
// histogram of tile ids.  MODE 0: the number of touched tiles per block;
// MODE 1: the touched tiles in increasing order and their entry counts.
template <int MODE>
__global__ void __launch_bounds__(kTileHistThreads) tile_pairs_kernel(int64_t n, int T, int ntc,
                                                                      const int64_t* __restrict__ rp,
                                                                      const int* __restrict__ ci,
                                                                      int* __restrict__ npairs,
                                                                      const int64_t* __restrict__ pair_ptr,
                                                                      int* __restrict__ ptile, int* __restrict__ pnnz) {
    extern __shared__ int h[];  // ntc counters, then kTileHistThreads scan slots
    int* scan = h + ntc;
    const int rb = blockIdx.x;
    const int64_t r0 = (int64_t)rb * T, r1 = min(n, r0 + T);
    for (int e = threadIdx.x; e < ntc; e += blockDim.x) h[e] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t row = r0 + warp; row < r1; row += blockDim.x / 32)
        for (int64_t k = rp[row] + lane; k < rp[row + 1]; k += 32) atomicAdd(&h[ci[k] / T], 1);
    __syncthreads();
    // each thread owns a contiguous range of tiles: count, block scan, write
    const int per = (ntc + blockDim.x - 1) / blockDim.x;
    const int t0 = threadIdx.x * per, t1 = min(ntc, t0 + per);
    int mine = 0;
    for (int t = t0; t < t1; ++t) mine += h[t] > 0;
    scan[threadIdx.x] = mine;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const int v = threadIdx.x >= off ? scan[threadIdx.x - off] : 0;
        __syncthreads();
        scan[threadIdx.x] += v;
        __syncthreads();
    }
    if (MODE == 0) {
        if (threadIdx.x == blockDim.x - 1) npairs[rb] = scan[threadIdx.x];
        return;
    }
    int64_t o = pair_ptr[rb] + scan[threadIdx.x] - mine;
    for (int t = t0; t < t1; ++t)
        if (h[t] > 0) {
            ptile[o] = t;
            pnnz[o] = h[t];
            ++o;
        }
}

// Entries of row block rb, pair by pair in tile order: per row its entries
// in the pair's tile (a cursor per row walks the sorted columns), a block
// scan for the row offsets, then the copies.
template <typename TM>
__global__ void __launch_bounds__(kTileHistThreads) tile_fill_kernel(int64_t n, int T, const int64_t* __restrict__ rp,
                                                                     const int* __restrict__ ci,
                                                                     const TM* __restrict__ va,
                                                                     const int64_t* __restrict__ pair_ptr,
                                                                     const int* __restrict__ ptile,
                                                                     const int64_t* __restrict__ pbase,
                                                                     unsigned short* __restrict__ off,
                                                                     unsigned short* __restrict__ lcol,
                                                                     TM* __restrict__ tval) {
    extern __shared__ int64_t cur[];  // T cursors, then T counts / offsets (int)
    int* cnt = reinterpret_cast<int*>(cur + T);
    __shared__ int wsum[kTileHistThreads / 32];
    const int rb = blockIdx.x;
    const int64_t r0 = (int64_t)rb * T;
    const int rows = (int)min((int64_t)T, n - r0);
    for (int q = threadIdx.x; q < T; q += blockDim.x) cur[q] = q < rows ? rp[r0 + q] : 0;
    __syncthreads();
    for (int64_t pr = pair_ptr[rb]; pr < pair_ptr[rb + 1]; ++pr) {
        const int t = ptile[pr];
        const int lim = (t + 1) * T;  // columns below lim belong to tiles <= t
        for (int q = threadIdx.x; q < T; q += blockDim.x) {
            int c = 0;
            if (q < rows) {
                const int64_t e = rp[r0 + q + 1];
                int64_t k = cur[q];
                while (k < e && ci[k] < lim) ++k;
                c = (int)(k - cur[q]);
            }
            cnt[q] = c;
        }
        __syncthreads();
        // exclusive scan of cnt[0..T) (T <= 8192): each thread a contiguous run
        const int per = (T + blockDim.x - 1) / blockDim.x;
        const int a = threadIdx.x * per, z = min(T, a + per);
        int s = 0;
        for (int q = a; q < z; ++q) s += cnt[q];
        int incl = s;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        int run = before + incl - s;
        for (int q = a; q < z; ++q) {
            const int c = cnt[q];
            cnt[q] = run;
            run += c;
        }
        if (threadIdx.x == blockDim.x - 1) cnt[T] = run;  // cnt holds T + 1 ints
        __syncthreads();
        unsigned short* po = off + pr * (T + 1);
        for (int q = threadIdx.x; q <= T; q += blockDim.x) po[q] = (unsigned short)cnt[q];
        // copies in slot-major order per 64-row slice (warp per slice): the
        // stream of lane l is row q0 + l's entries, then row q0 + 32 + l's
        const int64_t base = pbase[pr];
        const unsigned lt = (1u << lane) - 1u;
        for (int q0 = warp * 64; q0 < T; q0 += (int)(blockDim.x / 32) * 64) {
            const int qa = q0 + lane, qb = qa + 32;
            const int ca = qa < T ? cnt[qa + 1] - cnt[qa] : 0;
            const int cb = qb < T ? cnt[qb + 1] - cnt[qb] : 0;
            const int tot = ca + cb;
            const int smax = __reduce_max_sync(0xffffffffu, tot);
            int64_t o = base + cnt[q0];
            for (int sl = 0; sl < smax; ++sl) {
                const unsigned m = __ballot_sync(0xffffffffu, sl < tot);
                if (sl < tot) {
                    const int64_t k = sl < ca ? cur[qa] + sl : cur[qb] + (sl - ca);
                    const int64_t w = o + __popc(m & lt);
                    lcol[w] = (unsigned short)(ci[k] - t * T);
                    tval[w] = va[k];
                }
                o += __popc(m);
            }
            if (qa < T) cur[qa] += ca;
            if (qb < T) cur[qb] += cb;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ SpMM
constexpr int kTiledMaxThreads = 512;  // tiles of at most 1024 rows

__device__ __forceinline__ void tcp16(void* smem, const void* gmem, int src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void tcommit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void twait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename TX>
struct TiledVal {  // matrix value type in the product
    using type = TX;
};
template <>
struct TiledVal<df32> {
    using type = float;
};

template <typename TX, int N>
__device__ __forceinline__ void tload(const TX* p, TX (&o)[N]) {
    if constexpr (is_df32<TX>::value) {
        static_assert(N == 2, "df32 chunks of 2");
        const float4 x = *reinterpret_cast<const float4*>(p);
        o[0] = df32(x.x, x.y);
        o[1] = df32(x.z, x.w);
    } else if constexpr (sizeof(TX) == 4) {
        static_assert(N == 4, "float chunks of 4");
        const float4 x = *reinterpret_cast<const float4*>(p);
        o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
    } else {
        static_assert(N == 2, "double chunks of 2");
        const double2 x = *reinterpret_cast<const double2*>(p);
        o[0] = x.x; o[1] = x.y;
    }
}

template <typename TX, int N>
__device__ __forceinline__ void tstore(TX* p, const TX (&o)[N]) {
    if constexpr (is_df32<TX>::value) {
#pragma unroll
        for (int v = 0; v < N; ++v) {
            const df32 r = dfm::renorm(o[v].hi, o[v].lo);
            *reinterpret_cast<float2*>(p + v) = make_float2(r.hi, r.lo);
        }
    } else if constexpr (sizeof(TX) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    }
}

template <typename TX>
__device__ __forceinline__ TX tfma(typename TiledVal<TX>::type h, TX v, TX c) {
    if constexpr (is_df32<TX>::value) return dfm::fma(h, v, c);
    else return fma(h, v, c);
}

// Chunk of row r of a staged tile that holds its 16-byte chunk c (C chunks
// per row): c XOR a few bits of r, so that rows differing in their low bits
// spread their chunks over the eight 16-byte bank groups.
template <int C>
__device__ __forceinline__ int tswz(int r, int c) {
    if constexpr (C == 1) return 0;
    else return c ^ ((r / (8 / C)) & (C - 1));
}

// One CTA: row block rb = blockIdx.x, columns [c0, c0 + CB), c0 =
// blockIdx.y * CB; 32 * ceil(T / 64) threads.  Warp w owns rows 64 w + l and
// 64 w + 32 + l (lane l).  Shared memory: two T x CB tiles of V.  TM: stored
// value type; TX: block type (and, through TiledVal, the type of the value
// in the product).
template <typename TM, typename TX, int CB>
__global__ void __launch_bounds__(kTiledMaxThreads, 2) tiled_spmm_kernel(
    int64_t n, int T, int b, const int64_t* __restrict__ pair_ptr, const int* __restrict__ ptile,
    const int64_t* __restrict__ pbase, const unsigned short* __restrict__ off, const unsigned short* __restrict__ lcol,
    const TM* __restrict__ tval, const TX* __restrict__ V, TX* __restrict__ W) {
    using H = typename TiledVal<TX>::type;
    constexpr int VEC = 16 / (int)sizeof(TX);
    constexpr int C = CB / VEC;
    static_assert(CB % VEC == 0 && C <= 8, "column group of one to eight 16-byte chunks");
    extern __shared__ __align__(16) unsigned char smem[];
    TX* Sbuf = reinterpret_cast<TX*>(smem);  // [2][T * CB]
    const int rb = blockIdx.x;
    const int c0 = blockIdx.y * CB;
    const int64_t r0 = (int64_t)rb * T;
    const int rows = (int)min((int64_t)T, n - r0);
    const int nch = T * C;
    const int64_t p0 = pair_ptr[rb], p1 = pair_ptr[rb + 1];
    const int np = (int)(p1 - p0);
    const int lane = threadIdx.x & 31;
    const int q0 = (threadIdx.x >> 5) * 64;  // < T
    const int qa = q0 + lane, qb = qa + 32;
    const unsigned lt = (1u << lane) - 1u;

    // copy tile k (pair p0 + k) of V into buffer k & 1: rows t*T .. t*T + T - 1
    // (zeros past n), columns [c0, c0 + CB), chunks swizzled
    auto issue = [&](int k) {
        if (k < np) {
            const int t = ptile[p0 + k];
            TX* S = Sbuf + (size_t)(k & 1) * T * CB;
            const int64_t g0 = (int64_t)t * T;
            for (int ch = threadIdx.x; ch < nch; ch += blockDim.x) {
                const int q = ch / C, c = ch % C;
                const bool ok = g0 + q < n;
                tcp16(S + (q * C + tswz<C>(q, c)) * VEC,
                      ok ? (const void*)(V + (g0 + q) * b + c0 + c * VEC) : (const void*)V, ok ? 16 : 0);
            }
        }
        tcommit();
    };
    // the two rows' entry counts and the slice's first entry in pair k
    int na = 0, nb = 0, ns = 0;
    auto fetch = [&](int k) {
        na = nb = ns = 0;
        if (k < np) {
            const unsigned short* po = off + (p0 + k) * (T + 1);
            int a0 = 0;
            if (qa < T) {
                a0 = __ldg(po + qa);
                na = __ldg(po + qa + 1) - a0;
            }
            if (qb < T) nb = __ldg(po + qb + 1) - __ldg(po + qb);
            ns = __shfl_sync(0xffffffffu, a0, 0);  // lane 0: row q0 < T
        }
    };

    TX accA[CB], accB[CB];
#pragma unroll
    for (int v = 0; v < CB; ++v) accA[v] = accB[v] = TX(0.0f);
    issue(0);
    fetch(0);
    for (int k = 0; k < np; ++k) {
        issue(k + 1);  // buffer (k + 1) & 1 was released by the barrier at the end of step k - 1
        twait<1>();
        __syncthreads();  // tile k complete from every thread's copies
        const TX* S = Sbuf + (size_t)(k & 1) * T * CB;
        const int ca = na, tot = na + nb;
        int64_t pos = pbase[p0 + k] + ns;
        fetch(k + 1);
        const int smax = __reduce_max_sync(0xffffffffu, tot);
        const int send = (smax + 3) & ~3;
        TX cur[CB];
#pragma unroll
        for (int v = 0; v < CB; ++v) cur[v] = TX(0.0f);
        for (int s0 = 0; s0 < send; s0 += 4) {
            int lc[4];
            H h[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool on = s0 + u < tot;
                const unsigned m = __ballot_sync(0xffffffffu, on);
                const int64_t w = pos + __popc(m & lt);
                pos += __popc(m);
                lc[u] = on ? (int)__ldg(lcol + w) : 0;
                h[u] = on ? (H)__ldg(tval + w) : H(0.0f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (s0 + u == ca) {  // the lane's stream moves from row qa to row qb
#pragma unroll
                    for (int v = 0; v < CB; ++v) {
                        accA[v] += cur[v];
                        cur[v] = TX(0.0f);
                    }
                }
                if (s0 + u < tot) {
                    const TX* row = S + lc[u] * CB;
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        TX x[VEC];
                        tload<TX, VEC>(row + tswz<C>(lc[u], c) * VEC, x);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) cur[c * VEC + v] = tfma<TX>(h[u], x[v], cur[c * VEC + v]);
                    }
                }
            }
        }
        if (ca < send) {
#pragma unroll
            for (int v = 0; v < CB; ++v) accB[v] += cur[v];
        } else {
#pragma unroll
            for (int v = 0; v < CB; ++v) accA[v] += cur[v];
        }
        __syncthreads();  // every thread is done with buffer k & 1
    }
    twait<0>();
#pragma unroll
    for (int c = 0; c < C; ++c) {
        TX oa[VEC], ob[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            oa[v] = accA[c * VEC + v];
            ob[v] = accB[c * VEC + v];
        }
        if (qa < rows) tstore<TX, VEC>(W + (r0 + qa) * b + c0 + c * VEC, oa);
        if (qb < rows) tstore<TX, VEC>(W + (r0 + qb) * b + c0 + c * VEC, ob);
    }
}

constexpr size_t kTiledSmemMax = 200 * 1024;

template <typename TM, typename TX, int CB>
bbl_status launch_tiled_t(const bbl_matrix* A, int b, const TM* val, const TX* V, TX* W, cudaStream_t st) {
    auto kern = tiled_spmm_kernel<TM, TX, CB>;
    static bool attr = false;
    if (!attr) {
        BBL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTiledSmemMax));
        attr = true;
    }
    const int T = A->tile;
    const size_t smem = 2 * (size_t)T * CB * sizeof(TX);
    dim3 grid((unsigned)A->t_nrb, (unsigned)(b / CB));
    const unsigned threads = 32u * (unsigned)ceil_div(T, 64);
    kern<<<grid, threads, smem, st>>>(A->n, T, b, A->t_pair_ptr.as<int64_t>(), A->t_pair_tile.as<int>(),
                                      A->t_pair_base.as<int64_t>(), A->t_off.as<unsigned short>(),
                                      A->t_lcol.as<unsigned short>(), val, V, W);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

// Column group: 32 bytes of a row (or 16 when b holds no 32-byte group),
// two tiles within the shared-memory limit.
template <typename TM, typename TX>
bbl_status tiled_typed(const bbl_matrix* A, int b, const TM* val, const TX* V, TX* W, cudaStream_t st) {
    constexpr int VEC = 16 / (int)sizeof(TX);
    if (A->tile > 2 * kTiledMaxThreads)
        return set_error(BBL_ERR_UNSUPPORTED, "spmm: tiled tile %d above %d rows", A->tile, 2 * kTiledMaxThreads);
    for (int CB = 2 * VEC; CB >= VEC; CB /= 2) {
        if (b % CB) continue;
        if (2 * (size_t)A->tile * CB * sizeof(TX) > kTiledSmemMax) continue;
        if (CB == 2 * VEC) return launch_tiled_t<TM, TX, 2 * VEC>(A, b, val, V, W, st);
        return launch_tiled_t<TM, TX, VEC>(A, b, val, V, W, st);
    }
    return set_error(BBL_ERR_UNSUPPORTED,
                     "spmm: the tiled format needs b a multiple of %d and a tile of at most %lld rows", VEC,
                     (long long)(kTiledSmemMax / (2 * VEC * sizeof(TX))));
}

}  // namespace

bbl_status tiled_spmm(const bbl_matrix* A, int b, int dt, const void* V, void* W, cudaStream_t st) {
    if (dt == kDF32)
        return tiled_typed<float, df32>(A, b, A->t_val.as<float>(), static_cast<const df32*>(V), static_cast<df32*>(W),
                                        st);
    if (dt == BBL_FP64) {
        if (A->storage == BBL_FP64)
            return tiled_typed<double, double>(A, b, A->t_val.as<double>(), static_cast<const double*>(V),
                                               static_cast<double*>(W), st);
        return tiled_typed<float, double>(A, b, A->t_val.as<float>(), static_cast<const double*>(V),
                                          static_cast<double*>(W), st);
    }
    return tiled_typed<float, float>(A, b, A->t_val.as<float>(), static_cast<const float*>(V), static_cast<float*>(W),
                                     st);
}

// Builds the tiled copy of A's CSR (values of type TM, the storage type).
template <typename TM>
bbl_status tiled_build_t(bbl_matrix* A, int T, cudaStream_t st) {
    const int64_t n = A->n;
    const int64_t nrb = ceil_div(n, T);
    const int64_t ntc64 = nrb;
    const size_t hist_smem = sizeof(int) * ((size_t)ntc64 + kTileHistThreads);
    if (hist_smem > 200 * 1024)
        return set_error(BBL_ERR_UNSUPPORTED, "matrix_create: %lld column tiles of %d (use a larger tile)",
                         (long long)ntc64, T);
    const int ntc = (int)ntc64;
    BBL_CUDA(cudaFuncSetAttribute(tile_pairs_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    BBL_CUDA(cudaFuncSetAttribute(tile_pairs_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    DevBuf np;
    BBL_TRY(np.alloc(sizeof(int) * nrb));
    tile_pairs_kernel<0><<<(unsigned)nrb, kTileHistThreads, hist_smem, st>>>(
        n, T, ntc, A->row_ptr.as<int64_t>(), A->col.as<int>(), np.as<int>(), nullptr, nullptr, nullptr);
    BBL_LAUNCH_CHECK();
    std::vector<int> hnp(nrb);
    BBL_CUDA(cudaMemcpyAsync(hnp.data(), np.p, sizeof(int) * nrb, cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    std::vector<int64_t> pp(nrb + 1, 0);
    for (int64_t r = 0; r < nrb; ++r) pp[r + 1] = pp[r] + hnp[r];
    const int64_t npairs = pp[nrb];
    BBL_TRY(A->t_pair_ptr.alloc(sizeof(int64_t) * (nrb + 1)));
    BBL_TRY(A->t_pair_tile.alloc(sizeof(int) * std::max<int64_t>(npairs, 1)));
    BBL_TRY(A->t_pair_base.alloc(sizeof(int64_t) * std::max<int64_t>(npairs, 1)));
    DevBuf pnnz;
    BBL_TRY(pnnz.alloc(sizeof(int) * std::max<int64_t>(npairs, 1)));
    BBL_CUDA(cudaMemcpyAsync(A->t_pair_ptr.p, pp.data(), sizeof(int64_t) * (nrb + 1), cudaMemcpyHostToDevice, st));
    tile_pairs_kernel<1><<<(unsigned)nrb, kTileHistThreads, hist_smem, st>>>(
        n, T, ntc, A->row_ptr.as<int64_t>(), A->col.as<int>(), nullptr, A->t_pair_ptr.as<int64_t>(),
        A->t_pair_tile.as<int>(), pnnz.as<int>());
    BBL_LAUNCH_CHECK();
    std::vector<int> hpn(npairs);
    BBL_CUDA(cudaMemcpyAsync(hpn.data(), pnnz.p, sizeof(int) * npairs, cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    std::vector<int64_t> base(npairs);
    int64_t acc = 0;
    for (int64_t p = 0; p < npairs; ++p) {
        if (hpn[p] > 65535)
            return set_error(BBL_ERR_UNSUPPORTED,
                             "matrix_create: %d entries in one (row block, column tile) pair exceed 16-bit offsets "
                             "(use a smaller tile)", hpn[p]);
        base[p] = acc;
        acc += hpn[p];
    }
    if (acc != A->nnz) return set_error(BBL_ERR_NUMERICAL, "matrix_create: tiled entries %lld != nnz %lld",
                                        (long long)acc, (long long)A->nnz);
    BBL_CUDA(cudaMemcpyAsync(A->t_pair_base.p, base.data(), sizeof(int64_t) * npairs, cudaMemcpyHostToDevice, st));
    BBL_TRY(A->t_off.alloc(sizeof(unsigned short) * (size_t)std::max<int64_t>(npairs, 1) * (T + 1)));
    BBL_TRY(A->t_lcol.alloc(sizeof(unsigned short) * std::max<int64_t>(A->nnz, 1)));
    BBL_TRY(A->t_val.alloc(sizeof(TM) * std::max<int64_t>(A->nnz, 1)));
    const size_t fill_smem = sizeof(int64_t) * T + sizeof(int) * (T + 1);
    BBL_CUDA(cudaFuncSetAttribute(tile_fill_kernel<TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    tile_fill_kernel<TM><<<(unsigned)nrb, kTileHistThreads, fill_smem, st>>>(
        n, T, A->row_ptr.as<int64_t>(), A->col.as<int>(), A->val.as<TM>(), A->t_pair_ptr.as<int64_t>(),
        A->t_pair_tile.as<int>(), A->t_pair_base.as<int64_t>(), A->t_off.as<unsigned short>(),
        A->t_lcol.as<unsigned short>(), A->t_val.as<TM>());
    BBL_LAUNCH_CHECK();
    BBL_CUDA(cudaStreamSynchronize(st));
    A->tile = T;
    A->t_nrb = nrb;
    A->t_npairs = npairs;
    return BBL_OK;
}

bbl_status tiled_build(bbl_matrix* A, int T, cudaStream_t st) {
    if (T < 16 || T > 1024) return set_error(BBL_ERR_INVALID_ARG, "matrix_create: tile %d outside 16..1024", T);
    if (A->storage == BBL_FP64) return tiled_build_t<double>(A, T, st);
    return tiled_build_t<float>(A, T, st);
}

}  // namespace bbl
