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
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include <cuda_fp16.h>

#include "common.cuh"
#include "df32.cuh"

namespace bbl {
namespace {

// (d0, d1) += a * (b0, b1) as one packed FP32 FMA (fma.rn.f32x2): each half
// rounds as fmaf does
__device__ __forceinline__ void fma2_bcast(float& d0, float& d1, float a, float b0, float b1) {
    unsigned long long d, aa, bb;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(d0), "f"(d1));
    asm("mov.b64 %0, {%1, %1};" : "=l"(aa) : "f"(a));
    asm("mov.b64 %0, {%1, %2};" : "=l"(bb) : "f"(b0), "f"(b1));
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(aa), "l"(bb));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d0), "=f"(d1) : "l"(d));
}

template <typename T, int N>
__device__ __forceinline__ void ldvec(const T* p, T (&out)[N]) {
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

constexpr int kRT = 256;   // rows per shared-memory tile in gram
constexpr int kRitzReserveSMs = 8;
constexpr int kThreads = 256;

// -------------------------------------------------------------------- gram
// One CTA: the partial Gram of the row ranges handed out by next(r0, r1)
// (called by every thread, in step) for the Q columns of column group
// `cgrp`, written to out[m][B] (this CTA's partial slot).
template <typename T, int B, int CPT, typename Next>
__device__ __forceinline__ void gram_body(int64_t n, int m, Next next, int TC, int cgrp, const T* __restrict__ Q,
                                          const T* __restrict__ W, double* __restrict__ partial_slot) {
    __shared__ T ws[kRT * B];
    extern __shared__ double sred[];
    const int tid = threadIdx.x;
    const int RS = kThreads / TC;
    const int cg = tid % TC, rs = tid / TC;
    const int a0 = (cgrp * TC + cg) * CPT;
    const bool active = a0 < m;
    const int j = active ? a0 / B : 0, off = a0 % B;
    const T* qb = Q + (int64_t)j * n * B + off;
    // FP64 running sums: in registers for FP64 data; for FP32 data the
    // per-tile FP32 sums are added into this thread's shared-memory slot, so
    // that registers go to loads in flight instead.
    constexpr bool kF32 = sizeof(T) == 4;
    constexpr int U = 8;  // rows whose loads are issued together
    double* mine = sred + (size_t)tid * CPT * B;
    double acc64[kF32 ? 1 : CPT][kF32 ? 1 : B];
    if constexpr (kF32) {
        for (int e = 0; e < CPT * B; ++e) mine[e] = 0.0;
    } else {
#pragma unroll
        for (int i = 0; i < CPT; ++i)
#pragma unroll
            for (int c = 0; c < B; ++c) acc64[i][c] = 0.0;
    }
    int64_t r_begin = 0, r_end = 0;
    while (next(r_begin, r_end))
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
            int r = rs;
            for (; r + (U - 1) * RS < rows; r += U * RS) {
                T q[U][CPT];
#pragma unroll
                for (int u = 0; u < U; ++u) ldvec<T, CPT>(qb + (t0 + r + u * RS) * B, q[u]);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const T* wr = ws + (r + u * RS) * B;
#pragma unroll
                    for (int c = 0; c < B; ++c) {
                        const T w = wr[c];
#pragma unroll
                        for (int i = 0; i < CPT; ++i) acc[i][c] = fma(q[u][i], w, acc[i][c]);
                    }
                }
            }
            for (; r < rows; r += RS) {
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
            if constexpr (kF32) {
#pragma unroll
                for (int i = 0; i < CPT; ++i)
#pragma unroll
                    for (int c = 0; c < B; ++c) mine[i * B + c] += (double)acc[i][c];
            } else {
#pragma unroll
                for (int i = 0; i < CPT; ++i)
#pragma unroll
                    for (int c = 0; c < B; ++c) acc64[i][c] += (double)acc[i][c];
            }
        }
    }
    if constexpr (!kF32) {
        if (RS > 1) {
#pragma unroll
            for (int i = 0; i < CPT; ++i)
#pragma unroll
                for (int c = 0; c < B; ++c) mine[i * B + c] = acc64[i][c];
        }
    }
    if (RS > 1) {
        // deterministic tree over the row slots
        __syncthreads();
        for (int s = RS / 2; s > 0; s >>= 1) {
            if (rs < s) {
                const double* other = sred + (size_t)(tid + s * TC) * CPT * B;
                for (int e = 0; e < CPT * B; ++e) mine[e] += other[e];
            }
            __syncthreads();
        }
        if (rs == 0 && active) {
            double* out = partial_slot + (int64_t)a0 * B;
            for (int e = 0; e < CPT * B; ++e) out[e] = mine[e];
        }
    } else if (active) {
        double* out = partial_slot + (int64_t)a0 * B;
        if constexpr (kF32) {
            for (int e = 0; e < CPT * B; ++e) out[e] = mine[e];
        } else {
#pragma unroll
            for (int i = 0; i < CPT; ++i)
#pragma unroll
                for (int c = 0; c < B; ++c) out[i * B + c] = acc64[i][c];
        }
    }
}

// Hands out [r0, r1) once (one fixed range per CTA).
struct OneRange {
    int64_t r0, r1;
    bool done = false;
    __device__ bool operator()(int64_t& a, int64_t& b) {
        if (done) return false;
        done = true;
        a = r0;
        b = r1;
        return r1 > r0;
    }
};

// Hands out chunks of a shared ticket counter: CTAs that start late (their
// SM was busy) simply take fewer chunks, so there is no tail wave.
struct TicketRanges {
    int* ticket;
    int64_t n, rows_per_chunk;
    int nchunks;
    __device__ bool operator()(int64_t& a, int64_t& b) {
        __shared__ int s_c;
        __syncthreads();
        if (threadIdx.x == 0) s_c = atomicAdd(ticket, 1);
        __syncthreads();
        const int c = s_c;
        if (c >= nchunks) return false;
        a = (int64_t)c * rows_per_chunk;
        b = min(n, a + rows_per_chunk);
        return true;
    }
};

// Split-K Gram: persistent CTAs (x, y) = worker x of column group y; the row
// chunks of each column group are taken from ticket[y].
template <typename T, int B, int CPT>
__global__ void __launch_bounds__(kThreads) gram_kernel(int64_t n, int m, int64_t rows_per_chunk, int nchunks, int TC,
                                                        const T* __restrict__ Q, const T* __restrict__ W,
                                                        double* __restrict__ partial, int* __restrict__ tickets) {
    TicketRanges next{tickets + blockIdx.y, n, rows_per_chunk, nchunks};
    gram_body<T, B, CPT>(n, m, next, TC, blockIdx.y, Q, W, partial + (int64_t)blockIdx.x * m * B);
}

// Row-contiguous split-K Gram (b = 4, 8).  A CTA takes a chunk of rows from
// the ticket counter and stages W's rows of the chunk in shared memory; its
// warps walk the basis blocks.  A warp streams a block's rows of the chunk
// into its own shared-memory ring with asynchronous 16-byte copies
// (cp.async), NS stages of RL * U whole consecutive rows, so that NS - 1
// stages are in flight while it computes on the oldest: no registers hold
// data in flight.  Lane (g, t) multiplies its CPL columns of a row (LPR
// lanes per row, RL = 32 / LPR rows per step) by the row's B values of W and
// keeps CPL x B sums; at the end of the block's rows the RL row lanes are
// combined by a butterfly that halves the values each lane carries per
// round, and each lane adds its share of the B x B partial to the CTA's
// FP64 slot.  Blocks are dealt to warps round-robin; with fewer than 8
// blocks the rows of a chunk are split among wpb warps per block (one slot
// per row share).  FP32 data: products are summed in FP32 per stage, then
// over the stages of the chunk and the lane tree, and in FP64 across chunks.
template <typename T, int B>
struct GramRowsShape {
    static constexpr int CPL = 16 / (int)sizeof(T);         // Q columns per lane
    static constexpr int LPR = B / CPL;                     // lanes per row
    static constexpr int RL = 32 / LPR;                     // rows per warp step
    static constexpr int R = 32768 / (B * (int)sizeof(T));  // rows per chunk (32 KB of W)
    static constexpr int U = 4;                             // rows per lane per stage
    static constexpr int NS = 4;                            // ring stages per warp
    static constexpr int SROWS = RL * U;                    // rows per stage (2 KB)
    static constexpr int NV = CPL * B;                      // sums per lane
    static constexpr int LOGRL = RL >= 32 ? 5 : RL >= 16 ? 4 : RL >= 8 ? 3 : RL >= 4 ? 2 : RL >= 2 ? 1 : 0;
    static constexpr int kWarps = kThreads / 32;
    static constexpr size_t smem_bytes = (size_t)R * B * sizeof(T) + (size_t)kWarps * NS * SROWS * B * sizeof(T);
};

template <typename T>
__device__ __forceinline__ T add_any(T a, T b) {
    return a + b;
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// warps per basis block when a chunk has fewer blocks than warps
__host__ __device__ __forceinline__ int gram_rows_wpb(int nblocks) {
    int wpb = 1;
    while (wpb < kThreads / 32 && nblocks * wpb * 2 <= kThreads / 32) wpb <<= 1;
    return wpb;
}

// One chunk, rows [r0, r0 + rows) with rows <= R, for all threads of the
// CTA: W's rows staged in shared memory (ws), then each warp streams the
// chunk's rows of its blocks (share sub: rows [sub * rsub, (sub + 1) * rsub))
// through its ring and adds its B x B partials to slot sub of `slots`
// (wpb slots of m x B FP64).  The barrier after the W tile also orders any
// plain stores the caller made to `slots` before the adds.
template <typename T, int B>
__device__ __forceinline__ void gram_rows_chunk(int64_t n, int m, int wpb, int64_t r0, int rows, int rsub,
                                                const T* __restrict__ Q, const T* __restrict__ W,
                                                double* __restrict__ slots, T* __restrict__ ws) {
    using S = GramRowsShape<T, B>;
    constexpr int CPL = S::CPL, LPR = S::LPR, RL = S::RL, R = S::R, U = S::U, NV = S::NV, LOGRL = S::LOGRL;
    constexpr int NS = S::NS, SROWS = S::SROWS;
    constexpr int PIECES = SROWS * LPR / 32;  // 16-byte copies per lane per stage
    static_assert(LPR >= 1 && LPR <= 32 && 32 % LPR == 0 && B % CPL == 0 && (1 << LOGRL) == RL, "gram_rows shape");
    static_assert((SROWS * LPR) % 32 == 0, "stage pieces");
    const int nblocks = m / B;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane % LPR, t = lane / LPR;
    T* ring = ws + (size_t)R * B + (size_t)warp * NS * SROWS * B;
    const int ngrp = S::kWarps / wpb;
    const int grp = warp / wpb, sub = warp % wpb;
    double* part = slots + (int64_t)sub * m * B;
    // after the butterfly lane t holds sums vbase .. vbase + NK - 1; when
    // NV < RL the last rounds are plain all-reduces and only t < NV write
    constexpr int NK = NV >= RL ? NV / RL : 1;
    int vbase = 0;
#pragma unroll
    for (int k = 0; k < LOGRL; ++k)
        if ((NV >> k) > 1 && (t & (1 << k))) vbase += NV >> (k + 1);
    const bool writer = (NV >= RL) || (t < NV);
    for (int e = threadIdx.x; e < R * LPR; e += kThreads) {
        const int r = e / LPR, h = e % LPR;
        T v[CPL];
        if (r < rows) {
            ldvec<T, CPL>(W + (r0 + r) * B + h * CPL, v);
        } else {
#pragma unroll
            for (int q = 0; q < CPL; ++q) v[q] = T(0);
        }
#pragma unroll
        for (int q = 0; q < CPL; ++q) ws[(h * R + r) * CPL + q] = v[q];
    }
    __syncthreads();
    const int rb = sub * rsub;
    const int re = min(rows, rb + rsub);
    if (re <= rb) return;
    const int nst = (re - rb + SROWS - 1) / SROWS;       // stages per block
    const int nblk = (nblocks - grp + ngrp - 1) / ngrp;  // blocks of this warp
    const int total = nblk * nst;
    // stage k: block grp + (k / nst) * ngrp, rows rb + (k % nst) * SROWS ..
    auto issue = [&](int k) {
        T* buf = ring + (size_t)(k % NS) * SROWS * B;
        if (k < total) {
            const int j = grp + (k / nst) * ngrp;
            const int s0 = rb + (k % nst) * SROWS;
            const T* src = Q + ((int64_t)j * n + r0 + s0) * B;
#pragma unroll
            for (int i = 0; i < PIECES; ++i) {
                const int pc = lane + 32 * i;
                const int row = pc / LPR, h = pc % LPR;
                const bool ok = s0 + row < re;
                cp_async16(buf + (size_t)pc * CPL, ok ? (const void*)(src + (size_t)row * B + h * CPL) : (const void*)Q,
                           ok ? 16 : 0);
            }
        }
        cp_async_commit();  // an empty group past the end keeps the count uniform
    };
#pragma unroll
    for (int k = 0; k < NS - 1; ++k) issue(k);
    T acc[CPL][B];
#pragma unroll
    for (int i = 0; i < CPL; ++i)
#pragma unroll
        for (int cc = 0; cc < B; ++cc) acc[i][cc] = T(0);
    for (int k = 0; k < total; ++k) {
        cp_async_wait<NS - 2>();
        __syncwarp();
        issue(k + NS - 1);  // into the buffer consumed at k - 1
        const T* buf = ring + (size_t)(k % NS) * SROWS * B;
        const int s0 = rb + (k % nst) * SROWS;
        T bat[CPL][B];
#pragma unroll
        for (int i = 0; i < CPL; ++i)
#pragma unroll
            for (int cc = 0; cc < B; ++cc) bat[i][cc] = T(0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int rr = t + u * RL;              // row within the stage (zero past the share)
            const int row = min(s0 + rr, R - 1);    // row within the W tile
            T q[CPL];
            T w[B];
            const T* qs = buf + (size_t)rr * B + g * CPL;
            if constexpr (sizeof(T) == 4) {
                const float4 x = *reinterpret_cast<const float4*>(qs);
                q[0] = x.x;
                q[1] = x.y;
                q[2] = x.z;
                q[3] = x.w;
            } else {
#pragma unroll
                for (int i = 0; i < CPL; ++i) q[i] = qs[i];
            }
#pragma unroll
            for (int h = 0; h < LPR; ++h) {
                const T* src = ws + (h * R + row) * CPL;
                if constexpr (sizeof(T) == 4) {
                    const float4 x = *reinterpret_cast<const float4*>(src);
                    w[h * CPL + 0] = x.x;
                    w[h * CPL + 1] = x.y;
                    w[h * CPL + 2] = x.z;
                    w[h * CPL + 3] = x.w;
                } else {
#pragma unroll
                    for (int q2 = 0; q2 < CPL; ++q2) w[h * CPL + q2] = src[q2];
                }
            }
            if constexpr (std::is_same<T, float>::value && B % 2 == 0) {
                // two columns per packed FP32 FMA (each half an IEEE fma.rn: the
                // same results as two fmaf, in half the issued instructions)
#pragma unroll
                for (int i = 0; i < CPL; ++i)
#pragma unroll
                    for (int cc = 0; cc < B; cc += 2) fma2_bcast(bat[i][cc], bat[i][cc + 1], q[i], w[cc], w[cc + 1]);
            } else {
#pragma unroll
                for (int i = 0; i < CPL; ++i)
#pragma unroll
                    for (int cc = 0; cc < B; ++cc) bat[i][cc] = fma(q[i], w[cc], bat[i][cc]);
            }
        }
#pragma unroll
        for (int i = 0; i < CPL; ++i)
#pragma unroll
            for (int cc = 0; cc < B; ++cc) acc[i][cc] = add_any(acc[i][cc], bat[i][cc]);
        if ((k % nst) == nst - 1) {
            // last stage of block j: butterfly over the RL row lanes
            const int j = grp + (k / nst) * ngrp;
            T v[NV];
#pragma unroll
            for (int e = 0; e < NV; ++e) v[e] = acc[e / B][e % B];
#pragma unroll
            for (int kk = 0; kk < LOGRL; ++kk) {
                const int o = (1 << kk) * LPR;
                const bool up = (t & (1 << kk)) != 0;
                if ((NV >> kk) > 1) {
                    const int hv = NV >> (kk + 1);
#pragma unroll
                    for (int x = 0; x < NV / 2; ++x) {
                        if (x < hv) {
                            const T send = up ? v[x] : v[x + hv];
                            const T keep = up ? v[x + hv] : v[x];
                            v[x] = add_any(keep, shfl_xor_any(0xffffffffu, send, o));
                        }
                    }
                } else {
                    v[0] = add_any(v[0], shfl_xor_any(0xffffffffu, v[0], o));
                }
            }
            if (writer) {
#pragma unroll
                for (int x = 0; x < NK; ++x) {
                    const int e = vbase + x;
                    const int i = e / B, cc = e % B;
                    part[(int64_t)(j * B + g * CPL + i) * B + cc] += (double)v[x];
                }
            }
#pragma unroll
            for (int i = 0; i < CPL; ++i)
#pragma unroll
                for (int cc = 0; cc < B; ++cc) acc[i][cc] = T(0);
        }
    }
    cp_async_wait<0>();
    __syncwarp();
}

// Single problem: persistent CTAs take chunks of rc rows from the ticket
// counter and accumulate into their own wpb slots.
template <typename T, int B>
__global__ void __launch_bounds__(kThreads) gram_rows_kernel(int64_t n, int m, int wpb, int rc, int nchunks,
                                                             const T* __restrict__ Q, const T* __restrict__ W,
                                                             double* __restrict__ partial, int* __restrict__ ticket) {
    // [ W tile: layout [h][row][CPL] | per-warp rings: NS stages of SROWS rows ]
    extern __shared__ __align__(16) unsigned char gram_rows_smem[];
    T* ws = reinterpret_cast<T*>(gram_rows_smem);
    __shared__ int s_chunk;
    double* slots = partial + (int64_t)blockIdx.x * wpb * m * B;
    for (int64_t e = threadIdx.x; e < (int64_t)wpb * m * B; e += kThreads) slots[e] = 0.0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_chunk = atomicAdd(ticket, 1);
        __syncthreads();
        const int c = s_chunk;
        if (c >= nchunks) break;
        const int64_t r0 = (int64_t)c * rc;
        const int rows = (int)min((int64_t)rc, n - r0);
        gram_rows_chunk<T, B>(n, m, wpb, r0, rows, rc / wpb, Q, W, slots, ws);
    }
}

// Batch of problems stacked row-wise: CTA x takes chunk x, rows
// [chunks[3x+1], chunks[3x+2]) of segment chunks[3x] (at most R rows, never
// crossing a segment), and writes its own wpb slots at partial[x * wpb * m * B].
// m is read from device memory so that one captured graph serves every
// iteration; chunks of inactive segments do nothing.
template <typename T, int B>
__global__ void __launch_bounds__(kThreads) gram_rows_seg_kernel(int64_t n, const int* __restrict__ d_m,
                                                                 const int64_t* __restrict__ chunks,
                                                                 const int* __restrict__ seg_active,
                                                                 const T* __restrict__ Q, const T* __restrict__ W,
                                                                 double* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char gram_rows_smem[];
    const int64_t seg = chunks[3 * blockIdx.x];
    if (seg_active && !seg_active[seg]) return;
    const int m = *d_m;
    const int wpb = gram_rows_wpb(m / B);
    const int64_t r0 = chunks[3 * blockIdx.x + 1];
    const int rows = (int)(chunks[3 * blockIdx.x + 2] - r0);
    double* slots = partial + (int64_t)blockIdx.x * wpb * m * B;
    for (int64_t e = threadIdx.x; e < (int64_t)wpb * m * B; e += kThreads) slots[e] = 0.0;
    gram_rows_chunk<T, B>(n, m, wpb, r0, rows, (rows + wpb - 1) / wpb, Q, W, slots,
                          reinterpret_cast<T*>(gram_rows_smem));
}

// Segmented Gram for a batch of independent problems stacked row-wise:
// chunk x covers rows [chunks[3x+1], chunks[3x+2]) of segment chunks[3x];
// chunks of inactive segments do nothing.
template <typename T, int B, int CPT>
__global__ void __launch_bounds__(kThreads) gram_seg_kernel(int64_t n, int m, const int64_t* __restrict__ chunks,
                                                            const int* __restrict__ seg_active, int TC,
                                                            const T* __restrict__ Q, const T* __restrict__ W,
                                                            double* __restrict__ partial) {
    const int64_t seg = chunks[3 * blockIdx.x];
    if (seg_active && !seg_active[seg]) return;
    gram_body<T, B, CPT>(n, m, OneRange{chunks[3 * blockIdx.x + 1], chunks[3 * blockIdx.x + 2]}, TC, blockIdx.y, Q, W,
                         partial + (int64_t)blockIdx.x * m * B);
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

// out[e] = sum_p partial[p * count + e]: 32 entries per CTA, the parts split
// over 8 warps (coalesced 256-byte rows), combined in a fixed order.
__global__ void __launch_bounds__(256) reduce_partials_kernel(int64_t count, int nparts,
                                                              const double* __restrict__ partial,
                                                              double* __restrict__ out) {
    __shared__ double red[8][33];
    const int tx = threadIdx.x & 31, pg = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * 32 + tx;
    double s = 0.0;
    if (e < count) {
        int p = pg;
        for (; p + 24 < nparts; p += 32) {
            const double a0 = partial[(int64_t)p * count + e];
            const double a1 = partial[(int64_t)(p + 8) * count + e];
            const double a2 = partial[(int64_t)(p + 16) * count + e];
            const double a3 = partial[(int64_t)(p + 24) * count + e];
            s += a0;
            s += a1;
            s += a2;
            s += a3;
        }
        for (; p < nparts; p += 8) s += partial[(int64_t)p * count + e];
    }
    red[pg][tx] = s;
    __syncthreads();
    if (pg == 0 && e < count) {
        double t = red[0][tx];
        for (int q = 1; q < 8; ++q) t += red[q][tx];
        out[e] = t;
    }
}

void launch_reduce(int64_t count, int nparts, const double* partial, double* out, cudaStream_t st) {
    reduce_partials_kernel<<<(unsigned)ceil_div(count, 32), 256, 0, st>>>(count, nparts, partial, out);
}

// Self Gram G = W^T W for b <= 8 (CholQR2): a thread per row (grid-strided),
// the b(b+1)/2 distinct products in registers, then a warp-shuffle and
// shared-memory reduction to one B x B partial per CTA.
template <typename T, int B>
__global__ void __launch_bounds__(kThreads) syrk_kernel(int64_t n, const T* __restrict__ W, double* __restrict__ partial) {
    constexpr int NP = B * (B + 1) / 2;
    __shared__ double red[kThreads / 32][NP];
    T acc[NP];
#pragma unroll
    for (int e = 0; e < NP; ++e) acc[e] = T(0);
    double acc64[NP];
#pragma unroll
    for (int e = 0; e < NP; ++e) acc64[e] = 0.0;
    int cnt = 0;
    for (int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x; r < n; r += (int64_t)gridDim.x * kThreads) {
        T w[B];
        if constexpr (B * sizeof(T) >= 16) {
            constexpr int CH = 16 / (int)sizeof(T);
#pragma unroll
            for (int ch = 0; ch < B / CH; ++ch) {
                T t[CH];
                ldvec<T, CH>(W + r * B + ch * CH, t);
#pragma unroll
                for (int q = 0; q < CH; ++q) w[ch * CH + q] = t[q];
            }
        } else {
            ldvec<T, B>(W + r * B, w);
        }
        int e = 0;
#pragma unroll
        for (int i = 0; i < B; ++i)
#pragma unroll
            for (int k = i; k < B; ++k) {
                acc[e] = fma(w[i], w[k], acc[e]);
                ++e;
            }
        if (++cnt == 64) {  // FP32 runs of at most 64 rows, summed in FP64
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                acc64[q] += (double)acc[q];
                acc[q] = T(0);
            }
            cnt = 0;
        }
    }
    // warp tree in the data type (FP32 sums of at most 64 rows per lane,
    // then 32 lanes); the FP64 flushes only exist when a lane saw more rows
    const bool flushed = n > (int64_t)64 * gridDim.x * kThreads;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        T vt = acc[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) vt = add_any(vt, shfl_xor_any(0xffffffffu, vt, off));
        double v = (double)vt;
        if (flushed) {
            double v64 = acc64[q];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v64 += __shfl_xor_sync(0xffffffffu, v64, off);
            v += v64;
        }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < NP) {
        double v = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) v += red[w][threadIdx.x];
        // unpack the upper-triangle index into (i, k) and store both halves
        int i = 0, e = threadIdx.x;
        while (e >= B - i) {
            e -= B - i;
            ++i;
        }
        const int k = i + e;
        partial[(int64_t)blockIdx.x * B * B + i * B + k] = v;
        partial[(int64_t)blockIdx.x * B * B + k * B + i] = v;
    }
}

template <typename T, int B>
bbl_status launch_syrk(int64_t n, const T* W, double* G, DevBuf& partials, cudaStream_t st) {
    const int grid = (int)std::min<int64_t>(152 * 4, std::max<int64_t>(1, ceil_div(n, kThreads)));
    const size_t need = sizeof(double) * (size_t)grid * B * B;
    BBL_TRY(partials.grow(need));
    syrk_kernel<T, B><<<grid, kThreads, 0, st>>>(n, W, partials.as<double>());
    BBL_LAUNCH_CHECK();
    launch_reduce((int64_t)B * B, grid, partials.as<double>(), G, st);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    }
    return n;
}

// Column groups of the split-K Gram for m basis columns: each thread of a
// CTA owns CPT columns, so a group covers up to kThreads * CPT columns, and
// each group has its own chunk ticket.
template <int CPT>
int gram_groups(int m) {
    const int cols = (m + CPT - 1) / CPT;
    return (cols + kThreads - 1) / kThreads;
}

// Launches the persistent split-K Gram and the reduction of its per-worker
// partials.  partial: room for `cap` doubles; tickets: room for `ticket_cap`
// ints, of which gram_groups<CPT>(m) are zeroed here and used (a request
// needing more is refused before any launch).
template <typename T, int B, int CPT>
bbl_status gram_core(int64_t n, int m, const T* Q, const T* W, double* C, double* partial, int64_t cap, int* tickets,
                     int64_t ticket_cap, cudaStream_t st) {
    int cols = (m + CPT - 1) / CPT;
    int TC = 1;
    while (TC < cols && TC < kThreads) TC <<= 1;
    const int gy = (cols + TC - 1) / TC;
    if (gy != gram_groups<CPT>(m) || gy > ticket_cap)
        return set_error(BBL_ERR_INVALID_ARG, "gram: %d column groups exceed the %lld chunk tickets", gy,
                         (long long)ticket_cap);
    const int RS = kThreads / TC;
    // FP32 data keeps its FP64 running sums in shared memory; FP64 data needs
    // the buffer only for the reduction over row slots
    const size_t smem_max = sizeof(double) * kThreads * CPT * B;
    const size_t smem = (RS > 1 || sizeof(T) == 4) ? smem_max : 0;
    static int occ = 0;
    if (occ == 0) {
        BBL_CUDA(cudaFuncSetAttribute(gram_kernel<T, B, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
        BBL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gram_kernel<T, B, CPT>, kThreads, smem_max));
        if (occ < 1) occ = 1;
    }
    const int64_t rpc = 4 * kRT;
    const int nch = (int)std::max<int64_t>(1, ceil_div(n, rpc));
    const int64_t per = (int64_t)m * B;
    int64_t workers = std::max<int64_t>(1, (int64_t)sm_count() * occ / gy);
    workers = std::min<int64_t>(workers, nch);
    workers = std::min<int64_t>(workers, cap / per);
    if (workers < 1)
        return set_error(BBL_ERR_INVALID_ARG, "gram: %lld partial sums exceed the %lld-double scratch", (long long)per,
                         (long long)cap);
    BBL_CUDA(cudaMemsetAsync(tickets, 0, sizeof(int) * gy, st));
    dim3 grid((unsigned)workers, (unsigned)gy);
    gram_kernel<T, B, CPT><<<grid, kThreads, smem, st>>>(n, m, rpc, nch, TC, Q, W, partial, tickets);
    BBL_LAUNCH_CHECK();
    launch_reduce(per, (int)workers, partial, C, st);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

template <typename T, int B>
bbl_status launch_gram_rows(int64_t n, int m, const T* Q, const T* W, double* C, DevBuf& partials, cudaStream_t st) {
    using S = GramRowsShape<T, B>;
    static int occ = 0;
    if (occ == 0) {
        BBL_CUDA(cudaFuncSetAttribute(gram_rows_kernel<T, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)S::smem_bytes));
        BBL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gram_rows_kernel<T, B>, kThreads, S::smem_bytes));
        if (occ < 1) occ = 1;
    }
    const int nblocks = m / B;
    const int wpb = gram_rows_wpb(nblocks);  // warps per block when there are fewer blocks than warps
    // leave a few SMs to the Ritz solve that runs beside the main stream: a
    // persistent CTA that cannot start until such a kernel ends would hold the
    // whole Gram back
    const int64_t slots_max = (int64_t)std::max(1, sm_count() - kRitzReserveSMs) * occ;
    // rows per chunk: the full tile, or fewer so that small n still spreads
    // over the GPU (a multiple of RL * wpb)
    const int unit = S::RL * wpb;
    int64_t rc = ceil_div(n, slots_max);
    rc = std::max<int64_t>(unit * S::U, ceil_div(rc, unit) * unit);
    rc = std::min<int64_t>(rc, S::R);
    const int nch = (int)std::max<int64_t>(1, ceil_div(n, rc));
    const int64_t workers = std::min<int64_t>(slots_max, nch);
    const int64_t per = (int64_t)m * B;
    const int64_t slots = workers * wpb;
    const size_t need = sizeof(double) * (size_t)(slots * per) + 256;
    BBL_TRY(partials.grow(need));
    int* ticket = reinterpret_cast<int*>(partials.as<char>() + sizeof(double) * (size_t)(slots * per));
    BBL_CUDA(cudaMemsetAsync(ticket, 0, sizeof(int), st));
    gram_rows_kernel<T, B><<<(unsigned)workers, kThreads, S::smem_bytes, st>>>(n, m, wpb, (int)rc, nch, Q, W,
                                                                              partials.as<double>(), ticket);
    BBL_LAUNCH_CHECK();
    launch_reduce(per, (int)slots, partials.as<double>(), C, st);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

// First-pass Gram from an FP16 copy of an FP32 basis (b = 8): C ~= Q16^T W,
// on the tensor cores.  The first Gram-Schmidt pass only has to take out
// the bulk of W's component in span(Q) -- the FP32 second pass removes what
// is left, and A_j sums both passes' coefficients -- so its coefficients may
// carry FP16 roundings (relative 2^-11) of Q and of W, and the pass reads 2
// instead of 4 bytes per basis element.
//
// Persistent CTAs take chunks of kHalfRows rows from a ticket counter.  W's
// rows of the chunk are scaled by an exact power of two (the chunk's largest
// |W| lands in [2^13, 2^14)) and rounded to FP16 into shared memory.  Warp w
// owns the pairs of basis blocks p = w, w + 8, ...: per 16 rows a pair is a
// 16 x 16 FP16 tile A (16 basis columns x 16 rows), brought into a per-warp
// shared-memory ring by cp.async (one 16-byte row per lane, kHmSK tiles per
// stage, kHmNS stages) and loaded transposed with ldmatrix; W's 16 x 8 tile
// is the B operand; one mma.sync.m16n8k16 (FP16 in, FP32 accumulate) adds
// the pair's 16 x 8 block of C.  Over a chunk the sums stay in FP32; at the
// chunk's end they are unscaled (exactly) and added to the CTA's FP64 slot
// (m x 8), reduced over the CTAs afterwards.
constexpr int kHalfRows = 1024;
constexpr int kHmSK = 2;   // 16-row tiles per ring stage
constexpr int kHmNS = 3;   // ring stages per warp
constexpr int kHmWarps = kThreads / 32;

__device__ __forceinline__ void ldsm_x4_trans(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_trans(unsigned& r0, unsigned& r1, const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}
// D (16x8 FP32) += A (16x16 FP16, row) * B (16x8 FP16, col)
__device__ __forceinline__ void mma_16816(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(kThreads) gram_half_kernel(int64_t n, int m, int nchunks,
                                                             const __half* __restrict__ Q, const float* __restrict__ W,
                                                             double* __restrict__ partial, int* __restrict__ ticket) {
    constexpr int B = 8;
    constexpr int STAGE = kHmSK * 32 * B;  // halves per ring stage (kHmSK tiles of 32 rows of 16 bytes)
    __shared__ __align__(16) __half ws[kHalfRows * B];
    __shared__ __align__(16) __half ring[kHmWarps][kHmNS][STAGE];
    __shared__ float s_max[kHmWarps];
    __shared__ int s_chunk;
    const int nblocks = m / B;
    const int npairs = (nblocks + 1) / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tig = lane & 3;
    double* part = partial + (int64_t)blockIdx.x * m * B;
    for (int e = threadIdx.x; e < m * B; e += kThreads) part[e] = 0.0;
    const int mypairs = warp < npairs ? (npairs - warp + kHmWarps - 1) / kHmWarps : 0;
    constexpr int NST = kHalfRows / 16 / kHmSK;  // stages per pair per chunk
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_chunk = atomicAdd(ticket, 1);
        __syncthreads();
        const int c = s_chunk;
        if (c >= nchunks) break;
        const int64_t r0 = (int64_t)c * kHalfRows;
        const int rows = (int)min((int64_t)kHalfRows, n - r0);
        // the chunk's largest |W| -> power-of-two scale
        float mx = 0.f;
        for (int e = threadIdx.x; e < rows * B; e += kThreads) mx = fmaxf(mx, fabsf(W[r0 * B + e]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) s_max[warp] = mx;
        __syncthreads();
        mx = 0.f;
#pragma unroll
        for (int w = 0; w < kHmWarps; ++w) mx = fmaxf(mx, s_max[w]);
        int ex = 0;
        if (mx > 0.f) frexpf(mx, &ex);
        const float scale = ldexpf(1.f, 14 - ex);
        const double unscale = ldexp(1.0, ex - 14);
        for (int e = threadIdx.x; e < kHalfRows * B; e += kThreads)
            ws[e] = __float2half_rn(e < rows * B ? W[r0 * B + e] * scale : 0.f);
        __syncthreads();
        const int total = mypairs * NST;
        // ring stage k: pair warp + (k / NST) * kHmWarps, rows (k % NST) * 16 * kHmSK ..
        // lane L copies row (L & 15) of block 2p + (L >> 4) for each tile u
        auto issue = [&](int k) {
            if (k < total) {
                const int p = warp + (k / NST) * kHmWarps;
                const int j = 2 * p + (lane >> 4);
                __half* buf = ring[warp][k % kHmNS];
#pragma unroll
                for (int u = 0; u < kHmSK; ++u) {
                    const int rr = (k % NST) * 16 * kHmSK + u * 16 + (lane & 15);
                    const bool ok = j < nblocks && rr < rows;
                    cp_async16(buf + (u * 32 + lane) * B, ok ? (const void*)(Q + ((int64_t)j * n + r0 + rr) * B)
                                                             : (const void*)Q, ok ? 16 : 0);
                }
            }
            cp_async_commit();
        };
#pragma unroll
        for (int k = 0; k < kHmNS - 1; ++k) issue(k);
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        // ldmatrix row addresses: A, matrix q = lane >> 3 (rows 0-7 / 8-15 of blocks 0 / 1), row lane & 7
        const int a_row = ((lane >> 3) & 1) * 16 + (lane >> 4) * 8 + (lane & 7);
        const int b_row = ((lane >> 3) & 1) * 8 + (lane & 7);
        for (int k = 0; k < total; ++k) {
            cp_async_wait<kHmNS - 2>();
            __syncwarp();
            issue(k + kHmNS - 1);  // into the stage consumed at k - 1
            const __half* buf = ring[warp][k % kHmNS];
#pragma unroll
            for (int u = 0; u < kHmSK; ++u) {
                unsigned a[4], bq[2];
                ldsm_x4_trans(a[0], a[1], a[2], a[3], buf + (u * 32 + a_row) * B);
                const int kk = (k % NST) * kHmSK + u;  // 16-row tile of the chunk
                ldsm_x2_trans(bq[0], bq[1], ws + (kk * 16 + b_row) * B);
                mma_16816(acc, a, bq);
            }
            if ((k % NST) == NST - 1) {
                // the pair's sums over this chunk: rows g (block 2p) and g + 8 (block 2p + 1), columns 2 tig, 2 tig + 1
                const int p = warp + (k / NST) * kHmWarps;
                const int j0 = 2 * p, j1 = 2 * p + 1;
                double* o0 = part + ((int64_t)j0 * B + g) * B + 2 * tig;
                o0[0] += (double)acc[0] * unscale;
                o0[1] += (double)acc[1] * unscale;
                if (j1 < nblocks) {
                    double* o1 = part + ((int64_t)j1 * B + g) * B + 2 * tig;
                    o1[0] += (double)acc[2] * unscale;
                    o1[1] += (double)acc[3] * unscale;
                }
                acc[0] = acc[1] = acc[2] = acc[3] = 0.f;
            }
        }
        cp_async_wait<0>();
    }
}

bbl_status launch_gram_half(int64_t n, int m, const __half* Q, const float* W, double* C, DevBuf& partials,
                            cudaStream_t st) {
    static int occ = 0;
    if (occ == 0) {
        BBL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gram_half_kernel, kThreads, 0));
        if (occ < 1) occ = 1;
    }
    const int64_t slots_max = (int64_t)std::max(1, sm_count() - kRitzReserveSMs) * occ;
    const int nch = (int)std::max<int64_t>(1, ceil_div(n, kHalfRows));
    const int64_t workers = std::min<int64_t>(slots_max, nch);
    const int64_t per = (int64_t)m * 8;
    const size_t need = sizeof(double) * (size_t)(workers * per) + 256;
    BBL_TRY(partials.grow(need));
    int* ticket = reinterpret_cast<int*>(partials.as<char>() + sizeof(double) * (size_t)(workers * per));
    BBL_CUDA(cudaMemsetAsync(ticket, 0, sizeof(int), st));
    gram_half_kernel<<<(unsigned)workers, kThreads, 0, st>>>(n, m, nch, Q, W, partials.as<double>(), ticket);
    BBL_LAUNCH_CHECK();
    launch_reduce(per, (int)workers, partials.as<double>(), C, st);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

__global__ void f32_to_f16_kernel(int64_t count, const float* __restrict__ in, __half* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = __float2half_rn(in[e]);
}

template <typename T, int B, int CPT>
bbl_status launch_gram(int64_t n, int m, const T* Q, const T* W, double* C, DevBuf& partials, cudaStream_t st) {
    const int64_t per = (int64_t)m * B;
    const int64_t cap = per * (int64_t)sm_count() * 8;        // enough for any occupancy
    const int64_t gy = gram_groups<CPT>(m);                   // one ticket per column group
    const size_t ticket_bytes = 256 * (size_t)ceil_div(gy * (int64_t)sizeof(int), 256);
    const size_t need = sizeof(double) * (size_t)cap + ticket_bytes;
    BBL_TRY(partials.grow(need));
    int* tickets = reinterpret_cast<int*>(partials.as<char>() + sizeof(double) * (size_t)cap);
    return gram_core<T, B, CPT>(n, m, Q, W, C, partials.as<double>(), cap, tickets,
                                (int64_t)(ticket_bytes / sizeof(int)), st);
}

template <typename T>
bbl_status launch_gram_generic(int64_t n, int m, int b, const T* Q, const T* W, double* C, DevBuf& partials,
                               cudaStream_t st) {
    int TC = 1;
    while (TC < m && TC < kThreads) TC <<= 1;
    const int gy = (m + TC - 1) / TC;
    int64_t target = std::max<int64_t>(1, (152 * 2) / gy);
    int64_t rpc = std::max<int64_t>(kRT * 4, ceil_div(n, target));
    rpc = ceil_div(rpc, kRT) * kRT;
    const int64_t nch = std::max<int64_t>(1, ceil_div(n, rpc));
    const size_t need = sizeof(double) * (size_t)nch * m * b;
    BBL_TRY(partials.grow(need));
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
    launch_reduce(count, (int)nch, partials.as<double>(), C, st);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

template <typename T>
bbl_status gram_typed(int64_t n, int b, int m, const T* Q, const T* W, double* C, DevBuf& partials, cudaStream_t st) {
    switch (b) {
        case 1: return launch_gram<T, 1, 1>(n, m, Q, W, C, partials, st);
        case 2: return launch_gram<T, 2, 2>(n, m, Q, W, C, partials, st);
        case 4: return launch_gram_rows<T, 4>(n, m, Q, W, C, partials, st);
        case 8: return launch_gram_rows<T, 8>(n, m, Q, W, C, partials, st);
        case 16: return launch_gram<T, 16, 2>(n, m, Q, W, C, partials, st);
        default: return launch_gram_generic<T>(n, m, b, Q, W, C, partials, st);
    }
}

// -------------------------------------------------------------------- apply
// W[r][c] (SUB ? -= : =) sum_a Q[r][a] C[a][c], c < kc.  Q: nblocks blocks of
// n x B; C: m x kc FP64 row-major; W: n x kc (type TO).  TA: accumulation type.
constexpr int kKT = 256;
// One CTA: rows r = row0 + threadIdx.x (r < row_end) of W (-)= Q C.
template <typename T, int B, int KCT, bool SUB, typename TA, typename TO>
__device__ __forceinline__ void apply_body(int64_t n, int m, int kc, int64_t row0, int64_t row_end, const T* Q,
                                           const double* __restrict__ C, TO* W) {
    constexpr int KM = KCT > 0 ? KCT : kMaxB;
    // FP32 sums into an FP64 result: FP32 within a tile of kKT columns, FP64
    // across tiles
    constexpr bool kTiled = sizeof(TA) == 4 && !is_df32<TA>::value && sizeof(TO) == 8;
    __shared__ TA cs[kKT * KM];
    const int tid = threadIdx.x;
    const int64_t r = row0 + tid;
    const int64_t rlim = row_end;
    TA acc[KM];
    double acc64[kTiled ? KM : 1];
#pragma unroll
    for (int c = 0; c < KM; ++c) acc[c] = TA(0);
    if constexpr (kTiled) {
#pragma unroll
        for (int c = 0; c < KM; ++c) acc64[c] = 0.0;
    }
    for (int a0 = 0; a0 < m; a0 += kKT) {
        const int rows = min(kKT, m - a0);
        __syncthreads();
        for (int e = tid; e < rows * KM; e += kThreads) {
            const int a = e / KM, c = e % KM;
            cs[e] = (c < kc) ? (TA)C[(int64_t)(a0 + a) * kc + c] : TA(0);
        }
        __syncthreads();
        if (r < rlim) {
#pragma unroll 4
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
        if constexpr (kTiled) {
#pragma unroll
            for (int c = 0; c < KM; ++c) {
                acc64[c] += (double)acc[c];
                acc[c] = TA(0);
            }
        }
    }
    if (r < rlim) {
#pragma unroll
        for (int c = 0; c < KM; ++c) {
            if (c < kc) {
                TO* w = W + r * kc + c;
                if constexpr (kTiled) {
                    if (SUB) *w = (TO)((double)(*w) - acc64[c]);
                    else *w = (TO)acc64[c];
                } else {
                    if (SUB) *w = (TO)((TA)(*w) - acc[c]);
                    else *w = (TO)acc[c];
                }
            }
        }
    }
}

template <typename T, int B, int KCT, bool SUB, typename TA, typename TO>
__global__ void __launch_bounds__(kThreads) apply_kernel(int64_t n, int m, int kc, const T* Q, const double* __restrict__ C,
                                                         TO* W) {
    apply_body<T, B, KCT, SUB, TA, TO>(n, m, kc, (int64_t)blockIdx.x * kThreads, n, Q, C, W);
}

// Segmented apply: CTA x handles rows [ctas[3x+1], ctas[3x+2]) (at most 256)
// of segment s = ctas[3x], with that segment's coefficients C + s*cstride and
// m = ms[s * ms_stride] basis columns (ms_stride 0: one shared count; ms NULL:
// m_all); inactive segments skip.
template <typename T, int B, int KCT, bool SUB, typename TA, typename TO>
__global__ void __launch_bounds__(kThreads) apply_seg_kernel(int64_t n, int m_all, const int* __restrict__ ms,
                                                             int ms_stride, int kc,
                                                             const int64_t* __restrict__ ctas,
                                                             const int* __restrict__ seg_active, const T* Q,
                                                             const double* __restrict__ C, int64_t cstride, TO* W) {
    const int64_t seg = ctas[3 * blockIdx.x];
    if (seg_active && !seg_active[seg]) return;
    const int m = ms ? ms[seg * ms_stride] : m_all;
    apply_body<T, B, KCT, SUB, TA, TO>(n, m, kc, ctas[3 * blockIdx.x + 1], ctas[3 * blockIdx.x + 2], Q,
                                       C + seg * cstride, W);
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

// First-pass update of the FP32 stage, b = 8, with the older blocks read
// from the FP16 copy: W -= sum_j Q_j C_j.  In Lanczos the first pass's
// coefficients of the blocks older than the two newest are of the order of
// the lost orthogonality (about 1e-7 of ||W|| in FP32): the FP16 rounding
// of those blocks (2^-12 relative) changes W by about 2^-12 of that, far
// below W's own FP32 rounding, and a rounding of their coefficients is a
// change of the coefficients only (it stays in span(Q), and the second
// pass removes it).  So the older blocks' product runs on the tensor cores
// straight from the FP16 copy (mma.sync m16n8k16, FP16 in, FP32
// accumulate): C's rows of those blocks are scaled by one power of two s
// (the largest entry to [2^13, 2^14)) and rounded to FP16, and the sum is
// multiplied by 1/s.  The newest blocks (jsplit and up), whose coefficients
// are A_j and B_{j-1}^T, are FP32 FMA products with C rounded to FP32, as
// in the FP32 update.

// B fragments of the older blocks' product, per block pair q (blocks 2q,
// 2q + 1 < jsplit, the second zero past it) and lane (g = lane / 4, t = lane
// % 4): {C rows 16q + 2t, +1 | C rows 16q + 8 + 2t, +1}, column g, times s,
// in FP16 pairs (low half = lower row); scale[0] = 1/s.  One CTA.
__global__ void __launch_bounds__(256) half_old_prep_kernel(int jsplit, const double* __restrict__ C,
                                                            uint2* __restrict__ frag, float* __restrict__ scale) {
    __shared__ double smax[256];
    double mx = 0.0;
    for (int e = threadIdx.x; e < jsplit * 64; e += 256) mx = fmax(mx, fabs(C[e]));
    smax[threadIdx.x] = mx;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + w]);
        __syncthreads();
    }
    mx = smax[0];
    int ex = 0;
    if (mx > 0.0) (void)frexp(mx, &ex);  // mx = f 2^ex, f in [0.5, 1)
    // max * sc in [2^13, 2^14); coefficients below 2^-100 (negligible) keep
    // sc = 2^114, so that sc and 1/sc stay finite and normal in FP32
    ex = ex < -100 ? -100 : ex;
    const double sc = (mx > 0.0) ? ldexp(1.0, 14 - ex) : 1.0;
    if (threadIdx.x == 0) scale[0] = (float)(1.0 / sc);
    const int npo = (jsplit + 1) >> 1;
    for (int e = threadIdx.x; e < npo * 32; e += 256) {
        const int q = e >> 5, lane = e & 31, g = lane >> 2, t = lane & 3;
        const int ra = 16 * q + 2 * t, rb = 16 * q + 8 + 2 * t;
        const bool two = 2 * q + 1 < jsplit;
        const __half2 b0 = __floats2half2_rn((float)(C[ra * 8 + g] * sc), (float)(C[(ra + 1) * 8 + g] * sc));
        const __half2 b1 = two ? __floats2half2_rn((float)(C[rb * 8 + g] * sc), (float)(C[(rb + 1) * 8 + g] * sc))
                               : __floats2half2_rn(0.f, 0.f);
        frag[e] = make_uint2(*reinterpret_cast<const unsigned*>(&b0), *reinterpret_cast<const unsigned*>(&b1));
    }
}

// One warp per 16-row tile.  A fragments of the older blocks come straight
// from global memory (each 4-byte load of a warp covers 8 rows x 16 bytes
// of one block: one 128-byte line).
__global__ void __launch_bounds__(256) apply_half_old_kernel(int64_t n, int nblocks, int jsplit,
                                                             const __half* __restrict__ Q16,
                                                             const float* __restrict__ Q,
                                                             const double* __restrict__ C,
                                                             const uint2* __restrict__ frag,
                                                             const float* __restrict__ scale, float* __restrict__ W) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t r0 = tile * 16;
    if (r0 >= n) return;
    const int64_t ra = r0 + g, rb = r0 + g + 8;
    const bool oka = ra < n, okb = rb < n;
    const unsigned* Q16w = reinterpret_cast<const unsigned*>(Q16);  // two halves per word
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    const int npo = (jsplit + 1) >> 1;
    // groups of kHoU block pairs: every load of a group is issued before its products
    constexpr int kHoU = 8;
    for (int q0 = 0; q0 < npo; q0 += kHoU) {
        unsigned a[kHoU][4];
        unsigned b[kHoU][2];
#pragma unroll
        for (int u = 0; u < kHoU; ++u) {
            const int q = q0 + u;
            const bool on = q < npo;
            const int j0 = on ? 2 * q : 0;
            const int j1 = (on && 2 * q + 1 < nblocks) ? 2 * q + 1 : j0;  // past the basis: b1 is zero
            a[u][0] = (on && oka) ? __ldg(Q16w + (((int64_t)j0 * n + ra) * 8 + 2 * t) / 2) : 0u;
            a[u][1] = (on && okb) ? __ldg(Q16w + (((int64_t)j0 * n + rb) * 8 + 2 * t) / 2) : 0u;
            a[u][2] = (on && oka) ? __ldg(Q16w + (((int64_t)j1 * n + ra) * 8 + 2 * t) / 2) : 0u;
            a[u][3] = (on && okb) ? __ldg(Q16w + (((int64_t)j1 * n + rb) * 8 + 2 * t) / 2) : 0u;
            const uint2 f = on ? __ldg(frag + q * 32 + lane) : make_uint2(0u, 0u);
            b[u][0] = f.x;
            b[u][1] = f.y;
        }
#pragma unroll
        for (int u = 0; u < kHoU; ++u)
            if (q0 + u < npo) mma_16816(d, a[u], b[u]);
    }
    const float inv = npo > 0 ? __ldg(scale) : 0.f;
    // acc[row][col]: rows ra / rb, columns 2t, 2t + 1
    float acc[2][2] = {{d[0] * inv, d[1] * inv}, {d[2] * inv, d[3] * inv}};
    for (int j = jsplit; j < nblocks; ++j) {
        float cj[8][2];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            cj[i][0] = (float)__ldg(C + (8 * j + i) * 8 + 2 * t);
            cj[i][1] = (float)__ldg(C + (8 * j + i) * 8 + 2 * t + 1);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t rr = h ? rb : ra;
            if (rr < n) {
                const float4 x0 = __ldg(reinterpret_cast<const float4*>(Q + ((int64_t)j * n + rr) * 8));
                const float4 x1 = __ldg(reinterpret_cast<const float4*>(Q + ((int64_t)j * n + rr) * 8 + 4));
                const float qv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    acc[h][0] = fmaf(qv[i], cj[i][0], acc[h][0]);
                    acc[h][1] = fmaf(qv[i], cj[i][1], acc[h][1]);
                }
            }
        }
    }
    if (oka) {
        float2* w = reinterpret_cast<float2*>(W + ra * 8 + 2 * t);
        const float2 v = *w;
        *w = make_float2(v.x - acc[0][0], v.y - acc[0][1]);
    }
    if (okb) {
        float2* w = reinterpret_cast<float2*>(W + rb * 8 + 2 * t);
        const float2 v = *w;
        *w = make_float2(v.x - acc[1][0], v.y - acc[1][1]);
    }
}

// Update of the float-float polish, b = 8: W -= sum_j Q_j C_j with the
// blocks older than jsplit read from the FP32 copy of the basis (the high
// parts) with FP32 products and sums, the newer ones from the float-float
// basis with float-float products.  The older blocks' coefficients are the
// lost orthogonality and the FP32 first-pass Gram's error, so their FP32
// products (2^-24 relative) change W far below its float-float rounding;
// their bytes halve and their arithmetic is one FMA per product.
__global__ void __launch_bounds__(kThreads) apply_df32_f32old_kernel(int64_t n, int m, int jsplit,
                                                                     const float* __restrict__ Q32,
                                                                     const df32* __restrict__ Q,
                                                                     const double* __restrict__ C, df32* W) {
    constexpr int B = 8;
    __shared__ df32 cs[kKT * B];
    const int tid = threadIdx.x;
    const int64_t r = (int64_t)blockIdx.x * kThreads + tid;
    float a32[B];
    df32 adf[B];
#pragma unroll
    for (int c = 0; c < B; ++c) {
        a32[c] = 0.f;
        adf[c] = df32(0.f);
    }
    for (int a0 = 0; a0 < m; a0 += kKT) {
        const int rows = min(kKT, m - a0);
        __syncthreads();
        for (int e = tid; e < rows * B; e += kThreads) cs[e] = df32(C[(int64_t)a0 * B + e]);
        __syncthreads();
        if (r < n) {
            for (int jb = 0; jb < rows; jb += B) {
                const int j = (a0 + jb) / B;
                const df32* cr = cs + jb * B;
                if (j < jsplit) {
                    const float4 x0 = __ldg(reinterpret_cast<const float4*>(Q32 + ((int64_t)j * n + r) * B));
                    const float4 x1 = __ldg(reinterpret_cast<const float4*>(Q32 + ((int64_t)j * n + r) * B + 4));
                    const float q[B] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                    for (int i = 0; i < B; ++i)
#pragma unroll
                        for (int c = 0; c < B; ++c) a32[c] = fmaf(q[i], cr[i * B + c].hi, a32[c]);
                } else {
                    df32 q[B];
                    ldvec<df32, B>(Q + ((int64_t)j * n + r) * B, q);
#pragma unroll
                    for (int i = 0; i < B; ++i)
#pragma unroll
                        for (int c = 0; c < B; ++c) adf[c] = dfm::fma(q[i], cr[i * B + c], adf[c]);
                }
            }
        }
    }
    if (r < n) {
#pragma unroll
        for (int c = 0; c < B; ++c) {
            df32* w = W + r * B + c;
            *w = *w - (adf[c] + df32(a32[c]));
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
__device__ void chol_body(int b, const double* __restrict__ G, double thresh2, int relative, double* __restrict__ R,
                          double* __restrict__ Rinv, int* __restrict__ ndefl, int* __restrict__ mask,
                          int* __restrict__ status);

// One thread per segment: Cholesky of G + s*b*b with threshold thresh2[s].
__global__ void chol_seg_kernel(int b, int nseg, const double* __restrict__ G, const double* __restrict__ thresh2,
                                int relative, double* __restrict__ R, double* __restrict__ Rinv, int* __restrict__ ndefl,
                                int* __restrict__ mask, int* __restrict__ status, const int* __restrict__ active) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg || (active && !active[s])) return;
    const int64_t o = (int64_t)s * b * b;
    chol_body(b, G + o, thresh2 ? thresh2[s] : 0.0, relative, R + o, Rinv + o, ndefl ? ndefl + s : nullptr,
              mask ? mask + (int64_t)s * b : nullptr, status ? status + s : nullptr);
}

__global__ void trmul_seg_kernel(int b, int nseg, const double* __restrict__ R2, const double* __restrict__ R1,
                                 double* __restrict__ B, const int* __restrict__ active) {
    const int s = blockIdx.y;
    const int e = threadIdx.x;
    if (s >= nseg || e >= b * b || (active && !active[s])) return;
    const int64_t o = (int64_t)s * b * b;
    const int i = e / b, k = e % b;
    double acc = 0.0;
    for (int l = 0; l < b; ++l) acc += R2[o + i * b + l] * R1[o + l * b + k];
    B[o + e] = acc;
}

__device__ void chol_body(int b, const double* __restrict__ G, double thresh2, int relative, double* __restrict__ R,
                          double* __restrict__ Rinv, int* __restrict__ ndefl, int* __restrict__ mask,
                          int* __restrict__ status) {
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

// The same Cholesky with deflation by one warp: rows of R are formed one
// after the other (lane k computes R[i][k]), then lane c forms column c of
// R^{-1}.  Deflated columns get zero rows in R and zero columns in R^{-1}.
__global__ void __launch_bounds__(32) chol_warp_kernel(int b, const double* __restrict__ G, double thresh2, int relative,
                                                      double* __restrict__ R, double* __restrict__ Rinv,
                                                      int* __restrict__ ndefl, int* __restrict__ mask,
                                                      int* __restrict__ status) {
    __shared__ double Gs[kMaxB * kMaxB];
    __shared__ double Rs[kMaxB * kMaxB];
    __shared__ int dm[kMaxB];
    const int lane = threadIdx.x;
    int bad = 0;
    double gmax = 0.0;
    for (int e = lane; e < b * b; e += 32) {
        const double g = G[e];
        Gs[e] = g;
        Rs[e] = 0.0;
        if (!isfinite(g)) bad = 1;
    }
    bad = __any_sync(0xffffffffu, bad);
    __syncwarp();
    for (int q = 0; q < b; ++q) gmax = fmax(gmax, Gs[q * b + q]);
    if (relative) thresh2 *= gmax;
    int cnt = 0;
    for (int i = 0; i < b; ++i) {
        double d = Gs[i * b + i];
        for (int l = 0; l < i; ++l) d -= Rs[l * b + i] * Rs[l * b + i];
        const int defl = !(d > thresh2) || bad;
        cnt += defl;
        if (lane == 0) dm[i] = defl;
        if (!defl) {
            const double rii = sqrt(d);
            if (lane == i) Rs[i * b + i] = rii;
            if (lane > i && lane < b) {
                double t = Gs[i * b + lane];
                for (int l = 0; l < i; ++l) t -= Rs[l * b + i] * Rs[l * b + lane];
                Rs[i * b + lane] = t / rii;
            }
        }
        __syncwarp();
    }
    for (int e = lane; e < b * b; e += 32) R[e] = Rs[e];
    if (lane < b) {
        const int c = lane;
        double col[kMaxB];
#pragma unroll
        for (int q = 0; q < kMaxB; ++q) col[q] = 0.0;
        if (!dm[c]) {
            col[c] = 1.0 / Rs[c * b + c];
            for (int i = c - 1; i >= 0; --i) {
                if (dm[i]) continue;
                double t = 0.0;
                for (int k = i + 1; k <= c; ++k)
                    if (!dm[k]) t += Rs[i * b + k] * col[k];
                col[i] = -t / Rs[i * b + i];
            }
        }
        for (int q = 0; q < b; ++q) Rinv[q * b + c] = col[q];
        if (mask) mask[c] = dm[c];
    }
    if (lane == 0) {
        if (ndefl) *ndefl += cnt;
        if (bad && status) atomicOr(status, 1);
    }
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
void reduce_partials(int64_t count, int nparts, const double* partial, double* out, cudaStream_t st) {
    launch_reduce(count, nparts, partial, out, st);
}

int gram_worker_sms() { return std::max(1, sm_count() - kRitzReserveSMs); }

bbl_status gram(int64_t n, int b, int nblocks, int dtype, const void* Q, const void* W, double* C, DevBuf& partials,
                cudaStream_t st) {
    const int m = nblocks * b;
    if (dtype == BBL_FP64)
        return gram_typed<double>(n, b, m, static_cast<const double*>(Q), static_cast<const double*>(W), C, partials, st);
    if (dtype == kDF32)
        return gram_typed<df32>(n, b, m, static_cast<const df32*>(Q), static_cast<const df32*>(W), C, partials, st);
    return gram_typed<float>(n, b, m, static_cast<const float*>(Q), static_cast<const float*>(W), C, partials, st);
}

// C ~= Q16^T W for b = 8: Q16 the FP16 copy of an FP32 basis of nblocks blocks
bbl_status gram_half(int64_t n, int nblocks, const void* Q16, const float* W, double* C, DevBuf& partials,
                     cudaStream_t st) {
    return launch_gram_half(n, nblocks * 8, static_cast<const __half*>(Q16), W, C, partials, st);
}

// FP16 copy (round to nearest) of count FP32 values
bbl_status to_half(int64_t count, const float* in, void* out, cudaStream_t st) {
    f32_to_f16_kernel<<<152 * 8, 256, 0, st>>>(count, in, static_cast<__half*>(out));
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

bbl_status update(int64_t n, int b, int nblocks, int dtype, const void* Q, const double* C, void* W, cudaStream_t st) {
    const int m = nblocks * b;
    if (dtype == BBL_FP64)
        return apply_typed<double, true, double, double>(n, b, m, b, static_cast<const double*>(Q), C,
                                                         static_cast<double*>(W), st);
    if (dtype == kDF32)
        return apply_typed<df32, true, df32, df32>(n, b, m, b, static_cast<const df32*>(Q), C, static_cast<df32*>(W),
                                                   st);
    return apply_typed<float, true, float, float>(n, b, m, b, static_cast<const float*>(Q), C, static_cast<float*>(W),
                                                  st);
}

bbl_status update_half_old(int64_t n, int nblocks, int nnew, const void* Q16, const float* Q, const double* C,
                           float* W, DevBuf& work, cudaStream_t st) {
    const int jsplit = nblocks > nnew ? nblocks - nnew : 0;
    const int npo = (jsplit + 1) >> 1;
    BBL_TRY(work.grow(sizeof(uint2) * (size_t)npo * 32 + 256));
    uint2* frag = work.as<uint2>();
    float* scale = reinterpret_cast<float*>(work.as<char>() + sizeof(uint2) * (size_t)npo * 32);
    if (npo > 0) {
        half_old_prep_kernel<<<1, 256, 0, st>>>(jsplit, C, frag, scale);
        BBL_LAUNCH_CHECK();
    }
    const int64_t warps = ceil_div(n, (int64_t)16);
    apply_half_old_kernel<<<(unsigned)ceil_div(warps * 32, 256), 256, 0, st>>>(
        n, nblocks, jsplit, static_cast<const __half*>(Q16), Q, C, frag, scale, W);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

bbl_status update_df32_f32old(int64_t n, int nblocks, int nnew, const float* Q32, const void* Q, const double* C,
                             void* W, cudaStream_t st) {
    const int jsplit = nblocks > nnew ? nblocks - nnew : 0;
    apply_df32_f32old_kernel<<<(unsigned)ceil_div(n, kThreads), kThreads, 0, st>>>(
        n, nblocks * 8, jsplit, Q32, static_cast<const df32*>(Q), C, static_cast<df32*>(W));
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

bbl_status ritz_vectors(int64_t n, int b, int nblocks, int dtype, const void* Q, int k, const double* S, double* X,
                        cudaStream_t st) {
    const int m = nblocks * b;
    if (dtype == BBL_FP64)
        return apply_typed<double, false, double, double>(n, b, m, k, static_cast<const double*>(Q), S, X, st);
    if (dtype == kDF32)
        return apply_typed<df32, false, df32, double>(n, b, m, k, static_cast<const df32*>(Q), S, X, st);
    // FP32 blocks: FP32 products and sums (the vectors carry FP32 accuracy
    // anyway), FP64 output
    return apply_typed<float, false, float, double>(n, b, m, k, static_cast<const float*>(Q), S, X, st);
}

// small: >= 8*b*b doubles + 4*b ints.  B (device, b x b) receives R2 R1.
// G = W^T W (b x b): the dedicated kernel for b in {1, 2, 4, 8}, else the general Gram.
bbl_status self_gram(int64_t n, int b, int dtype, const void* W, double* G, DevBuf& partials, cudaStream_t st) {
    if (dtype == BBL_FP64) {
        auto w = static_cast<const double*>(W);
        switch (b) {
            case 1: return launch_syrk<double, 1>(n, w, G, partials, st);
            case 2: return launch_syrk<double, 2>(n, w, G, partials, st);
            case 4: return launch_syrk<double, 4>(n, w, G, partials, st);
            case 8: return launch_syrk<double, 8>(n, w, G, partials, st);
            default: break;
        }
    } else if (dtype == kDF32) {
        auto w = static_cast<const df32*>(W);
        switch (b) {
            case 1: return launch_syrk<df32, 1>(n, w, G, partials, st);
            case 2: return launch_syrk<df32, 2>(n, w, G, partials, st);
            case 4: return launch_syrk<df32, 4>(n, w, G, partials, st);
            case 8: return launch_syrk<df32, 8>(n, w, G, partials, st);
            default: break;
        }
    } else {
        auto w = static_cast<const float*>(W);
        switch (b) {
            case 1: return launch_syrk<float, 1>(n, w, G, partials, st);
            case 2: return launch_syrk<float, 2>(n, w, G, partials, st);
            case 4: return launch_syrk<float, 4>(n, w, G, partials, st);
            case 8: return launch_syrk<float, 8>(n, w, G, partials, st);
            default: break;
        }
    }
    return gram(n, b, 1, dtype, W, W, G, partials, st);
}

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
    BBL_TRY(self_gram(n, b, dtype, W, G, partials, st));
    chol_warp_kernel<<<1, 32, 0, st>>>(b, G, t1, relative, R1, R1i, d_ndefl, d_mask, status);
    BBL_LAUNCH_CHECK();
    if (dtype == BBL_FP64)
        BBL_TRY((apply_typed<double, false, double, double>(n, b, b, b, static_cast<double*>(W), R1i,
                                                             static_cast<double*>(W), st)));
    else if (dtype == kDF32)
        BBL_TRY((apply_typed<df32, false, df32, df32>(n, b, b, b, static_cast<df32*>(W), R1i, static_cast<df32*>(W),
                                                       st)));
    else
        BBL_TRY((apply_typed<float, false, float, float>(n, b, b, b, static_cast<float*>(W), R1i,
                                                          static_cast<float*>(W), st)));
    BBL_TRY(self_gram(n, b, dtype, W, G, partials, st));
    // second pass: columns of Q1 have norm ~1; a pivot below 1e-6 means the
    // first pass produced no usable direction (it was deflated or lost).
    chol_warp_kernel<<<1, 32, 0, st>>>(b, G, 1e-6, 0, R2, R2i, nullptr, nullptr, status);
    BBL_LAUNCH_CHECK();
    if (dtype == BBL_FP64)
        BBL_TRY((apply_typed<double, false, double, double>(n, b, b, b, static_cast<double*>(W), R2i,
                                                             static_cast<double*>(W), st)));
    else if (dtype == kDF32)
        BBL_TRY((apply_typed<df32, false, df32, df32>(n, b, b, b, static_cast<df32*>(W), R2i, static_cast<df32*>(W),
                                                       st)));
    else
        BBL_TRY((apply_typed<float, false, float, float>(n, b, b, b, static_cast<float*>(W), R2i,
                                                          static_cast<float*>(W), st)));
    if (B) {
        trmul_kernel<<<1, 256, 0, st>>>(b, R2, R1, B);
        BBL_LAUNCH_CHECK();
    }
    return BBL_OK;
}

// -------------------------------------------------------------------- segmented (batched) forms
// A batch of independent problems is stacked row-wise: segment s owns rows
// [off[s], off[s+1]) of every n_tot x b block.  Work tables are built once
// on the host: gram chunks (seg, r0, r1) never cross a segment, apply CTAs
// (seg, r0, r1) cover at most 256 rows of one segment.  The current number of
// basis columns may be read from device memory (d_m), so that one captured
// graph serves every iteration.
namespace {

// C[s] = sum of segment s's partial slots (rows_slots: the row-contiguous
// kernel's wpb slots per chunk, else one), in chunk order
__global__ void reduce_seg_kernel(int m_max, int b, const int* __restrict__ d_m, const int* __restrict__ seg_chunk_ptr,
                                  const int* __restrict__ active, const double* __restrict__ partial,
                                  double* __restrict__ C, int rows_slots) {
    const int s = blockIdx.y;
    if (active && !active[s]) return;
    const int m = d_m ? *d_m : m_max;
    const int per = rows_slots ? gram_rows_wpb(m / b) : 1;
    const int64_t count = (int64_t)m * b;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    double acc = 0.0;
    for (int c = seg_chunk_ptr[s] * per; c < seg_chunk_ptr[s + 1] * per; ++c) acc += partial[(int64_t)c * count + e];
    C[(int64_t)s * m_max * b + e] = acc;
}

template <typename T, int B>
bbl_status launch_gram_rows_seg(int64_t n, const int* d_m, const T* Q, const T* W, const int64_t* chunks, int nchunks,
                                const int* active, double* partial, cudaStream_t st) {
    using S = GramRowsShape<T, B>;
    static bool attr_set = false;
    if (!attr_set) {
        BBL_CUDA(cudaFuncSetAttribute(gram_rows_seg_kernel<T, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)S::smem_bytes));
        attr_set = true;
    }
    gram_rows_seg_kernel<T, B><<<(unsigned)nchunks, kThreads, S::smem_bytes, st>>>(n, d_m, chunks, active, Q, W,
                                                                                   partial);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

template <typename T, int B, int CPT>
__global__ void __launch_bounds__(kThreads) gram_seg_dyn_kernel(int64_t n, const int* __restrict__ d_m,
                                                                const int64_t* __restrict__ chunks,
                                                                const int* __restrict__ seg_active,
                                                                const T* __restrict__ Q, const T* __restrict__ W,
                                                                double* __restrict__ partial) {
    const int64_t seg = chunks[3 * blockIdx.x];
    if (seg_active && !seg_active[seg]) return;
    const int m = *d_m;
    const int cols = (m + CPT - 1) / CPT;
    int TC = 1;
    while (TC < cols && TC < kThreads) TC <<= 1;
    if ((int)blockIdx.y * TC * CPT >= m) return;
    gram_body<T, B, CPT>(n, m, OneRange{chunks[3 * blockIdx.x + 1], chunks[3 * blockIdx.x + 2]}, TC, blockIdx.y, Q, W,
                         partial + (int64_t)blockIdx.x * m * B);
}

template <typename T, int B, int CPT>
bbl_status launch_gram_seg(int64_t n, int m_max, const int* d_m, const T* Q, const T* W, const int64_t* chunks,
                           int nchunks, const int* active, double* partial, cudaStream_t st) {
    const int cols = (m_max + CPT - 1) / CPT;
    const int gy = (cols + kThreads - 1) / kThreads;
    static bool attr_set = false;
    if (!attr_set) {
        BBL_CUDA(cudaFuncSetAttribute(gram_seg_dyn_kernel<T, B, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(double) * kThreads * CPT * B)));
        attr_set = true;
    }
    dim3 grid((unsigned)nchunks, (unsigned)gy);
    gram_seg_dyn_kernel<T, B, CPT><<<grid, kThreads, sizeof(double) * kThreads * CPT * B, st>>>(n, d_m, chunks, active,
                                                                                                Q, W, partial);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

template <typename T, bool SUB, typename TA, typename TO, int B>
bbl_status launch_apply_seg(int64_t n, int kc, const int* ms, int mss, const int64_t* ctas, int nctas,
                            const int* active, const T* Q, const double* C, int64_t cstride, TO* W, cudaStream_t st) {
    if (kc == B)
        apply_seg_kernel<T, B, B, SUB, TA, TO><<<nctas, kThreads, 0, st>>>(n, 0, ms, mss, kc, ctas, active, Q, C,
                                                                          cstride, W);
    else
        apply_seg_kernel<T, B, 0, SUB, TA, TO><<<nctas, kThreads, 0, st>>>(n, 0, ms, mss, kc, ctas, active, Q, C,
                                                                          cstride, W);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

template <typename T, bool SUB, typename TA, typename TO>
bbl_status apply_seg_typed(int64_t n, int b, int kc, const int* ms, int mss, const int64_t* ctas, int nctas,
                           const int* active, const T* Q, const double* C, int64_t cstride, TO* W, cudaStream_t st) {
    switch (b) {
        case 1: return launch_apply_seg<T, SUB, TA, TO, 1>(n, kc, ms, mss, ctas, nctas, active, Q, C, cstride, W, st);
        case 2: return launch_apply_seg<T, SUB, TA, TO, 2>(n, kc, ms, mss, ctas, nctas, active, Q, C, cstride, W, st);
        case 4: return launch_apply_seg<T, SUB, TA, TO, 4>(n, kc, ms, mss, ctas, nctas, active, Q, C, cstride, W, st);
        case 8: return launch_apply_seg<T, SUB, TA, TO, 8>(n, kc, ms, mss, ctas, nctas, active, Q, C, cstride, W, st);
        case 16: return launch_apply_seg<T, SUB, TA, TO, 16>(n, kc, ms, mss, ctas, nctas, active, Q, C, cstride, W, st);
        default: return set_error(BBL_ERR_UNSUPPORTED, "batched: b=%d (supported: 1, 2, 4, 8, 16)", b);
    }
}

}  // namespace

int gram_seg_chunk_rows(int b, int dtype) {
    if (dtype == BBL_FP64) {
        if (b == 4) return GramRowsShape<double, 4>::R;
        if (b == 8) return GramRowsShape<double, 8>::R;
    } else if (dtype == BBL_FP32) {
        if (b == 4) return GramRowsShape<float, 4>::R;
        if (b == 8) return GramRowsShape<float, 8>::R;
        if (b == 16) return GramRowsShape<float, 16>::R;
    }
    return 0;
}

bbl_status gram_seg(int64_t n, int b, int m_max, const int* d_m, int dtype, const void* Q, const void* W,
                    const int64_t* chunks, int nchunks, const int* seg_chunk_ptr, int nseg, const int* active,
                    double* partial, double* C, cudaStream_t st) {
    constexpr int kC = 4;
    const int rows_slots = gram_seg_chunk_rows(b, dtype) > 0 ? 1 : 0;
    if (rows_slots) {
        if (dtype == BBL_FP64) {
            auto q = static_cast<const double*>(Q);
            auto w = static_cast<const double*>(W);
            if (b == 4) BBL_TRY((launch_gram_rows_seg<double, 4>(n, d_m, q, w, chunks, nchunks, active, partial, st)));
            else BBL_TRY((launch_gram_rows_seg<double, 8>(n, d_m, q, w, chunks, nchunks, active, partial, st)));
        } else {
            auto q = static_cast<const float*>(Q);
            auto w = static_cast<const float*>(W);
            if (b == 4) BBL_TRY((launch_gram_rows_seg<float, 4>(n, d_m, q, w, chunks, nchunks, active, partial, st)));
            else if (b == 8) BBL_TRY((launch_gram_rows_seg<float, 8>(n, d_m, q, w, chunks, nchunks, active, partial, st)));
            else BBL_TRY((launch_gram_rows_seg<float, 16>(n, d_m, q, w, chunks, nchunks, active, partial, st)));
        }
    } else if (dtype == BBL_FP64) {
        auto q = static_cast<const double*>(Q);
        auto w = static_cast<const double*>(W);
        switch (b) {
            case 1: BBL_TRY((launch_gram_seg<double, 1, 1>(n, m_max, d_m, q, w, chunks, nchunks, active, partial, st))); break;
            case 2: BBL_TRY((launch_gram_seg<double, 2, 2>(n, m_max, d_m, q, w, chunks, nchunks, active, partial, st))); break;
            case 4: BBL_TRY((launch_gram_seg<double, 4, 2>(n, m_max, d_m, q, w, chunks, nchunks, active, partial, st))); break;
            case 8: BBL_TRY((launch_gram_seg<double, 8, 2>(n, m_max, d_m, q, w, chunks, nchunks, active, partial, st))); break;
            case 16: BBL_TRY((launch_gram_seg<double, 16, 2>(n, m_max, d_m, q, w, chunks, nchunks, active, partial, st))); break;
            default: return set_error(BBL_ERR_UNSUPPORTED, "batched: b=%d", b);
        }
    } else {
        auto q = static_cast<const float*>(Q);
        auto w = static_cast<const float*>(W);
        switch (b) {
            case 1: BBL_TRY((launch_gram_seg<float, 1, 1>(n, m_max, d_m, q, w, chunks, nchunks, active, partial, st))); break;
            case 2: BBL_TRY((launch_gram_seg<float, 2, 2>(n, m_max, d_m, q, w, chunks, nchunks, active, partial, st))); break;
            case 4: BBL_TRY((launch_gram_seg<float, 4, kC>(n, m_max, d_m, q, w, chunks, nchunks, active, partial, st))); break;
            case 8: BBL_TRY((launch_gram_seg<float, 8, kC>(n, m_max, d_m, q, w, chunks, nchunks, active, partial, st))); break;
            case 16: BBL_TRY((launch_gram_seg<float, 16, 2>(n, m_max, d_m, q, w, chunks, nchunks, active, partial, st))); break;
            default: return set_error(BBL_ERR_UNSUPPORTED, "batched: b=%d", b);
        }
    }
    dim3 g((unsigned)ceil_div((int64_t)m_max * b, 256), (unsigned)nseg);
    reduce_seg_kernel<<<g, 256, 0, st>>>(m_max, b, d_m, seg_chunk_ptr, active, partial, C, rows_slots);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

bbl_status apply_seg(int64_t n, int b, int kc, const int* ms, int ms_stride, int dtype, const void* Q, const double* C,
                     int64_t cstride, void* W, bool sub, bool f64_out, const int64_t* ctas, int nctas, const int* active,
                     cudaStream_t st) {
    if (dtype == BBL_FP64) {
        auto q = static_cast<const double*>(Q);
        if (sub) return apply_seg_typed<double, true, double, double>(n, b, kc, ms, ms_stride, ctas, nctas, active, q, C, cstride,
                                                                      static_cast<double*>(W), st);
        return apply_seg_typed<double, false, double, double>(n, b, kc, ms, ms_stride, ctas, nctas, active, q, C, cstride,
                                                              static_cast<double*>(W), st);
    }
    auto q = static_cast<const float*>(Q);
    if (f64_out)
        return apply_seg_typed<float, false, double, double>(n, b, kc, ms, ms_stride, ctas, nctas, active, q, C, cstride,
                                                             static_cast<double*>(W), st);
    if (sub) return apply_seg_typed<float, true, float, float>(n, b, kc, ms, ms_stride, ctas, nctas, active, q, C, cstride,
                                                               static_cast<float*>(W), st);
    return apply_seg_typed<float, false, float, float>(n, b, kc, ms, ms_stride, ctas, nctas, active, q, C, cstride,
                                                       static_cast<float*>(W), st);
}

bbl_status chol_seg(int b, int nseg, const double* G, const double* thresh2, int relative, double* R, double* Rinv,
                    int* ndefl, int* mask, int* status, const int* active, cudaStream_t st) {
    chol_seg_kernel<<<(unsigned)ceil_div(nseg, 32), 32, 0, st>>>(b, nseg, G, thresh2, relative, R, Rinv, ndefl, mask,
                                                                 status, active);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

bbl_status trmul_seg(int b, int nseg, const double* R2, const double* R1, double* B, const int* active, cudaStream_t st) {
    trmul_seg_kernel<<<dim3(1, nseg), 256, 0, st>>>(b, nseg, R2, R1, B, active);
    BBL_LAUNCH_CHECK();
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

constexpr int64_t kNoAllocScratchDoubles = int64_t(1) << 20;  // 8 MiB: chunk tickets + FP64 partial sums
// The front of the array holds one chunk ticket (int) per column group of the
// Gram.  2048 doubles hold 4096 tickets, more than any request within the
// limit below needs (b = 1: m <= 2^20 - 2048 columns in groups of 256 give at
// most 4088; larger b have fewer groups); the rest holds the partial sums.
constexpr int64_t kNoAllocTicketDoubles = 2048;
constexpr int64_t kNoAllocPartialDoubles = kNoAllocScratchDoubles - kNoAllocTicketDoubles;
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
    // the front of the array holds the chunk tickets (the ones a call uses
    // are zeroed by that call), the rest the per-worker partial sums
    const int64_t per_worker = (int64_t)m * B;
    if (per_worker > kNoAllocPartialDoubles)
        return set_error(BBL_ERR_INVALID_ARG,
                         "block_gram_noalloc: nblocks*b*b = %lld exceeds the fixed scratch of %lld doubles",
                         (long long)per_worker, (long long)kNoAllocPartialDoubles);
    return gram_core<T, B, CPT>(n, m, Q, W, C, scratch + kNoAllocTicketDoubles, kNoAllocPartialDoubles,
                                reinterpret_cast<int*>(scratch),
                                kNoAllocTicketDoubles * (int64_t)(sizeof(double) / sizeof(int)), st);
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

// -------------------------------------------------------------------- pivot overlap diagnostic
// How much of each converged eigenvector lies in the span of the pivot block
// (Sec. II.B: the pivot must overlap the wanted eigenvectors; Sec. III.A:
// states the pivot misses come late or as intruders).
namespace bbl {
namespace {

constexpr int kOvRows = 64;

// partial[cta][a*k + i] = sum over the CTA's rows r of Q[r][a] X[r][i]
// (thread t < b*k owns the pair a = t / k, i = t % k; row tiles of Q and X
// are staged in shared memory).
__global__ void __launch_bounds__(256) cross_gram_kernel(int64_t n, int b, int k, const double* __restrict__ Q,
                                                         const double* __restrict__ X, double* __restrict__ partial) {
    __shared__ double qs[kOvRows * kMaxB];
    __shared__ double xs[kOvRows * kMaxB];
    const int t = threadIdx.x;
    const int a = t / k, i = t - (t / k) * k;
    double s = 0.0;
    for (int64_t r0 = (int64_t)blockIdx.x * kOvRows; r0 < n; r0 += (int64_t)gridDim.x * kOvRows) {
        const int rows = (int)min((int64_t)kOvRows, n - r0);
        __syncthreads();
        for (int e = t; e < rows * b; e += blockDim.x) qs[e] = Q[r0 * b + e];
        for (int e = t; e < rows * k; e += blockDim.x) xs[e] = X[r0 * k + e];
        __syncthreads();
        if (t < b * k)
            for (int r = 0; r < rows; ++r) s = fma(qs[r * b + a], xs[r * k + i], s);
    }
    if (t < b * k) partial[(int64_t)blockIdx.x * b * k + t] = s;
}

}  // namespace
}  // namespace bbl

extern "C" bbl_status bbl_pivot_overlap(int64_t n, int b, const double* P, int k, const double* X, double* overlap,
                                        void* stream) {
    using namespace bbl;
    if (n < 1 || b < 1 || b > kMaxB || k < 1 || k > kMaxB || !P || !X || !overlap)
        return set_error(BBL_ERR_INVALID_ARG, "pivot_overlap: bad arguments (b, k in 1..%d)", kMaxB);
    cudaStream_t st = as_stream(stream);
    DevBuf Q, Xd, partials, small, cnt, part, C;
    BBL_TRY(Q.alloc(sizeof(double) * n * b));
    BBL_CUDA(cudaMemcpyAsync(Q.p, P, sizeof(double) * n * b, cudaMemcpyDefault, st));
    const double* Xp = X;
    if (!is_device_pointer(X)) {
        BBL_TRY(Xd.alloc(sizeof(double) * n * k));
        BBL_CUDA(cudaMemcpyAsync(Xd.p, X, sizeof(double) * n * k, cudaMemcpyHostToDevice, st));
        Xp = Xd.as<double>();
    }
    // Q = orth(P) by CholQR2; a column dependent on the others to 1e-10 of
    // the largest column norm is dropped (a zero column of Q)
    BBL_TRY(cnt.alloc(sizeof(int)));
    BBL_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int), st));
    BBL_TRY(small.alloc(sizeof(double) * 8 * kMaxB * kMaxB + sizeof(int) * 4 * kMaxB));
    BBL_CUDA(cudaMemsetAsync(small.p, 0, small.bytes, st));
    DevBuf Bm;
    BBL_TRY(Bm.alloc(sizeof(double) * kMaxB * kMaxB));
    BBL_TRY(cholqr2_dev(n, b, BBL_FP64, Q.p, Bm.as<double>(), -1e-20, cnt.as<int>(), nullptr, partials, small, st));
    const int grid = (int)std::min<int64_t>(152 * 4, ceil_div(n, kOvRows));
    BBL_TRY(part.alloc(sizeof(double) * (size_t)grid * b * k));
    BBL_TRY(C.alloc(sizeof(double) * b * k));
    cross_gram_kernel<<<grid, 256, 0, st>>>(n, b, k, Q.as<double>(), Xp, part.as<double>());
    BBL_LAUNCH_CHECK();
    launch_reduce((int64_t)b * k, grid, part.as<double>(), C.as<double>(), st);
    BBL_LAUNCH_CHECK();
    std::vector<double> h(b * k);
    int bad = 0;
    BBL_CUDA(cudaMemcpyAsync(h.data(), C.p, sizeof(double) * b * k, cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaMemcpyAsync(&bad, reinterpret_cast<char*>(small.p) + sizeof(double) * 8 * kMaxB * kMaxB, sizeof(int),
                             cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    if (bad) return set_error(BBL_ERR_NUMERICAL, "pivot_overlap: non-finite pivot Gram matrix");
    for (int i = 0; i < k; ++i) {
        double s = 0.0;
        for (int a = 0; a < b; ++a) s += h[a * k + i] * h[a * k + i];
        overlap[i] = std::sqrt(s);
    }
    return BBL_OK;
}
