// S4: Ritz solve of the block-tridiagonal T (Sec. II.B, Eq. 12), which the
// paper hands to LAPACK.  T is symmetric with bandwidth p = b (its
// off-diagonal blocks B_j from CholQR2 are upper triangular), stored as a
// lower band: Tb[i*(p+1) + d] = T[i][i-d].
//
// Three kernels, all on the device:
//  1. bisect  - one CTA per wanted eigenvalue index i.  Sylvester's law of
//               inertia: the number of negative pivots of the LDL^T
//               factorisation of T - sigma I is the number of eigenvalues below
//               sigma.  For p in {1, 2, 4, 8, 16} a group of p+1 lanes holds
//               the elimination window in registers and evaluates one shift
//               (32/(p+1) shifts per warp, 24 per CTA for p = 8); for
//               p in {1, 2, 4, 8} every thread holds a whole window and
//               evaluates its own shift (256 per CTA); otherwise a warp per
//               shift with the window in shared memory.  Multisection runs in
//               FP32 (58x the FP64 rate on this GPU) to a bracket of
//               1e-5 * scale, starting from the previous Ritz value when one is
//               given (Cauchy interlacing makes it an upper bound); FP64 counts
//               check the bracket and FP64 multisection narrows it to
//               1e-8 * scale.
//  2. invit   - one warp per eigenvalue: banded LU with partial pivoting of
//               T - theta I (U has bandwidth 2p), three steps of inverse
//               iteration from a per-index pseudo-random start (register-window
//               triangular solves for p <= 8), Rayleigh quotient.
//  3. cluster - one CTA: eigenvalues closer than 1e-3 * scale are grouped;
//               their vectors are orthonormalised twice (modified
//               Gram-Schmidt) and rotated by a small Jacobi Rayleigh-Ritz;
//               columns get the sign convention (first largest-magnitude
//               entry positive).
#include <algorithm>

#include "common.cuh"
#include "df32.cuh"

namespace bbl {
namespace {

constexpr int kMaxP = kMaxB;            // bandwidth limit
constexpr int kWin = kMaxP + 1;         // LDL^T window edge
constexpr int kBisectWarps = 8;
constexpr size_t kBandSmemMax = 160 * 1024;  // band bytes staged in shared memory
constexpr int kMaxNev = 32;
constexpr size_t kInvitSmemMax = 220 * 1024;  // inverse iteration: window, vector and LU factors

// Per-segment addressing for a batch of independent T's (blockIdx.y = segment
// in bisect / invit, blockIdx.x in cluster).  The single-problem path passes
// d_m = active = nullptr and zero strides.
struct SegArgs {
    const int* d_m;       // current order m in device memory (overrides the argument)
    const int* active;    // per-segment flag; inactive segments are skipped
    int64_t sT, sTh, sS, sWs, sTmp;
};

__device__ __forceinline__ double band_get(const double* __restrict__ Tb, int p, int m, int r, int c) {
    // T[r][c] for any r, c (0 outside the band or the matrix)
    if (r < 0 || c < 0 || r >= m || c >= m) return 0.0;
    if (r >= c) return (r - c <= p) ? Tb[(int64_t)r * (p + 1) + (r - c)] : 0.0;
    return (c - r <= p) ? Tb[(int64_t)c * (p + 1) + (c - r)] : 0.0;
}

// Number of eigenvalues of T strictly below sigma (LDL^T of T - sigma I),
// evaluated by one warp.  win: this warp's (p+1)^2 shared-memory window.
template <typename F>
__device__ int inertia_count(const double* __restrict__ Tb, int p, int m, double sigma, double pivmin, F* win) {
    const int lane = threadIdx.x & 31;
    const int P1 = p + 1;
    // initial window: rows/cols 0..p
    for (int e = lane; e < P1 * P1; e += 32) {
        const int r = e / P1, c = e % P1;
        double v = band_get(Tb, p, m, r, c);
        if (r == c) v = (r < m) ? v - sigma : 1e300;
        win[e] = (F)((r == c && r >= m) ? (F)1e30 : (F)v);
    }
    __syncwarp();
    int neg = 0;
    const F fpivmin = (F)pivmin;
    for (int k = 0; k < m; ++k) {
        const int ks = k % P1;
        F d = win[ks * P1 + ks];
        if (fabs((double)d) < (double)fpivmin) d = -fpivmin;
        neg += (d < F(0));
        const F rd = F(1) / d;
        // lane c (1..p) updates window column k+c, rows k+c..k+p (lower triangle
        // plus the mirrored upper part it owns)
        if (lane >= 1 && lane <= p) {
            const int cs = (k + lane) % P1;
            const F u = win[ks * P1 + cs] * rd;
            for (int r = 1; r <= p; ++r) {
                const int rs = (k + r) % P1;
                win[rs * P1 + cs] -= win[rs * P1 + ks] * u;
            }
        }
        __syncwarp();
        // bring in row/column k+p+1 in the freed slot ks
        const int R = k + p + 1;
        if (lane <= p) {
            const int C = k + 1 + lane;  // C in [k+1, k+p+1]
            const int cs = C % P1;
            double v;
            if (R >= m) v = (C == R) ? 1e300 : 0.0;
            else v = band_get(Tb, p, m, R, C) - (C == R ? sigma : 0.0);
            const F fv = (R >= m && C == R) ? (F)1e30 : (F)v;
            win[ks * P1 + cs] = fv;
            win[cs * P1 + ks] = fv;
        }
        __syncwarp();
    }
    return neg;
}

// The same count with the active window in registers, for bandwidths
// P in {1, 2, 4, 8, 16}.  A group of P+1 lanes evaluates one shift (a warp
// holds 32 / (P+1) groups, each with its own sigma).  Lane r of a group holds
// one row of the window: at step k the rows k..k+P sit in lanes k mod (P+1),
// ..., and a lane keeps its row's entries in the not yet eliminated columns
// k..(its row) as f[0..delta], delta = its distance from the pivot row.  A
// step gathers column k (every lane's f[0]) with P+1 shuffles, each lane
// applies its multiplier f[0] / d_k to its row, shifts its entries by one
// column, and the pivot lane takes the next row of T (loaded one cycle of
// P+1 steps ahead).  All lanes of a group see the same pivots d_k.
template <typename F, int P>
__device__ int inertia_count_reg(const double* __restrict__ Tb, int m, double sigma, double pivmin) {
    constexpr int P1 = P + 1;
    const int lane = threadIdx.x & 31;
    const int base = (lane / P1) * P1;  // spare lanes past the last group run along harmlessly
    const int r = lane - base;
    const F big = (F)1e30;
    // entries of row R of T - sigma I in columns k1 .. k1 + P (lower triangle)
    auto load = [&](int R, int k1, F(&dst)[P1]) {
#pragma unroll
        for (int j = 0; j < P1; ++j) {
            const int C = k1 + j;
            const int d = R - C;
            F v = F(0);
            if (R >= m) {
                v = (d == 0) ? big : F(0);
            } else if (d >= 0 && d <= P && C >= 0) {
                double t = Tb[(int64_t)R * P1 + d];
                if (d == 0) t -= sigma;
                v = (F)t;
            }
            dst[j] = v;
        }
    };
    F f[P1], nf[P1];
    load(r, 0, f);            // row r, columns 0..P
    load(r + P1, r + 1, nf);  // the row this lane takes after pivoting at step r
    int delta = r < P ? r : P;
    int piv = 0;
    int neg = 0;
    const F fpivmin = (F)pivmin;
    for (int k = 0; k < m; ++k) {
        F g[P1];
#pragma unroll
        for (int j = 0; j < P1; ++j) {
            int src = piv + j;
            if (src >= P1) src -= P1;
            g[j] = __shfl_sync(0xffffffffu, f[0], base + src);
        }
        F d = g[0];
        if (fabs(d) < fpivmin) d = -fpivmin;
        neg += (d < F(0)) ? 1 : 0;
        if (delta == 0) {
#pragma unroll
            for (int j = 0; j < P1; ++j) f[j] = nf[j];
            load(k + 2 * P1, k + P1 + 1, nf);
            delta = P;
        } else {
            F mlt;
            if constexpr (sizeof(F) == 4) {
                mlt = __fdividef(f[0], d);
            } else {
                // reciprocal from an FP32 seed and one Newton step (relative
                // error ~2^-46, ample for the signs of the pivots)
                const double ad = fabs(d);
                double rd;
                if (ad > 1e-30 && ad < 1e30) {
                    const double r0 = (double)__frcp_rn((float)d);
                    rd = r0 * fma(-d, r0, 2.0);
                } else {
                    rd = 1.0 / d;
                }
                mlt = f[0] * rd;
            }
#pragma unroll
            for (int j = 1; j < P1; ++j)
                if (j <= delta) f[j] = fma(-mlt, g[j], f[j]);
#pragma unroll
            for (int j = 0; j < P; ++j) f[j] = f[j + 1];
            f[P] = F(0);
            delta -= 1;
        }
        piv = (piv + 1 == P1) ? 0 : piv + 1;
    }
    return neg;
}

// The same count by a single thread: the lower triangle of the (P+1)x(P+1)
// active window lives in the thread's registers, relative to the pivot row,
// and every thread of a CTA evaluates its own shift.  A step forms the
// multipliers of column k from one reciprocal, updates the remaining
// entries, shifts the window and takes the next row of T (the same address
// for all threads).  No thread talks to another.  The band comes as an FP32
// or float-float copy (band[i*(P+1) + d] = T[i][i-d]): GB300 issues one FP64
// warp instruction per 64 cycles per scheduler, so the recurrences run on
// the FP32 pipes only, in FP32 (F = float) or float-float (F = df32).
template <typename F>
struct RitzArith;

template <>
struct RitzArith<float> {
    static __device__ __forceinline__ float fms(float l, float e, float x) { return __fmaf_rn(-l, e, x); }  // x - l e
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float rcp(float a) { return __frcp_rn(a); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float hi(float a) { return a; }
    static __device__ __forceinline__ float make(float h) { return h; }
};

template <>
struct RitzArith<df32> {
    static __device__ __forceinline__ df32 fms(df32 l, df32 e, df32 x) { return dfm::dfma(dfm::dneg(l), e, x); }
    static __device__ __forceinline__ df32 mul(df32 a, df32 b) { return dfm::dmul(a, b); }
    static __device__ __forceinline__ df32 rcp(df32 a) { return dfm::drcp(a); }
    static __device__ __forceinline__ df32 sub(df32 a, df32 b) { return a - b; }
    static __device__ __forceinline__ float hi(df32 a) { return a.hi; }
    static __device__ __forceinline__ df32 make(float h) { return df32(h); }
};

template <typename F, int P>
__device__ int count_lane(const F* __restrict__ band, int m, F sigma, float pivmin) {
    using A = RitzArith<F>;
    constexpr int P1 = P + 1;
    const F big = A::make(1e30f);
    const F zero = A::make(0.0f);
    F E[P1][P1];
#pragma unroll
    for (int r = 0; r < P1; ++r)
#pragma unroll
        for (int c = 0; c < P1; ++c) {
            F v = zero;
            if (c <= r) {
                if (r >= m) {
                    v = (r == c) ? big : zero;
                } else {
                    v = band[r * P1 + (r - c)];
                    if (r == c) v = A::sub(v, sigma);
                }
            }
            E[r][c] = v;
        }
    int neg = 0;
    for (int k = 0; k < m; ++k) {
        F d = E[0][0];
        if (fabsf(A::hi(d)) < pivmin) d = A::make(-pivmin);
        neg += (A::hi(d) < 0.0f) ? 1 : 0;
        const F rd = A::rcp(d);
        F l[P1], e0[P1];
#pragma unroll
        for (int r = 1; r < P1; ++r) {
            e0[r] = E[r][0];
            l[r] = A::mul(e0[r], rd);
        }
        // in place: entry (r, c) moves to (r-1, c-1) after it has been read
#pragma unroll
        for (int r = 1; r < P1; ++r)
#pragma unroll
            for (int c = 1; c <= r; ++c) E[r - 1][c - 1] = A::fms(l[r], e0[c], E[r][c]);
        const int R = k + P1;  // row entering the window: columns k+1 .. k+P+1
        if (R < m) {
            const F* row = band + R * P1;
#pragma unroll
            for (int c = 0; c < P1; ++c) E[P][c] = row[P - c];
            E[P][P] = A::sub(E[P][P], sigma);
        } else {
#pragma unroll
            for (int c = 0; c < P1; ++c) E[P][c] = (c == P) ? big : zero;
        }
    }
    return neg;
}

// Bisection with one shift per thread (p in {1, 2, 4, 8}): FP32
// multisection with 256 shifts per round to a 1e-5 * scale bracket, then one
// float-float round whose first and last threads sit on the bracket ends
// (the check) and whose 254 others narrow it 255-fold; a failed check
// restarts from the Gershgorin interval (warm start) and then falls back to
// float-float multisection by one warp.  The band is staged in shared memory
// as FP32 and float-float copies (bands longer than the staging area use
// the slower copies in the caller-provided scratch).
template <int P>
__global__ void __launch_bounds__(256) bisect_lane_kernel(int m, int nev, const double* __restrict__ Tg,
                                                         double* __restrict__ theta_out, double* __restrict__ width_out,
                                                         int band_in_smem, SegArgs sa, const double* __restrict__ warm,
                                                         int warm_count) {
    constexpr int NT = 256;
    constexpr int p = P, P1 = P + 1;
    __shared__ int counts[NT];
    __shared__ double red[2][NT];
    __shared__ double s_lo, s_hi;
    __shared__ int s_tlo[NT / 32], s_thi[NT / 32];
    extern __shared__ __align__(16) unsigned char bl_smem[];
    const int i = blockIdx.x;
    const int seg = blockIdx.y;
    if (sa.active && !sa.active[seg]) return;
    if (sa.d_m) m = *sa.d_m;
    if (i >= min(nev, m)) return;
    Tg += seg * sa.sT;
    theta_out += seg * sa.sTh;
    width_out += seg * sa.sTh;
    const int tid = threadIdx.x;
    // FP32 and float-float copies of the band (shared memory)
    df32* bdf = reinterpret_cast<df32*>(bl_smem);
    float* b32 = reinterpret_cast<float*>(bdf + (size_t)m * P1);
    for (int e = tid; e < m * P1; e += NT) {
        const double v = Tg[e];
        bdf[e] = df32(v);
        b32[e] = (float)v;
    }
    __syncthreads();
    const double* Tb = Tg;
    double gmin = 1e308, gmax = -1e308;
    for (int r = tid; r < m; r += NT) {
        double off = 0.0;
        for (int c = max(0, r - p); c <= min(m - 1, r + p); ++c)
            if (c != r) off += fabs(band_get(Tb, p, m, r, c));
        const double d = band_get(Tb, p, m, r, r);
        gmin = fmin(gmin, d - off);
        gmax = fmax(gmax, d + off);
    }
    red[0][tid] = gmin;
    red[1][tid] = gmax;
    __syncthreads();
    if (tid == 0) {
        for (int t = 1; t < NT; ++t) {
            gmin = fmin(gmin, red[0][t]);
            gmax = fmax(gmax, red[1][t]);
        }
        const double scale = fmax(fabs(gmin), fabs(gmax));
        const double pad = 1e-10 * scale + 1e-300;
        s_lo = gmin - pad;
        s_hi = gmax + pad;
    }
    __syncthreads();
    const double scale = fmax(fmax(fabs(s_lo), fabs(s_hi)), 1e-300);
    const float pivmin32 = (float)(1e-7 * scale);
    const float pivmindf = (float)(1e-13 * scale);
    const double glo = s_lo, ghi = s_hi;
    double lo = glo, hi = ghi;
    const bool warm_used = warm && i < warm_count;
    if (warm_used) {
        const double w = warm[i];
        hi = fmin(ghi, w + 1e-9 * scale);
        lo = fmax(glo, w - 1e-3 * scale);
        if (!(lo < hi)) {
            lo = glo;
            hi = ghi;
        }
    }
    // New bracket from counts[t] at a + (b-a)(t+1)/(ns+1): the last sample
    // with at most i eigenvalues below it and the first with more, found by
    // integer max/min reductions (FP64 instructions are kept out of per-sample
    // work); false when the counts are inconsistent.
    auto update = [&](int ns, double& a, double& b) -> bool {
        const int lane = tid & 31, w = tid >> 5;
        int tl = -1, th = ns;
        if (tid < ns) {
            if (counts[tid] <= i) tl = tid;
            else th = tid;
        }
        tl = __reduce_max_sync(0xffffffffu, tl);
        th = __reduce_min_sync(0xffffffffu, th);
        if (lane == 0) {
            s_tlo[w] = tl;
            s_thi[w] = th;
        }
        __syncthreads();
        tl = -1;
        th = ns;
        for (int q = 0; q < NT / 32; ++q) {
            tl = max(tl, s_tlo[q]);
            th = min(th, s_thi[q]);
        }
        __syncthreads();
        if (tl >= th) return false;
        const double step = (b - a) / (double)(ns + 1);
        const double nlo = tl >= 0 ? a + step * (double)(tl + 1) : a;
        const double nhi = th < ns ? a + step * (double)(th + 1) : b;
        a = nlo;
        b = nhi;
        return true;
    };
    bool verified = false;
    for (int attempt = 0; attempt < (warm_used ? 2 : 1) && !verified; ++attempt) {
        if (attempt == 1) {
            lo = glo;
            hi = ghi;
        }
        for (int round = 0; round < 40 && (hi - lo) > 1e-5 * scale; ++round) {
            const double sg = lo + (hi - lo) * ((double)(tid + 1) * (1.0 / (double)(NT + 1)));
            counts[tid] = count_lane<float, P>(b32, m, (float)sg, pivmin32);
            __syncthreads();
            const bool ok = update(NT, lo, hi);
            __syncthreads();
            if (!ok) break;  // inconsistent FP32 counts: the float-float round decides
        }
        // float-float round: lane 0 at lo, lane 31 at hi, lanes 1..30 inside
        {
            // every thread evaluates one float-float shift (the wall time is
            // that of one thread's chain): 0 at lo, NT-1 at hi, the rest inside
            const double sg = tid == NT - 1 ? hi : lo + (hi - lo) * ((double)tid * (1.0 / (double)(NT - 1)));
            counts[tid] = count_lane<df32, P>(bdf, m, df32(sg), pivmindf);
        }
        __syncthreads();
        verified = counts[0] <= i && counts[NT - 1] > i;
        __syncthreads();
        if (verified) {
            // the inner samples: counts[1..NT-2] at lo + (hi-lo) t/(NT-1)
            const int c = (tid < NT - 2) ? counts[tid + 1] : 0;
            __syncthreads();
            if (tid < NT - 2) counts[tid] = c;
            __syncthreads();
            double a = lo, b = hi;
            if (update(NT - 2, a, b)) {
                lo = a;
                hi = b;
            }
        }
    }
    if (!verified) {
        // float-float multisection by warp 0 from the Gershgorin interval to 1e-8 * scale
        lo = glo;
        hi = ghi;
        for (int round = 0; round < 60 && (hi - lo) > 1e-8 * scale; ++round) {
            if (tid < 32) {
                const double sg = lo + (hi - lo) * ((double)(tid + 1) * (1.0 / 33.0));
                counts[tid] = count_lane<df32, P>(bdf, m, df32(sg), pivmindf);
            }
            __syncthreads();
            const bool ok = update(32, lo, hi);
            __syncthreads();
            if (!ok) break;
        }
    }
    if (tid == 0) {
        theta_out[i] = 0.5 * (lo + hi);
        width_out[i] = hi - lo;
    }
}

// Shifts evaluated at once per CTA: one per warp (window in shared memory,
// any p) or one per lane group (register window, P > 0).
template <int P>
struct BisectShape {
    static constexpr int G = P > 0 ? 32 / (P + 1) : 1;
    static constexpr int NSH = kBisectWarps * G;
};

template <typename F, int P>
__device__ __forceinline__ int count_below(const double* Tb, int p, int m, double sigma, double pivmin, F* win) {
    if constexpr (P > 0) return inertia_count_reg<F, P>(Tb, m, sigma, pivmin);
    else return inertia_count<F>(Tb, p, m, sigma, pivmin, win);
}

struct Bracket {
    double lo, hi;
};

template <int P>
__global__ void __launch_bounds__(32 * kBisectWarps) bisect_kernel(int m, int p, int nev, const double* __restrict__ Tg,
                                                                   double* __restrict__ theta_out,
                                                                   double* __restrict__ width_out, int band_in_smem,
                                                                   SegArgs sa, const double* __restrict__ warm,
                                                                   int warm_count) {
    constexpr int G = BisectShape<P>::G, NSH = BisectShape<P>::NSH;
    constexpr int WIN = P > 0 ? 1 : kWin * kWin;  // shared-memory windows only for the generic form
    __shared__ double win64[kBisectWarps][WIN];
    __shared__ float win32[kBisectWarps][WIN];
    __shared__ int counts[NSH];
    __shared__ double red[2][32 * kBisectWarps];
    __shared__ double s_lo, s_hi;
    extern __shared__ double tb_sh[];
    const int i = blockIdx.x;
    const int seg = blockIdx.y;
    if (sa.active && !sa.active[seg]) return;
    if (sa.d_m) m = *sa.d_m;
    if (i >= min(nev, m)) return;
    Tg += seg * sa.sT;
    theta_out += seg * sa.sTh;
    width_out += seg * sa.sTh;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid & 31;
    // shift slot of this lane: warp * G + its lane group; reporter: the group's first lane
    const int lgrp = P > 0 ? min(lane / (P + 1), G - 1) : 0;
    const int sidx = warp * G + lgrp;
    const bool reporter = P > 0 ? (lane % (P + 1) == 0 && lane / (P + 1) < G) : (lane == 0);
    // the elimination walks T row by row: keep its band in shared memory when it fits
    const double* Tb = Tg;
    if (band_in_smem) {
        for (int e = tid; e < m * (p + 1); e += blockDim.x) tb_sh[e] = Tg[e];
        __syncthreads();
        Tb = tb_sh;
    }
    // Gershgorin interval
    double gmin = 1e308, gmax = -1e308;
    for (int r = tid; r < m; r += blockDim.x) {
        double off = 0.0;
        for (int c = max(0, r - p); c <= min(m - 1, r + p); ++c)
            if (c != r) off += fabs(band_get(Tb, p, m, r, c));
        const double d = band_get(Tb, p, m, r, r);
        gmin = fmin(gmin, d - off);
        gmax = fmax(gmax, d + off);
    }
    red[0][tid] = gmin;
    red[1][tid] = gmax;
    __syncthreads();
    if (tid == 0) {
        for (int t = 1; t < blockDim.x; ++t) {
            gmin = fmin(gmin, red[0][t]);
            gmax = fmax(gmax, red[1][t]);
        }
        const double scale = fmax(fabs(gmin), fabs(gmax));
        const double pad = 1e-10 * scale + 1e-300;
        s_lo = gmin - pad;
        s_hi = gmax + pad;
    }
    __syncthreads();
    const double scale = fmax(fmax(fabs(s_lo), fabs(s_hi)), 1e-300);
    // pivots smaller than these are replaced by -pivmin (a perturbation of T
    // far below the bracket widths used): keeps the elimination finite
    const double pivmin64 = 1e-14 * scale;
    const double pivmin32 = 1e-7 * scale;
    const double glo = s_lo, ghi = s_hi;
    double lo = glo, hi = ghi;
    if (warm && i < warm_count) {
        // T of an earlier block is a leading principal submatrix of this T, so
        // its i-th Ritz value bounds this one from above (Cauchy interlacing);
        // a guessed lower end is checked with the final FP64 counts below
        const double w = warm[i];
        hi = fmin(ghi, w + 1e-9 * scale);
        lo = fmax(glo, w - 1e-3 * scale);
        if (!(lo < hi)) {
            lo = glo;
            hi = ghi;
        }
    }
    // phase 1: FP32 multisection to a 1e-5 * scale bracket (FP32 counts are
    // exact for a matrix within a few p * 2^-24 * scale of T, so narrower FP32
    // brackets are not trustworthy), checked with FP64
    // counts at its ends (warp 0 at lo, warp 1 at hi).  A warm bracket that
    // fails the check (the value moved further down than guessed) is retried
    // once from the Gershgorin interval.
    const bool warm_used = warm && i < warm_count && !(lo == glo && hi == ghi);
    bool verified = false;
    for (int attempt = 0; attempt < (warm_used ? 2 : 1) && !verified; ++attempt) {
        if (attempt == 1) {
            lo = glo;
            hi = ghi;
        }
        for (int round = 0; round < 40 && (hi - lo) > 1e-5 * scale; ++round) {
            const double sigma = lo + (hi - lo) * (double)(sidx + 1) / (double)(NSH + 1);
            const int cnt = count_below<float, P>(Tb, p, m, sigma, pivmin32, win32[warp]);
            if (reporter) counts[sidx] = cnt;
            __syncthreads();
            double nlo = lo, nhi = hi;
            for (int w = 0; w < NSH; ++w) {
                const double s = lo + (hi - lo) * (double)(w + 1) / (double)(NSH + 1);
                if (counts[w] <= i) nlo = fmax(nlo, s);
                else nhi = fmin(nhi, s);
            }
            __syncthreads();
            if (nlo >= nhi) break;  // inconsistent FP32 counts: stop, the FP64 check decides
            lo = nlo;
            hi = nhi;
        }
        if (warp < 2) {
            const int cnt = count_below<double, P>(Tb, p, m, warp == 0 ? lo : hi, pivmin64, win64[warp]);
            if (lane == 0) counts[warp] = cnt;
        }
        __syncthreads();
        verified = counts[0] <= i && counts[1] > i;
        __syncthreads();
    }
    // phase 2: FP64 multisection from the verified bracket (or, when the FP32
    // bracket failed the check, from the Gershgorin interval) to 1e-8 * scale;
    // inverse iteration then starts within 1e-8 * scale of the eigenvalue and
    // its Rayleigh quotient gives the value to working precision.
    if (!verified) {
        lo = glo;
        hi = ghi;
    }
    for (int round = 0; round < 200; ++round) {
        const double tolw = 1e-8 * scale + 1e-300;
        if (hi - lo <= tolw) break;
        const double sigma = lo + (hi - lo) * (double)(sidx + 1) / (double)(NSH + 1);
        const int cnt = count_below<double, P>(Tb, p, m, sigma, pivmin64, win64[warp]);
        if (reporter) counts[sidx] = cnt;
        __syncthreads();
        double nlo = lo, nhi = hi;
        for (int w = 0; w < NSH; ++w) {
            const double s = lo + (hi - lo) * (double)(w + 1) / (double)(NSH + 1);
            if (counts[w] <= i) nlo = fmax(nlo, s);
            else nhi = fmin(nhi, s);
        }
        __syncthreads();
        if (nlo >= nhi || (nlo == lo && nhi == hi)) break;
        lo = nlo;
        hi = nhi;
    }
    if (tid == 0) {
        theta_out[i] = 0.5 * (lo + hi);
        width_out[i] = hi - lo;
    }
}

__device__ __forceinline__ double hash_uniform(uint64_t a, uint64_t b) {
    uint64_t z = a * 0x9E3779B97F4A7C15ull + b + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((double)(z >> 11) + 0.5) * 0x1.0p-53 * 2.0 - 1.0;
}

// Inverse iteration for eigenvalue i.  ws: per-eigenvalue workspace of
// m*(3p+1) doubles + m ints (U rows of width 2p+1, L multipliers, pivots).
__global__ void __launch_bounds__(32) invit_kernel(int m, int p, const double* __restrict__ Tg,
                                                    double* __restrict__ theta, double* __restrict__ S, int nev,
                                                    double* __restrict__ ws, double scale_hint, int band_in_smem,
                                                    SegArgs sa) {
    extern __shared__ double sm[];
    const int i = blockIdx.x;
    const int seg = blockIdx.y;
    if (sa.active && !sa.active[seg]) return;
    if (sa.d_m) m = *sa.d_m;
    if (i >= min(nev, m)) return;
    Tg += seg * sa.sT;
    theta += seg * sa.sTh;
    S += seg * sa.sS;
    ws += seg * sa.sWs;
    const int lane = threadIdx.x;
    const int P1 = p + 1, UW = 2 * p + 1;
    double* win = sm;              // P1 x UW circular window
    double* x = win + P1 * UW;     // m
    double* lsh = x + m;           // p multipliers
    const double* Tb = Tg;
    if (band_in_smem) {            // band copy after the multipliers
        double* tb = lsh + p + 8;
        for (int e = lane; e < m * (p + 1); e += 32) tb[e] = Tg[e];
        __syncwarp();
        Tb = tb;
    }
    double* U = ws + (int64_t)i * m * (3 * p + 1);
    double* L = U + (int64_t)m * UW;
    int* piv = reinterpret_cast<int*>(ws + (int64_t)nev * m * (3 * p + 1)) + (int64_t)i * m;
    const double sigma = theta[i];
    double scale = 0.0;
    for (int r = lane; r < m; r += 32) {
        double s = 0.0;
        for (int c = max(0, r - p); c <= min(m - 1, r + p); ++c) s += fabs(band_get(Tb, p, m, r, c));
        scale = fmax(scale, s);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) scale = fmax(scale, __shfl_xor_sync(0xffffffffu, scale, off));
    scale = fmax(scale, scale_hint);
    const double tiny = 1e-14 * fmax(scale, 1e-300);
    // window init: rows 0..p, columns 0..2p
    for (int e = lane; e < P1 * UW; e += 32) {
        const int r = e / UW, c = e % UW;
        double v = (r < m && c < m) ? band_get(Tb, p, m, r, c) : 0.0;
        if (r == c && r < m) v -= sigma;
        win[(r % P1) * UW + (c % UW)] = v;
    }
    __syncwarp();
    for (int k = 0; k < m; ++k) {
        const int ks = k % P1;
        const int kc = k % UW;
        // pivot search over rows k..min(k+p, m-1)
        double best = -1.0;
        int bi = 0;
        if (lane <= p && k + lane < m) {
            best = fabs(win[((k + lane) % P1) * UW + kc]);
            bi = lane;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        const int ps = (k + bi) % P1;
        if (bi != 0) {
            for (int c = lane; c < UW; c += 32) {
                const int cs = (k + c) % UW;
                const double a = win[ks * UW + cs], b2 = win[ps * UW + cs];
                win[ks * UW + cs] = b2;
                win[ps * UW + cs] = a;
            }
        }
        __syncwarp();
        if (lane == 0) {
            piv[k] = k + bi;
            double u = win[ks * UW + kc];
            if (fabs(u) < tiny) u = (u < 0.0) ? -tiny : tiny;
            win[ks * UW + kc] = u;
        }
        __syncwarp();
        for (int c = lane; c < UW; c += 32) U[(int64_t)k * UW + c] = win[ks * UW + (k + c) % UW];
        const double u0 = win[ks * UW + kc];
        if (lane >= 1 && lane <= p) {
            const double l = (k + lane < m) ? win[((k + lane) % P1) * UW + kc] / u0 : 0.0;
            lsh[lane - 1] = l;
            L[(int64_t)k * p + lane - 1] = l;
        }
        __syncwarp();
        for (int c = lane; c < UW; c += 32) {
            if (c == 0) continue;
            const int cs = (k + c) % UW;
            const double top = win[ks * UW + cs];
            for (int r = 1; r <= p; ++r) {
                const int rs = (k + r) % P1;
                win[rs * UW + cs] -= lsh[r - 1] * top;
            }
        }
        __syncwarp();
        // slot ks now holds row k+p+1; column slot kc now holds column k+2p+1
        const int R = k + p + 1;
        for (int c = lane; c < UW; c += 32) {
            const int C = k + 1 + c;
            double v = 0.0;
            if (R < m && C < m) v = band_get(Tb, p, m, R, C) - (R == C ? sigma : 0.0);
            win[ks * UW + (C % UW)] = v;
        }
        if (lane >= 1 && lane <= p) {
            win[((k + lane) % P1) * UW + kc] = 0.0;  // (k+lane, k+2p+1) is outside the band
        }
        __syncwarp();
    }
    // inverse iteration
    for (int r = lane; r < m; r += 32) x[r] = hash_uniform((uint64_t)i + 1, (uint64_t)r);
    __syncwarp();
    // the shift is within 1e-6 * scale of the eigenvalue and other eigenvalues
    // closer than 1e-3 * scale are handled as a cluster, so each iteration
    // shrinks the other components by 5e-4 or more: five give working precision
    for (int it = 0; it < 5; ++it) {
        // forward: P and L
        for (int k = 0; k < m; ++k) {
            if (lane == 0) {
                const int pk = piv[k];
                if (pk != k) {
                    const double t = x[k];
                    x[k] = x[pk];
                    x[pk] = t;
                }
            }
            __syncwarp();
            if (lane >= 1 && lane <= p && k + lane < m) x[k + lane] -= L[(int64_t)k * p + lane - 1] * x[k];
            __syncwarp();
        }
        // backward: U (bandwidth 2p)
        for (int k = m - 1; k >= 0; --k) {
            double s = 0.0;
            for (int c = lane; c < UW; c += 32)
                if (c >= 1 && k + c < m) s += U[(int64_t)k * UW + c] * x[k + c];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) x[k] = (x[k] - s) / U[(int64_t)k * UW];
            __syncwarp();
        }
        // normalise
        double nn = 0.0;
        for (int r = lane; r < m; r += 32) nn += x[r] * x[r];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, off);
        const double inv = 1.0 / sqrt(nn);
        for (int r = lane; r < m; r += 32) x[r] *= inv;
        __syncwarp();
    }
    // Rayleigh quotient
    double rq = 0.0;
    for (int r = lane; r < m; r += 32) {
        double tx = 0.0;
        for (int c = max(0, r - p); c <= min(m - 1, r + p); ++c) tx += band_get(Tb, p, m, r, c) * x[c];
        rq += x[r] * tx;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) rq += __shfl_xor_sync(0xffffffffu, rq, off);
    if (lane == 0) theta[i] = rq;
    for (int r = lane; r < m; r += 32) S[(int64_t)r * nev + i] = x[r];
}

// Inverse iteration for bandwidths P in {1, 2, 4, 8}, in float-float
// arithmetic on the FP32 pipes (a chain of FP64 instructions would wait 64
// cycles per instruction on GB300).  The band is staged in shared memory as
// float-float values.  Banded LU with partial pivoting: the window rows
// k..k+P x columns k..k+2P, lane l holding column k + ((l - k) mod (2P+1))
// in registers col[r] = A_k[k+r][k+c]; the pivot column's lane finds the
// pivot row, every lane swaps rows 0 and bi of its column, the multipliers
// are broadcast, every lane updates its column, writes row k of U, shifts
// its rows up and takes its entry of the next row of T.  The factors live
// in shared memory when they fit.  Then three steps of inverse iteration
// with column-oriented triangular solves whose active rows live in
// registers (forward: rows k..k+P, backward: rows k-2P..k); the vector is
// normalised and its Rayleigh quotient formed in FP64.
template <int P>
__global__ void __launch_bounds__(32) invit_df_kernel(int m, const double* __restrict__ Tg, double* __restrict__ theta,
                                                       double* __restrict__ S, int nev, double* __restrict__ ws,
                                                       int lu_in_smem, SegArgs sa) {
    using dfm::dfma;
    using dfm::dmul;
    using dfm::dneg;
    using dfm::drcp;
    constexpr int p = P, P1 = P + 1, UW = 2 * P + 1;
    static_assert(UW <= 32, "backward window exceeds a warp");
    extern __shared__ __align__(16) unsigned char ism[];
    const int i = blockIdx.x;
    const int seg = blockIdx.y;
    if (sa.active && !sa.active[seg]) return;
    if (sa.d_m) m = *sa.d_m;
    if (i >= min(nev, m)) return;
    Tg += seg * sa.sT;
    theta += seg * sa.sTh;
    S += seg * sa.sS;
    ws += seg * sa.sWs;
    const int lane = threadIdx.x;
    df32* bdf = reinterpret_cast<df32*>(ism);   // band, m x (P+1)
    df32* x = bdf + (size_t)m * P1;              // m
    df32* U;
    df32* L;
    int* piv;
    if (lu_in_smem) {
        U = x + m;
        L = U + (size_t)m * UW;
        piv = reinterpret_cast<int*>(L + (size_t)m * p);
    } else {
        U = reinterpret_cast<df32*>(ws + (int64_t)i * m * (3 * p + 1));
        L = U + (size_t)m * UW;
        piv = reinterpret_cast<int*>(ws + (int64_t)nev * m * (3 * p + 1)) + (int64_t)i * m;
    }
    for (int e = lane; e < m * P1; e += 32) bdf[e] = df32(Tg[e]);
    __syncwarp();
    const double sigma = theta[i];
    const df32 sig(sigma);
    float scale = 0.0f;
    for (int r = lane; r < m; r += 32) {
        float s = 0.0f;
        for (int d = 0; d <= p && d <= r; ++d) s += fabsf(bdf[r * P1 + d].hi);
        for (int d = 1; d <= p && r + d < m; ++d) s += fabsf(bdf[(r + d) * P1 + d].hi);
        scale = fmaxf(scale, s);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) scale = fmaxf(scale, __shfl_xor_sync(0xffffffffu, scale, off));
    const float tiny = 1e-14f * fmaxf(scale, 1e-30f);
    const df32 zero(0.0f);
    auto tget = [&](int r, int c) -> df32 {  // T - sigma I, 0 outside
        if (r < 0 || c < 0 || r >= m || c >= m) return zero;
        const int d = r - c;
        if (d == 0) return bdf[r * P1] - sig;
        if (d > 0 && d <= p) return bdf[r * P1 + d];
        if (d < 0 && -d <= p) return bdf[c * P1 - d];
        return zero;
    };
    // ---- banded LU with partial pivoting of T - sigma I
    df32 col[P1];
    int cl = lane < UW ? lane : 0;  // this lane's column offset from k
#pragma unroll
    for (int r = 0; r < P1; ++r) col[r] = (lane < UW) ? tget(r, cl) : zero;
    int lk = 0;  // lane holding column k
    for (int k = 0; k < m; ++k) {
        int bi = 0;
        {
            float best = fabsf(col[0].hi);
#pragma unroll
            for (int r = 1; r < P1; ++r) {
                const float v = fabsf(col[r].hi);
                if (k + r < m && v > best) {
                    best = v;
                    bi = r;
                }
            }
        }
        bi = __shfl_sync(0xffffffffu, bi, lk);
#pragma unroll
        for (int r = 1; r < P1; ++r) {
            if (r == bi) {
                const df32 t = col[0];
                col[0] = col[r];
                col[r] = t;
            }
        }
        df32 u(__shfl_sync(0xffffffffu, col[0].hi, lk), __shfl_sync(0xffffffffu, col[0].lo, lk));
        if (fabsf(u.hi) < tiny) u = df32(u.hi < 0.0f ? -tiny : tiny);
        if (lane == lk) col[0] = u;
        const df32 ru = drcp(u);
        df32 lmul[P1];
#pragma unroll
        for (int r = 1; r < P1; ++r) {
            const df32 a(__shfl_sync(0xffffffffu, col[r].hi, lk), __shfl_sync(0xffffffffu, col[r].lo, lk));
            lmul[r] = (k + r < m) ? dmul(a, ru) : zero;
        }
        if (lane < UW) {
            U[(size_t)k * UW + cl] = col[0];
            if (lane != lk) {
#pragma unroll
                for (int r = 1; r < P1; ++r) col[r] = dfma(dneg(lmul[r]), col[0], col[r]);
            }
        }
        if (lane >= 1 && lane <= p) {
#pragma unroll
            for (int r = 1; r < P1; ++r)
                if (r == lane) L[(size_t)k * p + r - 1] = lmul[r];
        }
        if (lane == 0) piv[k] = k + bi;
        if (lane < UW) {
#pragma unroll
            for (int r = 0; r < P; ++r) col[r] = col[r + 1];
            if (lane == lk) {
                cl = UW - 1;  // this lane now holds column k+1+2P
#pragma unroll
                for (int r = 0; r < P; ++r) col[r] = zero;
            } else {
                cl -= 1;
            }
            col[P] = tget(k + P1, k + 1 + cl);
        }
        lk = (lk + 1 == UW) ? 0 : lk + 1;
    }
    __syncwarp();
    // reciprocals of U's diagonal for the backward solve
    for (int r = lane; r < m; r += 32) U[(size_t)r * UW] = drcp(U[(size_t)r * UW]);
    // pseudo-random start (splitmix-style hash of (index, row))
    for (int r = lane; r < m; r += 32) {
        uint64_t z = ((uint64_t)i + 1) * 0x9E3779B97F4A7C15ull + (uint64_t)r + 0x632BE59BD9B4E019ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x[r] = df32((float)(z >> 40) * 0x1.0p-23f - 1.0f);
    }
    __syncwarp();
    // the shift is within 4e-8 * scale of the eigenvalue and eigenvalues closer
    // than 1e-3 * scale form a cluster: each step shrinks the other components
    // by 4e-5 or more, three reach working precision
    for (int it = 0; it < 3; ++it) {
        // forward: row interchanges and L (row r in lane r mod (P+1))
        {
            df32 xv = (lane < P1 && lane < m) ? x[lane] : zero;
            int sk = 0;
            for (int k = 0; k < m; ++k) {
                const int pk = piv[k];
                int sp = sk + (pk - k);
                if (sp >= P1) sp -= P1;
                const df32 xn(__shfl_sync(0xffffffffu, xv.hi, sp), __shfl_sync(0xffffffffu, xv.lo, sp));
                const df32 xo(__shfl_sync(0xffffffffu, xv.hi, sk), __shfl_sync(0xffffffffu, xv.lo, sk));
                if (lane == sp) xv = xo;
                if (lane == sk) xv = xn;
                if (lane < P1 && lane != sk) {
                    const int d = lane - sk + (lane < sk ? P1 : 0);  // row k + d
                    if (k + d < m) xv = dfma(dneg(L[(size_t)k * p + d - 1]), xn, xv);
                }
                if (lane == sk) {
                    x[k] = xn;
                    xv = (k + P1 < m) ? x[k + P1] : zero;
                }
                sk = (sk + 1 == P1) ? 0 : sk + 1;
            }
        }
        __syncwarp();
        // backward: U x = y (row r in lane r mod (2P+1))
        {
            df32 yv = zero, rd = zero;
            int sk = (m - 1) % UW;
            {
                const int r = (m - 1) - ((sk - lane + UW) % UW);
                if (lane < UW && r >= 0) {
                    yv = x[r];
                    rd = U[(size_t)r * UW];
                }
            }
            for (int k = m - 1; k >= 0; --k) {
                const df32 t = dmul(yv, rd);
                const df32 xk(__shfl_sync(0xffffffffu, t.hi, sk), __shfl_sync(0xffffffffu, t.lo, sk));
                if (lane < UW && lane != sk) {
                    const int c = sk - lane + (lane > sk ? UW : 0);  // row k - c
                    if (k - c >= 0) yv = dfma(dneg(U[(size_t)(k - c) * UW + c]), xk, yv);
                }
                if (lane == sk) {
                    x[k] = xk;
                    const int r = k - UW;
                    yv = (r >= 0) ? x[r] : zero;
                    rd = (r >= 0) ? U[(size_t)r * UW] : zero;
                }
                sk = (sk == 0) ? UW - 1 : sk - 1;
            }
        }
        __syncwarp();
        // rescale (the exact normalisation comes at the end, in FP64)
        float nn = 0.0f;
        for (int r = lane; r < m; r += 32) nn = fmaf(x[r].hi, x[r].hi, nn);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, off);
        const float inv = rsqrtf(nn);
        for (int r = lane; r < m; r += 32) x[r] = dmul(x[r], df32(inv));
        __syncwarp();
    }
    // FP64: normalise, Rayleigh quotient, output
    double* xd = reinterpret_cast<double*>(x);
    for (int r = lane; r < m; r += 32) xd[r] = (double)x[r];
    __syncwarp();
    double nn = 0.0;
    for (int r = lane; r < m; r += 32) nn += xd[r] * xd[r];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, off);
    const double inv = 1.0 / sqrt(nn);
    for (int r = lane; r < m; r += 32) xd[r] *= inv;
    __syncwarp();
    double rq = 0.0;
    for (int r = lane; r < m; r += 32) {
        double tx = 0.0;
        for (int c = max(0, r - p); c <= min(m - 1, r + p); ++c) tx += band_get(Tg, p, m, r, c) * xd[c];
        rq += xd[r] * tx;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) rq += __shfl_xor_sync(0xffffffffu, rq, off);
    if (lane == 0) theta[i] = rq;
    for (int r = lane; r < m; r += 32) S[(int64_t)r * nev + i] = xd[r];
}

// Groups close eigenvalues, orthonormalises their vectors, Rayleigh-Ritz in
// each group (cyclic Jacobi), sorts, applies the sign convention.
__global__ void __launch_bounds__(256) cluster_kernel(int m, int p, int ldS, const double* __restrict__ Tb,
                                                      double* __restrict__ theta, double* __restrict__ S,
                                                      double* __restrict__ tmp /* m x ldS */, SegArgs sa) {
    __shared__ double K[kMaxNev * kMaxNev];
    __shared__ double Z[kMaxNev * kMaxNev];
    __shared__ double red[256];
    __shared__ double th[kMaxNev];
    __shared__ int start[kMaxNev + 1];
    __shared__ int ngroups;
    __shared__ double s_scale;
    const int seg = blockIdx.x;
    if (sa.active && !sa.active[seg]) return;
    if (sa.d_m) m = *sa.d_m;
    const int nev = min(ldS, m);  // columns computed; S keeps row stride ldS
    Tb += seg * sa.sT;
    theta += seg * sa.sTh;
    S += seg * sa.sS;
    tmp += seg * sa.sTmp;
    const int tid = threadIdx.x;
    // scale = max |theta|, at least the largest diagonal magnitude
    double sc = 0.0;
    for (int r = tid; r < m; r += 256) sc = fmax(sc, fabs(band_get(Tb, p, m, r, r)));
    for (int k = tid; k < nev; k += 256) sc = fmax(sc, fabs(theta[k]));
    red[tid] = sc;
    __syncthreads();
    if (tid == 0) {
        for (int t = 1; t < 256; ++t) sc = fmax(sc, red[t]);
        s_scale = fmax(sc, 1e-300);
        // sort theta (and remember the permutation in start[] temporarily): insertion sort
        for (int k = 0; k < nev; ++k) th[k] = theta[k];
    }
    __syncthreads();
    // sort columns by theta (selection on thread 0, column swaps in parallel)
    for (int a = 0; a < nev; ++a) {
        __shared__ int sel;
        if (tid == 0) {
            int best = a;
            for (int k = a + 1; k < nev; ++k)
                if (th[k] < th[best]) best = k;
            sel = best;
            const double t = th[a];
            th[a] = th[best];
            th[best] = t;
        }
        __syncthreads();
        if (sel != a) {
            for (int r = tid; r < m; r += 256) {
                const double t = S[(int64_t)r * ldS + a];
                S[(int64_t)r * ldS + a] = S[(int64_t)r * ldS + sel];
                S[(int64_t)r * ldS + sel] = t;
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        int g = 0;
        start[0] = 0;
        for (int k = 1; k < nev; ++k)
            if (th[k] - th[k - 1] > 1e-3 * s_scale) start[++g] = k;
        start[++g] = nev;
        ngroups = g;
    }
    __syncthreads();
    for (int g = 0; g < ngroups; ++g) {
        const int a0 = start[g], a1 = start[g + 1], k = a1 - a0;
        if (k < 2) continue;
        // MGS twice over the group's columns
        for (int pass = 0; pass < 2; ++pass) {
            for (int a = a0; a < a1; ++a) {
                for (int q = a0; q < a; ++q) {
                    double s = 0.0;
                    for (int r = tid; r < m; r += 256) s += S[(int64_t)r * ldS + q] * S[(int64_t)r * ldS + a];
                    red[tid] = s;
                    __syncthreads();
                    for (int w = 128; w > 0; w >>= 1) {
                        if (tid < w) red[tid] += red[tid + w];
                        __syncthreads();
                    }
                    const double dot = red[0];
                    __syncthreads();
                    for (int r = tid; r < m; r += 256) S[(int64_t)r * ldS + a] -= dot * S[(int64_t)r * ldS + q];
                    __syncthreads();
                }
                double s = 0.0;
                for (int r = tid; r < m; r += 256) s += S[(int64_t)r * ldS + a] * S[(int64_t)r * ldS + a];
                red[tid] = s;
                __syncthreads();
                for (int w = 128; w > 0; w >>= 1) {
                    if (tid < w) red[tid] += red[tid + w];
                    __syncthreads();
                }
                const double inv = 1.0 / sqrt(red[0]);
                __syncthreads();
                for (int r = tid; r < m; r += 256) S[(int64_t)r * ldS + a] *= inv;
                __syncthreads();
            }
        }
        // tmp = T * S_group
        for (int r = tid; r < m; r += 256) {
            for (int a = a0; a < a1; ++a) {
                double t = 0.0;
                for (int c = max(0, r - p); c <= min(m - 1, r + p); ++c) t += band_get(Tb, p, m, r, c) * S[(int64_t)c * ldS + a];
                tmp[(int64_t)r * ldS + a] = t;
            }
        }
        __syncthreads();
        // K = S_g^T T S_g
        for (int e = 0; e < k * k; ++e) {
            const int a = a0 + e / k, q = a0 + e % k;
            double s = 0.0;
            for (int r = tid; r < m; r += 256) s += S[(int64_t)r * ldS + a] * tmp[(int64_t)r * ldS + q];
            red[tid] = s;
            __syncthreads();
            for (int w = 128; w > 0; w >>= 1) {
                if (tid < w) red[tid] += red[tid + w];
                __syncthreads();
            }
            if (tid == 0) K[e] = red[0];
            __syncthreads();
        }
        // cyclic Jacobi on K (thread 0; k <= 64)
        if (tid == 0) {
            for (int e = 0; e < k * k; ++e) Z[e] = (e / k == e % k) ? 1.0 : 0.0;
            for (int a = 0; a < k; ++a)
                for (int q = a + 1; q < k; ++q) {
                    const double s = 0.5 * (K[a * k + q] + K[q * k + a]);
                    K[a * k + q] = K[q * k + a] = s;
                }
            for (int sweep = 0; sweep < 50; ++sweep) {
                double off = 0.0;
                for (int a = 0; a < k; ++a)
                    for (int q = a + 1; q < k; ++q) off += K[a * k + q] * K[a * k + q];
                if (off < 1e-32 * s_scale * s_scale) break;
                for (int a = 0; a < k; ++a)
                    for (int q = a + 1; q < k; ++q) {
                        const double apq = K[a * k + q];
                        if (fabs(apq) < 1e-300) continue;
                        const double tau = (K[q * k + q] - K[a * k + a]) / (2.0 * apq);
                        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                        for (int r = 0; r < k; ++r) {
                            const double kra = K[r * k + a], krq = K[r * k + q];
                            K[r * k + a] = c * kra - s * krq;
                            K[r * k + q] = s * kra + c * krq;
                        }
                        for (int r = 0; r < k; ++r) {
                            const double kar = K[a * k + r], kqr = K[q * k + r];
                            K[a * k + r] = c * kar - s * kqr;
                            K[q * k + r] = s * kar + c * kqr;
                        }
                        for (int r = 0; r < k; ++r) {
                            const double zra = Z[r * k + a], zrq = Z[r * k + q];
                            Z[r * k + a] = c * zra - s * zrq;
                            Z[r * k + q] = s * zra + c * zrq;
                        }
                    }
            }
            // sort eigenpairs of K ascending
            for (int a = 0; a < k; ++a) {
                int best = a;
                for (int q = a + 1; q < k; ++q)
                    if (K[q * k + q] < K[best * k + best]) best = q;
                if (best != a) {
                    const double t = K[a * k + a];
                    K[a * k + a] = K[best * k + best];
                    K[best * k + best] = t;
                    for (int r = 0; r < k; ++r) {
                        const double z = Z[r * k + a];
                        Z[r * k + a] = Z[r * k + best];
                        Z[r * k + best] = z;
                    }
                }
            }
            for (int a = 0; a < k; ++a) th[a0 + a] = K[a * k + a];
        }
        __syncthreads();
        // S_g <- S_g Z
        for (int r = tid; r < m; r += 256) {
            double row[kMaxNev];
            for (int a = 0; a < k; ++a) row[a] = S[(int64_t)r * ldS + a0 + a];
            for (int a = 0; a < k; ++a) {
                double s = 0.0;
                for (int q = 0; q < k; ++q) s += row[q] * Z[q * k + a];
                S[(int64_t)r * ldS + a0 + a] = s;
            }
        }
        __syncthreads();
    }
    // sign convention: the first entry of largest magnitude is positive
    for (int a = 0; a < nev; ++a) {
        double best = -1.0;
        int bi = 0;
        for (int r = tid; r < m; r += 256) {
            const double v = fabs(S[(int64_t)r * ldS + a]);
            if (v > best) {
                best = v;
                bi = r;
            }
        }
        __shared__ double bv[256];
        __shared__ int bix[256];
        bv[tid] = best;
        bix[tid] = bi;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (tid < w) {
                if (bv[tid + w] > bv[tid] || (bv[tid + w] == bv[tid] && bix[tid + w] < bix[tid])) {
                    bv[tid] = bv[tid + w];
                    bix[tid] = bix[tid + w];
                }
            }
            __syncthreads();
        }
        const bool flip = S[(int64_t)bix[0] * ldS + a] < 0.0;
        __syncthreads();
        if (flip)
            for (int r = tid; r < m; r += 256) S[(int64_t)r * ldS + a] = -S[(int64_t)r * ldS + a];
        __syncthreads();
    }
    for (int k = tid; k < nev; k += 256) theta[k] = th[k];
}

}  // namespace

size_t ritz_workspace_bytes(int m, int p, int nev) {
    return sizeof(double) * ((size_t)nev * m * (3 * p + 1) + (size_t)m * nev + 2 * (size_t)nev) +
           sizeof(int) * (size_t)nev * m + 256;
}

namespace {
bbl_status set_ritz_attrs() {
    static bool attr_set = false;
    if (!attr_set) {
        BBL_CUDA(cudaFuncSetAttribute(bisect_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBandSmemMax));
        BBL_CUDA(cudaFuncSetAttribute(bisect_lane_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBandSmemMax));
        BBL_CUDA(cudaFuncSetAttribute(bisect_lane_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBandSmemMax));
        BBL_CUDA(cudaFuncSetAttribute(bisect_lane_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBandSmemMax));
        BBL_CUDA(cudaFuncSetAttribute(bisect_lane_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBandSmemMax));
        BBL_CUDA(cudaFuncSetAttribute(bisect_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBandSmemMax));
        BBL_CUDA(cudaFuncSetAttribute(bisect_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBandSmemMax));
        BBL_CUDA(cudaFuncSetAttribute(bisect_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBandSmemMax));
        BBL_CUDA(cudaFuncSetAttribute(bisect_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBandSmemMax));
        BBL_CUDA(cudaFuncSetAttribute(bisect_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBandSmemMax));
        BBL_CUDA(cudaFuncSetAttribute(invit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(200 * 1024)));
        BBL_CUDA(cudaFuncSetAttribute(invit_df_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInvitSmemMax));
        BBL_CUDA(cudaFuncSetAttribute(invit_df_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInvitSmemMax));
        BBL_CUDA(cudaFuncSetAttribute(invit_df_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInvitSmemMax));
        BBL_CUDA(cudaFuncSetAttribute(invit_df_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInvitSmemMax));
        attr_set = true;
    }
    return BBL_OK;
}

// the register-window bisection for p in {1, 2, 4, 8, 16}, else the generic one
bbl_status launch_bisect(dim3 grid, int m, int p, int nev, const double* Tb, double* theta, double* width,
                         int band_smem, size_t band_bytes, SegArgs sa, const double* warm, int warm_count,
                         cudaStream_t st) {
    const size_t sm = band_smem ? band_bytes : 0;
    const unsigned th = 32 * kBisectWarps;
    // one shift per thread: FP32 + float-float band copies in shared memory
    const size_t lane_smem = (size_t)m * (p + 1) * (sizeof(float) + sizeof(df32));
    const bool lane = (p == 1 || p == 2 || p == 4 || p == 8) && lane_smem <= kBandSmemMax;
    if (lane) {
        switch (p) {
            case 1: bisect_lane_kernel<1><<<grid, 256, lane_smem, st>>>(m, nev, Tb, theta, width, 1, sa, warm, warm_count); break;
            case 2: bisect_lane_kernel<2><<<grid, 256, lane_smem, st>>>(m, nev, Tb, theta, width, 1, sa, warm, warm_count); break;
            case 4: bisect_lane_kernel<4><<<grid, 256, lane_smem, st>>>(m, nev, Tb, theta, width, 1, sa, warm, warm_count); break;
            default: bisect_lane_kernel<8><<<grid, 256, lane_smem, st>>>(m, nev, Tb, theta, width, 1, sa, warm, warm_count); break;
        }
    } else {
        switch (p) {
            case 1: bisect_kernel<1><<<grid, th, sm, st>>>(m, p, nev, Tb, theta, width, band_smem, sa, warm, warm_count); break;
            case 2: bisect_kernel<2><<<grid, th, sm, st>>>(m, p, nev, Tb, theta, width, band_smem, sa, warm, warm_count); break;
            case 4: bisect_kernel<4><<<grid, th, sm, st>>>(m, p, nev, Tb, theta, width, band_smem, sa, warm, warm_count); break;
            case 8: bisect_kernel<8><<<grid, th, sm, st>>>(m, p, nev, Tb, theta, width, band_smem, sa, warm, warm_count); break;
            case 16: bisect_kernel<16><<<grid, th, sm, st>>>(m, p, nev, Tb, theta, width, band_smem, sa, warm, warm_count); break;
            default: bisect_kernel<0><<<grid, th, sm, st>>>(m, p, nev, Tb, theta, width, band_smem, sa, warm, warm_count);
        }
    }
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

// inverse iteration: the register-window solves for p in {1, 2, 4, 8} (LU
// factors in shared memory when they fit), else the generic kernel
bbl_status launch_invit(dim3 grid, int m, int p, int nev, const double* Tb, double* theta, double* S, double* ws,
                        SegArgs sa, cudaStream_t st) {
    if (p == 1 || p == 2 || p == 4 || p == 8) {
        const int UW = 2 * p + 1, P1 = p + 1;
        const size_t base = sizeof(df32) * ((size_t)m * P1 + m) + 16;
        const size_t lu = sizeof(df32) * (size_t)m * (UW + p) + sizeof(int) * (size_t)m;
        if (base <= kInvitSmemMax) {
            const int lu_smem = (base + lu <= kInvitSmemMax) ? 1 : 0;
            const size_t smem = base + (lu_smem ? lu : 0);
            switch (p) {
                case 1: invit_df_kernel<1><<<grid, 32, smem, st>>>(m, Tb, theta, S, nev, ws, lu_smem, sa); break;
                case 2: invit_df_kernel<2><<<grid, 32, smem, st>>>(m, Tb, theta, S, nev, ws, lu_smem, sa); break;
                case 4: invit_df_kernel<4><<<grid, 32, smem, st>>>(m, Tb, theta, S, nev, ws, lu_smem, sa); break;
                default: invit_df_kernel<8><<<grid, 32, smem, st>>>(m, Tb, theta, S, nev, ws, lu_smem, sa); break;
            }
            BBL_LAUNCH_CHECK();
            return BBL_OK;
        }
    }
    const size_t band_bytes = sizeof(double) * (size_t)m * (p + 1);
    const size_t base = sizeof(double) * ((size_t)(p + 1) * (2 * p + 1) + m + p + 8);
    const int inv_smem = (base + band_bytes <= 200 * 1024) ? 1 : 0;
    const size_t smem = base + (inv_smem ? band_bytes : 0);
    if (smem > 200 * 1024) return set_error(BBL_ERR_UNSUPPORTED, "ritz: m=%d too large for the inverse iteration", m);
    invit_kernel<<<grid, 32, smem, st>>>(m, p, Tb, theta, S, nev, ws, 0.0, inv_smem, sa);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}
}  // namespace

bbl_status ritz_dev(int m, int p, int nev, const double* Tb, double* theta, double* S, DevBuf& work, cudaStream_t st,
                    const double* warm, int warm_count) {
    const size_t need = ritz_workspace_bytes(m, p, nev);
    if (work.bytes < need) BBL_TRY(work.alloc(need + need / 2));
    double* ws = work.as<double>();
    double* width = reinterpret_cast<double*>(reinterpret_cast<char*>(ws) + sizeof(double) * (size_t)nev * m * (3 * p + 1) +
                                      sizeof(int) * (size_t)nev * m + 64);
    width = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(width) + 15) & ~uintptr_t(15));
    double* tmp = width + nev + 2;
    const size_t band_bytes = sizeof(double) * (size_t)m * (p + 1);
    const int band_smem = band_bytes <= kBandSmemMax ? 1 : 0;
    BBL_TRY(set_ritz_attrs());
    const SegArgs one{nullptr, nullptr, 0, 0, 0, 0, 0};
    BBL_TRY(launch_bisect(dim3(nev), m, p, nev, Tb, theta, width, band_smem, band_bytes, one, warm, warm_count, st));
    BBL_TRY(launch_invit(dim3(nev), m, p, nev, Tb, theta, S, ws, one, st));
    cluster_kernel<<<1, 256, 0, st>>>(m, p, nev, Tb, theta, S, tmp, one);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

// Per-segment workspace (doubles) for orders up to m_max.
size_t ritz_seg_workspace_doubles(int m_max, int p, int nev) {
    const size_t d = (size_t)nev * m_max * (3 * p + 1) + (sizeof(int) * (size_t)nev * m_max + 7) / 8 + 16;
    return (d + 31) & ~size_t(31);
}

// Batched Ritz solves: nseg independent band matrices Tb + s*sT (order *d_m,
// at most m_max, bandwidth p), k = min(nev, m) lowest pairs each into
// theta + s*sTh and S + s*sS (row stride nev); segments with active[s] == 0
// are skipped.  ws: nseg * ritz_seg_workspace_doubles; tmp: nseg * m_max * nev.
bbl_status ritz_dev_batched(int m_max, int p, int nev, int nseg, const double* Tb, int64_t sT, double* theta,
                            int64_t sTh, double* width, double* S, int64_t sS, double* ws, double* tmp, const int* d_m,
                            const int* active, cudaStream_t st) {
    BBL_TRY(set_ritz_attrs());
    const size_t band_bytes = sizeof(double) * (size_t)m_max * (p + 1);
    const int band_smem = band_bytes <= kBandSmemMax ? 1 : 0;
    const int64_t sWs = (int64_t)ritz_seg_workspace_doubles(m_max, p, nev);
    const SegArgs sa{d_m, active, sT, sTh, sS, sWs, (int64_t)m_max * nev};
    dim3 g(nev, nseg);
    BBL_TRY(launch_bisect(g, m_max, p, nev, Tb, theta, width, band_smem, band_bytes, sa, nullptr, 0, st));
    BBL_TRY(launch_invit(g, m_max, p, nev, Tb, theta, S, ws, sa, st));
    cluster_kernel<<<nseg, 256, 0, st>>>(m_max, p, nev, Tb, theta, S, tmp, sa);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

}  // namespace bbl

extern "C" bbl_status bbl_ritz_banded(int m, int p, int nev, const double* Tband, double* theta, double* S,
                                      void* stream) {
    using namespace bbl;
    if (m < 1 || p < 0 || p > kMaxP || nev < 1 || nev > m || nev > kMaxNev || !Tband || !theta || !S)
        return set_error(BBL_ERR_INVALID_ARG, "ritz_banded: bad arguments (m=%d p=%d nev=%d)", m, p, nev);
    if (m > 16384) return set_error(BBL_ERR_UNSUPPORTED, "ritz_banded: m=%d above 16384", m);
    cudaStream_t st = as_stream(stream);
    DevBuf work;
    BBL_TRY(ritz_dev(m, p, nev, Tband, theta, S, work, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    return BBL_OK;
}
