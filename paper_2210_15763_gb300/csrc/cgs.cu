// Fused first update and second Gram of the FP32 stage's block Gram-Schmidt
// (Sec. II.A, full reorthogonalisation; Eqs. 7-8), on the tensor cores:
//
//     W1 = W - Q C1        (written over W)
//     C2 = Q^T W1          (FP64, m x 8)
//
// for an FP32 basis Q of nblocks blocks of n x 8 (row-major blocks, b = 8)
// and FP64 coefficients C1 (m x 8, m = 8 nblocks).  Two classical passes
// read the basis three times after the first Gram (update, Gram, update);
// here the first update and the second Gram share one read.  A CTA takes
// 16-row chunks of the basis in turn: the chunk's rows of every block (16 x
// 8 FP32 = 512 contiguous bytes per block) and of W are copied into a ring
// of shared-memory stages with cp.async, several chunks ahead, and from one
// staged chunk the CTA forms the chunk's W1 and then the chunk's
// contribution to Q^T W1.
//
// The products run as mma.sync.m16n8k16 BF16 with FP32 accumulation.  Each
// FP32 operand is split exactly into three BF16 parts, x = x1 + x2 + x3
// (x1 = bf16(x), x2 = bf16(x - x1), x3 = x - x1 - x2, which has at most 8
// significant bits), and of the nine partial products the six with i + j <=
// 4 are formed: a b = a1 b1 + a1 b2 + a2 b1 + a1 b3 + a2 b2 + a3 b1 + e with
// |e| <= 2^-23 |a b|, about the rounding of an FP32 product.
//  * Update: M = the chunk's 16 rows, N = 8, K = 16 = the columns of a pair
//    of basis blocks; the update group's warps split the pairs (two
//    accumulators each) and their partial sums are added in a fixed order.  The two newest blocks
//    are applied with FP32 FMAs instead (W's own-block and previous-block
//    coefficients in Lanczos are of the order of ||H||, the older ones of
//    the order of the lost orthogonality).
//  * Gram: M = 16 basis columns (a pair of blocks), N = 8, K = the chunk's
//    16 rows (k = 2t, 2t+1, 2t+8, 2t+9 read rows t, t+4, t+8, t+12, the same
//    order for W1); each Gram warp keeps its pairs' 16 x 8 sums in registers over
//    every chunk its CTA takes (a chunk's products are formed from zero and
//    added to the running sum in FP32, so the accumulation's rounding is
//    that of plain FP32 additions), and the CTAs' sums are added in FP64.
// Every shared-memory access pattern above is free of bank conflicts.
#include <cuda_bf16.h>

#include "common.cuh"

namespace bbl {
namespace {

constexpr int kFuRows = 16;                          // rows per chunk
constexpr int kFuWarps = 16;
constexpr int kFuThreads = 32 * kFuWarps;
constexpr int kFuMaxBlocks = 128;                    // 1024 basis columns
constexpr int kFuGramPairsPerWarp = kFuMaxBlocks / 2 / (kFuWarps / 2);  // register sums per Gram warp
constexpr int kFuMaxStages = 5;
constexpr size_t kFuSmemLimit = 220 * 1024;

// two FP32 values rounded to BF16 (nearest even), packed: lo in bits 0-15
__device__ __forceinline__ unsigned bf2_pack(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned*>(&h);
}
__device__ __forceinline__ float bf_lo(unsigned p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf_hi(unsigned p) { return __uint_as_float(p & 0xFFFF0000u); }
// (lo, hi) = p1 + p2 + p3 exactly, each a packed BF16 pair (both differences
// are exact in FP32; the last remainder has at most 8 significant bits)
__device__ __forceinline__ void bf16x3_split(float lo, float hi, unsigned& p1, unsigned& p2, unsigned& p3) {
    p1 = bf2_pack(lo, hi);
    const float rl = lo - bf_lo(p1), rh = hi - bf_hi(p1);
    p2 = bf2_pack(rl, rh);
    p3 = bf2_pack(rl - bf_lo(p2), rh - bf_hi(p2));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// d += A B from the three-part splits a[part][reg], b[part][reg]: the six
// partial products with i + j <= 4, the smallest first
__device__ __forceinline__ void mma_bf16x3(float (&d)[4], const unsigned (&a)[3][4], const unsigned (&b)[3][2]) {
    mma_bf16(d, a[2], b[0]);
    mma_bf16(d, a[1], b[1]);
    mma_bf16(d, a[0], b[2]);
    mma_bf16(d, a[1], b[0]);
    mma_bf16(d, a[0], b[1]);
    mma_bf16(d, a[0], b[0]);
}

__device__ __forceinline__ void fu_cp16(void* smem, const void* gmem, int src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void fu_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most `pending` of this thread's copy groups are in flight
__device__ __forceinline__ void fu_wait(int pending) {
    switch (pending) {
        case 0: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
        case 1: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
        case 2: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
        default: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
    }
}

// Blocks of the update on the tensor cores (the rest, the ne newest, by FMA)
__host__ __device__ inline int fu_tc_blocks(int nblocks) { return nblocks - (nblocks < 2 ? nblocks : 2); }
__host__ __device__ inline int fu_tc_pairs(int nblocks) { return (fu_tc_blocks(nblocks) + 1) >> 1; }

// C1 (FP64, m x 8) -> per tensor-core block pair q (blocks 2q, 2q + 1) and
// lane the update's B fragment, split: b0 = C1 rows 16q + 2t, 16q + 2t + 1,
// b1 = rows 16q + 8 + 2t, 16q + 9 + 2t, column g (g = lane / 4, t = lane %
// 4; b1 = 0 past the tensor-core blocks), C1 rounded to FP32 first as in the
// FP32 update.  fa = {b0 part 1, b1 part 1, b0 part 2, b1 part 2}, fb =
// {b0 part 3, b1 part 3}.
__global__ void cgs_split_c1_kernel(int nblocks, const double* __restrict__ C1, uint4* __restrict__ fa,
                                    uint2* __restrict__ fb) {
    const int nt = fu_tc_blocks(nblocks);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= fu_tc_pairs(nblocks) * 32) return;
    const int q = e >> 5, lane = e & 31, g = lane >> 2, t = lane & 3;
    const bool two = 2 * q + 1 < nt;
    const int r0 = 16 * q + 2 * t, r1 = 16 * q + 8 + 2 * t;
    unsigned b0[3], b1[3];
    bf16x3_split((float)C1[r0 * 8 + g], (float)C1[(r0 + 1) * 8 + g], b0[0], b0[1], b0[2]);
    bf16x3_split(two ? (float)C1[r1 * 8 + g] : 0.f, two ? (float)C1[(r1 + 1) * 8 + g] : 0.f, b1[0], b1[1], b1[2]);
    fa[e] = make_uint4(b0[0], b1[0], b0[1], b1[1]);
    fb[e] = make_uint2(b0[2], b1[2]);
}

// Named barriers of the two warp groups (id 0 is __syncthreads): the update
// group's own barrier, "W1 of chunk i is ready" (ids 2, 3 by the parity of
// i) and "the Gram group is done with chunk i" (ids 4, 5).  A group never
// arrives twice at one id before the other group has passed it: the next
// arrival at the same id is two chunks later, and each group's chunk i + 2
// waits for the other group's chunk i.
__device__ __forceinline__ void fu_bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void fu_bar_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}
constexpr int kFuGroupWarps = kFuWarps / 2;          // warps per group
constexpr int kFuGroupThreads = 32 * kFuGroupWarps;

// Shared memory: [stages x (the chunk's rows of every block, nblocks x 512
// B, then W's rows, 512 B)][update partials: kFuGroupWarps x 512 B][W1's
// rows, two buffers: 1024 B][C1's rows of the two newest blocks in FP32:
// 512 B].  The update's B fragments are read through the L1 cache.
__host__ __device__ inline size_t fu_stage_bytes(int nblocks) { return (size_t)nblocks * 512 + 512; }
inline size_t fu_smem_bytes(int nblocks, int stages) {
    return (size_t)stages * fu_stage_bytes(nblocks) + (size_t)kFuGroupWarps * 512 + 1536;
}

// Persistent CTAs take the 16-row chunks blockIdx.x, blockIdx.x + gridDim.x,
// ...; `stages` >= 3 shared-memory stages hold the chunks in flight.  Warps
// 0-7 (the update group) copy the chunks in, form W1 = W - Q C1 of chunk i
// and hand it over; warps 8-15 (the Gram group) meanwhile form chunk i - 1's
// contribution to Q^T W1.  A stage is refilled (with chunk i - 2 + stages)
// once both groups are done with its chunk i - 2.
__global__ void __launch_bounds__(kFuThreads, 1) cgs_update_gram_kernel(int64_t n, int nblocks, int64_t nchunks,
                                                                     int stages, const float* __restrict__ Q,
                                                                     const double* __restrict__ C1,
                                                                     const uint4* __restrict__ fa,
                                                                     const uint2* __restrict__ fb,
                                                                     float* __restrict__ W,
                                                                     double* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char fu_smem[];
    const int nt = fu_tc_blocks(nblocks), ne = nblocks - nt;  // tensor-core blocks, FMA blocks
    const int ntp = fu_tc_pairs(nblocks);
    const size_t sb = fu_stage_bytes(nblocks);
    unsigned char* stage0 = fu_smem;
    float* red = reinterpret_cast<float*>(stage0 + (size_t)stages * sb);  // [kFuGroupWarps][16][8]
    float* W1s = red + kFuGroupWarps * 128;                                 // [2][16][8]
    float* c1x = W1s + 256;  // [8 ne][8]: C1's rows of the ne newest blocks, FP32
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int64_t G = gridDim.x;

    for (int e = threadIdx.x; e < ne * 64; e += kFuThreads) c1x[e] = (float)C1[(int64_t)nt * 64 + e];
    __syncthreads();

    if (warp < kFuGroupWarps) {
        // ---------------- update group
        const int uw = warp;
        // 16-byte piece `lane` (row lane / 2, half lane % 2) of the chunk's
        // rows of blocks uw, uw + 8, ...; the last warp also copies W's.
        const int pr = lane >> 1, ph = lane & 1;
        auto stage_chunk = [&](int64_t c, int s) {
            if (c < nchunks) {
                const int64_t row = c * kFuRows + pr;
                const bool ok = row < n;
                float* dst = reinterpret_cast<float*>(stage0 + (size_t)s * sb) + uw * 128 + lane * 4;
                const float* src = Q + ((int64_t)uw * n + row) * 8 + ph * 4;
                const int64_t step = (int64_t)kFuGroupWarps * n * 8;
                for (int j = uw; j < nblocks; j += kFuGroupWarps, src += step, dst += kFuGroupWarps * 128)
                    fu_cp16(dst, ok ? (const void*)src : (const void*)Q, ok ? 16 : 0);
                if (uw == kFuGroupWarps - 1) {
                    float* wd = reinterpret_cast<float*>(stage0 + (size_t)s * sb) + nblocks * 128 + lane * 4;
                    fu_cp16(wd, ok ? (const void*)(W + row * 8 + ph * 4) : (const void*)W, ok ? 16 : 0);
                }
            }
            fu_commit();
        };
        for (int q = 0; q < stages; ++q) stage_chunk(blockIdx.x + q * G, q);
        int i = 0;
        for (int64_t c = blockIdx.x; c < nchunks; c += G, ++i) {
            const int s = i % stages;
            if (i >= 2) {
                // the Gram group is done with chunk i - 2: its stage takes chunk i - 2 + stages
                fu_bar_sync(4 + (i & 1), kFuThreads);
                stage_chunk(c + (int64_t)(stages - 2) * G, (i - 2) % stages);
            }
            // copy group k holds chunk k; at most stages - 2 later groups may be in flight
            fu_wait(stages - 2);
            fu_bar_sync(1, kFuGroupThreads);  // every piece of chunk i has landed
            const float* Qs = reinterpret_cast<const float*>(stage0 + (size_t)s * sb);
            const float* Ws = Qs + nblocks * 128;
            const int64_t r0 = c * kFuRows;
            float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
            auto upd = [&](int q, float (&d)[4]) {
                // A: rows g / g + 8, k = 2t, 2t + 1 of block 2q (a0, a1) and of block 2q + 1 (a2, a3)
                const float* T0 = Qs + (2 * q) * 128 + g * 8 + 2 * t;
                const float2 x0 = *reinterpret_cast<const float2*>(T0);
                const float2 x1 = *reinterpret_cast<const float2*>(T0 + 64);
                const float2 x2 = *reinterpret_cast<const float2*>(T0 + 128);
                const float2 x3 = *reinterpret_cast<const float2*>(T0 + 192);
                unsigned a[3][4];
                bf16x3_split(x0.x, x0.y, a[0][0], a[1][0], a[2][0]);
                bf16x3_split(x1.x, x1.y, a[0][1], a[1][1], a[2][1]);
                bf16x3_split(x2.x, x2.y, a[0][2], a[1][2], a[2][2]);
                bf16x3_split(x3.x, x3.y, a[0][3], a[1][3], a[2][3]);
                const uint4 f = __ldg(fa + q * 32 + lane);
                const uint2 f3 = __ldg(fb + q * 32 + lane);
                const unsigned b[3][2] = {{f.x, f.y}, {f.z, f.w}, {f3.x, f3.y}};
                mma_bf16x3(d, a, b);
            };
            int q = uw;
            for (; q + kFuGroupWarps < ntp; q += 2 * kFuGroupWarps) {
                upd(q, d0);
                upd(q + kFuGroupWarps, d1);
            }
            if (q < ntp) upd(q, d0);
            float* rw = red + uw * 128;
            *reinterpret_cast<float2*>(rw + g * 8 + 2 * t) = make_float2(d0[0] + d1[0], d0[1] + d1[1]);
            *reinterpret_cast<float2*>(rw + (g + 8) * 8 + 2 * t) = make_float2(d0[2] + d1[2], d0[3] + d1[3]);
            fu_bar_sync(1, kFuGroupThreads);
            if (threadIdx.x < 128) {
                const int e = threadIdx.x;  // 16 rows x 8 columns
                const int r = e >> 3, col = e & 7;
                float x = Ws[e];
                for (int cc = 0; cc < 8 * ne; ++cc)
                    x = fmaf(-Qs[(nt + (cc >> 3)) * 128 + r * 8 + (cc & 7)], c1x[cc * 8 + col], x);
                float sum = red[e];
#pragma unroll
                for (int w = 1; w < kFuGroupWarps; ++w) sum += red[w * 128 + e];
                const float w1 = x - sum;
                W1s[(i & 1) * 128 + e] = w1;
                if (r0 + r < n) W[r0 * 8 + e] = w1;
            }
            fu_bar_arrive(2 + (i & 1), kFuThreads);  // W1 of chunk i is ready
        }
        // the Gram group's last two chunks: their stages are not refilled, but
        // the arrivals are matched so that no barrier is left half-passed
        if (i >= 2) fu_bar_sync(4 + (i & 1), kFuThreads);
        if (i >= 1) fu_bar_sync(4 + ((i + 1) & 1), kFuThreads);
        fu_wait(0);
    } else {
        // ---------------- Gram group
        const int gw = warp - kFuGroupWarps;
        const int npairs = (nblocks + 1) >> 1;
        float acc[kFuGramPairsPerWarp][4];
#pragma unroll
        for (int k = 0; k < kFuGramPairsPerWarp; ++k) acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = 0.f;
        int i = 0;
        for (int64_t c = blockIdx.x; c < nchunks; c += G, ++i) {
            const int s = i % stages;
            fu_bar_sync(2 + (i & 1), kFuThreads);  // W1 of chunk i (and its stage) are ready
            const float* Qs = reinterpret_cast<const float*>(stage0 + (size_t)s * sb);
            const float* W1c = W1s + (i & 1) * 128;
            // B = W1 (k = 2t, 2t + 1 -> rows t, t + 4; k = 2t + 8, 2t + 9 -> rows t + 8, t + 12), split
            unsigned bw[3][2];
            bf16x3_split(W1c[t * 8 + g], W1c[(t + 4) * 8 + g], bw[0][0], bw[1][0], bw[2][0]);
            bf16x3_split(W1c[(t + 8) * 8 + g], W1c[(t + 12) * 8 + g], bw[0][1], bw[1][1], bw[2][1]);
#pragma unroll
            for (int k = 0; k < kFuGramPairsPerWarp; ++k) {
                const int p = gw + kFuGroupWarps * k;
                if (p < npairs) {
                    // A = [Q_2p Q_2p+1]^T: row = column of the pair (g: block 2p, g + 8:
                    // block 2p + 1; for an odd last pair the second block's rows are unused)
                    const float* T0 = Qs + (2 * p) * 128 + t * 8 + g;
                    const float* T1 = T0 + 128;
                    unsigned a[3][4];
                    bf16x3_split(T0[0], T0[32], a[0][0], a[1][0], a[2][0]);
                    bf16x3_split(T1[0], T1[32], a[0][1], a[1][1], a[2][1]);
                    bf16x3_split(T0[64], T0[96], a[0][2], a[1][2], a[2][2]);
                    bf16x3_split(T1[64], T1[96], a[0][3], a[1][3], a[2][3]);
                    // the chunk's products from zero (the tensor cores' FP32 accumulation
                    // truncates), then one rounded FP32 addition to the running sum
                    float d[4] = {0.f, 0.f, 0.f, 0.f};
                    mma_bf16x3(d, a, bw);
#pragma unroll
                    for (int r = 0; r < 4; ++r) acc[k][r] += d[r];
                }
            }
            fu_bar_arrive(4 + (i & 1), kFuThreads);  // done with chunk i's stage and W1
        }
        // this CTA's sums -> its FP64 slot (row-major m x 8)
        double* part = partial + (int64_t)blockIdx.x * nblocks * 64;
#pragma unroll
        for (int k = 0; k < kFuGramPairsPerWarp; ++k) {
            const int p = gw + kFuGroupWarps * k;
            if (p < npairs) {
                part[((2 * p) * 8 + g) * 8 + 2 * t] = (double)acc[k][0];
                part[((2 * p) * 8 + g) * 8 + 2 * t + 1] = (double)acc[k][1];
                if (2 * p + 1 < nblocks) {
                    part[((2 * p + 1) * 8 + g) * 8 + 2 * t] = (double)acc[k][2];
                    part[((2 * p + 1) * 8 + g) * 8 + 2 * t + 1] = (double)acc[k][3];
                }
            }
        }
    }
}

// stages of the ring for nblocks (0: the basis does not fit)
int fu_stages(int nblocks) {
    for (int s = kFuMaxStages; s >= 3; --s)
        if (fu_smem_bytes(nblocks, s) <= kFuSmemLimit) return s;
    return 0;
}

}  // namespace

bool update_gram_tc_supports(int nblocks) {
    return nblocks >= 1 && nblocks <= kFuMaxBlocks && fu_stages(nblocks) >= 3;
}

bbl_status update_gram_tc(int64_t n, int nblocks, const float* Q, const double* C1, float* W, double* C2,
                          DevBuf& work, cudaStream_t st) {
    if (!update_gram_tc_supports(nblocks))
        return set_error(BBL_ERR_UNSUPPORTED, "update_gram_tc: %d blocks outside 1..%d", nblocks, kFuMaxBlocks);
    static bool attr = false;
    if (!attr) {
        BBL_CUDA(cudaFuncSetAttribute(cgs_update_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kFuSmemLimit));
        attr = true;
    }
    const int stages = fu_stages(nblocks);
    const size_t smem = fu_smem_bytes(nblocks, stages);
    int occ = 0;
    BBL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cgs_update_gram_kernel, kFuThreads, smem));
    if (occ < 1) occ = 1;
    const int64_t nchunks = ceil_div(n, (int64_t)kFuRows);
    if (nchunks > ((int64_t)1 << 30)) return set_error(BBL_ERR_UNSUPPORTED, "update_gram_tc: n too large");
    const int64_t workers = std::max<int64_t>(1, std::min<int64_t>((int64_t)gram_worker_sms() * occ, nchunks));
    const int64_t per = (int64_t)nblocks * 64;
    // [ update B fragments: tc pairs x 32 x (16 + 8) bytes | CTA slots: workers x per doubles ]
    const int ntp = fu_tc_pairs(nblocks);
    const size_t frag_bytes = (size_t)ntp * 32 * 24 + 256;
    const size_t need = frag_bytes + sizeof(double) * (size_t)(workers * per);
    BBL_TRY(work.grow(need));
    uint4* fa = reinterpret_cast<uint4*>(work.as<char>());
    uint2* fb = reinterpret_cast<uint2*>(work.as<char>() + (size_t)ntp * 32 * 16);
    double* slots = reinterpret_cast<double*>(work.as<char>() + frag_bytes);
    if (ntp > 0) {
        cgs_split_c1_kernel<<<(unsigned)ceil_div(ntp * 32, 256), 256, 0, st>>>(nblocks, C1, fa, fb);
        BBL_LAUNCH_CHECK();
    }
    cgs_update_gram_kernel<<<(unsigned)workers, kFuThreads, smem, st>>>(n, nblocks, nchunks, stages, Q, C1, fa, fb,
                                                                        W, slots);
    BBL_LAUNCH_CHECK();
    reduce_partials(per, (int)workers, slots, C2, st);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

}  // namespace bbl
