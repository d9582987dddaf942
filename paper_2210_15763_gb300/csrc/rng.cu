// Counter-based random numbers: splitmix64 (Steele, Lea & Flood, OOPSLA 2014)
// evaluated as mix(seed + (counter + 1) * 0x9E3779B97F4A7C15).
//   uniform01(c) = ((mix >> 11) + 1) * 2^-53      in (0, 1]
//   normal(k)    = sqrt(-2 ln u(2k)) cos(2 pi u(2k+1))   (Box-Muller)
// Used for random pivots (Sec. III "randomly constructed pivot") and for the
// replacement directions of deflated columns.
#include "common.cuh"
#include "df32.cuh"

namespace bbl {
namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t counter) {
    uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t counter) {
    return ((double)(splitmix64(seed, counter) >> 11) + 1.0) * 0x1.0p-53;
}

__global__ void normal_kernel(int64_t count, uint64_t seed, uint64_t offset, double* __restrict__ P) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = offset + (uint64_t)e;
        const double u1 = uniform01(seed, 2ull * k);
        const double u2 = uniform01(seed, 2ull * k + 1ull);
        P[e] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    }
}

// Column c of Z (n x b row-major) is set to uniform(-1,1) where mask[c] != 0,
// to 0 elsewhere.  Element (i, c) uses counter offset + c * n + i.
template <typename T>
__global__ void uniform_cols_kernel(int64_t n, int b, uint64_t seed, uint64_t offset, const int* __restrict__ mask,
                                    T* __restrict__ Z) {
    const int64_t count = n * b;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / b;
        const int c = (int)(e % b);
        T v = T(0);
        if (mask[c]) v = (T)(2.0 * uniform01(seed, offset + (uint64_t)c * (uint64_t)n + (uint64_t)i) - 1.0);
        Z[e] = v;
    }
}

}  // namespace

bbl_status fill_normal(int64_t n, int b, uint64_t seed, uint64_t offset, double* P, cudaStream_t st) {
    normal_kernel<<<152 * 8, 256, 0, st>>>(n * b, seed, offset, P);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

bbl_status fill_uniform_cols(int64_t n, int b, int dtype, uint64_t seed, uint64_t offset, const int* mask, void* Z,
                             cudaStream_t st) {
    if (dtype == BBL_FP64)
        uniform_cols_kernel<double><<<152 * 8, 256, 0, st>>>(n, b, seed, offset, mask, static_cast<double*>(Z));
    else if (dtype == kDF32)
        uniform_cols_kernel<df32><<<152 * 8, 256, 0, st>>>(n, b, seed, offset, mask, static_cast<df32*>(Z));
    else
        uniform_cols_kernel<float><<<152 * 8, 256, 0, st>>>(n, b, seed, offset, mask, static_cast<float*>(Z));
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

}  // namespace bbl

extern "C" bbl_status bbl_pivot_random(int64_t n, int b, uint64_t seed, double* P, void* stream) {
    using namespace bbl;
    if (n < 1 || b < 1 || b > kMaxB || !P) return set_error(BBL_ERR_INVALID_ARG, "pivot_random: bad arguments");
    BBL_TRY(fill_normal(n, b, seed, 0, P, as_stream(stream)));
    return BBL_OK;
}
