// Arithmetic-rate probe (no counterpart in the paper): the FP32 and FP64
// fused multiply-add throughput of this GPU, measured with CUDA events.  The
// solver's precision choices rest on the ratio (the mixed-precision form
// keeps its long products on the FP32 pipes and uses float-float pairs
// rather than FP64 for the polish).
#include "common.cuh"

namespace bbl {
namespace {

constexpr int kChains = 8;

// kChains independent FMA chains per thread, `iters` steps each; the sum is
// stored so that nothing is optimised away.
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, T a, T c, T* __restrict__ out) {
    T x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = (T)(threadIdx.x + j);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
bbl_status probe(double* flops, cudaStream_t st) {
    int dev = 0, sms = 0;
    BBL_CUDA(cudaGetDevice(&dev));
    BBL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * 8, threads = 256;
    const int iters = sizeof(T) == 8 ? 2048 : 65536;
    DevBuf out;
    BBL_TRY(out.alloc(sizeof(T) * (size_t)grid * threads));
    cudaEvent_t e0, e1;
    BBL_CUDA(cudaEventCreate(&e0));
    BBL_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    bbl_status s = BBL_OK;
    for (int rep = 0; rep < 4 && s == BBL_OK; ++rep) {  // the first launch warms up
        cudaEventRecord(e0, st);
        fma_probe_kernel<T><<<grid, threads, 0, st>>>(iters, (T)0.999999, (T)1e-7, out.as<T>());
        count_launch();
        cudaEventRecord(e1, st);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            s = set_error(BBL_ERR_CUDA, "probe_fma_rate: launch failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = ms < best ? ms : best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != BBL_OK) return s;
    *flops = 2.0 * kChains * (double)iters * grid * threads / (best * 1e-3);
    return BBL_OK;
}

}  // namespace
}  // namespace bbl

extern "C" bbl_status bbl_probe_fma_rate(bbl_dtype dtype, double* flops_per_s, void* stream) {
    using namespace bbl;
    if (!flops_per_s || (dtype != BBL_FP32 && dtype != BBL_FP64))
        return set_error(BBL_ERR_INVALID_ARG, "probe_fma_rate: bad arguments");
    if (dtype == BBL_FP64) return probe<double>(flops_per_s, as_stream(stream));
    return probe<float>(flops_per_s, as_stream(stream));
}
