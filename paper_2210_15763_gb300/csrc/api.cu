// Error state, option defaults and small ABI helpers.
#include <atomic>
#include <cstring>

#include "common.cuh"

namespace bbl {

static thread_local std::string g_last_error;

bbl_status set_error(bbl_status s, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

void clear_error() { g_last_error.clear(); }

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

bool is_device_pointer(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace bbl

extern "C" {

const char* bbl_last_error(void) { return bbl::g_last_error.c_str(); }

const char* bbl_status_string(bbl_status s) {
    switch (s) {
        case BBL_OK: return "BBL_OK";
        case BBL_ERR_INVALID_ARG: return "BBL_ERR_INVALID_ARG";
        case BBL_ERR_NOT_SYMMETRIC: return "BBL_ERR_NOT_SYMMETRIC";
        case BBL_ERR_OOM: return "BBL_ERR_OOM";
        case BBL_ERR_CUDA: return "BBL_ERR_CUDA";
        case BBL_ERR_NOT_CONVERGED: return "BBL_ERR_NOT_CONVERGED";
        case BBL_ERR_NUMERICAL: return "BBL_ERR_NUMERICAL";
        case BBL_ERR_TIMEOUT: return "BBL_ERR_TIMEOUT";
        case BBL_ERR_UNSUPPORTED: return "BBL_ERR_UNSUPPORTED";
    }
    return "BBL_STATUS_UNKNOWN";
}

int bbl_version(void) { return 100; }

uint64_t bbl_kernel_launches(void) { return bbl::g_launches.load(); }

void bbl_options_default(bbl_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-8;
    o->max_vectors = 2000;
    o->criterion = 0;
    o->rms_tol = 1e-6;
    o->seed = 20221028ull;
    o->defl_tol = 0.0;
    o->storage = BBL_FP64;
    o->polish = 1;
    o->stage1_tol = 2e-6;
    o->check_every = 0;
    o->ritz_overlap = 1;
    o->stream = nullptr;
}

}  // extern "C"
