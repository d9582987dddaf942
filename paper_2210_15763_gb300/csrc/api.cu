// Error state, option defaults, the workspace cache and small ABI helpers.
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

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

// ------------------------------------------------------------------ workspace cache
namespace {
struct IdleBuf {
    void* p;
    size_t bytes;
    int dev;
    cudaEvent_t ready;  // recorded on the last stream that used it
};
std::mutex g_pool_mu;
std::vector<IdleBuf> g_idle;  // oldest first
constexpr int kPoolIdleMax = 8;

// frees the idle buffers of device dev; the caller holds g_pool_mu and has
// dev current
void free_idle_locked(int dev) {
    for (size_t i = 0; i < g_idle.size();) {
        IdleBuf& e = g_idle[i];
        if (e.dev == dev) {
            cudaEventSynchronize(e.ready);
            cudaEventDestroy(e.ready);
            cudaFree(e.p);
            g_idle.erase(g_idle.begin() + (std::ptrdiff_t)i);
        } else {
            ++i;
        }
    }
}
}  // namespace

bbl_status PoolBuf::alloc(size_t nbytes, cudaStream_t stream) {
    release();
    if (nbytes == 0) nbytes = 16;
    int d = 0;
    BBL_CUDA(cudaGetDevice(&d));
    std::lock_guard<std::mutex> lk(g_pool_mu);
    // reuse only a buffer at most 1/16 larger than the request: a much larger
    // one would strand its excess while other idle memory is counted as free
    int best = -1;
    for (size_t i = 0; i < g_idle.size(); ++i) {
        const IdleBuf& e = g_idle[i];
        if (e.dev == d && e.bytes >= nbytes && e.bytes - nbytes <= nbytes / 16 &&
            (best < 0 || e.bytes < g_idle[(size_t)best].bytes))
            best = (int)i;
    }
    if (best >= 0) {
        const IdleBuf e = g_idle[(size_t)best];
        g_idle.erase(g_idle.begin() + best);
        const cudaError_t w = cudaStreamWaitEvent(stream, e.ready, 0);
        cudaEventDestroy(e.ready);
        if (w != cudaSuccess) {
            cudaFree(e.p);
            return set_error(BBL_ERR_CUDA, "workspace: cudaStreamWaitEvent: %s", cudaGetErrorString(w));
        }
        p = e.p;
        bytes = e.bytes;
        st = stream;
        dev = d;
        return BBL_OK;
    }
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e == cudaErrorMemoryAllocation) {  // give the idle buffers back, then once more
        (void)cudaGetLastError();
        free_idle_locked(d);
        e = cudaMalloc(&p, nbytes);
    }
    if (e != cudaSuccess) {
        p = nullptr;
        (void)cudaGetLastError();
        return set_error(BBL_ERR_OOM, "cudaMalloc(%zu bytes): %s", nbytes, cudaGetErrorString(e));
    }
    bytes = nbytes;
    st = stream;
    dev = d;
    return BBL_OK;
}

void PoolBuf::release() {
    if (!p) return;
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess && cudaEventRecord(ev, st) == cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        g_idle.push_back(IdleBuf{p, bytes, dev, ev});
        int held = 0;
        for (const IdleBuf& e : g_idle) held += e.dev == dev;
        for (size_t i = 0; i < g_idle.size() && held > kPoolIdleMax;) {
            if (g_idle[i].dev == dev) {  // the oldest of this device (dev is current: it was allocated here)
                cudaEventSynchronize(g_idle[i].ready);
                cudaEventDestroy(g_idle[i].ready);
                cudaFree(g_idle[i].p);
                g_idle.erase(g_idle.begin() + (std::ptrdiff_t)i);
                --held;
            } else {
                ++i;
            }
        }
    } else {
        // reuse cannot be ordered: give it back (cudaFree waits for the device)
        if (ev) cudaEventDestroy(ev);
        (void)cudaGetLastError();
        cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
}

bool pool_free_idle_current_device() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    size_t before = g_idle.size();
    free_idle_locked(d);
    return g_idle.size() != before;
}

size_t pool_idle_bytes(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    size_t t = 0;
    for (const IdleBuf& e : g_idle)
        if (e.dev == dev) t += e.bytes;
    return t;
}

}  // namespace bbl

extern "C" {

size_t bbl_workspace_bytes(void) {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return bbl::pool_idle_bytes(d);
}

bbl_status bbl_workspace_release(void) {
    int d = 0;
    BBL_CUDA(cudaGetDevice(&d));
    std::lock_guard<std::mutex> lk(bbl::g_pool_mu);
    bbl::free_idle_locked(d);
    return BBL_OK;
}

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
    o->half_first_pass = 1;
    o->fused_update_gram = 0;
    o->narrow_old_updates = 1;
    o->stream = nullptr;
}

}  // extern "C"
