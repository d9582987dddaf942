// Learned pivot: a small MLP g -> coefficients on a stored basis U of
// converged eigenvectors, trained on this library's own solves.  The paper
// has no learned component; this is the proposal step in front of the
// bootstrapped pivot, which stays the fallback.
//
//   h1 = gelu(W1 g + b1)   1 -> H     (gelu(x) = x/2 (1 + erf(x/sqrt 2)))
//   h2 = gelu(W2 h1 + b2)  H -> H
//   y  = W3 h2 + b3        H -> O  (O = nbasis * b, reshaped nbasis x b)
//
// Weights are used in BF16 (round-to-nearest-even copies of FP32 master
// weights), activations and accumulation are FP32.  Loss: mean squared error.
// Optimiser: Adam (Kingma & Ba 2015) on the FP32 masters.  One training epoch
// (forward, loss, backward, Adam) is captured once in a CUDA graph and
// replayed.  The pivot P = U C(g) reuses the Ritz-vector kernel.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

struct bbl_mlp {
    int hidden = 0, out = 0, nparams = 0;
    int cap_batch = 0;
    bbl::DevBuf params, grads, m, v, wbf, act, tstep, lossbuf;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_batch = -1;
    const void* graph_g = nullptr;
    const void* graph_t = nullptr;
    float graph_lr = 0.f;
    ~bbl_mlp() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
    // packed offsets (FP32 params): W1[H], b1[H], W2[H*H], b2[H], W3[O*H], b3[O]
    int oW1() const { return 0; }
    int ob1() const { return hidden; }
    int oW2() const { return 2 * hidden; }
    int ob2() const { return 2 * hidden + hidden * hidden; }
    int oW3() const { return 3 * hidden + hidden * hidden; }
    int ob3() const { return 3 * hidden + hidden * hidden + out * hidden; }
};

namespace bbl {
namespace {

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}
__device__ __forceinline__ float bf(const __nv_bfloat16* w, int i) { return __bfloat162float(w[i]); }

// activations layout per sample: z1[H] h1[H] z2[H] h2[H] dz1[H] dz2[H] y[O] dy[O]
__global__ void forward_kernel(int H, int O, const float* __restrict__ P, const __nv_bfloat16* __restrict__ Wb,
                               const float* __restrict__ g, float* __restrict__ act, float* __restrict__ y_out) {
    extern __shared__ float sh[];
    float* h1 = sh;
    float* h2 = sh + H;
    const int s = blockIdx.x;
    const float x = g[s];
    float* a = act + (size_t)s * (6 * H + 2 * O);
    const __nv_bfloat16* W1 = Wb;
    const __nv_bfloat16* W2 = Wb + H;
    const __nv_bfloat16* W3 = Wb + H + H * H;
    const float* b1 = P + H;
    const float* b2 = P + 2 * H + H * H;
    const float* b3 = P + 3 * H + H * H + O * H;
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        const float z = fmaf(bf(W1, i), x, b1[i]);
        a[i] = z;
        const float hv = gelu(z);
        a[H + i] = hv;
        h1[i] = hv;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < H; o += blockDim.x) {
        float acc = b2[o];
        for (int i = 0; i < H; ++i) acc = fmaf(bf(W2, o * H + i), h1[i], acc);
        a[2 * H + o] = acc;
        const float hv = gelu(acc);
        a[3 * H + o] = hv;
        h2[o] = hv;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < O; o += blockDim.x) {
        float acc = b3[o];
        for (int i = 0; i < H; ++i) acc = fmaf(bf(W3, o * H + i), h2[i], acc);
        a[6 * H + o] = acc;
        if (y_out) y_out[(size_t)s * O + o] = acc;
    }
}

// dy = 2 (y - t) / N and per-sample partial losses
__global__ void loss_kernel(int batch, int H, int O, const float* __restrict__ target, float* __restrict__ act,
                            float* __restrict__ lossp) {
    __shared__ float red[256];
    const int s = blockIdx.x;
    float* a = act + (size_t)s * (6 * H + 2 * O);
    const float invN = 1.0f / ((float)batch * (float)O);
    float l = 0.f;
    for (int o = threadIdx.x; o < O; o += blockDim.x) {
        const float d = a[6 * H + o] - target[(size_t)s * O + o];
        l = fmaf(d, d, l);
        a[6 * H + O + o] = 2.0f * d * invN;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) lossp[s] = red[0] * invN;
}

// per-sample backward through the activations: dz2, dz1
__global__ void backward_act_kernel(int H, int O, const __nv_bfloat16* __restrict__ Wb, float* __restrict__ act) {
    extern __shared__ float sh[];
    float* dz2s = sh;
    const int s = blockIdx.x;
    float* a = act + (size_t)s * (6 * H + 2 * O);
    const __nv_bfloat16* W2 = Wb + H;
    const __nv_bfloat16* W3 = Wb + H + H * H;
    const float* dy = a + 6 * H + O;
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        float acc = 0.f;
        for (int o = 0; o < O; ++o) acc = fmaf(bf(W3, o * H + i), dy[o], acc);
        const float d = acc * gelu_grad(a[2 * H + i]);
        a[5 * H + i] = d;
        dz2s[i] = d;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        float acc = 0.f;
        for (int o = 0; o < H; ++o) acc = fmaf(bf(W2, o * H + i), dz2s[o], acc);
        a[4 * H + i] = acc * gelu_grad(a[i]);
    }
}

// weight gradients, one thread per parameter, summed over the batch in order
__global__ void backward_w_kernel(int batch, int H, int O, const float* __restrict__ g, const float* __restrict__ act,
                                  float* __restrict__ G) {
    const int np = 3 * H + H * H + O * H + O;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const size_t st = 6 * H + 2 * O;
    float acc = 0.f;
    if (p < H) {  // W1[o]
        for (int s = 0; s < batch; ++s) acc = fmaf(act[s * st + 4 * H + p], g[s], acc);
    } else if (p < 2 * H) {  // b1
        const int o = p - H;
        for (int s = 0; s < batch; ++s) acc += act[s * st + 4 * H + o];
    } else if (p < 2 * H + H * H) {  // W2[o][i]
        const int e = p - 2 * H, o = e / H, i = e % H;
        for (int s = 0; s < batch; ++s) acc = fmaf(act[s * st + 5 * H + o], act[s * st + H + i], acc);
    } else if (p < 3 * H + H * H) {  // b2
        const int o = p - 2 * H - H * H;
        for (int s = 0; s < batch; ++s) acc += act[s * st + 5 * H + o];
    } else if (p < 3 * H + H * H + O * H) {  // W3[o][i]
        const int e = p - 3 * H - H * H, o = e / H, i = e % H;
        for (int s = 0; s < batch; ++s) acc = fmaf(act[s * st + 6 * H + O + o], act[s * st + 3 * H + i], acc);
    } else {  // b3
        const int o = p - 3 * H - H * H - O * H;
        for (int s = 0; s < batch; ++s) acc += act[s * st + 6 * H + O + o];
    }
    G[p] = acc;
}

// bf16 copies of the weight matrices (W1 | W2 | W3)
__global__ void to_bf16_kernel(int H, int O, const float* __restrict__ P, __nv_bfloat16* __restrict__ Wb) {
    const int nw = H + H * H + O * H;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nw; e += gridDim.x * blockDim.x) {
        int src;
        if (e < H) src = e;                                   // W1
        else if (e < H + H * H) src = 2 * H + (e - H);        // W2
        else src = 3 * H + H * H + (e - H - H * H);           // W3
        Wb[e] = __float2bfloat16_rn(P[src]);
    }
}

__global__ void adam_kernel(int np, float lr, float b1, float b2, float eps, float* __restrict__ P,
                            const float* __restrict__ G, float* __restrict__ M, float* __restrict__ V,
                            int* __restrict__ tstep) {
    const int t = *tstep + 1;  // read before the increment below (one block writes it after a grid-wide pass)
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        const float gr = G[p];
        const float m = b1 * M[p] + (1.0f - b1) * gr;
        const float v = b2 * V[p] + (1.0f - b2) * gr * gr;
        M[p] = m;
        V[p] = v;
        P[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

__global__ void step_inc_kernel(int* tstep) { *tstep += 1; }

__global__ void sum_loss_kernel(int batch, const float* __restrict__ lossp, float* __restrict__ out, int slot) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.f;
        for (int i = 0; i < batch; ++i) s += lossp[i];
        out[slot] = s;
    }
}

__global__ void widen_kernel(int count, const float* __restrict__ y, double* __restrict__ C) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count) C[e] = (double)y[e];
}

bbl_status ensure_batch(bbl_mlp* M, int batch) {
    if (batch <= M->cap_batch) return BBL_OK;
    BBL_TRY(M->act.alloc(sizeof(float) * (size_t)batch * (6 * M->hidden + 2 * M->out)));
    BBL_TRY(M->lossbuf.alloc(sizeof(float) * (size_t)(batch + 8)));
    M->cap_batch = batch;
    if (M->exec) {
        cudaGraphExecDestroy(M->exec);
        cudaGraphDestroy(M->graph);
        M->exec = nullptr;
        M->graph = nullptr;
        M->graph_batch = -1;
    }
    return BBL_OK;
}

bbl_status launch_forward(const bbl_mlp* M, int batch, const float* g, float* y, cudaStream_t st) {
    forward_kernel<<<batch, 256, sizeof(float) * 2 * M->hidden, st>>>(
        M->hidden, M->out, M->params.as<float>(), M->wbf.as<__nv_bfloat16>(), g, M->act.as<float>(), y);
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

bbl_status launch_loss_backward(bbl_mlp* M, int batch, const float* g, const float* target, cudaStream_t st) {
    loss_kernel<<<batch, 256, 0, st>>>(batch, M->hidden, M->out, target, M->act.as<float>(), M->lossbuf.as<float>());
    BBL_LAUNCH_CHECK();
    backward_act_kernel<<<batch, 128, sizeof(float) * M->hidden, st>>>(M->hidden, M->out, M->wbf.as<__nv_bfloat16>(),
                                                                       M->act.as<float>());
    BBL_LAUNCH_CHECK();
    backward_w_kernel<<<(unsigned)ceil_div(M->nparams, 256), 256, 0, st>>>(batch, M->hidden, M->out, g,
                                                                          M->act.as<float>(), M->grads.as<float>());
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

bbl_status launch_adam(bbl_mlp* M, float lr, cudaStream_t st) {
    adam_kernel<<<(unsigned)ceil_div(M->nparams, 256), 256, 0, st>>>(M->nparams, lr, 0.9f, 0.999f, 1e-8f,
                                                                     M->params.as<float>(), M->grads.as<float>(),
                                                                     M->m.as<float>(), M->v.as<float>(),
                                                                     M->tstep.as<int>());
    BBL_LAUNCH_CHECK();
    step_inc_kernel<<<1, 1, 0, st>>>(M->tstep.as<int>());
    BBL_LAUNCH_CHECK();
    to_bf16_kernel<<<64, 256, 0, st>>>(M->hidden, M->out, M->params.as<float>(), M->wbf.as<__nv_bfloat16>());
    BBL_LAUNCH_CHECK();
    return BBL_OK;
}

}  // namespace
bbl_status ritz_vectors(int64_t n, int b, int nblocks, int dtype, const void* Q, int k, const double* S, double* X,
                        cudaStream_t st);
}  // namespace bbl

extern "C" {

bbl_status bbl_mlp_create(int hidden, int out_dim, bbl_mlp** out) {
    using namespace bbl;
    if (!out || hidden < 1 || hidden > 1024 || out_dim < 1 || out_dim > 4096)
        return set_error(BBL_ERR_INVALID_ARG, "mlp_create: bad arguments");
    bbl_mlp* M = new bbl_mlp();
    M->hidden = hidden;
    M->out = out_dim;
    M->nparams = 3 * hidden + hidden * hidden + out_dim * hidden + out_dim;
    const size_t pb = sizeof(float) * M->nparams;
    bbl_status s;
    if ((s = M->params.alloc(pb)) != BBL_OK || (s = M->grads.alloc(pb)) != BBL_OK || (s = M->m.alloc(pb)) != BBL_OK ||
        (s = M->v.alloc(pb)) != BBL_OK || (s = M->tstep.alloc(sizeof(int))) != BBL_OK ||
        (s = M->wbf.alloc(sizeof(__nv_bfloat16) * (hidden + hidden * hidden + out_dim * hidden))) != BBL_OK) {
        delete M;
        return s;
    }
    cudaMemset(M->params.p, 0, pb);
    cudaMemset(M->m.p, 0, pb);
    cudaMemset(M->v.p, 0, pb);
    cudaMemset(M->tstep.p, 0, sizeof(int));
    cudaMemset(M->wbf.p, 0, M->wbf.bytes);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        delete M;
        return set_error(BBL_ERR_CUDA, "mlp_create: initialisation failed");
    }
    *out = M;
    return BBL_OK;
}

void bbl_mlp_destroy(bbl_mlp* M) {
    if (M) {
        cudaDeviceSynchronize();
        delete M;
    }
}

int bbl_mlp_num_params(const bbl_mlp* M) { return M ? M->nparams : 0; }

bbl_status bbl_mlp_set_params(bbl_mlp* M, const float* packed, void* stream) {
    using namespace bbl;
    if (!M || !packed) return set_error(BBL_ERR_INVALID_ARG, "mlp_set_params: NULL argument");
    cudaStream_t st = as_stream(stream);
    BBL_CUDA(cudaMemcpyAsync(M->params.p, packed, sizeof(float) * M->nparams, cudaMemcpyDefault, st));
    BBL_CUDA(cudaMemsetAsync(M->m.p, 0, M->m.bytes, st));
    BBL_CUDA(cudaMemsetAsync(M->v.p, 0, M->v.bytes, st));
    BBL_CUDA(cudaMemsetAsync(M->tstep.p, 0, sizeof(int), st));
    to_bf16_kernel<<<64, 256, 0, st>>>(M->hidden, M->out, M->params.as<float>(), M->wbf.as<__nv_bfloat16>());
    BBL_LAUNCH_CHECK();
    BBL_CUDA(cudaStreamSynchronize(st));
    return BBL_OK;
}

bbl_status bbl_mlp_get_params(const bbl_mlp* M, float* packed, float* grads, void* stream) {
    using namespace bbl;
    if (!M) return set_error(BBL_ERR_INVALID_ARG, "mlp_get_params: NULL model");
    cudaStream_t st = as_stream(stream);
    if (packed) BBL_CUDA(cudaMemcpyAsync(packed, M->params.p, sizeof(float) * M->nparams, cudaMemcpyDefault, st));
    if (grads) BBL_CUDA(cudaMemcpyAsync(grads, M->grads.p, sizeof(float) * M->nparams, cudaMemcpyDefault, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    return BBL_OK;
}

bbl_status bbl_mlp_forward(bbl_mlp* M, int batch, const float* g, float* y, void* stream) {
    using namespace bbl;
    if (!M || !g || !y || batch < 1) return set_error(BBL_ERR_INVALID_ARG, "mlp_forward: bad arguments");
    BBL_TRY(ensure_batch(M, batch));
    cudaStream_t st = as_stream(stream);
    BBL_TRY(launch_forward(M, batch, g, y, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    return BBL_OK;
}

bbl_status bbl_mlp_loss_grad(bbl_mlp* M, int batch, const float* g, const float* target, float* loss, void* stream) {
    using namespace bbl;
    if (!M || !g || !target || batch < 1) return set_error(BBL_ERR_INVALID_ARG, "mlp_loss_grad: bad arguments");
    BBL_TRY(ensure_batch(M, batch));
    cudaStream_t st = as_stream(stream);
    BBL_TRY(launch_forward(M, batch, g, nullptr, st));
    BBL_TRY(launch_loss_backward(M, batch, g, target, st));
    float* lp = M->lossbuf.as<float>();
    sum_loss_kernel<<<1, 32, 0, st>>>(batch, lp, lp, batch);
    BBL_LAUNCH_CHECK();
    float h = 0.f;
    BBL_CUDA(cudaMemcpyAsync(&h, lp + batch, sizeof(float), cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    if (loss) *loss = h;
    return BBL_OK;
}

bbl_status bbl_mlp_adam_step(bbl_mlp* M, float lr, void* stream) {
    using namespace bbl;
    if (!M || !(lr > 0)) return set_error(BBL_ERR_INVALID_ARG, "mlp_adam_step: bad arguments");
    cudaStream_t st = as_stream(stream);
    BBL_TRY(launch_adam(M, lr, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    return BBL_OK;
}

bbl_status bbl_mlp_train(bbl_mlp* M, int batch, const float* g, const float* target, int epochs, float lr,
                         float* loss_hist, void* stream) {
    using namespace bbl;
    if (!M || !g || !target || batch < 1 || epochs < 0 || !(lr > 0))
        return set_error(BBL_ERR_INVALID_ARG, "mlp_train: bad arguments");
    BBL_TRY(ensure_batch(M, batch));
    cudaStream_t st = as_stream(stream);
    cudaStream_t cap = nullptr;
    if (!st) {  // graphs cannot be captured on the legacy stream
        BBL_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        st = cap;
    }
    if (!M->exec || M->graph_batch != batch || M->graph_g != g || M->graph_t != target || M->graph_lr != lr) {
        if (M->exec) {
            cudaGraphExecDestroy(M->exec);
            cudaGraphDestroy(M->graph);
            M->exec = nullptr;
            M->graph = nullptr;
        }
        BBL_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        bbl_status s = launch_forward(M, batch, g, nullptr, st);
        if (s == BBL_OK) s = launch_loss_backward(M, batch, g, target, st);
        if (s == BBL_OK) s = launch_adam(M, lr, st);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (s != BBL_OK) return s;
        if (e != cudaSuccess) return set_error(BBL_ERR_CUDA, "mlp_train: capture failed: %s", cudaGetErrorString(e));
        M->graph = graph;
        BBL_CUDA(cudaGraphInstantiate(&M->exec, graph, 0));
        M->graph_batch = batch;
        M->graph_g = g;
        M->graph_t = target;
        M->graph_lr = lr;
    }
    std::vector<float> hist;
    DevBuf lh;
    if (loss_hist) BBL_TRY(lh.alloc(sizeof(float) * (epochs + 1)));
    for (int e = 0; e < epochs; ++e) {
        BBL_CUDA(cudaGraphLaunch(M->exec, st));
        count_launch();
        if (loss_hist) {
            sum_loss_kernel<<<1, 32, 0, st>>>(batch, M->lossbuf.as<float>(), lh.as<float>(), e);
            BBL_LAUNCH_CHECK();
        }
    }
    if (loss_hist && epochs > 0)
        BBL_CUDA(cudaMemcpyAsync(loss_hist, lh.p, sizeof(float) * epochs, cudaMemcpyDeviceToHost, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    if (cap) cudaStreamDestroy(cap);
    return BBL_OK;
}

bbl_status bbl_pivot_learned(bbl_mlp* M, float g, int64_t n, int b_U, int nblocks_U, const float* U, int b, double* P,
                             void* stream) {
    using namespace bbl;
    if (!M || !U || !P || n < 1 || b_U < 1 || b_U > kMaxB || nblocks_U < 1 || b < 1 || b > kMaxB ||
        (int64_t)nblocks_U * b_U * b != M->out)
        return set_error(BBL_ERR_INVALID_ARG, "pivot_learned: shapes do not match the network output");
    cudaStream_t st = as_stream(stream);
    BBL_TRY(ensure_batch(M, 1));
    DevBuf gb, y, C;
    BBL_TRY(gb.alloc(sizeof(float)));
    BBL_TRY(y.alloc(sizeof(float) * M->out));
    BBL_TRY(C.alloc(sizeof(double) * M->out));
    BBL_CUDA(cudaMemcpyAsync(gb.p, &g, sizeof(float), cudaMemcpyHostToDevice, st));
    BBL_TRY(launch_forward(M, 1, gb.as<float>(), y.as<float>(), st));
    widen_kernel<<<(unsigned)ceil_div(M->out, 256), 256, 0, st>>>(M->out, y.as<float>(), C.as<double>());
    BBL_LAUNCH_CHECK();
    BBL_TRY(ritz_vectors(n, b_U, nblocks_U, BBL_FP32, U, b, C.as<double>(), P, st));
    BBL_CUDA(cudaStreamSynchronize(st));
    return BBL_OK;
}

}  // extern "C"
