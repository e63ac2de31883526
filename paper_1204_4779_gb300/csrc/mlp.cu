// Cost model of the variant tuner: a 3-layer MLP (tanh, tanh, linear) with its forward pass,
// back-propagation and Adam update as hand-written FP32 CUDA kernels.
//
// The network is small (input ~30 features, width 64, a few thousand samples), so each
// kernel gives one thread one output element and loops over the reduction index in a fixed
// order: deterministic results, no atomics.  The weight gradients sum over the samples in two
// fixed-order levels: chunks of kChunk samples in parallel, then the chunk partials in order.
//
// Flat parameter layout: W1 (H x d, row-major), b1 (H), W2 (H x H), b2 (H), W3 (1 x H), b3 (1).
// Workspace for n samples (floats): h1 (n H), h2 (n H), y (n), dy (n), dz2 (n H), dz1 (n H),
// grad (P), loss (1), the Adam step counter (one int), the weight-gradient chunk partials
// (ceil(n / kChunk) x H x (max(d, H) + 1)).
//
// Training replays captured epochs: the Adam step number lives in the workspace (the loss
// kernel advances it, the Adam kernel derives its bias corrections from it), so one epoch's
// launches are the same every epoch and a CUDA graph of kEpochsPerGraph epochs is replayed.
#include <math.h>
#include <string.h>

#include "../../include/hydro.h"
#include "hydro_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 128;  // samples per partial sum of the weight gradients

constexpr int kEpochsPerGraph = 16;

struct Sizes {
    long long P, h1, h2, y, dy, dz2, dz1, grad, loss, stepc, part, total;  // float offsets / count
};

Sizes sizes(int d, int H, long long n) {
    Sizes S;
    S.P = (long long)H * d + H + (long long)H * H + H + H + 1;
    long long o = 0;
    S.h1 = o; o += n * H;
    S.h2 = o; o += n * H;
    S.y = o; o += n;
    S.dy = o; o += n;
    S.dz2 = o; o += n * H;
    S.dz1 = o; o += n * H;
    S.grad = o; o += S.P;
    S.loss = o; o += 1;
    S.stepc = o; o += 1;
    S.part = o; o += (n + kChunk - 1) / kChunk * (long long)H * ((d > H ? d : H) + 1);
    S.total = o;
    return S;
}

// out[s][j] = act(b[j] + sum_i in[s][i] W[j][i])
template <bool TANH>
__global__ void __launch_bounds__(kThreads) dense_forward(const float *in, int din, const float *W,
                                                          const float *b, int dout, long long n,
                                                          float *out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * dout) return;
    const long long s = idx / dout;
    const int j = (int)(idx % dout);
    float acc = b[j];
    for (int i = 0; i < din; ++i) acc = fmaf(in[s * din + i], W[(long long)j * din + i], acc);
    out[idx] = TANH ? tanhf(acc) : acc;
}

// dy[s] = 2 (y[s] - t[s]) / n; loss = (1/n) sum_s (y[s] - t[s])^2 (one CTA, fixed order).
// Training (stepc non-null): also record the loss in hist[*stepc - step0] and advance the Adam
// step counter *stepc, which the Adam kernel of the same epoch reads.
__global__ void __launch_bounds__(kThreads) mse_kernel(const float *y, const float *t, long long n,
                                                       float *dy, float *loss, int *stepc = nullptr,
                                                       int step0 = 0, float *hist = nullptr) {
    __shared__ float s[kThreads];
    float acc = 0.0f;
    for (long long i = threadIdx.x; i < n; i += kThreads) {
        const float e = y[i] - t[i];
        dy[i] = 2.0f * e / (float)n;
        acc = fmaf(e, e, acc);
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *loss = s[0] / (float)n;
        if (stepc) {
            if (hist) hist[*stepc - step0] = s[0] / (float)n;
            *stepc += 1;
        }
    }
}

// dz[s][i] = (sum_j delta[s][j] W[j][i]) (1 - h[s][i]^2): back through a dense layer and tanh
__global__ void __launch_bounds__(kThreads) dense_backward(const float *delta, int dout,
                                                           const float *W, const float *h, int din,
                                                           long long n, float *dz) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * din) return;
    const long long s = idx / din;
    const int i = (int)(idx % din);
    float acc = 0.0f;
    for (int j = 0; j < dout; ++j) acc = fmaf(delta[s * dout + j], W[(long long)j * din + i], acc);
    const float hv = h[idx];
    dz[idx] = acc * (1.0f - hv * hv);
}

// Chunk partials of the weight gradient: part[c][j][i] = sum over samples s of chunk c of
// delta[s][j] in[s][i] (i = din: delta[s][j] alone, the bias), s in increasing order.
__global__ void __launch_bounds__(kThreads) dense_wgrad_part(const float *delta, int dout,
                                                             const float *in, int din, long long n,
                                                             float *part) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per = (long long)dout * (din + 1);
    if (idx >= per) return;
    const int j = (int)(idx / (din + 1));
    const int i = (int)(idx % (din + 1));
    const long long s0 = (long long)blockIdx.y * kChunk;
    const long long s1 = s0 + kChunk < n ? s0 + kChunk : n;
    float acc = 0.0f;
    if (i < din) {
        for (long long s = s0; s < s1; ++s) acc = fmaf(delta[s * dout + j], in[s * din + i], acc);
    } else {
        for (long long s = s0; s < s1; ++s) acc += delta[s * dout + j];
    }
    part[blockIdx.y * per + idx] = acc;
}

// gW[j][i] = sum_c part[c][j][i] in chunk order; gb[j] = the same for i = din
__global__ void __launch_bounds__(kThreads) dense_wgrad_sum(const float *part, int dout, int din,
                                                            int nchunks, float *gW, float *gb) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per = (long long)dout * (din + 1);
    if (idx >= per) return;
    float acc = 0.0f;
    for (int c = 0; c < nchunks; ++c) acc += part[c * per + idx];
    const int j = (int)(idx / (din + 1));
    const int i = (int)(idx % (din + 1));
    if (i < din)
        gW[(long long)j * din + i] = acc;
    else
        gb[j] = acc;
}

// Adam with the step number t = *stepc read on the device (bias corrections 1 - b^t)
__global__ void __launch_bounds__(kThreads) adam_kernel_dev(float *p, float *m, float *v,
                                                            const float *g, long long count,
                                                            float lr, float b1, float b2, float eps,
                                                            const int *stepc) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float t = (float)*stepc;
    const float c1 = 1.0f - powf(b1, t), c2 = 1.0f - powf(b2, t);
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void set_step_kernel(int *stepc, int value) { *stepc = value; }

__global__ void __launch_bounds__(kThreads) adam_kernel(float *p, float *m, float *v, const float *g,
                                                        long long count, float lr, float b1,
                                                        float b2, float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

unsigned blocks(long long work) { return (unsigned)((work + kThreads - 1) / kThreads); }

// gW, gb of a dense layer (delta: n x dout, in: n x din) through the chunk partials
void dense_wgrad(const float *delta, int dout, const float *in, int din, long long n, float *part,
                 float *gW, float *gb, cudaStream_t st) {
    const int nchunks = (int)((n + kChunk - 1) / kChunk);
    const long long per = (long long)dout * (din + 1);
    dense_wgrad_part<<<dim3(blocks(per), (unsigned)nchunks), kThreads, 0, st>>>(delta, dout, in,
                                                                                din, n, part);
    dense_wgrad_sum<<<blocks(per), kThreads, 0, st>>>(part, dout, din, nchunks, gW, gb);
}

cudaError_t forward_all(const float *p, int d, int H, const float *X, long long n, float *ws,
                        const Sizes &S, cudaStream_t st) {
    const float *W1 = p, *b1 = W1 + (long long)H * d, *W2 = b1 + H, *b2 = W2 + (long long)H * H;
    const float *W3 = b2 + H, *b3 = W3 + H;
    dense_forward<true><<<blocks(n * H), kThreads, 0, st>>>(X, d, W1, b1, H, n, ws + S.h1);
    dense_forward<true><<<blocks(n * H), kThreads, 0, st>>>(ws + S.h1, H, W2, b2, H, n, ws + S.h2);
    dense_forward<false><<<blocks(n), kThreads, 0, st>>>(ws + S.h2, H, W3, b3, 1, n, ws + S.y);
    return cudaGetLastError();
}

// Forward, loss and back-propagation into ws + S.grad.  Training: stepc/step0/hist as in
// mse_kernel.
cudaError_t gradient_all(const float *p, int d, int H, const float *X, const float *t, long long n,
                         float *ws, const Sizes &S, cudaStream_t st, int *stepc = nullptr,
                         int step0 = 0, float *hist = nullptr) {
    cudaError_t e = forward_all(p, d, H, X, n, ws, S, st);
    if (e != cudaSuccess) return e;
    const float *W2 = p + (long long)H * d + H, *W3 = W2 + (long long)H * H + H;
    float *g = ws + S.grad;
    float *gW1 = g, *gb1 = gW1 + (long long)H * d, *gW2 = gb1 + H, *gb2 = gW2 + (long long)H * H;
    float *gW3 = gb2 + H, *gb3 = gW3 + H;
    mse_kernel<<<1, kThreads, 0, st>>>(ws + S.y, t, n, ws + S.dy, ws + S.loss, stepc, step0, hist);
    // output layer (linear): delta = dy
    float *part = ws + S.part;
    dense_wgrad(ws + S.dy, 1, ws + S.h2, H, n, part, gW3, gb3, st);
    dense_backward<<<blocks(n * H), kThreads, 0, st>>>(ws + S.dy, 1, W3, ws + S.h2, H, n, ws + S.dz2);
    dense_wgrad(ws + S.dz2, H, ws + S.h1, H, n, part, gW2, gb2, st);
    dense_backward<<<blocks(n * H), kThreads, 0, st>>>(ws + S.dz2, H, W2, ws + S.h1, H, n, ws + S.dz1);
    dense_wgrad(ws + S.dz1, H, X, d, n, part, gW1, gb1, st);
    return cudaGetLastError();
}

bool dims_ok(int d, int H, long long n) {
    return d >= 1 && d <= 4096 && H >= 1 && H <= 4096 && n >= 1 && n <= 65535LL * kChunk;
}

}  // namespace

extern "C" {

int hydro_mlp_sizes(int32_t d, int32_t hidden, int64_t n, int64_t *param_count,
                    size_t *workspace_bytes) {
    if (!dims_ok(d, hidden, n)) return HYDRO_EINVAL;
    const Sizes S = sizes(d, hidden, n);
    if (param_count) *param_count = S.P;
    if (workspace_bytes) *workspace_bytes = sizeof(float) * (size_t)S.total;
    return HYDRO_OK;
}

int hydro_mlp_forward(const float *params, int32_t d, int32_t hidden, const float *X, int64_t n,
                      float *y_out, void *workspace, void *stream) {
    if (!params || !X || !y_out || !workspace || !dims_ok(d, hidden, n)) return HYDRO_EINVAL;
    const Sizes S = sizes(d, hidden, n);
    float *ws = static_cast<float *>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = forward_all(params, d, hidden, X, n, ws, S, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(y_out, ws + S.y, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? HYDRO_OK : hydro::record_cuda_error(e, "hydro_mlp_forward");
}

int hydro_mlp_gradient(const float *params, int32_t d, int32_t hidden, const float *X,
                       const float *t, int64_t n, void *workspace, float *grad_out,
                       float *loss_out, void *stream) {
    if (!params || !X || !t || !workspace || !dims_ok(d, hidden, n)) return HYDRO_EINVAL;
    const Sizes S = sizes(d, hidden, n);
    float *ws = static_cast<float *>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = gradient_all(params, d, hidden, X, t, n, ws, S, st);
    if (e == cudaSuccess && grad_out)
        e = cudaMemcpyAsync(grad_out, ws + S.grad, sizeof(float) * (size_t)S.P,
                            cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && loss_out)
        e = cudaMemcpyAsync(loss_out, ws + S.loss, sizeof(float), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? HYDRO_OK : hydro::record_cuda_error(e, "hydro_mlp_gradient");
}

int hydro_mlp_adam(float *params, float *m, float *v, const float *grad, int64_t count,
                   int32_t step, float lr, float beta1, float beta2, float eps, void *stream) {
    if (!params || !m || !v || !grad || count < 1 || step < 1) return HYDRO_EINVAL;
    const float c1 = 1.0f - powf(beta1, (float)step);
    const float c2 = 1.0f - powf(beta2, (float)step);
    adam_kernel<<<blocks(count), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        params, m, v, grad, count, lr, beta1, beta2, eps, c1, c2);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HYDRO_OK : hydro::record_cuda_error(e, "hydro_mlp_adam");
}

int hydro_mlp_train(float *params, float *m, float *v, int32_t d, int32_t hidden, const float *X,
                    const float *t, int64_t n, int32_t epochs, int32_t step0, float lr,
                    void *workspace, float *loss_out, void *stream) {
    if (!params || !m || !v || !X || !t || !workspace || epochs < 0 || step0 < 0 ||
        !dims_ok(d, hidden, n))
        return HYDRO_EINVAL;
    const Sizes S = sizes(d, hidden, n);
    float *ws = static_cast<float *>(workspace);
    int *stepc = reinterpret_cast<int *>(ws + S.stepc);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // one epoch: forward, loss (advances the step counter), back-propagation, Adam
    auto epoch = [&](cudaStream_t s) -> cudaError_t {
        cudaError_t e = gradient_all(params, d, hidden, X, t, n, ws, S, s, stepc, step0, loss_out);
        if (e != cudaSuccess) return e;
        adam_kernel_dev<<<blocks(S.P), kThreads, 0, s>>>(params, m, v, ws + S.grad, S.P, lr, 0.9f,
                                                         0.999f, 1e-8f, stepc);
        return cudaGetLastError();
    };
    set_step_kernel<<<1, 1, 0, st>>>(stepc, step0);
    cudaError_t e = cudaGetLastError();
    const int per = epochs < kEpochsPerGraph ? epochs : kEpochsPerGraph;
    const int reps = per > 0 ? epochs / per : 0;
    if (e == cudaSuccess && reps > 1) {
        // capture `per` epochs on a private stream and replay them on the caller's
        cudaStream_t cap = nullptr;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t ec = cudaSuccess;
            for (int k = 0; k < per && ec == cudaSuccess; ++k) ec = epoch(cap);
            e = cudaStreamEndCapture(cap, &g);
            if (e == cudaSuccess) e = ec;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(x, st);
        if (x) cudaGraphExecDestroy(x);
        if (g) cudaGraphDestroy(g);
        if (cap) cudaStreamDestroy(cap);
        for (int k = reps * per; k < epochs && e == cudaSuccess; ++k) e = epoch(st);
    } else {
        for (int k = 0; k < epochs && e == cudaSuccess; ++k) e = epoch(st);
    }
    return e == cudaSuccess ? HYDRO_OK : hydro::record_cuda_error(e, "hydro_mlp_train");
}

}  // extern "C"
