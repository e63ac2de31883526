// Device diagnostic with no counterpart in the paper: the measured fused multiply-add
// throughput of the current GPU, the denominator of the benchmark's FP32 roofline (and the
// FP64 rate that bounds the FP64 path).
//
// Every thread runs eight independent FMA chains x <- x a + b (a just below one, so the
// chains stay finite and normal); enough resident warps per SM hide the FMA latency, and the
// inner loop is unrolled so loop control is a small share of the issued instructions.  The
// result is written only under a condition the data never meets, so the chains stay live
// without memory traffic.
#include <cuda_runtime.h>

#include "../../include/hydro.h"
#include "hydro_internal.h"

namespace {

constexpr int kFmaThreads = 256;
constexpr int kChains = 8;

template <class T>
__global__ void __launch_bounds__(kFmaThreads) fma_chains_kernel(T a, T b, int iters, T *sink) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
#pragma unroll 1
    for (int i = 0; i < iters; i += 16) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == T(-1)) *sink = s;  // never true for these chains (all values stay positive)
}

template <class T>
int fma_rate_t(cudaStream_t st, int iters, double *out) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chains_kernel<T>,
                                                          kFmaThreads, 0);
    T *sink = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&sink), sizeof(T), st);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const unsigned blocks = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
    const T a = T(0.9999), b = T(1e-4);
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            fma_chains_kernel<T><<<blocks, kFmaThreads, 0, st>>>(a, b, iters, sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (sink) {
        const cudaError_t f = cudaFreeAsync(sink, st);
        if (e == cudaSuccess) e = f;
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return hydro::record_cuda_error(e, "hydro_fma_rate");
    const double ops = (double)blocks * kFmaThreads * kChains * (double)iters;
    *out = best > 0.f ? ops / (best * 1e-3) : 0.0;
    return HYDRO_OK;
}

}  // namespace

extern "C" int hydro_fma_rate(int32_t prec, void *stream, double *ops_per_s_out) {
    if (!ops_per_s_out) return HYDRO_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // about 4 ms per timed launch at the expected rates (FP64 runs far fewer FMAs per second)
    if (prec == HYDRO_F32) return fma_rate_t<float>(st, 1 << 16, ops_per_s_out);
    if (prec == HYDRO_F64) return fma_rate_t<double>(st, 1 << 11, ops_per_s_out);
    return HYDRO_EINVAL;
}
