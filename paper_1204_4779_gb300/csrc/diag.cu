// Device diagnostics with no counterpart in the paper: the measured fused multiply-add
// throughput of the current GPU, the denominator of the benchmark's FP32 roofline (and the
// FP64 rate that bounds the FP64 path); and a check that the bounded mbarrier wait of the
// TMA-staged stage kernels gives up on a phase that never completes.
//
// Every thread runs eight independent FMA chains x <- x a + b (a just below one, so the
// chains stay finite and normal); enough resident warps per SM hide the FMA latency, and the
// inner loop is unrolled so loop control is a small share of the issued instructions.  The
// result is written only under a condition the data never meets, so the chains stay live
// without memory traffic.
#include <cuda_runtime.h>

#include "../../include/hydro.h"
#include "hydro_internal.h"
#include "tma.cuh"

namespace {

// The bounded mbarrier wait of the TMA-staged stage kernels, on a phase that never completes:
// one mbarrier expecting one arrival that nobody makes; every thread waits on it and counts
// itself in *gave_up when the wait gives up.
__device__ unsigned int g_no_abort = 0u;  // abort bits that are never set

__global__ void wait_bound_kernel(int *gave_up) {
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = hydro::smem_u32(&bar);
    if (threadIdx.x == 0) {
        hydro::mbar_init(b, 1);
        hydro::mbar_init_fence();
    }
    __syncthreads();
    if (!hydro::mbar_wait(b, 0, &g_no_abort)) atomicAdd(gave_up, 1);
}

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

extern "C" int hydro_wait_bound_check(int32_t *gave_up_device, void *stream, int32_t *gave_up_out,
                                      double *elapsed_ms_out) {
    if (!gave_up_device || !gave_up_out) return HYDRO_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemsetAsync(gave_up_device, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        wait_bound_kernel<<<1, 32, 0, st>>>(gave_up_device);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(gave_up_out, gave_up_device, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return hydro::record_cuda_error(e, "hydro_wait_bound_check");
    if (elapsed_ms_out) *elapsed_ms_out = ms;
    return HYDRO_OK;
}
