// Plane staging by the Tensor Memory Accelerator (TMA) for the 3D marching stage kernel.
//
// One bulk tensor copy per field (cp.async.bulk.tensor.3d) moves a box of a z-plane of the
// stage's input U -- the tile plus a two-cell halo, widened in x so that the box starts on a
// 16-byte boundary -- from global into shared memory; its completion is counted in bytes on an
// mbarrier.  Only this GPU's own memory is read and nothing is multicast.  Waits on an mbarrier
// are bounded: after kMbarSpins tries the waiting thread records STATUS_TIMEOUT in the control
// block, stops waiting for later boxes and goes on (the step's result is then void and the host
// reports HYDRO_ETIMEOUT); every other waiter of the grid gives up as soon as it sees that bit.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hydro_device.cuh"

namespace hydro {

// Tensor maps of the five fields of the stage's input (3D, FP32).  Passed to the kernel as a
// __grid_constant__ parameter, so the copies read the maps from parameter space.
struct TmaMaps {
    CUtensorMap map[5];
};

// Box of one plane for a BX x BY tile: x from x0 - 4 (a multiple of four cells, i.e. of 16
// bytes) to x0 + BX + 4, y from y0 - 2 to y0 + BY + 2.  Out-of-range cells read as zero and are
// replaced by the boundary condition (plain loads) where the halo needs them.
template <int BX, int BY> struct TmaBox {
    static constexpr int slots = 2;  // planes in the ring
    static constexpr int W = BX + 8;
    static constexpr int H = BY + 4;
    static constexpr int cells = W * H;
    static constexpr unsigned bytes = 5u * cells * 4u;  // one plane, five FP32 fields
    // rows start on 16 bytes, fields and slots on 128 (checked where a TMA kernel is compiled)
    static constexpr bool aligned = (W * 4) % 16 == 0 && (cells * 4) % 128 == 0;
    // shared bytes of the ring plus one mbarrier per slot and 128 bytes of alignment slack
    static constexpr size_t smem_bytes = slots * (size_t)bytes + 8u * slots + 128u;
};

constexpr int kMbarSpins = 1 << 16;
constexpr unsigned long long kMbarMaxNs = 1000000000ull;  // and at most about one second

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Make the initialised mbarriers visible to the asynchronous proxy (the TMA unit).
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of copies to complete the current phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// Wait until the phase of parity `parity` has completed; false after kMbarSpins tries or about
// kMbarMaxNs of the global timer, or as soon as `abort_bits` has STATUS_TIMEOUT set by another
// waiter (both checked every 256 tries, so a wait that succeeds at once reads neither).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          const volatile unsigned int *abort_bits) {
    unsigned long long t0 = 0;
    for (int i = 0; i < kMbarSpins; ++i) {
        if ((i & 255) == 255) {
            if (*abort_bits & STATUS_TIMEOUT) return false;
            const unsigned long long t = globaltimer_ns();
            if (t0 == 0)
                t0 = t;
            else if (t - t0 > kMbarMaxNs)
                return false;
        }
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Order this thread's earlier shared-memory accesses (after a CTA barrier: everyone's) before
// the asynchronous proxy's next writes to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Copy the box at (x, y, z) of tensor map `map` into shared memory at `dst`, completing
// `bytes` on mbarrier `bar`.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Host: encode the five maps of FP32 planes of an n[0] x n[1] x n[2] grid (x fastest) with a
// box of box_w x box_h x 1.  Needs n[0] a multiple of 4 (16-byte row pitch) and 16-byte
// aligned planes; cudaErrorInvalidValue otherwise or if the driver refuses a map.
cudaError_t encode_plane_maps(TmaMaps *out, const void *const planes[5], const int n[3],
                              int box_w, int box_h);

}  // namespace hydro
