// FP32 batched RK-stage kernels (compiled with FMA contraction).
#include "batch_kernel.cuh"

namespace hydro {

cudaError_t batch_f32(const BatchLaunch &L, cudaStream_t st, int kind, bool prepare_only,
                      int *blocks_per_sm) {
    if (L.tile_x == 32 && L.tile_y == 8)
        return batch_dispatch_tile<float, 32, 8>(L, st, kind, prepare_only, blocks_per_sm);
    if (L.tile_x == 16 && L.tile_y == 16)
        return batch_dispatch_tile<float, 16, 16>(L, st, kind, prepare_only, blocks_per_sm);
    // row tiles (march along y), three-CTA-equivalent register budget
    if (L.tile_x == 32 && L.tile_y == 1)
        return batch_dispatch_tile<float, 32, 1, 3>(L, st, kind, prepare_only, blocks_per_sm);
    if (L.tile_x == 64 && L.tile_y == 1)
        return batch_dispatch_tile<float, 64, 1, 3>(L, st, kind, prepare_only, blocks_per_sm);
    if (L.tile_x == 128 && L.tile_y == 1)
        return batch_dispatch_tile<float, 128, 1, 3>(L, st, kind, prepare_only, blocks_per_sm);
    return cudaErrorInvalidValue;
}

}  // namespace hydro
