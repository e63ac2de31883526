// FP64 batched RK-stage kernels, compiled with --fmad=false like the FP64 single-grid path.
#include "batch_kernel.cuh"

namespace hydro {

cudaError_t batch_f64(const BatchLaunch &L, cudaStream_t st, int kind, bool prepare_only,
                      int *blocks_per_sm) {
    if (L.tile_x == 32 && L.tile_y == 8)
        return batch_dispatch_tile<double, 32, 8>(L, st, kind, prepare_only, blocks_per_sm);
    if (L.tile_x == 64 && L.tile_y == 1)
        return batch_dispatch_tile<double, 64, 1>(L, st, kind, prepare_only, blocks_per_sm);
    return cudaErrorInvalidValue;
}

}  // namespace hydro
