// FP32 RK-stage kernels, dims 1 and 2 (compiled with FMA contraction): one-plane tiles, and in
// dim 2 also row tiles that march along y.
#include "stage_launch.cuh"

namespace hydro {

cudaError_t stage_f32_d1(const StageLaunch &L, cudaStream_t st, bool prepare_only) {
    HYDRO_STAGE_CASE(float, 1, 128, 1, false)
    HYDRO_STAGE_CASE(float, 1, 256, 1, false)
    return cudaErrorInvalidValue;
}

cudaError_t stage_f32_d2(const StageLaunch &L, cudaStream_t st, bool prepare_only) {
    HYDRO_STAGE_CASE(float, 2, 32, 8, false)
    HYDRO_STAGE_CASE(float, 2, 64, 4, false)
    HYDRO_STAGE_CASE(float, 2, 16, 16, false)
    HYDRO_STAGE_CASE(float, 2, 32, 16, false)
    // row tiles: BX cells of x, marching along y
    HYDRO_STAGE_CASE(float, 2, 64, 1, true)
    HYDRO_STAGE_CASE(float, 2, 128, 1, true)
    HYDRO_STAGE_CASE(float, 2, 256, 1, true)
    return cudaErrorInvalidValue;
}

}  // namespace hydro
