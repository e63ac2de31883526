// FP32 RK-stage kernels, dim 3 (compiled with FMA contraction), both staging depths.
#include "stage_launch.cuh"

namespace hydro {

cudaError_t stage_f32_d3(const StageLaunch &L, cudaStream_t st, bool prepare_only) {
    HYDRO_STAGE_CASE(float, 3, 32, 8, true)
    HYDRO_STAGE_CASE(float, 3, 32, 4, true)
    HYDRO_STAGE_CASE(float, 3, 64, 4, true)
    HYDRO_STAGE_CASE(float, 3, 16, 16, true)
    HYDRO_STAGE_CASE(float, 3, 32, 16, true)
    HYDRO_STAGE_CASE(float, 3, 16, 8, true)
    return cudaErrorInvalidValue;
}

}  // namespace hydro
