// FP32 RK-stage kernels, dim 3 (compiled with FMA contraction).
#include "stage_launch.cuh"

namespace hydro {

cudaError_t stage_f32_d3(const StageLaunch &L, cudaStream_t st, bool prepare_only) {
    HYDRO_STAGE_CASE(float, 3, 32, 8)
    HYDRO_STAGE_CASE(float, 3, 32, 4)
    HYDRO_STAGE_CASE(float, 3, 64, 4)
    HYDRO_STAGE_CASE(float, 3, 16, 16)
    HYDRO_STAGE_CASE(float, 3, 32, 16)
    return cudaErrorInvalidValue;
}

}  // namespace hydro
