// FP32 RK-stage kernels, dim 3: tiles 16x16, 32x16, 16x8 (see stage_f32_d3.cu); 16x16 and 16x8
// also in the manifest forms, 16x8 also with TMA plane staging.
#include "stage_launch.cuh"

namespace hydro {

cudaError_t stage_f32_d3b(const StageLaunch &L, cudaStream_t st, bool prepare_only) {
    HYDRO_STAGE_CASE_M(float, 3, 16, 16, true)
    HYDRO_STAGE_CASE(float, 3, 32, 16, true)
    HYDRO_STAGE_CASE_MT(float, 3, 16, 8, true)
    return cudaErrorInvalidValue;
}

}  // namespace hydro
