// FP32 RK-stage kernels, dim 3 (compiled with FMA contraction), both staging depths and both
// occupancy targets: tiles 32x8, 32x4, 64x4 (the others are in stage_f32_d3b.cu).
#include "stage_launch.cuh"

namespace hydro {

cudaError_t stage_f32_d3b(const StageLaunch &L, cudaStream_t st, bool prepare_only);

cudaError_t stage_f32_d3(const StageLaunch &L, cudaStream_t st, bool prepare_only) {
    HYDRO_STAGE_CASE_M(float, 3, 32, 8, true)
    HYDRO_STAGE_CASE(float, 3, 32, 4, true)
    HYDRO_STAGE_CASE(float, 3, 64, 4, true)
    return stage_f32_d3b(L, st, prepare_only);
}

}  // namespace hydro
