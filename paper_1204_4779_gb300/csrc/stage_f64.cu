// FP64 RK-stage kernels, dims 1-3.  Compiled with --fmad=false: every operation of the
// stencil is one correctly rounded IEEE-754 operation, in the order of the plain formulas.
#include "stage_launch.cuh"

namespace hydro {

cudaError_t stage_f64(int dim, const StageLaunch &L, cudaStream_t st, bool prepare_only) {
    if (dim == 1) {
        HYDRO_STAGE_CASE(double, 1, 128, 1, false)
    } else if (dim == 2) {
        HYDRO_STAGE_CASE(double, 2, 32, 8, false)
        HYDRO_STAGE_CASE(double, 2, 128, 1, false)
    } else if (dim == 3) {
        HYDRO_STAGE_CASE_M(double, 3, 32, 8, false)
    }
    return cudaErrorInvalidValue;
}

const TileShape kTiles[] = {
    {1, 1, 128, 1, 0}, {1, 1, 256, 1, 0},
    {1, 2, 32, 8, 0},  {1, 2, 64, 4, 0},  {1, 2, 16, 16, 0}, {1, 2, 32, 16, 0},
    {1, 2, 64, 1, 1},  {1, 2, 128, 1, 1}, {1, 2, 256, 1, 1},
    {1, 3, 32, 8, 1, 1}, {1, 3, 32, 4, 1},  {1, 3, 64, 4, 1},  {1, 3, 16, 16, 1, 1},
    {1, 3, 32, 16, 1}, {1, 3, 16, 8, 1, 1, 1},
    {0, 1, 128, 1, 0}, {0, 2, 32, 8, 0},  {0, 2, 128, 1, 0}, {0, 3, 32, 8, 0, 1},
};
const int kNumTiles = sizeof(kTiles) / sizeof(kTiles[0]);

}  // namespace hydro
