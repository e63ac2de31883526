// Internal interface between the C-ABI host code and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace hydro {

// Arguments of one RK-stage launch (precision-free; the launcher casts).
struct StageLaunch {
    int stage;          // 1 or 2
    const void *uin[5];
    const void *ubase[5];
    void *uout[5];
    int n[3];
    int periodic[3];
    int march;
    int tile_x, tile_y;
    double dr[3];
    double gamma;
    void *ctrl;
};

// Launch (or, with prepare_only, set the kernel attributes of) the stage kernel with tile
// (L.tile_x, L.tile_y).  cudaErrorInvalidValue if that tile is not compiled.
cudaError_t stage_f32_d1(const StageLaunch &L, cudaStream_t st, bool prepare_only);
cudaError_t stage_f32_d2(const StageLaunch &L, cudaStream_t st, bool prepare_only);
cudaError_t stage_f32_d3(const StageLaunch &L, cudaStream_t st, bool prepare_only);
cudaError_t stage_f64(int dim, const StageLaunch &L, cudaStream_t st, bool prepare_only);

// Compiled tile shapes.
struct TileShape {
    int prec, dim, bx, by;
};
extern const TileShape kTiles[];
extern const int kNumTiles;

// Auxiliary kernels (aux_kernels.cu).
struct AuxArgs {
    int prec;
    int dim;
    long long ncell;
    const void *u[5];
    void *out[5];
    double dr[3];
    double gamma;
    void *ctrl;
};
// CFL pass: max signal of u -> dt of the first step in ctrl (ctrl must be initialised).
cudaError_t launch_cfl(const AuxArgs &A, cudaStream_t st);
// Totals: per-CTA partials into `partials` (dim+2 x nparts doubles), then the fixed-order
// final sum times the cell volume into ctrl->totals.
cudaError_t launch_totals(const AuxArgs &A, double *partials, int nparts, double vol,
                          cudaStream_t st);
cudaError_t launch_convert(const AuxArgs &A, int to_cons, cudaStream_t st);

constexpr int kTotalsParts = 1024;

}  // namespace hydro
