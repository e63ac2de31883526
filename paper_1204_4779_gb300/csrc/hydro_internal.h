// Internal interface between the C-ABI host code and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace hydro {

// Record the text of a failed CUDA call for hydro_last_cuda_error(); returns HYDRO_ECUDA.
int record_cuda_error(cudaError_t e, const char *what);

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
    int prefetch;       // dim 3: 1 = next plane's loads one plane ahead, 0 = at staging,
                        // 2 = planes staged by TMA (FP32 tiles compiled with it)
    int split;          // stage 2: 0 = dt reduction fused, 1 = left to a separate CFL pass
    int occupancy;      // dim 3 FP32: resident CTAs per SM the register budget targets (2 or 3)
    int order;          // reconstruction order (2 MinBee, 1 first order); 0 = 2
    int riemann;        // HLLC wave speeds: 0 Davis, 1 pressure-based
    int zchunk0;        // first march chunk to launch
    int zchunks;        // march chunks to launch (0: all from zchunk0)
    int manifest;       // dim 3: 0 nothing stored, 1 V stored by a pass, 2 face fluxes stored
    void *vbuf[5];      // manifest V: the primitive planes
    void *flux[3][5];   // manifest F: face-flux planes per axis
    int ana;            // bit a: axis a takes analytic ghost cells from frame (one-plane tiles)
    const void *frame[5];
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

// Compiled tile shapes (both_pf: both staging depths compiled).
struct TileShape {
    int prec, dim, bx, by, both_pf;
    int manifest;  // also compiled in the manifest forms (V and F)
    int tma;       // also compiled with TMA plane staging
};
extern const TileShape kTiles[];
extern const int kNumTiles;

// Auxiliary kernels (aux_kernels.cu).
struct AuxArgs {
    int prec;
    int dim;
    long long ncell;        // cells the launch covers (the CFL pass: from cell `first`)
    long long first;        // CFL pass over part of the grid: its first cell (0: all)
    unsigned total_blocks;  // CFL pass in parts: CTAs of all the parts' launches (0: this one)
    const void *u[5];
    void *out[5];
    double dr[3];
    double gamma;
    void *ctrl;
};
// CFL pass: max signal of u -> dt of the next step in ctrl.  advance = false: the first dt of
// a call (ctrl freshly initialised); true: after an RK step whose stage 2 left the reduction
// to this pass (t advances by the step's dt first).
cudaError_t launch_cfl(const AuxArgs &A, cudaStream_t st, bool advance = false);
// CTAs a CFL-pass launch over `ncell` cells uses (to sum over the parts of a split pass).
unsigned cfl_blocks(long long ncell);
// Totals: per-CTA partials into `partials` (dim+2 x nparts doubles), then the fixed-order
// final sum times the cell volume into ctrl->totals.
cudaError_t launch_totals(const AuxArgs &A, double *partials, int nparts, double vol,
                          cudaStream_t st);
cudaError_t launch_convert(const AuxArgs &A, int to_cons, cudaStream_t st);

constexpr int kTotalsParts = 1024;

// Analytic-solution boundaries (analytic.cu).  The frame is the ring of two ghost layers
// around an nx x ny grid (dim 1: the four cells beyond its ends), frame_cells cells per plane in
// the order of
// frame_index (stage_kernel.cuh); launch_analytic_frame fills it with the conserved form of the
// solution `kind` (1 entropy wave, 2 sound wave of amplitude amp, 3 Sod's shock tube, each
// travelling at angle theta from the x axis) at the time of RK stage `stage` of the step held
// in ctrl.
struct AnalyticLaunch {
    int prec, dim, nx, ny, kind;
    double lo[2], dr[2];
    double gamma, theta, amp;
    void *frame[5];
    void *ctrl;
};
long long frame_cells(int dim, long long nx, long long ny);

// Ghost exchange through buffers (exchange.cu): pack the two boundary layers at both ends of
// each exchange axis (bit a of axes) from the stage input uin into buf[a][side], then unpack
// each buffer into the ghost ring at the other end (the periodic wrap on one GPU).
struct ExchangeLaunch {
    int prec, dim, nx, ny, axes;
    const void *uin[5];
    void *buf[2][2];
    void *frame[5];
};
long long exchange_buffer_cells(int dim, long long nx, long long ny, int axis);
cudaError_t launch_exchange(const ExchangeLaunch &L, cudaStream_t st);
cudaError_t launch_analytic_frame(const AnalyticLaunch &L, int stage, cudaStream_t st);

// ---- batched 2D grids (batch_kernel.cuh) ----
struct BatchItem {  // one tile of one grid
    int g, x0, y0, pad;
};
struct BatchGrid {  // geometry of one grid of the batch
    long long off;    // first cell of the grid in every packed plane
    int nx, ny;
    int ntiles;       // work items of this grid
    int first_item;   // index of its first work item
    double dr[2];
    float inv_dr[2];
};
struct BatchLaunch {
    const void *uin[4];
    const void *ubase[4];
    void *uout[4];
    const BatchItem *items;
    int n_items;
    const BatchGrid *grids;
    int n_grids;
    void *ctrl;          // n_grids control blocks
    void *tile_sig;      // n_items CFL-signal maxima, one per work item (element type)
    unsigned int *claim; // work-item counters of the row kernels' stages 1 and 2 (zero before
                         // each stage launch: the init and finaliser kernels reset them)
    const double *t0;    // per-grid start times (init), may be null
    double t_end, cfl, gamma;
    int periodic[2];
    int n_blocks;        // persistent grid size
    int tile_x, tile_y;  // tile_y = 1: row tiles, which march along y
    int march;           // rows of a row tile's work item
};
// kind: 0 init, 1 CFL pass (tile maxima), 2 RK stage 1, 3 RK stage 2 (+ tile maxima),
// 4 per-grid totals, 5 per-grid dt from the tile maxima (first dt of a call), 6 the same after
// a step (time advances first).
// prepare_only: set kernel attributes and report resident CTAs per SM of the stage kernel.
cudaError_t batch_f32(const BatchLaunch &L, cudaStream_t st, int kind, bool prepare_only,
                      int *blocks_per_sm);
cudaError_t batch_f64(const BatchLaunch &L, cudaStream_t st, int kind, bool prepare_only,
                      int *blocks_per_sm);

}  // namespace hydro
