// hydro_step_static: the RK step for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code running inside
// another runtime that owns every allocation (a host framework with its own caching
// allocator), and small embedded or real-time callers that must not allocate after start-up.
// This entry point needs no workspace: the RK stage buffer U1 and the step control block live
// in one file-scope device array of fixed size, HYDRO_STATIC_SCRATCH_BYTES, which every GPU
// that loads the library holds until the process exits.  The caller still passes the state
// planes, which must live on the caller's current device: the call runs there.
//
// Host code cannot use that array's name as a device address (in host code it names a host
// stand-in), so the first call on each device, with that device current, looks the address
// up once with cudaGetSymbolAddress and sets the stage kernels' shared-memory attributes;
// later calls reuse it.
//
// The kernels are one fixed variant (not the tuned defaults of hydro_create): 32 x 8 tiles in
// 2D and 3D (3D marching up to 64 planes), 128-cell rows in 1D, look-ahead staging, the
// two-CTA register budget, the dt reduction fused into stage 2.  The call launches the CFL
// pass and then 2 n_steps stage kernels whatever t_end is (stages after t_end return at
// once), with no graph; it reads nothing back unless t_inout or steps_done asks for it, in
// which case it copies the control block to the host and synchronises the stream.
//
// Every call shares the one array and it keeps the last call's contents: the control block
// is rewritten at the start of each call and U1 is fully written by stage 1 before stage 2
// reads it.  Calls that overlap on the GPU (on different streams, or from different host
// threads without ordering) race on the array.
#include <string.h>

#include <mutex>

#include "../../include/hydro.h"
#include "hydro_device.cuh"
#include "hydro_internal.h"

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[HYDRO_STATIC_SCRATCH_BYTES];

unsigned char *g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup_mutex;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Start-of-call state of the control block (every field, so no earlier call leaks in).
__global__ void init_ctrl_kernel(hydro::Ctrl *c, double t0, double t_end, double cfl, double dr0,
                                 double dr1, double dr2) {
    hydro::Ctrl z = {};
    z.t = t0;
    z.t_end = t_end;
    z.cfl = cfl;
    z.dr[0] = dr0;
    z.dr[1] = dr1;
    z.dr[2] = dr2;
    *c = z;
}

cudaError_t stage_launch(int prec, int dim, const hydro::StageLaunch &L, cudaStream_t st,
                         bool prepare_only) {
    if (prec == HYDRO_F64) return hydro::stage_f64(dim, L, st, prepare_only);
    switch (dim) {
        case 1: return hydro::stage_f32_d1(L, st, prepare_only);
        case 2: return hydro::stage_f32_d2(L, st, prepare_only);
        default: return hydro::stage_f32_d3(L, st, prepare_only);
    }
}

}  // namespace

extern "C" int hydro_step_static(const hydro_grid_t *grid, double gamma, const int32_t bc[3],
                                 int32_t prec, double cfl, const hydro_state_t *state,
                                 int32_t n_steps, double t_end, double *t_inout,
                                 int32_t *steps_done, void *stream) {
    if (!grid || !bc || !state || grid->dim < 1 || grid->dim > 3 || n_steps < 0) return HYDRO_EINVAL;
    if (prec != HYDRO_F32 && prec != HYDRO_F64) return HYDRO_EINVAL;
    if (!(gamma > 1.0) || !(gamma < 1e300) || !(cfl > 0.0) || !(cfl < 1e300) || t_end != t_end)
        return HYDRO_EINVAL;
    const int dim = grid->dim;
    long long ncell = 1;
    int n[3] = {1, 1, 1}, periodic[3] = {1, 1, 1};
    double dr[3] = {1.0, 1.0, 1.0};
    for (int a = 0; a < dim; ++a) {
        if (grid->n[a] < 1 || grid->n[a] > (1LL << 31) - 1024 || !(grid->hi[a] > grid->lo[a]))
            return HYDRO_EINVAL;
        if (bc[a] != HYDRO_BC_PERIODIC && bc[a] != HYDRO_BC_OUTFLOW) return HYDRO_EINVAL;
        n[a] = (int)grid->n[a];
        periodic[a] = bc[a] == HYDRO_BC_PERIODIC;
        dr[a] = (grid->hi[a] - grid->lo[a]) / (double)grid->n[a];
        ncell *= grid->n[a];
        if (ncell >= (1LL << 31)) return HYDRO_EINVAL;
    }
    for (int k = 0; k < dim + 2; ++k)
        if (!state->plane[k]) return HYDRO_EINVAL;
    // the scratch holds the control block and dim+2 planes of U1
    const size_t esz = prec == HYDRO_F32 ? 4 : 8;
    const size_t plane = align_up((size_t)ncell * esz);
    const size_t u1_off = align_up(sizeof(hydro::Ctrl));
    if (u1_off + plane * (size_t)(dim + 2) > HYDRO_STATIC_SCRATCH_BYTES) return HYDRO_EINVAL;
    const double t0 = t_inout ? *t_inout : 0.0;
    if (t0 != t0) return HYDRO_EINVAL;

    hydro::StageLaunch L;
    memset(&L, 0, sizeof L);
    L.march = dim == 3 ? (n[2] < 64 ? n[2] : 64) : 1;
    L.tile_x = dim == 1 ? 128 : 32;
    L.tile_y = dim == 1 ? 1 : 8;
    // launch-grid limits of the stage kernels (y and z at most 65535 CTAs), checked here
    // rather than left to the array's size cap
    if (dim >= 2 && (n[1] + L.tile_y - 1) / L.tile_y > 65535) return HYDRO_EINVAL;
    if (dim == 3 && (n[2] + L.march - 1) / L.march > 65535) return HYDRO_EINVAL;
    L.prefetch = 1;
    L.split = 0;
    L.occupancy = 2;
    L.gamma = gamma;
    for (int a = 0; a < 3; ++a) {
        L.n[a] = n[a];
        L.periodic[a] = periodic[a];
        L.dr[a] = dr[a];
    }

    // set-up, once per device, with that device current
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HYDRO_ECUDA;
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess || !ptr) return HYDRO_ECUDA;
            for (int p = 0; p < 2; ++p)
                for (int d = 1; d <= 3; ++d) {
                    hydro::StageLaunch P = L;
                    P.tile_x = d == 1 ? 128 : 32;
                    P.tile_y = d == 1 ? 1 : 8;
                    if (stage_launch(p, d, P, nullptr, /*prepare_only=*/true) != cudaSuccess)
                        return HYDRO_ECUDA;
                }
            g_scratch_addr[dev] = static_cast<unsigned char *>(ptr);
        }
        base = g_scratch_addr[dev];
    }

    hydro::Ctrl *ctrl = reinterpret_cast<hydro::Ctrl *>(base);
    void *u1[5] = {};
    for (int k = 0; k < dim + 2; ++k) u1[k] = base + u1_off + plane * (size_t)k;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    init_ctrl_kernel<<<1, 1, 0, st>>>(ctrl, t0, t_end, cfl, dr[0], dr[1], dr[2]);
    if ((e = cudaGetLastError()) != cudaSuccess) return HYDRO_ECUDA;
    hydro::AuxArgs A;
    memset(&A, 0, sizeof A);
    A.prec = prec;
    A.dim = dim;
    A.ncell = ncell;
    A.gamma = gamma;
    A.ctrl = ctrl;
    for (int k = 0; k < dim + 2; ++k) A.u[k] = state->plane[k];
    for (int a = 0; a < 3; ++a) A.dr[a] = dr[a];
    if (hydro::launch_cfl(A, st) != cudaSuccess) return HYDRO_ECUDA;

    L.ctrl = ctrl;
    hydro::StageLaunch L1 = L, L2 = L;
    L1.stage = 1;
    L2.stage = 2;
    for (int k = 0; k < dim + 2; ++k) {
        L1.uin[k] = state->plane[k];
        L1.ubase[k] = state->plane[k];
        L1.uout[k] = u1[k];
        L2.uin[k] = u1[k];
        L2.ubase[k] = state->plane[k];
        L2.uout[k] = state->plane[k];
    }
    for (int i = 0; i < n_steps; ++i) {
        if (stage_launch(prec, dim, L1, st, false) != cudaSuccess) return HYDRO_ECUDA;
        if (stage_launch(prec, dim, L2, st, false) != cudaSuccess) return HYDRO_ECUDA;
    }
    if (!t_inout && !steps_done) return HYDRO_OK;
    hydro::Ctrl h;
    if (cudaMemcpyAsync(&h, ctrl, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return HYDRO_ECUDA;
    if (t_inout) *t_inout = h.t;
    if (steps_done) *steps_done = h.steps;
    return (h.status & hydro::STATUS_NONFINITE) ? HYDRO_ENONFINITE : HYDRO_OK;
}
