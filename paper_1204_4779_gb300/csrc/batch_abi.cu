// C ABI of the batched path (include/hydro.h, hydro_batch_*): many independent 2D grids of
// uneven size in packed planes, one persistent launch per RK stage, steps captured in CUDA
// graphs, per-grid dt and time on the device.
#include <string.h>

#include <new>
#include <vector>

#include "../../include/hydro.h"
#include "hydro_device.cuh"
#include "hydro_internal.h"

using hydro::BatchGrid;
using hydro::BatchItem;
using hydro::BatchLaunch;
using hydro::Ctrl;

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxChunk = 64;
constexpr int kGraphSlots = 8;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct BatchLayout {
    size_t ctrl_off, t0_off, grids_off, items_off, sig_off, claim_off, u1_off, plane_bytes, total;
    long long ncell, n_items;
};

bool shapes_ok(int32_t n_grids, const int64_t *nx, const int64_t *ny) {
    if (n_grids < 1 || !nx || !ny) return false;
    long long total = 0;
    for (int g = 0; g < n_grids; ++g) {
        if (nx[g] < 1 || ny[g] < 1 || nx[g] > (1 << 30) || ny[g] > (1 << 30)) return false;
        total += nx[g] * ny[g];
        if (total >= (1LL << 40)) return false;
    }
    return true;
}

// Tile of the batch kernels and the rows of one work item (the tile height, or for row tiles,
// tile_y = 1, the march along y).
// Default: FP32 row tiles of 32 columns marching 32 rows (4096 uneven grids: 24.3 G
// cell-updates/s against 16.4 G for the 32 x 8 tile kernel); FP64 the 32 x 8 tiles.
void tile_of(int prec, const hydro_variant_t *v, int *bx, int *by, int *rows) {
    *bx = 32;
    *by = prec == HYDRO_F32 ? 1 : 8;
    if (v && v->tile_x) *bx = v->tile_x;
    if (v && v->tile_y) *by = v->tile_y;
    *rows = *by;
    if (*by == 1) *rows = (v && v->march > 0) ? v->march : 32;
}

bool tile_ok(int prec, int bx, int by, const hydro_variant_t *v) {
    if (v && v->march < 0) return false;
    if (bx == 32 && by == 8) return true;
    if (by == 1) return prec == HYDRO_F32 ? (bx == 32 || bx == 64 || bx == 128) : bx == 64;
    return prec == HYDRO_F32 && bx == 16 && by == 16;
}

BatchLayout batch_layout(int32_t n_grids, const int64_t *nx, const int64_t *ny, int prec, int bx,
                         int rows) {
    BatchLayout L;
    L.ncell = 0;
    L.n_items = 0;
    for (int g = 0; g < n_grids; ++g) {
        L.ncell += nx[g] * ny[g];
        L.n_items += ((nx[g] + bx - 1) / bx) * ((ny[g] + rows - 1) / rows);
    }
    const size_t esz = prec == HYDRO_F32 ? 4 : 8;
    L.ctrl_off = 0;
    L.t0_off = align_up(sizeof(Ctrl) * (size_t)n_grids);
    L.grids_off = L.t0_off + align_up(sizeof(double) * (size_t)n_grids);
    L.items_off = L.grids_off + align_up(sizeof(BatchGrid) * (size_t)n_grids);
    L.sig_off = L.items_off + align_up(sizeof(BatchItem) * (size_t)L.n_items);
    L.claim_off = L.sig_off + align_up(sizeof(double) * (size_t)L.n_items);
    L.u1_off = L.claim_off + align_up(2 * sizeof(unsigned int));
    L.plane_bytes = align_up((size_t)L.ncell * esz);
    L.total = L.u1_off + 4 * L.plane_bytes;
    return L;
}

int bfail(cudaError_t e, const char *what) { return hydro::record_cuda_error(e, what); }

#define BCK(call)                                        \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return bfail(e_, #call);  \
    } while (0)

}  // namespace

struct hydro_batch {
    int device = 0;
    int prec = HYDRO_F32;
    int n_grids = 0;
    std::vector<long long> offsets;  // n_grids + 1
    BatchLayout lay = {};
    unsigned char *ws = nullptr;
    Ctrl *ctrl = nullptr;
    double *t0 = nullptr;
    BatchGrid *grids = nullptr;
    BatchItem *items = nullptr;
    void *tile_sig = nullptr;
    unsigned int *claim = nullptr;
    void *u1[4] = {};
    double gamma = 1.4, cfl = 0.4;
    int periodic[2] = {1, 1};
    int tile_x = 32, tile_y = 8;
    int rows = 8;  // rows of a work item
    int n_blocks = 1;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    struct Graph {
        int chunk = 0;
        void *planes[4] = {};
        cudaGraphExec_t exec = nullptr;
        unsigned long long last_use = 0;
    } graphs[kGraphSlots];
    unsigned long long use_clock = 0;
    bool profiling = false;
    std::vector<cudaEvent_t> events;
    double kms[3] = {0, 0, 0};
    long long klaunch[3] = {0, 0, 0};
};

namespace {

BatchLaunch launch_args(const hydro_batch *b, const hydro_state_t *s, int kind, const double *t0,
                        double t_end) {
    BatchLaunch L;
    memset(&L, 0, sizeof L);
    for (int k = 0; k < 4; ++k) {
        const bool stage2 = kind == 3;
        L.uin[k] = stage2 ? b->u1[k] : s->plane[k];
        L.ubase[k] = s->plane[k];
        L.uout[k] = kind == 2 ? b->u1[k] : s->plane[k];
    }
    L.items = b->items;
    L.n_items = (int)b->lay.n_items;
    L.grids = b->grids;
    L.n_grids = b->n_grids;
    L.ctrl = b->ctrl;
    L.tile_sig = b->tile_sig;
    L.claim = b->claim;
    L.t0 = t0;
    L.t_end = t_end;
    L.cfl = b->cfl;
    L.gamma = b->gamma;
    L.periodic[0] = b->periodic[0];
    L.periodic[1] = b->periodic[1];
    L.n_blocks = b->n_blocks;
    L.tile_x = b->tile_x;
    L.tile_y = b->tile_y;
    L.march = b->rows;
    return L;
}

cudaError_t launch(const hydro_batch *b, const BatchLaunch &L, cudaStream_t st, int kind) {
    return b->prec == HYDRO_F32 ? hydro::batch_f32(L, st, kind, false, nullptr)
                                : hydro::batch_f64(L, st, kind, false, nullptr);
}

bool state_ok(const hydro_state_t *s) {
    if (!s) return false;
    for (int k = 0; k < 4; ++k)
        if (!s->plane[k]) return false;
    return true;
}

int timed(hydro_batch *b, const BatchLaunch &L, int kind, int slot) {
    while (b->events.size() < 2) {
        cudaEvent_t e;
        BCK(cudaEventCreate(&e));
        b->events.push_back(e);
    }
    BCK(cudaEventRecord(b->events[0], b->stream));
    BCK(launch(b, L, b->stream, kind));
    BCK(cudaEventRecord(b->events[1], b->stream));
    BCK(cudaEventSynchronize(b->events[1]));
    float ms = 0;
    BCK(cudaEventElapsedTime(&ms, b->events[0], b->events[1]));
    b->kms[slot] += ms;
    b->klaunch[slot] += 1;
    return HYDRO_OK;
}

int get_graph(hydro_batch *b, const hydro_state_t *s, int chunk, cudaGraphExec_t *out) {
    hydro_batch::Graph *free_slot = nullptr, *oldest = &b->graphs[0];
    for (auto &g : b->graphs) {
        if (g.exec && g.chunk == chunk) {
            bool same = true;
            for (int k = 0; k < 4; ++k) same &= g.planes[k] == s->plane[k];
            if (same) {
                g.last_use = ++b->use_clock;
                *out = g.exec;
                return HYDRO_OK;
            }
        }
        if (!g.exec && !free_slot) free_slot = &g;
        if (g.last_use < oldest->last_use) oldest = &g;
    }
    hydro_batch::Graph *slot = free_slot ? free_slot : oldest;
    if (slot->exec) {
        cudaGraphExecDestroy(slot->exec);
        slot->exec = nullptr;
    }
    const BatchLaunch L1 = launch_args(b, s, 2, nullptr, 0.0), L2 = launch_args(b, s, 3, nullptr, 0.0);
    const BatchLaunch F = launch_args(b, s, 6, nullptr, 0.0);
    BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    for (int i = 0; i < chunk && le == cudaSuccess; ++i) {
        le = launch(b, L1, b->cap, 2);
        if (le == cudaSuccess) le = launch(b, L2, b->cap, 3);
        if (le == cudaSuccess) le = launch(b, F, b->cap, 6);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->cap, &graph);
    if (le != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return bfail(le, "batch stage launch during capture");
    }
    if (ee != cudaSuccess) return bfail(ee, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return bfail(ie, "cudaGraphInstantiate");
    slot->exec = exec;
    slot->chunk = chunk;
    for (int k = 0; k < 4; ++k) slot->planes[k] = s->plane[k];
    slot->last_use = ++b->use_clock;
    *out = exec;
    return HYDRO_OK;
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

int hydro_batch_workspace_bytes(int32_t n_grids, const int64_t *nx, const int64_t *ny, int32_t prec,
                                const hydro_variant_t *variant, size_t *bytes_out) {
    if (!bytes_out || !shapes_ok(n_grids, nx, ny)) return HYDRO_EINVAL;
    if (prec != HYDRO_F32 && prec != HYDRO_F64) return HYDRO_EINVAL;
    int bx, by, rows;
    tile_of(prec, variant, &bx, &by, &rows);
    if (!tile_ok(prec, bx, by, variant)) return HYDRO_EUNSUPPORTED;
    *bytes_out = batch_layout(n_grids, nx, ny, prec, bx, rows).total;
    return HYDRO_OK;
}

int hydro_batch_create(int32_t n_grids, const int64_t *nx, const int64_t *ny, double gamma,
                       const int32_t bc[2], int32_t prec, double cfl,
                       const hydro_variant_t *variant, void *workspace, size_t workspace_bytes,
                       void *stream, hydro_batch_t **out) {
    if (!out) return HYDRO_EINVAL;
    *out = nullptr;
    if (!shapes_ok(n_grids, nx, ny) || !bc || !workspace) return HYDRO_EINVAL;
    if (prec != HYDRO_F32 && prec != HYDRO_F64) return HYDRO_EINVAL;
    if (!(gamma > 1.0) || !(gamma < 1e300) || !(cfl > 0.0) || !(cfl < 1e300)) return HYDRO_EINVAL;
    for (int a = 0; a < 2; ++a)
        if (bc[a] != HYDRO_BC_PERIODIC && bc[a] != HYDRO_BC_OUTFLOW) return HYDRO_EINVAL;
    if (((uintptr_t)workspace) % kAlign) return HYDRO_EINVAL;
    int bx, by, rows;
    tile_of(prec, variant, &bx, &by, &rows);
    if (!tile_ok(prec, bx, by, variant)) return HYDRO_EUNSUPPORTED;
    const BatchLayout lay = batch_layout(n_grids, nx, ny, prec, bx, rows);
    if (workspace_bytes < lay.total) return HYDRO_EINVAL;
    if (lay.n_items >= (1LL << 31)) return HYDRO_EUNSUPPORTED;

    hydro_batch *b = new (std::nothrow) hydro_batch();
    if (!b) return HYDRO_EINVAL;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return bfail(cudaGetLastError(), "cudaGetDevice");
    }
    b->prec = prec;
    b->n_grids = n_grids;
    b->lay = lay;
    b->gamma = gamma;
    b->cfl = cfl;
    b->periodic[0] = bc[0] == HYDRO_BC_PERIODIC;
    b->periodic[1] = bc[1] == HYDRO_BC_PERIODIC;
    b->tile_x = bx;
    b->tile_y = by;
    b->rows = rows;
    b->stream = static_cast<cudaStream_t>(stream);
    b->ws = static_cast<unsigned char *>(workspace);
    b->ctrl = reinterpret_cast<Ctrl *>(b->ws + lay.ctrl_off);
    b->t0 = reinterpret_cast<double *>(b->ws + lay.t0_off);
    b->grids = reinterpret_cast<BatchGrid *>(b->ws + lay.grids_off);
    b->items = reinterpret_cast<BatchItem *>(b->ws + lay.items_off);
    b->tile_sig = b->ws + lay.sig_off;
    b->claim = reinterpret_cast<unsigned int *>(b->ws + lay.claim_off);
    for (int k = 0; k < 4; ++k) b->u1[k] = b->ws + lay.u1_off + lay.plane_bytes * (size_t)k;

    // host tables: grid geometry and the (grid, tile) work list, grid by grid, row-major
    std::vector<BatchGrid> hg((size_t)n_grids);
    std::vector<BatchItem> hi;
    hi.reserve((size_t)lay.n_items);
    b->offsets.resize((size_t)n_grids + 1);
    long long off = 0;
    for (int g = 0; g < n_grids; ++g) {
        BatchGrid &G = hg[(size_t)g];
        memset(&G, 0, sizeof G);
        G.off = off;
        G.nx = (int)nx[g];
        G.ny = (int)ny[g];
        G.dr[0] = 1.0 / (double)nx[g];
        G.dr[1] = 1.0 / (double)ny[g];
        G.inv_dr[0] = (float)(1.0 / G.dr[0]);
        G.inv_dr[1] = (float)(1.0 / G.dr[1]);
        const int tx = (G.nx + bx - 1) / bx, ty = (G.ny + rows - 1) / rows;
        G.ntiles = tx * ty;
        G.first_item = (int)hi.size();
        for (int j = 0; j < ty; ++j)
            for (int i = 0; i < tx; ++i) hi.push_back(BatchItem{g, i * bx, j * rows, 0});
        b->offsets[(size_t)g] = off;
        off += nx[g] * ny[g];
    }
    b->offsets[(size_t)n_grids] = off;

    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    BatchLaunch P;
    memset(&P, 0, sizeof P);
    P.tile_x = bx;
    P.tile_y = by;
    P.march = rows;
    int per_sm = 0, n_sm = 0;
    if (e == cudaSuccess)
        e = prec == HYDRO_F32 ? hydro::batch_f32(P, nullptr, 3, true, &per_sm)
                              : hydro::batch_f64(P, nullptr, 3, true, &per_sm);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->grids, hg.data(), sizeof(BatchGrid) * hg.size(),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->items, hi.data(), sizeof(BatchItem) * hi.size(),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        if (b->cap) cudaStreamDestroy(b->cap);
        delete b;
        return bfail(e, "hydro_batch_create");
    }
    long long nb = (long long)(per_sm > 0 ? per_sm : 1) * (n_sm > 0 ? n_sm : 1);
    if (nb > lay.n_items) nb = lay.n_items;
    b->n_blocks = (int)(nb < 1 ? 1 : nb);
    *out = b;
    return HYDRO_OK;
}

int hydro_batch_destroy(hydro_batch_t *b) {
    if (!b) return HYDRO_EINVAL;
    DevGuard dg(b->device);
    for (auto &g : b->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto e : b->events) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return HYDRO_OK;
}

int hydro_batch_offsets(const hydro_batch_t *b, int64_t *offsets_out) {
    if (!b || !offsets_out) return HYDRO_EINVAL;
    for (size_t g = 0; g < b->offsets.size(); ++g) offsets_out[g] = b->offsets[g];
    return HYDRO_OK;
}

int hydro_batch_set_stream(hydro_batch_t *b, void *stream) {
    if (!b) return HYDRO_EINVAL;
    b->stream = static_cast<cudaStream_t>(stream);
    return HYDRO_OK;
}

int hydro_batch_step(hydro_batch_t *b, const hydro_state_t *packed, int32_t n_steps, double t_end,
                     double *t_inout, int32_t *steps_done) {
    if (!b || !state_ok(packed) || n_steps < 0 || t_end != t_end) return HYDRO_EINVAL;
    DevGuard dg(b->device);
    if (t_inout)
        BCK(cudaMemcpyAsync(b->t0, t_inout, sizeof(double) * (size_t)b->n_grids,
                            cudaMemcpyHostToDevice, b->stream));
    const BatchLaunch I = launch_args(b, packed, 0, t_inout ? b->t0 : nullptr, t_end);
    BCK(launch(b, I, b->stream, 0));
    const BatchLaunch C = launch_args(b, packed, 1, nullptr, t_end);
    const BatchLaunch F0 = launch_args(b, packed, 5, nullptr, t_end);
    if (b->profiling) {
        int rc = timed(b, C, 1, 0);
        if (rc) return rc;
        BCK(launch(b, F0, b->stream, 5));
        const BatchLaunch L1 = launch_args(b, packed, 2, nullptr, 0.0);
        const BatchLaunch L2 = launch_args(b, packed, 3, nullptr, 0.0);
        const BatchLaunch F = launch_args(b, packed, 6, nullptr, 0.0);
        for (int i = 0; i < n_steps; ++i) {
            if ((rc = timed(b, L1, 2, 1))) return rc;
            if ((rc = timed(b, L2, 3, 2))) return rc;
            if ((rc = timed(b, F, 6, 0))) return rc;
        }
    } else {
        BCK(launch(b, C, b->stream, 1));
        BCK(launch(b, F0, b->stream, 5));
        int left = n_steps;
        while (left > 0) {
            int chunk = kMaxChunk;
            while (chunk > left) chunk >>= 1;
            cudaGraphExec_t g = nullptr;
            const int rc = get_graph(b, packed, chunk, &g);
            if (rc) return rc;
            BCK(cudaGraphLaunch(g, b->stream));
            left -= chunk;
        }
    }
    if (!t_inout && !steps_done) return HYDRO_OK;
    std::vector<Ctrl> h((size_t)b->n_grids);
    BCK(cudaMemcpyAsync(h.data(), b->ctrl, sizeof(Ctrl) * h.size(), cudaMemcpyDeviceToHost,
                        b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    bool bad = false;
    for (int g = 0; g < b->n_grids; ++g) {
        if (t_inout) t_inout[g] = h[(size_t)g].t;
        if (steps_done) steps_done[g] = h[(size_t)g].steps;
        bad |= (h[(size_t)g].status & hydro::STATUS_NONFINITE) != 0;
    }
    return bad ? HYDRO_ENONFINITE : HYDRO_OK;
}

int hydro_batch_totals(hydro_batch_t *b, const hydro_state_t *packed, double *out) {
    if (!b || !state_ok(packed) || !out) return HYDRO_EINVAL;
    DevGuard dg(b->device);
    const BatchLaunch T = launch_args(b, packed, 4, nullptr, 0.0);
    BCK(launch(b, T, b->stream, 4));
    std::vector<Ctrl> h((size_t)b->n_grids);
    BCK(cudaMemcpyAsync(h.data(), b->ctrl, sizeof(Ctrl) * h.size(), cudaMemcpyDeviceToHost,
                        b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    for (int g = 0; g < b->n_grids; ++g)
        for (int k = 0; k < 5; ++k) out[(size_t)g * 5 + k] = h[(size_t)g].totals[k];
    return HYDRO_OK;
}

int hydro_batch_set_profiling(hydro_batch_t *b, int32_t on) {
    if (!b) return HYDRO_EINVAL;
    b->profiling = on != 0;
    return HYDRO_OK;
}

int hydro_batch_kernel_times(hydro_batch_t *b, double *ms_out, int64_t *launches_out, int32_t n,
                             int32_t reset) {
    if (!b || n < 0 || (n > 0 && (!ms_out || !launches_out))) return HYDRO_EINVAL;
    for (int k = 0; k < n; ++k) {
        ms_out[k] = k < 3 ? b->kms[k] : 0.0;
        launches_out[k] = k < 3 ? b->klaunch[k] : 0;
    }
    if (reset)
        for (int k = 0; k < 3; ++k) {
            b->kms[k] = 0;
            b->klaunch[k] = 0;
        }
    return HYDRO_OK;
}

}  // extern "C"
