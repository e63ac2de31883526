// C ABI of libhydro.so (declared in include/hydro.h): argument checking, the solver context,
// the CUDA-graph cache of step chunks and the per-kernel event timing.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/hydro.h"
#include "hydro_device.cuh"
#include "hydro_internal.h"

using hydro::Ctrl;

namespace {

thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e, const char *what) {
    snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
    return HYDRO_ECUDA;
}

}  // namespace

int hydro::record_cuda_error(cudaError_t e, const char *what) { return cuda_fail(e, what); }

namespace {

#define CK(call)                                            \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

constexpr size_t kAlign = 256;
constexpr int kMaxChunk = 64;  // largest number of steps captured in one graph
constexpr int kGraphSlots = 16;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct GraphEntry {
    int chunk = 0;
    void *planes[5] = {};
    cudaGraphExec_t exec = nullptr;
    unsigned long long last_use = 0;
};

struct Layout {
    size_t ctrl_off, parts_off, u1_off, total;
    size_t v_off;            // manifest V: the primitive planes
    size_t f_off[3];         // manifest F: the face-flux planes of each axis
    size_t plane, fplane[3]; // bytes of one cell plane and of one face plane per axis
    size_t frame_off, frame_plane;  // dim 1, 2: the ghost-cell ring of analytic boundaries
    size_t ex_off[2][2];            // dim 1, 2: exchange buffers per axis and side
};

bool grid_ok(const hydro_grid_t *g, long long *ncell) {
    if (!g || g->dim < 1 || g->dim > 3) return false;
    long long n = 1;
    for (int a = 0; a < g->dim; ++a) {
        // (cell coordinates of a tile plus its halo stay below 2^31)
        if (g->n[a] < 1 || g->n[a] > (1LL << 31) - 1024) return false;
        if (!(g->hi[a] > g->lo[a])) return false;
        n *= g->n[a];
        if (n >= (1LL << 31)) return false;
    }
    *ncell = n;
    return true;
}

// Workspace: control block, totals partials, the stage buffer U1, for the manifest forms
// (manifest: 1 none, 2 V, 3 F in the ABI's spelling) the V planes or the face-flux planes, and
// in dim 1 and 2 the ring of ghost cells analytic and exchange boundaries fill and the exchange
// buffers (O(nx + ny) per plane).
Layout layout_for(int dim, const int64_t n[3], long long ncell, int prec, int manifest = 1) {
    Layout L;
    memset(&L, 0, sizeof L);
    const size_t esz = prec == HYDRO_F32 ? 4 : 8;
    L.ctrl_off = 0;
    L.parts_off = align_up(sizeof(Ctrl));
    L.u1_off = align_up(L.parts_off + sizeof(double) * 5 * hydro::kTotalsParts);
    L.plane = align_up((size_t)ncell * esz);
    L.total = L.u1_off + L.plane * (size_t)(dim + 2);
    if (manifest == 2) {
        L.v_off = L.total;
        L.total += L.plane * (size_t)(dim + 2);
    } else if (manifest == 3) {
        for (int a = 0; a < dim; ++a) {
            const size_t faces = (size_t)ncell / (size_t)n[a] * (size_t)(n[a] + 1);
            L.fplane[a] = align_up(faces * esz);
            L.f_off[a] = L.total;
            L.total += L.fplane[a] * (size_t)(dim + 2);
        }
    }
    if (dim <= 2) {
        L.frame_plane = align_up((size_t)hydro::frame_cells(dim, n[0], dim >= 2 ? n[1] : 1) * esz);
        L.frame_off = L.total;
        L.total += L.frame_plane * (size_t)(dim + 2);
        for (int a = 0; a < dim; ++a)
            for (int side = 0; side < 2; ++side) {
                L.ex_off[a][side] = L.total;
                L.total += align_up((size_t)hydro::exchange_buffer_cells(dim, n[0], dim >= 2 ? n[1] : 1, a) * esz);
            }
    }
    return L;
}

// 0: not compiled; 1: compiled with the default staging depth; 2: with both depths
int tile_compiled(int prec, int dim, int bx, int by) {
    for (int i = 0; i < hydro::kNumTiles; ++i) {
        const hydro::TileShape &t = hydro::kTiles[i];
        if (t.prec == prec && t.dim == dim && t.bx == bx && t.by == by) return t.both_pf ? 2 : 1;
    }
    return 0;
}

// 1 if the tile is also compiled in the manifest forms.
int tile_compiled_manifest(int prec, int dim, int bx, int by) {
    for (int i = 0; i < hydro::kNumTiles; ++i) {
        const hydro::TileShape &t = hydro::kTiles[i];
        if (t.prec == prec && t.dim == dim && t.bx == bx && t.by == by) return t.manifest;
    }
    return 0;
}

// Status code of a control block's status bits: a timed-out device wait first (the step's
// result is void), then a non-finite or non-positive state.
int status_code(unsigned int status) {
    if (status & hydro::STATUS_TIMEOUT) return HYDRO_ETIMEOUT;
    return (status & hydro::STATUS_NONFINITE) ? HYDRO_ENONFINITE : HYDRO_OK;
}

// 1 if the tile is also compiled with TMA plane staging.
int tile_compiled_tma(int prec, int dim, int bx, int by) {
    for (int i = 0; i < hydro::kNumTiles; ++i) {
        const hydro::TileShape &t = hydro::kTiles[i];
        if (t.prec == prec && t.dim == dim && t.bx == bx && t.by == by) return t.tma;
    }
    return 0;
}

// Defaults chosen by measurements on GB300.  dim 3: marching 64 planes; FP32 tile 16 x 8 with
// the three-CTA register budget (the variant tuner's best: 23.03 against 22.82 G
// cell-updates/s for 32 x 8 at 512^3), FP64 tile 32 x 8 (its one compiled 3D tile).  dim 2, FP32: row tiles of 256
// cells marching 16 rows along y, three-CTA budget (2048^2: 28.4 G cell-updates/s against 20.8
// G for the best one-plane tile).  dim 1 and FP64 dim 2: one-plane tiles.  The dt reduction is
// fused into stage 2 for marching tiles; for one-plane tiles, where a CTA updates one tile, the
// separate CFL pass (a fused per-CTA reduction costs more there than one extra read of the
// state).  The split is settled in resolve_variant, once the tile is known.
void default_variant(int prec, int dim, hydro_variant_t *v) {
    v->split = 0;
    v->staging = 1;
    v->occupancy = 2;
    v->march = 0;
    v->manifest = 1;
    if (dim == 1) {
        v->tile_x = 128;
        v->tile_y = 1;
    } else if (dim == 2 && prec == HYDRO_F32) {
        v->tile_x = 256;
        v->tile_y = 1;
        v->march = 16;
        v->occupancy = 3;
    } else if (dim == 3 && prec == HYDRO_F32) {
        v->tile_x = 16;
        v->tile_y = 8;
    } else {
        v->tile_x = 32;
        v->tile_y = 8;
    }
    if (dim == 3) {
        v->march = 64;
        if (prec == HYDRO_F32) v->occupancy = 3;
    }
}

// Default march of a 3D FP32 grid (a variant that names no march).  A CTA advances one tile
// through `march` planes after a short prologue; the launch's (tile, chunk) work items run in
// order, chunk by chunk, so the last chunk's items (shorter where the march does not divide
// the extent) finish the launch.  Among marches 8, 16, 32, ..., 128 whose items fill the GPU's
// resident CTAs at least three times, the one with the least modelled overhead: 0.5 plane per
// chunk (the prologue) plus 0.3 times the last chunk's planes (the launch's tail); 8 when none
// fills them three times.  The weights were fitted to blast runs on GB300 (marches 16-128, n =
// 256 ... 640); G cell-updates/s, the chosen march marked: 512^3 23.14 (64) 23.29 (80) 23.32
// (96*); 448^3 22.90 (64) 23.25 (48*); 384^3 22.62 (64) 22.87 (32*); 256^3 20.56 (64) 21.85
// (16) 22.08 (48*); 128^3 11.56 (64) 15.74 (16) 17.41 (8*).
// The march of `tiles` tiles marching through `extent` planes: among `marches` those whose
// work items fill `slots` resident CTAs `waves` times, the one with the least
// 0.5 chunks + 0.3 (planes of the last chunk); `fallback` when none does.
static int choose_march(long long tiles, long long extent, double slots, double waves,
                        const int *marches, int n_marches, int fallback) {
    int best = 0;
    double best_cost = 0.0;
    for (int i = 0; i < n_marches; ++i) {
        const int m = marches[i];
        const long long chunks = (extent + m - 1) / m;
        if ((double)tiles * (double)chunks < waves * slots) continue;
        const long long last = extent - (chunks - 1) * m;
        const double cost = 0.5 * (double)chunks + 0.3 * (double)last;
        if (best == 0 || cost < best_cost) {
            best = m;
            best_cost = cost;
        }
    }
    return best ? best : fallback;
}

static double resident_slots(const hydro_variant_t &v, int sm_count) {
    int per_sm = v.occupancy * 256 / (v.tile_x * v.tile_y);
    if (per_sm < 1) per_sm = 1;
    return (double)(sm_count > 0 ? sm_count : 1) * per_sm;
}

int default_march_3d(const int64_t n[3], const hydro_variant_t &v, int sm_count) {
    static const int kMarch[] = {8, 16, 32, 48, 64, 80, 96, 112, 128};
    const long long tiles = ((n[0] + v.tile_x - 1) / v.tile_x) * ((n[1] + v.tile_y - 1) / v.tile_y);
    return choose_march(tiles, n[2], resident_slots(v, sm_count), 3.0, kMarch, 9, 8);
}

// Default march of the 2D FP32 row tiles (a variant that names no march), with the same cost
// and marches 8, 16, 32, 64, 128 whose items fill the resident CTAs twice (launches of more
// items than resident CTAs run persistently, so a short last wave costs little); 16 when none
// does.  Measured on GB300 (shear layer, tile 256 x 1, G cell-updates/s, marches 8 / 16 / 32 /
// 64, chosen marked): 4096^2 32.3 / 34.3 / 34.0 / 35.6*; 2048^2 28.4 / 30.2* / 25.6 / 24.9;
// 1024^2 (no march fills them twice) 19.5 / 20.4* / 15.5 / -.
int default_march_rows(const int64_t n[3], const hydro_variant_t &v, int sm_count) {
    static const int kMarch[] = {8, 16, 32, 64, 128};
    const long long strips = (n[0] + v.tile_x - 1) / v.tile_x;
    return choose_march(strips, n[1], resident_slots(v, sm_count), 2.0, kMarch, 5, 16);
}

// Resolve a (possibly partial) variant against the defaults; false if not compiled.
bool resolve_variant(int prec, int dim, const hydro_variant_t *in, hydro_variant_t *out) {
    default_variant(prec, dim, out);
    if (in) {
        const bool tile_given = in->tile_x || in->tile_y;
        if (in->tile_x) out->tile_x = in->tile_x;
        if (in->tile_y) out->tile_y = in->tile_y;
        if (tile_given) {  // the default march and budget belong to the default tile
            hydro_variant_t d;
            default_variant(prec, dim, &d);
            if (out->tile_x != d.tile_x || out->tile_y != d.tile_y) {
                out->march = 0;
                out->occupancy = dim == 3 ? d.occupancy : 2;
            }
        }
        if (in->march) out->march = in->march;
        if (in->split) out->split = in->split;
        if (in->staging) out->staging = in->staging;
        if (in->occupancy) out->occupancy = in->occupancy;
        if (in->manifest) out->manifest = in->manifest;
    }
    // manifest forms: dim 3, tiles compiled with them, look-ahead staging, the default budget
    if (out->manifest < 1 || out->manifest > 3) return false;
    if (out->manifest > 1) {
        const int tm = tile_compiled_manifest(prec, dim, out->tile_x, out->tile_y);
        const int occ = prec == HYDRO_F32 ? 3 : 2;
        if (dim != 3 || !tm || out->staging != 1 || out->occupancy != occ) return false;
    }
    if (in && (in->split < 0 || in->split > 2)) return false;
    if (out->staging < 1 || out->staging > 3) return false;
    // TMA plane staging: 3D FP32 tiles compiled with it, nothing stored between the stage's parts
    if (out->staging == 3 && (dim != 3 || prec != HYDRO_F32 || out->manifest != 1 ||
                              !tile_compiled_tma(prec, dim, out->tile_x, out->tile_y)))
        return false;
    if (out->occupancy != 2 && out->occupancy != 3) return false;
    // marching tiles: dim 3, and the row tiles of dim 2 (tile_y = 1), which march along y
    const bool marching = dim == 3 || (dim == 2 && out->tile_y == 1);
    // split 0 = default: fused for marching tiles, the separate CFL pass for one-plane tiles;
    // internally 0 = fused, 1 = separate
    if (out->split == 0) out->split = marching ? 0 : 1;
    else if (out->split == 2) out->split = 0;
    if (out->occupancy == 3 && (!marching || prec != HYDRO_F32)) return false;
    if (marching && out->march == 0) out->march = dim == 3 ? 64 : 16;
    if (marching && out->march < 1) return false;
    if (!marching) {
        out->march = 1;
        out->staging = 1;  // one plane: nothing to look ahead to
    }
    const int comp = tile_compiled(prec, dim, out->tile_x, out->tile_y);
    return comp == 2 || (comp == 1 && out->staging == 1);
}

}  // namespace

struct hydro_ctx {
    int device = 0;
    int dim = 1;
    int prec = HYDRO_F64;
    long long ncell = 0;
    int n[3] = {1, 1, 1};
    int periodic[3] = {1, 1, 1};
    double dr[3] = {1, 1, 1};
    double gamma = 1.4, cfl = 0.4;
    int order = 2, riemann = 0;
    int ana_axes = 0;        // bit a: axis a has analytic boundaries
    int ex_axes = 0;         // bit a: axis a has exchange boundaries
    void *ex_buf[2][2] = {};
    int ana_kind = 0;        // their solution (hydro_set_analytic); 0 = not set yet
    double ana_theta = 0.0, ana_amp = 0.0;
    double lo[3] = {0, 0, 0};
    void *frame[5] = {};
    hydro_variant_t var = {};
    Layout lay = {};
    unsigned char *ws = nullptr;
    Ctrl *ctrl = nullptr;
    double *parts = nullptr;
    void *u1[5] = {};
    void *vbuf[5] = {};     // manifest V: primitive planes
    void *flux[3][5] = {};  // manifest F: face-flux planes per axis
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only to capture graphs
    cudaStream_t copy = nullptr;  // private stream of hydro_step_host's copies back to the host
    std::vector<cudaEvent_t> slab_events;  // one per stage-2 slab of hydro_step_host
    double *dt_probe = nullptr;            // pinned host: dt after a graph chunk (2 slots)
    cudaEvent_t probe_ev[2] = {nullptr, nullptr};
    GraphEntry graphs[kGraphSlots];
    unsigned long long use_clock = 0;
    bool profiling = false;
    std::vector<cudaEvent_t> events;
    double kms[3] = {0, 0, 0};
    long long klaunch[3] = {0, 0, 0};
};

namespace {

bool state_ok(const hydro_ctx *c, const hydro_state_t *s) {
    if (!s) return false;
    for (int k = 0; k < c->dim + 2; ++k)
        if (!s->plane[k]) return false;
    return true;
}

hydro::StageLaunch stage_args(const hydro_ctx *c, const hydro_state_t *s, int stage) {
    hydro::StageLaunch L;
    memset(&L, 0, sizeof L);
    L.stage = stage;
    for (int k = 0; k < c->dim + 2; ++k) {
        L.uin[k] = stage == 1 ? s->plane[k] : c->u1[k];
        L.ubase[k] = s->plane[k];
        L.uout[k] = stage == 1 ? c->u1[k] : s->plane[k];
    }
    for (int a = 0; a < 3; ++a) {
        L.n[a] = c->n[a];
        L.periodic[a] = c->periodic[a];
        L.dr[a] = c->dr[a];
    }
    L.march = c->var.march;
    L.tile_x = c->var.tile_x;
    L.tile_y = c->var.tile_y;
    L.prefetch = c->var.staging == 2 ? 0 : (c->var.staging == 3 ? 2 : 1);
    L.split = c->var.split;
    L.occupancy = c->var.occupancy;
    L.manifest = c->var.manifest == 2 ? 1 : (c->var.manifest == 3 ? 2 : 0);
    for (int k = 0; k < 5; ++k) L.vbuf[k] = c->vbuf[k];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 5; ++k) L.flux[a][k] = c->flux[a][k];
    L.order = c->order;
    L.riemann = c->riemann;
    L.gamma = c->gamma;
    L.ctrl = c->ctrl;
    L.ana = c->ana_axes | c->ex_axes;  // the axes whose ghost cells come from the ring
    for (int k = 0; k < 5; ++k) L.frame[k] = c->frame[k];
    return L;
}

cudaError_t launch_stage(const hydro_ctx *c, const hydro::StageLaunch &L, cudaStream_t st,
                         bool prepare_only = false) {
    if (c->ana_axes && !prepare_only) {  // the ghost ring at the stage's time first
        hydro::AnalyticLaunch A;
        memset(&A, 0, sizeof A);
        A.prec = c->prec;
        A.dim = c->dim;
        A.nx = c->n[0];
        A.ny = c->n[1];
        A.kind = c->ana_kind;
        for (int d = 0; d < 2; ++d) A.lo[d] = c->lo[d], A.dr[d] = c->dr[d];
        A.gamma = c->gamma;
        A.theta = c->ana_theta;
        A.amp = c->ana_amp;
        for (int k = 0; k < 5; ++k) A.frame[k] = c->frame[k];
        A.ctrl = c->ctrl;
        const cudaError_t e = hydro::launch_analytic_frame(A, L.stage, st);
        if (e != cudaSuccess) return e;
    }
    if (c->ex_axes && !prepare_only) {  // then the exchanged layers of the stage's input
        hydro::ExchangeLaunch X;
        memset(&X, 0, sizeof X);
        X.prec = c->prec;
        X.dim = c->dim;
        X.nx = c->n[0];
        X.ny = c->n[1];
        X.axes = c->ex_axes;
        for (int k = 0; k < 5; ++k) X.uin[k] = L.uin[k], X.frame[k] = c->frame[k];
        for (int a = 0; a < 2; ++a)
            for (int side = 0; side < 2; ++side) X.buf[a][side] = c->ex_buf[a][side];
        const cudaError_t e = hydro::launch_exchange(X, st);
        if (e != cudaSuccess) return e;
    }
    if (c->prec == HYDRO_F64) return hydro::stage_f64(c->dim, L, st, prepare_only);
    switch (c->dim) {
        case 1: return hydro::stage_f32_d1(L, st, prepare_only);
        case 2: return hydro::stage_f32_d2(L, st, prepare_only);
        default: return hydro::stage_f32_d3(L, st, prepare_only);
    }
}

hydro::AuxArgs aux_args(const hydro_ctx *c, const hydro_state_t *s) {
    hydro::AuxArgs A;
    memset(&A, 0, sizeof A);
    A.prec = c->prec;
    A.dim = c->dim;
    A.ncell = c->ncell;
    for (int k = 0; k < c->dim + 2; ++k) A.u[k] = s->plane[k];
    for (int a = 0; a < 3; ++a) A.dr[a] = c->dr[a];
    A.gamma = c->gamma;
    A.ctrl = c->ctrl;
    return A;
}

// Reset the control block for a call starting at t0.
int init_ctrl(hydro_ctx *c, double t0, double t_end) {
    Ctrl init;
    memset(&init, 0, sizeof init);
    init.t = t0;
    init.t_end = t_end;
    init.cfl = c->cfl;
    for (int a = 0; a < 3; ++a) init.dr[a] = c->dr[a];
    CK(cudaMemcpyAsync(c->ctrl, &init, sizeof init, cudaMemcpyHostToDevice, c->stream));
    return HYDRO_OK;
}

// Reset the control block and run the CFL pass: dt of the first step from `s`.
int begin_steps(hydro_ctx *c, const hydro_state_t *s, double t0, double t_end) {
    const int rc = init_ctrl(c, t0, t_end);
    if (rc) return rc;
    if (c->profiling) {
        while (c->events.size() < 2) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            c->events.push_back(e);
        }
        CK(cudaEventRecord(c->events[0], c->stream));
        CK(hydro::launch_cfl(aux_args(c, s), c->stream));
        CK(cudaEventRecord(c->events[1], c->stream));
        CK(cudaEventSynchronize(c->events[1]));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, c->events[0], c->events[1]));
        c->kms[0] += ms;
        c->klaunch[0] += 1;
        return HYDRO_OK;
    }
    CK(hydro::launch_cfl(aux_args(c, s), c->stream));
    return HYDRO_OK;
}

int get_graph(hydro_ctx *c, const hydro_state_t *s, int chunk, cudaGraphExec_t *out) {
    GraphEntry *free_slot = nullptr, *oldest = &c->graphs[0];
    for (auto &g : c->graphs) {
        if (g.exec && g.chunk == chunk) {
            bool same = true;
            for (int k = 0; k < c->dim + 2; ++k) same &= g.planes[k] == s->plane[k];
            if (same) {
                g.last_use = ++c->use_clock;
                *out = g.exec;
                return HYDRO_OK;
            }
        }
        if (!g.exec && !free_slot) free_slot = &g;
        if (g.last_use < oldest->last_use) oldest = &g;
    }
    GraphEntry *slot = free_slot ? free_slot : oldest;
    if (slot->exec) {
        cudaGraphExecDestroy(slot->exec);
        slot->exec = nullptr;
    }
    const hydro::StageLaunch L1 = stage_args(c, s, 1), L2 = stage_args(c, s, 2);
    const hydro::AuxArgs C = aux_args(c, s);
    CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    for (int i = 0; i < chunk && le == cudaSuccess; ++i) {
        le = launch_stage(c, L1, c->cap);
        if (le == cudaSuccess) le = launch_stage(c, L2, c->cap);
        if (le == cudaSuccess && c->var.split) le = hydro::launch_cfl(C, c->cap, /*advance=*/true);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(c->cap, &graph);
    if (le != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(le, "stage launch during capture");
    }
    if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate");
    slot->exec = exec;
    slot->chunk = chunk;
    for (int k = 0; k < 5; ++k) slot->planes[k] = s->plane[k];
    slot->last_use = ++c->use_clock;
    *out = exec;
    return HYDRO_OK;
}

// Profiling: the steps launched one by one with CUDA events around each launch, in batches of
// up to kMaxChunk steps (the events are reused); after each batch the times are collected and
// the stepping stops once no further step is to be taken (dt = 0).
int run_steps_profiled(hydro_ctx *c, const hydro_state_t *s, int n) {
    const hydro::StageLaunch L1 = stage_args(c, s, 1), L2 = stage_args(c, s, 2);
    const hydro::AuxArgs C = aux_args(c, s);
    const int per = c->var.split ? 3 : 2;  // launches per step
    const size_t need = (size_t)per * kMaxChunk + 1;
    while (c->events.size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        c->events.push_back(e);
    }
    for (int done = 0; done < n;) {
        const int b = n - done < kMaxChunk ? n - done : kMaxChunk;
        CK(cudaEventRecord(c->events[0], c->stream));
        for (int i = 0; i < b; ++i) {
            const int e0 = per * i;
            CK(launch_stage(c, L1, c->stream));
            CK(cudaEventRecord(c->events[e0 + 1], c->stream));
            CK(launch_stage(c, L2, c->stream));
            CK(cudaEventRecord(c->events[e0 + 2], c->stream));
            if (c->var.split) {
                CK(hydro::launch_cfl(C, c->stream, /*advance=*/true));
                CK(cudaEventRecord(c->events[e0 + 3], c->stream));
            }
        }
        CK(cudaMemcpyAsync(&c->dt_probe[0], &c->ctrl->dt, sizeof(double), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (int i = 0; i < b; ++i) {
            const int e0 = per * i;
            for (int k = 0; k < per; ++k) {
                float m = 0;
                CK(cudaEventElapsedTime(&m, c->events[e0 + k], c->events[e0 + k + 1]));
                const int kind = k < 2 ? k + 1 : 0;  // stage 1, stage 2, then the CFL pass
                c->kms[kind] += m;
                c->klaunch[kind] += 1;
            }
        }
        done += b;
        if (!(c->dt_probe[0] > 0.0)) break;
    }
    return HYDRO_OK;
}

// stop_early: the caller synchronises at the end anyway, so after each graph chunk the dt of
// the next step is copied to the host, and once it is 0 (t_end reached, or a failed step) the
// remaining chunks are not launched.  The check lags one chunk, so the GPU never waits on it:
// at most one chunk of steps that return at once is launched after the last real step.
int run_steps(hydro_ctx *c, const hydro_state_t *s, int n, bool stop_early = false) {
    if (n <= 0) return HYDRO_OK;
    if (c->profiling) return run_steps_profiled(c, s, n);
    int left = n, k = 0;
    while (left > 0) {
        int chunk = kMaxChunk;
        while (chunk > left) chunk >>= 1;
        cudaGraphExec_t g = nullptr;
        int rc = get_graph(c, s, chunk, &g);
        if (rc) return rc;
        CK(cudaGraphLaunch(g, c->stream));
        left -= chunk;
        if (stop_early && left > 0) {
            const int slot = k & 1;
            CK(cudaMemcpyAsync(&c->dt_probe[slot], &c->ctrl->dt, sizeof(double),
                               cudaMemcpyDeviceToHost, c->stream));
            CK(cudaEventRecord(c->probe_ev[slot], c->stream));
            if (k > 0) {  // the previous chunk's probe (the current chunk is already queued)
                CK(cudaEventSynchronize(c->probe_ev[slot ^ 1]));
                if (!(c->dt_probe[slot ^ 1] > 0.0)) break;
            }
            ++k;
        }
    }
    return HYDRO_OK;
}

int finish_steps(hydro_ctx *c, double *t_inout, int32_t *steps_done) {
    if (!t_inout && !steps_done) return HYDRO_OK;
    Ctrl h;
    CK(cudaMemcpyAsync(&h, c->ctrl, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (t_inout) *t_inout = h.t;
    if (steps_done) *steps_done = h.steps;
    return status_code(h.status);
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

int hydro_version(void) { return HYDRO_ABI_VERSION; }

const char *hydro_strerror(int status) {
    switch (status) {
        case HYDRO_OK: return "ok";
        case HYDRO_EINVAL: return "invalid argument";
        case HYDRO_ECUDA: return "CUDA runtime error";
        case HYDRO_ENONFINITE: return "non-finite value or non-positive density/pressure";
        case HYDRO_ETIMEOUT: return "bounded device wait timed out";
        case HYDRO_EUNSUPPORTED: return "no kernel compiled for this request";
        default: return "unknown status";
    }
}

const char *hydro_last_cuda_error(void) { return g_cuda_err; }

int hydro_variant_supported(int32_t prec, int32_t dim, const hydro_variant_t *variant) {
    if (prec != HYDRO_F32 && prec != HYDRO_F64) return 0;
    if (dim < 1 || dim > 3) return 0;
    hydro_variant_t v;
    return resolve_variant(prec, dim, variant, &v) ? 1 : 0;
}

int hydro_workspace_bytes(const hydro_grid_t *grid, int32_t prec, size_t *bytes_out) {
    long long ncell = 0;
    if (!bytes_out || !grid_ok(grid, &ncell)) return HYDRO_EINVAL;
    if (prec != HYDRO_F32 && prec != HYDRO_F64) return HYDRO_EINVAL;
    *bytes_out = layout_for(grid->dim, grid->n, ncell, prec).total;
    return HYDRO_OK;
}

int hydro_workspace_bytes_variant(const hydro_grid_t *grid, int32_t prec,
                                  const hydro_variant_t *variant, size_t *bytes_out) {
    long long ncell = 0;
    if (!bytes_out || !grid_ok(grid, &ncell)) return HYDRO_EINVAL;
    if (prec != HYDRO_F32 && prec != HYDRO_F64) return HYDRO_EINVAL;
    hydro_variant_t var;
    if (!resolve_variant(prec, grid->dim, variant, &var)) return HYDRO_EUNSUPPORTED;
    *bytes_out = layout_for(grid->dim, grid->n, ncell, prec, var.manifest).total;
    return HYDRO_OK;
}

int hydro_create(const hydro_grid_t *grid, double gamma, const int32_t bc[3], int32_t prec,
                 double cfl, const hydro_variant_t *variant, void *workspace,
                 size_t workspace_bytes, void *stream, hydro_ctx_t **out) {
    if (!out) return HYDRO_EINVAL;
    *out = nullptr;
    long long ncell = 0;
    if (!grid_ok(grid, &ncell) || !bc || !workspace) return HYDRO_EINVAL;
    if (prec != HYDRO_F32 && prec != HYDRO_F64) return HYDRO_EINVAL;
    if (!(gamma > 1.0) || !(gamma < 1e300) || !(cfl > 0.0) || !(cfl < 1e300)) return HYDRO_EINVAL;
    int ana_axes = 0, ex_axes = 0;
    for (int a = 0; a < grid->dim; ++a) {
        if (bc[a] < HYDRO_BC_PERIODIC || bc[a] > HYDRO_BC_EXCHANGE) return HYDRO_EINVAL;
        if (bc[a] == HYDRO_BC_ANALYTIC) ana_axes |= 1 << a;
        if (bc[a] == HYDRO_BC_EXCHANGE) {
            if (grid->n[a] < 2) return HYDRO_EUNSUPPORTED;  // two layers to exchange
            ex_axes |= 1 << a;
        }
    }
    if (((uintptr_t)workspace) % kAlign) return HYDRO_EINVAL;
    hydro_variant_t var;
    if (!resolve_variant(prec, grid->dim, variant, &var)) return HYDRO_EUNSUPPORTED;
    if (ana_axes | ex_axes) {  // one-plane tiles of dim 1 and 2 read the ghost ring
        if (grid->dim == 3) return HYDRO_EUNSUPPORTED;
        const bool tile_given = variant && (variant->tile_x || variant->tile_y);
        if (grid->dim == 2 && !tile_given) {  // the default 2D FP32 tile marches: take 32 x 8
            hydro_variant_t w = variant ? *variant : hydro_variant_t{};
            w.tile_x = 32;
            w.tile_y = 8;
            if (!resolve_variant(prec, grid->dim, &w, &var)) return HYDRO_EUNSUPPORTED;
        }
        if (grid->dim == 2 && var.tile_y == 1) return HYDRO_EUNSUPPORTED;
        if (hydro::frame_cells(grid->dim, grid->n[0], grid->dim >= 2 ? grid->n[1] : 1) >= (1LL << 31))
            return HYDRO_EUNSUPPORTED;  // the ring's int indices
    }
    const bool rows = grid->dim == 2 && var.tile_y == 1;
    if ((grid->dim == 3 || rows) && prec == HYDRO_F32 && !(variant && variant->march)) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            var.march = rows ? default_march_rows(grid->n, var, sms)
                             : default_march_3d(grid->n, var, sms);
    }
    const Layout lay = layout_for(grid->dim, grid->n, ncell, prec, var.manifest);
    if (workspace_bytes < lay.total) return HYDRO_EINVAL;
    // grid-dimension limits of the stage launch
    const bool marching = grid->dim == 3 || (grid->dim == 2 && var.tile_y == 1);
    if ((grid->dim == 3 || (grid->dim == 2 && !marching)) &&
        (grid->n[1] + var.tile_y - 1) / var.tile_y > 65535)
        return HYDRO_EUNSUPPORTED;
    if (marching && (grid->n[grid->dim - 1] + var.march - 1) / var.march > 65535)
        return HYDRO_EUNSUPPORTED;

    hydro_ctx *c = new (std::nothrow) hydro_ctx();
    if (!c) return HYDRO_EINVAL;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return cuda_fail(cudaGetLastError(), "cudaGetDevice");
    }
    c->dim = grid->dim;
    c->prec = prec;
    c->ncell = ncell;
    for (int a = 0; a < 3; ++a) {
        const bool act = a < grid->dim;
        c->n[a] = act ? (int)grid->n[a] : 1;
        c->periodic[a] = act ? (bc[a] == HYDRO_BC_PERIODIC) : 1;
        c->dr[a] = act ? (grid->hi[a] - grid->lo[a]) / (double)grid->n[a] : 1.0;
        c->lo[a] = act ? grid->lo[a] : 0.0;
    }
    c->ana_axes = ana_axes;
    c->ex_axes = ex_axes;
    if (marching && var.march > c->n[c->dim - 1]) var.march = c->n[c->dim - 1];
    c->gamma = gamma;
    c->cfl = cfl;
    c->var = var;
    c->lay = lay;
    c->ws = static_cast<unsigned char *>(workspace);
    c->ctrl = reinterpret_cast<Ctrl *>(c->ws + lay.ctrl_off);
    c->parts = reinterpret_cast<double *>(c->ws + lay.parts_off);
    const size_t plane = align_up((size_t)ncell * (prec == HYDRO_F32 ? 4 : 8));
    for (int k = 0; k < c->dim + 2; ++k) c->u1[k] = c->ws + lay.u1_off + plane * (size_t)k;
    if (var.manifest == 2)
        for (int k = 0; k < c->dim + 2; ++k) c->vbuf[k] = c->ws + lay.v_off + lay.plane * (size_t)k;
    if (var.manifest == 3)
        for (int a = 0; a < c->dim; ++a)
            for (int k = 0; k < c->dim + 2; ++k)
                c->flux[a][k] = c->ws + lay.f_off[a] + lay.fplane[a] * (size_t)k;
    if (c->dim <= 2) {
        for (int k = 0; k < c->dim + 2; ++k) c->frame[k] = c->ws + lay.frame_off + lay.frame_plane * (size_t)k;
        for (int a = 0; a < c->dim; ++a)
            for (int side = 0; side < 2; ++side) c->ex_buf[a][side] = c->ws + lay.ex_off[a][side];
    }
    c->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&c->dt_probe), 2 * sizeof(double), 0);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&c->probe_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (c->cap) cudaStreamDestroy(c->cap);
        if (c->copy) cudaStreamDestroy(c->copy);
        if (c->dt_probe) cudaFreeHost(c->dt_probe);
        for (auto ev : c->probe_ev)
            if (ev) cudaEventDestroy(ev);
        delete c;
        return cuda_fail(e, "context streams and events");
    }
    hydro_state_t dummy;
    memset(&dummy, 0, sizeof dummy);
    e = launch_stage(c, stage_args(c, &dummy, 1), c->stream, /*prepare_only=*/true);
    if (e != cudaSuccess) {
        cudaStreamDestroy(c->cap);
        cudaStreamDestroy(c->copy);
        cudaFreeHost(c->dt_probe);
        for (auto ev : c->probe_ev) cudaEventDestroy(ev);
        delete c;
        return cuda_fail(e, "stage kernel attributes");
    }
    *out = c;
    return HYDRO_OK;
}

int hydro_get_variant(const hydro_ctx_t *c, hydro_variant_t *out) {
    if (!c || !out) return HYDRO_EINVAL;
    *out = c->var;
    out->split = c->var.split ? 1 : 2;  // the ABI's spelling: 1 separate CFL pass, 2 fused
    return HYDRO_OK;
}

int hydro_destroy(hydro_ctx_t *c) {
    if (!c) return HYDRO_EINVAL;
    DeviceGuard dg(c->device);
    for (auto &g : c->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto e : c->events) cudaEventDestroy(e);
    for (auto e : c->slab_events) cudaEventDestroy(e);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->copy) cudaStreamDestroy(c->copy);
    if (c->dt_probe) cudaFreeHost(c->dt_probe);
    for (auto ev : c->probe_ev)
        if (ev) cudaEventDestroy(ev);
    delete c;
    return HYDRO_OK;
}

int hydro_set_scheme(hydro_ctx_t *c, int32_t order, int32_t riemann) {
    if (!c || (order != 1 && order != 2) || (riemann != 0 && riemann != 1)) return HYDRO_EINVAL;
    if (order == c->order && riemann == c->riemann) return HYDRO_OK;
    DeviceGuard dg(c->device);
    // captured graphs hold the old kernel arguments
    for (auto &g : c->graphs)
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            g.chunk = 0;
        }
    c->order = order;
    c->riemann = riemann;
    return HYDRO_OK;
}

int hydro_set_analytic(hydro_ctx_t *c, int32_t kind, double theta, double amplitude) {
    if (!c || kind < HYDRO_ANALYTIC_ENTROPY_WAVE || kind > HYDRO_ANALYTIC_SHOCK_TUBE) return HYDRO_EINVAL;
    if (!(theta == theta) || !(fabs(theta) < 1e6) || !(fabs(amplitude) < 1e300)) return HYDRO_EINVAL;
    if (!c->ana_axes) return HYDRO_EINVAL;
    DeviceGuard dg(c->device);
    for (auto &g : c->graphs)  // captured graphs hold the old fill arguments
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            g.chunk = 0;
        }
    c->ana_kind = kind;
    c->ana_theta = theta;
    c->ana_amp = amplitude;
    return HYDRO_OK;
}

int hydro_set_stream(hydro_ctx_t *c, void *stream) {
    if (!c) return HYDRO_EINVAL;
    c->stream = static_cast<cudaStream_t>(stream);
    return HYDRO_OK;
}

int hydro_step(hydro_ctx_t *c, const hydro_state_t *state, int32_t n_steps, double t_end,
               double *t_inout, int32_t *steps_done) {
    if (!c || !state_ok(c, state) || n_steps < 0) return HYDRO_EINVAL;
    if (t_end != t_end) return HYDRO_EINVAL;
    if (c->ana_axes && !c->ana_kind) return HYDRO_EINVAL;  // no analytic solution set
    DeviceGuard dg(c->device);
    const double t0 = t_inout ? *t_inout : 0.0;
    if (t0 != t0) return HYDRO_EINVAL;
    int rc = begin_steps(c, state, t0, t_end);
    if (rc) return rc;
    rc = run_steps(c, state, n_steps, /*stop_early=*/t_inout || steps_done);
    if (rc) return rc;
    return finish_steps(c, t_inout, steps_done);
}

// Copy the byte range [off, off + bytes) of each of n planes (dst[k] <- src[k]).  When both
// sides' planes are equally spaced (one tensor of planes), one strided copy moves all of them.
static cudaError_t copy_planes(void *const dst[5], const void *const src[5], int n, size_t off,
                               size_t bytes, cudaMemcpyKind kind, cudaStream_t st) {
    bool even = n > 1;
    const long long dp = n > 1 ? (long long)((const char *)dst[1] - (const char *)dst[0]) : 0;
    const long long sp = n > 1 ? (long long)((const char *)src[1] - (const char *)src[0]) : 0;
    for (int k = 2; k < n && even; ++k)
        even = (const char *)dst[k] - (const char *)dst[k - 1] == dp &&
               (const char *)src[k] - (const char *)src[k - 1] == sp;
    // positive pitches of at least the row width and below 2 GiB (the pitch limit of copies)
    even = even && dp >= (long long)bytes && sp >= (long long)bytes && dp < (1LL << 31) &&
           sp < (1LL << 31);
    if (even)
        return cudaMemcpy2DAsync(static_cast<char *>(dst[0]) + off, (size_t)dp,
                                 static_cast<const char *>(src[0]) + off, (size_t)sp, bytes,
                                 (size_t)n, kind, st);
    for (int k = 0; k < n; ++k) {
        const cudaError_t e = cudaMemcpyAsync(static_cast<char *>(dst[k]) + off,
                                              static_cast<const char *>(src[k]) + off, bytes,
                                              kind, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The last step of hydro_step_host in dim 3, with the copy back overlapped: stages 1 and 2
// slab by slab (groups of march chunks along z, the dt reduction left to a CFL pass), each
// slab's finished planes copied to the host on the private copy stream while the next slabs
// compute; the CFL pass (status, time, next dt) runs after the last slab.  A slab's U is final
// when its stage-2 launch ends: stage 2 writes only its own cells and reads other slabs' U1,
// not U.  Returns with the copy stream joined into the context's stream.
static int last_step_overlapped(hydro_ctx *c, const hydro_state_t *s, void *const host_out[5]) {
    const int march = c->var.march;
    const int nchunks = (c->n[2] + march - 1) / march;
    const int nslabs = nchunks < 8 ? nchunks : 8;
    while ((int)c->slab_events.size() < nslabs + 1) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c->slab_events.push_back(e);
    }
    const size_t esz = c->prec == HYDRO_F32 ? 4 : 8;
    const size_t plane_cells = (size_t)c->n[0] * (size_t)c->n[1];
    auto chunk0 = [&](int i) { return (int)((long long)nchunks * i / nslabs); };
    // Stage 1 runs by slabs too, interleaved so that slab i of stage 2 (which overwrites U0 in
    // place) follows every stage-1 slab that reads U0 planes of slab i (its neighbours, the last
    // slab through the periodic wrap): last, 0, 1, then stage 2 of slab i after stage 1 of slab
    // i + 1.  The copy back of the first slab can then start after two stage-1 slabs instead of
    // the whole of stage 1.
    hydro::StageLaunch L1 = stage_args(c, s, 1);
    auto stage1_slab = [&](int i) -> cudaError_t {
        L1.zchunk0 = chunk0(i);
        L1.zchunks = chunk0(i + 1) - chunk0(i);
        return launch_stage(c, L1, c->stream);
    };
    // (every slab at least two planes thick, so that the U0 planes a stage-1 slab reads lie in
    // its neighbouring slabs; otherwise stage 1 runs whole first)
    const bool interleave = march >= 2 && c->n[2] - chunk0(nslabs - 1) * march >= 2;
    if (interleave) {
        CK(stage1_slab(nslabs - 1));
        if (nslabs > 1) CK(stage1_slab(0));
    } else {
        CK(launch_stage(c, stage_args(c, s, 1), c->stream));
    }
    hydro::StageLaunch L2 = stage_args(c, s, 2);
    L2.split = 1;
    for (int i = 0; i < nslabs; ++i) {
        if (interleave && i + 1 <= nslabs - 2) CK(stage1_slab(i + 1));
        const int k0 = chunk0(i);
        const int k1 = chunk0(i + 1);
        L2.zchunk0 = k0;
        L2.zchunks = k1 - k0;
        CK(launch_stage(c, L2, c->stream));
        CK(cudaEventRecord(c->slab_events[(size_t)i], c->stream));
        CK(cudaStreamWaitEvent(c->copy, c->slab_events[(size_t)i], 0));
        const int z0 = k0 * march, z1 = k1 * march < c->n[2] ? k1 * march : c->n[2];
        const size_t off = (size_t)z0 * plane_cells * esz, bytes = (size_t)(z1 - z0) * plane_cells * esz;
        CK(copy_planes(host_out, s->plane, c->dim + 2, off, bytes, cudaMemcpyDeviceToHost, c->copy));
    }
    CK(hydro::launch_cfl(aux_args(c, s), c->stream, /*advance=*/true));
    CK(cudaEventRecord(c->slab_events[(size_t)nslabs], c->copy));
    CK(cudaStreamWaitEvent(c->stream, c->slab_events[(size_t)nslabs], 0));
    return HYDRO_OK;
}

// The copy in of hydro_step_host in dim 3 with the CFL pass overlapped: the state comes in
// z-slab by z-slab on the private copy stream, and each slab's part of the CFL pass runs on the
// context's stream as soon as the slab has arrived, so only the last part follows the copy.
// The parts share one running maximum; the last CTA of all of them sets dt.
static int copy_in_overlapped(hydro_ctx *c, const hydro_state_t *dev,
                              const void *const host_in[5], double t0, double t_end) {
    const int nslabs = c->n[2] < 8 ? c->n[2] : 8;
    while ((int)c->slab_events.size() < nslabs + 1) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c->slab_events.push_back(e);
    }
    const int rc = init_ctrl(c, t0, t_end);
    if (rc) return rc;
    // the copies start after the stream's earlier work on the state
    CK(cudaEventRecord(c->slab_events[(size_t)nslabs], c->stream));
    CK(cudaStreamWaitEvent(c->copy, c->slab_events[(size_t)nslabs], 0));
    const size_t esz = c->prec == HYDRO_F32 ? 4 : 8;
    const long long plane = (long long)c->n[0] * c->n[1];
    hydro::AuxArgs A = aux_args(c, dev);
    unsigned total = 0;
    for (int i = 0; i < nslabs; ++i) {
        const long long z0 = (long long)c->n[2] * i / nslabs, z1 = (long long)c->n[2] * (i + 1) / nslabs;
        total += hydro::cfl_blocks((z1 - z0) * plane);
    }
    A.total_blocks = total;
    for (int i = 0; i < nslabs; ++i) {
        const long long z0 = (long long)c->n[2] * i / nslabs, z1 = (long long)c->n[2] * (i + 1) / nslabs;
        const size_t off = (size_t)(z0 * plane) * esz, bytes = (size_t)((z1 - z0) * plane) * esz;
        CK(copy_planes(dev->plane, host_in, c->dim + 2, off, bytes, cudaMemcpyHostToDevice, c->copy));
        CK(cudaEventRecord(c->slab_events[(size_t)i], c->copy));
        CK(cudaStreamWaitEvent(c->stream, c->slab_events[(size_t)i], 0));
        A.first = z0 * plane;
        A.ncell = (z1 - z0) * plane;
        CK(hydro::launch_cfl(A, c->stream));
    }
    return HYDRO_OK;
}

// hydro_step_host and hydro_step_host_async: the copy in, the steps and the copy back,
// enqueued on the context's stream (and its private copy stream).  sync: stop launching once
// no further step is to be taken, then wait for the stream and return the time, the steps
// taken and the status; otherwise enqueue everything and return.
static int step_host_impl(hydro_ctx_t *c, const hydro_state_t *dev, const void *const host_in[5],
                          void *const host_out[5], int32_t n_steps, double t_end, double t,
                          bool sync, double *t_out, int32_t *steps_done) {
    if (!c || !state_ok(c, dev) || !host_in || !host_out || n_steps < 0) return HYDRO_EINVAL;
    if (t_end != t_end || t != t) return HYDRO_EINVAL;
    if (c->ana_axes && !c->ana_kind) return HYDRO_EINVAL;
    for (int k = 0; k < c->dim + 2; ++k)
        if (!host_in[k] || !host_out[k]) return HYDRO_EINVAL;
    DeviceGuard dg(c->device);
    const size_t bytes = (size_t)c->ncell * (c->prec == HYDRO_F32 ? 4 : 8);
    int32_t done = 0;
    // dim 3 outside profiling: the copy in overlaps the CFL pass and the last step's stage 2
    // overlaps the copy back
    const bool overlap = c->dim == 3 && n_steps >= 1 && !c->profiling && c->var.manifest == 1;
    int rc;
    if (overlap) {
        rc = copy_in_overlapped(c, dev, host_in, t, t_end);
    } else {
        for (int k = 0; k < c->dim + 2; ++k)
            CK(cudaMemcpyAsync(dev->plane[k], host_in[k], bytes, cudaMemcpyHostToDevice, c->stream));
        rc = begin_steps(c, dev, t, t_end);
    }
    if (!rc) rc = run_steps(c, dev, overlap ? n_steps - 1 : n_steps, /*stop_early=*/sync);
    if (!rc && overlap) rc = last_step_overlapped(c, dev, host_out);
    if (rc) return rc;
    if (!overlap)
        for (int k = 0; k < c->dim + 2; ++k)
            CK(cudaMemcpyAsync(host_out[k], dev->plane[k], bytes, cudaMemcpyDeviceToHost, c->stream));
    if (!sync) return HYDRO_OK;
    rc = finish_steps(c, &t, &done);
    if (t_out) *t_out = t;
    if (steps_done) *steps_done = done;
    return rc;
}

int hydro_step_host(hydro_ctx_t *c, const hydro_state_t *dev, const void *const host_in[5],
                    void *const host_out[5], int32_t n_steps, double t_end, double *t_inout,
                    int32_t *steps_done) {
    return step_host_impl(c, dev, host_in, host_out, n_steps, t_end, t_inout ? *t_inout : 0.0,
                          /*sync=*/true, t_inout, steps_done);
}

int hydro_step_host_async(hydro_ctx_t *c, const hydro_state_t *dev, const void *const host_in[5],
                          void *const host_out[5], int32_t n_steps, double t_end, double t) {
    return step_host_impl(c, dev, host_in, host_out, n_steps, t_end, t, /*sync=*/false, nullptr,
                          nullptr);
}

int hydro_cfl_dt(hydro_ctx_t *c, const hydro_state_t *state, double *dt_out) {
    if (!c || !state_ok(c, state) || !dt_out) return HYDRO_EINVAL;
    DeviceGuard dg(c->device);
    int rc = begin_steps(c, state, 0.0, 0.0);
    if (rc) return rc;
    Ctrl h;
    CK(cudaMemcpyAsync(&h, c->ctrl, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *dt_out = h.dt;
    return status_code(h.status);
}

int hydro_totals(hydro_ctx_t *c, const hydro_state_t *state, double out[5]) {
    if (!c || !state_ok(c, state) || !out) return HYDRO_EINVAL;
    DeviceGuard dg(c->device);
    double vol = 1.0;
    for (int a = 0; a < c->dim; ++a) vol *= c->dr[a];
    CK(hydro::launch_totals(aux_args(c, state), c->parts, hydro::kTotalsParts, vol, c->stream));
    CK(cudaMemcpyAsync(out, c->ctrl->totals, sizeof(double) * 5, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return HYDRO_OK;
}

int hydro_status(hydro_ctx_t *c) {
    if (!c) return HYDRO_EINVAL;
    DeviceGuard dg(c->device);
    unsigned int st = 0;
    CK(cudaMemcpyAsync(&st, &c->ctrl->status, sizeof st, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return status_code(st);
}

static int convert(int32_t dim, int64_t ncell, double gamma, int32_t prec, const hydro_state_t *in,
                   const hydro_state_t *out, void *stream, int to_cons) {
    if (dim < 1 || dim > 3 || ncell < 0 || !in || !out || !(gamma > 1.0)) return HYDRO_EINVAL;
    if (prec != HYDRO_F32 && prec != HYDRO_F64) return HYDRO_EINVAL;
    if (ncell == 0) return HYDRO_OK;
    hydro::AuxArgs A;
    memset(&A, 0, sizeof A);
    A.prec = prec;
    A.dim = dim;
    A.ncell = ncell;
    A.gamma = gamma;
    for (int k = 0; k < dim + 2; ++k) {
        if (!in->plane[k] || !out->plane[k]) return HYDRO_EINVAL;
        A.u[k] = in->plane[k];
        A.out[k] = out->plane[k];
    }
    CK(hydro::launch_convert(A, to_cons, static_cast<cudaStream_t>(stream)));
    return HYDRO_OK;
}

int hydro_prim_to_cons(int32_t dim, int64_t ncell, double gamma, int32_t prec,
                       const hydro_state_t *prim_in, const hydro_state_t *cons_out, void *stream) {
    return convert(dim, ncell, gamma, prec, prim_in, cons_out, stream, 1);
}

int hydro_cons_to_prim(int32_t dim, int64_t ncell, double gamma, int32_t prec,
                       const hydro_state_t *cons_in, const hydro_state_t *prim_out, void *stream) {
    return convert(dim, ncell, gamma, prec, cons_in, prim_out, stream, 0);
}

int hydro_set_profiling(hydro_ctx_t *c, int32_t on) {
    if (!c) return HYDRO_EINVAL;
    c->profiling = on != 0;
    return HYDRO_OK;
}

int hydro_kernel_times(hydro_ctx_t *c, double *ms_out, int64_t *launches_out, int32_t n,
                       int32_t reset) {
    if (!c || n < 0 || (n > 0 && (!ms_out || !launches_out))) return HYDRO_EINVAL;
    DeviceGuard dg(c->device);
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < n && k < 3; ++k) {
        ms_out[k] = c->kms[k];
        launches_out[k] = c->klaunch[k];
    }
    for (int k = 3; k < n; ++k) {
        ms_out[k] = 0;
        launches_out[k] = 0;
    }
    if (reset)
        for (int k = 0; k < 3; ++k) {
            c->kms[k] = 0;
            c->klaunch[k] = 0;
        }
    return HYDRO_OK;
}

}  // extern "C"
