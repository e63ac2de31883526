/*
 * hydro.h -- C ABI of libhydro.so: the second-order finite-volume step of the compressible
 * Euler equations (Paraiso, arXiv:1204.4779, section 4.1 "The Target Program") on one GB300
 * (sm_103a), FP32 or FP64.
 *
 * The step (section 4.1): with V = (rho, v_a, p) the primitive and U = (rho, m_a, E) the
 * conserved variables (Eqs. eqPrimitiveVars, eqConservedVars),
 *     F0_a = Flux_a(U0);   U1 = AddFlux(dt/2, F0, U0);
 *     F1_a = Flux_a(U1);   U2 = AddFlux(dt,   F1, U0),
 * where Flux_a recovers V from U, reconstructs face values with the piecewise-linear MinBee
 * limiter (Eqs. eqInterpolateV, eqInterpolateSingle) and evaluates the HLLC Riemann solver
 * on each face, and AddFlux is the conservative update of Eq. eqAddFlux.  dt comes from the
 * CFL condition, dt = cfl / max_i sum_a (|v_a| + c_s) / dr_a with c_s = sqrt(gamma p / rho),
 * evaluated on the state at the start of each step (the paper says only that dt is
 * "determined by the CFL condition"; this is the reading used).
 *
 * Layout of a state: structure of arrays, dim+2 planes (rho, m_x, [m_y, [m_z]], E), each a
 * dense n[0]*n[1]*n[2] array of the context's element type with x fastest, then y, then z.
 * Planes live in device memory owned by the caller; no ghost padding.
 *
 * Ownership: the library never allocates device memory.  The caller allocates the state
 * planes and one workspace block of hydro_workspace_bytes() bytes (256-byte aligned) and keeps
 * both alive while the context uses them.  The context owns only host memory, CUDA graphs,
 * events and one private capture stream.
 *
 * Errors: every call returns an int status (HYDRO_OK = 0); no call aborts or throws.
 * HYDRO_ENONFINITE means a step produced (or was given) a non-finite value, rho <= 0 or
 * p <= 0; the state then holds the output of that step and no further step runs in the call.
 *
 * Streams: every call is ordered on the context's stream (set at create or by
 * hydro_set_stream).  Calls that return host values (hydro_cfl_dt, hydro_totals, hydro_step
 * with t_inout or steps_done, hydro_step_host, hydro_status) synchronise that stream.
 * A context must not be used from two host threads at once.
 */
#ifndef HYDRO_H
#define HYDRO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HYDRO_ABI_VERSION 1

enum {
    HYDRO_OK = 0,
    HYDRO_EINVAL = 1,     /* bad argument: null pointer, bad grid/gamma/cfl/precision/variant,
                             workspace too small or misaligned */
    HYDRO_ECUDA = 2,      /* a CUDA runtime call failed (hydro_last_cuda_error tells which) */
    HYDRO_ENONFINITE = 3, /* non-finite value, rho <= 0 or p <= 0 seen on the device */
    HYDRO_ETIMEOUT = 4,   /* a bounded device-side wait gave up: a TMA-staged stage kernel
                             (variant staging 3) did not see its plane's copy complete on its
                             mbarrier within the bound; the step's result is void.  No kernel
                             waits on another CTA (the dt reductions use a last-CTA counter or
                             per-item slots and a finaliser kernel) */
    HYDRO_EUNSUPPORTED = 5 /* valid request that this build has no kernel for */
};

typedef enum {
    HYDRO_BC_PERIODIC = 0,
    HYDRO_BC_OUTFLOW = 1,
    HYDRO_BC_ANALYTIC = 2,
    HYDRO_BC_EXCHANGE = 3
} hydro_bc_t;
/* Analytic solutions of HYDRO_BC_ANALYTIC (section 4.3 convergence tests; hydro_set_analytic). */
typedef enum {
    HYDRO_ANALYTIC_ENTROPY_WAVE = 1,
    HYDRO_ANALYTIC_SOUND_WAVE = 2,
    HYDRO_ANALYTIC_SHOCK_TUBE = 3
} hydro_analytic_t;
typedef enum { HYDRO_F64 = 0, HYDRO_F32 = 1 } hydro_prec_t;

/* Grid: dim in {1,2,3}; n[a] >= 1 cells on active axes (n[a] is ignored and taken as 1 on
 * axes a >= dim); box [lo[a], hi[a]] with hi > lo, so dr_a = (hi[a] - lo[a]) / n[a].
 * n[a] <= 2^31 - 1024 and n[0]*n[1]*n[2] < 2^31. */
typedef struct {
    int32_t dim;
    int32_t reserved;
    int64_t n[3];
    double lo[3];
    double hi[3];
} hydro_grid_t;

/* Device pointers of the dim+2 conserved (or primitive) planes; entries >= dim+2 unused. */
typedef struct {
    void *plane[5];
} hydro_state_t;

/* Kernel variant (the tuning space).  Zero-initialised = library default.
 *   tile_x, tile_y: CTA tile (cells).  dim 3: a tile of the (x, y) plane that marches along
 *                   z; dim 2: a tile of the plane, or with tile_y = 1 a row of tile_x cells
 *                   that marches along y ("row tile"); dim 1: a row (tile_y = 1).  Which shapes
 *                   are compiled is answered by hydro_variant_supported().
 *   march:          marching tiles only (dim 3, dim-2 row tiles): planes one CTA marches
 *                   through (>= 1), i.e. the cells each thread updates per stage; 0 = default
 *                   (FP32: chosen by hydro_create from the grid: among 8, 16, 32, 48, ...,
 *                   128 in dim 3 (8, 16, 32, 64, 128 for row tiles) the marches whose
 *                   (tile, chunk) work items fill the GPU's resident CTAs three times (row
 *                   tiles: twice), the one with the least 0.5 x chunks + 0.3 x planes of the
 *                   last chunk, else 8 (row tiles: 16); FP64: 64 in dim 3, 16 for row tiles).
 *   split:          fusion split.  0 = library default (fused for marching tiles, separate
 *                   for one-plane tiles); 1 = a separate CFL pass after RK stage 2 (one more
 *                   launch and one more read of the state per step); 2 = the CFL signal and
 *                   the next dt reduced in the epilogue of stage 2 (fused).
 *   staging:        staging depth, marching tiles only.  0 = default (1); 1 = the next
 *                   plane's loads are issued one plane ahead of their use; 2 = each plane is
 *                   loaded when it is staged (no look-ahead, fewer registers); 3 = the planes
 *                   of the stage's input come into shared memory by TMA (bulk tensor copies of
 *                   the tile plus its halo, completion on an mbarrier, two planes in flight;
 *                   dim 3 FP32, tile 16 x 8, nothing stored between a stage's parts).  Grids
 *                   whose x extent is not a multiple of 4, or planes not 16-byte aligned, run
 *                   the staging-1 kernels instead.  A TMA wait that does not complete within
 *                   its bound makes the call return HYDRO_ETIMEOUT.
 *   occupancy:      FP32 marching tiles only: resident 256-thread CTAs' worth of warps per SM
 *                   the register budget of the stage kernels targets.  0 = library default
 *                   (3 for the default FP32 marching tiles, else 2); 2 (about 128 registers a
 *                   thread); 3 (about 80 registers, 24 warps per SM).
 *   manifest:       what a stage stores in HBM between its parts (the paper's choice of what
 *                   to "Manifest", section 3.1).  0 = library default (1); 1 = nothing: V, the
 *                   face states and fluxes live in registers and shared memory; 2 = V: a pass
 *                   stores the primitive planes of the stage's input, which the stage kernel
 *                   reads instead of U; 3 = F: the stage kernel stores every face flux and a
 *                   pass applies AddFlux (and stage 2's dt reduction).  All three compute the
 *                   same step: bit for bit in FP64; in FP32 to rounding (where V or a flux
 *                   stays in registers the compiler may fuse a product into its consumer).
 *                   dim 3 only, for the tiles compiled with them (FP32
 *                   16 x 8, 32 x 8, 16 x 16; FP64 32 x 8), with look-ahead staging and the
 *                   precision's default budget; 2 and 3 need more workspace
 *                   (hydro_workspace_bytes_variant).
 * Library defaults (measured on GB300): dim 3 FP32 tile 16 x 8 (march from the grid size: 96
 * at 512^3), FP64 32 x 8, march 64; dim 2 FP32 row tile 256 x 1 (march from the grid size: 16
 * at 2048^2, 64 at 4096^2); dim 2 FP64 tile 32 x 8; dim 1 tile 128.  A variant that names a tile other than the default gets that
 * tile's default march (as above in dim 3, 16 for row tiles) and budget unless it names them
 * too.
 * Every variant computes the same step; they differ in speed only. */
typedef struct {
    int32_t tile_x;
    int32_t tile_y;
    int32_t march;
    int32_t split;
    int32_t staging;
    int32_t occupancy;
    int32_t manifest;
} hydro_variant_t;

typedef struct hydro_ctx hydro_ctx_t;

/* Library version (HYDRO_ABI_VERSION). */
int hydro_version(void);

/* Human-readable text of a status code; never NULL. */
const char *hydro_strerror(int status);

/* Text of the last failing CUDA call seen by this host thread ("" if none). */
const char *hydro_last_cuda_error(void);

/* 1 if this build has kernels for (prec, dim, variant); variant may be NULL (default). */
int hydro_variant_supported(int32_t prec, int32_t dim, const hydro_variant_t *variant);

/* Bytes of device workspace hydro_create needs for this grid and precision: the RK stage
 * buffer U1 (dim+2 planes), the step control block and reduction partials. */
int hydro_workspace_bytes(const hydro_grid_t *grid, int32_t prec, size_t *bytes_out);

/* Workspace bytes for a given variant (the manifest forms store V or the face fluxes there);
 * the same as hydro_workspace_bytes for variants that store nothing.  Errors: HYDRO_EINVAL,
 * HYDRO_EUNSUPPORTED (variant not compiled). */
int hydro_workspace_bytes_variant(const hydro_grid_t *grid, int32_t prec,
                                  const hydro_variant_t *variant, size_t *bytes_out);

/* Create a solver context.
 *   grid      grid and box (copied)
 *   gamma     ratio of specific heats, > 1
 *   bc        per-axis boundary condition (hydro_bc_t); entries >= dim ignored.  Periodic
 *             wraps; outflow copies the nearest interior cell into the two ghost layers;
 *             analytic (dim 1 and 2 only, else HYDRO_EUNSUPPORTED) fills the two ghost layers
 *             outside that axis's ends with the exact solution set by hydro_set_analytic at
 *             the time of each RK stage.  Analytic boundaries run on one-plane tiles: with no
 *             tile given a 2D context takes 32 x 8; a row tile (tile_y = 1) is
 *             HYDRO_EUNSUPPORTED.  Exchange (dim 1 and 2, n >= 2 on the axis, one-plane
 *             tiles likewise): before each RK stage the two boundary layers at each end are
 *             packed into buffers and unpacked into the two ghost layers at the other end —
 *             the periodic wrap through the pack/unpack kernels a domain decomposition over
 *             several GPUs would put its transfers between; results equal HYDRO_BC_PERIODIC
 *             bit for bit
 *   prec      HYDRO_F32 (whole stencil in FP32; dt, time and totals in FP64) or HYDRO_F64
 *   cfl       Courant number, 0 < cfl
 *   variant   kernel variant or NULL for the default
 *   workspace device pointer, 256-byte aligned, >= hydro_workspace_bytes(); caller-owned
 *   stream    cudaStream_t the context issues work on (NULL = legacy default stream)
 *   out       receives the context
 * The current CUDA device at create is the context's device. */
int hydro_create(const hydro_grid_t *grid, double gamma, const int32_t bc[3], int32_t prec,
                 double cfl, const hydro_variant_t *variant, void *workspace,
                 size_t workspace_bytes, void *stream, hydro_ctx_t **out);

/* The variant a context runs: the one given to hydro_create with every default filled in
 * (split spelled 1 = separate CFL pass, 2 = fused).  Errors: HYDRO_EINVAL (null pointer). */
int hydro_get_variant(const hydro_ctx_t *ctx, hydro_variant_t *out);

int hydro_destroy(hydro_ctx_t *ctx);

/* The exact solution the analytic boundaries substitute (section 4.3: the tests' domain is
 * the unit square and the solution is given outside it at every time).  With the coordinate
 * along the wave s = (x - 1/2) cos(theta) + (y - 1/2) sin(theta) + 1/2 (dim 1: y = 1/2) and
 * w = sin(2 pi (s - t)), at the ghost-cell centres x = lo + (i + 1/2) dr:
 *   HYDRO_ANALYTIC_ENTROPY_WAVE: rho = 2 + w, v = (cos theta, sin theta), p = 1
 *   HYDRO_ANALYTIC_SOUND_WAVE:   rho = gamma (1 + A w), v = A w (cos theta, sin theta),
 *                                p = 1 + gamma A w   (A = amplitude)
 *   HYDRO_ANALYTIC_SHOCK_TUBE:   Sod's problem, (rho, u, p) = (1, 0, 1) for s < 1/2 and
 *                                (0.125, 0, 0.1) otherwise at t = 0, and its exact similarity
 *                                solution in (s - 1/2) / t after, u the velocity along
 *                                (cos theta, sin theta)
 * evaluated in FP64, converted to conserved variables and rounded to the precision of the
 * context.  Stage 1 of a step takes the solution at t, stage 2 at t + dt/2.  Until it is
 * called, steps of a context with analytic boundaries return HYDRO_EINVAL.  Errors:
 * HYDRO_EINVAL (no analytic axis, unknown kind, non-finite theta or amplitude). */
int hydro_set_analytic(hydro_ctx_t *ctx, int32_t kind, double theta, double amplitude);

/* The same exact solutions at every cell centre of a grid (dim 1 or 2) at time t: the conserved
 * state written to the dim+2 planes of `out` (device, caller-owned, prec elements), e.g. the
 * initial data and the reference of a convergence study.  Stream-ordered on `stream`, no
 * synchronisation.  Errors: HYDRO_EINVAL (dim 3, unknown kind, t < 0, bad grid or pointers). */
int hydro_analytic_state(const hydro_grid_t *grid, double gamma, int32_t prec, int32_t kind,
                         double theta, double amplitude, double t, const hydro_state_t *out,
                         void *stream);

/* Change the stream later calls are ordered on. */
int hydro_set_stream(hydro_ctx_t *ctx, void *stream);

/* Scheme options for later steps (section 4.2 interpolation listing; wave speeds of the cited
 * HLLC solver).  order: 2 = piecewise-linear MinBee reconstruction (default), 1 = first order
 * (the face values are the cell values).  riemann: 0 = Davis wave-speed estimates (default),
 * 1 = pressure-based estimates (Toro's PVRS: p* = max(0, (p_L+p_R)/2 - (u_R-u_L) rho_bar a_bar/2),
 * q_K = 1 if p* <= p_K else sqrt(1 + (gamma+1)/(2 gamma) (p* / p_K - 1)), S_L = u_L - a_L q_L,
 * S_R = u_R + a_R q_R).  HYDRO_EINVAL for other values. */
int hydro_set_scheme(hydro_ctx_t *ctx, int32_t order, int32_t riemann);

/* Advance `state` (in place) by up to n_steps midpoint-RK steps (section 4.1).
 *   t_end     > 0: the last step is clipped so that t lands exactly on t_end and no step
 *             runs once t >= t_end; <= 0: no clipping
 *   t_inout   in: time of `state` (NULL = 0); out: time after the call
 *   steps_done out: steps actually taken (may be NULL)
 * dt is computed on the device from the state at the start of each step (the first from
 * `state` by a CFL pass, later ones in the epilogue of the previous step) and never leaves
 * the device inside the call.  The steps run as CUDA graphs of captured launches (chunks of up
 * to 64 steps); once no further step is to be taken (t_end reached or a failed step) the steps
 * left return at once on the device, and a synchronous call stops launching chunks after
 * that (it reads dt back after each chunk, one chunk late, so n_steps may be a generous
 * bound when t_end is what ends the run).
 * If both t_inout and steps_done are NULL the call is asynchronous and a device-side error
 * is reported by the next synchronising call; otherwise it synchronises and returns
 * HYDRO_ENONFINITE if a step failed. */
int hydro_step(hydro_ctx_t *ctx, const hydro_state_t *state, int32_t n_steps, double t_end,
               double *t_inout, int32_t *steps_done);

/* Same as hydro_step, but the state comes from and goes back to HOST memory: the dim+2
 * planes at host_in[k] are copied into the device planes of `dev_state`, stepped, and copied
 * out to host_out[k] (host_out may equal host_in).  Pinned host memory gives full copy
 * bandwidth.  In dim 3 the copies overlap the work: the state comes in by z-slabs, each slab's
 * part of the first CFL pass starting on arrival, and the last step runs both stages slab by
 * slab, each finished slab going back while later slabs compute; planes that are equally
 * spaced on both sides (one tensor) move as one strided copy per slab.  Always synchronises. */
int hydro_step_host(hydro_ctx_t *ctx, const hydro_state_t *dev_state,
                    const void *const host_in[5], void *const host_out[5], int32_t n_steps,
                    double t_end, double *t_inout, int32_t *steps_done);

/* hydro_step_host without waiting (no counterpart in the paper): the same copy in, steps and
 * copy back, all enqueued on the context's stream (and its private copy stream), and the call
 * returns.  t: time of the state in host_in (as *t_inout of hydro_step_host).  The host
 * buffers must stay allocated, host_in unchanged and host_out unread until the context's
 * stream has reached the end of the call (cudaStreamSynchronize on it, or hydro_status, which
 * also returns the status of the steps).  All n_steps steps are launched (those after t_end or
 * after a failed step return at once on the device).  Calls on one context run one after the
 * other; calls on contexts with different streams overlap, so two problems in flight keep the
 * CPU-GPU link busy in both directions (one problem's copy in during another's copy back).
 * Setting up a copy of the control block from host memory may wait for the context's stream
 * to finish its earlier work.  Errors: HYDRO_EINVAL (as hydro_step_host, or t or t_end NaN),
 * HYDRO_ECUDA; a failed step is reported by the next synchronising call. */
int hydro_step_host_async(hydro_ctx_t *ctx, const hydro_state_t *dev_state,
                          const void *const host_in[5], void *const host_out[5],
                          int32_t n_steps, double t_end, double t);

/* dt = cfl / max_i sum_a (|v_a| + c_s)/dr_a of `state` (FP64 result).  Synchronises. */
int hydro_cfl_dt(hydro_ctx_t *ctx, const hydro_state_t *state, double *dt_out);

/* Conserved totals integrated over the box, in FP64: out = (mass, M_x, M_y, M_z, energy),
 * momenta of inactive axes 0.  Deterministic fixed-order two-level sum times the cell volume.
 * Synchronises. */
int hydro_totals(hydro_ctx_t *ctx, const hydro_state_t *state, double out[5]);

/* Device status word of the last step call: HYDRO_OK or HYDRO_ENONFINITE.  Synchronises. */
int hydro_status(hydro_ctx_t *ctx);

/* Element-wise conversions between primitive (rho, v, p) and conserved (rho, m, E) planes
 * (section 4.1: m_a = rho v_a, E = p/(gamma-1) + rho v^2/2) for ncell cells of precision
 * prec, on `stream`.  in and out may be the same planes.  Context-free. */
int hydro_prim_to_cons(int32_t dim, int64_t ncell, double gamma, int32_t prec,
                       const hydro_state_t *prim_in, const hydro_state_t *cons_out, void *stream);
int hydro_cons_to_prim(int32_t dim, int64_t ncell, double gamma, int32_t prec,
                       const hydro_state_t *cons_in, const hydro_state_t *prim_out, void *stream);

/* Per-kernel timing.  With profiling on, hydro_step launches its kernels directly (no graph)
 * with CUDA events recorded on the context's stream around each launch, in batches of up to 64
 * steps (the call synchronises after each batch and stops once no further step is to be
 * taken).  Stage times include the ghost-ring fills of analytic and exchange boundaries.
 * hydro_kernel_times fills, for each kernel kind k (0 = CFL pass, 1 = RK stage 1, 2 = RK
 * stage 2 with the fused dt reduction), ms_out[k] = summed device time and launches_out[k] =
 * launches since the last reset; it synchronises.  n = number of entries the arrays hold. */
int hydro_set_profiling(hydro_ctx_t *ctx, int32_t on);
int hydro_kernel_times(hydro_ctx_t *ctx, double *ms_out, int64_t *launches_out, int32_t n,
                       int32_t reset);

/* ---- Batched grids: many independent 2D grids of uneven size ----------------------------
 * The grids are advanced together by one persistent launch per RK stage, steps captured in
 * CUDA graphs.  Each grid is its own unit square (dr = 1/nx, 1/ny) with its own CFL dt and
 * time, the same scheme as hydro_step.  All grids share gamma, cfl, the boundary conditions
 * and the precision.
 * Packed layout: 4 planes (rho, m_x, m_y, E); plane k is one device array of sum_g nx_g ny_g
 * elements in which grid g occupies [offset_g, offset_g + nx_g ny_g), x fastest (offsets from
 * hydro_batch_offsets, grids in the order given).
 * Workspace: caller-owned, hydro_batch_workspace_bytes() bytes, 256-byte aligned: per-grid
 * control blocks and geometry, the (grid, tile) work list and the packed U1 stage buffer. */
typedef struct hydro_batch hydro_batch_t;

/* Bytes of workspace for n_grids grids of nx[g] x ny[g] cells (variant: tile, or NULL). */
int hydro_batch_workspace_bytes(int32_t n_grids, const int64_t *nx, const int64_t *ny,
                                int32_t prec, const hydro_variant_t *variant, size_t *bytes_out);

/* Create a batch (grid shapes copied; bc[0], bc[1] for x and y of every grid).  Uploads the
 * work list into the workspace and synchronises `stream` once. */
int hydro_batch_create(int32_t n_grids, const int64_t *nx, const int64_t *ny, double gamma,
                       const int32_t bc[2], int32_t prec, double cfl,
                       const hydro_variant_t *variant, void *workspace, size_t workspace_bytes,
                       void *stream, hydro_batch_t **out);
int hydro_batch_destroy(hydro_batch_t *batch);

/* offsets_out[0..n_grids]: first cell of each grid in the packed planes, then the total. */
int hydro_batch_offsets(const hydro_batch_t *batch, int64_t *offsets_out);
int hydro_batch_set_stream(hydro_batch_t *batch, void *stream);

/* Advance every grid by up to n_steps RK steps (each with its own dt).  t_inout: n_grids
 * start times in, end times out (NULL: all start at 0); steps_done: n_grids counts (NULL ok).
 * t_end as for hydro_step, per grid.  Synchronises when t_inout or steps_done is given and
 * then returns HYDRO_ENONFINITE if any grid failed (that grid stops; the others go on). */
int hydro_batch_step(hydro_batch_t *batch, const hydro_state_t *packed, int32_t n_steps,
                     double t_end, double *t_inout, int32_t *steps_done);

/* FP64 totals of every grid: out[5 g + (mass, M_x, M_y, 0, E)].  Synchronises. */
int hydro_batch_totals(hydro_batch_t *batch, const hydro_state_t *packed, double *out);

/* Per-kernel event timing as hydro_set_profiling / hydro_kernel_times (kinds 0 = CFL pass,
 * 1 = RK stage 1, 2 = RK stage 2). */
int hydro_batch_set_profiling(hydro_batch_t *batch, int32_t on);
int hydro_batch_kernel_times(hydro_batch_t *batch, double *ms_out, int64_t *launches_out,
                             int32_t n, int32_t reset);

/* ---- The linear-wave example (section 2.3) ---------------------------------------------
 * f_t = g, g_t = c^2 f_xx on n >= 3 cells of the periodic interval [0, length), dx = length/n,
 * advanced n_steps times by Eqs. eqLWDiscF and eqLWDiscG:
 *     f1[i] = f[i] + dt g[i];  g1[i] = g[i] + (c^2 dt/dx^2)(f1[i+1] + f1[i-1] - 2 f1[i]),
 * with the discrete energy E = sum_i (c^2 ((f1[i+1]-f1[i-1])/(2 dx))^2 + ((g[i]+g1[i])/2)^2)/2 dx
 * computed in FP64 after every step into energy_out[step] (host, n_steps doubles; may be NULL).
 * (The paper prints this energy with c^2 inside the square and no 1/2; the form above is the
 * one its listing computes and the scheme conserves.)  f and g: device arrays of n elements
 * of precision prec, updated in place.  Workspace: hydro_wave_workspace_bytes() bytes,
 * 256-byte aligned, caller-owned.  Synchronises `stream`. */
int hydro_wave_workspace_bytes(int64_t n, int32_t prec, int32_t n_steps, size_t *bytes_out);
int hydro_wave_run(int32_t prec, int64_t n, double c, double length, double dt, void *f, void *g,
                   int32_t n_steps, double *energy_out, void *workspace, size_t workspace_bytes,
                   void *stream);

/* ---- Cost model of the variant tuner: a 3-layer MLP trained on the GPU ---------------------
 * y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3, input width d, hidden width H, FP32.  All arrays
 * are device memory owned by the caller: params (hydro_mlp_sizes' param_count floats, layout
 * W1 (H x d, row-major), b1, W2 (H x H), b2, W3 (1 x H), b3), Adam moments m and v (same
 * size), inputs X (n x d, row-major), targets t (n), and a workspace of workspace_bytes for
 * n samples (1 <= n <= 65535 * 128, 1 <= d, H <= 4096; otherwise HYDRO_EINVAL).  Loss: mean
 * squared error over the n samples.  Calls are ordered on `stream` and do not synchronise.
 * Deterministic (fixed reduction order, no atomics). */
int hydro_mlp_sizes(int32_t d, int32_t hidden, int64_t n, int64_t *param_count,
                    size_t *workspace_bytes);
/* y_out[s] = network(X[s]) for s < n. */
int hydro_mlp_forward(const float *params, int32_t d, int32_t hidden, const float *X, int64_t n,
                      float *y_out, void *workspace, void *stream);
/* Gradient of the loss w.r.t. params (back-propagation) into grad_out (param_count floats) and
 * the loss into loss_out[0]; either may be NULL. */
int hydro_mlp_gradient(const float *params, int32_t d, int32_t hidden, const float *X,
                       const float *t, int64_t n, void *workspace, float *grad_out,
                       float *loss_out, void *stream);
/* One Adam step (step >= 1 is the 1-based update count for the bias corrections). */
int hydro_mlp_adam(float *params, float *m, float *v, const float *grad, int64_t count,
                   int32_t step, float lr, float beta1, float beta2, float eps, void *stream);
/* `epochs` full-batch Adam steps (numbered step0+1 ...); loss_out[k] (device, may be NULL)
 * receives the loss before step k.  The step number is kept in the workspace and advanced on
 * the device, so the epochs are captured once into a CUDA graph (on a private stream) and
 * replayed on `stream`; the Adam bias corrections are computed on the device. */
int hydro_mlp_train(float *params, float *m, float *v, int32_t d, int32_t hidden, const float *X,
                    const float *t, int64_t n, int32_t epochs, int32_t step0, float lr,
                    void *workspace, float *loss_out, void *stream);

/* Size of the device scratch array of hydro_step_static: 4 MiB, held by every GPU that loads
 * this library until the process exits. */
#define HYDRO_STATIC_SCRATCH_BYTES (4u << 20)

/* hydro_step for callers that cannot allocate device memory (no counterpart in the paper).
 *
 * Some callers cannot call cudaMalloc or give the library a workspace: code running inside
 * another runtime that owns every allocation (a framework with its own caching allocator),
 * and embedded or real-time callers that must not allocate after start-up.  This call takes
 * the grid, gamma, bc, prec and cfl of hydro_create plus the arguments of hydro_step, needs no
 * context and no workspace, and allocates nothing: the RK stage buffer U1 and the step control
 * block live in one file-scope device array of HYDRO_STATIC_SCRATCH_BYTES.  The caller still
 * owns and passes the state planes (device memory on the caller's CURRENT device, where the
 * call runs; layout as for hydro_step).
 *   Kernels: one fixed variant, not hydro_create's tuned defaults: 32 x 8 tiles in 2D and 3D
 *   (3D marching up to 64 planes), 128-cell rows in 1D, look-ahead staging, the two-CTA
 *   register budget, the dt reduction fused into stage 2.  Direct launches (no graph): one
 *   CFL pass, then 2 * n_steps stage kernels whatever t_end is (the stages after t_end return
 *   at once, but each still costs a launch, so keep n_steps near the steps needed).
 *   Size limit: the control block (256 bytes) plus dim+2 planes of n[0]*n[1]*n[2] cells, each
 *   rounded up to 256 bytes, must fit in HYDRO_STATIC_SCRATCH_BYTES (for example a 1D grid of
 *   10^5 cells in FP64, or 59^3 cells in FP32); larger grids return HYDRO_EINVAL.
 *   Set-up: the first call on each device (that device current) looks up the array's device
 *   address with cudaGetSymbolAddress and sets kernel attributes; later calls reuse both.
 *   Time: *t_inout (NULL: 0) is read on the host when the call is made.  With t_inout or
 *   steps_done non-NULL the call copies the control block back and synchronises the stream
 *   (as hydro_step does); with both NULL it only enqueues work and returns.
 *   Sharing: every call uses the same array, which keeps the last call's contents; each call
 *   rewrites the control block before use.  Calls that overlap on the GPU race on the array:
 *   order them (one stream, or events).
 * Errors as for hydro_step (stream = cudaStream_t to issue on). */
int hydro_step_static(const hydro_grid_t *grid, double gamma, const int32_t bc[3], int32_t prec,
                      double cfl, const hydro_state_t *state, int32_t n_steps, double t_end,
                      double *t_inout, int32_t *steps_done, void *stream);

/* Diagnostic with no counterpart in the paper: the measured fused multiply-add throughput of
 * the current device, in lane operations per second (one FMA counts one), for prec HYDRO_F32 or
 * HYDRO_F64.  A grid of every SM's resident 256-thread CTAs runs eight independent FMA chains
 * per thread; the best of three timed launches (CUDA events on `stream`, after one warm-up
 * launch) is returned in *ops_per_s_out.  Takes a few tens of milliseconds, allocates one
 * element with cudaMallocAsync on `stream` and frees it, and synchronises the stream.
 * Errors: HYDRO_EINVAL (null output, other prec), HYDRO_ECUDA. */
int hydro_fma_rate(int32_t prec, void *stream, double *ops_per_s_out);

/* Diagnostic with no counterpart in the paper: checks the bounded mbarrier wait that the
 * TMA-staged stage kernels (variant staging 3) use.  One CTA of 32 threads waits on an mbarrier
 * whose phase never completes (it expects an arrival nobody makes); each thread gives up after
 * the wait's bound (2^16 tries or about one second of the GPU's global timer) and counts itself
 * in *gave_up_device (one int32 of caller-owned device memory, zeroed by the call).  The count is
 * copied to *gave_up_out (32 when the bound works) and the kernel's time to *elapsed_ms_out (may
 * be NULL); the context stays usable.  Synchronises `stream`.  Errors: HYDRO_EINVAL (null
 * pointers), HYDRO_ECUDA. */
int hydro_wait_bound_check(int32_t *gave_up_device, void *stream, int32_t *gave_up_out,
                           double *elapsed_ms_out);

#ifdef __cplusplus
}
#endif

#endif /* HYDRO_H */
