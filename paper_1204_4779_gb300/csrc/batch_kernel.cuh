// Batched RK-stage kernels: thousands of independent 2D grids of uneven size advanced by one
// persistent launch per RK stage (the same midpoint-RK MinBee/HLLC step as stage_kernel.cuh,
// arXiv:1204.4779 section 4.1, on every grid).
//
// Layout: the grids' planes are packed: plane k of the batch is one array in which grid g
// occupies [off_g, off_g + nx_g ny_g), x fastest.  Work is a list of (grid, tile) items,
// ordered grid by grid; a persistent grid of CTAs walks it with a fixed stride, so CTAs that
// run at the same time work on neighbouring tiles of the same grid (halo reuse in L2).
//
// Each grid has its own control block (dt, time, status): every grid is its own unit square
// with its own CFL dt.  In stage 2 each tile reduces the CFL signal of its new cells and
// stores the maximum in its own slot (a plain store: no atomic, no fence on the tile's path);
// a small finaliser kernel, one warp per grid, reduces each grid's slots and sets its dt for
// the next step.
#pragma once

#include "hydro_device.cuh"
#include "hydro_internal.h"
#include "stage_kernel.cuh"

namespace hydro {

template <class T> struct BatchArgs {
    const T *uin[4];
    const T *ubase[4];
    T *uout[4];
    const BatchItem *items;
    int n_items;
    const BatchGrid *grids;
    Ctrl *ctrl;  // one per grid
    T *tile_sig;       // CFL-signal maximum of each work item (NaN: a bad cell)
    unsigned int *claim;  // row kernels: next work item of stage 1 / stage 2, minus gridDim.x
    const double *t0;  // per-grid start time (init kernel), may be null
    double t_end, cfl;
    int periodic[2];
    int rows;   // rows of a work item: the tile height, or the march of row tiles
    Gas<T> gas;
};

// Max over the CTA of a non-negative value or NaN (on the bit patterns: NaN > inf > finite),
// returned to thread 0.  Call from all threads.
template <class T, int NT> __device__ __forceinline__ T block_max(T v, T *sred) {
    using U = typename std::conditional<sizeof(T) == 4, unsigned int, unsigned long long>::type;
    U bits;
    if constexpr (sizeof(T) == 4)
        bits = __float_as_uint(v);
    else
        bits = (unsigned long long)__double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const U other = __shfl_xor_sync(0xffffffffu, bits, o);
        bits = other > bits ? other : bits;
    }
    U *sb = reinterpret_cast<U *>(sred);
    __syncthreads();  // the previous use of sred is over
    if ((threadIdx.x & 31) == 0) sb[threadIdx.x >> 5] = bits;
    __syncthreads();
    U m = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) m = sb[w] > m ? sb[w] : m;
    if constexpr (sizeof(T) == 4)
        return __uint_as_float((unsigned int)m);
    else
        return __longlong_as_double((long long)m);
}

template <class T, int BX, int BY, int STAGE>
__global__ void __launch_bounds__(BX * BY, (MinBlocks<T, BX * BY>::value))
    batch_stage_kernel(const BatchArgs<T> A) {
    using S = StageShape<T, 2, BX, BY>;
    constexpr int NV = 4, NT = S::NT, HX = S::HX, PL = S::PL;
    constexpr int NFX = S::NFX, NF = S::NF, HPT = S::HPT, FPT = S::FPT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const sV = reinterpret_cast<T *>(smem_raw);
    T *const sF = sV + NV * PL;
    T *const sRed = sF + NV * NF;
    const Gas<T> G = A.gas;

    const int tid = threadIdx.x;
    const int tx = tid % BX, ty = tid / BX;
    const int own_s = (ty + 2) * HX + (tx + 2);
    int h_lx[HPT], h_ly[HPT];
    bool h_ok[HPT];
#pragma unroll
    for (int j = 0; j < HPT; ++j) h_ok[j] = halo_task<2, BX, BY>((NT - 1 - tid) + j * NT, h_lx[j], h_ly[j]);
    int f_o[FPT], f_s[FPT], f_a[FPT], f_id[FPT];
    bool f_ok[FPT];
#pragma unroll
    for (int j = 0; j < FPT; ++j) f_ok[j] = face_task<2, BX, BY>(tid, j, f_o[j], f_s[j], f_a[j], f_id[j]);

    for (int it = blockIdx.x; it < A.n_items; it += gridDim.x) {
        const BatchItem W = A.items[it];
        const BatchGrid R = A.grids[W.g];
        Ctrl *ctrl = A.ctrl + W.g;
        const double dt = __ldcg(&ctrl->dt);
        if (!(dt > 0.0)) continue;  // this grid takes no step (same for the whole CTA)
        const T cx = T(__ldcg(&ctrl->coef[STAGE - 1][0]));
        const T cy = T(__ldcg(&ctrl->coef[STAGE - 1][1]));
        const int nx = R.nx, ny = R.ny;
        const int x = W.x0 + tx, y = W.y0 + ty;
        const bool active = (x < nx) && (y < ny);
        const long long off = R.off;

        // stage V of the tile and its halo
        {
            T u[NV], v[NV];
            const long long i = off + remap(y, ny, A.periodic[1]) * nx + remap(x, nx, A.periodic[0]);
#pragma unroll
            for (int k = 0; k < NV; ++k) u[k] = __ldg(A.uin[k] + i);
            prim_of_cons<T, 2>(u, v, G);
            Cells<T, NV>::put(sV, PL, own_s, v);
        }
#pragma unroll
        for (int j = 0; j < HPT; ++j) {
            if (h_ok[j]) {
                const int xg = remap(W.x0 + h_lx[j] - 2, nx, A.periodic[0]);
                const int yg = remap(W.y0 + h_ly[j] - 2, ny, A.periodic[1]);
                const long long i = off + (long long)yg * nx + xg;
                T u[NV], v[NV];
#pragma unroll
                for (int k = 0; k < NV; ++k) u[k] = __ldg(A.uin[k] + i);
                prim_of_cons<T, 2>(u, v, G);
                Cells<T, NV>::put(sV, PL, h_ly[j] * HX + h_lx[j], v);
            }
        }
        T base[NV];
        {
            const long long i = off + (active ? (long long)y * nx + x : 0);
#pragma unroll
            for (int k = 0; k < NV; ++k) base[k] = active ? A.ubase[k][i] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < FPT; ++j)
            if (f_ok[j]) inplane_face<T, 2, PL, NF>(sV, sF, f_o[j], f_s[j], f_a[j], f_id[j], G);
        __syncthreads();

        T smax = T(0);
        bool bad = false;
        if (active) {
            const int fxl = ty * (BX + 1) + tx;
            const int fyb = NFX + ty * BX + tx;
            T un[NV], fw[NV], fe[NV], fs[NV], fn[NV];
            Cells<T, NV>::get(sF, NF, fxl, fw);
            Cells<T, NV>::get(sF, NF, fxl + 1, fe);
            Cells<T, NV>::get(sF, NF, fyb, fs);
            Cells<T, NV>::get(sF, NF, fyb + BX, fn);
            add_fluxes<T, NV, true, false>(base, cx, fw, fe, cy, fs, fn, T(0), fw, fw, un);
            const long long i = off + (long long)y * nx + x;
#pragma unroll
            for (int k = 0; k < NV; ++k) A.uout[k][i] = un[k];
            if constexpr (STAGE == 2) {
                T v[NV];
                prim_of_cons<T, 2>(un, v, G);
                T cs, s = T(0);
                if constexpr (Arith<T>::exact) {
                    cs = sqrt(G.g * v[3] / v[0]);
                    s = s + (fabs(v[1]) + cs) / R.dr[0];
                    s = s + (fabs(v[2]) + cs) / R.dr[1];
                } else {
                    cs = Arith<float>::sqrt_(G.g * v[3] * Arith<float>::rcp(v[0]));
                    s = fmaf(fabsf(v[1]) + cs, R.inv_dr[0], s);
                    s = fmaf(fabsf(v[2]) + cs, R.inv_dr[1], s);
                }
                smax = s;
                bad = !(v[0] > T(0)) || !(v[3] > T(0));
            }
        }
        if constexpr (STAGE == 2) {
            const T m = block_max<T, NT>(bad ? T(NAN) : smax, sRed);
            if (threadIdx.x == 0) A.tile_sig[it] = m;
        }
    }
}

// Row tiles: a work item is a strip of BX columns of one grid and a chunk of `rows` rows,
// advanced by the single-grid kernels' per-tile code (stage_tile) marching along y, with the
// same per-tile CFL slot as the tile kernel above.  Items are claimed dynamically: CTA b takes
// item b first, then the next unclaimed item from a counter (items differ in size -- ragged
// strips and chunks, grids of 32 to 512 cells a side -- so a fixed stride leaves CTAs idle at
// the end of the launch); items are still taken in list order, grid by grid.  Every item's
// result and CFL slot are the same whichever CTA computes it.
template <class T, int BX, int STAGE, int OCC>
__global__ void __launch_bounds__(BX, (MinBlocks<T, BX, OCC>::value))
    batch_row_kernel(const BatchArgs<T> A) {
    using S = StageShape<T, 2, BX, 1>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const sRed = reinterpret_cast<T *>(smem_raw) + 2 * S::NV * S::PL + 2 * S::NV * S::NF;
    __shared__ int s_next;
    auto claim_next = [&]() -> int {
        __syncthreads();  // every thread has read the previous claim
        if (threadIdx.x == 0) s_next = (int)gridDim.x + (int)atomicAdd(A.claim + (STAGE - 1), 1u);
        __syncthreads();
        return s_next;
    };
    for (int it = blockIdx.x; it < A.n_items; it = claim_next()) {
        const BatchItem W = A.items[it];
        const BatchGrid R = A.grids[W.g];
        Ctrl *ctrl = A.ctrl + W.g;
        const double dt = __ldcg(&ctrl->dt);
        if (!(dt > 0.0)) continue;  // this grid takes no step (same for the whole CTA)
        const T cx = T(__ldcg(&ctrl->coef[STAGE - 1][0]));
        const T cy = T(__ldcg(&ctrl->coef[STAGE - 1][1]));
        StageArgs<T> V;  // the grid as a single-grid problem
        for (int k = 0; k < 4; ++k) {
            V.uin[k] = A.uin[k] + R.off;
            V.ubase[k] = A.ubase[k] + R.off;
            V.uout[k] = A.uout[k] + R.off;
        }
        V.uin[4] = V.ubase[4] = nullptr;
        V.uout[4] = nullptr;
        V.n[0] = R.nx, V.n[1] = R.ny, V.n[2] = 1;
        V.periodic[0] = A.periodic[0], V.periodic[1] = A.periodic[1], V.periodic[2] = 1;
        V.march = A.rows;
        V.zchunk0 = 0;
        V.order = 2;
        V.riemann = 0;
        V.dr[0] = R.dr[0], V.dr[1] = R.dr[1], V.dr[2] = 1.0;
        V.inv_dr[0] = T(R.inv_dr[0]), V.inv_dr[1] = T(R.inv_dr[1]), V.inv_dr[2] = T(1);
        V.gas = A.gas;
        V.ctrl = ctrl;
        V.ana = 0;  // the batch's grids are periodic or outflow
        V.items = 0;
        __syncthreads();  // the previous item's last shared-memory reads are done
        T smax = T(0);
        bool bad = false;
        stage_tile<T, 2, BX, 1, STAGE, 1, (STAGE == 2)>(V, W.x0, 0, W.y0, min(W.y0 + A.rows, R.ny),
                                                         smem_raw, cx, T(0), cy, smax, bad);
        if constexpr (STAGE == 2) {
            const T m = block_max<T, BX>(bad ? T(NAN) : smax, sRed);
            if (threadIdx.x == 0) A.tile_sig[it] = m;
        }
    }
}

// Per-grid start of a step call: control block of grid g reset, time t0[g] (or 0).
static __global__ void batch_init_kernel(Ctrl *ctrl, const BatchGrid *grids, int n_grids,
                                  const double *t0, double t_end, double cfl, unsigned int *claim) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g == 0 && claim) claim[0] = claim[1] = 0u;
    if (g >= n_grids) return;
    Ctrl z = {};
    z.t = t0 ? t0[g] : 0.0;
    z.t_end = t_end;
    z.cfl = cfl;
    z.dr[0] = grids[g].dr[0];
    z.dr[1] = grids[g].dr[1];
    z.dr[2] = 1.0;
    ctrl[g] = z;
}

// CFL pass over every tile: the first dt of each grid.
template <class T, int BX, int BY>
__global__ void __launch_bounds__(BX * BY) batch_cfl_kernel(const BatchArgs<T> A) {
    constexpr int NT = BX * BY;
    __shared__ T sRed[2 * NT / 32];
    const int tx = threadIdx.x % BX, ty = threadIdx.x / BX;
    for (int it = blockIdx.x; it < A.n_items; it += gridDim.x) {
        const BatchItem W = A.items[it];
        const BatchGrid R = A.grids[W.g];
        const int x = W.x0 + tx;
        T smax = T(0);
        bool bad = false;
        for (int y = W.y0 + ty; y < W.y0 + A.rows && y < R.ny && x < R.nx; y += BY) {
            const long long i = R.off + (long long)y * R.nx + x;
            T u[4], v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) u[k] = A.uin[k][i];
            prim_of_cons<T, 2>(u, v, A.gas);
            T s = T(0);
            if constexpr (Arith<T>::exact) {
                const T cs = sqrt(A.gas.g * v[3] / v[0]);
                s = s + (fabs(v[1]) + cs) / R.dr[0];
                s = s + (fabs(v[2]) + cs) / R.dr[1];
            } else {
                const T cs = Arith<float>::sqrt_(A.gas.g * v[3] * Arith<float>::rcp(v[0]));
                s = fmaf(fabsf(v[1]) + cs, R.inv_dr[0], s);
                s = fmaf(fabsf(v[2]) + cs, R.inv_dr[1], s);
            }
            smax = (s > smax || s != s) ? s : smax;
            bad |= !(v[0] > T(0)) || !(v[3] > T(0));
        }
        const T m = block_max<T, NT>(bad ? T(NAN) : smax, sRed);
        if (threadIdx.x == 0) A.tile_sig[it] = m;
    }
}

// dt of every grid from its tiles' signal maxima: one warp per grid reduces the grid's slots
// in a fixed pattern, lane 0 finalises (advance: a step has just completed).
template <class T, bool ADVANCE>
__global__ void __launch_bounds__(256) batch_finalize_kernel(const BatchArgs<T> A, int n_grids) {
    using U = typename std::conditional<sizeof(T) == 4, unsigned int, unsigned long long>::type;
    const int g = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    // the row kernels' work-item counters, for the next stage launches (this kernel runs after
    // a step's stage 2 and before the next stage 1)
    if (blockIdx.x == 0 && threadIdx.x == 0 && A.claim) A.claim[0] = A.claim[1] = 0u;
    if (g >= n_grids) return;
    const BatchGrid R = A.grids[g];
    U m = 0;
    for (int i = lane; i < R.ntiles; i += 32) {
        const T v = A.tile_sig[R.first_item + i];
        U b;
        if constexpr (sizeof(T) == 4)
            b = __float_as_uint(v);
        else
            b = (unsigned long long)__double_as_longlong(v);
        m = b > m ? b : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const U other = __shfl_xor_sync(0xffffffffu, m, o);
        m = other > m ? other : m;
    }
    if (lane == 0) {
        Ctrl *c = A.ctrl + g;
        if constexpr (sizeof(T) == 4)
            c->sig32 = (unsigned int)m;
        else
            c->sig64 = (unsigned long long)m;
        finalize_dt<T>(c, ADVANCE);
    }
}

// Conserved totals of every grid in FP64: one CTA per grid, fixed per-thread strides and a
// fixed shared-memory tree (deterministic), times the cell volume, into ctrl[g].totals.
template <class T>
__global__ void __launch_bounds__(256) batch_totals_kernel(const BatchArgs<T> A, int n_grids) {
    __shared__ double s[256];
    const int g = blockIdx.x;
    if (g >= n_grids) return;
    const BatchGrid R = A.grids[g];
    const long long n = (long long)R.nx * R.ny;
    const double vol = R.dr[0] * R.dr[1];
    for (int k = 0; k < 4; ++k) {
        double acc = 0.0;
        for (long long i = threadIdx.x; i < n; i += 256) acc += (double)A.uin[k][R.off + i];
        s[threadIdx.x] = acc;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) A.ctrl[g].totals[k == 3 ? 4 : k] = s[0] * vol;
        __syncthreads();
    }
    if (threadIdx.x == 0) A.ctrl[g].totals[3] = 0.0;
}

template <class T> BatchArgs<T> make_batch_args(const BatchLaunch &L) {
    BatchArgs<T> A;
    for (int k = 0; k < 4; ++k) {
        A.uin[k] = static_cast<const T *>(L.uin[k]);
        A.ubase[k] = static_cast<const T *>(L.ubase[k]);
        A.uout[k] = static_cast<T *>(L.uout[k]);
    }
    A.items = L.items;
    A.n_items = L.n_items;
    A.grids = L.grids;
    A.ctrl = static_cast<Ctrl *>(L.ctrl);
    A.tile_sig = static_cast<T *>(L.tile_sig);
    A.claim = L.claim;
    A.t0 = L.t0;
    A.t_end = L.t_end;
    A.cfl = L.cfl;
    A.periodic[0] = L.periodic[0];
    A.periodic[1] = L.periodic[1];
    A.rows = L.tile_y == 1 ? L.march : L.tile_y;
    A.gas = make_gas<T>(L.gamma);
    return A;
}

// The two RK-stage kernels of a batch tile shape: row tiles or one-plane tiles.
template <class T, int BX, int BY, int OCC, bool ROWS> struct BatchKernels {
    static constexpr auto s1 = batch_stage_kernel<T, BX, BY, 1>;
    static constexpr auto s2 = batch_stage_kernel<T, BX, BY, 2>;
};
template <class T, int BX, int BY, int OCC> struct BatchKernels<T, BX, BY, OCC, true> {
    static constexpr auto s1 = batch_row_kernel<T, BX, 1, OCC>;
    static constexpr auto s2 = batch_row_kernel<T, BX, 2, OCC>;
};

// Dispatch for one precision: kind 0 = init, 1 = CFL pass, 2/3 = RK stage 1/2, 4 = totals;
// prepare_only sets the shared-memory attribute and returns the resident CTAs per SM of the
// stage kernel in *blocks_per_sm.
template <class T, int BX, int BY, int OCC = 2>
cudaError_t batch_dispatch_tile(const BatchLaunch &L, cudaStream_t st, int kind, bool prepare_only,
                                int *blocks_per_sm) {
    using S = StageShape<T, 2, BX, BY>;
    constexpr bool rows = (BY == 1);  // row tiles march along y
    // the tile kernel keeps one primitive and one flux plane; row tiles use stage_tile's two each
    const size_t smem = sizeof(T) * (size_t)((rows ? 2 : 1) * 4 * (S::PL + S::NF) + 2 * (S::NT / 32));
    using K = BatchKernels<T, BX, BY, OCC, rows>;
    const auto s1 = K::s1, s2 = K::s2;
    if (prepare_only) {
        cudaError_t e = cudaFuncSetAttribute(s1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(s2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess && blocks_per_sm)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, s2, S::NT, smem);
        return e;
    }
    const BatchArgs<T> A = make_batch_args<T>(L);
    switch (kind) {
        case 0: batch_init_kernel<<<(L.n_grids + 255) / 256, 256, 0, st>>>(A.ctrl, A.grids, L.n_grids, A.t0, A.t_end, A.cfl, A.claim); break;
        case 1: batch_cfl_kernel<T, BX, BY><<<L.n_blocks, S::NT, 0, st>>>(A); break;
        case 2: s1<<<L.n_blocks, S::NT, smem, st>>>(A); break;
        case 3: s2<<<L.n_blocks, S::NT, smem, st>>>(A); break;
        case 4: batch_totals_kernel<T><<<L.n_grids, 256, 0, st>>>(A, L.n_grids); break;
        case 5: batch_finalize_kernel<T, false><<<(L.n_grids * 32 + 255) / 256, 256, 0, st>>>(A, L.n_grids); break;
        case 6: batch_finalize_kernel<T, true><<<(L.n_grids * 32 + 255) / 256, 256, 0, st>>>(A, L.n_grids); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hydro
