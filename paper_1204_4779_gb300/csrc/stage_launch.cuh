// Launch helpers of the fused RK-stage kernel: grid shape, dynamic shared memory and the
// table of compiled tile shapes (BX, BY) per precision and dimension.
#pragma once

#include "hydro_internal.h"
#include "stage_kernel.cuh"

namespace hydro {

template <class T> static StageArgs<T> make_stage_args(const StageLaunch &L) {
    StageArgs<T> A;
    for (int k = 0; k < 5; ++k) {
        A.uin[k] = static_cast<const T *>(L.uin[k]);
        A.ubase[k] = static_cast<const T *>(L.ubase[k]);
        A.uout[k] = static_cast<T *>(L.uout[k]);
    }
    for (int a = 0; a < 3; ++a) {
        A.n[a] = L.n[a];
        A.periodic[a] = L.periodic[a];
        A.dr[a] = L.dr[a];
        A.inv_dr[a] = T(1.0 / L.dr[a]);
    }
    A.march = L.march;
    A.zchunk0 = L.zchunk0;
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 5; ++k) A.flux[a][k] = static_cast<T *>(L.flux[a][k]);
    A.order = L.order == 1 ? 1 : 2;
    A.riemann = L.riemann;
    A.gas = make_gas<T>(L.gamma);
    A.ctrl = static_cast<Ctrl *>(L.ctrl);
    A.ana = L.ana;
    for (int k = 0; k < 5; ++k) A.frame[k] = static_cast<const T *>(L.frame[k]);
    A.items = 0;
    A.tiles_x = A.tiles_y = 0;
    return A;
}

// The kernels of one (T, D, tile) for one staging depth PF and occupancy target OCC: stage 1,
// stage 2 with the fused dt reduction, stage 2 without it.
// MAN 2 (manifest F): s1 is the flux kernel of both stages (it stores fluxes and never updates).
template <class T, int D, int BX, int BY, int PF, int OCC, int MAN = 0> struct StageKernels {
    static constexpr auto s1 = stage_kernel<T, D, BX, BY, 1, PF, true, OCC, MAN>;
    static constexpr auto s2 = stage_kernel<T, D, BX, BY, 2, PF, true, OCC, MAN>;
    static constexpr auto s2_split = stage_kernel<T, D, BX, BY, 2, PF, false, OCC, MAN>;
};
// Their persistent forms (2D row tiles).
template <class T, int D, int BX, int BY, int PF, int OCC> struct PersistentKernels {
    static constexpr auto s1 = stage_kernel_persistent<T, D, BX, BY, 1, PF, true, OCC>;
    static constexpr auto s2 = stage_kernel_persistent<T, D, BX, BY, 2, PF, true, OCC>;
    static constexpr auto s2_split = stage_kernel_persistent<T, D, BX, BY, 2, PF, false, OCC>;
};

// CTAs of each persistent stage kernel that the whole GPU holds at once (SMs x resident CTAs
// per SM), measured when the kernels are prepared; 0 = unknown (the one-item-per-CTA kernels
// run then).
template <class T, int D, int BX, int BY, int PF, int OCC> struct ResidentCtas {
    static inline int s1 = 0, s2 = 0, s2_split = 0;
};

template <class F> static int resident_ctas(F kernel, int nt, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, nt, smem) != cudaSuccess) return 0;
    return sms * per;
}

// Grid of a manifest pass: enough CTAs to fill every SM several times.
inline unsigned pass_blocks(long long ncell) {
    long long b = (ncell + kPassThreads - 1) / kPassThreads;
    return (unsigned)(b < 1 ? 1 : (b > 152LL * 8 ? 152LL * 8 : b));
}

template <class T, int D, int BX, int BY, int PF, int OCC = 2, int MAN = 0>
static cudaError_t launch_stage_pf(const StageLaunch &L, const StageArgs<T> &A0, cudaStream_t st) {
    using S = StageShape<T, D, BX, BY>;
    using GM = Geom<D, BY>;
    using K = StageKernels<T, D, BX, BY, PF, OCC, MAN>;
    StageArgs<T> A = A0;
    const long long ncell = (long long)A.n[0] * A.n[1] * A.n[2];
    if constexpr (MAN == 1) {  // V(U_in) into the V planes, which the stage kernel then reads
        StageArgs<T> P = A0;
        for (int k = 0; k < 5; ++k) P.uout[k] = static_cast<T *>(L.vbuf[k]);
        manifest_v_kernel<T><<<pass_blocks(ncell), kPassThreads, 0, st>>>(P);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        for (int k = 0; k < 5; ++k) A.uin[k] = static_cast<const T *>(L.vbuf[k]);
    }
    const dim3 grid((unsigned)((A.n[0] + BX - 1) / BX),
                    (unsigned)((GM::IN >= 2) ? (A.n[1] + BY - 1) / BY : 1),
                    (unsigned)(GM::march ? (L.zchunks > 0 ? L.zchunks
                                                          : (A.n[GM::MA] + A.march - 1) / A.march - L.zchunk0)
                                         : 1));
    const size_t smem = S::smem_bytes;
    if constexpr (MAN == 2) {  // fluxes to HBM, then AddFlux from them
        if (L.zchunk0 != 0 || L.zchunks != 0) return cudaErrorInvalidValue;  // whole grid only
        K::s1<<<grid, S::NT, smem, st>>>(A);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (L.stage == 1)
            addflux_kernel<T, 1, true><<<pass_blocks(ncell), kPassThreads, 0, st>>>(A);
        else if (L.split)
            addflux_kernel<T, 2, false><<<pass_blocks(ncell), kPassThreads, 0, st>>>(A);
        else
            addflux_kernel<T, 2, true><<<pass_blocks(ncell), kPassThreads, 0, st>>>(A);
        return cudaGetLastError();
    } else {
        // 2D row tiles with more work items than resident CTAs: a persistent grid of the
        // resident CTAs claims the items (stage_kernel_persistent)
        if constexpr (GM::rows && MAN == 0) {
            using R = ResidentCtas<T, D, BX, BY, PF, OCC>;
            using P = PersistentKernels<T, D, BX, BY, PF, OCC>;
            const int slots = L.stage == 1 ? R::s1 : (L.split ? R::s2_split : R::s2);
            const long long items = (long long)grid.x * grid.y * grid.z;
            if (slots > 0 && items > slots && items < (1LL << 31)) {
                A.items = (int)items;
                A.tiles_x = (int)grid.x;
                A.tiles_y = (int)grid.y;
                const dim3 g((unsigned)slots);
                if (L.stage == 1)
                    P::s1<<<g, S::NT, smem, st>>>(A);
                else if (L.split)
                    P::s2_split<<<g, S::NT, smem, st>>>(A);
                else
                    P::s2<<<g, S::NT, smem, st>>>(A);
                return cudaGetLastError();
            }
        }
        if (L.stage == 1)
            K::s1<<<grid, S::NT, smem, st>>>(A);
        else if (L.split)
            K::s2_split<<<grid, S::NT, smem, st>>>(A);
        else
            K::s2<<<grid, S::NT, smem, st>>>(A);
        return cudaGetLastError();
    }
}

template <class T, int D, int BX, int BY, int PF, int OCC = 2, int MAN = 0>
static cudaError_t prepare_stage_pf() {
    using K = StageKernels<T, D, BX, BY, PF, OCC, MAN>;
    const int smem = (int)StageShape<T, D, BX, BY>::smem_bytes;
    cudaError_t e = cudaFuncSetAttribute(K::s1, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if constexpr (MAN != 2) {  // the flux kernel is the only stage kernel of manifest F
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(K::s2, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(K::s2_split, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
    if constexpr (Geom<D, BY>::rows && MAN == 0) {
        using P = PersistentKernels<T, D, BX, BY, PF, OCC>;
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(P::s1, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(P::s2, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(P::s2_split, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) {
            using R = ResidentCtas<T, D, BX, BY, PF, OCC>;
            constexpr int nt = StageShape<T, D, BX, BY>::NT;
            R::s1 = resident_ctas(P::s1, nt, (size_t)smem);
            R::s2 = resident_ctas(P::s2, nt, (size_t)smem);
            R::s2_split = resident_ctas(P::s2_split, nt, (size_t)smem);
        }
    }
    return e;
}

template <class T, int D, int BX, int BY, int PF, int OCC, int MAN = 0>
static cudaError_t run_or_prepare(const StageLaunch &L, cudaStream_t st, bool prepare_only) {
    if (prepare_only) return prepare_stage_pf<T, D, BX, BY, PF, OCC, MAN>();
    return launch_stage_pf<T, D, BX, BY, PF, OCC, MAN>(L, make_stage_args<T>(L), st);
}

// TMA-staged kernels (3D FP32): the planes of U_in come in by bulk tensor copies.  Where the
// maps cannot be made (a row pitch that is not a multiple of 16 bytes, planes not 16-byte
// aligned) the launch falls back to the look-ahead kernels of the same tile and budget.
template <class T, int D, int BX, int BY, int OCC> struct TmaKernels {
    static constexpr auto s1 = stage_kernel_tma<T, D, BX, BY, 1, true, OCC>;
    static constexpr auto s2 = stage_kernel_tma<T, D, BX, BY, 2, true, OCC>;
    static constexpr auto s2_split = stage_kernel_tma<T, D, BX, BY, 2, false, OCC>;
    static constexpr size_t smem = StageShape<T, D, BX, BY>::smem_bytes + TmaBox<BX, BY>::smem_bytes;
};

template <class T, int D, int BX, int BY, int OCC>
static cudaError_t run_or_prepare_tma(const StageLaunch &L, cudaStream_t st, bool prepare_only) {
    using K = TmaKernels<T, D, BX, BY, OCC>;
    if (prepare_only) {
        cudaError_t e = cudaFuncSetAttribute(K::s1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(K::s2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(K::s2_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem);
        if (e == cudaSuccess) e = prepare_stage_pf<T, D, BX, BY, 1, OCC>();  // the fallback
        return e;
    }
    const StageArgs<T> A = make_stage_args<T>(L);
    TmaMaps M;
    if (encode_plane_maps(&M, L.uin, L.n, TmaBox<BX, BY>::W, TmaBox<BX, BY>::H) != cudaSuccess)
        return launch_stage_pf<T, D, BX, BY, 1, OCC>(L, A, st);
    const dim3 grid((unsigned)((A.n[0] + BX - 1) / BX), (unsigned)((A.n[1] + BY - 1) / BY),
                    (unsigned)(L.zchunks > 0 ? L.zchunks : (A.n[2] + A.march - 1) / A.march - L.zchunk0));
    if (L.stage == 1)
        K::s1<<<grid, BX * BY, K::smem, st>>>(A, M);
    else if (L.split)
        K::s2_split<<<grid, BX * BY, K::smem, st>>>(A, M);
    else
        K::s2<<<grid, BX * BY, K::smem, st>>>(A, M);
    return cudaGetLastError();
}

// Both staging depths and both occupancy targets exist only for marching tiles (dim 3, and the
// row tiles of dim 2); one-plane tiles have nothing to look ahead to and small register needs.
// The manifest forms (3D tiles compiled with them) exist for the look-ahead staging and the
// default budget of the precision.
template <class T, int D, int BX, int BY, bool BOTH_PF, bool MANIFEST = false, bool TMA = false>
static cudaError_t dispatch_tile(const StageLaunch &L, cudaStream_t st, bool prepare_only) {
    if constexpr (TMA && D == 3) {
        if (L.prefetch == 2)
            return L.occupancy == 3 ? run_or_prepare_tma<T, D, BX, BY, 3>(L, st, prepare_only)
                                    : run_or_prepare_tma<T, D, BX, BY, 2>(L, st, prepare_only);
    }
    if constexpr (MANIFEST && D == 3) {
        constexpr int OCC = sizeof(T) == 4 ? 3 : 2;
        if (L.manifest == 1) return run_or_prepare<T, D, BX, BY, 1, OCC, 1>(L, st, prepare_only);
        if (L.manifest == 2) return run_or_prepare<T, D, BX, BY, 1, OCC, 2>(L, st, prepare_only);
    }
    if constexpr (BOTH_PF && Geom<D, BY>::march) {
        const bool occ3 = L.occupancy == 3;
        if (L.prefetch == 0)
            return occ3 ? run_or_prepare<T, D, BX, BY, 0, 3>(L, st, prepare_only)
                        : run_or_prepare<T, D, BX, BY, 0, 2>(L, st, prepare_only);
        if (occ3) return run_or_prepare<T, D, BX, BY, 1, 3>(L, st, prepare_only);
    }
    return run_or_prepare<T, D, BX, BY, 1, 2>(L, st, prepare_only);
}

}  // namespace hydro

// One dispatch case: (BX, BY) compiled for (T, D), with both staging depths (PF2 = true) or
// only the default one.
#define HYDRO_STAGE_CASE(T, D, BX, BY, PF2) \
    if (L.tile_x == BX && L.tile_y == BY) return dispatch_tile<T, D, BX, BY, PF2>(L, st, prepare_only);
// The same with the manifest forms compiled too (dim 3).
#define HYDRO_STAGE_CASE_M(T, D, BX, BY, PF2) \
    if (L.tile_x == BX && L.tile_y == BY) return dispatch_tile<T, D, BX, BY, PF2, true>(L, st, prepare_only);
// The same with the TMA-staged kernels compiled too (dim 3 FP32).
#define HYDRO_STAGE_CASE_MT(T, D, BX, BY, PF2) \
    if (L.tile_x == BX && L.tile_y == BY) return dispatch_tile<T, D, BX, BY, PF2, true, true>(L, st, prepare_only);
