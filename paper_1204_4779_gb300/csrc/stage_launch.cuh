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
    A.order = L.order == 1 ? 1 : 2;
    A.riemann = L.riemann;
    A.gas = make_gas<T>(L.gamma);
    A.ctrl = static_cast<Ctrl *>(L.ctrl);
    return A;
}

// The kernels of one (T, D, tile) for one staging depth PF and occupancy target OCC: stage 1,
// stage 2 with the fused dt reduction, stage 2 without it.
template <class T, int D, int BX, int BY, int PF, int OCC> struct StageKernels {
    static constexpr auto s1 = stage_kernel<T, D, BX, BY, 1, PF, true, OCC>;
    static constexpr auto s2 = stage_kernel<T, D, BX, BY, 2, PF, true, OCC>;
    static constexpr auto s2_split = stage_kernel<T, D, BX, BY, 2, PF, false, OCC>;
};

template <class T, int D, int BX, int BY, int PF, int OCC = 2>
static cudaError_t launch_stage_pf(const StageLaunch &L, const StageArgs<T> &A, cudaStream_t st) {
    using S = StageShape<T, D, BX, BY>;
    using GM = Geom<D, BY>;
    using K = StageKernels<T, D, BX, BY, PF, OCC>;
    const dim3 grid((unsigned)((A.n[0] + BX - 1) / BX),
                    (unsigned)((GM::IN >= 2) ? (A.n[1] + BY - 1) / BY : 1),
                    (unsigned)(GM::march ? (L.zchunks > 0 ? L.zchunks
                                                          : (A.n[GM::MA] + A.march - 1) / A.march - L.zchunk0)
                                         : 1));
    const size_t smem = S::smem_bytes;
    if (L.stage == 1)
        K::s1<<<grid, S::NT, smem, st>>>(A);
    else if (L.split)
        K::s2_split<<<grid, S::NT, smem, st>>>(A);
    else
        K::s2<<<grid, S::NT, smem, st>>>(A);
    return cudaGetLastError();
}

template <class T, int D, int BX, int BY, int PF, int OCC = 2>
static cudaError_t prepare_stage_pf() {
    using K = StageKernels<T, D, BX, BY, PF, OCC>;
    const int smem = (int)StageShape<T, D, BX, BY>::smem_bytes;
    cudaError_t e = cudaFuncSetAttribute(K::s1, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(K::s2, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(K::s2_split, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

template <class T, int D, int BX, int BY, int PF, int OCC>
static cudaError_t run_or_prepare(const StageLaunch &L, cudaStream_t st, bool prepare_only) {
    if (prepare_only) return prepare_stage_pf<T, D, BX, BY, PF, OCC>();
    return launch_stage_pf<T, D, BX, BY, PF, OCC>(L, make_stage_args<T>(L), st);
}

// Both staging depths and both occupancy targets exist only for marching tiles (dim 3, and the
// row tiles of dim 2); one-plane tiles have nothing to look ahead to and small register needs.
template <class T, int D, int BX, int BY, bool BOTH_PF>
static cudaError_t dispatch_tile(const StageLaunch &L, cudaStream_t st, bool prepare_only) {
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
