// Launch helpers of the fused RK-stage kernel: grid shape, dynamic shared memory and the
// table of compiled tile shapes (BX, BY) per precision and dimension.
#pragma once

#include "hydro_internal.h"
#include "stage_kernel.cuh"

namespace hydro {

template <class T, int D, int BX, int BY>
static cudaError_t launch_stage_inst(int stage, const StageArgs<T> &A, cudaStream_t st) {
    using S = StageShape<T, D, BX, BY>;
    const dim3 grid((unsigned)((A.n[0] + BX - 1) / BX),
                    (unsigned)((D >= 2) ? (A.n[1] + BY - 1) / BY : 1),
                    (unsigned)((D == 3) ? (A.n[2] + A.march - 1) / A.march : 1));
    const size_t smem = S::smem_bytes;
    if (stage == 1)
        stage_kernel<T, D, BX, BY, 1><<<grid, S::NT, smem, st>>>(A);
    else
        stage_kernel<T, D, BX, BY, 2><<<grid, S::NT, smem, st>>>(A);
    return cudaGetLastError();
}

template <class T, int D, int BX, int BY>
static cudaError_t prepare_stage_inst() {
    using S = StageShape<T, D, BX, BY>;
    const int smem = (int)S::smem_bytes;
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<T, D, BX, BY, 1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(stage_kernel<T, D, BX, BY, 2>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

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
    A.gas = make_gas<T>(L.gamma);
    A.ctrl = static_cast<Ctrl *>(L.ctrl);
    return A;
}

}  // namespace hydro

// One dispatch case: (BX, BY) compiled for (T, D).
#define HYDRO_STAGE_CASE(T, D, BX, BY)                                                     \
    if (L.tile_x == BX && L.tile_y == BY) {                                                \
        if (prepare_only) return prepare_stage_inst<T, D, BX, BY>();                       \
        return launch_stage_inst<T, D, BX, BY>(L.stage, make_stage_args<T>(L), st);        \
    }
