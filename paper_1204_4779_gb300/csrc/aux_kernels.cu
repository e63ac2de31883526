// Auxiliary kernels: the CFL pass that gives the first dt of a step call, the FP64
// conserved-totals audit, and primitive <-> conserved conversion.  Compiled with
// --fmad=false so the FP64 forms follow the plain formulas operation by operation.
#include <type_traits>

#include "hydro_device.cuh"
#include "hydro_internal.h"

namespace hydro {

namespace {

constexpr int kAuxThreads = 256;

template <class T> struct AuxT {
    const T *u[5];
    T *out[5];
    long long ncell, first;
    unsigned total_blocks;
    double dr[3];
    T inv_dr[3];
    Gas<T> gas;
    Ctrl *ctrl;
};

template <class T> AuxT<T> make_aux(const AuxArgs &A) {
    AuxT<T> a;
    for (int k = 0; k < 5; ++k) {
        a.u[k] = static_cast<const T *>(A.u[k]);
        a.out[k] = static_cast<T *>(A.out[k]);
    }
    a.ncell = A.ncell;
    a.first = A.first;
    a.total_blocks = A.total_blocks;
    for (int d = 0; d < 3; ++d) {
        a.dr[d] = A.dr[d];
        a.inv_dr[d] = T(1.0 / A.dr[d]);
    }
    a.gas = make_gas<T>(A.gamma);
    a.ctrl = static_cast<Ctrl *>(A.ctrl);
    return a;
}

// Max over cells of sum_a (|v_a| + c_s) / dr_a, c_s = sqrt(gamma p / rho); flags rho <= 0 or
// p <= 0; the last CTA turns the max into dt (cfl / max, clipped onto t_end).  A pass may be
// split into launches over consecutive cell ranges [first, first + ncell) whose CTAs add up to
// total_blocks: the running maximum and the CTA count then span the launches.
template <class T, int D, bool ADVANCE>
__global__ void __launch_bounds__(kAuxThreads) cfl_kernel(const AuxT<T> A) {
    __shared__ T sred[2 * kAuxThreads / 32];
    constexpr int NV = D + 2;
    // after a step that did not run (dt = 0: t reached t_end, or a failed state) there is
    // nothing to reduce; the same for every CTA
    if (ADVANCE && !(__ldcg(&A.ctrl->dt) > 0.0)) return;
    T smax = T(0);
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long end = A.first + A.ncell;
    for (long long i = A.first + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < end;
         i += stride) {
        T u[NV], v[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) u[k] = A.u[k][i];
        prim_of_cons<T, D>(u, v, A.gas);
        T s = T(0);
        if constexpr (Arith<T>::exact) {
            const T cs = sqrt(A.gas.g * v[NV - 1] / v[0]);
#pragma unroll
            for (int a = 0; a < D; ++a) s = s + (fabs(v[1 + a]) + cs) / T(A.dr[a]);
        } else {
            const T cs = Arith<float>::sqrt_(A.gas.g * v[NV - 1] * Arith<float>::rcp(v[0]));
#pragma unroll
            for (int a = 0; a < D; ++a) s = fmaf(fabsf(v[1 + a]) + cs, A.inv_dr[a], s);
        }
        smax = (s > smax || s != s) ? s : smax;
        bad |= !(v[0] > T(0)) || !(v[NV - 1] > T(0));
    }
    reduce_signal_and_finalize<T, kAuxThreads>(A.ctrl, smax, bad, ADVANCE, sred, A.total_blocks);
}

// Totals, level 1: CTA b sums the contiguous chunk [b*chunk, (b+1)*chunk) of each plane
// (fixed per-thread strides, fixed shared-memory tree) into partials[k * nparts + b].  FP64
// states are summed in FP64.  FP32 states: each thread sums its cells in double-float (every
// FP32 value is exact in it; TwoSum and renormalisation per addition keep about 48 bits of the
// running sum) and converts its sums to FP64 once, so that the FP64 pipe, at 1/62 of the FP32
// rate, does not bound the pass; the tree over the threads runs in FP64.
template <class T, int NV>
__global__ void __launch_bounds__(kAuxThreads)
    totals_partial_kernel(const AuxT<T> A, double *partials, int nparts) {
    __shared__ double s[kAuxThreads];
    const long long chunk = (A.ncell + nparts - 1) / nparts;
    const long long b0 = (long long)blockIdx.x * chunk;
    const long long b1 = b0 + chunk < A.ncell ? b0 + chunk : A.ncell;
    double tsum[NV];
    if constexpr (sizeof(T) == 4) {
        DF acc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = {0.0f, 0.0f};
        for (long long i = b0 + threadIdx.x; i < b1; i += kAuxThreads) {
#pragma unroll
            for (int k = 0; k < NV; ++k) acc_add(acc[k], {A.u[k][i], 0.0f});
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) tsum[k] = (double)acc[k].hi + (double)acc[k].lo;
    } else {
#pragma unroll
        for (int k = 0; k < NV; ++k) tsum[k] = 0.0;
        for (long long i = b0 + threadIdx.x; i < b1; i += kAuxThreads) {
#pragma unroll
            for (int k = 0; k < NV; ++k) tsum[k] += (double)A.u[k][i];
        }
    }
    for (int k = 0; k < NV; ++k) {
        const double acc = tsum[k];
        s[threadIdx.x] = acc;
        __syncthreads();
        for (int w = kAuxThreads / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) partials[k * nparts + blockIdx.x] = s[0];
        __syncthreads();
    }
}

// Totals, level 2: one CTA sums the partials of each plane in a fixed order and scales by
// the cell volume; output (mass, M_x, M_y, M_z, E) into ctrl->totals.
template <int NV>
__global__ void __launch_bounds__(kAuxThreads)
    totals_final_kernel(const double *partials, int nparts, double vol, Ctrl *ctrl) {
    __shared__ double s[kAuxThreads];
    for (int k = 0; k < NV; ++k) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < nparts; i += kAuxThreads) acc += partials[k * nparts + i];
        s[threadIdx.x] = acc;
        __syncthreads();
        for (int w = kAuxThreads / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const int slot = (k == NV - 1) ? 4 : k;
            ctrl->totals[slot] = s[0] * vol;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = NV - 1; k < 4; ++k) ctrl->totals[k] = 0.0;  // inactive momenta
}

// U(V): m_a = rho v_a, E = p/(gamma-1) + rho v^2/2 (v^2 summed in axis order); V(U) inverse.
template <class T, int D>
__global__ void __launch_bounds__(kAuxThreads) convert_kernel(const AuxT<T> A, int to_cons) {
    constexpr int NV = D + 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.ncell; i += stride) {
        T in[NV], out[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) in[k] = A.u[k][i];
        if (to_cons) {
            const T rho = in[0];
            T v2 = T(0);
            out[0] = rho;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                out[1 + a] = rho * in[1 + a];
                v2 = v2 + in[1 + a] * in[1 + a];
            }
            out[NV - 1] = in[NV - 1] / A.gas.gm1 + T(0.5) * rho * v2;
        } else {
            // exact quotient form in both precisions
            const T rho = in[0];
            T kin = T(0);
            out[0] = rho;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                out[1 + a] = in[1 + a] / rho;
                kin = kin + in[1 + a] * out[1 + a];
            }
            out[NV - 1] = A.gas.gm1 * (in[NV - 1] - T(0.5) * kin);
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) A.out[k][i] = out[k];
    }
}

int grid_for(long long ncell) {
    long long b = (ncell + kAuxThreads - 1) / kAuxThreads;
    const long long cap = 152LL * 8;  // enough CTAs to fill every SM several times
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

template <class T, bool ADV> cudaError_t cfl_t(const AuxArgs &A, cudaStream_t st) {
    const AuxT<T> a = make_aux<T>(A);
    const int g = grid_for(A.ncell);
    switch (A.dim) {
        case 1: cfl_kernel<T, 1, ADV><<<g, kAuxThreads, 0, st>>>(a); break;
        case 2: cfl_kernel<T, 2, ADV><<<g, kAuxThreads, 0, st>>>(a); break;
        case 3: cfl_kernel<T, 3, ADV><<<g, kAuxThreads, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t totals_t(const AuxArgs &A, double *partials, int nparts, double vol, cudaStream_t st) {
    const AuxT<T> a = make_aux<T>(A);
    Ctrl *c = static_cast<Ctrl *>(A.ctrl);
    switch (A.dim + 2) {
        case 3:
            totals_partial_kernel<T, 3><<<nparts, kAuxThreads, 0, st>>>(a, partials, nparts);
            totals_final_kernel<3><<<1, kAuxThreads, 0, st>>>(partials, nparts, vol, c);
            break;
        case 4:
            totals_partial_kernel<T, 4><<<nparts, kAuxThreads, 0, st>>>(a, partials, nparts);
            totals_final_kernel<4><<<1, kAuxThreads, 0, st>>>(partials, nparts, vol, c);
            break;
        case 5:
            totals_partial_kernel<T, 5><<<nparts, kAuxThreads, 0, st>>>(a, partials, nparts);
            totals_final_kernel<5><<<1, kAuxThreads, 0, st>>>(partials, nparts, vol, c);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class T> cudaError_t convert_t(const AuxArgs &A, int to_cons, cudaStream_t st) {
    const AuxT<T> a = make_aux<T>(A);
    const int g = grid_for(A.ncell);
    switch (A.dim) {
        case 1: convert_kernel<T, 1><<<g, kAuxThreads, 0, st>>>(a, to_cons); break;
        case 2: convert_kernel<T, 2><<<g, kAuxThreads, 0, st>>>(a, to_cons); break;
        case 3: convert_kernel<T, 3><<<g, kAuxThreads, 0, st>>>(a, to_cons); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

unsigned cfl_blocks(long long ncell) { return (unsigned)grid_for(ncell); }

cudaError_t launch_cfl(const AuxArgs &A, cudaStream_t st, bool advance) {
    if (A.prec == 1) return advance ? cfl_t<float, true>(A, st) : cfl_t<float, false>(A, st);
    return advance ? cfl_t<double, true>(A, st) : cfl_t<double, false>(A, st);
}

cudaError_t launch_totals(const AuxArgs &A, double *partials, int nparts, double vol,
                          cudaStream_t st) {
    return A.prec == 1 ? totals_t<float>(A, partials, nparts, vol, st)
                       : totals_t<double>(A, partials, nparts, vol, st);
}

cudaError_t launch_convert(const AuxArgs &A, int to_cons, cudaStream_t st) {
    return A.prec == 1 ? convert_t<float>(A, to_cons, st) : convert_t<double>(A, to_cons, st);
}

}  // namespace hydro
