// Ghost-layer exchange through buffers: the pack and unpack kernels a slab decomposition of the
// grid over several GPUs puts its sends and receives between.  Pack copies the two cell layers
// next to a side of an axis (the layers the neighbour across that side needs as its ghost
// layers) from the stage's input into a contiguous buffer; unpack writes a received buffer into
// the ghost ring (frame_index) on the opposite side, where the stage kernel's halo loads read
// it.  On one GPU the grid is its own neighbour across both ends (the periodic wrap): the buffer
// packed at the high end is unpacked into the low-side ghosts and vice versa, which reproduces
// the periodic boundary through the exchange path.
//
// Buffer layout per (axis, side): [field k][layer l][j], j running along the grid's other axis
// (dim 1: one cell).  Layer l packed at the high end is cell n - 2 + l, at the low end cell l;
// the receiving ghost -2 + l (low side) or n + l (high side) takes layer l.
#include <string.h>

#include "../../include/hydro.h"
#include "hydro_device.cuh"
#include "hydro_internal.h"
#include "stage_kernel.cuh"

namespace hydro {
namespace {

constexpr int kExThreads = 256;

struct ExArgs {
    int dim, nx, ny, nv;
    int axes;                // bit a: axis a exchanges
    const void *uin[5];      // the stage's input planes
    void *buf[2][2];         // [axis][side]: nv * 2 * m elements each
    void *frame[5];
};

// cells along the other axis of axis a (the buffer's j extent)
__host__ __device__ inline int ex_m(const ExArgs &e, int a) { return a == 0 ? e.ny : e.nx; }

// One thread per (axis, side, layer, j): all fields of that cell.
template <class T>
__global__ void __launch_bounds__(kExThreads) pack_kernel(const ExArgs e) {
    int i = blockIdx.x * kExThreads + threadIdx.x;
    for (int a = 0; a < e.dim; ++a) {
        if (!(e.axes >> a & 1)) continue;
        const int m = ex_m(e, a), per_side = 2 * m;
        if (i >= 2 * per_side) {
            i -= 2 * per_side;
            continue;
        }
        const int side = i / per_side, r = i % per_side, l = r / m, j = r % m;
        const int n = a == 0 ? e.nx : e.ny;
        const int c = side ? n - 2 + l : l;  // the cell along the axis (n >= 2 checked at create)
        const long long idx = a == 0 ? (long long)j * e.nx + c : (long long)c * e.nx + j;
        T *b = static_cast<T *>(e.buf[a][side]);
        for (int k = 0; k < e.nv; ++k)
            b[(long long)k * per_side + r] = static_cast<const T *>(e.uin[k])[idx];
        return;
    }
}

// One thread per (axis, receiving side, layer, j): the buffer packed at the OTHER end of the
// same axis (the wrap) into the ghost ring.
template <class T>
__global__ void __launch_bounds__(kExThreads) unpack_kernel(const ExArgs e) {
    int i = blockIdx.x * kExThreads + threadIdx.x;
    for (int a = 0; a < e.dim; ++a) {
        if (!(e.axes >> a & 1)) continue;
        const int m = ex_m(e, a), per_side = 2 * m;
        if (i >= 2 * per_side) {
            i -= 2 * per_side;
            continue;
        }
        const int side = i / per_side, r = i % per_side, l = r / m, j = r % m;
        const int n = a == 0 ? e.nx : e.ny;
        const int g = side ? n + l : -2 + l;  // ghost position along the axis
        const int ring = a == 0 ? frame_index(g, e.dim >= 2 ? j : 0, e.nx, e.ny)
                                : frame_index(j, g, e.nx, e.ny);
        const T *b = static_cast<const T *>(e.buf[a][side ^ 1]);
        for (int k = 0; k < e.nv; ++k)
            static_cast<T *>(e.frame[k])[ring] = b[(long long)k * per_side + r];
        return;
    }
}

}  // namespace

long long exchange_buffer_cells(int dim, long long nx, long long ny, int axis) {
    const long long m = axis == 0 ? (dim >= 2 ? ny : 1) : nx;
    return (long long)(dim + 2) * 2 * m;
}

cudaError_t launch_exchange(const ExchangeLaunch &L, cudaStream_t st) {
    ExArgs e;
    memset(&e, 0, sizeof e);
    e.dim = L.dim;
    e.nx = L.nx;
    e.ny = L.dim >= 2 ? L.ny : 1;
    e.nv = L.dim + 2;
    e.axes = L.axes;
    long long total = 0;
    for (int a = 0; a < L.dim; ++a) {
        if (!(L.axes >> a & 1)) continue;
        total += 2LL * 2 * (a == 0 ? e.ny : e.nx);
        for (int s = 0; s < 2; ++s) e.buf[a][s] = L.buf[a][s];
    }
    for (int k = 0; k < e.nv; ++k) {
        e.uin[k] = L.uin[k];
        e.frame[k] = L.frame[k];
    }
    if (total == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((total + kExThreads - 1) / kExThreads);
    if (L.prec == HYDRO_F32) {
        pack_kernel<float><<<blocks, kExThreads, 0, st>>>(e);
        unpack_kernel<float><<<blocks, kExThreads, 0, st>>>(e);
    } else {
        pack_kernel<double><<<blocks, kExThreads, 0, st>>>(e);
        unpack_kernel<double><<<blocks, kExThreads, 0, st>>>(e);
    }
    return cudaGetLastError();
}

}  // namespace hydro
