// Fused RK-stage kernel of the compressible-Euler step (arXiv:1204.4779, section 4.1).
//
// One launch computes, for every cell i,
//     U_out[i] = U_base[i] + sum_a (c dt / dr_a) (F_a[i - e_a/2] - F_a[i + e_a/2]),
//     F_a = HLLC_a(MinBee faces of V(U_in)),
// i.e. Flux_a followed by AddFlux (Eq. eqAddFlux):
//     stage 1: U_in = U0, U_base = U0, U_out = U1, c = 1/2
//     stage 2: U_in = U1, U_base = U0, U_out = U0 (in place), c = 1
// Stage 2 also computes the CFL signal of every new cell and the dt of the next step
// (warp shuffle -> CTA -> one atomic per CTA -> the last CTA finalises dt on the device).
//
// Tiling.  A CTA owns a BX x BY tile of the (x, y) plane (dim 1: a BX row).  In dim 3 it
// marches through `march` z-planes.  Per plane:
//   * V of the tile plus a cross-shaped halo of two cells (the stencil needs no corners) is
//     recovered from U and staged in shared memory; the halo comes from global memory with
//     the boundary condition applied by index remapping (no ghost cells in HBM);
//   * every x- and y-face of the tile is evaluated ONCE (BX+1 per row, BY+1 per column),
//     spread over all threads, the fluxes kept in shared memory;
//   * the z-face above each column is evaluated by its own thread from a register pipeline
//     of the column's V(z), V(z+1), V(z+2), carrying the z-slope and the flux of the face
//     below from the previous plane, so z-faces are also evaluated once;
//   * the next plane's loads (own column three planes ahead, the halo of the plane after
//     next) are issued before the current plane's flux work, hiding their latency; the
//     shared planes are double-buffered, so a plane costs one barrier.
// HBM traffic per stage: read U_in and U_base, write U_out once; halo re-reads hit L2.
#pragma once

#include <type_traits>

#include "hydro_device.cuh"
#include "tma.cuh"

namespace hydro {

template <class T> struct StageArgs {
    const T *uin[5];    // flux source (never written by this launch)
    const T *ubase[5];  // U0
    T *uout[5];         // U1 (stage 1) or U0 (stage 2, in place over ubase)
    int n[3];
    int periodic[3];
    int march;          // planes per CTA along the march axis
    int zchunk0;        // march chunk of blockIdx.z = 0 (a launch may cover a slab of chunks)
    int order;          // reconstruction order: 2 = MinBee slopes, 1 = face values = cell values
    int riemann;        // HLLC wave speeds: 0 = Davis, 1 = pressure-based
    double dr[3];       // cell sizes (the FP64 CFL signal divides by them)
    T inv_dr[3];        // 1 / dr in the element type (the FP32 CFL signal multiplies)
    Gas<T> gas;
    Ctrl *ctrl;
    T *flux[3][5];      // manifest F: face-flux planes per axis (faces of the cells' low sides
                        // plus the grid's high boundary, x fastest, the face axis n_a + 1 long)
    const T *frame[5];  // analytic boundaries: the ghost-cell ring (frame_index), U at the
                        // stage's time
    int ana;            // bit a set: axis a takes its ghost cells from the frame (one-plane
                        // tiles of dim 1 and 2 only)
    int items;          // > 0: persistent launch over `items` (tile, march chunk) work items,
                        // tiles_x x tiles_y tiles per chunk, x fastest; 0: one item per CTA
    int tiles_x, tiles_y;
};

// Position of ghost cell (gx, gy) of an nx x ny grid (dim 1: ny = 1, gy = 0) in the frame ring
// of two ghost layers: first per grid row its four side cells (x = -2, -1, nx, nx + 1), then
// (dim 2) the two rows below the grid and the two above it, x from -2 to nx + 1.  Size
// 4 ny + 4 (nx + 4) in dim 2, 4 in dim 1.
__host__ __device__ __forceinline__ int frame_index(int gx, int gy, int nx, int ny) {
    const int w = nx + 4;
    if (gy < 0) return 4 * ny + (gy + 2) * w + gx + 2;
    if (gy >= ny) return 4 * ny + (gy - ny + 2) * w + gx + 2;
    return gy * 4 + (gx < 0 ? gx + 2 : gx - nx + 2);
}

// CFL signal of one cell's new state, sum_a (|v_a| + c_s) / dr_a, folded into the running
// maximum smax (NaN propagates); bad: rho <= 0 or p <= 0 seen.
template <class T, int D>
__device__ __forceinline__ void cfl_signal(const T (&un)[D + 2], const StageArgs<T> &A, T &smax,
                                           bool &bad) {
    constexpr int NV = D + 2;
    T v[NV];
    prim_of_cons<T, D>(un, v, A.gas);
    T cs, s = T(0);
    if constexpr (Arith<T>::exact) {
        cs = sqrt(A.gas.g * v[NV - 1] / v[0]);
#pragma unroll
        for (int a = 0; a < D; ++a) s = s + (fabs(v[1 + a]) + cs) / A.dr[a];
    } else {
        cs = Arith<float>::sqrt_(A.gas.g * v[NV - 1] * Arith<float>::rcp(v[0]));
#pragma unroll
        for (int a = 0; a < D; ++a) s = fmaf(fabsf(v[1 + a]) + cs, A.inv_dr[a], s);
    }
    smax = (s > smax || s != s) ? s : smax;
    bad |= !(v[0] > T(0)) || !(v[NV - 1] > T(0));
}

// Tile geometry.  dim 3: a BX x BY tile of the (x, y) plane marching along z.  dim 2: a BX x BY
// tile (one plane, no march), or with BY = 1 a row of BX cells marching along y ("row tiles").
// dim 1: a row of BX cells.  IN = the in-plane axes whose faces go through shared memory; the
// march axis D - 1 (if any) has its faces in the register pipeline.
template <int D, int BY> struct Geom {
    static constexpr bool rows = (D == 2 && BY == 1);
    static constexpr bool march = (D == 3) || rows;
    static constexpr int IN = (D == 3 || (D == 2 && BY > 1)) ? 2 : 1;
    static constexpr int MA = D - 1;  // march axis
};

template <class T, int D, int BX, int BY> struct StageShape {
    static constexpr int IN = Geom<D, BY>::IN;
    static constexpr int NV = D + 2;
    static constexpr int NT = BX * BY;
    static constexpr int HX = BX + 4;
    static constexpr int HY = (IN >= 2) ? BY + 4 : 1;
    // shared plane of one field, and the flux plane, in cells; multiples of four so that the
    // 16-byte records of Cells stay aligned from plane to plane
    static constexpr int PL = (HY * HX + 3) / 4 * 4;
    static constexpr int NFX = (BX + 1) * BY;
    static constexpr int NFY = (IN >= 2) ? BX * (BY + 1) : 0;
    static constexpr int NF = (NFX + NFY + 3) / 4 * 4;
    static constexpr int NH = (IN >= 2) ? 4 * BY + 4 * BX : 4;
    static constexpr int HPT = (NH + NT - 1) / NT;  // halo cells per thread
    static constexpr int FPT = (IN >= 2) ? 3 : 2;  // in-plane face rounds per thread
    static_assert((IN >= 2 ? BX + BY : 1) <= NT, "the tile's extra faces must fit in one round");
    static constexpr size_t smem_bytes = sizeof(T) * (size_t)(2 * NV * PL + 2 * NV * NF + 2 * (NT / 32));
};

// Shared-memory records of NV values per cell (primitive states, face fluxes) in arrays of
// `stride` cells.  Generic form: one array per value.  FP32 with four or five values: the
// first four are one float4 per cell and the fifth an array after them; FP64: pairs of
// doubles as double2 plus the odd fifth.  One 128-bit access then moves four (two) values.
// The base must be 16-byte aligned and `stride` a multiple of four.
template <class T, int NV> struct Cells {
    __device__ static __forceinline__ void put(T *b, int stride, int i, const T (&v)[NV]) {
#pragma unroll
        for (int k = 0; k < NV; ++k) b[k * stride + i] = v[k];
    }
    __device__ static __forceinline__ void get(const T *b, int stride, int i, T (&v)[NV]) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = b[k * stride + i];
    }
};
template <int NV> struct Cells4f {
    static_assert(NV == 4 || NV == 5, "float4 records hold four or five values");
    __device__ static __forceinline__ void put(float *b, int stride, int i, const float (&v)[NV]) {
        reinterpret_cast<float4 *>(b)[i] = make_float4(v[0], v[1], v[2], v[3]);
        if constexpr (NV == 5) b[4 * stride + i] = v[4];
    }
    __device__ static __forceinline__ void get(const float *b, int stride, int i, float (&v)[NV]) {
        const float4 q = reinterpret_cast<const float4 *>(b)[i];
        v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
        if constexpr (NV == 5) v[4] = b[4 * stride + i];
    }
};
template <> struct Cells<float, 4> : Cells4f<4> {};
template <> struct Cells<float, 5> : Cells4f<5> {};
template <int NV> struct Cells2d {
    static_assert(NV == 4 || NV == 5, "double2 records hold four or five values");
    __device__ static __forceinline__ void put(double *b, int stride, int i, const double (&v)[NV]) {
        reinterpret_cast<double2 *>(b)[i] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(b + 2 * stride)[i] = make_double2(v[2], v[3]);
        if constexpr (NV == 5) b[4 * stride + i] = v[4];
    }
    __device__ static __forceinline__ void get(const double *b, int stride, int i, double (&v)[NV]) {
        const double2 p = reinterpret_cast<const double2 *>(b)[i];
        const double2 q = reinterpret_cast<const double2 *>(b + 2 * stride)[i];
        v[0] = p.x, v[1] = p.y, v[2] = q.x, v[3] = q.y;
        if constexpr (NV == 5) v[4] = b[4 * stride + i];
    }
};
template <> struct Cells<double, 4> : Cells2d<4> {};
template <> struct Cells<double, 5> : Cells2d<5> {};

// FP32 values are processed in pairs (k, k+1) with f32x2 instructions, the last value alone
// when NV is odd; FP64 (and anything else) value by value.  Either way each value sees the
// same operations in the same order.
template <class T, int NV> struct Pairs {
    static constexpr int n = std::is_same<T, float>::value ? NV / 2 : 0;  // packed pairs
    static constexpr int first_scalar = 2 * n;
};

// MinBee slopes d = minbee(c - m, p - c) of three consecutive cells, value by value (all zero
// for first-order reconstruction).
template <class T, int NV>
__device__ __forceinline__ void minbee_slopes(const T (&m)[NV], const T (&c)[NV], const T (&p)[NV],
                                              bool order2, T (&d)[NV]) {
    using P = Pairs<T, NV>;
    if (!order2) {
#pragma unroll
        for (int k = 0; k < NV; ++k) d[k] = T(0);
        return;
    }
    if constexpr (P::n > 0) {
#pragma unroll
        for (int j = 0; j < P::n; ++j) {
            const int k = 2 * j;
            const F2 C = f2_pack(c[k], c[k + 1]);
            float a0, a1, b0, b1;
            f2_unpack(f2_sub(C, f2_pack(m[k], m[k + 1])), a0, a1);
            f2_unpack(f2_sub(f2_pack(p[k], p[k + 1]), C), b0, b1);
            d[k] = minbee(a0, b0);
            d[k + 1] = minbee(a1, b1);
        }
    }
#pragma unroll
    for (int k = P::first_scalar; k < NV; ++k) d[k] = minbee(c[k] - m[k], p[k] - c[k]);
}

// Face states from cell values and slopes: out = v + s * d / 2 (s = +1: the cell's upper face,
// -1: its lower face).
template <class T, int NV>
__device__ __forceinline__ void half_step(const T (&v)[NV], const T (&d)[NV], T s, T (&out)[NV]) {
    using P = Pairs<T, NV>;
    if constexpr (P::n > 0) {
        const F2 h = f2_pack(0.5f * s, 0.5f * s);
#pragma unroll
        for (int j = 0; j < P::n; ++j) {
            const int k = 2 * j;
            f2_unpack(f2_fma(h, f2_pack(d[k], d[k + 1]), f2_pack(v[k], v[k + 1])), out[k], out[k + 1]);
        }
    }
#pragma unroll
    for (int k = P::first_scalar; k < NV; ++k)
        out[k] = (s > T(0)) ? v[k] + T(0.5) * d[k] : v[k] - T(0.5) * d[k];
}

// MinBee faces of four consecutive cells q0..q3 along a normal: L = upper face of q1,
// R = lower face of q2 (the two sides of the face between q1 and q2).
template <class T, int NV>
__device__ __forceinline__ void minbee_face_pair(const T (&q0)[NV], const T (&q1)[NV],
                                                 const T (&q2)[NV], const T (&q3)[NV], T (&L)[NV],
                                                 T (&R)[NV]) {
    using P = Pairs<T, NV>;
    if constexpr (P::n > 0) {
        const F2 h = f2_pack(0.5f, 0.5f), mh = f2_pack(-0.5f, -0.5f);
#pragma unroll
        for (int j = 0; j < P::n; ++j) {
            const int k = 2 * j;
            const F2 Q1 = f2_pack(q1[k], q1[k + 1]), Q2 = f2_pack(q2[k], q2[k + 1]);
            float a0, a1, b0, b1, c0, c1;
            f2_unpack(f2_sub(Q1, f2_pack(q0[k], q0[k + 1])), a0, a1);
            f2_unpack(f2_sub(Q2, Q1), b0, b1);
            f2_unpack(f2_sub(f2_pack(q3[k], q3[k + 1]), Q2), c0, c1);
            f2_unpack(f2_fma(h, f2_pack(minbee(a0, b0), minbee(a1, b1)), Q1), L[k], L[k + 1]);
            f2_unpack(f2_fma(mh, f2_pack(minbee(b0, c0), minbee(b1, c1)), Q2), R[k], R[k + 1]);
        }
    }
#pragma unroll
    for (int k = P::first_scalar; k < NV; ++k) {
        const T d01 = q1[k] - q0[k], d12 = q2[k] - q1[k], d23 = q3[k] - q2[k];
        L[k] = q1[k] + T(0.5) * minbee(d01, d12);
        R[k] = q2[k] - T(0.5) * minbee(d12, d23);
    }
}

// AddFlux of one cell (Eq. eqAddFlux), the axes summed in order:
//     un = base + cx (fw - fe) [+ cy (fs - fn)] [+ cz (zm - zp)],
// the fluxes of its low and high faces per axis, all in axis order; HAS_Y: an in-plane y axis
// (faces fs, fn); HAS_M: a march axis (the last axis; faces zm, zp).
template <class T, int NV, bool HAS_Y, bool HAS_M>
__device__ __forceinline__ void add_fluxes(const T (&base)[NV], T cx, const T (&fw)[NV],
                                           const T (&fe)[NV], T cy, const T (&fs)[NV],
                                           const T (&fn)[NV], T cz, const T (&zm)[NV],
                                           const T (&zp)[NV], T (&un)[NV]) {
    using P = Pairs<T, NV>;
    if constexpr (P::n > 0) {
        const F2 CX = f2_pack(cx, cx), CY = f2_pack(cy, cy), CZ = f2_pack(cz, cz);
#pragma unroll
        for (int j = 0; j < P::n; ++j) {
            const int k = 2 * j;
            auto pk = [k](const float (&a)[NV]) { return f2_pack(a[k], a[k + 1]); };
            F2 sum = f2_mul(CX, f2_sub(pk(fw), pk(fe)));
            if constexpr (HAS_Y) sum = f2_fma(CY, f2_sub(pk(fs), pk(fn)), sum);
            if constexpr (HAS_M) sum = f2_fma(CZ, f2_sub(pk(zm), pk(zp)), sum);
            f2_unpack(f2_add(pk(base), sum), un[k], un[k + 1]);
        }
    }
#pragma unroll
    for (int k = P::first_scalar; k < NV; ++k) {
        T sum = cx * (fw[k] - fe[k]);
        if constexpr (HAS_Y) sum = sum + cy * (fs[k] - fn[k]);
        if constexpr (HAS_M) sum = sum + cz * (zm[k] - zp[k]);
        un[k] = base[k] + sum;
    }
}

// Flux of one in-plane face from the staged primitive plane.  `o`: shared index of the
// first of the four cells q0..q3 along the normal, `s`: their stride, `a`: the normal axis
// (0 or 1).  Face between q1 and q2.  Writes the flux in axis order to record f of sF.
template <class T, int D, int PL, int NF>
__device__ __forceinline__ void inplane_face(const T *__restrict__ sV, T *__restrict__ sF, int o,
                                             int s, int a, int f, const Gas<T> &G,
                                             int order = 2, int riemann = 0) {
    constexpr int NV = D + 2;
    using C = Cells<T, NV>;
    T q1[NV], q2[NV], L[NV], R[NV];  // axis order (rho, v_x, [v_y, [v_z]], p)
    C::get(sV, PL, o + s, q1);
    C::get(sV, PL, o + 2 * s, q2);
    if (order == 2) {
        T q0[NV], q3[NV];
        C::get(sV, PL, o, q0);
        C::get(sV, PL, o + 3 * s, q3);
        minbee_face_pair<T, NV>(q0, q1, q2, q3, L, R);
    } else {
#pragma unroll
        for (int k = 0; k < NV; ++k) L[k] = q1[k], R[k] = q2[k];
    }
    // velocities normal first, then the tangential ones in increasing axis order
    T vl[D], vr[D], F[NV];
    vl[0] = (D >= 2 && a) ? L[2] : L[1];
    vr[0] = (D >= 2 && a) ? R[2] : R[1];
    if constexpr (D >= 2) {
        vl[1] = a ? L[1] : L[2];
        vr[1] = a ? R[1] : R[2];
    }
    if constexpr (D == 3) vl[2] = L[3], vr[2] = R[3];
    hllc<T, D, false>(L[0], vl, L[NV - 1], R[0], vr, R[NV - 1], G, F, riemann);
    T Fa[NV];  // back to axis order
    Fa[0] = F[0];
    Fa[1] = (D >= 2 && a) ? F[2] : F[1];
    if constexpr (D >= 2) Fa[2] = a ? F[1] : F[2];
    if constexpr (D == 3) Fa[3] = F[3];
    Fa[NV - 1] = F[NV - 1];
    C::put(sF, NF, f, Fa);
}

// Flux of the march-axis face (z in dim 3, y for row tiles in dim 2) between a column's cells
// at plane z (lower) and z+1 (upper) from their primitive states and MinBee slopes.  Returned
// normal-first: (mass, m_normal, tangential momenta in axis order, E).
template <class T, int D>
__device__ __forceinline__ void march_face(const T (&Vlo)[D + 2], const T (&dlo)[D + 2],
                                           const T (&Vhi)[D + 2], const T (&dhi)[D + 2],
                                           const Gas<T> &G, T (&F)[D + 2], int riemann = 0) {
    T L[D + 2], R[D + 2];
    half_step<T, D + 2>(Vlo, dlo, T(1), L);
    half_step<T, D + 2>(Vhi, dhi, T(-1), R);
    T vl[D], vr[D];
    vl[0] = L[D];
    vr[0] = R[D];
#pragma unroll
    for (int b = 1; b < D; ++b) vl[b] = L[b], vr[b] = R[b];
    hllc<T, D, true>(L[0], vl, L[D + 1], R[0], vr, R[D + 1], G, F, riemann);
}

// Shared-memory position (lx, ly) of halo task h of a BX x BY tile (the cross-shaped two-cell
// halo: two columns left and right of the tile rows, two rows below and above the tile
// columns); false if h is past the last task.
template <int IN, int BX, int BY>
__device__ __forceinline__ bool halo_task(int h, int &lx, int &ly) {
    constexpr int NH = (IN >= 2) ? 4 * BY + 4 * BX : 4;
    if (h >= NH) {
        lx = ly = 0;
        return false;
    }
    if constexpr (IN >= 2) {
        if (h < 4 * BY) {
            const int c = h & 3;
            ly = (h >> 2) + 2;
            lx = c < 2 ? c : BX + c;
        } else {
            const int g = h - 4 * BY;
            const int r = g / BX;
            lx = g % BX + 2;
            ly = r < 2 ? r : BY + r;
        }
    } else {
        const int c = h & 3;
        lx = c < 2 ? c : BX + c;
        ly = 0;
    }
    return true;
}

// In-plane face task j of thread tid: shared base index o, stride s, normal axis a, face id.
// Round 0: the x-face on the low side of the thread's cell; round 1 (IN = 2): the y-face on
// its low side; last round: the tile's high x-column (BY faces) and high y-row (BX faces), on
// the lowest threads.  Rounds 0 and 1 give each warp one row of unit-stride faces.
template <int IN, int BX, int BY>
__device__ __forceinline__ bool face_task(int tid, int j, int &o, int &s, int &a, int &id) {
    constexpr int HX = BX + 4;
    constexpr int NFX = (BX + 1) * BY;
    const int tx = tid % BX, ty = tid / BX;
    int c, r;
    bool ok = true;
    if (j == 0) {
        c = tx, r = ty, a = 0;
    } else if (IN >= 2 && j == 1) {
        c = tx, r = ty, a = 1;
    } else {
        const int e = tid;
        if (e < BY) {
            c = BX, r = e, a = 0;
        } else {
            c = e - BY, r = BY, a = 1;
            ok = (IN >= 2) && e < BX + BY;
        }
    }
    if (!ok) c = r = a = 0;
    if (a == 0) {  // x-face between tile cells (c-1, r) and (c, r)
        o = ((IN >= 2) ? (r + 2) * HX : 0) + c;
        s = 1;
        id = r * (BX + 1) + c;
    } else {  // y-face between (c, r-1) and (c, r)
        o = r * HX + c + 2;
        s = HX;
        id = NFX + r * BX + c;
    }
    return ok;
}

// Resident CTAs per SM the register budget targets: OCC 256-thread CTAs' worth of warps in
// FP32 (OCC = 2: ~128 registers per thread, 3: ~80); FP64 keeps one CTA's budget.
template <class T, int NT, int OCC = 2> struct MinBlocks {
    static constexpr int v = OCC * 256 / NT;
    static constexpr int value = (sizeof(T) == 4) ? (v > 1 ? v : 1) : 1;
};

// One CTA's work: the tile at (x0, y0) of the in-plane axes, planes [zb, ze) of the march axis
// (one plane without a march).  The AddFlux coefficients (c dt)/dr_a of the in-plane x and y
// axes and of the march axis are cx, cy, cz.  CFL (stage 2): also return the CFL signal maximum
// of the thread's new cells in smax and whether any was non-positive or non-finite in bad.
// Uses the caller's dynamic shared memory (StageShape::smem_bytes).  A caller that runs it
// twice in one CTA puts a barrier between the calls: the second call's first shared-memory
// writes may hit planes the first call's last reads still use.
// MAN (dim 3 only): 0 = nothing stored in HBM between the parts of a stage; 1 = manifest V:
// A.uin holds primitive planes (a pass stored V(U_in)), so loaded cells need no recovery;
// 2 = manifest F: store every face flux in A.flux instead of updating (a pass applies them).
// PF = 2 (dim 3, FP32): the planes of U_in come into shared memory by TMA (tma.cuh): one box
// per plane (tile plus halo) in a ring of TmaBox::slots slots, the box of plane p issued once
// the box of plane p - slots has been read; the own cell of plane z + 2 and the halo of plane
// z + 1 are read from their boxes, cells outside the grid by plain loads with the boundary
// remap.  M: the tensor maps of U_in's fields (a __grid_constant__ kernel parameter).
template <class T, int D, int BX, int BY, int STAGE, int PF, bool CFL, int MAN = 0>
__device__ __forceinline__ void stage_tile(const StageArgs<T> &A, int x0, int y0, int zb, int ze,
                                           unsigned char *smem_raw, T cx, T cy, T cz, T &smax,
                                           bool &bad, const TmaMaps *M = nullptr) {
    static_assert(MAN == 0 || D == 3, "the manifest forms are compiled for 3D grids");
    using S = StageShape<T, D, BX, BY>;
    using GM = Geom<D, BY>;
    constexpr int NV = S::NV, NT = S::NT, HX = S::HX, PL = S::PL, IN = GM::IN, MA = GM::MA;
    constexpr bool MARCH = GM::march;
    constexpr int NFX = S::NFX, NF = S::NF, HPT = S::HPT, FPT = S::FPT;
    // two primitive planes and two flux planes, alternating between planes so that one barrier
    // per plane suffices
    T *const sV0 = reinterpret_cast<T *>(smem_raw);
    T *const sV1 = sV0 + NV * PL;
    T *const sF0 = sV1 + NV * PL;
    T *const sF1 = sF0 + NV * NF;
    const Gas<T> G = A.gas;
    const bool order2 = A.order == 2;
    constexpr bool TMA = PF == 2;
    static_assert(!TMA || (D == 3 && std::is_same<T, float>::value && MAN == 0),
                  "TMA staging is compiled for the 3D FP32 tiles");
    using TB = TmaBox<BX, BY>;
    // V of a loaded cell: recovered from U, or already V (manifest V)
    auto recover = [&](const T (&u)[NV], T (&v)[NV]) {
        if constexpr (MAN == 1) {
#pragma unroll
            for (int k = 0; k < NV; ++k) v[k] = u[k];
        } else {
            prim_of_cons<T, D>(u, v, G);
        }
    };

    const int tid = threadIdx.x;
    const int tx = tid % BX, ty = tid / BX;
    const int nx = A.n[0];
    const int ny = (IN >= 2) ? A.n[1] : 1;             // in-plane y extent
    const int nz = MARCH ? A.n[MA] : 1;                // march extent
    const int pstride = nx * ny;                       // cells per plane
    const int x = x0 + tx, y = y0 + ty;
    const bool active = (x < nx) && (y < ny);
    // plane offset of the cell (gx, gy) at most two cells outside the grid: boundary remap, or
    // for a cell outside on exactly one axis that takes analytic ghost cells, -(1 + its
    // position in the frame ring)
    auto cell_off = [&](int gx, int gy) -> int {
        if constexpr (!MARCH) {
            if (A.ana) {
                const bool ox = gx < 0 || gx >= nx;
                const bool oy = (IN >= 2) && (gy < 0 || gy >= ny);
                if (ox != oy && gx >= -2 && gx < nx + 2 && gy >= -2 && gy < ny + 2 &&
                    (A.ana & (ox ? 1 : 2)))
                    return -1 - frame_index(gx, (IN >= 2) ? gy : 0, nx, ny);
            }
        }
        const int yg = (IN >= 2) ? remap(gy, ny, A.periodic[1]) : 0;
        return yg * nx + remap(gx, nx, A.periodic[0]);
    };
    const int own_off = cell_off(x, y);
    const int own_s = (IN >= 2) ? (ty + 2) * HX + (tx + 2) : (tx + 2);

    // halo cells of this thread: plane offset and shared index.  Halo work goes to the
    // highest threads, the tile's extra row/column of faces to the lowest.
    int h_off[HPT], h_s[HPT], h_b[HPT];
    bool h_ok[HPT], h_in[HPT];
#pragma unroll
    for (int j = 0; j < HPT; ++j) {
        int lx, ly;
        h_ok[j] = halo_task<IN, BX, BY>((NT - 1 - tid) + j * NT, lx, ly);
        h_off[j] = cell_off(x0 + lx - 2, y0 + ly - 2);
        h_s[j] = ly * HX + lx;
        // TMA: the cell's place in the plane's box, and whether the box holds it (inside the
        // grid; outside, the box holds zeros and the boundary remap applies)
        h_b[j] = ly * TB::W + lx + 2;
        const int gx = x0 + lx - 2, gy = y0 + ly - 2;
        h_in[j] = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
    }
    const int own_b = (ty + 2) * TB::W + tx + 4;
    const bool own_in = active;

    // in-plane face tasks of this thread
    int f_o[FPT], f_s[FPT], f_a[FPT], f_id[FPT];
    bool f_ok[FPT];
#pragma unroll
    for (int j = 0; j < FPT; ++j) f_ok[j] = face_task<IN, BX, BY>(tid, j, f_o[j], f_s[j], f_a[j], f_id[j]);

    const int pz = MARCH ? A.periodic[MA] : 1;

    // TMA ring: TB::slots slots of one plane's box each, an mbarrier per slot.  Box of plane p:
    // slot q % slots and use q / slots of that slot, q = p - (zb + 1); boxes zb + 1 (if the
    // chunk has two planes or more: the halo of plane zb + 1) to ze + 1 (the own cell of plane
    // ze - 1 + 2) are issued, and every issued box is waited for.
    constexpr int NSL = TB::slots;
    float *sBox = nullptr;
    uint32_t bar0 = 0;
    if constexpr (TMA) {
        const uintptr_t a = (reinterpret_cast<uintptr_t>(smem_raw) + S::smem_bytes + 127) &
                            ~static_cast<uintptr_t>(127);
        sBox = reinterpret_cast<float *>(a);
        bar0 = smem_u32(sBox + NSL * 5 * TB::cells);
    }
    auto issue_box = [&](int p) {  // one thread
        const int q = p - (zb + 1);
        const uint32_t bar = bar0 + 8u * (q % NSL);
        const uint32_t dst = smem_u32(sBox + (q % NSL) * 5 * TB::cells);
        const int zr = remap(p, nz, pz);
        mbar_arrive_expect_tx(bar, TB::bytes);
#pragma unroll
        for (int k = 0; k < 5; ++k)
            tma_load_3d(dst + 4u * k * TB::cells, &M->map[k], x0 - 4, y0 - 2, zr, bar);
    };
    bool tma_dead = false;  // a wait of this thread timed out: wait no more
    auto wait_box = [&](int p) -> const float * {
        const int q = p - (zb + 1);
        if (!tma_dead && !mbar_wait(bar0 + 8u * (q % NSL), (q / NSL) & 1, &A.ctrl->status)) {
            atomicOr(&A.ctrl->status, STATUS_TIMEOUT);
            tma_dead = true;
        }
        return sBox + (q % NSL) * 5 * TB::cells;
    };
    if constexpr (TMA) {
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < NSL; ++k) mbar_init(bar0 + 8u * k, 1);
            mbar_init_fence();
            if (zb + 1 < ze) issue_box(zb + 1);
#pragma unroll
            for (int k = 2; k <= NSL; ++k)
                if (zb + k <= ze + 1) issue_box(zb + k);
        }
    }

    auto load_u = [&](T (&u)[NV], int zr, int off) {
        if constexpr (!MARCH) {
            if (off < 0) {  // analytic ghost cell
#pragma unroll
                for (int k = 0; k < NV; ++k) u[k] = __ldg(A.frame[k] + (-1 - off));
                return;
            }
        }
        const int i = zr * pstride + off;
#pragma unroll
        for (int k = 0; k < NV; ++k) u[k] = __ldg(A.uin[k] + i);
    };
    // V of one plane into shared memory: the own cell from registers, the halo recovered
    // from its prefetched conserved values
    auto stage_plane = [&](T *sV, const T (&Vown)[NV], T (&ph)[HPT][NV]) {
        Cells<T, NV>::put(sV, PL, own_s, Vown);
#pragma unroll
        for (int j = 0; j < HPT; ++j) {
            if (h_ok[j]) {
                T vh[NV];
                recover(ph[j], vh);
                Cells<T, NV>::put(sV, PL, h_s[j], vh);
            }
        }
    };

    // register pipeline along the march axis: V(z), V(z+1), slope at z, flux of face z - 1/2,
    // raw U of plane z+2 (own column) and of the next plane's halo
    T Vc[NV], Vn[NV], dzc[NV], Fzm[NV];
    T pown[NV];
    T phalo[HPT][NV];

    if constexpr (MARCH) {
        T u[NV], Vm2[NV], Vm1[NV], dzm[NV];
        load_u(u, remap(zb - 2, nz, pz), own_off);
        recover(u, Vm2);
        load_u(u, remap(zb - 1, nz, pz), own_off);
        recover(u, Vm1);
        load_u(u, remap(zb, nz, pz), own_off);
        recover(u, Vc);
        load_u(u, remap(zb + 1, nz, pz), own_off);
        recover(u, Vn);
        minbee_slopes<T, NV>(Vm2, Vm1, Vc, order2, dzm);
        minbee_slopes<T, NV>(Vm1, Vc, Vn, order2, dzc);
        march_face<T, D>(Vm1, dzm, Vc, dzc, G, Fzm, A.riemann);
        if constexpr (PF == 1) load_u(pown, remap(zb + 2, nz, pz), own_off);
    } else {
        T u[NV];
        load_u(u, 0, own_off);
        recover(u, Vc);
    }
#pragma unroll
    for (int j = 0; j < HPT; ++j)
        if (h_ok[j]) load_u(phalo[j], MARCH ? remap(zb, nz, pz) : 0, h_off[j]);
    stage_plane(sV0, Vc, phalo);
    if constexpr (MARCH && PF == 1) {
        if (zb + 1 < ze) {
#pragma unroll
            for (int j = 0; j < HPT; ++j)
                if (h_ok[j]) load_u(phalo[j], remap(zb + 1, nz, pz), h_off[j]);
        }
    }
    __syncthreads();

    // planes z + 1 ... z + 3 of the loop lie at or above 0: remap_ahead
    for (int z = zb; z < ze; ++z) {
        const bool odd = ((z - zb) & 1) != 0;
        T *const sVc = odd ? sV1 : sV0;
        T *const sVn = odd ? sV0 : sV1;
        T *const sF = odd ? sF1 : sF0;
        // U_base of the plane, consumed after the barrier
        T base[NV];
        {
            const int i = (MARCH ? z * pstride : 0) + (active ? y * nx + x : 0);
#pragma unroll
            for (int k = 0; k < NV; ++k) base[k] = active ? A.ubase[k][i] : T(0);
        }
        T Vnn[NV];
        if constexpr (MARCH && !TMA) {
            if constexpr (PF == 0) load_u(pown, remap_ahead(z + 2, nz, pz), own_off);
            recover(pown, Vnn);  // V(z+2)
            if constexpr (PF == 1) {
                if (z + 1 < ze) load_u(pown, remap_ahead(z + 3, nz, pz), own_off);
            }
        }

        // in-plane faces of plane z, each once
#pragma unroll
        for (int j = 0; j < FPT; ++j)
            if (f_ok[j])
                inplane_face<T, D, PL, NF>(sVc, sF, f_o[j], f_s[j], f_a[j], f_id[j], G, A.order,
                                           A.riemann);
        // march-axis face above this column
        T Fzp[NV], dzn[NV];
        if constexpr (MARCH) {
            if constexpr (TMA) {  // V(z+2) of the own cell from its box (issued a plane ago)
                const float *b = wait_box(z + 2);
                T u[NV];
                if (own_in) {
#pragma unroll
                    for (int k = 0; k < NV; ++k) u[k] = b[k * TB::cells + own_b];
                } else {
                    load_u(u, remap_ahead(z + 2, nz, pz), own_off);
                }
                recover(u, Vnn);
            }
            minbee_slopes<T, NV>(Vc, Vn, Vnn, order2, dzn);
            march_face<T, D>(Vc, dzc, Vn, dzn, G, Fzp, A.riemann);
            // stage plane z+1 into the other buffer, prefetch the halo of plane z+2
            if (z + 1 < ze) {
                if constexpr (PF == 0) {
#pragma unroll
                    for (int j = 0; j < HPT; ++j)
                        if (h_ok[j]) load_u(phalo[j], remap_ahead(z + 1, nz, pz), h_off[j]);
                }
                if constexpr (TMA) {  // the halo of plane z+1 from its box
                    const float *b = wait_box(z + 1);
#pragma unroll
                    for (int j = 0; j < HPT; ++j) {
                        if (!h_ok[j]) continue;
                        if (h_in[j]) {
#pragma unroll
                            for (int k = 0; k < NV; ++k) phalo[j][k] = b[k * TB::cells + h_b[j]];
                        } else {
                            load_u(phalo[j], remap_ahead(z + 1, nz, pz), h_off[j]);
                        }
                    }
                }
                stage_plane(sVn, Vn, phalo);
                if (PF == 1 && z + 2 < ze) {
#pragma unroll
                    for (int j = 0; j < HPT; ++j)
                        if (h_ok[j]) load_u(phalo[j], remap_ahead(z + 2, nz, pz), h_off[j]);
                }
            }
        }
        __syncthreads();
        // TMA: every thread is done with the box of plane z+1; its slot takes plane z+1+slots
        if constexpr (TMA) {
            if (tid == 0 && z + 1 + NSL <= ze + 1) {
                fence_proxy_async_smem();
                issue_box(z + 1 + NSL);
            }
        }

        if (active) {
            const int fxl = ty * (BX + 1) + tx;
            const int fyb = NFX + ty * BX + tx;
            T un[NV], fw[NV], fe[NV], fs[NV], fn[NV];
            Cells<T, NV>::get(sF, NF, fxl, fw);
            Cells<T, NV>::get(sF, NF, fxl + 1, fe);
            if constexpr (IN >= 2) {
                Cells<T, NV>::get(sF, NF, fyb, fs);
                Cells<T, NV>::get(sF, NF, fyb + BX, fn);
            }
            // march-axis fluxes in axis order (they come normal-first: mass, m_normal, the
            // tangential momenta in axis order, E)
            T zm[NV], zp[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const int kk = (!MARCH || k == 0 || k == NV - 1) ? k : (k == D ? 1 : k + 1);
                zm[k] = MARCH ? Fzm[kk] : T(0);
                zp[k] = MARCH ? Fzp[kk] : T(0);
            }
            if constexpr (MAN == 2) {
                // face fluxes to HBM: each cell its low faces, the last cell of a line also
                // the high face on the grid's boundary
                const long long ix = ((long long)z * ny + y) * (nx + 1) + x;
                const long long iy = ((long long)z * (ny + 1) + y) * nx + x;
                const long long iz = ((long long)z * ny + y) * nx + x;
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    A.flux[0][k][ix] = fw[k];
                    A.flux[1][k][iy] = fs[k];
                    A.flux[2][k][iz] = zm[k];
                    if (x == nx - 1) A.flux[0][k][ix + 1] = fe[k];
                    if (y == ny - 1) A.flux[1][k][iy + nx] = fn[k];
                    if (z == nz - 1) A.flux[2][k][iz + (long long)nx * ny] = zp[k];
                }
            } else {
                add_fluxes<T, NV, (IN >= 2), MARCH>(base, cx, fw, fe, cy, fs, fn, cz, zm, zp, un);
                const int i = (MARCH ? z * pstride : 0) + y * nx + x;
#pragma unroll
                for (int k = 0; k < NV; ++k) A.uout[k][i] = un[k];
                if constexpr (STAGE == 2 && CFL) cfl_signal<T, D>(un, A, smax, bad);
            }
        }
        if constexpr (MARCH) {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                Vc[k] = Vn[k];
                Vn[k] = Vnn[k];
                dzc[k] = dzn[k];
                Fzm[k] = Fzp[k];
            }
        }
    }
}

// STAGE: RK stage (1 or 2).  PF (staging depth, march tiles): 1 = the next plane's loads are
// issued one plane ahead of their use, 0 = each plane is loaded when it is staged.  FUSED
// (stage 2): 1 = the CFL signal and the next dt are reduced in this kernel's epilogue, 0 = left
// to a separate CFL pass.  OCC: resident CTAs per SM the register budget targets.
template <class T, int D, int BX, int BY, int STAGE, int PF = 1, bool FUSED = true, int OCC = 2,
          int MAN = 0>
__global__ void __launch_bounds__(BX * BY, (MinBlocks<T, BX * BY, OCC>::value))
    stage_kernel(const StageArgs<T> A) {
    using S = StageShape<T, D, BX, BY>;
    using GM = Geom<D, BY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const sRed = reinterpret_cast<T *>(smem_raw) + 2 * S::NV * S::PL + 2 * S::NV * S::NF;

    Ctrl *ctrl = A.ctrl;
    const double dt = __ldcg(&ctrl->dt);
    if (!(dt > 0.0)) return;  // uniform over the grid: no step to take
    // (c dt)/dr_a, computed once per step in FP64 by the dt finaliser
    const T cx = T(__ldcg(&ctrl->coef[STAGE - 1][0]));
    const T cy = (GM::IN >= 2) ? T(__ldcg(&ctrl->coef[STAGE - 1][1])) : T(0);
    const T cz = GM::march ? T(__ldcg(&ctrl->coef[STAGE - 1][GM::MA])) : T(0);
    const int x0 = blockIdx.x * BX;
    const int y0 = (GM::IN >= 2) ? blockIdx.y * BY : 0;
    const int zb = GM::march ? ((int)blockIdx.z + A.zchunk0) * A.march : 0;
    const int ze = GM::march ? min(zb + A.march, A.n[GM::MA]) : 1;
    T smax = T(0);
    bool bad = false;
    constexpr bool CFL = STAGE == 2 && FUSED && MAN != 2;
    stage_tile<T, D, BX, BY, STAGE, PF, CFL, MAN>(A, x0, y0, zb, ze, smem_raw, cx, cy, cz, smax, bad);
    if constexpr (CFL) reduce_signal_and_finalize<T, S::NT>(ctrl, smax, bad, true, sRed);
}

// The same stage over a persistent grid of resident CTAs (marching tiles, nothing manifest):
// A.items work items (tile, march chunk), A.tiles_x x A.tiles_y tiles per chunk, x fastest.
// CTA b takes item b, then claims the next unclaimed item from the control block's counter
// until none is left, so the last wave of a launch with few items per SM does not leave SMs
// idle.  The last CTA to stop claiming resets the counters for the next launch on the same
// control block.  Used where the items make only a few waves of CTAs (the row tiles of 2D
// grids): over many waves the hardware's own scheduling loses nothing and the claiming loop
// costs instructions.
template <class T, int D, int BX, int BY, int STAGE, int PF, bool FUSED = true, int OCC = 2>
__global__ void __launch_bounds__(BX * BY, (MinBlocks<T, BX * BY, OCC>::value))
    stage_kernel_persistent(const StageArgs<T> A) {
    using S = StageShape<T, D, BX, BY>;
    using GM = Geom<D, BY>;
    static_assert(GM::march, "persistent launches are compiled for marching tiles");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const sRed = reinterpret_cast<T *>(smem_raw) + 2 * S::NV * S::PL + 2 * S::NV * S::NF;
    __shared__ int s_item;

    Ctrl *ctrl = A.ctrl;
    const double dt = __ldcg(&ctrl->dt);
    if (!(dt > 0.0)) return;  // uniform over the grid: no step to take (and nothing claimed)
    const T cx = T(__ldcg(&ctrl->coef[STAGE - 1][0]));
    const T cy = (GM::IN >= 2) ? T(__ldcg(&ctrl->coef[STAGE - 1][1])) : T(0);
    const T cz = T(__ldcg(&ctrl->coef[STAGE - 1][GM::MA]));
    T smax = T(0);
    bool bad = false;
    constexpr bool CFL = STAGE == 2 && FUSED;
    for (int item = (int)blockIdx.x; item < A.items;) {
        const int ix = item % A.tiles_x;
        const int r = item / A.tiles_x;
        const int x0 = ix * BX;
        const int y0 = (GM::IN >= 2) ? (r % A.tiles_y) * BY : 0;
        const int zb = (r / A.tiles_y + A.zchunk0) * A.march;
        const int ze = min(zb + A.march, A.n[GM::MA]);
        stage_tile<T, D, BX, BY, STAGE, PF, CFL, 0>(A, x0, y0, zb, ze, smem_raw, cx, cy, cz, smax,
                                                    bad);
        __syncthreads();  // the tile's last shared-memory reads are done; s_item is free
        if (threadIdx.x == 0) s_item = (int)gridDim.x + (int)atomicAdd(&ctrl->claim, 1u);
        __syncthreads();
        item = s_item;
    }
    if (threadIdx.x == 0 && atomicAdd(&ctrl->claim_done, 1u) == gridDim.x - 1) {
        atomicExch(&ctrl->claim, 0u);
        atomicExch(&ctrl->claim_done, 0u);
    }
    if constexpr (CFL) reduce_signal_and_finalize<T, S::NT>(ctrl, smax, bad, true, sRed);
}

// The same stage with the planes of U_in staged by TMA (PF = 2; 3D FP32).  Dynamic shared
// memory: StageShape::smem_bytes + TmaBox::smem_bytes.
template <class T, int D, int BX, int BY, int STAGE, bool FUSED = true, int OCC = 2>
__global__ void __launch_bounds__(BX * BY, (MinBlocks<T, BX * BY, OCC>::value))
    stage_kernel_tma(const __grid_constant__ StageArgs<T> A, const __grid_constant__ TmaMaps M) {
    using S = StageShape<T, D, BX, BY>;
    using GM = Geom<D, BY>;
    static_assert(D == 3, "TMA staging marches along z");
    static_assert(TmaBox<BX, BY>::aligned, "TMA boxes of this tile would not stay aligned");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const sRed = reinterpret_cast<T *>(smem_raw) + 2 * S::NV * S::PL + 2 * S::NV * S::NF;

    Ctrl *ctrl = A.ctrl;
    const double dt = __ldcg(&ctrl->dt);
    if (!(dt > 0.0)) return;  // uniform over the grid: no step to take
    const T cx = T(__ldcg(&ctrl->coef[STAGE - 1][0]));
    const T cy = T(__ldcg(&ctrl->coef[STAGE - 1][1]));
    const T cz = T(__ldcg(&ctrl->coef[STAGE - 1][2]));
    const int x0 = blockIdx.x * BX;
    const int y0 = blockIdx.y * BY;
    const int zb = ((int)blockIdx.z + A.zchunk0) * A.march;
    const int ze = min(zb + A.march, A.n[GM::MA]);
    T smax = T(0);
    bool bad = false;
    constexpr bool CFL = STAGE == 2 && FUSED;
    stage_tile<T, D, BX, BY, STAGE, 2, CFL, 0>(A, x0, y0, zb, ze, smem_raw, cx, cy, cz, smax, bad,
                                               &M);
    if constexpr (CFL) reduce_signal_and_finalize<T, S::NT>(ctrl, smax, bad, true, sRed);
}

// ---- the passes of the manifest forms (dim 3) ---------------------------------------------

constexpr int kPassThreads = 256;

// Manifest V: the primitive planes of the stage's input, V(U_in) -> A.uout, with the same
// recovery the stage kernel applies to the cells it loads.
template <class T>
__global__ void __launch_bounds__(kPassThreads) manifest_v_kernel(const StageArgs<T> A) {
    constexpr int D = 3, NV = 5;
    const long long ncell = (long long)A.n[0] * A.n[1] * A.n[2];
    for (long long i = (long long)blockIdx.x * kPassThreads + threadIdx.x; i < ncell;
         i += (long long)gridDim.x * kPassThreads) {
        T u[NV], v[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) u[k] = __ldg(A.uin[k] + i);
        prim_of_cons<T, D>(u, v, A.gas);
#pragma unroll
        for (int k = 0; k < NV; ++k) A.uout[k][i] = v[k];
    }
}

// Manifest F: AddFlux from the stored face fluxes (Eq. eqAddFlux, the same arithmetic as the
// fused stage kernel's update), with stage 2's CFL signal and dt reduction when FUSED.
template <class T, int STAGE, bool FUSED>
__global__ void __launch_bounds__(kPassThreads) addflux_kernel(const StageArgs<T> A) {
    constexpr int D = 3, NV = 5;
    __shared__ T sRed[2 * kPassThreads / 32];
    Ctrl *ctrl = A.ctrl;
    const double dt = __ldcg(&ctrl->dt);
    if (!(dt > 0.0)) return;
    const T cx = T(__ldcg(&ctrl->coef[STAGE - 1][0]));
    const T cy = T(__ldcg(&ctrl->coef[STAGE - 1][1]));
    const T cz = T(__ldcg(&ctrl->coef[STAGE - 1][2]));
    const int nx = A.n[0], ny = A.n[1], nz = A.n[2];
    const long long plane = (long long)nx * ny, ncell = plane * nz;
    T smax = T(0);
    bool bad = false;
    for (long long i = (long long)blockIdx.x * kPassThreads + threadIdx.x; i < ncell;
         i += (long long)gridDim.x * kPassThreads) {
        const int x = (int)(i % nx);
        const long long yz = i / nx;
        const int y = (int)(yz % ny);
        const long long z = yz / ny;
        const long long ix = (z * ny + y) * (nx + 1) + x;
        const long long iy = (z * (ny + 1) + y) * nx + x;
        T base[NV], fw[NV], fe[NV], fs[NV], fn[NV], zm[NV], zp[NV], un[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            base[k] = A.ubase[k][i];
            fw[k] = A.flux[0][k][ix];
            fe[k] = A.flux[0][k][ix + 1];
            fs[k] = A.flux[1][k][iy];
            fn[k] = A.flux[1][k][iy + nx];
            zm[k] = A.flux[2][k][i];
            zp[k] = A.flux[2][k][i + plane];
        }
        add_fluxes<T, NV, true, true>(base, cx, fw, fe, cy, fs, fn, cz, zm, zp, un);
#pragma unroll
        for (int k = 0; k < NV; ++k) A.uout[k][i] = un[k];
        if constexpr (STAGE == 2 && FUSED) cfl_signal<T, D>(un, A, smax, bad);
    }
    if constexpr (STAGE == 2 && FUSED)
        reduce_signal_and_finalize<T, kPassThreads>(ctrl, smax, bad, true, sRed);
}

}  // namespace hydro
