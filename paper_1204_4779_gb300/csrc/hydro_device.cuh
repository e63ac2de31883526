// Device building blocks of the compressible-Euler step (arXiv:1204.4779, section 4.1):
// primitive recovery, the MinBee slope, the HLLC face flux, boundary index remapping and the
// on-device dt control block.
//
// Two arithmetic modes, chosen by the element type:
//  * double: every operation is written in the order of the plain formulas (divisions stay
//    divisions, no reciprocals), and the FP64 translation units are compiled with
//    --fmad=false, so each operation is one correctly rounded IEEE operation;
//  * float:  the stencil runs in FP32 with fused multiply-adds and the approximate MUFU
//    reciprocal and square root (rcp.approx / sqrt.approx).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace hydro {

// ----------------------------------------------------------------- control block ----------

// One per context, in the workspace.  Written by the CFL pass and by the last CTA of every
// RK stage-2 launch; read by every CTA of the stage kernels.
struct Ctrl {
    double t;               // time of the state the next step starts from
    double dt;              // dt of the next step; 0 = no further step in this call
    double t_end;           // <= 0: no clipping
    double cfl;
    double dt_last;         // dt of the last completed step
    unsigned long long sig64;  // running max of the CFL signal, FP64 bit pattern
    unsigned int sig32;        // running max of the CFL signal, FP32 bit pattern
    unsigned int blocks_done;  // CTAs finished in the current reduction launch
    unsigned int status;       // bit 0: non-finite / non-positive value seen
    int steps;              // steps completed since the CFL pass
    int clipped;            // the next step is clipped onto t_end
    unsigned int claim;       // persistent stage launches: work items claimed beyond the first
    unsigned int claim_done;  // CTAs of the current persistent launch that stopped claiming
    int pad;
    double totals[5];       // output of the totals reduction
    double dr[3];           // cell sizes (set by the host with t, t_end, cfl)
    double coef[2][3];      // (dt/2)/dr_a and dt/dr_a of the next step, for RK stages 1 and 2
};
static_assert(sizeof(Ctrl) <= 256, "the control block has 256 bytes in every workspace");

enum : unsigned int {
    STATUS_NONFINITE = 1u,  // non-finite, rho <= 0 or p <= 0 seen
    STATUS_TIMEOUT = 2u,    // a bounded wait on an mbarrier gave up
};

// ------------------------------------------------------------------- arithmetic -----------

template <class T> struct Arith;

template <> struct Arith<double> {
    static constexpr bool exact = true;
    __device__ static __forceinline__ double div(double a, double b) { return a / b; }
    __device__ static __forceinline__ double sqrt_(double a) { return sqrt(a); }
};

template <> struct Arith<float> {
    static constexpr bool exact = false;
    __device__ static __forceinline__ float rcp(float a) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
        return r;
    }
    __device__ static __forceinline__ float div(float a, float b) { return a * rcp(b); }
    __device__ static __forceinline__ float sqrt_(float a) {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
        return r;
    }
};

// Packed FP32 pairs: Blackwell's f32x2 add/sub/mul/fma apply one operation to two FP32 values
// held in a 64-bit register pair, so one issued instruction does the work of two.  Each lane
// rounds as the scalar instruction would (round to nearest, flush-to-zero like the FP32 units).
struct F2 {
    unsigned long long r;
};
__device__ __forceinline__ F2 f2_pack(float a, float b) {
    F2 v;
    asm("mov.b64 %0, {%1, %2};" : "=l"(v.r) : "f"(a), "f"(b));
    return v;
}
__device__ __forceinline__ void f2_unpack(F2 v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v.r));
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    F2 d;
    asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b) {
    F2 d;
    asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
    F2 d;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
// a * b + c, one rounding per lane
__device__ __forceinline__ F2 f2_fma(F2 a, F2 b, F2 c) {
    F2 d;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d.r) : "l"(a.r), "l"(b.r), "l"(c.r));
    return d;
}

// Double-float arithmetic: a value carried as an unevaluated sum hi + lo of two FP32 numbers
// (Dekker's and Knuth's error-free transformations, as used in double-double arithmetic).  The
// additions are plain IEEE operations in the order written; the translation units that use
// them either compile with --fmad=false or use no contractible product next to them.
struct DF {
    float hi, lo;
};
// a + b exactly as hi + lo (Knuth's TwoSum, six operations, any magnitudes)
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
// (hi + lo)^2 as a pair: hi^2 exactly by TwoProduct with an FMA, plus 2 hi lo (lo^2 dropped)
__device__ __forceinline__ DF square(DF x) {
    const float p = x.hi * x.hi;
    float e = fmaf(x.hi, x.hi, -p);
    e = fmaf(x.hi + x.hi, x.lo, e);
    return {p, e};
}
// running sum s += x: TwoSum of the high parts, low parts added, then renormalised so that
// |lo| <= ulp(hi) / 2 (Fast2Sum)
__device__ __forceinline__ void acc_add(DF &s, DF x) {
    const DF t = two_sum(s.hi, x.hi);
    const float e = t.lo + (s.lo + x.lo);
    const float h = t.hi + e;
    s.lo = e - (h - t.hi);
    s.hi = h;
}

template <class T> struct Gas {
    T g;        // gamma
    T gm1;      // gamma - 1
    T inv_gm1;  // 1 / (gamma - 1)  (FP32 mode only)
};

template <class T> __host__ __device__ inline Gas<T> make_gas(double gamma) {
    Gas<T> G;
    G.g = T(gamma);
    G.gm1 = T(gamma - 1.0);
    G.inv_gm1 = T(1.0 / (gamma - 1.0));
    return G;
}

// V(U) for one cell: v_a = m_a / rho, p = (gamma - 1)(E - rho v^2 / 2), the kinetic term
// summed in axis order as m_a v_a.
template <class T, int D>
__device__ __forceinline__ void prim_of_cons(const T (&u)[D + 2], T (&v)[D + 2], const Gas<T> &G) {
    const T rho = u[0];
    v[0] = rho;
    if constexpr (Arith<T>::exact) {
        T kin = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            v[1 + a] = u[1 + a] / rho;
            kin = kin + u[1 + a] * v[1 + a];
        }
        v[D + 1] = G.gm1 * (u[D + 1] - T(0.5) * kin);
    } else {
        const T ir = Arith<float>::rcp(rho);
        T kin = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            v[1 + a] = u[1 + a] * ir;
            kin = fmaf(u[1 + a], v[1 + a], kin);
        }
        v[D + 1] = G.gm1 * fmaf(-0.5f, kin, u[D + 1]);
    }
}

// MinBee slope of Eq. eqInterpolateSingle from the two one-sided differences:
// 0 if d01 d12 < 0, else the one of smaller magnitude (d12 on a tie).
__device__ __forceinline__ double minbee(double d01, double d12) {
    return (d01 * d12 < 0.0) ? 0.0 : (fabs(d01) < fabs(d12) ? d01 : d12);
}
// FP32 form in three ALU operations: min.xorsign.abs gives min(|a|, |b|) carrying a negative
// sign exactly when the signs of a and b differ; clamping at zero yields 0 for opposite signs;
// the sign of a restores the slope's sign.  Same values as the form above (up to the sign of
// a zero slope).
__device__ __forceinline__ float minbee(float d01, float d12) {
    float m;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(m) : "f"(d01), "f"(d12));
    return copysignf(fmaxf(m, 0.0f), d01);
}

// HLLC flux through a face whose normal is axis a (Toro, Spruce & Speares; Davis wave-speed
// estimates), from the reconstructed primitive states on its lower (L) and upper (R) side.
// Velocities and the returned flux are in NORMAL-FIRST order: (normal, tangential in
// increasing axis order).  Flux components: (mass, normal momentum, tangential momenta,
// energy).  NLAST: the normal axis is the last axis (only the kinetic-energy summation order
// of the exact mode depends on it: v^2 is summed in axis order).
// riemann: wave-speed estimate, 0 = Davis, 1 = pressure-based (Toro's PVRS: p_pv from the
// arithmetic means, p* = max(0, p_pv), q_K = 1 or sqrt(1 + (g+1)/(2g) (p*/p_K - 1)) behind a
// shock, S_L = u_L - a_L q_L, S_R = u_R + a_R q_R).
template <class T, int D, bool NLAST>
__device__ __forceinline__ void hllc(T rl, const T (&vl)[D], T pl, T rr, const T (&vr)[D], T pr,
                                     const Gas<T> &G, T (&F)[D + 2], int riemann = 0) {
    using A = Arith<T>;
    const T ul = vl[0], ur = vr[0];
    T al, ar, irl = T(0), irr = T(0);
    if constexpr (A::exact) {
        al = A::sqrt_(G.g * pl / rl);
        ar = A::sqrt_(G.g * pr / rr);
    } else {
        irl = Arith<float>::rcp(rl);
        irr = Arith<float>::rcp(rr);
        al = A::sqrt_(G.g * pl * irl);
        ar = A::sqrt_(G.g * pr * irr);
    }
    T SL, SR;
    if (riemann == 0) {
        SL = fmin(ul - al, ur - ar);
        SR = fmax(ul + al, ur + ar);
    } else {
        const T rbar = T(0.5) * (rl + rr);
        const T abar = T(0.5) * (al + ar);
        const T ppv = T(0.5) * (pl + pr) - T(0.5) * (ur - ul) * rbar * abar;
        const T ps = fmax(T(0), ppv);
        T ql = T(1), qr = T(1);
        if constexpr (A::exact) {
            const T c = (G.g + T(1)) / (T(2) * G.g);
            if (!(ps <= pl)) ql = sqrt(T(1) + c * (ps / pl - T(1)));
            if (!(ps <= pr)) qr = sqrt(T(1) + c * (ps / pr - T(1)));
        } else {
            const T c = (G.g + 1.0f) * (0.5f * Arith<float>::rcp(G.g));
            if (!(ps <= pl)) ql = A::sqrt_(fmaf(c, ps * Arith<float>::rcp(pl) - 1.0f, 1.0f));
            if (!(ps <= pr)) qr = A::sqrt_(fmaf(c, ps * Arith<float>::rcp(pr) - 1.0f, 1.0f));
        }
        SL = ul - al * ql;
        SR = ur + ar * qr;
    }
    const T ml = rl * (SL - ul);
    const T mr = rr * (SR - ur);
    T Ss;
    if constexpr (A::exact)
        Ss = (pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur)) / (ml - mr);
    else
        Ss = A::div(fmaf(ul, ml, pr - pl) - ur * mr, ml - mr);

    // F_L if S_L >= 0; F*_L if S* >= 0; F*_R if S_R > 0; else F_R.
    const bool left = (T(0) <= SL) || (T(0) <= Ss);
    const bool star = !(T(0) <= SL) && ((T(0) <= Ss) || (T(0) < SR));
    const T r = left ? rl : rr;
    const T p = left ? pl : pr;
    const T S = left ? SL : SR;
    T v[D];
#pragma unroll
    for (int b = 0; b < D; ++b) v[b] = left ? vl[b] : vr[b];
    const T u = v[0];

    // kinetic energy in axis order
    T v2 = T(0);
    if constexpr (NLAST) {
#pragma unroll
        for (int b = 1; b < D; ++b) v2 = v2 + v[b] * v[b];
        v2 = v2 + v[0] * v[0];
    } else {
#pragma unroll
        for (int b = 0; b < D; ++b) v2 = v2 + v[b] * v[b];
    }

    T U[D + 2], FK[D + 2];
    U[0] = r;
    FK[0] = r * u;
#pragma unroll
    for (int b = 0; b < D; ++b) U[1 + b] = r * v[b];
    if constexpr (A::exact)
        U[D + 1] = p / G.gm1 + T(0.5) * r * v2;
    else
        U[D + 1] = fmaf(0.5f * r, v2, p * G.inv_gm1);
    FK[1] = U[1] * u + p;
#pragma unroll
    for (int b = 1; b < D; ++b) FK[1 + b] = U[1 + b] * u;
    FK[D + 1] = u * (U[D + 1] + p);

    // star state: rho (S - u)/(S - S*) (1, S*, v_t, E/rho + (S* - u)(S* + p/(rho (S - u))))
    T chi, eterm;
    if constexpr (A::exact) {
        chi = r * (S - u) / (S - Ss);
        eterm = U[D + 1] / r + (Ss - u) * (Ss + p / (r * (S - u)));
    } else {
        // S - S* is non-zero in both star branches; outside them it is replaced by 1 so the
        // (discarded) star state stays finite and the blend below can be a single FMA.
        const T ir = left ? irl : irr;
        const T m = r * (S - u);
        chi = m * Arith<float>::rcp(star ? S - Ss : T(1));
        eterm = fmaf(Ss - u, fmaf(p, Arith<float>::rcp(m), Ss), U[D + 1] * ir);
    }
    T Us[D + 2];
    Us[0] = chi;
    Us[1] = chi * Ss;
#pragma unroll
    for (int b = 1; b < D; ++b) Us[1 + b] = chi * v[b];
    Us[D + 1] = chi * eterm;
    if constexpr (A::exact) {
#pragma unroll
        for (int k = 0; k < D + 2; ++k) F[k] = star ? FK[k] + S * (Us[k] - U[k]) : FK[k];
    } else {
        const T Se = star ? S : T(0);  // F_K + 0 (U* - U_K) = F_K outside the star branches
#pragma unroll
        for (int k = 0; k < D + 2; ++k) F[k] = fmaf(Se, Us[k] - U[k], FK[k]);
    }
}

// Boundary remap of a cell index at most two cells outside [0, n): periodic wraps once,
// outflow (zero gradient) clamps; the final clamp also keeps the unused positions of a ragged
// tile (more than two cells outside) in bounds.
__device__ __forceinline__ int remap(int i, int n, int periodic) {
    if (periodic) i = i < 0 ? i + n : (i >= n ? i - n : i);
    return min(max(i, 0), n - 1);
}
// The same for an index known to be >= 0 (the planes ahead of a marching tile): only the
// upper side can be outside, and the result equals remap(i, n, periodic).
__device__ __forceinline__ int remap_ahead(int i, int n, int periodic) {
    return min((periodic && i >= n) ? i - n : i, n - 1);
}

// ------------------------------------------------------------- dt finalisation ------------

template <class T> __device__ __forceinline__ double take_signal(Ctrl *c);
template <> __device__ __forceinline__ double take_signal<float>(Ctrl *c) {
    unsigned int b = atomicExch(&c->sig32, 0u);
    return (double)__uint_as_float(b);
}
template <> __device__ __forceinline__ double take_signal<double>(Ctrl *c) {
    unsigned long long b = atomicExch(&c->sig64, 0ull);
    return __longlong_as_double((long long)b);
}

template <class T> __device__ __forceinline__ void push_signal(Ctrl *c, T s);
template <> __device__ __forceinline__ void push_signal<float>(Ctrl *c, float s) {
    atomicMax(&c->sig32, __float_as_uint(s));
}
template <> __device__ __forceinline__ void push_signal<double>(Ctrl *c, double s) {
    atomicMax(&c->sig64, (unsigned long long)__double_as_longlong(s));
}

// Run by one thread of the last CTA of a reduction launch.  `advance`: a step with dt = c->dt
// has just completed (no step ran if that dt is 0, e.g. once t reached t_end).  Then dt of the
// next step = cfl / max signal, clipped onto t_end.
template <class T> __device__ void finalize_dt(Ctrl *c, bool advance) {
    volatile Ctrl *vc = c;
    if (advance && vc->dt > 0.0) {
        const double dt = vc->dt;
        vc->t = vc->clipped ? vc->t_end : vc->t + dt;
        vc->dt_last = dt;
        vc->steps = vc->steps + 1;
    }
    const double s = take_signal<T>(c);
    const double t = vc->t, t_end = vc->t_end;
    double dt = 0.0;
    int clipped = 0;
    if (!(s <= 1.7976931348623157e308) || !(s > 0.0)) {  // NaN, inf or no signal
        atomicOr(&c->status, STATUS_NONFINITE);
    } else if (vc->status == 0u) {
        dt = vc->cfl / s;
        if (t_end > 0.0) {
            if (t >= t_end) {
                dt = 0.0;
            } else if (dt >= t_end - t) {
                dt = t_end - t;
                clipped = 1;
            }
        }
    }
    if (atomicOr(&c->status, 0u) != 0u) dt = 0.0;
    vc->dt = dt;
    vc->clipped = clipped;
    // AddFlux coefficients of both stages, in the order of Eq. eqAddFlux: (c dt) / dr_a
    for (int a = 0; a < 3; ++a) {
        vc->coef[0][a] = (0.5 * dt) / vc->dr[a];
        vc->coef[1][a] = dt / vc->dr[a];
    }
    __threadfence();
}

// Block-wide max of a non-negative value (NaN propagates as the largest bit pattern), then
// one atomic per CTA; the last of `nblocks` contributions (0: every CTA of the launch)
// finalises dt.  Call from all threads.
template <class T, int NT>
__device__ __forceinline__ void reduce_signal_and_finalize(Ctrl *ctrl, T smax, bool bad,
                                                           bool advance, T *sred,
                                                           unsigned int nblocks = 0) {
    // warp max on the bit patterns (order-free and exact)
    using U = typename std::conditional<sizeof(T) == 4, unsigned int, unsigned long long>::type;
    U bits;
    if constexpr (sizeof(T) == 4)
        bits = __float_as_uint(smax);
    else
        bits = (unsigned long long)__double_as_longlong(smax);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        U other = __shfl_xor_sync(0xffffffffu, bits, o);
        bits = other > bits ? other : bits;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int anybad = __syncthreads_or(bad ? 1 : 0);
    U *sb = reinterpret_cast<U *>(sred);
    if (lane == 0) sb[warp] = bits;
    __syncthreads();
    if (threadIdx.x == 0) {
        U m = 0;
#pragma unroll 1
        for (int w = 0; w < NT / 32; ++w) m = sb[w] > m ? sb[w] : m;
        T bm;
        if constexpr (sizeof(T) == 4)
            bm = __uint_as_float(m);
        else
            bm = __longlong_as_double((long long)m);
        push_signal<T>(ctrl, bm);
        if (anybad) atomicOr(&ctrl->status, STATUS_NONFINITE);
        __threadfence();
        if (nblocks == 0) nblocks = gridDim.x * gridDim.y * gridDim.z;
        const unsigned int prev = atomicAdd(&ctrl->blocks_done, 1u);
        if (prev == nblocks - 1) {
            __threadfence();
            finalize_dt<T>(ctrl, advance);
            atomicExch(&ctrl->blocks_done, 0u);
        }
    }
}

}  // namespace hydro
