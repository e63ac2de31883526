// Analytic-solution boundaries (arXiv:1204.4779, section 4.3): outside the unit square the
// convergence tests substitute the exact solution as boundary condition at every time.  Before
// each RK stage a small kernel writes the conserved form of the solution at the stage's time
// (t for stage 1, t + dt/2 for stage 2, read from the device control block, so the fill is part
// of the captured step graphs) into the ring of two ghost layers around the grid; the stage
// kernel's halo loads read that ring for the cells outside the grid on an analytic axis.
//
// The solutions are the section's waves rotated by theta about (1/2, 1/2): with the coordinate
// along the wave s = (x - 1/2) cos theta + (y - 1/2) sin theta + 1/2,
//   1 entropy wave: rho = 2 + sin(2 pi (s - t)), v = (cos theta, sin theta), p = 1;
//   2 sound wave:   rho = gamma (1 + A w), v = A w (cos theta, sin theta), p = 1 + gamma A w,
//                   w = sin(2 pi (s - t)) (sound speed 1; exact to first order in A);
//   3 shock tube:   the exact solution of Sod's Riemann problem, (rho, u, p) = (1, 0, 1) for
//                   s < 1/2 and (0.125, 0, 0.1) for s > 1/2 at t = 0, sampled at s - 1/2 = xi t
//                   with the normal velocity u along (cos theta, sin theta).
// The ghost values are evaluated in FP64 and rounded to the element type.
#include <math.h>
#include <string.h>

#include "../../include/hydro.h"
#include "hydro_device.cuh"
#include "hydro_internal.h"

namespace hydro {
namespace {

constexpr int kFrameThreads = 256;

// Exact Riemann-problem solution of an ideal gas (the pressure-function iteration of Toro,
// Riemann Solvers and Numerical Methods for Fluid Dynamics, ch. 4): star pressure and velocity
// on the host, sampling on the device.
struct Prim1 {
    double r, u, p;
};

double pressure_fn(double p, const Prim1 &K, double g, double *dfdp) {
    const double a = sqrt(g * K.p / K.r);
    if (p > K.p) {  // shock
        const double Ak = 2.0 / ((g + 1.0) * K.r), Bk = (g - 1.0) / (g + 1.0) * K.p;
        const double q = sqrt(Ak / (p + Bk));
        *dfdp = q * (1.0 - 0.5 * (p - K.p) / (p + Bk));
        return (p - K.p) * q;
    }
    const double e = (g - 1.0) / (2.0 * g);  // rarefaction
    *dfdp = pow(p / K.p, -(g + 1.0) / (2.0 * g)) / (K.r * a);
    return 2.0 * a / (g - 1.0) * (pow(p / K.p, e) - 1.0);
}

void star_state(const Prim1 &L, const Prim1 &R, double g, double *ps, double *us) {
    const double aL = sqrt(g * L.p / L.r), aR = sqrt(g * R.p / R.r);
    // linearised guess, kept positive
    double p = 0.5 * (L.p + R.p) - 0.125 * (R.u - L.u) * (L.r + R.r) * (aL + aR);
    if (!(p > 1e-8)) p = 1e-8;
    for (int it = 0; it < 100; ++it) {
        double dL, dR;
        const double f = pressure_fn(p, L, g, &dL) + pressure_fn(p, R, g, &dR) + (R.u - L.u);
        double pn = p - f / (dL + dR);
        if (!(pn > 1e-12)) pn = 1e-12;
        const double change = fabs(pn - p) / (0.5 * (pn + p));
        p = pn;
        if (change < 1e-15) break;
    }
    double dL, dR;
    *ps = p;
    *us = 0.5 * (L.u + R.u) + 0.5 * (pressure_fn(p, R, g, &dR) - pressure_fn(p, L, g, &dL));
}

struct FrameArgs {
    int dim, nx, ny, kind, cells;
    double lo[2], dr[2];
    double gamma, cth, sth, amp;
    double rl, ul, pl, rr, ur, pr, ps, us;  // shock tube: the two states and the star state
    void *frame[5];
    const Ctrl *ctrl;
};

// Sample the exact solution at xi = (s - 1/2) / t; side < 0 / > 0 selects a side at t = 0.
__device__ void riemann_sample(const FrameArgs &a, double xi, double *r, double *u, double *p) {
    const double g = a.gamma;
    const double ps = a.ps, us = a.us;
    if (xi <= us) {  // left of the contact
        const double aL = sqrt(g * a.pl / a.rl);
        if (ps > a.pl) {
            const double SL = a.ul - aL * sqrt((g + 1.0) / (2.0 * g) * ps / a.pl + (g - 1.0) / (2.0 * g));
            if (xi <= SL) {
                *r = a.rl, *u = a.ul, *p = a.pl;
            } else {
                const double q = (g - 1.0) / (g + 1.0);
                *r = a.rl * (ps / a.pl + q) / (q * ps / a.pl + 1.0), *u = us, *p = ps;
            }
        } else {
            const double head = a.ul - aL;
            const double tail = us - aL * pow(ps / a.pl, (g - 1.0) / (2.0 * g));
            if (xi <= head) {
                *r = a.rl, *u = a.ul, *p = a.pl;
            } else if (xi >= tail) {
                *r = a.rl * pow(ps / a.pl, 1.0 / g), *u = us, *p = ps;
            } else {  // inside the fan
                const double c = 2.0 / (g + 1.0) * (aL + 0.5 * (g - 1.0) * (a.ul - xi));
                *u = 2.0 / (g + 1.0) * (aL + 0.5 * (g - 1.0) * a.ul + xi);
                *r = a.rl * pow(c / aL, 2.0 / (g - 1.0));
                *p = a.pl * pow(c / aL, 2.0 * g / (g - 1.0));
            }
        }
    } else {  // right of the contact (mirror image)
        const double aR = sqrt(g * a.pr / a.rr);
        if (ps > a.pr) {
            const double SR = a.ur + aR * sqrt((g + 1.0) / (2.0 * g) * ps / a.pr + (g - 1.0) / (2.0 * g));
            if (xi >= SR) {
                *r = a.rr, *u = a.ur, *p = a.pr;
            } else {
                const double q = (g - 1.0) / (g + 1.0);
                *r = a.rr * (ps / a.pr + q) / (q * ps / a.pr + 1.0), *u = us, *p = ps;
            }
        } else {
            const double head = a.ur + aR;
            const double tail = us + aR * pow(ps / a.pr, (g - 1.0) / (2.0 * g));
            if (xi >= head) {
                *r = a.rr, *u = a.ur, *p = a.pr;
            } else if (xi <= tail) {
                *r = a.rr * pow(ps / a.pr, 1.0 / g), *u = us, *p = ps;
            } else {
                const double c = 2.0 / (g + 1.0) * (aR - 0.5 * (g - 1.0) * (a.ur - xi));
                *u = 2.0 / (g + 1.0) * (-aR + 0.5 * (g - 1.0) * a.ur + xi);
                *r = a.rr * pow(c / aR, 2.0 / (g - 1.0));
                *p = a.pr * pow(c / aR, 2.0 * g / (g - 1.0));
            }
        }
    }
}

// The conserved state of the solution at the point (x, y) and time t (dim 1: y = 1/2), stored
// at index i of the planes `out`.
template <class T>
__device__ void store_solution(const FrameArgs &a, double x, double y, double t, void *const *out,
                               long long i) {
    const double s = (x - 0.5) * a.cth + (y - 0.5) * a.sth + 0.5;
    double rho, un, p;
    if (a.kind == 3) {
        if (t > 0.0) {
            riemann_sample(a, (s - 0.5) / t, &rho, &un, &p);
        } else if (s < 0.5) {
            rho = a.rl, un = a.ul, p = a.pl;
        } else {
            rho = a.rr, un = a.ur, p = a.pr;
        }
    } else {
        const double wv = sin(2.0 * 3.14159265358979323846 * (s - t));
        if (a.kind == 1) {
            rho = 2.0 + wv, un = 1.0, p = 1.0;
        } else {
            rho = a.gamma * (1.0 + a.amp * wv), un = a.amp * wv, p = 1.0 + a.gamma * a.amp * wv;
        }
    }
    const double v[2] = {un * a.cth, un * a.sth};
    double kin = 0.0;
    for (int d = 0; d < a.dim; ++d) kin += v[d] * v[d];
    T *const *f = reinterpret_cast<T *const *>(out);
    f[0][i] = T(rho);
    for (int d = 0; d < a.dim; ++d) f[1 + d][i] = T(rho * v[d]);
    f[a.dim + 1][i] = T(p / (a.gamma - 1.0) + 0.5 * rho * kin);
}

template <class T>
__global__ void __launch_bounds__(kFrameThreads) frame_kernel(const FrameArgs a, int stage) {
    const int i = blockIdx.x * kFrameThreads + threadIdx.x;
    if (i >= a.cells) return;
    // ring position -> ghost cell (gx, gy), the inverse of frame_index
    const int w = a.nx + 4;
    int gx, gy;
    if (i < 4 * a.ny) {
        const int c = i % 4;
        gy = i / 4, gx = c < 2 ? c - 2 : a.nx + c - 2;
    } else if (i < 4 * a.ny + 2 * w) {
        const int j = i - 4 * a.ny;
        gy = j / w - 2, gx = j % w - 2;
    } else {
        const int j = i - 4 * a.ny - 2 * w;
        gy = a.ny + j / w, gx = j % w - 2;
    }
    const double t = stage == 2 ? a.ctrl->t + 0.5 * a.ctrl->dt : a.ctrl->t;
    const double x = a.lo[0] + (gx + 0.5) * a.dr[0];
    const double y = a.dim >= 2 ? a.lo[1] + (gy + 0.5) * a.dr[1] : 0.5;
    store_solution<T>(a, x, y, t, a.frame, i);
}

// The solution at every cell centre of the grid at time t (grid-stride over the cells).
template <class T>
__global__ void __launch_bounds__(kFrameThreads) solution_kernel(const FrameArgs a, double t,
                                                                 long long ncell) {
    for (long long i = (long long)blockIdx.x * kFrameThreads + threadIdx.x; i < ncell;
         i += (long long)gridDim.x * kFrameThreads) {
        const long long gx = i % a.nx, gy = i / a.nx;
        const double x = a.lo[0] + ((double)gx + 0.5) * a.dr[0];
        const double y = a.dim >= 2 ? a.lo[1] + ((double)gy + 0.5) * a.dr[1] : 0.5;
        store_solution<T>(a, x, y, t, a.frame, i);
    }
}

}  // namespace

long long frame_cells(int dim, long long nx, long long ny) {
    return dim >= 2 ? 4 * ny + 4 * (nx + 4) : 4;
}

static FrameArgs frame_args(const AnalyticLaunch &L) {
    FrameArgs a;
    memset(&a, 0, sizeof a);
    a.dim = L.dim;
    a.nx = L.nx;
    a.ny = L.dim >= 2 ? L.ny : 1;
    a.kind = L.kind;
    a.cells = (int)frame_cells(L.dim, L.nx, L.ny);  // below 2^31: checked at create
    for (int d = 0; d < 2; ++d) a.lo[d] = L.lo[d], a.dr[d] = L.dr[d];
    a.gamma = L.gamma;
    a.cth = cos(L.theta);
    a.sth = sin(L.theta);
    a.amp = L.amp;
    if (L.kind == 3) {  // Sod's shock tube
        const Prim1 l = {1.0, 0.0, 1.0}, r = {0.125, 0.0, 0.1};
        a.rl = l.r, a.ul = l.u, a.pl = l.p, a.rr = r.r, a.ur = r.u, a.pr = r.p;
        star_state(l, r, L.gamma, &a.ps, &a.us);
    }
    for (int k = 0; k < 5; ++k) a.frame[k] = L.frame[k];
    a.ctrl = static_cast<const Ctrl *>(L.ctrl);
    return a;
}

cudaError_t launch_analytic_frame(const AnalyticLaunch &L, int stage, cudaStream_t st) {
    const FrameArgs a = frame_args(L);
    const unsigned blocks = (unsigned)((a.cells + kFrameThreads - 1) / kFrameThreads);
    if (L.prec == HYDRO_F32)
        frame_kernel<float><<<blocks, kFrameThreads, 0, st>>>(a, stage);
    else
        frame_kernel<double><<<blocks, kFrameThreads, 0, st>>>(a, stage);
    return cudaGetLastError();
}

}  // namespace hydro

extern "C" int hydro_analytic_state(const hydro_grid_t *grid, double gamma, int32_t prec,
                                    int32_t kind, double theta, double amplitude, double t,
                                    const hydro_state_t *out, void *stream) {
    if (!grid || !out || grid->dim < 1 || grid->dim > 2) return HYDRO_EINVAL;
    if (prec != HYDRO_F32 && prec != HYDRO_F64) return HYDRO_EINVAL;
    if (kind < HYDRO_ANALYTIC_ENTROPY_WAVE || kind > HYDRO_ANALYTIC_SHOCK_TUBE) return HYDRO_EINVAL;
    if (!(gamma > 1.0) || !(gamma < 1e300) || !(t >= 0.0) || !(t < 1e300)) return HYDRO_EINVAL;
    if (!(fabs(theta) < 1e6) || !(fabs(amplitude) < 1e300)) return HYDRO_EINVAL;
    long long ncell = 1;
    for (int d = 0; d < grid->dim; ++d) {
        if (grid->n[d] < 1 || grid->n[d] > (1LL << 31) - 1024 || !(grid->hi[d] > grid->lo[d]))
            return HYDRO_EINVAL;
        ncell *= grid->n[d];
    }
    if (ncell >= (1LL << 31)) return HYDRO_EINVAL;
    for (int k = 0; k < grid->dim + 2; ++k)
        if (!out->plane[k]) return HYDRO_EINVAL;
    hydro::AnalyticLaunch L;
    memset(&L, 0, sizeof L);
    L.prec = prec;
    L.dim = grid->dim;
    L.nx = (int)grid->n[0];
    L.ny = grid->dim >= 2 ? (int)grid->n[1] : 1;
    L.kind = kind;
    for (int d = 0; d < grid->dim; ++d) {
        L.lo[d] = grid->lo[d];
        L.dr[d] = (grid->hi[d] - grid->lo[d]) / (double)grid->n[d];
    }
    L.gamma = gamma;
    L.theta = theta;
    L.amp = amplitude;
    for (int k = 0; k < grid->dim + 2; ++k) L.frame[k] = out->plane[k];
    const hydro::FrameArgs a = hydro::frame_args(L);
    const long long want = (ncell + hydro::kFrameThreads - 1) / hydro::kFrameThreads;
    const unsigned blocks = (unsigned)(want < 152LL * 16 ? want : 152LL * 16);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (prec == HYDRO_F32)
        hydro::solution_kernel<float><<<blocks, hydro::kFrameThreads, 0, st>>>(a, t, ncell);
    else
        hydro::solution_kernel<double><<<blocks, hydro::kFrameThreads, 0, st>>>(a, t, ncell);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HYDRO_OK : hydro::record_cuda_error(e, "hydro_analytic_state");
}
