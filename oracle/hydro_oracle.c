/*
 * hydro_oracle.c -- plain, slow FP64 CPU oracle of the second-order
 * compressible-Euler step of Paraiso (Muranushi, arXiv:1204.4779, section 4.1
 * "The Target Program").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load it.  It shares no code, header, table or
 * constant with the CUDA library: every formula below is written out here, from
 * the paper, in the paper's order.
 *
 * Compile: gcc -O2 -ffp-contract=off [-fopenmp] -shared -fPIC (no fast-math), so
 * every operation is one IEEE-754 round-to-nearest operation.
 *
 * Layout of the arrays passed in and out: structure of arrays, dim+2 planes
 * (rho, m_0..m_{dim-1}, E) or (rho, v_0..v_{dim-1}, p), each plane n0*n1*n2
 * doubles with axis 0 (x) fastest.  Inactive axes have n = 1.
 *
 * Readings of the paper used here (the paper is silent or garbled on them):
 *  - flux row 1 is the mass flux rho*v_a and the PDE is dU/dt + d_a F_a = 0;
 *    the sign of AddFlux (Eq. eqAddFlux) is the conservative one and is used.
 *  - HLLC (cited, not written out, section 4.1): Davis wave-speed estimates
 *    S_L = min(u_L - a_L, u_R - a_R), S_R = max(u_L + a_L, u_R + a_R); the
 *    contact speed S* and the star states of Toro, Spruce & Speares (1994).
 *    Branch tie-breaks: F_L if S_L >= 0, F*_L if S* >= 0, F*_R if S_R > 0,
 *    else F_R.
 *  - CFL (section 4.1 says only "determined by the CFL condition"):
 *    dt = CFL / max_i sum_a (|v_a| + c_s) / dr_a, c_s = sqrt(gamma p / rho),
 *    evaluated on the state at the start of the RK step and used by both stages.
 *  - Interpolate (Eq. eqInterpolateSingle): dy = 0 if dy01*dy12 < 0, dy01 if
 *    |dy01| < |dy12|, dy12 otherwise, applied to the primitive variables V
 *    along the face normal only (Eq. eqInterpolateV).
 *  - Boundaries: periodic wrap, or outflow = zero-gradient copy of the nearest
 *    interior cell, into two ghost layers, refilled before every stage; or (the
 *    convergence tests of section 4.3) the analytic solution substituted into the
 *    ghost layers at the time of each stage (t for stage 1, t + dt/2 for stage 2): the
 *    entropy and sound waves, or Sod's shock tube (its exact Riemann solution).
 *  - Time: the last step is clipped so that t lands on t_end; a clipped step
 *    sets t = t_end exactly.
 *  - No positivity floors.
 *  Scheme options (defaults: order 2, Davis speeds):
 *  - order 1: the first-order branch of the paper's interpolation (section 4.2 listing): the
 *    face values are the cell values, no slopes.
 *  - pressure-based HLLC wave speeds (Toro's PVRS estimate): p_pv = (p_L + p_R)/2 -
 *    (u_R - u_L) rho_bar a_bar / 2 with rho_bar, a_bar the arithmetic means,
 *    p_star = max(0, p_pv), q_K = 1 if p_star <= p_K else
 *    sqrt(1 + (gamma+1)/(2 gamma) (p_star / p_K - 1)), S_L = u_L - a_L q_L, S_R = u_R + a_R q_R.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NG 2 /* ghost layers per side on every active axis */

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ENONFINITE = 3 };

typedef struct {
    int dim;         /* 1, 2 or 3 */
    long n[3];       /* interior cells per axis (1 on inactive axes) */
    long p[3];       /* padded extent per axis: n + 2*NG on active axes */
    long g[3];       /* ghost offset per axis: NG on active axes, else 0 */
    double dr[3];    /* cell size per axis */
    double gamma;
    int bc[3];       /* 0 periodic, 1 outflow, 2 analytic solution */
    long ncell;      /* interior cells */
    long npad;       /* padded cells */
    int ana;         /* analytic solution of bc 2: 1 entropy wave, 2 sound wave */
    double ana_theta, ana_amp;  /* its direction (radians from x) and amplitude */
    double ana_ps, ana_us;      /* shock tube: star pressure and velocity */
} grid_t;

static int make_grid(grid_t *G, int dim, const long n[3], const double dr[3],
                     double gamma, const int bc[3]) {
    if (dim < 1 || dim > 3 || !(gamma > 1.0)) return ORC_EINVAL;
    memset(G, 0, sizeof *G);
    G->dim = dim;
    G->gamma = gamma;
    G->ncell = 1;
    G->npad = 1;
    for (int a = 0; a < 3; ++a) {
        int active = a < dim;
        G->n[a] = active ? n[a] : 1;
        if (G->n[a] < 1) return ORC_EINVAL;
        G->g[a] = active ? NG : 0;
        G->p[a] = G->n[a] + 2 * G->g[a];
        G->dr[a] = active ? dr[a] : 1.0;
        if (active && !(dr[a] > 0.0)) return ORC_EINVAL;
        G->bc[a] = active ? bc[a] : 0;
        G->ncell *= G->n[a];
        G->npad *= G->p[a];
    }
    return ORC_OK;
}

/* linear index of interior coordinate (i0,i1,i2), ghosts at negative / >= n */
static long pidx(const grid_t *G, long i0, long i1, long i2) {
    return ((i2 + G->g[2]) * G->p[1] + (i1 + G->g[1])) * G->p[0] + (i0 + G->g[0]);
}

static long wrap(long i, long n) {
    long r = i % n;
    return r < 0 ? r + n : r;
}

/* ---------------------------------------------------------------- ghosts -- */

/* Fill the NG ghost layers of one padded array along every active axis, axis
 * by axis; each pass covers the full padded extent of the other axes. */
static void fill_ghosts(const grid_t *G, double *q) {
    for (int a = 0; a < G->dim; ++a) {
        if (G->bc[a] == 2) continue; /* analytic: filled from the solution, all fields at once */
        long lo[3], hi[3];
        for (int b = 0; b < 3; ++b) {
            lo[b] = -G->g[b];
            hi[b] = G->n[b] + G->g[b];
        }
        for (long i2 = lo[2]; i2 < hi[2]; ++i2)
            for (long i1 = lo[1]; i1 < hi[1]; ++i1)
                for (long i0 = lo[0]; i0 < hi[0]; ++i0) {
                    long c[3] = {i0, i1, i2};
                    long ia = c[a];
                    if (ia >= 0 && ia < G->n[a]) continue;
                    long src[3] = {i0, i1, i2};
                    if (G->bc[a] == 0)
                        src[a] = wrap(ia, G->n[a]);
                    else
                        src[a] = ia < 0 ? 0 : G->n[a] - 1;
                    q[pidx(G, i0, i1, i2)] = q[pidx(G, src[0], src[1], src[2])];
                }
    }
}

/* ------------------------------------- exact Riemann solution (Sod's tube) -- */

/* The exact solution of the Riemann problem of an ideal gas (Toro, Riemann Solvers and
 * Numerical Methods for Fluid Dynamics, ch. 4): across the left and right waves the pressure
 * p* and velocity u* of the star region satisfy f_L(p*) + f_R(p*) + u_R - u_L = 0 with
 *   f_K(p) = (p - p_K) sqrt(A_K / (p + B_K)),  A_K = 2 / ((gamma+1) rho_K),
 *            B_K = (gamma-1)/(gamma+1) p_K                         if p > p_K (shock),
 *   f_K(p) = 2 a_K / (gamma-1) ((p / p_K)^((gamma-1)/(2 gamma)) - 1) otherwise (rarefaction),
 * and u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2.  f_L + f_R is increasing in p, so p* is found
 * by bisection. */
static double riemann_f(double p, double rk, double pk, double g) {
    if (p > pk) {
        double A = 2.0 / ((g + 1.0) * rk), B = (g - 1.0) / (g + 1.0) * pk;
        return (p - pk) * sqrt(A / (p + B));
    }
    double a = sqrt(g * pk / rk);
    return 2.0 * a / (g - 1.0) * (pow(p / pk, (g - 1.0) / (2.0 * g)) - 1.0);
}

static void riemann_star(const double L[3], const double R[3], double g, double *ps, double *us) {
    double lo = 0.0, hi = L[2] > R[2] ? L[2] : R[2];
    while (riemann_f(hi, L[0], L[2], g) + riemann_f(hi, R[0], R[2], g) + R[1] - L[1] < 0.0)
        hi *= 2.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break; /* adjacent doubles */
        if (riemann_f(mid, L[0], L[2], g) + riemann_f(mid, R[0], R[2], g) + R[1] - L[1] < 0.0)
            lo = mid;
        else
            hi = mid;
    }
    *ps = 0.5 * (lo + hi);
    *us = 0.5 * (L[1] + R[1]) + 0.5 * (riemann_f(*ps, R[0], R[2], g) - riemann_f(*ps, L[0], L[2], g));
}

/* (rho, u, p) of the self-similar solution at xi = (x - x0) / t.  One side of the contact
 * (speed u*): with side sign q = -1 (left) or +1 (right) the outer state K, the wave between K
 * and the star region is a shock of speed u_K + q a_K sqrt((gamma+1)/(2 gamma) p* / p_K +
 * (gamma-1)/(2 gamma)) if p* > p_K, else a rarefaction with head u_K + q a_K, tail
 * u* + q a_K (p* / p_K)^((gamma-1)/(2 gamma)) and, inside the fan, the isentropic state with
 * u = 2/(gamma+1) (-q a_K + (gamma-1)/2 u_K + xi).  At a discontinuity the state on the
 * outer (K) side is taken, and at the contact the left star state. */
static void riemann_sample(const double L[3], const double R[3], double g, double ps, double us,
                           double xi, double out[3]) {
    int right = xi > us;
    const double *K = right ? R : L;
    double q = right ? 1.0 : -1.0;
    double a = sqrt(g * K[2] / K[0]);
    if (ps > K[2]) {
        double S = K[1] + q * a * sqrt((g + 1.0) / (2.0 * g) * ps / K[2] + (g - 1.0) / (2.0 * g));
        if (q * (xi - S) >= 0.0) { /* outside the shock */
            out[0] = K[0], out[1] = K[1], out[2] = K[2];
        } else {
            double r = ps / K[2], m = (g - 1.0) / (g + 1.0);
            out[0] = K[0] * (r + m) / (m * r + 1.0), out[1] = us, out[2] = ps;
        }
        return;
    }
    double head = K[1] + q * a;
    double astar = a * pow(ps / K[2], (g - 1.0) / (2.0 * g));
    double tail = us + q * astar;
    if (q * (xi - head) >= 0.0) {
        out[0] = K[0], out[1] = K[1], out[2] = K[2];
    } else if (q * (xi - tail) <= 0.0) {
        out[0] = K[0] * pow(ps / K[2], 1.0 / g), out[1] = us, out[2] = ps;
    } else {
        double u = 2.0 / (g + 1.0) * (-q * a + 0.5 * (g - 1.0) * K[1] + xi);
        double c = q * (xi - u); /* sound speed in the fan: xi = u + q c */
        out[0] = K[0] * pow(c / a, 2.0 / (g - 1.0));
        out[1] = u;
        out[2] = K[2] * pow(c / a, 2.0 * g / (g - 1.0));
    }
}

/* Sod's shock tube of section 4.3: (rho, u, p) = (1, 0, 1) | (0.125, 0, 0.1). */
static const double SOD_L[3] = {1.0, 0.0, 1.0}, SOD_R[3] = {0.125, 0.0, 0.1};

/* Exact Sod solution at xi for the tests: out = (rho, u, p); also p*, u*. */
void oracle_sod_sample(double gamma, double xi, double out[3], double star[2]) {
    double ps, us;
    riemann_star(SOD_L, SOD_R, gamma, &ps, &us);
    riemann_sample(SOD_L, SOD_R, gamma, ps, us, xi, out);
    if (star) star[0] = ps, star[1] = us;
}

/* The analytic solutions of the convergence tests of section 4.3, rotated by theta about
 * (1/2, 1/2): the coordinate along the wave s = (x - 1/2) cos(theta) + (y - 1/2) sin(theta) + 1/2
 * and the phase 2 pi (s - t).
 *  1 entropy wave: rho = 2 + sin(phase), v = (cos theta, sin theta), p = 1 (exact);
 *  2 sound wave:   rho = gamma (1 + A sin(phase)), v = A sin(phase) (cos theta, sin theta),
 *                  p = 1 + gamma A sin(phase) (sound speed 1 for rho = gamma, p = 1; exact to
 *                  first order in the amplitude A);
 *  3 shock tube:   Sod's problem with the discontinuity at s = 1/2, the exact solution at
 *                  xi = (s - 1/2) / t (t = 0: the left state for s < 1/2, else the right one),
 *                  its velocity along (cos theta, sin theta). */
static void analytic_prim(const grid_t *G, double x, double y, double t, double *V) {
    const double pi = 3.14159265358979323846;
    double c = cos(G->ana_theta), sn = sin(G->ana_theta);
    double s = (x - 0.5) * c + (y - 0.5) * sn + 0.5;
    int dim = G->dim;
    double dir[3] = {c, sn, 0.0};
    if (G->ana == 3) {
        double W[3];
        if (t > 0.0)
            riemann_sample(SOD_L, SOD_R, G->gamma, G->ana_ps, G->ana_us, (s - 0.5) / t, W);
        else
            for (int k = 0; k < 3; ++k) W[k] = s < 0.5 ? SOD_L[k] : SOD_R[k];
        V[0] = W[0];
        for (int a = 0; a < dim; ++a) V[1 + a] = W[1] * dir[a];
        V[dim + 1] = W[2];
        return;
    }
    double w = sin(2.0 * pi * (s - t));
    if (G->ana == 1) {
        V[0] = 2.0 + w;
        for (int a = 0; a < dim; ++a) V[1 + a] = dir[a];
        V[dim + 1] = 1.0;
    } else {
        double A = G->ana_amp;
        V[0] = G->gamma * (1.0 + A * w);
        for (int a = 0; a < dim; ++a) V[1 + a] = A * w * dir[a];
        V[dim + 1] = 1.0 + G->gamma * A * w;
    }
}

static void cons_of_prim(int dim, double gamma, const double *V, double *U);

/* Ghost cells outside the interior on an analytic axis: the conserved form of the analytic
 * solution at the cell centre and time t. */
static void fill_analytic(const grid_t *G, double *const *Upad, double t) {
    int nv = G->dim + 2;
    for (long i2 = -G->g[2]; i2 < G->n[2] + G->g[2]; ++i2)
        for (long i1 = -G->g[1]; i1 < G->n[1] + G->g[1]; ++i1)
            for (long i0 = -G->g[0]; i0 < G->n[0] + G->g[0]; ++i0) {
                long c[3] = {i0, i1, i2};
                int outside = 0;
                for (int a = 0; a < G->dim; ++a)
                    if (G->bc[a] == 2 && (c[a] < 0 || c[a] >= G->n[a])) outside = 1;
                if (!outside) continue;
                double V[5], U[5];
                double x = (i0 + 0.5) * G->dr[0];
                double y = G->dim >= 2 ? (i1 + 0.5) * G->dr[1] : 0.5;
                analytic_prim(G, x, y, t, V);
                cons_of_prim(G->dim, G->gamma, V, U);
                long p = pidx(G, i0, i1, i2);
                for (int k = 0; k < nv; ++k) Upad[k][p] = U[k];
            }
}

/* ------------------------------------------------- variables (Eqs. 1-2) -- */

/* V(U): v_a = m_a / rho, p = (gamma-1) (E - 1/2 rho v^2)  (section 4.1) */
static void prim_of_cons(int dim, double gamma, const double *U, double *V) {
    double rho = U[0];
    double kin = 0.0;
    V[0] = rho;
    for (int a = 0; a < dim; ++a) {
        V[1 + a] = U[1 + a] / rho;
        kin += U[1 + a] * V[1 + a];
    }
    V[dim + 1] = (gamma - 1.0) * (U[dim + 1] - 0.5 * kin);
}

/* U(V): m_a = rho v_a, E = p/(gamma-1) + 1/2 rho v^2  (section 4.1) */
static void cons_of_prim(int dim, double gamma, const double *V, double *U) {
    double rho = V[0];
    double v2 = 0.0;
    U[0] = rho;
    for (int a = 0; a < dim; ++a) {
        U[1 + a] = rho * V[1 + a];
        v2 += V[1 + a] * V[1 + a];
    }
    U[dim + 1] = V[dim + 1] / (gamma - 1.0) + 0.5 * rho * v2;
}

/* Euler flux along normal axis a of primitive state V (section 4.1, F_a):
 * (rho v_a, rho v_a v_b + p delta_ab, v_a (E + p)) */
static void euler_flux(int dim, int a, double gamma, const double *V, double *F) {
    double U[5];
    cons_of_prim(dim, gamma, V, U);
    double un = V[1 + a];
    double p = V[dim + 1];
    F[0] = U[0] * un;
    for (int b = 0; b < dim; ++b) F[1 + b] = U[1 + b] * un + (b == a ? p : 0.0);
    F[dim + 1] = un * (U[dim + 1] + p);
}

/* ------------------------------------- Interpolate, Eq. eqInterpolateSingle */

void oracle_interpolate(double y0, double y1, double y2, double *left, double *right) {
    double dy01 = y1 - y0;
    double dy12 = y2 - y1;
    double dy;
    if (dy01 * dy12 < 0.0)
        dy = 0.0;
    else if (fabs(dy01) < fabs(dy12))
        dy = dy01;
    else
        dy = dy12;
    *left = y1 - 0.5 * dy;  /* value at the cell's lower face */
    *right = y1 + 0.5 * dy; /* value at the cell's upper face */
}

/* Interpolate of the given order: order 1 leaves the cell value on both faces. */
static void interpolate_order(int order, double y0, double y1, double y2, double *left,
                              double *right) {
    if (order == 1) {
        *left = y1;
        *right = y1;
        return;
    }
    oracle_interpolate(y0, y1, y2, left, right);
}

/* ------------------------------------------------- HLLC (section 4.1) ----- */

/* HLLC_a(VL, VR): flux through a face whose normal is axis a, from the
 * primitive states on its lower (L) and upper (R) side; riemann selects the wave-speed
 * estimate (0 Davis, 1 pressure-based). */
void oracle_hllc_opt(int dim, int a, double gamma, int riemann, const double *VL,
                     const double *VR, double *F) {
    double rl = VL[0], ul = VL[1 + a], pl = VL[dim + 1];
    double rr = VR[0], ur = VR[1 + a], pr = VR[dim + 1];
    double UL[5], UR[5], FL[5], FR[5];
    cons_of_prim(dim, gamma, VL, UL);
    cons_of_prim(dim, gamma, VR, UR);
    euler_flux(dim, a, gamma, VL, FL);
    euler_flux(dim, a, gamma, VR, FR);

    double al = sqrt(gamma * pl / rl);
    double ar = sqrt(gamma * pr / rr);
    double SL, SR;
    if (riemann == 0) { /* Davis */
        SL = fmin(ul - al, ur - ar);
        SR = fmax(ul + al, ur + ar);
    } else { /* pressure-based (PVRS) */
        double rbar = 0.5 * (rl + rr);
        double abar = 0.5 * (al + ar);
        double ppv = 0.5 * (pl + pr) - 0.5 * (ur - ul) * rbar * abar;
        double ps = fmax(0.0, ppv);
        double ql = ps <= pl ? 1.0 : sqrt(1.0 + (gamma + 1.0) / (2.0 * gamma) * (ps / pl - 1.0));
        double qr = ps <= pr ? 1.0 : sqrt(1.0 + (gamma + 1.0) / (2.0 * gamma) * (ps / pr - 1.0));
        SL = ul - al * ql;
        SR = ur + ar * qr;
    }
    double Ss = (pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur)) /
                (rl * (SL - ul) - rr * (SR - ur));

    int nv = dim + 2;
    if (0.0 <= SL) { /* whole fan moves right: F_L */
        for (int k = 0; k < nv; ++k) F[k] = FL[k];
        return;
    }
    if (!(0.0 <= Ss) && !(0.0 < SR)) { /* whole fan moves left: F_R */
        for (int k = 0; k < nv; ++k) F[k] = FR[k];
        return;
    }
    /* star region: F*_K = F_K + S_K (U*_K - U_K), K = L if S* >= 0 else R */
    int left = 0.0 <= Ss;
    const double *V = left ? VL : VR;
    const double *U = left ? UL : UR;
    const double *FK = left ? FL : FR;
    double S = left ? SL : SR;
    double r = V[0], u = V[1 + a], p = V[dim + 1];
    /* star state of Toro, Spruce & Speares: rho_K (S_K-u_K)/(S_K-S*) times
     * (1, velocity with normal part S*, E_K/rho_K + (S*-u_K)(S* + p_K/(rho_K (S_K-u_K)))) */
    double chi = r * (S - u) / (S - Ss);
    double Us[5];
    Us[0] = chi;
    for (int b = 0; b < dim; ++b) Us[1 + b] = chi * (b == a ? Ss : V[1 + b]);
    Us[dim + 1] = chi * (U[dim + 1] / r + (Ss - u) * (Ss + p / (r * (S - u))));
    for (int k = 0; k < nv; ++k) F[k] = FK[k] + S * (Us[k] - U[k]);
}

void oracle_hllc(int dim, int a, double gamma, const double *VL, const double *VR,
                 double *F) {
    oracle_hllc_opt(dim, a, gamma, 0, VL, VR, F);
}

/* Euler flux, exported for the special-case pins (HLLC(V,V) = F(V)). */
void oracle_euler_flux(int dim, int a, double gamma, const double *V, double *F) {
    euler_flux(dim, a, gamma, V, F);
}

/* ------------------------------------------------------------ the step ---- */

typedef struct {
    grid_t G;
    int nv;
    int order;         /* reconstruction order, 1 or 2 */
    int riemann;       /* HLLC wave speeds: 0 Davis, 1 pressure-based */
    double *U[5];      /* padded conserved planes (scratch copy of a stage input) */
    double *V[5];      /* padded primitive planes */
    double *VL[3][5];  /* face values, lower side, per axis */
    double *VR[3][5];  /* face values, upper side, per axis */
    double *F[3][5];   /* face fluxes per axis */
    long nface[3];     /* faces per axis: (n_a + 1) * prod_{b != a} n_b */
} work_t;

static void free_work(work_t *W) {
    for (int k = 0; k < 5; ++k) {
        free(W->U[k]);
        free(W->V[k]);
        for (int a = 0; a < 3; ++a) {
            free(W->VL[a][k]);
            free(W->VR[a][k]);
            free(W->F[a][k]);
        }
    }
}

static int alloc_work(work_t *W, const grid_t *G) {
    memset(W, 0, sizeof *W);
    W->G = *G;
    W->nv = G->dim + 2;
    W->order = 2;
    for (int k = 0; k < W->nv; ++k) {
        W->U[k] = (double *)calloc((size_t)G->npad, sizeof(double));
        W->V[k] = (double *)calloc((size_t)G->npad, sizeof(double));
        if (!W->U[k] || !W->V[k]) return ORC_ENOMEM;
    }
    for (int a = 0; a < G->dim; ++a) {
        long nf = G->n[a] + 1;
        for (int b = 0; b < 3; ++b)
            if (b != a) nf *= G->n[b];
        W->nface[a] = nf;
        for (int k = 0; k < W->nv; ++k) {
            W->VL[a][k] = (double *)calloc((size_t)nf, sizeof(double));
            W->VR[a][k] = (double *)calloc((size_t)nf, sizeof(double));
            W->F[a][k] = (double *)calloc((size_t)nf, sizeof(double));
            if (!W->VL[a][k] || !W->VR[a][k] || !W->F[a][k]) return ORC_ENOMEM;
        }
    }
    return ORC_OK;
}

/* face index on axis a for the face between interior cells c-e_a and c,
 * where c[a] runs over 0..n_a (face c[a] - 1/2) */
static long fidx(const grid_t *G, int a, const long c[3]) {
    long e[3];
    for (int b = 0; b < 3; ++b) e[b] = G->n[b] + (b == a ? 1 : 0);
    return (c[2] * e[1] + c[1]) * e[0] + c[0];
}

/* Flux_a(U) for every axis: V = V(U); Interpolate -> (VR, VL); F = HLLC_a.
 * U_int holds interior planes (unpadded, caller layout). */
static void flux_all_axes(work_t *W, double *const *U_int, double t_stage) {
    const grid_t *G = &W->G;
    int nv = W->nv, dim = G->dim;
    /* load the stage input into the padded scratch and fill the ghosts */
    for (int k = 0; k < nv; ++k) {
        for (long i2 = 0; i2 < G->n[2]; ++i2)
            for (long i1 = 0; i1 < G->n[1]; ++i1)
                for (long i0 = 0; i0 < G->n[0]; ++i0)
                    W->U[k][pidx(G, i0, i1, i2)] =
                        U_int[k][(i2 * G->n[1] + i1) * G->n[0] + i0];
        fill_ghosts(G, W->U[k]);
    }
    for (int a = 0; a < dim; ++a)
        if (G->bc[a] == 2) {
            fill_analytic(G, W->U, t_stage);
            break;
        }
    /* V0 = V(U0) on interior and ghost cells */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < G->npad; ++c) {
        double u[5], v[5];
        for (int k = 0; k < nv; ++k) u[k] = W->U[k][c];
        prim_of_cons(dim, G->gamma, u, v);
        for (int k = 0; k < nv; ++k) W->V[k][c] = v[k];
    }
    for (int a = 0; a < dim; ++a) {
        /* Eq. eqInterpolateV: every cell i with -1 <= i_a <= n_a (interior on
         * the other axes) yields VR at face i - 1/2 and VL at face i + 1/2 */
        long lo[3] = {0, 0, 0}, hi[3] = {G->n[0], G->n[1], G->n[2]};
        lo[a] = -1;
        hi[a] = G->n[a] + 1;
        long stride = a == 0 ? 1 : (a == 1 ? G->p[0] : G->p[0] * G->p[1]);
#pragma omp parallel for collapse(2) schedule(static)
        for (long i2 = lo[2]; i2 < hi[2]; ++i2)
            for (long i1 = lo[1]; i1 < hi[1]; ++i1)
                for (long i0 = lo[0]; i0 < hi[0]; ++i0) {
                    long c[3] = {i0, i1, i2};
                    long ci = pidx(G, i0, i1, i2);
                    for (int k = 0; k < nv; ++k) {
                        double lft, rgt;
                        interpolate_order(W->order, W->V[k][ci - stride], W->V[k][ci],
                                          W->V[k][ci + stride], &lft, &rgt);
                        if (c[a] >= 0) { /* face c - 1/2 exists: VR there */
                            W->VR[a][k][fidx(G, a, c)] = lft;
                        }
                        if (c[a] + 1 <= G->n[a]) { /* face c + 1/2: VL there */
                            long cu[3] = {c[0], c[1], c[2]};
                            cu[a] += 1;
                            W->VL[a][k][fidx(G, a, cu)] = rgt;
                        }
                    }
                }
        /* F_a[i + 1/2] = HLLC_a(VL[i + 1/2], VR[i + 1/2]) */
#pragma omp parallel for schedule(static)
        for (long f = 0; f < W->nface[a]; ++f) {
            double vl[5], vr[5], fl[5];
            for (int k = 0; k < nv; ++k) {
                vl[k] = W->VL[a][k][f];
                vr[k] = W->VR[a][k][f];
            }
            oracle_hllc_opt(dim, a, G->gamma, W->riemann, vl, vr, fl);
            for (int k = 0; k < nv; ++k) W->F[a][k][f] = fl[k];
        }
    }
}

/* AddFlux(dt, F, Ubase) -> Uout, Eq. eqAddFlux:
 * Uout[i] = Ubase[i] + sum_a (dt/dr_a) (F_a[i - 1/2] - F_a[i + 1/2]) */
static void add_flux(work_t *W, double dt, double *const *Ubase, double *const *Uout) {
    const grid_t *G = &W->G;
    int nv = W->nv, dim = G->dim;
    double coef[3];
    for (int a = 0; a < dim; ++a) coef[a] = dt / G->dr[a];
#pragma omp parallel for collapse(2) schedule(static)
    for (long i2 = 0; i2 < G->n[2]; ++i2)
        for (long i1 = 0; i1 < G->n[1]; ++i1)
            for (long i0 = 0; i0 < G->n[0]; ++i0) {
                long c[3] = {i0, i1, i2};
                long li = (i2 * G->n[1] + i1) * G->n[0] + i0;
                for (int k = 0; k < nv; ++k) {
                    double sum = 0.0;
                    for (int a = 0; a < dim; ++a) {
                        long cu[3] = {c[0], c[1], c[2]};
                        cu[a] += 1;
                        double fm = W->F[a][k][fidx(G, a, c)];  /* F_a[i - 1/2] */
                        double fp = W->F[a][k][fidx(G, a, cu)]; /* F_a[i + 1/2] */
                        sum += coef[a] * (fm - fp);
                    }
                    Uout[k][li] = Ubase[k][li] + sum;
                }
            }
}

/* per-cell CFL signal sum_a (|v_a| + c_s) / dr_a; its maximum over cells */
static double max_signal(const grid_t *G, double *const *U) {
    double smax = 0.0;
    int dim = G->dim;
    for (long c = 0; c < G->ncell; ++c) {
        double u[5], v[5];
        for (int k = 0; k < dim + 2; ++k) u[k] = U[k][c];
        prim_of_cons(dim, G->gamma, u, v);
        double cs = sqrt(G->gamma * v[dim + 1] / v[0]);
        double s = 0.0;
        for (int a = 0; a < dim; ++a) s += (fabs(v[1 + a]) + cs) / G->dr[a];
        if (!(s <= smax)) smax = s; /* NaN propagates */
    }
    return smax;
}

static int all_finite_positive(const grid_t *G, double *const *U) {
    int dim = G->dim;
    for (long c = 0; c < G->ncell; ++c) {
        double u[5], v[5];
        for (int k = 0; k < dim + 2; ++k) {
            u[k] = U[k][c];
            if (!isfinite(u[k])) return 0;
        }
        prim_of_cons(dim, G->gamma, u, v);
        if (!(v[0] > 0.0) || !(v[dim + 1] > 0.0)) return 0;
    }
    return 1;
}

/* One midpoint RK step (section 4.1):
 *   F0 = Flux(U0); U1 = AddFlux(dt/2, F0, U0); F1 = Flux(U1); U2 = AddFlux(dt, F1, U0)
 * U (in/out) holds U0 on entry and U2 on return. */
static void rk_step(work_t *W, double *const *U, double *const *U1, double dt, double t) {
    flux_all_axes(W, U, t);
    add_flux(W, 0.5 * dt, U, U1);
    flux_all_axes(W, U1, t + 0.5 * dt);
    add_flux(W, dt, U, U);
}

/* -------------------------------------------------------- exported API --- */

static void split_planes(double *base, int nv, long ncell, double **planes) {
    for (int k = 0; k < nv; ++k) planes[k] = base + (size_t)k * (size_t)ncell;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_has_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int oracle_prim_to_cons(int dim, const long n[3], double gamma, const double *V, double *U) {
    long ncell = 1;
    for (int a = 0; a < dim; ++a) ncell *= n[a];
    int nv = dim + 2;
    for (long c = 0; c < ncell; ++c) {
        double v[5], u[5];
        for (int k = 0; k < nv; ++k) v[k] = V[(size_t)k * ncell + c];
        cons_of_prim(dim, gamma, v, u);
        for (int k = 0; k < nv; ++k) U[(size_t)k * ncell + c] = u[k];
    }
    return ORC_OK;
}

int oracle_cons_to_prim(int dim, const long n[3], double gamma, const double *U, double *V) {
    long ncell = 1;
    for (int a = 0; a < dim; ++a) ncell *= n[a];
    int nv = dim + 2;
    for (long c = 0; c < ncell; ++c) {
        double v[5], u[5];
        for (int k = 0; k < nv; ++k) u[k] = U[(size_t)k * ncell + c];
        prim_of_cons(dim, gamma, u, v);
        for (int k = 0; k < nv; ++k) V[(size_t)k * ncell + c] = v[k];
    }
    return ORC_OK;
}

/* dt = cfl / max_i sum_a (|v_a| + c_s)/dr_a on state U (SoA, dim+2 planes) */
int oracle_cfl_dt(int dim, const long n[3], const double dr[3], double gamma,
                  const double *U, double cfl, double *dt_out) {
    grid_t G;
    int bc[3] = {0, 0, 0};
    int rc = make_grid(&G, dim, n, dr, gamma, bc);
    if (rc) return rc;
    double *P[5];
    split_planes((double *)U, dim + 2, G.ncell, P);
    *dt_out = cfl / max_signal(&G, P);
    return ORC_OK;
}

/* Face fluxes Flux_a(U) of every axis, for the per-face pins.  F_out[a] points
 * to (dim+2) planes of (n_a+1)*prod_{b!=a} n_b faces, face c-1/2 of cell c. */
int oracle_fluxes(int dim, const long n[3], const double dr[3], double gamma,
                  const int bc[3], const double *U, double **F_out) {
    grid_t G;
    int rc = make_grid(&G, dim, n, dr, gamma, bc);
    if (rc) return rc;
    work_t W;
    rc = alloc_work(&W, &G);
    if (rc) {
        free_work(&W);
        return rc;
    }
    for (int a = 0; a < dim; ++a)
        if (bc[a] == 2) { /* no analytic solution is given here */
            free_work(&W);
            return ORC_EINVAL;
        }
    double *P[5];
    split_planes((double *)U, dim + 2, G.ncell, P);
    flux_all_axes(&W, P, 0.0);
    for (int a = 0; a < dim; ++a)
        for (int k = 0; k < dim + 2; ++k)
            memcpy(F_out[a] + (size_t)k * W.nface[a], W.F[a][k],
                   sizeof(double) * (size_t)W.nface[a]);
    free_work(&W);
    return ORC_OK;
}

/* Advance U (SoA, dim+2 planes, in/out) by up to n_steps RK steps.
 * Each step: dt = cfl / max signal of the step's initial state; if t_end > 0,
 * dt = min(dt, t_end - t) and a clipped step sets t = t_end; stop once
 * t >= t_end.  Returns ORC_ENONFINITE if a step leaves a non-finite value,
 * rho <= 0 or p <= 0 (the state then holds that step's output). */
int oracle_run_opt(int dim, const long n[3], const double dr[3], double gamma,
                   const int bc[3], double cfl, int order, int riemann, double *U, int n_steps,
                   double t_end, double *t_inout, int *steps_done, int nthreads, int ana,
                   double ana_theta, double ana_amp) {
    grid_t G;
    int rc = make_grid(&G, dim, n, dr, gamma, bc);
    if (rc) return rc;
    if ((order != 1 && order != 2) || (riemann != 0 && riemann != 1)) return ORC_EINVAL;
    for (int a = 0; a < dim; ++a)
        if (bc[a] < 0 || bc[a] > 2 || (bc[a] == 2 && (ana < 1 || ana > 3))) return ORC_EINVAL;
    G.ana = ana;
    G.ana_theta = ana_theta;
    G.ana_amp = ana_amp;
    if (ana == 3) riemann_star(SOD_L, SOD_R, gamma, &G.ana_ps, &G.ana_us);
    set_threads(nthreads);
    work_t W;
    rc = alloc_work(&W, &G);
    W.order = order;
    W.riemann = riemann;
    double *u1 = rc ? NULL : (double *)calloc((size_t)(dim + 2) * (size_t)G.ncell, sizeof(double));
    if (rc || !u1) {
        free_work(&W);
        free(u1);
        return ORC_ENOMEM;
    }
    double *P[5], *P1[5];
    split_planes(U, dim + 2, G.ncell, P);
    split_planes(u1, dim + 2, G.ncell, P1);
    double t = t_inout ? *t_inout : 0.0;
    int done = 0;
    rc = ORC_OK;
    for (int s = 0; s < n_steps; ++s) {
        if (t_end > 0.0 && t >= t_end) break;
        double dt = cfl / max_signal(&G, P);
        int clipped = 0;
        if (t_end > 0.0 && dt >= t_end - t) {
            dt = t_end - t;
            clipped = 1;
        }
        rk_step(&W, P, P1, dt, t);
        t = clipped ? t_end : t + dt;
        ++done;
        if (!all_finite_positive(&G, P)) {
            rc = ORC_ENONFINITE;
            break;
        }
    }
    if (t_inout) *t_inout = t;
    if (steps_done) *steps_done = done;
    free(u1);
    free_work(&W);
    return rc;
}

int oracle_run(int dim, const long n[3], const double dr[3], double gamma,
               const int bc[3], double cfl, double *U, int n_steps, double t_end,
               double *t_inout, int *steps_done, int nthreads) {
    return oracle_run_opt(dim, n, dr, gamma, bc, cfl, 2, 0, U, n_steps, t_end, t_inout,
                          steps_done, nthreads, 0, 0.0, 0.0);
}

/* fixed-order pairwise sum of x[0..n) */
static double pairwise_sum(const double *x, long n) {
    if (n <= 8) {
        double s = 0.0;
        for (long i = 0; i < n; ++i) s += x[i];
        return s;
    }
    long h = n / 2;
    return pairwise_sum(x, h) + pairwise_sum(x + h, n - h);
}

/* Totals (mass, momentum_0..2, energy) = pairwise sums times the cell volume.
 * Momenta of inactive axes are 0. */
int oracle_totals(int dim, const long n[3], const double dr[3], const double *U,
                  double out[5]) {
    long ncell = 1;
    double vol = 1.0;
    for (int a = 0; a < dim; ++a) {
        ncell *= n[a];
        vol *= dr[a];
    }
    for (int k = 0; k < 5; ++k) out[k] = 0.0;
    out[0] = pairwise_sum(U, ncell) * vol;
    for (int a = 0; a < dim; ++a)
        out[1 + a] = pairwise_sum(U + (size_t)(1 + a) * ncell, ncell) * vol;
    out[4] = pairwise_sum(U + (size_t)(dim + 1) * ncell, ncell) * vol;
    return ORC_OK;
}
