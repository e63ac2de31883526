// The paper's linear-wave example (arXiv:1204.4779, section 2.3): f_t = g, g_t = c^2 f_xx on a
// periodic 1D grid, advanced by Eqs. eqLWDiscF and eqLWDiscG,
//     f1[i] = f[i] + dt g[i]
//     g1[i] = g[i] + (c^2 dt / dx^2) (f1[i+1] + f1[i-1] - 2 f1[i]),
// with the discrete energy
//     E = sum_i (1/2) (c^2 ((f1[i+1] - f1[i-1]) / (2 dx))^2 + ((g[i] + g1[i]) / 2)^2) dx
// audited after every step (the form of the paper's listing, which the scheme conserves to
// round-off).
//
// One launch per step: a CTA walks tiles of cells (tile b, b + G, ... for G CTAs); a one-CTA
// kernel sums the G energy partials in fixed order.  State ping-pongs between the caller's
// arrays and two workspace arrays.  The translation unit is compiled with --fmad=false: every
// product and sum of the update formulas is its own IEEE operation, in the formulas' order.
//
// FP64, n even and arrays 16-byte aligned (wave_step_kernel_f64v): two cells per thread with
// 128-bit loads and stores, the neighbours' f1 from the adjacent lanes by warp shuffles; the
// energy as K1 sum D^2 + K2 sum G^2 (below), each thread's two sums kept in FP64 by fused
// multiply-adds, so a cell costs 11 FP64 operations (the update's 7, the energy's 4) on
// GB300's FP64 pipe (1/62 of the FP32 rate).  Otherwise (wave_step_kernel) a tile's f1 (plus
// one halo cell each side) goes through shared memory and each cell's energy term is evaluated
// as the formula reads (the centred difference multiplied by a precomputed 1 / (2 dx) rather
// than divided by 2 dx), the tile's terms reduced by a fixed tree and summed in tile order into
// the CTA's partial.  Either energy differs from the oracle's evaluation by rounding only, well
// inside the 1e-13 relative agreement the tests require; the states are identical.
//
// FP32: the stencil runs in FP32 and the energy keeps FP64 accuracy without per-cell FP64
// arithmetic (GB300's FP64 pipe runs at 1/62 of the FP32 rate).  Each cell recomputes f1 at
// i-1, i, i+1 from f and g (one FP32 operation each, the neighbours' loads hitting cache), so
// the tile loop has no barrier; where n is a multiple of four and the arrays are 16-byte
// aligned a thread takes four consecutive cells with 128-bit loads and stores.  With D = f1[i+1] - f1[i-1] and G = g[i] + g1[i], the energy is
// K1 sum D^2 + K2 sum G^2, K1 = c^2 dx / (8 dx^2), K2 = dx / 8.  D and G are formed exactly as
// FP32 pairs (hi + lo) by Knuth's TwoSum, their squares as pairs by the FMA form of Dekker's
// TwoProduct (dropping lo^2, 2^-48 of the square), and each thread adds them to two running
// double-float sums (TwoSum of the high parts, the low parts added, renormalised; Dekker's and
// Knuth's algorithms as used in double-double arithmetic).  Once per CTA the running sums go to
// FP64, are scaled by K1 and K2 and reduced by the same fixed tree.  The result agrees with an
// FP64 evaluation of the FP32 state's energy to about 2^-48 times the cells a thread visits.
#include <string.h>

#include "../../include/hydro.h"
#include "hydro_device.cuh"
#include "hydro_internal.h"

namespace {

using hydro::acc_add;
using hydro::DF;
using hydro::square;
using hydro::two_sum;

constexpr int kWaveThreads = 256;

// FP32 step with the double-float energy audit (see the file comment).  k1, k2: K1 and K2.
__global__ void __launch_bounds__(kWaveThreads)
    wave_step_kernel_f32(const float *__restrict__ f, const float *__restrict__ g,
                         float *__restrict__ fo, float *__restrict__ go, long long n,
                         long long ntiles, float dt, float k, double k1, double k2,
                         double *partial) {
    __shared__ double s_e[kWaveThreads / 32];
    DF sd = {0.0f, 0.0f}, sg = {0.0f, 0.0f};  // this thread's sums of D^2 and G^2, cell order
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long i = tile * kWaveThreads + threadIdx.x;
        if (i >= n) continue;
        const long long l = i == 0 ? n - 1 : i - 1;
        const long long r = i == n - 1 ? 0 : i + 1;
        const float gi = g[i];
        const float fm = f[l] + dt * g[l];
        const float f1 = f[i] + dt * gi;
        const float fp = f[r] + dt * g[r];
        const float g1 = gi + k * (fp + fm - 2.0f * f1);
        fo[i] = f1;
        go[i] = g1;
        acc_add(sd, square(two_sum(fp, -fm)));
        acc_add(sg, square(two_sum(gi, g1)));
    }
    double e = k1 * ((double)sd.hi + (double)sd.lo) + k2 * ((double)sg.hi + (double)sg.lo);
    // fixed-order tree: a butterfly within each warp, then the warp sums in warp order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) s_e[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kWaveThreads / 32; ++w) t += s_e[w];
        partial[blockIdx.x] = t;
    }
}

// The same step with four cells per thread: 128-bit loads and stores of f and g (n a multiple
// of four, arrays 16-byte aligned), each cell's formulas and energy terms as in
// wave_step_kernel_f32, the four cells added to the running sums in cell order.
__global__ void __launch_bounds__(kWaveThreads)
    wave_step_kernel_f32v(const float *__restrict__ f, const float *__restrict__ g,
                          float *__restrict__ fo, float *__restrict__ go, long long n4,
                          long long ntiles, float dt, float k, double k1, double k2,
                          double *partial) {
    __shared__ double s_e[kWaveThreads / 32];
    const float4 *f4 = reinterpret_cast<const float4 *>(f);
    const float4 *g4 = reinterpret_cast<const float4 *>(g);
    DF sd = {0.0f, 0.0f}, sg = {0.0f, 0.0f};
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long q = tile * kWaveThreads + threadIdx.x;  // index of the cell quadruple
        if (q >= n4) continue;
        const long long n = 4 * n4;
        const long long l = q == 0 ? n - 1 : 4 * q - 1;
        const long long r = q == n4 - 1 ? 0 : 4 * q + 4;
        const float4 fv = f4[q], gv = g4[q];
        const float fi[6] = {f[l], fv.x, fv.y, fv.z, fv.w, f[r]};
        const float gi[6] = {g[l], gv.x, gv.y, gv.z, gv.w, g[r]};
        float f1[6], g1[4];
#pragma unroll
        for (int c = 0; c < 6; ++c) f1[c] = fi[c] + dt * gi[c];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            g1[c] = gi[c + 1] + k * (f1[c + 2] + f1[c] - 2.0f * f1[c + 1]);
            acc_add(sd, square(two_sum(f1[c + 2], -f1[c])));
            acc_add(sg, square(two_sum(gi[c + 1], g1[c])));
        }
        reinterpret_cast<float4 *>(fo)[q] = make_float4(f1[1], f1[2], f1[3], f1[4]);
        reinterpret_cast<float4 *>(go)[q] = make_float4(g1[0], g1[1], g1[2], g1[3]);
    }
    double e = k1 * ((double)sd.hi + (double)sd.lo) + k2 * ((double)sg.hi + (double)sg.lo);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) s_e[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kWaveThreads / 32; ++w) t += s_e[w];
        partial[blockIdx.x] = t;
    }
}

// FP64 step with two cells per thread: 128-bit loads and stores of f and g (n even, arrays
// 16-byte aligned).  The update formulas are evaluated exactly as in wave_step_kernel (the same
// IEEE operations in the same order, so the states are identical); the neighbours' f1 come
// from the adjacent lanes by warp shuffles (the warp's first and last lanes and the last pair
// of the grid compute theirs from memory), so the loop has no barrier and evaluates each f1
// once.  Energy: with D = f1[i+1] - f1[i-1] and G = g[i] + g1[i], E = K1 sum D^2 + K2 sum G^2
// (K1 = c^2 dx / (8 dx^2), K2 = dx / 8), each thread keeping its two sums in FP64 by fused
// multiply-adds in cell order; once per CTA they go through the fixed tree and are scaled.
__global__ void __launch_bounds__(kWaveThreads)
    wave_step_kernel_f64v(const double *__restrict__ f, const double *__restrict__ g,
                          double *__restrict__ fo, double *__restrict__ go, long long n2,
                          long long ntiles, double dt, double k, double k1, double k2,
                          double *partial) {
    __shared__ double s_d[kWaveThreads / 32], s_g[kWaveThreads / 32];
    const double2 *f2 = reinterpret_cast<const double2 *>(f);
    const double2 *g2 = reinterpret_cast<const double2 *>(g);
    const long long n = 2 * n2;
    const int lane = threadIdx.x & 31;
    double sd = 0.0, sg = 0.0;  // this thread's sums of D^2 and G^2, cell order
    // every thread of the CTA walks the same tiles, so the shuffles below are warp-uniform
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long q = tile * kWaveThreads + threadIdx.x;  // index of the cell pair
        const bool active = q < n2;
        double2 fv = make_double2(0.0, 0.0), gv = make_double2(0.0, 0.0);
        if (active) {
            fv = f2[q];
            gv = g2[q];
        }
        const double f1a = fv.x + dt * gv.x;  // cells 2q, 2q + 1
        const double f1b = fv.y + dt * gv.y;
        double fl = __shfl_up_sync(0xffffffffu, f1b, 1);    // f1 of cell 2q - 1
        double fr = __shfl_down_sync(0xffffffffu, f1a, 1);  // f1 of cell 2q + 2
        if (!active) continue;
        if (lane == 0) {
            const long long l = q == 0 ? n - 1 : 2 * q - 1;
            fl = f[l] + dt * g[l];
        }
        if (lane == 31 || q == n2 - 1) {
            const long long r = q == n2 - 1 ? 0 : 2 * q + 2;
            fr = f[r] + dt * g[r];
        }
        const double g1a = gv.x + k * (f1b + fl - 2.0 * f1a);
        const double g1b = gv.y + k * (fr + f1a - 2.0 * f1b);
        reinterpret_cast<double2 *>(fo)[q] = make_double2(f1a, f1b);
        reinterpret_cast<double2 *>(go)[q] = make_double2(g1a, g1b);
        const double da = f1b - fl, db = fr - f1a;
        const double ga = gv.x + g1a, gb = gv.y + g1b;
        sd = fma(da, da, sd);
        sd = fma(db, db, sd);
        sg = fma(ga, ga, sg);
        sg = fma(gb, gb, sg);
    }
    // fixed-order tree: a butterfly within each warp, then the warp sums in warp order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sd += __shfl_xor_sync(0xffffffffu, sd, o);
        sg += __shfl_xor_sync(0xffffffffu, sg, o);
    }
    if (lane == 0) {
        s_d[threadIdx.x >> 5] = sd;
        s_g[threadIdx.x >> 5] = sg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double td = 0.0, tg = 0.0;
#pragma unroll
        for (int w = 0; w < kWaveThreads / 32; ++w) {
            td += s_d[w];
            tg += s_g[w];
        }
        partial[blockIdx.x] = k1 * td + k2 * tg;
    }
}

template <class T>
__global__ void __launch_bounds__(kWaveThreads)
    wave_step_kernel(const T *__restrict__ f, const T *__restrict__ g, T *__restrict__ fo,
                     T *__restrict__ go, long long n, long long ntiles, T dt, T k, double c2,
                     double dx, double inv_2dx, double *partial) {
    __shared__ T s_f1[kWaveThreads + 2];
    __shared__ double s_e[kWaveThreads];
    double acc = 0.0;  // this CTA's tiles, summed in tile order (thread 0)
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long base = tile * kWaveThreads;
        const long long i = base + threadIdx.x;
        const bool active = i < n;
        // f1 on the tile and its two halo cells (periodic)
        if (active) s_f1[threadIdx.x + 1] = f[i] + dt * g[i];
        if (threadIdx.x == 0) {
            const long long l = base == 0 ? n - 1 : base - 1;
            s_f1[0] = f[l] + dt * g[l];
        }
        if (threadIdx.x == kWaveThreads - 1 || i == n - 1) {
            const long long r = i + 1 >= n ? 0 : i + 1;
            s_f1[threadIdx.x + 2] = f[r] + dt * g[r];
        }
        __syncthreads();
        double e = 0.0;
        if (active) {
            const T fm = s_f1[threadIdx.x], f1 = s_f1[threadIdx.x + 1], fp = s_f1[threadIdx.x + 2];
            const T g1 = g[i] + k * (fp + fm - T(2) * f1);
            fo[i] = f1;
            go[i] = g1;
            // FP64 divisions are long instruction sequences: multiply by 1 / (2 dx) instead
            const double dfdx = ((double)fp - (double)fm) * inv_2dx;
            const double gm = ((double)g[i] + (double)g1) * 0.5;
            e = 0.5 * (c2 * dfdx * dfdx + gm * gm) * dx;
        }
        // fixed-order tree: a butterfly within each warp (lane 0's order), then the warp sums
        // in warp order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if ((threadIdx.x & 31) == 0) s_e[threadIdx.x >> 5] = e;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
#pragma unroll
            for (int w = 0; w < kWaveThreads / 32; ++w) t += s_e[w];
            acc += t;
        }
        __syncthreads();  // the next tile reuses s_f1 and s_e
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kWaveThreads)
    wave_energy_kernel(const double *partial, int nparts, double *out) {
    __shared__ double s[kWaveThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += kWaveThreads) acc += partial[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kWaveThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

size_t align_up(size_t x) { return (x + 255) / 256 * 256; }

struct WaveLayout {
    size_t f_off, g_off, part_off, e_off, total;
    long long ntiles;   // tiles of kWaveThreads cells
    long long nblocks;  // CTAs of the step kernel (each walks tiles b, b + nblocks, ...)
};

WaveLayout wave_layout(long long n, int prec, int n_steps) {
    WaveLayout L;
    const size_t esz = prec == HYDRO_F32 ? 4 : 8;
    L.ntiles = (n + kWaveThreads - 1) / kWaveThreads;
    // enough CTAs to fill every SM several times; the energy partials stay few, so the final
    // fixed-order sum of them is short
    L.nblocks = L.ntiles < 152LL * 8 ? L.ntiles : 152LL * 8;
    L.f_off = 0;
    L.g_off = align_up((size_t)n * esz);
    L.part_off = L.g_off + align_up((size_t)n * esz);
    L.e_off = L.part_off + align_up(sizeof(double) * (size_t)L.nblocks);
    L.total = L.e_off + align_up(sizeof(double) * (size_t)(n_steps > 0 ? n_steps : 1));
    return L;
}

template <class T>
int wave_run_t(long long n, double c, double length, double dt, T *f, T *g, int n_steps,
               double *energy_out, unsigned char *ws, const WaveLayout &L, cudaStream_t st) {
    T *fa = f, *ga = g;
    T *fb = reinterpret_cast<T *>(ws + L.f_off), *gb = reinterpret_cast<T *>(ws + L.g_off);
    double *part = reinterpret_cast<double *>(ws + L.part_off);
    double *energy = reinterpret_cast<double *>(ws + L.e_off);
    const double dx = length / (double)n;
    const T k = T(c * c * dt / (dx * dx));
    // the FP32 energy's factors: (1/2) c^2 (D / (2 dx))^2 dx = K1 D^2, (1/2) (G / 2)^2 dx = K2 G^2
    const double k1 = c * c * dx / (8.0 * dx * dx), k2 = dx / 8.0;
    // FP32: four cells per thread where n and the arrays allow 128-bit accesses
    const bool vec = sizeof(T) == 4 && n % 4 == 0 && n >= 8 &&
                     reinterpret_cast<uintptr_t>(f) % 16 == 0 && reinterpret_cast<uintptr_t>(g) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(fb) % 16 == 0 && reinterpret_cast<uintptr_t>(gb) % 16 == 0;
    const long long vtiles = (n / 4 + kWaveThreads - 1) / kWaveThreads;
    const unsigned vblocks = (unsigned)(vtiles < L.nblocks ? vtiles : L.nblocks);
    // FP64: two cells per thread where n is even and the arrays allow 128-bit accesses
    const bool vec2 = sizeof(T) == 8 && n % 2 == 0 && reinterpret_cast<uintptr_t>(f) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(g) % 16 == 0 && reinterpret_cast<uintptr_t>(fb) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(gb) % 16 == 0;
    const long long ptiles = (n / 2 + kWaveThreads - 1) / kWaveThreads;
    const unsigned pblocks = (unsigned)(ptiles < L.nblocks ? ptiles : L.nblocks);
    const int nparts = vec ? (int)vblocks : (vec2 ? (int)pblocks : (int)L.nblocks);
    for (int s = 0; s < n_steps; ++s) {
        if constexpr (sizeof(T) == 4) {
            if (vec)
                wave_step_kernel_f32v<<<vblocks, kWaveThreads, 0, st>>>(
                    fa, ga, fb, gb, n / 4, vtiles, T(dt), k, k1, k2, part);
            else
                wave_step_kernel_f32<<<(unsigned)L.nblocks, kWaveThreads, 0, st>>>(
                    fa, ga, fb, gb, n, L.ntiles, T(dt), k, k1, k2, part);
        } else if (vec2) {
            wave_step_kernel_f64v<<<pblocks, kWaveThreads, 0, st>>>(
                reinterpret_cast<const double *>(fa), reinterpret_cast<const double *>(ga),
                reinterpret_cast<double *>(fb), reinterpret_cast<double *>(gb), n / 2, ptiles,
                (double)dt, (double)k, k1, k2, part);
        } else
            wave_step_kernel<T><<<(unsigned)L.nblocks, kWaveThreads, 0, st>>>(
                fa, ga, fb, gb, n, L.ntiles, T(dt), k, c * c, dx, 1.0 / (2.0 * dx), part);
        wave_energy_kernel<<<1, kWaveThreads, 0, st>>>(part, nparts, energy + s);
        T *t = fa;
        fa = fb;
        fb = t;
        t = ga;
        ga = gb;
        gb = t;
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && fa != f) {  // odd step count: the result is in the workspace
        e = cudaMemcpyAsync(f, fa, sizeof(T) * (size_t)n, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g, ga, sizeof(T) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    }
    if (e == cudaSuccess && energy_out && n_steps > 0)
        e = cudaMemcpyAsync(energy_out, energy, sizeof(double) * (size_t)n_steps,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? HYDRO_OK : hydro::record_cuda_error(e, "hydro_wave_run");
}

}  // namespace

extern "C" {

int hydro_wave_workspace_bytes(int64_t n, int32_t prec, int32_t n_steps, size_t *bytes_out) {
    if (!bytes_out || n < 3 || n >= (1LL << 40) || n_steps < 0) return HYDRO_EINVAL;
    if (prec != HYDRO_F32 && prec != HYDRO_F64) return HYDRO_EINVAL;
    *bytes_out = wave_layout(n, prec, n_steps).total;
    return HYDRO_OK;
}

int hydro_wave_run(int32_t prec, int64_t n, double c, double length, double dt, void *f, void *g,
                   int32_t n_steps, double *energy_out, void *workspace, size_t workspace_bytes,
                   void *stream) {
    if (!f || !g || !workspace || n < 3 || n_steps < 0) return HYDRO_EINVAL;
    if (prec != HYDRO_F32 && prec != HYDRO_F64) return HYDRO_EINVAL;
    if (!(c > 0.0) || !(length > 0.0) || !(dt > 0.0) || ((uintptr_t)workspace) % 256)
        return HYDRO_EINVAL;
    const WaveLayout L = wave_layout(n, prec, n_steps);
    if (workspace_bytes < L.total || L.nblocks >= (1LL << 31)) return HYDRO_EINVAL;
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (prec == HYDRO_F32)
        return wave_run_t<float>(n, c, length, dt, static_cast<float *>(f), static_cast<float *>(g),
                                 n_steps, energy_out, ws, L, st);
    return wave_run_t<double>(n, c, length, dt, static_cast<double *>(f), static_cast<double *>(g),
                              n_steps, energy_out, ws, L, st);
}

}  // extern "C"
