// CFL time step of the FP64 paths (the paper states no rule; the reading
// used here):
//   dt = cfl * min over non-inner interior cells and axes d of
//        dx_d / (|v_d| + max(c_f,d(B'), c_f,d(B' + B_d))).
// Grid-stride pass, warp-shuffle and block min, then the last block to finish
// (atomic ticket, no floating-point atomics) combines the per-block minima and
// resets the ticket.  EX: the reference's expressions (cfl.cu, compiled
// without contraction: bit-identical dt); otherwise the pressure once per cell,
// one reciprocal of rho, square roots as x * rsqrt(x), sign and order tests of
// non-negative values on the integer pipe and, given the reciprocal widths,
// the rate max (|v_d| + c_f,d) / dx_d in place of the quotients, inverted once
// per thread (cfl_fp64.cu, with contraction).  Both forms take the inner
// sphere from the per-cell mask when the context has one (computed on the
// host with the reference's expression).
//
// Two-pass form (single domain, both FP64 forms): a screening pass first
// evaluates every cell's bound in float arithmetic (the mixed path's
// double-float pressure, float wave speeds and dipole: no FP64 work) and the
// smallest positive finite one, m; the FP64 pass then evaluates only the
// cells whose float bound is at most (1 + 1 %) m, or not a positive finite
// number.  The float bound is within ~1e-4 of the FP64 one (the fast-speed
// discriminant's cancellation being the worst case), so the cell holding the
// FP64 minimum is always among them and dt is the one-pass result bit for
// bit, at the cost of a float pass (HBM-bound) instead of FP64 work on every
// cell.
#pragma once
#include <math.h>

#include "sweep.cuh"

namespace ppmlr {

constexpr int CFL_THREADS = 256;
constexpr float CFL_SCREEN_MARGIN = 0.01f;

static __device__ __forceinline__ double fast2d(double rho, double p, double Bn, double B1, double B2, double gam)
{
    double a2 = gam * p / rho;
    double b2 = (Bn * Bn + B1 * B1 + B2 * B2) / rho;
    double bn2 = Bn * Bn / rho;
    double s = a2 + b2;
    double disc = s * s - 4.0 * a2 * bn2;
    if (disc < 0.0) disc = 0.0;
    return 0.5 * (s + sqrt(disc));
}

// x * rsqrt(x) for x >= 0 (zero at zero): a few ulp from the correctly
// rounded square root at about two thirds of its FP64-pipe cost
static __device__ __forceinline__ double sqrt_fast(double x)
{
    const double r = x * rsqrt(x);
    return __double_as_longlong(x) > 0 ? r : 0.0;
}

static __device__ __forceinline__ double block_min(double v)
{
    __shared__ double red[CFL_THREADS / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        double o = __shfl_down_sync(0xffffffffu, v, off);
        v = o < v ? o : v;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < CFL_THREADS / 32 ? red[threadIdx.x] : INFINITY;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            double o = __shfl_down_sync(0xffffffffu, v, off);
            v = o < v ? o : v;
        }
    }
    return v;
}

static __device__ __forceinline__ float block_min_screen(float v)
{
    __shared__ float red[CFL_THREADS / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fminf(v, __shfl_down_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < CFL_THREADS / 32 ? red[threadIdx.x] : INFINITY;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v = fminf(v, __shfl_down_sync(0xffffffffu, v, off));
    }
    return v;
}

// Division by a fixed divisor d >= 1 of dividends n < 2^31 by one 32 x 32 ->
// 64-bit multiply and a shift (Granlund & Montgomery 1994, Thm. 4.2): with
// l = ceil(log2 d), k = 31 + l and m = ceil(2^k / d) (< 2^32),
// floor(n / d) = (n m) >> k.  The cell index of a grid stays below 2^31.
struct FastDiv { unsigned m; int k; };
static __device__ __forceinline__ FastDiv make_fastdiv(unsigned d)
{
    int l = 0;
    while ((1ull << l) < d) l++;
    const int k = 31 + l;
    return FastDiv{(unsigned)(((1ull << k) + d - 1) / d), k};
}
static __device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv &f)
{
    return (unsigned)(((unsigned long long)n * f.m) >> f.k);
}

// Double-float quotient with a fast first approximation (the remainder step
// restores ~44 bits) and the mixed path's double-float pressure built on it.
static __device__ __forceinline__ df screen_df_div(df x, df y)
{
    const float q1 = __fdividef(x.h, y.h);
    const float p = q1 * y.h;
    const float pe = fmaf(q1, y.h, -p);
    const float r = ((x.h - p) - pe + x.l) - q1 * y.l;
    return quick_two_sum(q1, __fdividef(r, y.h));
}
static __device__ __forceinline__ float screen_pressure(const df *q, float gm1)
{
    const df mm = df_add(df_add(df_sqr(q[1]), df_sqr(q[2])), df_sqr(q[3]));
    const df bb = df_add(df_add(df_sqr(q[4]), df_sqr(q[5])), df_sqr(q[6]));
    df t = df_add(screen_df_div(mm, q[0]), bb);
    t.h *= 0.5f;
    t.l *= 0.5f;
    const df e = df_add(q[7], df_neg(t));
    return gm1 * (e.h + e.l);
}
// sqrt(max(x, 0)) to a few ulp
static __device__ __forceinline__ float screen_sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
// fast magnetosonic speed squared along n: (s + sqrt(s^2 - 4 a^2 bn^2)) / 2
static __device__ __forceinline__ float screen_fast2(float a2, float ir, float Bn, float B1, float B2)
{
    const float bn2 = Bn * Bn * ir;
    const float s = a2 + fmaf(B2, B2, fmaf(B1, B1, Bn * Bn)) * ir;
    return 0.5f * (s + screen_sqrt(s * s - 4.0f * a2 * bn2));
}

// Screen value of cell i = (ix, iy, iz): +inf inside the inner sphere (the
// same test as the FP64 pass), -1 where the float bound is not a positive
// finite number (the FP64 pass then always evaluates the cell), else the
// float bound min over d of dx_d / (|v_d| + max(c_f,d(B'), c_f,d(B' + B_d))).
static __device__ __forceinline__ float screen_bound(const CflArgs &a, const long long i, const int ix, const int iy,
                                                    const int iz)
{
    if (a.inner_mask) {
        if (a.inner_mask[i]) return INFINITY;
    } else if (a.r_inner > 0.0) {
        const double x = a.c[0][ix + GH], y = a.c[1][iy + GH], z = a.c[2][iz + GH];
        if (x * x + y * y + z * z < a.r_inner * a.r_inner) return INFINITY;
    }
    df q[8];
#pragma unroll
    for (int v = 0; v < 8; v++) q[v] = split_double_fast(__ldg(a.U[v] + i));
    float pr = screen_pressure(q, a.gammaf - 1.0f);
    if (!(pr == pr)) return -1.0f;
    if (pr < a.p_minf) pr = a.p_minf;
    float Bd[3];
    dipole_f(a.Mf, a.cf[0][ix + GH], a.cf[1][iy + GH], a.cf[2][iz + GH], Bd);
    const float ir = __fdividef(1.0f, q[0].h);
    const float a2 = a.gammaf * pr * ir;
    const int idx[3] = {ix, iy, iz};
    float best = INFINITY;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
        const float Bn = q[4 + d].h, B1 = q[4 + t1].h, B2 = q[4 + t2].h;
        const float c1 = screen_fast2(a2, ir, Bn, B1, B2);
        const float c2 = screen_fast2(a2, ir, Bn + Bd[d], B1 + Bd[t1], B2 + Bd[t2]);
        const float cf = screen_sqrt(fmaxf(c1, c2));
        best = fminf(best, __fdividef(a.wf[d][idx[d] + GH], fabsf(q[1 + d].h * ir) + cf));
    }
    return best > 0.0f && best < INFINITY ? best : -1.0f;
}

// Screening pass: every cell's screen value to a.screen, and the threshold
// (1 + margin) x the smallest positive finite bound (+inf if none) to
// *a.screen_thr, written by the last block (atomic ticket; resets it).  EX
// only selects the translation unit's copy.
template <bool EX>
__global__ void __launch_bounds__(CFL_THREADS) cfl_screen_kernel(CflArgs a)
{
    const unsigned ncell = (unsigned)a.n[0] * a.n[1] * a.n[2];      // < 2^31 (checked at creation)
    const FastDiv fx = make_fastdiv((unsigned)a.n[0]), fy = make_fastdiv((unsigned)a.n[1]);
    float best = INFINITY;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
        const unsigned row = fdiv(i, fx), iz = fdiv(row, fy);
        const float v = screen_bound(a, i, (int)(i - row * a.n[0]), (int)(row - iz * a.n[1]), (int)iz);
        a.screen[i] = v;
        if (v > 0.0f) best = fminf(best, v);
    }
    best = block_min_screen(best);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        a.partial[blockIdx.x] = (double)best;
        __threadfence();
        const unsigned int ticket = atomicAdd(a.counter, 1u);
        last = (ticket == gridDim.x - 1u);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        float m = INFINITY;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) m = fminf(m, (float)__ldcg(a.partial + b));
        m = block_min_screen(m);
        if (threadIdx.x == 0) {
            *a.screen_thr = m * (1.0f + CFL_SCREEN_MARGIN);
            *a.counter = 0u;
        }
    }
}

// Block `bid` of `nb` blocks working on the domain described by `a`; with a
// screen, only the cells it marks are evaluated.
template <bool EX>
__device__ __forceinline__ void cfl_body(const CflArgs &a, const int bid, const int nb)
{
    const long long nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const long long ncell = nx * ny * nz;
    double best = INFINITY;
    double rate = 0.0;        // contracted form with reciprocal widths: max rate of the thread's cells
    const float thr = a.screen ? __ldcg(a.screen_thr) : 0.0f;
    for (long long i = (long long)bid * blockDim.x + threadIdx.x; i < ncell;
         i += (long long)nb * blockDim.x) {
        if (a.screen && !(__ldcg(a.screen + i) <= thr)) continue;
        const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / (nx * ny));
        if (a.inner_mask) {
            if (a.inner_mask[i]) continue;
        } else if (a.r_inner > 0.0) {
            const double x = a.c[0][ix + GH], y = a.c[1][iy + GH], z = a.c[2][iz + GH];
            if (x * x + y * y + z * z < a.r_inner * a.r_inner) continue;
        }
        double U[8];
#pragma unroll
        for (int v = 0; v < 8; v++) U[v] = __ldg(a.U[v] + i);
        double Bd[3] = {0.0, 0.0, 0.0};
        if (a.bd) {            // the sweeps' dipole table (same formula as below in the exact form)
            Bd[0] = __ldg(a.bd + i);
            Bd[1] = __ldg(a.bd + a.bd_vs + i);
            Bd[2] = __ldg(a.bd + 2 * a.bd_vs + i);
        } else {
            const double x = a.c[0][ix + GH], y = a.c[1][iy + GH], z = a.c[2][iz + GH];
            double r2 = x * x + y * y + z * z;
            if (a.M != 0.0 && r2 != 0.0) {
                double r = sqrt(r2);
                double r5 = r2 * r2 * r;
                double mr = -z;
                Bd[0] = a.M * (3.0 * mr * x) / r5;
                Bd[1] = a.M * (3.0 * mr * y) / r5;
                Bd[2] = a.M * (3.0 * mr * z + r2) / r5;
            }
        }
        const int idx[3] = {ix, iy, iz};
        if constexpr (EX) {
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
                double rho = U[0];
                double mn = U[1 + d], m1 = U[1 + t1], m2 = U[1 + t2];
                double Bn = U[4 + d], B1 = U[4 + t1], B2 = U[4 + t2];
                double pr = (a.gamma - 1.0) * (U[7] - 0.5 * (mn * mn + m1 * m1 + m2 * m2) / rho
                                               - 0.5 * (Bn * Bn + B1 * B1 + B2 * B2));
                if (pr < a.p_min) pr = a.p_min;
                double c1 = fast2d(rho, pr, Bn, B1, B2, a.gamma);
                double c2 = fast2d(rho, pr, Bn + Bd[d], B1 + Bd[t1], B2 + Bd[t2], a.gamma);
                double cf = sqrt(c1 > c2 ? c1 : c2);
                double s = a.w[d][idx[d] + GH] / (fabs(mn / rho) + cf);
                if (s < best) best = s;
            }
        } else {
            // one reciprocal of rho, the pressure once per cell
            const double ir = 1.0 / U[0];
            double pr = (a.gamma - 1.0) * (U[7] - 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) * ir
                                           - 0.5 * (U[4] * U[4] + U[5] * U[5] + U[6] * U[6]));
            if (__double_as_longlong(pr) < __double_as_longlong(a.p_min)) pr = a.p_min;   // p_min >= 0
            const double a2 = a.gamma * pr * ir;
            const double bp2 = (U[4] * U[4] + U[5] * U[5] + U[6] * U[6]) * ir;
            const double Bt[3] = {U[4] + Bd[0], U[5] + Bd[1], U[6] + Bd[2]};
            const double bt2 = (Bt[0] * Bt[0] + Bt[1] * Bt[1] + Bt[2] * Bt[2]) * ir;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                // c1, c2 >= 0 and the rates >= 0: ordered as their bit patterns;
                // sqrt_fast gives 0 for a negative discriminant
                double s1 = a2 + bp2, s2 = a2 + bt2;
                double q1 = s1 * s1 - 4.0 * a2 * (U[4 + d] * U[4 + d] * ir);
                double q2 = s2 * s2 - 4.0 * a2 * (Bt[d] * Bt[d] * ir);
                double c1 = 0.5 * (s1 + sqrt_fast(q1));
                double c2 = 0.5 * (s2 + sqrt_fast(q2));
                double cf = sqrt_fast(__double_as_longlong(c1) > __double_as_longlong(c2) ? c1 : c2);
                if (a.iw[0]) {
                    // a NaN rate (bit patterns above +inf) is skipped, as the
                    // quotient form's comparison skips a NaN bound
                    const double r = (fabs(U[1 + d] * ir) + cf) * a.iw[d][idx[d] + GH];
                    const long long rb = __double_as_longlong(r);
                    if (rb > __double_as_longlong(rate) && rb <= 0x7FF0000000000000LL) rate = r;
                } else {
                    double s = a.w[d][idx[d] + GH] / (fabs(U[1 + d] * ir) + cf);
                    if (s < best) best = s;
                }
            }
        }
    }
    if (!EX && a.iw[0]) best = 1.0 / rate;     // no cell: 1 / 0 = inf, as the quotient form
    best = block_min(best);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        a.partial[bid] = best;
        __threadfence();
        unsigned int ticket = atomicAdd(a.counter, 1u);
        last = (ticket == (unsigned int)nb - 1u);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double m = INFINITY;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            double v = __ldcg(a.partial + b);
            m = v < m ? v : m;
        }
        m = block_min(m);
        if (threadIdx.x == 0) {
            const double dt = a.cfl * m;
            *a.dt_out = dt;
            if (a.t_acc) *a.t_acc += dt;
            *a.counter = 0u;
        }
    }
}

template <bool EX>
__global__ void __launch_bounds__(CFL_THREADS) cfl_kernel(CflArgs a) { cfl_body<EX>(a, blockIdx.x, gridDim.x); }

// Ensemble: block b works for the last instance i with first_block[i] <= b.
template <bool EX>
__global__ void __launch_bounds__(CFL_THREADS) cfl_ensemble_kernel(EnsCflArgs e)
{
    const int b = blockIdx.x;
    int lo = 0, hi = e.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (e.first_block[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const int nb = (lo + 1 < e.count ? e.first_block[lo + 1] : (int)gridDim.x) - e.first_block[lo];
    cfl_body<EX>(e.args[lo], b - e.first_block[lo], nb);
}

template <bool EX>
struct CflVariant {
    static cudaError_t single(const CflArgs &a, int blocks, cudaStream_t s)
    {
        if (a.screen) {           // two-pass form: the float screen first
            cfl_screen_kernel<EX><<<blocks, CFL_THREADS, 0, s>>>(a);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        cfl_kernel<EX><<<blocks, CFL_THREADS, 0, s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t ens(const EnsCflArgs &e, int blocks, cudaStream_t s)
    {
        cfl_ensemble_kernel<EX><<<blocks, CFL_THREADS, 0, s>>>(e);
        return cudaGetLastError();
    }
    static constexpr CflLaunchers table() { return {single, ens}; }
};

}  // namespace ppmlr
