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
#pragma once
#include <math.h>

#include "ppmlr_internal.h"

namespace ppmlr {

constexpr int CFL_THREADS = 256;

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

// Block `bid` of `nb` blocks working on the domain described by `a`.
template <bool EX>
__device__ __forceinline__ void cfl_body(const CflArgs &a, const int bid, const int nb)
{
    const long long nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const long long ncell = nx * ny * nz;
    double best = INFINITY;
    double rate = 0.0;        // contracted form with reciprocal widths: max rate of the thread's cells
    for (long long i = (long long)bid * blockDim.x + threadIdx.x; i < ncell;
         i += (long long)nb * blockDim.x) {
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
