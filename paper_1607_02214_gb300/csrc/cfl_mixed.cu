// CFL time step of the mixed-precision path: the same rule as cfl.cu,
//   dt = cfl * min over non-inner cells and axes of dx_d / (|v_d| + max(c_f(B'), c_f(B' + B_d))),
// with float wave speeds, the double-float pressure recovery of the mixed
// sweep and no FP64 instructions in the per-cell work.  Block minima and the
// last-block combine (atomic ticket, no float atomics) as in cfl.cu.
#include "cfl.cuh"

namespace ppmlr {

constexpr int CFLM_THREADS = 256;

__device__ __forceinline__ float block_min_f(float v)
{
    __shared__ float red[CFLM_THREADS / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fminf(v, __shfl_down_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < CFLM_THREADS / 32 ? red[threadIdx.x] : INFINITY;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v = fminf(v, __shfl_down_sync(0xffffffffu, v, off));
    }
    return v;
}

// Bound dx_d / (|v_d| + c_f,d) of one cell (INFINITY inside the inner sphere)
// from its 8 conserved values.
__device__ __forceinline__ float cell_bound(const CflArgs &a, const int ix, const int iy, const int iz,
                                            const double *u)
{
    const float x = a.cf[0][ix + GH], y = a.cf[1][iy + GH], z = a.cf[2][iz + GH];
    if (a.r_innerf > 0.0f) {
        const float r2 = x * x + y * y + z * z, ri2 = a.r_innerf * a.r_innerf;
        if (r2 < ri2 * (1.0f - 1e-5f)) return INFINITY;
        if (r2 < ri2 * (1.0f + 1e-5f)) {
            const double xd = a.c[0][ix + GH], yd = a.c[1][iy + GH], zd = a.c[2][iz + GH];
            if (xd * xd + yd * yd + zd * zd < a.r_inner * a.r_inner) return INFINITY;
        }
    }
    const float gm1 = a.gammaf - 1.0f;
    df q[8];
#pragma unroll
    for (int v = 0; v < 8; v++) q[v] = split_double_fast(u[v]);
    float pr = pressure_df(q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7], gm1);
    if (pr < a.p_minf) pr = a.p_minf;
    float Bd[3];
    dipole_f(a.Mf, x, y, z, Bd);
    const float rho = q[0].h, ir = 1.0f / rho;
    const int idx[3] = {ix, iy, iz};
    float best = INFINITY;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
        const float Bn = q[4 + d].h, B1 = q[4 + t1].h, B2 = q[4 + t2].h;
        const float c1 = fast2<float>(rho, pr, Bn, B1, B2, a.gammaf);
        const float c2 = fast2<float>(rho, pr, Bn + Bd[d], B1 + Bd[t1], B2 + Bd[t2], a.gammaf);
        const float cf = sqrtf(fmaxf(c1, c2));
        const float sv = a.wf[d][idx[d] + GH] / (fabsf(q[1 + d].h * ir) + cf);
        best = fminf(best, sv);
    }
    return best;
}

// Grid-stride pass over the cells, two cells per iteration: both cells' 16
// loads are issued before either is used, doubling the loads in flight.
// Cell indices (ix, iy, iz) of i < 2^31 by two fixed-divisor divisions.
__device__ __forceinline__ void cell_xyz(const unsigned i, const CflArgs &a, const FastDiv &fx, const FastDiv &fy,
                                         int &ix, int &iy, int &iz)
{
    const unsigned row = fdiv(i, fx), z = fdiv(row, fy);
    ix = (int)(i - row * (unsigned)a.n[0]);
    iy = (int)(row - z * (unsigned)a.n[1]);
    iz = (int)z;
}

__device__ __forceinline__ void cfl_mixed_body(const CflArgs &a, const int bid, const int nb)
{
    const unsigned ncell = (unsigned)a.n[0] * a.n[1] * a.n[2];      // < 2^31 (checked at creation)
    const unsigned step = (unsigned)nb * blockDim.x;
    const FastDiv fx = make_fastdiv((unsigned)a.n[0]), fy = make_fastdiv((unsigned)a.n[1]);
    float best = INFINITY;
    for (unsigned i0 = (unsigned)bid * blockDim.x + threadIdx.x; i0 < ncell; i0 += 2 * step) {
        const unsigned i1 = i0 + step;
        const bool two = i1 < ncell;
        double u0[8], u1[8];
#pragma unroll
        for (int v = 0; v < 8; v++) u0[v] = __ldg(a.U[v] + i0);
#pragma unroll
        for (int v = 0; v < 8; v++) u1[v] = two ? __ldg(a.U[v] + i1) : u0[v];
        int x0, y0, z0, x1, y1, z1;
        cell_xyz(i0, a, fx, fy, x0, y0, z0);
        best = fminf(best, cell_bound(a, x0, y0, z0, u0));
        if (two) {
            cell_xyz(i1, a, fx, fy, x1, y1, z1);
            best = fminf(best, cell_bound(a, x1, y1, z1, u1));
        }
    }
    best = block_min_f(best);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        a.partial[bid] = widen(best);
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
        float mf = block_min_f((float)m);   // exact: every partial is a widened float
        if (threadIdx.x == 0) {
            const double dt = a.cfl * widen(mf);
            *a.dt_out = dt;
            if (a.t_acc) *a.t_acc += dt;
            *a.counter = 0u;
        }
    }
}

__global__ void __launch_bounds__(CFLM_THREADS, 4) cfl_mixed_kernel(CflArgs a) { cfl_mixed_body(a, blockIdx.x, gridDim.x); }

__global__ void __launch_bounds__(CFLM_THREADS) cfl_mixed_ensemble_kernel(EnsCflArgs e)
{
    const int b = blockIdx.x;
    int lo = 0, hi = e.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (e.first_block[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const int nb = (lo + 1 < e.count ? e.first_block[lo + 1] : (int)gridDim.x) - e.first_block[lo];
    cfl_mixed_body(e.args[lo], b - e.first_block[lo], nb);
}

static cudaError_t launch_single(const CflArgs &a, int blocks, cudaStream_t s)
{
    cfl_mixed_kernel<<<blocks, CFLM_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

static cudaError_t launch_ens(const EnsCflArgs &e, int blocks, cudaStream_t s)
{
    cfl_mixed_ensemble_kernel<<<blocks, CFLM_THREADS, 0, s>>>(e);
    return cudaGetLastError();
}

const CflLaunchers k_cfl_mixed = {launch_single, launch_ens};

}  // namespace ppmlr
