// Ionosphere shell (Sec. II): field-aligned current from the magnetosphere,
// electrostatic potential on the two polar caps, E x B flow of the inner
// cells.  Five small FP64 kernels per solve, all on the caller's stream:
//   iono_current_kernel  one thread per cap node: curl B' at the 8 cells
//                        around the node's mapping point, trilinear, J_par,
//                        times the node's flux-tube and radial factor;
//   iono_dft_kernel      one thread per (cap, ring, mode): real DFT in
//                        longitude of the scaled source;
//   iono_tridiag_kernel  one thread per (cap, mode): the colatitude system of
//                        that Fourier mode (Thomas algorithm);
//   iono_idft_kernel     one thread per cap node: inverse DFT, and the pole
//                        value (ring-0 mean) per cap;
//   iono_inner_kernel    one thread per inner cell: the potential at its six
//                        neighbours (bilinear stencils on the caps), E = -grad
//                        Phi, v = E x B_d/B_d^2, the cell's conserved state.
// The Fourier modes diagonalise the periodic second difference in longitude
// exactly (eigenvalue (2 - 2 cos(2 pi m / n_phi)) / dphi^2), so the result is
// the five-point system's solution to rounding.  Everything that depends only
// on the grid and the shell's configuration is a host-computed table (api.cu):
// each node's mapping point (trilinear cell and weights, B_d there, the
// factor |B_d(foot)|/|B_d(point)| x B_r/|B_d| at the foot / |B_d(foot)|), the
// twiddle factors, the colatitude rows, the mode eigenvalues, and each inner
// cell's interpolation stencils and B_d / |B_d|^2.
#include <math.h>

#include "ppmlr_internal.h"

namespace ppmlr {

constexpr int IONO_THREADS = 128;

__global__ void __launch_bounds__(IONO_THREADS) iono_current_kernel(IonoArgs a)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * a.nt * a.np) return;
    const IonoNode &q = a.nodes[t];
    if (q.factor == 0.0) { a.jr[t] = 0.0; return; }          // the line closes below r_fac
    const long long nx = a.n[0], nxy = (long long)a.n[0] * a.n[1];
    double J[3] = {0.0, 0.0, 0.0}, Bp[3] = {0.0, 0.0, 0.0};
    const double *Bx = a.B[0], *By = a.B[1], *Bz = a.B[2];
#pragma unroll
    for (int dz = 0; dz < 2; dz++)
#pragma unroll
        for (int dy = 0; dy < 2; dy++)
#pragma unroll
            for (int dx = 0; dx < 2; dx++) {
                const int ix = q.i0[0] + dx, iy = q.i0[1] + dy, iz = q.i0[2] + dz;
                const double wt = (dz ? q.w[2] : 1.0 - q.w[2]) * (dy ? q.w[1] : 1.0 - q.w[1]) *
                                  (dx ? q.w[0] : 1.0 - q.w[0]);
                const long long g = iz * nxy + iy * nx + ix;
                // centred differences over the centre-to-centre span
                const double hx = a.c[0][GH + ix + 1] - a.c[0][GH + ix - 1];
                const double hy = a.c[1][GH + iy + 1] - a.c[1][GH + iy - 1];
                const double hz = a.c[2][GH + iz + 1] - a.c[2][GH + iz - 1];
                const double dBz_dy = (Bz[g + nx] - Bz[g - nx]) / hy, dBy_dz = (By[g + nxy] - By[g - nxy]) / hz;
                const double dBx_dz = (Bx[g + nxy] - Bx[g - nxy]) / hz, dBz_dx = (Bz[g + 1] - Bz[g - 1]) / hx;
                const double dBy_dx = (By[g + 1] - By[g - 1]) / hx, dBx_dy = (Bx[g + nx] - Bx[g - nx]) / hy;
                J[0] += wt * (dBz_dy - dBy_dz);
                J[1] += wt * (dBx_dz - dBz_dx);
                J[2] += wt * (dBy_dx - dBx_dy);
                Bp[0] += wt * Bx[g];
                Bp[1] += wt * By[g];
                Bp[2] += wt * Bz[g];
            }
    const double B[3] = {Bp[0] + q.Bd[0], Bp[1] + q.Bd[1], Bp[2] + q.Bd[2]};
    const double jpar = (J[0] * B[0] + J[1] * B[1] + J[2] * B[2]) / sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    a.jr[t] = jpar * q.factor;
}

// spec layout: [cap][ring][mode][re, im], modes 0..n_phi/2
__global__ void __launch_bounds__(IONO_THREADS) iono_dft_kernel(IonoArgs a)
{
    const int nm = a.np / 2 + 1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * a.nt * nm) return;
    const int h = t / (a.nt * nm), j = (t / nm) % a.nt, m = t % nm;
    const double *f = a.jr + ((long long)h * a.nt + j) * a.np;
    double re = 0.0, im = 0.0;
    for (int k = 0, q = 0; k < a.np; k++) {                  // q = m k mod n_phi
        re += f[k] * a.tw[2 * q];
        im -= f[k] * a.tw[2 * q + 1];
        q += m;
        if (q >= a.np) q -= a.np;
    }
    const double scale = a.r_iono * a.r_iono / a.sigma_p;    // Laplacian on the unit sphere
    a.spec[2 * t] = scale * re;
    a.spec[2 * t + 1] = scale * im;
}

__global__ void __launch_bounds__(IONO_THREADS) iono_tridiag_kernel(IonoArgs a)
{
    const int nm = a.np / 2 + 1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * nm) return;
    const int h = t / nm, m = t % nm;
    const int nt = a.nt;
    const double lam = a.lam[m];
    double *X = a.spec;
    auto at = [&](int j) { return 2 * ((((long long)h * nt + j) * nm) + m); };
    // the column in thread-local memory (independent loads, then the serial
    // recurrence at L1 latency)
    double xr[IONO_MAX_NT], xi[IONO_MAX_NT], cp[IONO_MAX_NT];
    for (int j = 0; j < nt; j++) { xr[j] = X[at(j)]; xi[j] = X[at(j) + 1]; }
    // forward elimination, rows j = 0 .. nt-1:
    //   lo_j Phi_{j-1} + (d_j - lam_m / sin^2) Phi_j + up_j Phi_{j+1} = rhs_j
    double prev_c = 0.0, prev_re = 0.0, prev_im = 0.0;
    for (int j = 0; j < nt; j++) {
        const double lo = a.rows[4 * j], up = a.rows[4 * j + 1], d = a.rows[4 * j + 2], is2 = a.rows[4 * j + 3];
        const double den = (d - lam * is2) - lo * prev_c;
        const double r = 1.0 / den;
        cp[j] = up * r;
        xr[j] = (xr[j] - lo * prev_re) * r;
        xi[j] = (xi[j] - lo * prev_im) * r;
        prev_c = cp[j]; prev_re = xr[j]; prev_im = xi[j];
    }
    for (int j = nt - 2; j >= 0; j--) {                     // back substitution
        xr[j] -= cp[j] * xr[j + 1];
        xi[j] -= cp[j] * xi[j + 1];
    }
    for (int j = 0; j < nt; j++) { X[at(j)] = xr[j]; X[at(j) + 1] = xi[j]; }
}

__global__ void __launch_bounds__(IONO_THREADS) iono_idft_kernel(IonoArgs a)
{
    const int nm = a.np / 2 + 1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * a.nt * a.np) return;
    const int h = t / (a.nt * a.np), j = (t / a.np) % a.nt, k = t % a.np;
    const double *X = a.spec + 2 * (((long long)h * a.nt + j) * nm);
    double v = X[0];
    for (int m = 1, q = k; m < a.np / 2; m++) {              // q = m k mod n_phi
        v += 2.0 * (X[2 * m] * a.tw[2 * q] - X[2 * m + 1] * a.tw[2 * q + 1]);
        q += k;
        if (q >= a.np) q -= a.np;
    }
    v += X[2 * (a.np / 2)] * ((k & 1) ? -1.0 : 1.0);
    a.phi[t] = v / a.np;
    if (j == 0 && k == 0) a.pole[h] = X[0] / a.np;           // ring-0 mean
}

__global__ void __launch_bounds__(IONO_THREADS) iono_inner_kernel(IonoArgs a)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_inner) return;
    const IonoInner &q = a.inner[t];
    // E_d = -(Phi(+) - Phi(-)) / span_d: the signed interpolation weights over
    // span_d of the two neighbours' stencils (node index >= 0, or -1 - cap
    // for that cap's pole value)
    double E[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        double e = 0.0;
#pragma unroll
        for (int s = 0; s < 8; s++) {
            const int k = q.idx[d][s];
            const double v = k >= 0 ? a.phi[k] : a.pole[-1 - k];
            e += q.coef[d][s] * v;
        }
        E[d] = e;
    }
    const double v[3] = {E[1] * q.bt[2] - E[2] * q.bt[1], E[2] * q.bt[0] - E[0] * q.bt[2],
                         E[0] * q.bt[1] - E[1] * q.bt[0]};
    const double rho = a.rho_in;
    const long long n = a.n_inner;
    a.inner_state[0 * n + t] = rho;
    a.inner_state[1 * n + t] = rho * v[0];
    a.inner_state[2 * n + t] = rho * v[1];
    a.inner_state[3 * n + t] = rho * v[2];
    a.inner_state[4 * n + t] = 0.0;
    a.inner_state[5 * n + t] = 0.0;
    a.inner_state[6 * n + t] = 0.0;
    a.inner_state[7 * n + t] = a.p_in / (a.gamma - 1.0) + 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
}

static int blocks_for(long long n, int threads = IONO_THREADS) { return (int)((n + threads - 1) / threads); }

cudaError_t launch_ionosphere(const IonoArgs &a, cudaStream_t s, int *launches)
{
    const int nm = a.np / 2 + 1;
    // the gather kernels in one-warp blocks: their time is load latency, so
    // spread them over as many SMs as possible
    iono_current_kernel<<<blocks_for(2LL * a.nt * a.np, 32), 32, 0, s>>>(a);
    iono_dft_kernel<<<blocks_for(2LL * a.nt * nm), IONO_THREADS, 0, s>>>(a);
    iono_tridiag_kernel<<<blocks_for(2LL * nm), IONO_THREADS, 0, s>>>(a);
    iono_idft_kernel<<<blocks_for(2LL * a.nt * a.np), IONO_THREADS, 0, s>>>(a);
    int n = 4;
    if (a.n_inner > 0) {
        iono_inner_kernel<<<blocks_for(a.n_inner, 32), 32, 0, s>>>(a);
        n++;
    }
    if (launches) *launches = n;
    return cudaGetLastError();
}

}  // namespace ppmlr
