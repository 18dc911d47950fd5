// Ionosphere shell (Sec. II): field-aligned current from the magnetosphere,
// electrostatic potential on the two polar caps, E x B flow of the inner
// cells.  Five small FP64 kernels per solve, all on the caller's stream:
//   iono_current_kernel  one thread per cap node: curl B' at the 8 cells
//                        around the node's mapping point, trilinear, J_par,
//                        flux-tube scaling, radial component;
//   iono_dft_kernel      one thread per (cap, ring, mode): real DFT in
//                        longitude of the scaled source;
//   iono_tridiag_kernel  one thread per (cap, mode): the colatitude system of
//                        that Fourier mode (Thomas algorithm);
//   iono_idft_kernel     one thread per cap node: inverse DFT, and the pole
//                        value (ring-0 mean) per cap;
//   iono_inner_kernel    one thread per inner cell: the potential mapped to
//                        its six neighbours, E = -grad Phi, v = E x B_d/B_d^2,
//                        the cell's conserved inner state.
// The Fourier modes diagonalise the periodic second difference in longitude
// exactly (eigenvalue (2 - 2 cos(2 pi m / n_phi)) / dphi^2), so the result is
// the five-point system's solution to rounding.
#include <math.h>

#include "ppmlr_internal.h"

namespace ppmlr {

constexpr int IONO_THREADS = 128;

// Earth dipole along -z: B = M (3 (m.r) r - m r^2) / r^5, m = -z.
__device__ __forceinline__ void iono_dipole(double M, double x, double y, double z, double *B)
{
    const double r2 = x * x + y * y + z * z;
    if (M == 0.0 || r2 == 0.0) { B[0] = B[1] = B[2] = 0.0; return; }
    const double f = M / (r2 * r2 * sqrt(r2));
    const double mr = -z;
    B[0] = f * (3.0 * mr * x);
    B[1] = f * (3.0 * mr * y);
    B[2] = f * (3.0 * mr * z + r2);
}

// Interior cell index i with c[i] <= p < c[i + 1], clamped to [0, n - 2]
// (c: ghost-extended centres, interior centre i at c[GH + i]).
__device__ __forceinline__ int bracket(const double *c, int n, double p)
{
    int lo = 0, hi = n - 1;            // find the last i with c[i] <= p
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (c[GH + mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo < 0 ? 0 : (lo > n - 2 ? n - 2 : lo);
}

__global__ void __launch_bounds__(IONO_THREADS) iono_current_kernel(IonoArgs a)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nt = a.nt, np = a.np;
    if (t >= 2 * nt * np) return;
    const int h = t / (nt * np), j = (t / np) % nt, k = t % np;
    const double th = (j + 0.5) * a.dth, ph = k * a.dph;
    const double st = sin(th), ct = cos(th);
    const double s2m = (a.r_fac / a.r_iono) * st * st;     // sin^2 at r_fac on the same field line
    if (s2m > 1.0) { a.jr[t] = 0.0; return; }
    const double zs = h == 0 ? 1.0 : -1.0;
    double sp, cp;
    sincos(ph, &sp, &cp);
    const double sm = sqrt(s2m), cm = sqrt(1.0 - s2m);
    const double p[3] = {a.r_fac * sm * cp, a.r_fac * sm * sp, zs * a.r_fac * cm};
    int i0[3];
    double w[3];
    for (int d = 0; d < 3; d++) {
        // the configuration keeps [-r_fac, r_fac] inside centres 1 .. n-2; the
        // clamp keeps every curl stencil (cells i0 - 1 .. i0 + 2) in the grid
        i0[d] = min(max(bracket(a.c[d], a.n[d], p[d]), 1), a.n[d] - 3);
        const double c0 = a.c[d][GH + i0[d]], c1 = a.c[d][GH + i0[d] + 1];
        w[d] = (p[d] - c0) / (c1 - c0);
    }
    const long long nx = a.n[0], nxy = (long long)a.n[0] * a.n[1];
    double J[3] = {0.0, 0.0, 0.0}, Bp[3] = {0.0, 0.0, 0.0};
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++) {
                const int ix = i0[0] + dx, iy = i0[1] + dy, iz = i0[2] + dz;
                const double wt = (dz ? w[2] : 1.0 - w[2]) * (dy ? w[1] : 1.0 - w[1]) * (dx ? w[0] : 1.0 - w[0]);
                const long long g = iz * nxy + iy * nx + ix;
                const double *Bx = a.B[0], *By = a.B[1], *Bz = a.B[2];
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
    double Bm[3];
    iono_dipole(a.M, p[0], p[1], p[2], Bm);
    const double B[3] = {Bp[0] + Bm[0], Bp[1] + Bm[1], Bp[2] + Bm[2]};
    const double jpar = (J[0] * B[0] + J[1] * B[1] + J[2] * B[2]) / sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    // foot point on the shell: J_par scaled by |B_d(foot)| / |B_d(p)|, radial part B_r / |B_d(foot)|
    const double f[3] = {a.r_iono * st * cp, a.r_iono * st * sp, zs * a.r_iono * ct};
    double Bf[3];
    iono_dipole(a.M, f[0], f[1], f[2], Bf);
    const double br = (Bf[0] * f[0] + Bf[1] * f[1] + Bf[2] * f[2]) / a.r_iono;
    const double bm = sqrt(Bm[0] * Bm[0] + Bm[1] * Bm[1] + Bm[2] * Bm[2]);
    a.jr[t] = jpar * br / bm;
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
    for (int k = 0; k < a.np; k++) {
        const int q = (int)(((long long)m * k) % a.np);      // exact reduction of the phase
        double s, c;
        sincospi(2.0 * q / a.np, &s, &c);
        re += f[k] * c;
        im -= f[k] * s;
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
    const double dth2 = a.dth * a.dth;
    const double lam = 4.0 * sinpi((double)m / a.np) * sinpi((double)m / a.np) / (a.dph * a.dph);
    double *cp = a.work + (long long)t * nt;                 // modified upper coefficients
    double *X = a.spec;
    auto at = [&](int j) { return 2 * ((((long long)h * nt + j) * nm) + m); };
    // forward elimination, rows j = 0 .. nt-1:
    //   lo_j Phi_{j-1} + di_j Phi_j + up_j Phi_{j+1} = rhs_j
    double prev_c = 0.0, prev_re = 0.0, prev_im = 0.0;
    for (int j = 0; j < nt; j++) {
        const double th = (j + 0.5) * a.dth, s = sin(th);
        const double sp = sin(th + 0.5 * a.dth), sm = j > 0 ? sin(th - 0.5 * a.dth) : 0.0;
        const double lo = sm / (s * dth2), up = sp / (s * dth2);
        double di = -(sp + sm) / (s * dth2) - lam / (s * s);
        if (j == nt - 1) di -= up;                          // Phi = 0 at theta_max (odd ghost)
        const double den = di - lo * prev_c;
        const double c = j < nt - 1 ? up / den : 0.0;
        const long long q = at(j);
        const double re = (X[q] - lo * prev_re) / den, im = (X[q + 1] - lo * prev_im) / den;
        cp[j] = c;
        X[q] = re;
        X[q + 1] = im;
        prev_c = c; prev_re = re; prev_im = im;
    }
    for (int j = nt - 2; j >= 0; j--) {                     // back substitution
        const long long q = at(j), q1 = at(j + 1);
        X[q] -= cp[j] * X[q1];
        X[q + 1] -= cp[j] * X[q1 + 1];
    }
}

__global__ void __launch_bounds__(IONO_THREADS) iono_idft_kernel(IonoArgs a)
{
    const int nm = a.np / 2 + 1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * a.nt * a.np) return;
    const int h = t / (a.nt * a.np), j = (t / a.np) % a.nt, k = t % a.np;
    const double *X = a.spec + 2 * (((long long)h * a.nt + j) * nm);
    double v = X[0];
    for (int m = 1; m < a.np / 2; m++) {
        const int q = (int)(((long long)m * k) % a.np);
        double s, c;
        sincospi(2.0 * q / a.np, &s, &c);
        v += 2.0 * (X[2 * m] * c - X[2 * m + 1] * s);
    }
    v += X[2 * (a.np / 2)] * ((k & 1) ? -1.0 : 1.0);
    a.phi[t] = v / a.np;
    if (j == 0 && k == 0) a.pole[h] = X[0] / a.np;           // ring-0 mean
}

// Potential carried along the dipole field line through (x, y, z).
__device__ double iono_phi_at(const IonoArgs &a, double x, double y, double z)
{
    const double r2 = x * x + y * y + z * z;
    if (r2 == 0.0) return 0.0;
    const double r = sqrt(r2);
    const double s2i = (a.r_iono / r) * ((x * x + y * y) / r2);
    if (s2i > 1.0) return 0.0;                              // the line closes below the shell
    const double th = asin(sqrt(s2i));
    if (!(th < a.theta_max)) return 0.0;                    // off the caps
    double ph = atan2(y, x);
    if (ph < 0.0) ph += 2.0 * M_PI;
    const int h = z >= 0.0 ? 0 : 1;
    const int nt = a.nt, np = a.np;
    const double *P = a.phi + (long long)h * nt * np;
    const double u = ph / a.dph, fl = floor(u);
    const int k0 = ((int)fl % np + np) % np, k1 = (k0 + 1) % np;
    const double fu = u - fl;
    auto ring = [&](int j) {
        if (j < 0) return a.pole[h];
        if (j >= nt) return 0.0;
        return (1.0 - fu) * P[j * np + k0] + fu * P[j * np + k1];
    };
    const double t = th / a.dth - 0.5;
    if (t < 0.0) {
        const double w = (t + 0.5) / 0.5;
        return (1.0 - w) * ring(-1) + w * ring(0);
    }
    if (t > nt - 1) {
        const double w = (t - (nt - 1)) / 0.5;
        return (1.0 - w) * ring(nt - 1);
    }
    const int j = (int)floor(t);
    const double w = t - j;
    return (1.0 - w) * ring(j) + w * ring(j + 1);
}

__global__ void __launch_bounds__(IONO_THREADS) iono_inner_kernel(IonoArgs a)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_inner) return;
    const long long gi = a.inner_cells[t];
    const long long nx = a.n[0], ny = a.n[1];
    const int idx[3] = {(int)(gi % nx), (int)((gi / nx) % ny), (int)(gi / (nx * ny))};
    const double x0[3] = {a.c[0][GH + idx[0]], a.c[1][GH + idx[1]], a.c[2][GH + idx[2]]};
    double E[3];
    for (int d = 0; d < 3; d++) {
        const int lo = idx[d] > 0 ? idx[d] - 1 : 0, hi = idx[d] < a.n[d] - 1 ? idx[d] + 1 : a.n[d] - 1;
        double pm[3] = {x0[0], x0[1], x0[2]}, pp[3] = {x0[0], x0[1], x0[2]};
        pm[d] = a.c[d][GH + lo];
        pp[d] = a.c[d][GH + hi];
        const double fm = iono_phi_at(a, pm[0], pm[1], pm[2]), fp = iono_phi_at(a, pp[0], pp[1], pp[2]);
        E[d] = -(fp - fm) / (a.c[d][GH + hi] - a.c[d][GH + lo]);
    }
    double B[3];
    iono_dipole(a.M, x0[0], x0[1], x0[2], B);
    const double b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    double v[3] = {0.0, 0.0, 0.0};
    if (b2 > 0.0) {
        v[0] = (E[1] * B[2] - E[2] * B[1]) / b2;
        v[1] = (E[2] * B[0] - E[0] * B[2]) / b2;
        v[2] = (E[0] * B[1] - E[1] * B[0]) / b2;
    }
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

static int blocks_for(long long n) { return (int)((n + IONO_THREADS - 1) / IONO_THREADS); }

cudaError_t launch_ionosphere(const IonoArgs &a, cudaStream_t s, int *launches)
{
    const int nm = a.np / 2 + 1;
    iono_current_kernel<<<blocks_for(2LL * a.nt * a.np), IONO_THREADS, 0, s>>>(a);
    iono_dft_kernel<<<blocks_for(2LL * a.nt * nm), IONO_THREADS, 0, s>>>(a);
    iono_tridiag_kernel<<<blocks_for(2LL * nm), IONO_THREADS, 0, s>>>(a);
    iono_idft_kernel<<<blocks_for(2LL * a.nt * a.np), IONO_THREADS, 0, s>>>(a);
    int n = 4;
    if (a.n_inner > 0) {
        iono_inner_kernel<<<blocks_for(a.n_inner), IONO_THREADS, 0, s>>>(a);
        n++;
    }
    if (launches) *launches = n;
    return cudaGetLastError();
}

}  // namespace ppmlr
