/*
 * ppmlr_oracle.c -- plain, slow FP64 CPU reference of the split PPMLR-MHD sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the GPU library is
 * checked against.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the GPU library neither links nor calls it, and
 * the two share no code, header or table.
 *
 * What it computes (Guo et al., "Large Scale GPU Accelerated PPMLR-MHD
 * Simulations for Space Weather Forecast"):
 *   - the ideal-MHD system written for B' = B - B_d with the dipole coupling
 *     terms on the right-hand side and gamma = 5/3 (Sec. II, the MHD equations
 *     and their closure), in code units with mu0 = 1;
 *   - the PPMLR scheme outlined in Sec. II: zone-centred volume averages,
 *     piecewise-parabolic profiles, edge states traced along characteristics,
 *     a Lagrangian update, then a remap to the fixed Eulerian grid.  The paper
 *     defers the formulas to Colella & Woodward (1984); the PPM interface
 *     formula, slope limiter, flattening, monotonicity constraint and
 *     domain-of-dependence averages below restate that published method;
 *   - the dimensional split of Sec. III-A: the 3D update is three 1D sweeps,
 *     each independent across the two transverse directions;
 *   - the magnetosphere boundaries of Secs. II and IV-A: solar-wind inflow,
 *     outflow, an inner sphere held at a fixed state, and an Earth dipole.
 * Where the paper is silent (Riemann solver, source split, boundary details,
 * CFL rule) the readings are the ones listed in the design notes; each is
 * marked [R] where it is used.
 *
 * Everything is IEEE double, evaluated left to right as written.  Build with
 * -ffp-contract=off so that no multiply-add is fused.  Pencils are independent,
 * so the OpenMP loop over pencils gives results independent of thread count.
 *
 * Parity pins: every routine here is pinned by the CPU tests (cubic exactness
 * of the interface formula, parabola averages, Riemann-invariant and symmetry
 * checks, exact Sod solution, Brio-Wu self-convergence, Alfven-wave order,
 * conservation, equilibria, split symmetry, flattening values worked out by
 * hand, the CFL step against hand-computed states and the eigenvalues of the
 * MHD Jacobian, boundary ghosts against their definitions).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define G 7                  /* ghost cells per pencil end (stencil radius) */
#define NVAR 8               /* conserved: rho, m_x, m_y, m_z, B'_x, B'_y, B'_z, E */
#define NREC 7               /* reconstructed: rho, u, v1, v2, B1, B2, p (Lagrangian) */
#define NTR 9                /* traced: the 7 above along the fast family, B1, B2 along the Alfven one */

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_INFLOW = 2 };
enum { FLAG_CFL = 1, FLAG_NONFINITE = 2 };

/* Flattening constants of Colella & Woodward (1984), Appendix A. */
static const double FLAT_EPS = 0.33, FLAT_W1 = 0.75, FLAT_W2 = 10.0;
/* Contact-steepening constants of Colella & Woodward (1984), Sec. 1. */
static const double ST_ETA1 = 20.0, ST_ETA2 = 0.05, ST_EPS = 0.01, ST_K0 = 0.1;

typedef struct {
    int n[3];
    double *w[3];            /* widths, n[d] + 2G, index 0 = ghost -G */
    double *c[3];            /* centres, same indexing */
    double gamma;
    int bc[3][2];
    double inflow[8];        /* rho, vx, vy, vz, Bx, By, Bz (total field), p */
    double M;                /* dipole moment B_E R_E^3 along -z; 0 = no dipole */
    double r_inner;
    double inner[8];         /* rho, vx, vy, vz, (B ignored: B' = 0 inside), p */
    double p_min;
    int powell;
    int riemann_iters;       /* 0: two-wave Riemann solver; k > 0: k two-shock Newton steps */
    int steepen;             /* 1: contact steepening in the remap */
    double *inner_v;         /* [3][nz][ny][nx] flow of the inner cells (ionosphere), or NULL: at rest */
    double *U;               /* [8][nz][ny][nx], x fastest */
    double *Unew;
    long long floors;
    long long steps;
} orc_ctx;

/* ------------------------------------------------------------------------- */
/* Earth dipole, moment M along -z (GSM, zero tilt):                          */
/* B_d = M [3 (m.r) r - m r^2] / r^5 with m = -z_hat  [R: moment, sign].       */
void orc_dipole(double M, double x, double y, double z, double *B)
{
    double r2 = x * x + y * y + z * z;
    if (M == 0.0 || r2 == 0.0) { B[0] = B[1] = B[2] = 0.0; return; }
    double r = sqrt(r2);
    double r5 = r2 * r2 * r;
    double mr = -z;                        /* m_hat . r */
    B[0] = M * (3.0 * mr * x) / r5;
    B[1] = M * (3.0 * mr * y) / r5;
    B[2] = M * (3.0 * mr * z + r2) / r5;   /* -m_z r^2 = +r^2 */
}

/* Fast magnetosonic speed squared along the normal direction:
 * cf^2 = 1/2 [a^2 + b^2 + sqrt((a^2 + b^2)^2 - 4 a^2 bn^2)],
 * a^2 = gamma p / rho, b^2 = |B|^2 / rho, bn^2 = Bn^2 / rho (mu0 = 1). */
double orc_fast_speed2(double rho, double p, double Bn, double B1, double B2, double gamma)
{
    double a2 = gamma * p / rho;
    double b2 = (Bn * Bn + B1 * B1 + B2 * B2) / rho;
    double bn2 = Bn * Bn / rho;
    double s = a2 + b2;
    double disc = s * s - 4.0 * a2 * bn2;
    if (disc < 0.0) disc = 0.0;
    return 0.5 * (s + sqrt(disc));
}

/* ------------------------------------------------------------------------- */
/* PPM on a non-uniform coordinate xi (Colella & Woodward 1984, Sec. 1).      */

/* Average slope in zone i (uses i-1, i, i+1). */
static double ppm_slope(const double *xi, const double *a, int i)
{
    double dp = a[i + 1] - a[i];
    double dm = a[i] - a[i - 1];
    double s3 = xi[i - 1] + xi[i] + xi[i + 1];
    return xi[i] / s3 * ((2.0 * xi[i - 1] + xi[i]) / (xi[i + 1] + xi[i]) * dp
                         + (xi[i] + 2.0 * xi[i + 1]) / (xi[i - 1] + xi[i]) * dm);
}

/* Limited slope: zero at an extremum, else bounded by twice either one-sided
 * difference. */
static double ppm_limit(const double *a, int i, double da)
{
    double dp = a[i + 1] - a[i];
    double dm = a[i] - a[i - 1];
    if (dp * dm > 0.0) {
        double m = fabs(da);
        double lim_m = 2.0 * fabs(dm), lim_p = 2.0 * fabs(dp);
        if (lim_m < m) m = lim_m;
        if (lim_p < m) m = lim_p;
        return da > 0.0 ? m : (da < 0.0 ? -m : 0.0);
    }
    return 0.0;
}

/* Interface value a_{i+1/2} (uses i-1 .. i+2) from the slopes of zones i, i+1. */
static double ppm_edge(const double *xi, const double *a, int i, double dmi, double dmi1)
{
    double x0 = xi[i - 1], x1 = xi[i], x2 = xi[i + 1], x3 = xi[i + 2];
    double z1 = (x0 + x1) / (2.0 * x1 + x2);
    double z2 = (x3 + x2) / (2.0 * x2 + x1);
    double d = a[i + 1] - a[i];
    double s4 = x0 + x1 + x2 + x3;
    return a[i] + x1 / (x1 + x2) * d
           + 1.0 / s4 * (2.0 * x2 * x1 / (x1 + x2) * (z1 - z2) * d
                         - x1 * z1 * dmi1 + x2 * z2 * dmi);
}

/* Exported for the pins: interface values for i in [1, n-3] into edge[i]
 * (edge i is the interface between zones i and i+1); other entries are NaN.
 * limited = 0 uses the raw slopes (the interpolant is then exact for cubics). */
void orc_ppm_edges(int n, const double *xi, const double *a, int limited, double *edge)
{
    double *dm = (double *)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i < n; i++) { dm[i] = NAN; edge[i] = NAN; }
    for (int i = 1; i <= n - 2; i++) {
        double da = ppm_slope(xi, a, i);
        dm[i] = limited ? ppm_limit(a, i, da) : da;
    }
    for (int i = 1; i <= n - 3; i++) edge[i] = ppm_edge(xi, a, i, dm[i], dm[i + 1]);
    free(dm);
}

/* Monotonicity constraint of the parabola (a_L, a_i, a_R) (CW84 eq. 1.10);
 * returns a_L, a_R and a6 = 6 (a_i - (a_L + a_R)/2). */
static void ppm_monotone(double ai, double *aL, double *aR, double *a6)
{
    double l = *aL, r = *aR;
    if ((r - ai) * (ai - l) <= 0.0) {
        l = ai; r = ai;
    } else {
        double da = r - l;
        double m6 = 6.0 * (ai - 0.5 * (l + r));
        if (da * m6 > da * da) l = 3.0 * ai - 2.0 * r;
        else if (-(da * da) > da * m6) r = 3.0 * ai - 2.0 * l;
    }
    *aL = l; *aR = r;
    *a6 = 6.0 * (ai - 0.5 * (l + r));
}

/* Exported for the pins: flatten with coefficient f, then constrain. */
void orc_ppm_parabola(double ai, double aL, double aR, double f, double *out3)
{
    double l = f * ai + (1.0 - f) * aL;
    double r = f * ai + (1.0 - f) * aR;
    double a6;
    ppm_monotone(ai, &l, &r, &a6);
    out3[0] = l; out3[1] = r; out3[2] = a6;
}

/* Averages of the parabola over the fraction y of the zone next to its right
 * and left ends (CW84 eq. 1.12). */
double orc_avg_right(double aL, double aR, double a6, double y)
{
    return aR - 0.5 * y * ((aR - aL) - (1.0 - 2.0 / 3.0 * y) * a6);
}
double orc_avg_left(double aL, double aR, double a6, double y)
{
    return aL + 0.5 * y * ((aR - aL) + (1.0 - 2.0 / 3.0 * y) * a6);
}

/* ------------------------------------------------------------------------- */
/* Linearised Lagrangian MHD Riemann solver at one interface [R: the paper    */
/* names no solver].  Each side's state is s = (rho, u, v1, v2, B1, B2, p,     */
/* B1a, B2a): B1, B2 traced along the fast characteristic (they enter the      */
/* total pressure and the fast impedance), B1a, B2a and v1, v2 traced along    */
/* the Alfven characteristic (they enter the transverse subsystem).  Bn is the */
/* face normal field.  Normal subsystem: impedance W = rho c_f, total pressure */
/* P = p + |B_t|^2 / 2.  Transverse subsystem: sigma = Bn B_t, impedance       */
/* Z = sqrt(rho) |Bn|.  Both take the two-wave acoustic solution, i.e. the     */
/* intersection of the two incoming Riemann invariants.                        */
/* out = (u*, P*, S* = P* - Bn^2/2, v1*, v2*, sigma1*, sigma2*, F_E).           */
/*                                                                            */
/* iters > 0 selects the nonlinear variant of the normal subsystem [R: the    */
/* two-shock Riemann solver of Colella & Woodward (1984), which the paper     */
/* cites for its scheme, carried over to MHD by taking the fast Lagrangian    */
/* speed C = rho c_f for the gas's rho c and the total pressure P for p].     */
/* Each side's wave is treated as a shock whose Lagrangian speed depends on   */
/* the middle pressure, W(P) = C sqrt(1 + (gamma+1)/(2 gamma) (P/P_s - 1)),   */
/* so that u*_L(P) = u_L - (P - P_L)/W_L(P) and u*_R(P) = u_R + (P - P_R)/     */
/* W_R(P).  Starting from the two-wave P*, `iters` Newton steps on            */
/* u*_R(P) - u*_L(P) = 0, with the slope of each curve dP/du = Z =            */
/* 2 W^3 / (W^2 + C^2) (the derivative of the curve above), move P* towards   */
/* their intersection (P clipped at 0 where W is evaluated).  u* and P* then  */
/* follow from the two-wave formulas with W_L, W_R at the final P*; at        */
/* convergence they lie on both curves.  With B = 0 this is the gas-dynamic   */
/* two-shock solver, exact when both waves are shocks.  The transverse        */
/* (Alfven) subsystem is linear in this model and stays as above.  Without    */
/* positive total pressures on both sides the two-wave solution is kept.      */
void orc_riemann_nl(const double *L, const double *R, double Bn, double gamma, int iters, double *out)
{
    double PL = L[6] + 0.5 * (L[4] * L[4] + L[5] * L[5]);
    double PR = R[6] + 0.5 * (R[4] * R[4] + R[5] * R[5]);
    double WL = L[0] * sqrt(orc_fast_speed2(L[0], L[6], Bn, L[4], L[5], gamma));
    double WR = R[0] * sqrt(orc_fast_speed2(R[0], R[6], Bn, R[4], R[5], gamma));
    if (iters > 0 && PL > 0.0 && PR > 0.0) {
        double CL = WL, CR = WR;
        double a = (gamma + 1.0) / (2.0 * gamma);
        double P = (WR * PL + WL * PR + WL * WR * (L[1] - R[1])) / (WL + WR);
        for (int k = 0; k < iters; k++) {
            double Pc = P > 0.0 ? P : 0.0;
            double WLk = CL * sqrt(1.0 + a * (Pc / PL - 1.0));
            double WRk = CR * sqrt(1.0 + a * (Pc / PR - 1.0));
            double uLk = L[1] - (Pc - PL) / WLk;
            double uRk = R[1] + (Pc - PR) / WRk;
            double ZL = 2.0 * WLk * WLk * WLk / (WLk * WLk + CL * CL);
            double ZR = 2.0 * WRk * WRk * WRk / (WRk * WRk + CR * CR);
            P = Pc - ZL * ZR * (uRk - uLk) / (ZL + ZR);
        }
        double Pc = P > 0.0 ? P : 0.0;
        WL = CL * sqrt(1.0 + a * (Pc / PL - 1.0));
        WR = CR * sqrt(1.0 + a * (Pc / PR - 1.0));
    }
    double us = (WL * L[1] + WR * R[1] + PL - PR) / (WL + WR);
    double Ps = (WR * PL + WL * PR + WL * WR * (L[1] - R[1])) / (WL + WR);
    double Ss = Ps - 0.5 * Bn * Bn;
    double ZL = sqrt(L[0]) * fabs(Bn);
    double ZR = sqrt(R[0]) * fabs(Bn);
    double vs[2], ss[2];
    for (int t = 0; t < 2; t++) {
        double vL = L[2 + t], vR = R[2 + t];
        double sL = Bn * L[7 + t], sR = Bn * R[7 + t];
        if (ZL + ZR == 0.0) {
            vs[t] = 0.5 * (vL + vR);
            ss[t] = 0.0;
        } else {
            vs[t] = (ZL * vL + ZR * vR + sR - sL) / (ZL + ZR);
            ss[t] = (ZR * sL + ZL * sR + ZL * ZR * (vR - vL)) / (ZL + ZR);
        }
    }
    out[0] = us; out[1] = Ps; out[2] = Ss;
    out[3] = vs[0]; out[4] = vs[1]; out[5] = ss[0]; out[6] = ss[1];
    out[7] = Ss * us - ss[0] * vs[0] - ss[1] * vs[1];
}

void orc_riemann(const double *L, const double *R, double Bn, double gamma, double *out)
{
    orc_riemann_nl(L, R, Bn, gamma, 0, out);
}

/* ------------------------------------------------------------------------- */
/* Context                                                                    */

static size_t ncell(const orc_ctx *c) { return (size_t)c->n[0] * c->n[1] * c->n[2]; }

/* Ghost widths [R]: periodic faces wrap; other faces mirror the interior
 * widths (clamped to the pencil).  Centres extend the grid by those widths. */
static void build_axis(orc_ctx *c, int d, const double *edges)
{
    int n = c->n[d];
    double *w = (double *)malloc(sizeof(double) * (size_t)(n + 2 * G));
    double *ce = (double *)malloc(sizeof(double) * (size_t)(n + 2 * G));
    for (int i = 0; i < n; i++) w[G + i] = edges[i + 1] - edges[i];
    for (int k = 1; k <= G; k++) {
        int lo, hi;
        if (c->bc[d][0] == BC_PERIODIC) lo = ((-k) % n + n) % n;
        else { lo = k - 1; if (lo > n - 1) lo = n - 1; }
        if (c->bc[d][1] == BC_PERIODIC) hi = (k - 1) % n;
        else { hi = n - k; if (hi < 0) hi = 0; }
        w[G - k] = w[G + lo];
        w[G + n - 1 + k] = w[G + hi];
    }
    for (int i = 0; i < n; i++) ce[G + i] = 0.5 * (edges[i] + edges[i + 1]);
    double e = edges[0];
    for (int k = 1; k <= G; k++) { ce[G - k] = e - 0.5 * w[G - k]; e -= w[G - k]; }
    e = edges[n];
    for (int k = 1; k <= G; k++) { ce[G + n - 1 + k] = e + 0.5 * w[G + n - 1 + k]; e += w[G + n - 1 + k]; }
    c->w[d] = w; c->c[d] = ce;
}

orc_ctx *orc_create(int nx, int ny, int nz, const double *ex, const double *ey, const double *ez,
                    double gamma, const int *bc, const double *inflow, double dipole_moment,
                    double r_inner, const double *inner, double p_min, int powell)
{
    if (nx < 1 || ny < 1 || nz < 1) return NULL;
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    c->n[0] = nx; c->n[1] = ny; c->n[2] = nz;
    c->gamma = gamma;
    for (int d = 0; d < 3; d++) { c->bc[d][0] = bc[2 * d]; c->bc[d][1] = bc[2 * d + 1]; }
    memcpy(c->inflow, inflow, sizeof(c->inflow));
    c->M = dipole_moment;
    c->r_inner = r_inner;
    memcpy(c->inner, inner, sizeof(c->inner));
    c->p_min = p_min;
    c->powell = powell;
    build_axis(c, 0, ex); build_axis(c, 1, ey); build_axis(c, 2, ez);
    c->U = (double *)calloc((size_t)NVAR * ncell(c), sizeof(double));
    c->Unew = (double *)calloc((size_t)NVAR * ncell(c), sizeof(double));
    return c;
}

void orc_destroy(orc_ctx *c)
{
    if (!c) return;
    for (int d = 0; d < 3; d++) { free(c->w[d]); free(c->c[d]); }
    free(c->inner_v); free(c->U); free(c->Unew); free(c);
}

/* Flow of the inner-sphere cells set by the ionosphere shell (Sec. II): v =
 * 3 arrays of ncell values (x fastest), copied; NULL puts the inner state back
 * at rest. */
void orc_set_inner_velocity(orc_ctx *c, const double *v)
{
    if (!v) { free(c->inner_v); c->inner_v = NULL; return; }
    if (!c->inner_v) c->inner_v = (double *)malloc(sizeof(double) * 3 * ncell(c));
    memcpy(c->inner_v, v, sizeof(double) * 3 * ncell(c));
}

void orc_set_state(orc_ctx *c, const double *U) { memcpy(c->U, U, sizeof(double) * NVAR * ncell(c)); }
void orc_get_state(const orc_ctx *c, double *U) { memcpy(U, c->U, sizeof(double) * NVAR * ncell(c)); }
long long orc_floor_hits(const orc_ctx *c) { return c->floors; }
long long orc_step_count(const orc_ctx *c) { return c->steps; }
void orc_set_step_count(orc_ctx *c, long long s) { c->steps = s; }
void orc_set_riemann(orc_ctx *c, int iters) { c->riemann_iters = iters > 0 ? iters : 0; }
void orc_set_steepening(orc_ctx *c, int on) { c->steepen = on ? 1 : 0; }

int orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
    return omp_get_max_threads();
#else
    (void)t;
    return 1;
#endif
}

/* Conserved state of a primitive state (rho, v, B', p): closure of Sec. II. */
/* Flattening coefficient of Colella & Woodward (1984), Appendix A, on a
 * pencil of NP zones, with the total pressure Pt = p + |B'|^2/2 in place of
 * the gas pressure [R: MHD] and the normal velocity u.
 *   Shock indicator of zone p (2 <= p <= NP-3): the zone is in a shock when
 *   the pressure jump across it exceeds FLAT_EPS of the smaller neighbour,
 *   |Pt[p+1] - Pt[p-1]| > FLAT_EPS min(Pt[p+1], Pt[p-1]), and the flow is
 *   compressive there, u[p-1] > u[p+1].  Then
 *   ft = clamp((steep - FLAT_W1) FLAT_W2, 0, 1) with the steepness
 *   steep = (Pt[p+1] - Pt[p-1]) / (Pt[p+2] - Pt[p-2]) (1 where the wide
 *   difference vanishes); elsewhere ft = 0.
 *   Coefficient of zone p (3 <= p <= NP-4): f = max(ft[p], ft[p - s]),
 *   s = sign(Pt[p+1] - Pt[p-1]) -- the neighbour on the low-pressure side
 *   (s = 0 is taken as +1 [R]).
 * ft is written for every zone (0 outside 2..NP-3); f only for 3..NP-4. */
void orc_flatten(int NP, const double *Pt, const double *u, double *ft, double *f)
{
    for (int p = 0; p < NP; p++) ft[p] = 0.0;
    for (int p = 2; p <= NP - 3; p++) {
        double dP = Pt[p + 1] - Pt[p - 1];
        double pmin = Pt[p + 1] < Pt[p - 1] ? Pt[p + 1] : Pt[p - 1];
        if (fabs(dP) > FLAT_EPS * pmin && u[p - 1] - u[p + 1] > 0.0) {
            double den = Pt[p + 2] - Pt[p - 2];
            double steep = den != 0.0 ? dP / den : 1.0;
            double fz = (steep - FLAT_W1) * FLAT_W2;
            if (fz < 0.0) fz = 0.0;
            if (fz > 1.0) fz = 1.0;
            ft[p] = fz;
        }
    }
    for (int p = 3; p <= NP - 4; p++) {
        double up = Pt[p + 1] - Pt[p - 1] < 0.0 ? ft[p + 1] : ft[p - 1];
        f[p] = ft[p] > up ? ft[p] : up;
    }
}

static void prim_to_cons(double rho, const double *v, const double *Bp, double p, double gamma, double *U)
{
    U[0] = rho;
    U[1] = rho * v[0]; U[2] = rho * v[1]; U[3] = rho * v[2];
    U[4] = Bp[0]; U[5] = Bp[1]; U[6] = Bp[2];
    U[7] = p / (gamma - 1.0) + 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2])
           + 0.5 * (Bp[0] * Bp[0] + Bp[1] * Bp[1] + Bp[2] * Bp[2]);
}

static int is_inner(const orc_ctx *c, double x, double y, double z)
{
    return c->r_inner > 0.0 && x * x + y * y + z * z < c->r_inner * c->r_inner;
}

/* Fixed inner state of cell gi: density, pressure and flow of the
 * configuration, B' = 0; the flow replaced by the ionosphere's when set. */
static void inner_state(const orc_ctx *c, size_t gi, double *U)
{
    const double zero[3] = {0.0, 0.0, 0.0};
    double v[3] = {c->inner[1], c->inner[2], c->inner[3]};
    if (c->inner_v)
        for (int m = 0; m < 3; m++) v[m] = c->inner_v[(size_t)m * ncell(c) + gi];
    prim_to_cons(c->inner[0], v, zero, c->inner[7], c->gamma, U);
}

/* ------------------------------------------------------------------------- */
/* One pencil of one sweep.  Local frame: n = axis, t1 = axis+1, t2 = axis+2  */
/* (cyclic), so (n, t1, t2) is right-handed.                                  */

typedef struct {
    /* per position, NP = N + 2G */
    double *U[NVAR];      /* conserved, global component order */
    double *dx, *pos;     /* width and centre along n */
    double *Bd[3];        /* dipole at the centre, local frame (n, t1, t2) */
    double *q[NREC];      /* rho, u, v1, v2, B1, B2, p */
    double *Bn, *Pt, *W, *ft, *f;
    double *edge[NREC];
    double *aL[NREC], *aR[NREC], *a6[NREC];
    double *sl[NTR], *sr[NTR];     /* traced state left of i+1/2 (zone i), right of i-1/2 (zone i) */
    double *rs[8];                 /* Riemann output at i+1/2 */
    double *Bnf;
    double *dxL, *rq[NREC], *dC[NREC];  /* Lagrangian width, remap densities, content increments */
    double *F[NREC];                    /* remap flux through Eulerian edge i+1/2 */
    double *slq[NREC], *d2, *eta;       /* contact steepening: limited slopes of the remap densities,
                                           second differences of rho^L, weights */
    double *tmp;
} pencil_buf;

static void pb_alloc(pencil_buf *b, int NP)
{
    size_t s = sizeof(double) * (size_t)NP;
    double **all[] = {&b->dx, &b->pos, &b->Bn, &b->Pt, &b->W, &b->ft, &b->f, &b->Bnf, &b->dxL, &b->tmp,
                      &b->d2, &b->eta};
    for (size_t k = 0; k < sizeof(all) / sizeof(all[0]); k++) *all[k] = (double *)malloc(s);
    for (int v = 0; v < NVAR; v++) b->U[v] = (double *)malloc(s);
    for (int v = 0; v < 3; v++) b->Bd[v] = (double *)malloc(s);
    for (int v = 0; v < 8; v++) b->rs[v] = (double *)malloc(s);
    for (int v = 0; v < NTR; v++) { b->sl[v] = (double *)malloc(s); b->sr[v] = (double *)malloc(s); }
    for (int v = 0; v < NREC; v++) {
        b->q[v] = (double *)malloc(s); b->edge[v] = (double *)malloc(s);
        b->aL[v] = (double *)malloc(s); b->aR[v] = (double *)malloc(s); b->a6[v] = (double *)malloc(s);
        b->rq[v] = (double *)malloc(s); b->dC[v] = (double *)malloc(s); b->F[v] = (double *)malloc(s);
        b->slq[v] = (double *)malloc(s);
    }
}

static void pb_free(pencil_buf *b)
{
    double *all[] = {b->dx, b->pos, b->Bn, b->Pt, b->W, b->ft, b->f, b->Bnf, b->dxL, b->tmp, b->d2, b->eta};
    for (size_t k = 0; k < sizeof(all) / sizeof(all[0]); k++) free(all[k]);
    for (int v = 0; v < NVAR; v++) free(b->U[v]);
    for (int v = 0; v < 3; v++) free(b->Bd[v]);
    for (int v = 0; v < 8; v++) free(b->rs[v]);
    for (int v = 0; v < NTR; v++) { free(b->sl[v]); free(b->sr[v]); }
    for (int v = 0; v < NREC; v++) {
        free(b->q[v]); free(b->edge[v]); free(b->aL[v]); free(b->aR[v]); free(b->a6[v]);
        free(b->rq[v]); free(b->dC[v]); free(b->F[v]); free(b->slq[v]);
    }
}

/* Global linear index of cell i along axis d in the pencil (j, k) with
 * (j, k) = the two other indices in increasing axis order. */
static size_t gidx(const orc_ctx *c, int d, int i, int j, int k)
{
    int ix, iy, iz;
    if (d == 0) { ix = i; iy = j; iz = k; }
    else if (d == 1) { ix = j; iy = i; iz = k; }
    else { ix = j; iy = k; iz = i; }
    return ((size_t)iz * c->n[1] + iy) * c->n[0] + ix;
}

static void sweep_pencil(orc_ctx *c, int d, int j, int k, double dt, pencil_buf *b,
                         long long *floors, int *flags)
{
    const int N = c->n[d], NP = N + 2 * G;
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const double gam = c->gamma;
    /* transverse centre coordinates of this pencil */
    double tc[3];
    {
        int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;   /* the other axes, increasing */
        tc[a1] = c->c[a1][G + j];
        tc[a2] = c->c[a2][G + k];
    }

    /* 1. load the pencil with its ghosts [R: ghost rules] */
    for (int p = 0; p < NP; p++) {
        int g = p - G;
        b->dx[p] = c->w[d][p];
        b->pos[p] = c->c[d][p];
        double xyz[3] = {tc[0], tc[1], tc[2]};
        xyz[d] = b->pos[p];
        double Bdg[3];
        orc_dipole(c->M, xyz[0], xyz[1], xyz[2], Bdg);
        b->Bd[0][p] = Bdg[d]; b->Bd[1][p] = Bdg[t1]; b->Bd[2][p] = Bdg[t2];
        int src = g;
        if (g < 0 || g >= N) {
            int side = g < 0 ? 0 : 1;
            int kind = c->bc[d][side];
            if (kind == BC_PERIODIC) src = ((g % N) + N) % N;
            else if (kind == BC_OUTFLOW) src = side == 0 ? 0 : N - 1;
            else {
                double Bp[3] = {c->inflow[4] - Bdg[0], c->inflow[5] - Bdg[1], c->inflow[6] - Bdg[2]};
                double Ug[NVAR];
                prim_to_cons(c->inflow[0], &c->inflow[1], Bp, c->inflow[7], gam, Ug);
                for (int v = 0; v < NVAR; v++) b->U[v][p] = Ug[v];
                continue;
            }
        }
        size_t gi = gidx(c, d, src, j, k);
        for (int v = 0; v < NVAR; v++) b->U[v][p] = c->U[(size_t)v * ncell(c) + gi];
    }

    /* 2. primitives (local frame), pressure floor counted on interior cells */
    for (int p = 0; p < NP; p++) {
        double rho = b->U[0][p];
        double mn = b->U[1 + d][p], m1 = b->U[1 + t1][p], m2 = b->U[1 + t2][p];
        double Bn = b->U[4 + d][p], B1 = b->U[4 + t1][p], B2 = b->U[4 + t2][p];
        double E = b->U[7][p];
        double pr = (gam - 1.0) * (E - 0.5 * (mn * mn + m1 * m1 + m2 * m2) / rho
                                   - 0.5 * (Bn * Bn + B1 * B1 + B2 * B2));
        if (pr < c->p_min) {
            pr = c->p_min;
            if (p >= G && p < G + N) (*floors)++;
        }
        b->q[0][p] = rho; b->q[1][p] = mn / rho; b->q[2][p] = m1 / rho; b->q[3][p] = m2 / rho;
        b->q[4][p] = B1; b->q[5][p] = B2; b->q[6][p] = pr;
        b->Bn[p] = Bn;
        b->Pt[p] = pr + 0.5 * (Bn * Bn + B1 * B1 + B2 * B2);
        b->W[p] = rho * sqrt(orc_fast_speed2(rho, pr, Bn, B1, B2, gam));
        b->tmp[p] = rho * b->dx[p];        /* mass width dm */
    }
    const double *dm = b->tmp;

    /* 3. flattening coefficient (CW84 App. A) on total pressure and u [R] */
    orc_flatten(NP, b->Pt, b->q[1], b->ft, b->f);

    /* 4. Lagrangian PPM of the 7 primitives on the mass coordinate, then the
     *    domain-of-dependence averages (CW84 eq. 1.12), each over the mass its
     *    own characteristic family sweeps in dt: y = W dt / dm for the fast
     *    family (rho, u, p and B_t for the total pressure), y = Z dt / dm for
     *    the Alfven family (v_t and B_t for sigma) [R]. */
    for (int v = 0; v < NREC; v++) orc_ppm_edges(NP, dm, b->q[v], 1, b->edge[v]);
    for (int p = 3; p <= NP - 4; p++) {
        double yf = b->W[p] * dt / dm[p];
        double ya = sqrt(b->q[0][p]) * fabs(b->Bn[p]) * dt / dm[p];
        for (int v = 0; v < NREC; v++) {
            double o[3];
            orc_ppm_parabola(b->q[v][p], b->edge[v][p - 1], b->edge[v][p], b->f[p], o);
            double y = (v == 2 || v == 3) ? ya : yf;
            b->sl[v][p] = orc_avg_right(o[0], o[1], o[2], y);
            b->sr[v][p] = orc_avg_left(o[0], o[1], o[2], y);
            if (v == 4 || v == 5) {
                b->sl[v + 3][p] = orc_avg_right(o[0], o[1], o[2], ya);
                b->sr[v + 3][p] = orc_avg_left(o[0], o[1], o[2], ya);
            }
        }
    }

    /* 5. Riemann problem at each interface i+1/2, i in [3, NP-5] */
    for (int p = 3; p <= NP - 5; p++) {
        double Ls[NTR], Rs[NTR], o[8];
        for (int v = 0; v < NTR; v++) { Ls[v] = b->sl[v][p]; Rs[v] = b->sr[v][p + 1]; }
        double Bnf = 0.5 * (b->Bn[p] + b->Bn[p + 1]);
        orc_riemann_nl(Ls, Rs, Bnf, gam, c->riemann_iters, o);
        for (int v = 0; v < 8; v++) b->rs[v][p] = o[v];
        b->Bnf[p] = Bnf;
    }

    /* 6. Lagrangian update, cells [4, NP-5]: interfaces p-1 (left), p (right) */
    for (int p = 4; p <= NP - 5; p++) {
        double dmp = dm[p];
        double dxL = b->dx[p] + dt * (b->rs[0][p] - b->rs[0][p - 1]);
        if (!(dxL > 0.0)) *flags |= FLAG_CFL;
        double uL = b->q[1][p] - dt * (b->rs[2][p] - b->rs[2][p - 1]) / dmp;
        double v1L = b->q[2][p] + dt * (b->rs[5][p] - b->rs[5][p - 1]) / dmp;
        double v2L = b->q[3][p] + dt * (b->rs[6][p] - b->rs[6][p - 1]) / dmp;
        double bv1 = dt * (b->Bnf[p] * b->rs[3][p] - b->Bnf[p - 1] * b->rs[3][p - 1]);
        double bv2 = dt * (b->Bnf[p] * b->rs[4][p] - b->Bnf[p - 1] * b->rs[4][p - 1]);
        double B1dx = b->q[4][p] * b->dx[p] + bv1;
        double B2dx = b->q[5][p] * b->dx[p] + bv2;
        double eL = b->U[7][p] / b->q[0][p] - dt * (b->rs[7][p] - b->rs[7][p - 1]) / dmp;
        double rhoL = dmp / dxL;
        b->dxL[p] = dxL;
        b->rq[0][p] = rhoL;
        b->rq[1][p] = rhoL * uL;
        b->rq[2][p] = rhoL * v1L;
        b->rq[3][p] = rhoL * v2L;
        b->rq[4][p] = B1dx / dxL;
        b->rq[5][p] = B2dx / dxL;
        b->rq[6][p] = rhoL * eL;
        /* content increments of the Lagrangian step (exact differences of
         * the Lagrangian contents and the old contents) */
        b->dC[0][p] = 0.0;
        b->dC[1][p] = -dt * (b->rs[2][p] - b->rs[2][p - 1]);
        b->dC[2][p] = dt * (b->rs[5][p] - b->rs[5][p - 1]);
        b->dC[3][p] = dt * (b->rs[6][p] - b->rs[6][p - 1]);
        b->dC[4][p] = bv1;
        b->dC[5][p] = bv2;
        b->dC[6][p] = -dt * (b->rs[7][p] - b->rs[7][p - 1]);
    }

    /* 7. remap: PPM of the 7 conserved densities on the Lagrangian widths (no
     *    flattening [R]) and the sliver fluxes through the Eulerian edges. */
    for (int v = 0; v < NREC; v++) {
        /* edges over the Lagrangian cells [4, NP-5]: shift the arrays so that
         * orc_ppm_edges sees only valid cells */
        int n4 = NP - 8;
        orc_ppm_edges(n4, b->dxL + 4, b->rq[v] + 4, 1, b->edge[v] + 4);
    }
    /* contact steepening (option) [R: Colella & Woodward (1984), Sec. 1,
     * applied in the remap, where contacts move across the fixed grid].  The
     * weight eta of zone p comes from the Lagrangian density on the Lagrangian
     * widths: its second differences d2 must change sign across the zone, its
     * jump exceed ST_EPS of the smaller neighbour, and the zone must not sit
     * in a shock (total-pressure jump of the sweep input, relative, times
     * gamma ST_K0, at least the relative density jump).  The same eta blends
     * the parabola ends of all seven densities towards the one-sided values
     * a_{p-1} + slope_{p-1}/2 and a_{p+1} - slope_{p+1}/2, so that quantities
     * that are affine in the density across a contact stay consistent. */
    if (c->steepen) {
        for (int v = 0; v < NREC; v++)
            for (int p = 5; p <= NP - 6; p++)
                b->slq[v][p] = ppm_limit(b->rq[v] + 4, p - 4, ppm_slope(b->dxL + 4, b->rq[v] + 4, p - 4));
        const double *r = b->rq[0], *w = b->dxL;
        for (int p = 5; p <= NP - 6; p++)
            b->d2[p] = ((r[p + 1] - r[p]) / (w[p + 1] + w[p]) - (r[p] - r[p - 1]) / (w[p] + w[p - 1])) /
                       (w[p - 1] + w[p] + w[p + 1]);
        for (int p = 6; p <= NP - 7; p++) {
            double eta = 0.0;
            double dr = r[p + 1] - r[p - 1];
            double rmin = fabs(r[p + 1]) < fabs(r[p - 1]) ? fabs(r[p + 1]) : fabs(r[p - 1]);
            double Pp = b->Pt[p + 1], Pm = b->Pt[p - 1], rp = b->q[0][p + 1], rm = b->q[0][p - 1];
            int shock = gam * ST_K0 * fabs(Pp - Pm) / (Pp < Pm ? Pp : Pm) >= fabs(rp - rm) / (rp < rm ? rp : rm);
            if (b->d2[p + 1] * b->d2[p - 1] < 0.0 && fabs(dr) - ST_EPS * rmin > 0.0 && !shock) {
                double xl = 0.5 * (w[p - 1] + w[p]), xr = 0.5 * (w[p] + w[p + 1]);
                double et = -(b->d2[p + 1] - b->d2[p - 1]) / dr * (xl * xl * xl + xr * xr * xr) / (xl + xr);
                eta = ST_ETA1 * (et - ST_ETA2);
                if (eta < 0.0) eta = 0.0;
                if (eta > 1.0) eta = 1.0;
            }
            b->eta[p] = eta;
        }
    }
    for (int p = 6; p <= NP - 7; p++) {
        for (int v = 0; v < NREC; v++) {
            double l = b->edge[v][p - 1], r = b->edge[v][p], a6;
            if (c->steepen && b->eta[p] > 0.0) {
                double eta = b->eta[p];
                double ld = b->rq[v][p - 1] + 0.5 * b->slq[v][p - 1];
                double rd = b->rq[v][p + 1] - 0.5 * b->slq[v][p + 1];
                l = l * (1.0 - eta) + eta * ld;
                r = r * (1.0 - eta) + eta * rd;
            }
            ppm_monotone(b->rq[v][p], &l, &r, &a6);
            b->aL[v][p] = l; b->aR[v][p] = r; b->a6[v][p] = a6;
        }
    }
    for (int p = 6; p <= NP - 8; p++) {        /* edge p+1/2 between zones p, p+1 */
        double del = dt * b->rs[0][p];
        for (int v = 0; v < NREC; v++) b->F[v][p] = 0.0;
        if (del > 0.0) {
            double y = del / b->dxL[p];
            if (y >= 1.0) *flags |= FLAG_CFL;
            for (int v = 0; v < NREC; v++)
                b->F[v][p] = del * orc_avg_right(b->aL[v][p], b->aR[v][p], b->a6[v][p], y);
        } else if (del < 0.0) {
            double y = -del / b->dxL[p + 1];
            if (y >= 1.0) *flags |= FLAG_CFL;
            for (int v = 0; v < NREC; v++)
                b->F[v][p] = del * orc_avg_left(b->aL[v][p + 1], b->aR[v][p + 1], b->a6[v][p + 1], y);
        }
    }

    /* 8. new Eulerian state of the interior cells: remap increment, then the
     *    directional part of the dipole and Powell source terms [R], then the
     *    inner-sphere reset [R]. */
    const int cmap[NREC] = {0, 1 + d, 1 + t1, 1 + t2, 4 + t1, 4 + t2, 7};
    const int do_src = c->M != 0.0 || c->powell;
    for (int p = G; p < G + N; p++) {
        double Un[NVAR];
        for (int v = 0; v < NVAR; v++) Un[v] = b->U[v][p];
        for (int v = 0; v < NREC; v++) {
            double dU = (b->dC[v][p] + b->F[v][p - 1] - b->F[v][p]) / b->dx[p];
            Un[cmap[v]] = Un[cmap[v]] + dU;
        }
        if (do_src) {
            double h = 0.5 * b->dx[p - 1] + b->dx[p] + 0.5 * b->dx[p + 1];
            /* local-frame vectors at p-1, p, p+1 */
            double vv[3][3], BB[3][3], A[3][3];
            for (int s = 0; s < 3; s++) {
                int pp = p - 1 + s;
                double rho = b->U[0][pp];
                vv[s][0] = b->U[1 + d][pp] / rho;
                vv[s][1] = b->U[1 + t1][pp] / rho;
                vv[s][2] = b->U[1 + t2][pp] / rho;
                BB[s][0] = b->U[4 + d][pp]; BB[s][1] = b->U[4 + t1][pp]; BB[s][2] = b->U[4 + t2][pp];
                double Bx = b->Bd[0][pp], By = b->Bd[1][pp], Bz = b->Bd[2][pp];
                A[s][0] = vv[s][1] * Bz - vv[s][2] * By;    /* v x B_d */
                A[s][1] = vv[s][2] * Bx - vv[s][0] * Bz;
                A[s][2] = vv[s][0] * By - vv[s][1] * Bx;
            }
            double DB[3], DA[3];
            for (int m = 0; m < 3; m++) { DB[m] = (BB[2][m] - BB[0][m]) / h; DA[m] = (A[2][m] - A[0][m]) / h; }
            double J[3] = {0.0, -DB[2], DB[1]};              /* e_n x D B' */
            double cA[3] = {0.0, -DA[2], DA[1]};             /* e_n x D (v x B_d) */
            double Bd0 = b->Bd[0][p], Bd1 = b->Bd[1][p], Bd2 = b->Bd[2][p];
            double Sm[3] = {J[1] * Bd2 - J[2] * Bd1, J[2] * Bd0 - J[0] * Bd2, J[0] * Bd1 - J[1] * Bd0};
            double divB = DB[0];
            double SB[3], pw = c->powell ? 1.0 : 0.0;
            for (int m = 0; m < 3; m++) SB[m] = cA[m] - pw * vv[1][m] * divB;
            double SE = vv[1][0] * Sm[0] + vv[1][1] * Sm[1] + vv[1][2] * Sm[2]
                        + BB[1][0] * cA[0] + BB[1][1] * cA[1] + BB[1][2] * cA[2];
            const int mi[3] = {1 + d, 1 + t1, 1 + t2}, bi[3] = {4 + d, 4 + t1, 4 + t2};
            for (int m = 0; m < 3; m++) {
                Un[mi[m]] = Un[mi[m]] + dt * Sm[m];
                Un[bi[m]] = Un[bi[m]] + dt * SB[m];
            }
            Un[7] = Un[7] + dt * SE;
        }
        double xyz[3] = {tc[0], tc[1], tc[2]};
        xyz[d] = b->pos[p];
        size_t gi = gidx(c, d, p - G, j, k);
        if (is_inner(c, xyz[0], xyz[1], xyz[2])) inner_state(c, gi, Un);
        for (int v = 0; v < NVAR; v++) {
            if (!isfinite(Un[v])) *flags |= FLAG_NONFINITE;
            c->Unew[(size_t)v * ncell(c) + gi] = Un[v];
        }
    }
}

/* A sweep along an axis of one cell with periodic faces and no dipole is an
 * exact no-op (every pencil is uniform); it is skipped. */
static int sweep_is_noop(const orc_ctx *c, int d)
{
    return c->n[d] == 1 && c->bc[d][0] == BC_PERIODIC && c->bc[d][1] == BC_PERIODIC && c->M == 0.0;
}

int orc_sweep(orc_ctx *c, int d, double dt)
{
    if (sweep_is_noop(c, d)) return 0;
    int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
    int nj = c->n[a1], nk = c->n[a2];
    long long floors = 0;
    int flags = 0;
    long total = (long)nj * nk;
#pragma omp parallel reduction(+ : floors) reduction(| : flags)
    {
        pencil_buf b;
        pb_alloc(&b, c->n[d] + 2 * G);
#pragma omp for schedule(static)
        for (long t = 0; t < total; t++) {
            int j = (int)(t % nj), k = (int)(t / nj);
            sweep_pencil(c, d, j, k, dt, &b, &floors, &flags);
        }
        pb_free(&b);
    }
    double *tmp = c->U; c->U = c->Unew; c->Unew = tmp;
    c->floors += floors;
    return flags;
}

/* One sweep of only the listed pencils (j[p], k[p]: the two transverse
 * indices in increasing axis order), for sampled comparisons on grids too
 * large to sweep whole.  The state is not modified; out receives, per pencil,
 * the 8 conserved arrays of its n[axis] cells ([pencil][var][cell]). */
int orc_sweep_sampled(orc_ctx *c, int d, double dt, int npencil, const int *j, const int *k, double *out)
{
    const int N = c->n[d];
    long long floors = 0;
    int flags = 0;
    if (sweep_is_noop(c, d)) {
        for (int q = 0; q < npencil; q++)
            for (int v = 0; v < NVAR; v++)
                for (int i = 0; i < N; i++)
                    out[((size_t)q * NVAR + v) * N + i] = c->U[(size_t)v * ncell(c) + gidx(c, d, i, j[q], k[q])];
        return 0;
    }
#pragma omp parallel reduction(+ : floors) reduction(| : flags)
    {
        pencil_buf b;
        pb_alloc(&b, N + 2 * G);
#pragma omp for schedule(static)
        for (int q = 0; q < npencil; q++) {
            sweep_pencil(c, d, j[q], k[q], dt, &b, &floors, &flags);
            for (int v = 0; v < NVAR; v++)
                for (int i = 0; i < N; i++)
                    out[((size_t)q * NVAR + v) * N + i] = c->Unew[(size_t)v * ncell(c) + gidx(c, d, i, j[q], k[q])];
        }
        pb_free(&b);
    }
    return flags;
}

/* One full step [R: sweep order alternates x,y,z / z,y,x with step parity]. */
int orc_step(orc_ctx *c, double dt)
{
    int flags = 0;
    if ((c->steps & 1) == 0) { for (int d = 0; d < 3; d++) flags |= orc_sweep(c, d, dt); }
    else { for (int d = 2; d >= 0; d--) flags |= orc_sweep(c, d, dt); }
    c->steps++;
    return flags;
}

/* CFL time step [R]: dt = cfl * min over non-inner interior cells and axes of
 * dx_d / (|v_d| + max(c_f,d(B'), c_f,d(B' + B_d))). */
double orc_cfl_dt(const orc_ctx *c, double cfl)
{
    const double gam = c->gamma;
    double best = INFINITY;
    long total = (long)c->n[1] * c->n[2];
#pragma omp parallel for reduction(min : best) schedule(static)
    for (long t = 0; t < total; t++) {
        int iy = (int)(t % c->n[1]), iz = (int)(t / c->n[1]);
        for (int ix = 0; ix < c->n[0]; ix++) {
            double x = c->c[0][G + ix], y = c->c[1][G + iy], z = c->c[2][G + iz];
            if (is_inner(c, x, y, z)) continue;
            size_t gi = ((size_t)iz * c->n[1] + iy) * c->n[0] + ix;
            size_t nc = ncell(c);
            double U[NVAR];
            for (int v = 0; v < NVAR; v++) U[v] = c->U[(size_t)v * nc + gi];
            double Bd[3];
            orc_dipole(c->M, x, y, z, Bd);
            int idx[3] = {ix, iy, iz};
            for (int d = 0; d < 3; d++) {
                int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
                double rho = U[0];
                double mn = U[1 + d], m1 = U[1 + t1], m2 = U[1 + t2];
                double Bn = U[4 + d], B1 = U[4 + t1], B2 = U[4 + t2];
                double pr = (gam - 1.0) * (U[7] - 0.5 * (mn * mn + m1 * m1 + m2 * m2) / rho
                                           - 0.5 * (Bn * Bn + B1 * B1 + B2 * B2));
                if (pr < c->p_min) pr = c->p_min;
                double c1 = orc_fast_speed2(rho, pr, Bn, B1, B2, gam);
                double c2 = orc_fast_speed2(rho, pr, Bn + Bd[d], B1 + Bd[t1], B2 + Bd[t2], gam);
                double cf = sqrt(c1 > c2 ? c1 : c2);
                double s = c->w[d][G + idx[d]] / (fabs(mn / rho) + cf);
                if (s < best) best = s;
            }
        }
    }
    return cfl * best;
}
