// Mixed-precision sweep, marching form: one thread per pencil, walking it
// cell by cell (Sec. II scheme, Sec. III-A split; the same arithmetic as the
// tile form of sweep.cuh for R = float).
//
// The tile form gives every cell of a tile its own thread and passes the
// values a neighbour needs through shared memory between barrier-separated
// phases; on GB300 that exchange, the per-phase index work and the halo
// positions cost more issue slots than the arithmetic itself.  Here a warp
// holds 32 pencils (lanes) and all its threads advance together along the
// sweep axis.  At input cell g a thread runs every stage of the scheme once,
// each on the newest cell whose inputs are complete:
//   S1  cell g:     load (with the boundary ghosts), primitives, p floor
//   S2  zone g-1:   limited slopes; flattening indicator of zone g-2;
//                   directional sources of zone g-1
//   S3  edge g-3/2: interface values
//   S4  zone g-3:   flattening, parabolas, domain-of-dependence states
//   S5  edge g-7/2: Lagrangian Riemann problem
//   S6  zone g-4:   Lagrangian update
//   S7  zone g-5:   remap slopes
//   S8  edge g-11/2: remap interface values
//   S9  zone g-6:   remap parabola, donor fluxes through its edges
//   S10 zone g-7:   new state, sources, inner sphere, store
// Neighbour values come from register windows shifted once per cell; the
// two values that wait longest (the sources of a zone, six cells, and its
// Lagrangian content changes, three cells) wait in a per-thread ring in
// shared memory.  A chunk of C output cells reads C + 14 input cells (7
// ghost cells at each end); the first 14 iterations fill the pipeline and
// their stage results outside the dependency cone of the outputs are never
// stored or flagged.
//
// Loads: y and z sweeps run lanes along x (consecutive x cells: every warp
// access is one contiguous row segment per variable); the x sweep runs lanes
// across pencils and reads each pencil's consecutive cells through L1.
#pragma once
#include "sweep.cuh"

namespace ppmlr {

constexpr int MARCH_WARPS = 4;                      // warps per block (independent)
constexpr int MARCH_SRC_SLOTS = 8;                  // ring slots of the source terms (a delay of 6 cells)
constexpr int MARCH_DC_SLOTS = 4;                   // ring slots of the content changes (a delay of 3 cells)
constexpr int MARCH_RING = MARCH_SRC_SLOTS * 7 + MARCH_DC_SLOTS * 6;   // floats per thread
constexpr size_t march_smem_bytes() { return (size_t)MARCH_RING * 32 * MARCH_WARPS * sizeof(float); }

// Warps of a marching sweep launch: lane groups of 32 pencils x chunks.
__host__ __device__ inline int march_warps(const SweepArgs &a, int dir)
{
    const int other = dir == 0 ? 1 : (dir == 1 ? a.n[2] : a.n[1]);
    return a.ngx * a.nchunk * other;
}

template <int DIR>
__global__ void __launch_bounds__(32 * MARCH_WARPS, 1) sweep_march_kernel(const SweepArgs a)
{
    extern __shared__ __align__(16) float march_ring[];
    constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * MARCH_WARPS + (threadIdx.x >> 5);
    if (warp >= march_warps(a, DIR)) return;
    const int nt = blockDim.x;
    float *const ring = march_ring + threadIdx.x;
#define RSRC(slot, k) ring[(((slot) & (MARCH_SRC_SLOTS - 1)) * 7 + (k)) * nt]
#define RDC(slot, k) ring[(MARCH_SRC_SLOTS * 7 + ((slot) & (MARCH_DC_SLOTS - 1)) * 6 + (k)) * nt]

    // ---- lane decode (lanes past the domain edge follow the last pencil and store nothing)
    const int chunk = warp % a.nchunk, grp = warp / a.nchunk;
    int ix = 0, iy = 0, iz = 0;
    bool lane_ok;
    if (DIR == 0) {
        const long long np = (long long)a.n[1] * a.n[2];
        long long q = (long long)grp * 32 + lane;
        lane_ok = q < np;
        if (!lane_ok) q = np - 1;
        iy = (int)(q % a.n[1]);
        iz = (int)(q / a.n[1]);
    } else {
        const int xg = grp % a.ngx, t = grp / a.ngx;
        ix = xg * 32 + lane;
        lane_ok = ix < a.n[0];
        if (!lane_ok) ix = a.n[0] - 1;
        if (DIR == 1) iz = t; else iy = t;
    }
    long long base, stride;
    if (DIR == 0) { base = ((long long)iz * a.n[1] + iy) * a.n[0]; stride = 1; }
    else if (DIR == 1) { base = (long long)iz * a.n[1] * a.n[0] + ix; stride = a.n[0]; }
    else { base = (long long)iy * a.n[0] + ix; stride = (long long)a.n[0] * a.n[1]; }
    const double *__restrict__ Uin = a.U;
    double *__restrict__ Uout = a.Un;
    const long long vs = a.vs;
    const int N = a.N;
    const int g0 = chunk * a.C;
    const int Ce = min(a.C, N - g0);
    const double dt = a.dt_dev ? *a.dt_dev : a.dt;
    const float dtr = (float)dt;
    const float gam = a.gammaf, gm1 = a.gammaf - 1.0f;
    const float *__restrict__ wf = a.wf + GH;          // widths along the axis, index = cell (ghosts < 0, >= N)
    const float *__restrict__ caxf = (DIR == 0 ? a.cxf : DIR == 1 ? a.cyf : a.czf) + GH;
    // transverse centres of this lane (float for the dipole, double for the
    // exact test of centres near the inner sphere)
    const float pxl = DIR == 0 ? 0.0f : a.cxf[ix + GH];
    const float pyl = DIR == 1 ? 0.0f : a.cyf[iy + GH];
    const float pzl = DIR == 2 ? 0.0f : a.czf[iz + GH];

    // ---- register windows (suffix: cells behind the newest input cell g)
    float rho0 = 0, u0 = 0, v1_0 = 0, v2_0 = 0, B1_0 = 0, B2_0 = 0, p0 = 0;
    float rho1 = 0, u1 = 0, v1_1 = 0, v2_1 = 0, B1_1 = 0, B2_1 = 0, p1 = 0;
    float rho2 = 0, u2 = 0, v1_2 = 0, v2_2 = 0, B1_2 = 0, B2_2 = 0, p2 = 0;
    float rho3 = 0, u3 = 0, v1_3 = 0, v2_3 = 0, B1_3 = 0, B2_3 = 0, p3 = 0;
    float u4 = 0, v1_4 = 0, v2_4 = 0, B1_4 = 0, B2_4 = 0;
    float Bn0 = 0, Bn1 = 0, Bn2 = 0, Bn3 = 0, Bn4 = 0;
    float dm0 = 0, dm1 = 0, dm2 = 0, dm3 = 0, dm4 = 0;
    float e0 = 0, e1 = 0, e2 = 0, e3 = 0, e4 = 0;
    float Pt0 = 0, Pt1 = 0, Pt2 = 0, Pt3 = 0, Pt4 = 0;
    float W0 = 0, W1 = 0, W2 = 0, W3 = 0;
    float ft3 = 0, ft4 = 0;
    float AY0 = 0, AY1 = 0, AY2 = 0, AZ0 = 0, AZ1 = 0, AZ2 = 0;
    float Bdn1 = 0, Bdt1_1 = 0, Bdt2_1 = 0;           // dipole of zone g-1 (normal, t1, t2)
    float da2[7] = {0, 0, 0, 0, 0, 0, 0};             // limited slopes of zone g-2
    float eA[7] = {0, 0, 0, 0, 0, 0, 0};              // interface values at g-7/2
    float eB[7] = {0, 0, 0, 0, 0, 0, 0};              // interface values at g-5/2
    float dtm4 = 0;                                   // dt / dm of zone g-4
    float slP[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};       // right-end states of zone g-4
    float rsP[7] = {0, 0, 0, 0, 0, 0, 0};             // Riemann output at g-9/2
    float us9 = 0, us11 = 0, us13 = 0;                // u* at g-9/2, g-11/2, g-13/2
    float qL5[7] = {0, 0, 0, 0, 0, 0, 0}, qL6[7] = {0, 0, 0, 0, 0, 0, 0};
    float dxL5 = 0, dxL6 = 0, dxL7 = 0, idxL5 = 0, idxL6 = 0;
    float rda6[7] = {0, 0, 0, 0, 0, 0, 0};            // remap slopes of zone g-6
    float reP[7] = {0, 0, 0, 0, 0, 0, 0};             // remap interface values at g-13/2
    float Fc[7] = {0, 0, 0, 0, 0, 0, 0};              // flux through g-13/2 if zone g-7 is its donor
    float Fm[7] = {0, 0, 0, 0, 0, 0, 0};              // flux through g-15/2
    int flags = 0;
    unsigned floors = 0;

    // source cell of input cell g along the pencil (boundary ghosts); -1: the inflow state
    auto source_cell = [&](int g) -> int {
        if (g >= 0 && g < N) return g;
        const int kind = g < 0 ? a.bc_lo : a.bc_hi;
        if (kind == PPMLR_BC_PERIODIC) return ((g % N) + N) % N;
        if (kind == PPMLR_BC_OUTFLOW) return g < 0 ? 0 : N - 1;
        return -1;
    };
    double cur[8], nxt[8];
    {
        const int src = source_cell(g0 - GH);
        if (src >= 0) {
            const long long gi = base + (long long)src * stride;
#pragma unroll
            for (int v = 0; v < 8; v++) cur[v] = __ldg(Uin + v * vs + gi);
        }
    }

    const int gend = g0 + Ce + GH;
    for (int g = g0 - GH; g < gend; g++) {
        // prefetch of the next input cell
        {
            const int src = g + 1 < gend ? source_cell(g + 1) : -1;
            if (src >= 0) {
                const long long gi = base + (long long)src * stride;
#pragma unroll
                for (int v = 0; v < 8; v++) nxt[v] = __ldg(Uin + v * vs + gi);
            }
        }

        // ---------------- S1: cell g ----------------
        float Bd0f, Bd1f, Bd2f;                     // dipole at cell g: normal, t1, t2
        {
            const float pa = caxf[g];
            float B[3];
            dipole_f(a.Mf, DIR == 0 ? pa : pxl, DIR == 1 ? pa : pyl, DIR == 2 ? pa : pzl, B);
            Bd0f = B[DIR]; Bd1f = B[T1]; Bd2f = B[T2];
            const bool out_cell = g >= g0 && g < g0 + Ce;
            float pabs;                                 // p; the windows hold p - p_reff
            if (source_cell(g) < 0) {
                const float *f = a.inflowf;
                rho0 = f[0];
                u0 = f[1 + DIR]; v1_0 = f[1 + T1]; v2_0 = f[1 + T2];
                Bn0 = f[4 + DIR] - Bd0f; B1_0 = f[4 + T1] - Bd1f; B2_0 = f[4 + T2] - Bd2f;
                pabs = f[7];
                p0 = f[7] - a.p_reff;
                e0 = pabs / (gm1 * rho0) + 0.5f * (u0 * u0 + v1_0 * v1_0 + v2_0 * v2_0) +
                     0.5f * (Bn0 * Bn0 + B1_0 * B1_0 + B2_0 * B2_0) / rho0;
            } else {
                df q[8];
#pragma unroll
                for (int v = 0; v < 8; v++) q[v] = split_double_fast(cur[v]);
                const df pp = pressure_df_pair(q[0], q[1 + DIR], q[1 + T1], q[1 + T2], q[4 + DIR], q[4 + T1],
                                               q[4 + T2], q[7], gm1);
                pabs = pp.h + pp.l;
                p0 = (pp.h - a.p_reff) + pp.l;
                rho0 = q[0].h;
                const float ir = 1.0f / rho0;
                u0 = q[1 + DIR].h * ir; v1_0 = q[1 + T1].h * ir; v2_0 = q[1 + T2].h * ir;
                Bn0 = q[4 + DIR].h; B1_0 = q[4 + T1].h; B2_0 = q[4 + T2].h;
                e0 = q[7].h * ir;
            }
            if (pabs < a.p_minf) {
                pabs = a.p_minf;
                p0 = a.p_minf - a.p_reff;
                floors += (out_cell && lane_ok) ? 1u : 0u;
            }
            dm0 = rho0 * wf[g];
            Pt0 = pabs + 0.5f * (Bn0 * Bn0 + B1_0 * B1_0 + B2_0 * B2_0);
            W0 = rho0 * fsqrt<float, false>(fast2<float, false>(rho0, pabs, Bn0, B1_0, B2_0, gam));
            AY0 = v2_0 * Bd0f - u0 * Bd2f;
            AZ0 = u0 * Bd1f - v1_0 * Bd0f;
        }

        // ---------------- S2: slopes of zone g-1, flattening indicator of zone g-2, sources of zone g-1
        float da1[7];
        {
            const SlopeCoef<float> k = slope_coef<float, false>(dm2, dm1, dm0);
            const float am[7] = {rho2, u2, v1_2, v2_2, B1_2, B2_2, p2};
            const float a0[7] = {rho1, u1, v1_1, v2_1, B1_1, B2_1, p1};
            const float ap[7] = {rho0, u0, v1_0, v2_0, B1_0, B2_0, p0};
#pragma unroll
            for (int v = 0; v < 7; v++) da1[v] = limit_slope<float, false>(am[v], a0[v], ap[v], k.c1, k.c2, k.c3);
        }
        float ft2 = 0.0f;
        {
            const float dP = Pt1 - Pt3;
            const float pmin = Pt1 < Pt3 ? Pt1 : Pt3;
            if (fabsf(dP) > 0.33f * pmin && u3 - u1 > 0.0f) {
                const float den = Pt0 - Pt4;
                const float steep = den != 0.0f ? dP / den : 1.0f;
                float f = (steep - 0.75f) * 10.0f;
                if (f < 0.0f) f = 0.0f;
                if (f > 1.0f) f = 1.0f;
                ft2 = f;
            }
        }
        if (a.do_src) {
            // (the first two iterations have no zone g-2 / g-1 in the table:
            // clamped, their results are outside every output's dependencies)
            const float h = 0.5f * wf[max(g - 2, g0 - GH)] + wf[max(g - 1, g0 - GH)] + 0.5f * wf[g];
            const float ih = 1.0f / h;
            const float DB0 = (Bn0 - Bn2) * ih, DB1 = (B1_0 - B1_2) * ih, DB2 = (B2_0 - B2_2) * ih;
            const float DA1 = (AY0 - AY2) * ih, DA2 = (AZ0 - AZ2) * ih;
            const float J1 = -DB2, J2 = DB1, cA1 = -DA2, cA2 = DA1, divB = DB0;
            const float sm0 = J1 * Bdt2_1 - J2 * Bdt1_1, sm1 = J2 * Bdn1, sm2 = -(J1 * Bdn1);
            float sb0 = 0.0f, sb1 = cA1, sb2 = cA2;
            if (a.powell) {
                sb0 = -(u1 * divB);
                sb1 = cA1 - v1_1 * divB;
                sb2 = cA2 - v2_1 * divB;
            }
            const float se = u1 * sm0 + v1_1 * sm1 + v2_1 * sm2 + B1_1 * cA1 + B2_1 * cA2;
            const int z = g - 1;
            RSRC(z, 0) = sm0; RSRC(z, 1) = sm1; RSRC(z, 2) = sm2;
            RSRC(z, 3) = sb0; RSRC(z, 4) = sb1; RSRC(z, 5) = sb2; RSRC(z, 6) = se;
        }

        // ---------------- S3: interface values at g-3/2 (zones g-2 | g-1)
        float en[7];
        {
            const EdgeCoef<float> k = edge_coef<float, false>(dm3, dm2, dm1, dm0);
            const float a0[7] = {rho2, u2, v1_2, v2_2, B1_2, B2_2, p2};
            const float a1[7] = {rho1, u1, v1_1, v2_1, B1_1, B2_1, p1};
#pragma unroll
            for (int v = 0; v < 7; v++) en[v] = edge_value_d<float>(k, a0[v], a1[v] - a0[v], da2[v], da1[v]);
        }

        // ---------------- S4: zone g-3: flattening, parabolas, traced states
        float sl[9], sr[9];
        const float dtm3 = dtr / dm3;                 // dt / dm of zone g-3 (S6 of the next cell)
        {
            const float up = Pt2 - Pt4 < 0.0f ? ft2 : ft4;
            const float flat = ft3 > up ? ft3 : up;
            const float dtm = dtm3;
            const float yf = W3 * dtm;
            const float ya = fsqrt<float, false>(rho3) * fabsf(Bn3) * dtm;
            const float own[7] = {rho3, u3, v1_3, v2_3, B1_3, B2_3, p3};
            const bool blend = flat != 0.0f;
            const AvgCoef<float> kf = avg_coef<float>(yf), ka = avg_coef<float>(ya);
#pragma unroll
            for (int v = 0; v < 7; v++) {
                float lft = eA[v], rgt = eB[v];
                if (blend) {
                    lft = flat * own[v] + (1.0f - flat) * lft;
                    rgt = flat * own[v] + (1.0f - flat) * rgt;
                }
                float dl2, dr2;
                monotone_d(own[v], lft, rgt, dl2, dr2);
                const AvgCoef<float> &k = (v == 2 || v == 3) ? ka : kf;
                sl[v] = avg_right_d<float>(own[v], dl2, dr2, k);
                sr[v] = avg_left_d<float>(own[v], dl2, dr2, k);
                if (v == 4 || v == 5) {
                    sl[v + 3] = avg_right_d<float>(own[v], dl2, dr2, ka);
                    sr[v + 3] = avg_left_d<float>(own[v], dl2, dr2, ka);
                }
            }
        }

        // ---------------- S5: Riemann problem at g-7/2 (zone g-4 left, zone g-3 right)
        float rs[7];
        {
            const float Bnf = 0.5f * (Bn4 + Bn3);
            const float PL = slP[6] + 0.5f * (slP[4] * slP[4] + slP[5] * slP[5]);
            const float PR = sr[6] + 0.5f * (sr[4] * sr[4] + sr[5] * sr[5]);
            // (PL, PR, P* and S* relative to p_reff; absolute pressures for the
            // impedances, the nonlinear solver and the energy flux)
            const float pref = a.p_reff;
            float WL = slP[0] * sqrtf(fast2<float, false>(slP[0], slP[6] + pref, Bnf, slP[4], slP[5], gam));
            float WR = sr[0] * sqrtf(fast2<float, false>(sr[0], sr[6] + pref, Bnf, sr[4], sr[5], gam));
            const float PLa = PL + pref, PRa = PR + pref;
            if (a.riemann_iters > 0 && PLa > 0.0f && PRa > 0.0f)
                two_shock<float, false>(a.riemann_iters, slP[1], sr[1], PLa, PRa, gam, WL, WR);
            const float iW = 1.0f / (WL + WR);
            const float us = (WL * slP[1] + WR * sr[1] + PL - PR) * iW;
            const float Ps = (WR * PL + WL * PR + WL * WR * (slP[1] - sr[1])) * iW;
            const float Ss = Ps - 0.5f * Bnf * Bnf;
            const float ZL = fsqrt<float, false>(slP[0]) * fabsf(Bnf);
            const float ZR = fsqrt<float, false>(sr[0]) * fabsf(Bnf);
            const float zsum = ZL + ZR;
            const bool zero_z = zsum == 0.0f;
            const float iZ = zero_z ? 0.0f : 1.0f / zsum;
            float vst[2], sst[2];
#pragma unroll
            for (int t = 0; t < 2; t++) {
                const float vL = slP[2 + t], vR = sr[2 + t];
                const float sL = Bnf * slP[7 + t], sR = Bnf * sr[7 + t];
                if (zero_z) {
                    vst[t] = 0.5f * (vL + vR);
                    sst[t] = 0.0f;
                } else {
                    vst[t] = (ZL * vL + ZR * vR + sR - sL) * iZ;
                    sst[t] = (ZR * sL + ZL * sR + ZL * ZR * (vR - vL)) * iZ;
                }
            }
            rs[0] = us; rs[1] = Ss; rs[2] = sst[0]; rs[3] = sst[1];
            rs[4] = Bnf * vst[0]; rs[5] = Bnf * vst[1];
            rs[6] = (Ss + pref) * us - sst[0] * vst[0] - sst[1] * vst[1];
        }

        // ---------------- S6: Lagrangian update of zone g-4 (edges g-9/2 | g-7/2)
        float qL4[7], dxL4, idxL4;
        {
            const int z = g - 4;
            const float dxr = wf[max(z, g0 - GH)];          // (clamped while the pipeline fills)
            dxL4 = dxr + dtr * (rs[0] - rsP[0]);
            if (!(dxL4 > 0.0f) && z >= g0 - 3 && z <= g0 + Ce + 2) flags |= FLAG_CFL;
            const float bv1 = dtr * (rs[4] - rsP[4]);
            const float bv2 = dtr * (rs[5] - rsP[5]);
            const float B1dx = B1_4 * dxr + bv1;
            const float B2dx = B2_4 * dxr + bv2;
            const float dtm = dtm4;
            idxL4 = 1.0f / dxL4;
            const float uL = u4 - (rs[1] - rsP[1]) * dtm;
            const float v1L = v1_4 + (rs[2] - rsP[2]) * dtm;
            const float v2L = v2_4 + (rs[3] - rsP[3]) * dtm;
            const float eL = e4 - (rs[6] - rsP[6]) * dtm;
            const float rhoL = dm4 * idxL4;
            qL4[0] = rhoL; qL4[1] = rhoL * uL; qL4[2] = rhoL * v1L; qL4[3] = rhoL * v2L;
            qL4[4] = B1dx * idxL4; qL4[5] = B2dx * idxL4; qL4[6] = rhoL * eL;
            RDC(z, 0) = -dtr * (rs[1] - rsP[1]);
            RDC(z, 1) = dtr * (rs[2] - rsP[2]);
            RDC(z, 2) = dtr * (rs[3] - rsP[3]);
            RDC(z, 3) = bv1;
            RDC(z, 4) = bv2;
            RDC(z, 5) = -dtr * (rs[6] - rsP[6]);
        }

        // ---------------- S7: remap slopes of zone g-5
        float rda5[7];
        {
            const SlopeCoef<float> k = slope_coef<float, false>(dxL6, dxL5, dxL4);
#pragma unroll
            for (int v = 0; v < 7; v++) rda5[v] = limit_slope<float, false>(qL6[v], qL5[v], qL4[v], k.c1, k.c2, k.c3);
        }

        // ---------------- S8: remap interface values at g-11/2 (zones g-6 | g-5)
        float ren[7];
        {
            const EdgeCoef<float> k = edge_coef<float, false>(dxL7, dxL6, dxL5, dxL4);
#pragma unroll
            for (int v = 0; v < 7; v++) ren[v] = edge_value_d<float>(k, qL6[v], qL5[v] - qL6[v], rda6[v], rda5[v]);
        }

        // ---------------- S9: remap parabola of zone g-6, donor fluxes through g-13/2 and g-11/2
        float Fp[7];                                   // flux through g-13/2
        {
            const int z = g - 6;
            const float del_m = dtr * us13, del_p = dtr * us11;
            float dl2[7], dr2[7];                      // one-sided differences of the constrained parabola
#pragma unroll
            for (int v = 0; v < 7; v++) monotone_d(qL6[v], reP[v], ren[v], dl2[v], dr2[v]);
            if (del_m < 0.0f) {                        // zone g-6 is the donor of g-13/2
                const float y = -del_m * idxL6;
                if (sliver_too_wide<float, false>(y) && z >= g0 && z <= g0 + Ce) flags |= FLAG_CFL;
                const AvgCoef<float> k = avg_coef<float>(y);
#pragma unroll
                for (int v = 0; v < 7; v++) Fp[v] = del_m * avg_left_d<float>(qL6[v], dl2[v], dr2[v], k);
            } else {
#pragma unroll
                for (int v = 0; v < 7; v++) Fp[v] = Fc[v];
            }
            if (del_p > 0.0f) {                        // zone g-6 is the donor of g-11/2
                const float y = del_p * idxL6;
                if (sliver_too_wide<float, false>(y) && z >= g0 - 1 && z <= g0 + Ce - 1) flags |= FLAG_CFL;
                const AvgCoef<float> k = avg_coef<float>(y);
#pragma unroll
                for (int v = 0; v < 7; v++) Fc[v] = del_p * avg_right_d<float>(qL6[v], dl2[v], dr2[v], k);
            } else {
#pragma unroll
                for (int v = 0; v < 7; v++) Fc[v] = 0.0f;
            }
        }

        // ---------------- S10: zone g-7: new state, sources, inner sphere, store
        {
            const int z = g - 7;
            if (z >= g0 && lane_ok) {
                const long long gi = base + (long long)z * stride;
                double Un[8];
#pragma unroll
                for (int v = 0; v < 8; v++) Un[v] = __ldg(Uin + v * vs + gi);
                const int cmap[7] = {0, 1 + DIR, 1 + T1, 1 + T2, 4 + T1, 4 + T2, 7};
                const float idx = 1.0f / wf[z];
                float dU[8];
                dU[0] = (0.0f + Fm[0] - Fp[0]) * idx;
#pragma unroll
                for (int v = 1; v < 7; v++) dU[cmap[v]] = (RDC(z, v - 1) + Fm[v] - Fp[v]) * idx;
                dU[4 + DIR] = 0.0f;
                if (a.do_src) {
                    dU[1 + DIR] += dtr * RSRC(z, 0); dU[1 + T1] += dtr * RSRC(z, 1); dU[1 + T2] += dtr * RSRC(z, 2);
                    dU[4 + DIR] += dtr * RSRC(z, 3); dU[4 + T1] += dtr * RSRC(z, 4); dU[4 + T2] += dtr * RSRC(z, 5);
                    dU[7] += dtr * RSRC(z, 6);
                }
#pragma unroll
                for (int v = 0; v < 8; v++) Un[v] = Un[v] + widen(dU[v]);
                bool inner = false;
                if (a.inner_mask) {
                    inner = a.inner_mask[gi] != 0;
                } else if (a.r_innerf > 0.0f) {
                    // float test with an exact double test for centres within 1e-5 of the sphere
                    const float pa = caxf[z];
                    const float px = DIR == 0 ? pa : pxl, py = DIR == 1 ? pa : pyl, pz = DIR == 2 ? pa : pzl;
                    const float r2 = px * px + py * py + pz * pz, ri2 = a.r_innerf * a.r_innerf;
                    if (r2 < ri2 * (1.0f - 1e-5f)) inner = true;
                    else if (r2 < ri2 * (1.0f + 1e-5f)) {
                        const double x = a.cx[(DIR == 0 ? z : ix) + GH], y = a.cy[(DIR == 1 ? z : iy) + GH],
                                     zz = a.cz[(DIR == 2 ? z : iz) + GH];
                        inner = x * x + y * y + zz * zz < a.r_inner * a.r_inner;
                    }
                }
                if (inner && a.inner_cells) {     // the ionosphere's state of this cell
                    int lo = 0, hi = a.n_inner - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (a.inner_cells[mid] < gi) lo = mid + 1; else hi = mid;
                    }
                    if (a.inner_cells[lo] == gi) {
#pragma unroll
                        for (int v = 0; v < 8; v++) Un[v] = a.inner_state[(long long)v * a.n_inner + lo];
                        inner = false;
                    }
                }
                if (inner) {
                    const double *q = a.inner;
                    const double rh = q[0];
                    Un[0] = rh;
                    Un[1] = rh * q[1]; Un[2] = rh * q[2]; Un[3] = rh * q[3];
                    Un[4] = 0.0; Un[5] = 0.0; Un[6] = 0.0;
                    Un[7] = q[7] / (a.gamma - 1.0) + 0.5 * rh * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3])
                            + 0.5 * (0.0 * 0.0 + 0.0 * 0.0 + 0.0 * 0.0);
                }
                bool bad = false;
#pragma unroll
                for (int v = 0; v < 8; v++) {   // non-finite test on the exponent bits (integer pipe)
                    bad |= ((__double2hiint(Un[v]) >> 20) & 0x7FF) == 0x7FF;
                    Uout[v * vs + gi] = Un[v];
                }
                if (bad) flags |= FLAG_NONFINITE;
            }
        }

        // ---------------- shift the windows by one cell
#pragma unroll
        for (int v = 0; v < 7; v++) {
            Fm[v] = Fp[v];
            reP[v] = ren[v];
            rda6[v] = rda5[v];
            qL6[v] = qL5[v];
            qL5[v] = qL4[v];
            rsP[v] = rs[v];
            eA[v] = eB[v];
            eB[v] = en[v];
            da2[v] = da1[v];
        }
#pragma unroll
        for (int v = 0; v < 9; v++) slP[v] = sl[v];
        dxL7 = dxL6; dxL6 = dxL5; dxL5 = dxL4;
        idxL6 = idxL5; idxL5 = idxL4;
        us13 = us11; us11 = us9; us9 = rs[0];
        dtm4 = dtm3;
        u4 = u3; v1_4 = v1_3; v2_4 = v2_3; B1_4 = B1_3; B2_4 = B2_3;
        rho3 = rho2; u3 = u2; v1_3 = v1_2; v2_3 = v2_2; B1_3 = B1_2; B2_3 = B2_2; p3 = p2;
        rho2 = rho1; u2 = u1; v1_2 = v1_1; v2_2 = v2_1; B1_2 = B1_1; B2_2 = B2_1; p2 = p1;
        rho1 = rho0; u1 = u0; v1_1 = v1_0; v2_1 = v2_0; B1_1 = B1_0; B2_1 = B2_0; p1 = p0;
        Bn4 = Bn3; Bn3 = Bn2; Bn2 = Bn1; Bn1 = Bn0;
        dm4 = dm3; dm3 = dm2; dm2 = dm1; dm1 = dm0;
        e4 = e3; e3 = e2; e2 = e1; e1 = e0;
        Pt4 = Pt3; Pt3 = Pt2; Pt2 = Pt1; Pt1 = Pt0;
        W3 = W2; W2 = W1; W1 = W0;
        ft4 = ft3; ft3 = ft2;
        AY2 = AY1; AY1 = AY0; AZ2 = AZ1; AZ1 = AZ0;
        Bdn1 = Bd0f; Bdt1_1 = Bd1f; Bdt2_1 = Bd2f;
#pragma unroll
        for (int v = 0; v < 8; v++) cur[v] = nxt[v];
    }
#undef RSRC
#undef RDC

    // flags and the floor count: one atomic per warp
    const unsigned fl = __reduce_or_sync(0xffffffffu, (unsigned)flags);
    const unsigned nf = __reduce_add_sync(0xffffffffu, floors);
    if (lane == 0) {
        if (fl) atomicOr(a.flags, (int)fl);
        if (nf) atomicAdd(a.floors, (unsigned long long)nf);
    }
}

}  // namespace ppmlr
