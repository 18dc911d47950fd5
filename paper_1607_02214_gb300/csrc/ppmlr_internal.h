// Internal declarations of the GB300 split-sweep library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ppmlr.h"

namespace ppmlr {

constexpr int GH = 7;          // ghost cells per pencil end: the stencil radius of one sweep
constexpr int NSM = 28;        // shared-memory exchange arrays per tile (see sweep.cuh)
constexpr int MAXT = 512;      // threads per tile (one thread per cell position and lane)

enum : int { FLAG_CFL = 1, FLAG_NONFINITE = 2 };

// Arguments of one sweep launch (passed by value).
struct SweepArgs {
    const double *U[8];        // input state, 8 SoA arrays
    double *Un[8];             // output state
    int n[3];                  // nx, ny, nz
    int N;                     // cells along the sweep axis
    int C;                     // output cells per chunk along the axis
    int L;                     // lanes (pencils) per tile
    int NP;                    // C + 2*GH positions per lane
    int nchunk;                // chunks per pencil
    int ngx;                   // lane groups along x (y/z sweeps) or pencil groups (x sweep)
    const double *w;           // widths along the sweep axis, N + 2*GH entries (ghosts first)
    const double *c;           // centres along the sweep axis, same indexing
    const double *cx, *cy, *cz;  // centres of every axis, n[d] + 2*GH entries each
    int bc_lo, bc_hi;
    double inflow[8];          // rho, vx, vy, vz, Bx, By, Bz (total), p
    double gamma, p_min, M, r_inner;
    double inner[8];           // rho, vx, vy, vz, -, -, -, p
    int powell, do_src;
    double dt;                 // used when dt_dev == nullptr
    const double *dt_dev;
    int *flags;
    unsigned long long *floors;
    // float copies for the mixed path (geometry and parameters)
    const float *wf;           // widths along the sweep axis, ghost-extended
    const float *cxf, *cyf, *czf;
    float gammaf, p_minf, Mf, r_innerf;
    float inflowf[8];
};

struct CflArgs {
    const double *U[8];
    int n[3];
    const double *w[3];        // ghost-extended widths of each axis
    const double *c[3];        // ghost-extended centres
    double gamma, p_min, M, r_inner;
    double cfl;
    // float copies for the mixed path
    const float *wf[3], *cf[3];
    float gammaf, p_minf, Mf, r_innerf;
    double *partial;           // one entry per block
    unsigned int *counter;     // zero between launches; the last block resets it
    double *dt_out;            // device scalar
};

// Tile shape of one sweep direction.
struct Tile {
    int C, L, NP, nchunk, ngx, ntiles, threads;
    size_t smem;
};

// launchers (defined in the kernel translation units)
cudaError_t launch_sweep_fp64(int dir, const SweepArgs &a, const Tile &t, cudaStream_t s);
cudaError_t launch_sweep_mixed(int dir, const SweepArgs &a, const Tile &t, cudaStream_t s);
cudaError_t launch_cfl(const CflArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_cfl_mixed(const CflArgs &a, int blocks, cudaStream_t s);
int cfl_threads();

}  // namespace ppmlr
