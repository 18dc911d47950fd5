// Internal declarations of the GB300 split-sweep library (not part of the ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ppmlr.h"

namespace ppmlr {

constexpr int GH = 7;          // ghost cells per pencil end: the stencil radius of one sweep
constexpr int NSM = 28;        // shared-memory exchange values per slot (see sweep.cuh)
constexpr int NSMP = 29;       // slot pitch in values: odd, so consecutive slots hit distinct banks
constexpr int MAXT = 512;      // threads per tile (one thread per cell position and lane), mixed path
constexpr int MAXT_F64 = 448;  // FP64 path: fewer threads, up to 146 registers each
// Contracted FP64 x sweep: its kernel is held to 96 registers, so a block of
// up to 640 threads fits one SM (its 20 warps' registers split over the four
// schedulers); the budget covers two whole 256-cell pencils (540 threads)
constexpr int MAXT_F64_X = 576;

// Thread budget of a tile: the limit on (C + 2*GH) * L.
inline int tile_budget(int prec, int dir)
{
    if (prec == PPMLR_MIXED) return MAXT;
    return prec == PPMLR_FP64 && dir == 0 ? MAXT_F64_X : MAXT_F64;
}

enum : int { FLAG_CFL = 1, FLAG_NONFINITE = 2, FLAG_TIMEOUT = 4, FLAG_BOUNDS = 8 };

// Arguments of one sweep launch (passed by value).
struct SweepArgs {
    const double *U;           // input state: array v at U + v * vs
    double *Un;                // output state: array v at Un + v * vs
    long long vs;              // element stride between the 8 arrays of a state
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
    int riemann_iters;         // 0: two-wave Riemann solver; k > 0: k two-shock Newton steps
    int steepen;               // 1: contact steepening of the remapped densities
    double dt;                 // used when dt_dev == nullptr
    const double *dt_dev;
    const double *bd;          // FP64 forms: dipole table (component k at bd + k * vs + cell) or null
    const double *iw, *ih;     // FP64 forms: 1 / width and 1 / (w_-/2 + w + w_+/2) along the axis, or null
    const unsigned char *inner_mask;   // per cell: 1 inside the inner sphere, or null
    // ionosphere shell on: sorted linear indices of the inner cells and their
    // conserved states (array v at inner_state + v * n_inner); null otherwise
    const long long *inner_cells;
    const double *inner_state;
    int n_inner;
    int *flags;
    unsigned long long *floors;
    // float copies for the mixed path (geometry and parameters)
    const float *wf;           // widths along the sweep axis, ghost-extended
    const float *cxf, *cyf, *czf;
    float gammaf, p_minf, Mf, r_innerf;
    float inflowf[8];
    // mixed path: the sweeps reconstruct and trace p - p_reff and form the
    // Riemann problem's total pressures relative to it (the scheme is
    // invariant under a constant pressure offset; float differences of
    // pressures near p_reff keep their digits).  0 for the FP64 forms.
    float p_reff;
};

// Pressure offset p_reff of the mixed sweeps: the inflow pressure when any
// face is an inflow face (the solar wind fills most of a magnetosphere
// domain), else 0 (the plain arithmetic).
inline float mixed_pressure_reference(const ppmlr_bc &bc)
{
    for (int d = 0; d < 3; d++)
        for (int s = 0; s < 2; s++)
            if (bc.face[d][s] == PPMLR_BC_INFLOW) return (float)bc.inflow.p;
    return 0.0f;
}

// Persistent ensemble sweep: per-instance arguments (input state = U, output
// = Un; flip = 1 swaps them), the first global tile of every instance and a
// work counter that must be zero at launch.
struct EnsSweepArgs {
    const SweepArgs *__restrict__ args;   // device array, one entry per instance (this direction)
    const int *first_tile;     // device array, count entries, ascending
    int count;
    int total_tiles;
    int flip;
    unsigned int *queue;
};

// Ensembles of up to ENS_PARAM_MAX instances also travel as one by-value
// kernel parameter (constant bank) for the one-block-per-tile launch form.
constexpr int ENS_PARAM_MAX = 64;
struct EnsSweepParams {
    SweepArgs args[ENS_PARAM_MAX];
    int first_tile[ENS_PARAM_MAX];
    int count;
    int flip;
    int total_tiles;           // persistent parameter form: tiles of all instances
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
    double *t_acc;             // device scalar or null: the last block adds dt (simulated time)
    const double *bd;          // FP64 forms: dipole table of the domain (component k at bd + k * bd_vs) or null
    long long bd_vs;
    const double *iw[3];       // contracted FP64 form: ghost-extended reciprocal widths, or null
    const unsigned char *inner_mask;   // per cell: 1 inside the inner sphere, or null
    // FP64 forms, two-pass step (null: one pass): per cell the float screen
    // bound written by the first pass, and the threshold it leaves (device)
    float *screen;
    float *screen_thr;
};

// Ionosphere shell (ionosphere.cu).  Static per cap node: the trilinear cell
// i0 (interior indices, 1 .. n-3) and weights of its mapping point at r_fac,
// B_d there, and factor = |B_d(foot)| / |B_d(point)| x B_r(foot) / |B_d(foot)|
// (0: the node's field line closes below r_fac).
struct IonoNode {
    int i0[3];
    double w[3];
    double Bd[3];
    double factor;
};
// Static per inner cell: for each axis d the potential stencils of its two
// neighbours along d, as 8 (node, coefficient) pairs giving E_d directly
// (node >= 0: index into the potential; -1 - cap: that cap's pole value;
// coefficients -w / span for the upper neighbour, +w / span for the lower),
// and bt = B_d / |B_d|^2 at the cell (v = E x bt).
struct IonoInner {
    int idx[3][8];
    double coef[3][8];
    double bt[3];
};
constexpr int IONO_MAX_NT = 256;      // rings per cap
// One ionosphere solve: state, geometry, tables and the device buffers it fills.
struct IonoArgs {
    const double *B[3];        // B' of the state (arrays 4..6)
    int n[3];
    const double *c[3];        // ghost-extended cell centres of each axis
    double r_iono, sigma_p;
    int nt, np;                // rings and longitudes per cap
    const IonoNode *nodes;     // 2 * nt * np
    double *jr;                // 2 * nt * np: radial current per cap node
    double *phi;               // 2 * nt * np: potential
    double *spec;              // 2 * nt * (np/2 + 1) * 2: Fourier coefficients
    double *pole;              // 2: ring-0 mean per cap
    const double *tw;          // np x (cos, sin) of 2 pi q / np
    const double *rows;        // nt x (lower, upper, diagonal without the longitude term, 1 / sin^2)
    const double *lam;         // np/2 + 1: (2 - 2 cos(2 pi m / np)) / dphi^2
    const IonoInner *inner;    // n_inner
    int n_inner;
    double *inner_state;       // 8 * n_inner
    double rho_in, p_in, gamma;
};
cudaError_t launch_ionosphere(const IonoArgs &a, cudaStream_t s, int *launches);
// selftest.cu: one block waits, with at most `polls` polls, on an mbarrier that
// nothing completes, then raises FLAG_TIMEOUT in *flags
cudaError_t launch_wait_selftest(int *flags, int polls, cudaStream_t s);

// Tile shape of one sweep direction.
struct Tile {
    int C, L, NP, nchunk, ngx, ntiles, threads;
    size_t smem;
};

// host helpers shared by the single-domain and ensemble code (api.cu)
void build_axis(int n, const double *edges, int bc_lo, int bc_hi, std::vector<double> &w, std::vector<double> &ce);
Tile choose_tile(int dir, const int n[3], size_t real_size);
Tile make_tile(int dir, const int n[3], size_t real_size, int C, int L);   // C cells per chunk, L lanes
bool validate_grid_bc(const ppmlr_grid *grid, const ppmlr_bc *bc);

// Launchers of one arithmetic variant (defined in the kernel translation
// units: sweep_fp64.cu, sweep_fp64_exact.cu, sweep_mixed.cu).
struct SweepLaunchers {
    cudaError_t (*single)(int dir, const SweepArgs &a, const Tile &t, cudaStream_t s);
    cudaError_t (*ens)(int dir, const EnsSweepArgs &e, int blocks, int threads, size_t smem, cudaStream_t s);
    cudaError_t (*param)(int dir, const EnsSweepParams &p, int blocks, int threads, size_t smem, cudaStream_t s);
    int (*per_sm)(int dir, int threads, size_t smem);
    // persistent y/z sweep with TMA-staged input boxes
    cudaError_t (*tma)(int dir, int persist, const SweepArgs &a, const CUtensorMap &map, int blocks, int threads,
                       size_t smem, cudaStream_t s);
    int (*tma_per_sm)(int dir, int persist, int threads, size_t smem);
    // dipole table of a single domain (null for the mixed path, which evaluates it in float)
    cudaError_t (*dipole_table)(double M, const int n[3], const double *cx, const double *cy, const double *cz,
                                double *bd, long long vs, cudaStream_t s);
    // ensemble y/z sweep, input boxes staged by TMA through per-instance tensor maps
    cudaError_t (*ens_tma)(int dir, const EnsSweepArgs &e, const CUtensorMap *maps, int blocks, int threads,
                           size_t smem, cudaStream_t s);
    int (*ens_tma_per_sm)(int dir, int threads, size_t smem);
    // ensemble, persistent blocks taking tiles from a work counter (zero at
    // launch), all instances' arguments in the kernel parameter
    cudaError_t (*param_persist)(int dir, const EnsSweepParams &p, unsigned int *queue, int blocks, int threads,
                                 size_t smem, cudaStream_t s);
    int (*param_persist_per_sm)(int dir, int threads, size_t smem);
    // ensemble, one block per tile, input box staged by TMA, all instances'
    // arguments in the kernel parameter
    cudaError_t (*ens_tma_param)(int dir, const EnsSweepParams &p, const CUtensorMap *maps, int blocks,
                                 int threads, size_t smem, cudaStream_t s);
    int (*ens_tma_param_per_sm)(int dir, int threads, size_t smem);
    // marching form (one thread per pencil; PPMLR_MIXED only, else cudaErrorNotSupported):
    // `a` carries the chunk length C, nchunk and the lane groups ngx (of 32)
    cudaError_t (*march)(int dir, const SweepArgs &a, cudaStream_t s);
};

// cuTensorMapEncodeTiled from the driver (null if unavailable)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn tensor_map_encoder();
// bytes of a tile's staged input box along direction d, padded to 1 KB (the
// exchange arrays follow it); x boxes hold NP + 2 cells per lane row
inline size_t stage_pad_bytes(const Tile &t, int d = 1)
{
    const size_t rows = (size_t)(d == 0 ? t.NP + 2 : t.NP) * t.L;
    return (8 * rows * sizeof(double) + 1023) / 1024 * 1024;
}
extern const SweepLaunchers k_sweep_fp64, k_sweep_fp64_exact, k_sweep_mixed;
inline const SweepLaunchers &sweep_launchers(ppmlr_precision p)
{
    return p == PPMLR_MIXED ? k_sweep_mixed : p == PPMLR_FP64_EXACT ? k_sweep_fp64_exact : k_sweep_fp64;
}

// Ensemble CFL: block b belongs to the last instance i with first_block[i] <= b.
struct EnsCflArgs {
    const CflArgs *args;       // device array, one entry per instance
    const int *first_block;
    int count;
};
struct CflLaunchers {
    cudaError_t (*single)(const CflArgs &a, int blocks, cudaStream_t s);
    cudaError_t (*ens)(const EnsCflArgs &e, int blocks, cudaStream_t s);
};
extern const CflLaunchers k_cfl_fp64, k_cfl_fp64_exact, k_cfl_mixed;
inline const CflLaunchers &cfl_launchers(ppmlr_precision p)
{
    return p == PPMLR_MIXED ? k_cfl_mixed : p == PPMLR_FP64_EXACT ? k_cfl_fp64_exact : k_cfl_fp64;
}
int cfl_threads();

}  // namespace ppmlr
