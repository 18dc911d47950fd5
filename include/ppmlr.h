/*
 * ppmlr.h -- C ABI of the GB300 (sm_103a) split-sweep PPMLR-MHD library.
 *
 * The library advances the ideal-MHD system in B' form of Guo et al.,
 * "Large Scale GPU Accelerated PPMLR-MHD Simulations for Space Weather
 * Forecast" (arXiv:1607.02214): conservation laws for rho, rho v, B' = B - B_d
 * and E with the dipole-coupling terms on the right-hand side, closure
 * E = p/(gamma-1) + rho v^2/2 + B'^2/2 (Sec. II, mu0 = 1 in code units).  One
 * step is three directionally split 1D sweeps (Sec. III-A), each a PPM
 * reconstruction, a characteristic Lagrangian step and a remap to the Eulerian
 * grid (Sec. II), with the solar-wind inflow, outflow, inner-boundary and
 * dipole treatment of Secs. II and IV-A.
 *
 * Conventions for every call:
 *   - Status codes: every call returns a ppmlr_status; ppmlr_last_error() gives
 *     the text of the last failure on that context.  Device-side conditions
 *     (non-finite state, CFL violation) are raised by kernels into a device
 *     flag word and reported by the next synchronising call (ppmlr_cfl_dt,
 *     ppmlr_get_state, ppmlr_check).  Kernels never trap and never spin.
 *   - State layout: 8 arrays of nx*ny*nz doubles, x fastest then y then z, in
 *     the order rho, m_x, m_y, m_z, B'_x, B'_y, B'_z, E (interior cells only;
 *     no ghost cells are stored).  Callers' arrays are only copied.
 *   - Ownership: the context owns all the device memory it allocates
 *     (ppmlr_create) and frees it in ppmlr_destroy.  Pointers passed in remain
 *     the caller's.
 *   - Streams: all work of a context is issued on its CUDA stream (the one
 *     given at create time or by ppmlr_set_stream; NULL = legacy default).
 */
#ifndef PPMLR_H
#define PPMLR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PPMLR_OK = 0,
    PPMLR_E_INVALID = 1,    /* bad argument (NULL, size, enum, non-positive width ...) */
    PPMLR_E_CUDA = 2,       /* a CUDA runtime call failed */
    PPMLR_E_OOM = 3,        /* device allocation failed */
    PPMLR_E_NONFINITE = 4,  /* a sweep produced a non-finite conserved value */
    PPMLR_E_CFL = 5,        /* dt too large: a Lagrangian width <= 0 or a remap sliver >= one zone */
    PPMLR_E_TIMEOUT = 6,    /* a bounded device wait (TMA copy completion) gave up */
    PPMLR_E_BOUNDS = 7      /* checked build (-DPPMLR_CHECK) only: a kernel index left its array */
} ppmlr_status;

typedef enum {
    PPMLR_FP64 = 0,         /* every stage in IEEE double; fused multiply-add and one reciprocal
                               per shared denominator; products, reciprocals and square roots
                               partly on the integer pipes, each correctly rounded (subnormals
                               flush to zero); agrees with the CPU reference to roundoff */
    PPMLR_MIXED = 1,        /* FP32 reconstruction, Riemann, remap and sources; pressure recovered
                               in double-float arithmetic; FP64 state accumulation */
    PPMLR_FP64_EXACT = 2    /* every stage in IEEE double with the CPU reference's expression
                               trees and no contraction: bit-identical to it */
} ppmlr_precision;

typedef enum { PPMLR_BC_PERIODIC = 0, PPMLR_BC_OUTFLOW = 1, PPMLR_BC_INFLOW = 2 } ppmlr_bc_kind;

/* Grid: n[d] cells along axis d (x, y, z); edges[d] points to n[d]+1 strictly
 * ascending cell edges in host memory (copied at create time).  A stretched
 * Cartesian grid as in Sec. III-B is given by its edges. */
typedef struct {
    int n[3];
    const double *edges[3];
} ppmlr_grid;

/* Primitive state: density, velocity, TOTAL magnetic field B, thermal pressure. */
typedef struct {
    double rho, v[3], B[3], p;
} ppmlr_prim;

/* Boundary specification (Secs. II and IV-A):
 *   face[axis][0|1]: kind of the low/high face of each axis.  PERIODIC wraps
 *     (both faces of an axis must then be periodic); OUTFLOW copies the edge
 *     cell; INFLOW imposes `inflow` with B' = inflow.B - B_d(ghost centre).
 *     Ghost widths wrap on periodic faces and mirror the edge cells otherwise.
 *   dipole_moment: M = B_E R_E^3 in code units, moment along -z (GSM, zero
 *     tilt): B_d = M [3 (m.r) r - m r^2] / r^5, m = -z.  0 disables B_d and
 *     its source terms.
 *   r_inner, inner: cells with centre radius < r_inner are reset after every
 *     sweep to rho = inner.rho, v = inner.v, p = inner.p and B' = 0 (inner.B is
 *     ignored).  r_inner <= 0 disables the inner sphere.
 *   p_min: pressure floor applied when recovering p from E; every use is
 *     counted (ppmlr_get_diagnostics).
 *   powell: 1 adds the -v div B' term of the induction equation. */
typedef struct {
    int face[3][2];
    ppmlr_prim inflow;
    double dipole_moment;
    double r_inner;
    ppmlr_prim inner;
    double p_min;
    int powell;
} ppmlr_bc;

typedef struct ppmlr_ctx ppmlr_ctx;

/* Create a context on the current CUDA device: copies the grid, builds the
 * ghost-extended geometry, allocates the state (2 x 8 arrays) and scratch.
 * gamma > 1.  cuda_stream: a cudaStream_t (NULL = default stream).
 * Errors: PPMLR_E_INVALID (NULL pointers, n < 1, non-ascending edges, bad
 * face kinds, periodic on one face only), PPMLR_E_OOM, PPMLR_E_CUDA.  On
 * failure *out is set to NULL. */
ppmlr_status ppmlr_create(const ppmlr_grid *grid, double gamma, const ppmlr_bc *bc,
                          ppmlr_precision prec, void *cuda_stream, ppmlr_ctx **out);

/* Replace the stream used for all later work of the context. */
ppmlr_status ppmlr_set_stream(ppmlr_ctx *ctx, void *cuda_stream);

/* Copy a state in (U[v] = 8 arrays of nx*ny*nz doubles, layout above).
 * on_device = 1: device pointers (copied on the context stream, asynchronous);
 * 0: host pointers (the call returns once the copy is done).  Resets the
 * device flag word. */
ppmlr_status ppmlr_set_state(ppmlr_ctx *ctx, const double *const U[8], int on_device);

/* Copy the state out (same layout).  Synchronises the context stream and
 * reports pending device flags (PPMLR_E_NONFINITE / PPMLR_E_CFL) after the
 * copy has completed. */
ppmlr_status ppmlr_get_state(ppmlr_ctx *ctx, double *const U[8], int on_device);

/* Layers k0 .. k0+nk-1 along z (the slowest axis) of the state: copied out of
 * (get) or into (set) the context; U: 8 arrays of nk * n[1] * n[0] doubles
 * (x fastest), host or device memory (on_device), caller-owned.  For a
 * domain split along z across ranks (block decomposition, the paper's own
 * scaling axis, Secs. III-A and III-B): each rank's context holds its slab
 * plus 7 halo layers (the stencil radius of one sweep) toward each
 * neighbour, and the halos are refreshed from the neighbours' owned layers
 * after every z sweep.  Stream-ordered on the context's stream; host copies
 * synchronise it.  PPMLR_E_INVALID for k0 < 0, nk < 0, k0 + nk > n[2] or a
 * NULL array. */
ppmlr_status ppmlr_get_layers(ppmlr_ctx *ctx, int k0, int nk, double *const U[8], int on_device);
ppmlr_status ppmlr_set_layers(ppmlr_ctx *ctx, int k0, int nk, const double *const U[8], int on_device);

/* CFL time step (reading of the paper, which states none):
 *   dt = cfl * min over non-inner interior cells and axes d of
 *        dx_d / (|v_d| + max(c_f,d(B'), c_f,d(B' + B_d))).
 * Computed on the device by a block-min reduction (no float atomics) and
 * copied to *dt_out (synchronises).  The FP64 forms take two passes: a float
 * screen bounds every cell, then the form's own FP64 expressions evaluate
 * only the cells within 1 % of the smallest float bound (and any whose float
 * bound is not a positive finite number), which always include the cell of
 * the minimum: the same dt bit for bit as one FP64 pass over every cell, at
 * the cost of a float pass.  The value also stays on the device for
 * ppmlr_step_cfl.  Reports pending device flags. */
ppmlr_status ppmlr_cfl_dt(ppmlr_ctx *ctx, double cfl, double *dt_out);

/* One full step with the given dt: three sweeps, x,y,z on even steps and
 * z,y,x on odd steps (Strang-type alternation; the paper does not state the
 * order).  Asynchronous: device flags are reported by the next synchronising
 * call.  dt must be finite and > 0 (else PPMLR_E_INVALID). */
ppmlr_status ppmlr_step(ppmlr_ctx *ctx, double dt);

/* nsteps steps, each with its dt computed on the device from the state at
 * the start of that step (as ppmlr_cfl_dt with `cfl`), with no host
 * synchronisation.  Asynchronous. */
ppmlr_status ppmlr_step_cfl(ppmlr_ctx *ctx, double cfl, int nsteps);

/* A single sweep along `axis` (0, 1, 2) with the given dt; does not advance
 * the step counter.  For testing a sweep in isolation. */
ppmlr_status ppmlr_sweep(ppmlr_ctx *ctx, int axis, double dt);

/* Synchronise the context stream and report pending device flags. */
ppmlr_status ppmlr_check(ppmlr_ctx *ctx);

/* Diagnostics (synchronises): steps taken, pressure-floor uses so far
 * (summed over sweeps), parity of the next step's sweep order (0: x,y,z). */
ppmlr_status ppmlr_get_diagnostics(ppmlr_ctx *ctx, long long *step, long long *floor_hits, int *order_parity);

/* Restore the step counter (checkpoint/resume: the state plus this counter
 * reproduce a run bit for bit). */
ppmlr_status ppmlr_set_step_count(ppmlr_ctx *ctx, long long step);

/* dt of the most recent ppmlr_cfl_dt / ppmlr_step_cfl step (synchronises). */
ppmlr_status ppmlr_get_dt(ppmlr_ctx *ctx, double *dt_out);

/* Text of the last error on this context ("" if none; static string for a
 * NULL context). */
const char *ppmlr_last_error(const ppmlr_ctx *ctx);

/* Free everything the context owns.  NULL is ignored. */
void ppmlr_destroy(ppmlr_ctx *ctx);

/* Kernel launches issued by this context so far (all kinds). */
long long ppmlr_launch_count(const ppmlr_ctx *ctx);

/* Per-kernel timing.  While enabled, CUDA events are recorded on the context
 * stream immediately before and after every kernel the context launches
 * (no synchronisation is added).  ppmlr_read_timing synchronises, returns the
 * summed device time in milliseconds and the launch count per kind since the
 * last read, and clears the records.  Kinds: 0, 1, 2 = x, y, z sweep;
 * 3 = CFL reduction.  total_ms and launches point to 4 entries each. */
ppmlr_status ppmlr_enable_timing(ppmlr_ctx *ctx, int on);
ppmlr_status ppmlr_read_timing(ppmlr_ctx *ctx, double *total_ms, long long *launches);

/* Tile-shape autotuner of one context: for each sweep direction, times a set
 * of candidate tile shapes (chunk length along the sweep axis x lanes per
 * tile) on the current state, out of place (the state is unchanged), and keeps
 * the fastest.  Results do not depend on the tile shape, only the speed does.
 * Shapes are cached per process by (direction, grid, precision), so a second
 * context of the same shape reuses them without timing.  best_ms (3 entries,
 * may be NULL) receives the tuned sweep times.  Synchronises. */
ppmlr_status ppmlr_autotune(ppmlr_ctx *ctx, double *best_ms);

/* Tile shape in use per direction: C (cells per chunk) and L (lanes);
 * C and L point to 3 entries each.  A direction in the marching form (3)
 * reports its chunk length and L = 32 (pencils per warp). */
ppmlr_status ppmlr_get_tiles(ppmlr_ctx *ctx, int *C, int *L);

/* Chunk length of the marching form along one axis (1 <= C <= n[axis];
 * default n[axis], whole pencils): each warp walks C output cells of 32
 * pencils and reads C + 14 input cells.  Results do not depend on it.
 * PPMLR_E_INVALID (state unchanged) outside those bounds. */
ppmlr_status ppmlr_set_march_chunk(ppmlr_ctx *ctx, int axis, int C);

/* Force the tile shape of one direction (axis 0, 1, 2): C cells per chunk
 * (1 <= C <= n[axis]) and L lanes (L >= 1) with (C + 14) * L within the
 * thread budget (512 for PPMLR_MIXED; 448 for the FP64 forms, except 576
 * for the x sweep of PPMLR_FP64).  Resets that
 * direction's launch form to 0.  Results do not depend on the shape.  Returns
 * PPMLR_E_INVALID (state unchanged) for shapes outside those bounds. */
ppmlr_status ppmlr_set_tiles(ppmlr_ctx *ctx, int axis, int C, int L);

/* Riemann solver of the sweeps.  iters = 0 (default): the linearised
 * two-wave solver (total pressure, fast impedance rho c_f; Alfven subsystem
 * with impedance sqrt(rho) |B_n|).  iters = 1..16: the nonlinear variant --
 * the two-shock solver of Colella & Woodward (1984), which the paper cites
 * for its scheme (Sec. II), on the fast mode: each side's wave is a shock
 * with Lagrangian speed W(P) = rho c_f sqrt(1 + (gamma+1)/(2 gamma)
 * (P/P_s - 1)) in the total pressure P; `iters` Newton steps from the
 * two-wave P* (4 reach the exact two-shock solution to roundoff for strong
 * shocks).  The Alfven subsystem stays linear.  Same arithmetic forms as the
 * rest of the sweep (PPMLR_FP64_EXACT: the reference's expressions).
 * PPMLR_E_INVALID outside [0, 16]. */
ppmlr_status ppmlr_set_riemann_solver(ppmlr_ctx *ctx, int iters);

/* Contact steepening (on = 1; default 0): the discontinuity detection of
 * Colella & Woodward (1984), which the paper cites for its scheme, applied in
 * the remap.  A zone whose Lagrangian density has second differences of
 * opposite sign on its two sides, a jump above 1 % of the smaller neighbour
 * and no shock (gamma 0.1 |dP|/P_min < |d rho|/rho_min on the sweep input,
 * P the total pressure) gets a weight eta in [0, 1] (20 (eta~ - 0.05)); the
 * parabola ends of all seven remapped densities move by eta towards the
 * neighbours' one-sided values a_{i-1} + slope/2 and a_{i+1} - slope/2.  One
 * weight for all densities keeps pressure and velocity uniform across an
 * advected contact. */
ppmlr_status ppmlr_set_steepening(ppmlr_ctx *ctx, int on);

/* Failure-path self-test of the kernels' bounded waits: launches one block
 * that waits, with the wait helper of the TMA-staged sweeps (here bounded at
 * 4096 polls), on an mbarrier that nothing completes; the wait gives up, the
 * block raises the timeout flag and returns.  The next synchronising call
 * (ppmlr_check, ppmlr_get_state, ppmlr_cfl_dt) returns PPMLR_E_TIMEOUT once;
 * the context stays usable.  No paper counterpart. */
ppmlr_status ppmlr_selftest_wait_timeout(ppmlr_ctx *ctx);

/* Ionosphere shell (Sec. II): a thin conducting sphere at r_iono closes the
 * field-aligned currents and is tied to the inner boundary by dipole field
 * lines; its electrostatic potential sets the flow of the inner-sphere cells.
 * Once per step, before the step's sweeps and from the state at the start of
 * the step:
 *   1. J = curl B' at the cell centres (centred differences), sampled with
 *      B' at the mapping sphere r_fac by trilinear interpolation along the
 *      dipole field lines of the shell nodes; J_par = J.B/|B|, B = B' + B_d;
 *   2. down the flux tube J_par scales with |B_d|; the shell takes the radial
 *      part J_r = J_par(r_iono) B_r/|B| (0 where the line closes below r_fac);
 *   3. Sigma_P Laplacian Phi = J_r on each polar cap 0 <= theta <= theta_max
 *      (theta from the cap's own pole, sin^2 theta_max = r_iono / r_inner),
 *      Phi = 0 at theta_max; cell-centred (n_theta x n_phi) grid, conservative
 *      five-point spherical Laplacian, solved exactly (Fourier in longitude,
 *      tridiagonal in colatitude);
 *   4. Phi carried along the field lines to the neighbours of every inner
 *      cell (bilinear on the caps, ring mean at the pole, 0 off the caps),
 *      E = -grad Phi by centred differences, v = E x B_d / |B_d|^2;
 *   5. every inner cell is reset to (inner rho, rho v, B' = 0,
 *      p_inner/(gamma-1) + rho v^2/2) instead of the configuration's rest
 *      state.
 * The calculation is in FP64 for every precision.  Units: Sigma_P in code
 * units (mu0 v0 Sigma_SI); radii in R_E. */
typedef struct {
    double r_iono;                   /* shell radius, 0 < r_iono < r_inner */
    double r_fac;                    /* current-mapping radius, r_fac > r_iono */
    double sigma_p;                  /* Pedersen conductance (code units), > 0 */
    int n_theta;                     /* colatitude rings per cap, 2..256 */
    int n_phi;                       /* longitudes, even, 4..1024 */
} ppmlr_iono;
/* Turns the shell on (cfg copied) or off (cfg = NULL: the inner cells return
 * to the configuration's fixed state at the next sweep).  Needs r_inner > 0,
 * a dipole, and the mapping sphere one cell inside the interior of every axis
 * (the centres of cells 1 and n-2 bracket [-r_fac, r_fac]).  Allocates per
 * cap node about 4 doubles (current, potential, Fourier coefficients) and a
 * 72-byte table entry, per inner cell 8 doubles and a 312-byte stencil entry,
 * plus the solve tables (2 n_phi + 4 n_theta + n_phi/2 + 1 doubles); drops
 * the step graphs.  Device-dt steps run the solve beside the CFL reduction
 * on a second stream.  Until the first solve (a step, or
 * ppmlr_ionosphere_solve) the inner cells keep the configuration's fixed
 * state, so a lone ppmlr_sweep resets them as without the shell.
 * PPMLR_E_INVALID (shell unchanged) otherwise, PPMLR_E_OOM on allocation
 * failure. */
ppmlr_status ppmlr_set_ionosphere(ppmlr_ctx *ctx, const ppmlr_iono *cfg);
/* One ionosphere solve from the current state (what every step does first
 * while the shell is on), on the context's stream.  PPMLR_E_INVALID when the
 * shell is off. */
ppmlr_status ppmlr_ionosphere_solve(ppmlr_ctx *ctx);
/* Copies the last solve's potential and radial current to host arrays of
 * 2 * n_theta * n_phi doubles (cap-major: north then south, ring-major,
 * longitude fastest); either pointer may be NULL.  Synchronises the stream.
 * PPMLR_E_INVALID when the shell is off. */
ppmlr_status ppmlr_get_ionosphere(ppmlr_ctx *ctx, double *phi, double *jr);

/* Launch form of each sweep direction (3 entries): 0 = one block per tile
 * reading its input from global memory; 1 = persistent blocks whose input
 * boxes (8 arrays x positions x lanes) are staged into shared memory by the
 * tensor memory accelerator, double-buffered so the next tile's copy overlaps
 * the current tile's arithmetic; 2 = one block per tile with its input box
 * staged by the tensor memory accelerator.  Forms 1 and 2 apply to the y and
 * z sweeps with an even number of lanes, nx even and at most 256 positions
 * per tile; 3 = the marching form of PPMLR_MIXED: one thread per pencil
 * walking it cell by cell, every stage of the scheme on the newest zone whose
 * inputs are complete, neighbour values in register windows (no
 * shared-memory exchange, no barriers), 32 pencils per warp; a context with
 * contact steepening on runs the tile form 0 in its place.  The autotuner
 * chooses the form with the tile shape; results do not depend on it beyond
 * roundoff on the contracted paths. */
ppmlr_status ppmlr_get_sweep_forms(ppmlr_ctx *ctx, int *form);
/* Select a launch form for one axis (PPMLR_E_INVALID if not available). */
ppmlr_status ppmlr_set_sweep_form(ppmlr_ctx *ctx, int axis, int form);

/* ---- Long runs: graph replay, simulated time, checkpoints -----------------
 * The paper's production use is a magnetosphere driven to a steady state
 * over many steps, run faster than real time (Secs. I and IV-A); none of the
 * calls below changes the arithmetic of a step. */

/* nsteps steps exactly as ppmlr_step_cfl (same dt, same results bit for
 * bit), replayed from CUDA graphs of graph_steps steps each (a CFL pass and
 * three sweeps per step; graph_steps even, 2..4096), with any remainder
 * launched directly; graph_steps = 0 launches every kernel directly.  Graphs
 * are captured on first use for the current step parity, input buffer,
 * length and cfl, kept by the context and dropped when the tile shapes or
 * launch forms change.  Asynchronous.  PPMLR_E_INVALID for cfl <= 0,
 * nsteps < 0 or an odd or out-of-range graph_steps. */
ppmlr_status ppmlr_run(ppmlr_ctx *ctx, double cfl, long long nsteps, int graph_steps);

/* Simulated time in code units (R_E / v0 with v0 = 100 km/s: 63.712 s): the
 * FP64 sum of the dt of every step since creation or the last
 * ppmlr_set_time / ppmlr_checkpoint_load.  Device-dt steps (ppmlr_step_cfl,
 * ppmlr_run) add on the device; ppmlr_step adds its dt on the host.
 * Synchronises. */
ppmlr_status ppmlr_get_time(ppmlr_ctx *ctx, double *t_out);
ppmlr_status ppmlr_set_time(ppmlr_ctx *ctx, double t);

/* Checkpoint of the state, step counter and simulated time.  File layout
 * (little-endian): a 56-byte header -- magic "PPMLRCK1", u32 version (1),
 * u32 precision, i32 n[3], i32 0, i64 step, f64 time, f64 gamma -- then the
 * grid edges of x, y, z (n[d] + 1 doubles each), the 8 conserved arrays
 * (n0*n1*n2 doubles each, x fastest; rho, m_x, m_y, m_z, B'_x, B'_y, B'_z,
 * E) and a u64 checksum: FNV-1a (offset 0xcbf29ce484222325, prime
 * 0x100000001b3) over all preceding bytes taken as 64-bit words.
 * ppmlr_checkpoint_save synchronises, writes `path`.part and renames it to
 * `path` (PPMLR_E_INVALID if the file cannot be written); it then reports
 * pending device flags.  ppmlr_checkpoint_load verifies the whole file
 * (magic, version, checksum, grid size, edges bit for bit and gamma against
 * the context's) before it replaces the state, step counter and simulated
 * time; otherwise PPMLR_E_INVALID with the state unchanged.  A checkpoint of
 * any precision loads into a context of any precision (the state is FP64 in
 * every form; ppmlr_checkpoint_info reports the writer's precision).  If a
 * device copy fails while saving, no file (and no `path`.part) is left.
 * Loading a checkpoint of step k and continuing reproduces an uninterrupted
 * run bit for bit (state and time). */
ppmlr_status ppmlr_checkpoint_save(ppmlr_ctx *ctx, const char *path);
ppmlr_status ppmlr_checkpoint_load(ppmlr_ctx *ctx, const char *path);
/* Host only (no device, no context): verify a checkpoint file and read its
 * header fields (any output pointer may be NULL).  PPMLR_E_INVALID if the
 * file is missing, truncated or corrupt. */
ppmlr_status ppmlr_checkpoint_info(const char *path, int n[3], long long *step, double *time, int *precision);

/* ---- Batched ensemble ----------------------------------------------------
 * count independent instances, each with its own grid and boundary
 * specification (e.g. different solar-wind and IMF inputs, uneven grid
 * sizes), advanced together: per step one device CFL pass giving every
 * instance its own dt, then one persistent launch per sweep direction whose
 * blocks take (instance, tile) work items from a global counter.  A step is
 * captured once as a CUDA graph (x,y,z and z,y,x variants) and replayed.
 * The results of every instance are bit-identical to a single context
 * advanced with ppmlr_step_cfl.  The ensemble owns all its device memory. */
typedef struct ppmlr_ens ppmlr_ens;

ppmlr_status ppmlr_ensemble_create(int count, const ppmlr_grid *grids, const ppmlr_bc *bcs, double gamma,
                                   ppmlr_precision prec, void *cuda_stream, ppmlr_ens **out);
ppmlr_status ppmlr_ensemble_set_stream(ppmlr_ens *ens, void *cuda_stream);
/* State of instance i (layout as for a context). */
ppmlr_status ppmlr_ensemble_set_state(ppmlr_ens *ens, int i, const double *const U[8], int on_device);
ppmlr_status ppmlr_ensemble_get_state(ppmlr_ens *ens, int i, double *const U[8], int on_device);
/* nsteps graph-replayed steps with per-instance device dt (asynchronous). */
ppmlr_status ppmlr_ensemble_step(ppmlr_ens *ens, double cfl, int nsteps);
/* The same steps with direct launches and CUDA events around every kernel;
 * avg_ms (4 entries) receives the mean time per launch of the x, y, z sweeps
 * and the CFL pass.  Synchronises. */
ppmlr_status ppmlr_ensemble_time_kernels(ppmlr_ens *ens, double cfl, int nsteps, double *avg_ms);
/* Tile-shape autotuner of the ensemble: per direction, the thread budget of
 * the tiles of all instances and the launch form (0: persistent blocks taking
 * tiles from a work counter; 1: one block per tile, arguments from a device
 * table; 2: one block per tile, arguments of all instances in the kernel
 * parameter, up to 64 instances; 3: one block per tile with the input box
 * staged by TMA; 4: persistent blocks taking tiles from a work counter,
 * arguments of all instances in the kernel parameter, up to 64 instances;
 * 5: one block per tile with the input box staged by TMA and the arguments
 * of all instances in the kernel parameter, up to 64 instances), timed out
 * of place; a persistent form (0 or 4) is kept when it is within 2 % of the
 * fastest; best_ms: 3 entries or NULL. */
ppmlr_status ppmlr_ensemble_autotune(ppmlr_ens *ens, double *best_ms);
/* Fix the launch of one sweep direction instead of autotuning it: form 0 =
 * persistent blocks taking tiles from a work counter, 1 = one block per tile
 * (arguments from a device table), 2 = one block per tile (arguments of all
 * instances in the kernel parameter; at most 64 instances), 3 = one block per
 * tile with the tile's input box staged by the tensor memory accelerator
 * through per-instance tensor maps (every instance needs nx even and at most
 * 256 positions per tile; along x also C even and ny a multiple of the
 * lanes), 4 = persistent blocks taking tiles from a work counter with the
 * arguments of all instances in the kernel parameter (at most 64
 * instances), 5 = one block per tile with the box staged as in form 3 and
 * the arguments of all instances in the kernel parameter (the conditions of
 * form 3; at most 64 instances); budget = positions x lanes per
 * tile (15..448 for the FP64 forms, ..512 for PPMLR_MIXED).  Tiles: whole
 * pencils when they fit (else equal chunks), then as many lanes as fit; for
 * y and z, budget + 10000 selects the other rule: the most lanes (a power of
 * two up to 16) for which chunks of at least min(n, 48) cells fit.  Drops the
 * step graphs.  PPMLR_E_INVALID (launch unchanged) when the form does not
 * fit. */
ppmlr_status ppmlr_ensemble_set_launch(ppmlr_ens *ens, int axis, int form, int budget);
/* Riemann solver of every instance's sweeps, as ppmlr_set_riemann_solver
 * (0: two-wave; 1..16: two-shock Newton steps on the fast mode).  Drops the
 * captured step graphs.  PPMLR_E_INVALID outside [0, 16]. */
ppmlr_status ppmlr_ensemble_set_riemann_solver(ppmlr_ens *ens, int iters);
/* Contact steepening of every instance's remap, as ppmlr_set_steepening.
 * Drops the captured step graphs. */
ppmlr_status ppmlr_ensemble_set_steepening(ppmlr_ens *ens, int on);
/* Launch form, tile rule and thread budget per direction in use:
 * 10000 * lanes_first + 1000 * form + budget (3 entries). */
ppmlr_status ppmlr_ensemble_get_tiles(ppmlr_ens *ens, int *maxt);
/* dt of the last step of every instance (count entries; synchronises). */
ppmlr_status ppmlr_ensemble_get_dt(ppmlr_ens *ens, double *dt_out);
ppmlr_status ppmlr_ensemble_check(ppmlr_ens *ens);
ppmlr_status ppmlr_ensemble_get_diagnostics(ppmlr_ens *ens, long long *step, long long *floor_hits);
const char *ppmlr_ensemble_last_error(const ppmlr_ens *ens);
long long ppmlr_ensemble_launch_count(const ppmlr_ens *ens);
void ppmlr_ensemble_destroy(ppmlr_ens *ens);

/* Arithmetic-pipe rates of the current GPU (measurement support, no paper
 * counterpart): instructions per second of FP64 fused multiply-add
 * (rates[0]), FP64 add (rates[1]) and FP32 fused multiply-add (rates[2]),
 * each from eight independent dependency chains per thread, 8 blocks of 256
 * threads per SM, timed with CUDA events on `cuda_stream` (NULL = default)
 * after a warm-up launch.  Allocates and frees a small output buffer;
 * synchronises the stream.  The FP64 rate x 2 flops is the peak of the FP64
 * sweeps' roofline.  Errors: PPMLR_E_INVALID (rates NULL), PPMLR_E_OOM,
 * PPMLR_E_CUDA. */
ppmlr_status ppmlr_measure_pipe_rates(void *cuda_stream, double rates[3]);

/* Co-issue of the PPMLR_FP64 form's integer-pipe double product with the
 * FP64 pipe (no paper counterpart): rates[0] products per second of that
 * product alone (eight independent chains per thread, as above), rates[1]
 * operations per second of four FP64 FMA chains beside four product chains
 * per thread -- above rates[0] and above the FP64 FMA rate of
 * ppmlr_measure_pipe_rates when the two pipes issue side by side.  Runs on
 * `cuda_stream` (NULL = default), allocates and frees one scratch buffer,
 * synchronises the stream.  Errors: PPMLR_E_INVALID (rates NULL),
 * PPMLR_E_OOM, PPMLR_E_CUDA. */
ppmlr_status ppmlr_measure_coissue(void *cuda_stream, double rates[2]);

/* Self-test of the PPMLR_FP64 form's own square root, reciprocal and
 * product (integer and FP32 arithmetic, each correctly rounded); no paper
 * counterpart.  Over n >= 1 arguments (1 + f) 2^e, e cycling over
 * -1000..1000, every fourth one an exact square moved by -3..3 units in its
 * last place instead: max_ulp[0] and max_ulp[1] the largest errors of the
 * square root and the reciprocal in ulps of the correctly rounded result
 * (both 0 for the form's accuracy claim), max_ulp[2] the count of
 * square roots that differ from the correctly rounded ones (0), max_ulp[3]
 * the count of n products of normal doubles with normal results (a quarter
 * of them built to round a tie) that differ from the IEEE product (0).
 * Runs on `cuda_stream` (NULL = default), allocates and frees 32 bytes,
 * synchronises the stream.  Errors: PPMLR_E_INVALID (max_ulp NULL or
 * n < 1), PPMLR_E_OOM, PPMLR_E_CUDA. */
ppmlr_status ppmlr_selftest_fp64_arith(void *cuda_stream, long long n, double max_ulp[4]);

/* Allocation-free CFL time step.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory -- a host
 * solver whose device memory belongs to another allocator that forbids raw
 * cudaMalloc, a coupling loop that cannot afford the device synchronisation
 * an allocation may cause, or a program with a fixed device-memory budget.
 * It needs no context: every input and the output are caller-owned device
 * memory, and it performs no cudaMalloc, cudaFree or other allocation.
 *   U: 8 device arrays of the state (layout above); n: cells per axis;
 *   width[d], centre[d]: device arrays of the n[d] cell widths and centres of
 *   each axis (no ghost cells); gamma, p_min, dipole_moment, r_inner: as in
 *   ppmlr_bc; cfl > 0; blocks: reduction blocks, 0 = automatic, at most 1024
 *   (the size of the static scratch; larger values return PPMLR_E_INVALID);
 *   dt_out: device pointer that receives dt; cuda_stream: stream (NULL =
 *   default).  Asynchronous.  The formula of ppmlr_cfl_dt in the exact double
 *   arithmetic of the CPU reference: the dt equals that of a
 *   PPMLR_FP64_EXACT context bit for bit, and that of a PPMLR_FP64 context
 *   (contracted arithmetic) to roundoff.
 * Scratch: a static device array of 1056 doubles (8.4 KB) that every GPU that
 * loads the library holds until the process exits.  All calls on a device
 * share it and it keeps the last call's contents (its ticket counter is
 * cleared at the start of each call); calls whose kernels overlap on the GPU
 * race on it and must be serialised by the caller.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) and
 * caches it with the unique ID of the current CUDA context; a call under a
 * different context of the device (after cudaDeviceReset, say) looks it up
 * again.  Make the first call on a device before capturing any stream work.
 * Errors: PPMLR_E_INVALID (NULL pointer, n < 1, too many cells or blocks,
 * gamma <= 1, cfl <= 0), PPMLR_E_CUDA. */
ppmlr_status ppmlr_cfl_dt_noalloc(const double *const U[8], const int n[3], const double *const width[3],
                                  const double *const centre[3], double gamma, double p_min, double dipole_moment,
                                  double r_inner, double cfl, int blocks, double *dt_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* PPMLR_H */
