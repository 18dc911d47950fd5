// Host side of the C ABI declared in include/ppmlr.h: context lifetime,
// ghost-extended geometry, state copies, sweep/step/CFL launches and the
// device status word.  Built with -ffp-contract=off so that the geometry is
// computed with the same IEEE double operations as the CPU reference.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "ppmlr_internal.h"

using namespace ppmlr;

struct ppmlr_ctx {
    int n[3];
    long long ncell;
    double gamma;
    ppmlr_bc bc;
    ppmlr_precision prec;
    cudaStream_t stream;
    int device;
    double *state;               // 16 arrays: U (8) then Unew (8), each padded
    size_t stride;               // elements between arrays
    double *U[8], *Un[8];
    double *geo;                 // w[3], c[3], 1/w[3], 1/h[3]
    double *w[3], *c[3], *iw[3], *ih[3];
    unsigned char *inner_mask;   // per cell: centre inside the inner sphere (r_inner > 0), else null
    float *geof;                 // float copies of w[3], c[3] (mixed path)
    float *wf[3], *cf[3];
    int *flags;
    unsigned long long *floors;
    double *dt_dev;
    double *bd;                  // FP64 forms with a dipole: B_d at every cell (3 arrays, stride `stride`)
    float *screen;               // FP64 forms: the CFL screen (one float per cell, then the threshold)
    double *partial;
    unsigned int *counter;
    int cfl_blocks;
    Tile tile[3];
    int mode[3];                 // 0: one block per tile; 1: persistent, TMA-staged input (y, z);
                                 // 2: one block per tile, TMA-staged input (y, z);
                                 // 3: marching form (one thread per pencil; mixed path)
    int march_C[3];              // marching form: output cells per chunk along each axis
    CUtensorMap tmap[3][2];      // per direction, per state buffer (input = buffer 0 or 1)
    int tma_blocks[3];
    size_t tma_smem[3];
    int sms;
    long long steps;
    long long launches;
    std::string err;
    // simulated time: device accumulator (dt_dev[1], steps with a device dt)
    // plus the explicit dt of ppmlr_step, summed on the host
    double t_host;
    int riemann_iters;              // 0: two-wave Riemann solver; k > 0: k two-shock Newton steps
    int steepen;                    // 1: contact steepening in the remap
    std::vector<double> edges[3];   // host copies of the grid edges (checkpoint validation)
    // graph replay of ppmlr_run: one executable graph per starting step
    // parity, input buffer, length and CFL number; dropped when the tiles or
    // launch forms change
    cudaStream_t cap;
    // with the ionosphere shell on, device-dt steps run the shell's solve on
    // `side` concurrently with the CFL pass (fork / join events)
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
    struct Graph { int parity, buf, ksteps; double cfl; cudaGraphExec_t exec; long long launches; };
    std::vector<Graph> graphs;
    // per-kernel timing records (kind, start, stop) and a pool of spare events
    bool timing;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    // ionosphere shell: the inner cells (ascending linear index, from the
    // inner mask) and, while the shell is on, its configuration and buffers
    std::vector<long long> inner_list;
    struct Iono {
        bool on;
        ppmlr_iono cfg;
        double *buf;                // jr, phi, spectra, poles, solve tables (IonoLayout)
        IonoNode *nodes;            // per cap node
        IonoInner *inner;           // per inner cell
        long long *cells;           // inner_list on the device
        double *state;              // 8 x inner_list.size()
    } iono;
};

static cudaEvent_t take_event(ppmlr_ctx *c)
{
    if (!c->pool.empty()) { cudaEvent_t e = c->pool.back(); c->pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Records the start event of a timed launch; returns the record index or -1.
static int timing_begin(ppmlr_ctx *c, int kind)
{
    if (!c->timing) return -1;
    ppmlr_ctx::Rec r{kind, take_event(c), take_event(c)};
    if (!r.a || !r.b || cudaEventRecord(r.a, c->stream) != cudaSuccess) {
        if (r.a) c->pool.push_back(r.a);
        if (r.b) c->pool.push_back(r.b);
        return -1;
    }
    c->recs.push_back(r);
    return (int)c->recs.size() - 1;
}

static void timing_end(ppmlr_ctx *c, int idx)
{
    if (idx >= 0) cudaEventRecord(c->recs[idx].b, c->stream);
}

static const char *k_null_ctx = "null context";

static ppmlr_status fail(ppmlr_ctx *c, ppmlr_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

static ppmlr_status cuda_fail(ppmlr_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, e == cudaErrorMemoryAllocation ? PPMLR_E_OOM : PPMLR_E_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(c, call, what)                                \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

// Ghost-extended widths and centres of one axis (same rules and arithmetic as
// the CPU reference): periodic faces wrap, other faces mirror the edge widths
// (clamped to the axis); centres extend the grid by the ghost widths.
void ppmlr::build_axis(int n, const double *edges, int bc_lo, int bc_hi, std::vector<double> &w,
                       std::vector<double> &ce)
{
    w.assign(n + 2 * GH, 0.0);
    ce.assign(n + 2 * GH, 0.0);
    for (int i = 0; i < n; i++) w[GH + i] = edges[i + 1] - edges[i];
    for (int k = 1; k <= GH; k++) {
        int lo, hi;
        if (bc_lo == PPMLR_BC_PERIODIC) lo = ((-k) % n + n) % n;
        else { lo = k - 1; if (lo > n - 1) lo = n - 1; }
        if (bc_hi == PPMLR_BC_PERIODIC) hi = (k - 1) % n;
        else { hi = n - k; if (hi < 0) hi = 0; }
        w[GH - k] = w[GH + lo];
        w[GH + n - 1 + k] = w[GH + hi];
    }
    for (int i = 0; i < n; i++) ce[GH + i] = 0.5 * (edges[i] + edges[i + 1]);
    double e = edges[0];
    for (int k = 1; k <= GH; k++) { ce[GH - k] = e - 0.5 * w[GH - k]; e -= w[GH - k]; }
    e = edges[n];
    for (int k = 1; k <= GH; k++) { ce[GH + n - 1 + k] = e + 0.5 * w[GH + n - 1 + k]; e += w[GH + n - 1 + k]; }
}

// Tile shape for a sweep along an axis of N cells: whole pencils when they fit
// in MAXT positions, else equal chunks; as many lanes as fit (powers of two
// for the y/z sweeps, whose lanes are consecutive x cells).
Tile ppmlr::make_tile(int dir, const int n[3], size_t real_size, int C, int L)
{
    Tile t;
    const int N = n[dir];
    t.C = C < 1 ? 1 : (C > N ? N : C);
    t.nchunk = (N + t.C - 1) / t.C;
    t.NP = t.C + 2 * GH;
    if (L < 1) L = 1;
    if (dir == 0) {
        long long pencils = (long long)n[1] * n[2];
        if (L > pencils) L = (int)pencils;
        t.L = L;
        t.ngx = (int)((pencils + L - 1) / L);
        t.ntiles = t.ngx * t.nchunk;
    } else {
        t.L = L;
        t.ngx = (n[0] + t.L - 1) / t.L;
        int other = dir == 1 ? n[2] : n[1];
        t.ntiles = t.ngx * other * t.nchunk;
    }
    t.threads = ((t.NP * t.L + 31) / 32) * 32;
    t.smem = (size_t)NSMP * t.NP * t.L * real_size;
    return t;
}

// Default tile policy: whole pencils when they fit the thread budget, else
// equal chunks; as many lanes as fit (powers of two for the y/z sweeps, whose
// lanes are consecutive x cells).
Tile ppmlr::choose_tile(int dir, const int n[3], size_t real_size)
{
    const int N = n[dir];
    const int maxt = real_size == sizeof(double) ? MAXT_F64 : MAXT;
    int nchunk = 1, C = N;
    while (C + 2 * GH > maxt) {
        nchunk++;
        C = (N + nchunk - 1) / nchunk;
    }
    int L = maxt / (C + 2 * GH);
    if (L < 1) L = 1;
    if (dir != 0) {
        int p2 = 1;
        while (p2 * 2 <= L && p2 * 2 <= 16) p2 *= 2;
        while (p2 > 1 && p2 / 2 >= n[0]) p2 /= 2;
        L = p2;
    }
    return make_tile(dir, n, real_size, C, L);
}

bool ppmlr::validate_grid_bc(const ppmlr_grid *grid, const ppmlr_bc *bc)
{
    if (!grid || !bc) return false;
    for (int d = 0; d < 3; d++) {
        if (grid->n[d] < 1 || !grid->edges[d]) return false;
        for (int i = 0; i < grid->n[d]; i++)
            if (!(grid->edges[d][i + 1] > grid->edges[d][i])) return false;
        for (int s = 0; s < 2; s++)
            if (bc->face[d][s] < PPMLR_BC_PERIODIC || bc->face[d][s] > PPMLR_BC_INFLOW) return false;
        if ((bc->face[d][0] == PPMLR_BC_PERIODIC) != (bc->face[d][1] == PPMLR_BC_PERIODIC)) return false;
    }
    bool any_inflow = false;
    for (int d = 0; d < 3; d++) any_inflow |= bc->face[d][0] == PPMLR_BC_INFLOW || bc->face[d][1] == PPMLR_BC_INFLOW;
    if (!(bc->p_min >= 0.0)) return false;
    if (any_inflow && !(bc->inflow.rho > 0.0 && bc->inflow.p > 0.0)) return false;
    if (bc->r_inner > 0.0 && !(bc->inner.rho > 0.0 && bc->inner.p >= 0.0)) return false;
    long long ncell = (long long)grid->n[0] * grid->n[1] * grid->n[2];
    return ncell <= (1LL << 31) - 1;
}

static EncodeTiledFn encode_fn() { return tensor_map_encoder(); }

EncodeTiledFn ppmlr::tensor_map_encoder()
{
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {     // looked up once (thread-safe)
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (EncodeTiledFn)p;
        return nullptr;
    }();
    return fn;
}


// The TMA forms apply where the tile's box fits the copy engine's rules: rows
// 16-byte aligned (nx even) and every box dimension at most 256.  y/z sweeps:
// lanes (the x extent of the box) even.  x sweep (one tile per block only):
// C even so that the box's x origin g0 - 8 is even, and L pencils that lie in
// one z plane (ny a multiple of L).  The staging buffer(s) plus the exchange
// arrays must fit in shared memory.
static const char *tma_ineligible(const ppmlr_ctx *c, int d, const Tile &t, int form)
{
    if (!encode_fn()) return "cuTensorMapEncodeTiled is not available from the driver";
    if (c->n[0] & 1) return "the TMA form needs nx even (16-byte aligned rows)";
    if (t.threads > (c->prec == PPMLR_MIXED ? MAXT : MAXT_F64))
        return "the TMA kernels take at most 512 (mixed) or 448 (FP64) threads per tile";
    if (d == 0) {
        if (form != 2) return "the x sweep has only the one-tile TMA form (2)";
        if (t.C & 1) return "the x-sweep TMA form needs an even chunk length C";
        if (t.NP + 2 > 256) return "the x-sweep TMA form needs at most 254 positions per tile (C + 14)";
        if (c->n[1] % t.L) return "the x-sweep TMA form needs ny to be a multiple of the lanes L";
    } else {
        if (t.L < 2 || (t.L & 1)) return "the TMA form needs an even number of lanes";
        if (t.NP > 256) return "the TMA form needs at most 256 positions per tile (C + 14)";
    }
    const int persist = form == 1;
    const size_t smem = (persist ? 2 : 1) * stage_pad_bytes(t, d) + t.smem;
    if (smem > 226 * 1024) return "the TMA staging buffers do not fit in shared memory";   // 1 KB static
    if (sweep_launchers(c->prec).tma_per_sm(d, persist, t.threads, smem) < 1)
        return "the TMA kernel cannot be resident with this tile shape";
    return nullptr;
}
static bool tma_eligible(const ppmlr_ctx *c, int d, const Tile &t, int form)
{
    return tma_ineligible(c, d, t, form) == nullptr;
}

// Tensor maps of direction d for both state buffers: a 4D view (x, y, z,
// variable) of the 8 equally spaced arrays; box = L lanes x NP positions
// (x sweep: NP + 2 cells x L pencils).
// Returns nullptr on success, else the reason.
static const char *setup_tma_why(ppmlr_ctx *c, int d, int form)
{
    const Tile &t = c->tile[d];
    if (const char *why = tma_ineligible(c, d, t, form)) return why;
    const cuuint64_t dims[4] = {(cuuint64_t)c->n[0], (cuuint64_t)c->n[1], (cuuint64_t)c->n[2], 8};
    const cuuint64_t strides[3] = {(cuuint64_t)c->n[0] * 8, (cuuint64_t)c->n[0] * c->n[1] * 8,
                                   (cuuint64_t)c->stride * 8};
    cuuint32_t box[4] = {(cuuint32_t)t.L, 1, 1, 8};
    box[d] = (cuuint32_t)t.NP;
    if (d == 0) { box[0] = (cuuint32_t)(t.NP + 2); box[1] = (cuuint32_t)t.L; }   // L pencils of one z plane
    const cuuint32_t es[4] = {1, 1, 1, 1};
    for (int b = 0; b < 2; b++) {
        void *base = c->state + (size_t)b * 8 * c->stride;
        CUresult r = encode_fn()(&c->tmap[d][b], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, base, dims, strides, box, es,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return "cuTensorMapEncodeTiled rejected the state layout";
    }
    const int persist = form == 1;
    c->tma_smem[d] = (persist ? 2 : 1) * stage_pad_bytes(t, d) + t.smem;
    const int per_sm = sweep_launchers(c->prec).tma_per_sm(d, persist, t.threads, c->tma_smem[d]);
    const long long b = (long long)per_sm * c->sms;
    c->tma_blocks[d] = persist ? (int)(b < t.ntiles ? b : t.ntiles) : t.ntiles;
    return nullptr;
}
static bool setup_tma(ppmlr_ctx *c, int d, int form) { return setup_tma_why(c, d, form) == nullptr; }

static bool is_sweep_noop(const ppmlr_ctx *c, int d)
{
    return c->n[d] == 1 && c->bc.face[d][0] == PPMLR_BC_PERIODIC && c->bc.face[d][1] == PPMLR_BC_PERIODIC &&
           c->bc.dipole_moment == 0.0;
}

extern "C" {

ppmlr_status ppmlr_create(const ppmlr_grid *grid, double gamma, const ppmlr_bc *bc, ppmlr_precision prec,
                          void *cuda_stream, ppmlr_ctx **out)
{
    if (!out) return PPMLR_E_INVALID;
    *out = nullptr;
    if (!grid || !bc) return PPMLR_E_INVALID;
    if (!(gamma > 1.0) || (prec != PPMLR_FP64 && prec != PPMLR_MIXED && prec != PPMLR_FP64_EXACT))
        return PPMLR_E_INVALID;
    if (!validate_grid_bc(grid, bc)) return PPMLR_E_INVALID;
    long long ncell = (long long)grid->n[0] * grid->n[1] * grid->n[2];

    ppmlr_ctx *c = new ppmlr_ctx();
    memcpy(c->n, grid->n, sizeof(c->n));
    c->ncell = ncell;
    c->gamma = gamma;
    c->bc = *bc;
    c->prec = prec;
    c->stream = (cudaStream_t)cuda_stream;
    c->steps = 0;
    c->launches = 0;
    c->timing = false;
    c->t_host = 0.0;
    c->riemann_iters = 0;
    c->steepen = 0;
    c->cap = nullptr;
    for (int d = 0; d < 3; d++) c->edges[d].assign(grid->edges[d], grid->edges[d] + grid->n[d] + 1);
    if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return PPMLR_E_CUDA; }

    // state: 16 arrays, each padded to 256-byte multiples
    c->stride = ((size_t)ncell + 31) / 32 * 32;
    cudaError_t e = cudaMalloc(&c->state, sizeof(double) * c->stride * 16);
    if (e != cudaSuccess) { delete c; return e == cudaErrorMemoryAllocation ? PPMLR_E_OOM : PPMLR_E_CUDA; }
    for (int v = 0; v < 8; v++) { c->U[v] = c->state + v * c->stride; c->Un[v] = c->state + (8 + v) * c->stride; }

    // geometry
    std::vector<double> host;
    size_t off[12];
    for (int d = 0; d < 3; d++) {
        std::vector<double> w, ce;
        build_axis(grid->n[d], grid->edges[d], bc->face[d][0], bc->face[d][1], w, ce);
        off[d] = host.size(); host.insert(host.end(), w.begin(), w.end());
        off[3 + d] = host.size(); host.insert(host.end(), ce.begin(), ce.end());
    }
    // reciprocal geometry for the contracted FP64 form: 1 / w and 1 / h with
    // h = w_-/2 + w + w_+/2 (the span of the centred source differences)
    for (int d = 0; d < 3; d++) {
        const size_t len = (size_t)grid->n[d] + 2 * GH;
        const double *w = host.data() + off[d];
        std::vector<double> iw(len), ih(len, 0.0);
        for (size_t k = 0; k < len; k++) iw[k] = 1.0 / w[k];
        for (size_t k = 1; k + 1 < len; k++) ih[k] = 1.0 / (0.5 * w[k - 1] + w[k] + 0.5 * w[k + 1]);
        off[6 + d] = host.size(); host.insert(host.end(), iw.begin(), iw.end());
        off[9 + d] = host.size(); host.insert(host.end(), ih.begin(), ih.end());
    }
    int dev_sms = 152;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device);
    c->cfl_blocks = dev_sms * 4;
    long long need_blocks = (ncell + cfl_threads() - 1) / cfl_threads();
    if (need_blocks < c->cfl_blocks) c->cfl_blocks = (int)need_blocks;
    size_t scratch_bytes = sizeof(double) * (host.size() + 2 + c->cfl_blocks) + 64;
    e = cudaMalloc(&c->geo, scratch_bytes);
    if (e != cudaSuccess) { cudaFree(c->state); delete c; return PPMLR_E_OOM; }
    for (int d = 0; d < 3; d++) {
        c->w[d] = c->geo + off[d]; c->c[d] = c->geo + off[3 + d];
        c->iw[d] = c->geo + off[6 + d]; c->ih[d] = c->geo + off[9 + d];
    }
    c->dt_dev = c->geo + host.size();
    c->partial = c->dt_dev + 2;
    unsigned char *tail = reinterpret_cast<unsigned char *>(c->partial + c->cfl_blocks);
    c->flags = reinterpret_cast<int *>(tail);
    c->counter = reinterpret_cast<unsigned int *>(tail + 8);
    c->floors = reinterpret_cast<unsigned long long *>(tail + 16);
    e = cudaMemcpyAsync(c->geo, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dt_dev, 0, sizeof(double) * (2 + c->cfl_blocks) + 64, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->state, 0, sizeof(double) * c->stride * 16, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { cudaFree(c->geo); cudaFree(c->state); delete c; return PPMLR_E_CUDA; }
    {
        std::vector<float> hf(host.size());
        for (size_t k = 0; k < host.size(); k++) hf[k] = (float)host[k];
        e = cudaMalloc(&c->geof, sizeof(float) * hf.size());
        if (e != cudaSuccess) { cudaFree(c->geo); cudaFree(c->state); delete c; return PPMLR_E_OOM; }
        for (int d = 0; d < 3; d++) { c->wf[d] = c->geof + off[d]; c->cf[d] = c->geof + off[3 + d]; }
        e = cudaMemcpyAsync(c->geof, hf.data(), sizeof(float) * hf.size(), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) { cudaFree(c->geof); cudaFree(c->geo); cudaFree(c->state); delete c; return PPMLR_E_CUDA; }
    }
    size_t rs = prec == PPMLR_MIXED ? sizeof(float) : sizeof(double);
    for (int d = 0; d < 3; d++) { c->tile[d] = choose_tile(d, c->n, rs); c->mode[d] = 0; c->march_C[d] = c->n[d]; }
    c->sms = dev_sms;
    c->bd = nullptr;
    c->inner_mask = nullptr;
    if (bc->r_inner > 0.0) {
        // the inner-sphere test of every cell, once, with the CPU reference's expression
        std::vector<unsigned char> mask((size_t)ncell);
        const double *cx = host.data() + off[3] + GH, *cy = host.data() + off[4] + GH, *cz = host.data() + off[5] + GH;
        const double r2 = bc->r_inner * bc->r_inner;
        size_t i = 0;
        for (int iz = 0; iz < c->n[2]; iz++)
            for (int iy = 0; iy < c->n[1]; iy++)
                for (int ix = 0; ix < c->n[0]; ix++, i++) {
                    mask[i] = cx[ix] * cx[ix] + cy[iy] * cy[iy] + cz[iz] * cz[iz] < r2 ? 1 : 0;
                    if (mask[i]) c->inner_list.push_back((long long)i);
                }
        e = cudaMalloc(&c->inner_mask, mask.size());
        if (e == cudaSuccess) e = cudaMemcpy(c->inner_mask, mask.data(), mask.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(c->inner_mask); cudaFree(c->geof); cudaFree(c->geo); cudaFree(c->state); delete c;
            return e == cudaErrorMemoryAllocation ? PPMLR_E_OOM : PPMLR_E_CUDA;
        }
    }
    if (prec != PPMLR_MIXED && bc->dipole_moment != 0.0) {
        // the dipole at every cell centre, evaluated once by the sweeps' own formula
        e = cudaMalloc(&c->bd, sizeof(double) * c->stride * 3);
        if (e == cudaSuccess)
            e = sweep_launchers(prec).dipole_table(bc->dipole_moment, c->n, c->c[0], c->c[1], c->c[2], c->bd,
                                                   (long long)c->stride, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            cudaFree(c->bd); cudaFree(c->inner_mask); cudaFree(c->geof); cudaFree(c->geo); cudaFree(c->state);
            delete c;
            return e == cudaErrorMemoryAllocation ? PPMLR_E_OOM : PPMLR_E_CUDA;
        }
    }
    if (prec != PPMLR_MIXED) {
        // the two-pass CFL step's screen: a float bound per cell and the threshold
        e = cudaMalloc(&c->screen, sizeof(float) * ((size_t)ncell + 1));
        if (e != cudaSuccess) {
            cudaFree(c->bd); cudaFree(c->inner_mask); cudaFree(c->geof); cudaFree(c->geo); cudaFree(c->state);
            delete c;
            return e == cudaErrorMemoryAllocation ? PPMLR_E_OOM : PPMLR_E_CUDA;
        }
    }
    *out = c;
    return PPMLR_OK;
}

static void drop_graphs(ppmlr_ctx *c)
{
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

void ppmlr_destroy(ppmlr_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    for (auto &r : c->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : c->pool) cudaEventDestroy(e);
    cudaFree(c->iono.buf); cudaFree(c->iono.cells); cudaFree(c->iono.state);
    cudaFree(c->iono.nodes); cudaFree(c->iono.inner);
    cudaFree(c->bd);
    cudaFree(c->screen);
    cudaFree(c->inner_mask);
    cudaFree(c->geof);
    cudaFree(c->geo);
    cudaFree(c->state);
    delete c;
}

const char *ppmlr_last_error(const ppmlr_ctx *c) { return c ? c->err.c_str() : k_null_ctx; }

long long ppmlr_launch_count(const ppmlr_ctx *c) { return c ? c->launches : 0; }

ppmlr_status ppmlr_set_stream(ppmlr_ctx *c, void *stream)
{
    if (!c) return PPMLR_E_INVALID;
    c->stream = (cudaStream_t)stream;
    return PPMLR_OK;
}

ppmlr_status ppmlr_set_state(ppmlr_ctx *c, const double *const U[8], int on_device)
{
    if (!c) return PPMLR_E_INVALID;
    if (!U) return fail(c, PPMLR_E_INVALID, "set_state: null array list");
    for (int v = 0; v < 8; v++)
        if (!U[v]) return fail(c, PPMLR_E_INVALID, "set_state: null array");
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int v = 0; v < 8; v++)
        CK(c, cudaMemcpyAsync(c->U[v], U[v], sizeof(double) * c->ncell, kind, c->stream), "set_state copy");
    CK(c, cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream), "set_state flags");
    if (!on_device) CK(c, cudaStreamSynchronize(c->stream), "set_state sync");
    return PPMLR_OK;
}

static ppmlr_status read_flags(ppmlr_ctx *c)
{
    int f = 0;
    CK(c, cudaMemcpyAsync(&f, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flags copy");
    CK(c, cudaStreamSynchronize(c->stream), "stream sync");
    if (f) {
        CK(c, cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream), "flags reset");
        if (f & FLAG_BOUNDS) return fail(c, PPMLR_E_BOUNDS, "checked build: a kernel index left its array");
        if (f & FLAG_TIMEOUT) return fail(c, PPMLR_E_TIMEOUT, "a bounded device wait gave up");
        if (f & FLAG_NONFINITE) return fail(c, PPMLR_E_NONFINITE, "a sweep produced a non-finite state");
        return fail(c, PPMLR_E_CFL, "time step too large for the CFL condition");
    }
    return PPMLR_OK;
}

// z-layer ranges of the state (z is the slowest axis: layers k0 .. k0+nk-1
// of array v are one contiguous block), for the halo exchange of a domain
// split along z.
static const char *layer_range_error(const ppmlr_ctx *c, int k0, int nk, const void *const *U)
{
    if (!U) return "layers: null array list";
    for (int v = 0; v < 8; v++)
        if (!U[v]) return "layers: null array";
    if (k0 < 0 || nk < 0 || k0 + nk > c->n[2]) return "layers: need 0 <= k0 and k0 + nk <= n[2]";
    return nullptr;
}

ppmlr_status ppmlr_get_layers(ppmlr_ctx *c, int k0, int nk, double *const U[8], int on_device)
{
    if (!c) return PPMLR_E_INVALID;
    if (const char *why = layer_range_error(c, k0, nk, (const void *const *)U)) return fail(c, PPMLR_E_INVALID, why);
    const size_t plane = (size_t)c->n[0] * c->n[1];
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int v = 0; v < 8; v++)
        if (nk > 0)
            CK(c, cudaMemcpyAsync(U[v], c->U[v] + (size_t)k0 * plane, sizeof(double) * plane * nk, kind, c->stream),
               "get_layers copy");
    if (!on_device) CK(c, cudaStreamSynchronize(c->stream), "get_layers sync");
    return PPMLR_OK;
}

ppmlr_status ppmlr_set_layers(ppmlr_ctx *c, int k0, int nk, const double *const U[8], int on_device)
{
    if (!c) return PPMLR_E_INVALID;
    if (const char *why = layer_range_error(c, k0, nk, (const void *const *)U)) return fail(c, PPMLR_E_INVALID, why);
    const size_t plane = (size_t)c->n[0] * c->n[1];
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int v = 0; v < 8; v++)
        if (nk > 0)
            CK(c, cudaMemcpyAsync(c->U[v] + (size_t)k0 * plane, U[v], sizeof(double) * plane * nk, kind, c->stream),
               "set_layers copy");
    if (!on_device) CK(c, cudaStreamSynchronize(c->stream), "set_layers sync");
    return PPMLR_OK;
}

ppmlr_status ppmlr_check(ppmlr_ctx *c)
{
    if (!c) return PPMLR_E_INVALID;
    CK(c, cudaStreamSynchronize(c->stream), "stream sync");
    return read_flags(c);
}

ppmlr_status ppmlr_get_state(ppmlr_ctx *c, double *const U[8], int on_device)
{
    if (!c) return PPMLR_E_INVALID;
    if (!U) return fail(c, PPMLR_E_INVALID, "get_state: null array list");
    for (int v = 0; v < 8; v++)
        if (!U[v]) return fail(c, PPMLR_E_INVALID, "get_state: null array");
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int v = 0; v < 8; v++)
        CK(c, cudaMemcpyAsync(U[v], c->U[v], sizeof(double) * c->ncell, kind, c->stream), "get_state copy");
    return read_flags(c);
}

static ppmlr_status launch_one_sweep(ppmlr_ctx *c, int d, double dt, const double *dt_dev)
{
    if (is_sweep_noop(c, d)) return PPMLR_OK;
    SweepArgs a;
    memset(&a, 0, sizeof(a));
    a.U = c->U[0]; a.Un = c->Un[0]; a.vs = (long long)c->stride;
    for (int k = 0; k < 3; k++) a.n[k] = c->n[k];
    const Tile &t = c->tile[d];
    a.N = c->n[d];
    a.C = t.C; a.L = t.L; a.NP = t.NP; a.nchunk = t.nchunk; a.ngx = t.ngx;
    a.w = c->w[d]; a.c = c->c[d];
    a.cx = c->c[0]; a.cy = c->c[1]; a.cz = c->c[2];
    a.bc_lo = c->bc.face[d][0]; a.bc_hi = c->bc.face[d][1];
    const ppmlr_prim &f = c->bc.inflow;
    double infl[8] = {f.rho, f.v[0], f.v[1], f.v[2], f.B[0], f.B[1], f.B[2], f.p};
    memcpy(a.inflow, infl, sizeof(infl));
    const ppmlr_prim &q = c->bc.inner;
    double inn[8] = {q.rho, q.v[0], q.v[1], q.v[2], 0.0, 0.0, 0.0, q.p};
    memcpy(a.inner, inn, sizeof(inn));
    a.gamma = c->gamma; a.p_min = c->bc.p_min; a.M = c->bc.dipole_moment; a.r_inner = c->bc.r_inner;
    a.powell = c->bc.powell ? 1 : 0;
    a.do_src = (a.M != 0.0 || a.powell) ? 1 : 0;
    a.riemann_iters = c->riemann_iters;
    a.steepen = c->steepen;
    a.dt = dt; a.dt_dev = dt_dev;
    a.bd = c->bd;
    if (c->prec != PPMLR_MIXED) { a.iw = c->iw[d]; a.ih = c->ih[d]; }
    a.inner_mask = c->inner_mask;
    if (c->iono.on) {
        a.inner_cells = c->iono.cells;
        a.inner_state = c->iono.state;
        a.n_inner = (int)c->inner_list.size();
    }
    a.flags = c->flags; a.floors = c->floors;
    a.wf = c->wf[d];
    a.cxf = c->cf[0]; a.cyf = c->cf[1]; a.czf = c->cf[2];
    a.gammaf = (float)a.gamma; a.p_minf = (float)a.p_min; a.Mf = (float)a.M; a.r_innerf = (float)a.r_inner;
    for (int k = 0; k < 8; k++) a.inflowf[k] = (float)a.inflow[k];
    a.p_reff = c->prec == PPMLR_MIXED ? mixed_pressure_reference(c->bc) : 0.0f;
    int rec = timing_begin(c, d);
    cudaError_t e;
    if (c->mode[d] == 3 && !c->steepen) {          // marching form (no contact steepening)
        a.C = c->march_C[d];
        a.nchunk = (a.N + a.C - 1) / a.C;
        a.L = 32;
        a.NP = a.C + 2 * GH;
        a.ngx = d == 0 ? (int)(((long long)c->n[1] * c->n[2] + 31) / 32) : (c->n[0] + 31) / 32;
        e = sweep_launchers(c->prec).march(d, a, c->stream);
    } else if (c->mode[d] == 1 || c->mode[d] == 2) {
        const int b = c->U[0] == c->state ? 0 : 1;     // buffer holding the input state
        e = sweep_launchers(c->prec).tma(d, c->mode[d] == 1, a, c->tmap[d][b], c->tma_blocks[d], t.threads,
                                         c->tma_smem[d], c->stream);
    } else {
        e = sweep_launchers(c->prec).single(d, a, t, c->stream);
    }
    timing_end(c, rec);
    if (e != cudaSuccess) return cuda_fail(c, e, "sweep launch");
    c->launches++;
    for (int v = 0; v < 8; v++) { double *tmp = c->U[v]; c->U[v] = c->Un[v]; c->Un[v] = tmp; }
    return PPMLR_OK;
}

ppmlr_status ppmlr_sweep(ppmlr_ctx *c, int axis, double dt)
{
    if (!c) return PPMLR_E_INVALID;
    if (axis < 0 || axis > 2) return fail(c, PPMLR_E_INVALID, "sweep: axis must be 0, 1 or 2");
    if (!(dt > 0.0) || !isfinite(dt)) return fail(c, PPMLR_E_INVALID, "sweep: dt must be finite and > 0");
    return launch_one_sweep(c, axis, dt, nullptr);
}

// Device buffer of the shell (doubles): jr, phi (2 nt np each), Fourier
// coefficients (2 nt (np/2+1) x 2), poles (2), then the host tables: twiddles
// (2 np), colatitude rows (4 nt), mode eigenvalues (np/2+1).
struct IonoLayout {
    size_t nodes, nm, jr, phi, spec, pole, tw, rows, lam, total;
    explicit IonoLayout(const ppmlr_iono &g)
    {
        nodes = 2 * (size_t)g.n_theta * g.n_phi;
        nm = (size_t)g.n_phi / 2 + 1;
        jr = 0; phi = jr + nodes; spec = phi + nodes; pole = spec + 2 * (size_t)g.n_theta * nm * 2;
        tw = pole + 2; rows = tw + 2 * (size_t)g.n_phi; lam = rows + 4 * (size_t)g.n_theta; total = lam + nm;
    }
};

// The ionosphere solve from the current state (five small kernels) on stream s.
static ppmlr_status launch_iono(ppmlr_ctx *c, cudaStream_t s)
{
    const ppmlr_iono &g = c->iono.cfg;
    const IonoLayout L(g);
    IonoArgs a;
    memset(&a, 0, sizeof(a));
    for (int d = 0; d < 3; d++) { a.B[d] = c->U[4 + d]; a.n[d] = c->n[d]; a.c[d] = c->c[d]; }
    a.r_iono = g.r_iono; a.sigma_p = g.sigma_p;
    a.nt = g.n_theta; a.np = g.n_phi;
    a.nodes = c->iono.nodes;
    double *b = c->iono.buf;
    a.jr = b + L.jr; a.phi = b + L.phi; a.spec = b + L.spec; a.pole = b + L.pole;
    a.tw = b + L.tw; a.rows = b + L.rows; a.lam = b + L.lam;
    a.inner = c->iono.inner;
    a.n_inner = (int)c->inner_list.size();
    a.inner_state = c->iono.state;
    a.rho_in = c->bc.inner.rho; a.p_in = c->bc.inner.p; a.gamma = c->gamma;
    int n = 0;
    cudaError_t e = launch_ionosphere(a, s, &n);
    if (e != cudaSuccess) return cuda_fail(c, e, "ionosphere launch");
    c->launches += n;
    return PPMLR_OK;
}

// shell_done: the step's ionosphere solve is already on the stream
static ppmlr_status do_step(ppmlr_ctx *c, double dt, const double *dt_dev, bool shell_done = false)
{
    if (c->iono.on && !shell_done) {
        ppmlr_status s = launch_iono(c, c->stream);
        if (s != PPMLR_OK) return s;
    }
    const int order_even[3] = {0, 1, 2}, order_odd[3] = {2, 1, 0};
    const int *ord = (c->steps & 1) ? order_odd : order_even;
    for (int k = 0; k < 3; k++) {
        ppmlr_status s = launch_one_sweep(c, ord[k], dt, dt_dev);
        if (s != PPMLR_OK) return s;
    }
    c->steps++;
    return PPMLR_OK;
}

ppmlr_status ppmlr_step(ppmlr_ctx *c, double dt)
{
    if (!c) return PPMLR_E_INVALID;
    if (!(dt > 0.0) || !isfinite(dt)) return fail(c, PPMLR_E_INVALID, "step: dt must be finite and > 0");
    ppmlr_status s = do_step(c, dt, nullptr);
    if (s == PPMLR_OK) c->t_host += dt;
    return s;
}

// advance_time: the kernel also adds the new dt to the device time accumulator
static ppmlr_status launch_cfl_kernel(ppmlr_ctx *c, double cfl, bool advance_time = false)
{
    CflArgs a;
    memset(&a, 0, sizeof(a));
    for (int v = 0; v < 8; v++) a.U[v] = c->U[v];
    for (int d = 0; d < 3; d++) { a.n[d] = c->n[d]; a.w[d] = c->w[d]; a.c[d] = c->c[d]; }
    a.gamma = c->gamma; a.p_min = c->bc.p_min; a.M = c->bc.dipole_moment; a.r_inner = c->bc.r_inner;
    a.cfl = cfl;
    a.partial = c->partial; a.counter = c->counter; a.dt_out = c->dt_dev;
    a.t_acc = advance_time ? c->dt_dev + 1 : nullptr;
    a.bd = c->bd;
    a.bd_vs = (long long)c->stride;
    if (c->prec == PPMLR_FP64)
        for (int d = 0; d < 3; d++) a.iw[d] = c->iw[d];
    a.inner_mask = c->inner_mask;
    for (int d = 0; d < 3; d++) { a.wf[d] = c->wf[d]; a.cf[d] = c->cf[d]; }
    a.gammaf = (float)a.gamma; a.p_minf = (float)a.p_min; a.Mf = (float)a.M; a.r_innerf = (float)a.r_inner;
    if (c->screen) { a.screen = c->screen; a.screen_thr = c->screen + c->ncell; }
    int rec = timing_begin(c, 3);
    cudaError_t e = cfl_launchers(c->prec).single(a, c->cfl_blocks, c->stream);
    timing_end(c, rec);
    if (e != cudaSuccess) return cuda_fail(c, e, "cfl launch");
    c->launches += c->screen ? 2 : 1;
    return PPMLR_OK;
}

ppmlr_status ppmlr_cfl_dt(ppmlr_ctx *c, double cfl, double *dt_out)
{
    if (!c) return PPMLR_E_INVALID;
    if (!dt_out || !(cfl > 0.0)) return fail(c, PPMLR_E_INVALID, "cfl_dt: need cfl > 0 and an output pointer");
    ppmlr_status s = launch_cfl_kernel(c, cfl);
    if (s != PPMLR_OK) return s;
    CK(c, cudaMemcpyAsync(dt_out, c->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "dt copy");
    return read_flags(c);
}

// One device-dt step: the CFL pass and, with the shell on, the shell's solve
// on the side stream at the same time (both only read the state), joined
// before the first sweep; then the three sweeps.
static ppmlr_status cfl_step(ppmlr_ctx *c, double cfl)
{
    if (!c->iono.on) {
        ppmlr_status s = launch_cfl_kernel(c, cfl, true);
        return s != PPMLR_OK ? s : do_step(c, 0.0, c->dt_dev);
    }
    if (!c->side) CK(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "side stream");
    if (!c->ev_fork) CK(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "event");
    if (!c->ev_join) CK(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "event");
    CK(c, cudaEventRecord(c->ev_fork, c->stream), "fork");
    CK(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0), "fork");
    ppmlr_status s = launch_iono(c, c->side);
    if (s != PPMLR_OK) return s;
    CK(c, cudaEventRecord(c->ev_join, c->side), "join");
    s = launch_cfl_kernel(c, cfl, true);
    if (s != PPMLR_OK) return s;
    CK(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0), "join");
    return do_step(c, 0.0, c->dt_dev, true);
}

static ppmlr_status step_cfl_direct(ppmlr_ctx *c, double cfl, long long nsteps)
{
    for (long long k = 0; k < nsteps; k++) {
        ppmlr_status s = cfl_step(c, cfl);
        if (s != PPMLR_OK) return s;
    }
    return PPMLR_OK;
}

ppmlr_status ppmlr_step_cfl(ppmlr_ctx *c, double cfl, int nsteps)
{
    if (!c) return PPMLR_E_INVALID;
    if (!(cfl > 0.0) || nsteps < 0) return fail(c, PPMLR_E_INVALID, "step_cfl: need cfl > 0, nsteps >= 0");
    return step_cfl_direct(c, cfl, nsteps);
}

ppmlr_status ppmlr_get_dt(ppmlr_ctx *c, double *dt_out)
{
    if (!c) return PPMLR_E_INVALID;
    if (!dt_out) return fail(c, PPMLR_E_INVALID, "get_dt: null output");
    CK(c, cudaMemcpyAsync(dt_out, c->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "dt copy");
    CK(c, cudaStreamSynchronize(c->stream), "stream sync");
    return PPMLR_OK;
}

ppmlr_status ppmlr_get_diagnostics(ppmlr_ctx *c, long long *step, long long *floor_hits, int *order_parity)
{
    if (!c) return PPMLR_E_INVALID;
    unsigned long long fl = 0;
    CK(c, cudaMemcpyAsync(&fl, c->floors, sizeof(fl), cudaMemcpyDeviceToHost, c->stream), "floors copy");
    CK(c, cudaStreamSynchronize(c->stream), "stream sync");
    if (step) *step = c->steps;
    if (floor_hits) *floor_hits = (long long)fl;
    if (order_parity) *order_parity = (int)(c->steps & 1);
    return PPMLR_OK;
}

// The marching form serves the mixed path without contact steepening.
static bool march_eligible(const ppmlr_ctx *c) { return c->prec == PPMLR_MIXED && !c->steepen; }

// Per-process cache of tuned tile shapes: (dir, nx, ny, nz, prec) -> (C, L, form).
static std::mutex g_tune_mutex;
static std::map<std::tuple<int, int, int, int, int>, std::tuple<int, int, int>> g_tune_cache;

ppmlr_status ppmlr_autotune(ppmlr_ctx *c, double *best_ms)
{
    if (!c) return PPMLR_E_INVALID;
    const size_t rs = c->prec == PPMLR_MIXED ? sizeof(float) : sizeof(double);
    unsigned long long floors_before = 0;
    CK(c, cudaMemcpyAsync(&floors_before, c->floors, sizeof(floors_before), cudaMemcpyDeviceToHost, c->stream),
       "floors copy");
    ppmlr_status st = launch_cfl_kernel(c, 0.4);      // a valid device dt for the timing runs
    if (st != PPMLR_OK) return st;
    cudaEvent_t t0, t1;
    CK(c, cudaEventCreate(&t0), "event");
    CK(c, cudaEventCreate(&t1), "event");
    const bool was_timing = c->timing;
    c->timing = false;
    drop_graphs(c);
    for (int d = 0; d < 3; d++) {
        if (best_ms) best_ms[d] = 0.0;
        if (is_sweep_noop(c, d)) continue;
        auto key = std::make_tuple(d, c->n[0], c->n[1], c->n[2], (int)c->prec);
        {
            std::lock_guard<std::mutex> lk(g_tune_mutex);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                const int f = std::get<2>(it->second);
                if (f == 3) {
                    c->march_C[d] = std::get<0>(it->second);
                    c->mode[d] = 3;
                } else {
                    c->tile[d] = make_tile(d, c->n, rs, std::get<0>(it->second), std::get<1>(it->second));
                    c->mode[d] = f != 0 && setup_tma(c, d, f) ? f : 0;
                }
                continue;
            }
        }
        const int N = c->n[d];
        const int maxt = tile_budget(c->prec, d);
        std::vector<std::pair<int, int>> cands;
        for (int nchunk = 1; nchunk <= 4; nchunk++) {
            const int C = (N + nchunk - 1) / nchunk;
            if (C + 2 * GH > maxt) continue;
            if (nchunk > 1 && C < 48) break;
            for (int L = 1; L <= 16; L *= 2) {
                if ((C + 2 * GH) * L > maxt) break;
                if (d != 0 && L > 1 && L / 2 >= c->n[0]) break;
                if (d == 0 && L > 1 && (long long)L > (long long)c->n[1] * c->n[2]) break;
                cands.push_back({C, L});
            }
        }
        float best = 1e30f;
        std::tuple<int, int, int> pick = {c->tile[d].C, c->tile[d].L, c->mode[d]};
        const Tile keep = c->tile[d];
        const int keep_mode = c->mode[d];
        std::vector<std::tuple<int, int, int>> trials;
        for (auto &cl : cands) {
            trials.push_back({cl.first, cl.second, 0});
            for (int f = 1; f <= 2; f++)
                if (tma_eligible(c, d, make_tile(d, c->n, rs, cl.first, cl.second), f))
                    trials.push_back({cl.first, cl.second, f});
        }
        const int keep_march = c->march_C[d];
        if (march_eligible(c))            // marching form: whole pencils or 2..4 equal chunks
            for (int k = 1; k <= 4; k++) {
                const int C = (N + k - 1) / k;
                if (k > 1 && C < 32) break;
                trials.push_back({C, 32, 3});
            }
        for (auto &tr : trials) {
            const int f = std::get<2>(tr);
            if (f == 3) {
                c->march_C[d] = std::get<0>(tr);
                c->mode[d] = 3;
            } else {
                c->tile[d] = make_tile(d, c->n, rs, std::get<0>(tr), std::get<1>(tr));
                c->mode[d] = f != 0 && setup_tma(c, d, f) ? f : 0;
                if (c->mode[d] != f) continue;
            }
            float tot = 0.0f;
            for (int rep = 0; rep < 3; rep++) {
                CK(c, cudaEventRecord(t0, c->stream), "event");
                st = launch_one_sweep(c, d, 0.0, c->dt_dev);
                if (st != PPMLR_OK) {
                    c->tile[d] = keep; c->mode[d] = keep_mode; c->march_C[d] = keep_march;
                    return st;
                }
                CK(c, cudaEventRecord(t1, c->stream), "event");
                CK(c, cudaEventSynchronize(t1), "event sync");
                // undo the buffer swap of launch_one_sweep: the state stays in place
                for (int v = 0; v < 8; v++) { double *tmp = c->U[v]; c->U[v] = c->Un[v]; c->Un[v] = tmp; }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, t0, t1);
                if (rep > 0) tot += ms;
            }
            if (tot < best) { best = tot; pick = tr; }
        }
        const int fp = std::get<2>(pick);
        if (fp == 3) {
            c->tile[d] = keep;
            c->march_C[d] = std::get<0>(pick);
            c->mode[d] = 3;
        } else {
            c->tile[d] = make_tile(d, c->n, rs, std::get<0>(pick), std::get<1>(pick));
            c->march_C[d] = keep_march;
            c->mode[d] = fp != 0 && setup_tma(c, d, fp) ? fp : 0;
        }
        if (best_ms) best_ms[d] = best / 2.0f;
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune_cache[key] = pick;
    }
    c->timing = was_timing;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    CK(c, cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream), "flags reset");
    CK(c, cudaMemcpyAsync(c->floors, &floors_before, sizeof(floors_before), cudaMemcpyHostToDevice, c->stream),
       "floors restore");
    CK(c, cudaStreamSynchronize(c->stream), "sync");
    return PPMLR_OK;
}

ppmlr_status ppmlr_get_tiles(ppmlr_ctx *c, int *C, int *L)
{
    if (!c || !C || !L) return PPMLR_E_INVALID;
    for (int d = 0; d < 3; d++) {
        const bool m = c->mode[d] == 3 && !c->steepen;
        C[d] = m ? c->march_C[d] : c->tile[d].C;
        L[d] = m ? 32 : c->tile[d].L;
    }
    return PPMLR_OK;
}

ppmlr_status ppmlr_set_march_chunk(ppmlr_ctx *c, int axis, int C)
{
    if (!c) return PPMLR_E_INVALID;
    if (axis < 0 || axis > 2) return fail(c, PPMLR_E_INVALID, "set_march_chunk: bad axis");
    if (C < 1 || C > c->n[axis]) return fail(c, PPMLR_E_INVALID, "set_march_chunk: need 1 <= C <= n[axis]");
    c->march_C[axis] = C;
    drop_graphs(c);
    return PPMLR_OK;
}

ppmlr_status ppmlr_set_tiles(ppmlr_ctx *c, int axis, int C, int L)
{
    if (!c) return PPMLR_E_INVALID;
    if (axis < 0 || axis > 2) return fail(c, PPMLR_E_INVALID, "set_tiles: bad axis");
    const int N = c->n[axis];
    if (C < 1 || C > N || L < 1) return fail(c, PPMLR_E_INVALID, "set_tiles: need 1 <= C <= n[axis] and L >= 1");
    const size_t rs = c->prec == PPMLR_MIXED ? sizeof(float) : sizeof(double);
    const int maxt = tile_budget(c->prec, axis);
    if ((long long)(C + 2 * GH) * L > maxt) return fail(c, PPMLR_E_INVALID, "set_tiles: (C + 14) * L exceeds the thread budget");
    c->tile[axis] = make_tile(axis, c->n, rs, C, L);
    c->mode[axis] = 0;
    drop_graphs(c);
    return PPMLR_OK;
}

ppmlr_status ppmlr_set_riemann_solver(ppmlr_ctx *c, int iters)
{
    if (!c) return PPMLR_E_INVALID;
    if (iters < 0 || iters > 16) return fail(c, PPMLR_E_INVALID, "set_riemann_solver: iters must be in [0, 16]");
    c->riemann_iters = iters;
    drop_graphs(c);
    return PPMLR_OK;
}

static void free_iono(ppmlr_ctx *c)
{
    cudaFree(c->iono.buf); cudaFree(c->iono.cells); cudaFree(c->iono.state);
    cudaFree(c->iono.nodes); cudaFree(c->iono.inner);
    c->iono = ppmlr_ctx::Iono{};
}

// Earth dipole along -z (host): B = M (3 (m.r) r - m r^2) / r^5, m = -z.
static void dipole_host(double M, double x, double y, double z, double *B)
{
    const double r2 = x * x + y * y + z * z;
    if (M == 0.0 || r2 == 0.0) { B[0] = B[1] = B[2] = 0.0; return; }
    const double f = M / (r2 * r2 * sqrt(r2));
    B[0] = f * (3.0 * -z * x);
    B[1] = f * (3.0 * -z * y);
    B[2] = f * (3.0 * -z * z + r2);
}

// Bilinear stencil of the cap potential at the foot point of the dipole field
// line through (x, y, z): up to 4 (node, weight) pairs (node -1 - cap: that
// cap's pole value, the ring-0 mean); none off the caps or where the line
// closes below the shell.  Returns the number of pairs.
static int cap_stencil(const ppmlr_iono &g, double theta_max, double dth, double dph, double x, double y, double z,
                       int *idx, double *w)
{
    const double r2 = x * x + y * y + z * z;
    if (r2 == 0.0) return 0;
    const double r = sqrt(r2);
    const double s2i = (g.r_iono / r) * ((x * x + y * y) / r2);
    if (s2i > 1.0) return 0;
    const double th = asin(sqrt(s2i));
    if (!(th < theta_max)) return 0;
    double ph = atan2(y, x);
    if (ph < 0.0) ph += 2.0 * M_PI;
    const int h = z >= 0.0 ? 0 : 1, nt = g.n_theta, np = g.n_phi;
    const double u = ph / dph, fl = floor(u);
    const int k0 = ((int)fl % np + np) % np, k1 = (k0 + 1) % np;
    const double fu = u - fl;
    int n = 0;
    auto ring = [&](int j, double wr) {
        if (j < 0) { idx[n] = -1 - h; w[n++] = wr; return; }
        if (j >= nt) return;
        const int base = (h * nt + j) * np;
        idx[n] = base + k0; w[n++] = wr * (1.0 - fu);
        idx[n] = base + k1; w[n++] = wr * fu;
    };
    const double t = th / dth - 0.5;
    if (t < 0.0) {
        const double q = (t + 0.5) / 0.5;
        ring(-1, 1.0 - q);
        ring(0, q);
    } else if (t > nt - 1) {
        ring(nt - 1, 1.0 - (t - (nt - 1)) / 0.5);
    } else {
        const int j = (int)floor(t);
        ring(j, 1.0 - (t - j));
        ring(j + 1, t - j);
    }
    return n;
}

ppmlr_status ppmlr_set_ionosphere(ppmlr_ctx *c, const ppmlr_iono *cfg)
{
    if (!c) return PPMLR_E_INVALID;
    if (!cfg) {
        CK(c, cudaStreamSynchronize(c->stream), "stream sync");
        free_iono(c);
        drop_graphs(c);
        return PPMLR_OK;
    }
    const ppmlr_iono g = *cfg;
    if (!(c->bc.r_inner > 0.0) || c->bc.dipole_moment == 0.0)
        return fail(c, PPMLR_E_INVALID, "set_ionosphere: needs an inner sphere and a dipole");
    if (!(g.r_iono > 0.0) || !(g.r_iono < c->bc.r_inner) || !(g.r_fac > g.r_iono) || !isfinite(g.r_fac) ||
        !(g.sigma_p > 0.0) || !isfinite(g.sigma_p) || g.n_theta < 2 || g.n_theta > IONO_MAX_NT || g.n_phi < 4 ||
        g.n_phi > 1024 || (g.n_phi & 1))
        return fail(c, PPMLR_E_INVALID, "set_ionosphere: need 0 < r_iono < r_inner, r_fac > r_iono, sigma_p > 0, "
                                        "2 <= n_theta <= 256, even 4 <= n_phi <= 1024");
    std::vector<double> ce[3];        // interior centres
    for (int d = 0; d < 3; d++) {     // the mapping sphere's curl stencils inside the grid
        const std::vector<double> &e = c->edges[d];
        const int n = c->n[d];
        if (n < 4) return fail(c, PPMLR_E_INVALID, "set_ionosphere: every axis needs at least 4 cells");
        ce[d].resize(n);
        for (int i = 0; i < n; i++) ce[d][i] = 0.5 * (e[i] + e[i + 1]);
        const double rf = g.r_fac * (1.0 + 1e-12);
        if (!(ce[d][1] < -rf) || !(rf < ce[d][n - 2]))
            return fail(c, PPMLR_E_INVALID, "set_ionosphere: the mapping sphere must lie inside centres 1 .. n-2");
    }
    const IonoLayout L(g);
    const double M = c->bc.dipole_moment;
    const double theta_max = asin(sqrt(g.r_iono / c->bc.r_inner));
    const double dth = theta_max / g.n_theta, dph = 2.0 * M_PI / g.n_phi;
    // cap solve tables: twiddles, colatitude rows (conservative five-point
    // form on the unit sphere, no flux through the pole, odd ghost at
    // theta_max), eigenvalues of the longitude second difference
    std::vector<double> tab(L.total - L.tw);
    for (int q = 0; q < g.n_phi; q++) {
        tab[2 * q] = cos(2.0 * M_PI * q / g.n_phi);
        tab[2 * q + 1] = sin(2.0 * M_PI * q / g.n_phi);
    }
    double *rows = tab.data() + (L.rows - L.tw);
    for (int j = 0; j < g.n_theta; j++) {
        const double th = (j + 0.5) * dth, s = sin(th);
        const double sp = sin(th + 0.5 * dth), sm = j > 0 ? sin(th - 0.5 * dth) : 0.0;
        rows[4 * j] = sm / (s * dth * dth);
        rows[4 * j + 1] = j < g.n_theta - 1 ? sp / (s * dth * dth) : 0.0;
        rows[4 * j + 2] = -(sp + sm) / (s * dth * dth) - (j == g.n_theta - 1 ? sp / (s * dth * dth) : 0.0);
        rows[4 * j + 3] = 1.0 / (s * s);
    }
    double *lam = tab.data() + (L.lam - L.tw);
    for (size_t m = 0; m < L.nm; m++) {
        const double sn = sin(M_PI * (double)m / g.n_phi);
        lam[m] = 4.0 * sn * sn / (dph * dph);
    }
    // per node: mapping point along the node's dipole field line at r_fac
    std::vector<IonoNode> nodes(L.nodes);
    for (int h = 0; h < 2; h++)
        for (int j = 0; j < g.n_theta; j++)
            for (int k = 0; k < g.n_phi; k++) {
                IonoNode &q = nodes[((size_t)h * g.n_theta + j) * g.n_phi + k];
                for (int d = 0; d < 3; d++) { q.i0[d] = 1; q.w[d] = 0.0; q.Bd[d] = 0.0; }
                q.factor = 0.0;
                const double th = (j + 0.5) * dth, ph = k * dph, st = sin(th), ct = cos(th);
                const double s2m = (g.r_fac / g.r_iono) * st * st;       // sin^2 at r_fac, same line
                if (s2m > 1.0) continue;
                const double zs = h == 0 ? 1.0 : -1.0, sp = sin(ph), cp = cos(ph);
                const double sm = sqrt(s2m), cm = sqrt(1.0 - s2m);
                const double p[3] = {g.r_fac * sm * cp, g.r_fac * sm * sp, zs * g.r_fac * cm};
                for (int d = 0; d < 3; d++) {
                    const std::vector<double> &cc = ce[d];
                    int i = (int)(std::upper_bound(cc.begin(), cc.end(), p[d]) - cc.begin()) - 1;
                    i = i < 1 ? 1 : (i > c->n[d] - 3 ? c->n[d] - 3 : i);
                    q.i0[d] = i;
                    q.w[d] = (p[d] - cc[i]) / (cc[i + 1] - cc[i]);
                }
                dipole_host(M, p[0], p[1], p[2], q.Bd);
                const double f[3] = {g.r_iono * st * cp, g.r_iono * st * sp, zs * g.r_iono * ct};
                double Bf[3];
                dipole_host(M, f[0], f[1], f[2], Bf);
                const double br = (Bf[0] * f[0] + Bf[1] * f[1] + Bf[2] * f[2]) / g.r_iono;
                q.factor = br / sqrt(q.Bd[0] * q.Bd[0] + q.Bd[1] * q.Bd[1] + q.Bd[2] * q.Bd[2]);
            }
    // per inner cell: stencils of its six neighbours, E = -grad Phi folded in
    const size_t ninner = c->inner_list.size();
    std::vector<IonoInner> inner(ninner);
    for (size_t t = 0; t < ninner; t++) {
        const long long gi = c->inner_list[t];
        const int id[3] = {(int)(gi % c->n[0]), (int)((gi / c->n[0]) % c->n[1]),
                           (int)(gi / ((long long)c->n[0] * c->n[1]))};
        const double x0[3] = {ce[0][id[0]], ce[1][id[1]], ce[2][id[2]]};
        IonoInner &q = inner[t];
        for (int d = 0; d < 3; d++) {
            for (int s = 0; s < 8; s++) { q.idx[d][s] = 0; q.coef[d][s] = 0.0; }
            const int lo = id[d] > 0 ? id[d] - 1 : 0, hi = id[d] < c->n[d] - 1 ? id[d] + 1 : c->n[d] - 1;
            const double span = ce[d][hi] - ce[d][lo];
            for (int side = 0; side < 2; side++) {
                double pt[3] = {x0[0], x0[1], x0[2]};
                pt[d] = ce[d][side == 0 ? hi : lo];
                int ix[4];
                double wv[4];
                const int m = cap_stencil(g, theta_max, dth, dph, pt[0], pt[1], pt[2], ix, wv);
                for (int s = 0; s < m; s++) {
                    q.idx[d][4 * side + s] = ix[s];
                    q.coef[d][4 * side + s] = (side == 0 ? -wv[s] : wv[s]) / span;
                }
            }
        }
        double B[3];
        dipole_host(M, x0[0], x0[1], x0[2], B);
        const double b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
        for (int d = 0; d < 3; d++) q.bt[d] = b2 > 0.0 ? B[d] / b2 : 0.0;
    }
    // until the first solve, every inner cell holds the configuration's fixed
    // inner state (what the sweeps wrote without the shell)
    std::vector<double> rest(8 * ninner);
    {
        const ppmlr_prim &q = c->bc.inner;
        const double u[8] = {q.rho, q.rho * q.v[0], q.rho * q.v[1], q.rho * q.v[2], 0.0, 0.0, 0.0,
                             q.p / (c->gamma - 1.0) + 0.5 * q.rho * (q.v[0] * q.v[0] + q.v[1] * q.v[1] + q.v[2] * q.v[2])};
        for (int v = 0; v < 8; v++)
            for (size_t t = 0; t < ninner; t++) rest[(size_t)v * ninner + t] = u[v];
    }
    double *buf = nullptr, *state = nullptr;
    long long *cells = nullptr;
    IonoNode *dnodes = nullptr;
    IonoInner *dinner = nullptr;
    cudaError_t e = cudaMalloc(&buf, sizeof(double) * L.total);
    if (e == cudaSuccess) e = cudaMalloc(&dnodes, sizeof(IonoNode) * nodes.size());
    if (e == cudaSuccess && ninner) e = cudaMalloc(&cells, sizeof(long long) * ninner);
    if (e == cudaSuccess && ninner) e = cudaMalloc(&state, sizeof(double) * 8 * ninner);
    if (e == cudaSuccess && ninner) e = cudaMalloc(&dinner, sizeof(IonoInner) * ninner);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, sizeof(double) * L.total, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(buf + L.tw, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dnodes, nodes.data(), sizeof(IonoNode) * nodes.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && ninner)
        e = cudaMemcpyAsync(cells, c->inner_list.data(), sizeof(long long) * ninner, cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess && ninner)
        e = cudaMemcpyAsync(dinner, inner.data(), sizeof(IonoInner) * ninner, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && ninner)
        e = cudaMemcpyAsync(state, rest.data(), sizeof(double) * rest.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(buf); cudaFree(cells); cudaFree(state); cudaFree(dnodes); cudaFree(dinner);
        return e == cudaErrorMemoryAllocation ? fail(c, PPMLR_E_OOM, "set_ionosphere: out of device memory")
                                              : cuda_fail(c, e, "set_ionosphere");
    }
    free_iono(c);
    c->iono.on = true;
    c->iono.cfg = g;
    c->iono.buf = buf; c->iono.cells = cells; c->iono.state = state;
    c->iono.nodes = dnodes; c->iono.inner = dinner;
    drop_graphs(c);
    return PPMLR_OK;
}

ppmlr_status ppmlr_ionosphere_solve(ppmlr_ctx *c)
{
    if (!c) return PPMLR_E_INVALID;
    if (!c->iono.on) return fail(c, PPMLR_E_INVALID, "ionosphere_solve: the shell is off");
    return launch_iono(c, c->stream);
}

ppmlr_status ppmlr_get_ionosphere(ppmlr_ctx *c, double *phi, double *jr)
{
    if (!c) return PPMLR_E_INVALID;
    if (!c->iono.on) return fail(c, PPMLR_E_INVALID, "get_ionosphere: the shell is off");
    const IonoLayout L(c->iono.cfg);
    if (jr)
        CK(c, cudaMemcpyAsync(jr, c->iono.buf + L.jr, sizeof(double) * L.nodes, cudaMemcpyDeviceToHost, c->stream),
           "copy");
    if (phi)
        CK(c, cudaMemcpyAsync(phi, c->iono.buf + L.phi, sizeof(double) * L.nodes, cudaMemcpyDeviceToHost, c->stream),
           "copy");
    CK(c, cudaStreamSynchronize(c->stream), "stream sync");
    return read_flags(c);
}

ppmlr_status ppmlr_selftest_wait_timeout(ppmlr_ctx *c)
{
    if (!c) return PPMLR_E_INVALID;
    cudaError_t e = launch_wait_selftest(c->flags, 1 << 12, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "selftest launch");
    c->launches++;
    return PPMLR_OK;
}

ppmlr_status ppmlr_set_steepening(ppmlr_ctx *c, int on)
{
    if (!c) return PPMLR_E_INVALID;
    c->steepen = on ? 1 : 0;
    drop_graphs(c);
    return PPMLR_OK;
}

ppmlr_status ppmlr_get_sweep_forms(ppmlr_ctx *c, int *form)
{
    if (!c || !form) return PPMLR_E_INVALID;
    for (int d = 0; d < 3; d++) form[d] = c->mode[d];
    return PPMLR_OK;
}

ppmlr_status ppmlr_set_sweep_form(ppmlr_ctx *c, int axis, int form)
{
    if (!c) return PPMLR_E_INVALID;
    if (axis < 0 || axis > 2 || form < 0 || form > 3) return fail(c, PPMLR_E_INVALID, "set_sweep_form: bad axis or form");
    drop_graphs(c);
    if (form == 0) { c->mode[axis] = 0; return PPMLR_OK; }
    if (form == 3) {
        if (c->prec != PPMLR_MIXED) return fail(c, PPMLR_E_INVALID, "the marching form (3) is a PPMLR_MIXED form");
        c->mode[axis] = 3;
        return PPMLR_OK;
    }
    if (const char *why = setup_tma_why(c, axis, form)) return fail(c, PPMLR_E_INVALID, why);
    c->mode[axis] = form;
    return PPMLR_OK;
}

ppmlr_status ppmlr_enable_timing(ppmlr_ctx *c, int on)
{
    if (!c) return PPMLR_E_INVALID;
    c->timing = on != 0;
    return PPMLR_OK;
}

ppmlr_status ppmlr_read_timing(ppmlr_ctx *c, double *total_ms, long long *launches)
{
    if (!c) return PPMLR_E_INVALID;
    if (!total_ms || !launches) return fail(c, PPMLR_E_INVALID, "read_timing: null output");
    for (int k = 0; k < 4; k++) { total_ms[k] = 0.0; launches[k] = 0; }
    CK(c, cudaStreamSynchronize(c->stream), "stream sync");
    for (auto &r : c->recs) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            total_ms[r.kind] += ms;
            launches[r.kind] += 1;
        }
        c->pool.push_back(r.a);
        c->pool.push_back(r.b);
    }
    c->recs.clear();
    return PPMLR_OK;
}

ppmlr_status ppmlr_set_step_count(ppmlr_ctx *c, long long step)
{
    if (!c) return PPMLR_E_INVALID;
    if (step < 0) return fail(c, PPMLR_E_INVALID, "set_step_count: negative");
    c->steps = step;
    return PPMLR_OK;
}

// ---- long runs: simulated time, graph replay, checkpoints ----

ppmlr_status ppmlr_get_time(ppmlr_ctx *c, double *t_out)
{
    if (!c) return PPMLR_E_INVALID;
    if (!t_out) return fail(c, PPMLR_E_INVALID, "get_time: null output");
    double td = 0.0;
    CK(c, cudaMemcpyAsync(&td, c->dt_dev + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "time copy");
    CK(c, cudaStreamSynchronize(c->stream), "stream sync");
    *t_out = c->t_host + td;
    return PPMLR_OK;
}

static ppmlr_status put_device_time(ppmlr_ctx *c, double t)
{
    CK(c, cudaMemcpyAsync(c->dt_dev + 1, &t, sizeof(double), cudaMemcpyHostToDevice, c->stream), "time copy");
    CK(c, cudaStreamSynchronize(c->stream), "stream sync");
    c->t_host = 0.0;
    return PPMLR_OK;
}

ppmlr_status ppmlr_set_time(ppmlr_ctx *c, double t)
{
    if (!c) return PPMLR_E_INVALID;
    if (!isfinite(t)) return fail(c, PPMLR_E_INVALID, "set_time: t must be finite");
    return put_device_time(c, t);
}

// Captures ksteps steps (CFL pass + three sweeps each) from the current step
// parity and input buffer into an executable graph.  The host-side view
// (step count, launch count, buffer roles) is left as it was: the graph has
// not run yet.
static ppmlr_status capture_run_graph(ppmlr_ctx *c, double cfl, int ksteps, ppmlr_ctx::Graph &g)
{
    if (!c->cap) CK(c, cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking), "capture stream");
    const cudaStream_t user = c->stream;
    const bool was_timing = c->timing;
    const long long steps0 = c->steps, launches0 = c->launches;
    double *U0[8], *Un0[8];
    memcpy(U0, c->U, sizeof(U0));
    memcpy(Un0, c->Un, sizeof(Un0));
    g.parity = (int)(c->steps & 1);
    g.buf = c->U[0] == c->state ? 0 : 1;
    g.ksteps = ksteps;
    g.cfl = cfl;
    g.exec = nullptr;
    c->timing = false;
    c->stream = c->cap;
    cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    ppmlr_status st = e == cudaSuccess ? PPMLR_OK : cuda_fail(c, e, "begin capture");
    for (int k = 0; st == PPMLR_OK && k < ksteps; k++) st = cfl_step(c, cfl);
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) {
        cudaError_t e2 = cudaStreamEndCapture(c->cap, &graph);
        if (st == PPMLR_OK && e2 != cudaSuccess) st = cuda_fail(c, e2, "end capture");
    }
    g.launches = c->launches - launches0;
    c->stream = user;
    c->timing = was_timing;
    c->steps = steps0;
    c->launches = launches0;
    memcpy(c->U, U0, sizeof(U0));
    memcpy(c->Un, Un0, sizeof(Un0));
    if (st == PPMLR_OK) {
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        if (e != cudaSuccess) st = cuda_fail(c, e, "graph instantiate");
    }
    if (graph) cudaGraphDestroy(graph);
    return st;
}

ppmlr_status ppmlr_run(ppmlr_ctx *c, double cfl, long long nsteps, int graph_steps)
{
    if (!c) return PPMLR_E_INVALID;
    if (!(cfl > 0.0) || !isfinite(cfl) || nsteps < 0 || graph_steps < 0 || (graph_steps & 1) || graph_steps > 4096)
        return fail(c, PPMLR_E_INVALID, "run: need cfl > 0, nsteps >= 0 and an even graph_steps in [0, 4096]");
    long long left = nsteps;
    while (graph_steps > 0 && left >= graph_steps) {
        const int parity = (int)(c->steps & 1), buf = c->U[0] == c->state ? 0 : 1;
        ppmlr_ctx::Graph *g = nullptr;
        for (auto &x : c->graphs)
            if (x.parity == parity && x.buf == buf && x.ksteps == graph_steps && x.cfl == cfl) { g = &x; break; }
        if (!g) {
            ppmlr_ctx::Graph ng;
            ppmlr_status st = capture_run_graph(c, cfl, graph_steps, ng);
            if (st != PPMLR_OK) return st;
            c->graphs.push_back(ng);
            g = &c->graphs.back();
        }
        CK(c, cudaGraphLaunch(g->exec, c->stream), "graph launch");
        // an even number of steps swaps the buffers an even number of times
        c->steps += graph_steps;
        c->launches += g->launches;
        left -= graph_steps;
    }
    return step_cfl_direct(c, cfl, left);
}

}  // extern "C"

// Checkpoint file (little-endian): a 56-byte header (magic "PPMLRCK1",
// u32 version 1, u32 precision, i32 n[3], i32 0, i64 step, f64 simulated
// time, f64 gamma), the grid edges of x, y, z (n[d] + 1 doubles each), the
// 8 state arrays (n0*n1*n2 doubles each, x fastest), then a u64 checksum:
// FNV-1a over the preceding bytes taken as 64-bit words.
namespace {
struct CkHeader {
    char magic[8];
    uint32_t version, precision;
    int32_t n[3], reserved;
    int64_t step;
    double time, gamma;
};
static_assert(sizeof(CkHeader) == 56, "checkpoint header layout");
const char k_magic[8] = {'P', 'P', 'M', 'L', 'R', 'C', 'K', '1'};

struct Fnv64 {
    uint64_t h = 0xcbf29ce484222325ull;
    void add(const void *p, size_t bytes)      // bytes: a multiple of 8
    {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t k = 0; k + 8 <= bytes; k += 8) {
            uint64_t w;
            memcpy(&w, b + k, 8);
            h ^= w;
            h *= 0x100000001b3ull;
        }
    }
};

struct File {
    FILE *f = nullptr;
    ~File() { if (f) fclose(f); }
};

// Reads and verifies a checkpoint; `sink(v, data)` receives state array v.
// Returns nullptr or the reason it is not a valid checkpoint.
template <typename Sink>
const char *read_checkpoint(const char *path, CkHeader &h, std::vector<double> edges[3], Sink sink)
{
    File in;
    in.f = fopen(path, "rb");
    if (!in.f) return "checkpoint: cannot open the file";
    Fnv64 hash;
    if (fread(&h, sizeof(h), 1, in.f) != 1) return "checkpoint: truncated header";
    if (memcmp(h.magic, k_magic, 8) != 0 || h.version != 1) return "checkpoint: not a version-1 checkpoint";
    if (h.n[0] < 1 || h.n[1] < 1 || h.n[2] < 1 || (long long)h.n[0] * h.n[1] * h.n[2] > (1LL << 31) - 1)
        return "checkpoint: bad grid size";
    hash.add(&h, sizeof(h));
    for (int d = 0; d < 3; d++) {
        edges[d].resize((size_t)h.n[d] + 1);
        if (fread(edges[d].data(), sizeof(double), edges[d].size(), in.f) != edges[d].size())
            return "checkpoint: truncated edges";
        hash.add(edges[d].data(), sizeof(double) * edges[d].size());
    }
    const size_t ncell = (size_t)h.n[0] * h.n[1] * h.n[2];
    std::vector<double> buf(ncell);
    for (int v = 0; v < 8; v++) {
        if (fread(buf.data(), sizeof(double), ncell, in.f) != ncell) return "checkpoint: truncated state";
        hash.add(buf.data(), sizeof(double) * ncell);
        if (const char *why = sink(v, buf.data())) return why;
    }
    uint64_t sum = 0;
    if (fread(&sum, sizeof(sum), 1, in.f) != 1) return "checkpoint: missing checksum";
    if (fgetc(in.f) != EOF) return "checkpoint: trailing bytes";
    if (sum != hash.h) return "checkpoint: checksum mismatch";
    return nullptr;
}
}  // namespace

extern "C" {

ppmlr_status ppmlr_checkpoint_save(ppmlr_ctx *c, const char *path)
{
    if (!c) return PPMLR_E_INVALID;
    if (!path || !*path) return fail(c, PPMLR_E_INVALID, "checkpoint_save: empty path");
    double t = 0.0;
    ppmlr_status st = ppmlr_get_time(c, &t);
    if (st != PPMLR_OK) return st;
    CkHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, k_magic, 8);
    h.version = 1;
    h.precision = (uint32_t)c->prec;
    for (int d = 0; d < 3; d++) h.n[d] = c->n[d];
    h.step = c->steps;
    h.time = t;
    h.gamma = c->gamma;
    const std::string tmp = std::string(path) + ".part";
    File out;
    out.f = fopen(tmp.c_str(), "wb");
    if (!out.f) return fail(c, PPMLR_E_INVALID, "checkpoint_save: cannot create " + tmp);
    Fnv64 hash;
    bool ok = fwrite(&h, sizeof(h), 1, out.f) == 1;
    hash.add(&h, sizeof(h));
    for (int d = 0; d < 3 && ok; d++) {
        ok = fwrite(c->edges[d].data(), sizeof(double), c->edges[d].size(), out.f) == c->edges[d].size();
        hash.add(c->edges[d].data(), sizeof(double) * c->edges[d].size());
    }
    std::vector<double> buf((size_t)c->ncell);
    for (int v = 0; v < 8 && ok; v++) {
        cudaError_t e = cudaMemcpyAsync(buf.data(), c->U[v], sizeof(double) * buf.size(), cudaMemcpyDeviceToHost,
                                        c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {            // no partial file left behind
            fclose(out.f);
            out.f = nullptr;
            remove(tmp.c_str());
            return cuda_fail(c, e, "checkpoint copy");
        }
        ok = fwrite(buf.data(), sizeof(double), buf.size(), out.f) == buf.size();
        hash.add(buf.data(), sizeof(double) * buf.size());
    }
    if (ok) ok = fwrite(&hash.h, sizeof(hash.h), 1, out.f) == 1;
    if (fclose(out.f) != 0) ok = false;
    out.f = nullptr;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return fail(c, PPMLR_E_INVALID, std::string("checkpoint_save: write failed for ") + path);
    }
    return read_flags(c);
}

ppmlr_status ppmlr_checkpoint_load(ppmlr_ctx *c, const char *path)
{
    if (!c) return PPMLR_E_INVALID;
    if (!path) return fail(c, PPMLR_E_INVALID, "checkpoint_load: null path");
    CK(c, cudaStreamSynchronize(c->stream), "stream sync");
    CkHeader h;
    std::vector<double> edges[3];
    cudaError_t ce = cudaSuccess;
    // the arrays go to the output buffers first: the state changes only once
    // the whole file has been verified
    const char *why = read_checkpoint(path, h, edges, [&](int v, const double *data) -> const char * {
        if (v == 0) {
            for (int d = 0; d < 3; d++)
                if (h.n[d] != c->n[d]) return "checkpoint: grid size differs from the context's";
            for (int d = 0; d < 3; d++)
                if (memcmp(edges[d].data(), c->edges[d].data(), sizeof(double) * edges[d].size()) != 0)
                    return "checkpoint: grid edges differ from the context's";
            if (!(h.gamma == c->gamma)) return "checkpoint: gamma differs from the context's";
        }
        ce = cudaMemcpy(c->Un[v], data, sizeof(double) * (size_t)c->ncell, cudaMemcpyHostToDevice);
        return ce == cudaSuccess ? nullptr : "checkpoint: device copy failed";
    });
    if (ce != cudaSuccess) return cuda_fail(c, ce, "checkpoint copy");
    if (why) return fail(c, PPMLR_E_INVALID, why);
    for (int v = 0; v < 8; v++) { double *tmp = c->U[v]; c->U[v] = c->Un[v]; c->Un[v] = tmp; }
    c->steps = h.step;
    CK(c, cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream), "flags reset");
    return put_device_time(c, h.time);
}

ppmlr_status ppmlr_checkpoint_info(const char *path, int n[3], long long *step, double *time, int *precision)
{
    if (!path) return PPMLR_E_INVALID;
    CkHeader h;
    std::vector<double> edges[3];
    if (read_checkpoint(path, h, edges, [](int, const double *) -> const char * { return nullptr; }))
        return PPMLR_E_INVALID;
    if (n) for (int d = 0; d < 3; d++) n[d] = h.n[d];
    if (step) *step = h.step;
    if (time) *time = h.time;
    if (precision) *precision = (int)h.precision;
    return PPMLR_OK;
}

}  // extern "C"
