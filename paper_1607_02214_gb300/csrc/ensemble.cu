// Batched ensemble: many independent magnetosphere instances (different
// grids, solar-wind and IMF inputs) advanced together.  Each step is one
// ensemble CFL launch (a per-instance dt on the device) and one persistent
// sweep launch per direction whose blocks take (instance, tile) items from a
// global work counter; the whole step is captured once as a CUDA graph (one
// graph for x,y,z steps, one for z,y,x steps) and replayed.
//
// State buffers: every instance owns two sets of 8 arrays, A and B.  Even
// steps start in A and end in B (sweeps read A, B, A), odd steps start in B
// and end in A; the sweep arguments hold A as input and B as output and a
// per-launch flip swaps them.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <tuple>
#include <vector>

#include "ppmlr_internal.h"

using namespace ppmlr;

struct ppmlr_ens {
    int count;
    ppmlr_precision prec;
    double gamma;
    cudaStream_t stream;
    cudaStream_t cap;            // private stream used for graph capture
    int device, sms;
    std::vector<int> n;          // 3 per instance
    std::vector<long long> ncell;
    std::vector<ppmlr_bc> bc;
    int riemann_iters;           // 0: two-wave Riemann solver; k > 0: k two-shock Newton steps
    int steepen;                 // 1: contact steepening in the remap
    double *state;               // all instances, A and B sets
    std::vector<double *> A, B;  // 8 per instance
    double *geo;                 // per instance: w[3], c[3] (double)
    float *geof;                 // float copies
    double *dt;                  // per instance
    double *partial;             // CFL block minima, all instances
    unsigned int *tickets;       // CFL tickets, one per instance
    unsigned int *queue;         // three sweep work counters
    int *flags;
    unsigned long long *floors;
    // per direction
    SweepArgs *d_args[3];
    int *d_first_tile[3];
    int total_tiles[3], threads[3], blocks[3];
    size_t smem[3];
    int maxt[3];                 // tile thread budget chosen per direction
    int lanes_first[3];          // y/z tile rule: 1 = most lanes, pencils chunked to >= 48 cells
    int mode[3];                 // 0: persistent work queue, 1: one block per tile (table),
                                 // 2: one block per tile (arguments in the kernel parameter),
                                 // 3: one block per tile, input box staged by TMA (y, z),
                                 // 4: persistent work queue, arguments in the kernel parameter,
                                 // 5: one block per tile, input box staged by TMA, arguments in
                                 //    the kernel parameter
    CUtensorMap *d_maps[3];      // modes 3, 5: per instance the maps of its two state sets
    std::vector<SweepArgs> host_args[3];
    std::vector<Tile> tiles[3];
    // CFL tables for states in A and in B
    CflArgs *d_cfl[2];
    int *d_first_block;
    int cfl_blocks;
    // graphs
    cudaGraphExec_t exec[2];
    double graph_cfl;
    bool graphs_ok;
    long long steps, launches;
    std::string err;
    void *dev_alloc;             // single allocation for the small tables
};

static ppmlr_status efail(ppmlr_ens *e, ppmlr_status s, const std::string &m)
{
    if (e) e->err = m;
    return s;
}

#define ECK(e, call, what)                                                                   \
    do {                                                                                     \
        cudaError_t r_ = (call);                                                             \
        if (r_ != cudaSuccess)                                                               \
            return efail(e, r_ == cudaErrorMemoryAllocation ? PPMLR_E_OOM : PPMLR_E_CUDA,    \
                         std::string(what) + ": " + cudaGetErrorString(r_));                 \
    } while (0)

static size_t real_size(const ppmlr_ens *e) { return e->prec == PPMLR_MIXED ? sizeof(float) : sizeof(double); }

// Tile shapes of every instance for one direction under a thread budget;
// false (nothing changed) when `mode` cannot serve every instance.
// Tile of one instance along d within `maxt` positions x lanes.  Default
// rule: whole pencils when they fit (else equal chunks), then as many lanes
// as fit (y/z: a power of two up to 16, at most 2 nx).  lanes_first (y/z):
// the most lanes (power of two up to 16) for which chunks of at least
// min(N, 48) cells fit, then the fewest equal chunks.
static void pick_tile(const int *n, int d, int maxt, bool lanes_first, int &C, int &L)
{
    const int N = n[d];
    if (lanes_first && d != 0) {
        const int cmin = N < 48 ? N : 48;
        L = 1;
        for (int l = 16; l >= 2; l /= 2) {
            if (l / 2 >= n[0]) continue;
            if (maxt / l - 2 * GH >= cmin) { L = l; break; }
        }
        const int cmax = maxt / L - 2 * GH;
        int nchunk = (N + cmax - 1) / cmax;
        if (nchunk < 1) nchunk = 1;
        C = (N + nchunk - 1) / nchunk;
        return;
    }
    int nchunk = 1;
    C = N;
    while (C + 2 * GH > maxt) { nchunk++; C = (N + nchunk - 1) / nchunk; }
    L = maxt / (C + 2 * GH);
    if (L < 1) L = 1;
    if (d != 0) {
        int p2 = 1;
        while (p2 * 2 <= L && p2 * 2 <= 16) p2 *= 2;
        while (p2 > 1 && p2 / 2 >= n[0]) p2 /= 2;
        L = p2;
    }
}

static bool plan_direction(ppmlr_ens *e, int d, int maxt, int mode, bool lanes_first = false)
{
    if ((mode == 2 || mode == 4 || mode == 5) && e->count > ENS_PARAM_MAX) return false;
    if (mode == 3 || mode == 5) {     // TMA staging: every instance's box within the copy engine's rules
        if (!tensor_map_encoder()) return false;
        size_t sm = 0;
        int thr = 32;
        for (int i = 0; i < e->count; i++) {
            const int *n = &e->n[3 * i];
            int C, L;
            pick_tile(n, d, maxt, lanes_first, C, L);
            const Tile t = make_tile(d, n, real_size(e), C, L);
            if (n[0] & 1) return false;
            if (d == 0 && ((t.C & 1) || t.NP + 2 > 256 || n[1] % t.L)) return false;   // x: even origin, one z plane
            if (d != 0 && (t.L < 2 || (t.L & 1) || t.NP > 256)) return false;
            sm = std::max(sm, stage_pad_bytes(t, d) + t.smem);
            thr = std::max(thr, t.threads);
        }
        const int fit = mode == 5 ? sweep_launchers(e->prec).ens_tma_param_per_sm(d, thr, sm)
                                  : sweep_launchers(e->prec).ens_tma_per_sm(d, thr, sm);
        if (sm > 224 * 1024 || fit < 1) return false;
    }
    e->maxt[d] = maxt;
    e->mode[d] = mode;
    e->lanes_first[d] = lanes_first && d != 0 ? 1 : 0;
    e->tiles[d].clear();
    int thr = 32;
    size_t sm = 0;
    int total = 0;
    for (int i = 0; i < e->count; i++) {
        const int *n = &e->n[3 * i];
        int C, L;
        pick_tile(n, d, maxt, lanes_first, C, L);
        Tile t = make_tile(d, n, real_size(e), C, L);
        e->tiles[d].push_back(t);
        if (t.threads > thr) thr = t.threads;
        const size_t need = mode == 3 || mode == 5 ? stage_pad_bytes(t, d) + t.smem : t.smem;
        if (need > sm) sm = need;
        total += t.ntiles;
    }
    e->threads[d] = thr;
    e->smem[d] = sm;
    e->total_tiles[d] = total;
    const bool persist = mode == 0 || mode == 4;
    int per_sm = mode == 4 ? sweep_launchers(e->prec).param_persist_per_sm(d, thr, sm)
                           : sweep_launchers(e->prec).per_sm(d, thr, sm);
    int b = per_sm * e->sms;
    e->blocks[d] = (!persist || b > total) ? total : b;
    if (persist && e->blocks[d] == total && total > 1) e->blocks[d] = total - 1;   // keep it persistent
    return true;
}

// Tensor maps of every instance's two state sets for the TMA form along d:
// a 4D view (x, y, z, variable) with box L lanes x NP positions x 8 arrays
// (x: NP + 2 cells x L pencils x 8 arrays).
static ppmlr_status upload_maps(ppmlr_ens *e, int d)
{
    std::vector<CUtensorMap> maps(2 * (size_t)e->count);
    for (int i = 0; i < e->count; i++) {
        const int *n = &e->n[3 * i];
        const Tile &t = e->tiles[d][i];
        const long long vs = (long long)(e->A[8 * i + 1] - e->A[8 * i]);
        const cuuint64_t dims[4] = {(cuuint64_t)n[0], (cuuint64_t)n[1], (cuuint64_t)n[2], 8};
        const cuuint64_t strides[3] = {(cuuint64_t)n[0] * 8, (cuuint64_t)n[0] * n[1] * 8, (cuuint64_t)vs * 8};
        cuuint32_t box[4] = {(cuuint32_t)t.L, 1, 1, 8};
        box[d] = (cuuint32_t)t.NP;
        if (d == 0) { box[0] = (cuuint32_t)(t.NP + 2); box[1] = (cuuint32_t)t.L; }
        const cuuint32_t es[4] = {1, 1, 1, 1};
        for (int b = 0; b < 2; b++) {
            void *base = b == 0 ? e->A[8 * i] : e->B[8 * i];
            CUresult r = tensor_map_encoder()(&maps[2 * i + b], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, base, dims, strides,
                                              box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return efail(e, PPMLR_E_INVALID, "ensemble: tensor map rejected");
        }
    }
    if (!e->d_maps[d]) ECK(e, cudaMalloc(&e->d_maps[d], sizeof(CUtensorMap) * maps.size()), "tensor map table");
    ECK(e, cudaMemcpyAsync(e->d_maps[d], maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                           e->stream), "tensor map upload");
    return PPMLR_OK;
}

// Upload the per-instance sweep arguments and first-tile table of a direction.
static ppmlr_status upload_direction(ppmlr_ens *e, int d)
{
    std::vector<SweepArgs> args(e->count);
    std::vector<int> first(e->count);
    int acc = 0;
    size_t goff = 0;
    for (int i = 0; i < e->count; i++) {
        const int *n = &e->n[3 * i];
        SweepArgs a;
        memset(&a, 0, sizeof(a));
        a.U = e->A[8 * i]; a.Un = e->B[8 * i]; a.vs = (long long)(e->A[8 * i + 1] - e->A[8 * i]);
        for (int k = 0; k < 3; k++) a.n[k] = n[k];
        const Tile &t = e->tiles[d][i];
        a.N = n[d]; a.C = t.C; a.L = t.L; a.NP = t.NP; a.nchunk = t.nchunk; a.ngx = t.ngx;
        // geometry block of instance i: w0, c0, w1, c1, w2, c2 (each n + 2GH)
        size_t o[6], q = goff;
        for (int k = 0; k < 3; k++) { o[2 * k] = q; q += n[k] + 2 * GH; o[2 * k + 1] = q; q += n[k] + 2 * GH; }
        a.w = e->geo + o[2 * d]; a.c = e->geo + o[2 * d + 1];
        a.cx = e->geo + o[1]; a.cy = e->geo + o[3]; a.cz = e->geo + o[5];
        a.wf = e->geof + o[2 * d];
        a.cxf = e->geof + o[1]; a.cyf = e->geof + o[3]; a.czf = e->geof + o[5];
        goff = q;
        const ppmlr_bc &b = e->bc[i];
        a.bc_lo = b.face[d][0]; a.bc_hi = b.face[d][1];
        double infl[8] = {b.inflow.rho, b.inflow.v[0], b.inflow.v[1], b.inflow.v[2],
                          b.inflow.B[0], b.inflow.B[1], b.inflow.B[2], b.inflow.p};
        double inn[8] = {b.inner.rho, b.inner.v[0], b.inner.v[1], b.inner.v[2], 0.0, 0.0, 0.0, b.inner.p};
        memcpy(a.inflow, infl, sizeof(infl));
        memcpy(a.inner, inn, sizeof(inn));
        a.gamma = e->gamma; a.p_min = b.p_min; a.M = b.dipole_moment; a.r_inner = b.r_inner;
        a.powell = b.powell ? 1 : 0;
        a.do_src = (a.M != 0.0 || a.powell) ? 1 : 0;
        a.riemann_iters = e->riemann_iters;
        a.steepen = e->steepen;
        a.dt = 0.0; a.dt_dev = e->dt + i;
        a.flags = e->flags; a.floors = e->floors;
        a.gammaf = (float)a.gamma; a.p_minf = (float)a.p_min; a.Mf = (float)a.M; a.r_innerf = (float)a.r_inner;
        for (int k = 0; k < 8; k++) a.inflowf[k] = (float)a.inflow[k];
        a.p_reff = e->prec == PPMLR_MIXED ? mixed_pressure_reference(b) : 0.0f;
        args[i] = a;
        first[i] = acc;
        acc += t.ntiles;
    }
    e->host_args[d] = args;
    if (e->mode[d] == 3 || e->mode[d] == 5) {
        ppmlr_status st = upload_maps(e, d);
        if (st != PPMLR_OK) return st;
    }
    ECK(e, cudaMemcpyAsync(e->d_args[d], args.data(), sizeof(SweepArgs) * e->count, cudaMemcpyHostToDevice,
                           e->stream), "ensemble args upload");
    ECK(e, cudaMemcpyAsync(e->d_first_tile[d], first.data(), sizeof(int) * e->count, cudaMemcpyHostToDevice,
                           e->stream), "ensemble tile table upload");
    ECK(e, cudaStreamSynchronize(e->stream), "ensemble upload sync");
    return PPMLR_OK;
}

// One ensemble sweep launch along d in the direction's launch form.
static cudaError_t launch_dir(ppmlr_ens *e, int d, int flip, unsigned int *queue, cudaStream_t s)
{
    const SweepLaunchers &L = sweep_launchers(e->prec);
    if (e->mode[d] == 2 || e->mode[d] == 4 || e->mode[d] == 5) {
        EnsSweepParams p;
        memset(&p, 0, sizeof(p));
        for (int i = 0; i < e->count; i++) p.args[i] = e->host_args[d][i];
        int acc = 0;
        for (int i = 0; i < e->count; i++) { p.first_tile[i] = acc; acc += e->tiles[d][i].ntiles; }
        p.count = e->count;
        p.flip = flip;
        p.total_tiles = acc;
        if (e->mode[d] == 4) return L.param_persist(d, p, queue, e->blocks[d], e->threads[d], e->smem[d], s);
        if (e->mode[d] == 5) return L.ens_tma_param(d, p, e->d_maps[d], e->blocks[d], e->threads[d], e->smem[d], s);
        return L.param(d, p, e->blocks[d], e->threads[d], e->smem[d], s);
    }
    EnsSweepArgs ea{e->d_args[d], e->d_first_tile[d], e->count, e->total_tiles[d], flip, queue};
    if (e->mode[d] == 3) return L.ens_tma(d, ea, e->d_maps[d], e->blocks[d], e->threads[d], e->smem[d], s);
    return L.ens(d, ea, e->blocks[d], e->threads[d], e->smem[d], s);
}

// Enqueue one step (parity 0: x,y,z from A; 1: z,y,x from B) on stream s.
static ppmlr_status enqueue_step(ppmlr_ens *e, int parity, double cfl, cudaStream_t s)
{
    ECK(e, cudaMemsetAsync(e->queue, 0, 3 * sizeof(unsigned int), s), "queue reset");
    EnsCflArgs ca;
    ca.args = e->d_cfl[parity];
    ca.first_block = e->d_first_block;
    ca.count = e->count;
    (void)cfl;   // the CFL number is part of the uploaded CflArgs tables
    cudaError_t r = cfl_launchers(e->prec).ens(ca, e->cfl_blocks, s);
    ECK(e, r, "ensemble cfl launch");
    e->launches++;
    const int ord[2][3] = {{0, 1, 2}, {2, 1, 0}};
    const int flip[2][3] = {{0, 1, 0}, {1, 0, 1}};
    for (int k = 0; k < 3; k++) {
        const int d = ord[parity][k];
        r = launch_dir(e, d, flip[parity][k], e->queue + k, s);
        ECK(e, r, "ensemble sweep launch");
        e->launches++;
    }
    return PPMLR_OK;
}

static ppmlr_status upload_cfl(ppmlr_ens *e, double cfl)
{
    std::vector<CflArgs> tab[2];
    std::vector<int> first(e->count);
    int acc = 0;
    size_t goff = 0, poff = 0;
    for (int i = 0; i < e->count; i++) {
        const int *n = &e->n[3 * i];
        long long nb = (e->ncell[i] + cfl_threads() - 1) / cfl_threads();
        if (nb > 64) nb = 64;
        size_t o[6], q = goff;
        for (int k = 0; k < 3; k++) { o[2 * k] = q; q += n[k] + 2 * GH; o[2 * k + 1] = q; q += n[k] + 2 * GH; }
        for (int side = 0; side < 2; side++) {
            CflArgs a;
            memset(&a, 0, sizeof(a));
            for (int v = 0; v < 8; v++) a.U[v] = side == 0 ? e->A[8 * i + v] : e->B[8 * i + v];
            for (int k = 0; k < 3; k++) {
                a.n[k] = n[k];
                a.w[k] = e->geo + o[2 * k]; a.c[k] = e->geo + o[2 * k + 1];
                a.wf[k] = e->geof + o[2 * k]; a.cf[k] = e->geof + o[2 * k + 1];
            }
            const ppmlr_bc &b = e->bc[i];
            a.gamma = e->gamma; a.p_min = b.p_min; a.M = b.dipole_moment; a.r_inner = b.r_inner;
            a.cfl = cfl;
            a.gammaf = (float)a.gamma; a.p_minf = (float)a.p_min; a.Mf = (float)a.M; a.r_innerf = (float)a.r_inner;
            a.partial = e->partial + poff;
            a.counter = e->tickets + i;
            a.dt_out = e->dt + i;
            tab[side].push_back(a);
        }
        goff = q;
        poff += (size_t)nb;
        first[i] = acc;
        acc += (int)nb;
    }
    e->cfl_blocks = acc;
    for (int side = 0; side < 2; side++)
        ECK(e, cudaMemcpyAsync(e->d_cfl[side], tab[side].data(), sizeof(CflArgs) * e->count,
                               cudaMemcpyHostToDevice, e->stream), "cfl table upload");
    ECK(e, cudaMemcpyAsync(e->d_first_block, first.data(), sizeof(int) * e->count, cudaMemcpyHostToDevice,
                           e->stream), "cfl block table upload");
    ECK(e, cudaStreamSynchronize(e->stream), "cfl upload sync");
    return PPMLR_OK;
}

static void drop_graphs(ppmlr_ens *e)
{
    for (int k = 0; k < 2; k++)
        if (e->exec[k]) { cudaGraphExecDestroy(e->exec[k]); e->exec[k] = nullptr; }
    e->graphs_ok = false;
}

static ppmlr_status build_graphs(ppmlr_ens *e, double cfl)
{
    drop_graphs(e);
    ppmlr_status st = upload_cfl(e, cfl);
    if (st != PPMLR_OK) return st;
    for (int parity = 0; parity < 2; parity++) {
        cudaGraph_t g = nullptr;
        ECK(e, cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        long long l0 = e->launches;
        st = enqueue_step(e, parity, cfl, e->cap);
        e->launches = l0;
        cudaError_t r = cudaStreamEndCapture(e->cap, &g);
        if (st != PPMLR_OK) { if (g) cudaGraphDestroy(g); return st; }
        ECK(e, r, "end capture");
        r = cudaGraphInstantiate(&e->exec[parity], g, 0);
        cudaGraphDestroy(g);
        ECK(e, r, "graph instantiate");
    }
    e->graph_cfl = cfl;
    e->graphs_ok = true;
    return PPMLR_OK;
}

extern "C" {

ppmlr_status ppmlr_ensemble_create(int count, const ppmlr_grid *grids, const ppmlr_bc *bcs, double gamma,
                                   ppmlr_precision prec, void *cuda_stream, ppmlr_ens **out)
{
    if (!out) return PPMLR_E_INVALID;
    *out = nullptr;
    if (count < 1 || !grids || !bcs || !(gamma > 1.0) ||
        (prec != PPMLR_FP64 && prec != PPMLR_MIXED && prec != PPMLR_FP64_EXACT))
        return PPMLR_E_INVALID;
    for (int i = 0; i < count; i++)
        if (!validate_grid_bc(&grids[i], &bcs[i])) return PPMLR_E_INVALID;
    ppmlr_ens *e = new ppmlr_ens();
    e->count = count; e->prec = prec; e->gamma = gamma;
    e->stream = (cudaStream_t)cuda_stream;
    e->steps = 0; e->launches = 0; e->graphs_ok = false; e->graph_cfl = 0.0;
    e->exec[0] = e->exec[1] = nullptr;
    e->state = nullptr; e->geo = nullptr; e->geof = nullptr; e->dev_alloc = nullptr; e->cap = nullptr;
    if (cudaGetDevice(&e->device) != cudaSuccess) { delete e; return PPMLR_E_CUDA; }
    e->sms = 152;
    cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, e->device);
    size_t total = 0, geo_total = 0;
    for (int i = 0; i < count; i++) {
        for (int k = 0; k < 3; k++) { e->n.push_back(grids[i].n[k]); geo_total += 2 * (grids[i].n[k] + 2 * GH); }
        long long nc = (long long)grids[i].n[0] * grids[i].n[1] * grids[i].n[2];
        e->ncell.push_back(nc);
        e->bc.push_back(bcs[i]);
        total += ((size_t)nc + 31) / 32 * 32;
    }
    auto cleanup = [&](ppmlr_status s) { ppmlr_ensemble_destroy(e); return s; };
    if (cudaMalloc(&e->state, sizeof(double) * total * 16) != cudaSuccess) return cleanup(PPMLR_E_OOM);
    {
        size_t off = 0;
        for (int i = 0; i < count; i++) {
            size_t stride = ((size_t)e->ncell[i] + 31) / 32 * 32;
            for (int v = 0; v < 8; v++) e->A.push_back(e->state + off + v * stride);
            for (int v = 0; v < 8; v++) e->B.push_back(e->state + off + (8 + v) * stride);
            off += 16 * stride;
        }
    }
    // geometry
    std::vector<double> host;
    for (int i = 0; i < count; i++)
        for (int k = 0; k < 3; k++) {
            std::vector<double> w, ce;
            build_axis(grids[i].n[k], grids[i].edges[k], bcs[i].face[k][0], bcs[i].face[k][1], w, ce);
            host.insert(host.end(), w.begin(), w.end());
            host.insert(host.end(), ce.begin(), ce.end());
        }
    std::vector<float> hostf(host.begin(), host.end());
    if (cudaMalloc(&e->geo, sizeof(double) * geo_total) != cudaSuccess) return cleanup(PPMLR_E_OOM);
    if (cudaMalloc(&e->geof, sizeof(float) * geo_total) != cudaSuccess) return cleanup(PPMLR_E_OOM);
    // small tables: dt, partials (<= 64 per instance), tickets, queue, flags,
    // floors, sweep args and tile tables, CFL tables; laid out twice: a dry
    // run from address 0 gives the size, the second pass assigns pointers
    size_t bytes = 0;
    for (int pass = 0; pass < 2; pass++) {
        unsigned char *base = pass == 0 ? nullptr : (unsigned char *)e->dev_alloc;
        size_t off = 0;
        auto take = [&](size_t nb) { unsigned char *r = base + off; off += (nb + 255) / 256 * 256; return r; };
        e->dt = (double *)take(sizeof(double) * count);
        e->partial = (double *)take(sizeof(double) * 64 * count);
        e->tickets = (unsigned int *)take(sizeof(unsigned) * count);
        e->queue = (unsigned int *)take(16);
        e->flags = (int *)take(8);
        e->floors = (unsigned long long *)take(8);
        for (int d = 0; d < 3; d++) {
            e->d_args[d] = (SweepArgs *)take(sizeof(SweepArgs) * count);
            e->d_first_tile[d] = (int *)take(sizeof(int) * count);
        }
        e->d_cfl[0] = (CflArgs *)take(sizeof(CflArgs) * count);
        e->d_cfl[1] = (CflArgs *)take(sizeof(CflArgs) * count);
        e->d_first_block = (int *)take(sizeof(int) * count);
        if (pass == 0) {
            bytes = off;
            if (cudaMalloc(&e->dev_alloc, bytes) != cudaSuccess) return cleanup(PPMLR_E_OOM);
        }
    }
    if (cudaMemsetAsync(e->dev_alloc, 0, bytes, e->stream) != cudaSuccess) return cleanup(PPMLR_E_CUDA);
    if (cudaMemsetAsync(e->state, 0, sizeof(double) * total * 16, e->stream) != cudaSuccess)
        return cleanup(PPMLR_E_CUDA);
    if (cudaMemcpyAsync(e->geo, host.data(), sizeof(double) * geo_total, cudaMemcpyHostToDevice, e->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(e->geof, hostf.data(), sizeof(float) * geo_total, cudaMemcpyHostToDevice, e->stream) !=
            cudaSuccess)
        return cleanup(PPMLR_E_CUDA);
    if (cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking) != cudaSuccess) return cleanup(PPMLR_E_CUDA);
    const int default_maxt = prec == PPMLR_MIXED ? MAXT : MAXT_F64;
    for (int d = 0; d < 3; d++) {
        plan_direction(e, d, default_maxt, count <= ENS_PARAM_MAX ? 2 : 0);
        if (upload_direction(e, d) != PPMLR_OK) return cleanup(PPMLR_E_CUDA);
    }
    if (cudaStreamSynchronize(e->stream) != cudaSuccess) return cleanup(PPMLR_E_CUDA);
    *out = e;
    return PPMLR_OK;
}

void ppmlr_ensemble_destroy(ppmlr_ens *e)
{
    if (!e) return;
    cudaStreamSynchronize(e->stream);
    drop_graphs(e);
    if (e->cap) cudaStreamDestroy(e->cap);
    cudaFree(e->dev_alloc);
    for (int d = 0; d < 3; d++) cudaFree(e->d_maps[d]);
    cudaFree(e->geof);
    cudaFree(e->geo);
    cudaFree(e->state);
    delete e;
}

const char *ppmlr_ensemble_last_error(const ppmlr_ens *e) { return e ? e->err.c_str() : "null ensemble"; }

long long ppmlr_ensemble_launch_count(const ppmlr_ens *e) { return e ? e->launches : 0; }

ppmlr_status ppmlr_ensemble_set_state(ppmlr_ens *e, int i, const double *const U[8], int on_device)
{
    if (!e) return PPMLR_E_INVALID;
    if (i < 0 || i >= e->count || !U) return efail(e, PPMLR_E_INVALID, "ensemble_set_state: bad index or arrays");
    for (int v = 0; v < 8; v++)
        if (!U[v]) return efail(e, PPMLR_E_INVALID, "ensemble_set_state: null array");
    double *const *dst = (e->steps & 1) ? &e->B[8 * i] : &e->A[8 * i];
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int v = 0; v < 8; v++)
        ECK(e, cudaMemcpyAsync(dst[v], U[v], sizeof(double) * e->ncell[i], kind, e->stream), "set_state copy");
    if (!on_device) ECK(e, cudaStreamSynchronize(e->stream), "set_state sync");
    return PPMLR_OK;
}

static ppmlr_status ens_flags(ppmlr_ens *e)
{
    int f = 0;
    ECK(e, cudaMemcpyAsync(&f, e->flags, sizeof(int), cudaMemcpyDeviceToHost, e->stream), "flags copy");
    ECK(e, cudaStreamSynchronize(e->stream), "stream sync");
    if (f) {
        ECK(e, cudaMemsetAsync(e->flags, 0, sizeof(int), e->stream), "flags reset");
        if (f & FLAG_BOUNDS) return efail(e, PPMLR_E_BOUNDS, "checked build: a kernel index left its array");
        if (f & FLAG_TIMEOUT) return efail(e, PPMLR_E_TIMEOUT, "a bounded device wait gave up");
        if (f & FLAG_NONFINITE) return efail(e, PPMLR_E_NONFINITE, "a sweep produced a non-finite state");
        return efail(e, PPMLR_E_CFL, "time step too large for the CFL condition");
    }
    return PPMLR_OK;
}

ppmlr_status ppmlr_ensemble_get_state(ppmlr_ens *e, int i, double *const U[8], int on_device)
{
    if (!e) return PPMLR_E_INVALID;
    if (i < 0 || i >= e->count || !U) return efail(e, PPMLR_E_INVALID, "ensemble_get_state: bad index or arrays");
    for (int v = 0; v < 8; v++)
        if (!U[v]) return efail(e, PPMLR_E_INVALID, "ensemble_get_state: null array");
    double *const *src = (e->steps & 1) ? &e->B[8 * i] : &e->A[8 * i];
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int v = 0; v < 8; v++)
        ECK(e, cudaMemcpyAsync(U[v], src[v], sizeof(double) * e->ncell[i], kind, e->stream), "get_state copy");
    return ens_flags(e);
}

ppmlr_status ppmlr_ensemble_step(ppmlr_ens *e, double cfl, int nsteps)
{
    if (!e) return PPMLR_E_INVALID;
    if (!(cfl > 0.0) || nsteps < 0) return efail(e, PPMLR_E_INVALID, "ensemble_step: need cfl > 0, nsteps >= 0");
    if (!e->graphs_ok || e->graph_cfl != cfl) {
        ppmlr_status st = build_graphs(e, cfl);
        if (st != PPMLR_OK) return st;
    }
    for (int k = 0; k < nsteps; k++) {
        ECK(e, cudaGraphLaunch(e->exec[e->steps & 1], e->stream), "graph launch");
        e->launches += 4;
        e->steps++;
    }
    return PPMLR_OK;
}

ppmlr_status ppmlr_ensemble_check(ppmlr_ens *e)
{
    if (!e) return PPMLR_E_INVALID;
    return ens_flags(e);
}

ppmlr_status ppmlr_ensemble_get_dt(ppmlr_ens *e, double *dt_out)
{
    if (!e) return PPMLR_E_INVALID;
    if (!dt_out) return efail(e, PPMLR_E_INVALID, "ensemble_get_dt: null output");
    ECK(e, cudaMemcpyAsync(dt_out, e->dt, sizeof(double) * e->count, cudaMemcpyDeviceToHost, e->stream), "dt copy");
    ECK(e, cudaStreamSynchronize(e->stream), "stream sync");
    return PPMLR_OK;
}

ppmlr_status ppmlr_ensemble_get_diagnostics(ppmlr_ens *e, long long *step, long long *floor_hits)
{
    if (!e) return PPMLR_E_INVALID;
    unsigned long long fl = 0;
    ECK(e, cudaMemcpyAsync(&fl, e->floors, sizeof(fl), cudaMemcpyDeviceToHost, e->stream), "floors copy");
    ECK(e, cudaStreamSynchronize(e->stream), "stream sync");
    if (step) *step = e->steps;
    if (floor_hits) *floor_hits = (long long)fl;
    return PPMLR_OK;
}

ppmlr_status ppmlr_ensemble_set_stream(ppmlr_ens *e, void *stream)
{
    if (!e) return PPMLR_E_INVALID;
    e->stream = (cudaStream_t)stream;
    return PPMLR_OK;
}

// Autotuner: for each direction try thread budgets for the tiles of all
// instances, time the persistent sweep on the current state (out of place:
// the state is not modified), keep the fastest, then rebuild the graphs.
// Results do not depend on the tile shapes (each cell's arithmetic is the
// same), only the speed does.  best_ms receives the tuned time per direction.
ppmlr_status ppmlr_ensemble_autotune(ppmlr_ens *e, double *best_ms)
{
    if (!e) return PPMLR_E_INVALID;
    const int cands_mixed[] = {128, 192, 256, 320, 384, 448, 512};
    const int cands_f64[] = {128, 192, 256, 320, 384, 448};
    const int *cands = e->prec == PPMLR_MIXED ? cands_mixed : cands_f64;
    const int nc = e->prec == PPMLR_MIXED ? 7 : 6;
    unsigned long long floors_before = 0;
    ECK(e, cudaMemcpyAsync(&floors_before, e->floors, sizeof(floors_before), cudaMemcpyDeviceToHost, e->stream),
        "floors copy");
    ECK(e, cudaStreamSynchronize(e->stream), "sync");
    cudaEvent_t t0, t1;
    ECK(e, cudaEventCreate(&t0), "event");
    ECK(e, cudaEventCreate(&t1), "event");
    // a valid dt for the timing runs
    {
        ppmlr_status st = upload_cfl(e, 0.4);
        if (st != PPMLR_OK) return st;
        EnsCflArgs ca{e->d_cfl[e->steps & 1], e->d_first_block, e->count};
        ECK(e, cfl_launchers(e->prec).ens(ca, e->cfl_blocks, e->stream), "cfl");
    }
    for (int d = 0; d < 3; d++) {
        float best = 1e30f;
        int best_t = e->maxt[d], best_m = e->mode[d], best_r = e->lanes_first[d];
        const int rules = d == 0 ? 1 : 2;
        // per candidate (budget, form, tile rule) the time of two sweeps
        std::vector<std::tuple<float, int, int, int>> timed;
        constexpr int NF = 6;           // launch forms 0..5
        for (int k = 0; k < NF * nc * rules; k++) {
            const int mode = (k / nc) % NF, rule = k / (NF * nc);
            if ((mode == 2 || mode == 4 || mode == 5) && e->count > ENS_PARAM_MAX) continue;
            if (!plan_direction(e, d, cands[k % nc], mode, rule == 1)) continue;
            ppmlr_status st = upload_direction(e, d);
            if (st != PPMLR_OK) return st;
            float tot = 0.0f;
            for (int rep = 0; rep < 3; rep++) {
                ECK(e, cudaMemsetAsync(e->queue, 0, sizeof(unsigned), e->stream), "queue");
                ECK(e, cudaEventRecord(t0, e->stream), "event");
                ECK(e, launch_dir(e, d, (int)(e->steps & 1), e->queue, e->stream), "tune launch");
                ECK(e, cudaEventRecord(t1, e->stream), "event");
                ECK(e, cudaEventSynchronize(t1), "event sync");
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, t0, t1);
                if (rep > 0) tot += ms;
            }
            timed.push_back({tot, cands[k % nc], mode, rule});
            if (tot < best) { best = tot; best_t = cands[k % nc]; best_m = mode; best_r = rule; }
        }
        // a persistent form (one launch of resident blocks taking tiles from
        // the work counter) is kept when it is within 2 % of the fastest
        if (best_m != 0 && best_m != 4) {
            float pbest = 1e30f;
            for (auto &tc : timed)
                if ((std::get<2>(tc) == 0 || std::get<2>(tc) == 4) && std::get<0>(tc) < pbest) {
                    pbest = std::get<0>(tc);
                    if (pbest <= 1.02f * best) {
                        best_t = std::get<1>(tc); best_m = std::get<2>(tc); best_r = std::get<3>(tc);
                    }
                }
            if (pbest <= 1.02f * best) best = pbest;
        }
        plan_direction(e, d, best_t, best_m, best_r == 1);
        ppmlr_status st = upload_direction(e, d);
        if (st != PPMLR_OK) return st;
        if (best_ms) best_ms[d] = best / 2.0f;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    // the tuning runs may have raised flags or counted floors on the discarded output
    ECK(e, cudaMemsetAsync(e->flags, 0, sizeof(int), e->stream), "flags reset");
    ECK(e, cudaMemcpyAsync(e->floors, &floors_before, sizeof(floors_before), cudaMemcpyHostToDevice, e->stream),
        "floors restore");
    ECK(e, cudaStreamSynchronize(e->stream), "sync");
    drop_graphs(e);
    return PPMLR_OK;
}

// nsteps steps with direct launches (no graph) and CUDA events around every
// kernel on the ensemble stream; avg_ms receives the mean time per launch of
// the x, y, z sweeps and the CFL pass.  Advances the state like ensemble_step.
ppmlr_status ppmlr_ensemble_time_kernels(ppmlr_ens *e, double cfl, int nsteps, double *avg_ms)
{
    if (!e) return PPMLR_E_INVALID;
    if (!avg_ms || !(cfl > 0.0) || nsteps < 1) return efail(e, PPMLR_E_INVALID, "time_kernels: bad arguments");
    ppmlr_status st = upload_cfl(e, cfl);
    if (st != PPMLR_OK) return st;
    drop_graphs(e);
    std::vector<cudaEvent_t> ev(8 * nsteps);
    for (auto &x : ev) ECK(e, cudaEventCreate(&x), "event");
    const int ord[2][3] = {{0, 1, 2}, {2, 1, 0}};
    const int flip[2][3] = {{0, 1, 0}, {1, 0, 1}};
    std::vector<int> kind(4 * nsteps);
    for (int k = 0; k < nsteps; k++) {
        const int parity = (int)(e->steps & 1);
        ECK(e, cudaMemsetAsync(e->queue, 0, 3 * sizeof(unsigned int), e->stream), "queue reset");
        EnsCflArgs ca{e->d_cfl[parity], e->d_first_block, e->count};
        ECK(e, cudaEventRecord(ev[8 * k], e->stream), "event");
        ECK(e, cfl_launchers(e->prec).ens(ca, e->cfl_blocks, e->stream), "cfl");
        ECK(e, cudaEventRecord(ev[8 * k + 1], e->stream), "event");
        kind[4 * k] = 3;
        for (int j = 0; j < 3; j++) {
            const int d = ord[parity][j];
            ECK(e, cudaEventRecord(ev[8 * k + 2 + 2 * j], e->stream), "event");
            ECK(e, launch_dir(e, d, flip[parity][j], e->queue + j, e->stream), "sweep");
            ECK(e, cudaEventRecord(ev[8 * k + 3 + 2 * j], e->stream), "event");
            kind[4 * k + 1 + j] = d;
        }
        e->launches += 4;
        e->steps++;
    }
    ECK(e, cudaStreamSynchronize(e->stream), "sync");
    double tot[4] = {0, 0, 0, 0};
    int cnt[4] = {0, 0, 0, 0};
    for (int k = 0; k < nsteps; k++)
        for (int j = 0; j < 4; j++) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, ev[8 * k + 2 * j], ev[8 * k + 2 * j + 1]);
            tot[kind[4 * k + j]] += ms;
            cnt[kind[4 * k + j]]++;
        }
    for (auto &x : ev) cudaEventDestroy(x);
    for (int j = 0; j < 4; j++) avg_ms[j] = cnt[j] ? tot[j] / cnt[j] : 0.0;
    return PPMLR_OK;
}

ppmlr_status ppmlr_ensemble_set_launch(ppmlr_ens *e, int axis, int form, int budget)
{
    if (!e) return PPMLR_E_INVALID;
    const int maxb = e->prec == PPMLR_MIXED ? MAXT : MAXT_F64;
    const bool lanes_first = budget >= 10000;
    if (lanes_first) budget -= 10000;
    if (axis < 0 || axis > 2 || form < 0 || form > 5 || budget < 2 * GH + 1 || budget > maxb ||
        (lanes_first && axis == 0))
        return efail(e, PPMLR_E_INVALID, "set_launch: bad axis, form or budget");
    if ((form == 2 || form == 4 || form == 5) && e->count > ENS_PARAM_MAX)
        return efail(e, PPMLR_E_INVALID, "set_launch: forms 2, 4 and 5 take at most 64 instances");
    if (!plan_direction(e, axis, budget, form, lanes_first))
        return efail(e, PPMLR_E_INVALID, "set_launch: the TMA form does not fit every instance along this axis");
    ppmlr_status st = upload_direction(e, axis);
    if (st != PPMLR_OK) return st;
    drop_graphs(e);
    return PPMLR_OK;
}

ppmlr_status ppmlr_ensemble_set_steepening(ppmlr_ens *e, int on)
{
    if (!e) return PPMLR_E_INVALID;
    e->steepen = on ? 1 : 0;
    for (int d = 0; d < 3; d++) {
        ppmlr_status st = upload_direction(e, d);
        if (st != PPMLR_OK) return st;
    }
    drop_graphs(e);
    return PPMLR_OK;
}

ppmlr_status ppmlr_ensemble_set_riemann_solver(ppmlr_ens *e, int iters)
{
    if (!e) return PPMLR_E_INVALID;
    if (iters < 0 || iters > 16) return efail(e, PPMLR_E_INVALID, "set_riemann_solver: iters must be in [0, 16]");
    e->riemann_iters = iters;
    for (int d = 0; d < 3; d++) {
        ppmlr_status st = upload_direction(e, d);
        if (st != PPMLR_OK) return st;
    }
    ECK(e, cudaStreamSynchronize(e->stream), "sync");
    drop_graphs(e);
    return PPMLR_OK;
}

ppmlr_status ppmlr_ensemble_get_tiles(ppmlr_ens *e, int *maxt_out)
{
    if (!e || !maxt_out) return PPMLR_E_INVALID;
    for (int d = 0; d < 3; d++) maxt_out[d] = 10000 * e->lanes_first[d] + 1000 * e->mode[d] + e->maxt[d];
    return PPMLR_OK;
}

}  // extern "C"
