// Allocation-free variant of the CFL time-step reduction.
//
// Why it exists: some programs that call this library must not allocate device
// memory themselves -- for example a host solver whose device memory is owned
// by another allocator that forbids raw cudaMalloc, or a coupling loop that
// must not risk the implicit device synchronisation an allocation can cause,
// or a caller running under a fixed device-memory budget.  Such callers hold
// no ppmlr context (creating one allocates), so this entry point takes every
// input and the output as caller-owned device memory and keeps its only
// scratch (one minimum per block plus a ticket counter) in a static device
// array of this file.
//
// Static scratch: every GPU that loads the library holds it until the process
// exits; every call on a device shares it and it keeps the last call's
// contents.  The ticket counter is cleared at the start of every call.  Calls
// whose kernels overlap on the GPU (different streams, or host threads) race
// on the scratch and must be serialised by the caller.
//
// Set-up: the first call on each device looks up the device address of the
// static array with cudaGetSymbolAddress (the host-side name of a __device__
// array is only a stand-in, not a device address) and caches it per device
// together with the unique ID of the CUDA context that was current then.  A
// later call under another context of that device (after cudaDeviceReset, or
// a context created and destroyed through the driver API) repeats the lookup,
// since the module and its array may then sit at another address.  Make the
// first call on a device before capturing any stream work.
//
// The arithmetic is the IEEE double sequence of the exact-form CFL kernel
// (compiled without contraction), which is the CPU reference's sequence: the
// dt equals ppmlr_cfl_dt of a PPMLR_FP64_EXACT context bit for bit, and that
// of the default PPMLR_FP64 context (contracted rate form) to roundoff.
#include <cuda.h>
#include <math.h>
#include <mutex>

#include "ppmlr_internal.h"

namespace ppmlr {
namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 1024;                 // one double per block
constexpr int NA_SCRATCH_DOUBLES = NA_MAX_BLOCKS + 32;  // + ticket counter (padded)

static __device__ __align__(256) double g_cfl_scratch[NA_SCRATCH_DOUBLES];

__device__ __forceinline__ double na_fast2(double rho, double p, double Bn, double B1, double B2, double gam)
{
    double a2 = gam * p / rho;
    double b2 = (Bn * Bn + B1 * B1 + B2 * B2) / rho;
    double bn2 = Bn * Bn / rho;
    double s = a2 + b2;
    double disc = s * s - 4.0 * a2 * bn2;
    if (disc < 0.0) disc = 0.0;
    return 0.5 * (s + sqrt(disc));
}

__device__ __forceinline__ double na_block_min(double v)
{
    __shared__ double red[NA_THREADS / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        double o = __shfl_down_sync(0xffffffffu, v, off);
        v = o < v ? o : v;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < NA_THREADS / 32 ? red[threadIdx.x] : INFINITY;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            double o = __shfl_down_sync(0xffffffffu, v, off);
            v = o < v ? o : v;
        }
    }
    return v;
}

struct NaArgs {
    const double *U[8];
    int n[3];
    const double *w[3];     // cell widths, n[d] entries (no ghosts)
    const double *c[3];     // cell centres, n[d] entries
    double gamma, p_min, M, r_inner, cfl;
    double *scratch;        // device address of g_cfl_scratch
    double *dt_out;
};

__global__ void __launch_bounds__(NA_THREADS) cfl_noalloc_kernel(NaArgs a)
{
    double *partial = a.scratch;
    unsigned int *counter = reinterpret_cast<unsigned int *>(a.scratch + NA_MAX_BLOCKS);
    const long long nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const long long ncell = nx * ny * nz;
    double best = INFINITY;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ncell;
         i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / (nx * ny));
        const double x = a.c[0][ix], y = a.c[1][iy], z = a.c[2][iz];
        if (a.r_inner > 0.0 && x * x + y * y + z * z < a.r_inner * a.r_inner) continue;
        double U[8];
#pragma unroll
        for (int v = 0; v < 8; v++) U[v] = __ldg(a.U[v] + i);
        double Bd[3] = {0.0, 0.0, 0.0};
        {
            double r2 = x * x + y * y + z * z;
            if (a.M != 0.0 && r2 != 0.0) {
                double r = sqrt(r2);
                double r5 = r2 * r2 * r;
                double mr = -z;
                Bd[0] = a.M * (3.0 * mr * x) / r5;
                Bd[1] = a.M * (3.0 * mr * y) / r5;
                Bd[2] = a.M * (3.0 * mr * z + r2) / r5;
            }
        }
        const int idx[3] = {ix, iy, iz};
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
            double rho = U[0];
            double mn = U[1 + d], m1 = U[1 + t1], m2 = U[1 + t2];
            double Bn = U[4 + d], B1 = U[4 + t1], B2 = U[4 + t2];
            double pr = (a.gamma - 1.0) * (U[7] - 0.5 * (mn * mn + m1 * m1 + m2 * m2) / rho
                                           - 0.5 * (Bn * Bn + B1 * B1 + B2 * B2));
            if (pr < a.p_min) pr = a.p_min;
            double c1 = na_fast2(rho, pr, Bn, B1, B2, a.gamma);
            double c2 = na_fast2(rho, pr, Bn + Bd[d], B1 + Bd[t1], B2 + Bd[t2], a.gamma);
            double cf = sqrt(c1 > c2 ? c1 : c2);
            double s = a.w[d][idx[d]] / (fabs(mn / rho) + cf);
            if (s < best) best = s;
        }
    }
    best = na_block_min(best);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = best;
        __threadfence();
        unsigned int ticket = atomicAdd(counter, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double m = INFINITY;
        for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
            double v = __ldcg(partial + b);
            m = v < m ? v : m;
        }
        m = na_block_min(m);
        if (threadIdx.x == 0) {
            *a.dt_out = a.cfl * m;
            *counter = 0u;
        }
    }
}

// Per-device cache of the scratch array's device address, keyed by the unique
// ID of the context it was looked up under.
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
double *g_na_ptr[NA_MAX_DEVICES] = {nullptr};
unsigned long long g_na_ctx[NA_MAX_DEVICES] = {0};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Unique ID of the current context (0: none current, or the driver offers no
// context IDs -- then every call looks the address up again).
unsigned long long current_context_id()
{
    static const CtxGetCurrentFn get_current = []() -> CtxGetCurrentFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        return cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
                       q == cudaDriverEntryPointSuccess
                   ? (CtxGetCurrentFn)p
                   : nullptr;
    }();
    static const CtxGetIdFn get_id = []() -> CtxGetIdFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        return cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                       q == cudaDriverEntryPointSuccess
                   ? (CtxGetIdFn)p
                   : nullptr;
    }();
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

cudaError_t scratch_address(int device, double **out)
{
    std::lock_guard<std::mutex> lock(g_na_mutex);
    const unsigned long long id = current_context_id();
    if (!g_na_ptr[device] || id == 0 || id != g_na_ctx[device]) {
        double *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&ptr, g_cfl_scratch);   // makes the context current if none was
        if (e != cudaSuccess) return e;
        g_na_ptr[device] = ptr;
        g_na_ctx[device] = id != 0 ? id : current_context_id();
    }
    *out = g_na_ptr[device];
    return cudaSuccess;
}

}  // namespace
}  // namespace ppmlr

using namespace ppmlr;

extern "C" ppmlr_status ppmlr_cfl_dt_noalloc(const double *const U[8], const int n[3],
                                             const double *const width[3], const double *const centre[3],
                                             double gamma, double p_min, double dipole_moment, double r_inner,
                                             double cfl, int blocks, double *dt_out, void *cuda_stream)
{
    if (!U || !n || !width || !centre || !dt_out) return PPMLR_E_INVALID;
    for (int v = 0; v < 8; v++)
        if (!U[v]) return PPMLR_E_INVALID;
    for (int d = 0; d < 3; d++)
        if (n[d] < 1 || !width[d] || !centre[d]) return PPMLR_E_INVALID;
    if (!(gamma > 1.0) || !(cfl > 0.0) || !(p_min >= 0.0)) return PPMLR_E_INVALID;
    const long long ncell = (long long)n[0] * n[1] * n[2];
    if (ncell > (1LL << 31) - 1) return PPMLR_E_INVALID;
    if (blocks < 0 || blocks > NA_MAX_BLOCKS) return PPMLR_E_INVALID;   // beyond the static scratch

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return PPMLR_E_CUDA;
    if (device < 0 || device >= NA_MAX_DEVICES) return PPMLR_E_INVALID;
    double *scratch = nullptr;
    if (scratch_address(device, &scratch) != cudaSuccess) return PPMLR_E_CUDA;

    if (blocks == 0) {
        int sms = 152;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return PPMLR_E_CUDA;
        long long need = (ncell + NA_THREADS - 1) / NA_THREADS;
        long long b = 4LL * sms;
        if (b > need) b = need;
        if (b > NA_MAX_BLOCKS) b = NA_MAX_BLOCKS;
        blocks = (int)b;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the ticket counter must start at zero on every call
    if (cudaMemsetAsync(scratch + NA_MAX_BLOCKS, 0, sizeof(unsigned int), s) != cudaSuccess) return PPMLR_E_CUDA;
    NaArgs a;
    for (int v = 0; v < 8; v++) a.U[v] = U[v];
    for (int d = 0; d < 3; d++) { a.n[d] = n[d]; a.w[d] = width[d]; a.c[d] = centre[d]; }
    a.gamma = gamma; a.p_min = p_min; a.M = dipole_moment; a.r_inner = r_inner; a.cfl = cfl;
    a.scratch = scratch;
    a.dt_out = dt_out;
    cfl_noalloc_kernel<<<blocks, NA_THREADS, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? PPMLR_OK : PPMLR_E_CUDA;
}
