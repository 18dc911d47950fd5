// Mixed-precision sweep kernels: FP32 reconstruction, Riemann solve, remap and
// sources; FP64 pressure recovery and FP64 accumulation of the state (see
// sweep.cuh).  Compiled with contraction and fast FP32 division and sqrt.
#include "sweep.cuh"

namespace ppmlr {

template <int DIR>
static cudaError_t go(const SweepArgs &a, const Tile &t, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(sweep_kernel<DIR, float>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    sweep_kernel<DIR, float><<<t.ntiles, t.threads, t.smem, s>>>(a);
    return cudaGetLastError();
}

// (the shared-memory attribute is set by occ(), which planning always calls first)
template <int DIR>
static cudaError_t go_ens(const EnsSweepArgs &e, int blocks, int threads, size_t smem, cudaStream_t s)
{
    if (blocks == e.total_tiles) {   // one block per tile
        sweep_ensemble_grid_kernel<DIR, float><<<blocks, threads, smem, s>>>(e);
        return cudaGetLastError();
    }
    sweep_ensemble_kernel<DIR, float><<<blocks, threads, smem, s>>>(e);
    return cudaGetLastError();
}

template <int DIR>
static int occ(int threads, size_t smem)
{
    cudaFuncSetAttribute(sweep_ensemble_kernel<DIR, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(sweep_ensemble_grid_kernel<DIR, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_ensemble_kernel<DIR, float>, threads, smem) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_sweep_mixed(int dir, const SweepArgs &a, const Tile &t, cudaStream_t s)
{
    switch (dir) {
        case 0: return go<0>(a, t, s);
        case 1: return go<1>(a, t, s);
        default: return go<2>(a, t, s);
    }
}

cudaError_t launch_sweep_ensemble_mixed(int dir, const EnsSweepArgs &e, int blocks, int threads, size_t smem,
                                       cudaStream_t s)
{
    switch (dir) {
        case 0: return go_ens<0>(e, blocks, threads, smem, s);
        case 1: return go_ens<1>(e, blocks, threads, smem, s);
        default: return go_ens<2>(e, blocks, threads, smem, s);
    }
}

template <int DIR>
static cudaError_t go_param(const EnsSweepParams &p, int blocks, int threads, size_t smem, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t r = cudaFuncSetAttribute(sweep_ensemble_param_kernel<DIR, float>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (r != cudaSuccess) return r;
        attr = true;
    }
    sweep_ensemble_param_kernel<DIR, float><<<blocks, threads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_sweep_ensemble_param_mixed(int dir, const EnsSweepParams &p, int blocks, int threads, size_t smem,
                                             cudaStream_t s)
{
    switch (dir) {
        case 0: return go_param<0>(p, blocks, threads, smem, s);
        case 1: return go_param<1>(p, blocks, threads, smem, s);
        default: return go_param<2>(p, blocks, threads, smem, s);
    }
}

int sweep_blocks_per_sm_mixed(int dir, int threads, size_t smem)
{
    switch (dir) {
        case 0: return occ<0>(threads, smem);
        case 1: return occ<1>(threads, smem);
        default: return occ<2>(threads, smem);
    }
}

}  // namespace ppmlr
