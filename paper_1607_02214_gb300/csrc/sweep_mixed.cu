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

cudaError_t launch_sweep_mixed(int dir, const SweepArgs &a, const Tile &t, cudaStream_t s)
{
    switch (dir) {
        case 0: return go<0>(a, t, s);
        case 1: return go<1>(a, t, s);
        default: return go<2>(a, t, s);
    }
}

}  // namespace ppmlr
