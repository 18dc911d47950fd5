// FP64 sweep kernels.  Compiled without floating-point contraction so that
// every stage evaluates the same IEEE double expression trees as the CPU
// reference (correctly rounded division and square root on both sides).
#include "sweep.cuh"

namespace ppmlr {

template <int DIR>
static cudaError_t go(const SweepArgs &a, const Tile &t, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(sweep_kernel<DIR, double>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    sweep_kernel<DIR, double><<<t.ntiles, t.threads, t.smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sweep_fp64(int dir, const SweepArgs &a, const Tile &t, cudaStream_t s)
{
    switch (dir) {
        case 0: return go<0>(a, t, s);
        case 1: return go<1>(a, t, s);
        default: return go<2>(a, t, s);
    }
}

}  // namespace ppmlr
