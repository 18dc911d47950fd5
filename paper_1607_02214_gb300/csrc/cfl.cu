// CFL kernels of the exact FP64 path (bit-identical to the CPU reference).
#include "cfl.cuh"

namespace ppmlr {
int cfl_threads() { return CFL_THREADS; }
const CflLaunchers k_cfl_fp64_exact = CflVariant<true>::table();
}  // namespace ppmlr
