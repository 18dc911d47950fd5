// CFL kernels of the default FP64 path (contraction, shared reciprocal).
#include "cfl.cuh"

namespace ppmlr {
const CflLaunchers k_cfl_fp64 = CflVariant<false>::table();
}  // namespace ppmlr
