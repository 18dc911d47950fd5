// FP64 sweep kernels, exact form: the same IEEE double expression trees as the
// CPU reference, compiled without contraction, so that the results are
// bit-identical to it (correctly rounded division and square root on both
// sides).
#include "launch.cuh"

namespace ppmlr {
const SweepLaunchers k_sweep_fp64_exact = SweepVariant<double, true>::table();
}  // namespace ppmlr
