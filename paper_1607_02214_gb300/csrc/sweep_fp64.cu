// FP64 sweep kernels, default form: IEEE double throughout, compiled with
// contraction (fused multiply-add) and one reciprocal per shared denominator.
// Agrees with the CPU reference to roundoff (parity bar: relative L1 1e-11).
#include "launch.cuh"

namespace ppmlr {
const SweepLaunchers k_sweep_fp64 = SweepVariant<double, false>::table();
}  // namespace ppmlr
