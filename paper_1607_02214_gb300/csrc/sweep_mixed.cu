// Mixed-precision sweep kernels: FP32 reconstruction, Riemann solve, remap and
// sources; pressure recovery in double-float arithmetic and the state
// accumulated in FP64 (see sweep.cuh and mixed_util.cuh).  Compiled with
// contraction and fast FP32 division and square root.
#include "launch.cuh"

namespace ppmlr {
const SweepLaunchers k_sweep_mixed = SweepVariant<float, false>::table();
}  // namespace ppmlr
