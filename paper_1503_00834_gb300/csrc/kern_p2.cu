// Residual kernels of order p = 2 (N = 3 solution points per direction).
// Elements per CTA: 6 (FP64 form), 12 (FP32 perturbation form); chosen so that a CTA's state block
// is a multiple of 16 bytes (bulk-copy granularity) and the CTA stays near 128 threads.
// Tile 1 halves the FP32 elements per CTA (a candidate of the batched-shell autotuner).
#include "kern_inst.cuh"

namespace chorus {
LaunchSet launchers_p2(int tile) {
  return tile == 1 ? Inst<3, 6, 6>::set() : Inst<3, 6, 12>::set();
}
}  // namespace chorus
