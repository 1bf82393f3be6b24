// Residual kernels of order p = 3 (N = 4 solution points per direction).
// Elements per CTA: 4 (FP64 form), 8 (FP32 perturbation form); chosen so that a CTA's state block
// is a multiple of 16 bytes (bulk-copy granularity) and the CTA stays near 128 threads.
// Tile 1 halves the FP32 elements per CTA (a candidate of the batched-shell autotuner).
// This translation unit is compiled with the approximate FP32 square root (build.py).
#include "kern_inst.cuh"

namespace chorus {
LaunchSet launchers_p3(int tile) {
  return tile == 1 ? Inst<4, 4, 4>::set() : Inst<4, 4, 8>::set();
}
}  // namespace chorus
