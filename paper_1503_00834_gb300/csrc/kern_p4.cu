// Residual kernels of order p = 4 (N = 5 solution points per direction).
// Elements per CTA: 2 (FP64 form), 4 (FP32 perturbation form); chosen so that a CTA's state block
// is a multiple of 16 bytes (bulk-copy granularity) and the CTA stays near 128 threads.
// Tile 1 halves the FP32 elements per CTA (a candidate of the batched-shell autotuner).
#include "kern_inst.cuh"

namespace chorus {
LaunchSet launchers_p4(int tile) {
  return tile == 1 ? Inst<5, 2, 2>::set() : Inst<5, 2, 4>::set();
}
}  // namespace chorus
