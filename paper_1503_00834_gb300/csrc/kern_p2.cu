// Residual kernels of order p = 2 (N = 3 solution points per direction).
// Elements per CTA: 6 (FP64 form), 14 (FP32 perturbation form: 126 threads, four warps nearly full;
// 12 elements left 20 of 128 lanes idle and ran 8 % slower).
// Tile 1 halves the FP32 elements per CTA (a candidate of the batched-shell autotuner).
#include "kern_inst.cuh"

namespace chorus {
LaunchSet launchers_p2(int tile) {
  return tile == 1 ? Inst<3, 6, 6>::set() : Inst<3, 6, 14>::set();
}
}  // namespace chorus
