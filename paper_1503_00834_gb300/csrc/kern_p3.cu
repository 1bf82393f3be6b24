// Residual kernels of order p = 3 (N = 4 solution points per direction).
// Elements per CTA: 4 (FP64 form), 4 (FP32 perturbation form, both kernels: 64-thread CTAs, eight
// lifting and six residual CTAs per SM; the residual kernel 8 % faster than with eight-element CTAs
// at the same warps per SM).  Tile 1 (eight elements per CTA, the previous default) is the other
// candidate of the batched-shell autotuner.
// This translation unit is compiled with the approximate FP32 square root (build.py).
#include "kern_inst.cuh"

namespace chorus {
LaunchSet launchers_p3(int tile) {
  return tile == 1 ? Inst<4, 4, 8>::set() : Inst<4, 4, 4>::set();
}
}  // namespace chorus
