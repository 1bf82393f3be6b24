// Residual kernels of order p = 5 (N = 6 solution points per direction).
// Elements per CTA: 2 (FP64 form), 2 (FP32 perturbation form, both kernels: 72-thread CTAs, four
// per SM; the residual kernel 5 % and the lifting kernel 3 % faster than with four-element CTAs at two
// per SM).  A CTA's state block stays a multiple of 16 bytes (bulk-copy granularity).
// Tile 1 (four elements per CTA, the previous default) is the other candidate of the batched-shell
// autotuner.
#include "kern_inst.cuh"

namespace chorus {
LaunchSet launchers_p5(int tile) {
  return tile == 1 ? Inst<6, 2, 4>::set() : Inst<6, 2, 2>::set();
}
}  // namespace chorus
