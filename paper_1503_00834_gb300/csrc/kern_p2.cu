// Residual kernels of order p = 2 (N = 3 solution points per direction).
// Elements per CTA: 6 (FP64 form); FP32 perturbation form: 14 in the lifting kernel (126 threads,
// four warps nearly full; 12 elements left 20 of 128 lanes idle and ran 8 % slower) and 7 in the
// residual kernel (63 threads, six CTAs per SM: 4.6 % faster than 14).
// Tile 1 (six elements per CTA in both) is the other candidate of the batched-shell autotuner.
#include "kern_inst.cuh"

namespace chorus {
LaunchSet launchers_p2(int tile) {
  return tile == 1 ? Inst<3, 6, 6>::set() : Inst<3, 6, 14, 7>::set();
}
}  // namespace chorus
