// Residual kernels of order p = 4 (N = 5 solution points per direction).
// Elements per CTA: 2 (FP64 form); FP32 perturbation form: 5 (125 threads: three CTAs per SM fill 12
// warps in both kernels; 4 elements left 28 of 128 lanes idle: the residual kernel ran 14 % slower,
// the lifting kernel 24 % slower even at four CTAs per SM).
// Tile 1 (two elements per CTA) is the other candidate of the batched-shell autotuner.
#include "kern_inst.cuh"

namespace chorus {
LaunchSet launchers_p4(int tile) {
  return tile == 1 ? Inst<5, 2, 2>::set() : Inst<5, 2, 5, 5>::set();
}
}  // namespace chorus
