// Residual kernels of order p = 4 (N = 5 solution points per direction).
// Elements per CTA: 2 (FP64 form); FP32 perturbation form: 4 in the lifting kernel (four 100-thread
// CTAs per SM) and 5 in the residual kernel (125 threads: three CTAs per SM fill 12 warps; 4 left 28
// of 128 lanes idle and ran 14 % slower).
// Tile 1 halves the FP32 elements per CTA (a candidate of the batched-shell autotuner).
#include "kern_inst.cuh"

namespace chorus {
LaunchSet launchers_p4(int tile) {
  return tile == 1 ? Inst<5, 2, 2>::set() : Inst<5, 2, 4, 5>::set();
}
}  // namespace chorus
