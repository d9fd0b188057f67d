// Brick-tiled FP32 semi-Lagrangian launchers with a BF16 gradient history, halo 2 (see sl_kernels.cuh).
#include "sl_kernels.cuh"

namespace claire {
CLAIRE_SL_LAUNCHERS_G(, float, 2, __nv_bfloat16)
}  // namespace claire
