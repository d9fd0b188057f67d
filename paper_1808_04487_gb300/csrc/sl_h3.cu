// Brick-tiled FP32 semi-Lagrangian launchers for halo 3 (see sl_kernels.cuh).
#include "sl_kernels.cuh"

namespace claire {
CLAIRE_SL_LAUNCHERS(, float, 3)
}  // namespace claire
