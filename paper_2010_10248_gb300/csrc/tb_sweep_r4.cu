// Sweep kernels of radius 4 (space order 8), T = 1..4 fused steps.
#include "tb_sweep.cuh"

namespace tbi {
TBI_DEFINE_RADIUS(4)
}  // namespace tbi
