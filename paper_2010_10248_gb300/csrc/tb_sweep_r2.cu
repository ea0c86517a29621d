// Sweep kernels of radius 2 (space order 4), T = 1..4 fused steps.
#include "tb_sweep.cuh"

namespace tbi {
TBI_DEFINE_RADIUS(2)
}  // namespace tbi
