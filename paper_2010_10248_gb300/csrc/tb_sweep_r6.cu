// Sweep kernels of radius 6 (space order 12), T = 1..4 fused steps.
#include "tb_sweep.cuh"

namespace tbi {
TBI_DEFINE_RADIUS(6)
}  // namespace tbi
