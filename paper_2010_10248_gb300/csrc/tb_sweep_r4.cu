// Sweep kernels of radius 4 (space order 8), T = 1..4 fused steps.
#include "tb_sweep.cuh"

namespace tbi {
// what: 0 launch, 1 occupancy query, 2 shape query
cudaError_t sweep_dispatch_r4(int what, int T, int sk, const SweepParams* p, int nctas, bool coop,
                               cudaStream_t st, int* per_sm, SweepShape* s) {
  switch (T) {
    TBI_DEFINE_RADIUS_T(4, 1)
    TBI_DEFINE_RADIUS_T(4, 2)
    TBI_DEFINE_RADIUS_T(4, 3)
    TBI_DEFINE_RADIUS_T(4, 4)
  }
  return cudaErrorInvalidValue;
}
cudaError_t sweep_batch_dispatch_r4(const BatchParams* p, int nctas, cudaStream_t st) {
  return sweep_batch_launch_t<4>(*p, nctas, st);
}
}  // namespace tbi
