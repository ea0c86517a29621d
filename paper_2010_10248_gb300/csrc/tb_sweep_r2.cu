// Sweep kernels of radius 2 (space order 4), T = 1..4 fused steps.
#include "tb_sweep.cuh"

namespace tbi {
// what: 0 launch, 1 occupancy query, 2 shape query
cudaError_t sweep_dispatch_r2(int what, int T, int sk, const SweepParams* p, int nctas, bool coop,
                               cudaStream_t st, int* per_sm, SweepShape* s) {
  switch (T) {
    TBI_DEFINE_RADIUS_T(2, 1)
    TBI_DEFINE_RADIUS_T(2, 2)
    TBI_DEFINE_RADIUS_T(2, 3)
    TBI_DEFINE_RADIUS_T(2, 4)
  }
  return cudaErrorInvalidValue;
}
cudaError_t sweep_batch_dispatch_r2(const BatchParams* p, int nctas, cudaStream_t st) {
  return sweep_batch_launch_t<2>(*p, nctas, st);
}
}  // namespace tbi
