// Sweep kernels of radius 6 (space order 12), T = 1..2 fused steps.
#include "tb_sweep.cuh"

namespace tbi {
// what: 0 launch, 1 occupancy query, 2 shape query
cudaError_t sweep_dispatch_r6(int what, int T, int sk, const SweepParams* p, int nctas, bool coop,
                               cudaStream_t st, int* per_sm, SweepShape* s) {
  switch (T) {
    TBI_DEFINE_RADIUS_T(6, 1)
    TBI_DEFINE_RADIUS_T(6, 2)
  }
  return cudaErrorInvalidValue;
}
cudaError_t sweep_batch_dispatch_r6(const BatchParams* p, int nctas, cudaStream_t st) {
  return sweep_batch_launch_t<6>(*p, nctas, st);
}
}  // namespace tbi
