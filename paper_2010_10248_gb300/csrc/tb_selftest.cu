// Self-test of the bounded wait used by the blocked sweep: one thread waits
// on a flag that nothing sets, gives up after the limit and reports it.
#include "tb_sweep.cuh"

namespace tbi {

__global__ void k_selftest_wait(const unsigned long long* flag, long long timeout_ns, int* err) {
  if (threadIdx.x != 0) return;
  const bool ok = bounded_wait_ge(flag, 1ull, global_ns(), timeout_ns);
  *err = ok ? 0 : 1;
}

cudaError_t selftest_wait(long long timeout_ns, cudaStream_t st, int* timed_out) {
  unsigned long long* flag = nullptr;
  int* err = nullptr;
  cudaError_t e = dmalloc(&flag, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = dmalloc(&err, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0xff, sizeof(int), st);
  if (e == cudaSuccess) {
    count_launch();
    k_selftest_wait<<<1, 32, 0, st>>>(flag, timeout_ns, err);
    e = cudaGetLastError();
  }
  int h = -1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dfree(flag, st);
  dfree(err, st);
  *timed_out = h;
  return e;
}

}  // namespace tbi
