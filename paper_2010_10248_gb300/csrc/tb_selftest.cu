// Diagnostics: a self-test of the bounded wait used by the blocked sweep (one
// thread waits on a flag that nothing sets, gives up after the limit and
// reports it), and the two peaks the rooflines are read against, measured
// with this build's own kernels: a float4 copy (HBM) and chains of packed
// FP32 FMAs.
#include <algorithm>

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

// dst = src over n float4 values, grid-stride, streaming loads and stores
__global__ void __launch_bounds__(256) k_copy4(const float4* __restrict__ src, float4* __restrict__ dst, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) __stcs(dst + i, __ldcs(src + i));
}

// 8 independent chains of packed FMAs per thread (each f32x2 FMA = 4 flops);
// the sums go to out so that the chains are not removed
__global__ void __launch_bounds__(256) k_fma_chains(float* out, int iters, float a, float b) {
  float2 acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = make_float2((float)(threadIdx.x + k), (float)(blockIdx.x - k));
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = __ffma2_rn(acc[k], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += acc[k].x + acc[k].y;
  if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // practically never taken
}

cudaError_t measure_peaks(double* hbm_gbs, double* fp32_tflops, cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const size_t n4 = (size_t)1 << 26;  // 64 Mi float4 = 1 GiB per buffer, far above L2
  float4 *a = nullptr, *b = nullptr;
  float* out = nullptr;
  e = dmalloc(&a, sizeof(float4) * n4, st);
  if (e == cudaSuccess) e = dmalloc(&b, sizeof(float4) * n4, st);
  if (e == cudaSuccess) e = dmalloc(&out, sizeof(float) * (size_t)nsm * 4 * 256, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a, 0, sizeof(float4) * n4, st);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  float best = 1e30f;
  for (int r = 0; r < 6 && e == cudaSuccess; ++r) {  // copy: best of 6, after one warm-up
    cudaEventRecord(t0, st);
    count_launch();
    k_copy4<<<nsm * 8, 256, 0, st>>>(r & 1 ? b : a, r & 1 ? a : b, n4);
    cudaEventRecord(t1, st);
    e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (r > 0) best = std::min(best, ms);
  }
  if (e == cudaSuccess) *hbm_gbs = 2.0 * sizeof(float4) * (double)n4 / (best * 1e-3) / 1e9;
  const int iters = 1 << 15, blocks = nsm * 4;
  best = 1e30f;
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
    cudaEventRecord(t0, st);
    count_launch();
    k_fma_chains<<<blocks, 256, 0, st>>>(out, iters, 0.999f, 1e-3f);
    cudaEventRecord(t1, st);
    e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (r > 0) best = std::min(best, ms);
  }
  if (e == cudaSuccess) *fp32_tflops = 4.0 * 8.0 * iters * (double)blocks * 256 / (best * 1e-3) / 1e12;
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  dfree(a, st);
  dfree(b, st);
  dfree(out, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  return e != cudaSuccess ? e : e2;
}

}  // namespace tbi
