// Acoustic one-step propagation (Eq. 1) with the wavefields stored in
// 16 bits (FP16 or BF16) and every operation in FP32: stored value = u / s
// with a per-field power-of-two scale s, so that scaling is exact and the
// FP16 range holds the field.  u^{n+1} is stored with the scale
//   s_{n+1} = 2^(ceil(log2(4 max|u^n| + max|src step n|)) - 8)
// (the field can grow by well under 4x per step at the CFL limit, so the
// stored values stay below 2^8 of FP16's 2^16 range), computed on the device
// from the running maximum of the previous step, so no step waits for the host.
// The same kernel instantiated for float storage is the FP32 baseline of
// equal structure.
//
// A thread owns one (y, z) column of a chunk of planes and keeps the axis-0
// neighbours in a register queue (FP32); axis-1/axis-2 neighbours come
// through the L1 cache.  Injection and receiver sampling are separate small
// kernels after the update, as in the TTI / elastic path.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "tb_internal.cuh"

namespace tbi {

static unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <class ST>
struct Store;
template <>
struct Store<float> {
  static __device__ __forceinline__ float get(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ float make(float v) { return v; }
};
template <>
struct Store<__half> {
  static __device__ __forceinline__ float get(const __half* p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ __half make(float v) { return __float2half_rn(v); }
};
template <>
struct Store<__nv_bfloat16> {
  static __device__ __forceinline__ float get(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
  static __device__ __forceinline__ __nv_bfloat16 make(float v) { return __float2bfloat16_rn(v); }
};

namespace {
__device__ __forceinline__ size_t lidx(const PhysGrid& g, int x, int y, int z) {
  return ((size_t)x * g.n1 + y) * g.n2p + z;
}
template <class ST>
__device__ __forceinline__ float lz(const PhysGrid& g, const ST* f, int x, int y, int z, float s) {
  return (x >= 0 && x < g.n0 && y >= 0 && y < g.n1 && z >= 0 && z < g.n2) ? __fmul_rn(Store<ST>::get(f + lidx(g, x, y, z)), s)
                                                                        : 0.f;
}
// warp max, then one atomic per warp (non-negative floats order as their bits)
__device__ __forceinline__ void atomic_max_warp(unsigned* dst, float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(dst, __float_as_uint(v));
}
}  // namespace

// scales: s[k] is the scale of u^{k-1} (s[0] for u^{-1}); mx[k]: max |u^{k-1}|
template <class ST, int R>
__global__ void __launch_bounds__(256) k_ac_lp(PhysGrid g, LapW w, int nchunks, const ST* __restrict__ uc,
                                               ST* up, const float* __restrict__ c2,
                                               const float* __restrict__ damp_b, float* scales,
                                               const float* __restrict__ srcmax, int n, unsigned* __restrict__ mx) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  const bool ok = z < g.n2 && y < g.n1;
  // planes [x0, x1) of chunk blockIdx.z (all chunks of a step in one launch)
  const int x0 = (int)((int64_t)g.n0 * blockIdx.z / nchunks), x1 = (int)((int64_t)g.n0 * (blockIdx.z + 1) / nchunks);
  const float s_out = lp_next_scale(mx, srcmax, n);
  const float s_cur = scales[n + 1], s_prev = scales[n], inv_out = 1.0f / s_out;  // powers of two
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && threadIdx.y == 0)
    scales[n + 2] = s_out;  // for the kernels after the step
  float q[2 * R + 1];
#pragma unroll
  for (int s = 0; s < 2 * R + 1; ++s) q[s] = ok ? lz(g, uc, x0 - 1 - R + s, y, z, s_cur) : 0.f;
  const float byz = ok ? __fadd_rn(__ldg(damp_b + g.n0 + y), __ldg(damp_b + g.n0 + g.n1 + z)) : 0.f;
  float vmax = 0.f;
  for (int x = x0; x < x1; ++x) {
#pragma unroll
    for (int s = 0; s < 2 * R; ++s) q[s] = q[s + 1];
    q[2 * R] = ok ? lz(g, uc, x + R, y, z, s_cur) : 0.f;
    if (!ok) continue;
    const float u = q[R];
    float l = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float acc = 0.f;
#pragma unroll
      for (int i = 1; i <= R; ++i) {
        const float a = d == 0 ? q[R + i] : (d == 1 ? lz(g, uc, x, y + i, z, s_cur) : lz(g, uc, x, y, z + i, s_cur));
        const float b = d == 0 ? q[R - i] : (d == 1 ? lz(g, uc, x, y - i, z, s_cur) : lz(g, uc, x, y, z - i, s_cur));
        acc = __fmaf_rn(w.c[d][i - 1], __fadd_rn(__fsub_rn(a, u), __fsub_rn(b, u)), acc);
      }
      l = __fadd_rn(l, acc);
    }
    const size_t i0 = lidx(g, x, y, z);
    const float cc = __ldg(c2 + i0);
    const float gd = __fmul_rn(__fadd_rn(__ldg(damp_b + x), byz), cc);
    const float uprev = __fmul_rn(Store<ST>::get(up + i0), s_prev);
    // the quotient is exact without a division outside the sponge (1 + gd = 1)
    const float num = __fmaf_rn(cc, l, __fmul_rn(__fsub_rn(1.f, gd), __fsub_rn(u, uprev)));
    const float den = __fadd_rn(1.f, gd);
    const float un = __fadd_rn(u, den == 1.f ? num : __fdiv_rn(num, den));
    up[i0] = Store<ST>::make(__fmul_rn(un, inv_out));
    vmax = fmaxf(vmax, fabsf(un));
  }
  atomic_max_warp(mx + n + 2, vmax);
}

// u^{n+1}(p_id) += dcmp[id], in the stored scale; updates the running max
template <class ST>
__global__ void k_lp_inject(PhysGrid g, int64_t npts, const int64_t* __restrict__ lin, const float* __restrict__ dcmp,
                            ST* u, const float* __restrict__ scales, int n, unsigned* mx) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= npts) return;
  const int64_t l = lin[id];
  const int z = (int)(l % g.n2), y = (int)((l / g.n2) % g.n1), x = (int)(l / ((int64_t)g.n1 * g.n2));
  const size_t i0 = lidx(g, x, y, z);
  const float s = scales[n + 2];
  const float v = __fadd_rn(__fmul_rn(Store<ST>::get(u + i0), s), dcmp[id]);
  u[i0] = Store<ST>::make(__fmul_rn(v, 1.0f / s));
  atomicMax(mx + n + 2, __float_as_uint(fabsf(v)));
}

template <class ST>
__global__ void k_lp_sample(PhysGrid g, int64_t npts, const int2* __restrict__ ent, const int64_t* __restrict__ lin,
                            const ST* u, const float* __restrict__ scales, int n, float* __restrict__ row) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npts) return;
  const int64_t l = lin[ent[e].y];
  const int z = (int)(l % g.n2), y = (int)((l / g.n2) % g.n1), x = (int)(l / ((int64_t)g.n1 * g.n2));
  row[e] = __fmul_rn(Store<ST>::get(u + lidx(g, x, y, z)), scales[n + 2]);
}

// largest |src_dcmp[t][.]| of every step t (one block per step)
__global__ void k_lp_srcmax(int64_t npts, const float* __restrict__ dcmp, float* out) {
  const int t = blockIdx.x;
  float m = 0.f;
  for (int64_t i = threadIdx.x; i < npts; i += blockDim.x) m = fmaxf(m, fabsf(dcmp[(int64_t)t * npts + i]));
  __shared__ float red[256];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[t] = red[0];
}

template <class ST>
__global__ void k_lp_unpack(PhysGrid g, const ST* __restrict__ u, float s, float* __restrict__ out) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, x = blockIdx.z;
  if (z >= g.n2 || y >= g.n1) return;
  out[((size_t)x * g.n1 + y) * g.n2 + z] = __fmul_rn(Store<ST>::get(u + lidx(g, x, y, z)), s);
}

// ------------------------------------------------------------- launch --
template <class ST, int R>
static cudaError_t lp_step_t(const PhysGrid& g, const LapW& w, int nchunks, const void* uc, void* up, const float* c2,
                             const float* damp_b, float* scales, const float* srcmax, int n, unsigned* mx,
                             cudaStream_t st) {
  const dim3 blk(32, 8), grd((unsigned)((g.n2 + 31) / 32), (unsigned)((g.n1 + 7) / 8), (unsigned)nchunks);
  count_launch();
  k_ac_lp<ST, R><<<grd, blk, 0, st>>>(g, w, nchunks, (const ST*)uc, (ST*)up, c2, damp_b, scales, srcmax, n, mx);
  return cudaGetLastError();
}
template <class ST>
static cudaError_t lp_step_st(int R, const PhysGrid& g, const LapW& w, int nchunks, const void* uc, void* up,
                              const float* c2, const float* damp_b, float* scales, const float* srcmax, int n,
                              unsigned* mx, cudaStream_t st) {
  switch (R) {
    case 2: return lp_step_t<ST, 2>(g, w, nchunks, uc, up, c2, damp_b, scales, srcmax, n, mx, st);
    case 4: return lp_step_t<ST, 4>(g, w, nchunks, uc, up, c2, damp_b, scales, srcmax, n, mx, st);
    case 6: return lp_step_t<ST, 6>(g, w, nchunks, uc, up, c2, damp_b, scales, srcmax, n, mx, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t lowprec_step(int storage, int R, const PhysGrid& g, const LapW& w, int nchunks, const void* uc, void* up,
                         const float* c2, const float* damp_b, float* scales, const float* srcmax, int n,
                         unsigned* mx, cudaStream_t st) {
  switch (storage) {
    case 1: return lp_step_st<__half>(R, g, w, nchunks, uc, up, c2, damp_b, scales, srcmax, n, mx, st);
    case 2: return lp_step_st<__nv_bfloat16>(R, g, w, nchunks, uc, up, c2, damp_b, scales, srcmax, n, mx, st);
    case 3: return lp_step_st<float>(R, g, w, nchunks, uc, up, c2, damp_b, scales, srcmax, n, mx, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t lowprec_inject(int storage, const PhysGrid& g, int64_t npts, const int64_t* lin, const float* dcmp_row,
                           void* u, const float* scales, int n, unsigned* mx, cudaStream_t st) {
  if (npts <= 0) return cudaSuccess;
  count_launch();
  const unsigned gb = grid_for(npts, 128);
  if (storage == 1) k_lp_inject<__half><<<gb, 128, 0, st>>>(g, npts, lin, dcmp_row, (__half*)u, scales, n, mx);
  else if (storage == 2)
    k_lp_inject<__nv_bfloat16><<<gb, 128, 0, st>>>(g, npts, lin, dcmp_row, (__nv_bfloat16*)u, scales, n, mx);
  else k_lp_inject<float><<<gb, 128, 0, st>>>(g, npts, lin, dcmp_row, (float*)u, scales, n, mx);
  return cudaGetLastError();
}

cudaError_t lowprec_sample(int storage, const PhysGrid& g, int64_t npts, const int2* ent, const int64_t* lin,
                           const void* u, const float* scales, int n, float* row, cudaStream_t st) {
  if (npts <= 0) return cudaSuccess;
  count_launch();
  const unsigned gb = grid_for(npts, 128);
  if (storage == 1) k_lp_sample<__half><<<gb, 128, 0, st>>>(g, npts, ent, lin, (const __half*)u, scales, n, row);
  else if (storage == 2)
    k_lp_sample<__nv_bfloat16><<<gb, 128, 0, st>>>(g, npts, ent, lin, (const __nv_bfloat16*)u, scales, n, row);
  else k_lp_sample<float><<<gb, 128, 0, st>>>(g, npts, ent, lin, (const float*)u, scales, n, row);
  return cudaGetLastError();
}

cudaError_t lowprec_srcmax(int64_t npts, int nt, const float* dcmp, float* out, cudaStream_t st) {
  if (npts <= 0 || nt <= 0) return cudaSuccess;
  count_launch();
  k_lp_srcmax<<<nt, 256, 0, st>>>(npts, dcmp, out);
  return cudaGetLastError();
}

cudaError_t lowprec_unpack(int storage, const PhysGrid& g, const void* u, float s, float* out, cudaStream_t st) {
  count_launch();
  const dim3 blk(32, 8), grd((unsigned)((g.n2 + 31) / 32), (unsigned)((g.n1 + 7) / 8), (unsigned)g.n0);
  if (storage == 1) k_lp_unpack<__half><<<grd, blk, 0, st>>>(g, (const __half*)u, s, out);
  else if (storage == 2) k_lp_unpack<__nv_bfloat16><<<grd, blk, 0, st>>>(g, (const __nv_bfloat16*)u, s, out);
  else k_lp_unpack<float><<<grd, blk, 0, st>>>(g, (const float*)u, s, out);
  return cudaGetLastError();
}

}  // namespace tbi
