// Adjoint of the acoustic one-step recurrence and the adjoint-state
// gradient with respect to vp (the FWI / RTM use of the propagator, Sec. I).
//
// Forward, per point: u^{k} = D L u^{k-1} + B u^{k-1} + C u^{k-2} + M S^{k-1}
// with, in the library's variables c2 = dt^2/m and g = a/m (a = eta dt/2),
//   D = c2/(1+g),  B = 2/(1+g),  C = (g-1)/(1+g),  M = c2,
// receivers d[k-1] = P u^{k}.  Adjoint for residual traces r (backward):
//   lam^{k} = L (D lam^{k+1}) + B lam^{k+1} + C lam^{k+2} + P^T r[k-1]
// (the centred Laplacian is symmetric), and the gradient of <d, r> is
//   d/dm(p) = sum_k lam^k(p) c2 [2 g (u^{k-1} - u^{k-2}) - c2 L u^{k-1}](p)
//             / (dt^2 (1+g)^2)  -  sum_k lam^k(p) c2(p) S^{k-1}(p) c2(p)/dt^2,
// evaluated through the recurrence from three stored states (k_adj_grad),
//   d/dvp = d/dm * (-2/vp^3),  vp = sqrt(c2)/dt,
// accumulated in FP64 (the per-step term in FP32).  One plane of columns per
// block; a neighbour load tests only the coordinate it moves along.
#include <cstdint>

#include "tb_internal.cuh"

namespace tbi {

static unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

namespace {
struct AdjCol {
  int y, z;
  bool ok;
};
__device__ __forceinline__ AdjCol adj_col(const PhysGrid& g) {
  AdjCol c;
  c.z = blockIdx.x * blockDim.x + threadIdx.x;
  c.y = blockIdx.y * blockDim.y + threadIdx.y;
  c.ok = c.z < g.n2 && c.y < g.n1;
  return c;
}
__device__ __forceinline__ size_t aidx(const PhysGrid& g, int x, int y, int z) {
  return ((size_t)x * g.n1 + y) * g.n2p + z;
}
__device__ __forceinline__ float ldz(const PhysGrid& g, const float* __restrict__ f, int x, int y, int z) {
  return (x >= 0 && x < g.n0 && y >= 0 && y < g.n1 && z >= 0 && z < g.n2) ? __ldg(f + aidx(g, x, y, z)) : 0.f;
}
// g = (sum of per-axis eta/(2 dt)) * c2
__device__ __forceinline__ float damp_g(const PhysGrid& g, const float* __restrict__ damp_b, float c2, int x, int y,
                                        int z) {
  return __fmul_rn(__fadd_rn(__fadd_rn(__ldg(damp_b + x), __ldg(damp_b + g.n0 + y)), __ldg(damp_b + g.n0 + g.n1 + z)),
                   c2);
}
// neighbour at offset o along axis d of the in-grid point (x, y, z): only
// that coordinate can leave the grid
template <int D>
__device__ __forceinline__ float ld_ax(const PhysGrid& g, const float* __restrict__ f, size_t i0, int x, int y, int z,
                                       int o) {
  const int c = D == 0 ? x : (D == 1 ? y : z);
  const int n = D == 0 ? g.n0 : (D == 1 ? g.n1 : g.n2);
  const ptrdiff_t st = D == 0 ? (ptrdiff_t)g.n1 * g.n2p : (D == 1 ? (ptrdiff_t)g.n2p : 1);
  return (unsigned)(c + o) < (unsigned)n ? __ldg(f + (ptrdiff_t)i0 + o * st) : 0.f;
}
// centred Laplacian in differences form at the in-grid point (x, y, z)
// (w2[d][i-1] = c_i / h_d^2)
template <int R>
__device__ __forceinline__ float lap_at(const PhysGrid& g, const float* __restrict__ f, const LapW& w, int x, int y,
                                        int z) {
  const size_t i0 = aidx(g, x, y, z);
  const float u = __ldg(f + i0);
  float l = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float s = 0.f;
#pragma unroll
    for (int i = 1; i <= R; ++i) {
      const float a = d == 0 ? ld_ax<0>(g, f, i0, x, y, z, i) : (d == 1 ? ld_ax<1>(g, f, i0, x, y, z, i) : ld_ax<2>(g, f, i0, x, y, z, i));
      const float b = d == 0 ? ld_ax<0>(g, f, i0, x, y, z, -i) : (d == 1 ? ld_ax<1>(g, f, i0, x, y, z, -i) : ld_ax<2>(g, f, i0, x, y, z, -i));
      s = __fmaf_rn(w.c[d][i - 1], __fadd_rn(__fsub_rn(a, u), __fsub_rn(b, u)), s);
    }
    l = __fadd_rn(l, s);
  }
  return l;
}
// n / den, exact when den is 1 (outside the sponge) without a division
__device__ __forceinline__ float div_sponge(float n, float den) { return den == 1.f ? n : __fdiv_rn(n, den); }
}  // namespace

// w = D lam^{k+1}
__global__ void k_adj_scale(PhysGrid g, const float* __restrict__ lam1, const float* __restrict__ c2,
                            const float* __restrict__ damp_b, float* __restrict__ w) {
  const AdjCol c = adj_col(g);
  if (!c.ok) return;
  const int x = blockIdx.z;
  const size_t i0 = aidx(g, x, c.y, c.z);
  const float cc = __ldg(c2 + i0);
  const float gd = damp_g(g, damp_b, cc, x, c.y, c.z);
  w[i0] = div_sponge(__fmul_rn(cc, lam1[i0]), __fadd_rn(1.f, gd));
}

// lam^{k} = L w + B lam^{k+1} + C lam^{k+2} (before the residual injection)
template <int R>
__global__ void k_adj_step(PhysGrid g, LapW lw, const float* __restrict__ w, const float* __restrict__ lam1,
                           const float* __restrict__ lam2, const float* __restrict__ c2,
                           const float* __restrict__ damp_b, float* __restrict__ lam0) {
  const AdjCol c = adj_col(g);
  if (!c.ok) return;
  const int x = blockIdx.z;
  const size_t i0 = aidx(g, x, c.y, c.z);
  const float gd = damp_g(g, damp_b, __ldg(c2 + i0), x, c.y, c.z);
  const float opg = __fadd_rn(1.f, gd);
  const float l = lap_at<R>(g, w, lw, x, c.y, c.z);
  lam0[i0] = __fadd_rn(l, div_sponge(__fmaf_rn(2.f, lam1[i0], __fmul_rn(__fsub_rn(gd, 1.f), lam2[i0])), opg));
}

// grad_m += lam^k c2 [2 g (u^{k-1} - u^{k-2}) - c2 L u^{k-1}] / (dt^2 (1+g)^2).  By the
// forward recurrence, (1+g) (u^k - c2 S^{k-1}) = c2 L u^{k-1} + 2 u^{k-1} - (1-g) u^{k-2},
// the bracket equals -(1+g) [(u^k - c2 S^{k-1}) - 2 u^{k-1} + u^{k-2}]: the term is
// -lam^k c2 [(u^k - u^{k-1}) - (u^{k-1} - u^{k-2})] / (dt^2 (1+g)), pointwise on three
// stored states (no stencil), with the c2 S part added at the source points
// (k_adj_grad_src).  The term in FP32 (the differences of neighbouring states
// first), the sum over steps in FP64.
__global__ void k_adj_grad(PhysGrid g, float inv_dt2, const float* __restrict__ lam0, const float* __restrict__ u0,
                           const float* __restrict__ u1, const float* __restrict__ u2, const float* __restrict__ c2,
                           const float* __restrict__ damp_b, double* __restrict__ gm) {
  const AdjCol c = adj_col(g);
  if (!c.ok) return;
  const int x = blockIdx.z;
  const size_t i0 = aidx(g, x, c.y, c.z);
  const float cc = __ldg(c2 + i0);
  const float gd = damp_g(g, damp_b, cc, x, c.y, c.z);
  const float b1 = __ldg(u1 + i0);
  const float d2 = __fsub_rn(__fsub_rn(__ldg(u0 + i0), b1), __fsub_rn(b1, __ldg(u2 + i0)));
  const float dr = div_sponge(__fmul_rn(__fmul_rn(cc, d2), inv_dt2), __fadd_rn(1.f, gd));
  gm[i0] -= (double)__ldg(lam0 + i0) * (double)dr;
}

// source points: the term of M = c2 (d(c2 S)/dm = -c2 (c2 S)/dt^2) and the c2 S
// part of the imaging term, +lam^k c2 (c2 S) / (dt^2 (1+g)); together
// grad_m(p_id) -= lam^k c2 (c2 S^{k-1}) g / (dt^2 (1+g))  (src_dcmp = c2 S; zero
// outside the sponge)
__global__ void k_adj_grad_src(PhysGrid g, int64_t npts, const int64_t* __restrict__ lin,
                               const float* __restrict__ dcmp_row, double inv_dt2, const float* __restrict__ lam0,
                               const float* __restrict__ c2, const float* __restrict__ damp_b,
                               double* __restrict__ gm) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= npts) return;
  const int64_t l = lin[id];
  const int z = (int)(l % g.n2), y = (int)((l / g.n2) % g.n1), x = (int)(l / ((int64_t)g.n1 * g.n2));
  const size_t i0 = aidx(g, x, y, z);
  const float cc = c2[i0];
  const double gd = (double)damp_g(g, damp_b, cc, x, y, z);
  gm[i0] -= (double)lam0[i0] * (double)cc * (double)dcmp_row[id] * inv_dt2 * (gd / (1.0 + gd));
}

// source-wavelet gradient row: value at each source point of M lam = c2 lam
__global__ void k_adj_sample_src(PhysGrid g, int64_t npts, const int2* __restrict__ ent,
                                 const int64_t* __restrict__ lin, const float* __restrict__ lam0,
                                 const float* __restrict__ c2, float* __restrict__ row) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npts) return;
  const int64_t l = lin[ent[e].y];
  const int z = (int)(l % g.n2), y = (int)((l / g.n2) % g.n1), x = (int)(l / ((int64_t)g.n1 * g.n2));
  const size_t i0 = aidx(g, x, y, z);
  row[e] = __fmul_rn(c2[i0], lam0[i0]);
}

// grad_vp = grad_m * (-2 / vp^3), vp = sqrt(c2)/dt, into a dense [n0][n1][n2] array
__global__ void k_adj_finish(PhysGrid g, double dt, const double* __restrict__ gm, const float* __restrict__ c2,
                             float* __restrict__ out) {
  const AdjCol c = adj_col(g);
  if (!c.ok) return;
  const int x = blockIdx.z;
  const size_t i0 = aidx(g, x, c.y, c.z);
  const double vp = sqrt((double)c2[i0]) / dt;
  out[((size_t)x * g.n1 + c.y) * g.n2 + c.z] = (float)(gm[i0] * (-2.0 / (vp * vp * vp)));
}

static dim3 adj_grid(const PhysGrid& g) {
  return dim3((unsigned)((g.n2 + 31) / 32), (unsigned)((g.n1 + 7) / 8), (unsigned)g.n0);
}

template <int R>
static cudaError_t adj_step_r(const PhysGrid& g, const LapW& lw, const float* lam1, const float* lam2, float* lam0,
                              float* w, const float* c2, const float* damp_b, cudaStream_t st) {
  count_launch(2);
  k_adj_scale<<<adj_grid(g), dim3(32, 8), 0, st>>>(g, lam1, c2, damp_b, w);
  k_adj_step<R><<<adj_grid(g), dim3(32, 8), 0, st>>>(g, lw, w, lam1, lam2, c2, damp_b, lam0);
  return cudaGetLastError();
}
cudaError_t adjoint_step(int R, const PhysGrid& g, const LapW& lw, const float* lam1, const float* lam2, float* lam0,
                         float* w, const float* c2, const float* damp_b, cudaStream_t st) {
  switch (R) {
    case 2: return adj_step_r<2>(g, lw, lam1, lam2, lam0, w, c2, damp_b, st);
    case 4: return adj_step_r<4>(g, lw, lam1, lam2, lam0, w, c2, damp_b, st);
    case 6: return adj_step_r<6>(g, lw, lam1, lam2, lam0, w, c2, damp_b, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t adjoint_grad(const PhysGrid& g, double dt, const float* lam0, const float* u0, const float* u1,
                         const float* u2, const float* c2, const float* damp_b, double* gm, cudaStream_t st) {
  count_launch();
  k_adj_grad<<<adj_grid(g), dim3(32, 8), 0, st>>>(g, (float)(1.0 / (dt * dt)), lam0, u0, u1, u2, c2, damp_b, gm);
  return cudaGetLastError();
}

cudaError_t adjoint_grad_src(const PhysGrid& g, int64_t npts, const int64_t* lin, const float* dcmp_row, double dt,
                             const float* lam0, const float* c2, const float* damp_b, double* gm, cudaStream_t st) {
  if (npts <= 0) return cudaSuccess;
  count_launch();
  k_adj_grad_src<<<grid_for(npts, 128), 128, 0, st>>>(g, npts, lin, dcmp_row, 1.0 / (dt * dt), lam0, c2, damp_b, gm);
  return cudaGetLastError();
}

cudaError_t adjoint_sample_src(const PhysGrid& g, int64_t npts, const int2* ent, const int64_t* lin,
                               const float* lam0, const float* c2, float* row, cudaStream_t st) {
  if (npts <= 0) return cudaSuccess;
  count_launch();
  k_adj_sample_src<<<grid_for(npts, 128), 128, 0, st>>>(g, npts, ent, lin, lam0, c2, row);
  return cudaGetLastError();
}

cudaError_t adjoint_finish(const PhysGrid& g, double dt, const double* gm, const float* c2, float* out,
                           cudaStream_t st) {
  count_launch();
  k_adj_finish<<<adj_grid(g), dim3(32, 8), 0, st>>>(g, dt, gm, c2, out);
  return cudaGetLastError();
}

}  // namespace tbi

namespace tbi {
// out[c][r] = in[r][c] for a rows x cols float matrix
__global__ void k_transpose(int64_t rows, int64_t cols, const float* __restrict__ in, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const int64_t r = i / cols, c = i - r * cols;
  out[c * rows + r] = in[i];
}
cudaError_t transpose_f32(int64_t rows, int64_t cols, const float* in, float* out, cudaStream_t st) {
  if (rows * cols <= 0) return cudaSuccess;
  count_launch();
  k_transpose<<<grid_for(rows * cols, 256), 256, 0, st>>>(rows, cols, in, out);
  return cudaGetLastError();
}
}  // namespace tbi
