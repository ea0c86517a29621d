// Adjoint of the acoustic one-step recurrence and the adjoint-state
// gradient with respect to vp (the FWI / RTM use of the propagator, Sec. I).
//
// Forward, per point: u^{k} = D L u^{k-1} + B u^{k-1} + C u^{k-2} + M S^{k-1}
// with, in the library's variables c2 = dt^2/m and g = a/m (a = eta dt/2),
//   D = c2/(1+g),  B = 2/(1+g),  C = (g-1)/(1+g),  M = c2,
// receivers d[k-1] = P u^{k}.  Adjoint for residual traces r (backward):
//   lam^{k} = L (D lam^{k+1}) + B lam^{k+1} + C lam^{k+2} + P^T r[k-1]
// (the centred Laplacian is symmetric).  B, C and D are pointwise, so
// mu = D lam obeys the forward recurrence itself, backward in time:
//   mu^{k} = D L mu^{k+1} + B mu^{k+1} + C mu^{k+2} + D P^T r[k-1],
// which the forward sweep kernel computes (the residual injected at the
// receiver points, scaled by D).  The gradient of <d, r>,
//   d/dm(p) = sum_k lam^k c2 [2 g (u^{k-1} - u^{k-2}) - c2 L u^{k-1}] / (dt^2 (1+g)^2)
//             - sum_k lam^k c2 S^{k-1} c2 / dt^2,
// becomes, with the forward recurrence for c2 L u^{k-1} (see k_adj_grad),
//   d/dm(p) = -sum_k mu^k [(u^k - u^{k-1}) - (u^{k-1} - u^{k-2})] / dt^2
//             - sum_k mu^k (c2 S^{k-1}) g / dt^2     (source points),
//   d/dvp = d/dm * (-2/vp^3),  vp = sqrt(c2)/dt,
// accumulated in FP64 (the per-step term in FP32).
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
// g = (sum of per-axis eta/(2 dt)) * c2
__device__ __forceinline__ float damp_g(const PhysGrid& g, const float* __restrict__ damp_b, float c2, int x, int y,
                                        int z) {
  return __fmul_rn(__fadd_rn(__fadd_rn(__ldg(damp_b + x), __ldg(damp_b + g.n0 + y)), __ldg(damp_b + g.n0 + g.n1 + z)),
                   c2);
}
// n / den, exact when den is 1 (outside the sponge) without a division
__device__ __forceinline__ float div_sponge(float n, float den) { return den == 1.f ? n : __fdiv_rn(n, den); }
}  // namespace

// rows[t][id] *= D(p_id) = c2/(1+g): the residual injection of the mu recurrence
__global__ void k_adj_scale_rows(PhysGrid g, int nt, int64_t npts, const int64_t* __restrict__ lin,
                                 const float* __restrict__ c2, const float* __restrict__ damp_b,
                                 float* __restrict__ rows) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nt * npts) return;
  const int64_t l = lin[i % npts];
  const int z = (int)(l % g.n2), y = (int)((l / g.n2) % g.n1), x = (int)(l / ((int64_t)g.n1 * g.n2));
  const size_t i0 = aidx(g, x, y, z);
  const float cc = __ldg(c2 + i0);
  rows[i] = div_sponge(__fmul_rn(cc, rows[i]), __fadd_rn(1.f, damp_g(g, damp_b, cc, x, y, z)));
}

// grad_m += lam^k c2 [2 g (u^{k-1} - u^{k-2}) - c2 L u^{k-1}] / (dt^2 (1+g)^2).  By the
// forward recurrence, (1+g) (u^k - c2 S^{k-1}) = c2 L u^{k-1} + 2 u^{k-1} - (1-g) u^{k-2},
// the bracket equals -(1+g) [(u^k - c2 S^{k-1}) - 2 u^{k-1} + u^{k-2}], and with
// lam = mu (1+g)/c2 the term is -mu^k [(u^k - u^{k-1}) - (u^{k-1} - u^{k-2})] / dt^2:
// pointwise on three stored states, no stencil; the c2 S part is added at the
// source points (k_adj_grad_src).  The term in FP32 (the differences of
// neighbouring states first), the sum over steps in FP64.
__global__ void k_adj_grad(PhysGrid g, float inv_dt2, const float* __restrict__ mu, const float* __restrict__ u0,
                           const float* __restrict__ u1, const float* __restrict__ u2, double* __restrict__ gm) {
  const AdjCol c = adj_col(g);
  if (!c.ok) return;
  const int x = blockIdx.z;
  const size_t i0 = aidx(g, x, c.y, c.z);
  const float b1 = __ldg(u1 + i0);
  const float d2 = __fsub_rn(__fsub_rn(__ldg(u0 + i0), b1), __fsub_rn(b1, __ldg(u2 + i0)));
  gm[i0] -= (double)__ldg(mu + i0) * (double)__fmul_rn(d2, inv_dt2);
}

// source points: the term of M = c2 (d(c2 S)/dm = -c2 (c2 S)/dt^2) and the c2 S
// part of the imaging term, +lam^k c2 (c2 S) / (dt^2 (1+g)); together
// -lam^k c2 (c2 S^{k-1}) g / (dt^2 (1+g)) = -mu^k (c2 S^{k-1}) g / dt^2
// (src_dcmp = c2 S; zero outside the sponge)
__global__ void k_adj_grad_src(PhysGrid g, int64_t npts, const int64_t* __restrict__ lin,
                               const float* __restrict__ dcmp_row, double inv_dt2, const float* __restrict__ mu,
                               const float* __restrict__ c2, const float* __restrict__ damp_b,
                               double* __restrict__ gm) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= npts) return;
  const int64_t l = lin[id];
  const int z = (int)(l % g.n2), y = (int)((l / g.n2) % g.n1), x = (int)(l / ((int64_t)g.n1 * g.n2));
  const size_t i0 = aidx(g, x, y, z);
  const double gd = (double)damp_g(g, damp_b, c2[i0], x, y, z);
  gm[i0] -= (double)mu[i0] * (double)dcmp_row[id] * gd * inv_dt2;
}

// source-wavelet gradient row: value at each source point of M lam = c2 lam = (1+g) mu
__global__ void k_adj_sample_src(PhysGrid g, int64_t npts, const int2* __restrict__ ent,
                                 const int64_t* __restrict__ lin, const float* __restrict__ mu,
                                 const float* __restrict__ c2, const float* __restrict__ damp_b,
                                 float* __restrict__ row) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npts) return;
  const int64_t l = lin[ent[e].y];
  const int z = (int)(l % g.n2), y = (int)((l / g.n2) % g.n1), x = (int)(l / ((int64_t)g.n1 * g.n2));
  const size_t i0 = aidx(g, x, y, z);
  row[e] = __fmul_rn(__fadd_rn(1.f, damp_g(g, damp_b, c2[i0], x, y, z)), mu[i0]);
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

cudaError_t adjoint_scale_rows(const PhysGrid& g, int nt, int64_t npts, const int64_t* lin, const float* c2,
                               const float* damp_b, float* rows, cudaStream_t st) {
  if (npts <= 0 || nt <= 0) return cudaSuccess;
  count_launch();
  k_adj_scale_rows<<<grid_for((int64_t)nt * npts, 256), 256, 0, st>>>(g, nt, npts, lin, c2, damp_b, rows);
  return cudaGetLastError();
}

cudaError_t adjoint_grad(const PhysGrid& g, double dt, const float* mu, const float* u0, const float* u1,
                         const float* u2, double* gm, cudaStream_t st) {
  count_launch();
  k_adj_grad<<<adj_grid(g), dim3(32, 8), 0, st>>>(g, (float)(1.0 / (dt * dt)), mu, u0, u1, u2, gm);
  return cudaGetLastError();
}

cudaError_t adjoint_grad_src(const PhysGrid& g, int64_t npts, const int64_t* lin, const float* dcmp_row, double dt,
                             const float* mu, const float* c2, const float* damp_b, double* gm, cudaStream_t st) {
  if (npts <= 0) return cudaSuccess;
  count_launch();
  k_adj_grad_src<<<grid_for(npts, 128), 128, 0, st>>>(g, npts, lin, dcmp_row, 1.0 / (dt * dt), mu, c2, damp_b, gm);
  return cudaGetLastError();
}

cudaError_t adjoint_sample_src(const PhysGrid& g, int64_t npts, const int2* ent, const int64_t* lin,
                               const float* mu, const float* c2, const float* damp_b, float* row, cudaStream_t st) {
  if (npts <= 0) return cudaSuccess;
  count_launch();
  k_adj_sample_src<<<grid_for(npts, 128), 128, 0, st>>>(g, npts, ent, lin, mu, c2, damp_b, row);
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
