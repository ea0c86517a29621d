// One-step propagators of the other two wave equations of Sec. III:
//
//   TTI pseudo-acoustic (Sec. III-B, Eq. 2): two fields p, r,
//     m p_tt = (1 + 2 eps) H_h p + sqrt(1 + 2 delta) H_z r
//     m r_tt = sqrt(1 + 2 delta) H_h p + H_z r
//   with H_z r = div(zbar (zbar . grad r)) and H_h p = div(grad p - zbar
//   (zbar . grad p)), grad and div the centred first derivative of order so
//   (fields and fluxes zero outside the grid), zbar = (sin t cos f,
//   sin t sin f, cos t) the symmetry axis of the frame that Eq. 2's rotated
//   derivative belongs to; H_h is -(D_xbar^T D_xbar + D_ybar^T D_ybar)
//   rewritten with the frame's orthonormality (xbar xbar^T + ybar ybar^T =
//   I - zbar zbar^T).  Two kernels per step: the fluxes F = grad p - zbar
//   (zbar . grad p) and G = zbar (zbar . grad r), then their divergences and
//   the leapfrog update of both fields (same damping and increment form as
//   the acoustic kernel).
//
//   Isotropic elastic velocity-stress (Sec. III-C, Eq. 3) on the staggered
//   grid: a velocity kernel (v += dt b div tau) and a stress kernel (tau +=
//   dt (lam tr(e) I + 2 mu e)), each value divided by 1 + eta dt (sponge).
//
// Both stream along axis 0: a thread owns one (y, z) column of a chunk of
// planes and keeps the axis-0 neighbours of its column in a register queue;
// axis-1 and axis-2 neighbours come through the L1 cache.  Source injection
// (grid-aligned table of Sec. II-A) and receiver sampling are separate small
// kernels after the update of each step.
#include <algorithm>
#include <cstddef>
#include <cstdint>

#include "tb_async.cuh"
#include "tb_internal.cuh"

namespace tbi {

static unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Column of a thread: z fastest (coalesced), y from blockIdx.y / threadIdx.y.
struct Col {
  int y, z;
  bool ok;
};
__device__ __forceinline__ Col thread_col(const PhysGrid& g) {
  Col c;
  c.z = blockIdx.x * blockDim.x + threadIdx.x;
  c.y = blockIdx.y * blockDim.y + threadIdx.y;
  c.ok = c.z < g.n2 && c.y < g.n1;
  return c;
}
__device__ __forceinline__ size_t pidx(const PhysGrid& g, int x, int y, int z) {
  return ((size_t)x * g.n1 + y) * g.n2p + z;
}
// value of a padded field at (x, y, z), zero outside the grid
__device__ __forceinline__ float ld0(const PhysGrid& g, const float* __restrict__ f, int x, int y, int z) {
  return (x >= 0 && x < g.n0 && y >= 0 && y < g.n1 && z >= 0 && z < g.n2) ? __ldg(f + pidx(g, x, y, z)) : 0.f;
}

// planes [x0, x1) of the chunk blockIdx.z of nchunks along axis 0 (all chunks
// of a step run in one launch)
__device__ __forceinline__ void chunk_planes(const PhysGrid& g, int nchunks, int& x0, int& x1) {
  x0 = (int)((int64_t)g.n0 * blockIdx.z / nchunks);
  x1 = (int)((int64_t)g.n0 * (blockIdx.z + 1) / nchunks);
}
// n / den, exact when den is 1 (outside the sponge) without a division
__device__ __forceinline__ float div_sponge(float n, float den) { return den == 1.f ? n : __fdiv_rn(n, den); }

// ------------------------------------------------------------------ TTI --
// centred first derivative along axis 1 / 2 at (x, y, z): sum_i a_i (f_{+i} - f_{-i})
// Neighbours of a point inside the grid along one axis: only that axis'
// coordinate can leave the grid, so only it is tested.
__device__ __forceinline__ float ld_y(const PhysGrid& g, const float* __restrict__ f, size_t i0, int y, int dy) {
  return (unsigned)(y + dy) < (unsigned)g.n1 ? __ldg(f + (ptrdiff_t)i0 + (ptrdiff_t)dy * g.n2p) : 0.f;
}
__device__ __forceinline__ float ld_z(const PhysGrid& g, const float* __restrict__ f, size_t i0, int z, int dz) {
  return (unsigned)(z + dz) < (unsigned)g.n2 ? __ldg(f + (ptrdiff_t)i0 + dz) : 0.f;
}
template <int R>
__device__ __forceinline__ float dc_y(const PhysGrid& g, const float* f, const float* a, int x, int y, int z) {
  const size_t i0 = pidx(g, x, y, z);
  float s = 0.f;
#pragma unroll
  for (int i = R; i >= 1; --i) s = __fmaf_rn(a[i - 1], __fsub_rn(ld_y(g, f, i0, y, i), ld_y(g, f, i0, y, -i)), s);
  return s;
}
template <int R>
__device__ __forceinline__ float dc_z(const PhysGrid& g, const float* f, const float* a, int x, int y, int z) {
  const size_t i0 = pidx(g, x, y, z);
  float s = 0.f;
#pragma unroll
  for (int i = R; i >= 1; --i) s = __fmaf_rn(a[i - 1], __fsub_rn(ld_z(g, f, i0, z, i), ld_z(g, f, i0, z, -i)), s);
  return s;
}
template <int R>
__device__ __forceinline__ float dc_q(const float* q, const float* a) {  // q[R] is the centre
  float s = 0.f;
#pragma unroll
  for (int i = R; i >= 1; --i) s = __fmaf_rn(a[i - 1], __fsub_rn(q[R + i], q[R - i]), s);
  return s;
}

// pass 1: F = grad p - zbar (zbar . grad p), G = zbar (zbar . grad r) on
// planes [x0, x1) of column c.  Reads p, r on planes x0 - R .. x1 - 1 + R.
template <int R>
__device__ __forceinline__ void tti_flux_cols(const PhysGrid& g, const DerivW& w, const Col& c, int x0, int x1,
                                              const float* __restrict__ p, const float* __restrict__ r,
                                              const float* __restrict__ nz, float* __restrict__ flux) {
  const size_t Np = (size_t)g.n0 * g.n1 * g.n2p;
  float qp[2 * R + 1], qr[2 * R + 1];
  qp[0] = qr[0] = 0.f;  // shifted out before its first use
#pragma unroll
  for (int s = 1; s < 2 * R + 1; ++s) {  // planes x0-R .. x0+R-1 before the first shift
    qp[s] = ld0(g, p, x0 - 1 - R + s, c.y, c.z);
    qr[s] = ld0(g, r, x0 - 1 - R + s, c.y, c.z);
  }
  for (int x = x0; x < x1; ++x) {
#pragma unroll
    for (int s = 0; s < 2 * R; ++s) {
      qp[s] = qp[s + 1];
      qr[s] = qr[s + 1];
    }
    qp[2 * R] = ld0(g, p, x + R, c.y, c.z);
    qr[2 * R] = ld0(g, r, x + R, c.y, c.z);
    const size_t i0 = pidx(g, x, c.y, c.z);
    const float gp0 = dc_q<R>(qp, w.a[0]), gp1 = dc_y<R>(g, p, w.a[1], x, c.y, c.z),
                gp2 = dc_z<R>(g, p, w.a[2], x, c.y, c.z);
    const float gr0 = dc_q<R>(qr, w.a[0]), gr1 = dc_y<R>(g, r, w.a[1], x, c.y, c.z),
                gr2 = dc_z<R>(g, r, w.a[2], x, c.y, c.z);
    const float n0 = __ldg(nz + i0), n1 = __ldg(nz + Np + i0), n2 = __ldg(nz + 2 * Np + i0);
    const float sp = __fmaf_rn(n2, gp2, __fmaf_rn(n1, gp1, __fmul_rn(n0, gp0)));
    const float sr = __fmaf_rn(n2, gr2, __fmaf_rn(n1, gr1, __fmul_rn(n0, gr0)));
    flux[i0] = __fmaf_rn(-n0, sp, gp0);
    flux[Np + i0] = __fmaf_rn(-n1, sp, gp1);
    flux[2 * Np + i0] = __fmaf_rn(-n2, sp, gp2);
    flux[3 * Np + i0] = __fmul_rn(n0, sr);
    flux[4 * Np + i0] = __fmul_rn(n1, sr);
    flux[5 * Np + i0] = __fmul_rn(n2, sr);
  }
}
template <int R>
__global__ void __launch_bounds__(256) k_tti_flux(PhysGrid g, DerivW w, int nchunks, const float* __restrict__ p,
                                                  const float* __restrict__ r, const float* __restrict__ nz,
                                                  float* __restrict__ flux) {
  const Col c = thread_col(g);
  if (!c.ok) return;
  int x0, x1;
  chunk_planes(g, nchunks, x0, x1);
  tti_flux_cols<R>(g, w, c, x0, x1, p, r, nz, flux);
}

// pass 2: H_h p = div F, H_z r = div G; leapfrog update of p and r written
// over p^{n-1}, r^{n-1} on planes [x0, x1) of column c.  Reads the fluxes on
// planes x0 - R .. x1 - 1 + R.
template <int R>
__device__ __forceinline__ void tti_update_cols(const PhysGrid& g, const DerivW& w, const Col& c, int x0, int x1,
                                                const float* __restrict__ flux, const float* __restrict__ pc, float* pp,
                                                const float* __restrict__ rc, float* rp, const float* __restrict__ c2,
                                                const float* __restrict__ coef, const float* __restrict__ damp_b) {
  const size_t Np = (size_t)g.n0 * g.n1 * g.n2p;
  const float* F0 = flux;
  const float* G0 = flux + 3 * Np;
  float qf[2 * R + 1], qg[2 * R + 1];
  qf[0] = qg[0] = 0.f;
#pragma unroll
  for (int s = 1; s < 2 * R + 1; ++s) {
    qf[s] = ld0(g, F0, x0 - 1 - R + s, c.y, c.z);
    qg[s] = ld0(g, G0, x0 - 1 - R + s, c.y, c.z);
  }
  const float byz = __fadd_rn(__ldg(damp_b + g.n0 + c.y), __ldg(damp_b + g.n0 + g.n1 + c.z));
  for (int x = x0; x < x1; ++x) {
#pragma unroll
    for (int s = 0; s < 2 * R; ++s) {
      qf[s] = qf[s + 1];
      qg[s] = qg[s + 1];
    }
    qf[2 * R] = ld0(g, F0, x + R, c.y, c.z);
    qg[2 * R] = ld0(g, G0, x + R, c.y, c.z);
    const size_t i0 = pidx(g, x, c.y, c.z);
    const float hh = __fadd_rn(__fadd_rn(dc_q<R>(qf, w.a[0]), dc_y<R>(g, flux + Np, w.a[1], x, c.y, c.z)),
                               dc_z<R>(g, flux + 2 * Np, w.a[2], x, c.y, c.z));
    const float hz = __fadd_rn(__fadd_rn(dc_q<R>(qg, w.a[0]), dc_y<R>(g, flux + 4 * Np, w.a[1], x, c.y, c.z)),
                               dc_z<R>(g, flux + 5 * Np, w.a[2], x, c.y, c.z));
    const float cpp = __ldg(coef + i0), cpr = __ldg(coef + Np + i0);
    const float rhs_p = __fmaf_rn(cpp, hh, __fmul_rn(cpr, hz));
    const float rhs_r = __fmaf_rn(cpr, hh, hz);
    const float c2v = __ldg(c2 + i0);
    const float gdamp = __fmul_rn(__fadd_rn(__ldg(damp_b + x), byz), c2v);
    const float opg = __fadd_rn(1.f, gdamp), omg = __fsub_rn(1.f, gdamp);
    const float up = pc[i0], upp = pp[i0], ur = rc[i0], urp = rp[i0];
    pp[i0] = __fadd_rn(up, div_sponge(__fmaf_rn(c2v, rhs_p, __fmul_rn(omg, __fsub_rn(up, upp))), opg));
    rp[i0] = __fadd_rn(ur, div_sponge(__fmaf_rn(c2v, rhs_r, __fmul_rn(omg, __fsub_rn(ur, urp))), opg));
  }
}
template <int R>
__global__ void __launch_bounds__(256) k_tti_update(PhysGrid g, DerivW w, int nchunks, const float* __restrict__ flux,
                                                    const float* __restrict__ pc, float* pp, const float* __restrict__ rc,
                                                    float* rp, const float* __restrict__ c2,
                                                    const float* __restrict__ coef, const float* __restrict__ damp_b) {
  const Col c = thread_col(g);
  if (!c.ok) return;
  int x0, x1;
  chunk_planes(g, nchunks, x0, x1);
  tti_update_cols<R>(g, w, c, x0, x1, flux, pc, pp, rc, rp, c2, coef, damp_b);
}

// ------------------------------------------------------- fused TTI step --
// Both passes of a TTI step in one kernel.  A CTA owns a tile of kFY x TZ
// columns and streams a chunk of planes; one thread per column of the tile
// widened by r on each side along axes 1 and 2.  At flux plane x every
// thread takes p, r of its column from register queues (planes x - r ..
// x + r) and the axis-1/2 neighbours from shared planes that reach 2r beyond
// the tile, and computes F, G there: F0, G0 stay in the owning thread's
// register queue (planes x - 2r .. x), F1, G1 (rows -r .. kFY + r) and F2,
// G2 (columns -r .. TZ + r) go into a ring of r + 1 shared planes.  The
// update of plane x - r then reads all six fluxes on chip.  Every operation
// is that of k_tti_flux and k_tti_update in the same order (fluxes zero
// outside the grid), so the step equals the two-kernel step bit for bit,
// and the fluxes never reach memory (per point and step: p, r, p^{n-1},
// r^{n-1}, the six coefficients read, p, r written).
constexpr int kFY = 8;
template <int R>
struct TtiFusedCfg {
  static constexpr int TZ = R == 2 ? 32 : 24;               // tile columns (about 512-720 threads)
  static constexpr int EH = kFY + 2 * R, EW = TZ + 2 * R;   // thread columns
  static constexpr int NT = EH * EW;
  static constexpr int PH = kFY + 4 * R, PW = TZ + 4 * R;   // shared p, r planes
  static constexpr int NFAR = 2 * R * (kFY + TZ);          // plane cells read beyond the thread columns
  static constexpr int NRING = R + 1;                      // flux planes kept for the divergence
  static constexpr int FYS = EH * TZ, FZS = kFY * EW;     // F1 / G1 and F2 / G2 plane sizes
  static constexpr int SMEM = (int)sizeof(float) * (2 * PH * PW + NRING * 2 * (FYS + FZS));
  static_assert(NFAR <= NT && NT <= 1024, "thread columns");
};

// d/dy, d/dz of a shared plane with row pitch `pitch` at index c: the sums
// of dc_y / dc_z (offsets r .. 1, zeros outside the grid already stored)
template <int R>
__device__ __forceinline__ float dcs(const float* f, int c, int step, const float* a) {
  float s = 0.f;
#pragma unroll
  for (int i = R; i >= 1; --i) s = __fmaf_rn(a[i - 1], __fsub_rn(f[c + i * step], f[c - i * step]), s);
  return s;
}

// Every global value a step needs (p, r at plane x + r, the far cells at x,
// the frame at x, the update's operands at x - r) is loaded one step ahead,
// so that a step's loads are in flight during the previous step's work.
template <int R>
__device__ __forceinline__ void tti_fused_tile(const PhysGrid& g, const DerivW& w, int y0, int z0, int x0, int x1,
                                               const float* __restrict__ pc, float* pp, const float* __restrict__ rc,
                                               float* rp, const float* __restrict__ c2, const float* __restrict__ coef,
                                               const float* __restrict__ nz, const float* __restrict__ damp_b,
                                               float* sm) {
  using C = TtiFusedCfg<R>;
  constexpr int TZ = C::TZ;
  const size_t Np = (size_t)g.n0 * g.n1 * g.n2p;
  const int t = threadIdx.x;
  const int ey = t / C::EW - R, ez = t % C::EW - R;  // column relative to the tile
  const int y = y0 + ey, z = z0 + ez;
  const bool in_yz = (unsigned)y < (unsigned)g.n1 && (unsigned)z < (unsigned)g.n2;
  const bool ycross = ez >= 0 && ez < TZ;   // F1, G1 wanted here
  const bool zcross = ey >= 0 && ey < kFY;  // F2, G2 wanted here
  const bool own = ycross && zcross;
  const bool flux_col = in_yz && (ycross || zcross);
  const bool upd_col = own && in_yz;
  float* sp = sm;
  float* sr = sm + C::PH * C::PW;
  float* ring = sm + 2 * C::PH * C::PW;  // [NRING][F1 | G1 | F2 | G2]
  const int cs = (ey + 2 * R) * C::PW + ez + 2 * R;  // this column in the shared planes
  // the far cell of this thread: 2r rows beyond the thread rows at the tile's
  // columns, 2r columns beyond the thread columns at the tile's rows
  int fy = 0, fz = 0;
  const bool far = t < C::NFAR;
  if (far) {
    if (t < 2 * R * TZ) {
      const int row = t / TZ;
      fy = row < R ? row - 2 * R : kFY + row;
      fz = t % TZ;
    } else {
      const int f = t - 2 * R * TZ, col = f % (2 * R);
      fy = f / (2 * R);
      fz = col < R ? col - 2 * R : TZ + col;
    }
  }
  const int fyg = y0 + fy, fzg = z0 + fz;
  const bool far_in = far && (unsigned)fyg < (unsigned)g.n1 && (unsigned)fzg < (unsigned)g.n2;
  const int cf = (fy + 2 * R) * C::PW + fz + 2 * R;
  const size_t col = (size_t)(in_yz ? y : 0) * g.n2p + (in_yz ? z : 0);
  const size_t colf = (size_t)(far_in ? fyg : 0) * g.n2p + (far_in ? fzg : 0);
  const size_t plane = (size_t)g.n1 * g.n2p;
  auto ldx = [&](const float* f, size_t c, bool ok, int x) -> float {
    return (ok && (unsigned)x < (unsigned)g.n0) ? __ldg(f + (size_t)x * plane + c) : 0.f;
  };
  float qp[2 * R + 1], qr[2 * R + 1], qf[2 * R + 1], qg[2 * R + 1];
  const int xs = x0 - R, xe = x1 + R;  // flux planes
  qp[0] = qr[0] = 0.f;  // shifted out before its first use
#pragma unroll
  for (int s = 1; s < 2 * R + 1; ++s) {  // planes xs - r .. xs + r - 1
    qp[s] = ldx(pc, col, in_yz, xs - 1 - R + s);
    qr[s] = ldx(rc, col, in_yz, xs - 1 - R + s);
  }
#pragma unroll
  for (int s = 0; s < 2 * R + 1; ++s) qf[s] = qg[s] = 0.f;
  const float byz = upd_col ? __fadd_rn(__ldg(damp_b + g.n0 + y), __ldg(damp_b + g.n0 + g.n1 + z)) : 0.f;
  // values of the coming step, loaded one step ahead
  float np_ = 0.f, nr_ = 0.f, fp_ = 0.f, fr_ = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f;
  float o_pp = 0.f, o_rp = 0.f, o_c2 = 0.f, o_cp = 0.f, o_cr = 0.f;
  auto prefetch = [&](int x) {
    np_ = ldx(pc, col, in_yz, x + R);
    nr_ = ldx(rc, col, in_yz, x + R);
    if (far) {
      fp_ = ldx(pc, colf, far_in, x);
      fr_ = ldx(rc, colf, far_in, x);
    }
    if (flux_col && (unsigned)x < (unsigned)g.n0) {
      const size_t i0 = (size_t)x * plane + col;
      m0 = __ldg(nz + i0);
      m1 = __ldg(nz + Np + i0);
      m2 = __ldg(nz + 2 * Np + i0);
    }
    const int u = x - R;
    if (upd_col && u >= x0 && u < x1) {
      const size_t i0 = (size_t)u * plane + col;
      o_pp = pp[i0];
      o_rp = rp[i0];
      o_c2 = __ldg(c2 + i0);
      o_cp = __ldg(coef + i0);
      o_cr = __ldg(coef + Np + i0);
    }
  };
  prefetch(xs);
  for (int x = xs; x < xe; ++x) {
#pragma unroll
    for (int s = 0; s < 2 * R; ++s) {
      qp[s] = qp[s + 1];
      qr[s] = qr[s + 1];
    }
    qp[2 * R] = np_;
    qr[2 * R] = nr_;
    sp[cs] = qp[R];
    sr[cs] = qr[R];
    if (far) {
      sp[cf] = fp_;
      sr[cf] = fr_;
    }
    const bool pin = flux_col && (unsigned)x < (unsigned)g.n0;
    const float n0 = m0, n1 = m1, n2 = m2;
    const float upp = o_pp, urp = o_rp, c2v = o_c2, cpp = o_cp, cpr = o_cr;
    if (x + 1 < xe) prefetch(x + 1);
    __syncthreads();
    float F0 = 0.f, F1 = 0.f, F2 = 0.f, G0 = 0.f, G1 = 0.f, G2 = 0.f;
    if (pin) {
      const float gp0 = dc_q<R>(qp, w.a[0]), gp1 = dcs<R>(sp, cs, C::PW, w.a[1]), gp2 = dcs<R>(sp, cs, 1, w.a[2]);
      const float gr0 = dc_q<R>(qr, w.a[0]), gr1 = dcs<R>(sr, cs, C::PW, w.a[1]), gr2 = dcs<R>(sr, cs, 1, w.a[2]);
      const float spn = __fmaf_rn(n2, gp2, __fmaf_rn(n1, gp1, __fmul_rn(n0, gp0)));
      const float srn = __fmaf_rn(n2, gr2, __fmaf_rn(n1, gr1, __fmul_rn(n0, gr0)));
      F0 = __fmaf_rn(-n0, spn, gp0);
      F1 = __fmaf_rn(-n1, spn, gp1);
      F2 = __fmaf_rn(-n2, spn, gp2);
      G0 = __fmul_rn(n0, srn);
      G1 = __fmul_rn(n1, srn);
      G2 = __fmul_rn(n2, srn);
    }
    float* slot = ring + ((x - xs) % C::NRING) * 2 * (C::FYS + C::FZS);
    if (ycross) {
      slot[(ey + R) * TZ + ez] = F1;
      slot[C::FYS + (ey + R) * TZ + ez] = G1;
    }
    if (zcross) {
      slot[2 * C::FYS + ey * C::EW + ez + R] = F2;
      slot[2 * C::FYS + C::FZS + ey * C::EW + ez + R] = G2;
    }
#pragma unroll
    for (int s = 0; s < 2 * R; ++s) {
      qf[s] = qf[s + 1];
      qg[s] = qg[s + 1];
    }
    qf[2 * R] = F0;
    qg[2 * R] = G0;
    __syncthreads();
    const int u = x - R;  // the plane updated at this step
    if (upd_col && u >= x0) {
      const float* su = ring + ((u - xs) % C::NRING) * 2 * (C::FYS + C::FZS);
      const int cy = (ey + R) * TZ + ez, cz = ey * C::EW + ez + R;
      const float hh = __fadd_rn(__fadd_rn(dc_q<R>(qf, w.a[0]), dcs<R>(su, cy, TZ, w.a[1])),
                                 dcs<R>(su + 2 * C::FYS, cz, 1, w.a[2]));
      const float hz = __fadd_rn(__fadd_rn(dc_q<R>(qg, w.a[0]), dcs<R>(su + C::FYS, cy, TZ, w.a[1])),
                                 dcs<R>(su + 2 * C::FYS + C::FZS, cz, 1, w.a[2]));
      const size_t i0 = (size_t)u * plane + col;
      const float rhs_p = __fmaf_rn(cpp, hh, __fmul_rn(cpr, hz));
      const float rhs_r = __fmaf_rn(cpr, hh, hz);
      const float gdamp = __fmul_rn(__fadd_rn(__ldg(damp_b + u), byz), c2v);
      const float opg = __fadd_rn(1.f, gdamp), omg = __fsub_rn(1.f, gdamp);
      const float up = qp[0], ur = qr[0];
      pp[i0] = __fadd_rn(up, div_sponge(__fmaf_rn(c2v, rhs_p, __fmul_rn(omg, __fsub_rn(up, upp))), opg));
      rp[i0] = __fadd_rn(ur, div_sponge(__fmaf_rn(c2v, rhs_r, __fmul_rn(omg, __fsub_rn(ur, urp))), opg));
    }
  }
}

template <int R>
__global__ void __launch_bounds__(TtiFusedCfg<R>::NT, 1)
    k_tti_fused(PhysGrid g, DerivW w, int nchunks, const float* __restrict__ pc, float* pp,
                const float* __restrict__ rc, float* rp, const float* __restrict__ c2,
                const float* __restrict__ coef, const float* __restrict__ nz, const float* __restrict__ damp_b) {
  extern __shared__ float4 tti_smem4[];
  int x0, x1;
  chunk_planes(g, nchunks, x0, x1);
  tti_fused_tile<R>(g, w, blockIdx.y * kFY, blockIdx.x * TtiFusedCfg<R>::TZ, x0, x1, pc, pp, rc, rp, c2, coef, nz,
                    damp_b,
                    reinterpret_cast<float*>(tti_smem4));
}

// wavefront form: item blockIdx.z is one fused step on one slab (a: p^n,
// b: p^{n-1} -> p^{n+1}, c: r^n, d: r^{n-1} -> r^{n+1})
template <int R>
__global__ void __launch_bounds__(TtiFusedCfg<R>::NT, 1)
    k_tti_fused_wave(PhysGrid g, DerivW w, WaveItems L, const float* __restrict__ c2, const float* __restrict__ coef,
                     const float* __restrict__ nz, const float* __restrict__ damp_b) {
  extern __shared__ float4 tti_smem4[];
  const WaveItem it = L.it[blockIdx.z];
  tti_fused_tile<R>(g, w, blockIdx.y * kFY, blockIdx.x * TtiFusedCfg<R>::TZ, it.x0, it.x1, it.a, it.b, it.c, it.d,
                    c2, coef, nz,
                    damp_b, reinterpret_cast<float*>(tti_smem4));
}

// ------------------------------------------------------------- elastic --
// node -> half-node: sum_k c_k (f[i+k] - f[i-k+1]); half-node -> node:
// sum_k c_k (f[i+k-1] - f[i-k]), along axis d at (x, y, z)
template <int R, int D>
__device__ __forceinline__ float dstag(const PhysGrid& g, const float* f, const float* cw, int x, int y, int z,
                                       bool plus) {
  float s = 0.f;
#pragma unroll
  for (int k = R; k >= 1; --k) {
    const int hi = plus ? k : k - 1, lo = plus ? -(k - 1) : -k;
    const size_t i0 = pidx(g, x, y, z);
    const float a = D == 0 ? ld0(g, f, x + hi, y, z) : (D == 1 ? ld_y(g, f, i0, y, hi) : ld_z(g, f, i0, z, hi));
    const float b = D == 0 ? ld0(g, f, x + lo, y, z) : (D == 1 ? ld_y(g, f, i0, y, lo) : ld_z(g, f, i0, z, lo));
    s = __fmaf_rn(cw[k - 1], __fsub_rn(a, b), s);
  }
  return s;
}

// staggered derivative along axis 0 from a register queue (q[R + s] is
// plane x + s): the same sums as dstag<R, 0>
template <int R>
__device__ __forceinline__ float dstag_q(const float* q, const float* cw, bool plus) {
  float s = 0.f;
#pragma unroll
  for (int k = R; k >= 1; --k) {
    const int hi = plus ? k : k - 1, lo = plus ? -(k - 1) : -k;
    s = __fmaf_rn(cw[k - 1], __fsub_rn(q[R + hi], q[R + lo]), s);
  }
  return s;
}

// fields: [9][Np] vx vy vz txx tyy tzz txy txz tyz; mat: [8][Np] bx by bz lam mu mxy mxz myz.
// Each thread streams its column through the planes of one chunk; the axis-0
// neighbours of the three fields it differentiates along axis 0 sit in
// register queues of planes x-R .. x+R.
// velocity update on planes [x0, x1) of column c; reads the stresses on
// planes x0 - R .. x1 - 1 + R
template <int R>
__device__ __forceinline__ void ela_velocity_cols(const PhysGrid& g, const DerivW& w, const Col& c, float dt, int x0,
                                                  int x1, float* __restrict__ f, const float* __restrict__ mat,
                                                  const float* __restrict__ eta_dt) {
  const size_t Np = (size_t)g.n0 * g.n1 * g.n2p;
  const float *txx = f + 3 * Np, *tyy = f + 4 * Np, *tzz = f + 5 * Np, *txy = f + 6 * Np, *txz = f + 7 * Np,
              *tyz = f + 8 * Np;
  float qa[2 * R + 1], qb[2 * R + 1], qc[2 * R + 1];  // txx, txy, txz
  qa[0] = qb[0] = qc[0] = 0.f;
#pragma unroll
  for (int s = 1; s < 2 * R + 1; ++s) {
    qa[s] = ld0(g, txx, x0 - 1 - R + s, c.y, c.z);
    qb[s] = ld0(g, txy, x0 - 1 - R + s, c.y, c.z);
    qc[s] = ld0(g, txz, x0 - 1 - R + s, c.y, c.z);
  }
  const float ey = __ldg(eta_dt + g.n0 + c.y), ez = __ldg(eta_dt + g.n0 + g.n1 + c.z);
  for (int x = x0; x < x1; ++x) {
#pragma unroll
    for (int s = 0; s < 2 * R; ++s) {
      qa[s] = qa[s + 1];
      qb[s] = qb[s + 1];
      qc[s] = qc[s + 1];
    }
    qa[2 * R] = ld0(g, txx, x + R, c.y, c.z);
    qb[2 * R] = ld0(g, txy, x + R, c.y, c.z);
    qc[2 * R] = ld0(g, txz, x + R, c.y, c.z);
    const size_t i0 = pidx(g, x, c.y, c.z);
    const float fx = __fadd_rn(__fadd_rn(dstag_q<R>(qa, w.a[0], true), dstag<R, 1>(g, txy, w.a[1], x, c.y, c.z, false)),
                               dstag<R, 2>(g, txz, w.a[2], x, c.y, c.z, false));
    const float fy = __fadd_rn(__fadd_rn(dstag_q<R>(qb, w.a[0], false), dstag<R, 1>(g, tyy, w.a[1], x, c.y, c.z, true)),
                               dstag<R, 2>(g, tyz, w.a[2], x, c.y, c.z, false));
    const float fz = __fadd_rn(__fadd_rn(dstag_q<R>(qc, w.a[0], false), dstag<R, 1>(g, tyz, w.a[1], x, c.y, c.z, false)),
                               dstag<R, 2>(g, tzz, w.a[2], x, c.y, c.z, true));
    const float den = __fadd_rn(1.f, __fadd_rn(__fadd_rn(__ldg(eta_dt + x), ey), ez));
    f[i0] = div_sponge(__fmaf_rn(__fmul_rn(dt, __ldg(mat + i0)), fx, f[i0]), den);
    f[Np + i0] = div_sponge(__fmaf_rn(__fmul_rn(dt, __ldg(mat + Np + i0)), fy, f[Np + i0]), den);
    f[2 * Np + i0] = div_sponge(__fmaf_rn(__fmul_rn(dt, __ldg(mat + 2 * Np + i0)), fz, f[2 * Np + i0]), den);
  }
}
template <int R>
__global__ void __launch_bounds__(256, 4) k_ela_velocity(PhysGrid g, DerivW w, float dt, int nchunks, float* __restrict__ f,
                                                      const float* __restrict__ mat, const float* __restrict__ eta_dt) {
  const Col c = thread_col(g);
  if (!c.ok) return;
  int x0, x1;
  chunk_planes(g, nchunks, x0, x1);
  ela_velocity_cols<R>(g, w, c, dt, x0, x1, f, mat, eta_dt);
}

// stress update on planes [x0, x1) of column c; reads the velocities on
// planes x0 - R .. x1 - 1 + R
template <int R>
__device__ __forceinline__ void ela_stress_cols(const PhysGrid& g, const DerivW& w, const Col& c, float dt, int x0,
                                                int x1, float* __restrict__ f, const float* __restrict__ mat,
                                                const float* __restrict__ eta_dt) {
  const size_t Np = (size_t)g.n0 * g.n1 * g.n2p;
  const float *vx = f, *vy = f + Np, *vz = f + 2 * Np;
  float qa[2 * R + 1], qb[2 * R + 1], qc[2 * R + 1];  // vx, vy, vz
  qa[0] = qb[0] = qc[0] = 0.f;
#pragma unroll
  for (int s = 1; s < 2 * R + 1; ++s) {
    qa[s] = ld0(g, vx, x0 - 1 - R + s, c.y, c.z);
    qb[s] = ld0(g, vy, x0 - 1 - R + s, c.y, c.z);
    qc[s] = ld0(g, vz, x0 - 1 - R + s, c.y, c.z);
  }
  const float ey = __ldg(eta_dt + g.n0 + c.y), ez = __ldg(eta_dt + g.n0 + g.n1 + c.z);
  for (int x = x0; x < x1; ++x) {
#pragma unroll
    for (int s = 0; s < 2 * R; ++s) {
      qa[s] = qa[s + 1];
      qb[s] = qb[s + 1];
      qc[s] = qc[s + 1];
    }
    qa[2 * R] = ld0(g, vx, x + R, c.y, c.z);
    qb[2 * R] = ld0(g, vy, x + R, c.y, c.z);
    qc[2 * R] = ld0(g, vz, x + R, c.y, c.z);
    const size_t i0 = pidx(g, x, c.y, c.z);
    const float exx = dstag_q<R>(qa, w.a[0], false);
    const float eyy = dstag<R, 1>(g, vy, w.a[1], x, c.y, c.z, false);
    const float ezz = dstag<R, 2>(g, vz, w.a[2], x, c.y, c.z, false);
    const float gxy = __fadd_rn(dstag<R, 1>(g, vx, w.a[1], x, c.y, c.z, true), dstag_q<R>(qb, w.a[0], true));
    const float gxz = __fadd_rn(dstag<R, 2>(g, vx, w.a[2], x, c.y, c.z, true), dstag_q<R>(qc, w.a[0], true));
    const float gyz = __fadd_rn(dstag<R, 2>(g, vy, w.a[2], x, c.y, c.z, true), dstag<R, 1>(g, vz, w.a[1], x, c.y, c.z, true));
    const float lam = __ldg(mat + 3 * Np + i0), mu = __ldg(mat + 4 * Np + i0);
    const float ltr = __fmul_rn(lam, __fadd_rn(__fadd_rn(exx, eyy), ezz));
    const float den = __fadd_rn(1.f, __fadd_rn(__fadd_rn(__ldg(eta_dt + x), ey), ez));
    const float mu2 = __fmul_rn(2.f, mu);
    f[3 * Np + i0] = div_sponge(__fmaf_rn(dt, __fmaf_rn(mu2, exx, ltr), f[3 * Np + i0]), den);
    f[4 * Np + i0] = div_sponge(__fmaf_rn(dt, __fmaf_rn(mu2, eyy, ltr), f[4 * Np + i0]), den);
    f[5 * Np + i0] = div_sponge(__fmaf_rn(dt, __fmaf_rn(mu2, ezz, ltr), f[5 * Np + i0]), den);
    f[6 * Np + i0] = div_sponge(__fmaf_rn(__fmul_rn(dt, __ldg(mat + 5 * Np + i0)), gxy, f[6 * Np + i0]), den);
    f[7 * Np + i0] = div_sponge(__fmaf_rn(__fmul_rn(dt, __ldg(mat + 6 * Np + i0)), gxz, f[7 * Np + i0]), den);
    f[8 * Np + i0] = div_sponge(__fmaf_rn(__fmul_rn(dt, __ldg(mat + 7 * Np + i0)), gyz, f[8 * Np + i0]), den);
  }
}
template <int R>
__global__ void __launch_bounds__(256, 4) k_ela_stress(PhysGrid g, DerivW w, float dt, int nchunks, float* __restrict__ f,
                                                    const float* __restrict__ mat, const float* __restrict__ eta_dt) {
  const Col c = thread_col(g);
  if (!c.ok) return;
  int x0, x1;
  chunk_planes(g, nchunks, x0, x1);
  ela_stress_cols<R>(g, w, c, dt, x0, x1, f, mat, eta_dt);
}

// ------------------------------------------------- elastic, TMA-staged --
// The velocity and stress updates with every operand staged by TMA: a CTA
// owns a kEY x kEZ tile (one compute thread per column) and streams a range
// of planes; a producer warp loads, per plane x, the planes the axis-1/2
// derivatives read (with an r-cell halo, zeros outside the grid), the
// plane x + r of the three fields differentiated along axis 0 (the head of
// each column's register queue), the fields updated in place and the
// material, into a ring of stages several planes ahead of the compute
// warps.  The per-point arithmetic is that of k_ela_velocity / k_ela_stress
// (same operations in the same order), so the results are bit for bit
// those of the plain kernels.
template <int R>
struct ElaCfg {
  static constexpr int RZ = (R + 3) / 4 * 4;  // axis-2 halo rounded to 16 bytes (TMA)
  static constexpr int HH = kEY + 2 * R, HW = kEZ + 2 * RZ;
  static constexpr int HALO = HH * HW, OWN = kEY * kEZ;
  // velocity: halo planes txy tyy tyz txz tzz (x); own planes txx txy txz
  // (x + r), vx vy vz, bx by bz (x).  Stress: halo planes vx vy vz (x); own
  // planes vx vy vz (x + r), txx .. tyz, lam mu mxy mxz myz (x).
  static constexpr int NHV = 5, NOV = 9, NHS = 3, NOS = 14;
  static constexpr int SV = NHV * HALO + NOV * OWN, SS = NHS * HALO + NOS * OWN;
  static constexpr int STAGE = SV > SS ? SV : SS;  // floats
  static constexpr int NST = 3;                    // stages in flight
  static constexpr int NT = kEY * kEZ + 32;        // compute warps + producer warp
  static constexpr int MINB = R <= 4 ? 3 : 2;      // CTAs per SM the shared memory allows
  static constexpr int SMEM = 4 * NST * STAGE + 16 * NST + 128;  // + alignment of the ring to 128 B
  static_assert(HALO % 32 == 0 && OWN % 32 == 0 && STAGE % 32 == 0, "128-byte aligned TMA boxes");
  static constexpr unsigned BYTES_V = 4u * SV, BYTES_S = 4u * SS;
};

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// staggered derivative along axis 1 or 2 of a shared plane (pitch `step`
// between neighbours): the sums of dstag<R, 1 | 2>
template <int R>
__device__ __forceinline__ float dstag_s(const float* f, int c, int step, const float* cw, bool plus) {
  float s = 0.f;
#pragma unroll
  for (int k = R; k >= 1; --k) {
    const int hi = plus ? k : k - 1, lo = plus ? -(k - 1) : -k;
    s = __fmaf_rn(cw[k - 1], __fsub_rn(f[c + hi * step], f[c + lo * step]), s);
  }
  return s;
}

// kind 0: velocity, 1: stress, on planes [x0, x1) of the tile at (y0, z0)
template <int R>
__device__ __forceinline__ void ela_tma_tile(const PhysGrid& g, const DerivW& w, float dt, const ElaMaps& M,
                                             int kind, int y0, int z0, int x0, int x1, float* __restrict__ f,
                                             const float* __restrict__ eta_dt, float* ring, uint64_t* full,
                                             uint64_t* empty, long long tmo, int* err) {
  using C = ElaCfg<R>;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int nsteps = x1 - x0;
  if (warp == kEY) {
    // ============================ producer warp ============================
    if (lane != 0) return;
    int issued = 0;
    bool ok = true;
    for (int i = 0; i < nsteps && ok; ++i) {
      const int st = i % C::NST, x = x0 + i;
      if (i >= C::NST && !mbar_wait(&empty[st], ((i / C::NST) - 1) & 1, tmo)) {
        atomicExch(err, 1);
        ok = false;
        break;
      }
      float* base = ring + (size_t)st * C::STAGE;
      uint64_t* bar = &full[st];
      if (kind == 0) {
        mbar_expect_tx(bar, C::BYTES_V);
        const int hf[5] = {6, 4, 8, 7, 5};  // txy tyy tyz txz tzz
#pragma unroll
        for (int k = 0; k < 5; ++k) tma_load_4d(base + k * C::HALO, &M.fh, bar, z0 - C::RZ, y0 - R, x, hf[k]);
        float* own = base + C::NHV * C::HALO;
        const int qf[3] = {3, 6, 7};  // txx txy txz at x + r
#pragma unroll
        for (int k = 0; k < 3; ++k) tma_load_4d(own + k * C::OWN, &M.fo, bar, z0, y0, x + R, qf[k]);
#pragma unroll
        for (int k = 0; k < 3; ++k) tma_load_4d(own + (3 + k) * C::OWN, &M.fo, bar, z0, y0, x, k);
#pragma unroll
        for (int k = 0; k < 3; ++k) tma_load_4d(own + (6 + k) * C::OWN, &M.mo, bar, z0, y0, x, k);
      } else {
        mbar_expect_tx(bar, C::BYTES_S);
#pragma unroll
        for (int k = 0; k < 3; ++k) tma_load_4d(base + k * C::HALO, &M.fh, bar, z0 - C::RZ, y0 - R, x, k);
        float* own = base + C::NHS * C::HALO;
#pragma unroll
        for (int k = 0; k < 3; ++k) tma_load_4d(own + k * C::OWN, &M.fo, bar, z0, y0, x + R, k);
#pragma unroll
        for (int k = 0; k < 6; ++k) tma_load_4d(own + (3 + k) * C::OWN, &M.fo, bar, z0, y0, x, 3 + k);
#pragma unroll
        for (int k = 0; k < 5; ++k) tma_load_4d(own + (9 + k) * C::OWN, &M.mo, bar, z0, y0, x, 3 + k);
      }
      issued = i + 1;
    }
    // copies still in flight complete on their stages' full barriers
    for (int i = (issued > C::NST ? issued - C::NST : 0); i < issued; ++i)
      mbar_wait(&full[i % C::NST], (i / C::NST) & 1, tmo);
    return;
  }
  // ============================= compute warps =============================
  const int ey = warp, ez = lane;
  const int y = y0 + ey, z = z0 + ez;
  const bool in = y < g.n1 && z < g.n2;
  const size_t Np = (size_t)g.n0 * g.n1 * g.n2p;
  const size_t col = (size_t)(in ? y : 0) * g.n2p + (in ? z : 0);
  const int ch = (ey + R) * C::HW + ez + C::RZ, co = ey * kEZ + ez;
  // axis-0 queues (planes x - r .. x + r) of txx txy txz (velocity) or vx vy vz (stress)
  const float* q0 = f + (kind == 0 ? 3 * Np : 0);
  const float* q1 = f + (kind == 0 ? 6 * Np : Np);
  const float* q2 = f + (kind == 0 ? 7 * Np : 2 * Np);
  float qa[2 * R + 1], qb[2 * R + 1], qc[2 * R + 1];
  qa[0] = qb[0] = qc[0] = 0.f;  // shifted out before its first use
  const int yc = in ? y : 0, zc = in ? z : 0;
#pragma unroll
  for (int s = 1; s < 2 * R + 1; ++s) {  // planes x0 - r .. x0 + r - 1 before the first shift
    qa[s] = in ? ld0(g, q0, x0 - 1 - R + s, yc, zc) : 0.f;
    qb[s] = in ? ld0(g, q1, x0 - 1 - R + s, yc, zc) : 0.f;
    qc[s] = in ? ld0(g, q2, x0 - 1 - R + s, yc, zc) : 0.f;
  }
  const float eyz_y = __ldg(eta_dt + g.n0 + (in ? y : 0)), eyz_z = __ldg(eta_dt + g.n0 + g.n1 + (in ? z : 0));
  float eta_next = nsteps > 0 ? __ldg(eta_dt + x0) : 0.f;  // the plane's damping, loaded a step ahead
  for (int i = 0; i < nsteps; ++i) {
    const int st = i % C::NST, x = x0 + i;
    const float eta_x = eta_next;
    if (i + 1 < nsteps) eta_next = __ldg(eta_dt + x + 1);
    const bool ok = mbar_wait(&full[st], (i / C::NST) & 1, tmo);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) atomicExch(err, 1);
      break;
    }
    const float* base = ring + (size_t)st * C::STAGE;
#pragma unroll
    for (int s = 0; s < 2 * R; ++s) {
      qa[s] = qa[s + 1];
      qb[s] = qb[s + 1];
      qc[s] = qc[s + 1];
    }
    const float den = __fadd_rn(1.f, __fadd_rn(__fadd_rn(eta_x, eyz_y), eyz_z));
    const size_t i0 = (size_t)x * g.n1 * g.n2p + col;
    if (kind == 0) {
      const float* own = base + C::NHV * C::HALO;
      qa[2 * R] = own[co];
      qb[2 * R] = own[C::OWN + co];
      qc[2 * R] = own[2 * C::OWN + co];
      const float *txy = base, *tyy = base + C::HALO, *tyz = base + 2 * C::HALO, *txz = base + 3 * C::HALO,
                  *tzz = base + 4 * C::HALO;
      const float fx = __fadd_rn(__fadd_rn(dstag_q<R>(qa, w.a[0], true), dstag_s<R>(txy, ch, C::HW, w.a[1], false)),
                                 dstag_s<R>(txz, ch, 1, w.a[2], false));
      const float fy = __fadd_rn(__fadd_rn(dstag_q<R>(qb, w.a[0], false), dstag_s<R>(tyy, ch, C::HW, w.a[1], true)),
                                 dstag_s<R>(tyz, ch, 1, w.a[2], false));
      const float fz = __fadd_rn(__fadd_rn(dstag_q<R>(qc, w.a[0], false), dstag_s<R>(tyz, ch, C::HW, w.a[1], false)),
                                 dstag_s<R>(tzz, ch, 1, w.a[2], true));
      const float vx = own[3 * C::OWN + co], vy = own[4 * C::OWN + co], vz = own[5 * C::OWN + co];
      const float bx = own[6 * C::OWN + co], by = own[7 * C::OWN + co], bz = own[8 * C::OWN + co];
      if (in) {
        f[i0] = div_sponge(__fmaf_rn(__fmul_rn(dt, bx), fx, vx), den);
        f[Np + i0] = div_sponge(__fmaf_rn(__fmul_rn(dt, by), fy, vy), den);
        f[2 * Np + i0] = div_sponge(__fmaf_rn(__fmul_rn(dt, bz), fz, vz), den);
      }
    } else {
      const float* own = base + C::NHS * C::HALO;
      qa[2 * R] = own[co];
      qb[2 * R] = own[C::OWN + co];
      qc[2 * R] = own[2 * C::OWN + co];
      const float *vxp = base, *vyp = base + C::HALO, *vzp = base + 2 * C::HALO;
      const float exx = dstag_q<R>(qa, w.a[0], false);
      const float eyy = dstag_s<R>(vyp, ch, C::HW, w.a[1], false);
      const float ezz = dstag_s<R>(vzp, ch, 1, w.a[2], false);
      const float gxy = __fadd_rn(dstag_s<R>(vxp, ch, C::HW, w.a[1], true), dstag_q<R>(qb, w.a[0], true));
      const float gxz = __fadd_rn(dstag_s<R>(vxp, ch, 1, w.a[2], true), dstag_q<R>(qc, w.a[0], true));
      const float gyz = __fadd_rn(dstag_s<R>(vyp, ch, 1, w.a[2], true), dstag_s<R>(vzp, ch, C::HW, w.a[1], true));
      const float lam = own[9 * C::OWN + co], mu = own[10 * C::OWN + co];
      const float ltr = __fmul_rn(lam, __fadd_rn(__fadd_rn(exx, eyy), ezz));
      const float mu2 = __fmul_rn(2.f, mu);
      const float sxx = own[3 * C::OWN + co], syy = own[4 * C::OWN + co], szz = own[5 * C::OWN + co];
      const float sxy = own[6 * C::OWN + co], sxz = own[7 * C::OWN + co], syz = own[8 * C::OWN + co];
      const float mxy = own[11 * C::OWN + co], mxz = own[12 * C::OWN + co], myz = own[13 * C::OWN + co];
      if (in) {
        f[3 * Np + i0] = div_sponge(__fmaf_rn(dt, __fmaf_rn(mu2, exx, ltr), sxx), den);
        f[4 * Np + i0] = div_sponge(__fmaf_rn(dt, __fmaf_rn(mu2, eyy, ltr), syy), den);
        f[5 * Np + i0] = div_sponge(__fmaf_rn(dt, __fmaf_rn(mu2, ezz, ltr), szz), den);
        f[6 * Np + i0] = div_sponge(__fmaf_rn(__fmul_rn(dt, mxy), gxy, sxy), den);
        f[7 * Np + i0] = div_sponge(__fmaf_rn(__fmul_rn(dt, mxz), gxz, sxz), den);
        f[8 * Np + i0] = div_sponge(__fmaf_rn(__fmul_rn(dt, myz), gyz, syz), den);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
  }
}

// one-step (L.n == 0: `kind` over nchunks chunks of planes) or wavefront items
template <int R>
__global__ void __launch_bounds__(ElaCfg<R>::NT, ElaCfg<R>::MINB)
    k_ela_tma(PhysGrid g, DerivW w, float dt, const __grid_constant__ ElaMaps M, int kind, int nchunks,
              const WaveItems L, float* f, const float* __restrict__ eta_dt, long long tmo, int* err) {
  using C = ElaCfg<R>;
  extern __shared__ float4 ela_smem4[];
  float* ring = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(ela_smem4) + 127) & ~uintptr_t(127));
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)C::NST * C::STAGE);
  uint64_t* empty = full + C::NST;
  if (threadIdx.x == 0) {
    for (int i = 0; i < C::NST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kEY);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int x0, x1;
  if (L.n == 0) {
    chunk_planes(g, nchunks, x0, x1);
  } else {
    const WaveItem& it = L.it[blockIdx.z];
    kind = it.kind;
    x0 = it.x0;
    x1 = it.x1;
  }
  ela_tma_tile<R>(g, w, dt, M, kind, blockIdx.y * kEY, blockIdx.x * kEZ, x0, x1, f, eta_dt, ring, full, empty, tmo,
                  err);
}

// ----------------------------------------------------- TTI, TMA-staged --
// The flux and update passes with every operand staged by TMA, as the
// elastic updates above: per plane x the producer warp loads the planes the
// axis-1/2 derivatives read (p, r for the fluxes; F1, G1, F2, G2 for the
// divergence) with an r-cell halo, the axis-0 queue heads at x + r (p, r;
// F0, G0) and the point's other operands.  Same arithmetic as k_tti_flux /
// k_tti_update, so bit for bit their results.
template <int R>
struct TtiCfg {
  static constexpr int RZ = (R + 3) / 4 * 4;
  static constexpr int HH = kEY + 2 * R, HW = kEZ + 2 * RZ;
  static constexpr int HALO = HH * HW, OWN = kEY * kEZ;
  // flux: halo p r (x); own p r (x + r), n0 n1 n2 (x).  Update: halo F1 G1
  // F2 G2 (x); own F0 G0 (x + r), p^n p^{n-1} r^n r^{n-1} c2 coef0 coef1 (x).
  static constexpr int NHF = 2, NOF = 5, NHU = 4, NOU = 9;
  static constexpr int SF = NHF * HALO + NOF * OWN, SU = NHU * HALO + NOU * OWN;
  static constexpr int STAGE = SF > SU ? SF : SU;
  static constexpr int NST = 3;
  static constexpr int NT = kEY * kEZ + 32;
  static constexpr int MINB = R <= 4 ? 3 : 2;
  static constexpr int SMEM = 4 * NST * STAGE + 16 * NST + 128;
  static constexpr unsigned BYTES_F = 4u * SF, BYTES_U = 4u * SU;
  static_assert(HALO % 32 == 0 && OWN % 32 == 0 && STAGE % 32 == 0, "128-byte aligned TMA boxes");
};

template <int R>
__device__ __forceinline__ void tti_tma_tile(const PhysGrid& g, const DerivW& w, const TtiMaps& M,
                                             const WaveItem& it, int y0, int z0, int x0, int x1,
                                             float* __restrict__ flux, const float* __restrict__ damp_b, float* ring,
                                             uint64_t* full, uint64_t* empty, long long tmo, int* err) {
  using C = TtiCfg<R>;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int nsteps = x1 - x0, kind = it.kind;
  if (warp == kEY) {
    // ============================ producer warp ============================
    if (lane != 0) return;
    int issued = 0;
    for (int i = 0; i < nsteps; ++i) {
      const int st = i % C::NST, x = x0 + i;
      if (i >= C::NST && !mbar_wait(&empty[st], ((i / C::NST) - 1) & 1, tmo)) {
        atomicExch(err, 1);
        break;
      }
      float* base = ring + (size_t)st * C::STAGE;
      uint64_t* bar = &full[st];
      if (kind == 0) {
        mbar_expect_tx(bar, C::BYTES_F);
        tma_load_3d(base, &M.bh[it.ia], bar, z0 - C::RZ, y0 - R, x);
        tma_load_3d(base + C::HALO, &M.bh[it.ic], bar, z0 - C::RZ, y0 - R, x);
        float* own = base + C::NHF * C::HALO;
        tma_load_3d(own, &M.bo[it.ia], bar, z0, y0, x + R);
        tma_load_3d(own + C::OWN, &M.bo[it.ic], bar, z0, y0, x + R);
#pragma unroll
        for (int k = 0; k < 3; ++k) tma_load_4d(own + (2 + k) * C::OWN, &M.nzo, bar, z0, y0, x, k);
      } else {
        mbar_expect_tx(bar, C::BYTES_U);
        const int hf[4] = {1, 4, 2, 5};  // F1 G1 F2 G2
#pragma unroll
        for (int k = 0; k < 4; ++k) tma_load_4d(base + k * C::HALO, &M.fh, bar, z0 - C::RZ, y0 - R, x, hf[k]);
        float* own = base + C::NHU * C::HALO;
        tma_load_4d(own, &M.fo, bar, z0, y0, x + R, 0);            // F0
        tma_load_4d(own + C::OWN, &M.fo, bar, z0, y0, x + R, 3);  // G0
        tma_load_3d(own + 2 * C::OWN, &M.bo[it.ia], bar, z0, y0, x);
        tma_load_3d(own + 3 * C::OWN, &M.bo[it.ib], bar, z0, y0, x);
        tma_load_3d(own + 4 * C::OWN, &M.bo[it.ic], bar, z0, y0, x);
        tma_load_3d(own + 5 * C::OWN, &M.bo[it.id], bar, z0, y0, x);
        tma_load_3d(own + 6 * C::OWN, &M.co, bar, z0, y0, x);
        tma_load_4d(own + 7 * C::OWN, &M.ko, bar, z0, y0, x, 0);
        tma_load_4d(own + 8 * C::OWN, &M.ko, bar, z0, y0, x, 1);
      }
      issued = i + 1;
    }
    for (int i = (issued > C::NST ? issued - C::NST : 0); i < issued; ++i)
      mbar_wait(&full[i % C::NST], (i / C::NST) & 1, tmo);
    return;
  }
  // ============================= compute warps =============================
  const int ey = warp, ez = lane;
  const int y = y0 + ey, z = z0 + ez;
  const bool in = y < g.n1 && z < g.n2;
  const size_t Np = (size_t)g.n0 * g.n1 * g.n2p;
  const size_t col = (size_t)(in ? y : 0) * g.n2p + (in ? z : 0);
  const int yc = in ? y : 0, zc = in ? z : 0;
  const int ch = (ey + R) * C::HW + ez + C::RZ, co = ey * kEZ + ez;
  const float* q0 = kind == 0 ? it.a : flux;           // p^n or F0
  const float* q1 = kind == 0 ? it.c : flux + 3 * Np;  // r^n or G0
  float qa[2 * R + 1], qb[2 * R + 1];
  qa[0] = qb[0] = 0.f;  // shifted out before its first use
#pragma unroll
  for (int s = 1; s < 2 * R + 1; ++s) {
    qa[s] = in ? ld0(g, q0, x0 - 1 - R + s, yc, zc) : 0.f;
    qb[s] = in ? ld0(g, q1, x0 - 1 - R + s, yc, zc) : 0.f;
  }
  const float byz = in ? __fadd_rn(__ldg(damp_b + g.n0 + y), __ldg(damp_b + g.n0 + g.n1 + z)) : 0.f;
  float bx_next = nsteps > 0 ? __ldg(damp_b + x0) : 0.f;  // the plane's damping, loaded a step ahead
  for (int i = 0; i < nsteps; ++i) {
    const int st = i % C::NST, x = x0 + i;
    const float bx_x = bx_next;
    if (i + 1 < nsteps) bx_next = __ldg(damp_b + x + 1);
    const bool ok = mbar_wait(&full[st], (i / C::NST) & 1, tmo);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) atomicExch(err, 1);
      break;
    }
    const float* base = ring + (size_t)st * C::STAGE;
#pragma unroll
    for (int s = 0; s < 2 * R; ++s) {
      qa[s] = qa[s + 1];
      qb[s] = qb[s + 1];
    }
    const size_t i0 = (size_t)x * g.n1 * g.n2p + col;
    if (kind == 0) {
      const float* own = base + C::NHF * C::HALO;
      qa[2 * R] = own[co];
      qb[2 * R] = own[C::OWN + co];
      const float* hp = base;
      const float* hr = base + C::HALO;
      const float gp0 = dc_q<R>(qa, w.a[0]), gp1 = dcs<R>(hp, ch, C::HW, w.a[1]), gp2 = dcs<R>(hp, ch, 1, w.a[2]);
      const float gr0 = dc_q<R>(qb, w.a[0]), gr1 = dcs<R>(hr, ch, C::HW, w.a[1]), gr2 = dcs<R>(hr, ch, 1, w.a[2]);
      const float n0 = own[2 * C::OWN + co], n1 = own[3 * C::OWN + co], n2 = own[4 * C::OWN + co];
      const float sp = __fmaf_rn(n2, gp2, __fmaf_rn(n1, gp1, __fmul_rn(n0, gp0)));
      const float sr = __fmaf_rn(n2, gr2, __fmaf_rn(n1, gr1, __fmul_rn(n0, gr0)));
      if (in) {
        flux[i0] = __fmaf_rn(-n0, sp, gp0);
        flux[Np + i0] = __fmaf_rn(-n1, sp, gp1);
        flux[2 * Np + i0] = __fmaf_rn(-n2, sp, gp2);
        flux[3 * Np + i0] = __fmul_rn(n0, sr);
        flux[4 * Np + i0] = __fmul_rn(n1, sr);
        flux[5 * Np + i0] = __fmul_rn(n2, sr);
      }
    } else {
      const float* own = base + C::NHU * C::HALO;
      qa[2 * R] = own[co];
      qb[2 * R] = own[C::OWN + co];
      const float *hF1 = base, *hG1 = base + C::HALO, *hF2 = base + 2 * C::HALO, *hG2 = base + 3 * C::HALO;
      const float hh = __fadd_rn(__fadd_rn(dc_q<R>(qa, w.a[0]), dcs<R>(hF1, ch, C::HW, w.a[1])),
                                 dcs<R>(hF2, ch, 1, w.a[2]));
      const float hz = __fadd_rn(__fadd_rn(dc_q<R>(qb, w.a[0]), dcs<R>(hG1, ch, C::HW, w.a[1])),
                                 dcs<R>(hG2, ch, 1, w.a[2]));
      const float up = own[2 * C::OWN + co], upp = own[3 * C::OWN + co];
      const float ur = own[4 * C::OWN + co], urp = own[5 * C::OWN + co];
      const float c2v = own[6 * C::OWN + co], cpp = own[7 * C::OWN + co], cpr = own[8 * C::OWN + co];
      const float rhs_p = __fmaf_rn(cpp, hh, __fmul_rn(cpr, hz));
      const float rhs_r = __fmaf_rn(cpr, hh, hz);
      const float gdamp = __fmul_rn(__fadd_rn(bx_x, byz), c2v);
      const float opg = __fadd_rn(1.f, gdamp), omg = __fsub_rn(1.f, gdamp);
      if (in) {
        it.b[i0] = __fadd_rn(up, div_sponge(__fmaf_rn(c2v, rhs_p, __fmul_rn(omg, __fsub_rn(up, upp))), opg));
        it.d[i0] = __fadd_rn(ur, div_sponge(__fmaf_rn(c2v, rhs_r, __fmul_rn(omg, __fsub_rn(ur, urp))), opg));
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
  }
}

template <int R>
__global__ void __launch_bounds__(TtiCfg<R>::NT, TtiCfg<R>::MINB)
    k_tti_tma(PhysGrid g, DerivW w, const __grid_constant__ TtiMaps M, int nchunks, const WaveItem one,
              const WaveItems L, float* flux, const float* __restrict__ damp_b, long long tmo, int* err) {
  using C = TtiCfg<R>;
  extern __shared__ float4 tti_tma_smem4[];
  float* ring = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(tti_tma_smem4) + 127) & ~uintptr_t(127));
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)C::NST * C::STAGE);
  uint64_t* empty = full + C::NST;
  if (threadIdx.x == 0) {
    for (int i = 0; i < C::NST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kEY);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int x0, x1;
  WaveItem it;
  if (L.n == 0) {
    it = one;
    chunk_planes(g, nchunks, x0, x1);
  } else {
    it = L.it[blockIdx.z];
    x0 = it.x0;
    x1 = it.x1;
  }
  tti_tma_tile<R>(g, w, M, it, blockIdx.y * kEY, blockIdx.x * kEZ, x0, x1, flux, damp_b, ring, full, empty, tmo,
                  err);
}

// material at the staggered positions from vp, vs, rho (dense [N]):
// b = 1/rho at half-nodes (mean of two nodes), lam, mu at nodes, mu at edge
// centres (harmonic mean of four nodes, 0 if one is 0); a neighbour past
// the last node takes the last node's value
__global__ void k_ela_material(PhysGrid g, const float* __restrict__ vp, const float* __restrict__ vs,
                               const float* __restrict__ rho, float* __restrict__ mat, int* bad) {
  const Col c = thread_col(g);
  if (!c.ok) return;
  const int x = blockIdx.z;
  const size_t Np = (size_t)g.n0 * g.n1 * g.n2p;
  auto di = [&](int xx, int yy, int zz) { return ((size_t)xx * g.n1 + yy) * g.n2 + zz; };
  const int x1 = min(x + 1, g.n0 - 1), y1 = min(c.y + 1, g.n1 - 1), z1 = min(c.z + 1, g.n2 - 1);
  auto mu_at = [&](int xx, int yy, int zz) {
    const double r = rho[di(xx, yy, zz)], s = vs[di(xx, yy, zz)];
    return r * s * s;
  };
  auto harm4 = [](double a, double b, double cc, double d) {
    if (a <= 0 || b <= 0 || cc <= 0 || d <= 0) return 0.0;
    return 4.0 / (1.0 / a + 1.0 / b + 1.0 / cc + 1.0 / d);
  };
  const size_t q = di(x, c.y, c.z);
  const double r0 = rho[q], p0 = vp[q], s0 = vs[q];
  if (!(r0 > 0) || !(p0 > 0) || !(s0 >= 0) || !(2.0 * s0 * s0 <= p0 * p0) || !isfinite(r0 + p0 + s0)) atomicExch(bad, 1);
  const size_t i0 = pidx(g, x, c.y, c.z);
  mat[i0] = (float)(0.5 * (1.0 / r0 + 1.0 / (double)rho[di(x1, c.y, c.z)]));
  mat[Np + i0] = (float)(0.5 * (1.0 / r0 + 1.0 / (double)rho[di(x, y1, c.z)]));
  mat[2 * Np + i0] = (float)(0.5 * (1.0 / r0 + 1.0 / (double)rho[di(x, c.y, z1)]));
  mat[3 * Np + i0] = (float)(r0 * (p0 * p0 - 2.0 * s0 * s0));
  const double m00 = mu_at(x, c.y, c.z);
  mat[4 * Np + i0] = (float)m00;
  mat[5 * Np + i0] = (float)harm4(m00, mu_at(x1, c.y, c.z), mu_at(x, y1, c.z), mu_at(x1, y1, c.z));
  mat[6 * Np + i0] = (float)harm4(m00, mu_at(x1, c.y, c.z), mu_at(x, c.y, z1), mu_at(x1, c.y, z1));
  mat[7 * Np + i0] = (float)harm4(m00, mu_at(x, y1, c.z), mu_at(x, c.y, z1), mu_at(x, y1, z1));
}

// TTI coefficients from eps, delta, theta, phi (dense [N]): 1 + 2 eps,
// sqrt(1 + 2 delta) and zbar; eps < delta (or delta <= -1/2) flags bad
__global__ void k_tti_coef(PhysGrid g, const float* __restrict__ aux, float* __restrict__ coef,
                           float* __restrict__ nz, unsigned* emax_bits, int* bad) {
  const Col c = thread_col(g);
  if (!c.ok) return;
  const int x = blockIdx.z;
  const size_t N = (size_t)g.n0 * g.n1 * g.n2, Np = (size_t)g.n0 * g.n1 * g.n2p;
  const size_t q = ((size_t)x * g.n1 + c.y) * g.n2 + c.z;
  const double e = aux[q], d = aux[N + q], th = aux[2 * N + q], ph = aux[3 * N + q];
  if (!(e >= d) || !(d > -0.5) || !isfinite(e + d + th + ph)) atomicExch(bad, 1);
  const size_t i0 = pidx(g, x, c.y, c.z);
  coef[i0] = (float)(1.0 + 2.0 * e);
  coef[Np + i0] = (float)sqrt(1.0 + 2.0 * d);
  nz[i0] = (float)(sin(th) * cos(ph));
  nz[Np + i0] = (float)(sin(th) * sin(ph));
  nz[2 * Np + i0] = (float)cos(th);
  if (e > 0) atomicMax(emax_bits, __float_as_uint((float)e));  // non-negative floats order as their bits
}

// ------------------------------------------------- sparse operators --
// grid-aligned injection: f_k[lin(id)] += dcmp[id] for the fields f_k
__global__ void k_inject(PhysGrid g, int64_t npts, const int64_t* __restrict__ lin,
                         const float* __restrict__ dcmp, float* f0, float* f1, float* f2) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= npts) return;
  const int64_t l = lin[id];
  const int z = (int)(l % g.n2), y = (int)((l / g.n2) % g.n1), x = (int)(l / ((int64_t)g.n1 * g.n2));
  const size_t i0 = pidx(g, x, y, z);
  const float a = dcmp[id];
  if (f0) f0[i0] = __fadd_rn(f0[i0], a);
  if (f1) f1[i0] = __fadd_rn(f1[i0], a);
  if (f2) f2[i0] = __fadd_rn(f2[i0], a);
}

// receiver sampling: row[e] = value at the point of entry e (entries in
// column order, as the trace finalisation expects); mean of up to three
// fields (the normal stresses) or one field
__global__ void k_sample(PhysGrid g, int64_t npts, const int2* __restrict__ ent, const int64_t* __restrict__ lin,
                         const float* f0, const float* f1, const float* f2, float* __restrict__ row) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npts) return;
  const int64_t l = lin[ent[e].y];
  const int z = (int)(l % g.n2), y = (int)((l / g.n2) % g.n1), x = (int)(l / ((int64_t)g.n1 * g.n2));
  const size_t i0 = pidx(g, x, y, z);
  float v = f0[i0];
  if (f1) v = __fdiv_rn(__fadd_rn(__fadd_rn(v, f1[i0]), f2[i0]), 3.f);
  row[e] = v;
}

// ------------------------------------------------- wavefront sweeps --
// Temporal blocking of the two-pass steps (Sec. II-B, Fig. 7b): T steps are
// 2T sub-updates (TTI: flux, update; elastic: velocity, stress), each
// reading the previous one's output within r planes along axis 0.  Axis 0
// is cut into slabs of at least r planes and sub-update u of slab s runs in
// launch s + 2u: every value a sub-update reads was written in an earlier
// launch, and no value is overwritten before the launch after its last
// reader, so the fields stay in place and every point sees the operands of
// the one-step order.  One launch runs all of its (sub-update, slab) items,
// blockIdx.z selecting the item; the per-point code is the one-step code.
template <int R>
__global__ void __launch_bounds__(256) k_tti_wave(PhysGrid g, DerivW w, WaveItems L, const float* __restrict__ c2,
                                                  const float* __restrict__ coef, const float* __restrict__ nz,
                                                  const float* __restrict__ damp_b, float* flux) {
  const Col c = thread_col(g);
  if (!c.ok) return;
  const WaveItem it = L.it[blockIdx.z];
  if (it.kind == 0) tti_flux_cols<R>(g, w, c, it.x0, it.x1, it.a, it.c, nz, flux);
  else tti_update_cols<R>(g, w, c, it.x0, it.x1, flux, it.a, it.b, it.c, it.d, c2, coef, damp_b);
}

template <int R>
__global__ void __launch_bounds__(256, 4) k_ela_wave(PhysGrid g, DerivW w, float dt, WaveItems L, float* f,
                                                  const float* __restrict__ mat, const float* __restrict__ eta_dt) {
  const Col c = thread_col(g);
  if (!c.ok) return;
  const WaveItem it = L.it[blockIdx.z];
  if (it.kind == 0) ela_velocity_cols<R>(g, w, c, dt, it.x0, it.x1, f, mat, eta_dt);
  else ela_stress_cols<R>(g, w, c, dt, it.x0, it.x1, f, mat, eta_dt);
}

__device__ __forceinline__ int point_plane(const PhysGrid& g, int64_t l) { return (int)(l / ((int64_t)g.n1 * g.n2)); }

// grid-aligned injection of the steps whose last sub-update finished slabs
// in this launch: item blockIdx.y adds its step's table row to the points on
// its planes (the one-step injection, restricted to a slab)
__global__ void k_wave_inject(PhysGrid g, int64_t npts, const int64_t* __restrict__ lin, WavePosts P) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= npts) return;
  const WavePost q = P.it[blockIdx.y];
  const int64_t l = lin[id];
  const int x = point_plane(g, l);
  if (x < q.x0 || x >= q.x1) return;
  const int z = (int)(l % g.n2), y = (int)((l / g.n2) % g.n1);
  const size_t i0 = pidx(g, x, y, z);
  const float a = q.dcmp[id];
  if (q.f0) q.f0[i0] = __fadd_rn(q.f0[i0], a);
  if (q.f1) q.f1[i0] = __fadd_rn(q.f1[i0], a);
  if (q.f2) q.f2[i0] = __fadd_rn(q.f2[i0], a);
}

// receiver sampling of the same steps on the same slabs (after injection)
__global__ void k_wave_sample(PhysGrid g, int64_t npts, const int2* __restrict__ ent, const int64_t* __restrict__ lin,
                              WavePosts P) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npts) return;
  const WavePost q = P.it[blockIdx.y];
  const int64_t l = lin[ent[e].y];
  const int x = point_plane(g, l);
  if (x < q.x0 || x >= q.x1) return;
  const int z = (int)(l % g.n2), y = (int)((l / g.n2) % g.n1);
  const size_t i0 = pidx(g, x, y, z);
  float v = q.s0[i0];
  if (q.s1) v = __fdiv_rn(__fadd_rn(__fadd_rn(v, q.s1[i0]), q.s2[i0]), 3.f);
  q.row[e] = v;
}

// ------------------------------------------------------------- launch --
static dim3 col_grid(const PhysGrid& g, int nz_planes) {
  return dim3((unsigned)((g.n2 + 31) / 32), (unsigned)((g.n1 + 7) / 8), (unsigned)nz_planes);
}

template <int R>
static cudaError_t tti_step_r(const PhysGrid& g, const DerivW& w, int nchunks, const float* pc, float* pp,
                              const float* rc, float* rp, const float* c2, const float* coef, const float* nz,
                              const float* damp_b, float* flux, cudaStream_t st) {
  // chunks of planes, all in one launch: each column streams its chunk (the
  // queue warms up on R planes before the chunk)
  const dim3 blk(32, 8);
  count_launch(2);
  k_tti_flux<R><<<col_grid(g, nchunks), blk, 0, st>>>(g, w, nchunks, pc, rc, nz, flux);
  k_tti_update<R><<<col_grid(g, nchunks), blk, 0, st>>>(g, w, nchunks, flux, pc, pp, rc, rp, c2, coef, damp_b);
  return cudaGetLastError();
}

template <int R>
static cudaError_t tti_fused_r(const PhysGrid& g, const DerivW& w, int nchunks, const WaveItems* L, const float* pc,
                               float* pp, const float* rc, float* rp, const float* c2, const float* coef,
                               const float* nz, const float* damp_b, cudaStream_t st) {
  using C = TtiFusedCfg<R>;
  // shared memory above 48 KB (r = 6) needs the opt-in; once per process (a
  // function-local static is initialised once even with concurrent callers)
  static const cudaError_t attr = [] {
    const cudaError_t e = cudaFuncSetAttribute(k_tti_fused<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    return e != cudaSuccess
               ? e
               : cudaFuncSetAttribute(k_tti_fused_wave<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  }();
  if (attr != cudaSuccess) return attr;
  const unsigned gz = (unsigned)((g.n2 + C::TZ - 1) / C::TZ), gy = (unsigned)((g.n1 + kFY - 1) / kFY);
  count_launch();
  if (L)
    k_tti_fused_wave<R><<<dim3(gz, gy, L->n), C::NT, C::SMEM, st>>>(g, w, *L, c2, coef, nz, damp_b);
  else
    k_tti_fused<R><<<dim3(gz, gy, nchunks), C::NT, C::SMEM, st>>>(g, w, nchunks, pc, pp, rc, rp, c2, coef, nz,
                                                                    damp_b);
  return cudaGetLastError();
}

cudaError_t tti_fused(int R, const PhysGrid& g, const DerivW& w, int nchunks, const WaveItems* L, const float* pc,
                      float* pp, const float* rc, float* rp, const float* c2, const float* coef, const float* nz,
                      const float* damp_b, cudaStream_t st) {
  if (L && (L->n < 1 || L->n > kWaveItemsMax)) return cudaErrorInvalidValue;
  switch (R) {
    case 2: return tti_fused_r<2>(g, w, nchunks, L, pc, pp, rc, rp, c2, coef, nz, damp_b, st);
    case 4: return tti_fused_r<4>(g, w, nchunks, L, pc, pp, rc, rp, c2, coef, nz, damp_b, st);
    case 6: return tti_fused_r<6>(g, w, nchunks, L, pc, pp, rc, rp, c2, coef, nz, damp_b, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t tti_step(int R, const PhysGrid& g, const DerivW& w, int nchunks, const float* pc, float* pp,
                     const float* rc, float* rp, const float* c2, const float* coef, const float* nz,
                     const float* damp_b, float* flux, cudaStream_t st) {
  switch (R) {
    case 2: return tti_step_r<2>(g, w, nchunks, pc, pp, rc, rp, c2, coef, nz, damp_b, flux, st);
    case 4: return tti_step_r<4>(g, w, nchunks, pc, pp, rc, rp, c2, coef, nz, damp_b, flux, st);
    case 6: return tti_step_r<6>(g, w, nchunks, pc, pp, rc, rp, c2, coef, nz, damp_b, flux, st);
  }
  return cudaErrorInvalidValue;
}

template <int R>
static cudaError_t ela_step_r(const PhysGrid& g, const DerivW& w, float dt, int nchunks, float* f, const float* mat,
                              const float* eta_dt, cudaStream_t st) {
  const dim3 blk(32, 8);
  count_launch(2);
  k_ela_velocity<R><<<col_grid(g, nchunks), blk, 0, st>>>(g, w, dt, nchunks, f, mat, eta_dt);
  k_ela_stress<R><<<col_grid(g, nchunks), blk, 0, st>>>(g, w, dt, nchunks, f, mat, eta_dt);
  return cudaGetLastError();
}

cudaError_t elastic_step(int R, const PhysGrid& g, const DerivW& w, float dt, int nchunks, float* f, const float* mat,
                         const float* eta_dt, cudaStream_t st) {
  switch (R) {
    case 2: return ela_step_r<2>(g, w, dt, nchunks, f, mat, eta_dt, st);
    case 4: return ela_step_r<4>(g, w, dt, nchunks, f, mat, eta_dt, st);
    case 6: return ela_step_r<6>(g, w, dt, nchunks, f, mat, eta_dt, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t wave_launch(int physics, int R, const PhysGrid& g, const DerivW& w, float dt, const WaveItems& L,
                        const float* c2, const float* coef, const float* nz, const float* damp_b, float* flux,
                        float* ef, const float* mat, const float* eta_dt, cudaStream_t st) {
  if (L.n < 1 || L.n > kWaveItemsMax) return cudaErrorInvalidValue;
  const dim3 grid = col_grid(g, L.n), blk(32, 8);
  count_launch();
  if (physics == TB_TTI) {
    switch (R) {
      case 2: k_tti_wave<2><<<grid, blk, 0, st>>>(g, w, L, c2, coef, nz, damp_b, flux); break;
      case 4: k_tti_wave<4><<<grid, blk, 0, st>>>(g, w, L, c2, coef, nz, damp_b, flux); break;
      case 6: k_tti_wave<6><<<grid, blk, 0, st>>>(g, w, L, c2, coef, nz, damp_b, flux); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (R) {
      case 2: k_ela_wave<2><<<grid, blk, 0, st>>>(g, w, dt, L, ef, mat, eta_dt); break;
      case 4: k_ela_wave<4><<<grid, blk, 0, st>>>(g, w, dt, L, ef, mat, eta_dt); break;
      case 6: k_ela_wave<6><<<grid, blk, 0, st>>>(g, w, dt, L, ef, mat, eta_dt); break;
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

int wave_plan(int n0, int slab, int U, std::vector<int>* items) {
  if (n0 < 1 || slab < 1 || U < 1) return -1;
  const int ns = (n0 + slab - 1) / slab;
  items->clear();
  for (int L = 0; L < ns + 2 * (U - 1); ++L)
    for (int u = 0; u < U; ++u) {
      const int sl = L - 2 * u;
      if (sl < 0 || sl >= ns) continue;
      items->insert(items->end(), {L, u, sl * slab, std::min(n0, (sl + 1) * slab)});
    }
  return 0;
}

cudaError_t wave_post(const PhysGrid& g, const WavePosts& P, int64_t nsrc_pts, const int64_t* src_lin,
                      int64_t nrec_pts, const int2* rec_ent, const int64_t* rec_lin, cudaStream_t st) {
  if (P.n < 1 || P.n > kWavePostsMax) return cudaErrorInvalidValue;
  if (nsrc_pts > 0) {
    count_launch();
    k_wave_inject<<<dim3(grid_for(nsrc_pts, 128), P.n), 128, 0, st>>>(g, nsrc_pts, src_lin, P);
  }
  if (nrec_pts > 0) {
    count_launch();
    k_wave_sample<<<dim3(grid_for(nrec_pts, 128), P.n), 128, 0, st>>>(g, nrec_pts, rec_ent, rec_lin, P);
  }
  return cudaGetLastError();
}

template <int R>
static cudaError_t ela_tma_r(const PhysGrid& g, const DerivW& w, float dt, const ElaMaps& M, int kind, int nchunks,
                             const WaveItems* L, float* f, const float* eta_dt, long long tmo, int* err,
                             cudaStream_t st) {
  using C = ElaCfg<R>;
  // more than 48 KB of shared memory needs the opt-in; once per process
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_ela_tma<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  if (attr != cudaSuccess) return attr;
  WaveItems none{};
  const dim3 grid((unsigned)((g.n2 + kEZ - 1) / kEZ), (unsigned)((g.n1 + kEY - 1) / kEY),
                  (unsigned)(L ? L->n : nchunks));
  count_launch();
  k_ela_tma<R><<<grid, C::NT, C::SMEM, st>>>(g, w, dt, M, kind, nchunks, L ? *L : none, f, eta_dt, tmo, err);
  return cudaGetLastError();
}

cudaError_t elastic_tma(int R, const PhysGrid& g, const DerivW& w, float dt, const ElaMaps& M, int kind,
                        int nchunks, const WaveItems* L, float* f, const float* eta_dt, long long tmo, int* err,
                        cudaStream_t st) {
  if (L && (L->n < 1 || L->n > kWaveItemsMax)) return cudaErrorInvalidValue;
  switch (R) {
    case 2: return ela_tma_r<2>(g, w, dt, M, kind, nchunks, L, f, eta_dt, tmo, err, st);
    case 4: return ela_tma_r<4>(g, w, dt, M, kind, nchunks, L, f, eta_dt, tmo, err, st);
    case 6: return ela_tma_r<6>(g, w, dt, M, kind, nchunks, L, f, eta_dt, tmo, err, st);
  }
  return cudaErrorInvalidValue;
}

template <int R>
static cudaError_t tti_tma_r(const PhysGrid& g, const DerivW& w, const TtiMaps& M, int nchunks, const WaveItem* one,
                             const WaveItems* L, float* flux, const float* damp_b, long long tmo, int* err,
                             cudaStream_t st) {
  using C = TtiCfg<R>;
  // more than 48 KB of shared memory needs the opt-in; once per process
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_tti_tma<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  if (attr != cudaSuccess) return attr;
  WaveItems none{};
  WaveItem nil{};
  const dim3 grid((unsigned)((g.n2 + kEZ - 1) / kEZ), (unsigned)((g.n1 + kEY - 1) / kEY),
                  (unsigned)(L ? L->n : nchunks));
  count_launch();
  k_tti_tma<R><<<grid, C::NT, C::SMEM, st>>>(g, w, M, nchunks, one ? *one : nil, L ? *L : none, flux, damp_b, tmo,
                                             err);
  return cudaGetLastError();
}

cudaError_t tti_tma(int R, const PhysGrid& g, const DerivW& w, const TtiMaps& M, int nchunks, const WaveItem* one,
                    const WaveItems* L, float* flux, const float* damp_b, long long tmo, int* err, cudaStream_t st) {
  if (L ? (L->n < 1 || L->n > kWaveItemsMax) : !one) return cudaErrorInvalidValue;
  switch (R) {
    case 2: return tti_tma_r<2>(g, w, M, nchunks, one, L, flux, damp_b, tmo, err, st);
    case 4: return tti_tma_r<4>(g, w, M, nchunks, one, L, flux, damp_b, tmo, err, st);
    case 6: return tti_tma_r<6>(g, w, M, nchunks, one, L, flux, damp_b, tmo, err, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t elastic_material(const PhysGrid& g, const float* vp, const float* vs, const float* rho, float* mat,
                             int* d_bad, cudaStream_t st) {
  count_launch();
  k_ela_material<<<col_grid(g, g.n0), dim3(32, 8), 0, st>>>(g, vp, vs, rho, mat, d_bad);
  return cudaGetLastError();
}

cudaError_t tti_coefficients(const PhysGrid& g, const float* aux, float* coef, float* nz, unsigned* d_emax,
                             int* d_bad, cudaStream_t st) {
  count_launch();
  k_tti_coef<<<col_grid(g, g.n0), dim3(32, 8), 0, st>>>(g, aux, coef, nz, d_emax, d_bad);
  return cudaGetLastError();
}

cudaError_t inject_points(const PhysGrid& g, int64_t npts, const int64_t* lin, const float* dcmp_row, float* f0,
                          float* f1, float* f2, cudaStream_t st) {
  if (npts <= 0) return cudaSuccess;
  count_launch();
  k_inject<<<grid_for(npts, 128), 128, 0, st>>>(g, npts, lin, dcmp_row, f0, f1, f2);
  return cudaGetLastError();
}

cudaError_t sample_points(const PhysGrid& g, int64_t npts, const int2* ent, const int64_t* lin, const float* f0,
                          const float* f1, const float* f2, float* row, cudaStream_t st) {
  if (npts <= 0) return cudaSuccess;
  count_launch();
  k_sample<<<grid_for(npts, 128), 128, 0, st>>>(g, npts, ent, lin, f0, f1, f2, row);
  return cudaGetLastError();
}

}  // namespace tbi
