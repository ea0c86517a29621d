// Acoustic propagator sweep: T time steps of Eq. 1 fused in one pass
// (T = 1 is the spatially blocked one-step kernel).
//
// Layout.  Fields are [n0][n1][n2p] floats, axis 2 contiguous (row pitch
// n2p = n2 rounded up to 4).  A CTA owns a tile of TY rows (axis 1) by 64
// columns (axis 2) and streams it along axis 0: one warp per row, each lane
// owns two adjacent columns (float2 access, fully coalesced rows).
//
// Temporal blocking (Sec. II-B, re-designed for the GPU).  Fused step k
// (k = 0..T-1) computes level n+k+1 at plane q_k = j - k r while step j of
// the stream loads level n at plane j + r.  Each fused step keeps, per owned
// column, a register queue of the 2r+1 planes of its input level around
// q_k; the axis-0 neighbours of the stencil come from that queue, the axis-1
// and axis-2 neighbours from a shared-memory plane filled once per stream
// step.  A step's output goes straight into the next step's queue, so the
// intermediate levels never reach HBM: per T steps a point costs one read of
// u^n, u^{n-1}, c2 and one write of u^{n+T}, u^{n+T-1}.
//
// Halo exchange.  All CTAs of a pass stream in lockstep (cooperative launch,
// co-resident).  The r-wide boundary strips of every intermediate level are
// published to a small ring in global memory (L2-resident), and a CTA reads
// its neighbours' strips r stream steps after they were produced, after an
// acquire on the neighbour's progress counter.  Waits are bounded by a
// timeout; on expiry the CTA sets the error flag and returns.  Within a
// pass there is no redundant computation; passes (bands along axis 1,
// chunks along axis 0) overlap by (T-1) r rows or planes.
//
// Grid-aligned sparse operators (Sec. II-A).  Per column, the inspector's
// entries (x, id) are sorted by x; each fused step walks them with its own
// cursor, adds src_dcmp[step][id] right after the stencil update of that
// point (Listing 5's fused z2 loop, here along the streamed axis), and
// records u at receiver points into rec_dcmp[step][rid].
//
// Rounding.  Every floating-point operation of the point update is an
// explicit round-to-nearest intrinsic, so that each fused step and the
// one-step kernel produce bitwise-identical values.
#pragma once

#include "tb_internal.cuh"

namespace tbi {

template <int R, int T, int TY>
struct SweepCfg {
  static constexpr int TZ = 64;
  static constexpr int NT = 32 * TY;
  static constexpr int SW = TZ + 2 * R;  // shared plane row stride (floats)
  static constexpr int SH = TY + 2 * R;
  static constexpr int PLANE = SW * SH;
  static constexpr int Q = 2 * R + 1;    // queue length
  static constexpr int D = 2 * R + 2;    // ring slots per fused step
  static constexpr int STRIP = 2 * R * TZ + 2 * R * TY;
  static constexpr int RING_PER_CTA = (T > 1 ? (T - 1) * D * STRIP : 0);
  static constexpr size_t SMEM =
      sizeof(float) * T * PLANE + sizeof(int) * (2 * T * 2 * NT + 2 * 2 * NT);
  static_assert(R % 2 == 0, "radius must be even for aligned float2 access");
  static_assert(TY >= R && TZ >= R, "halo must come from one neighbour tile");
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Spin (one thread) until *flag >= target, at most timeout_ns after t0 and
// at most 2^26 polls.  Returns false when the limit ran out.
__device__ __forceinline__ bool bounded_wait_ge(const unsigned long long* flag,
                                                unsigned long long target, unsigned long long t0,
                                                long long timeout_ns) {
  long long spins = 0;
  while (ld_acquire_u64(flag) < target) {
    if (++spins > (1ll << 26) || (long long)(global_ns() - t0) > timeout_ns) return false;
    __nanosleep(32);
  }
  return true;
}

// Eq. 1 at one point: u^{n+1} = [dt^2 L u + m(2u - u_prev) + a u_prev]/(m + a)
// rewritten with c2 = dt^2/m and g = a/m = (eta/(2 dt)) c2:
//   u^{n+1} = (c2 L u + 2u - (1 - g) u_prev) / (1 + g).
__device__ __forceinline__ float point_update(float uc, float up, float lap, float c2,
                                              float bsum) {
  const float two_u = __fadd_rn(uc, uc);
  if (bsum == 0.f) return __fmaf_rn(c2, lap, __fsub_rn(two_u, up));
  const float g = __fmul_rn(bsum, c2);
  const float num = __fmaf_rn(c2, lap, __fsub_rn(two_u, __fmul_rn(__fsub_rn(1.f, g), up)));
  return __fdiv_rn(num, __fadd_rn(1.f, g));
}

template <int R, int T, int TY>
__global__ void __launch_bounds__(32 * TY, T == 1 ? 2 : 1) sweep_kernel(const SweepParams P) {
  using C = SweepCfg<R, T, TY>;
  constexpr int TZ = C::TZ, NT = C::NT, SW = C::SW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* planes = reinterpret_cast<float*>(smem_raw);
  int* cur = reinterpret_cast<int*>(planes + T * C::PLANE);  // [2 kinds][T][2 cols][NT]
  int* cend = cur + 2 * T * 2 * NT;                           // [2 kinds][2 cols][NT]
  __shared__ int s_abort;

  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int b = blockIdx.x;
  int pi = 0;
  for (int i = 1; i < P.npass; ++i)
    if (P.pass[i].cta0 <= b) pi = i;
  const PassDesc pd = P.pass[pi];

  const int tl = b - pd.cta0, ty = tl / pd.ntz, tz = tl - ty * pd.ntz;
  const int y0 = pd.yb0 + ty * TY, z0 = tz * TZ;
  const int y = y0 + w, z = z0 + 2 * lane;
  const bool vrow = y < P.n1;
  const bool v0 = vrow && z < P.n2, v1 = vrow && z + 1 < P.n2;
  const int nb_up = ty > 0 ? b - pd.ntz : -1;
  const int nb_dn = ty + 1 < pd.nty ? b + pd.ntz : -1;
  const int nb_lf = tz > 0 ? b - 1 : -1;
  const int nb_rt = tz + 1 < pd.ntz ? b + 1 : -1;
  const bool own_row = y >= pd.yo0 && y < pd.yo1;
  const size_t ps = (size_t)P.n1 * P.n2p;       // plane stride
  const size_t coff = (size_t)y * P.n2p + z;    // column offset (valid if v0)

  float byz0 = 0.f, byz1 = 0.f;
  if (v0) byz0 = __fadd_rn(__ldg(&P.damp_b[P.n0 + y]), __ldg(&P.damp_b[P.n0 + P.n1 + z]));
  if (v1) byz1 = __fadd_rn(__ldg(&P.damp_b[P.n0 + y]), __ldg(&P.damp_b[P.n0 + P.n1 + z + 1]));

  // Per-column cursors into the grid-aligned source / receiver entries.
  int flags = 0;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    if (!(i == 0 ? v0 : v1)) continue;
    const int c = y * P.n2 + z + i;
    if (P.s_colptr) {
      const int sb = __ldg(&P.s_colptr[c]), se = __ldg(&P.s_colptr[c + 1]);
      if (se > sb) {
        flags |= 1 << i;
        for (int k = 0; k < T; ++k) cur[((0 * T + k) * 2 + i) * NT + tid] = sb;
        cend[(0 * 2 + i) * NT + tid] = se;
      }
    }
    if (P.r_colptr) {
      const int rb = __ldg(&P.r_colptr[c]), re = __ldg(&P.r_colptr[c + 1]);
      if (re > rb) {
        flags |= 4 << i;
        for (int k = 0; k < T; ++k) cur[((1 * T + k) * 2 + i) * NT + tid] = rb;
        cend[(1 * 2 + i) * NT + tid] = re;
      }
    }
  }

  auto load_u = [&](const float* base, int plane) -> float2 {
    float2 v = make_float2(0.f, 0.f);
    if (v0 && plane >= 0 && plane < P.n0) {
      v = __ldg(reinterpret_cast<const float2*>(base + (size_t)plane * ps + coff));
      if (!v1) v.y = 0.f;
    }
    return v;
  };
  auto ring_strip = [&](int tile, int ridx, int q) -> float* {
    return P.ring + (((size_t)tile * (T - 1) + ridx) * C::D + (q % C::D)) * C::STRIP;
  };

  const int jstart = pd.xc0;
  const int jend = pd.xo1 - 1 + (T - 1) * R;  // inclusive

  float2 Qs[T][C::Q];
#pragma unroll
  for (int k = 0; k < T; ++k)
#pragma unroll
    for (int s = 0; s < C::Q; ++s) Qs[k][s] = make_float2(0.f, 0.f);
  // stage 0 holds planes [jstart-1-R, jstart-1+R] of u^n before the first shift
#pragma unroll
  for (int s = 0; s < C::Q; ++s) Qs[0][s] = load_u(P.u_cur, jstart - 1 - R + s);

  if (tid == 0) s_abort = 0;

#pragma unroll 1
  for (int j = jstart; j <= jend; ++j) {
    const float2 newq = load_u(P.u_cur, j + R);
    const bool act0 = j >= pd.xc0 && j < pd.xc1;
    float2 up0 = make_float2(0.f, 0.f);
    if (act0 && v0) {
      // plain load: in the one-step kernel u_prev aliases out0 (in place)
      up0 = *reinterpret_cast<const float2*>(P.u_prev + (size_t)j * ps + coff);
      if (!v1) up0.y = 0.f;
    }
    __syncthreads();  // previous step finished with planes, ring and cursors

    if constexpr (T > 1) {
      if (tid == 0) {
        if (j > jstart) {
          __threadfence();
          st_release_u64(&P.progress[b], P.prog_base + (unsigned long long)(j - jstart));
        }
        bool need = false;
#pragma unroll
        for (int k = 1; k < T; ++k) {
          const int q = j - k * R;
          need |= (q >= pd.xc0 && q < pd.xc1);
        }
        if (need && j - R >= jstart) {
          const unsigned long long target = P.prog_base + (unsigned long long)(j - R - jstart + 1);
          const int nbs[4] = {nb_up, nb_dn, nb_lf, nb_rt};
          const unsigned long long t0 = global_ns();
          bool ok = true;
          for (int i = 0; i < 4 && ok; ++i)
            if (nbs[i] >= 0) ok = bounded_wait_ge(&P.progress[nbs[i]], target, t0, P.timeout_ns);
          if (!ok) {
            atomicExch(P.err, 1);
            s_abort = 1;
          }
        }
        __threadfence();
      }
      __syncthreads();
      if (s_abort) return;
    }

    // ---- fill the shared planes: centre from the queues, halos from u^n
    //      (fused step 0) or from the neighbours' ring strips
#pragma unroll
    for (int k = 0; k < T; ++k) {
      const int q = j - k * R;
      if (q < pd.xc0 || q >= pd.xc1) continue;
      float* pl = planes + k * C::PLANE;
      *reinterpret_cast<float2*>(&pl[(R + w) * SW + R + 2 * lane]) = Qs[k][R + 1];
      for (int e = tid; e < 2 * R * TZ; e += NT) {
        const int hr = e / TZ, hz = e - hr * TZ;
        const bool top = hr < R;
        const int yy = top ? y0 - R + hr : y0 + TY + (hr - R);
        const int zz = z0 + hz;
        float v = 0.f;
        if (yy >= 0 && yy < P.n1 && zz < P.n2) {
          if (k == 0) {
            v = __ldg(P.u_cur + (size_t)q * ps + (size_t)yy * P.n2p + zz);
          } else {
            const int nb = top ? nb_up : nb_dn;
            if (nb >= 0)
              v = __ldcg(ring_strip(nb, k - 1, q) + (top ? (R + hr) * TZ + hz : (hr - R) * TZ + hz));
          }
        }
        pl[(top ? hr : TY + hr) * SW + R + hz] = v;
      }
      for (int e = tid; e < TY * 2 * R; e += NT) {
        const int row = e / (2 * R), hc = e - row * (2 * R);
        const bool left = hc < R;
        const int zz = left ? z0 - R + hc : z0 + TZ + (hc - R);
        const int yy = y0 + row;
        float v = 0.f;
        if (yy < P.n1 && zz >= 0 && zz < P.n2) {
          if (k == 0) {
            v = __ldg(P.u_cur + (size_t)q * ps + (size_t)yy * P.n2p + zz);
          } else {
            const int nb = left ? nb_lf : nb_rt;
            if (nb >= 0)
              v = __ldcg(ring_strip(nb, k - 1, q) + 2 * R * TZ + (left ? TY * R : 0) + row * R +
                         (left ? hc : hc - R));
          }
        }
        pl[(R + row) * SW + (left ? hc : TZ + hc)] = v;
      }
    }
    __syncthreads();

    // ---- fused steps
#pragma unroll
    for (int s = 0; s < C::Q - 1; ++s) Qs[0][s] = Qs[0][s + 1];
    Qs[0][C::Q - 1] = newq;

#pragma unroll
    for (int k = 0; k < T; ++k) {
      const int q = j - k * R;
      const bool act = q >= pd.xc0 && q < pd.xc1;
      float2 un = make_float2(0.f, 0.f);
      if (act) {
        const float* pl = planes + k * C::PLANE;
        const float2 upv = (k == 0) ? up0 : Qs[k > 0 ? k - 1 : 0][0];
        float2 c2v = make_float2(0.f, 0.f);
        if (v0) c2v = __ldg(reinterpret_cast<const float2*>(P.c2 + (size_t)q * ps + coff));
        const float bx = __ldg(&P.damp_b[q]);
        const float2 uc = Qs[k][R];
        // axis-2 window: zw[m] = value at tile column 2*lane - R + m
        float zw[2 * R + 2];
#pragma unroll
        for (int m = 0; m < R; m += 2) {
          const float2 a = *reinterpret_cast<const float2*>(&pl[(R + w) * SW + 2 * lane + m]);
          const float2 c = *reinterpret_cast<const float2*>(&pl[(R + w) * SW + 2 * lane + R + 2 + m]);
          zw[m] = a.x;
          zw[m + 1] = a.y;
          zw[R + 2 + m] = c.x;
          zw[R + 3 + m] = c.y;
        }
        zw[R] = uc.x;
        zw[R + 1] = uc.y;
        float lap0 = __fmul_rn(P.wc, uc.x);
        float lap1 = __fmul_rn(P.wc, uc.y);
#pragma unroll
        for (int d = 1; d <= R; ++d) {
          const float2 yp = *reinterpret_cast<const float2*>(&pl[(R + w + d) * SW + R + 2 * lane]);
          const float2 ym = *reinterpret_cast<const float2*>(&pl[(R + w - d) * SW + R + 2 * lane]);
          lap0 = __fmaf_rn(P.wx[d - 1], __fadd_rn(Qs[k][R + d].x, Qs[k][R - d].x), lap0);
          lap1 = __fmaf_rn(P.wx[d - 1], __fadd_rn(Qs[k][R + d].y, Qs[k][R - d].y), lap1);
          lap0 = __fmaf_rn(P.wy[d - 1], __fadd_rn(yp.x, ym.x), lap0);
          lap1 = __fmaf_rn(P.wy[d - 1], __fadd_rn(yp.y, ym.y), lap1);
          lap0 = __fmaf_rn(P.wz[d - 1], __fadd_rn(zw[R + d], zw[R - d]), lap0);
          lap1 = __fmaf_rn(P.wz[d - 1], __fadd_rn(zw[R + 1 + d], zw[R + 1 - d]), lap1);
        }
        if (v0) un.x = point_update(uc.x, upv.x, lap0, c2v.x, __fadd_rn(bx, byz0));
        if (v1) un.y = point_update(uc.y, upv.y, lap1, c2v.y, __fadd_rn(bx, byz1));

        const int step = P.step0 + k;
        if (flags & 3) {  // fused grid-aligned injection (Listing 5)
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            if (!((flags >> i) & 1)) continue;
            int* cp = &cur[((0 * T + k) * 2 + i) * NT + tid];
            int cc = *cp;
            const int ce = cend[(0 * 2 + i) * NT + tid];
            while (cc < ce) {
              const int2 e = __ldg(&P.s_ent[cc]);
              if (e.x < q) { ++cc; continue; }
              if (e.x == q) {
                const float add = __ldg(&P.src_dcmp[(size_t)step * P.npts + e.y]);
                if (i == 0) un.x = __fadd_rn(un.x, add);
                else un.y = __fadd_rn(un.y, add);
                ++cc;
              }
              break;
            }
            *cp = cc;
          }
        }
        if ((flags & 12) && own_row && q >= pd.xo0 && q < pd.xo1) {  // receiver points
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            if (!((flags >> (2 + i)) & 1)) continue;
            int* cp = &cur[((1 * T + k) * 2 + i) * NT + tid];
            int cc = *cp;
            const int ce = cend[(1 * 2 + i) * NT + tid];
            while (cc < ce) {
              const int2 e = __ldg(&P.r_ent[cc]);
              if (e.x < q) { ++cc; continue; }
              if (e.x == q) {
                P.rec_dcmp[(size_t)(step - P.rec_base) * P.nrpts + e.y] = (i == 0 ? un.x : un.y);
                ++cc;
              }
              break;
            }
            *cp = cc;
          }
        }
      }
      if (k + 1 < T) {
        // hand the new level to the next fused step, publish its halo strips
#pragma unroll
        for (int s = 0; s < C::Q - 1; ++s) Qs[k + 1 < T ? k + 1 : 0][s] = Qs[k + 1 < T ? k + 1 : 0][s + 1];
        Qs[k + 1 < T ? k + 1 : 0][C::Q - 1] = un;
        if (act) {
          float* rs = ring_strip(b, k, q);
          if (w < R) __stcg(reinterpret_cast<float2*>(rs + w * TZ + 2 * lane), un);
          if (w >= TY - R) __stcg(reinterpret_cast<float2*>(rs + (R + w - (TY - R)) * TZ + 2 * lane), un);
          if (2 * lane < R) __stcg(reinterpret_cast<float2*>(rs + 2 * R * TZ + w * R + 2 * lane), un);
          if (2 * lane >= TZ - R)
            __stcg(reinterpret_cast<float2*>(rs + 2 * R * TZ + TY * R + w * R + 2 * lane - (TZ - R)), un);
        }
      } else if (act && own_row && q >= pd.xo0 && q < pd.xo1 && v0) {
        __stcs(reinterpret_cast<float2*>(P.out0 + (size_t)q * ps + coff), un);
        if constexpr (T > 1) __stcs(reinterpret_cast<float2*>(P.out1 + (size_t)q * ps + coff), Qs[k][R]);
      }
    }
  }
  if constexpr (T > 1) {
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release_u64(&P.progress[b], P.prog_base + (unsigned long long)(jend - jstart + 1));
    }
  }
}

template <int R, int T>
struct SweepTraits {
  static constexpr int TY = 16;
  using Cfg = SweepCfg<R, T, TY>;
};

template <int R, int T>
cudaError_t sweep_launch_t(const SweepParams& p, int nctas, bool cooperative, cudaStream_t st) {
  using Tr = SweepTraits<R, T>;
  using Cf = typename Tr::Cfg;
  auto fn = sweep_kernel<R, T, Tr::TY>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cf::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  count_launch();
  if (cooperative) {
    SweepParams pc = p;
    void* args[] = {&pc};
    return cudaLaunchCooperativeKernel((const void*)fn, dim3(nctas), dim3(Cf::NT), args, Cf::SMEM, st);
  }
  fn<<<nctas, Cf::NT, Cf::SMEM, st>>>(p);
  return cudaGetLastError();
}

template <int R, int T>
cudaError_t sweep_occupancy_t(int* per_sm) {
  using Tr = SweepTraits<R, T>;
  using Cf = typename Tr::Cfg;
  auto fn = sweep_kernel<R, T, Tr::TY>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cf::SMEM);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, Cf::NT, Cf::SMEM);
}

template <int R, int T>
void sweep_shape_t(SweepShape* s) {
  using Tr = SweepTraits<R, T>;
  using Cf = typename Tr::Cfg;
  s->R = R;
  s->T = T;
  s->TY = Tr::TY;
  s->threads = Cf::NT;
  s->smem = Cf::SMEM;
  s->ring_floats_per_cta = Cf::RING_PER_CTA;
}

// Per-radius entry points (one translation unit per radius).
#define TBI_DECLARE_RADIUS(RR)                                                                \
  cudaError_t sweep_launch_r##RR(int T, const SweepParams& p, int nctas, bool coop,           \
                                 cudaStream_t st);                                            \
  cudaError_t sweep_occupancy_r##RR(int T, int* per_sm);                                      \
  bool sweep_shape_r##RR(int T, SweepShape* s);

TBI_DECLARE_RADIUS(2)
TBI_DECLARE_RADIUS(4)
TBI_DECLARE_RADIUS(6)

#define TBI_DEFINE_RADIUS(RR)                                                                 \
  cudaError_t sweep_launch_r##RR(int T, const SweepParams& p, int nctas, bool coop,           \
                                 cudaStream_t st) {                                           \
    switch (T) {                                                                              \
      case 1: return sweep_launch_t<RR, 1>(p, nctas, coop, st);                               \
      case 2: return sweep_launch_t<RR, 2>(p, nctas, coop, st);                               \
      case 3: return sweep_launch_t<RR, 3>(p, nctas, coop, st);                               \
      case 4: return sweep_launch_t<RR, 4>(p, nctas, coop, st);                               \
    }                                                                                         \
    return cudaErrorInvalidValue;                                                             \
  }                                                                                           \
  cudaError_t sweep_occupancy_r##RR(int T, int* per_sm) {                                     \
    switch (T) {                                                                              \
      case 1: return sweep_occupancy_t<RR, 1>(per_sm);                                        \
      case 2: return sweep_occupancy_t<RR, 2>(per_sm);                                        \
      case 3: return sweep_occupancy_t<RR, 3>(per_sm);                                        \
      case 4: return sweep_occupancy_t<RR, 4>(per_sm);                                        \
    }                                                                                         \
    return cudaErrorInvalidValue;                                                             \
  }                                                                                           \
  bool sweep_shape_r##RR(int T, SweepShape* s) {                                              \
    switch (T) {                                                                              \
      case 1: sweep_shape_t<RR, 1>(s); return true;                                           \
      case 2: sweep_shape_t<RR, 2>(s); return true;                                           \
      case 3: sweep_shape_t<RR, 3>(s); return true;                                           \
      case 4: sweep_shape_t<RR, 4>(s); return true;                                           \
    }                                                                                         \
    return false;                                                                             \
  }

}  // namespace tbi
