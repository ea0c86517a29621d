// Acoustic propagator sweep: T time steps of Eq. 1 fused in one pass
// (T = 1 is the spatially blocked one-step kernel).
//
// Layout.  Fields are [n0][n1][n2p] floats, axis 2 contiguous (row pitch
// n2p = n2 rounded up to 4).  A CTA owns a tile of TY rows (axis 1) by 64
// columns (axis 2) and streams it along axis 0: one warp per row, each lane
// owns two adjacent columns (float2 / packed f32x2 arithmetic).
//
// Data movement (per stream step j, asynchronous and prefetched):
//   * u^n plane j+r as a (TY+2r) x (64+2rp) box with its halo, by a 3-D TMA
//     load into a ring of shared-memory planes (out-of-grid cells arrive as
//     zeros, which is the zero boundary of Eq. 1);
//   * the own tiles of u^{n-1} and c2 = dt^2/m by TMA into their rings;
//   * for fused steps k >= 1, the neighbours' halo strips of level n+k by
//     16-byte cp.async from a small L2-resident ring in global memory, one
//     stream step ahead.
// Every ring slot has an mbarrier; one thread refills a slot right after
// the stream step that last reads it.
//
// Temporal blocking (Sec. II-B, re-designed for the GPU).  Fused step k
// (k = 0..T-1) computes level n+k+1 at plane q_k = j - k r.  Each fused step
// keeps, per owned column, a register queue of the 2r+1 planes of its input
// level around q_k (the axis-0 neighbours of the stencil); axis-1 and axis-2
// neighbours come from a shared plane.  A step's output goes straight into
// the next step's queue, so intermediate levels never reach HBM: per T
// steps a point costs one read of u^n, u^{n-1}, c2 and one write of
// u^{n+T}, u^{n+T-1}.
//
// Halo exchange between CTAs.  All CTAs of a pass stream in lockstep
// (cooperative launch, co-resident).  The boundary strips of every
// intermediate level are published to the ring; a CTA prefetches its
// neighbours' strips of stream step j+1 during step j, after an acquire on
// the neighbours' progress counters.  Waits are bounded by a timeout; on
// expiry the CTA sets the error flag, drains its own copies and returns.
// Within a pass there is no redundant computation; passes (bands along axis
// 1, chunks along axis 0) overlap by (T-1) r rows or planes.
//
// Grid-aligned sparse operators (Sec. II-A).  Per column, the inspector's
// entries (x, id) are sorted by x; each fused step walks them with its own
// cursor, adds src_dcmp[step][id] right after the stencil update of that
// point (Listing 5's fused injection loop, here along the streamed axis),
// and records u at receiver points into rec_dcmp[step][rid].
//
// Rounding.  Every floating-point operation of the point update is an
// explicit round-to-nearest operation, so each fused step and the one-step
// kernel produce bitwise-identical values.
#pragma once

#include <cuda.h>

#include "tb_internal.cuh"

namespace tbi {

constexpr size_t align128(size_t b) { return (b + 127) / 128 * 128; }

template <int R, int T, int TY>
struct SweepCfg {
  static constexpr int TZ = 64;
  static constexpr int NT = 32 * TY;
  static constexpr int RP = (R + 3) / 4 * 4;  // axis-2 halo width in shared memory
  static constexpr int SW = TZ + 2 * RP;      // plane row stride (floats)
  static constexpr int SH = TY + 2 * R;
  static constexpr int PLANE = SW * SH;
  static constexpr int PSLOT = (int)(align128(PLANE * 4) / 4);
  static constexpr int TILE = TY * TZ;
  static constexpr int Q = 2 * R + 1;               // queue length
  static constexpr int PF = 2;                      // prefetch distance in planes
  static constexpr int NU = R + 1 + PF;             // u^n box ring
  static constexpr int NP = PF + 1;                 // u^{n-1} tile ring
  static constexpr int NC = (T - 1) * R + 1 + PF;   // c2 tile ring
  static constexpr int D = 2 * R + 2;               // halo ring slots per fused step (global)
  static constexpr int STRIP = 2 * R * TZ + 2 * TY * RP;
  static constexpr int RING_PER_CTA = T > 1 ? (T - 1) * D * STRIP : 0;
  static constexpr size_t OFF_U = 0;
  static constexpr size_t OFF_P = OFF_U + align128((size_t)NU * PSLOT * 4);
  static constexpr size_t OFF_C = OFF_P + align128((size_t)NP * TILE * 4);
  static constexpr size_t OFF_S = OFF_C + align128((size_t)NC * TILE * 4);
  static constexpr size_t OFF_BASE = OFF_S + align128((size_t)(T > 1 ? 2 * (T - 1) : 0) * PSLOT * 4);
  static constexpr size_t OFF_CNT = OFF_BASE + 4 * 2 * 2 * NT;
  static constexpr size_t OFF_CUR = OFF_CNT + 2 * 2 * 2 * NT;
  static constexpr size_t OFF_BAR = align128(OFF_CUR + 2 * 2 * T * 2 * NT);
  static constexpr size_t SMEM = OFF_BAR + 8 * (NU + NP + NC) + 128;  // + base alignment
  static_assert(R % 2 == 0, "radius must be even for aligned float2 access");
  static_assert(TY >= R && TZ >= RP, "a halo must come from one neighbour tile");
  static_assert(SMEM <= 232448, "shared memory budget exceeded");
};

// ---------------------------------------------------------------- PTX ----
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
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
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase; false when the time limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if ((long long)(global_ns() - t0) > timeout_ns) return false;
  return true;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

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

// ------------------------------------------------------------ arithmetic --
// Eq. 1 at one point: u^{n+1} = [dt^2 L u + m(2u - u_prev) + a u_prev]/(m + a)
// rewritten with c2 = dt^2/m and g = a/m = (eta/(2 dt)) c2 as an increment:
//   u^{n+1} = u + (c2 L u + (1 - g)(u - u_prev)) / (1 + g).
__device__ __forceinline__ float point_update(float uc, float up, float lap, float c2,
                                              float bsum) {
  const float d = __fsub_rn(uc, up);
  if (bsum == 0.f) return __fadd_rn(uc, __fmaf_rn(c2, lap, d));
  const float g = __fmul_rn(bsum, c2);
  const float inc = __fmaf_rn(c2, lap, __fmul_rn(__fsub_rn(1.f, g), d));
  return __fadd_rn(uc, __fdiv_rn(inc, __fadd_rn(1.f, g)));
}

// One neighbour pair of the Laplacian in differences form on a column pair,
// acc + w ((a - u) + (b - u)), as packed f32x2 round-to-nearest operations.
// The differences of close values are exact, so the large centre term never
// cancels against the neighbour sum (in FP32 this keeps 1000-step runs ~40x
// closer to the FP64 result than the c0 u + sum c_i (u_+i + u_-i) form).
__device__ __forceinline__ unsigned long long pk2(float2 v) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ float2 pair_term2(float2 acc, unsigned long long w2, float2 a, float2 b,
                                             float2 u) {
  unsigned long long da, db, e, r;
  const unsigned long long uu = pk2(u);
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(da) : "l"(pk2(a)), "l"(uu));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(db) : "l"(pk2(b)), "l"(uu));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(e) : "l"(da), "l"(db));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(w2), "l"(e), "l"(pk2(acc)));
  return upk2(r);
}

// ----------------------------------------------------------------- kernel --
template <int R, int T, int TY>
__global__ void __launch_bounds__(32 * TY, T == 1 ? 2 : 1)
    sweep_kernel(const __grid_constant__ SweepParams P) {
  using C = SweepCfg<R, T, TY>;
  constexpr int TZ = C::TZ, NT = C::NT, SW = C::SW, RP = C::RP;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // TMA destinations need 128-byte alignment: align the base explicitly
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  float* uring = reinterpret_cast<float*>(smem + C::OFF_U);
  float* pring = reinterpret_cast<float*>(smem + C::OFF_P);
  float* cring = reinterpret_cast<float*>(smem + C::OFF_C);
  float* splane = reinterpret_cast<float*>(smem + C::OFF_S);
  int* cbase = reinterpret_cast<int*>(smem + C::OFF_BASE);                      // [kind][col][NT]
  unsigned short* ccnt = reinterpret_cast<unsigned short*>(smem + C::OFF_CNT);  // [kind][col][NT]
  unsigned short* ccur = reinterpret_cast<unsigned short*>(smem + C::OFF_CUR);  // [kind][T][col][NT]
  uint64_t* bar_u = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
  uint64_t* bar_p = bar_u + C::NU;
  uint64_t* bar_c = bar_p + C::NP;
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
  const size_t ps = (size_t)P.n1 * P.n2p;        // plane stride
  const size_t coff = (size_t)y * P.n2p + z;     // column offset (valid if v0)
  const int own = (R + w) * SW + RP + 2 * lane;  // own pair in a plane slot
  const int own_t = w * TZ + 2 * lane;           // own pair in a tile slot
  const int jstart = pd.xc0;
  const int jend = pd.xo1 - 1 + (T - 1) * R;  // inclusive
  const long long tmo = P.timeout_ns;

  float byz0 = 0.f, byz1 = 0.f;
  if (v0) byz0 = __fadd_rn(__ldg(&P.damp_b[P.n0 + y]), __ldg(&P.damp_b[P.n0 + P.n1 + z]));
  if (v1) byz1 = __fadd_rn(__ldg(&P.damp_b[P.n0 + y]), __ldg(&P.damp_b[P.n0 + P.n1 + z + 1]));

  // Per-column cursors into the grid-aligned source / receiver entries.
  int flags = 0;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    if (!(i == 0 ? v0 : v1)) continue;
    const int c = y * P.n2 + z + i;
#pragma unroll
    for (int kind = 0; kind < 2; ++kind) {
      const int* colptr = kind == 0 ? P.s_colptr : P.r_colptr;
      if (!colptr) continue;
      const int cb = __ldg(&colptr[c]), ce = __ldg(&colptr[c + 1]);
      if (ce > cb) {
        flags |= 1 << (2 * kind + i);
        cbase[(kind * 2 + i) * NT + tid] = cb;
        ccnt[(kind * 2 + i) * NT + tid] = (unsigned short)(ce - cb);
        for (int k = 0; k < T; ++k) ccur[((kind * T + k) * 2 + i) * NT + tid] = 0;
      }
    }
  }

  // Missing neighbours leave zero halos in the fused-step planes for good.
  if constexpr (T > 1) {
    for (int e = tid; e < 2 * (T - 1) * C::PSLOT; e += NT) splane[e] = 0.f;
  }
  if (tid == 0) {
    s_abort = 0;
    for (int i = 0; i < C::NU + C::NP + C::NC; ++i) mbar_init(bar_u + i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  auto issue_u = [&](int p) {
    const int s = (p - jstart) % C::NU;
    mbar_expect_tx(bar_u + s, C::PLANE * 4);
    tma_load_3d(uring + s * C::PSLOT, &P.tm_u, bar_u + s, z0 - RP, y0 - R, p);
  };
  auto issue_p = [&](int p) {
    const int s = (p - jstart) % C::NP;
    mbar_expect_tx(bar_p + s, C::TILE * 4);
    tma_load_3d(pring + s * C::TILE, &P.tm_p, bar_p + s, z0, y0, p);
  };
  auto issue_c = [&](int p) {
    const int s = (p - jstart) % C::NC;
    mbar_expect_tx(bar_c + s, C::TILE * 4);
    tma_load_3d(cring + s * C::TILE, &P.tm_c, bar_c + s, z0, y0, p);
  };
  // Wait (bounded) for every prefetch issued for stream steps >= jn.
  auto drain = [&](int jn) {
    for (int p = jn; p < jn + C::NU; ++p)
      mbar_wait(bar_u + (p - jstart) % C::NU, ((p - jstart) / C::NU) & 1, tmo);
    for (int p = jn; p <= jn + C::PF; ++p) {
      mbar_wait(bar_p + (p - jstart) % C::NP, ((p - jstart) / C::NP) & 1, tmo);
      mbar_wait(bar_c + (p - jstart) % C::NC, ((p - jstart) / C::NC) & 1, tmo);
    }
  };
  if (tid == 0) {
    for (int p = jstart; p < jstart + C::NU; ++p) issue_u(p);
    for (int p = jstart; p <= jstart + C::PF; ++p) {
      issue_p(p);
      issue_c(p);
    }
  }

  auto ring_strip = [&](int tile, int ridx, int q) -> float* {
    return P.ring + (((size_t)tile * (T - 1) + ridx) * C::D + (q % C::D)) * C::STRIP;
  };
  // Prefetch of the fused steps' halo strips for stream step jn.
  auto prefetch_halos = [&](int jn) {
    constexpr int CH_ROW = TZ / 4;           // 16-byte chunks per strip row
    constexpr int CH_Y = 2 * R * CH_ROW;     // top + bottom strips
    constexpr int CH_Z = 2 * TY * (RP / 4);  // left + right strips
    constexpr int CH = CH_Y + CH_Z;
    float* buf = splane + (size_t)(jn & 1) * (T - 1) * C::PSLOT;
    for (int e = tid; e < (T - 1) * CH; e += NT) {
      const int k = 1 + e / CH, r = e - (k - 1) * CH;
      const int q = jn - k * R;
      if (q < pd.xc0 || q >= pd.xc1) continue;
      float* pl = buf + (k - 1) * C::PSLOT;
      if (r < CH_Y) {
        const int hr = r / CH_ROW, c4 = 4 * (r - hr * CH_ROW);
        if (hr < R) {
          if (nb_up >= 0)
            cp_async16(pl + hr * SW + RP + c4, ring_strip(nb_up, k - 1, q) + (R + hr) * TZ + c4);
        } else if (nb_dn >= 0) {
          cp_async16(pl + (TY + hr) * SW + RP + c4, ring_strip(nb_dn, k - 1, q) + (hr - R) * TZ + c4);
        }
      } else {
        const int r2 = r - CH_Y, row = r2 / (RP / 2), cc = r2 - row * (RP / 2);
        const bool left = cc < RP / 4;
        const int c4 = 4 * (left ? cc : cc - RP / 4);
        if (left) {
          if (nb_lf >= 0)
            cp_async16(pl + (R + row) * SW + c4,
                       ring_strip(nb_lf, k - 1, q) + 2 * R * TZ + TY * RP + row * RP + c4);
        } else if (nb_rt >= 0) {
          cp_async16(pl + (R + row) * SW + RP + TZ + c4,
                     ring_strip(nb_rt, k - 1, q) + 2 * R * TZ + row * RP + c4);
        }
      }
    }
  };

  // Stage-0 queue before the first shift: planes [jstart-1-R, jstart-1+R] of u^n.
  float2 Qs[T][C::Q];
#pragma unroll
  for (int k = 0; k < T; ++k)
#pragma unroll
    for (int s = 0; s < C::Q; ++s) Qs[k][s] = make_float2(0.f, 0.f);
#pragma unroll
  for (int s = 0; s < C::Q; ++s) {
    const int plane = jstart - 1 - R + s;
    if (v0 && plane >= 0 && plane < P.n0) {
      Qs[0][s] = __ldg(reinterpret_cast<const float2*>(P.u_cur + (size_t)plane * ps + coff));
      if (!v1) Qs[0][s].y = 0.f;
    }
  }
  // (fused steps k >= 1 are idle at the first stream step: their planes
  //  precede the chunk, so nothing is staged for them yet)

#pragma unroll 1
  for (int j = jstart; j <= jend; ++j) {
    const bool act0 = j >= pd.xc0 && j < pd.xc1;
    bool next_need = false;  // a fused step k >= 1 works at stream step j + 1
#pragma unroll
    for (int k = 1; k < T; ++k) {
      const int q = j + 1 - k * R;
      next_need |= (q >= pd.xc0 && q < pd.xc1);
    }
    if constexpr (T > 1) {
      if (tid == 0 && next_need && j + 1 - R >= jstart) {
        // the strips used at stream step j+1 were produced at step j+1-R
        const unsigned long long target = P.prog_base + (unsigned long long)(j + 1 - R - jstart + 1);
        const int nbs[4] = {nb_up, nb_dn, nb_lf, nb_rt};
        const unsigned long long t0 = global_ns();
        bool okn = true;
        for (int i = 0; i < 4 && okn; ++i)
          if (nbs[i] >= 0) okn = bounded_wait_ge(&P.progress[nbs[i]], target, t0, tmo);
        if (!okn) {
          atomicExch(P.err, 1);
          s_abort = 1;
        }
        __threadfence();
      }
    }
    // this step's TMA data, and the halos prefetched during the previous step
    const int su0 = (j - jstart) % C::NU, suR = (j + R - jstart) % C::NU;
    bool ok = mbar_wait(bar_u + su0, ((j - jstart) / C::NU) & 1, tmo);
    ok = ok && mbar_wait(bar_u + suR, ((j + R - jstart) / C::NU) & 1, tmo);
    if (act0) {
      ok = ok && mbar_wait(bar_p + (j - jstart) % C::NP, ((j - jstart) / C::NP) & 1, tmo);
      ok = ok && mbar_wait(bar_c + (j - jstart) % C::NC, ((j - jstart) / C::NC) & 1, tmo);
    }
    if (!ok) {
      atomicExch(P.err, 2);
      s_abort = 1;
    }
    if constexpr (T > 1) cp_async_wait_all();
    __syncthreads();
    if (s_abort) {
      if (tid == 0) drain(j);
      return;
    }
    if constexpr (T > 1) {
      if (next_need) prefetch_halos(j + 1);
    }

    // ---- fused steps
    const float* ub = uring + su0 * C::PSLOT;  // u^n plane j with its halo
    {
      const float2 nq = *reinterpret_cast<const float2*>(uring + suR * C::PSLOT + own);
#pragma unroll
      for (int s = 0; s < C::Q - 1; ++s) Qs[0][s] = Qs[0][s + 1];
      Qs[0][C::Q - 1] = nq;
    }
#pragma unroll
    for (int k = 0; k < T; ++k) {
      const int q = j - k * R;
      const bool act = q >= pd.xc0 && q < pd.xc1;
      float2 un = make_float2(0.f, 0.f);
      if (act) {
        const float* pl =
            (k == 0) ? ub : splane + ((size_t)(j & 1) * (T - 1) + (k > 0 ? k - 1 : 0)) * C::PSLOT;
        const float2 upv =
            (k == 0) ? *reinterpret_cast<const float2*>(pring + ((j - jstart) % C::NP) * C::TILE + own_t)
                     : Qs[k > 0 ? k - 1 : 0][0];
        const float2 c2v = *reinterpret_cast<const float2*>(cring + ((q - jstart) % C::NC) * C::TILE + own_t);
        const float bx = __ldg(&P.damp_b[q]);
        const float2 uc = Qs[k][R];
        // axis-2 window as column pairs: zp[m] = columns (2 lane - R + 2m, +1)
        float2 zp[R + 1];
#pragma unroll
        for (int m = 0; m <= R; ++m)
          zp[m] = (m == R / 2) ? uc : *reinterpret_cast<const float2*>(&pl[own - R + 2 * m]);
        float2 lap = make_float2(0.f, 0.f);
#pragma unroll
        for (int d = 1; d <= R; ++d) {
          const float2 yp = *reinterpret_cast<const float2*>(&pl[own + d * SW]);
          const float2 ym = *reinterpret_cast<const float2*>(&pl[own - d * SW]);
          float2 zpl, zmi;
          if (d % 2 == 0) {
            zpl = zp[R / 2 + d / 2];
            zmi = zp[R / 2 - d / 2];
          } else {
            zpl = make_float2(zp[R / 2 + (d - 1) / 2].y, zp[R / 2 + (d + 1) / 2].x);
            zmi = make_float2(zp[R / 2 - (d + 1) / 2].y, zp[R / 2 - (d - 1) / 2].x);
          }
          lap = pair_term2(lap, P.w2[0][d - 1], Qs[k][R + d], Qs[k][R - d], uc);
          lap = pair_term2(lap, P.w2[1][d - 1], yp, ym, uc);
          lap = pair_term2(lap, P.w2[2][d - 1], zpl, zmi, uc);
        }
        if (v0) un.x = point_update(uc.x, upv.x, lap.x, c2v.x, __fadd_rn(bx, byz0));
        if (v1) un.y = point_update(uc.y, upv.y, lap.y, c2v.y, __fadd_rn(bx, byz1));

        const int step = P.step0 + k;
        if (flags & 3) {  // fused grid-aligned injection (Listing 5)
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            if (!((flags >> i) & 1)) continue;
            unsigned short* cp = &ccur[((0 * T + k) * 2 + i) * NT + tid];
            int cc = *cp;
            const int cn = ccnt[(0 * 2 + i) * NT + tid], cb = cbase[(0 * 2 + i) * NT + tid];
            while (cc < cn) {
              const int2 e = __ldg(&P.s_ent[cb + cc]);
              if (e.x < q) {
                ++cc;
                continue;
              }
              if (e.x == q) {
                const float add = __ldg(&P.src_dcmp[(size_t)step * P.npts + e.y]);
                if (i == 0) un.x = __fadd_rn(un.x, add);
                else un.y = __fadd_rn(un.y, add);
                ++cc;
              }
              break;
            }
            *cp = (unsigned short)cc;
          }
        }
        if ((flags & 12) && own_row && q >= pd.xo0 && q < pd.xo1) {  // receiver points
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            if (!((flags >> (2 + i)) & 1)) continue;
            unsigned short* cp = &ccur[((1 * T + k) * 2 + i) * NT + tid];
            int cc = *cp;
            const int cn = ccnt[(1 * 2 + i) * NT + tid], cb = cbase[(1 * 2 + i) * NT + tid];
            while (cc < cn) {
              const int2 e = __ldg(&P.r_ent[cb + cc]);
              if (e.x < q) {
                ++cc;
                continue;
              }
              if (e.x == q) {
                P.rec_dcmp[(size_t)(step - P.rec_base) * P.nrpts + e.y] = (i == 0 ? un.x : un.y);
                ++cc;
              }
              break;
            }
            *cp = (unsigned short)cc;
          }
        }
      }
      if (k + 1 < T) {
        const int kn = (k + 1 < T) ? k + 1 : 0;
        // hand the new level to the next fused step ...
#pragma unroll
        for (int s = 0; s < C::Q - 1; ++s) Qs[kn][s] = Qs[kn][s + 1];
        Qs[kn][C::Q - 1] = un;
        // ... stage its centre for the next stream step ...
        const int qn = j + 1 - (k + 1) * R;
        if (qn >= pd.xc0 && qn < pd.xc1)
          *reinterpret_cast<float2*>(splane + ((size_t)((j + 1) & 1) * (T - 1) + k) * C::PSLOT + own) =
              Qs[kn][R + 1];
        // ... and publish its halo strips
        if (act) {
          float* rs = ring_strip(b, k, q);
          if (w < R) __stcg(reinterpret_cast<float2*>(rs + w * TZ + 2 * lane), un);
          if (w >= TY - R) __stcg(reinterpret_cast<float2*>(rs + (R + w - (TY - R)) * TZ + 2 * lane), un);
          if (2 * lane < RP) __stcg(reinterpret_cast<float2*>(rs + 2 * R * TZ + w * RP + 2 * lane), un);
          if (2 * lane >= TZ - RP)
            __stcg(reinterpret_cast<float2*>(rs + 2 * R * TZ + TY * RP + w * RP + 2 * lane - (TZ - RP)), un);
        }
      } else if (act && own_row && q >= pd.xo0 && q < pd.xo1 && v0) {
        __stcs(reinterpret_cast<float2*>(P.out0 + (size_t)q * ps + coff), un);
        if constexpr (T > 1) __stcs(reinterpret_cast<float2*>(P.out1 + (size_t)q * ps + coff), Qs[k][R]);
      }
    }
    __syncthreads();  // every read of this step's slots is done
    if (tid == 0) {
      if constexpr (T > 1) {
        __threadfence();
        st_release_u64(&P.progress[b], P.prog_base + (unsigned long long)(j - jstart + 1));
      }
      // refill u^n plane j's slot, u^{n-1} plane j's slot, c2 plane j-(T-1)r's slot
      issue_u(j + C::NU);
      issue_p(j + C::PF + 1);
      issue_c(j + C::PF + 1);
    }
  }
  if (tid == 0) drain(jend + 1);  // the prefetches still in flight
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
    void* args[] = {const_cast<SweepParams*>(&p)};
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
  s->box_w = Cf::SW;
  s->box_h = Cf::SH;
  s->halo_w = Cf::RP;
}

// Per-radius entry points (one translation unit per radius), T = 1..TMAX.
#define TBI_DEFINE_RADIUS_T(RR, TT)                                                \
  case TT:                                                                         \
    if (what == 0) return sweep_launch_t<RR, TT>(*p, nctas, coop, st);             \
    if (what == 1) return sweep_occupancy_t<RR, TT>(per_sm);                       \
    sweep_shape_t<RR, TT>(s);                                                      \
    return cudaSuccess;

}  // namespace tbi
