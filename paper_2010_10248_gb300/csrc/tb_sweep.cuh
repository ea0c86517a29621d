// Acoustic propagator sweep: T time steps of Eq. 1 fused in one pass
// (T = 1 is the spatially blocked one-step kernel).
//
// Layout.  Fields are [n0][n1][n2p] floats, axis 2 contiguous (row pitch
// n2p = n2 rounded up to 4).  A CTA owns a tile of TY rows (axis 1) by 64
// columns (axis 2) and streams it along axis 0.  TY compute warps own one
// row each (a lane owns two adjacent columns: float2 loads and packed f32x2
// arithmetic); one more warp is the producer.
//
// Producer warp (asynchronous data movement, runs ahead of the compute):
//   * per stream step j, one mbarrier covers three TMA loads: the u^n plane
//     j+r as a (TY+2r) x (64+2rp) box with halo (out-of-grid cells arrive as
//     zeros: the zero boundary of Eq. 1) and the own tiles of u^{n-1} and
//     c2 = dt^2/m at plane j, each into its ring of planes;
//   * retires stream steps (an mbarrier the compute warps arrive on) and
//     frees their ring slots.
// Halo warp (blocked sweeps, T > 1): for fused steps k >= 1 it copies the
// neighbours' halo strips of level n+k from a small L2-resident ring in
// global memory into a coming stream step's shared planes (bulk TMA copies,
// one per strip row), once the neighbours' progress counters (polled by
// four lanes at once) show the strips are written: the top and bottom
// strips with one bulk TMA copy each, completing on that step's centre
// barrier, the left and right columns with 16-byte L2 loads and shared
// stores; then the warp's one arrival on the centre barrier.
// Publisher warp (T > 1): publishes each retired step in the CTA's progress
// counter (a release store, whose fence can take microseconds: it is kept
// off the producer's and the halo warp's paths).
// Receiver warp: records u at the tile's receiver points for every fused
// step (levels n+1 .. n+T-1 from the staged shared planes, level n+T from
// the sweep's output once the step is retired), so that a receiver plane
// costs the compute warps nothing.
// Compute warps wait on two mbarriers per stream step (the step's data and
// the centre/halo planes); every wait is bounded by a timeout, after which
// the CTA records an error and returns (helper warps first drain their own
// copies in flight).
//
// Temporal blocking (Sec. II-B, re-designed for the GPU).  Fused step k
// (k = 0..T-1) computes level n+k+1 at plane q_k = j - k r of stream step
// j.  Step 0 reads all its neighbours from the u^n ring.  Steps k >= 1 keep,
// per owned column, a register queue of the 2r+1 planes of their input
// level around q_k (the axis-0 neighbours) and read axis-1/axis-2
// neighbours from a double-buffered shared plane (centres written by the
// compute warps, halos copied from the neighbours' strips).  A step's output goes
// straight into the next step's queue, so intermediate levels never reach
// HBM: per T steps a point costs one read of u^n, u^{n-1}, c2 and one write
// of u^{n+T}, u^{n+T-1}.  All CTAs of a pass stream in lockstep
// (cooperative launch, co-resident); within a pass there is no redundant
// computation, passes (bands along axis 1, chunks along axis 0) overlap by
// (T-1) r rows or planes.  A launch may hold passes of two consecutive time
// tiles (SweepParams::set[0] and set[1]): the last band of tile k and the
// first rows of tile k + 1, which depend only on rows of tile k finished by
// earlier launches, so that every launch fills the GPU.
//
// Grid-aligned sparse operators (Sec. II-A).  Sources: each lane's column
// pair has one range of planes that holds source points (built from the
// inspector's per-column entries when the sources are set), and each fused
// step adds the pair's injection right after the stencil update of a plane
// in that range (Listing 5's fused injection, along the streamed axis); the
// test is branch-light and stateless so that it does not split the step's
// code.  Receivers: the receiver warp walks the per-column entries (x, id)
// with one cursor per fused step and records u into rec_dcmp[step mod
// rec_cap][rid] (rec_cap a power of two).
//
// Rounding.  Every floating-point operation of the point update is an
// explicit round-to-nearest operation, so each fused step and the one-step
// kernel produce bitwise-identical values.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tb_async.cuh"
#include "tb_internal.cuh"

namespace tbi {

// Wavefield storage of a sweep: SK = 0 FP32; SK = 1 FP16, SK = 2 BF16 (one-
// step kernel only), where a stored field holds u / s with a power-of-two
// scale s per field and step.  Arithmetic is FP32 in every case.
template <int SK> struct StoreT { using type = float; };
template <> struct StoreT<1> { using type = __half; };
template <> struct StoreT<2> { using type = __nv_bfloat16; };
constexpr size_t align128(size_t b) { return (b + 127) / 128 * 128; }

template <int R, int T, int TY, int SK = 0>
struct SweepCfg {
  using ST = typename StoreT<SK>::type;
  static constexpr int ESZ = (int)sizeof(ST);  // bytes of a stored wavefield value
  static_assert(SK == 0 || T == 1, "16-bit storage: one-step kernel only");
  static constexpr int TZ = 64;
  static constexpr int NCOL = TY * TZ;         // columns of a tile
  // compute lanes own CW adjacent columns of one tile row (CW / 2 packed
  // f32x2 pairs).  The one-step kernel takes four (float4 accesses; a warp
  // covers two rows; two CTAs per SM keep 16 compute warps on an SM); the
  // blocked sweep, one CTA per SM whose fused steps form a long dependency
  // chain per stream step, takes two so that 16 compute warps hide it.
  static constexpr int CW = T == 1 ? 4 : 2;
  static constexpr int NPAIR = CW / 2;
  static constexpr int RPW = 32 * CW / TZ;   // tile rows per warp
  static constexpr int NWC = TY / RPW;
  static constexpr int NT = 32 * NWC;          // compute threads
  static constexpr bool HALO = T > 1;          // halo and publisher warps present
  // + producer, receiver (+ halo, publisher) warps
  static constexpr int NTHREADS = NT + 64 + (HALO ? 64 : 0);
  static constexpr int WPRO = NWC, WREC = NWC + 1;       // producer, receiver warps
  static constexpr int WHALO = NWC + 2, WPUB = NWC + 3;  // halo, publisher warps (T > 1)
  // axis-2 halo width in shared memory: a multiple of four values (16-byte
  // rows for the float4 accesses); with 16-bit values 8 keeps the TMA box's
  // first column z0 - RP on a 16-byte boundary
  static constexpr int RP = SK ? 8 : (R + 3) / 4 * 4;
  static constexpr int SW = TZ + 2 * RP;       // plane row stride (values)
  static constexpr int SH = TY + 2 * R;
  static constexpr int PLANE = SW * SH;
  static constexpr int PSLOT = (int)(align128(PLANE * ESZ) / ESZ);
  static constexpr int TILE = TY * TZ;
  static constexpr int Q = 2 * R + 1;                // queue length (planes around the centre)
  static constexpr int PF = 2;                       // planes of prefetch beyond need
  // fused step 0 takes its axis-0 neighbours from a register queue where
  // the registers allow (up to three queues of Q column groups: measured
  // 12 % faster at T = 3, r = 4 than reading them from the u^n ring), else
  // from the u^n ring
  static constexpr bool X0Q = T <= 3;
  static constexpr int NQ = X0Q ? T : T - 1;         // register queues
  static constexpr int NU = (X0Q ? R + 1 : 2 * R + 1) + PF;  // u^n box ring
  static constexpr int ULAG = X0Q ? 0 : R;           // plane p is last read at step p + ULAG
  static constexpr int NP = PF + 1;                  // u^{n-1} tile ring
  static constexpr int NC = (T - 1) * R + 1 + PF;    // c2 tile ring
  static constexpr int ND = PF + 2;                  // per-step data barriers
  // the data of stream step s may be loaded once step s - LEAD is retired
  static constexpr int LEAD = PF + 1;
  static_assert(NU - R - ULAG >= LEAD && NP >= LEAD && NC - (T - 1) * R >= LEAD && ND >= LEAD,
                "ring depths must cover the prefetch distance");
  static constexpr int NDONE = 8;                    // step-retirement barriers
  // helper warps' polls back off up to this many ns (their issue slots are
  // the compute warps')
  static constexpr unsigned kNapMax = 512;
  // the stream loop is unrolled by the queue length, so that the axis-0
  // register queues rotate by renaming; else they shift every step
  static constexpr bool UNROLL = true;
  static constexpr int D = 2 * R + 2;                // halo ring slots per fused step (global)
  // halo strips of one tile and fused step in the global ring: the top and
  // bottom R rows with the plane's row pitch SW (so that each lands in
  // shared memory with one contiguous copy), then the left and right RP
  // columns of the TY rows
  static constexpr int STRIP_Y = R * SW;
  static constexpr int STRIP = 2 * STRIP_Y + 2 * TY * RP;
  static constexpr int RING_PER_CTA = T > 1 ? (T - 1) * D * STRIP : 0;
  static constexpr int NSP = T > 1 ? 2 * (T - 1) : 0;  // fused-step planes
  static constexpr int CTR_COUNT = NT + (HALO ? 2 : 0);   // arrivals per centre phase: + halo, receiver
  static constexpr size_t OFF_U = 0;
  static constexpr size_t OFF_P = OFF_U + align128((size_t)NU * PSLOT * ESZ);
  static constexpr size_t OFF_C = OFF_P + align128((size_t)NP * TILE * ESZ);
  static constexpr size_t OFF_S = OFF_C + align128((size_t)NC * TILE * 4);
  static constexpr size_t OFF_BASE = OFF_S + align128((size_t)NSP * PSLOT * 4);
  static constexpr size_t OFF_CNT = OFF_BASE + 4 * NCOL;
  static constexpr size_t OFF_CUR = OFF_CNT + 2 * NCOL;
  static constexpr size_t OFF_XF = OFF_CUR + 2 * T * NCOL;      // receiver columns' first x
  static constexpr size_t OFF_RL = OFF_XF + 2 * NCOL;   // receiver warp: list of receiver columns
  static constexpr size_t OFF_BAR = align128(OFF_RL + 2 * NCOL);
  static constexpr int NBAR = 1 + ND + 2 + NDONE;    // prologue, data, centre[2], done
  static constexpr size_t SMEM = OFF_BAR + 8 * NBAR + 128;    // + base alignment
  static_assert(R % 2 == 0, "radius must be even for aligned float2 access");
  // a halo comes from one neighbour tile, and the top and bottom strips a tile
  // publishes (its first and last r rows) must not overlap
  static_assert(TY % 2 == 0 && TY >= 2 * R && TZ >= RP, "tile too small for the stencil radius");
  static_assert(SMEM <= 232448, "shared memory budget exceeded");
};

__device__ __forceinline__ int j_mod(int j, int d) { return j % d; }

// ------------------------------------------------------------ arithmetic --
// A lane's CW = 2 NP adjacent columns as NP column pairs (packed f32x2
// operands), moved as one float2 (NP = 1) or float4 (NP = 2).
template <int NP>
struct FV {
  float2 p[NP];
};
template <int NP>
__device__ __forceinline__ FV<NP> fvzero() {
  FV<NP> v;
#pragma unroll
  for (int i = 0; i < NP; ++i) v.p[i] = make_float2(0.f, 0.f);
  return v;
}
template <int NP>
__device__ __forceinline__ FV<NP> ldv(const float* p) {
  FV<NP> v;
  if constexpr (NP == 1) {
    v.p[0] = *reinterpret_cast<const float2*>(p);
  } else {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v.p[0] = make_float2(q.x, q.y);
    v.p[1] = make_float2(q.z, q.w);
  }
  return v;
}
__device__ __forceinline__ float2 h2f(unsigned x) { return __half22float2(*reinterpret_cast<const __half2*>(&x)); }
__device__ __forceinline__ float2 b2f(unsigned x) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&x));
}
template <int NP>
__device__ __forceinline__ FV<NP> ldv(const __half* p) {
  FV<NP> v;
  if constexpr (NP == 1) {
    v.p[0] = h2f(*reinterpret_cast<const unsigned*>(p));
  } else {
    const uint2 q = *reinterpret_cast<const uint2*>(p);
    v.p[0] = h2f(q.x);
    v.p[1] = h2f(q.y);
  }
  return v;
}
template <int NP>
__device__ __forceinline__ FV<NP> ldv(const __nv_bfloat16* p) {
  FV<NP> v;
  if constexpr (NP == 1) {
    v.p[0] = b2f(*reinterpret_cast<const unsigned*>(p));
  } else {
    const uint2 q = *reinterpret_cast<const uint2*>(p);
    v.p[0] = b2f(q.x);
    v.p[1] = b2f(q.y);
  }
  return v;
}
// stores: plain (shared memory), .cg (halo strips, kept in L2), .cs (outputs)
template <int NP>
__device__ __forceinline__ void stv(float* p, const FV<NP>& v) {
  if constexpr (NP == 1)
    *reinterpret_cast<float2*>(p) = v.p[0];
  else
    *reinterpret_cast<float4*>(p) = make_float4(v.p[0].x, v.p[0].y, v.p[1].x, v.p[1].y);
}
template <int NP>
__device__ __forceinline__ void stvcg(float* p, const FV<NP>& v) {
  if constexpr (NP == 1)
    __stcg(reinterpret_cast<float2*>(p), v.p[0]);
  else
    __stcg(reinterpret_cast<float4*>(p), make_float4(v.p[0].x, v.p[0].y, v.p[1].x, v.p[1].y));
}
// Stores of v to p where `on`, each one predicated instruction: a fused
// step's conditional stores (halo strips, staged centres, the sweep's output)
// then leave its code one block the compiler schedules across (branches
// around them cost the blocked sweep 10 % at T = 3).  Global with .cg (to L2)
// and .cs (streaming), or shared.
template <int NP>
__device__ __forceinline__ void st_pred_cg(bool on, float* p, const FV<NP>& v) {
  if constexpr (NP == 1)
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n @q st.global.cg.v2.f32 [%1], {%2, %3};\n}" ::"r"((int)on),
                 "l"(p), "f"(v.p[0].x), "f"(v.p[0].y));
  else
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n @q st.global.cg.v4.f32 [%1], {%2, %3, %4, %5};\n}" ::"r"((int)on),
                 "l"(p), "f"(v.p[0].x), "f"(v.p[0].y), "f"(v.p[1].x), "f"(v.p[1].y));
}
template <int NP>
__device__ __forceinline__ void st_pred_sh(bool on, float* p, const FV<NP>& v) {
  if constexpr (NP == 1)
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n @q st.shared.v2.f32 [%1], {%2, %3};\n}" ::"r"((int)on),
                 "r"(smem_u32(p)), "f"(v.p[0].x), "f"(v.p[0].y));
  else
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n @q st.shared.v4.f32 [%1], {%2, %3, %4, %5};\n}" ::"r"((int)on),
                 "r"(smem_u32(p)), "f"(v.p[0].x), "f"(v.p[0].y), "f"(v.p[1].x), "f"(v.p[1].y));
}
template <int NP>
__device__ __forceinline__ void st_pred_cs(bool on, float* p, const FV<NP>& v) {
  if constexpr (NP == 1)
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n @q st.global.cs.v2.f32 [%1], {%2, %3};\n}" ::"r"((int)on),
                 "l"(p), "f"(v.p[0].x), "f"(v.p[0].y));
  else
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n @q st.global.cs.v4.f32 [%1], {%2, %3, %4, %5};\n}" ::"r"((int)on),
                 "l"(p), "f"(v.p[0].x), "f"(v.p[0].y), "f"(v.p[1].x), "f"(v.p[1].y));
}
template <int NP>
__device__ __forceinline__ void stvcs(float* p, const FV<NP>& v) {
  if constexpr (NP == 1)
    __stcs(reinterpret_cast<float2*>(p), v.p[0]);
  else
    __stcs(reinterpret_cast<float4*>(p), make_float4(v.p[0].x, v.p[0].y, v.p[1].x, v.p[1].y));
}
__device__ __forceinline__ unsigned f2h(float2 v) {
  const __half2 h = __float22half2_rn(v);
  return *reinterpret_cast<const unsigned*>(&h);
}
__device__ __forceinline__ unsigned f2b(float2 v) {
  const __nv_bfloat162 h = __float22bfloat162_rn(v);
  return *reinterpret_cast<const unsigned*>(&h);
}
template <int NP>
__device__ __forceinline__ void stvcs(__half* p, const FV<NP>& v) {
  if constexpr (NP == 1)
    __stcs(reinterpret_cast<unsigned*>(p), f2h(v.p[0]));
  else
    __stcs(reinterpret_cast<uint2*>(p), make_uint2(f2h(v.p[0]), f2h(v.p[1])));
}
template <int NP>
__device__ __forceinline__ void stvcs(__nv_bfloat16* p, const FV<NP>& v) {
  if constexpr (NP == 1)
    __stcs(reinterpret_cast<unsigned*>(p), f2b(v.p[0]));
  else
    __stcs(reinterpret_cast<uint2*>(p), make_uint2(f2b(v.p[0]), f2b(v.p[1])));
}
// one value from global memory through L2
__device__ __forceinline__ float ld1cg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ float ld1cg(const __half* p) {
  return __half2float(__ushort_as_half(__ldcg(reinterpret_cast<const unsigned short*>(p))));
}
__device__ __forceinline__ float ld1cg(const __nv_bfloat16* p) {
  return __bfloat162float(__ushort_as_bfloat16(__ldcg(reinterpret_cast<const unsigned short*>(p))));
}

// Eq. 1 at one point: u^{n+1} = [dt^2 L u + m(2u - u_prev) + a u_prev]/(m + a)
// rewritten with c2 = dt^2/m and g = a/m = (eta/(2 dt)) c2 as an increment:
//   u^{n+1} = u + (c2 L u + (1 - g)(u - u_prev)) / (1 + g),
// on a column pair with packed f32x2 round-to-nearest operations.  x - y is
// formed as fma(y, -1, x) (the product is exact, so one rounding, as a
// subtraction).  Inside the sponge the quotient is the reciprocal times the
// numerator (within 2 ulp of the correctly rounded division); where g = 0
// every operation reduces exactly to point_update2_free, so the choice
// between the two never changes a result.
__device__ __forceinline__ float2 point_update2(float2 uc, float2 up, float2 lap, float2 c2, float2 bsum) {
  const float2 m1 = make_float2(-1.f, -1.f), one = make_float2(1.f, 1.f);
  const float2 d = __ffma2_rn(up, m1, uc);
  const float2 g = __fmul2_rn(bsum, c2);
  const float2 inc = __ffma2_rn(c2, lap, __fmul2_rn(__ffma2_rn(g, m1, one), d));
  const float2 opg = __fadd2_rn(one, g);
  // where g = 0 the quotient is inc itself, as in point_update2_free
  return __fadd2_rn(uc, make_float2(g.x == 0.f ? inc.x : __fdividef(inc.x, opg.x),
                                    g.y == 0.f ? inc.y : __fdividef(inc.y, opg.y)));
}
// The same update where no damping acts (g = 0): u + (c2 L u + (u - u_prev)).
__device__ __forceinline__ float2 point_update2_free(float2 uc, float2 up, float2 lap, float2 c2) {
  const float2 m1 = make_float2(-1.f, -1.f);
  return __fadd2_rn(uc, __ffma2_rn(c2, lap, __ffma2_rn(up, m1, uc)));
}

// Neighbour pairs of the Laplacian on a column pair.  The pairs with the two
// largest weights (offsets 1 and 2) are taken in differences form,
// acc + w ((a - u) + (b - u)): differences of close values are exact, so
// the large centre term never cancels against the neighbour sum (in FP32
// the c0 u + sum c_i (u_+i + u_-i) form lost ~40x accuracy over 1000 steps).
// The pairs further out (weights below 3 % of the nearest one at space order
// 8 and 12) are summed directly, acc + w (a + b), and their centre term
// -2 sum w u is added once per point: the cancellation there is against
// values ~30x smaller than the centre term of the direct form.
__device__ __forceinline__ float2 pair_diff2(float2 acc, float2 w2, float2 a, float2 b, float2 u) {
  const float2 m1 = make_float2(-1.f, -1.f);
  return __ffma2_rn(w2, __fadd2_rn(__ffma2_rn(u, m1, a), __ffma2_rn(u, m1, b)), acc);
}
__device__ __forceinline__ float2 pair_sum2(float2 acc, float2 w2, float2 a, float2 b) {
  return __ffma2_rn(w2, __fadd2_rn(a, b), acc);
}
constexpr int kDiffPairs = 2;  // offsets taken in differences form

// ----------------------------------------------------------------- kernel --
// The sweep of one CTA: pass pd (the CTA's place in the launch), block
// index b within the launch, time tile s1 (launches holding two), first
// step step0.  P holds the fields, tables and model of the propagation.
template <int R, int T, int TY, int SK, bool TWO, bool PRE>
__device__ __forceinline__ void sweep_body(const SweepParams& P, const PassDesc& pd, const int b, const bool s1,
                                           const int step0) {
  using C = SweepCfg<R, T, TY, SK>;
  using ST = typename C::ST;
  constexpr int TZ = C::TZ, NT = C::NT, SW = C::SW, RP = C::RP, NCOL = C::NCOL;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // TMA destinations need 128-byte alignment: align the base explicitly
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  ST* uring = reinterpret_cast<ST*>(smem + C::OFF_U);
  ST* pring = reinterpret_cast<ST*>(smem + C::OFF_P);
  float* cring = reinterpret_cast<float*>(smem + C::OFF_C);
  float* splane = reinterpret_cast<float*>(smem + C::OFF_S);
  uint64_t* bar_pro = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);  // u^n planes before the first step
  uint64_t* bar_dat = bar_pro + 1;     // [ND] data of stream step j
  uint64_t* bar_ctr = bar_dat + C::ND; // [2] centres and halos of stream step j in buffer j & 1
  uint64_t* bar_done = bar_ctr + 2;    // [NDONE] compute warps finished a stream step
  // per-column state of the grid-aligned receivers (receiver warp)
  int* cbase = reinterpret_cast<int*>(smem + C::OFF_BASE);                      // [NCOL]
  unsigned short* ccnt = reinterpret_cast<unsigned short*>(smem + C::OFF_CNT);  // [NCOL]
  unsigned short* ccur = reinterpret_cast<unsigned short*>(smem + C::OFF_CUR);  // [T][NCOL]
  unsigned short* cxf = reinterpret_cast<unsigned short*>(smem + C::OFF_XF);    // [NCOL]

  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  // the pass's time tile: launches holding two time tiles run the TWO
  // instantiation, which selects the fields by the block index (the select
  // costs ~2 % more instructions in the fused steps, so single-tile
  // launches take the other one)
  float* const out0 = s1 ? P.set[1].out0 : P.set[0].out0;
  float* const out1 = s1 ? P.set[1].out1 : P.set[0].out1;
  const float* const u_cur = s1 ? P.set[1].u_cur : P.set[0].u_cur;
  const CUtensorMap* const tm_u = s1 ? &P.set[1].tm_u : &P.set[0].tm_u;
  const CUtensorMap* const tm_p = s1 ? &P.set[1].tm_p : &P.set[0].tm_p;
  const int tl = b - pd.cta0, ty = tl / pd.ntz, tz = tl - ty * pd.ntz;
  const int y0 = pd.yb0 + ty * TY, z0 = tz * TZ;
  const int jstart = pd.xc0;
  const int jend = pd.xo1 - 1 + (T - 1) * R;  // inclusive
  const int pu0 = jstart - C::ULAG;           // first u^n plane in the ring
  const long long tmo = P.timeout_ns;
  __shared__ int s_ret;  // last stream step retired (written by the producer)

  if (tid == 0) {
    s_ret = jstart - 1;
    mbar_init(bar_pro, 1);
    for (int i = 0; i < C::ND; ++i) mbar_init(bar_dat + i, 1);
    mbar_init(bar_ctr + 0, C::CTR_COUNT);
    mbar_init(bar_ctr + 1, C::CTR_COUNT);
    for (int i = 0; i < C::NDONE; ++i) mbar_init(bar_done + i, NT);  // every compute thread arrives
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // Missing neighbours leave zero halos in the fused-step planes for good.
  if constexpr (T > 1) {
    for (int e = tid; e < C::NSP * C::PSLOT; e += C::NTHREADS) splane[e] = 0.f;
  }
  __syncthreads();  // the only CTA-wide barrier: set-up done

  const int nb_up = ty > 0 ? b - pd.ntz : -1;
  const int nb_dn = ty + 1 < pd.nty ? b + pd.ntz : -1;
  const int nb_lf = tz > 0 ? b - 1 : -1;
  const int nb_rt = tz + 1 < pd.ntz ? b + 1 : -1;

  if (w == C::WPRO) {
    // =========================== producer warp ===========================
    if (lane != 0) return;
    auto u_slot = [&](int p) { return uring + ((p - pu0) % C::NU) * C::PSLOT; };
    // u^n planes pu0 .. jstart+R-1, needed before the first step
    {
      const int np = jstart + R - pu0;
      mbar_expect_tx(bar_pro, (unsigned)(np * C::PLANE * C::ESZ));
      for (int p = pu0; p < jstart + R; ++p) tma_load_3d(u_slot(p), tm_u, bar_pro, z0 - RP, y0 - R, p);
    }
    // the data of stream step s: u^n plane s+R, u^{n-1} and c2 plane s
    auto issue = [&](int s) {
      uint64_t* bar = bar_dat + (s - jstart) % C::ND;
      mbar_expect_tx(bar, (unsigned)((C::PLANE + C::TILE) * C::ESZ + C::TILE * 4));
      tma_load_3d(u_slot(s + R), tm_u, bar, z0 - RP, y0 - R, s + R);
      tma_load_3d(pring + ((s - jstart) % C::NP) * C::TILE, tm_p, bar, z0, y0, s);
      tma_load_3d(cring + ((s - jstart) % C::NC) * C::TILE, &P.tm_c, bar, z0, y0, s);
    };
    int ns = jstart, ret = jstart - 1;
    bool ok = true;
    while (ret < jend) {
      while (ns <= jend && ns - C::LEAD <= ret) issue(ns++);
      // retire the next stream step (polled with a short back-off so the
      // refills above go out as soon as a step is done)
      const int s = ret + 1;
      // (suspending on the barrier: a polling loop here took issue slots
      // from the compute warps of the producer's sub-partition)
      if (!mbar_wait(bar_done + (s - jstart) % C::NDONE, ((s - jstart) / C::NDONE) & 1, tmo)) {
        atomicExch(P.err, 2);
        ok = false;
        break;
      }
      ret = s;
      st_release_cta_s32(&s_ret, ret);  // for the publisher and the receiver warp
    }
    // drain: wait (bounded) for every load this thread issued; after a full
    // run the compute warps consumed them all
    if (!ok) {
      mbar_wait(bar_pro, 0, tmo);
      for (int s = max(jstart, ns - C::ND); s < ns; ++s)
        mbar_wait(bar_dat + (s - jstart) % C::ND, ((s - jstart) / C::ND) & 1, tmo);
    }
    return;
  }

  if (w == C::WREC) {
    // ============================ receiver warp ============================
    // the tile's receiver columns (own rows), their per-column state and a
    // compact list of their slots (bit 15: entries contiguous in x)
    int* rbase = cbase;
    unsigned short* rcnt = ccnt;
    unsigned short* rcur = ccur;  // [T][NCOL]
    unsigned short* rlist = reinterpret_cast<unsigned short*>(smem + C::OFF_RL);
    int nlist = 0;
    int xlo = 0x7fffffff, xhi = -1;  // planes holding the tile's receiver points
    // tile column sl: row sl / TZ, column sl mod TZ
    for (int s0 = 0; s0 < NCOL; s0 += 32) {
      const int sl = s0 + lane;
      const int yy = y0 + sl / TZ, zz = z0 + sl % TZ;
      bool has = false, dense = false;
      if (P.r_colptr && yy < P.n1 && zz < P.n2 && yy >= pd.yo0 && yy < pd.yo1) {
        const int c = yy * P.n2 + zz;
        const int cb = __ldg(&P.r_colptr[c]), ce = __ldg(&P.r_colptr[c + 1]);
        if (ce > cb) {
          has = true;
          rbase[sl] = cb;
          rcnt[sl] = (unsigned short)(ce - cb);
          const int xf = __ldg(&P.r_ent[cb].x), xl = __ldg(&P.r_ent[ce - 1].x);
          cxf[sl] = (unsigned short)xf;
          dense = xl - xf + 1 == ce - cb;
          xlo = min(xlo, xf);
          xhi = max(xhi, xl);
          for (int k = 0; k < T; ++k) rcur[k * NCOL + sl] = 0;
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, has);
      if (has) rlist[nlist + __popc(m & ((1u << lane) - 1u))] = (unsigned short)(sl | (dense ? 0x8000 : 0));
      nlist += __popc(m);
    }
    __syncwarp();
    xlo = max(__reduce_min_sync(0xffffffffu, xlo), pd.xo0);
    xhi = min(__reduce_max_sync(0xffffffffu, xhi), pd.xo1 - 1);
    const size_t ps = (size_t)P.n1 * P.n2p;
    // u at the receiver points of plane q of level n+kk+1 (fused step kk):
    // from a staged plane, or from the sweep's output in global memory (a
    // plane without receiver points of the tile costs two compares)
    auto record = [&](int kk, int q, const float* plane) {
      if (q < xlo || q > xhi) return;
      float* rrow = P.rec_dcmp + (size_t)((step0 + kk) & (P.rec_cap - 1)) * P.nrpts;
      for (int e = lane; e < nlist; e += 32) {
        const int en = rlist[e], sl = en & 0x7fff, row = sl / TZ, col = sl % TZ;
        const int cn = rcnt[sl], cb = rbase[sl];
        int pos = -1;
        if (en & 0x8000) {
          const unsigned off = (unsigned)(q - (int)cxf[sl]);
          if (off < (unsigned)cn) pos = cb + (int)off;
        } else {
          unsigned short* cp = &rcur[kk * NCOL + sl];
          int cc = *cp;
          while (cc < cn) {
            const int x = __ldg(&P.r_ent[cb + cc].x);
            if (x < q) {
              ++cc;
              continue;
            }
            if (x == q) pos = cb + cc++;
            break;
          }
          *cp = (unsigned short)cc;
        }
        if (pos >= 0) {
          const size_t go = (size_t)q * ps + (size_t)(y0 + row) * P.n2p + z0 + col;
          if constexpr (SK != 0)  // one-step only: u^{n+1} is stored as u / s
            rrow[pos] = __fmul_rn(ld1cg(reinterpret_cast<const ST*>(out0) + go),
                                  lp_next_scale(P.lp_mx, P.lp_srcmax, step0));
          else
            rrow[pos] = plane ? plane[(R + row) * SW + RP + col] : __ldcg(out0 + go);
        }
      }
    };
    // steps retired by the producer (its level-n+T planes are in global memory)
    auto wait_retired = [&](int jr) -> bool {
      const unsigned long long t0 = global_ns();
      unsigned nap = 64;
      while (ld_acquire_cta_s32(&s_ret) < jr) {
        if ((long long)(global_ns() - t0) > tmo) return false;
        __nanosleep(nap);
        nap = nap < C::kNapMax ? 2 * nap : nap;
      }
      return true;
    };
    bool ok = true;
    if constexpr (T == 1) {
      for (int j = jstart; j <= jend && ok; ++j) {
        ok = __all_sync(0xffffffffu, wait_retired(j));
        if (ok) record(0, j, nullptr);
      }
    } else {
      for (int j = jstart; j <= jend + 1 && ok; ++j) {
        if (j <= jend) {
          // levels n+1 .. n+T-1 of this step's centre planes; then release
          // the buffer to the compute warps' staging of step j+2
          if (j > jstart) {
            ok = __all_sync(0xffffffffu, mbar_wait(bar_ctr + (j & 1), ((j - jstart - 1) >> 1) & 1, tmo));
            if (!ok) break;
            const float* rdbuf = splane + (size_t)(j & 1) * (T - 1) * C::PSLOT;
            for (int k = 1; k < T; ++k) record(k - 1, j - k * R, rdbuf + (size_t)(k - 1) * C::PSLOT);
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(bar_ctr + ((j + 1) & 1));
        }
        // level n+T of the step before, written to the output (ctr(j) implies
        // it for j <= jend; the last step waits for its retirement)
        if (j - 1 >= jstart) {
          if (j > jend) ok = __all_sync(0xffffffffu, wait_retired(j - 1));
          if (ok) record(T - 1, j - 1 - (T - 1) * R, nullptr);
        }
      }
    }
    if (!ok) atomicExch(P.err, 2);
    return;
  }

  if constexpr (C::HALO) {
    if (w == C::WPUB) {
      // =========================== publisher warp ===========================
      // publishes the producer's latest retired step (it may skip steps
      // while a release is in flight: the counter is monotonic)
      if (lane != 0) return;
      unsigned nap = 64;
      int pub = jstart - 1;
      unsigned long long t0 = global_ns();
      while (pub < jend) {
        const int r = ld_acquire_cta_s32(&s_ret);
        if (r > pub) {
          // release: cumulative over the compute warps' strip stores, which
          // happen before their arrival on the step's mbarrier, which the
          // producer observed before it wrote s_ret
          st_release_u64(&P.progress[(size_t)b * kProgressStride], P.prog_base + (unsigned long long)(r - jstart + 1));
          pub = r;
          t0 = global_ns();
          nap = 64;
        } else {
          if ((long long)(global_ns() - t0) > tmo) {
            atomicExch(P.err, 2);
            break;
          }
          __nanosleep(nap);
          nap = nap < C::kNapMax ? 2 * nap : nap;
        }
      }
      return;
    }
    if (w == C::WHALO) {
      // ============================= halo warp =============================
      // progress of neighbour `lane` (lanes 0..3: up, down, left, right)
      const int nb = lane == 0 ? nb_up : lane == 1 ? nb_dn : lane == 2 ? nb_lf : lane == 3 ? nb_rt : -1;
      unsigned long long seen = 0;
      constexpr unsigned BYTES_Y = C::STRIP_Y * 4;  // one top or bottom strip
      constexpr int CH_Z = TY * (RP / 4);           // 16-byte chunks per side strip
      const size_t tile_stride = (size_t)(T - 1) * C::D * C::STRIP;
      const unsigned bytes_k = (nb_up >= 0 ? BYTES_Y : 0) + (nb_dn >= 0 ? BYTES_Y : 0);
      bool ok = true;
      int last = jstart;  // last step whose copies were issued
      for (int jn = jstart + 1; jn <= jend && ok; ++jn) {
        // the strips of step jn are written by the neighbours' step jn - R
        if (jn - R >= jstart) {
          const unsigned long long target = P.prog_base + (unsigned long long)(jn - R - jstart + 1);
          const unsigned long long t0 = global_ns();
          unsigned nap = 32;  // back-off: the warp's polls take issue slots from the compute warps
          while (true) {
            if (nb >= 0 && seen < target) seen = ld_acquire_u64(&P.progress[(size_t)nb * kProgressStride]);
            if (__all_sync(0xffffffffu, nb < 0 || seen >= target)) break;
            if (__any_sync(0xffffffffu, (long long)(global_ns() - t0) > tmo)) {  // warp-uniform
              ok = false;
              break;
            }
            __nanosleep(nap);
            nap = nap < C::kNapMax ? 2 * nap : nap;
          }
          if (!ok) {
            atomicExch(P.err, 1);
            break;
          }
        }
        // buffer jn & 1 was last read during step jn - 2
        if (jn - 2 >= jstart) {
          const int s = jn - 2;
          ok = __all_sync(0xffffffffu,
                          mbar_wait(bar_done + (s - jstart) % C::NDONE, ((s - jstart) / C::NDONE) & 1, tmo));
          if (!ok) {
            atomicExch(P.err, 2);
            break;
          }
        }
        // the acquiring lanes' observations precede every lane's reads; the
        // bulk copies read through the async proxy
        __syncwarp();
        asm volatile("fence.proxy.async.global;" ::: "memory");
        uint64_t* bar = bar_ctr + (jn & 1);
        float* buf = splane + (size_t)(jn & 1) * (T - 1) * C::PSLOT;
        if (lane == 0) {
          unsigned bytes = 0;
          for (int k = 1; k < T; ++k) {
            const int q = jn - k * R;
            if (q >= pd.xc0 && q < pd.xc1) bytes += bytes_k;
          }
          mbar_expect_tx_only(bar, bytes);
        }
        __syncwarp();
        // top / bottom strips: one bulk copy each per fused step
        if (lane < 2 * (T - 1)) {
          const int k = 1 + (lane >> 1);
          const int q = jn - k * R;
          const int nbv = (lane & 1) ? nb_dn : nb_up;
          if (q >= pd.xc0 && q < pd.xc1 && nbv >= 0) {
            float* pl = buf + (k - 1) * C::PSLOT;
            const float* src = P.ring + (size_t)nbv * tile_stride + (size_t)(k - 1) * C::D * C::STRIP +
                               (size_t)(q % C::D) * C::STRIP;
            if (lane & 1)  // bottom halo rows: the lower neighbour's top strip
              bulk_load(pl + (TY + R) * SW, src, BYTES_Y, bar);
            else  // top halo rows: the upper neighbour's bottom strip
              bulk_load(pl, src + C::STRIP_Y, BYTES_Y, bar);
          }
        }
        // left / right columns: 16-byte L2 loads (issued together), then stores
        constexpr int NZ = (T - 1) * 2 * CH_Z;
        constexpr int PER = (NZ + 31) / 32;
        float4 v[PER];
        float* dst[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
          const int e = lane + 32 * i;
          dst[i] = nullptr;
          if (e < NZ) {
            const int k = 1 + e / (2 * CH_Z), r = e - (k - 1) * 2 * CH_Z;
            const int q = jn - k * R;
            const bool left = r < CH_Z;
            const int rr = left ? r : r - CH_Z, row = rr / (RP / 4), c4 = 4 * (rr - row * (RP / 4));
            const int nbv = left ? nb_lf : nb_rt;
            if (q >= pd.xc0 && q < pd.xc1 && nbv >= 0) {
              float* pl = buf + (k - 1) * C::PSLOT;
              const float* src = P.ring + (size_t)nbv * tile_stride + (size_t)(k - 1) * C::D * C::STRIP +
                                 (size_t)(q % C::D) * C::STRIP + 2 * C::STRIP_Y;
              // left halo: the left neighbour's right strip; right: the right one's left strip
              src += (left ? TY * RP : 0) + row * RP + c4;
              dst[i] = pl + (R + row) * SW + (left ? 0 : RP + TZ) + c4;
              v[i] = __ldcg(reinterpret_cast<const float4*>(src));
            }
          }
        }
#pragma unroll
        for (int i = 0; i < PER; ++i)
          if (dst[i]) *reinterpret_cast<float4*>(dst[i]) = v[i];
        __syncwarp();  // every lane's stores precede lane 0's arrival
        if (lane == 0) mbar_arrive(bar);
        last = jn;
      }
      if (!ok) {
        // copies of the last two issued steps may be in flight: they complete
        // on the centre phases; wait for those (bounded) before exiting
        for (int jn = max(jstart + 1, last - 1); jn <= last; ++jn)
          mbar_wait(bar_ctr + (jn & 1), ((jn - jstart - 1) >> 1) & 1, tmo);
      }
      return;
    }
  }

  // ============================== compute warps ==============================
  // A lane owns the CW adjacent columns c0 .. c0 + CW - 1 of tile row r: a
  // warp covers RPW rows (lanes 0-15 and 16-31 with four columns each, or
  // all 32 lanes of one row with two).
  constexpr int CW = C::CW, NPR = C::NPAIR;
  using V = FV<NPR>;
  constexpr int LPR = TZ / CW;                    // lanes per tile row
  const int r = C::RPW * w + lane / LPR, c0 = CW * (lane % LPR);
  const int y = y0 + r, z = z0 + c0;
  const bool vrow = y < P.n1;
  const bool vz = vrow && z < P.n2;               // the lane's first column is in the grid
  const bool own_row = y >= pd.yo0 && y < pd.yo1;
  const size_t ps = (size_t)P.n1 * P.n2p;         // plane stride
  const size_t coff = (size_t)y * P.n2p + z;      // column offset (valid if vz)
  const int own = (R + r) * SW + RP + c0;         // own columns in a plane slot
  const int own_t = r * TZ + c0;                  // own columns in a tile slot
  // this thread's place in the halo strips it publishes (-1: none)
  const int strip_y = r < R ? r * SW + RP + c0 : (r >= TY - R ? (R + r - (TY - R)) * SW + RP + c0 : -1);
  const int strip_z = c0 < RP ? 2 * C::STRIP_Y + r * RP + c0
                              : (c0 >= TZ - RP ? 2 * C::STRIP_Y + TY * RP + r * RP + c0 - (TZ - RP) : -1);

  // damping along axes 1 and 2 of the lane's columns (zero outside the
  // grid), and whether none acts anywhere in the warp's columns: then the
  // update takes the undamped form wherever the plane is outside the axis-0
  // sponge
  float bzc[CW];
#pragma unroll
  for (int c = 0; c < CW; ++c) bzc[c] = 0.f;
  if (vrow) {
    const float by = __ldg(&P.damp_b[P.n0 + y]);
#pragma unroll
    for (int c = 0; c < CW; ++c)
      if (z + c < P.n2) bzc[c] = __fadd_rn(by, __ldg(&P.damp_b[P.n0 + P.n1 + z + c]));
  }
  V byz;
  bool nodamp = true;
#pragma unroll
  for (int p = 0; p < NPR; ++p) {
    byz.p[p] = make_float2(bzc[2 * p], bzc[2 * p + 1]);
    nodamp = nodamp && bzc[2 * p] == 0.f && bzc[2 * p + 1] == 0.f;
  }
  const bool yz_free = __all_sync(0xffffffffu, nodamp);

  // centre weight of the directly summed pairs, -2 sum_d sum_{i > 2} c_i / h_d^2
  float2 wcen = make_float2(0.f, 0.f);
  if constexpr (R > kDiffPairs) {
    float s = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int i = kDiffPairs; i < R; ++i) s = __fadd_rn(s, P.w2[d][i].x);
    wcen = make_float2(-2.f * s, -2.f * s);
  }

  // The column pairs' grid-aligned source points (Sec. II-A, Listing 5): the
  // planes ev_x .. ev_x + ev_n - 1 carry the pair's injections, read from
  // src_ev[step][ev_b + plane - ev_x] (zero for a column without a point at
  // that plane).  The check is a compare and a predicated load per fused
  // step and pair, with no loop, cursor or shared-memory store in the step's
  // code.
  int ev_x[NPR], ev_n[NPR];
  const float2* evrow[NPR];
  bool any_src = false;
#pragma unroll
  for (int p = 0; p < NPR; ++p) {
    ev_x[p] = 0;
    ev_n[p] = 0;
    evrow[p] = nullptr;
    if (vz && P.ev_pair && z + 2 * p < P.n2) {
      const int2 d = __ldg(&P.ev_pair[(size_t)y * P.npair + (z >> 1) + p]);
      ev_x[p] = d.x & 0xffff;
      ev_n[p] = (int)((unsigned)d.x >> 16);
      if (ev_n[p] > 0) evrow[p] = P.src_ev + (size_t)step0 * P.nev + d.y;
    }
    any_src = any_src || ev_n[p] > 0;
  }
  // warp-uniform: the fused steps of a warp without source points skip the
  // check (1 % of the blocked sweep's time with one source)
  const bool any_src_w = __any_sync(0xffffffffu, any_src);

  // Register queues along axis 0, rotated by renaming: the stream loop is
  // unrolled by Q = 2r + 1, and at stream step j (phase i = (j - jstart) mod
  // Q) logical entry s of a queue (plane centre - r + s) is register
  // (i + s) mod Q.  Queue QI(k) holds level n+k around the plane of fused
  // step k (level n only with X0Q).
  constexpr int Q = C::Q, NQ = C::NQ;
  auto QI = [](int k) { return C::X0Q ? k : k - 1; };
  V qq[NQ][Q];
#pragma unroll
  for (int k = 0; k < NQ; ++k)
#pragma unroll
    for (int s = 0; s < Q; ++s) qq[k][s] = fvzero<NPR>();
  if constexpr (C::X0Q) {
    // planes jstart - r .. jstart + r - 1 of u^n (logical 0 .. 2r - 1 at phase 0)
#pragma unroll
    for (int s = 0; s < 2 * R; ++s) {
      const int plane = jstart - R + s;
      if (vz && plane >= 0 && plane < P.n0) {
        V v = ldv<NPR>(reinterpret_cast<const ST*>(u_cur) + (size_t)plane * ps + coff);
#pragma unroll
        for (int p = 0; p < NPR; ++p) {
          if (z + 2 * p >= P.n2) v.p[p].x = 0.f;
          if (z + 2 * p + 1 >= P.n2) v.p[p].y = 0.f;
        }
        qq[0][s] = v;
      }
    }
  }
  // damping along axis 0 at fused step k's plane: held by lane k, loaded one
  // stream step ahead, broadcast by shuffle when used
  const int kl = lane % T;  // lane holds fused step (lane mod T)
  float bxn;
  {
    const int q = jstart - kl * R;
    bxn = __ldg(&P.damp_b[min(max(q, 0), P.n0 - 1)]);
  }

  // 16-bit storage: scales of u^{n-1}, u^n and u^{n+1} (powers of two, set
  // by the step's scale kernel) and the running max |u^{n+1}| of this thread
  float2 sc2 = make_float2(1.f, 1.f), sp2 = sc2, io2 = sc2;
  float vmax = 0.f;
  if constexpr (SK != 0) {
    const float so = lp_next_scale(P.lp_mx, P.lp_srcmax, step0);
    const float a = __ldg(P.lp_scales + step0 + 1), p = __ldg(P.lp_scales + step0), o = 1.f / so;
    if (blockIdx.x == 0 && threadIdx.x == 0) P.lp_scales[step0 + 2] = so;  // for the kernels after the step
    sc2 = make_float2(a, a);
    sp2 = make_float2(p, p);
    io2 = make_float2(o, o);
  }

  // Laplacian (differences form for the nearest pairs, direct sums further
  // out, see pair_diff2) of the lane's columns at a plane slot `pl` (axes 1
  // and 2) with centre uc; xn(d) gives the axis-0 neighbours at +d (d > 0)
  // and -d (d < 0).  Every point's terms are summed in one fixed order, so
  // every fused step and the one-step kernel round alike.
  constexpr int NZ = (R + CW - 1) / CW;  // chunks of CW axis-2 neighbours on each side
  auto laplacian = [&](const auto* pl, const V& uc, auto&& xn) -> V {
    float zv[CW * (2 * NZ + 1)];
#pragma unroll
    for (int m = 0; m < NZ; ++m) {
      const V lf = ldv<NPR>(pl + own - CW * (m + 1)), rt = ldv<NPR>(pl + own + CW * (m + 1));
#pragma unroll
      for (int p = 0; p < NPR; ++p) {
        zv[CW * (NZ - 1 - m) + 2 * p] = lf.p[p].x;
        zv[CW * (NZ - 1 - m) + 2 * p + 1] = lf.p[p].y;
        zv[CW * (NZ + 1 + m) + 2 * p] = rt.p[p].x;
        zv[CW * (NZ + 1 + m) + 2 * p + 1] = rt.p[p].y;
      }
    }
#pragma unroll
    for (int p = 0; p < NPR; ++p) {
      zv[CW * NZ + 2 * p] = uc.p[p].x;
      zv[CW * NZ + 2 * p + 1] = uc.p[p].y;
    }
    float2 lx[NPR], ly[NPR], lz[NPR];
#pragma unroll
    for (int d = 1; d <= R; ++d) {
      const V xp = xn(d), xm = xn(-d);
      const V yp = ldv<NPR>(pl + own + d * SW), ym = ldv<NPR>(pl + own - d * SW);
#pragma unroll
      for (int p = 0; p < NPR; ++p) {
        const float2 u = uc.p[p];
        const int c = CW * NZ + 2 * p;
        const float2 cp = make_float2(zv[c + d], zv[c + 1 + d]), cm = make_float2(zv[c - d], zv[c + 1 - d]);
        if (d == 1) {
          const float2 m1 = make_float2(-1.f, -1.f);
          lx[p] = __fmul2_rn(P.w2[0][0], __fadd2_rn(__ffma2_rn(u, m1, xp.p[p]), __ffma2_rn(u, m1, xm.p[p])));
          ly[p] = __fmul2_rn(P.w2[1][0], __fadd2_rn(__ffma2_rn(u, m1, yp.p[p]), __ffma2_rn(u, m1, ym.p[p])));
          lz[p] = __fmul2_rn(P.w2[2][0], __fadd2_rn(__ffma2_rn(u, m1, cp), __ffma2_rn(u, m1, cm)));
        } else if (d <= kDiffPairs) {
          lx[p] = pair_diff2(lx[p], P.w2[0][d - 1], xp.p[p], xm.p[p], u);
          ly[p] = pair_diff2(ly[p], P.w2[1][d - 1], yp.p[p], ym.p[p], u);
          lz[p] = pair_diff2(lz[p], P.w2[2][d - 1], cp, cm, u);
        } else {
          lx[p] = pair_sum2(lx[p], P.w2[0][d - 1], xp.p[p], xm.p[p]);
          ly[p] = pair_sum2(ly[p], P.w2[1][d - 1], yp.p[p], ym.p[p]);
          lz[p] = pair_sum2(lz[p], P.w2[2][d - 1], cp, cm);
        }
      }
    }
    V out;
#pragma unroll
    for (int p = 0; p < NPR; ++p) {
      float2 l = __fadd2_rn(__fadd2_rn(lx[p], ly[p]), lz[p]);
      if constexpr (R > kDiffPairs) l = __ffma2_rn(wcen, uc.p[p], l);
      out.p[p] = l;
    }
    return out;
  };
  // Eq. 1's update of the lane's columns; `free` (warp-uniform): no damping
  // at any of the warp's points
  auto update = [&](const V& uc, const V& up, const V& lap, const V& c2v, float bx, bool free) -> V {
    V o;
    if (free) {
#pragma unroll
      for (int p = 0; p < NPR; ++p) o.p[p] = point_update2_free(uc.p[p], up.p[p], lap.p[p], c2v.p[p]);
    } else {
      const float2 bxx = make_float2(bx, bx);
#pragma unroll
      for (int p = 0; p < NPR; ++p)
        o.p[p] = point_update2(uc.p[p], up.p[p], lap.p[p], c2v.p[p], __fadd2_rn(bxx, byz.p[p]));
    }
    return o;
  };

  bool ok = mbar_wait(bar_pro, 0, tmo);  // u^n planes pu0 .. jstart+R-1

  // fused grid-aligned injection of fused step k at plane q (Listing 5).
  // PRE (sources with long plane ranges): the T values of a stream step are
  // loaded at its top (inj), so that their latency overlaps the steps'
  // arithmetic instead of stalling the fused step that adds them.
  float2 inj[PRE ? T : 1][NPR];
  auto inject = [&](int k, int q, V& un) {
#pragma unroll
    for (int p = 0; p < NPR; ++p) {
      const unsigned off = (unsigned)(q - ev_x[p]);
      if constexpr (PRE) {
        if (off < (unsigned)ev_n[p]) un.p[p] = __fadd2_rn(un.p[p], inj[k][p]);
      } else {
        if (off < (unsigned)ev_n[p]) un.p[p] = __fadd2_rn(un.p[p], __ldg(evrow[p] + (size_t)k * P.nev + off));
      }
    }
  };

  int su = (jstart - pu0) % C::NU;  // ring slot of u^n plane j
  int sp = 0, sc = 0;               // ring slots of u^{n-1}, c2 plane j
  int jd = j_mod(jstart, C::D);     // j mod D (halo ring slot of plane j)
  float* const rs_base = P.ring + (size_t)b * (T > 1 ? (T - 1) * C::D * C::STRIP : 0);
  constexpr int UNR = C::UNROLL ? Q : 1;
#pragma unroll 1
  for (int jb = jstart; jb <= jend && ok; jb += UNR) {
#pragma unroll
    for (int i = 0; i < UNR; ++i) {
      const int j = jb + i;
      if (j <= jend && ok) {
        const bool act0 = j >= pd.xc0 && j < pd.xc1;
        if constexpr (PRE) {
#pragma unroll
          for (int k = 0; k < T; ++k)
#pragma unroll
            for (int p = 0; p < NPR; ++p) {
              const unsigned off = (unsigned)(j - k * R - ev_x[p]);
              inj[k][p] = off < (unsigned)ev_n[p] ? __ldg(evrow[p] + (size_t)k * P.nev + off) : make_float2(0.f, 0.f);
            }
        }
        const float bxc = bxn;
        bxn = __ldg(&P.damp_b[min(max(j + 1 - kl * R, 0), P.n0 - 1)]);
        // u^n plane j+R, u^{n-1} and c2 plane j
        ok = mbar_wait(bar_dat + (j - jstart) % C::ND, ((j - jstart) / C::ND) & 1, tmo);
        if constexpr (T > 1) {
          // centres and halo strips of this step, staged during the previous one;
          // the phase also means every compute thread finished step j-1
          if (j > jstart) ok = ok && mbar_wait(bar_ctr + (j & 1), ((j - jstart - 1) >> 1) & 1, tmo);
        }
        if (ok) {
          const ST* ub = uring + su * C::PSLOT;
          if constexpr (C::X0Q) {
            int suR = su + R;
            suR -= suR >= C::NU ? C::NU : 0;
            qq[0][(i + 2 * R) % Q] = ldv<NPR>(uring + suR * C::PSLOT + own);
          }
          // ---- fused step 0
          V un = fvzero<NPR>();
          if (act0) {
            const V uc = C::X0Q ? qq[0][(i + R) % Q] : ldv<NPR>(ub + own);
            const V up = ldv<NPR>(pring + sp * C::TILE + own_t);
            const V c2v = ldv<NPR>(cring + sc * C::TILE + own_t);
            const V lap = laplacian(ub, uc, [&](int d) -> V {
              if constexpr (C::X0Q) {
                return qq[0][(i + R + d) % Q];
              } else {
                int sf = su + d;
                sf -= sf >= C::NU ? C::NU : 0;
                sf += sf < 0 ? C::NU : 0;
                return ldv<NPR>(uring + sf * C::PSLOT + own);
              }
            });
            const float bx = __shfl_sync(0xffffffffu, bxc, 0);
            if constexpr (SK != 0) {  // stored values are u / s: scale back (exact, s a power of two)
              V ucs, ups, ls;
#pragma unroll
              for (int p = 0; p < NPR; ++p) {
                ucs.p[p] = __fmul2_rn(uc.p[p], sc2);
                ups.p[p] = __fmul2_rn(up.p[p], sp2);
                ls.p[p] = __fmul2_rn(lap.p[p], sc2);
              }
              un = update(ucs, ups, ls, c2v, bx, CW == 4 && yz_free && bx == 0.f);
            } else {
              un = update(uc, up, lap, c2v, bx, CW == 4 && yz_free && bx == 0.f);
            }
            if constexpr (T == 1) {
              if (any_src) inject(0, j, un);
            } else {
              if (any_src_w) inject(0, j, un);
            }
          }

          if constexpr (T == 1) {
            if (act0 && own_row && j >= pd.xo0 && j < pd.xo1 && vz) {
              if constexpr (SK != 0) {
                V sv;
#pragma unroll
                for (int p = 0; p < NPR; ++p) {
                  vmax = fmaxf(vmax, fmaxf(fabsf(un.p[p].x), fabsf(un.p[p].y)));
                  sv.p[p] = __fmul2_rn(un.p[p], io2);
                }
                stvcs<NPR>(reinterpret_cast<ST*>(out0) + (size_t)j * ps + coff, sv);
              } else {
                stvcs<NPR>(out0 + (size_t)j * ps + coff, un);
              }
            }
          } else {
            const float* rdbuf = splane + (size_t)(j & 1) * (T - 1) * C::PSLOT;
            float* wrbuf = splane + (size_t)((j + 1) & 1) * (T - 1) * C::PSLOT;
            bool act = act0;
#pragma unroll
            for (int k = 0; k < T; ++k) {
              const int q = j - k * R;
              if (k > 0) {
                act = q >= pd.xc0 && q < pd.xc1;
                un = fvzero<NPR>();
                if (act) {
                  const float* pl = rdbuf + (k - 1) * C::PSLOT;
                  // u_prev of step k: level n+k-1 at plane q
                  V upv;
                  if (k == 1 && !C::X0Q) {
                    int sq = su - R;
                    sq += sq < 0 ? C::NU : 0;
                    upv = ldv<NPR>(uring + sq * C::PSLOT + own);
                  } else {
                    upv = qq[QI(k - 1)][i % Q];
                  }
                  int scq = sc - k * R;
                  scq += scq < 0 ? C::NC : 0;
                  const V c2v = ldv<NPR>(cring + scq * C::TILE + own_t);
                  const V uc = qq[QI(k)][(i + R) % Q];
                  const V lap = laplacian(pl, uc, [&](int d) -> V { return qq[QI(k)][(i + R + d) % Q]; });
                  const float bx = __shfl_sync(0xffffffffu, bxc, k);
                  un = update(uc, upv, lap, c2v, bx, CW == 4 && yz_free && bx == 0.f);
                  if (any_src_w) inject(k, q, un);
                }
              }
              if (k + 1 < T) {
                // hand the new level to fused step k+1 ...
                qq[QI(k + 1)][(i + 2 * R) % Q] = un;
                // ... stage its centre for the next stream step ...
                const int qn = j + 1 - (k + 1) * R;
                st_pred_sh<NPR>(qn >= pd.xc0 && qn < pd.xc1, wrbuf + (size_t)k * C::PSLOT + own,
                                qq[QI(k + 1)][(i + R + 1) % Q]);
                // ... and publish its halo strips for the neighbours
                {
                  int qd = jd - (k * R) % C::D;
                  qd += qd < 0 ? C::D : 0;
                  float* rs = rs_base + ((size_t)k * C::D + qd) * C::STRIP;
                  st_pred_cg<NPR>(act && strip_y >= 0, rs + (strip_y >= 0 ? strip_y : 0), un);
                  st_pred_cg<NPR>(act && strip_z >= 0, rs + (strip_z >= 0 ? strip_z : 0), un);
                }
              } else {
                const bool st_out = act && own_row && q >= pd.xo0 && q < pd.xo1 && vz;
                const size_t qo = (size_t)(st_out ? q : 0) * ps + coff;
                st_pred_cs<NPR>(st_out, out0 + qo, un);
                st_pred_cs<NPR>(st_out, out1 + qo, qq[QI(T - 1)][(i + R) % Q]);
              }
            }
            mbar_arrive(bar_ctr + ((j + 1) & 1));
          }
          mbar_arrive(bar_done + (j - jstart) % C::NDONE);
          if constexpr (!C::UNROLL) {  // the queues move one plane down
#pragma unroll
            for (int k = 0; k < NQ; ++k)
#pragma unroll
              for (int s2 = 0; s2 < Q - 1; ++s2) qq[k][s2] = qq[k][s2 + 1];
          }
          // advance the ring slots
          su = su + 1 == C::NU ? 0 : su + 1;
          sp = sp + 1 == C::NP ? 0 : sp + 1;
          sc = sc + 1 == C::NC ? 0 : sc + 1;
          jd = jd + 1 == C::D ? 0 : jd + 1;
        }
      }
    }
  }
  if constexpr (SK != 0) {  // max |u^{n+1}| over the grid, for the next step's scale
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if (lane == 0 && vmax > 0.f) atomicMax(P.lp_mx + step0 + 2, __float_as_uint(vmax));
  }
  if (!ok) atomicExch(P.err, 2);
}

// two CTAs per SM for the one-step kernel where its register queue fits in
// half the register file (r <= 4), else one
template <int R, int T, int TY, int SK = 0, bool TWO = false, bool PRE = false>
__global__ void __launch_bounds__(SweepCfg<R, T, TY, SK>::NTHREADS, (T == 1 && R <= 4) ? 2 : 1)
    sweep_kernel(const __grid_constant__ SweepParams P) {
  const int b = blockIdx.x;
  int pi = 0;
  for (int i = 1; i < P.npass; ++i)
    if (P.pass[i].cta0 <= b) pi = i;
  const PassDesc pd = P.pass[pi];
  const bool s1 = TWO && b >= P.set1_cta0;
  sweep_body<R, T, TY, SK, TWO, PRE>(P, pd, b, s1, s1 ? P.set[1].step0 : P.set[0].step0);
}

// One time step of several shots in one launch (the one-step sweep): the
// launch's pass table concatenates the shots' passes, each naming its shot
// and the launch at which the shot started, and the CTAs of a pass run the
// sweep of that shot's step with the shot's parameters (fields, tensor
// maps, tables), read from device memory: L.shots[2 s + parity of the step].
template <int R>
__global__ void __launch_bounds__(SweepCfg<R, 1, 16, 0>::NTHREADS, R <= 4 ? 2 : 1)
    sweep_batch_kernel(const __grid_constant__ BatchParams L) {
  const int b = blockIdx.x;
  int lo = 0, hi = L.npass - 1;  // the last pass with cta0 <= b (sorted by cta0)
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.pass[mid].cta0 <= b) lo = mid;
    else hi = mid - 1;
  }
  const PassDesc pd = L.pass[lo];
  const int step = L.step - pd.step_off;
  sweep_body<R, 1, 16, 0, false, false>(L.shots[2 * pd.shot + (step & 1)], pd, b, false, step);
}

template <int R, int T, int SK = 0>
struct SweepTraits {
  static constexpr int TY = 16;
  using Cfg = SweepCfg<R, T, TY, SK>;
};

template <int R, int T, int SK, bool TWO, bool PRE>
cudaError_t sweep_launch_t(const SweepParams& p, int nctas, bool cooperative, cudaStream_t st) {
  using Tr = SweepTraits<R, T, SK>;
  using Cf = typename Tr::Cfg;
  auto fn = sweep_kernel<R, T, Tr::TY, SK, TWO, PRE>;
  // once per process (a function-local static: initialised once even when
  // several host threads launch at the same time)
  static const cudaError_t attr =
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cf::SMEM);
  if (attr != cudaSuccess) return attr;
  count_launch();
  if (cooperative) {
    void* args[] = {const_cast<SweepParams*>(&p)};
    return cudaLaunchCooperativeKernel((const void*)fn, dim3(nctas), dim3(Cf::NTHREADS), args, Cf::SMEM, st);
  }
  fn<<<nctas, Cf::NTHREADS, Cf::SMEM, st>>>(p);
  return cudaGetLastError();
}

template <int R>
cudaError_t sweep_batch_launch_t(const BatchParams& p, int nctas, cudaStream_t st) {
  using Cf = SweepCfg<R, 1, 16, 0>;
  auto fn = sweep_batch_kernel<R>;
  static const cudaError_t attr =
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cf::SMEM);
  if (attr != cudaSuccess) return attr;
  count_launch();
  fn<<<nctas, Cf::NTHREADS, Cf::SMEM, st>>>(p);
  return cudaGetLastError();
}

template <int R, int T, int SK, bool TWO, bool PRE>
cudaError_t sweep_occupancy_t(int* per_sm) {
  using Tr = SweepTraits<R, T, SK>;
  using Cf = typename Tr::Cfg;
  auto fn = sweep_kernel<R, T, Tr::TY, SK, TWO, PRE>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cf::SMEM);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, Cf::NTHREADS, Cf::SMEM);
}

template <int R, int T, int SK>
void sweep_shape_t(SweepShape* s) {
  using Tr = SweepTraits<R, T, SK>;
  using Cf = typename Tr::Cfg;
  s->R = R;
  s->T = T;
  s->TY = Tr::TY;
  s->threads = Cf::NTHREADS;
  s->smem = Cf::SMEM;
  s->ring_floats_per_cta = Cf::RING_PER_CTA;
  s->box_w = Cf::SW;
  s->box_h = Cf::SH;
  s->halo_w = Cf::RP;
}

// what: 0 launch, 1 occupancy query, 2 shape query; sk: storage kind (16-bit
// storage only in the one-step kernel)
template <int R, int T, int SK>
cudaError_t sweep_do(int what, const SweepParams* p, int nctas, bool coop, cudaStream_t st, int* per_sm,
                     SweepShape* s) {
  constexpr bool kTwo = T > 1 && SK == 0;  // passes of two time tiles exist
  // prefetched injections, where the registers allow (T - 1 axis-0 queues of
  // 2r + 1 pairs up to 18 pairs; r = 4, T = 4 spilled)
  constexpr bool kPre = kTwo && (T - 1) * (2 * R + 1) <= 18;
  if (what == 0) {
    const bool two = p->set1_cta0 < nctas, pre = p->src_prefetch != 0;
    if constexpr (kTwo) {
      if constexpr (kPre) {
        if (pre) return two ? sweep_launch_t<R, T, SK, true, true>(*p, nctas, coop, st)
                            : sweep_launch_t<R, T, SK, false, true>(*p, nctas, coop, st);
      }
      if (two) return sweep_launch_t<R, T, SK, true, false>(*p, nctas, coop, st);
    }
    (void)two;
    (void)pre;
    return sweep_launch_t<R, T, SK, false, false>(*p, nctas, coop, st);
  }
  if (what == 1) {
    cudaError_t e = sweep_occupancy_t<R, T, SK, false, false>(per_sm);
    int o = 0;
    if constexpr (kTwo) {
      if (e == cudaSuccess) e = sweep_occupancy_t<R, T, SK, true, false>(&o);
      if (e == cudaSuccess) *per_sm = *per_sm < o ? *per_sm : o;
    }
    if constexpr (kPre) {
      if (e == cudaSuccess) e = sweep_occupancy_t<R, T, SK, false, true>(&o);
      if (e == cudaSuccess) *per_sm = *per_sm < o ? *per_sm : o;
      if (e == cudaSuccess) e = sweep_occupancy_t<R, T, SK, true, true>(&o);
      if (e == cudaSuccess) *per_sm = *per_sm < o ? *per_sm : o;
    }
    return e;
  }
  sweep_shape_t<R, T, SK>(s);
  return cudaSuccess;
}
template <int R, int T>
cudaError_t sweep_do_sk(int what, int sk, const SweepParams* p, int nctas, bool coop, cudaStream_t st,
                        int* per_sm, SweepShape* s) {
  if constexpr (T == 1) {
    if (sk == 1) return sweep_do<R, 1, 1>(what, p, nctas, coop, st, per_sm, s);
    if (sk == 2) return sweep_do<R, 1, 2>(what, p, nctas, coop, st, per_sm, s);
  }
  if (sk != 0) return cudaErrorInvalidValue;
  return sweep_do<R, T, 0>(what, p, nctas, coop, st, per_sm, s);
}

// Per-radius entry points (one translation unit per radius), T = 1..TMAX.
#define TBI_DEFINE_RADIUS_T(RR, TT) \
  case TT:                          \
    return sweep_do_sk<RR, TT>(what, sk, p, nctas, coop, st, per_sm, s);

}  // namespace tbi
