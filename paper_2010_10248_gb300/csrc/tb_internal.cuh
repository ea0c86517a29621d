// Internal declarations of the CUDA path (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "tb.h"

namespace tbi {

// Counts kernel launches made by the library (tb_launch_count).
void count_launch(int n = 1);

// Progress counters of the blocked sweep sit one 128-byte line apart: with
// several counters per line, every publish and every neighbour poll of the
// CTAs sharing a line queued at the same L2 slice (packed counters measured
// 1.8 us from publish to observation, one line each 0.5 us).
constexpr int kProgressStride = 16;

// Blocked sweeps keep one tile of (TY x 64) columns per CTA; the pass table
// describes which CTAs stream which (x-chunk, y-band) of the grid.
struct PassDesc {
  int cta0;      // first CTA of the pass (blockIdx.x)
  int nty, ntz;  // tiles along axis 1 and axis 2
  int yb0;       // first row (axis 1) of the band's tile coverage
  int yo0, yo1;  // rows whose results this pass owns (written out)
  int xc0, xc1;  // planes (axis 0) the first fused step computes
  int xo0, xo1;  // planes whose results this pass owns
  int set;       // time tile of the pass: SweepParams::set[set] (set-1 passes
                 // follow the set-0 passes of a launch)
  int shot;      // batched launches: the pass's shot (BatchParams::shots)
  int step_off;  // batched launches: the launch at which the shot started
};

// The fields and first step of one time tile (T fused steps from step n).
struct SweepSet {
  CUtensorMap tm_u;             // u^n: (TY+2r) x (64+2rp) boxes with halo
  CUtensorMap tm_p;             // u^{n-1}: TY x 64 tiles
  const float* u_cur;           // u^n
  const float* u_prev;          // u^{n-1}
  float* out0;                  // u^{n+T}   (one-step: may alias u_prev)
  float* out1;                  // u^{n+T-1} (T > 1)
  int step0;                    // n
};

// Launch parameters of one sweep (one-step or T fused steps).  A launch may
// hold passes of two consecutive time tiles (set[0]: tile k, set[1]: tile
// k + 1) when bands of the blocked sweep are pipelined across time tiles.
struct SweepParams {
  SweepSet set[2];
  int set1_cta0;                // CTAs from this index on compute set[1]
                                // (INT_MAX: the launch holds set[0] only)
  CUtensorMap tm_c;             // c2: TY x 64 tiles
  int n0, n1, n2, n2p;          // grid, and row pitch of the padded fields
  const float* c2;              // dt^2 vp^2 (padded layout)
  const float* damp_b;          // [n0 + n1 + n2] eta_d / (2 dt) per axis
  float2 w2[3][6];              // c_i / h_d^2 (i = 1..r) as (w, w) pairs
  // grid-aligned sources (Sec. II-A) as event ranges per column pair: for the
  // columns (y, 2p) and (y, 2p + 1), ev_pair[y * npair + p] = (first plane |
  // span << 16, base), and src_ev[n][base + x - first plane] holds the pair's
  // injections at plane x in step n (zero for a column without a point there)
  const int2* ev_pair;          // [n1][npair]; NULL: no sources
  const float2* src_ev;         // [nt][nev]
  int64_t nev;
  int npair;
  int src_prefetch;             // blocked sweep: load a stream step's injections
                                // at its top (some pair spans many planes)
  // grid-aligned receivers
  const int* r_colptr;
  const int2* r_ent;
  float* rec_dcmp;              // [rec_cap][nrpts] ring: row = step mod rec_cap,
                                // column = position in r_ent
  int64_t nrpts;
  int rec_cap;                  // a power of two
  // blocked-sweep coupling between CTAs
  float* ring;                  // per tile, per stage, per slot: halo strips
  unsigned long long* progress; // per CTA: completed steps (monotonic), kProgressStride apart
  unsigned long long prog_base;
  int* err;                     // device error flag (1 = wait timed out)
  long long timeout_ns;
  const PassDesc* pass;         // device copy of the pass table
  int npass;
  // 16-bit storage (one-step kernel): scales[n] of u^{n-1} (stored = u / s),
  // running max |u| per step (float bits), the steps' largest injections
  // (may be null); the sweep of step n sets scales[n + 2] (lp_next_scale)
  float* lp_scales;
  unsigned* lp_mx;
  const float* lp_srcmax;
};

// Scale of u^{n+1} with 16-bit storage, s = 2^(ceil(log2(4 max|u^n| + max
// |src step n|)) - 8) (a power of two, exact to multiply by), from the
// running maximum mx[n + 1] of |u^n| and the step's largest injection.
// Every thread of the step's launch computes it (no separate launch); the
// same arithmetic everywhere, so every reader gets the same value.
__device__ __forceinline__ float lp_next_scale(const unsigned* mx, const float* srcmax, int n) {
  const float bound = 4.f * __uint_as_float(mx[n + 1]) + (srcmax ? srcmax[n] : 0.f);
  int e = 0;
  if (bound > 0.f) {
    frexpf(bound, &e);  // bound = f 2^e, f in [0.5, 1)
    e -= 8;
  }
  return ldexpf(1.f, max(min(e, 100), -100));
}

// A batched one-step launch over several shots: pass table (sorted by
// cta0), per shot two parameter sets (even and odd steps: u^n in field 0 or
// 1) in device memory, and the launch's index (a shot's step is step -
// pass.step_off).
struct BatchParams {
  const PassDesc* pass;
  int npass;
  const SweepParams* shots;
  int step;
};

struct SweepShape {
  int R, T, TY;
  int threads;
  size_t smem;
  int ring_floats_per_cta;      // floats of ring storage per CTA
  int box_w, box_h;             // u^n box (axis 2, axis 1) incl. halo
  int halo_w;                   // axis-2 halo width of the box
};

// Kernel configuration and launch (tb_acoustic*.cu).
// sk: wavefield storage of the sweep (0 FP32; 1 FP16, 2 BF16 with per-step
// power-of-two scales, one-step kernel only)
bool sweep_shape(int R, int T, SweepShape* s, int sk = 0);
cudaError_t sweep_max_ctas(int R, int T, int* per_sm, int sk = 0);
cudaError_t sweep_launch(int R, int T, const SweepParams& p, int nctas, bool cooperative,
                         cudaStream_t st, int sk = 0);
cudaError_t sweep_batch_launch(int R, const BatchParams& p, int nctas, cudaStream_t st);

// Inspector and setup kernels (tb_inspector.cu).
struct PointTables {
  int npt = 0;                  // off-grid points given
  int64_t npts = 0;             // unique affected grid points
  int64_t nvalid = 0;           // corner entries with weight != 0
  int64_t* lin = nullptr;       // [npts] ascending unpadded linear index
  int* colptr = nullptr;        // [n1*n2 + 1]
  int2* ent = nullptr;          // [npts] (x, id) by column then x
  int* eid_of_id = nullptr;     // [npts] position of each point in ent
  int* corner_id = nullptr;     // [npt*8] point id of each corner, -1 if weight 0 (receivers)
  int* corner_eid = nullptr;    // [npt*8] position in ent of each corner (receivers)
  float* corner_w = nullptr;    // [npt*8] (receivers)
  // inspector scratch kept for the decomposition
  unsigned long long* keys = nullptr;  // sorted corner keys [P]
  double* w8 = nullptr;         // [npt*8] corner weights
  int64_t* gstart = nullptr;    // [npts + 1] first sorted entry of each point
  int* ent_id = nullptr;        // [P] point id of each sorted entry
  size_t bytes = 0;
};

// Grid of a padded field and first-derivative weights (per axis, offsets
// 1..r, divided by the spacing) for the TTI and elastic kernels (tb_physics.cu).
struct PhysGrid {
  int n0, n1, n2, n2p;
};
struct DerivW {
  float a[3][6];
};
cudaError_t tti_step(int R, const PhysGrid& g, const DerivW& w, int nchunks, const float* pc, float* pp,
                     const float* rc, float* rp, const float* c2, const float* coef, const float* nz,
                     const float* damp_b, float* flux, cudaStream_t st);
cudaError_t tti_coefficients(const PhysGrid& g, const float* aux, float* coef, float* nz, unsigned* d_emax,
                             int* d_bad, cudaStream_t st);
cudaError_t elastic_step(int R, const PhysGrid& g, const DerivW& w, float dt, int nchunks, float* f, const float* mat,
                         const float* eta_dt, cudaStream_t st);
// Wavefront schedule of the TTI / elastic sub-updates (tb_physics.cu): the
// (sub-update, slab) items of one launch, and the injection / sampling of the
// steps whose last sub-update finished a slab in it.
constexpr int kWaveItemsMax = 32;  // 2 x the deepest time tile (16)
constexpr int kWavePostsMax = 16;
struct WaveItem {
  int kind;   // 0: TTI flux / elastic velocity; 1: TTI update / elastic stress
  int x0, x1;  // planes of the slab
  const float* a;  // TTI: p^n (kind 0 and 1)
  float* b;        // TTI: p^{n-1}, overwritten by p^{n+1} (kind 1)
  const float* c;  // TTI: r^n
  float* d;        // TTI: r^{n-1}, overwritten by r^{n+1}
  int ia, ib, ic, id;  // TTI: the field buffers (0..3) of a, b, c, d, for their tensor maps
};
struct WaveItems {
  int n;
  WaveItem it[kWaveItemsMax];
};
struct WavePost {
  int x0, x1;
  const float* dcmp;    // the step's injection table row (unused without sources)
  float *f0, *f1, *f2;  // injected fields (TTI: p, r; elastic: txx, tyy, tzz)
  float* row;           // the step's receiver row (unused without receivers)
  const float *s0, *s1, *s2;  // sampled: s0 (TTI: p), or the mean of s0..s2 (elastic)
};
struct WavePosts {
  int n;
  WavePost it[kWavePostsMax];
};
cudaError_t wave_launch(int physics, int R, const PhysGrid& g, const DerivW& w, float dt, const WaveItems& L,
                        const float* c2, const float* coef, const float* nz, const float* damp_b, float* flux,
                        float* ef, const float* mat, const float* eta_dt, cudaStream_t st);
cudaError_t wave_post(const PhysGrid& g, const WavePosts& P, int64_t nsrc_pts, const int64_t* src_lin,
                      int64_t nrec_pts, const int2* rec_ent, const int64_t* rec_lin, cudaStream_t st);
// One TTI step with both passes fused on chip (no flux fields in memory):
// chunks along axis 0 (L null), or the items of one wavefront launch.
cudaError_t tti_fused(int R, const PhysGrid& g, const DerivW& w, int nchunks, const WaveItems* L, const float* pc,
                      float* pp, const float* rc, float* rp, const float* c2, const float* coef, const float* nz,
                      const float* damp_b, cudaStream_t st);
// Elastic velocity (kind 0) / stress (kind 1) update with TMA-staged
// operands (tb_physics.cu): kEY x kEZ tiles, chunks along axis 0 (L null)
// or the items of one wavefront launch.  A stalled copy sets *err after
// `tmo` ns.
constexpr int kEY = 8, kEZ = 32;
struct ElaMaps {
  CUtensorMap fh;  // the nine fields [9][n0][n1][n2p], (kEZ + 2 rz) x (kEY + 2r) boxes, rz = r rounded up to 4
  CUtensorMap fo;  // the nine fields, kEZ x kEY boxes
  CUtensorMap mo;  // the eight material fields, kEZ x kEY boxes
};
cudaError_t elastic_tma(int R, const PhysGrid& g, const DerivW& w, float dt, const ElaMaps& M, int kind,
                        int nchunks, const WaveItems* L, float* f, const float* eta_dt, long long tmo, int* err,
                        cudaStream_t st);
// TTI flux (kind 0) / update (kind 1) passes with TMA-staged operands, same
// tiles; one-step (L null: the buffers of WaveItem `one` over nchunks chunks)
// or the items of one wavefront launch.
struct TtiMaps {
  CUtensorMap bh[4];  // the four p, r buffers, (kEZ + 2 rz) x (kEY + 2r) boxes
  CUtensorMap bo[4];  // the four p, r buffers, kEZ x kEY boxes
  CUtensorMap fh;     // fluxes [6][n0][n1][n2p], halo boxes
  CUtensorMap fo;     // fluxes, own boxes
  CUtensorMap nzo;    // frame [3][..], own boxes
  CUtensorMap co;     // c2, own boxes
  CUtensorMap ko;     // coef [2][..], own boxes
};
cudaError_t tti_tma(int R, const PhysGrid& g, const DerivW& w, const TtiMaps& M, int nchunks, const WaveItem* one,
                    const WaveItems* L, float* flux, const float* damp_b, long long tmo, int* err, cudaStream_t st);
// items (launch, sub-update, x0, x1) of the wavefront over n0 planes in slabs
// of `slab` planes for U sub-updates, launches in order; -1 on bad arguments
int wave_plan(int n0, int slab, int U, std::vector<int>* items);
cudaError_t elastic_material(const PhysGrid& g, const float* vp, const float* vs, const float* rho, float* mat,
                             int* d_bad, cudaStream_t st);
cudaError_t inject_points(const PhysGrid& g, int64_t npts, const int64_t* lin, const float* dcmp_row, float* f0,
                          float* f1, float* f2, cudaStream_t st);
cudaError_t sample_points(const PhysGrid& g, int64_t npts, const int2* ent, const int64_t* lin, const float* f0,
                          const float* f1, const float* f2, float* row, cudaStream_t st);

// Adjoint of the acoustic one-step recurrence and the vp gradient (tb_adjoint.cu).
// The adjoint runs on mu = D lam (D = c2/(1+g)) with the forward sweep kernel.
struct LapW {
  float c[3][6];  // c_i / h_d^2, i = 1..r
};
// rows[t][id] *= D at the receiver point id (the residual injected into mu)
cudaError_t adjoint_scale_rows(const PhysGrid& g, int nt, int64_t npts, const int64_t* lin, const float* c2,
                               const float* damp_b, float* rows, cudaStream_t st);
// imaging term of step k from mu^k and u^k, u^{k-1}, u^{k-2} (pointwise), and
// its source-point part
cudaError_t adjoint_grad(const PhysGrid& g, double dt, const float* mu, const float* u0, const float* u1,
                         const float* u2, double* gm, cudaStream_t st);
cudaError_t adjoint_grad_src(const PhysGrid& g, int64_t npts, const int64_t* lin, const float* dcmp_row, double dt,
                             const float* mu, const float* c2, const float* damp_b, double* gm, cudaStream_t st);
cudaError_t adjoint_sample_src(const PhysGrid& g, int64_t npts, const int2* ent, const int64_t* lin,
                               const float* mu, const float* c2, const float* damp_b, float* row, cudaStream_t st);
cudaError_t adjoint_finish(const PhysGrid& g, double dt, const double* gm, const float* c2, float* out,
                           cudaStream_t st);
cudaError_t transpose_f32(int64_t rows, int64_t cols, const float* in, float* out, cudaStream_t st);

// Stream-ordered device memory (cudaMallocFromPoolAsync / cudaFreeAsync):
// creating, reconfiguring or destroying a handle never synchronises the whole
// device, so work of other handles on other streams keeps running meanwhile.
// The library's pool of the current device keeps up to 4 GiB of freed memory
// mapped (the default pool returns it at once, and remapping the staging
// buffer of a 512^3 model cost every shot), NULL if it cannot be made.
cudaMemPool_t library_pool();
template <class T>
inline cudaError_t dmalloc(T** p, size_t bytes, cudaStream_t st) {
  cudaMemPool_t pool = library_pool();
  if (pool) return cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), bytes ? bytes : 1, pool, st);
  return cudaMallocAsync(reinterpret_cast<void**>(p), bytes ? bytes : 1, st);
}
inline void dfree(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

// 16-bit (or plain FP32) storage one-step path (tb_lowprec.cu); storage: 1 FP16,
// 2 BF16, 3 FP32.  scales[k] / mx[k]: scale and max |u| of u^{k-1}.
// HBM copy bandwidth (GB/s, read + write bytes of a 2 x 1 GiB float4 copy,
// best of 5) and packed-FP32 FMA throughput (TFLOP/s), with this build's
// kernels (tb_selftest.cu).  Synchronises st.
cudaError_t measure_peaks(double* hbm_gbs, double* fp32_tflops, cudaStream_t st);
// one step; the step's kernel also sets scales[n + 2] (lp_next_scale)
cudaError_t lowprec_step(int storage, int R, const PhysGrid& g, const LapW& w, int nchunks, const void* uc, void* up,
                         const float* c2, const float* damp_b, float* scales, const float* srcmax, int n,
                         unsigned* mx, cudaStream_t st);
cudaError_t lowprec_inject(int storage, const PhysGrid& g, int64_t npts, const int64_t* lin, const float* dcmp_row,
                           void* u, const float* scales, int n, unsigned* mx, cudaStream_t st);
cudaError_t lowprec_sample(int storage, const PhysGrid& g, int64_t npts, const int2* ent, const int64_t* lin,
                           const void* u, const float* scales, int n, float* row, cudaStream_t st);
cudaError_t lowprec_srcmax(int64_t npts, int nt, const float* dcmp, float* out, cudaStream_t st);
cudaError_t lowprec_unpack(int storage, const PhysGrid& g, const void* u, float s, float* out, cudaStream_t st);

void free_tables(PointTables* t, cudaStream_t st);
// Builds lin, colptr, ent (+ corner tables when want_corners).  coords on
// the device.  Returns TB_OK / TB_EINVAL / TB_ENOMEM / TB_ECUDA.
int inspect(const int64_t n[3], const double h[3], int npt, const double* d_coords,
            bool want_corners, PointTables* t, cudaStream_t st, const char** why);
// src_dcmp[t][id] = s(p_id) * sum_e w_e q_{s(e)}[t]  (FP64 sum, FP32 out) with
// s = c2(p_id) = dt^2/m, or the constant `scale` when c2 is NULL
cudaError_t decompose(const PointTables* t, int nt, const float* d_wav, const float* c2, double scale,
                      int n1, int n2, int n2p, float* d_dcmp, cudaStream_t st);
// ev[t][slot[i]] = dcmp[t][i] for the sweep kernel's per-column-pair table
// (row length ev_row floats).
cudaError_t source_events(int nt, int64_t npts, const int* slot, const float* dcmp, float* ev, int64_t ev_row,
                          cudaStream_t st);
cudaError_t finalize_traces(int nsteps, int nrec, const int* corner_id, const float* corner_w,
                            const float* rec_dcmp, int64_t nrpts, float* traces,
                            cudaStream_t st);
cudaError_t model_vmax(const float* vp, int64_t N, float* d_out, int* d_bad, cudaStream_t st);
cudaError_t model_c2(const float* vp, int n0, int n1, int n2, int n2p, double dt2, float* c2,
                     cudaStream_t st);
cudaError_t pad_copy(const float* src, float* dst, int n0, int n1, int n2, int n2p,
                     cudaStream_t st);
cudaError_t unpad_copy(const float* src, float* dst, int n0, int n1, int n2, int n2p,
                       cudaStream_t st);
cudaError_t count_nonfinite(const float* a, int64_t n, int* d_count, cudaStream_t st);

// binomial checkpoint schedule of the adjoint gradient (tb_checkpoint.cu):
// ADVANCE computes X_to from X_from held at src into dst; REVERSE runs the
// adjoint step of forward step `from` with X_from held at src.  Locations:
// a slot 0 .. S-1, kCkptZero (the zero state X_0) or kCkptWork (the work
// pair).
enum { kCkptAdvance = 0, kCkptReverse = 1 };
enum { kCkptZero = -1, kCkptWork = -2 };
struct CkptAction {
  int kind, from, to, src, dst;
};
int plan_binomial(int nt, int S, std::vector<CkptAction>* out, int64_t* forward_steps);

}  // namespace tbi
