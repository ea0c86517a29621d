// C ABI of the propagator (see include/tb.h): handle, validation, host
// setup arithmetic (FD weights, CFL, sponge, Ricker), pass planning for the
// blocked sweep, and the time loop of tb_forward.
#include <algorithm>
#include <climits>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cudaTypedefs.h>

#include "tb_internal.cuh"

namespace tbi {
cudaError_t sweep_dispatch_r2(int what, int T, int sk, const SweepParams* p, int nctas, bool coop,
                              cudaStream_t st, int* per_sm, SweepShape* s);
cudaError_t sweep_dispatch_r4(int what, int T, int sk, const SweepParams* p, int nctas, bool coop,
                              cudaStream_t st, int* per_sm, SweepShape* s);
cudaError_t sweep_dispatch_r6(int what, int T, int sk, const SweepParams* p, int nctas, bool coop,
                              cudaStream_t st, int* per_sm, SweepShape* s);

cudaError_t sweep_batch_dispatch_r2(const BatchParams* p, int nctas, cudaStream_t st);
cudaError_t sweep_batch_dispatch_r4(const BatchParams* p, int nctas, cudaStream_t st);
cudaError_t sweep_batch_dispatch_r6(const BatchParams* p, int nctas, cudaStream_t st);
cudaError_t sweep_batch_launch(int R, const BatchParams& p, int nctas, cudaStream_t st) {
  switch (R) {
    case 2: return sweep_batch_dispatch_r2(&p, nctas, st);
    case 4: return sweep_batch_dispatch_r4(&p, nctas, st);
    case 6: return sweep_batch_dispatch_r6(&p, nctas, st);
  }
  return cudaErrorInvalidValue;
}

static cudaError_t sweep_dispatch(int R, int what, int T, int sk, const SweepParams* p, int nctas, bool coop,
                                  cudaStream_t st, int* per_sm, SweepShape* s) {
  switch (R) {
    case 2: return sweep_dispatch_r2(what, T, sk, p, nctas, coop, st, per_sm, s);
    case 4: return sweep_dispatch_r4(what, T, sk, p, nctas, coop, st, per_sm, s);
    case 6: return sweep_dispatch_r6(what, T, sk, p, nctas, coop, st, per_sm, s);
  }
  return cudaErrorInvalidValue;
}
bool sweep_shape(int R, int T, SweepShape* s, int sk) {
  return sweep_dispatch(R, 2, T, sk, nullptr, 0, false, nullptr, nullptr, s) == cudaSuccess;
}
cudaError_t sweep_max_ctas(int R, int T, int* per_sm, int sk) {
  return sweep_dispatch(R, 1, T, sk, nullptr, 0, false, nullptr, per_sm, nullptr);
}
cudaError_t sweep_launch(int R, int T, const SweepParams& p, int nctas, bool cooperative,
                         cudaStream_t st, int sk) {
  return sweep_dispatch(R, 0, T, sk, &p, nctas, cooperative, st, nullptr, nullptr);
}
}  // namespace tbi

namespace tbi {
cudaMemPool_t library_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = 4ull << 30;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}

static unsigned long long g_launches = 0;
void count_launch(int n) { __atomic_fetch_add(&g_launches, (unsigned long long)n, __ATOMIC_RELAXED); }
}  // namespace tbi

using namespace tbi;

extern "C" uint64_t tb_launch_count(void) { return __atomic_load_n(&tbi::g_launches, __ATOMIC_RELAXED); }

struct tb_handle {
  int64_t n[3] = {0, 0, 0};
  int n2p = 0;
  double h[3] = {0, 0, 0};
  int so = 0, R = 0;
  tb_options opt{};
  int device = 0, num_sms = 0;
  double c[8] = {0};     // centred 2nd-derivative weights
  double dt = 0.0, vmax = 0.0;
  bool have_model = false;
  float* field[4] = {nullptr, nullptr, nullptr, nullptr};
  float* c2 = nullptr;
  CUtensorMap tm_box[4];   // u^n boxes with halo, per field buffer
  CUtensorMap tm_tile[4];  // own tiles, per field buffer
  CUtensorMap tm_c2;       // own tiles of c2
  ElaMaps ela_maps;        // elastic fields and material for the TMA-staged updates
  TtiMaps tti_maps;        // TTI fields, fluxes and coefficients for the TMA-staged passes
  float* damp_b = nullptr;
  // other physics (Sec. III-B/C): physics id, TTI coefficients [2][Np]
  // (1+2eps, sqrt(1+2delta)), symmetry axis [3][Np], fluxes [6][Np];
  // elastic fields [9][Np], material [8][Np] and per-axis eta*dt
  int physics = TB_ACOUSTIC;
  float* coef = nullptr;
  float* nzb = nullptr;
  float* flux = nullptr;
  float* efield = nullptr;
  float* emat = nullptr;
  float* eta_dt = nullptr;
  double aux_max = 0.0;  // eps_max (TTI)
  // 16-bit / plain storage (acoustic): two stored fields (u^n, u^{n-1}; the
  // update writes u^{n+1} over u^{n-1}), per-step scales and maxima, per-step
  // largest source increment
  int storage = TB_F32;
  int sk = 0;  // storage kind of the sweep kernel: 0 FP32, 1 FP16, 2 BF16 (one-step)
  void* lp[2] = {nullptr, nullptr};
  int lp_cur = 0;
  float* lp_scales = nullptr;
  unsigned* lp_mx = nullptr;
  int lp_cap = 0;
  float* lp_srcmax = nullptr;
  // sources
  PointTables src;
  int src_nt = 0;
  float* src_dcmp = nullptr;
  // the sweep kernel's view of the sources: one plane range per column pair
  int2* ev_pair = nullptr;      // [n1][npair] (first plane | span << 16, base)
  float2* src_ev = nullptr;     // [src_nt][nev]
  int64_t nev = 0;
  int npair = 0;
  int ev_max_span = 0;          // longest plane range of a column pair
  bool have_src = false;
  // receivers
  PointTables rec;
  bool have_rec = false;
  float* rec_dcmp = nullptr;
  int rec_cap = 0;
  // blocked-sweep scratch
  float* ring = nullptr;
  size_t ring_floats = 0;
  unsigned long long* progress = nullptr;
  int progress_n = 0;
  unsigned long long prog_base = 0;
  int* err = nullptr;      // [4]: wait timeout flag, nonfinite counter, ...
  PassDesc* d_pass = nullptr;
  int pass_cap = 0;
  float* traces_dev = nullptr;
  size_t traces_cap = 0;
  // result of the last forward
  int last_nt = -1;
  int64_t last_fwd_steps = -1;  // forward steps of the last adjoint gradient
  size_t last_scratch = 0;      // device bytes it allocated
  int cur_idx = 0, prev_idx = 1;
  // profiling
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kind;
  int ev_used = 0;
  cudaStream_t ev_stream = nullptr;
  cudaStream_t last_stream = nullptr;  // stream of the latest call (destroy frees on it)
  char msg[512] = {0};
};

static int fail(tb_handle* h, int code, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->msg, sizeof(h->msg), fmt, ap);
    va_end(ap);
  }
  return code;
}
static int cuda_fail(tb_handle* h, cudaError_t e, const char* where) {
  cudaGetLastError();
  return fail(h, e == cudaErrorMemoryAllocation ? TB_ENOMEM : TB_ECUDA, "%s: %s", where,
              cudaGetErrorString(e));
}
#define TB_CUDA(h, call)                                      \
  do {                                                        \
    cudaError_t e__ = (call);                                 \
    if (e__ != cudaSuccess) return cuda_fail((h), e__, #call); \
  } while (0)

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Host or device input -> device pointer (copy into *tmp when host).
static cudaError_t to_device(const void* src, size_t bytes, void** tmp, const void** out,
                             cudaStream_t st) {
  *tmp = nullptr;
  if (is_device_ptr(src)) {
    *out = src;
    return cudaSuccess;
  }
  cudaError_t e = dmalloc(tmp, bytes, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(*tmp, src, bytes, cudaMemcpyHostToDevice, st);
  *out = *tmp;
  return e;
}

// ---------------------------------------------------------------- setup --
extern "C" int tb_fd_weights(int so, double* c) {
  // closed form of the centred 2nd-derivative weights of order 2r:
  // c_i = 2 (-1)^(i+1) (r!)^2 / (i^2 (r-i)! (r+i)!),  c_0 = -2 sum_{i>=1} c_i
  if (so < 2 || so > 16 || so % 2 || !c) return TB_EINVAL;
  const int r = so / 2;
  auto fact = [](int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
  };
  double s = 0.0;
  for (int i = 1; i <= r; ++i) {
    const double v = 2.0 * (i % 2 ? 1.0 : -1.0) * fact(r) * fact(r) / ((double)i * i * fact(r - i) * fact(r + i));
    c[i] = v;
    s += v;
  }
  c[0] = -2.0 * s;
  return TB_OK;
}

extern "C" double tb_cfl_dt_max(int so, const double h[3], double vmax) {
  double c[9];
  if (!h || !(vmax > 0) || tb_fd_weights(so, c) != TB_OK) return -1.0;
  const int r = so / 2;
  double S = c[0];
  for (int i = 1; i <= r; ++i) S += 2.0 * (i % 2 ? -c[i] : c[i]);
  S = std::fabs(S);
  double inv = 0.0;
  for (int d = 0; d < 3; ++d) {
    if (!(h[d] > 0)) return -1.0;
    inv += 1.0 / (h[d] * h[d]);
  }
  return 2.0 / (vmax * std::sqrt(S * inv));
}

// Centred first-derivative weights a_1..a_r of order 2r (closed form):
// a_i = (-1)^(i+1) (r!)^2 / (i (r-i)! (r+i)!).
static void d1_weights(int r, double* a) {
  auto fact = [](int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
  };
  for (int i = 1; i <= r; ++i)
    a[i] = (i % 2 ? 1.0 : -1.0) * fact(r) * fact(r) / ((double)i * fact(r - i) * fact(r + i));
}
// Staggered first-derivative weights c_1..c_r (nodes at +-(k - 1/2)) from
// the moment conditions sum_k 2 c_k (k - 1/2)^(2m+1) = [m == 0], m < r,
// solved by Gaussian elimination with partial pivoting.
static void stag_weights(int r, double* c) {
  double A[8][9];
  for (int m = 0; m < r; ++m) {
    for (int k = 1; k <= r; ++k) A[m][k - 1] = 2.0 * std::pow(k - 0.5, 2 * m + 1);
    A[m][r] = m == 0 ? 1.0 : 0.0;
  }
  for (int col = 0; col < r; ++col) {
    int piv = col;
    for (int i = col + 1; i < r; ++i)
      if (std::fabs(A[i][col]) > std::fabs(A[piv][col])) piv = i;
    for (int j = 0; j <= r; ++j) std::swap(A[col][j], A[piv][j]);
    for (int i = 0; i < r; ++i) {
      if (i == col) continue;
      const double f = A[i][col] / A[col][col];
      for (int j = col; j <= r; ++j) A[i][j] -= f * A[col][j];
    }
  }
  for (int k = 1; k <= r; ++k) c[k] = A[k - 1][r] / A[k - 1][k - 1];
}
// max over t in [0, pi] of |2 sum_i w_i sin((i - shift) t)|: dense samples,
// then golden-section refinement around the best one
static double symbol_peak(const double* w, int r, double shift) {
  auto f = [&](double t) {
    double v = 0.0;
    for (int i = 1; i <= r; ++i) v += w[i] * std::sin((i - shift) * t);
    return std::fabs(2.0 * v);
  };
  const double pi = 3.14159265358979323846;
  const int ns = 4096;
  int best = 0;
  for (int s = 1; s <= ns; ++s)
    if (f(pi * s / ns) > f(pi * best / ns)) best = s;
  double lo = pi * std::max(0, best - 1) / ns, hi = pi * std::min(ns, best + 1) / ns;
  const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
  for (int it = 0; it < 100; ++it) {
    const double a = hi - gr * (hi - lo), b = lo + gr * (hi - lo);
    if (f(a) > f(b)) hi = b;
    else lo = a;
  }
  return std::max(f(0.5 * (lo + hi)), f(pi * best / ns));
}

extern "C" double tb_tti_dt_max(int so, const double h[3], double vmax, double eps_max) {
  if (!h || !(vmax > 0) || !(eps_max > -0.5) || so < 2 || so > 12 || so % 2) return -1.0;
  double a[8];
  d1_weights(so / 2, a);
  const double S1 = symbol_peak(a, so / 2, 0.0);
  double s2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    if (!(h[d] > 0)) return -1.0;
    s2 += (S1 / h[d]) * (S1 / h[d]);
  }
  return 2.0 / (vmax * std::sqrt((1.0 + 2.0 * std::max(eps_max, 0.0)) * s2));
}

extern "C" double tb_elastic_dt_max(int so, const double h[3], double vpmax) {
  if (!h || !(vpmax > 0) || so < 2 || so > 12 || so % 2) return -1.0;
  double c[8];
  stag_weights(so / 2, c);
  const double S = symbol_peak(c, so / 2, 0.5);
  double s2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    if (!(h[d] > 0)) return -1.0;
    s2 += (S / h[d]) * (S / h[d]);
  }
  return 2.0 / (vpmax * std::sqrt(s2));
}

extern "C" int tb_sponge_profile(int64_t n, int nbl, double h, double vmax, double* eta) {
  if (n < 1 || nbl < 0 || !eta || !(h > 0)) return TB_EINVAL;
  const double emax = nbl > 0 ? 3.0 * vmax * std::log(1000.0) / (2.0 * nbl * h) : 0.0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t d = 0;
    if (i < nbl) d = nbl - i;
    else if (i > n - 1 - nbl) d = i - (n - 1 - nbl);
    const double f = nbl > 0 ? (double)d / nbl : 0.0;
    eta[i] = emax * f * f;
  }
  return TB_OK;
}

extern "C" int tb_ricker(double f0, double dt, int nt, double t0, float* out) {
  if (!(f0 > 0) || nt < 0 || !out) return TB_EINVAL;
  if (t0 <= 0) t0 = 1.0 / f0;
  const double pi = 3.14159265358979323846;
  for (int n = 0; n < nt; ++n) {
    const double a = (pi * f0 * (n * dt - t0)) * (pi * f0 * (n * dt - t0));
    out[n] = (float)((1.0 - 2.0 * a) * std::exp(-a));
  }
  return TB_OK;
}

// --------------------------------------------------------------- handle --
extern "C" const char* tb_last_error(const tb_handle* h) { return h ? h->msg : "null handle"; }

extern "C" int tb_destroy(tb_handle* h) {
  if (!h) return TB_OK;
  // stream-ordered frees after the handle's latest work (no device-wide sync)
  cudaStream_t st = h->last_stream;
  for (auto& f : h->field) dfree(f, st);
  dfree(h->lp[0], st);
  dfree(h->lp[1], st);
  dfree(h->lp_scales, st);
  dfree(h->lp_mx, st);
  dfree(h->lp_srcmax, st);
  dfree(h->coef, st);
  dfree(h->nzb, st);
  dfree(h->flux, st);
  dfree(h->efield, st);
  dfree(h->emat, st);
  dfree(h->eta_dt, st);
  dfree(h->c2, st);
  dfree(h->damp_b, st);
  free_tables(&h->src, st);
  free_tables(&h->rec, st);
  dfree(h->src_dcmp, st);
  dfree(h->ev_pair, st);
  dfree(h->src_ev, st);
  dfree(h->rec_dcmp, st);
  dfree(h->ring, st);
  dfree(h->progress, st);
  dfree(h->err, st);
  dfree(h->d_pass, st);
  dfree(h->traces_dev, st);
  for (auto e : h->ev) cudaEventDestroy(e);
  delete h;
  return TB_OK;
}

// TMA descriptor of a padded field [n0][n1][n2p] (only n2 columns are in
// the tensor, so cells past n2 read as zeros) with a box of bw x bh x 1.
static cudaError_t make_tmap(CUtensorMap* m, void* base, const int64_t n[3], int n2p, int bw, int bh,
                             CUtensorMapDataType dtype = CU_TENSOR_MAP_DATA_TYPE_FLOAT32, int esz = 4) {
  // looked up once (a function-local static: safe with concurrent callers)
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                           cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess) return nullptr;
    return (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }();
  if (!encode) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)n[2], (cuuint64_t)n[1], (cuuint64_t)n[0]};
  const cuuint64_t strides[2] = {(cuuint64_t)n2p * esz, (cuuint64_t)n2p * esz * n[1]};
  const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(m, dtype, 3, base, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// [nf][n0][n1][n2p] floats as a 4-D tensor (axis 2 innermost), bw x bh boxes of one plane of one field
static cudaError_t make_tmap4(CUtensorMap* m, void* base, const int64_t n[3], int n2p, int nf, int bw, int bh) {
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                           cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess) return nullptr;
    return (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }();
  if (!encode) return cudaErrorNotSupported;
  const cuuint64_t dims[4] = {(cuuint64_t)n[2], (cuuint64_t)n[1], (cuuint64_t)n[0], (cuuint64_t)nf};
  const cuuint64_t row = (cuuint64_t)n2p * 4;
  const cuuint64_t strides[3] = {row, row * n[1], row * n[1] * n[0]};
  const cuuint32_t box[4] = {(cuuint32_t)bw, (cuuint32_t)bh, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

extern "C" int tb_create(const int64_t n[3], const double hsp[3], int so, int physics,
                         const tb_options* opt, tb_handle** out) {
  if (!out || !n || !hsp) return TB_EINVAL;
  *out = nullptr;
  if (physics != TB_ACOUSTIC && physics != TB_TTI && physics != TB_ELASTIC) return TB_EINVAL;
  if (so != 4 && so != 8 && so != 12) return TB_EINVAL;
  for (int d = 0; d < 3; ++d) {
    if (n[d] < so + 2 || n[d] > 65535 || !(hsp[d] > 0)) return TB_EINVAL;
  }
  if (n[0] * n[1] * n[2] >= (1ll << 40)) return TB_EINVAL;
  tb_handle* h = new tb_handle();
  for (int d = 0; d < 3; ++d) {
    h->n[d] = n[d];
    h->h[d] = hsp[d];
  }
  // allocations on this thread's default stream, complete before returning
  cudaStream_t st = cudaStreamPerThread;
  h->last_stream = st;
  h->so = so;
  h->R = so / 2;
  h->physics = physics;
  if (opt) h->opt = *opt;
  h->storage = h->opt.storage;
  if (h->storage < TB_F32 || h->storage > TB_F32_PLAIN || (h->storage != TB_F32 && physics != TB_ACOUSTIC)) {
    delete h;
    return TB_EINVAL;
  }
  // more fused so12 steps exceed shared memory; 16-bit and plain storage run
  // one step per launch; the TTI / elastic wavefront takes up to 8 steps
  const int tmax = physics != TB_ACOUSTIC ? 16 : (h->storage != TB_F32 ? 1 : (so == 12 ? 2 : 4));
  // default: the fused depth measured fastest at 512^3 (so8: T = 3 computes
  // each level faster than T = 4, whose three register queues crowd the
  // registers); TTI / elastic: 16 (at 384^3 so8 the deepest wavefront costs
  // least per step: fewer ramp launches per step)
  if (h->opt.time_tile == 0)
    h->opt.time_tile = physics != TB_ACOUSTIC ? 16 : ((tmax > 1 && so == 8) ? 3 : tmax);
  if (h->opt.time_tile < 1 || h->opt.time_tile > tmax || h->opt.nbl < 0 || h->opt.y_bands < 0 ||
      h->opt.x_chunks < 0 || h->opt.band_ctas < 0 || h->opt.slab_planes < 0 ||
      (h->opt.slab_planes > 0 &&
       h->opt.slab_planes < ((physics == TB_TTI && h->opt.tti_fused) ? so : so / 2))) {
    delete h;
    return TB_EINVAL;
  }
  if (h->opt.wait_timeout_s <= 0) h->opt.wait_timeout_s = 2.0;
  tb_fd_weights(so, h->c);
  // row pitch: 16-byte rows for TMA (8 values at 16 bits)
  h->sk = (h->storage == TB_F16) ? 1 : (h->storage == TB_BF16 ? 2 : 0);
  h->n2p = (int)(h->sk ? (n[2] + 7) / 8 * 8 : (n[2] + 3) / 4 * 4);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) {
    // keep freed blocks in the device's default pool for the next handle
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, h->device) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  const size_t fbytes = sizeof(float) * (size_t)n[0] * n[1] * h->n2p;
  const int nfield = (physics == TB_ELASTIC || h->storage != TB_F32) ? 0 : 4;
  if (h->storage != TB_F32) {
    const size_t es = h->storage == TB_F32_PLAIN ? 4 : 2;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
      e = dmalloc(&h->lp[i], es * (size_t)n[0] * n[1] * h->n2p, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(h->lp[i], 0, es * (size_t)n[0] * n[1] * h->n2p, st);
    }
  }
  for (int i = 0; i < nfield && e == cudaSuccess; ++i) {
    e = dmalloc(&h->field[i], fbytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->field[i], 0, fbytes, st);
  }
  if (physics == TB_TTI) {
    if (e == cudaSuccess) e = dmalloc(&h->coef, 2 * fbytes, st);
    if (e == cudaSuccess) e = dmalloc(&h->nzb, 3 * fbytes, st);
    if (e == cudaSuccess && !h->opt.tti_fused) e = dmalloc(&h->flux, 6 * fbytes, st);
    if (e == cudaSuccess && !h->opt.tti_fused) e = cudaMemsetAsync(h->flux, 0, 6 * fbytes, st);
  } else if (physics == TB_ELASTIC) {
    if (e == cudaSuccess) e = dmalloc(&h->efield, 9 * fbytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->efield, 0, 9 * fbytes, st);
    if (e == cudaSuccess) e = dmalloc(&h->emat, 8 * fbytes, st);
    if (e == cudaSuccess) e = dmalloc(&h->eta_dt, sizeof(float) * (n[0] + n[1] + n[2]), st);
    const int rz = (so / 2 + 3) / 4 * 4;
    if (e == cudaSuccess && !h->opt.stream_l1)
      e = make_tmap4(&h->ela_maps.fh, h->efield, n, h->n2p, 9, kEZ + 2 * rz, kEY + so);
    if (e == cudaSuccess && !h->opt.stream_l1) e = make_tmap4(&h->ela_maps.fo, h->efield, n, h->n2p, 9, kEZ, kEY);
    if (e == cudaSuccess && !h->opt.stream_l1) e = make_tmap4(&h->ela_maps.mo, h->emat, n, h->n2p, 8, kEZ, kEY);
  }
  if (e == cudaSuccess) e = dmalloc(&h->c2, fbytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->c2, 0, fbytes, st);
  if (physics == TB_TTI && !h->opt.tti_fused && !h->opt.stream_l1) {
    const int rz = (so / 2 + 3) / 4 * 4;
    TtiMaps& M = h->tti_maps;
    for (int i = 0; i < nfield && e == cudaSuccess; ++i) {
      e = make_tmap(&M.bh[i], h->field[i], n, h->n2p, kEZ + 2 * rz, kEY + so);
      if (e == cudaSuccess) e = make_tmap(&M.bo[i], h->field[i], n, h->n2p, kEZ, kEY);
    }
    if (e == cudaSuccess) e = make_tmap4(&M.fh, h->flux, n, h->n2p, 6, kEZ + 2 * rz, kEY + so);
    if (e == cudaSuccess) e = make_tmap4(&M.fo, h->flux, n, h->n2p, 6, kEZ, kEY);
    if (e == cudaSuccess) e = make_tmap4(&M.nzo, h->nzb, n, h->n2p, 3, kEZ, kEY);
    if (e == cudaSuccess) e = make_tmap(&M.co, h->c2, n, h->n2p, kEZ, kEY);
    if (e == cudaSuccess) e = make_tmap4(&M.ko, h->coef, n, h->n2p, 2, kEZ, kEY);
  }
  if (e == cudaSuccess) e = dmalloc(&h->damp_b, sizeof(float) * (n[0] + n[1] + n[2]), st);
  if (e == cudaSuccess) e = dmalloc(&h->err, sizeof(int) * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, sizeof(int) * 4, st);
  SweepShape sh;
  if (e == cudaSuccess && !sweep_shape(h->R, 1, &sh, h->sk)) e = cudaErrorInvalidValue;
  for (int i = 0; i < 4 && e == cudaSuccess && physics == TB_ACOUSTIC && h->storage == TB_F32; ++i) {
    e = make_tmap(&h->tm_box[i], h->field[i], n, h->n2p, sh.box_w, sh.box_h);
    if (e == cudaSuccess) e = make_tmap(&h->tm_tile[i], h->field[i], n, h->n2p, 64, sh.TY);
  }
  // 16-bit storage: the two stored fields, read by the one-step sweep
  const CUtensorMapDataType dt16 = h->sk == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  for (int i = 0; i < 2 && e == cudaSuccess && physics == TB_ACOUSTIC && h->sk; ++i) {
    e = make_tmap(&h->tm_box[i], h->lp[i], n, h->n2p, sh.box_w, sh.box_h, dt16, 2);
    if (e == cudaSuccess) e = make_tmap(&h->tm_tile[i], h->lp[i], n, h->n2p, 64, sh.TY, dt16, 2);
  }
  if (e == cudaSuccess && physics == TB_ACOUSTIC && (h->storage == TB_F32 || h->sk))
    e = make_tmap(&h->tm_c2, h->c2, n, h->n2p, 64, sh.TY);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    int code = e == cudaErrorMemoryAllocation ? TB_ENOMEM : TB_ECUDA;
    cudaGetLastError();
    tb_destroy(h);
    return code;
  }
  *out = h;
  return TB_OK;
}

extern "C" double tb_get_dt(const tb_handle* h) { return (h && h->have_model) ? h->dt : 0.0; }

extern "C" size_t tb_workspace_bytes(const tb_handle* h) {
  if (!h) return 0;
  const size_t fbytes = sizeof(float) * (size_t)h->n[0] * h->n[1] * h->n2p;
  // wavefields (four FP32 buffers, or two stored 16-bit / plain-FP32 ones) and c2
  // (fbytes / 4 is one value per padded point)
  const size_t wave = h->storage == TB_F32 ? 4 * fbytes : 2 * (h->storage == TB_F32_PLAIN ? 4 : 2) * (fbytes / 4);
  size_t b = wave + fbytes + sizeof(float) * (h->n[0] + h->n[1] + h->n[2]) + sizeof(int) * 4;
  if (h->storage != TB_F32) b += 2 * sizeof(float) * h->lp_cap;
  if (h->physics == TB_TTI) b += (h->opt.tti_fused ? 5 : 11) * fbytes;
  if (h->physics == TB_ELASTIC) b += 17 * fbytes - 4 * fbytes + sizeof(float) * (h->n[0] + h->n[1] + h->n[2]);
  b += h->src.bytes + h->rec.bytes;
  b += sizeof(float) * (size_t)h->src_nt * std::max<int64_t>(h->src.npts, 0);
  if (h->ev_pair) b += sizeof(int2) * (size_t)h->n[1] * h->npair + sizeof(float2) * (size_t)h->src_nt * h->nev;
  b += sizeof(float) * (size_t)h->rec_cap * std::max<int64_t>(h->rec.npts, 0);
  b += sizeof(float) * h->ring_floats + sizeof(unsigned long long) * kProgressStride * h->progress_n;
  b += sizeof(PassDesc) * h->pass_cap + sizeof(float) * h->traces_cap;
  return b;
}

extern "C" int tb_set_model(tb_handle* h, const float* vp, const float* aux, const float* damp,
                            double dt, void* stream) {
  if (!h) return TB_EINVAL;
  if (!vp) return fail(h, TB_EINVAL, "vp is NULL");
  if (h->physics == TB_ACOUSTIC && aux) return fail(h, TB_EINVAL, "aux must be NULL for acoustic physics");
  if (h->physics != TB_ACOUSTIC && !aux)
    return fail(h, TB_EINVAL, "aux is required (TTI: eps, delta, theta, phi; elastic: vs, rho)");
  if (dt < 0 || !std::isfinite(dt)) return fail(h, TB_EINVAL, "dt must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  const int64_t N = h->n[0] * h->n[1] * h->n[2];
  void* tmp = nullptr;
  const void* dvp = nullptr;
  TB_CUDA(h, to_device(vp, sizeof(float) * N, &tmp, &dvp, st));
  float* d_vmax = reinterpret_cast<float*>(h->err + 2);
  int* d_bad = h->err + 3;
  cudaError_t e = model_vmax((const float*)dvp, N, d_vmax, d_bad, st);
  float vmax = 0.f;
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&vmax, d_vmax, sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    dfree(tmp, st);
    return cuda_fail(h, e, "tb_set_model vmax");
  }
  if (bad) {
    dfree(tmp, st);
    return fail(h, TB_EINVAL, "vp must be finite and > 0 everywhere");
  }
  double dtmax = tb_cfl_dt_max(h->so, h->h, vmax);
  if (h->physics != TB_ACOUSTIC) {
    // per-point coefficients of the TTI / elastic operator from aux
    const int naux = h->physics == TB_TTI ? 4 : 2;
    void* tmpa = nullptr;
    const void* daux = nullptr;
    e = to_device(aux, sizeof(float) * N * naux, &tmpa, &daux, st);
    const PhysGrid g{(int)h->n[0], (int)h->n[1], (int)h->n[2], h->n2p};
    unsigned* d_emax = reinterpret_cast<unsigned*>(h->err + 2);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->err + 2, 0, sizeof(int) * 2, st);
    if (e == cudaSuccess) {
      if (h->physics == TB_TTI)
        e = tti_coefficients(g, (const float*)daux, h->coef, h->nzb, d_emax, d_bad, st);
      else
        e = elastic_material(g, (const float*)dvp, (const float*)daux, (const float*)daux + N, h->emat, d_bad,
                             st);
    }
    unsigned emax_bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&emax_bits, d_emax, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(tmpa, st);
    if (e != cudaSuccess) {
      dfree(tmp, st);
      return cuda_fail(h, e, "tb_set_model coefficients");
    }
    if (bad) {
      dfree(tmp, st);
      return fail(h, h->physics == TB_TTI ? TB_EUNSTABLE : TB_EINVAL,
                  h->physics == TB_TTI ? "TTI needs eps >= delta > -1/2 and finite angles everywhere"
                                       : "elastic needs rho > 0, vs >= 0 and 2 vs^2 <= vp^2 everywhere");
    }
    float emax = 0.f;
    memcpy(&emax, &emax_bits, sizeof(float));
    h->aux_max = h->physics == TB_TTI ? (double)emax : 0.0;
    dtmax = h->physics == TB_TTI ? tb_tti_dt_max(h->so, h->h, vmax, h->aux_max)
                                 : tb_elastic_dt_max(h->so, h->h, vmax);
  }
  if (dt == 0.0) dt = 0.8 * dtmax;
  if (dt > dtmax) {
    dfree(tmp, st);
    return fail(h, TB_EUNSTABLE, "dt = %g exceeds the CFL limit %g for vmax = %g", dt, dtmax, (double)vmax);
  }
  // damping: per-axis eta (1/s) -> b = eta / (2 dt)
  const int64_t nsum = h->n[0] + h->n[1] + h->n[2];
  std::vector<double> eta(nsum, 0.0);
  if (damp) {
    std::vector<float> hd(nsum);
    if (is_device_ptr(damp)) {
      e = cudaMemcpyAsync(hd.data(), damp, sizeof(float) * nsum, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        dfree(tmp, st);
        return cuda_fail(h, e, "tb_set_model damp");
      }
    } else {
      memcpy(hd.data(), damp, sizeof(float) * nsum);
    }
    for (int64_t i = 0; i < nsum; ++i) {
      if (!(hd[i] >= 0.f) || !std::isfinite(hd[i])) {
        dfree(tmp, st);
        return fail(h, TB_EINVAL, "damping coefficients must be finite and >= 0");
      }
      eta[i] = hd[i];
    }
  } else {
    int64_t off = 0;
    for (int d = 0; d < 3; ++d) {
      tb_sponge_profile(h->n[d], h->opt.nbl, h->h[d], vmax, eta.data() + off);
      off += h->n[d];
    }
  }
  std::vector<float> b(nsum), edt(nsum);
  for (int64_t i = 0; i < nsum; ++i) {
    b[i] = (float)(eta[i] / (2.0 * dt));
    edt[i] = (float)(eta[i] * dt);
  }
  e = cudaMemcpyAsync(h->damp_b, b.data(), sizeof(float) * nsum, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && h->physics == TB_ELASTIC)
    e = cudaMemcpyAsync(h->eta_dt, edt.data(), sizeof(float) * nsum, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = model_c2((const float*)dvp, (int)h->n[0], (int)h->n[1], (int)h->n[2], h->n2p, dt * dt, h->c2, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // b (host vector) must outlive the copy
  dfree(tmp, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "tb_set_model c2");
  (void)edt;
  h->dt = dt;
  h->vmax = vmax;
  h->have_model = true;
  h->have_src = false;  // the source table depends on dt and m
  h->last_nt = -1;
  h->msg[0] = 0;
  return TB_OK;
}

// The sweep kernel's source event layout (host only): the points of each
// column pair (y, 2p), (y, 2p + 1) share one range of planes [first, last];
// ev_pair[y * npair + p] = (first | span << 16, base) and the injection of the
// point at plane x of column 2p + c goes to slot 2 (base + x - first) + c of
// every step's row (nev = the sum of the spans).  Returns TB_EINVAL when a
// plane or span does not fit 16 bits or the rows exceed the int32 slot range.
static int event_layout(const int64_t* lin, int64_t np, int64_t n1, int64_t n2, std::vector<int2>& evp,
                        std::vector<int>& slot, int64_t* nev, int* max_span) {
  const int64_t npair = (n2 + 1) / 2;
  std::vector<int64_t> ord(np);
  for (int64_t i = 0; i < np; ++i) ord[i] = i;
  // points ordered by (row, pair, plane)
  auto key = [&](int64_t i) {
    const int64_t z = lin[i] % n2, y = (lin[i] / n2) % n1, x = lin[i] / (n1 * n2);
    return std::make_pair(y * npair + z / 2, x);
  };
  std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return key(a) < key(b); });
  evp.assign((size_t)(n1 * npair), make_int2(0, 0));
  slot.assign((size_t)np, 0);
  int64_t base = 0;
  int mspan = 0;
  for (int64_t g = 0; g < np;) {
    const int64_t pr = key(ord[g]).first;
    int64_t g1 = g;
    while (g1 < np && key(ord[g1]).first == pr) ++g1;
    const int64_t xf = key(ord[g]).second, xl = key(ord[g1 - 1]).second, span = xl - xf + 1;
    if (xf > 0xffff || span > 0xffff) return TB_EINVAL;
    evp[pr] = make_int2((int)(xf | (span << 16)), (int)base);
    mspan = std::max(mspan, (int)span);
    for (int64_t i = g; i < g1; ++i) slot[ord[i]] = (int)(2 * (base + key(ord[i]).second - xf) + (lin[ord[i]] % n2) % 2);
    base += span;
    if (2 * base >= (int64_t)INT32_MAX) return TB_EINVAL;
    g = g1;
  }
  *nev = base;
  *max_span = mspan;
  return TB_OK;
}

extern "C" int tb_source_event_layout(int64_t npts, const int64_t* lin, int64_t n1, int64_t n2, int* ev_pair,
                                      int* slot, int64_t* nev) {
  if (npts < 0 || n1 < 1 || n2 < 1 || (npts > 0 && (!lin || !slot)) || !ev_pair || !nev) return TB_EINVAL;
  for (int64_t i = 0; i < npts; ++i)
    if (lin[i] < 0) return TB_EINVAL;
  std::vector<int2> evp;
  std::vector<int> sl;
  int mspan = 0;
  const int s = event_layout(lin, npts, n1, n2, evp, sl, nev, &mspan);
  if (s != TB_OK) return s;
  for (size_t i = 0; i < evp.size(); ++i) {
    ev_pair[2 * i] = evp[i].x;
    ev_pair[2 * i + 1] = evp[i].y;
  }
  for (int64_t i = 0; i < npts; ++i) slot[i] = sl[(size_t)i];
  return TB_OK;
}

extern "C" int tb_set_sources(tb_handle* h, int nsrc, const double* coords, int nt,
                              const float* wav, void* stream) {
  if (!h) return TB_EINVAL;
  if (!h->have_model) return fail(h, TB_ESTATE, "tb_set_model must come before tb_set_sources");
  if (nsrc < 0 || (nsrc > 0 && (!coords || !wav || nt <= 0)))
    return fail(h, TB_EINVAL, "bad source arguments");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  void *t1 = nullptr, *t2 = nullptr;
  const void *dc = nullptr, *dw = nullptr;
  if (nsrc > 0) {
    TB_CUDA(h, to_device(coords, sizeof(double) * 3 * nsrc, &t1, &dc, st));
    cudaError_t e = to_device(wav, sizeof(float) * (size_t)nsrc * nt, &t2, &dw, st);
    if (e != cudaSuccess) {
      dfree(t1, st);
      return cuda_fail(h, e, "tb_set_sources wavelets");
    }
  }
  const char* why = "";
  h->have_src = false;
  // corner tables too: the adjoint gathers the source-wavelet gradient with them
  int s = inspect(h->n, h->h, nsrc, (const double*)dc, true, &h->src, st, &why);
  if (s != TB_OK) {
    dfree(t1, st);
    dfree(t2, st);
    return fail(h, s, "source inspector: %s", why);
  }
  dfree(h->src_dcmp, st);
  h->src_dcmp = nullptr;
  dfree(h->ev_pair, st);
  h->ev_pair = nullptr;
  dfree(h->src_ev, st);
  h->src_ev = nullptr;
  h->nev = 0;
  h->ev_max_span = 0;
  h->src_nt = nsrc > 0 ? nt : 0;
  cudaError_t e = cudaSuccess;
  int* d_slot = nullptr;
  if (h->src.npts > 0) {
    e = dmalloc(&h->src_dcmp, sizeof(float) * (size_t)nt * h->src.npts, st);
    if (e == cudaSuccess)
      // acoustic / TTI: dt^2/m at the point (Eq. 1's s dt^2/m); elastic:
      // explosive source into the normal stresses, dt q
      e = decompose(&h->src, nt, (const float*)dw, h->physics == TB_ELASTIC ? nullptr : h->c2, h->dt,
                    (int)h->n[1], (int)h->n[2], h->n2p, h->src_dcmp, st);
    if (e == cudaSuccess && h->physics == TB_ACOUSTIC) {
      // the sweep kernel's event table: the points of each column pair
      // (y, 2p), (y, 2p + 1) share one range of planes [first, last]; the
      // injection of the point at plane x of column 2p + c goes to slot
      // 2 (base + x - first) + c of every step's row
      const int64_t np = h->src.npts, n1 = h->n[1], n2 = h->n[2];
      h->npair = (int)((n2 + 1) / 2);
      std::vector<int64_t> lin(np);
      e = cudaMemcpyAsync(lin.data(), h->src.lin, sizeof(int64_t) * np, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      std::vector<int> slot(np);
      std::vector<int2> evp;
      if (e == cudaSuccess && event_layout(lin.data(), np, n1, n2, evp, slot, &h->nev, &h->ev_max_span) != TB_OK)
        e = cudaErrorInvalidValue;
      if (e == cudaSuccess) e = dmalloc(&h->ev_pair, sizeof(int2) * evp.size(), st);
      if (e == cudaSuccess) e = dmalloc(&h->src_ev, sizeof(float2) * (size_t)nt * h->nev, st);
      if (e == cudaSuccess) e = dmalloc(&d_slot, sizeof(int) * np, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->ev_pair, evp.data(), sizeof(int2) * evp.size(), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_slot, slot.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(h->src_ev, 0, sizeof(float2) * (size_t)nt * h->nev, st);
      if (e == cudaSuccess)
        e = source_events(nt, np, d_slot, h->src_dcmp, reinterpret_cast<float*>(h->src_ev), 2 * h->nev, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host tables copied before they go
    }
  }
  dfree(d_slot, st);
  if (e == cudaSuccess && h->storage != TB_F32 && h->src.npts > 0) {
    dfree(h->lp_srcmax, st);
    h->lp_srcmax = nullptr;
    e = dmalloc(&h->lp_srcmax, sizeof(float) * nt, st);
    if (e == cudaSuccess) e = lowprec_srcmax(h->src.npts, nt, h->src_dcmp, h->lp_srcmax, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dfree(t1, st);
  dfree(t2, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "tb_set_sources decomposition");
  h->have_src = true;
  h->last_nt = -1;
  h->msg[0] = 0;
  return TB_OK;
}

extern "C" int tb_set_receivers(tb_handle* h, int nrec, const double* coords, void* stream) {
  if (!h) return TB_EINVAL;
  if (nrec < 0 || (nrec > 0 && !coords)) return fail(h, TB_EINVAL, "bad receiver arguments");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  void* t1 = nullptr;
  const void* dc = nullptr;
  if (nrec > 0) TB_CUDA(h, to_device(coords, sizeof(double) * 3 * nrec, &t1, &dc, st));
  const char* why = "";
  h->have_rec = false;
  int s = inspect(h->n, h->h, nrec, (const double*)dc, true, &h->rec, st, &why);
  dfree(t1, st);
  if (s != TB_OK) return fail(h, s, "receiver inspector: %s", why);
  h->have_rec = true;
  h->last_nt = -1;
  h->msg[0] = 0;
  return TB_OK;
}

// ------------------------------------------------------------- planning --
struct Plan {
  std::vector<PassDesc> launch_passes;  // all passes, in launch order
  std::vector<int> launch_first;        // first pass index of each launch
  std::vector<int> launch_ctas;         // CTAs per launch
  std::vector<int> launch_tile;         // pipelined plans: time tile k of set 0
  int max_ctas = 0;
};

// Split the grid into (x-chunk, y-band) passes for a sweep of T fused
// steps.  A pass computes rows [yo0 - (T-1) r, yo1 + (T-1) r) and planes
// [xo0 - (T-1) r, xo1 + (T-1) r) (clipped to the grid) and owns
// [yo0, yo1) x [xo0, xo1).
static int plan_sweep(tb_handle* h, int T, Plan* pl) {
  const int R = h->R;
  SweepShape sh;
  const int sk = T == 1 ? h->sk : 0;
  if (!sweep_shape(R, T, &sh, sk)) return fail(h, TB_EINVAL, "unsupported time tile %d", T);
  int per_sm = 0;
  cudaError_t e = sweep_max_ctas(R, T, &per_sm, sk);
  if (e != cudaSuccess) return cuda_fail(h, e, "occupancy");
  if (per_sm < 1) return fail(h, TB_ECUDA, "sweep kernel does not fit on an SM");
  const int cap = per_sm * h->num_sms;
  const int n0 = (int)h->n[0], n1 = (int)h->n[1], n2 = (int)h->n[2];
  const int TY = sh.TY, TZ = 64;
  const int ntz = (n2 + TZ - 1) / TZ;
  const int halo = (T - 1) * R;
  int nbands = h->opt.y_bands;
  if (T == 1) nbands = std::max(1, nbands);
  if (nbands == 0) {
    for (nbands = 1; nbands <= n1; ++nbands) {
      const int rows = (n1 + nbands - 1) / nbands;
      const int in_rows = std::min(n1, rows + (nbands > 1 ? 2 * halo : 0));
      const int nty = (in_rows + TY - 1) / TY;
      if (nty * ntz <= cap) break;
    }
    if (nbands > n1) return fail(h, TB_EINVAL, "grid too wide for a co-resident blocked sweep");
  }
  int nchunks = h->opt.x_chunks;
  if (nchunks == 0) {
    if (T == 1) {
      // one-step: enough CTAs to fill the GPU a few times over
      const int nty = (n1 + TY - 1) / TY;
      nchunks = std::max(1, std::min(n0 / std::max(8, 2 * R), (4 * cap + nty * ntz - 1) / (nty * ntz)));
    } else {
      nchunks = 1;
    }
  }
  nchunks = std::min(nchunks, n0);
  nbands = std::min(nbands, n1);
  std::vector<PassDesc> passes;
  for (int c = 0; c < nchunks; ++c) {
    const int xo0 = (int)((int64_t)n0 * c / nchunks), xo1 = (int)((int64_t)n0 * (c + 1) / nchunks);
    for (int bnd = 0; bnd < nbands; ++bnd) {
      const int yo0 = (int)((int64_t)n1 * bnd / nbands), yo1 = (int)((int64_t)n1 * (bnd + 1) / nbands);
      PassDesc p{};
      p.yo0 = yo0;
      p.yo1 = yo1;
      p.xo0 = xo0;
      p.xo1 = xo1;
      p.yb0 = std::max(0, yo0 - halo);
      const int yb1 = std::min(n1, yo1 + halo);
      p.nty = (yb1 - p.yb0 + TY - 1) / TY;
      p.ntz = ntz;
      p.xc0 = std::max(0, xo0 - halo);
      p.xc1 = std::min(n0, xo1 + halo);
      passes.push_back(p);
    }
  }
  // group passes into launches: cooperative launches must fit co-resident
  pl->launch_passes.clear();
  pl->launch_first.clear();
  pl->launch_ctas.clear();
  int ctas = 0;
  for (size_t i = 0; i < passes.size(); ++i) {
    const int need = passes[i].nty * passes[i].ntz;
    if (T > 1 && need > cap) return fail(h, TB_EINVAL, "blocked pass of %d CTAs exceeds %d co-resident", need, cap);
    const bool new_launch = pl->launch_first.empty() || (T > 1 && ctas + need > cap);
    if (new_launch) {
      if (!pl->launch_first.empty()) pl->launch_ctas.push_back(ctas);
      pl->launch_first.push_back((int)i);
      ctas = 0;
    }
    passes[i].cta0 = ctas;
    ctas += need;
    pl->launch_passes.push_back(passes[i]);
  }
  pl->launch_ctas.push_back(ctas);
  pl->max_ctas = 0;
  for (int c : pl->launch_ctas) pl->max_ctas = std::max(pl->max_ctas, c);
  (void)sh;
  return TB_OK;
}

// Blocked sweep of K time tiles with the bands pipelined across time tiles.
// Each launch fills up to `cap` CTAs: first with the rows of time tile k not
// yet computed (a band of rows [y, y1), cut where the CTAs run out), then,
// once tile k reaches the last row, with the first rows [0, c) of tile k + 1.
// A pass owning rows [y0, y1) of tile k + 1 depends on rows
// [0, y1 + T r) of tile k (T steps of reach r each); those must have been
// owned by earlier launches, so c <= y - T r.  The same bound keeps tile
// k + 1's writes (into the fields tile k reads) below every row that tile
// k's band in the launch reads.  Rows a pass computes beyond what its owned
// rows depend on may read fields in flight; they are never written out.  A
// grid whose time tile fits one launch gets one launch per tile.
// The planner itself (host only): returns 0, or -1 when a launch of `cap`
// CTAs cannot hold a band of the grid.
static int pipeline_passes(int n0, int n1, int n2, int R, int T, int TY, int K, int cap, Plan* pl) {
  const int TZ = 64;
  const int ntz = (n2 + TZ - 1) / TZ;
  const int halo = (T - 1) * R, reach = T * R;
  const int tiles_cap = cap / ntz;  // tile rows per launch
  auto make = [&](int set, int y0, int y1) {
    PassDesc p{};
    p.yo0 = y0;
    p.yo1 = y1;
    p.xo0 = 0;
    p.xo1 = n0;
    p.yb0 = std::max(0, y0 - halo);
    p.nty = (std::min(n1, y1 + halo) - p.yb0 + TY - 1) / TY;
    p.ntz = ntz;
    p.xc0 = 0;
    p.xc1 = n0;
    p.set = set;
    return p;
  };
  // the last row y1 <= n1 a pass from row y0 can own within `tiles` tile rows
  auto last_row = [&](int y0, int tiles) {
    const int cover = std::max(0, y0 - halo) + tiles * TY;
    return cover >= n1 ? n1 : cover - halo;
  };
  pl->launch_passes.clear();
  pl->launch_first.clear();
  pl->launch_ctas.clear();
  pl->launch_tile.clear();
  pl->max_ctas = 0;
  int k = 0, y = 0;  // rows [0, y) of time tile k are done
  while (k < K) {
    const int y1 = last_row(y, tiles_cap);
    if (y1 <= y) return -1;
    pl->launch_first.push_back((int)pl->launch_passes.size());
    pl->launch_tile.push_back(k);
    PassDesc a = make(0, y, y1);
    a.cta0 = 0;
    int ctas = a.nty * ntz;
    pl->launch_passes.push_back(a);
    if (y1 < n1) {
      y = y1;
    } else {
      int c = 0;
      if (k + 1 < K && tiles_cap > a.nty) c = std::min(last_row(0, tiles_cap - a.nty), y - reach);
      if (c > 0) {
        PassDesc b = make(1, 0, c);
        b.cta0 = ctas;
        ctas += b.nty * ntz;
        pl->launch_passes.push_back(b);
      }
      ++k;
      y = std::max(c, 0);
    }
    pl->launch_ctas.push_back(ctas);
    pl->max_ctas = std::max(pl->max_ctas, ctas);
  }
  return 0;
}

static int plan_pipeline(tb_handle* h, int T, int K, Plan* pl) {
  SweepShape sh;
  if (!sweep_shape(h->R, T, &sh, 0)) return fail(h, TB_EINVAL, "unsupported time tile %d", T);
  int per_sm = 0;
  cudaError_t e = sweep_max_ctas(h->R, T, &per_sm, 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "occupancy");
  if (per_sm < 1) return fail(h, TB_ECUDA, "sweep kernel does not fit on an SM");
  int cap = per_sm * h->num_sms;
  if (h->opt.band_ctas > 0) cap = std::min(cap, h->opt.band_ctas);
  if (pipeline_passes((int)h->n[0], (int)h->n[1], (int)h->n[2], h->R, T, sh.TY, K, cap, pl) != 0)
    return fail(h, TB_EINVAL, "a blocked launch of %d CTAs cannot hold a band of this grid (%d tile columns)", cap,
                (int)((h->n[2] + 63) / 64));
  return TB_OK;
}

extern "C" int tb_plan_wavefront(int n0, int slab, int n_sub, int* items, int max_items) {
  std::vector<int> v;
  if (wave_plan(n0, slab, n_sub, &v) != 0) return -TB_EINVAL;
  const int n = (int)(v.size() / 4);
  if (items) {
    if (max_items < n) return -TB_EINVAL;
    std::copy(v.begin(), v.end(), items);
  }
  return n;
}

extern "C" int tb_plan_pipeline(int n1, int n2, int space_order, int time_tile, int n_tiles, int cap, int* passes,
                                int max_passes) {
  const int R = space_order / 2;
  if ((space_order != 4 && space_order != 8 && space_order != 12) || time_tile < 2 || n1 < 1 || n2 < 1 ||
      n_tiles < 0 || cap < 1 || max_passes < 0 || (max_passes > 0 && !passes))
    return -TB_EINVAL;
  SweepShape sh;
  if (!sweep_shape(R, time_tile, &sh, 0)) return -TB_EINVAL;
  Plan pl;
  if (pipeline_passes(1, n1, n2, R, time_tile, sh.TY, n_tiles, cap, &pl) != 0) return -TB_EINVAL;
  const int np = (int)pl.launch_passes.size();
  for (int L = 0, i = 0; L < (int)pl.launch_first.size(); ++L) {
    const int last = L + 1 < (int)pl.launch_first.size() ? pl.launch_first[L + 1] : np;
    for (; i < last; ++i) {
      if (i >= max_passes) continue;
      const PassDesc& d = pl.launch_passes[i];
      int* o = passes + 7 * (size_t)i;
      o[0] = L;
      o[1] = pl.launch_tile[L] + d.set;
      o[2] = d.yo0;
      o[3] = d.yo1;
      o[4] = d.yb0;
      o[5] = d.nty;
      o[6] = d.cta0;
    }
  }
  return np;
}

static int ensure_capacity(tb_handle* h, int T, const Plan& pl, int nt, bool host_traces, int nrec,
                           cudaStream_t st) {
  SweepShape sh;
  sweep_shape(h->R, T, &sh);
  if (T > 1) {
    const size_t need = (size_t)sh.ring_floats_per_cta * pl.max_ctas;
    if (need > h->ring_floats) {
      dfree(h->ring, st);
      h->ring = nullptr;
      h->ring_floats = 0;
      TB_CUDA(h, dmalloc(&h->ring, sizeof(float) * need, st));
      h->ring_floats = need;
    }
    if (pl.max_ctas > h->progress_n) {
      dfree(h->progress, st);
      h->progress = nullptr;
      h->progress_n = 0;
      TB_CUDA(h, dmalloc(&h->progress, sizeof(unsigned long long) * kProgressStride * pl.max_ctas, st));
      TB_CUDA(h, cudaMemsetAsync(h->progress, 0, sizeof(unsigned long long) * kProgressStride * pl.max_ctas, st));
      h->progress_n = pl.max_ctas;
      h->prog_base = 0;
    }
  }
  if ((int)pl.launch_passes.size() > h->pass_cap) {
    dfree(h->d_pass, st);
    h->d_pass = nullptr;
    h->pass_cap = 0;
    TB_CUDA(h, dmalloc(&h->d_pass, sizeof(PassDesc) * pl.launch_passes.size(), st));
    h->pass_cap = (int)pl.launch_passes.size();
  }
  if (h->have_rec && h->rec.npts > 0) {
    // ring rows, a power of two: two time tiles in flight, plus slack
    int cap = 16;
    while (cap < 3 * T) cap *= 2;
    if (cap > h->rec_cap) {
      dfree(h->rec_dcmp, st);
      h->rec_dcmp = nullptr;
      h->rec_cap = 0;
      TB_CUDA(h, dmalloc(&h->rec_dcmp, sizeof(float) * (size_t)cap * h->rec.npts, st));
      h->rec_cap = cap;
    }
  }
  if (host_traces && nrec > 0) {
    const size_t need = (size_t)nt * nrec;
    if (need > h->traces_cap) {
      dfree(h->traces_dev, st);
      h->traces_dev = nullptr;
      h->traces_cap = 0;
      TB_CUDA(h, dmalloc(&h->traces_dev, sizeof(float) * need, st));
      h->traces_cap = need;
    }
  }
  return TB_OK;
}

static void ev_reset(tb_handle* h, cudaStream_t st) {
  h->ev_used = 0;
  h->ev_kind.clear();
  h->ev_stream = st;
}
static cudaEvent_t ev_next(tb_handle* h) {
  if (h->ev_used >= (int)h->ev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->ev.push_back(e);
  }
  return h->ev[h->ev_used++];
}

// TTI / elastic: one step per launch (Sec. III-B/C), grid-aligned injection
// and receiver sampling as separate kernels after each step.
static size_t Np_of(const tb_handle* h) { return (size_t)h->n[0] * h->n[1] * h->n2p; }

// Scale buffers of the 16-bit storage for nt steps: scales[k] of u^{k-1}
// (the zero fields u^{-1}, u^0 get 1) and the running max |u^{k-1}| (zeros).
static int ensure_scales(tb_handle* h, int nt, cudaStream_t st) {
  if (nt + 3 > h->lp_cap) {
    dfree(h->lp_scales, st);
    dfree(h->lp_mx, st);
    h->lp_scales = nullptr;
    h->lp_mx = nullptr;
    h->lp_cap = 0;
    TB_CUDA(h, dmalloc(&h->lp_scales, sizeof(float) * (nt + 3), st));
    TB_CUDA(h, dmalloc(&h->lp_mx, sizeof(unsigned) * (nt + 3), st));
    h->lp_cap = nt + 3;
  }
  const float ones[2] = {1.0f, 1.0f};
  TB_CUDA(h, cudaMemcpyAsync(h->lp_scales, ones, sizeof(ones), cudaMemcpyHostToDevice, st));
  TB_CUDA(h, cudaMemsetAsync(h->lp_mx, 0, sizeof(unsigned) * (nt + 3), st));
  TB_CUDA(h, cudaStreamSynchronize(st));  // `ones` outlives the copy
  return TB_OK;
}

static int forward_other(tb_handle* h, int nt, float* traces, int schedule, cudaStream_t st) {
  const int nrec = h->have_rec ? h->rec.npt : 0;
  const bool rec_on = h->have_rec && h->rec.npts > 0 && nrec > 0 && traces;
  const bool host_traces = traces && nrec > 0 && !is_device_ptr(traces);
  const size_t fbytes = sizeof(float) * (size_t)h->n[0] * h->n[1] * h->n2p;
  if (rec_on && h->rec_cap < 16) {
    dfree(h->rec_dcmp, st);
    h->rec_dcmp = nullptr;
    h->rec_cap = 0;
    TB_CUDA(h, dmalloc(&h->rec_dcmp, sizeof(float) * 16 * h->rec.npts, st));
    h->rec_cap = 16;
  }
  if (host_traces && (size_t)nt * nrec > h->traces_cap) {
    dfree(h->traces_dev, st);
    h->traces_dev = nullptr;
    h->traces_cap = 0;
    TB_CUDA(h, dmalloc(&h->traces_dev, sizeof(float) * (size_t)nt * nrec, st));
    h->traces_cap = (size_t)nt * nrec;
  }
  float* dtr = host_traces ? h->traces_dev : traces;
  const PhysGrid g{(int)h->n[0], (int)h->n[1], (int)h->n[2], h->n2p};
  DerivW w{};
  double a[8];
  if (h->physics == TB_TTI) d1_weights(h->R, a);
  else stag_weights(h->R, a);
  for (int d = 0; d < 3; ++d)
    for (int i = 1; i <= h->R; ++i) w.a[d][i - 1] = (float)(a[i] / h->h[d]);
  if (h->opt.profile) ev_reset(h, st);
  const bool lowp = h->physics == TB_ACOUSTIC;  // acoustic here means 16-bit or plain storage
  const size_t es = h->storage == TB_F32_PLAIN ? 4 : 2;
  LapW lw{};
  if (lowp) {
    for (int d = 0; d < 3; ++d)
      for (int i = 1; i <= h->R; ++i) lw.c[d][i - 1] = (float)(h->c[i] / (h->h[d] * h->h[d]));
    int s = ensure_scales(h, nt, st);
    if (s != TB_OK) return s;
    TB_CUDA(h, cudaMemsetAsync(h->lp[0], 0, es * Np_of(h), st));
    TB_CUDA(h, cudaMemsetAsync(h->lp[1], 0, es * Np_of(h), st));
    h->lp_cur = 0;
  } else if (h->physics == TB_TTI) {
    for (int i = 0; i < 4; ++i) TB_CUDA(h, cudaMemsetAsync(h->field[i], 0, fbytes, st));
  } else {
    TB_CUDA(h, cudaMemsetAsync(h->efield, 0, 9 * fbytes, st));
  }
  // chunks of planes along axis 0 for the streaming kernels (all chunks of a
  // step in one launch): enough columns x chunks for about eight waves of
  // full SMs (measured best for TTI and elastic at 384^3 among 2, 8 and one
  // plane per chunk), chunks no shorter than 4r planes (each re-reads 2r
  // planes to warm up its queue)
  const int64_t cols = h->n[1] * h->n[2];
  const int nchunks = (int)std::max<int64_t>(1, std::min<int64_t>(h->n[0] / std::max(4, 4 * h->R),
                                                                   (int64_t)h->num_sms * 2048 * 8 / std::max<int64_t>(cols, 1)));
  int pc = 0, pp = 1, rc = 2, rp = 3;  // TTI field indices
  int fill = 0, base = 0;
  const size_t Np = (size_t)h->n[0] * h->n[1] * h->n2p;
  auto flush = [&]() -> int {
    if (rec_on && fill > 0) {
      cudaError_t e = finalize_traces(fill, nrec, h->rec.corner_eid, h->rec.corner_w, h->rec_dcmp, h->rec.npts,
                                      dtr + (size_t)base * nrec, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "receiver finalize");
    }
    base += fill;
    fill = 0;
    return TB_OK;
  };
  // TTI / elastic blocked: T steps per wavefront over slabs of axis 0 (the
  // nt mod T remaining steps one step per launch)
  const int T = (!lowp && schedule == TB_BLOCKED) ? h->opt.time_tile : 1;
  // 32-plane slabs: measured fastest at 384^3 among 4 .. 64 (thin slabs
  // re-read 2r planes per slab to fill their register queues)
  const int slab = h->opt.slab_planes > 0 ? h->opt.slab_planes : 32;
  const bool src_on = h->have_src && h->src.npts > 0;
  // TTI with tti_fused: both passes of a step in one kernel (a step is one
  // sub-update of reach 2r)
  const bool fused = h->physics == TB_TTI && h->opt.tti_fused;
  const int per_step = fused ? 1 : 2;
  std::vector<int> plan;
  if (T > 1 && wave_plan((int)h->n[0], slab, per_step * T, &plan) != 0) return fail(h, TB_EINVAL, "bad wavefront");
  // fused TTI: chunks along axis 0 for about four CTAs per SM in all (one
  // CTA per SM fits), no chunk shorter than 8r planes (each computes the
  // fluxes of 2r planes beyond it)
  // elastic: the TMA-staged updates (chunks for about twelve CTAs per SM
  // in all, three fit at once; chunks no shorter than 4r planes), unless the
  // L1 streaming kernels are asked for
  const bool ela_tma = h->physics == TB_ELASTIC && !h->opt.stream_l1;
  const bool tti_tma_on = h->physics == TB_TTI && !h->opt.stream_l1 && !h->opt.tti_fused;
  const long long tmo = (long long)(h->opt.wait_timeout_s * 1e9);
  const int64_t etiles = ((h->n[2] + kEZ - 1) / kEZ) * ((h->n[1] + kEY - 1) / kEY);
  const int echunks = (int)std::max<int64_t>(
      1, std::min<int64_t>(h->n[0] / (4 * h->R), (12 * (int64_t)h->num_sms + etiles - 1) / etiles));
  if (ela_tma || tti_tma_on) TB_CUDA(h, cudaMemsetAsync(h->err, 0, sizeof(int), st));
  const int64_t ftiles = ((h->n[2] + 31) / 32) * ((h->n[1] + 7) / 8);
  const int fchunks = (int)std::max<int64_t>(
      1, std::min<int64_t>(h->n[0] / (8 * h->R), (4 * (int64_t)h->num_sms + ftiles - 1) / ftiles));
  for (int n = 0; n < nt;) {
    if (T > 1 && nt - n >= T) {
      if (rec_on && fill + T > h->rec_cap) {
        int s = flush();
        if (s != TB_OK) return s;
      }
      // level k of the block: TTI fields p^{n+k} and p^{n+k-1} (their roles
      // alternate with k), elastic fields in place
      int pcur[2] = {pc, pp}, rcur[2] = {rc, rp};
      WaveItems L{};
      WavePosts P{};
      for (size_t i = 0; i < plan.size(); i += 4) {
        const int u = plan[i + 1], k = u / per_step;
        WaveItem& it = L.it[L.n++];
        it.kind = fused ? 1 : (u & 1);
        it.x0 = plan[i + 2];
        it.x1 = plan[i + 3];
        if (h->physics == TB_TTI) {
          it.ia = pcur[k & 1];
          it.ib = pcur[(k + 1) & 1];
          it.ic = rcur[k & 1];
          it.id = rcur[(k + 1) & 1];
          it.a = h->field[it.ia];
          it.b = h->field[it.ib];
          it.c = h->field[it.ic];
          it.d = h->field[it.id];
        }
        if (it.kind == 1 && (src_on || rec_on)) {
          WavePost& q = P.it[P.n++];
          q.x0 = it.x0;
          q.x1 = it.x1;
          if (src_on) q.dcmp = h->src_dcmp + (size_t)(n + k) * h->src.npts;
          if (h->physics == TB_TTI) {
            q.f0 = it.b;  // p^{n+k+1}, r^{n+k+1}
            q.f1 = it.d;
            q.s0 = it.b;
          } else {
            q.f0 = h->efield + 3 * Np;
            q.f1 = h->efield + 4 * Np;
            q.f2 = h->efield + 5 * Np;
            q.s0 = q.f0;
            q.s1 = q.f1;
            q.s2 = q.f2;
          }
          if (rec_on) q.row = h->rec_dcmp + (size_t)(fill + k) * h->rec.npts;
        }
        const bool last = i + 4 == plan.size() || plan[i + 4] != plan[i];
        if (!last) continue;
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (h->opt.profile) {
          ea = ev_next(h);
          eb = ev_next(h);
          h->ev_kind.push_back(0);
          if (ea) cudaEventRecord(ea, st);
        }
        cudaError_t e = fused ? tti_fused(h->R, g, w, 0, &L, nullptr, nullptr, nullptr, nullptr, h->c2, h->coef,
                                          h->nzb, h->damp_b, st)
                        : ela_tma ? elastic_tma(h->R, g, w, (float)h->dt, h->ela_maps, 0, 0, &L, h->efield,
                                                h->eta_dt, tmo, h->err, st)
                        : tti_tma_on ? tti_tma(h->R, g, w, h->tti_maps, 0, nullptr, &L, h->flux, h->damp_b, tmo,
                                               h->err, st)
                                  : wave_launch(h->physics, h->R, g, w, (float)h->dt, L, h->c2, h->coef, h->nzb,
                                                h->damp_b, h->flux, h->efield, h->emat, h->eta_dt, st);
        if (h->opt.profile && eb) cudaEventRecord(eb, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "wavefront launch");
        if (P.n > 0) {
          e = wave_post(g, P, src_on ? h->src.npts : 0, h->src.lin, rec_on ? h->rec.npts : 0, h->rec.ent, h->rec.lin,
                        st);
          if (e != cudaSuccess) return cuda_fail(h, e, "wavefront injection / sampling");
        }
        L.n = 0;
        P.n = 0;
      }
      if (T & 1) {
        std::swap(pc, pp);
        std::swap(rc, rp);
      }
      n += T;
      if (rec_on) {
        fill += T;
        if (fill == h->rec_cap) {
          int s = flush();
          if (s != TB_OK) return s;
        }
      }
      continue;
    }
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (h->opt.profile) {
      ea = ev_next(h);
      eb = ev_next(h);
      h->ev_kind.push_back(0);
      if (ea) cudaEventRecord(ea, st);
    }
    cudaError_t e;
    float *f0, *f1 = nullptr, *f2 = nullptr, *s1 = nullptr, *s2 = nullptr;
    if (lowp) {
      void* uc = h->lp[h->lp_cur];
      void* up = h->lp[1 - h->lp_cur];
      e = lowprec_step(h->storage, h->R, g, lw, nchunks, uc, up, h->c2, h->damp_b, h->lp_scales,
                       (h->have_src && h->src.npts > 0) ? h->lp_srcmax : nullptr, n, h->lp_mx, st);
      if (h->opt.profile && eb) cudaEventRecord(eb, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
      h->lp_cur = 1 - h->lp_cur;  // u^{n+1} is now the current field
      if (h->have_src && h->src.npts > 0) {
        e = lowprec_inject(h->storage, g, h->src.npts, h->src.lin, h->src_dcmp + (size_t)n * h->src.npts, up,
                           h->lp_scales, n, h->lp_mx, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "injection");
      }
      if (rec_on) {
        e = lowprec_sample(h->storage, g, h->rec.npts, h->rec.ent, h->rec.lin, up, h->lp_scales, n,
                           h->rec_dcmp + (size_t)fill * h->rec.npts, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "receiver sampling");
        if (++fill == h->rec_cap) {
          int s = flush();
          if (s != TB_OK) return s;
        }
      }
      ++n;
      continue;
    }
    if (h->physics == TB_TTI) {
      if (fused) {
        e = tti_fused(h->R, g, w, fchunks, nullptr, h->field[pc], h->field[pp], h->field[rc], h->field[rp], h->c2,
                      h->coef, h->nzb, h->damp_b, st);
      } else if (tti_tma_on) {
        WaveItem one{};
        one.ia = pc;
        one.ib = pp;
        one.ic = rc;
        one.id = rp;
        one.a = h->field[pc];
        one.b = h->field[pp];
        one.c = h->field[rc];
        one.d = h->field[rp];
        e = tti_tma(h->R, g, w, h->tti_maps, echunks, &one, nullptr, h->flux, h->damp_b, tmo, h->err, st);
        one.kind = 1;
        if (e == cudaSuccess)
          e = tti_tma(h->R, g, w, h->tti_maps, echunks, &one, nullptr, h->flux, h->damp_b, tmo, h->err, st);
      } else {
        e = tti_step(h->R, g, w, nchunks, h->field[pc], h->field[pp], h->field[rc], h->field[rp], h->c2, h->coef,
                     h->nzb, h->damp_b, h->flux, st);
      }
      std::swap(pc, pp);
      std::swap(rc, rp);
      f0 = h->field[pc];
      f1 = h->field[rc];
    } else {
      if (ela_tma) {
        e = elastic_tma(h->R, g, w, (float)h->dt, h->ela_maps, 0, echunks, nullptr, h->efield, h->eta_dt, tmo,
                        h->err, st);
        if (e == cudaSuccess)
          e = elastic_tma(h->R, g, w, (float)h->dt, h->ela_maps, 1, echunks, nullptr, h->efield, h->eta_dt, tmo,
                          h->err, st);
      } else {
        e = elastic_step(h->R, g, w, (float)h->dt, nchunks, h->efield, h->emat, h->eta_dt, st);
      }
      f0 = h->efield + 3 * Np;
      f1 = h->efield + 4 * Np;
      f2 = h->efield + 5 * Np;
      s1 = f1;
      s2 = f2;
    }
    if (h->opt.profile && eb) cudaEventRecord(eb, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
    if (h->have_src && h->src.npts > 0) {
      e = inject_points(g, h->src.npts, h->src.lin, h->src_dcmp + (size_t)n * h->src.npts, f0, f1, f2, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "injection");
    }
    if (rec_on) {
      e = sample_points(g, h->rec.npts, h->rec.ent, h->rec.lin, f0, s1, s2, h->rec_dcmp + (size_t)fill * h->rec.npts,
                        st);
      if (e != cudaSuccess) return cuda_fail(h, e, "receiver sampling");
      if (++fill == h->rec_cap) {
        int s = flush();
        if (s != TB_OK) return s;
      }
    }
    ++n;
  }
  int s = flush();
  if (s != TB_OK) return s;
  h->cur_idx = pc;
  h->prev_idx = pp;
  h->last_nt = nt;
  if ((ela_tma || tti_tma_on) && nt > 0) {
    int err = 0;
    TB_CUDA(h, cudaMemcpyAsync(&err, h->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TB_CUDA(h, cudaStreamSynchronize(st));
    if (err) return fail(h, TB_ETIMEOUT, "a TTI / elastic CTA timed out waiting for its staged operands");
  }
  if (host_traces) {
    TB_CUDA(h, cudaMemcpyAsync(traces, h->traces_dev, sizeof(float) * (size_t)nt * nrec, cudaMemcpyDeviceToHost, st));
    TB_CUDA(h, cudaStreamSynchronize(st));
  }
  if (h->opt.check_nan && traces && nrec > 0 && nt > 0) {
    int cnt = 0;
    TB_CUDA(h, count_nonfinite(dtr, (int64_t)nt * nrec, h->err + 1, st));
    TB_CUDA(h, cudaMemcpyAsync(&cnt, h->err + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    TB_CUDA(h, cudaStreamSynchronize(st));
    if (cnt) return fail(h, TB_EDIVERGED, "%d non-finite trace samples", cnt);
  }
  h->msg[0] = 0;
  return TB_OK;
}

extern "C" int tb_forward(tb_handle* h, int nt, float* traces, int schedule, void* stream) {
  if (!h) return TB_EINVAL;
  if (!h->have_model) return fail(h, TB_ESTATE, "tb_set_model must come before tb_forward");
  if (nt < 0) return fail(h, TB_EINVAL, "nt < 0");
  if (schedule != TB_ONESTEP && schedule != TB_BLOCKED) return fail(h, TB_EINVAL, "bad schedule");
  if (h->have_src && h->src.npts > 0 && nt > h->src_nt)
    return fail(h, TB_EINVAL, "nt = %d exceeds the wavelet length %d", nt, h->src_nt);
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  if (h->physics != TB_ACOUSTIC) return forward_other(h, nt, traces, schedule, st);
  if (h->storage != TB_F32) {
    if (schedule != TB_ONESTEP)
      return fail(h, TB_EINVAL, "16-bit and plain storage run one step per launch (TB_ONESTEP)");
    // FP16 / BF16 storage runs the one-step sweep below; plain-FP32 storage
    // its streaming kernel
    if (!h->sk) return forward_other(h, nt, traces, schedule, st);
  }
  const int nrec = h->have_rec ? h->rec.npt : 0;
  const bool host_traces = traces && nrec > 0 && !is_device_ptr(traces);
  float* dtr = host_traces ? nullptr : traces;
  const int T = schedule == TB_BLOCKED ? h->opt.time_tile : 1;

  // blocked: bands pipelined across the K full time tiles unless the user
  // fixed the decomposition (y_bands, x_chunks); the nt mod T remaining
  // steps run one step per sweep
  const int K = T > 1 ? nt / T : 0;
  const bool pipelined = T > 1 && h->opt.y_bands == 0 && h->opt.x_chunks <= 1;
  Plan p1, pT;
  int s = plan_sweep(h, 1, &p1);
  if (s != TB_OK) return s;
  if (T > 1 && (s = pipelined ? plan_pipeline(h, T, K, &pT) : plan_sweep(h, T, &pT)) != TB_OK) return s;
  if ((s = ensure_capacity(h, 1, p1, nt, host_traces, nrec, st)) != TB_OK) return s;
  if (T > 1 && (s = ensure_capacity(h, T, pT, nt, host_traces, nrec, st)) != TB_OK) return s;
  if (host_traces) dtr = h->traces_dev;

  // the wavefield buffers: four FP32 fields, or the two 16-bit stored fields
  float* fld[4] = {h->field[0], h->field[1], h->field[2], h->field[3]};
  if (h->sk) {
    fld[0] = static_cast<float*>(h->lp[0]);
    fld[1] = static_cast<float*>(h->lp[1]);
  }
  const size_t fbytes = (h->sk ? 2 : sizeof(float)) * (size_t)h->n[0] * h->n[1] * h->n2p;
  // zero initial conditions (Eq. 1)
  TB_CUDA(h, cudaMemsetAsync(fld[0], 0, fbytes, st));
  TB_CUDA(h, cudaMemsetAsync(fld[1], 0, fbytes, st));
  TB_CUDA(h, cudaMemsetAsync(h->err, 0, sizeof(int), st));
  if (h->sk) {
    // per-step scales: scales[k] of u^{k-1} (u^{-1}, u^0 zero: 1), running max
    if ((s = ensure_scales(h, nt, st)) != TB_OK) return s;
    h->lp_cur = 0;
  }
  if (h->opt.profile) ev_reset(h, st);

  SweepParams P{};
  P.n0 = (int)h->n[0];
  P.n1 = (int)h->n[1];
  P.n2 = (int)h->n[2];
  P.n2p = h->n2p;
  P.c2 = h->c2;
  P.damp_b = h->damp_b;
  for (int d = 0; d < 3; ++d)
    for (int i = 1; i <= h->R; ++i) {
      const float wf = (float)(h->c[i] / (h->h[d] * h->h[d]));
      P.w2[d][i - 1] = make_float2(wf, wf);
    }
  const bool src_on = h->have_src && h->src.npts > 0;
  P.ev_pair = src_on ? h->ev_pair : nullptr;
  P.src_ev = h->src_ev;
  P.nev = h->nev;
  P.npair = h->npair;
  // a column pair injecting over more than 8 planes loads in most of its
  // stream steps: the blocked sweep then prefetches (a single source spans 2)
  P.src_prefetch = src_on && h->ev_max_span > 8;
  const bool rec_on = h->have_rec && h->rec.npts > 0 && nrec > 0;
  P.r_colptr = rec_on ? h->rec.colptr : nullptr;
  P.r_ent = rec_on ? h->rec.ent : nullptr;
  P.rec_dcmp = h->rec_dcmp;
  P.nrpts = h->rec.npts;
  P.ring = h->ring;
  P.progress = h->progress;
  P.err = h->err;
  P.timeout_ns = (long long)(h->opt.wait_timeout_s * 1e9);

  // upload both pass tables (one-step first, blocked after it)
  std::vector<PassDesc> all(p1.launch_passes);
  const int off_T = (int)all.size();
  if (T > 1) all.insert(all.end(), pT.launch_passes.begin(), pT.launch_passes.end());
  if ((int)all.size() > h->pass_cap) {
    dfree(h->d_pass, st);
    h->d_pass = nullptr;
    h->pass_cap = 0;
    TB_CUDA(h, dmalloc(&h->d_pass, sizeof(PassDesc) * all.size(), st));
    h->pass_cap = (int)all.size();
  }
  TB_CUDA(h, cudaMemcpyAsync(h->d_pass, all.data(), sizeof(PassDesc) * all.size(),
                             cudaMemcpyHostToDevice, st));

  int cur = 0, prev = 1;  // field indices of u^n and u^{n-1}
  // receiver samples of step n sit in ring row n mod rec_cap until the
  // traces of steps [flushed, done) are finalised (done: every row complete)
  int flushed = 0;
  auto flush_receivers = [&](int done) -> int {
    while (rec_on && dtr && flushed < done) {
      const int row = flushed % h->rec_cap, cnt = std::min(done - flushed, h->rec_cap - row);
      cudaEvent_t a = nullptr, b = nullptr;
      if (h->opt.profile) {
        a = ev_next(h);
        b = ev_next(h);
        h->ev_kind.push_back(1);
        if (a) cudaEventRecord(a, st);
      }
      cudaError_t e = finalize_traces(cnt, nrec, h->rec.corner_eid, h->rec.corner_w,
                                      h->rec_dcmp + (size_t)row * h->rec.npts, h->rec.npts,
                                      dtr + (size_t)flushed * nrec, st);
      if (h->opt.profile && b) cudaEventRecord(b, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "receiver finalize");
      flushed += cnt;
    }
    flushed = done;
    return TB_OK;
  };
  // before a launch recording steps below `hi` (steps below `done` complete)
  auto make_room = [&](int done, int hi) -> int {
    return rec_on && hi - flushed > h->rec_cap ? flush_receivers(done) : TB_OK;
  };
  P.rec_cap = h->rec_cap > 0 ? h->rec_cap : 1;
  P.lp_scales = h->lp_scales;
  P.lp_mx = h->lp_mx;
  P.lp_srcmax = (h->have_src && h->src.npts > 0) ? h->lp_srcmax : nullptr;
  // set `i` of the launch: the time tile from step n reading (fld[c], fld[p])
  auto set_fields = [&](int i, int c, int p, int out0, int out1, int step0) {
    SweepSet& S = P.set[i];
    S.u_cur = fld[c];
    S.u_prev = fld[p];
    S.tm_u = h->tm_box[c];
    S.tm_p = h->tm_tile[p];
    S.out0 = fld[out0];
    S.out1 = out1 >= 0 ? fld[out1] : nullptr;
    S.step0 = step0;
  };
  P.tm_c = h->tm_c2;
  auto launch = [&](int TT, const Plan& pl, int pass_off, size_t L) -> int {
    const int first = pl.launch_first[L];
    const int last = L + 1 < pl.launch_first.size() ? pl.launch_first[L + 1] : (int)pl.launch_passes.size();
    P.pass = h->d_pass + pass_off + first;
    P.npass = last - first;
    P.set1_cta0 = INT_MAX;
    for (int i = first; i < last; ++i)
      if (pl.launch_passes[i].set != 0) P.set1_cta0 = std::min(P.set1_cta0, pl.launch_passes[i].cta0);
    P.prog_base = h->prog_base;
    int maxsteps = 0;
    for (int i = first; i < last; ++i) {
      const PassDesc& d = pl.launch_passes[i];
      maxsteps = std::max(maxsteps, d.xo1 - 1 + (TT - 1) * h->R - d.xc0 + 1);
    }
    h->prog_base += (unsigned long long)maxsteps + 2;
    cudaEvent_t a = nullptr, b = nullptr;
    if (h->opt.profile) {
      a = ev_next(h);
      b = ev_next(h);
      h->ev_kind.push_back(0);
      if (a) cudaEventRecord(a, st);
    }
    cudaError_t e = sweep_launch(h->R, TT, P, pl.launch_ctas[L], TT > 1, st, TT == 1 ? h->sk : 0);
    if (h->opt.profile && b) cudaEventRecord(b, st);
    if (e != cudaSuccess) return cuda_fail(h, e, TT > 1 ? "blocked sweep launch" : "one-step launch");
    return TB_OK;
  };
  // every launch of a plan on the time tile (or step) from step n
  auto run = [&](int TT, const Plan& pl, int pass_off, int out0, int out1, int step0) -> int {
    set_fields(0, cur, prev, out0, out1, step0);
    for (size_t L = 0; L < pl.launch_first.size(); ++L) {
      int r = launch(TT, pl, pass_off, L);
      if (r != TB_OK) return r;
    }
    return TB_OK;
  };

  int n = 0;
  if (pipelined && K > 0) {
    // time tile k reads fields (0, 1) for even k and (2, 3) for odd k and
    // writes (u^{n+T}, u^{n+T-1}) into the other pair
    for (size_t L = 0; L < pT.launch_first.size(); ++L) {
      const int k = pT.launch_tile[L];
      const int c = (k & 1) ? 2 : 0, o = 2 - c;
      set_fields(0, c, c + 1, o, o + 1, k * T);
      set_fields(1, o, o + 1, c, c + 1, (k + 1) * T);
      if ((s = make_room(k * T, (k + 2) * T)) != TB_OK) return s;
      if ((s = launch(T, pT, off_T, L)) != TB_OK) return s;
    }
    cur = (K & 1) ? 2 : 0;
    prev = cur + 1;
    n = K * T;
  }
  while (n < nt) {
    if (T > 1 && !pipelined && n + T <= nt) {
      if ((s = make_room(n, n + T)) != TB_OK) return s;
      // the two fields not holding (u^n, u^{n-1}) receive (u^{n+T}, u^{n+T-1})
      int free_idx[2], nf = 0;
      for (int i = 0; i < 4; ++i)
        if (i != cur && i != prev) free_idx[nf++] = i;
      if ((s = run(T, pT, off_T, free_idx[0], free_idx[1], n)) != TB_OK) return s;
      cur = free_idx[0];
      prev = free_idx[1];
      n += T;
    } else {
      if ((s = make_room(n, n + 1)) != TB_OK) return s;
      if ((s = run(1, p1, 0, prev, -1, n)) != TB_OK) return s;
      std::swap(cur, prev);
      n += 1;
    }
  }
  if ((s = flush_receivers(nt)) != TB_OK) return s;
  h->cur_idx = cur;
  h->prev_idx = prev;
  if (h->sk) h->lp_cur = cur;
  h->last_nt = nt;

  if (T > 1) {
    int err = 0;
    TB_CUDA(h, cudaMemcpyAsync(&err, h->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TB_CUDA(h, cudaStreamSynchronize(st));
    if (err) return fail(h, TB_ETIMEOUT, "a blocked-sweep CTA timed out waiting for a neighbour");
  }
  if (host_traces) {
    TB_CUDA(h, cudaMemcpyAsync(traces, h->traces_dev, sizeof(float) * (size_t)nt * nrec,
                               cudaMemcpyDeviceToHost, st));
    TB_CUDA(h, cudaStreamSynchronize(st));
  }
  if (h->opt.check_nan && traces && nrec > 0 && nt > 0) {
    int cnt = 0;
    TB_CUDA(h, count_nonfinite(dtr, (int64_t)nt * nrec, h->err + 1, st));
    TB_CUDA(h, cudaMemcpyAsync(&cnt, h->err + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    TB_CUDA(h, cudaStreamSynchronize(st));
    if (cnt) return fail(h, TB_EDIVERGED, "%d non-finite trace samples", cnt);
  }
  h->msg[0] = 0;
  return TB_OK;
}

extern "C" int tb_get_field(tb_handle* h, int which, float* out, void* stream) {
  if (!h) return TB_EINVAL;
  if (h->last_nt < 0) return fail(h, TB_ESTATE, "no forward run yet");
  const int nwhich = h->physics == TB_ACOUSTIC ? 2 : (h->physics == TB_TTI ? 4 : 9);
  if (which < 0 || which >= nwhich || !out) return fail(h, TB_EINVAL, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  const float* src = nullptr;
  if (h->physics == TB_ACOUSTIC && h->storage != TB_F32) {
    // stored u / s: unpack with the step's scale into a dense FP32 array
    float sc = 1.f;
    const int k = h->last_nt - which + 1;  // scales[k] belongs to u^{k-1}
    TB_CUDA(h, cudaMemcpyAsync(&sc, h->lp_scales + k, sizeof(float), cudaMemcpyDeviceToHost, st));
    TB_CUDA(h, cudaStreamSynchronize(st));
    const void* u = h->lp[which == 0 ? h->lp_cur : 1 - h->lp_cur];
    const PhysGrid g{(int)h->n[0], (int)h->n[1], (int)h->n[2], h->n2p};
    const size_t N = (size_t)h->n[0] * h->n[1] * h->n[2];
    float* dst = out;
    float* tmp = nullptr;
    if (!is_device_ptr(out)) {
      TB_CUDA(h, dmalloc(&tmp, sizeof(float) * N, st));
      dst = tmp;
    }
    cudaError_t e = lowprec_unpack(h->storage, g, u, sc, dst, st);
    if (e == cudaSuccess && tmp) e = cudaMemcpyAsync(out, tmp, sizeof(float) * N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && tmp) e = cudaStreamSynchronize(st);
    dfree(tmp, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "tb_get_field");
    return TB_OK;
  }
  if (h->physics == TB_ACOUSTIC) {
    src = h->field[which == 0 ? h->cur_idx : h->prev_idx];
  } else if (h->physics == TB_TTI) {
    // p^n, p^{n-1}, r^n, r^{n-1}: p in fields {cur_idx, prev_idx}, r in the other two
    const int rc = h->cur_idx == 0 ? 2 : 3, rp = h->cur_idx == 0 ? 3 : 2;
    const int idx[4] = {h->cur_idx, h->prev_idx, rc, rp};
    src = h->field[idx[which]];
  } else {
    src = h->efield + (size_t)which * h->n[0] * h->n[1] * h->n2p;
  }
  const size_t N = (size_t)h->n[0] * h->n[1] * h->n[2];
  if (is_device_ptr(out)) {
    TB_CUDA(h, unpad_copy(src, out, (int)h->n[0], (int)h->n[1], (int)h->n[2], h->n2p, st));
    return TB_OK;
  }
  float* tmp = nullptr;
  TB_CUDA(h, dmalloc(&tmp, sizeof(float) * N, st));
  cudaError_t e = unpad_copy(src, tmp, (int)h->n[0], (int)h->n[1], (int)h->n[2], h->n2p, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, sizeof(float) * N, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dfree(tmp, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "tb_get_field");
  return TB_OK;
}

extern "C" int tb_get_source_points(tb_handle* h, int64_t* npts, int64_t* lin, float* dcmp) {
  if (!h || !npts) return TB_EINVAL;
  if (!h->have_src) return fail(h, TB_ESTATE, "no sources set");
  *npts = h->src.npts;
  if (h->src.npts > 0) {
    if (lin) TB_CUDA(h, cudaMemcpy(lin, h->src.lin, sizeof(int64_t) * h->src.npts, cudaMemcpyDeviceToHost));
    if (dcmp)
      TB_CUDA(h, cudaMemcpy(dcmp, h->src_dcmp, sizeof(float) * (size_t)h->src_nt * h->src.npts,
                            cudaMemcpyDeviceToHost));
  }
  return TB_OK;
}

extern "C" int tb_get_receiver_points(tb_handle* h, int64_t* npts, int64_t* lin, int32_t* corner_id,
                                      float* corner_w) {
  if (!h || !npts) return TB_EINVAL;
  if (!h->have_rec) return fail(h, TB_ESTATE, "no receivers set");
  *npts = h->rec.npts;
  if (h->rec.npts > 0 && lin)
    TB_CUDA(h, cudaMemcpy(lin, h->rec.lin, sizeof(int64_t) * h->rec.npts, cudaMemcpyDeviceToHost));
  if (h->rec.npt > 0) {
    if (corner_id)
      TB_CUDA(h, cudaMemcpy(corner_id, h->rec.corner_id, sizeof(int) * 8 * h->rec.npt, cudaMemcpyDeviceToHost));
    if (corner_w)
      TB_CUDA(h, cudaMemcpy(corner_w, h->rec.corner_w, sizeof(float) * 8 * h->rec.npt, cudaMemcpyDeviceToHost));
  }
  return TB_OK;
}

extern "C" int tb_kernel_time(tb_handle* h, int kind, int* launches, double* ms) {
  if (!h || !launches || !ms) return TB_EINVAL;
  *launches = 0;
  *ms = 0.0;
  if (!h->opt.profile) return fail(h, TB_ESTATE, "profiling is off (tb_options.profile)");
  if (h->ev_used > 0) TB_CUDA(h, cudaStreamSynchronize(h->ev_stream));
  for (size_t i = 0; i < h->ev_kind.size(); ++i) {
    if (h->ev_kind[i] != kind) continue;
    float t = 0.f;
    TB_CUDA(h, cudaEventElapsedTime(&t, h->ev[2 * i], h->ev[2 * i + 1]));
    *ms += t;
    ++*launches;
  }
  return TB_OK;
}

// ------------------------------------------------------------- adjoint --
// One-step sweeps for the adjoint's forward passes (no receiver recording).
struct StepRunner {
  Plan p1;
  SweepParams P{};
};
static int runner_init(tb_handle* h, StepRunner* r, cudaStream_t st) {
  int s = plan_sweep(h, 1, &r->p1);
  if (s != TB_OK) return s;
  if ((s = ensure_capacity(h, 1, r->p1, 0, false, 0, st)) != TB_OK) return s;
  TB_CUDA(h, cudaMemcpyAsync(h->d_pass, r->p1.launch_passes.data(), sizeof(PassDesc) * r->p1.launch_passes.size(),
                             cudaMemcpyHostToDevice, st));
  SweepParams& P = r->P;
  P.n0 = (int)h->n[0];
  P.n1 = (int)h->n[1];
  P.n2 = (int)h->n[2];
  P.n2p = h->n2p;
  P.c2 = h->c2;
  P.damp_b = h->damp_b;
  for (int d = 0; d < 3; ++d)
    for (int i = 1; i <= h->R; ++i) {
      const float wf = (float)(h->c[i] / (h->h[d] * h->h[d]));
      P.w2[d][i - 1] = make_float2(wf, wf);
    }
  const bool src_on = h->have_src && h->src.npts > 0;
  P.ev_pair = src_on ? h->ev_pair : nullptr;
  P.src_ev = h->src_ev;
  P.nev = h->nev;
  P.npair = h->npair;
  P.r_colptr = nullptr;
  P.r_ent = nullptr;
  P.err = h->err;
  P.timeout_ns = (long long)(h->opt.wait_timeout_s * 1e9);
  return TB_OK;
}
// one step of the sweep: u^{step+1} into out (fp when NULL) from fc = u^{step}
// and fp = u^{step-1}; box_c, tile_p: their TMA descriptors
static int runner_step_on(tb_handle* h, StepRunner* r, float* fc, float* fp, const CUtensorMap& box_c,
                          const CUtensorMap& tile_p, int step, cudaStream_t st, float* out = nullptr) {
  SweepParams& P = r->P;
  SweepSet& S = P.set[0];
  S.u_cur = fc;
  S.u_prev = fp;
  S.tm_u = box_c;
  S.tm_p = tile_p;
  S.out0 = out ? out : fp;
  S.out1 = nullptr;
  S.step0 = step;
  P.tm_c = h->tm_c2;
  P.rec_cap = 1;
  P.set1_cta0 = INT_MAX;
  const Plan& pl = r->p1;
  for (size_t L = 0; L < pl.launch_first.size(); ++L) {
    const int first = pl.launch_first[L];
    const int last = L + 1 < pl.launch_first.size() ? pl.launch_first[L + 1] : (int)pl.launch_passes.size();
    P.pass = h->d_pass + first;
    P.npass = last - first;
    cudaError_t e = sweep_launch(h->R, 1, P, pl.launch_ctas[L], false, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint sweep launch");
  }
  return TB_OK;
}
// u^{step+1} over field[prev] from field[cur] = u^{step}, field[prev] = u^{step-1}
static int runner_step(tb_handle* h, StepRunner* r, int cur, int prev, int step, cudaStream_t st) {
  return runner_step_on(h, r, h->field[cur], h->field[prev], h->tm_box[cur], h->tm_tile[prev], step, st);
}

// Adjoint-state gradient with one of two ways to provide the forward states
// the backward pass needs (u^k, u^{k-1}, u^{k-2} at adjoint step k):
//   TB_CKPT_SEGMENTS: a checkpoint every ceil(nt/S) steps and a segment
//     buffer of ceil(nt/S) + 2 states, every step recomputed once;
//   TB_CKPT_BINOMIAL: S stored states in Griewank's binomial schedule
//     (tb_checkpoint.cu), the least recomputation S states allow.
// Both give bit-identical gradients: every forward state is the same
// sequence of one-step sweeps from the zero initial condition.
static int adjoint_gradient_impl(tb_handle* h, int nt, const float* residual, float* grad_vp, float* grad_src,
                                 int n_snapshots, int ckpt, cudaStream_t st) {
  if (!h) return TB_EINVAL;
  if (h->physics != TB_ACOUSTIC || h->storage != TB_F32)
    return fail(h, TB_EINVAL, "the adjoint is implemented for the FP32 acoustic equation");
  if (!h->have_model || !h->have_src || !h->have_rec)
    return fail(h, TB_ESTATE, "tb_set_model, tb_set_sources and tb_set_receivers must come first");
  if (nt <= 0 || !residual || n_snapshots < 1 || (!grad_vp && !grad_src)) return fail(h, TB_EINVAL, "bad arguments");
  if (ckpt != TB_CKPT_SEGMENTS && ckpt != TB_CKPT_BINOMIAL) return fail(h, TB_EINVAL, "bad checkpointing");
  if (ckpt == TB_CKPT_BINOMIAL && n_snapshots > 4096) return fail(h, TB_EINVAL, "n_snapshots > 4096");
  if (h->src.npts > 0 && nt > h->src_nt)
    return fail(h, TB_EINVAL, "nt = %d exceeds the wavelet length %d", nt, h->src_nt);
  h->last_stream = st;
  const int nrec = h->rec.npt, nsrc = h->src.npt;
  const int64_t nrp = h->rec.npts, nsp = h->src.npts;
  const size_t Np = (size_t)h->n[0] * h->n[1] * h->n2p, fbytes = sizeof(float) * Np;
  const int K = (nt + n_snapshots - 1) / n_snapshots;  // segments: steps per segment
  const int nseg = (nt + K - 1) / K;
  std::vector<CkptAction> plan;
  int64_t fsteps = 0;
  if (ckpt == TB_CKPT_BINOMIAL && plan_binomial(nt, n_snapshots, &plan, &fsteps) != TB_OK)
    return fail(h, TB_EINVAL, "checkpoint schedule");
  StepRunner run;
  int s = runner_init(h, &run, st);
  if (s != TB_OK) return s;
  std::vector<void*> bufs;
  size_t scratch = 0;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (dmalloc(&p, bytes ? bytes : 1, st) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    scratch += bytes ? bytes : 1;
    return p;
  };
  auto cleanup = [&]() {
    for (void* p : bufs) dfree(p, st);
    bufs.clear();
  };
  // state storage.  Segments: checkpoints (u^{jK}, u^{jK-1}) of segments
  // j >= 1 and a segment of K + 2 states (u^{k0-1} .. u^{k1}).  Binomial: S
  // slots of two fields, a work pair, a zero field (X_0) and the handle's
  // four wavefields as scratch of the advances and the reverse steps.
  float* snap = nullptr;
  float* seg = nullptr;
  float* slots = nullptr;
  float* work = nullptr;
  float* zero = nullptr;
  if (ckpt == TB_CKPT_SEGMENTS) {
    snap = (float*)alloc(fbytes * 2 * std::max(nseg - 1, 1));
    seg = (float*)alloc(fbytes * (K + 2));
  } else {
    slots = (float*)alloc(fbytes * 2 * n_snapshots);
    work = (float*)alloc(fbytes * 2);
    zero = (float*)alloc(fbytes);
  }
  float* lam = (float*)alloc(fbytes * 2);
  double* gm = (double*)alloc(sizeof(double) * Np);
  float* resT = (float*)alloc(sizeof(float) * (size_t)nt * std::max(nrec, 1));
  float* rdcmp = (float*)alloc(sizeof(float) * (size_t)nt * std::max<int64_t>(nrp, 1));
  float* srow = (float*)alloc(sizeof(float) * (size_t)nt * std::max<int64_t>(nsp, 1));
  float* gsrc = (float*)alloc(sizeof(float) * (size_t)nt * std::max(nsrc, 1) * 2);
  float* gvp_dev = nullptr;
  const bool gvp_host = grad_vp && !is_device_ptr(grad_vp);
  if (gvp_host) gvp_dev = (float*)alloc(sizeof(float) * (size_t)h->n[0] * h->n[1] * h->n[2]);
  const bool have_states = ckpt == TB_CKPT_SEGMENTS ? (snap && seg) : (slots && work && zero);
  if (!have_states || !lam || !gm || !resT || !rdcmp || !srow || !gsrc || (gvp_host && !gvp_dev)) {
    cleanup();
    cudaGetLastError();
    return fail(h, TB_ENOMEM, "adjoint scratch");
  }
  const PhysGrid g{(int)h->n[0], (int)h->n[1], (int)h->n[2], h->n2p};
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess && x != cudaSuccess) e = x;
    return e == cudaSuccess;
  };
  // residual [nt][nrec] -> [nrec][nt] -> per receiver point: sum_c w r (FP64)
  {
    void* tmp = nullptr;
    const void* dres = nullptr;
    ok(to_device(residual, sizeof(float) * (size_t)nt * nrec, &tmp, &dres, st));
    if (tmp) {
      bufs.push_back(tmp);
      scratch += sizeof(float) * (size_t)nt * nrec;
    }
    ok(transpose_f32(nt, nrec, (const float*)dres, resT, st));
    if (nrp > 0) ok(decompose(&h->rec, nt, resT, nullptr, 1.0, (int)h->n[1], (int)h->n[2], h->n2p, rdcmp, st));
    // injected into mu = D lam: scaled by D at each receiver point
    if (nrp > 0) ok(adjoint_scale_rows(g, nt, nrp, h->rec.lin, h->c2, h->damp_b, rdcmp, st));
  }
  // TMA descriptors of every buffer a forward or adjoint step reads
  SweepShape sh;
  if (!sweep_shape(h->R, 1, &sh, 0)) ok(cudaErrorInvalidValue);
  struct Buf {
    float* p;
    CUtensorMap box, tile;
  };
  auto mkbuf = [&](float* p) {
    Buf b{p, {}, {}};
    ok(make_tmap(&b.box, p, h->n, h->n2p, sh.box_w, sh.box_h));
    ok(make_tmap(&b.tile, p, h->n, h->n2p, 64, sh.TY));
    return b;
  };
  // the adjoint sweeps: the forward sweep kernel on the mu fields, without
  // the sources (the residual is injected after each step)
  StepRunner arun = run;
  arun.P.ev_pair = nullptr;
  Buf mub[2] = {mkbuf(lam), mkbuf(lam + Np)};
  int mc = 0, mp = 1;  // mu^{k+1} in mub[mc], mu^{k+2} in mub[mp]
  ok(cudaMemsetAsync(lam, 0, fbytes * 2, st));
  ok(cudaMemsetAsync(gm, 0, sizeof(double) * Np, st));
  ok(cudaMemsetAsync(h->err, 0, sizeof(int), st));
  // adjoint step k (k = nt .. 1, in that order) with the forward states
  // u^k, u^{k-1}, u^{k-2}
  auto adjoint_step = [&](int k, const float* uk, const float* uk1, const float* uk2) -> int {
    // mu^k over mu^{k+2}, then + D P^T r[k-1]
    int r = runner_step_on(h, &arun, mub[mc].p, mub[mp].p, mub[mc].box, mub[mp].tile, nt - k, st);
    if (r != TB_OK) return r;
    std::swap(mc, mp);
    float* m0 = mub[mc].p;
    if (nrp > 0) ok(inject_points(g, nrp, h->rec.lin, rdcmp + (size_t)(k - 1) * nrp, m0, nullptr, nullptr, st));
    if (grad_vp) {
      ok(adjoint_grad(g, h->dt, m0, uk, uk1, uk2, gm, st));
      if (nsp > 0)
        ok(adjoint_grad_src(g, nsp, h->src.lin, h->src_dcmp + (size_t)(k - 1) * nsp, h->dt, m0, h->c2, h->damp_b,
                            gm, st));
    }
    if (grad_src && nsp > 0)
      ok(adjoint_sample_src(g, nsp, h->src.ent, h->src.lin, m0, h->c2, h->damp_b, srow + (size_t)(k - 1) * nsp, st));
    return TB_OK;
  };
  if (ckpt == TB_CKPT_SEGMENTS) {
    // seg[s] = u^{k0 - 1 + s}; the recomputation writes each state straight
    // into its segment slot
    std::vector<Buf> sb;
    for (int i = 0; i < K + 2; ++i) sb.push_back(mkbuf(seg + (size_t)i * Np));
    // forward pass, keeping the checkpoints
    int cur = 0, prev = 1;
    ok(cudaMemsetAsync(h->field[0], 0, fbytes, st));
    ok(cudaMemsetAsync(h->field[1], 0, fbytes, st));
    for (int n = 0; n < nt && e == cudaSuccess; ++n) {
      if (n > 0 && n % K == 0) {
        const int j = n / K;
        ok(cudaMemcpyAsync(snap + (size_t)(2 * (j - 1)) * Np, h->field[cur], fbytes, cudaMemcpyDeviceToDevice, st));
        ok(cudaMemcpyAsync(snap + (size_t)(2 * (j - 1) + 1) * Np, h->field[prev], fbytes, cudaMemcpyDeviceToDevice,
                           st));
      }
      if ((s = runner_step(h, &run, cur, prev, n, st)) != TB_OK) break;
      std::swap(cur, prev);
    }
    // backward over the segments, each recomputed once from its checkpoint
    for (int j = nseg - 1; j >= 0 && e == cudaSuccess && s == TB_OK; --j) {
      const int k0 = j * K, k1 = std::min((j + 1) * K, nt);
      if (j == 0) {
        ok(cudaMemsetAsync(seg, 0, fbytes * 2, st));
      } else {
        ok(cudaMemcpyAsync(seg + Np, snap + (size_t)(2 * (j - 1)) * Np, fbytes, cudaMemcpyDeviceToDevice, st));
        ok(cudaMemcpyAsync(seg, snap + (size_t)(2 * (j - 1) + 1) * Np, fbytes, cudaMemcpyDeviceToDevice, st));
      }
      for (int n = k0; n <= k1 - 1 && e == cudaSuccess && s == TB_OK; ++n) {
        const int sc = n - k0 + 1;  // slot of u^n
        s = runner_step_on(h, &run, sb[sc].p, sb[sc - 1].p, sb[sc].box, sb[sc - 1].tile, n, st, sb[sc + 1].p);
      }
      for (int k = k1; k >= k0 + 1 && e == cudaSuccess && s == TB_OK; --k)
        s = adjoint_step(k, sb[k - k0 + 1].p, sb[k - k0].p, sb[k - k0 - 1].p);
    }
  } else {
    // slot i holds a state X_n = (u^n, u^{n-1}) in fields 2i, 2i + 1
    std::vector<Buf> sl;
    for (int i = 0; i < 2 * n_snapshots; ++i) sl.push_back(mkbuf(slots + (size_t)i * Np));
    Buf wk[2] = {mkbuf(work), mkbuf(work + Np)};
    Buf zb = mkbuf(zero);
    Buf hf[4];
    for (int i = 0; i < 4; ++i) hf[i] = Buf{h->field[i], h->tm_box[i], h->tm_tile[i]};
    ok(cudaMemsetAsync(zero, 0, fbytes, st));
    auto loc = [&](int L, int which) -> Buf* {
      if (L >= 0) return &sl[2 * L + which];
      return L == kCkptWork ? &wk[which] : &zb;
    };
    for (size_t ai = 0; ai < plan.size() && e == cudaSuccess && s == TB_OK; ++ai) {
      const CkptAction& a = plan[ai];
      Buf* c = loc(a.src, 0);  // u^from
      Buf* p = loc(a.src, 1);  // u^{from-1}
      if (a.kind == kCkptAdvance) {
        // X_to into dst: the last two states go to the destination's fields,
        // the ones before them to a scratch wavefield that is neither input
        Buf* d0 = loc(a.dst, 0);
        Buf* d1 = loc(a.dst, 1);
        if (a.to - a.from == 1) {
          if (a.src == kCkptZero) ok(cudaMemsetAsync(d1->p, 0, fbytes, st));
          else ok(cudaMemcpyAsync(d1->p, c->p, fbytes, cudaMemcpyDeviceToDevice, st));
        }
        for (int n = a.from; n < a.to && e == cudaSuccess && s == TB_OK; ++n) {
          Buf* out = n + 1 == a.to ? d0 : (n + 1 == a.to - 1 ? d1 : nullptr);
          for (int i = 0; i < 3 && !out; ++i)
            if (hf[i].p != c->p && hf[i].p != p->p) out = &hf[i];
          s = runner_step_on(h, &run, c->p, p->p, c->box, p->tile, n, st, out->p);
          p = c;
          c = out;
        }
      } else {
        // reverse step `from`: u^{from+1} by one forward step, then the adjoint
        // step k = from + 1 with u^k, u^{k-1}, u^{k-2}
        s = runner_step_on(h, &run, c->p, p->p, c->box, p->tile, a.from, st, hf[3].p);
        if (s == TB_OK) s = adjoint_step(a.from + 1, hf[3].p, c->p, p->p);
      }
    }
  }
  if (s != TB_OK) {
    cleanup();
    return s;
  }
  if (grad_vp && e == cudaSuccess) {
    ok(adjoint_finish(g, h->dt, gm, h->c2, gvp_host ? gvp_dev : grad_vp, st));
    if (gvp_host)
      ok(cudaMemcpyAsync(grad_vp, gvp_dev, sizeof(float) * (size_t)h->n[0] * h->n[1] * h->n[2],
                         cudaMemcpyDeviceToHost, st));
  }
  if (grad_src && nsrc > 0 && e == cudaSuccess) {
    // [nt][nsrc] by the source corner weights, then [nsrc][nt]
    if (nsp > 0) ok(finalize_traces(nt, nsrc, h->src.corner_eid, h->src.corner_w, srow, nsp, gsrc, st));
    else ok(cudaMemsetAsync(gsrc, 0, sizeof(float) * (size_t)nt * nsrc, st));
    float* gT = gsrc + (size_t)nt * nsrc;
    ok(transpose_f32(nt, nsrc, gsrc, gT, st));
    ok(cudaMemcpyAsync(grad_src, gT, sizeof(float) * (size_t)nt * nsrc,
                       is_device_ptr(grad_src) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  int err = 0;
  ok(cudaMemcpyAsync(&err, h->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  ok(cudaStreamSynchronize(st));
  cleanup();
  if (e != cudaSuccess) return cuda_fail(h, e, "tb_adjoint_gradient");
  if (err) return fail(h, TB_ETIMEOUT, "a sweep CTA timed out");
  h->last_nt = -1;  // the fields hold recomputation scratch now
  h->last_fwd_steps = ckpt == TB_CKPT_BINOMIAL ? fsteps : 2 * (int64_t)nt;
  h->last_scratch = scratch;
  h->msg[0] = 0;
  return TB_OK;
}

extern "C" int tb_adjoint_gradient(tb_handle* h, int nt, const float* residual, float* grad_vp, float* grad_src,
                                   int n_snapshots, void* stream) {
  return adjoint_gradient_impl(h, nt, residual, grad_vp, grad_src, n_snapshots, TB_CKPT_SEGMENTS,
                               (cudaStream_t)stream);
}

extern "C" int tb_adjoint_gradient_ckpt(tb_handle* h, int nt, const float* residual, float* grad_vp,
                                        float* grad_src, int n_snapshots, int checkpointing, void* stream) {
  return adjoint_gradient_impl(h, nt, residual, grad_vp, grad_src, n_snapshots, checkpointing,
                               (cudaStream_t)stream);
}

extern "C" int tb_adjoint_stats(const tb_handle* h, int64_t* forward_steps, size_t* scratch_bytes) {
  if (!h || !forward_steps || !scratch_bytes) return TB_EINVAL;
  *forward_steps = h->last_fwd_steps;
  *scratch_bytes = h->last_fwd_steps < 0 ? 0 : h->last_scratch;
  return TB_OK;
}

namespace tbi {
cudaError_t selftest_wait(long long timeout_ns, cudaStream_t st, int* timed_out);
}

extern "C" int tb_measure_peaks(double* hbm_gbs, double* fp32_tflops, void* stream) {
  if (!hbm_gbs || !fp32_tflops) return TB_EINVAL;
  *hbm_gbs = 0.0;
  *fp32_tflops = 0.0;
  const cudaError_t e = tbi::measure_peaks(hbm_gbs, fp32_tflops, (cudaStream_t)stream);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return TB_ENOMEM;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TB_ECUDA;
  }
  return TB_OK;
}

extern "C" int tb_selftest_wait(double timeout_s, void* stream) {
  if (!(timeout_s > 0) || timeout_s > 10) return TB_EINVAL;
  int timed_out = -1;
  cudaError_t e = tbi::selftest_wait((long long)(timeout_s * 1e9), (cudaStream_t)stream, &timed_out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TB_ECUDA;
  }
  return timed_out == 1 ? TB_ETIMEOUT : (timed_out == 0 ? TB_OK : TB_ECUDA);
}

// --------------------------------------------------------------- batch --
// Several small acoustic shots advanced together, one launch per time step
// for all of them (the one-step sweep over a concatenated pass table).
struct tb_batch {
  struct Shot {
    tb_handle* h;
    int nt, done, flushed, admit, slot;
    float* traces;  // device [nt][nrec] or NULL
    Plan p1;
  };
  int R = 0;
  int max_shots = 0;
  std::vector<Shot> active;
  std::vector<tb_handle*> finished;
  std::vector<char> slot_used;
  SweepParams* d_params = nullptr;  // [2 max_shots]: even / odd steps of each slot
  PassDesc* d_pass = nullptr;
  int pass_cap = 0, npass = 0, nctas = 0;
  bool dirty = true;
  int step = 0;
  cudaStream_t last_stream = nullptr;
};

extern "C" int tb_batch_create(int max_shots, tb_batch** out) {
  if (!out || max_shots < 1 || max_shots > 4096) return TB_EINVAL;
  *out = nullptr;
  tb_batch* b = new (std::nothrow) tb_batch();
  if (!b) return TB_ENOMEM;
  b->max_shots = max_shots;
  b->slot_used.assign(max_shots, 0);
  if (dmalloc(&b->d_params, sizeof(SweepParams) * 2 * max_shots, nullptr) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return TB_ENOMEM;
  }
  *out = b;
  return TB_OK;
}

extern "C" int tb_batch_destroy(tb_batch* b) {
  if (!b) return TB_OK;
  dfree(b->d_params, b->last_stream);
  dfree(b->d_pass, b->last_stream);
  delete b;
  return TB_OK;
}

extern "C" int tb_batch_active(const tb_batch* b) { return b ? (int)b->active.size() : 0; }

extern "C" int tb_batch_add(tb_batch* b, tb_handle* h, int nt, float* traces, void* stream) {
  if (!b || !h) return TB_EINVAL;
  if (h->physics != TB_ACOUSTIC || h->storage != TB_F32)
    return fail(h, TB_EINVAL, "batched shots: FP32 acoustic propagation only");
  if (!h->have_model) return fail(h, TB_ESTATE, "tb_set_model must come before tb_batch_add");
  if (nt < 0) return fail(h, TB_EINVAL, "nt < 0");
  if (h->have_src && h->src.npts > 0 && nt > h->src_nt)
    return fail(h, TB_EINVAL, "nt = %d exceeds the wavelet length %d", nt, h->src_nt);
  const int nrec = h->have_rec ? h->rec.npt : 0;
  if (traces && nrec > 0 && !is_device_ptr(traces)) return fail(h, TB_EINVAL, "batched traces must be device memory");
  if (b->R && b->R != h->R) return fail(h, TB_EINVAL, "a batch holds shots of one space order");
  for (const auto& s : b->active)
    if (s.h == h) return fail(h, TB_EINVAL, "the handle is already in the batch");
  int slot = -1;
  for (int i = 0; i < b->max_shots && slot < 0; ++i)
    if (!b->slot_used[i]) slot = i;
  if (slot < 0) return fail(h, TB_EINVAL, "the batch is full (%d shots)", b->max_shots);
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  b->last_stream = st;
  tb_batch::Shot s{h, nt, 0, 0, b->step, slot, traces, Plan{}};
  int r = plan_sweep(h, 1, &s.p1);
  if (r != TB_OK) return r;
  if ((r = ensure_capacity(h, 1, s.p1, nt, false, nrec, st)) != TB_OK) return r;
  const size_t fbytes = sizeof(float) * (size_t)h->n[0] * h->n[1] * h->n2p;
  TB_CUDA(h, cudaMemsetAsync(h->field[0], 0, fbytes, st));
  TB_CUDA(h, cudaMemsetAsync(h->field[1], 0, fbytes, st));
  TB_CUDA(h, cudaMemsetAsync(h->err, 0, sizeof(int), st));
  // the shot's parameters for even steps (u^n in field 0) and odd steps
  SweepParams P[2] = {};
  for (int par = 0; par < 2; ++par) {
    SweepParams& Q = P[par];
    const int c = par, p = 1 - par;
    Q.n0 = (int)h->n[0];
    Q.n1 = (int)h->n[1];
    Q.n2 = (int)h->n[2];
    Q.n2p = h->n2p;
    Q.c2 = h->c2;
    Q.damp_b = h->damp_b;
    for (int d = 0; d < 3; ++d)
      for (int i = 1; i <= h->R; ++i) {
        const float wf = (float)(h->c[i] / (h->h[d] * h->h[d]));
        Q.w2[d][i - 1] = make_float2(wf, wf);
      }
    const bool src_on = h->have_src && h->src.npts > 0;
    Q.ev_pair = src_on ? h->ev_pair : nullptr;
    Q.src_ev = h->src_ev;
    Q.nev = h->nev;
    Q.npair = h->npair;
    const bool rec_on = h->have_rec && h->rec.npts > 0 && nrec > 0 && traces;
    Q.r_colptr = rec_on ? h->rec.colptr : nullptr;
    Q.r_ent = rec_on ? h->rec.ent : nullptr;
    Q.rec_dcmp = h->rec_dcmp;
    Q.nrpts = h->rec.npts;
    Q.rec_cap = h->rec_cap > 0 ? h->rec_cap : 1;
    Q.err = h->err;
    Q.timeout_ns = (long long)(h->opt.wait_timeout_s * 1e9);
    Q.set1_cta0 = INT_MAX;
    Q.tm_c = h->tm_c2;
    SweepSet& S = Q.set[0];
    S.u_cur = h->field[c];
    S.u_prev = h->field[p];
    S.tm_u = h->tm_box[c];
    S.tm_p = h->tm_tile[p];
    S.out0 = h->field[p];  // u^{n+1} over u^{n-1}
    S.out1 = nullptr;
  }
  TB_CUDA(h, cudaMemcpyAsync(b->d_params + 2 * slot, P, sizeof(P), cudaMemcpyHostToDevice, st));
  b->slot_used[slot] = 1;
  b->R = h->R;
  h->last_nt = -1;
  if (nt == 0) {
    h->cur_idx = 0;
    h->prev_idx = 1;
    h->last_nt = 0;
    b->slot_used[slot] = 0;
    b->finished.push_back(h);
  } else {
    b->active.push_back(std::move(s));
    b->dirty = true;
  }
  h->msg[0] = 0;
  return TB_OK;
}

extern "C" int tb_batch_step(tb_batch* b, int nsteps, void* stream) {
  if (!b || nsteps < 0) return TB_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  b->last_stream = st;
  for (int k = 0; k < nsteps && !b->active.empty(); ++k) {
    if (b->dirty) {
      // the shots' passes, concatenated with running CTA offsets
      std::vector<PassDesc> all;
      int off = 0;
      for (const auto& s : b->active) {
        const Plan& pl = s.p1;
        for (size_t L = 0; L < pl.launch_first.size(); ++L) {
          const int first = pl.launch_first[L];
          const int last = L + 1 < pl.launch_first.size() ? pl.launch_first[L + 1] : (int)pl.launch_passes.size();
          for (int i = first; i < last; ++i) {
            PassDesc d = pl.launch_passes[i];
            d.cta0 += off;
            d.shot = s.slot;
            d.step_off = s.admit;
            all.push_back(d);
          }
          off += pl.launch_ctas[L];
        }
      }
      if ((int)all.size() > b->pass_cap) {
        dfree(b->d_pass, st);
        b->d_pass = nullptr;
        b->pass_cap = 0;
        if (dmalloc(&b->d_pass, sizeof(PassDesc) * all.size(), st) != cudaSuccess) {
          cudaGetLastError();
          return TB_ENOMEM;
        }
        b->pass_cap = (int)all.size();
      }
      if (cudaMemcpyAsync(b->d_pass, all.data(), sizeof(PassDesc) * all.size(), cudaMemcpyHostToDevice, st) !=
          cudaSuccess) {
        cudaGetLastError();
        return TB_ECUDA;
      }
      // the pageable copy above is staged before it returns: `all` may go
      b->npass = (int)all.size();
      b->nctas = off;
      b->dirty = false;
    }
    BatchParams L{b->d_pass, b->npass, b->d_params, b->step};
    cudaError_t e = sweep_batch_launch(b->R, L, b->nctas, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return TB_ECUDA;
    }
    ++b->step;
    for (size_t i = 0; i < b->active.size();) {
      tb_batch::Shot& s = b->active[i];
      tb_handle* h = s.h;
      ++s.done;
      const int nrec = h->have_rec ? h->rec.npt : 0;
      const bool rec_on = h->have_rec && h->rec.npts > 0 && nrec > 0 && s.traces;
      // receiver samples of steps [flushed, done) to traces before the ring wraps
      if (rec_on && (s.done - s.flushed == h->rec_cap || s.done == s.nt)) {
        const int row = s.flushed % h->rec_cap, cnt = s.done - s.flushed;
        e = finalize_traces(cnt, nrec, h->rec.corner_eid, h->rec.corner_w, h->rec_dcmp + (size_t)row * h->rec.npts,
                            h->rec.npts, s.traces + (size_t)s.flushed * nrec, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "batched receiver finalize");
        s.flushed = s.done;
      }
      if (s.done == s.nt) {
        h->cur_idx = s.nt & 1;
        h->prev_idx = 1 - h->cur_idx;
        h->last_nt = s.nt;
        b->slot_used[s.slot] = 0;
        b->finished.push_back(h);
        b->active.erase(b->active.begin() + i);
        b->dirty = true;
      } else {
        ++i;
      }
    }
  }
  return TB_OK;
}

extern "C" int tb_batch_finished(tb_batch* b, tb_handle** out, int max_out, int* n) {
  if (!b || !n || max_out < 0 || (max_out > 0 && !out)) return TB_EINVAL;
  const int k = std::min<int>(max_out, (int)b->finished.size());
  for (int i = 0; i < k; ++i) out[i] = b->finished[i];
  b->finished.erase(b->finished.begin(), b->finished.begin() + k);
  *n = k;
  return TB_OK;
}
