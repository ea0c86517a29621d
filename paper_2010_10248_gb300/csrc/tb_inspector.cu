// Inspector of Sec. II-A on the device, plus the small setup kernels.
//
// Off-grid points -> trilinear corners with FP64 weights (Sec. I, Fig. 3)
// -> keys (linear index << 24 | point*8 + corner), zero-weight corners get
// the sentinel key -> bitonic sort (keys unique, so the order of equal
// linear indices is the point order: contributions are later summed in
// source order) -> one scan marks unique affected points and gives them
// ascending IDs (the paper's SM / SID, Sec. II-A.2) -> a second sort by
// (column, x) gives the per-column reduced index (nnz_mask / Sp_SID of
// Sec. II-A.4, here along axis 0 because the propagator streams axis 0)
// -> the decomposition src_dcmp (Listing 3) sums each point's
// contributions in FP64.
#include <cstdio>

#include "tb_internal.cuh"

namespace tbi {

static constexpr unsigned long long kSentinel = ~0ull;
static constexpr int kLowBits = 24;

__global__ void k_corners(int npt, const double* __restrict__ xyz, int64_t n0, int64_t n1,
                          int64_t n2, double h0, double h1, double h2,
                          unsigned long long* keys, double* w8, int* bad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npt) return;
  const int64_t n[3] = {n0, n1, n2};
  const double h[3] = {h0, h1, h2};
  int64_t base[3];
  double f[3];
  bool ok = true;
  for (int d = 0; d < 3; ++d) {
    const double xi = xyz[3 * p + d];
    const double ext = (double)(n[d] - 1) * h[d];
    if (!(xi >= 0.0) || !(xi <= ext)) ok = false;
    const double t = xi / h[d];
    int64_t i = (int64_t)floor(ok ? t : 0.0);
    if (i < 0) i = 0;
    if (i > n[d] - 2) i = n[d] - 2;
    base[d] = i;
    f[d] = (ok ? t : 0.0) - (double)i;
  }
  if (!ok) atomicOr(bad, 1);
  for (int c = 0; c < 8; ++c) {
    const int bx = (c >> 2) & 1, by = (c >> 1) & 1, bz = c & 1;
    const double w = (bx ? f[0] : 1.0 - f[0]) * (by ? f[1] : 1.0 - f[1]) * (bz ? f[2] : 1.0 - f[2]);
    const int64_t lin = ((base[0] + bx) * n1 + (base[1] + by)) * n2 + (base[2] + bz);
    const unsigned long long id = (unsigned long long)p * 8 + c;
    keys[id] = (ok && w != 0.0) ? (((unsigned long long)lin << kLowBits) | id) : kSentinel;
    w8[id] = w;
  }
}

__global__ void k_fill_u64(unsigned long long* a, int64_t from, int64_t to, unsigned long long v) {
  const int64_t i = from + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < to) a[i] = v;
}

// Bitonic sort, ascending.  Global step for partner distance j >= 1024;
// the shared-memory kernel finishes all distances < 1024 of one stage.
__global__ void k_bitonic_global(unsigned long long* a, int64_t P, int64_t j, int64_t k) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const int64_t l = i ^ j;
  if (l <= i) return;
  const unsigned long long x = a[i], y = a[l];
  const bool up = (i & k) == 0;
  if ((x > y) == up) {
    a[i] = y;
    a[l] = x;
  }
}

__global__ void k_bitonic_shared(unsigned long long* a, int64_t P, int64_t k, int64_t jmax) {
  __shared__ unsigned long long s[2048];
  const int64_t base = (int64_t)blockIdx.x * 2048;
  for (int t = threadIdx.x; t < 2048; t += blockDim.x) s[t] = base + t < P ? a[base + t] : kSentinel;
  __syncthreads();
  for (int64_t j = jmax; j >= 1; j >>= 1) {
    for (int t = threadIdx.x; t < 2048; t += blockDim.x) {
      const int l = t ^ (int)j;
      if (l > t) {
        const unsigned long long x = s[t], y = s[l];
        const bool up = ((base + t) & k) == 0;
        if ((x > y) == up) {
          s[t] = y;
          s[l] = x;
        }
      }
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < 2048; t += blockDim.x)
    if (base + t < P) a[base + t] = s[t];
}

static cudaError_t bitonic_sort(unsigned long long* a, int64_t P, cudaStream_t st) {
  // P is a power of two >= 2048
  for (int64_t k = 2; k <= P; k <<= 1) {
    int64_t j = k >> 1;
    for (; j >= 1024; j >>= 1) {
      count_launch();
      k_bitonic_global<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(a, P, j, k);
    }
    count_launch();
    k_bitonic_shared<<<(unsigned)(P / 2048), 1024, 0, st>>>(a, P, k, j);
  }
  return cudaGetLastError();
}

// One CTA: mark the first entry of every distinct linear index among the
// sorted keys, number the distinct points in ascending order.
__global__ void __launch_bounds__(1024) k_unique(const unsigned long long* __restrict__ keys,
                                                 int64_t P, int64_t* lin, int64_t* gstart,
                                                 int* ent_id, int64_t* counts) {
  __shared__ int64_t warp_sums[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t nvalid = 0;
  for (int64_t b0 = 0; b0 < P; b0 += 1024) {
    const int64_t i = b0 + threadIdx.x;
    int flag = 0;
    unsigned long long g = 0;
    bool valid = false;
    if (i < P) {
      const unsigned long long k = keys[i];
      valid = k != kSentinel;
      g = k >> kLowBits;
      flag = valid && (i == 0 || (keys[i - 1] >> kLowBits) != g || keys[i - 1] == kSentinel);
    }
    // block inclusive scan of flag
    int v = flag;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    if (lane == 31) warp_sums[wid] = v;
    __syncthreads();
    if (wid == 0) {
      int64_t s = warp_sums[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
      }
      warp_sums[lane] = s;
    }
    __syncthreads();
    const int64_t incl = carry + v + (wid > 0 ? warp_sums[wid - 1] : 0);
    if (valid) {
      const int64_t id = incl - 1;
      ent_id[i] = (int)id;
      if (flag) {
        lin[id] = (int64_t)g;
        gstart[id] = i;
      }
      ++nvalid;
    } else if (i < P) {
      ent_id[i] = -1;
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry = incl;
    __syncthreads();
  }
  // totals
  __shared__ int64_t nv[1024];
  nv[threadIdx.x] = nvalid;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (threadIdx.x < s) nv[threadIdx.x] += nv[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    counts[0] = carry;  // npts
    counts[1] = nv[0];  // nvalid
    gstart[carry] = nv[0];
  }
}

// keys2 = ((y*n2 + z)*n0 + x) << 24 | id for each unique point
__global__ void k_colkeys(int64_t npts, const int64_t* __restrict__ lin, int64_t n0, int64_t n1,
                          int64_t n2, unsigned long long* keys2) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= npts) return;
  const int64_t l = lin[id];
  const int64_t z = l % n2, y = (l / n2) % n1, x = l / (n1 * n2);
  keys2[id] = ((unsigned long long)((y * n2 + z) * n0 + x) << kLowBits) | (unsigned long long)id;
}

__global__ void k_colptr(int64_t ncol, const unsigned long long* __restrict__ keys2, int64_t npts,
                         int64_t n0, int* colptr) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c > ncol) return;
  const unsigned long long target = (unsigned long long)(c * n0) << kLowBits;
  int64_t lo = 0, hi = npts;  // first index with key >= target
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (keys2[mid] < target) lo = mid + 1;
    else hi = mid;
  }
  colptr[c] = (int)lo;
}

__global__ void k_entries(int64_t npts, const unsigned long long* __restrict__ keys2, int64_t n0,
                          int2* ent, int* eid_of_id) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const unsigned long long k = keys2[i];
  const int64_t cx = (int64_t)(k >> kLowBits);
  const int id = (int)(k & ((1ull << kLowBits) - 1));
  ent[i] = make_int2((int)(cx % n0), id);
  eid_of_id[id] = (int)i;  // position of point id in the column-ordered entries
}

__global__ void k_corner_tables(int64_t nvalid, const unsigned long long* __restrict__ keys,
                                const int* __restrict__ ent_id, const int* __restrict__ eid_of_id,
                                const double* __restrict__ w8, int* corner_id, int* corner_eid,
                                float* corner_w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvalid) return;
  const unsigned long long pc = keys[i] & ((1ull << kLowBits) - 1);
  corner_id[pc] = ent_id[i];
  corner_eid[pc] = eid_of_id[ent_id[i]];
  corner_w[pc] = (float)w8[pc];
}

__global__ void k_fill_i32(int* a, int64_t n, int v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

void free_tables(PointTables* t, cudaStream_t st) {
  dfree(t->lin, st);
  dfree(t->colptr, st);
  dfree(t->ent, st);
  dfree(t->corner_id, st);
  dfree(t->corner_eid, st);
  dfree(t->corner_w, st);
  dfree(t->eid_of_id, st);
  dfree(t->keys, st);
  dfree(t->w8, st);
  dfree(t->gstart, st);
  dfree(t->ent_id, st);
  *t = PointTables();
}

static unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

int inspect(const int64_t n[3], const double h[3], int npt, const double* d_coords,
            bool want_corners, PointTables* t, cudaStream_t st, const char** why) {
  free_tables(t, st);
  t->npt = npt;
  const int64_t ncol = n[1] * n[2];
  if (npt <= 0) {
    // empty set: all-zero column pointers
    if (dmalloc(&t->colptr, sizeof(int) * (ncol + 1), st) != cudaSuccess) return TB_ENOMEM;
    cudaMemsetAsync(t->colptr, 0, sizeof(int) * (ncol + 1), st);
    t->bytes = sizeof(int) * (ncol + 1);
    return cudaGetLastError() == cudaSuccess ? TB_OK : TB_ECUDA;
  }
  if (npt >= (1 << (kLowBits - 3))) {
    *why = "too many points (limit 2^21)";
    return TB_EINVAL;
  }
  int64_t P = 2048;
  while (P < (int64_t)npt * 8) P <<= 1;
  int* d_bad = nullptr;
  int64_t* d_counts = nullptr;
  unsigned long long* keys2 = nullptr;
  int status = TB_OK;
  auto ok = [&](cudaError_t e) {
    if (e != cudaSuccess && status == TB_OK) status = (e == cudaErrorMemoryAllocation) ? TB_ENOMEM : TB_ECUDA;
    return e == cudaSuccess;
  };
  if (!ok(dmalloc(&t->keys, sizeof(unsigned long long) * P, st)) ||
      !ok(dmalloc(&t->w8, sizeof(double) * npt * 8, st)) ||
      !ok(dmalloc(&t->ent_id, sizeof(int) * P, st)) || !ok(dmalloc(&d_bad, sizeof(int) * 4, st)) ||
      !ok(dmalloc(&d_counts, sizeof(int64_t) * 2, st))) {
    dfree(d_bad, st);
    dfree(d_counts, st);
    return status;
  }
  ok(cudaMemsetAsync(d_bad, 0, sizeof(int) * 4, st));
  if (P > (int64_t)npt * 8) {  // sentinel tail (empty when 8 npt is a power of two)
    count_launch();
    k_fill_u64<<<grid_for(P - (int64_t)npt * 8, 256), 256, 0, st>>>(t->keys, (int64_t)npt * 8, P, kSentinel);
  }
  count_launch();
  k_corners<<<grid_for(npt, 128), 128, 0, st>>>(npt, d_coords, n[0], n[1], n[2], h[0], h[1], h[2],
                                                t->keys, t->w8, d_bad);
  ok(cudaGetLastError());
  ok(bitonic_sort(t->keys, P, st));
  // upper bound for npts is the number of corners; allocate that much
  const int64_t maxpts = (int64_t)npt * 8;
  ok(dmalloc(&t->lin, sizeof(int64_t) * maxpts, st));
  ok(dmalloc(&t->gstart, sizeof(int64_t) * (maxpts + 1), st));
  if (status != TB_OK) goto fail;
  count_launch();
  k_unique<<<1, 1024, 0, st>>>(t->keys, P, t->lin, t->gstart, t->ent_id, d_counts);
  ok(cudaGetLastError());
  {
    int64_t counts[2] = {0, 0};
    int bad = 0;
    ok(cudaMemcpyAsync(counts, d_counts, sizeof(counts), cudaMemcpyDeviceToHost, st));
    ok(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    ok(cudaStreamSynchronize(st));
    if (status != TB_OK) goto fail;
    if (bad) {
      *why = "coordinate outside [0, (n-1) h]";
      status = TB_EINVAL;
      goto fail;
    }
    t->npts = counts[0];
    t->nvalid = counts[1];
  }
  // per-column reduced index
  {
    int64_t P2 = 2048;
    while (P2 < t->npts) P2 <<= 1;
    ok(dmalloc(&keys2, sizeof(unsigned long long) * P2, st));
    ok(dmalloc(&t->colptr, sizeof(int) * (ncol + 1), st));
    ok(dmalloc(&t->ent, sizeof(int2) * (t->npts > 0 ? t->npts : 1), st));
    ok(dmalloc(&t->eid_of_id, sizeof(int) * (t->npts > 0 ? t->npts : 1), st));
    if (status != TB_OK) goto fail;
    count_launch();
    k_fill_u64<<<grid_for(P2, 256), 256, 0, st>>>(keys2, 0, P2, kSentinel);
    count_launch();
    k_colkeys<<<grid_for(t->npts, 256), 256, 0, st>>>(t->npts, t->lin, n[0], n[1], n[2], keys2);
    ok(bitonic_sort(keys2, P2, st));
    count_launch();
    k_colptr<<<grid_for(ncol + 1, 256), 256, 0, st>>>(ncol, keys2, t->npts, n[0], t->colptr);
    count_launch();
    k_entries<<<grid_for(t->npts, 256), 256, 0, st>>>(t->npts, keys2, n[0], t->ent, t->eid_of_id);
    ok(cudaGetLastError());
  }
  if (want_corners) {
    ok(dmalloc(&t->corner_id, sizeof(int) * npt * 8, st));
    ok(dmalloc(&t->corner_eid, sizeof(int) * npt * 8, st));
    ok(dmalloc(&t->corner_w, sizeof(float) * npt * 8, st));
    if (status != TB_OK) goto fail;
    count_launch();
    k_fill_i32<<<grid_for((int64_t)npt * 8, 256), 256, 0, st>>>(t->corner_id, (int64_t)npt * 8, -1);
    count_launch();
    k_fill_i32<<<grid_for((int64_t)npt * 8, 256), 256, 0, st>>>(t->corner_eid, (int64_t)npt * 8, -1);
    ok(cudaMemsetAsync(t->corner_w, 0, sizeof(float) * npt * 8, st));
    count_launch();
    k_corner_tables<<<grid_for(t->nvalid, 256), 256, 0, st>>>(
        t->nvalid, t->keys, t->ent_id, t->eid_of_id, t->w8, t->corner_id, t->corner_eid, t->corner_w);
    ok(cudaGetLastError());
  }
  ok(cudaStreamSynchronize(st));
  if (status != TB_OK) goto fail;
  dfree(keys2, st);
  dfree(d_bad, st);
  dfree(d_counts, st);
  t->bytes = sizeof(unsigned long long) * P + sizeof(double) * npt * 8 + sizeof(int) * P +
             sizeof(int64_t) * (2 * maxpts + 1) + sizeof(int) * (ncol + 1) + (sizeof(int2) + sizeof(int)) * t->npts +
             (want_corners ? (2 * sizeof(int) + sizeof(float)) * npt * 8 : 0);
  return TB_OK;
fail:
  dfree(keys2, st);
  dfree(d_bad, st);
  dfree(d_counts, st);
  free_tables(t, st);
  return status;
}

// src_dcmp[t][id] = c2(p_id) * sum_e w_e * q_{s(e)}[t]: FP64 sum in source
// order, then scaled by dt^2/m at the point (Listing 3, expression s*dt^2/m).
__global__ void k_decompose(int nt, int64_t npts, const int64_t* __restrict__ gstart,
                            const unsigned long long* __restrict__ keys,
                            const double* __restrict__ w8, const float* __restrict__ wav,
                            const int64_t* __restrict__ lin, const float* __restrict__ c2, double scale,
                            int64_t n1, int64_t n2, int64_t n2p, float* dcmp) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (id >= npts || t >= nt) return;
  double acc = 0.0;
  for (int64_t e = gstart[id]; e < gstart[id + 1]; ++e) {
    const unsigned long long pc = keys[e] & ((1ull << kLowBits) - 1);
    const int64_t p = (int64_t)(pc >> 3);
    acc += w8[pc] * (double)wav[p * nt + t];
  }
  const int64_t l = lin[id];
  const int64_t z = l % n2, y = (l / n2) % n1, x = l / (n1 * n2);
  const double s = c2 ? (double)c2[(x * n1 + y) * n2p + z] : scale;
  dcmp[(int64_t)t * npts + id] = (float)(acc * s);
}

cudaError_t decompose(const PointTables* t, int nt, const float* d_wav, const float* c2, double scale,
                      int n1, int n2, int n2p, float* d_dcmp, cudaStream_t st) {
  if (t->npts <= 0 || nt <= 0) return cudaSuccess;
  dim3 grid(grid_for(t->npts, 128), nt);
  count_launch();
  k_decompose<<<grid, 128, 0, st>>>(nt, t->npts, t->gstart, t->keys, t->w8, d_wav, t->lin, c2, scale, n1,
                                    n2, n2p, d_dcmp);
  return cudaGetLastError();
}

// ev[t][slot[i]] = dcmp[t][i]: the decomposed injections of every step
// rearranged by column pair and plane for the sweep kernel (slots of planes
// without a point keep the zero they were cleared to)
__global__ void k_events(int nt, int64_t npts, const int* __restrict__ slot, const float* __restrict__ dcmp,
                         float* __restrict__ ev, int64_t ev_row) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (i >= npts || t >= nt) return;
  ev[(size_t)t * ev_row + slot[i]] = dcmp[(size_t)t * npts + i];
}

cudaError_t source_events(int nt, int64_t npts, const int* slot, const float* dcmp, float* ev, int64_t ev_row,
                          cudaStream_t st) {
  if (npts <= 0 || nt <= 0) return cudaSuccess;
  dim3 grid(grid_for(npts, 128), nt);
  count_launch();
  k_events<<<grid, 128, 0, st>>>(nt, npts, slot, dcmp, ev, ev_row);
  return cudaGetLastError();
}

// trace[s][r] = sum_c w_rc * rec_dcmp[s][e_rc], corners in fixed order; the
// recorded receiver points are indexed by their position e in the
// column-ordered entry list
__global__ void k_finalize(int nsteps, int nrec, const int* __restrict__ cid,
                           const float* __restrict__ cw, const float* __restrict__ rec_dcmp,
                           int64_t nrpts, float* traces) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (r >= nrec || s >= nsteps) return;
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int id = cid[r * 8 + c];
    if (id >= 0) acc = __fmaf_rn(cw[r * 8 + c], rec_dcmp[(int64_t)s * nrpts + id], acc);
  }
  traces[(int64_t)s * nrec + r] = acc;
}

cudaError_t finalize_traces(int nsteps, int nrec, const int* corner_id, const float* corner_w,
                            const float* rec_dcmp, int64_t nrpts, float* traces, cudaStream_t st) {
  if (nsteps <= 0 || nrec <= 0) return cudaSuccess;
  dim3 grid(grid_for(nrec, 256), nsteps);
  count_launch();
  k_finalize<<<grid, 256, 0, st>>>(nsteps, nrec, corner_id, corner_w, rec_dcmp, nrpts, traces);
  return cudaGetLastError();
}

__global__ void k_vmax(const float* __restrict__ vp, int64_t N, unsigned* out, int* bad) {
  float m = 0.f;
  int b = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = vp[i];
    if (!(v > 0.f) || !isfinite(v)) b = 1;
    else m = fmaxf(m, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    b |= __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, __float_as_uint(m));  // positive floats order like their bits
    if (b) atomicOr(bad, 1);
  }
}

cudaError_t model_vmax(const float* vp, int64_t N, float* d_out, int* d_bad, cudaStream_t st) {
  cudaMemsetAsync(d_out, 0, sizeof(float), st);
  cudaMemsetAsync(d_bad, 0, sizeof(int), st);
  count_launch();
  k_vmax<<<1024, 256, 0, st>>>(vp, N, reinterpret_cast<unsigned*>(d_out), d_bad);
  return cudaGetLastError();
}

__global__ void k_c2(const float* __restrict__ vp, int64_t n0, int64_t n1, int64_t n2, int64_t n2p,
                     double dt2, float* c2) {
  const int64_t N = n0 * n1 * n2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t z = i % n2, xy = i / n2;
    const double v = (double)vp[i];
    c2[xy * n2p + z] = (float)(dt2 * v * v);
  }
}

cudaError_t model_c2(const float* vp, int n0, int n1, int n2, int n2p, double dt2, float* c2,
                     cudaStream_t st) {
  count_launch();
  k_c2<<<4096, 256, 0, st>>>(vp, n0, n1, n2, n2p, dt2, c2);
  return cudaGetLastError();
}

__global__ void k_pad(const float* __restrict__ s, float* d, int64_t n0, int64_t n1, int64_t n2,
                      int64_t n2p, int dir) {
  const int64_t N = n0 * n1 * n2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t z = i % n2, xy = i / n2;
    if (dir == 0) d[xy * n2p + z] = s[i];
    else d[i] = s[xy * n2p + z];
  }
}

cudaError_t pad_copy(const float* src, float* dst, int n0, int n1, int n2, int n2p,
                     cudaStream_t st) {
  count_launch();
  k_pad<<<4096, 256, 0, st>>>(src, dst, n0, n1, n2, n2p, 0);
  return cudaGetLastError();
}

cudaError_t unpad_copy(const float* src, float* dst, int n0, int n1, int n2, int n2p,
                       cudaStream_t st) {
  count_launch();
  k_pad<<<4096, 256, 0, st>>>(src, dst, n0, n1, n2, n2p, 1);
  return cudaGetLastError();
}

__global__ void k_nonfinite(const float* __restrict__ a, int64_t n, int* cnt) {
  int c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    c += !isfinite(a[i]);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

cudaError_t count_nonfinite(const float* a, int64_t n, int* d_count, cudaStream_t st) {
  cudaMemsetAsync(d_count, 0, sizeof(int), st);
  if (n > 0) k_nonfinite<<<1024, 256, 0, st>>>(a, n, d_count);
  return cudaGetLastError();
}



// ---------------------------------------------------------------------------
// Allocation-free variant of the source-point inspector (tb_inspect_points_noalloc).
//
// Some callers cannot call cudaMalloc while they run: code that must not
// touch the allocator once started (a pre-sized device memory budget, or a
// real-time loop where an allocation would synchronise the device), and
// hosts whose memory is owned by another allocator.  This entry point takes
// the inspector's scratch (sort keys, per-entry ids, group starts, corner
// weights, counters) from a fixed array in device memory that every GPU
// loading the library holds until the process exits.  It computes the
// ascending unique affected points of a set of off-grid points, exactly as
// tb_set_sources does, into the caller's buffers.
// ---------------------------------------------------------------------------
namespace {
constexpr int64_t kNoAllocKeys = 1 << 16;  // corner slots: 8 per point -> 8192 points
constexpr size_t kNoAllocKeysOff = 0;
constexpr size_t kNoAllocEntOff = kNoAllocKeysOff + sizeof(unsigned long long) * kNoAllocKeys;
constexpr size_t kNoAllocStartOff = kNoAllocEntOff + sizeof(int) * kNoAllocKeys;
constexpr size_t kNoAllocW8Off = kNoAllocStartOff + sizeof(int64_t) * (kNoAllocKeys + 2);
constexpr size_t kNoAllocCountOff = kNoAllocW8Off + sizeof(double) * kNoAllocKeys;
constexpr size_t kNoAllocBadOff = kNoAllocCountOff + sizeof(int64_t) * 2;
constexpr size_t kNoAllocBytes = kNoAllocBadOff + 256;
}  // namespace

// The scratch of tb_inspect_points_noalloc (about 1.8 MB per device).
static __device__ __align__(256) unsigned char g_tb_noalloc_scratch[kNoAllocBytes];

__global__ void k_noalloc_result(const int* bad, const int64_t* counts, int64_t* npts_out) {
  *npts_out = *bad ? -1 : counts[0];
}

}  // namespace tbi

#include <mutex>

namespace {
// Device address of the scratch array, looked up once per device with that
// device current (the host-side symbol is not a device address).
void* noalloc_scratch(int dev, cudaError_t* err) {
  constexpr int kMaxDevices = 256;
  static void* ptr[kMaxDevices] = {nullptr};
  static std::mutex mu;
  *err = cudaSuccess;
  if (dev < 0 || dev >= kMaxDevices) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!ptr[dev]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, tbi::g_tb_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    ptr[dev] = p;
  }
  return ptr[dev];
}
}  // namespace

extern "C" int tb_inspect_points_noalloc(const int64_t n[3], const double h[3], int npt,
                                         const double* coords, int64_t* lin, int64_t* npts,
                                         void* stream) {
  using namespace tbi;
  if (!n || !h || !npts || npt < 0) return TB_EINVAL;
  if ((int64_t)npt * 8 > kNoAllocKeys) return TB_EINVAL;  // more than 8192 points
  if (npt > 0 && (!coords || !lin)) return TB_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (n[d] < 2 || n[d] > 65535 || !(h[d] > 0)) return TB_EINVAL;
  // the sort key holds the linear index above 24 bits of corner number: the
  // same grid-size limit as tb_create
  if (n[0] * n[1] * n[2] >= (1ll << 40)) return TB_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return TB_ECUDA;
  if (st) {  // the scratch address is per device: the stream must be the current device's
    int sdev = -1;
    if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
      cudaGetLastError();
      return TB_EINVAL;
    }
    if (sdev != dev) return TB_EINVAL;
  }
  unsigned char* base = (unsigned char*)noalloc_scratch(dev, &e);
  if (!base) {
    cudaGetLastError();
    return TB_ECUDA;
  }
  if (npt == 0) return cudaMemsetAsync(npts, 0, sizeof(int64_t), st) == cudaSuccess ? TB_OK : TB_ECUDA;
  unsigned long long* keys = (unsigned long long*)(base + kNoAllocKeysOff);
  int* ent_id = (int*)(base + kNoAllocEntOff);
  int64_t* gstart = (int64_t*)(base + kNoAllocStartOff);
  double* w8 = (double*)(base + kNoAllocW8Off);
  int64_t* counts = (int64_t*)(base + kNoAllocCountOff);
  int* bad = (int*)(base + kNoAllocBadOff);
  int64_t P = 2048;
  while (P < (int64_t)npt * 8) P <<= 1;
  // the array keeps the previous call's contents: reset what must start at zero
  e = cudaMemsetAsync(bad, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    count_launch(3);
    if (P > (int64_t)npt * 8) {
      count_launch();
      k_fill_u64<<<grid_for(P - (int64_t)npt * 8, 256), 256, 0, st>>>(keys, (int64_t)npt * 8, P, kSentinel);
    }
    k_corners<<<grid_for(npt, 128), 128, 0, st>>>(npt, coords, n[0], n[1], n[2], h[0], h[1], h[2], keys, w8,
                                                  bad);
    e = bitonic_sort(keys, P, st);
  }
  if (e == cudaSuccess) {
    k_unique<<<1, 1024, 0, st>>>(keys, P, lin, gstart, ent_id, counts);
    k_noalloc_result<<<1, 1, 0, st>>>(bad, counts, npts);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TB_ECUDA;
  }
  return TB_OK;
}
