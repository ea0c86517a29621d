/*
 * tb_oracle.c -- plain FP64 CPU oracle for the temporally blocked wave
 * propagator with off-the-grid sources (arXiv 2010.10248).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (FP64 throughout, no blocking, no fusion unless a
 * function says it follows a specific listing of the paper):
 *
 *   Eq. 1 (Sec. III-A), isotropic acoustic:  m u_tt - Lap u = delta(x_s) q(t),
 *   zero initial conditions, d(t,.) = u(t, x_r).  Discretised 2nd order in
 *   time, space order so in {4, 8, 12} (centred Fornberg weights), with the
 *   absorbing damping term eta*u_t of Sec. IV-B:
 *
 *     u^{n+1} = [dt^2 L u^n + m (2u^n - u^{n-1}) + (eta dt/2) u^{n-1}]
 *               / (m + eta dt/2)
 *
 *   Source injection follows the Devito expression s.inject(u.forward,
 *   expr = s*dt^2/m) of the listing in Sec. III-A, applied after the stencil
 *   sweep as in Listing 1 (Sec. I): for every source, for every trilinear
 *   corner c with weight w != 0:  u^{n+1}(c) += w q_s[n] dt^2 / m(c).
 *   Receivers interpolate trilinearly: trace[n][r] = sum_c w_rc u^{n+1}(c).
 *
 *   Outside the grid the wavefield is identically zero (a zero halo of width
 *   so/2 that is never updated).  A periodic mode exists only for the
 *   closed-form eigenmode pin in the tests.
 *
 * Readings where the paper is silent, and the reading taken here:
 *   - affected points are the trilinear corners with FP64 weight != 0
 *     (structural, independent of the wavelet values; Sec. II-A.1);
 *   - the unique IDs of Sec. II-A.2 ascend with the linear index
 *     (x*n1 + y)*n2 + z;
 *   - m in s*dt^2/m is evaluated at the affected grid point;
 *   - trace[n] samples u^{n+1} after the step-n injection;
 *   - the sponge is eta(d) = eta_max (d/nbl)^2 per axis, d = 1..nbl cells
 *     into the layer, summed over axes, eta_max = 3 vmax ln(1/R)/(2 nbl h),
 *     R = 1e-3, inside the stated grid;
 *   - trilinear base index floor(xi/h) clamped to [0, n-2].
 *
 * Other entry points restate, for tests only, the paper's reordered forms:
 *   orc_inspect_points      Sec. II-A.1-2 (SM / SID) and Listing 3 (src_dcmp)
 *   orc_acoustic_decomposed Listing 5: fused, reduced z2 loop (nnz_mask,
 *                           Sp_SID), unblocked
 *   orc_acoustic_wtb        Listing 6: wave-front temporal blocking over
 *                           t x x x y tiles with space blocks, skewed by the
 *                           stencil radius per in-tile step (Sec. II-B)
 *   orc_acoustic_wtb_naive  the schedule of Fig. 4b: WTB with the off-grid
 *                           injection applied when the tile holding the
 *                           source is visited (a dependence violation; used
 *                           as a negative test)
 *
 * The other two propagators of Sec. III, unblocked with direct injection:
 *   orc_tti_forward         Sec. III-B, Eq. 2: pseudo-acoustic TTI (two fields)
 *   orc_elastic_forward     Sec. III-C, Eq. 3: isotropic elastic velocity-stress
 * Parity unpinned (readings, no invariant fixes them): the edge averaging of
 * the elastic material parameters, the elastic sponge form, and which TTI
 * field the receivers sample.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

typedef struct {
  int64_t n[3];   /* grid points per axis; axis 2 is contiguous            */
  double h[3];    /* grid spacing in metres                                */
  int so;         /* space order: 4, 8 or 12                               */
  int nbl;        /* sponge width in cells (0: no damping)                 */
  int periodic;   /* 1: periodic wrap (eigenmode test only); 0: zero halo  */
  int nthreads;   /* OpenMP threads, 0 = runtime default                   */
  double dt;      /* time step in seconds                                  */
  int nt;         /* number of time steps                                  */
} orc_grid;

/* ------------------------------------------------------------------------
 * Finite-difference weights.  Fornberg's recursion (B. Fornberg, "Generation
 * of finite difference formulas on arbitrarily spaced grids", Math. Comp.
 * 1988) for the derivative of order `order` at z over the nodes x[0..np-1].
 * Output w[j] is the weight of node j.  Written from the published
 * recurrence; the tests pin it against closed rational weights.
 * ---------------------------------------------------------------------- */
static int fornberg(double z, const double* x, int np, int order, double* w) {
  /* C[j][k]: weight of node j for derivative k, k = 0..order */
  int K = order + 1;
  double* C = (double*)calloc((size_t)np * K, sizeof(double));
  if (!C) return ORC_ENOMEM;
  double c1 = 1.0, c4 = x[0] - z;
  C[0] = 1.0;
  for (int i = 1; i < np; ++i) {
    int mn = i < order ? i : order;
    double c2 = 1.0, c5 = c4;
    c4 = x[i] - z;
    for (int j = 0; j < i; ++j) {
      double c3 = x[i] - x[j];
      c2 *= c3;
      if (j == i - 1) {
        for (int k = mn; k >= 1; --k)
          C[i * K + k] = c1 * (k * C[(i - 1) * K + k - 1] - c5 * C[(i - 1) * K + k]) / c2;
        C[i * K + 0] = -c1 * c5 * C[(i - 1) * K + 0] / c2;
      }
      for (int k = mn; k >= 1; --k)
        C[j * K + k] = (c4 * C[j * K + k] - k * C[j * K + k - 1]) / c3;
      C[j * K + 0] = c4 * C[j * K + 0] / c3;
    }
    c1 = c2;
  }
  for (int j = 0; j < np; ++j) w[j] = C[j * K + order];
  free(C);
  return ORC_OK;
}

/* Centred 2nd-derivative weights c[0..r] (c[0] centre, c[i] for offsets
 * +-i), r = so/2, unit spacing. */
int orc_fd_weights_d2(int so, double* c) {
  if (so < 2 || so % 2) return ORC_EINVAL;
  int r = so / 2, np = 2 * r + 1;
  double x[64], w[64];
  for (int j = 0; j < np; ++j) x[j] = (double)(j - r);
  int st = fornberg(0.0, x, np, 2, w);
  if (st) return st;
  for (int i = 0; i <= r; ++i) c[i] = w[r + i];
  return ORC_OK;
}

/* Centred 1st-derivative weights c[1..r] (antisymmetric; c[0] = 0). */
int orc_fd_weights_d1(int so, double* c) {
  if (so < 2 || so % 2) return ORC_EINVAL;
  int r = so / 2, np = 2 * r + 1;
  double x[64], w[64];
  for (int j = 0; j < np; ++j) x[j] = (double)(j - r);
  int st = fornberg(0.0, x, np, 1, w);
  if (st) return st;
  for (int i = 0; i <= r; ++i) c[i] = w[r + i];
  return ORC_OK;
}

/* Staggered 1st-derivative weights c[1..r] for nodes at +-(i - 1/2):
 * d/dx f(0) ~ sum_i c[i] (f(i-1/2) - f(-(i-1/2))).  c[0] = 0. */
int orc_fd_weights_stag(int so, double* c) {
  if (so < 2 || so % 2) return ORC_EINVAL;
  int r = so / 2, np = 2 * r;
  double x[64], w[64];
  for (int j = 0; j < np; ++j) x[j] = (double)(j - r) + 0.5;
  int st = fornberg(0.0, x, np, 1, w);
  if (st) return st;
  c[0] = 0.0;
  for (int i = 1; i <= r; ++i) c[i] = w[r - 1 + i];
  return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Stability limit of the leapfrog scheme with the so-order Laplacian
 * (von Neumann): (v dt)^2 * S * sum_d 1/h_d^2 <= 4 where
 * S = max_theta -(c0 + 2 sum c_i cos(i theta)) = |c0 + 2 sum (-1)^i c_i|.
 * ---------------------------------------------------------------------- */
double orc_cfl_dt_max(int so, const double h[3], double vmax) {
  double c[32];
  if (orc_fd_weights_d2(so, c)) return -1.0;
  int r = so / 2;
  double S = c[0];
  for (int i = 1; i <= r; ++i) S += 2.0 * ((i % 2) ? -c[i] : c[i]);
  S = fabs(S);
  double inv = 1.0 / (h[0] * h[0]) + 1.0 / (h[1] * h[1]) + 1.0 / (h[2] * h[2]);
  return 2.0 / (vmax * sqrt(S * inv));
}

/* Sponge profile along one axis: eta[i] for i = 0..n-1 (1/s). */
void orc_damping_axis(int64_t n, int nbl, double h, double vmax, double* eta) {
  for (int64_t i = 0; i < n; ++i) eta[i] = 0.0;
  if (nbl <= 0) return;
  double eta_max = 3.0 * vmax * log(1.0 / 1e-3) / (2.0 * nbl * h);
  for (int64_t i = 0; i < n; ++i) {
    double d = 0.0;
    if (i < nbl) d = (double)(nbl - i);
    else if (i > n - 1 - nbl) d = (double)(i - (n - 1 - nbl));
    double f = d / nbl;
    eta[i] = eta_max * f * f;
  }
}

/* ------------------------------------------------------------------------
 * Padded wavefield: halo of r cells on every side.  Linear index of grid
 * point (x, y, z) is ((x + r) P1 + (y + r)) P2 + (z + r).
 * ---------------------------------------------------------------------- */
typedef struct {
  int64_t n0, n1, n2, r, P0, P1, P2, NP;
} pad_t;

static pad_t make_pad(const orc_grid* g) {
  pad_t p;
  p.n0 = g->n[0]; p.n1 = g->n[1]; p.n2 = g->n[2];
  p.r = g->so / 2;
  p.P0 = p.n0 + 2 * p.r; p.P1 = p.n1 + 2 * p.r; p.P2 = p.n2 + 2 * p.r;
  p.NP = p.P0 * p.P1 * p.P2;
  return p;
}
static inline int64_t pidx(const pad_t* p, int64_t x, int64_t y, int64_t z) {
  return ((x + p->r) * p->P1 + (y + p->r)) * p->P2 + (z + p->r);
}
static inline int64_t gidx(const pad_t* p, int64_t x, int64_t y, int64_t z) {
  return (x * p->n1 + y) * p->n2 + z;
}

/* Periodic wrap of the halo (test-only boundary). */
static void wrap_halo(const pad_t* p, double* u) {
  int64_t r = p->r;
  for (int64_t X = 0; X < p->P0; ++X)
    for (int64_t Y = 0; Y < p->P1; ++Y)
      for (int64_t Z = 0; Z < p->P2; ++Z) {
        int64_t x = X - r, y = Y - r, z = Z - r;
        int inside = x >= 0 && x < p->n0 && y >= 0 && y < p->n1 && z >= 0 && z < p->n2;
        if (inside) continue;
        int64_t xs = ((x % p->n0) + p->n0) % p->n0;
        int64_t ys = ((y % p->n1) + p->n1) % p->n1;
        int64_t zs = ((z % p->n2) + p->n2) % p->n2;
        u[(X * p->P1 + Y) * p->P2 + Z] = u[pidx(p, xs, ys, zs)];
      }
}

/* Per-problem coefficients shared by every schedule of this file. */
typedef struct {
  pad_t p;
  int r;
  double c[32];      /* centred 2nd-derivative weights                     */
  double ih2[3];     /* 1 / h_d^2                                          */
  double dt, dt2;
  double* m;         /* [N] squared slowness 1/vp^2 (unpadded)             */
  double* eta;       /* [N] damping (unpadded), 0 inside                   */
  int periodic;
} model_t;

static int model_init(model_t* M, const orc_grid* g, const double* vp, const double* eta_in) {
  memset(M, 0, sizeof(*M));
  if (g->so != 4 && g->so != 8 && g->so != 12) return ORC_EINVAL;
  M->p = make_pad(g);
  M->r = g->so / 2;
  for (int d = 0; d < 3; ++d) {
    if (g->n[d] < 2 * M->r + 2) return ORC_EINVAL;
    M->ih2[d] = 1.0 / (g->h[d] * g->h[d]);
  }
  if (orc_fd_weights_d2(g->so, M->c)) return ORC_EINVAL;
  M->dt = g->dt;
  M->dt2 = g->dt * g->dt;
  M->periodic = g->periodic;
  int64_t N = g->n[0] * g->n[1] * g->n[2];
  M->m = (double*)malloc(sizeof(double) * N);
  M->eta = (double*)malloc(sizeof(double) * N);
  if (!M->m || !M->eta) return ORC_ENOMEM;
  double vmax = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    if (!(vp[i] > 0.0)) return ORC_EINVAL;
    M->m[i] = 1.0 / (vp[i] * vp[i]);
    if (vp[i] > vmax) vmax = vp[i];
  }
  if (eta_in) {
    memcpy(M->eta, eta_in, sizeof(double) * N);
  } else {
    double* ea[3];
    for (int d = 0; d < 3; ++d) {
      ea[d] = (double*)malloc(sizeof(double) * g->n[d]);
      orc_damping_axis(g->n[d], g->nbl, g->h[d], vmax, ea[d]);
    }
    for (int64_t x = 0; x < g->n[0]; ++x)
      for (int64_t y = 0; y < g->n[1]; ++y)
        for (int64_t z = 0; z < g->n[2]; ++z)
          M->eta[gidx(&M->p, x, y, z)] = ea[0][x] + ea[1][y] + ea[2][z];
    for (int d = 0; d < 3; ++d) free(ea[d]);
  }
  return ORC_OK;
}
static void model_free(model_t* M) { free(M->m); free(M->eta); }

/* Eq. 1 at one grid point: returns u^{n+1}(x,y,z). */
static inline double point_update(const model_t* M, const double* up, const double* uc,
                                  int64_t x, int64_t y, int64_t z) {
  const pad_t* p = &M->p;
  int64_t q = pidx(p, x, y, z);
  int64_t stride[3] = {p->P1 * p->P2, p->P2, 1};
  double lap = 0.0;
  for (int d = 0; d < 3; ++d) {
    double s = M->c[0] * uc[q];
    for (int i = 1; i <= M->r; ++i) s += M->c[i] * (uc[q + i * stride[d]] + uc[q - i * stride[d]]);
    lap += s * M->ih2[d];
  }
  int64_t gq = gidx(p, x, y, z);
  double m = M->m[gq];
  double a = M->eta[gq] * M->dt * 0.5;
  return (M->dt2 * lap + m * (2.0 * uc[q] - up[q]) + a * up[q]) / (m + a);
}

/* ------------------------------------------------------------------------
 * Trilinear off-grid weights (Fig. 3, trilinear f of Sec. I).
 * ---------------------------------------------------------------------- */
static int trilinear(const orc_grid* g, const double* xyz, int64_t base[3], double frac[3]) {
  for (int d = 0; d < 3; ++d) {
    double xi = xyz[d];
    double ext = (double)(g->n[d] - 1) * g->h[d];
    if (!(xi >= 0.0) || !(xi <= ext)) return ORC_EINVAL;
    double t = xi / g->h[d];
    int64_t i = (int64_t)floor(t);
    if (i < 0) i = 0;
    if (i > g->n[d] - 2) i = g->n[d] - 2;
    base[d] = i;
    frac[d] = t - (double)i;
  }
  return ORC_OK;
}
static inline double corner_weight(const double f[3], int c) {
  double w = 1.0;
  for (int d = 0; d < 3; ++d) {
    int b = (c >> (2 - d)) & 1;
    w *= b ? f[d] : (1.0 - f[d]);
  }
  return w;
}

/* ------------------------------------------------------------------------
 * Listing 1 form: stencil sweep over the whole grid, then the sparse
 * source loop through the indirection, then the receiver interpolation.
 * ---------------------------------------------------------------------- */
int orc_acoustic_forward(const orc_grid* g, const double* vp, const double* eta,
                         int nsrc, const double* src_xyz, const double* src_wav,
                         int nrec, const double* rec_xyz, double* traces,
                         const double* u_init, const double* uprev_init,
                         double* u_out, double* uprev_out) {
  model_t M;
  int st = model_init(&M, g, vp, eta);
  if (st) { model_free(&M); return st; }
  const pad_t* p = &M.p;
  int64_t N = p->n0 * p->n1 * p->n2;
#ifdef _OPENMP
  if (g->nthreads > 0) omp_set_num_threads(g->nthreads);
#endif
  /* source / receiver corners */
  int64_t* sb = (int64_t*)malloc(sizeof(int64_t) * 3 * (nsrc > 0 ? nsrc : 1));
  double* sf = (double*)malloc(sizeof(double) * 3 * (nsrc > 0 ? nsrc : 1));
  int64_t* rb = (int64_t*)malloc(sizeof(int64_t) * 3 * (nrec > 0 ? nrec : 1));
  double* rf = (double*)malloc(sizeof(double) * 3 * (nrec > 0 ? nrec : 1));
  double* ua = (double*)calloc(p->NP, sizeof(double));
  double* ub = (double*)calloc(p->NP, sizeof(double));
  double* uc = (double*)calloc(p->NP, sizeof(double));
  if (!sb || !sf || !rb || !rf || !ua || !ub || !uc) { st = ORC_ENOMEM; goto done; }
  for (int s = 0; s < nsrc; ++s)
    if (trilinear(g, src_xyz + 3 * s, sb + 3 * s, sf + 3 * s)) { st = ORC_EINVAL; goto done; }
  for (int r = 0; r < nrec; ++r)
    if (trilinear(g, rec_xyz + 3 * r, rb + 3 * r, rf + 3 * r)) { st = ORC_EINVAL; goto done; }

  double* uprev = ua; /* u^{n-1} */
  double* ucur = ub;  /* u^n     */
  double* unext = uc; /* u^{n+1} */
  if (u_init)
    for (int64_t x = 0; x < p->n0; ++x)
      for (int64_t y = 0; y < p->n1; ++y)
        for (int64_t z = 0; z < p->n2; ++z) {
          ucur[pidx(p, x, y, z)] = u_init[gidx(p, x, y, z)];
          if (uprev_init) uprev[pidx(p, x, y, z)] = uprev_init[gidx(p, x, y, z)];
        }

  for (int n = 0; n < g->nt; ++n) {
    if (M.periodic) { wrap_halo(p, ucur); }
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < p->n0; ++x)
      for (int64_t y = 0; y < p->n1; ++y)
        for (int64_t z = 0; z < p->n2; ++z)
          unext[pidx(p, x, y, z)] = point_update(&M, uprev, ucur, x, y, z);
    /* sparse injection through the indirection (Listing 1) */
    for (int s = 0; s < nsrc; ++s) {
      double q = src_wav[(int64_t)s * g->nt + n];
      for (int c = 0; c < 8; ++c) {
        double w = corner_weight(sf + 3 * s, c);
        if (w == 0.0) continue;
        int64_t x = sb[3 * s] + ((c >> 2) & 1), y = sb[3 * s + 1] + ((c >> 1) & 1),
                z = sb[3 * s + 2] + (c & 1);
        unext[pidx(p, x, y, z)] += w * q * M.dt2 / M.m[gidx(p, x, y, z)];
      }
    }
    /* receiver interpolation of u^{n+1} */
    for (int r = 0; r < nrec; ++r) {
      double acc = 0.0;
      for (int c = 0; c < 8; ++c) {
        double w = corner_weight(rf + 3 * r, c);
        if (w == 0.0) continue;
        int64_t x = rb[3 * r] + ((c >> 2) & 1), y = rb[3 * r + 1] + ((c >> 1) & 1),
                z = rb[3 * r + 2] + (c & 1);
        acc += w * unext[pidx(p, x, y, z)];
      }
      traces[(int64_t)n * nrec + r] = acc;
    }
    double* t = uprev; uprev = ucur; ucur = unext; unext = t;
  }
  if (u_out || uprev_out)
    for (int64_t x = 0; x < p->n0; ++x)
      for (int64_t y = 0; y < p->n1; ++y)
        for (int64_t z = 0; z < p->n2; ++z) {
          if (u_out) u_out[gidx(p, x, y, z)] = ucur[pidx(p, x, y, z)];
          if (uprev_out) uprev_out[gidx(p, x, y, z)] = uprev[pidx(p, x, y, z)];
        }
  (void)N;
done:
  free(sb); free(sf); free(rb); free(rf); free(ua); free(ub); free(uc);
  model_free(&M);
  return st;
}

/* ------------------------------------------------------------------------
 * Inspector of Sec. II-A for a set of off-grid points (sources or
 * receivers).  Step 1: "inject" every point's structural weights into an
 * empty grid and keep the non-zero grid points (SM).  Step 2: give each
 * affected point a unique ascending ID (SID) in linear-index order.
 * ---------------------------------------------------------------------- */
typedef struct {
  int64_t npts;
  int64_t* lin;   /* [npts] linear index of each affected point, ascending */
  int32_t* sid;   /* [N] dense SID grid, -1 where SM = 0                   */
  uint8_t* sm;    /* [N] dense binary mask SM                              */
} inspect_t;

static int inspect_build(const orc_grid* g, int npt, const double* xyz, inspect_t* I) {
  int64_t N = g->n[0] * g->n[1] * g->n[2];
  memset(I, 0, sizeof(*I));
  I->sm = (uint8_t*)calloc(N, 1);
  I->sid = (int32_t*)malloc(sizeof(int32_t) * N);
  if (!I->sm || !I->sid) return ORC_ENOMEM;
  pad_t p = make_pad(g);
  for (int s = 0; s < npt; ++s) {
    int64_t b[3]; double f[3];
    if (trilinear(g, xyz + 3 * s, b, f)) return ORC_EINVAL;
    for (int c = 0; c < 8; ++c) {
      if (corner_weight(f, c) == 0.0) continue;
      I->sm[gidx(&p, b[0] + ((c >> 2) & 1), b[1] + ((c >> 1) & 1), b[2] + (c & 1))] = 1;
    }
  }
  int64_t cnt = 0;
  for (int64_t i = 0; i < N; ++i) cnt += I->sm[i];
  I->npts = cnt;
  I->lin = (int64_t*)malloc(sizeof(int64_t) * (cnt > 0 ? cnt : 1));
  if (!I->lin) return ORC_ENOMEM;
  int64_t id = 0;
  for (int64_t i = 0; i < N; ++i) {
    if (I->sm[i]) { I->lin[id] = i; I->sid[i] = (int32_t)id; ++id; }
    else I->sid[i] = -1;
  }
  return ORC_OK;
}
static void inspect_free(inspect_t* I) { free(I->lin); free(I->sid); free(I->sm); }

/* Listing 3: src_dcmp[t][SID(c)] += f(src(t,s)) over sources and corners,
 * with f = w * q * dt^2 / m(c) (the injection expression of Sec. III-A).
 * Contributions to one point are summed in source order. */
static int decompose_sources(const orc_grid* g, const model_t* M, const inspect_t* I, int nsrc,
                             const double* xyz, const double* wav, double* dcmp) {
  pad_t p = make_pad(g);
  memset(dcmp, 0, sizeof(double) * (size_t)g->nt * (I->npts > 0 ? I->npts : 1));
  for (int t = 0; t < g->nt; ++t)
    for (int s = 0; s < nsrc; ++s) {
      int64_t b[3]; double f[3];
      if (trilinear(g, xyz + 3 * s, b, f)) return ORC_EINVAL;
      for (int c = 0; c < 8; ++c) {
        double w = corner_weight(f, c);
        if (w == 0.0) continue;
        int64_t gq = gidx(&p, b[0] + ((c >> 2) & 1), b[1] + ((c >> 1) & 1), b[2] + (c & 1));
        dcmp[(int64_t)t * I->npts + I->sid[gq]] += w * wav[(int64_t)s * g->nt + t] * M->dt2 / M->m[gq];
      }
    }
  return ORC_OK;
}

/* Public form of the inspector, for comparing tables in the tests:
 * returns npts, the ascending linear indices of the affected points, and
 * (if dcmp != NULL) the decomposition table [nt][npts]. Call once with
 * lin == NULL to get npts. */
int orc_inspect_points(const orc_grid* g, const double* vp, int npt, const double* xyz,
                       const double* wav, int64_t* npts_out, int64_t* lin, double* dcmp) {
  inspect_t I;
  int st = inspect_build(g, npt, xyz, &I);
  if (st) { inspect_free(&I); return st; }
  *npts_out = I.npts;
  if (lin) memcpy(lin, I.lin, sizeof(int64_t) * I.npts);
  if (dcmp && wav) {
    model_t M;
    st = model_init(&M, g, vp, NULL);
    if (!st) st = decompose_sources(g, &M, &I, npt, xyz, wav, dcmp);
    model_free(&M);
  }
  inspect_free(&I);
  return st;
}

/* Iteration-space reduction of Sec. II-A.4: nnz_mask[x][y] = number of
 * affected z in column (x, y); Sp_SID[x][y][k] = k-th affected z. */
typedef struct {
  int32_t* nnz;   /* [n0*n1]                 */
  int64_t* off;   /* [n0*n1 + 1] into zind   */
  int32_t* zind;  /* [npts]                  */
} columns_t;

static int columns_build(const orc_grid* g, const inspect_t* I, columns_t* C) {
  int64_t n0 = g->n[0], n1 = g->n[1], n2 = g->n[2];
  C->nnz = (int32_t*)calloc(n0 * n1, sizeof(int32_t));
  C->off = (int64_t*)calloc(n0 * n1 + 1, sizeof(int64_t));
  C->zind = (int32_t*)malloc(sizeof(int32_t) * (I->npts > 0 ? I->npts : 1));
  if (!C->nnz || !C->off || !C->zind) return ORC_ENOMEM;
  for (int64_t xy = 0; xy < n0 * n1; ++xy) {
    C->off[xy] = (xy ? C->off[xy - 1] + C->nnz[xy - 1] : 0);
    for (int64_t z = 0; z < n2; ++z)
      if (I->sm[xy * n2 + z]) C->zind[C->off[xy] + C->nnz[xy]++] = (int32_t)z;
  }
  C->off[n0 * n1] = C->off[n0 * n1 - 1] + C->nnz[n0 * n1 - 1];
  return ORC_OK;
}
static void columns_free(columns_t* C) { free(C->nnz); free(C->off); free(C->zind); }

/* State of the decomposed (grid-aligned) schedules. */
typedef struct {
  model_t M;
  inspect_t S, R;       /* source and receiver inspections            */
  columns_t SC, RC;     /* their column structures                    */
  double* src_dcmp;     /* [nt][S.npts]                               */
  double* rec_dcmp;     /* [nt][R.npts] u^{n+1} at receiver points    */
  int64_t* rb; double* rf; int nrec;
  double* buf[2];       /* padded wavefields, time level t in buf[t&1] */
} dcmp_t;

static void dcmp_free(dcmp_t* D) {
  model_free(&D->M);
  inspect_free(&D->S); inspect_free(&D->R);
  columns_free(&D->SC); columns_free(&D->RC);
  free(D->src_dcmp); free(D->rec_dcmp); free(D->rb); free(D->rf);
  free(D->buf[0]); free(D->buf[1]);
}

static int dcmp_init(dcmp_t* D, const orc_grid* g, const double* vp, const double* eta,
                     int nsrc, const double* src_xyz, const double* src_wav,
                     int nrec, const double* rec_xyz) {
  memset(D, 0, sizeof(*D));
  int st = model_init(&D->M, g, vp, eta);
  if (st) return st;
  if ((st = inspect_build(g, nsrc, src_xyz, &D->S))) return st;
  if ((st = inspect_build(g, nrec, rec_xyz, &D->R))) return st;
  if ((st = columns_build(g, &D->S, &D->SC))) return st;
  if ((st = columns_build(g, &D->R, &D->RC))) return st;
  D->src_dcmp = (double*)malloc(sizeof(double) * (size_t)g->nt * (D->S.npts > 0 ? D->S.npts : 1));
  D->rec_dcmp = (double*)calloc((size_t)g->nt * (D->R.npts > 0 ? D->R.npts : 1), sizeof(double));
  D->rb = (int64_t*)malloc(sizeof(int64_t) * 3 * (nrec > 0 ? nrec : 1));
  D->rf = (double*)malloc(sizeof(double) * 3 * (nrec > 0 ? nrec : 1));
  D->buf[0] = (double*)calloc(D->M.p.NP, sizeof(double));
  D->buf[1] = (double*)calloc(D->M.p.NP, sizeof(double));
  if (!D->src_dcmp || !D->rec_dcmp || !D->rb || !D->rf || !D->buf[0] || !D->buf[1]) return ORC_ENOMEM;
  if ((st = decompose_sources(g, &D->M, &D->S, nsrc, src_xyz, src_wav, D->src_dcmp))) return st;
  D->nrec = nrec;
  for (int r = 0; r < nrec; ++r)
    if (trilinear(g, rec_xyz + 3 * r, D->rb + 3 * r, D->rf + 3 * r)) return ORC_EINVAL;
  return ORC_OK;
}

/* Listing 5 body for one column (x, y) at time t: the stencil z loop,
 * then the reduced z2 loop over nnz_mask[x][y] affected points, then the
 * mirrored receiver loop that records u^{t+1} at receiver points. */
static inline void column_update(dcmp_t* D, const orc_grid* g, int t, int64_t x, int64_t y) {
  const pad_t* p = &D->M.p;
  double* unew = D->buf[(t + 1) & 1];  /* holds u^{t-1}, overwritten in place */
  const double* ucur = D->buf[t & 1];
  for (int64_t z = 0; z < p->n2; ++z)
    unew[pidx(p, x, y, z)] = point_update(&D->M, unew, ucur, x, y, z);
  int64_t xy = x * p->n1 + y;
  for (int32_t k = 0; k < D->SC.nnz[xy]; ++k) {
    int64_t zind = D->SC.zind[D->SC.off[xy] + k];
    unew[pidx(p, x, y, zind)] += D->src_dcmp[(int64_t)t * D->S.npts + D->S.sid[xy * p->n2 + zind]];
  }
  for (int32_t k = 0; k < D->RC.nnz[xy]; ++k) {
    int64_t zind = D->RC.zind[D->RC.off[xy] + k];
    D->rec_dcmp[(int64_t)t * D->R.npts + D->R.sid[xy * p->n2 + zind]] = unew[pidx(p, x, y, zind)];
  }
  (void)g;
}

/* Receiver traces from the recorded receiver-point series. */
static void finalize_traces(dcmp_t* D, const orc_grid* g, double* traces) {
  pad_t p = make_pad(g);
  for (int t = 0; t < g->nt; ++t)
    for (int r = 0; r < D->nrec; ++r) {
      double acc = 0.0;
      for (int c = 0; c < 8; ++c) {
        double w = corner_weight(D->rf + 3 * r, c);
        if (w == 0.0) continue;
        int64_t gq = gidx(&p, D->rb[3 * r] + ((c >> 2) & 1), D->rb[3 * r + 1] + ((c >> 1) & 1),
                          D->rb[3 * r + 2] + (c & 1));
        acc += w * D->rec_dcmp[(int64_t)t * D->R.npts + D->R.sid[gq]];
      }
      traces[(int64_t)t * D->nrec + r] = acc;
    }
}

static void copy_out(const dcmp_t* D, const orc_grid* g, double* u_out, double* uprev_out) {
  const pad_t* p = &D->M.p;
  const double* un = D->buf[g->nt & 1];
  const double* upr = D->buf[(g->nt + 1) & 1];
  for (int64_t x = 0; x < p->n0; ++x)
    for (int64_t y = 0; y < p->n1; ++y)
      for (int64_t z = 0; z < p->n2; ++z) {
        if (u_out) u_out[gidx(p, x, y, z)] = un[pidx(p, x, y, z)];
        if (uprev_out) uprev_out[gidx(p, x, y, z)] = upr[pidx(p, x, y, z)];
      }
}

/* Listing 5: unblocked, fused and reduced injection (zero halo only). */
int orc_acoustic_decomposed(const orc_grid* g, const double* vp, const double* eta,
                            int nsrc, const double* src_xyz, const double* src_wav,
                            int nrec, const double* rec_xyz, double* traces,
                            double* u_out, double* uprev_out) {
  if (g->periodic) return ORC_EINVAL;
  dcmp_t D;
  int st = dcmp_init(&D, g, vp, eta, nsrc, src_xyz, src_wav, nrec, rec_xyz);
  if (st) { dcmp_free(&D); return st; }
#ifdef _OPENMP
  if (g->nthreads > 0) omp_set_num_threads(g->nthreads);
#endif
  for (int t = 0; t < g->nt; ++t) {
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < D.M.p.n0; ++x)
      for (int64_t y = 0; y < D.M.p.n1; ++y) column_update(&D, g, t, x, y);
  }
  if (traces) finalize_traces(&D, g, traces);
  copy_out(&D, g, u_out, uprev_out);
  dcmp_free(&D);
  return ORC_OK;
}

/* Listing 6: wave-front temporal blocking.  Time tiles of depth tt; space
 * tiles tile_x x tile_y in (x, y); inside a tile and a time step, blocks of
 * block_x x block_y (independent, run in parallel).  The tile origin moves
 * back by the stencil radius r at every in-tile step (the wave-front angle
 * of Sec. II-B), which with two in-place time buffers keeps every flow and
 * anti-dependence of the unblocked order.
 *
 * naive != 0 gives the schedule of Fig. 4b: the fused grid-aligned injection
 * is replaced by the off-grid Listing-1 injection of every source, applied
 * right after the block that contains the source's base corner is updated;
 * corners in blocks not yet updated at that time step receive the impulse
 * too early (a dependence violation the tests must detect). */
static int wtb_run(const orc_grid* g, const double* vp, const double* eta,
                   int nsrc, const double* src_xyz, const double* src_wav,
                   int nrec, const double* rec_xyz, double* traces,
                   double* u_out, double* uprev_out,
                   int tt, int tile_x, int tile_y, int block_x, int block_y, int naive) {
  if (g->periodic || tt < 1 || tile_x < 1 || tile_y < 1 || block_x < 1 || block_y < 1) return ORC_EINVAL;
  dcmp_t D;
  int st = dcmp_init(&D, g, vp, eta, nsrc, src_xyz, src_wav, nrec, rec_xyz);
  if (st) { dcmp_free(&D); return st; }
  int64_t* sb = NULL; double* sf = NULL;
  if (naive) {
    sb = (int64_t*)malloc(sizeof(int64_t) * 3 * (nsrc > 0 ? nsrc : 1));
    sf = (double*)malloc(sizeof(double) * 3 * (nsrc > 0 ? nsrc : 1));
    for (int s = 0; s < nsrc; ++s) trilinear(g, src_xyz + 3 * s, sb + 3 * s, sf + 3 * s);
  }
#ifdef _OPENMP
  if (g->nthreads > 0) omp_set_num_threads(g->nthreads);
#endif
  const pad_t* p = &D.M.p;
  int64_t r = D.M.r;
  int64_t nxt = (p->n0 + (int64_t)(tt - 1) * r + tile_x - 1) / tile_x;
  int64_t nyt = (p->n1 + (int64_t)(tt - 1) * r + tile_y - 1) / tile_y;
  for (int t0 = 0; t0 < g->nt; t0 += tt) {
    int t1 = t0 + tt < g->nt ? t0 + tt : g->nt;
    for (int64_t X = 0; X < nxt; ++X)
      for (int64_t Y = 0; Y < nyt; ++Y)
        for (int t = t0; t < t1; ++t) {
          int64_t s = t - t0;
          int64_t xa = X * tile_x - s * r, xb = xa + tile_x;
          int64_t ya = Y * tile_y - s * r, yb = ya + tile_y;
          if (xa < 0) xa = 0;
          if (ya < 0) ya = 0;
          if (xb > p->n0) xb = p->n0;
          if (yb > p->n1) yb = p->n1;
          if (xa >= xb || ya >= yb) continue;
          int64_t nbx = (xb - xa + block_x - 1) / block_x, nby = (yb - ya + block_y - 1) / block_y;
#pragma omp parallel for schedule(dynamic) collapse(2) if (!naive)
          for (int64_t bx = 0; bx < nbx; ++bx)
            for (int64_t by = 0; by < nby; ++by) {
              int64_t x0 = xa + bx * block_x, x1 = x0 + block_x < xb ? x0 + block_x : xb;
              int64_t y0 = ya + by * block_y, y1 = y0 + block_y < yb ? y0 + block_y : yb;
              for (int64_t x = x0; x < x1; ++x)
                for (int64_t y = y0; y < y1; ++y) {
                  if (!naive) { column_update(&D, g, t, x, y); continue; }
                  double* unew = D.buf[(t + 1) & 1];
                  const double* ucur = D.buf[t & 1];
                  for (int64_t z = 0; z < p->n2; ++z)
                    unew[pidx(p, x, y, z)] = point_update(&D.M, unew, ucur, x, y, z);
                }
              if (naive) {
                /* off-grid injection when the source's home block is done */
                double* unew = D.buf[(t + 1) & 1];
                for (int si = 0; si < nsrc; ++si) {
                  if (sb[3 * si] < x0 || sb[3 * si] >= x1 || sb[3 * si + 1] < y0 || sb[3 * si + 1] >= y1) continue;
                  double q = src_wav[(int64_t)si * g->nt + t];
                  for (int c = 0; c < 8; ++c) {
                    double w = corner_weight(sf + 3 * si, c);
                    if (w == 0.0) continue;
                    int64_t cx = sb[3 * si] + ((c >> 2) & 1), cy = sb[3 * si + 1] + ((c >> 1) & 1),
                            cz = sb[3 * si + 2] + (c & 1);
                    unew[pidx(p, cx, cy, cz)] += w * q * D.M.dt2 / D.M.m[gidx(p, cx, cy, cz)];
                  }
                }
              }
            }
        }
  }
  if (traces && !naive) finalize_traces(&D, g, traces);
  copy_out(&D, g, u_out, uprev_out);
  free(sb); free(sf);
  dcmp_free(&D);
  return ORC_OK;
}

int orc_acoustic_wtb(const orc_grid* g, const double* vp, const double* eta,
                     int nsrc, const double* src_xyz, const double* src_wav,
                     int nrec, const double* rec_xyz, double* traces,
                     double* u_out, double* uprev_out,
                     int tt, int tile_x, int tile_y, int block_x, int block_y) {
  return wtb_run(g, vp, eta, nsrc, src_xyz, src_wav, nrec, rec_xyz, traces, u_out, uprev_out,
                 tt, tile_x, tile_y, block_x, block_y, 0);
}

int orc_acoustic_wtb_naive(const orc_grid* g, const double* vp, const double* eta,
                           int nsrc, const double* src_xyz, const double* src_wav,
                           double* u_out, double* uprev_out,
                           int tt, int tile_x, int tile_y, int block_x, int block_y) {
  return wtb_run(g, vp, eta, nsrc, src_xyz, src_wav, 0, NULL, NULL, u_out, uprev_out,
                 tt, tile_x, tile_y, block_x, block_y, 1);
}

/* Discrete energy of the leapfrog scheme without damping:
 * E^{n+1/2} = sum m ((u^{n+1}-u^n)/dt)^2 - sum u^{n+1} (L u^n).
 * Inputs are unpadded; zero halo. */
double orc_acoustic_energy(const orc_grid* g, const double* vp, const double* u_next,
                           const double* u_cur) {
  model_t M;
  orc_grid g2 = *g;
  g2.nbl = 0;
  if (model_init(&M, &g2, vp, NULL)) { model_free(&M); return NAN; }
  const pad_t* p = &M.p;
  double* uc = (double*)calloc(p->NP, sizeof(double));
  for (int64_t x = 0; x < p->n0; ++x)
    for (int64_t y = 0; y < p->n1; ++y)
      for (int64_t z = 0; z < p->n2; ++z) uc[pidx(p, x, y, z)] = u_cur[gidx(p, x, y, z)];
  if (M.periodic) wrap_halo(p, uc);
  int64_t stride[3] = {p->P1 * p->P2, p->P2, 1};
  double kin = 0.0, pot = 0.0;
  for (int64_t x = 0; x < p->n0; ++x)
    for (int64_t y = 0; y < p->n1; ++y)
      for (int64_t z = 0; z < p->n2; ++z) {
        int64_t q = pidx(p, x, y, z), gq = gidx(p, x, y, z);
        double lap = 0.0;
        for (int d = 0; d < 3; ++d) {
          double s = M.c[0] * uc[q];
          for (int i = 1; i <= M.r; ++i) s += M.c[i] * (uc[q + i * stride[d]] + uc[q - i * stride[d]]);
          lap += s * M.ih2[d];
        }
        double v = (u_next[gq] - u_cur[gq]) / M.dt;
        kin += M.m[gq] * v * v;
        pot += u_next[gq] * lap;
      }
  free(uc);
  model_free(&M);
  return kin - pot;
}

/* =========================================================================
 * Shared helpers of the TTI and elastic oracles: padded copies and the
 * maximum of a trigonometric symbol (for the stability limits).
 * ======================================================================= */
static void to_padded(const pad_t* p, const double* src, double* dst) {
  for (int64_t x = 0; x < p->n0; ++x)
    for (int64_t y = 0; y < p->n1; ++y)
      for (int64_t z = 0; z < p->n2; ++z) dst[pidx(p, x, y, z)] = src[gidx(p, x, y, z)];
}
static void from_padded(const pad_t* p, const double* src, double* dst) {
  for (int64_t x = 0; x < p->n0; ++x)
    for (int64_t y = 0; y < p->n1; ++y)
      for (int64_t z = 0; z < p->n2; ++z) dst[gidx(p, x, y, z)] = src[pidx(p, x, y, z)];
}
/* max over theta in [0, pi] of |2 sum_i c[i] sin((i - shift) theta)|, by
 * dense sampling (the symbols are smooth; 2e5 samples). */
static double symbol_max(const double* c, int r, double shift) {
  double best = 0.0;
  const int ns = 200000;
  for (int s = 0; s <= ns; ++s) {
    double th = M_PI * (double)s / ns, v = 0.0;
    for (int i = 1; i <= r; ++i) v += c[i] * sin(((double)i - shift) * th);
    v = fabs(2.0 * v);
    if (v > best) best = v;
  }
  return best;
}

/* =========================================================================
 * Anisotropic pseudo-acoustic (TTI) propagator, Sec. III-B.
 *
 * Eq. 2 gives the rotated first derivative
 *   D_xbar = cos t cos f d/dx + cos t sin f d/dy - sin t d/dz
 * (t = theta, tilt; f = phi, azimuth).  The paper does not print the full
 * system; this oracle takes the self-adjoint pseudo-acoustic system of the
 * work it cites for it (Zhang, Zhang and Zhang 2011):
 *   m p_tt = (1 + 2 eps) H_h p + sqrt(1 + 2 delta) H_z r
 *   m r_tt = sqrt(1 + 2 delta) H_h p + H_z r
 *   H_h = -(D_xbar^T D_xbar + D_ybar^T D_ybar),   H_z = -D_zbar^T D_zbar
 * on the orthonormal frame completing Eq. 2 (axis order x, y, z = 0, 1, 2):
 *   xbar = ( cos t cos f,  cos t sin f, -sin t)
 *   ybar = (-sin f,        cos f,        0    )
 *   zbar = ( sin t cos f,  sin t sin f,  cos t)
 * Discretisation: D_nbar u (p) = sum_d nbar_d(p) (Dc_d u)(p), Dc_d the centred
 * first derivative of order so with the field zero outside the grid.  Its
 * transpose is -sum_d Dc_d (nbar_d .), so
 *   H_h p = sum_d Dc_d F_d,  F = xbar (xbar . Dc p) + ybar (ybar . Dc p)
 *   H_z r = sum_d Dc_d G_d,  G = zbar (zbar . Dc r)
 * with the fluxes F, G zero outside the grid.  Each field is stepped like
 * Eq. 1 (same leapfrog, damping and dt^2/m source scaling); sources are
 * injected into p and r alike, receivers sample p.
 * ======================================================================= */
typedef struct {
  pad_t p;
  int r;
  double a[32];     /* centred 1st-derivative weights a[1..r], unit spacing */
  double ih[3];     /* 1 / h_d */
  double dt, dt2;
  double *m, *eta, *cpp, *cpr;   /* [N]: 1/vp^2, damping, 1+2eps, sqrt(1+2delta) */
  double *nx, *ny, *nz;          /* [3][N] frame vectors xbar, ybar, zbar       */
  int periodic;
} tti_t;

static void tti_free(tti_t* T) {
  free(T->m); free(T->eta); free(T->cpp); free(T->cpr);
  free(T->nx); free(T->ny); free(T->nz);
}

static int tti_init(tti_t* T, const orc_grid* g, const double* vp, const double* eps,
                    const double* delta, const double* theta, const double* phi,
                    const double* eta_in) {
  memset(T, 0, sizeof(*T));
  if (g->so != 4 && g->so != 8 && g->so != 12) return ORC_EINVAL;
  T->p = make_pad(g);
  T->r = g->so / 2;
  for (int d = 0; d < 3; ++d) {
    if (g->n[d] < 2 * T->r + 2) return ORC_EINVAL;
    T->ih[d] = 1.0 / g->h[d];
  }
  if (orc_fd_weights_d1(g->so, T->a)) return ORC_EINVAL;
  T->dt = g->dt;
  T->dt2 = g->dt * g->dt;
  T->periodic = g->periodic;
  int64_t N = g->n[0] * g->n[1] * g->n[2];
  T->m = (double*)malloc(sizeof(double) * N);
  T->eta = (double*)malloc(sizeof(double) * N);
  T->cpp = (double*)malloc(sizeof(double) * N);
  T->cpr = (double*)malloc(sizeof(double) * N);
  T->nx = (double*)malloc(sizeof(double) * 3 * N);
  T->ny = (double*)malloc(sizeof(double) * 3 * N);
  T->nz = (double*)malloc(sizeof(double) * 3 * N);
  if (!T->m || !T->eta || !T->cpp || !T->cpr || !T->nx || !T->ny || !T->nz) return ORC_ENOMEM;
  double vmax = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    if (!(vp[i] > 0.0)) return ORC_EINVAL;
    if (!(eps[i] >= delta[i]) || !(delta[i] > -0.5)) return ORC_EINVAL; /* C must be PSD */
    T->m[i] = 1.0 / (vp[i] * vp[i]);
    T->cpp[i] = 1.0 + 2.0 * eps[i];
    T->cpr[i] = sqrt(1.0 + 2.0 * delta[i]);
    double ct = cos(theta[i]), st = sin(theta[i]), cf = cos(phi[i]), sf = sin(phi[i]);
    T->nx[i] = ct * cf; T->nx[N + i] = ct * sf; T->nx[2 * N + i] = -st;
    T->ny[i] = -sf;     T->ny[N + i] = cf;      T->ny[2 * N + i] = 0.0;
    T->nz[i] = st * cf; T->nz[N + i] = st * sf; T->nz[2 * N + i] = ct;
    if (vp[i] > vmax) vmax = vp[i];
  }
  if (eta_in) {
    memcpy(T->eta, eta_in, sizeof(double) * N);
  } else {
    double* ea[3];
    for (int d = 0; d < 3; ++d) {
      ea[d] = (double*)malloc(sizeof(double) * g->n[d]);
      orc_damping_axis(g->n[d], g->nbl, g->h[d], vmax, ea[d]);
    }
    for (int64_t x = 0; x < g->n[0]; ++x)
      for (int64_t y = 0; y < g->n[1]; ++y)
        for (int64_t z = 0; z < g->n[2]; ++z)
          T->eta[gidx(&T->p, x, y, z)] = ea[0][x] + ea[1][y] + ea[2][z];
    for (int d = 0; d < 3; ++d) free(ea[d]);
  }
  return ORC_OK;
}

/* centred first derivative along axis d of a padded field at padded index q */
static inline double tti_dc(const tti_t* T, const double* u, int64_t q, int d) {
  const pad_t* p = &T->p;
  int64_t s = d == 0 ? p->P1 * p->P2 : (d == 1 ? p->P2 : 1);
  double acc = 0.0;
  for (int i = 1; i <= T->r; ++i) acc += T->a[i] * (u[q + i * s] - u[q - i * s]);
  return acc * T->ih[d];
}

/* Hh = H_h p and Hz = H_z r ([N], unpadded) from padded p, r (halos already
 * zero or wrapped).  F[3], G[3] are padded scratch fields whose halos are
 * zero on entry. */
static void tti_apply(const tti_t* T, const double* pc, const double* rc, double* F[3],
                      double* G[3], double* Hh, double* Hz) {
  const pad_t* p = &T->p;
  const int64_t N = p->n0 * p->n1 * p->n2;
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < p->n0; ++x)
    for (int64_t y = 0; y < p->n1; ++y)
      for (int64_t z = 0; z < p->n2; ++z) {
        int64_t q = pidx(p, x, y, z), gq = gidx(p, x, y, z);
        double gp[3], gr[3];
        for (int d = 0; d < 3; ++d) {
          gp[d] = tti_dc(T, pc, q, d);
          gr[d] = tti_dc(T, rc, q, d);
        }
        double ax = 0.0, ay = 0.0, bz = 0.0;
        for (int d = 0; d < 3; ++d) {
          ax += T->nx[d * N + gq] * gp[d];
          ay += T->ny[d * N + gq] * gp[d];
          bz += T->nz[d * N + gq] * gr[d];
        }
        for (int d = 0; d < 3; ++d) {
          F[d][q] = T->nx[d * N + gq] * ax + T->ny[d * N + gq] * ay;
          G[d][q] = T->nz[d * N + gq] * bz;
        }
      }
  if (T->periodic)
    for (int d = 0; d < 3; ++d) { wrap_halo(p, F[d]); wrap_halo(p, G[d]); }
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < p->n0; ++x)
    for (int64_t y = 0; y < p->n1; ++y)
      for (int64_t z = 0; z < p->n2; ++z) {
        int64_t q = pidx(p, x, y, z), gq = gidx(p, x, y, z);
        double hh = 0.0, hz = 0.0;
        for (int d = 0; d < 3; ++d) {
          hh += tti_dc(T, F[d], q, d);
          hz += tti_dc(T, G[d], q, d);
        }
        Hh[gq] = hh;
        Hz[gq] = hz;
      }
}

/* Stability limit of the TTI leapfrog: the largest eigenvalue of the
 * per-point 2x2 system is at most (1 + 2 eps) |s|^2 when eps >= delta, with
 * |s_d| <= S1/h_d, S1 = max |2 sum a_i sin(i theta)| (centred 1st
 * derivative), so dt_max = 2 / (vmax sqrt(1 + 2 eps_max) sqrt(sum (S1/h_d)^2)). */
double orc_tti_dt_max(int so, const double h[3], double vmax, double eps_max) {
  double a[32];
  if (orc_fd_weights_d1(so, a)) return -1.0;
  double S1 = symbol_max(a, so / 2, 0.0);
  double s2 = 0.0;
  for (int d = 0; d < 3; ++d) s2 += (S1 / h[d]) * (S1 / h[d]);
  return 2.0 / (vmax * sqrt((1.0 + 2.0 * eps_max) * s2));
}

/* init: NULL or [4][N] = p^0, p^{-1}, r^0, r^{-1}; out: NULL or [4][N] =
 * p^{nt}, p^{nt-1}, r^{nt}, r^{nt-1}; traces [nt][nrec] sample p^{n+1}. */
int orc_tti_forward(const orc_grid* g, const double* vp, const double* eps, const double* delta,
                    const double* theta, const double* phi, const double* eta, int nsrc,
                    const double* src_xyz, const double* src_wav, int nrec, const double* rec_xyz,
                    double* traces, const double* init, double* out) {
  tti_t T;
  int st = tti_init(&T, g, vp, eps, delta, theta, phi, eta);
  if (st) { tti_free(&T); return st; }
  const pad_t* p = &T.p;
  const int64_t N = p->n0 * p->n1 * p->n2;
#ifdef _OPENMP
  if (g->nthreads > 0) omp_set_num_threads(g->nthreads);
#endif
  int64_t* sb = (int64_t*)malloc(sizeof(int64_t) * 3 * (nsrc > 0 ? nsrc : 1));
  double* sf = (double*)malloc(sizeof(double) * 3 * (nsrc > 0 ? nsrc : 1));
  int64_t* rb = (int64_t*)malloc(sizeof(int64_t) * 3 * (nrec > 0 ? nrec : 1));
  double* rf = (double*)malloc(sizeof(double) * 3 * (nrec > 0 ? nrec : 1));
  double* buf = (double*)calloc((size_t)p->NP * 12, sizeof(double));
  double* Hh = (double*)malloc(sizeof(double) * N);
  double* Hz = (double*)malloc(sizeof(double) * N);
  if (!sb || !sf || !rb || !rf || !buf || !Hh || !Hz) { st = ORC_ENOMEM; goto done; }
  for (int s = 0; s < nsrc; ++s)
    if (trilinear(g, src_xyz + 3 * s, sb + 3 * s, sf + 3 * s)) { st = ORC_EINVAL; goto done; }
  for (int r = 0; r < nrec; ++r)
    if (trilinear(g, rec_xyz + 3 * r, rb + 3 * r, rf + 3 * r)) { st = ORC_EINVAL; goto done; }
  {
    double* pp = buf;                 /* p^{n-1} */
    double* pc = buf + p->NP;         /* p^n     */
    double* pn = buf + 2 * p->NP;     /* p^{n+1} */
    double* rp = buf + 3 * p->NP;
    double* rc = buf + 4 * p->NP;
    double* rn = buf + 5 * p->NP;
    double* F[3] = {buf + 6 * p->NP, buf + 7 * p->NP, buf + 8 * p->NP};
    double* G[3] = {buf + 9 * p->NP, buf + 10 * p->NP, buf + 11 * p->NP};
    if (init) {
      to_padded(p, init, pc);
      to_padded(p, init + N, pp);
      to_padded(p, init + 2 * N, rc);
      to_padded(p, init + 3 * N, rp);
    }
    for (int n = 0; n < g->nt; ++n) {
      if (T.periodic) { wrap_halo(p, pc); wrap_halo(p, rc); }
      tti_apply(&T, pc, rc, F, G, Hh, Hz);
#pragma omp parallel for schedule(static)
      for (int64_t x = 0; x < p->n0; ++x)
        for (int64_t y = 0; y < p->n1; ++y)
          for (int64_t z = 0; z < p->n2; ++z) {
            int64_t q = pidx(p, x, y, z), gq = gidx(p, x, y, z);
            double m = T.m[gq], a = T.eta[gq] * T.dt * 0.5;
            double rhs_p = T.cpp[gq] * Hh[gq] + T.cpr[gq] * Hz[gq];
            double rhs_r = T.cpr[gq] * Hh[gq] + Hz[gq];
            pn[q] = (T.dt2 * rhs_p + m * (2.0 * pc[q] - pp[q]) + a * pp[q]) / (m + a);
            rn[q] = (T.dt2 * rhs_r + m * (2.0 * rc[q] - rp[q]) + a * rp[q]) / (m + a);
          }
      for (int s = 0; s < nsrc; ++s) {
        double qv = src_wav[(int64_t)s * g->nt + n];
        for (int c = 0; c < 8; ++c) {
          double w = corner_weight(sf + 3 * s, c);
          if (w == 0.0) continue;
          int64_t x = sb[3 * s] + ((c >> 2) & 1), y = sb[3 * s + 1] + ((c >> 1) & 1),
                  z = sb[3 * s + 2] + (c & 1);
          double add = w * qv * T.dt2 / T.m[gidx(p, x, y, z)];
          pn[pidx(p, x, y, z)] += add;
          rn[pidx(p, x, y, z)] += add;
        }
      }
      for (int r = 0; r < nrec; ++r) {
        double acc = 0.0;
        for (int c = 0; c < 8; ++c) {
          double w = corner_weight(rf + 3 * r, c);
          if (w == 0.0) continue;
          int64_t x = rb[3 * r] + ((c >> 2) & 1), y = rb[3 * r + 1] + ((c >> 1) & 1),
                  z = rb[3 * r + 2] + (c & 1);
          acc += w * pn[pidx(p, x, y, z)];
        }
        traces[(int64_t)n * nrec + r] = acc;
      }
      double* t = pp; pp = pc; pc = pn; pn = t;
      t = rp; rp = rc; rc = rn; rn = t;
    }
    if (out) {
      from_padded(p, pc, out);
      from_padded(p, pp, out + N);
      from_padded(p, rc, out + 2 * N);
      from_padded(p, rp, out + 3 * N);
    }
  }
done:
  free(sb); free(sf); free(rb); free(rf); free(buf); free(Hh); free(Hz);
  tti_free(&T);
  return st;
}

/* Discrete energy of the undamped TTI leapfrog (eps > delta everywhere):
 *   E^{n+1/2} = sum_pts D^T (m C^{-1}) D / dt^2 - (p^{n+1}.H_h p^n + r^{n+1}.H_z r^n)
 * with D = (p^{n+1} - p^n, r^{n+1} - r^n) and C = [[1+2eps, s], [s, 1]],
 * s = sqrt(1+2delta).  Constant in n for a symmetric H (no source). */
double orc_tti_energy(const orc_grid* g, const double* vp, const double* eps, const double* delta,
                      const double* theta, const double* phi, const double* p_next,
                      const double* p_cur, const double* r_next, const double* r_cur) {
  tti_t T;
  orc_grid g2 = *g;
  g2.nbl = 0;
  if (tti_init(&T, &g2, vp, eps, delta, theta, phi, NULL)) { tti_free(&T); return NAN; }
  const pad_t* p = &T.p;
  const int64_t N = p->n0 * p->n1 * p->n2;
  double* buf = (double*)calloc((size_t)p->NP * 8, sizeof(double));
  double* Hh = (double*)malloc(sizeof(double) * N);
  double* Hz = (double*)malloc(sizeof(double) * N);
  double E = NAN;
  if (buf && Hh && Hz) {
    double* pc = buf;
    double* rc = buf + p->NP;
    double* F[3] = {buf + 2 * p->NP, buf + 3 * p->NP, buf + 4 * p->NP};
    double* G[3] = {buf + 5 * p->NP, buf + 6 * p->NP, buf + 7 * p->NP};
    to_padded(p, p_cur, pc);
    to_padded(p, r_cur, rc);
    if (T.periodic) { wrap_halo(p, pc); wrap_halo(p, rc); }
    tti_apply(&T, pc, rc, F, G, Hh, Hz);
    double kin = 0.0, pot = 0.0;
    for (int64_t i = 0; i < N; ++i) {
      double a = T.cpp[i], s = T.cpr[i], det = a - s * s;
      double dp = (p_next[i] - p_cur[i]) / T.dt, dr = (r_next[i] - r_cur[i]) / T.dt;
      kin += T.m[i] * (dp * dp - 2.0 * s * dp * dr + a * dr * dr) / det;
      pot += p_next[i] * Hh[i] + r_next[i] * Hz[i];
    }
    E = kin - pot;
  }
  free(buf); free(Hh); free(Hz);
  tti_free(&T);
  return E;
}

/* =========================================================================
 * Isotropic elastic velocity-stress propagator, Eq. 3 (Sec. III-C).
 *
 * Standard staggered grid (Virieux 1986, which the paper cites):
 *   vx (i+1/2, j, k)   vy (i, j+1/2, k)   vz (i, j, k+1/2)
 *   txx, tyy, tzz (i, j, k)
 *   txy (i+1/2, j+1/2, k)   txz (i+1/2, j, k+1/2)   tyz (i, j+1/2, k+1/2)
 * Every field is an n0 x n1 x n2 array (index i of a half-node stands for
 * i + 1/2) and is zero outside it.  Staggered derivatives of order so with
 * the weights c_k of nodes at +-(k - 1/2):
 *   Dp_d f (i) = sum_k c_k (f[i+k] - f[i-k+1]) / h_d    (node -> half-node)
 *   Dm_d g (i) = sum_k c_k (g[i+k-1] - g[i-k]) / h_d    (half-node -> node)
 * (Dp^T = -Dm on these arrays, which makes the scheme energy conserving).
 * One time step n (v at n-1/2 -> n+1/2, stresses at n -> n+1):
 *   vx += dt bx (Dp_x txx + Dm_y txy + Dm_z txz)
 *   vy += dt by (Dm_x txy + Dp_y tyy + Dm_z tyz)
 *   vz += dt bz (Dm_x txz + Dm_y tyz + Dp_z tzz)
 *   tii += dt (lam tr(e) + 2 mu e_ii),  e_ii = Dm_i v_i
 *   txy += dt mu_xy (Dp_y vx + Dp_x vy), and likewise txz, tyz
 * with b = 1/rho, lam = rho (vp^2 - 2 vs^2), mu = rho vs^2; b at a half-node
 * is the arithmetic mean of its two nodes, mu at an edge the harmonic mean
 * of its four nodes (0 if one of them is 0); a neighbour beyond the last
 * node takes the last node's value.
 * Damping: each updated value is (old + dt rhs) / (1 + eta dt), eta the
 * sponge at the array index.  Explosive source: after the stress update of
 * step n, txx, tyy, tzz += dt w q[n] at each trilinear corner.  Receivers:
 * trace[n] = sum_c w (txx + tyy + tzz)(c) / 3 of the stresses at n+1.
 * ======================================================================= */
typedef struct {
  pad_t p;
  int r;
  double c[32];   /* staggered weights c[1..r], unit spacing */
  double ih[3];
  double dt;
  double *bx, *by, *bz, *lam, *mu, *mxy, *mxz, *myz, *eta;   /* [N] */
  int periodic;
} ela_t;

enum { EVX, EVY, EVZ, ETXX, ETYY, ETZZ, ETXY, ETXZ, ETYZ };

static void ela_free(ela_t* E) {
  free(E->bx); free(E->by); free(E->bz); free(E->lam); free(E->mu);
  free(E->mxy); free(E->mxz); free(E->myz); free(E->eta);
}

static double harm4(double a, double b, double c, double d) {
  if (a <= 0.0 || b <= 0.0 || c <= 0.0 || d <= 0.0) return 0.0;
  return 4.0 / (1.0 / a + 1.0 / b + 1.0 / c + 1.0 / d);
}

static int ela_init(ela_t* E, const orc_grid* g, const double* vp, const double* vs,
                    const double* rho, const double* eta_in) {
  memset(E, 0, sizeof(*E));
  if (g->so != 4 && g->so != 8 && g->so != 12) return ORC_EINVAL;
  E->p = make_pad(g);
  E->r = g->so / 2;
  for (int d = 0; d < 3; ++d) {
    if (g->n[d] < 2 * E->r + 2) return ORC_EINVAL;
    E->ih[d] = 1.0 / g->h[d];
  }
  if (orc_fd_weights_stag(g->so, E->c)) return ORC_EINVAL;
  E->dt = g->dt;
  E->periodic = g->periodic;
  const pad_t* p = &E->p;
  int64_t N = p->n0 * p->n1 * p->n2;
  double** arr[9] = {&E->bx, &E->by, &E->bz, &E->lam, &E->mu, &E->mxy, &E->mxz, &E->myz, &E->eta};
  for (int i = 0; i < 9; ++i) {
    *arr[i] = (double*)malloc(sizeof(double) * N);
    if (!*arr[i]) return ORC_ENOMEM;
  }
  double vmax = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    if (!(vp[i] > 0.0) || !(rho[i] > 0.0) || !(vs[i] >= 0.0) || !(2.0 * vs[i] * vs[i] <= vp[i] * vp[i]))
      return ORC_EINVAL;
    E->lam[i] = rho[i] * (vp[i] * vp[i] - 2.0 * vs[i] * vs[i]);
    E->mu[i] = rho[i] * vs[i] * vs[i];
    if (vp[i] > vmax) vmax = vp[i];
  }
  for (int64_t x = 0; x < p->n0; ++x)
    for (int64_t y = 0; y < p->n1; ++y)
      for (int64_t z = 0; z < p->n2; ++z) {
        int64_t x1 = x + 1 < p->n0 ? x + 1 : x, y1 = y + 1 < p->n1 ? y + 1 : y,
                z1 = z + 1 < p->n2 ? z + 1 : z;
        int64_t q = gidx(p, x, y, z);
        E->bx[q] = 0.5 * (1.0 / rho[q] + 1.0 / rho[gidx(p, x1, y, z)]);
        E->by[q] = 0.5 * (1.0 / rho[q] + 1.0 / rho[gidx(p, x, y1, z)]);
        E->bz[q] = 0.5 * (1.0 / rho[q] + 1.0 / rho[gidx(p, x, y, z1)]);
        E->mxy[q] = harm4(E->mu[q], E->mu[gidx(p, x1, y, z)], E->mu[gidx(p, x, y1, z)],
                          E->mu[gidx(p, x1, y1, z)]);
        E->mxz[q] = harm4(E->mu[q], E->mu[gidx(p, x1, y, z)], E->mu[gidx(p, x, y, z1)],
                          E->mu[gidx(p, x1, y, z1)]);
        E->myz[q] = harm4(E->mu[q], E->mu[gidx(p, x, y1, z)], E->mu[gidx(p, x, y, z1)],
                          E->mu[gidx(p, x, y1, z1)]);
      }
  if (eta_in) {
    memcpy(E->eta, eta_in, sizeof(double) * N);
  } else {
    double* ea[3];
    for (int d = 0; d < 3; ++d) {
      ea[d] = (double*)malloc(sizeof(double) * g->n[d]);
      orc_damping_axis(g->n[d], g->nbl, g->h[d], vmax, ea[d]);
    }
    for (int64_t x = 0; x < p->n0; ++x)
      for (int64_t y = 0; y < p->n1; ++y)
        for (int64_t z = 0; z < p->n2; ++z)
          E->eta[gidx(p, x, y, z)] = ea[0][x] + ea[1][y] + ea[2][z];
    for (int d = 0; d < 3; ++d) free(ea[d]);
  }
  return ORC_OK;
}

/* Test hook: the material arrays of the staggered scheme as ela_init builds
 * them (R18's averaging), so that a test can restate them independently.
 * out: [8][N] = bx, by, bz (half-nodes along x, y, z), lam, mu (nodes),
 * mu_xy, mu_xz, mu_yz (edge centres). */
int orc_elastic_materials(const orc_grid* g, const double* vp, const double* vs, const double* rho,
                          double* out) {
  ela_t E;
  int st = ela_init(&E, g, vp, vs, rho, NULL);
  if (st == ORC_OK) {
    int64_t N = g->n[0] * g->n[1] * g->n[2];
    const double* src[8] = {E.bx, E.by, E.bz, E.lam, E.mu, E.mxy, E.mxz, E.myz};
    for (int i = 0; i < 8; ++i) memcpy(out + (int64_t)i * N, src[i], sizeof(double) * N);
  }
  ela_free(&E);
  return st;
}

static inline int64_t ela_stride(const pad_t* p, int d) {
  return d == 0 ? p->P1 * p->P2 : (d == 1 ? p->P2 : 1);
}
/* node -> half-node derivative along d at padded index q */
static inline double ela_dp(const ela_t* E, const double* f, int64_t q, int d) {
  int64_t s = ela_stride(&E->p, d);
  double acc = 0.0;
  for (int k = 1; k <= E->r; ++k) acc += E->c[k] * (f[q + k * s] - f[q - (k - 1) * s]);
  return acc * E->ih[d];
}
/* half-node -> node derivative along d at padded index q */
static inline double ela_dm(const ela_t* E, const double* g, int64_t q, int d) {
  int64_t s = ela_stride(&E->p, d);
  double acc = 0.0;
  for (int k = 1; k <= E->r; ++k) acc += E->c[k] * (g[q + (k - 1) * s] - g[q - k * s]);
  return acc * E->ih[d];
}

/* Stability limit of the staggered velocity-stress leapfrog:
 * dt vp |s| <= 2 with |s_d| <= S/h_d, S = max |2 sum c_k sin((k - 1/2) theta)|. */
double orc_elastic_dt_max(int so, const double h[3], double vpmax) {
  double c[32];
  if (orc_fd_weights_stag(so, c)) return -1.0;
  double S = symbol_max(c, so / 2, 0.5);
  double s2 = 0.0;
  for (int d = 0; d < 3; ++d) s2 += (S / h[d]) * (S / h[d]);
  return 2.0 / (vpmax * sqrt(s2));
}

/* init / out: NULL or [9][N] in the order vx, vy, vz (at n - 1/2), txx, tyy,
 * tzz, txy, txz, tyz (at n); out holds v^{nt-1/2} and the stresses at nt. */
int orc_elastic_forward(const orc_grid* g, const double* vp, const double* vs, const double* rho,
                        const double* eta, int nsrc, const double* src_xyz, const double* src_wav,
                        int nrec, const double* rec_xyz, double* traces, const double* init,
                        double* out) {
  ela_t E;
  int st = ela_init(&E, g, vp, vs, rho, eta);
  if (st) { ela_free(&E); return st; }
  const pad_t* p = &E.p;
  const int64_t N = p->n0 * p->n1 * p->n2;
#ifdef _OPENMP
  if (g->nthreads > 0) omp_set_num_threads(g->nthreads);
#endif
  int64_t* sb = (int64_t*)malloc(sizeof(int64_t) * 3 * (nsrc > 0 ? nsrc : 1));
  double* sf = (double*)malloc(sizeof(double) * 3 * (nsrc > 0 ? nsrc : 1));
  int64_t* rb = (int64_t*)malloc(sizeof(int64_t) * 3 * (nrec > 0 ? nrec : 1));
  double* rf = (double*)malloc(sizeof(double) * 3 * (nrec > 0 ? nrec : 1));
  double* buf = (double*)calloc((size_t)p->NP * 9, sizeof(double));
  if (!sb || !sf || !rb || !rf || !buf) { st = ORC_ENOMEM; goto done; }
  for (int s = 0; s < nsrc; ++s)
    if (trilinear(g, src_xyz + 3 * s, sb + 3 * s, sf + 3 * s)) { st = ORC_EINVAL; goto done; }
  for (int r = 0; r < nrec; ++r)
    if (trilinear(g, rec_xyz + 3 * r, rb + 3 * r, rf + 3 * r)) { st = ORC_EINVAL; goto done; }
  {
    double* F[9];
    for (int i = 0; i < 9; ++i) F[i] = buf + (size_t)i * p->NP;
    if (init)
      for (int i = 0; i < 9; ++i) to_padded(p, init + (size_t)i * N, F[i]);
    const double dt = E.dt;
    for (int n = 0; n < g->nt; ++n) {
      if (E.periodic)
        for (int i = ETXX; i <= ETYZ; ++i) wrap_halo(p, F[i]);
      /* velocities: n - 1/2 -> n + 1/2 (reads stresses only) */
#pragma omp parallel for schedule(static)
      for (int64_t x = 0; x < p->n0; ++x)
        for (int64_t y = 0; y < p->n1; ++y)
          for (int64_t z = 0; z < p->n2; ++z) {
            int64_t q = pidx(p, x, y, z), gq = gidx(p, x, y, z);
            double damp = 1.0 + E.eta[gq] * dt;
            double fx = ela_dp(&E, F[ETXX], q, 0) + ela_dm(&E, F[ETXY], q, 1) + ela_dm(&E, F[ETXZ], q, 2);
            double fy = ela_dm(&E, F[ETXY], q, 0) + ela_dp(&E, F[ETYY], q, 1) + ela_dm(&E, F[ETYZ], q, 2);
            double fz = ela_dm(&E, F[ETXZ], q, 0) + ela_dm(&E, F[ETYZ], q, 1) + ela_dp(&E, F[ETZZ], q, 2);
            F[EVX][q] = (F[EVX][q] + dt * E.bx[gq] * fx) / damp;
            F[EVY][q] = (F[EVY][q] + dt * E.by[gq] * fy) / damp;
            F[EVZ][q] = (F[EVZ][q] + dt * E.bz[gq] * fz) / damp;
          }
      if (E.periodic)
        for (int i = EVX; i <= EVZ; ++i) wrap_halo(p, F[i]);
      /* stresses: n -> n + 1 (reads velocities only) */
#pragma omp parallel for schedule(static)
      for (int64_t x = 0; x < p->n0; ++x)
        for (int64_t y = 0; y < p->n1; ++y)
          for (int64_t z = 0; z < p->n2; ++z) {
            int64_t q = pidx(p, x, y, z), gq = gidx(p, x, y, z);
            double damp = 1.0 + E.eta[gq] * dt;
            double exx = ela_dm(&E, F[EVX], q, 0), eyy = ela_dm(&E, F[EVY], q, 1),
                   ezz = ela_dm(&E, F[EVZ], q, 2);
            double lam = E.lam[gq], mu = E.mu[gq], tr = exx + eyy + ezz;
            F[ETXX][q] = (F[ETXX][q] + dt * (lam * tr + 2.0 * mu * exx)) / damp;
            F[ETYY][q] = (F[ETYY][q] + dt * (lam * tr + 2.0 * mu * eyy)) / damp;
            F[ETZZ][q] = (F[ETZZ][q] + dt * (lam * tr + 2.0 * mu * ezz)) / damp;
            F[ETXY][q] = (F[ETXY][q] + dt * E.mxy[gq] * (ela_dp(&E, F[EVX], q, 1) + ela_dp(&E, F[EVY], q, 0))) / damp;
            F[ETXZ][q] = (F[ETXZ][q] + dt * E.mxz[gq] * (ela_dp(&E, F[EVX], q, 2) + ela_dp(&E, F[EVZ], q, 0))) / damp;
            F[ETYZ][q] = (F[ETYZ][q] + dt * E.myz[gq] * (ela_dp(&E, F[EVY], q, 2) + ela_dp(&E, F[EVZ], q, 1))) / damp;
          }
      /* explosive source into the normal stresses */
      for (int s = 0; s < nsrc; ++s) {
        double qv = src_wav[(int64_t)s * g->nt + n];
        for (int c = 0; c < 8; ++c) {
          double w = corner_weight(sf + 3 * s, c);
          if (w == 0.0) continue;
          int64_t q = pidx(p, sb[3 * s] + ((c >> 2) & 1), sb[3 * s + 1] + ((c >> 1) & 1),
                           sb[3 * s + 2] + (c & 1));
          F[ETXX][q] += dt * w * qv;
          F[ETYY][q] += dt * w * qv;
          F[ETZZ][q] += dt * w * qv;
        }
      }
      for (int r = 0; r < nrec; ++r) {
        double acc = 0.0;
        for (int c = 0; c < 8; ++c) {
          double w = corner_weight(rf + 3 * r, c);
          if (w == 0.0) continue;
          int64_t q = pidx(p, rb[3 * r] + ((c >> 2) & 1), rb[3 * r + 1] + ((c >> 1) & 1),
                           rb[3 * r + 2] + (c & 1));
          acc += w * (F[ETXX][q] + F[ETYY][q] + F[ETZZ][q]) / 3.0;
        }
        traces[(int64_t)n * nrec + r] = acc;
      }
    }
    if (out)
      for (int i = 0; i < 9; ++i) from_padded(p, F[i], out + (size_t)i * N);
  }
done:
  free(sb); free(sf); free(rb); free(rf); free(buf);
  ela_free(&E);
  return st;
}

/* Discrete energy of the undamped staggered scheme (vs > 0 everywhere):
 *   E^n = 1/2 sum v^{n+1/2} . W v^{n-1/2} + 1/2 sum tau^n : S tau^n
 * W = 1/b at each velocity position, S the compliance (inverse of the
 * stress update's stiffness: normal block [[lam+2mu, lam, lam], ...], shear
 * 1/mu_edge).  v_next, v_prev: [3][N]; tau: [6][N]. */
double orc_elastic_energy(const orc_grid* g, const double* vp, const double* vs, const double* rho,
                          const double* v_next, const double* v_prev, const double* tau) {
  ela_t E;
  orc_grid g2 = *g;
  g2.nbl = 0;
  if (ela_init(&E, &g2, vp, vs, rho, NULL)) { ela_free(&E); return NAN; }
  const int64_t N = E.p.n0 * E.p.n1 * E.p.n2;
  double kin = 0.0, pot = 0.0;
  const double* b[3] = {E.bx, E.by, E.bz};
  const double* ms[3] = {E.mxy, E.mxz, E.myz};
  for (int64_t i = 0; i < N; ++i) {
    for (int d = 0; d < 3; ++d) kin += v_next[d * N + i] * v_prev[d * N + i] / b[d][i];
    double lam = E.lam[i], mu = E.mu[i];
    double sxx = tau[i], syy = tau[N + i], szz = tau[2 * N + i];
    double tr = sxx + syy + szz;
    /* S sigma = (sigma - lam/(3 lam + 2 mu) tr I) / (2 mu) */
    double k = lam / (3.0 * lam + 2.0 * mu);
    pot += (sxx * sxx + syy * syy + szz * szz - k * tr * tr) / (2.0 * mu);
    for (int d = 0; d < 3; ++d) {
      double t = tau[(3 + d) * N + i];
      if (t != 0.0 || ms[d][i] > 0.0) pot += t * t / ms[d][i];
    }
  }
  ela_free(&E);
  return 0.5 * (kin + pot);
}

/* =========================================================================
 * Adjoint of the acoustic forward map and the velocity gradient (the FWI /
 * RTM use the paper cites in Sec. I).  Written for the discrete recurrence
 * of orc_acoustic_forward:
 *   u^{k} = D L u^{k-1} + B u^{k-1} + C u^{k-2} + M S^{k-1},  k = 1..nt
 *   D = dt^2/(m+a), B = 2m/(m+a), C = (a-m)/(m+a), M = dt^2/m, a = eta dt/2,
 *   S^{n} = sum_s w_s q_s[n] spread to the corners, d[n] = P u^{n+1}.
 * For adjoint traces r[n][k] (the residual) the adjoint state runs backward,
 *   lam^{k} = P^T r[k-1] + L (D lam^{k+1}) + B lam^{k+1} + C lam^{k+2},
 * (L symmetric), and gives
 *   d<d, r>/d q_s[n] = sum_c w_s(c) M(c) lam^{n+1}(c)           (grad_src)
 *   d<d, r>/d m(p)   = sum_k lam^k(p) [ (2a (u^{k-1} - u^{k-2}) - dt^2 L u^{k-1})
 *                      / (m+a)^2 - dt^2/m^2 S^{k-1} ](p)           (grad_m)
 *   d<d, r>/d vp(p)  = grad_m(p) * (-2 / vp(p)^3),
 * with dt and eta held fixed.  The forward history is kept whole (small
 * grids only).
 * ======================================================================= */
static void lap_apply(const model_t* M, const double* uc, double* out) {
  const pad_t* p = &M->p;
  int64_t stride[3] = {p->P1 * p->P2, p->P2, 1};
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < p->n0; ++x)
    for (int64_t y = 0; y < p->n1; ++y)
      for (int64_t z = 0; z < p->n2; ++z) {
        int64_t q = pidx(p, x, y, z);
        double lap = 0.0;
        for (int d = 0; d < 3; ++d) {
          double s = M->c[0] * uc[q];
          for (int i = 1; i <= M->r; ++i) s += M->c[i] * (uc[q + i * stride[d]] + uc[q - i * stride[d]]);
          lap += s * M->ih2[d];
        }
        out[gidx(p, x, y, z)] = lap;
      }
}

int orc_acoustic_adjoint(const orc_grid* g, const double* vp, const double* eta, int nsrc,
                         const double* src_xyz, const double* src_wav, int nrec, const double* rec_xyz,
                         const double* resid, double* grad_src, double* grad_vp) {
  model_t M;
  int st = model_init(&M, g, vp, eta);
  if (st) { model_free(&M); return st; }
  const pad_t* p = &M.p;
  const int64_t N = p->n0 * p->n1 * p->n2;
  const int nt = g->nt;
  int64_t* sb = (int64_t*)malloc(sizeof(int64_t) * 3 * (nsrc > 0 ? nsrc : 1));
  double* sf = (double*)malloc(sizeof(double) * 3 * (nsrc > 0 ? nsrc : 1));
  int64_t* rb = (int64_t*)malloc(sizeof(int64_t) * 3 * (nrec > 0 ? nrec : 1));
  double* rf = (double*)malloc(sizeof(double) * 3 * (nrec > 0 ? nrec : 1));
  /* forward history u^k, k = -1..nt (padded), stored as hist[k + 1] */
  double* hist = (double*)calloc((size_t)(nt + 2) * p->NP, sizeof(double));
  double* S = (double*)calloc((size_t)(nt > 0 ? nt : 1) * N, sizeof(double)); /* S^{n} unpadded */
  double* lam = (double*)calloc((size_t)3 * p->NP, sizeof(double));            /* lam^{k}, k+1, k+2 */
  double* w = (double*)calloc(p->NP, sizeof(double));
  double* lw = (double*)malloc(sizeof(double) * N);
  double* lu = (double*)malloc(sizeof(double) * N);
  double* gm = (double*)calloc(N, sizeof(double));
  if (!sb || !sf || !rb || !rf || !hist || !S || !lam || !w || !lw || !lu || !gm) { st = ORC_ENOMEM; goto done; }
  for (int s = 0; s < nsrc; ++s)
    if (trilinear(g, src_xyz + 3 * s, sb + 3 * s, sf + 3 * s)) { st = ORC_EINVAL; goto done; }
  for (int r = 0; r < nrec; ++r)
    if (trilinear(g, rec_xyz + 3 * r, rb + 3 * r, rf + 3 * r)) { st = ORC_EINVAL; goto done; }
  /* spread sources S^{n} */
  for (int n = 0; n < nt; ++n)
    for (int s = 0; s < nsrc; ++s)
      for (int c = 0; c < 8; ++c) {
        double wc = corner_weight(sf + 3 * s, c);
        if (wc == 0.0) continue;
        int64_t x = sb[3 * s] + ((c >> 2) & 1), y = sb[3 * s + 1] + ((c >> 1) & 1), z = sb[3 * s + 2] + (c & 1);
        S[(int64_t)n * N + gidx(p, x, y, z)] += wc * src_wav[(int64_t)s * nt + n];
      }
  /* forward, keeping every state */
  for (int k = 1; k <= nt; ++k) {
    double* up = hist + (size_t)(k - 1) * p->NP; /* u^{k-2} */
    double* uc = hist + (size_t)k * p->NP;       /* u^{k-1} */
    double* un = hist + (size_t)(k + 1) * p->NP; /* u^{k}   */
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < p->n0; ++x)
      for (int64_t y = 0; y < p->n1; ++y)
        for (int64_t z = 0; z < p->n2; ++z) {
          int64_t gq = gidx(p, x, y, z);
          un[pidx(p, x, y, z)] = point_update(&M, up, uc, x, y, z) + S[(int64_t)(k - 1) * N + gq] * M.dt2 / M.m[gq];
        }
  }
  /* backward: lam^{k} for k = nt..1 */
  double* l0 = lam;               /* lam^{k}   */
  double* l1 = lam + p->NP;       /* lam^{k+1} */
  double* l2 = lam + 2 * p->NP;   /* lam^{k+2} */
  if (grad_src) memset(grad_src, 0, sizeof(double) * (size_t)(nsrc > 0 ? nsrc : 0) * nt);
  for (int k = nt; k >= 1; --k) {
    /* w = D lam^{k+1} (zero halo), then L w */
    for (int64_t x = 0; x < p->n0; ++x)
      for (int64_t y = 0; y < p->n1; ++y)
        for (int64_t z = 0; z < p->n2; ++z) {
          int64_t gq = gidx(p, x, y, z);
          double a = M.eta[gq] * M.dt * 0.5;
          w[pidx(p, x, y, z)] = M.dt2 / (M.m[gq] + a) * l1[pidx(p, x, y, z)];
        }
    lap_apply(&M, w, lw);
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < p->n0; ++x)
      for (int64_t y = 0; y < p->n1; ++y)
        for (int64_t z = 0; z < p->n2; ++z) {
          int64_t q = pidx(p, x, y, z), gq = gidx(p, x, y, z);
          double m = M.m[gq], a = M.eta[gq] * M.dt * 0.5;
          l0[q] = lw[gq] + 2.0 * m / (m + a) * l1[q] + (a - m) / (m + a) * l2[q];
        }
    /* receiver residual injected at the corners: P^T r[k-1] */
    for (int r = 0; r < nrec; ++r)
      for (int c = 0; c < 8; ++c) {
        double wc = corner_weight(rf + 3 * r, c);
        if (wc == 0.0) continue;
        int64_t x = rb[3 * r] + ((c >> 2) & 1), y = rb[3 * r + 1] + ((c >> 1) & 1), z = rb[3 * r + 2] + (c & 1);
        l0[pidx(p, x, y, z)] += wc * resid[(int64_t)(k - 1) * nrec + r];
      }
    /* source gradient: sum_c w_s(c) M(c) lam^{k}(c) for step k-1 */
    if (grad_src)
      for (int s = 0; s < nsrc; ++s) {
        double acc = 0.0;
        for (int c = 0; c < 8; ++c) {
          double wc = corner_weight(sf + 3 * s, c);
          if (wc == 0.0) continue;
          int64_t x = sb[3 * s] + ((c >> 2) & 1), y = sb[3 * s + 1] + ((c >> 1) & 1), z = sb[3 * s + 2] + (c & 1);
          acc += wc * M.dt2 / M.m[gidx(p, x, y, z)] * l0[pidx(p, x, y, z)];
        }
        grad_src[(int64_t)s * nt + (k - 1)] = acc;
      }
    /* velocity gradient contribution of equation k */
    if (grad_vp) {
      double* um2 = hist + (size_t)(k - 1) * p->NP; /* u^{k-2} */
      double* um1 = hist + (size_t)k * p->NP;       /* u^{k-1} */
      lap_apply(&M, um1, lu);
      for (int64_t x = 0; x < p->n0; ++x)
        for (int64_t y = 0; y < p->n1; ++y)
          for (int64_t z = 0; z < p->n2; ++z) {
            int64_t q = pidx(p, x, y, z), gq = gidx(p, x, y, z);
            double m = M.m[gq], a = M.eta[gq] * M.dt * 0.5;
            double dr = (2.0 * a * (um1[q] - um2[q]) - M.dt2 * lu[gq]) / ((m + a) * (m + a)) -
                        M.dt2 / (m * m) * S[(int64_t)(k - 1) * N + gq];
            gm[gq] += l0[q] * dr;
          }
    }
    double* t = l2; l2 = l1; l1 = l0; l0 = t;
    memset(l0, 0, sizeof(double) * p->NP);
  }
  if (grad_vp)
    for (int64_t i = 0; i < N; ++i) grad_vp[i] = gm[i] * (-2.0 / (vp[i] * vp[i] * vp[i]));
done:
  free(sb); free(sf); free(rb); free(rf); free(hist); free(S); free(lam); free(w); free(lw); free(lu);
  free(gm);
  model_free(&M);
  return st;
}
