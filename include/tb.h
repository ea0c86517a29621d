/*
 * tb.h -- C ABI of the GB300 temporally blocked finite-difference wave
 * propagator with off-the-grid sources (arXiv 2010.10248).
 *
 * Problem (Sec. III-A, Eq. 1): isotropic acoustic wave equation
 *     m(x) u_tt - Lap u = delta(x - x_s) q(t),  m = 1/vp^2,
 *     zero initial conditions, receivers d(t, .) = u(t, x_r),
 * discretised 2nd order in time and space order 4/8/12, with absorbing
 * damping layers (Sec. IV-B).  Sources and receivers sit off the grid and
 * act through trilinear weights (Sec. I, Fig. 3).  Before propagation an
 * inspector rewrites them into grid-aligned form (Sec. II-A: affected-point
 * mask and unique IDs, decomposed source table src_dcmp, per-column reduced
 * iteration space), which lets the propagator fuse several time steps into
 * one temporally blocked sweep (Sec. II-B).
 *
 * The two other wave equations of Sec. III are propagated one step per
 * launch with the same grid-aligned sources and receivers:
 *   TB_TTI (Sec. III-B, Eq. 2): pseudo-acoustic tilted transversely
 *     isotropic medium, fields p and r, 2nd order in time:
 *       m p_tt = (1 + 2 eps) H_h p + sqrt(1 + 2 delta) H_z r
 *       m r_tt = sqrt(1 + 2 delta) H_h p + H_z r
 *     H_z = -D_zbar^T D_zbar, H_h = -(D_xbar^T D_xbar + D_ybar^T D_ybar) with
 *     Eq. 2's rotated first derivatives (centred, order so); sources enter p
 *     and r (dt^2/m scaling), receivers sample p.
 *   TB_ELASTIC (Sec. III-C, Eq. 3): isotropic velocity-stress on the
 *     staggered grid (staggered first derivatives of order so); explosive
 *     sources add dt q to the three normal stresses, receivers sample their
 *     mean.
 *
 * Conventions for every call:
 *   - Grid shape n[3] with axis 2 contiguous (the paper's u[t][x][y][z] with
 *     z innermost).  A "field" argument is a dense float array [n0][n1][n2].
 *   - Coordinates are FP64 metres with the origin at grid index 0; a point
 *     must lie in [0, (n_d - 1) h_d] on every axis, else TB_EINVAL.
 *   - Array pointers may point to host or device memory; the library tells
 *     them apart with cudaPointerGetAttributes.  Host inputs are copied to
 *     the device on `stream` before the call returns (pageable host memory
 *     makes the copy synchronous).  The caller keeps ownership of every
 *     pointer it passes; the library never frees or retains them after the
 *     call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL: the legacy default
 *     stream).  Device work is enqueued asynchronously on it unless stated.
 *   - Every function returns a tb_status.  The library never aborts or
 *     exits; on error the handle keeps a message readable with
 *     tb_last_error().  A failing call leaves the handle usable.
 *   - One handle must not be used from two host threads at once.
 */
#ifndef TB_H
#define TB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TB_OK = 0,
  TB_EINVAL = 1,     /* invalid argument (shape, order, coordinate, size)   */
  TB_ENOMEM = 2,     /* device allocation failed                            */
  TB_ECUDA = 3,      /* a CUDA runtime call failed                          */
  TB_EUNSTABLE = 4,  /* dt above the CFL limit of the model                 */
  TB_ETIMEOUT = 5,   /* a bounded device-side wait ran out (blocked sweep)  */
  TB_EDIVERGED = 6,  /* NaN/Inf found in the receiver traces                */
  TB_ESTATE = 7      /* call order violated (e.g. forward before set_model) */
} tb_status;

enum { TB_ACOUSTIC = 0, TB_TTI = 1, TB_ELASTIC = 2 };
enum { TB_ONESTEP = 0, TB_BLOCKED = 1 };
/* Wavefield storage (tb_options.storage), acoustic physics:
 *   TB_F32       FP32 fields, TMA-staged one-step and blocked sweeps (default);
 *   TB_F16       FP16 fields, FP32 arithmetic, per-field power-of-two scales
 *                (stored value u / s, s set on the device each step from the
 *                previous step's max |u|), through the TMA-staged one-step
 *                sweep: half the wavefield bytes and footprint of TB_F32;
 *   TB_BF16      BF16 fields, likewise;
 *   TB_F32_PLAIN FP32 fields with the same per-step scales through a plain
 *                streaming one-step kernel (a second, independent
 *                implementation of the scaled step).
 * The 16-bit and plain modes run one step per launch (TB_ONESTEP). */
enum { TB_F32 = 0, TB_F16 = 1, TB_BF16 = 2, TB_F32_PLAIN = 3 };

typedef struct tb_handle tb_handle;

/* Tuning and behaviour options; zero-initialise and set what you need.
 * All-zero options give the defaults noted per field. */
typedef struct {
  int time_tile;   /* T: time steps fused per blocked sweep (Sec. II-B).
                      Supported: 1..4 (space order 4, 8), 1..2 (space order 12);
                      0 -> the fastest measured on GB300 at 512^3: 4 (space
                      order 4), 3 (8), 2 (12).  TB_TTI, TB_ELASTIC: 1..16
                      steps per wavefront (below); 0 -> 16.                   */
  int nbl;         /* width in cells of the built-in sponge (Sec. IV-B); 0: none  */
  int y_bands;     /* blocked sweep: number of bands along axis 1, each time
                      tile split the same way; 0 -> bands pipelined across time
                      tiles: every launch fills the co-resident CTAs with the
                      rows of time tile k still to do and, once k is finished
                      in that launch, the first rows of tile k + 1 (rows at
                      least T r below the rows of tile k still running)      */
  int x_chunks;    /* chunks along axis 0 processed as independent sweeps; 0 -> 1
                      (blocked) or automatic (one-step); > 1 with the blocked
                      schedule turns the pipelining off                         */
  int profile;     /* 1: time every propagator launch with CUDA events on the
                      launching stream (read back with tb_kernel_time)            */
  int check_nan;   /* 1: tb_forward scans the traces and returns TB_EDIVERGED on
                      NaN/Inf (adds a device->host sync)                         */
  double wait_timeout_s; /* blocked sweep: bound on any device-side wait for a
                      neighbouring tile, seconds; 0 -> 2.0                         */
  int storage;     /* TB_F32 (0), TB_F16, TB_BF16 or TB_F32_PLAIN; the 16-bit
                      stored value is u / s with s = 2^(ceil(log2(4 max|u^n| +
                      max|source step n|)) - 8), set on the device each step     */
  int band_ctas;   /* pipelined blocked sweep: most CTAs per launch; 0 -> every
                      CTA that fits co-resident on the GPU (one per SM)          */
  int slab_planes; /* TB_TTI / TB_ELASTIC blocked sweep: planes per slab of the
                      wavefront along axis 0, at least the reach of one
                      sub-update: space_order / 2, or space_order for TTI with
                      tti_fused, else TB_EINVAL; 0 -> 32                         */
  int tti_fused;   /* TB_TTI: 0 (default) a flux kernel writing the six flux
                      fields and an update kernel reading them; 1: both passes
                      of a step in one kernel, the fluxes kept on chip (the
                      same values bit for bit, 6 fields less device memory,
                      48 B less memory traffic per point and step, slower on
                      GB300: one CTA per SM with two barriers per plane)        */
  int stream_l1;   /* TB_TTI (two-pass) / TB_ELASTIC: 0 (default) passes with
                      every operand staged in shared memory by TMA; 1: the
                      streaming kernels that read axis-1/2 neighbours through
                      the L1 cache (the same values bit for bit)                */
} tb_options;

/* Create a propagator for a grid of shape n[3] with spacing h[3] (metres),
 * space order 4, 8 or 12 (the space orders of Sec. IV) and physics
 * TB_ACOUSTIC, TB_TTI or TB_ELASTIC.  Requires n_d >= space_order + 2 on
 * every axis.  `opt` may be NULL (defaults).  Allocates the wavefields and
 * model buffers on the current CUDA device (acoustic: 5 x n0 n1 n2 floats,
 * with TB_F16 / TB_BF16 storage two 16-bit wavefields and one float field;
 * TTI: 16, 10 with opt.tti_fused; elastic: 18).  Errors: TB_EINVAL (also: 16-bit or plain storage
 * with TTI or elastic physics), TB_ENOMEM, TB_ECUDA. */
int tb_create(const int64_t n[3], const double h[3], int space_order, int physics,
              const tb_options* opt, tb_handle** out);

/* Release every device allocation of the handle and the handle itself
 * (stream-ordered frees on the handle's last stream).  NULL is accepted.
 * Returns TB_OK. */
int tb_destroy(tb_handle* h);

/* Set the velocity model (Eq. 1: m = 1/vp^2).  vp: field of P velocities in
 * m/s, all > 0.  aux: further per-point parameters, fields stacked [k][n0]
 * [n1][n2]: acoustic: NULL; TTI: k = 4: eps, delta (Thomsen parameters,
 * eps >= delta > -1/2, else TB_EUNSTABLE), theta (tilt), phi (azimuth) in
 * radians (Eq. 2); elastic: k = 2: vs (m/s, 0 <= 2 vs^2 <= vp^2) and rho
 * (> 0).  damp: NULL for the built-in sponge of opt.nbl cells, or
 * n0 + n1 + n2 per-axis damping coefficients eta (1/s) whose sum over the
 * three axes is the damping of a grid point.  dt: time step in seconds; 0
 * selects 0.8 of the stability limit (tb_cfl_dt_max, tb_tti_dt_max or
 * tb_elastic_dt_max for the model's maxima).  Computes the maxima on the
 * device (the call synchronises `stream`).
 * Errors: TB_EINVAL (vp <= 0 or not finite), TB_EUNSTABLE (dt > limit). */
int tb_set_model(tb_handle* h, const float* vp, const float* aux, const float* damp,
                 double dt, void* stream);

/* Time step in seconds in use after tb_set_model; 0 for a NULL handle or
 * before tb_set_model. */
double tb_get_dt(const tb_handle* h);

/* Register nsrc off-grid sources and run the inspector on the device
 * (Sec. II-A.1-3): trilinear corners with FP64 weight != 0 become affected
 * points with ascending unique IDs, and the wavelets are decomposed into the
 * grid-aligned table src_dcmp[t][id] = (dt^2/m(p_id)) sum_s w_s(p_id) q_s[t]
 * (Listing 3, injection expression s*dt^2/m of Sec. III-A; elastic: dt
 * instead of dt^2/m).
 * coords: [nsrc][3] FP64 metres.  wavelets: [nsrc][nt] float.  Requires
 * tb_set_model first (TB_ESTATE).  nsrc may be 0 (no sources).
 * Limits: nsrc < 2^21.  Errors: TB_EINVAL (coordinate outside the grid). */
int tb_set_sources(tb_handle* h, int nsrc, const double* coords, int nt,
                   const float* wavelets, void* stream);

/* Register nrec off-grid receivers (trilinear interpolation, Fig. 3b) and
 * build their grid-aligned form: unique receiver points, a per-column
 * reduced index (mirror of Sec. II-A.4), and per receiver its 8 (point,
 * weight) pairs.  coords: [nrec][3] FP64 metres.  nrec may be 0.
 * Limits: nrec < 2^21.  Errors: TB_EINVAL. */
int tb_set_receivers(tb_handle* h, int nrec, const double* coords, void* stream);

/* Propagate nt steps from zero initial conditions (Eq. 1) and write the
 * receiver traces traces[n][r] = sum_c w_rc u^{n+1}(c) (u^{n+1} after the
 * step-n injection), an [nt][nrec] float array (host or device; may be
 * NULL).  schedule: TB_ONESTEP (one launch per time step, spatial blocking
 * only) or TB_BLOCKED (opt.time_tile steps fused per sweep, Sec. II-B).
 * Both give bitwise-identical wavefields and traces.  TB_TTI and
 * TB_ELASTIC: each step is two sub-updates (elastic: velocity, then
 * stress, Fig. 7b; TTI: fluxes, then divergence and leapfrog update) or one
 * (TTI with opt.tti_fused); TB_BLOCKED runs opt.time_tile steps as
 * one wavefront over slabs of opt.slab_planes planes along axis 0,
 * sub-update u of slab s in launch s + 2u (the nt mod time_tile remaining
 * steps one step per launch); traces sample p (TTI) or
 * the mean normal stress at n+1 (elastic).  16-bit and plain storage:
 * TB_ONESTEP only (TB_EINVAL).  Source tables scale:
 * dt^2/m (acoustic, TTI), dt (elastic).  nt must not exceed the
 * wavelet length given to tb_set_sources (when sources are set).
 * Device traces: asynchronous on `stream`.  Host traces: synchronous.
 * Errors: TB_ESTATE, TB_EINVAL, TB_ETIMEOUT, TB_EDIVERGED, TB_ECUDA. */
int tb_forward(tb_handle* h, int nt, float* traces, int schedule, void* stream);

/* Copy a wavefield after tb_forward into out (dense [n0][n1][n2] float,
 * host or device).  Acoustic: which = 0 -> u^{nt}, 1 -> u^{nt-1}.  TTI:
 * 0 -> p^{nt}, 1 -> p^{nt-1}, 2 -> r^{nt}, 3 -> r^{nt-1}.  Elastic: 0..8 ->
 * vx, vy, vz (at nt - 1/2; vx at (i+1/2, j, k) etc.), txx, tyy, tzz, txy,
 * txz, tyz (at nt; txy at (i+1/2, j+1/2, k) etc.).  16-bit storage returns
 * the stored value times its step's scale.  Ordered on `stream` (a host
 * destination makes the call synchronous).  Errors: TB_EINVAL (NULL handle
 * or out, `which` out of range), TB_ESTATE (no tb_forward yet, or the fields
 * were overwritten by tb_adjoint_gradient), TB_ECUDA. */
int tb_get_field(tb_handle* h, int which, float* out, void* stream);

/* Inspector tables, for checking against an independent implementation.
 * Source points: *npts receives the number of affected points; lin (host,
 * may be NULL) receives their ascending linear indices (x n1 + y) n2 + z,
 * which is the paper's SID order; dcmp (host, may be NULL) receives
 * src_dcmp as [nt][npts] float (nt: the wavelet length given to
 * tb_set_sources).  Caller-owned arrays; call first with lin = dcmp = NULL
 * to size them.  Synchronous.  Errors: TB_EINVAL (NULL handle or npts),
 * TB_ESTATE (no sources set), TB_ECUDA. */
int tb_get_source_points(tb_handle* h, int64_t* npts, int64_t* lin, float* dcmp);

/* Receiver points: *npts, ascending linear indices (host, may be NULL), and
 * per receiver its 8 corner point ids (-1 for a zero weight) and weights
 * (host arrays [nrec][8], may be NULL).  Caller-owned arrays.  Synchronous.
 * Errors: TB_EINVAL (NULL handle or npts), TB_ESTATE (no receivers set),
 * TB_ECUDA. */
int tb_get_receiver_points(tb_handle* h, int64_t* npts, int64_t* lin, int32_t* corner_id,
                           float* corner_w);

/* Device bytes held by the handle (fields, model, tables, scratch); 0 for a
 * NULL handle.  Never fails. */
size_t tb_workspace_bytes(const tb_handle* h);

/* Host-side layout of the sweep kernel's source table (Sec. II-A's
 * grid-aligned injection, as the blocked sweep reads it; no GPU needed).
 * For npts grid points given by their unpadded linear indices lin[i] =
 * (x n1 + y) n2 + z on a grid with n1 x n2 points on axes 1 and 2, the points
 * of each column pair (y, 2p), (y, 2p + 1) share one range of planes
 * [first, first + span): writes ev_pair[2 (y ceil(n2/2) + p) + 0] = first |
 * span << 16 and [.. + 1] = base (caller-owned, 2 n1 ceil(n2/2) ints; zero
 * for pairs without points), slot[i] = 2 (base + x - first) + (z mod 2) (the
 * float offset of point i in every step's row of the table) and nev (the sum
 * of the spans: a row holds 2 nev floats).  Errors: TB_EINVAL (bad
 * arguments, a plane or span beyond 65535, more than 2^30 slots). */
int tb_source_event_layout(int64_t npts, const int64_t* lin, int64_t n1, int64_t n2, int* ev_pair, int* slot,
                           int64_t* nev);

/* Host-side schedule of the blocked sweep with bands pipelined across time
 * tiles (the default when y_bands = 0 and x_chunks <= 1; Sec. II-B's temporal
 * blocking, split into co-resident bands).  No GPU is needed.  For a grid of
 * n1 x n2 points on axes 1 and 2, space order 4, 8 or 12, time_tile >= 2 fused
 * steps, n_tiles time tiles and launches of at most `cap` CTAs (one 16 x 64
 * tile each), writes up to max_passes passes to `passes` (caller-owned,
 * 7 ints each, in launch order): launch index, time tile, first and end owned
 * row of axis 1, first computed row, tile rows, first CTA in the launch.  A
 * pass computes its owned rows plus (time_tile - 1) r rows on each side
 * (clipped), with r = space_order / 2.  Returns the number of passes (which
 * may exceed max_passes), or -TB_EINVAL for bad arguments or a cap too small
 * for one band of the grid. */
int tb_plan_pipeline(int n1, int n2, int space_order, int time_tile, int n_tiles, int cap, int* passes,
                     int max_passes);

/* Host-side planner of the TTI / elastic wavefront (tb_forward with
 * TB_BLOCKED, Sec. II-B): n0 planes along axis 0 in slabs of `slab` planes,
 * `n_sub` sub-updates (2 per fused step).  Writes up to max_items items of 4
 * ints (launch, sub-update u, first plane, end plane) into items (may be
 * NULL to count), launches ascending; sub-update u of slab s is in launch
 * s + 2u.  Returns the number of items, or -TB_EINVAL for n0 < 1, slab < 1,
 * n_sub < 1 or too small a buffer. */
int tb_plan_wavefront(int n0, int slab, int n_sub, int* items, int max_items);

/* With opt.profile = 1: number of propagator launches of the last
 * tb_forward and their summed device time in ms, measured with CUDA events
 * on the launching stream; kind 0 = propagator sweeps, 1 = receiver
 * finalize.  Synchronises the stream of the last forward.  Errors: TB_EINVAL
 * (NULL arguments), TB_ESTATE (profiling off). */
int tb_kernel_time(tb_handle* h, int kind, int* launches, double* ms);

/* Message of the last failing call on this handle ("" if the last call
 * succeeded; "null handle" for NULL).  Owned by the handle, valid until its
 * next call. */
const char* tb_last_error(const tb_handle* h);

/* --- Setup arithmetic (host, FP64), exported for testing --------------- */

/* Centred 2nd-derivative weights on a unit grid, c[0..so/2] (c[0] centre,
 * c[i] for offsets +-i), from the closed form
 * c_i = 2 (-1)^(i+1) (r!)^2 / (i^2 (r-i)! (r+i)!), c_0 = -2 sum c_i.
 * Errors: TB_EINVAL. */
int tb_fd_weights(int space_order, double* c);

/* CFL limit of the leapfrog scheme: dt_max = 2 / (vmax sqrt(S sum_d 1/h_d^2)),
 * S = |c0 + 2 sum_i (-1)^i c_i|.  Returns a negative value on bad input. */
double tb_cfl_dt_max(int space_order, const double h[3], double vmax);

/* Built-in sponge along one axis: eta[i] = eta_max (d/nbl)^2, d the
 * distance in cells into the layer (1..nbl), eta_max = 3 vmax ln(1000) /
 * (2 nbl h) (Sec. IV-B).  eta: caller-owned host array of n doubles.
 * Errors: TB_EINVAL (n < 1, nbl < 0, h <= 0, NULL eta). */
int tb_sponge_profile(int64_t n, int nbl, double h, double vmax, double* eta);

/* Ricker wavelet q(t_n) = (1 - 2 a) exp(-a), a = (pi f0 (n dt - t0))^2,
 * t0 = 1/f0 when t0 <= 0.  out: caller-owned host array of nt floats.
 * Errors: TB_EINVAL (f0 <= 0, nt < 0, NULL out). */
int tb_ricker(double f0, double dt, int nt, double t0, float* out);

/* --- Diagnostics ---------------------------------------------------- */

/* Run the blocked sweep's bounded device-side wait once, on a device flag
 * that nothing sets, with the given time limit (seconds, > 0 and <= 10).
 * The waiting kernel gives up after the limit, records the timeout in a
 * device flag and returns, leaving the context usable; the call then
 * returns TB_ETIMEOUT.  Any other result means the wait is broken.
 * Synchronises `stream`.  Errors: TB_EINVAL, TB_ECUDA. */
int tb_selftest_wait(double timeout_s, void* stream);

/* Measure, with this library's own kernels, the two peaks its rooflines are
 * read against: *hbm_gbs = HBM copy bandwidth in GB/s (read + write bytes
 * of a float4 copy between two 1 GiB device buffers, best of 5 after a
 * warm-up), *fp32_tflops = FP32 throughput in TFLOP/s of independent chains
 * of packed f32x2 FMAs on every SM (4 flops per packed FMA).  Allocates and
 * frees 2 GiB of device memory on `stream` and synchronises it.  Output
 * pointers are host memory.  Errors: TB_EINVAL (NULL output), TB_ENOMEM,
 * TB_ECUDA; on error both outputs are 0. */
int tb_measure_peaks(double* hbm_gbs, double* fp32_tflops, void* stream);

/* --- Allocation-free inspection --------------------------------------- */

/* The source-point inspector of tb_set_sources (affected grid points of a
 * set of off-grid points, ascending linear index), for callers that must not
 * allocate device memory while they run: code with a device memory budget
 * fixed at start-up, or a real-time loop where a cudaMalloc would
 * synchronise the device.  This call allocates nothing: its scratch is a
 * fixed array of about 1.8 MB in device memory, which every GPU that loads
 * the library holds until the process exits.  (The paper has no
 * counterpart; it is an interface addition of this library.)
 *   n, h       grid shape and spacing (host arrays): 2 <= n_d <= 65535,
 *              n0 n1 n2 < 2^40, h_d > 0, else TB_EINVAL.
 *   npt        number of points, 0..8192; more is rejected with TB_EINVAL.
 *   coords     device array [npt][3] of FP64 metres.
 *   lin        device array with room for 8 * npt int64 values; receives the
 *              ascending linear indices (x n1 + y) n2 + z of the affected
 *              points (the paper's SID order).
 *   npts       device int64: receives their number, or -1 when a coordinate
 *              lies outside [0, (n_d - 1) h_d].
 * Asynchronous on `stream`, which must belong to the current device
 * (TB_EINVAL otherwise; NULL is the current device's legacy stream).  The
 * first call on each device looks up the device address of the scratch
 * array (with that device current) and keeps it for the process: make that
 * first call before any stream capture, and make no call on a device after
 * a cudaDeviceReset of it.  Nothing in the array has to
 * start at zero: each call clears its own out-of-grid flag and overwrites
 * the rest before reading it.  Every call shares the one array and it keeps
 * the last call's contents: calls that overlap on the GPU
 * (different streams without ordering between them) race and give wrong
 * results; order them, e.g. on one stream.  Errors: TB_EINVAL, TB_ECUDA. */
int tb_inspect_points_noalloc(const int64_t n[3], const double h[3], int npt, const double* coords,
                              int64_t* lin, int64_t* npts, void* stream);

/* Adjoint-state gradient of the acoustic propagation (the FWI / RTM use of
 * the propagator that Sec. I motivates), for the model, sources and
 * receivers set on the handle, dt and damping held fixed:
 *   residual  [nt][nrec] float (host or device): adjoint traces r, e.g. the
 *             derivative of a misfit with respect to the traces;
 *   grad_vp   [n0][n1][n2] float (host or device, may be NULL): receives
 *             d<d(vp), r>/d vp with d the traces of tb_forward;
 *   grad_src  [nsrc][nt] float (host or device, may be NULL): receives
 *             d<d, r>/d q (the adjoint of the wavelet-to-trace map);
 *   n_snapshots >= 1: the forward pass keeps a checkpoint (u^n, u^{n-1})
 *             every ceil(nt / n_snapshots) steps; the backward pass
 *             recomputes each segment once from its checkpoint (one step
 *             into the next segment) into a buffer of
 *             ceil(nt / n_snapshots) + 2 states.
 * The adjoint is the exact transpose of the discrete one-step recurrence:
 * lam^k = L(D lam^{k+1}) + B lam^{k+1} + C lam^{k+2} + P^T r[k-1] with
 * D = dt^2/(m + a), B = 2m/(m + a), C = (a - m)/(m + a), a = eta dt/2,
 * computed as mu = D lam, which obeys the forward recurrence backward in
 * time (the forward sweep kernel runs it); the gradient sums
 * lam^k d(step k)/dm over the steps in FP64.  Device scratch about
 * (2 n_snapshots + ceil(nt / n_snapshots) + 5) fields, allocated and freed
 * by the call.  Synchronises `stream`.  Overwrites the handle's
 * wavefields (tb_get_field needs a new tb_forward).  Acoustic only.
 * Errors: TB_ESTATE, TB_EINVAL, TB_ENOMEM, TB_ECUDA, TB_ETIMEOUT. */
int tb_adjoint_gradient(tb_handle* h, int nt, const float* residual, float* grad_vp, float* grad_src,
                        int n_snapshots, void* stream);

/* Checkpointing of tb_adjoint_gradient_ckpt. */
enum { TB_CKPT_SEGMENTS = 0, TB_CKPT_BINOMIAL = 1 };

/* tb_adjoint_gradient with a choice of how the backward pass gets the
 * forward states it needs (same arguments and results otherwise; both give
 * bit-identical gradients, every state being the same sequence of one-step
 * sweeps from the zero initial condition):
 *   TB_CKPT_SEGMENTS  as tb_adjoint_gradient: a checkpoint every
 *     ceil(nt/S) steps and a segment buffer of ceil(nt/S) + 2 states; every
 *     step is recomputed once (2 nt forward steps in all); device scratch
 *     about (2 S + ceil(nt/S) + 5) fields;
 *   TB_CKPT_BINOMIAL  exactly S = n_snapshots stored states (two fields
 *     each) in Griewank's binomial schedule (tb_plan_checkpoints), the least
 *     recomputation S states allow; device scratch (2 S + 3) fields plus
 *     the adjoint's own 4 (two mu fields, the FP64 gradient sum), whatever
 *     nt is.  1 <= n_snapshots <= 4096.
 * tb_adjoint_stats reports the forward steps the call ran and its scratch.
 * Errors: as tb_adjoint_gradient, TB_EINVAL for another checkpointing. */
int tb_adjoint_gradient_ckpt(tb_handle* h, int nt, const float* residual, float* grad_vp, float* grad_src,
                             int n_snapshots, int checkpointing, void* stream);

/* Accounting of the last adjoint gradient of the handle: *forward_steps =
 * the forward time steps (one-step sweeps) it ran, its reverse steps' own
 * recomputations included (-1 before any), *scratch_bytes = the device
 * bytes it allocated for its own use and freed before returning (states,
 * adjoint fields, FP64 sum, tables).  Host outputs.  Errors: TB_EINVAL
 * (NULL argument). */
int tb_adjoint_stats(const tb_handle* h, int64_t* forward_steps, size_t* scratch_bytes);

/* Host-side binomial checkpoint schedule (no GPU needed), the one
 * TB_CKPT_BINOMIAL runs.  X_n = (u^n, u^{n-1}) is the forward state after n
 * steps (X_0 = 0, never stored); reversing forward step n (adjoint step
 * n + 1) needs X_n and runs that forward step once itself.  With
 * n_snapshots = S storage slots, writes up to max_actions actions of 5 ints
 * (kind, from, to, src, dst) in execution order (caller-owned):
 *   kind 0, advance: compute X_to from X_from held at src into dst;
 *   kind 1, reverse: reverse forward step `from` (= to) with X_from at src;
 * locations: a slot 0 .. S-1, -1 the zero state X_0, -2 a work pair.  The
 * reverse actions come in the order nt-1 .. 0.  *forward_steps (may be
 * NULL) receives the forward steps of the schedule (advanced steps plus one
 * per reverse action), the minimum for S slots: t l - C(S + t + 1, t - 1)
 * advanced steps, t the least integer with C(S + 1 + t, t) >= nt.  Returns
 * the number of actions (which may exceed max_actions), or -TB_EINVAL for
 * nt < 1, S < 0 or S > 4096. */
int tb_plan_checkpoints(int nt, int n_snapshots, int* actions, int max_actions, int64_t* forward_steps);

/* Stability limits of the TTI and elastic schemes (seconds), -1 on bad
 * arguments.  TTI: 2 / (vmax sqrt(1 + 2 eps_max) sqrt(sum_d (S1/h_d)^2)),
 * S1 = max |2 sum a_i sin(i t)| over the centred first-derivative weights
 * (the largest eigenvalue of the coupled p, r system is at most (1 + 2 eps)
 * |s|^2 when eps >= delta).  Elastic: 2 / (vpmax sqrt(sum_d (S/h_d)^2)),
 * S = max |2 sum c_k sin((k - 1/2) t)| over the staggered weights. */
double tb_tti_dt_max(int space_order, const double h[3], double vmax, double eps_max);
double tb_elastic_dt_max(int space_order, const double h[3], double vpmax);

/* --- Batched small shots (continuous batching) ------------------------ */

/* A batch advances several acoustic shots (FP32 storage, one space order)
 * together: every time step of every shot in the batch is one launch of the
 * one-step sweep (Sec. IV-C's spatially blocked kernel) whose CTAs take the
 * (shot, tile) entries of a concatenated pass table and read each shot's
 * fields, tensor maps and tables from device memory.  Shots join and leave
 * between steps, so a serving loop admits new shots while others run
 * (continuous batching); each shot gives the same traces and wavefields,
 * bit for bit, as tb_forward(TB_ONESTEP) alone.  Large shots are better
 * served alone with TB_BLOCKED.  A batch lives on the device that is current
 * at tb_batch_create; use one stream for all calls on a batch and its
 * shots, and keep a shot's handle alive and untouched (no other call on it)
 * from tb_batch_add until tb_batch_finished returns it.  The paper has no
 * counterpart; this is the serving path of the library. */
typedef struct tb_batch tb_batch;

/* Create a batch for at most max_shots (1..4096) shots at a time; allocates
 * about 2.3 KB of device memory per shot.  Errors: TB_EINVAL, TB_ENOMEM. */
int tb_batch_create(int max_shots, tb_batch** out);

/* Release the batch (stream-ordered frees on its last stream); its shots'
 * handles stay the caller's.  NULL is accepted.  Returns TB_OK. */
int tb_batch_destroy(tb_batch* b);

/* Admit a shot: handle h with tb_set_model done (sources and receivers
 * optional, as for tb_forward), nt steps from zero initial conditions,
 * traces: device [nt][nrec] float (caller-owned, may be NULL).  The shot's
 * wavefields are zeroed on `stream`; its first step is the batch's next
 * launch.  nt = 0 finishes at once.  Errors: TB_EINVAL (not acoustic FP32,
 * a space order other than the batch's, host traces, nt beyond the wavelet
 * length, the batch full, h already in it), TB_ESTATE (no model), TB_ECUDA. */
int tb_batch_add(tb_batch* b, tb_handle* h, int nt, float* traces, void* stream);

/* Advance every shot in the batch by up to nsteps steps (one launch per
 * step; fewer when the batch empties), asynchronously on `stream`; a shot's
 * receiver traces are finalised every 16 steps and at its last step, and a
 * shot that reaches its nt leaves the batch (tb_batch_finished).  Errors:
 * TB_EINVAL, TB_ENOMEM, TB_ECUDA. */
int tb_batch_step(tb_batch* b, int nsteps, void* stream);

/* Shots in the batch that have not finished. */
int tb_batch_active(const tb_batch* b);

/* Pop up to max_out finished shots' handles into out (caller-owned array),
 * *n = how many.  Their traces and final wavefields (tb_get_field) are ready
 * once the work enqueued so far on the batch's stream completes.  Errors:
 * TB_EINVAL. */
int tb_batch_finished(tb_batch* b, tb_handle** out, int max_out, int* n);

/* Number of CUDA kernels this library has launched in this process (all
 * handles, all devices), for accounting in benchmarks. */
uint64_t tb_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* TB_H */
