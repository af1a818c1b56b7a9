/*
 * mmod.h — C ABI of the GB300 (sm_103a) acoustic propagator library.
 *
 * The library time-steps the acoustic isotropic constant-density wave
 * equation of Minimod (arXiv 2007.06048):
 *   Eq. 1   (1/v^2) p_tt - lap p = f
 *   Eq. 5   p^{n+1} - Q p^n + p^{n-1} = dt^2 v^2 f^n,  Q = 2 + dt^2 v^2 lap
 *   Sec. 3  lap as the 25-point star  sum_m c_am [p(+m) + p(-m) - 2 p],
 *           order-8 Taylor weights (radius 4 per axis)
 *   Alg. 1  p^0 = 0, then per step: solve for p^{n+1}, add the source term
 *   Alg. 2  the inner region (Eq. 5) surrounded by six damping regions
 * with damping layers, point sources and grid-point receivers.  The readings
 * taken where the paper is silent are fixed by this ABI:
 *   - u = 0 outside the grid;
 *   - inside the layers the update is
 *       u^{n+1} = [2u^n - (1 - e) u^{n-1} + c (lap u^n + s^n)] / (1 + e),
 *     c = dt^2 v^2, e = dt (eta_x(i) + eta_y(j) + eta_z(k)),
 *     eta_a(i) = eta_max,a (d/L)^2, d = max(L - i, i - (n_a - 1 - L), 0),
 *     eta_max,a = 3 vmax ln(1/R) / (2 L h_a)   (e = 0 gives Eq. 5 exactly);
 *   - a point source adds c(x_s) w[n] / (hx hy hz) to the numerator above;
 *   - traces[n][r] = u^{n+1} at receiver r, after the source add of step n.
 *
 * Conventions.  Grid index (i, j, k) along (x, y, z); k = 0 is the surface.
 * Volumes are FP32 [nz][ny][nx] (x fastest), dense, no padding.  The layers
 * are part of the grid.  All arithmetic on the GPU is FP32.
 *
 * Pointers.  Every array argument may point to device memory or to host
 * memory (pageable or pinned); the library detects which and stages host
 * buffers through its own device buffers on the given stream.  The caller
 * owns every pointer it passes; the handle owns its internal wavefields,
 * coefficient volume, profiles and staging buffers.
 *
 * Streams.  `stream` is a cudaStream_t (NULL = the legacy default stream).
 * Calls are stream-ordered; a call returns once its work is enqueued, except
 * where a call says it synchronises.  With host output buffers the call
 * synchronises the stream before returning so that the data is in place.
 *
 * Errors.  Every call returns an mmod_status; on failure nothing is enqueued
 * (argument errors) or the CUDA error is latched in the handle and returned
 * by this and every later call.  mmod_last_error() describes the last failure.
 * A handle is not thread-safe: one host thread at a time.
 */
#ifndef MMOD_H
#define MMOD_H

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, declared without the CUDA headers. */
typedef struct CUstream_st *mmod_stream;

typedef enum {
    MMOD_OK = 0,
    MMOD_ERR_ARG = -1,          /* invalid argument or configuration */
    MMOD_ERR_UNSTABLE = -2,     /* dt too large for the model (CFL bound) */
    MMOD_ERR_OOM = -3,          /* device allocation failed */
    MMOD_ERR_CUDA = -4,         /* a CUDA call failed; see mmod_last_error */
    MMOD_ERR_TIMEOUT = -5,      /* a bounded device-side wait gave up */
    MMOD_ERR_STATE = -6,        /* call out of order (e.g. forward before set_model) */
    MMOD_ERR_UNSUPPORTED = -7   /* valid for the oracle, not on this GPU path */
} mmod_status;

typedef struct mmod_handle mmod_handle;

/* Problem description.  Mirrors the paper's run parameters (--ngrid,
 * --dgrid, --nsteps; "stencil", "ndamping", "source_loc", "nreceivers" of
 * the Sec. 5.3 printout). */
typedef struct {
    int nx, ny, nz;          /* grid points, damping layers included; each >= 1 and >= 2*nbl */
    double hx, hy, hz;       /* grid spacing, metres, > 0 */
    double dt;               /* time step, seconds, > 0 */
    int nt;                  /* number of time steps, >= 0 */
    int order;               /* spatial order; the GPU path supports 8 only */
    int nbl;                 /* damping width in cells on all six faces, >= 0 */
    double damp_R;           /* target reflection of the layers, 0 < R < 1 (1e-3 typical) */
    int nsrc;                /* number of point sources, >= 0 */
    const int *src_ijk;      /* host [nsrc][3] (i, j, k); copied by mmod_create */
    int nrec;                /* number of receivers, >= 0 */
    const int *rec_ijk;      /* host [nrec][3] (i, j, k); copied by mmod_create */
    int free_surface;        /* 1: free surface at k = 0 (the paper's surface option,
                                Sec. 3): p = 0 on that plane through the odd image
                                u(-m) = -u(m), no damping layer under it, sources on
                                the plane do nothing and receivers there read 0;
                                needs nz >= 5.  0: damping layers on all six faces. */
    int boundary;            /* MMOD_BOUNDARY_DAMPING (0): the layers damp (u_tt + 2 eta u_t);
                                MMOD_BOUNDARY_CPML (1): the nbl-cell layers are a
                                convolutional PML (the paper's boundary, Sec. 3) with
                                memory variables psi_a, zeta_a per axis, profiles
                                d = d0 (x/L)^2, d0 = 3 vmax ln(1/damp_R) / (2 L h),
                                alpha = pi cpml_f0 (1 - x/L); forward runs only
                                (adjoint, gradient, fused batches, persistent runs and
                                the allocation-free path answer UNSUPPORTED). */
    double cpml_f0;          /* CPML frequency shift, Hz (>= 0; the source's peak
                                frequency is typical) */
} mmod_config;

enum { MMOD_BOUNDARY_DAMPING = 0, MMOD_BOUNDARY_CPML = 1 };

/* Create a handle on CUDA device `device`: validates the configuration,
 * copies the source/receiver lists and allocates the wavefields and
 * coefficient volume (about 3 * 4 * nx*ny*nz bytes, rows padded to 128 B).
 * Errors: ARG (bad sizes, positions outside the grid, null lists with
 * nonzero counts, order != 8 -> UNSUPPORTED), OOM, CUDA.  *out is NULL on
 * failure. */
mmod_status mmod_create(const mmod_config *cfg, int device, mmod_handle **out);

/* Release everything the handle owns.  Synchronises the device work it
 * enqueued.  NULL is accepted. */
mmod_status mmod_destroy(mmod_handle *h);

/* Load a velocity model vel [nz][ny][nx] (m/s, FP32, all > 0): computes
 * c = dt^2 v^2 (rounded once from FP64 to FP32), the model maximum vmax and
 * the damping profiles.  Synchronises `stream` (vmax is read back for the
 * stability check).  Errors: ARG (null, non-positive or non-finite values),
 * UNSTABLE when dt * vmax * sqrt(sum_a 6.5016 / h_a^2) > 2 (the order-8
 * stencil's largest symbol magnitude is 6.5016 / h^2 per axis), CUDA. */
mmod_status mmod_set_model(mmod_handle *h, const float *vel, mmod_stream stream);

/* Forward modelling, Alg. 1: nt steps from u^{-1} = u^0 = 0 (or from the
 * state given by mmod_set_state, consumed by this call).
 *   wavelet  [nsrc][nt] FP32 source time functions w[n] (n = 0..nt-1);
 *            may be NULL when nsrc == 0
 *   traces   [nt][nrec] FP32 output, traces[n][r] = u^{n+1}(x_r); may be
 *            NULL when nrec == 0
 *   final_u  optional [nz][ny][nx] FP32 output u^{nt}
 * Each pointer may be host or device memory.  Host traces are downloaded
 * in eight row chunks on an internal stream while the time loop still runs
 * (each chunk once the steps that finish its rows are done); with any host
 * output the call returns after the data is in host memory.
 * Errors: STATE (no model), ARG, CUDA, TIMEOUT. */
mmod_status mmod_forward(mmod_handle *h, const float *wavelet, float *traces,
                         float *final_u, mmod_stream stream);

/* Adjoint of the forward map wavelet -> traces (for a fixed model): given
 * resid [nt][nrec] (FP32, the data-space vector r), writes adj_src [nsrc][nt]
 * = F^T r, i.e. <F w, r> = <w, F^T r> for every wavelet w.  It is the
 * transpose of the scheme above, run backward in time (the paper's Eq. 5
 * is linear in the source term; the transpose is this library's addition for
 * inversion, which the paper names as the use of forward modelling).  Uses
 * the handle's wavefield buffers (the forward state is overwritten).
 * Errors: STATE (no model), ARG, CUDA, TIMEOUT. */
mmod_status mmod_adjoint(mmod_handle *h, const float *resid, float *adj_src, mmod_stream stream);

/* Checkpoint storage of mmod_gradient. */
/* MMOD_CKPT_BF16 / MMOD_CKPT_FP16: the value divided by max |u| over its z
 * plane, rounded to BF16 / FP16 (one FP32 scale per plane).
 * MMOD_CKPT_BFP16: block floating point, one FP32 scale s = max |u| over each
 * block of 32 consecutive x values and round(u * 32767 / s) as int16 per
 * value (error <= s / 65534; 2.125 bytes per value). */
enum { MMOD_CKPT_FP32 = 0, MMOD_CKPT_BF16 = 1, MMOD_CKPT_FP16 = 2, MMOD_CKPT_BFP16 = 3 };

/* Gradient of J = 1/2 sum_n |traces^n - d_obs^n|^2 with respect to the
 * velocity, for the current model, given wavelet [nsrc][nt] and the residual
 * resid [nt][nrec] = traces - d_obs of that model.  Writes grad_v
 * [nz][ny][nx] (FP32, dJ/dv in J-units per m/s):
 *   dJ/dv = 2 dt^2 v sum_n mu^{n+1} (L u^n + s^n) = (2 / v) sum_n psi^{n+1} g^n,
 * mu = psi / c the adjoint state (zero-lag imaging condition), g^n = L u^n +
 * s^n written by the step kernel that advances u^n; all of it FP32.  The forward states are recomputed from
 * ckpt_count checkpoints, by the handle's scheme (mmod_set_option
 * MMOD_OPT_CKPT_SCHEME):
 *   MMOD_SCHEME_SEGMENTS (default): the run is cut into ckpt_count segments;
 *     each is replayed once, writing g^n of its ceil(nt / ckpt_count) steps
 *     into FP32 volumes (plus two for the replayed state), so the cost is two
 *     forward runs and one adjoint run; with FP32 storage and ckpt_count >= nt
 *     g^n of every step is kept instead (nt + 2 volumes, one forward run and
 *     one adjoint run);
 *   MMOD_SCHEME_REVOLVE: binomial checkpointing (mmod_revolve_schedule) with
 *     ckpt_count slots and two FP32 work volumes; the forward steps replayed
 *     are the fewest any schedule with that many slots needs (about r forward
 *     runs when C(ckpt_count + 1 + r, r) >= nt).
 * Every scheme also holds two adjoint volumes and the FP32 accumulator.  A
 * checkpoint holds (u^{n-1}, u^n), stored as MMOD_CKPT_FP32 (exact replay:
 * both schemes give the same bits) or in 16 bits per value (BF16 / FP16 with
 * one scale per z plane, BFP16 with one per 32 values; stepping stays FP32).  The rounding of a 16-bit checkpoint is noise at the
 * grid scale, which L in g^n amplifies by the ratio of the stencil's largest
 * symbol to the wavefield's: the gradient error grows with the points per
 * wavelength.  Device memory: mmod_gradient_memory().  Errors: STATE, ARG,
 * OOM, CUDA, TIMEOUT. */
mmod_status mmod_gradient(mmod_handle *h, const float *wavelet, const float *resid, float *grad_v,
                          int ckpt_count, int ckpt_dtype, mmod_stream stream);

/* Bytes of device memory mmod_gradient allocates for this checkpoint layout
 * under the handle's current scheme (on top of the handle's own volumes);
 * -1 for invalid arguments. */
long long mmod_gradient_memory(const mmod_handle *h, int ckpt_count, int ckpt_dtype);

/* Binomial checkpointing schedule (Griewank 1992; Griewank & Walther,
 * revolve) reversing nsteps time steps with `snaps` checkpoint slots besides
 * the initial state (zero, never stored).  Host code: no device is touched.
 * Writes up to cap actions as int triples {kind, a, b} into `actions`:
 *   MMOD_REV_ADVANCE  a, b: step the working state from step a to step b;
 *   MMOD_REV_SAVE     a, b: store the working state (at step b) in slot a;
 *   MMOD_REV_RESTORE  a, b: load the state of step b from slot a (a = -1:
 *                           the zero initial state, b = 0);
 *   MMOD_REV_REVERSE  a:    with the working state at step a, take forward
 *                           step a and the matching adjoint step (steps are
 *                           reversed in the order nsteps-1, ..., 0).
 * *count = number of actions, *advanced = steps advanced by ADVANCE actions
 * (both optional).  actions = NULL with cap = 0 only queries the sizes.
 * Errors: ARG (negative argument, or cap too small with actions given). */
enum { MMOD_REV_ADVANCE = 0, MMOD_REV_SAVE = 1, MMOD_REV_RESTORE = 2, MMOD_REV_REVERSE = 3 };
mmod_status mmod_revolve_schedule(int nsteps, int snaps, int *actions, long long cap, long long *count,
                                  long long *advanced);

/* ---- Stencil weights ----------------------------------------------------
 * The Laplacian's weights c_1..c_4 (unit spacing; the kernels use
 * c_m / h_a^2 on axis a).  Default: the order-8 Taylor weights 8/5, -1/5,
 * 8/315, -1/560 (Sec. 3).  Sec. 3 also allows weights that give up formal
 * order for a smaller dispersion error; the library computes them
 * as the minimiser of  int_0^kmax (sum_m 2 c_m (1 - cos m k) / k^2 - 1)^2 dk
 * (relative error of the 1-D symbol over the band kh in [0, kmax], radians
 * per cell, 0 < kmax <= pi) subject to sum_m m^2 c_m = 1.
 *
 * mmod_optimized_coefficients: writes c_1..c_4 into c4 (host).  Errors: ARG.
 * mmod_set_fd_coefficients: the handle uses c4 (host, 4 doubles; NULL = the
 *   Taylor weights) from its next run on; c4 must satisfy sum m^2 c_m = 1
 *   to 1e-6.  The stability bound follows the weights (max over k of
 *   sum 2 c_m (1 - cos m k), 2048/315 for Taylor); a loaded model that
 *   violates it is dropped (UNSTABLE).  The allocation-free entry point uses
 *   the Taylor weights.  Errors: ARG, UNSTABLE. */
mmod_status mmod_optimized_coefficients(double kmax, double *c4);
mmod_status mmod_set_fd_coefficients(mmod_handle *h, const double *c4);

/* FP64 sum of a[i] * b[i] over n FP32 device values (dot-product tests,
 * gradient norms).  Synchronises `stream`.  Errors: ARG, OOM, CUDA. */
mmod_status mmod_dot(const float *a, const float *b, long long n, double *out, mmod_stream stream);

/* Test hook: the next mmod_forward starts from u^{-1} = u_prev, u^0 = u_cur
 * ([nz][ny][nx] FP32, either may be NULL for zeros) instead of zeros (with a
 * free surface, the plane k = 0 of both is set to 0). */
mmod_status mmod_set_state(mmod_handle *h, const float *u_prev, const float *u_cur,
                           mmod_stream stream);

/* Copy the last forward's final state u^{nt-1}, u^{nt} (either may be NULL). */
mmod_status mmod_get_state(mmod_handle *h, float *u_prev, float *u_cur, mmod_stream stream);

/* Kernel selection: MMOD_KERNEL_AUTO (default) and MMOD_KERNEL_TMA run the
 * TMA-pipelined kernel; MMOD_KERNEL_SIMPLE runs the plain one-thread-per-point
 * kernel, which performs the identical FP32 operations per point
 * (validation).  All kernels produce the same bits.  Errors: ARG (unknown
 * id), UNSUPPORTED (the grid has no TMA plan). */
enum { MMOD_KERNEL_AUTO = 0, MMOD_KERNEL_SIMPLE = 1, MMOD_KERNEL_TMA = 2 };
mmod_status mmod_set_kernel(mmod_handle *h, int kernel);

/* Compiled variants of the TMA kernel (tile shape, points per thread, z
 * queue handling), for tuning.  mmod_tma_variant_name returns a static
 * description ("" out of range).  mmod_set_tma_variant selects one for the
 * handle (-1 = automatic).  All variants produce the same bits.  Errors:
 * ARG (out of range), UNSUPPORTED (no TMA plan). */
int mmod_tma_variant_count(void);
/* Resources of variant v on the current device, 14 ints: threads per CTA,
 * dynamic shared bytes, then {registers per thread, local bytes per thread,
 * static shared bytes, resident CTAs per SM} for its one-step, batch and
 * persistent kernels (-1 where not compiled).  Errors: ARG (out of range). */
mmod_status mmod_tma_variant_info(int v, int *out14);
const char *mmod_tma_variant_name(int v);
mmod_status mmod_set_tma_variant(mmod_handle *h, int v);

/* Options of a handle:
 *   MMOD_OPT_PDL          0 / 1: launch each TMA step as a programmatic
 *                         dependent of the previous one, so its set-up
 *                         overlaps the previous step's tail (default 1; the
 *                         same bits either way);
 *   MMOD_OPT_CKPT_SCHEME  MMOD_SCHEME_SEGMENTS (default) or
 *                         MMOD_SCHEME_REVOLVE: checkpointing of mmod_gradient;
 *   MMOD_OPT_PERSISTENT   0 / 1: run the time loop of mmod_forward and
 *                         mmod_adjoint as one cooperative launch in which each
 *                         work unit (64 x 16 tile x z range) starts a step as
 *                         soon as its neighbours finished the previous one
 *                         (default 0: slower than one launch per step on the
 *                         measured grids; the same bits either way; variants
 *                         without a persistent form ignore it);
 *   MMOD_OPT_ZLEN         >= 0: planes per z range of a CTA (0 = the plan's
 *                         choice, which fills one wave of resident CTAs; in a
 *                         batch created after it is set: the shot's z ranges,
 *                         at least 4 planes, 0 = 256); the same bits for any
 *                         value;
 *   MMOD_OPT_PERSISTENT_CTAS  >= 0: at most this many CTAs for the persistent
 *                         run (0 = as many as fit at once; a small value makes
 *                         each CTA serve many units, for tests);
 *   MMOD_OPT_CLAIM        0..2^20: planes per work unit of a work-claiming
 *                         step launch (0 = off: one CTA per unit of the
 *                         plan).  At most one wave of CTAs serves the units
 *                         (64 x 16 tile x this many planes): each CTA takes
 *                         its first unit by its index, then claims the next
 *                         free unit from a per-launch counter until none is
 *                         left, so early finishers take the remaining work
 *                         (TMA variants 1, 2 and 6; others ignore it); the
 *                         same bits for any value;
 *   MMOD_OPT_CPML_PLANES  0..4096: about this many layer lines per thread
 *                         (row segments per warp along x) in the CPML
 *                         layer passes (0 = the default, 1); the same bits
 *                         for any value;
 *   MMOD_OPT_CPML_TILES   0 / 1 (default 1): run the CPML layer pass of an
 *                         axis as tiles of 128 lines loaded whole into shared
 *                         memory by bulk-tensor copies, where the axis allows
 *                         it (layer width 8 or 20, the two layer ranges
 *                         apart; along x also nx a multiple of 4); 0: the
 *                         marching passes only.  The same bits either way;
 *   MMOD_OPT_TEST_STALL   1: test hook of the failure path.  The next
 *                         persistent run (of this handle, or of a persistent
 *                         batch holding it) waits for neighbour counters that
 *                         nothing sets; every wait gives up after 100 ms, the
 *                         kernel returns and the call reports MMOD_ERR_TIMEOUT
 *                         (the handle stays in that state; the device and
 *                         other handles stay usable).
 * Errors: ARG (unknown option or value). */
enum { MMOD_OPT_PDL = 2, MMOD_OPT_CKPT_SCHEME = 3, MMOD_OPT_PERSISTENT = 4, MMOD_OPT_PERSISTENT_CTAS = 5,
       MMOD_OPT_TEST_STALL = 6, MMOD_OPT_ZLEN = 7, MMOD_OPT_CPML_PLANES = 8, MMOD_OPT_CLAIM = 9,
       MMOD_OPT_CPML_TILES = 10 };
enum { MMOD_SCHEME_SEGMENTS = 0, MMOD_SCHEME_REVOLVE = 1 };
mmod_status mmod_set_option(mmod_handle *h, int option, int value);

/* CTAs of the persistent kernel the next mmod_forward / mmod_adjoint of this
 * handle will launch; 0 when it runs one launch per step (plain kernel, a
 * variant without a persistent form, z ranges thinner than the stencil
 * radius, or MMOD_OPT_PERSISTENT off); -1 for a null handle. */
int mmod_persistent_grid(const mmod_handle *h);

/* Launch plan of the active TMA variant: writes 8 ints {variant, tiles_x,
 * tiles_y, z_chunks, planes_per_chunk, grid, block, resident_ctas_per_sm}.
 * Errors: ARG, UNSUPPORTED (no TMA plan). */
mmod_status mmod_get_plan(const mmod_handle *h, int *out8);

/* Number of kernel launches the last mmod_forward enqueued (all of this
 * library's kernels, including set-up and gathers). */
long long mmod_last_launch_count(const mmod_handle *h);

/* Device time in milliseconds of the last mmod_forward's time loop (all
 * step and gather kernels between two CUDA events recorded on the call's
 * stream inside the captured graph).  Waits for that work to finish.
 * Returns a negative value when no loop has run. */
float mmod_last_loop_ms(mmod_handle *h);

/* dt = cfl * hmin / vmax (the CFL reading of the workloads).  Returns a
 * negative value for non-positive arguments. */
double mmod_cfl_dt(double cfl, double hmin, double vmax);

/* Human-readable description of the handle's last failure ("" if none).
 * The string is owned by the handle and valid until its next call.  With
 * h == NULL: the calling thread's last mmod_create or mmod_forward_noalloc
 * failure. */
const char *mmod_last_error(const mmod_handle *h);

/* Self-check of the damping reciprocal used by the step kernels (hardware
 * approximate reciprocal plus one Newton-Raphson step) against CUDA's
 * correctly rounded reciprocal, on n values of d in [1, 8), on the current
 * device.  Writes the largest difference in units in the last place.
 * Synchronous; returns MMOD_OK, ARG, OOM or CUDA. */
int mmod_check_recip(int n, unsigned int *max_ulp_out);

/* Allocation-free forward run, for callers that may not allocate device
 * memory (a framework that accounts for every byte through its own pool, a
 * process that reserves all device memory at start-up, real-time code that
 * cannot afford an allocation's implicit synchronisation or failure).  The
 * paper has no counterpart; this is a service of the library.
 *
 * Computes exactly what mmod_create + mmod_set_model + mmod_forward compute
 * for the same configuration, from zero initial state, without a handle and
 * without calling cudaMalloc, cudaFree or any allocating library routine: its
 * scratch (wavefields, coefficient volume, profiles, source/receiver tables)
 * is one fixed block of device memory inside the library, about 25 MB, that
 * every GPU loading the library keeps until the process exits.
 *   Limits: nx, ny, nz <= 4096; (nx rounded up to 32) * ny * nz <= 2097152;
 *   nsrc <= 64; nrec <= 65536; order 8.  Larger problems are rejected with
 *   MMOD_ERR_ARG (use the handle API).
 *   vel, wavelet, traces, final_u: memory of `device` (or managed memory),
 *   layouts as in mmod_set_model / mmod_forward; final_u may be NULL.
 * Synchronous: returns after the work on `stream` has finished, also when a
 * call fails after enqueuing work.  Every call shares the block (each call
 * clears what must start at zero), so calls that overlap on the GPU race:
 * serialise them.  Each call looks up the block's device address
 * (cudaGetSymbolAddress, which allocates nothing) with `device` current; the
 * first call on a device may load the library's device code, so make it
 * before any stream capture.  Errors: ARG, UNSTABLE, UNSUPPORTED, CUDA,
 * TIMEOUT; the message is available from mmod_last_error(NULL) on the
 * calling thread. */
mmod_status mmod_forward_noalloc(const mmod_config *cfg, int device, const float *vel,
                                 const float *wavelet, float *traces, float *final_u,
                                 mmod_stream stream);

/* ---- Batched shots ------------------------------------------------------
 * A batch advances several shots (one handle each: any grid sizes, the same
 * nt, the same device) together, in one of two modes (mmod_batch_set_mode):
 *   MMOD_BATCH_STREAMS (default): each shot's own time loop (the handle's
 *     graph of one-step kernels) on one of four internal streams forked
 *     from and joined back to the caller's stream, so the shots' kernels
 *     overlap;
 *   MMOD_BATCH_FUSED: one kernel launch per time step covers all shots, the
 *     nt launches captured once into a CUDA graph;
 *   MMOD_BATCH_PERSISTENT: one cooperative launch runs every shot's whole
 *     time loop: each work unit (a shot's 64 x 16 tile and z range) starts a
 *     step once the neighbouring units of its shot have finished the
 *     previous one (per-unit counters, waits bounded at 100 ms: a give-up
 *     is reported as MMOD_ERR_TIMEOUT); TMA variants 2 and 5 only.
 * Both give every shot the bits it gets alone.  The batch refers to the
 * handles (they keep their buffers, models and geometry); destroy the batch
 * before its handles.  Each handle's buffers hold its shot's final state
 * after mmod_batch_forward (mmod_get_state). */
typedef struct mmod_batch mmod_batch;

/* Errors: ARG (null or mismatched handles), UNSUPPORTED (a grid without TMA
 * plan), OOM, CUDA; message from mmod_last_error(NULL). */
mmod_status mmod_batch_create(mmod_handle *const *shots, int nshots, mmod_batch **out);
mmod_status mmod_batch_destroy(mmod_batch *b);

/* Forward run of every shot from zero state: wavelets[i] [nsrc_i][nt] and
 * traces[i] [nt][nrec_i] are DEVICE pointers (host arrays of nshots
 * pointers; entries may be NULL for shots without sources / receivers).
 * Stream-ordered.  Errors: STATE (a shot without model), ARG, CUDA, TIMEOUT;
 * message from mmod_batch_last_error. */
mmod_status mmod_batch_forward(mmod_batch *b, const float *const *wavelets, float *const *traces,
                               mmod_stream stream);

/* Select the TMA variant used by the batch (see mmod_tma_variant_count); in
 * streams mode it is set on every handle of the batch. */
mmod_status mmod_batch_set_variant(mmod_batch *b, int v);

/* MMOD_BATCH_STREAMS or MMOD_BATCH_FUSED.  Errors: ARG. */
enum { MMOD_BATCH_STREAMS = 0, MMOD_BATCH_FUSED = 1, MMOD_BATCH_PERSISTENT = 2 };
mmod_status mmod_batch_set_mode(mmod_batch *b, int mode);

/* Device time (ms) of the last mmod_batch_forward's loop; waits for it. */
float mmod_batch_last_loop_ms(mmod_batch *b);
const char *mmod_batch_last_error(const mmod_batch *b);

/* ---- Autotuner --------------------------------------------------------
 * Times every compiled TMA variant (points per thread, z-window unroll,
 * ring depths) for `steps` time steps on the handle's (or batch's) own grids
 * and model, without sources, and selects the fastest; *variant_out (may be
 * NULL) receives it.  Synchronises `stream`; overwrites the wavefields.
 * Errors: ARG, STATE (no model), UNSUPPORTED, CUDA. */
mmod_status mmod_autotune(mmod_handle *h, int steps, mmod_stream stream, int *variant_out);
mmod_status mmod_batch_autotune(mmod_batch *b, int steps, mmod_stream stream, int *variant_out);

/* ---- Variable-density propagator (staggered Yee grid) ------------------
 * The paper's first-order acoustic system with variable density (Sec. 3,
 * the "acoustic_iso" kernel):
 *     (1 / (rho v^2)) p_t - div vel = f,      rho vel_t - grad p = 0,
 * on a staggered grid: p, rho, v at the grid points (i, j, k); the particle
 * velocity along axis a half a cell further along a (vx at (i + 1/2, j, k)).
 * Leapfrog with the velocities at half steps; per step n:
 *   vel_a^{n+1/2} = [(1 - e/2) vel_a^{n-1/2} + dt b_a D+_a p^n] / (1 + e/2)
 *   p^{n+1}       = [(1 - e/2) p^n + dt K (sum_a D-_a vel_a^{n+1/2} + s^n)] / (1 + e/2)
 * K = rho v^2, b_a the mean of 1/rho over the half point's two grid points
 * (1/rho of the point itself past the last one), D+_a / D-_a the order-8
 * staggered differences  sum_m a_m (q(i+m) - q(i-m+1)) / h  and
 * sum_m a_m (q(i+m-1) - q(i-m)) / h,  a_m = 1225/1024, -245/3072, 49/5120,
 * -5/7168, with p = vel = 0 outside the grid; e = dt eta, eta the damping
 * profile of mmod.h summed over the axes at each field's own (possibly half)
 * position; s^n = w[n] / (hx hy hz) at a source point; traces[n][r] = p^{n+1}
 * at receiver r.  With cfg->boundary = MMOD_BOUNDARY_CPML the layers are a
 * CPML instead: each derivative gains a memory variable m = B m + G D on its
 * axis's layers (B = exp(-(d + alpha) dt), G = d (B - 1) / (d + alpha), the
 * profiles of the CPML above at the continuous depth into the layer), and
 * e = 0.  cfg->free_surface = 1: p = 0 on the plane k = 0 (the paper's
 * surface option), imposed through images above it, the odd image
 * p(-m) = -p(m) and for v_z, which sits at the half points, the even image
 * v_z(-m) = v_z(m - 1); no top layer; sources on the plane do nothing and
 * receivers there read 0; needs nz >= 5 (ARG otherwise).  Order 8 only
 * (UNSUPPORTED otherwise).  All pointers are DEVICE pointers (ARG
 * otherwise).  Streams, errors and latching as above.
 *
 * mmod_vd_create: as mmod_create; allocates p, vx, vy, vz, dt K, dt / rho
 *   (6 padded volumes; 12 with CPML).  Message: mmod_vd_last_error(NULL).
 * mmod_vd_set_model: vel and rho [nz][ny][nx] FP32 (m/s, kg/m^3, finite and
 *   > 0); synchronises `stream`.  UNSTABLE when
 *   dt veff (2 S) sqrt(sum_a 1/h_a^2) > 2, S = sum_m |a_m| (the symbol's
 *   largest magnitude), veff^2 = max over points of rho v^2 / min(rho over
 *   the point and its six neighbours).
 * mmod_vd_set_state: the next forward starts from state [4][nz][ny][nx] =
 *   p^0, vx, vy, vz at -1/2 (NULL: zeros) instead of zeros (with a free
 *   surface the plane k = 0 of p is set to 0).
 * mmod_vd_forward: nt steps; wavelet [nsrc][nt], traces [nt][nrec],
 *   final_state [4][nz][ny][nx] (p^{nt}, velocities at nt - 1/2; may be NULL).
 * mmod_vd_set_kernel: MMOD_KERNEL_AUTO / MMOD_KERNEL_TMA (the TMA-pipelined
 *   velocity and pressure kernels) or MMOD_KERNEL_SIMPLE (one thread per
 *   point, the same FP32 operations: the same bits).
 * mmod_vd_uses_tma: 1 when the next run uses the TMA kernels (-1: NULL).
 * mmod_vd_set_option: MMOD_OPT_PDL 0 / 1 (default 0): launch the TMA
 *   kernels as programmatic dependents, so that each requests the data its
 *   predecessor does not write (own velocities and buoyancy; p and dt K)
 *   while the predecessor finishes; MMOD_OPT_ZLEN >= 0: planes per z range
 *   of a CTA (0 = the plan's choice).  The same bits for every value.  ARG
 *   otherwise.
 * mmod_vd_get_plan: 6 ints {tiles_x, tiles_y, z_chunks, planes_per_chunk,
 *   CTAs per kernel, threads per CTA}; UNSUPPORTED when no TMA plan.
 * mmod_vd_last_loop_ms / mmod_vd_last_launch_count: as for mmod_forward. */
typedef struct mmod_vd mmod_vd;
mmod_status mmod_vd_create(const mmod_config *cfg, int device, mmod_vd **out);
mmod_status mmod_vd_destroy(mmod_vd *h);
mmod_status mmod_vd_set_model(mmod_vd *h, const float *vel, const float *rho, mmod_stream stream);
mmod_status mmod_vd_set_state(mmod_vd *h, const float *state, mmod_stream stream);
mmod_status mmod_vd_forward(mmod_vd *h, const float *wavelet, float *traces, float *final_state,
                            mmod_stream stream);
mmod_status mmod_vd_set_kernel(mmod_vd *h, int kernel);
int mmod_vd_uses_tma(const mmod_vd *h);
mmod_status mmod_vd_set_option(mmod_vd *h, int option, int value);
mmod_status mmod_vd_get_plan(const mmod_vd *h, int *out6);
float mmod_vd_last_loop_ms(mmod_vd *h);
long long mmod_vd_last_launch_count(const mmod_vd *h);
const char *mmod_vd_last_error(const mmod_vd *h);

/* Library version string, e.g. "mmod-gb300 0.1 sm_103a". */
const char *mmod_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MMOD_H */
