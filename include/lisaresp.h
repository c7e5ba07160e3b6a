/*
 * lisaresp.h -- C ABI of the GB300 (sm_103a) generic LISA time-domain response library.
 *
 * The library computes the response of the LISA constellation to a gravitational-wave
 * strain given as two polarisation time series on a uniform grid (Katz, Bayle, Chua &
 * Vallisneri, arXiv:2204.06633):
 *   - projection (Sec. "Projection on the constellation arms", Eq. instrument-response-to-gw):
 *       y_rs(t) = [H_rs(t - L_rs(t) - k.x_s(t)/c) - H_rs(t - k.x_r(t)/c)] / (2 (1 - k.n_rs(t))),
 *       H_rs = xi+ h+ + xix hx (Eq. projected-strain-ssb), n_rs from emitter s to receiver r;
 *   - TDI (Sec. "Time-delay interferometry", Eqs. tdi1 and tdi2): first- and second-generation
 *     Michelson X, Y, Z built from chained delays D_{i1..in} x(t) = x(t - sum L(t)) (summed,
 *     as in the paper) or nested;
 *   - every delayed read is a centered Lagrange fractional-delay FIR of odd degree p
 *     (Sec. "Implementation"): taps m-(p-1)/2 .. m+(p+1)/2 around m = floor(x);
 *   - orbits: spacecraft positions and link delays on a coarse uniform knot grid, cubic-spline
 *     interpolated to each sample (Sec. "Implementation"); delays not given are solved from
 *     the Newtonian light-time equation L_rs(t) = |x_r(t) - x_s(t - L_rs)| / c.
 *
 * Conventions
 *   - Units: metres, seconds.  c = 299792458 m/s.
 *   - Links are ordered 12, 23, 31, 13, 32, 21 (receiver first); link arrays are [6][n].
 *   - TDI outputs are [3][n]: X, Y, Z (Y, Z by the cyclic permutation 1->2->3->1).
 *   - Output sample n is at time t0 + n*dt; input sample j at t0_h + j*dt (same dt).
 *   - Samples outside an array are zero (zero extension): the operators stay linear and
 *     their transposes exact.  lr_required_margin() gives the input span a full-stencil
 *     output needs.
 *   - h+, hx are the un-rotated polarisations; the polarisation angle psi is applied inside
 *     the response by rotating the antenna patterns by 2 psi (the matrix of Sec. "Template
 *     generation").  For the paper's SSB sign convention pass -h+, -hx.
 *
 * Memory and threading
 *   - Array arguments of compute calls are DEVICE pointers owned by the caller (float64,
 *     contiguous), unless documented as host.  The library never frees or keeps them.
 *   - The library allocates only its own tables (orbit spline coefficients, plan tables,
 *     batch tile tables, the device error word) and frees them in the *_destroy calls.
 *   - Compute calls are asynchronous on `stream` (a cudaStream_t passed as void*, NULL =
 *     legacy default stream) and return after enqueueing.  Argument and range checks happen
 *     on the host before any launch.  Device-side faults the kernels detect (a stencil index
 *     outside its staged window, a bounded wait that ran out) are recorded in the plan's
 *     error word and reported by lr_plan_check().
 *   - Handles are not thread-safe: use one plan per host thread / stream.
 *
 * Errors: every call returns an lr_status; no exception crosses the ABI.
 */
#ifndef LISARESP_H
#define LISARESP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LR_API __attribute__((visibility("default")))

typedef enum {
    LR_OK = 0,
    LR_ERR_INVALID_ARG = 1,   /* null pointer, bad enum, non-positive size, ... */
    LR_ERR_RANGE = 2,         /* sizes beyond what the plan or a table supports */
    LR_ERR_OOM = 3,           /* device or host allocation failed */
    LR_ERR_CUDA = 4,          /* a CUDA runtime call failed (see lr_last_cuda_error) */
    LR_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out */
    LR_ERR_NONFINITE = 6,     /* NaN or Inf found where finite values are required */
    LR_ERR_UNSUPPORTED = 7,   /* valid request the library does not implement (e.g. even order) */
    LR_ERR_DEVICE = 8         /* a kernel recorded an internal fault in the plan's error word */
} lr_status;

enum { LR_FP64 = 0, LR_MIXED = 1 };                       /* plan precision */
enum { LR_DELAY_SUM = 0, LR_DELAY_NESTED = 1 };           /* chained-delay model */
enum { LR_SPLINE_NOT_A_KNOT = 0, LR_SPLINE_NATURAL = 1 }; /* spline end conditions */

typedef struct lr_ctx lr_ctx;
typedef struct lr_orbit lr_orbit;
typedef struct lr_plan lr_plan;

/* Sky position (ecliptic longitude lambda, latitude beta) and polarisation angle psi, rad.
 * k = -e_r, u = -e_phi, v = -e_theta of the SSB spherical basis (Sec. "Reference frames"). */
typedef struct { double lam, beta, psi; } lr_sky;

/* Galactic-binary parameters (Sec. "Template generation"): amplitude A, initial frequency f0 (Hz)
 * and its derivatives fdot (Hz/s), fddot (Hz/s^2; the paper takes 11 fdot^2 / (3 f0)), initial
 * phase phi0 and inclination iota (rad), with t measured on the library's time axis.  The
 * polarisations are h+ = A (1 + cos^2 iota) cos Phi and hx = 2 A cos iota sin Phi,
 * Phi = 2 pi (f0 t + fdot t^2 / 2 + fddot t^3 / 6) + phi0: the un-rotated inputs of the response
 * (psi is the sky's; pass -A for the paper's SSB sign). */
typedef struct { double A, f0, fdot, fddot, phi0, iota; } lr_gb;

typedef struct {
    int order;            /* Lagrange degree p: odd, 1 <= p <= 63 (a compiled subset; see lr_order_supported) */
    int precision;        /* LR_FP64 or LR_MIXED */
    int tdi_generation;   /* 1 (X1: Eq. tdi1) or 2 (X2: Eq. tdi2) */
    int delay_mode;       /* LR_DELAY_SUM (the paper's summed delays) or LR_DELAY_NESTED */
    double dt;            /* sample spacing (s), > 0 */
    double t0;            /* time of output sample 0 (s) */
    int64_t n;            /* output length of the single-source calls (>= 1) */
    const lr_orbit *proj_orbit;  /* positions + delays used by the projection */
    const lr_orbit *tdi_orbit;   /* delays used by TDI; may differ (hybrid templates) */
    int tile;             /* output samples per CTA tile; 0 = default.  Mixed plans stage a tile in
                             fixed shared-memory arrays: at most 340 outputs at order 25 and dt =
                             10 s (less for longer TDI halos); a larger tile is LR_ERR_RANGE */
    int threads;          /* threads per CTA; 0 = default */
} lr_plan_desc;

/* ------------------------------------------------------------------ misc */
LR_API const char *lr_strerror(int status);
LR_API int lr_version(void);                        /* major*10000 + minor*100 + patch */
LR_API int lr_order_supported(int order);           /* 1 if a kernel for this degree is compiled */
/* Failure injection for tests: after `after` more successful device allocations, every further
 * library allocation fails with LR_ERR_OOM (after < 0 disables; process-wide, not thread-safe). */
LR_API int lr_debug_fail_allocations(int after);

/* ------------------------------------------------------------------ context */
/* Binds the library to CUDA device `device` (>= 0).  *out is owned by the caller and freed
 * by lr_ctx_destroy.  Also resolves the device addresses of the fixed arrays used by
 * lr_response_batched_noalloc on this device (the CUDA runtime loads them here, not during that
 * call). */
LR_API int lr_ctx_create(int device, lr_ctx **out);
LR_API int lr_ctx_destroy(lr_ctx *ctx);
/* cudaError_t of the last failing CUDA call made through this context (0 if none). */
LR_API int lr_last_cuda_error(const lr_ctx *ctx);

/* ------------------------------------------------------------------ orbits */
/* Spacecraft positions and link delays on a uniform knot grid, interpolated by cubic
 * splines (Sec. "Implementation"; the spline kind is not stated in the paper: not-a-knot
 * by default).
 *   t_knots : HOST [n_knots], strictly increasing and uniformly spaced (rel. 1e-9), n_knots >= 4
 *   pos     : HOST [3 spacecraft][3 xyz][n_knots] (m)
 *   delays  : HOST [6 links][n_knots] (s), or NULL: solve L_rs(t) = |x_r(t) - x_s(t - L_rs)|/c
 *             on each knot by fixed-point iteration on the position spline
 *   spline_bc : LR_SPLINE_NOT_A_KNOT or LR_SPLINE_NATURAL
 * The host arrays are copied; the device tables belong to the orbit. */
LR_API int lr_orbit_create(lr_ctx *ctx, const double *t_knots, int64_t n_knots, const double *pos,
                           const double *delays, int spline_bc, lr_orbit **out);
LR_API int lr_orbit_destroy(lr_orbit *orbit);
/* Copies the delays on the knots (given or solved) to HOST out[6][n_knots]. */
LR_API int lr_orbit_delays(const lr_orbit *orbit, double *out, int64_t n_knots);

/* ------------------------------------------------------------------ plans */
/* Validates the descriptor and precomputes the plan's device tables (TDI chain tables,
 * halo sizes).  The orbits must outlive the plan. */
LR_API int lr_plan_create(lr_ctx *ctx, const lr_plan_desc *desc, lr_plan **out);
LR_API int lr_plan_destroy(lr_plan *plan);
/* Input samples an output sample needs on each side of its own time: an input series that
 * covers [t0 - left*dt, t0 + (n-1)*dt + right*dt] gives every output a full stencil. */
LR_API int lr_required_margin(const lr_plan *plan, int64_t *left, int64_t *right);
/* Output samples per CTA tile the plan uses (the descriptor's tile, or the default chosen for it;
 * lr_plan_autotune may change it).  Errors: LR_ERR_INVALID_ARG for null pointers. */
LR_API int lr_plan_tile(const lr_plan *plan, int *tile);
/* Outputs of the plan's span [0, n) whose TDI reads all have full stencils inside that span
 * (Eqs. tdi1/tdi2 with the reads of Sec. "Implementation"): every chained delay of output k,
 * at most tdi_generation-dependent 3 or 7 link delays (the TDI orbit's bound), reads link
 * samples floor(k - D/dt) - (p-1)/2 .. floor(k - D/dt) + (p+1)/2, so
 *   *first = ceil(q * L_max / dt) + (p-1)/2 + 1,   *last = n - 2 - (p-1)/2.
 * Outside [*first, *last] the zero extension of the link series before sample 0 and after
 * sample n-1 enters the result; inside it the outputs equal those of a longer span, provided the
 * strain covers lr_required_margin.  *first > *last means no output has full stencils.
 * Errors: LR_ERR_INVALID_ARG for null pointers. */
LR_API int lr_valid_range(const lr_plan *plan, int64_t *first, int64_t *last);
/* Waits for `stream`, then reads and clears the plan's device error word: LR_OK, or
 * LR_ERR_DEVICE / LR_ERR_TIMEOUT if a kernel recorded a fault since the last check, or
 * LR_ERR_NONFINITE if the only thing recorded is a NaN or infinity in the strain a forward tile
 * staged or in the likelihood data it read (the outputs it touched are then non-finite too). */
LR_API int lr_plan_check(lr_plan *plan, void *stream);

/* ------------------------------------------------------------------ forward */
/* Projection only: y[6][plan.n] from h+, hx (each [n_h], input grid t0_h + j*dt).
 * Eq. instrument-response-to-gw with the projection orbit. */
LR_API int lr_project(lr_plan *plan, const double *hp, const double *hc, int64_t n_h, double t0_h,
                      lr_sky sky, double *y, void *stream);
/* TDI only: xyz[3][plan.n] from y[6][plan.n] (Eqs. tdi1/tdi2 with the TDI orbit's delays). */
LR_API int lr_tdi(lr_plan *plan, const double *y, double *xyz, void *stream);
/* Fused projection + TDI: xyz[3][plan.n]; the link series stay on chip. */
LR_API int lr_response(lr_plan *plan, const double *hp, const double *hc, int64_t n_h, double t0_h,
                       lr_sky sky, double *xyz, void *stream);

/* ------------------------------------------------------------------ backward */
/* Transpose of lr_response applied to g_xyz[3][plan.n] (e.g. dLoss/dXYZ):
 *   g_hp, g_hc [n_h]   = P^T T^T g_xyz            (overwritten)
 *   g_sky[3] (DEVICE)  = d<g_xyz, R(h)>/d(lambda, beta, psi)   (overwritten; may be NULL)
 * The link series and their gradient are recomputed, not stored.  Deterministic: gathers
 * over inverted tap windows and fixed-order reductions, no atomics on the data. */
LR_API int lr_backward(lr_plan *plan, const double *hp, const double *hc, int64_t n_h, double t0_h,
                       lr_sky sky, const double *g_xyz, double *g_hp, double *g_hc, double *g_sky,
                       void *stream);

/* ------------------------------------------------------------------ batched */
/* S independent sources with their own lengths in one persistent launch.
 *   h_off   : DEVICE int64[S+1], source s reads hp/hc[h_off[s] .. h_off[s+1])
 *   out_off : DEVICE int64[S+1], source s has n_s = out_off[s+1]-out_off[s] outputs, written
 *             to xyz[3*out_off[s] ..) as [3][n_s]; output sample n at t0 + n*dt
 *   t0_h    : DEVICE double[S], time of each source's input sample 0
 *   sky     : DEVICE lr_sky[S]
 * S <= 2^24.  The plan's n is ignored.  Offsets must be non-decreasing (checked on device:
 * a violation records LR_ERR_DEVICE). */
LR_API int lr_response_batched(lr_plan *plan, int64_t S, const int64_t *h_off, const int64_t *out_off,
                               const double *t0_h, const lr_sky *sky, const double *hp, const double *hc,
                               double *xyz, void *stream);
/* Batched forward on HOST buffers: the same arguments and results as lr_response_batched, but
 * h_off, out_off, t0_h, sky, hp, hc and xyz are host arrays (h_off[0] = out_off[0] = 0, both
 * non-decreasing).  The batch is cut into chunks of whole sources (about 2^25 outputs each) and
 * (LR_PIPELINE_CHUNK_OUTPUTS in the environment overrides the chunk size)
 * the copy-in of one chunk, the fused kernel on the previous one and the copy-out of the one
 * before run concurrently on three library streams, in two plan-owned device slots (allocated on
 * first use and grown when a larger chunk arrives; freed with the plan).  Work queued earlier on
 * `stream` is waited for; the call returns when every result is in xyz (synchronous).  hp, hc and
 * xyz should be page-locked (cudaHostAlloc / cudaHostRegister) for the copies to overlap; pageable
 * memory gives the same results with serialised copies.  The paper's method is unchanged: this
 * is the library's transfer schedule for data that lives in host memory.
 * Errors: LR_ERR_INVALID_ARG for null pointers, S < 1 or non-monotone offsets, LR_ERR_RANGE for
 * S > 2^24, LR_ERR_OOM / LR_ERR_CUDA as elsewhere; device-detected faults are read with
 * lr_plan_check. */
LR_API int lr_response_batched_host(lr_plan *plan, int64_t S, const int64_t *h_off, const int64_t *out_off,
                                    const double *t0_h, const lr_sky *sky, const double *hp, const double *hc,
                                    double *xyz, void *stream);
/* ------------------------------------------------------------------ graphs and tuning */
typedef struct lr_graph lr_graph;
/* Captures one lr_response_batched call (batch-table kernels + persistent fused kernel) into an
 * instantiated CUDA graph.  The graph owns its batch tables (tile prefix sums and sky frames,
 * allocated before the capture, freed by lr_graph_destroy), so later calls on the same plan, with
 * any batch size, do not disturb it.  The graph keeps the given device pointers: rewrite the
 * inputs in place between replays; the batch shape (S, offsets) must not change while the graph
 * is used.  The plan (its error word and orbit tables) and the orbits must outlive the graph.
 * Owned by the caller. */
LR_API int lr_response_batched_graph(lr_plan *plan, int64_t S, const int64_t *h_off, const int64_t *out_off,
                                     const double *t0_h, const lr_sky *sky, const double *hp, const double *hc,
                                     double *xyz, lr_graph **out);
LR_API int lr_graph_launch(lr_graph *graph, void *stream);  /* replay on `stream` */
LR_API int lr_graph_destroy(lr_graph *graph);
/* Times the fused forward on a synthetic single source of n_samples outputs for a few candidate
 * tile sizes and keeps the fastest in the plan (*tile_out).  With use_cache the choice is read
 * from / appended to a text cache (path from LR_AUTOTUNE_CACHE, default
 * $HOME/.cache/lisaresp_autotune.txt) keyed by GPU name, precision, order, TDI generation and
 * log2 length bucket.  Allocates and frees temporary device buffers; synchronizes `stream`. */
LR_API int lr_plan_autotune(lr_plan *plan, int64_t n_samples, int use_cache, void *stream, int *tile_out);

/* The tile autotuner for a ragged batch: times the candidate tiles on a synthetic batch with the
 * given batch's length distribution (up to 48 of its length quantiles, scaled to at most 2^24
 * outputs in total), each candidate as one batched call (batch tables + persistent fused kernel),
 * and keeps the fastest in the plan.  Cached like lr_plan_autotune, keyed by GPU, precision,
 * order, TDI generation, S and the log2 of the batch's 10/50/90 % length quantiles.
 *   lengths : HOST int64[S], output samples per source (>= 0)
 * Allocates and frees temporary device buffers; synchronizes `stream`.
 * Errors: LR_ERR_INVALID_ARG for null pointers or a negative length; LR_ERR_RANGE for S outside
 * [1, 2^24] or an all-empty batch. */
LR_API int lr_plan_autotune_batch(lr_plan *plan, int64_t S, const int64_t *lengths, int use_cache, void *stream,
                                  int *tile_out);
/* The Lagrange order for a signal band: the smallest compiled odd degree p whose centered read of
 * a unit complex sinusoid of f_dt cycles per sample (the band edge f_max * dt) is within tol at
 * every fractional offset (129 offsets in [0, 1]; host arithmetic, weights by direct products of
 * Sec. "Implementation"'s centered Lagrange polynomials).  The response's own error is this read
 * error amplified by the projection and TDI cancellations (|y|/|h| ~ 2 pi f L and more), so tol is
 * the read accuracy the caller needs, not the response's relative error.
 * Errors: LR_ERR_INVALID_ARG for f_dt outside [0, 0.5) or tol <= 0; LR_ERR_RANGE when no compiled
 * order reaches tol. */
LR_API int lr_choose_order(double f_dt, double tol, int *order);

/* Batched forward that allocates no device memory.  Same arguments, results and asynchrony as
 * lr_response_batched, which allocates its per-batch tables on first use; this variant keeps
 * them in fixed device arrays inside the library, for callers that may not allocate device
 * memory once their run has started (a sampler or service that has budgeted all device memory
 * up front, or that cannot take the device-wide synchronisation of cudaMalloc / cudaFree).
 * The paper has no counterpart: it is an allocation policy of this library.
 *   S <= LR_NOALLOC_MAX_SOURCES, else LR_ERR_RANGE (nothing is launched).
 *   The arrays (the tile table, 8 * (LR_NOALLOC_MAX_SOURCES + 1) bytes, and the sources' sky
 *   frames, 88 * LR_NOALLOC_MAX_SOURCES bytes) are held by every GPU that loads the library until
 *   the process exits, and are shared by every call on that GPU: each call rewrites the entries
 *   it uses before reading them, and calls that overlap on the GPU (other streams, other threads,
 *   other plans) race on them.  The arrays' device addresses are looked up (cudaGetSymbolAddress,
 *   with that device current) by lr_ctx_create, which is also when the CUDA runtime loads the
 *   module holding them, so this call itself allocates nothing. */
#define LR_NOALLOC_MAX_SOURCES 65536
LR_API int lr_response_batched_noalloc(lr_plan *plan, int64_t S, const int64_t *h_off, const int64_t *out_off,
                                       const double *t0_h, const lr_sky *sky, const double *hp, const double *hc,
                                       double *xyz, void *stream);

/* ------------------------------------------------------------------ generated strain */
/* The Galactic-binary waveform of Sec. "Template generation" generated on the device instead of
 * read from arrays: the fused kernels compute the strain window each tile reads directly from the
 * parameters (lr_gb), on the output grid t0 + i dt at every index i (no zero extension: the
 * waveform exists at all times), so no strain crosses HBM.  The phase is formed in double-double
 * and reduced modulo one cycle before the FP64 sincos (a few 1e-16 rad at any t and f0).
 *
 * h+, hx [n] at t0 + j dt into DEVICE arrays, the same generator as the fused kernels.  Errors:
 * LR_ERR_INVALID_ARG for null pointers or n < 0, LR_ERR_NONFINITE for a non-finite parameter. */
LR_API int lr_gb_polarisations(const lr_gb *gb /* HOST */, double t0, double dt, int64_t n, double *hp, double *hc,
                               void *stream);
/* Fused response of one Galactic binary over the plan's span: xyz DEVICE [3][plan.n].  Errors as
 * lr_response; LR_ERR_NONFINITE for a non-finite parameter. */
LR_API int lr_response_gb(lr_plan *plan, lr_gb gb, lr_sky sky, double *xyz, void *stream);
/* Batched: S sources with output offsets out_off (DEVICE int64[S+1]), parameters gb (DEVICE lr_gb[S])
 * and sky (DEVICE lr_sky[S]); xyz as lr_response_batched.  Non-finite parameters give non-finite
 * outputs for that source.  Errors as lr_response_batched. */
LR_API int lr_response_gb_batched(lr_plan *plan, int64_t S, const int64_t *out_off, const lr_gb *gb,
                                  const lr_sky *sky, double *xyz, void *stream);
/* Per-source log-likelihood <d|h> - <h|h>/2 of generated templates (the sampler's step: parameters
 * in, one number per walker out): logl DEVICE double[S]; data, n_total, weights, xyz as
 * lr_log_likelihood_batched. */
LR_API int lr_log_likelihood_gb_batched(lr_plan *plan, int64_t S, const int64_t *out_off, const lr_gb *gb,
                                        const lr_sky *sky, const double *data, int64_t n_total,
                                        const double *weights, double *logl, double *xyz, void *stream);

/* ------------------------------------------------------------------ likelihood */
/* Fused likelihood epilogue of the forward (the log-likelihood of Eq. like,
 * log L = -(<d|d> + <h|h> - 2 <d|h>)/2, with the inner product summed over the uncorrelated
 * channels A = (Z - X)/sqrt 2, E = (X - 2Y + Z)/sqrt 6, T = (X + Y + Z)/sqrt 3 of Sec.
 * "Time-delay interferometry").  The inner product is taken in the time domain with white noise
 * of variance 1/w_c in channel c: <a|b> = sum_c w_c sum_n a_c[n] b_c[n] (the paper weights it
 * by a noise PSD in the frequency domain; that needs the whole series and is not fused here).
 * Each tile of the fused forward forms A, E, T of its outputs on chip and its partial sums; a
 * second kernel adds the tiles of each source in a fixed order (deterministic, no atomics).
 *   data    : DEVICE [3][plan.n], the data in A, E, T (channel-major)
 *   weights : HOST double[3], w_A, w_E, w_T (finite, >= 0)
 *   dh_hh   : DEVICE double[2], written with <d|h>, <h|h> (<d|d> is the caller's constant)
 *   xyz     : DEVICE [3][plan.n] receiving X, Y, Z as lr_response, or NULL (not written)
 * Allocates the plan's per-tile partial buffer on first use (freed with the plan).
 * Errors as lr_response; LR_ERR_INVALID_ARG for a negative or non-finite weight. */
LR_API int lr_likelihood(lr_plan *plan, const double *hp, const double *hc, int64_t n_h, double t0_h,
                         lr_sky sky, const double *data, const double *weights, double *dh_hh, double *xyz,
                         void *stream);
/* Batched form: offsets, times and sky as lr_response_batched; data is DEVICE packed like xyz
 * (source s at data[3*out_off[s] ..] as [3][n_s]) and holds n_total = out_off[S] samples per
 * channel block; dh_hh is DEVICE [S][2].  Sources whose offsets run past n_total get NaN and
 * record LR_ERR_DEVICE (read with lr_plan_check); no read goes past the data.  S <= 2^24,
 * n_total <= 2^40. */
LR_API int lr_likelihood_batched(lr_plan *plan, int64_t S, const int64_t *h_off, const int64_t *out_off,
                                 const double *t0_h, const lr_sky *sky, const double *hp, const double *hc,
                                 const double *data, int64_t n_total, const double *weights, double *dh_hh,
                                 double *xyz, void *stream);

/* The log-likelihood of Eq. like up to the caller's constant -<d|d>/2, <d|h> - <h|h>/2, formed by
 * the library from the same fused epilogue and per-source reduction as lr_likelihood: the only
 * value that leaves the GPU per source (the paper's MCMC use, Sec. "Implementation").
 *   logl : DEVICE double[1]; other arguments and errors as lr_likelihood. */
LR_API int lr_log_likelihood(lr_plan *plan, const double *hp, const double *hc, int64_t n_h, double t0_h,
                             lr_sky sky, const double *data, const double *weights, double *logl, double *xyz,
                             void *stream);
/* Batched form: logl is DEVICE double[S]; other arguments and errors as lr_likelihood_batched. */
LR_API int lr_log_likelihood_batched(lr_plan *plan, int64_t S, const int64_t *h_off, const int64_t *out_off,
                                     const double *t0_h, const lr_sky *sky, const double *hp, const double *hc,
                                     const double *data, int64_t n_total, const double *weights, double *logl,
                                     double *xyz, void *stream);

/* Gradient of the time-domain log-likelihood (up to the constant -<d|d>/2),
 * <d|h> - <h|h>/2 over A, E, T with the weights of lr_likelihood, with respect to the template's
 * X, Y, Z: g_xyz = scale * M^T W (data - M xyz), M the A, E, T map, W = diag(weights).  Feed
 * g_xyz to lr_backward for the gradient with respect to h+, hx and the sky angles.
 *   xyz, data, g_xyz : DEVICE [3][plan.n] (X, Y, Z; A, E, T; X, Y, Z); g_xyz may alias neither.
 *   weights : HOST double[3] (finite, >= 0); scale: host factor (e.g. the upstream gradient).
 * Elementwise, FP64 in both plan precisions.  LR_ERR_INVALID_ARG for null pointers or bad
 * weights, LR_ERR_NONFINITE for a non-finite scale. */
LR_API int lr_likelihood_grad(lr_plan *plan, const double *xyz, const double *data, const double *weights,
                              double scale, double *g_xyz, void *stream);
/* Batched form: out_off DEVICE int64[S+1] as lr_response_batched (source s at 3*out_off[s] as
 * [3][n_s] in xyz, data and g_xyz, which hold n_total samples per channel block); S <= 2^24.
 * Sources whose offsets decrease or run past n_total are skipped and record LR_ERR_DEVICE. */
LR_API int lr_likelihood_grad_batched(lr_plan *plan, int64_t S, const int64_t *out_off, int64_t n_total,
                                      const double *xyz, const double *data, const double *weights, double scale,
                                      double *g_xyz, void *stream);

/* Batched transpose; g_sky is DEVICE [S][3] (may be NULL). */
LR_API int lr_backward_batched(lr_plan *plan, int64_t S, const int64_t *h_off, const int64_t *out_off,
                               const double *t0_h, const lr_sky *sky, const double *hp, const double *hc,
                               const double *g_xyz, double *g_hp, double *g_hc, double *g_sky, void *stream);

/* ------------------------------------------------------------------ multi-GPU partitioning */
/* Host-only helpers (no device, context or plan needed) for running the response on several GPUs,
 * one process per GPU, with no collective on the data path.
 *
 * Across sources: the sources of a batch are independent.  Length-balanced greedy deal: sources in
 * order of decreasing length (equal lengths by index) each go to the rank with the smallest total
 * length so far (ties to the lower rank).  Deterministic, so every rank computes the same deal.
 *   lengths : HOST int64[S] (>= 0, e.g. output samples per source)
 *   rank_of : HOST int[S], written with each source's rank
 *   load    : HOST int64[ranks], written with each rank's total length (may be NULL)
 * Errors: LR_ERR_INVALID_ARG for S < 0, ranks < 1, null arrays or a negative length. */
LR_API int lr_partition_sources(int64_t S, const int64_t *lengths, int ranks, int *rank_of, int64_t *load);

/* Across time for one long source: rank `rank` of `ranks` owns outputs [first, first + count) of the
 * span [0, n) (whole units of `align` outputs, dealt as evenly as possible in rank order, the extra units to
 * the last ranks: the owned counts differ by at most `align`) and
 * computes the span [lo, hi): the owned range widened by halo_left / halo_right outputs, rounded
 * out to multiples of `align` and clamped to [0, n).  Run it as a plan of hi - lo outputs starting at
 * t0 + lo*dt, with the unsplit run's strain shifted by lo samples (input sample 0 at t0_h + lo*dt;
 * the same fractional read offsets, so the same arithmetic) covering lr_required_margin around
 * that span, and keep outputs
 * first - lo .. first - lo + count - 1: they equal the unsplit run's outputs first .. first + count - 1
 * when halo_left = *first and halo_right = n - 1 - *last of lr_valid_range (every TDI read of an
 * owned output then lies inside [lo, hi) or outside [0, n) for both runs), and align is the plan's
 * tile (the span's tiles are then the unsplit run's tiles).  The only exchange is the replicated
 * strain halo at set-up.  For the adjoint, give each rank g_xyz on its owned outputs only (zero on
 * the rest of its span): the ranks' sky-angle gradients then add up to the unsplit one (a sum of
 * three numbers), and their strain gradients add up where their input windows overlap.
 * Errors: LR_ERR_INVALID_ARG for a null out, n < 0, negative halos, align < 1 or a rank outside
 * [0, ranks). */
typedef struct {
    int64_t first, count;  /* outputs this rank owns */
    int64_t lo, hi;        /* output span this rank computes */
} lr_time_shard;
LR_API int lr_partition_time(int64_t n, int64_t halo_left, int64_t halo_right, int64_t align, int ranks, int rank,
                             lr_time_shard *out);

#ifdef __cplusplus
}
#endif
#endif /* LISARESP_H */
