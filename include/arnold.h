/*
 * arnold.h -- C ABI of libarnold.so, the B300 (sm_103a) ensemble propagator
 * for the Arnold-web scan of Seibert, Denisov, Ponomarev & Haenggi,
 * "Mapping the Arnold web with a GPU-supercomputer" (arXiv:1107.4107).
 *
 * What it computes (the paper's Sec. II-IV):
 *   H(P, X) = |P|^2 / 2 + eps * cos x cos y (1 + cos 2z)          (Eqs. 1-2)
 * propagated for an ensemble of independent trajectories by a symmetric
 * composition of drift-kick-drift leapfrog substeps (a sixth-order
 * symplectic integrator, Sec. III), angles on the torus [0, 2pi)^3 with lap
 * counters, each trajectory carrying the tangent-map vector for the
 * finite-time Lyapunov indicator, the finite-time averaged velocity
 * V = [X(t + dt) - X(t)] / dt of Sec. IV, and the energy error of Sec. III.
 *
 * Conventions for every entry point:
 *   - Status: 0 on success, a negative ARNOLD_E* code otherwise; no call
 *     aborts, throws or traps.  arnold_strerror() names a code.
 *   - Ownership: the library owns each context and all device memory inside
 *     it (state, tangent, tables, checkpoints, reduction scratch).  The caller
 *     owns every buffer it passes in; the library never keeps a caller pointer
 *     past the call.
 *   - ptr_kind: ARNOLD_HOST for host memory (pageable or pinned), ARNOLD_DEVICE
 *     for device memory of the context's device.
 *   - Layout: per-trajectory arrays are structure-of-arrays, component-major:
 *     a "[3][n] f64" array holds all x, then all y, then all z (row-major C).
 *   - Streams: work is enqueued on the stream given at creation (NULL = the
 *     legacy default stream).  Calls that return data to the host synchronise
 *     that stream; others return before the GPU finishes.  An error raised by
 *     a kernel is reported by the next call that synchronises.
 *   - Threads: a context may be used from one host thread at a time.
 *   - Current device: calls on a context (or batch) leave that context's device
 *     current in the calling host thread; arnold_stats_arrays_noalloc restores
 *     the caller's.
 */
#ifndef ARNOLD_H
#define ARNOLD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define ARNOLD_OK            0
#define ARNOLD_EINVAL       -1  /* bad argument: NULL, n <= 0, h == 0, unknown enum, size mismatch */
#define ARNOLD_ENOMEM       -2  /* device or host allocation failed                                */
#define ARNOLD_ECUDA        -3  /* a CUDA runtime call or kernel failed                             */
#define ARNOLD_ETIMEOUT     -4  /* a bounded device-side wait ran out                               */
#define ARNOLD_ENONFINITE   -5  /* the state became NaN/Inf (checked when results are read)         */
#define ARNOLD_EUNSUPPORTED -6  /* combination not built (e.g. no CUDA device)                      */
#define ARNOLD_ESTATE       -7  /* call out of order (e.g. arnold_grad before arnold_forward_ckpt)  */
#define ARNOLD_ERANGE       -8  /* outside the precision mode's range (h |q| per step > 160 for DF64 and DF64F, > 400 for FP32C) */

/* ---- enums --------------------------------------------------------------- */
/* Integrators (Sec. III names a sixth-order symplectic scheme whose reference
 * is missing; Yoshida's solution A is the default reading). */
#define ARNOLD_SCHEME_YOSHIDA6A   0  /* Yoshida 1990, 6th order, solution A, 7 kicks/step */
#define ARNOLD_SCHEME_TRIPLEJUMP6 1  /* recursive triple jump, 6th order, 9 kicks/step   */
#define ARNOLD_SCHEME_LEAPFROG2   2  /* drift-kick-drift leapfrog, 2nd order, 1 kick/step */

#define ARNOLD_FP64  0  /* state, tangent and sincos to FP64 accuracy (the paper used double precision,
                           Sec. III); FP64 instructions only where that accuracy needs them             */
#define ARNOLD_FP32C 1  /* compensated FP32: float-pair angles (held in a [1024, 2048) rad window, whole
                           turns removed exactly) and momenta, two-sum updates; FP64 logs and energy.
                           Forces and tangent in FP32: a short-horizon mode (its chi field holds the
                           scan's agreement bar to ~1e4 steps, not to 1e6).                             */
#define ARNOLD_DF64  2  /* double-float: state, kicks and tangent in float pairs (~48-bit), FP64-grade
                           trajectories on the FP32 pipes.  No adjoint.                                 */
#define ARNOLD_DF64F 3  /* DF64 with a faster sincos: the same double-float state, products, sums and
                           tangent, but sines and cosines to ~3e-10 (FP32 reduced argument joined to the
                           table's float pairs).  The compensated-FP32 mode for long horizons: its 1e6-step
                           indicator field matches FP64's.  No adjoint.                                  */

#define ARNOLD_HOST   0
#define ARNOLD_DEVICE 1

/* Indicator kinds for arnold_indicator(). */
#define ARNOLD_IND_CHI      0  /* [n] f64: FTLE chi_t = ln(|w(t)|/|w(0)|) / t, t = steps * h          */
#define ARNOLD_IND_V        1  /* [3][n] f64: V of Sec. IV (last closed window, or whole run if window=0) */
#define ARNOLD_IND_DE       2  /* [n] f64: |H(now) - H(t=0)| (Sec. III energy error)                      */
#define ARNOLD_IND_DE_MAX   3  /* [n] f64: max |H - H(0)| sampled every renorm_every steps               */
#define ARNOLD_IND_CLASS    4  /* [n] u8: 1 = chaotic, chi_t > kappa * ln(max(t, e)) / t                  */
#define ARNOLD_IND_X        5  /* [3][n] f64: angles x, y, z reduced into [0, 2pi)                       */
#define ARNOLD_IND_P        6  /* [3][n] f64: momenta p_x, p_y, p_z                                      */
#define ARNOLD_IND_DX       7  /* [3][n] f64: unwrapped X(now) - X(window start) (window 0: since start)  */
#define ARNOLD_IND_TANGENT  8  /* [6][n] f64: (dx, dy, dz, dp_x, dp_y, dp_z), as renormalised             */
#define ARNOLD_IND_LOGSUM   9  /* [n] f64: sum of ln|w| taken at renormalisations                        */
#define ARNOLD_IND_LEFT    10  /* [n] u8: 1 if the momentum direction left the tracked patch (area filter) */
/* MEGNO (mean exponential growth factor of nearby orbits; Cincotta & Simo,
 * Astron. Astrophys. Suppl. 147 (2000) 205) -- not in the paper, a second
 * tangent-based indicator beside chi.  Sampled at the m = steps / R
 * renormalisations so far, l_j the log growth of |w| over interval j:
 * Y_m = (2/m) sum_j j l_j and <Y>_m = (1/m) sum_{k<=m} Y_k.  <Y> tends to 0 on
 * stable periodic orbits, to 2 on quasi-periodic ones and grows like
 * lambda t / 2 on chaotic ones.  Both read 0 before the first renormalisation.
 * Needs a context created with megno = 1 (EINVAL otherwise). */
#define ARNOLD_IND_MEGNO   11  /* [n] f64: mean MEGNO <Y>_m                                              */
#define ARNOLD_IND_MEGNO_Y 12  /* [n] f64: MEGNO Y_m at the last renormalisation                         */
/* The paper's own reading of V (Sec. IV): a regular trajectory's averaged
 * velocity stays close to its initial momentum vector, a chaotic one's wanders
 * off; |V - P(0)| puts a number on it beside chi. */
#define ARNOLD_IND_VDEV    13  /* [n] f64: |V - P(t=0)|, V as ARNOLD_IND_V                                */

/* ---- parameters ------------------------------------------------------------ */
typedef struct arnold_params {
  double  eps;           /* eps of Eq. 1 (the paper uses 1, Eq. 3)                          */
  double  h;             /* composite step, != 0 (paper: 0.01 * 2 pi, Sec. III)             */
  int32_t scheme;        /* ARNOLD_SCHEME_*                                                 */
  int32_t precision;     /* ARNOLD_FP64, ARNOLD_FP32C, ARNOLD_DF64 or ARNOLD_DF64F          */
  int32_t tangent;       /* 1: carry the tangent vector and FTLE; 0: state only            */
  int32_t renorm_every;  /* R >= 1: tangent renormalisation / energy sampling interval      */
  int64_t window;        /* W >= 0: steps per averaging window of V; 0 = whole run          */
  double  chaos_kappa;   /* kappa > 0 of the regular/chaotic threshold (default 10)         */
  int32_t block_size;    /* threads per block, multiple of 32 in [32, 256]; 0 = default    */
  int32_t launch_steps;  /* max composite steps per kernel launch; 0 = automatic (~0.2 s)   */
  int32_t megno;         /* 1: also accumulate MEGNO (needs tangent = 1); 0: off            */
  int32_t reserved;      /* must be 0                                                       */
} arnold_params;

/* Fill defaults: eps 1, h 0.02 pi, Yoshida-6A, FP64, tangent on, R 100,
 * window 0, kappa 10, automatic launch shape.  Never fails. */
void arnold_params_default(arnold_params* prm);

typedef struct arnold_ctx arnold_ctx;

/* Create a context for n_traj trajectories on `device`, enqueuing on
 * `cuda_stream` (a cudaStream_t, or NULL).  Allocates all device state.
 * Errors: EINVAL (bad params, n_traj <= 0, out == NULL), ENOMEM, ECUDA,
 * EUNSUPPORTED (no device).  On error *out is NULL. */
int arnold_create(const arnold_params* prm, int64_t n_traj, int device, void* cuda_stream,
                  arnold_ctx** out);

/* Release the context and its device memory (synchronises its stream).
 * NULL is a no-op. */
void arnold_destroy(arnold_ctx* ctx);

/* Set the phase-space state of all trajectories and reset the clock,
 * indicators and energy reference H(t=0).  x, p: [3][n] f64 (angles may be
 * any real; they are reduced into [0, 2pi)); w: [6][n] f64 initial tangent
 * (dx, dy, dz, dp_x, dp_y, dp_z) normalised by the library, or NULL for
 * (1, ..., 1) / sqrt 6.  Errors: EINVAL, ECUDA. */
int arnold_set_state(arnold_ctx* ctx, const double* x, const double* p, const double* w,
                     int ptr_kind);

/* Initial conditions on a 2-D slice of initial actions, generated on the
 * device (the scans of Sec. IV, Figs. 2-3, on a grid): trajectory t = j*G + i
 * (global index, row j = row0 + t / G) gets p_x = (2 (i + 1/2)/G - 1) a,
 * p_y = (2 (j + 1/2)/G - 1) a, a = 0.9 sqrt(E - 2|eps|), angles uniform on
 * [0, 2pi) from SplitMix64(seed) counters 3 t_g .. 3 t_g + 2, and
 * p_z = +sqrt(2 (E - eps Hp(X)) - p_x^2 - p_y^2) from the fixed-energy
 * condition (Sec. IV, Fig. 4 caption).  The context must hold
 * n = rows * G trajectories for some rows >= 1 with row0 + rows <= G.
 * If raw_out (device, [6][n] f64) is not NULL it receives the generated
 * x, y, z, p_x, p_y, p_z.  Resets the clock like arnold_set_state.
 * Errors: EINVAL (E <= 2|eps|, size mismatch), ECUDA. */
int arnold_init_grid(arnold_ctx* ctx, int64_t G, int64_t row0, double E, uint64_t seed,
                     double* raw_out);

/* Initial conditions on the energy shell (the ensembles of Sec. IV, uniform
 * over the sphere S or a patch of it, and the Gaussian cloud of Fig. 4): x is
 * [3][n] angles; with mode ARNOLD_SHELL_DIRECTION p holds unit directions and
 * P = sqrt(2 (E - eps Hp(X))) p; with ARNOLD_SHELL_PZ p holds (p_x, p_y, -)
 * and p_z = +sqrt(2 (E - eps Hp) - p_x^2 - p_y^2).  Otherwise as
 * arnold_set_state (tangent (1,...,1)/sqrt 6).  A negative radicand gives NaN
 * momenta, reported as ENONFINITE by the next sync.  Errors: EINVAL, ECUDA. */
#define ARNOLD_SHELL_DIRECTION 1
#define ARNOLD_SHELL_PZ        2
int arnold_set_state_shell(arnold_ctx* ctx, const double* x, const double* p, int mode, double E,
                           int ptr_kind);

/* Initial conditions drawn on the device from SplitMix64(seed): candidate
 * t = offset + k draws counters 5t .. 5t+4 (three angles uniform on the torus,
 * then two uniforms u, w in [0, 1) for the momentum), the same stream as the
 * host generator, so an ensemble can be built in pieces (offset) or sharded.
 *
 * arnold_init_sphere (Sec. IV, Figs. 2-3: ensembles uniform over the sphere S
 * or a patch of it): trajectory k is candidate offset + k, with direction
 * cos theta = cos_lo + (cos_hi - cos_lo) u, phi = phi_lo + (phi_hi - phi_lo) w
 * and |P| = sqrt(2 (E - eps Hp(X))).  Resets the clock like arnold_set_state.
 * Errors: EINVAL (offset < 0, E <= 2|eps|, a patch outside [-1, 1] or reversed),
 * ECUDA. */
int arnold_init_sphere(arnold_ctx* ctx, double E, uint64_t seed, int64_t offset, double cos_lo, double cos_hi,
                       double phi_lo, double phi_hi);

/* arnold_init_gaussian (Sec. IV, Fig. 4: the cloud injected at W): candidate t
 * has (p_x, p_y) = (px0, py0) + sigma r (cos 2 pi w, sin 2 pi w) with
 * r = sqrt(-2 ln(1 - u)) (Box-Muller) and p_z = +sqrt(2 (E - eps Hp) - p_x^2 -
 * p_y^2); candidates whose radicand is negative have no real p_z and are
 * skipped.  The n trajectories are the first n candidates from `offset` that
 * have one, in candidate order; *n_drawn (if not NULL) receives the number of
 * candidates examined up to the last one kept.  Synchronises the stream.
 * Uses ~0.8 MB of library-owned device scratch (allocated on first use).
 * Errors: EINVAL (offset < 0, sigma < 0, non-finite input), ERANGE (fewer than
 * n real p_z among the first 64 n + 2^24 candidates; the trajectories are then
 * only partly set and must be initialised again), ENOMEM, ECUDA. */
int arnold_init_gaussian(arnold_ctx* ctx, double E, double px0, double py0, double sigma, uint64_t seed,
                         int64_t offset, int64_t* n_drawn);

/* Area tracking (Sec. IV, Fig. 3 zooms: trajectories that leave the scanned
 * area are dropped): from now on, every renorm_every steps, a trajectory whose
 * momentum direction (cos theta = p_z/|P|, phi = atan2(p_y, p_x) in [0, 2pi))
 * is outside [cos_lo, cos_hi] x [phi_lo, phi_hi] is flagged (ARNOLD_IND_LEFT).
 * Flags reset at set_state, init_grid, init_sphere, init_gaussian and this
 * call.  Errors: EINVAL, ENOMEM. */
int arnold_track_patch(arnold_ctx* ctx, double cos_lo, double cos_hi, double phi_lo, double phi_hi);

/* Snapshots of V (Sec. IV: one F per window Delta t): while enabled, the kernel
 * that closes averaging window w (w = 1, 2, ... counted from the last clock
 * reset; window = W steps, W > 0 in the params) also writes that window's V
 * into slot w - 1 of v_snap, a caller-owned DEVICE array [k_max][3][n] f64
 * (x, y, z components, SoA), for w <= k_max; later windows are not stored.
 * One long arnold_iterate thus records every window without host round
 * trips.  v_snap must stay valid until the iterations that write it have
 * completed on the stream; NULL disables.  The library keeps only the pointer
 * (not part of checkpoints).  Errors: EINVAL (window = 0, k_max < 1, pointer
 * not 8-byte aligned). */
int arnold_set_snapshots(arnold_ctx* ctx, double* v_snap, int64_t k_max);

/* Density of V on the momentum sphere (F of Sec. IV, Figs. 2-4): counts of the
 * direction of V (ARNOLD_IND_V) in n_cos x n_phi equal-width cells of
 * cos theta in [cos_lo, cos_hi] and phi in [phi_lo, phi_hi]; directions
 * outside are not counted, nor (filtered != 0) flagged trajectories.  counts:
 * [n_cos][n_phi] u64; accumulate != 0 adds to its contents (time-averaged F
 * over several windows), else it is overwritten.  Host counts synchronise.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int arnold_velocity_histogram(arnold_ctx* ctx, int n_cos, int n_phi, double cos_lo, double cos_hi,
                              double phi_lo, double phi_hi, int filtered, uint64_t* counts, int ptr_kind,
                              int accumulate);

/* Advance every trajectory n_steps >= 0 composite steps (asynchronous).
 * Work is split into launches of at most launch_steps steps; the result does
 * not depend on the split.  Errors: EINVAL, ECUDA. */
int arnold_iterate(arnold_ctx* ctx, int64_t n_steps);

/* Composite steps taken since the last set_state / init_grid. */
int64_t arnold_steps_done(const arnold_ctx* ctx);

/* Write one indicator (ARNOLD_IND_*) of all trajectories into `out`
 * (layout per kind above).  Host outputs synchronise the stream.
 * Errors: EINVAL (unknown kind, NULL out, CHI/CLASS/LOGSUM/TANGENT with
 * tangent off), ECUDA. */
int arnold_indicator(arnold_ctx* ctx, int kind, void* out, int ptr_kind);

/* Ensemble statistics (an ensemble statistic of the indicators, like the
 * density F of Sec. IV).  Histogram of log10 chi over [-8, 1) in 200 bins
 * (chi <= 0 or below -8: `under`; at or above 1: `over`), chaotic count,
 * maximum sampled energy error, mean and population variance of each
 * momentum component.  Reductions run on the device in a fixed order. */
#define ARNOLD_HIST_BINS 200
typedef struct arnold_stats {
  uint64_t hist[ARNOLD_HIST_BINS];
  uint64_t under, over, chaotic, n;
  double   dE_max;       /* max over trajectories of the energy-error input          */
  double   p_mean[3];
  double   p_var[3];
  double   t;            /* steps * h (or the t passed in)                            */
} arnold_stats;

/* Statistics of the context's own trajectories (chi, sampled dE_max, P).
 * Fills *out (host struct); synchronises.  Errors: EINVAL (tangent off),
 * ECUDA. */
int arnold_stats_compute(arnold_ctx* ctx, arnold_stats* out);

/* Same statistics over caller arrays (device pointers, f64): chi[n], dE[n]
 * (or NULL), p[3][n], for time t and threshold factor kappa.  Uses the
 * context's device, stream and reduction scratch.  Errors: EINVAL, ECUDA. */
int arnold_stats_arrays(arnold_ctx* ctx, int64_t n, const double* chi, const double* dE,
                        const double* p, double t, double kappa, arnold_stats* out);

/* Same statistics with no device allocation at all, and no context.  The
 * paper has no counterpart: this exists for callers that must not call
 * cudaMalloc -- for instance code running after another framework's caching
 * allocator has reserved nearly all device memory, code that must avoid the
 * device-wide synchronisation that cudaMalloc/cudaFree can cause, or a service
 * whose memory budget is fixed at start-up.  The reduction's block partials
 * live in a fixed ~1.7 MB array inside the library image (held by every GPU
 * that loads the library until the process exits).
 *   device, cuda_stream: where to run (stream NULL = legacy default stream).
 *   n, chi, dE, p, t, kappa, out: as arnold_stats_arrays (device f64 inputs,
 *   dE may be NULL, host output struct); synchronises the stream.
 * The first call on a device looks up the array's device address (set-up);
 * make that first call before any stream capture.  The caller's current
 * device is the same after the call as before it.  All calls share the array:
 * calls whose kernels overlap on the GPU race and must be serialised by the
 * caller.  Errors: EINVAL (NULL, n <= 0 or n > ARNOLD_NOALLOC_MAX_N, kappa <= 0,
 * t == 0, bad device), EUNSUPPORTED, ECUDA. */
#define ARNOLD_NOALLOC_MAX_N (1LL << 40)
int arnold_stats_arrays_noalloc(int device, void* cuda_stream, int64_t n, const double* chi,
                                const double* dE, const double* p, double t, double kappa,
                                arnold_stats* out);

/* ---- differentiation ------------------------------------------------------
 * Reverse-mode derivatives of the n_steps map of Sec. III (composite step,
 * angles wrapped: wrapping adds constants and does not change derivatives)
 * with respect to the initial state and to (h, eps).
 *
 * arnold_forward_ckpt: advance the ensemble n_steps >= 1 steps like
 * arnold_iterate, storing the state every ckpt_every steps (0: ceil(sqrt(n)))
 * in library-owned device memory (ceil(n_steps/C) + C states per trajectory).
 * Any later set_state / init_grid / iterate discards the checkpoints.
 * FP64 and FP32C contexts only (FP32C with the FP32 window reduction).
 * Errors: EINVAL, ENOMEM, ECUDA, EUNSUPPORTED (DF64, DF64F, the FP32C
 * FP64-reduction variant). */
int arnold_forward_ckpt(arnold_ctx* ctx, int64_t n_steps, int64_t ckpt_every);

/* arnold_grad: given dL/dX_N and dL/dP_N ([3][n] f64 each, in the paper's
 * coordinates; either may be NULL for zero) at the state reached by the last
 * arnold_forward_ckpt, write dL/dX_0 and dL/dP_0 ([3][n] f64) and
 * g_params[0] = dL/dh, g_params[1] = dL/deps (summed over trajectories).
 * The state and checkpoints are left unchanged, so grad may be called again
 * with another upstream gradient.  FP64 contexts differentiate in FP64;
 * FP32C contexts recompute in compensated FP32 and differentiate in FP32
 * (parameter sums in float pairs, then FP64).  ptr_kind applies to all five
 * arrays.  Errors: EINVAL, ESTATE (no valid forward_ckpt), ECUDA. */
int arnold_grad(arnold_ctx* ctx, const double* dL_dx, const double* dL_dp, double* g_x0, double* g_p0,
                double* g_params, int ptr_kind);

/* ---- batched persistent launch ----------------------------------------------
 * Many parameter sets (the scans of Sec. IV repeated over a grid of (K, eps)),
 * each a grid slice of initial actions with its own ensemble size and step
 * count, advanced together by one CUDA-graph launch of persistent kernels in
 * compensated FP32 (ARNOLD_FP32C) or double-float (ARNOLD_DF64F, ARNOLD_DF64).
 * Each set's trajectories are bit-identical to those of a single context of
 * the same precision with the same parameters. */
typedef struct arnold_batch_set {
  double   eps;       /* eps of Eq. 1                                         */
  double   h;         /* composite step (K = eps h^2)                         */
  double   E;         /* energy of the grid-slice ICs (E > 2|eps|)            */
  int64_t  G;         /* grid width: the set holds G * G trajectories         */
  int64_t  n_steps;   /* steps this set advances per arnold_batch_run         */
  uint64_t seed;      /* SplitMix64 seed of the initial angles                */
} arnold_batch_set;

typedef struct arnold_batch_tuning {
  int32_t block_size;       /* threads per block: multiple of 32 in [32, 256]        */
  int32_t traj_per_thread;  /* 1 or 2 trajectories advanced interleaved per thread
                               (FP32C); 1 for DF64 and DF64F                         */
  int32_t renorm_every;     /* R >= 1 for every set                                  */
  int32_t epoch_ms;         /* target GPU time of one persistent launch (ms)         */
} arnold_batch_tuning;

typedef struct arnold_batch arnold_batch;

/* Defaults: block 256, 1 trajectory per thread, R 100, 200 ms epochs. */
void arnold_batch_tuning_default(arnold_batch_tuning* t);

/* Create a batch of n_sets sets (allocates every set's device state and plans
 * the epochs).  precision: ARNOLD_FP32C, ARNOLD_DF64F or ARNOLD_DF64.  tuning
 * NULL = defaults.  Errors: EINVAL (bad set, precision ARNOLD_FP64,
 * traj_per_thread != 1 with a double-float precision), ENOMEM, ECUDA,
 * EUNSUPPORTED. */
int arnold_batch_create(const arnold_batch_set* sets, int n_sets, int scheme, int precision, int tangent,
                        const arnold_batch_tuning* tuning, int device, void* cuda_stream,
                        arnold_batch** out);

/* Grid-slice initial conditions for every set (as arnold_init_grid, row0 0). */
int arnold_batch_init(arnold_batch* b);

/* Advance every set by its n_steps: one graph launch (captured on first use;
 * asynchronous on the batch's stream).  Repeated runs continue the sets. */
int arnold_batch_run(arnold_batch* b);

/* Indicator / statistics of one set (as arnold_indicator / arnold_stats_compute). */
int arnold_batch_indicator(arnold_batch* b, int set, int kind, void* out, int ptr_kind);
int arnold_batch_stats(arnold_batch* b, int set, arnold_stats* out);

/* Plan size: epochs (persistent launches per run), work items per run, and
 * map steps per run (sum over sets of G^2 n_steps). */
int arnold_batch_info(const arnold_batch* b, int64_t* epochs, int64_t* items, int64_t* map_steps_per_run);

int arnold_batch_sync(arnold_batch* b);
int64_t arnold_batch_launch_count(const arnold_batch* b);
void arnold_batch_destroy(arnold_batch* b);

/* ---- checkpoint / resume ----------------------------------------------------
 * The complete per-trajectory state (phase-space state, tangent, laps, window
 * references, log sums, energy references and maxima, V, initial momenta, MEGNO
 * sums when enabled, area-tracking flags when tracking is on) plus the step counter, so
 * that a run resumed from a checkpoint continues bit for bit as if
 * uninterrupted (the paper's 24 h runs, Sec. IV, motivate it).  Layout: a
 * 128-byte header (magic "ARNOLDC2", precision, tangent, n, steps, scheme,
 * megno, eps, h, tracking on/off and the tracked patch) followed by the device
 * arrays.  The buffer is host memory owned by the caller. */
int arnold_checkpoint_size(const arnold_ctx* ctx, size_t* bytes);
/* Synchronises.  Errors: EINVAL (NULL, bytes too small), ECUDA. */
int arnold_checkpoint_save(arnold_ctx* ctx, void* host_buf, size_t bytes);
/* The context must have the same n, precision, tangent, scheme, megno, eps and h,
 * and the same area tracking: off in both, or on in both with the same patch
 * (call arnold_track_patch on a fresh context before loading a tracked
 * checkpoint; the flags are then restored).
 * Errors: EINVAL (mismatch, bad magic, size), ECUDA. */
int arnold_checkpoint_load(arnold_ctx* ctx, const void* host_buf, size_t bytes);

/* Synchronise the context's stream; returns the first pending error. */
int arnold_sync(arnold_ctx* ctx);

/* Number of kernels this context has launched (for accounting). */
int64_t arnold_launch_count(const arnold_ctx* ctx);

/* Human-readable name of a status code (static string, never NULL). */
const char* arnold_strerror(int status);

/* ---- diagnostics --------------------------------------------------------- */
/* Device sincos used by the kernels, for accuracy tests: s[k], c[k] for
 * x[k] in [0, 2pi] (device f64 arrays of length n).  precision selects the
 * FP64 table method or the FP32 variant (results widened to f64). */
int arnold_debug_sincos(arnold_ctx* ctx, int precision, int64_t n, const double* x, double* s,
                        double* c);

/* Pipe-throughput probe on `device`: kind 0 = DFMA, 1 = FFMA, 2 = MUFU sin, at
 * full occupancy with 8 independent chains per thread; *ops_per_s receives
 * lane-operations per second (best of 6 launches of ~100 ms after ~300 ms of
 * warm-up, so the clocks have risen; ~1 s in all).  Sample the SM clock while
 * it runs to turn the rate into operations per SM per clock.
 * Errors: EINVAL, ECUDA, EUNSUPPORTED. */
int arnold_probe_peak(int device, int kind, double* ops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* ARNOLD_H */
