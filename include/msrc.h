/*
 * msrc.h - C ABI of the GB300 moving-source image-source synthesis library.
 *
 * Method: arXiv 2508.03065, "Fast Algorithm for Moving Sound Source".
 *   - Every image source of a shoebox room (Sec. II-A, Eq. 1; lattice set
 *     |n_x|+|n_y|+|n_z| <= max_order times 8 parities) follows the mirrored
 *     source trajectory.
 *   - Its distance d_i(t) to the microphone gives the delay tau_i = d_i / c and
 *     the gain A_i = beta_i / (4 pi d_i) (Sec. II-A, text after Eq. 2).
 *   - d_i is evaluated exactly at knots whose spacing depends on the image's
 *     reflection count (dense for low orders, sparse for high orders) and is
 *     linearly interpolated to audio rate (Sec. II-C, "Fast Architecture"),
 *     or first upsampled band-limited (tier_upsample).
 *   - Each image is a discrete time-varying fractional delay realised with a
 *     Farrow structure (Sec. II-B, Eq. 3-5) approximating an L-tap windowed
 *     sinc (Hann or Kaiser) or following a least-squares design; the outputs
 *     of all images are summed (Eq. 8).
 *   - Options: microphones on a moving array (msrc_set_array_trajectory),
 *     emission-time (retarded) distances (delay_model), knot rates chosen
 *     from the motion (msrc_suggest_knot_rates, msrc_suggest_bandlimited_rates).
 *     Reverse mode
 *     (msrc_synthesize_backward) gives gradients for the signal, trajectory
 *     parameters and wall coefficients.
 *
 * Conventions for every entry point:
 *   - Every call returns an msrc_status; nothing aborts and no C++ exception
 *     crosses this boundary. msrc_last_error() gives a thread-local message
 *     describing the last failure of the calling thread.
 *   - Device work is asynchronous on the given stream (a cudaStream_t passed
 *     as void*, NULL = legacy default stream). Device-side errors (a bounded
 *     wait that timed out, a window clamp, a scratch overflow) are recorded in
 *     the workspace and reported by msrc_workspace_errors().
 *   - Device buffers (signals, outputs, workspace) are owned by the caller; the
 *     library never allocates device memory and never frees caller memory.
 *     Rooms are host objects owned by the library between create and destroy.
 *   - Device pointers must be 16-byte aligned; host arrays are read during the
 *     call only.
 *   - Units: metres, seconds, Hz. Wall order everywhere: x=0, x=Lx, y=0, y=Ly,
 *     z=0, z=Lz.
 */
#ifndef MSRC_H
#define MSRC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MSRC_OK = 0,
  MSRC_ERR_INVALID_ARG = 1,  /* null pointer, out-of-range value, geometry not valid */
  MSRC_ERR_UNSUPPORTED = 2,  /* valid request outside what the library supports */
  MSRC_ERR_WORKSPACE = 3,    /* workspace too small or misaligned */
  MSRC_ERR_CUDA = 4,         /* a CUDA runtime call failed (message in msrc_last_error) */
  MSRC_ERR_TIMEOUT = 5,      /* a bounded device wait gave up */
  MSRC_ERR_STATE = 6         /* call made on an object in the wrong state */
} msrc_status;

typedef struct msrc_room* msrc_room_t;

#define MSRC_MAX_TIERS 4
#define MSRC_MAX_MICS 16
#define MSRC_MAX_ORDER 60
#define MSRC_MAX_CTRL 16

/* Room and synthesis parameters (Sec. II-A, II-B, II-C). */
typedef struct {
  double dims[3];            /* room size Lx, Ly, Lz (m), each > 0 */
  double beta[6];            /* pressure reflection coefficient per wall, in [0, 1] */
  double c;                  /* speed of sound (m/s), > 0 */
  double fs;                 /* audio sample rate (Hz), > 0 */
  int32_t max_order;         /* image set |n_x|+|n_y|+|n_z| <= max_order, 0..MSRC_MAX_ORDER */
  int32_t n_tiers;           /* 1..MSRC_MAX_TIERS sampling tiers */
  int32_t tier_max_rho[4];   /* an image with reflection count rho = sum_d |2 n_d - p_d| goes to
                                the first tier t with rho <= tier_max_rho[t], else to the last */
  double tier_rate_hz[4];    /* knot rate of each tier; fs / rate must be an integer >= 1 */
  int32_t taps;              /* fractional-delay length L: even, 8..64 */
  int32_t window;            /* tap weights h(k; alpha), k = -L/2 .. L/2-1:
                                0 = Hann-windowed sinc, 1 = Kaiser-windowed sinc,
                                2 = least-squares Farrow design (Sec. II-B, Eq. 3-4):
                                    h(k; alpha) = sum_{q<=M} c_q(k) alpha^q minimising the
                                    integral over alpha in [0,1] and w in [0,pi] of
                                    V(w) |sum_k h(k; alpha) e^{-jwk} - e^{jw alpha}|^2,
                                    V = 1 up to passband*pi and 1e-3 above */
  double kaiser_beta;        /* Kaiser shape (used when window == 1), 0..20 */
  int32_t farrow_order;      /* window 2: polynomial order M, 1..4 */
  double passband;           /* window 2: passband edge as a fraction of pi, 0.05..0.98 */
  int32_t tier_upsample[4];  /* knot upsampler of each tier (Sec. II-C "recovered using an
                                upsampling algorithm"): 0 or 1 = linear interpolation of the
                                distance between knots; U > 1 (dividing fs / rate, at most 512) =
                                the distance at U virtual knots per interval from a band-limited
                                interpolation of the knots (sinc times a Kaiser window of shape 8
                                over 2 upsample_halfwidth knots, weights normalised to sum 1),
                                then linear between virtual knots. Knots before t = 0 and after
                                the end follow the trajectory's extension (line and circle
                                continue, the spline clamps). Reverse mode differentiates
                                through the interpolation (the weights' exact derivatives). */
  int32_t upsample_halfwidth;/* Q, half-width of that kernel in knots: 0 (= 4) or 1..8 */
  int32_t delay_model;       /* 0: an image's distance at a knot is taken at the reception time,
                                d = |r_i(t) - m(t)| (Sec. II-A, Eq. 2 evaluated at the output time);
                                1: emission-time (retarded) path length d = c tau with
                                c tau = |r_i(t - tau) - m(t)|, the sound reaching the microphone
                                at t having left the moving image at t - tau. Delay and gain
                                follow from d in both models. Model 1 needs linear knot
                                interpolation (tier_upsample <= 1) and the path valid
                                over [-(largest delay), end] (line and circle continue before
                                t = 0, the spline clamps); its reverse mode differentiates
                                through the emission time (implicit derivative of the equation). */
} msrc_room_desc;

/* Source trajectory s(t) (Sec. II-C: a band-limited trajectory p(n)). */
typedef struct {
  int32_t kind;              /* 0 line, 1 circle, 2 clamped uniform cubic B-spline */
  int32_t n_ctrl;            /* spline: number of control points, 4..MSRC_MAX_CTRL */
  double params[48];         /* line:   p0[3], direction[3] (any length > 0), speed v
                                circle: centre[3], radius R, speed v, start angle theta0
                                        (s = centre + R (cos, sin, 0)(theta0 + v t / R))
                                spline: control points P_0..P_{n_ctrl-1}, 3 doubles each */
  double duration_s;         /* trajectory duration T (> 0); the spline parameter is
                                u = clamp(t / T, 0, 1) */
} msrc_traj_desc;

/* Creates a room; validates the description and fits the Farrow coefficients
 * of the windowed-sinc fractional delay (Sec. II-B, Eq. 3-4) on the host.
 * *out receives a library-owned handle. No device call is made. */
msrc_status msrc_create_room(const msrc_room_desc* desc, msrc_room_t* out);

/* Destroys a room handle (NULL is accepted). Device work that used it must have
 * completed or been enqueued (the library keeps no device state per room). */
msrc_status msrc_destroy_room(msrc_room_t room);

/* Sets the source trajectory and the static microphone positions
 * (mics_xyz: n_mics x 3 doubles, host memory, 1 <= n_mics <= MSRC_MAX_MICS).
 * Validation: microphones strictly inside the room; the trajectory sampled
 * every millisecond over [0, T] stays strictly inside the room, at least 0.1 m
 * from every microphone, with speed below c. */
msrc_status msrc_set_trajectory(msrc_room_t room, const msrc_traj_desc* traj,
                                const double* mics_xyz, int32_t n_mics);

/* Moves the microphones rigidly with an array trajectory a(t) (same kinds and
 * parameters as the source's msrc_traj_desc): microphone m sits at
 * mics_xyz[m] + a(t) - a(0), mics_xyz as given to msrc_set_trajectory (their
 * positions at t = 0). Image distances use the microphone position at each knot
 * time (Sec. II-A distance |r_i(t) - mic|, with a moving receiver). traj = NULL
 * makes the array static again. Validation (1 ms grid, up to the source
 * duration): every microphone strictly inside the room and at least 0.1 m from
 * the source, source speed plus array speed below c (below c/2 for
 * msrc_synthesize_backward). On failure the room keeps its previous state.
 * Reverse mode differentiates with respect to the source trajectory only. */
msrc_status msrc_set_array_trajectory(msrc_room_t room, const msrc_traj_desc* traj);

/* Source positions s(t_k) of the room's trajectory at n_times times (seconds,
 * host array) into out (n_times x 3 doubles, host), by the same formulas the
 * knot kernel uses (Sec. II-C trajectory). Host only; used by tools that need
 * positions along the path (e.g. static responses sampled along it). */
msrc_status msrc_trajectory_positions(msrc_room_t room, const double* times, int64_t n_times, double* out);

/* Knot rates from the motion (Sec. II-C, "Bandwidth Analysis of d_i(t)": the
 * distance of an image changes as smoothly as the motion allows, and the
 * farther the image, the more slowly; dense knots for the direct sound and
 * low orders, sparse knots for high orders). For every tier of the room,
 * writes to rates_hz[t] (host array of n_tiers doubles) the lowest rate fs / N
 * (N an integer in [1, max_step]) at which linear interpolation between knots
 * keeps the delay of every image of the tier within tol_samples of its exact
 * value over [0, duration]. It uses the chord bound (N / fs)^2 / 8 * max |d''|
 * * fs / c with |d''| <= (|s'| + |m'|)^2 / d_min + |s''| + |m''|: speeds and
 * accelerations of the source (and array) from second differences on a 1 ms
 * grid, d_min the tier's smallest image distance on a 256-point grid, lowered
 * by the largest motion between grid points, and a safety factor of 1.25. For
 * a spline path (source or array) N also divides the path's length in samples,
 * so that its clamped end, where the velocity jumps, is a knot.
 * tol_samples > 0, max_step >= 1; needs a trajectory (MSRC_ERR_STATE). The
 * room's own tier rates are not changed: create a room with these rates. */
msrc_status msrc_suggest_knot_rates(msrc_room_t room, double tol_samples, int32_t max_step, double* rates_hz);

/* Knot rates for band-limited upsampling (Sec. II-C: the image distance is
 * band-limited by the motion, so knots at a rate above twice its bandwidth
 * recover it; the nearer the image, the wider the band). For every tier,
 * writes to rates_hz[t] the lowest rate fs / N (N an integer, rates tried
 * from 1 / duration up in steps of 1.25x) at which the room's band-limited
 * kernel (upsample_halfwidth) reproduces the distances of the tier's four
 * nearest images within tol_samples of delay. The error is checked at 16
 * points per knot interval over [0, duration], for microphone 0 carried by
 * the array, with the knots beyond the ends on the path's extension. Use the
 * rates with tier_upsample; linear interpolation between the virtual knots
 * adds its own chord error. tol_samples > 0; needs a trajectory (MSRC_ERR_STATE). */
msrc_status msrc_suggest_bandlimited_rates(msrc_room_t room, double tol_samples, double* rates_hz);

/* Replaces the six wall reflection coefficients of a room (beta: 6 doubles in
 * [0, 1], host memory); the Farrow fit and the trajectory are kept. Used by
 * optimisation loops that update the walls between forward calls. */
msrc_status msrc_set_reflection(msrc_room_t room, const double* beta);

/* Workspace bytes needed by msrc_synthesize (*fwd_bytes) and by
 * msrc_synthesize_backward (*bwd_bytes) for these rooms, input lengths
 * n_in[r] and output lengths n_out[r] (host arrays of n_rooms entries).
 * Either output pointer may be NULL. */
msrc_status msrc_workspace_size(const msrc_room_t* rooms, int32_t n_rooms,
                                const int64_t* n_in, const int64_t* n_out,
                                size_t* fwd_bytes, size_t* bwd_bytes);

/* Forward synthesis, Eq. 8: for every room r and microphone m,
 *   y_dev[r][m * n_out[r] + n] = sum_i A_i(n) * (fractional delay of x_dev[r] by tau_i(n))
 * for n in [0, n_out[r]). x_dev[r]: n_in[r] floats (device); x is zero outside
 * [0, n_in). y_dev[r]: n_mics x n_out[r] floats (device), fully overwritten.
 * rooms, x_dev, n_in, y_dev, n_out are host arrays of n_rooms entries; all rooms
 * must share taps, window and kaiser_beta. n_rooms > 1 runs every scene in the
 * same launches (one persistent synthesis launch over a work queue).
 * workspace_dev: >= msrc_workspace_size(...).fwd_bytes, 256-byte aligned.
 * The result is bitwise reproducible for the same inputs and tile configuration;
 * a batched call equals the single calls of its scenes bitwise when both run in
 * the same tile configuration (name one: the automatic default may choose
 * differently for a batch and for one of its scenes). */
msrc_status msrc_synthesize(const msrc_room_t* rooms, int32_t n_rooms,
                            const float* const* x_dev, const int64_t* n_in,
                            float* const* y_dev, const int64_t* n_out,
                            void* workspace_dev, size_t workspace_bytes, void* stream);

/* Tile configuration of a call (the synthesis launch's CTA shape, window and
 * record capacity; msrc_tile_configs() lists how many exist):
 * MSRC_TILE_DEFAULT = the process default (msrc_set_tile_config, initially
 * MSRC_TILE_AUTO); MSRC_TILE_AUTO = chosen from the call's knot layout (tiles
 * of 768 samples with two CTAs per SM; per-knot records, which hold twice as
 * many images per block, when most images sit on knots at most 24 samples
 * apart, interval records otherwise); else 0 .. msrc_tile_configs() - 1. The _cfg entry points take it per call, so
 * that workloads tuned differently (msrc_autotune) share a process without
 * overwriting each other's choice. The workspace size depends on it: size the
 * workspace with the configuration the call uses. An id out of range is
 * MSRC_ERR_INVALID_ARG. Results of every configuration agree within FP32
 * rounding; for a fixed configuration they are bitwise reproducible. */
#define MSRC_TILE_DEFAULT (-1)
#define MSRC_TILE_AUTO (-2)
msrc_status msrc_workspace_size_cfg(const msrc_room_t* rooms, int32_t n_rooms,
                                    const int64_t* n_in, const int64_t* n_out, int32_t tile_config,
                                    size_t* fwd_bytes, size_t* bwd_bytes);
msrc_status msrc_synthesize_cfg(const msrc_room_t* rooms, int32_t n_rooms,
                                const float* const* x_dev, const int64_t* n_in,
                                float* const* y_dev, const int64_t* n_out, int32_t tile_config,
                                void* workspace_dev, size_t workspace_bytes, void* stream);

/* Same computation with HOST signal buffers: x_host[r] is copied to the
 * workspace, the scene is synthesised and y is copied back into y_host[r]
 * (n_mics x n_out[r] floats), all enqueued on `stream`. The caller synchronises
 * the stream before reading y_host; pinned host memory makes the copies
 * asynchronous. Workspace: msrc_workspace_size(...).fwd_bytes plus the signal
 * bytes (sum_r 4*(n_in[r] + n_mics*n_out[r]), each rounded up to 256). */
msrc_status msrc_synthesize_host(const msrc_room_t* rooms, int32_t n_rooms,
                                 const float* const* x_host, const int64_t* n_in,
                                 float* const* y_host, const int64_t* n_out,
                                 void* workspace_dev, size_t workspace_bytes, void* stream);

/* Extra workspace bytes msrc_synthesize_host needs on top of the forward size. */
msrc_status msrc_host_io_bytes(const msrc_room_t* rooms, int32_t n_rooms,
                               const int64_t* n_in, const int64_t* n_out, size_t* bytes);

/* Adjoint of msrc_synthesize (reverse mode), for an upstream gradient
 * dy_dev[r] (n_mics x n_out[r] floats, device) of a scalar loss:
 *   dx_dev[r]     (n_in[r] floats, device, nullable): dL/dx
 *   dparams_dev[r] (48 doubles, device, nullable): dL/d traj.params (spline
 *                 control points; line p0 and speed; circle centre, radius and speed)
 *   dbeta_dev[r]  (6 doubles, device, nullable): dL/d beta per wall
 * Delays are recomputed from the trajectory, not stored. Every tier kind is
 * differentiated: linear knots, band-limited knots (through the upsampler's
 * weights) and emission-time delays (through the implicit emission time,
 * dd/dtheta = (sigma o u)^T J(e) / (1 + (sigma o u) . s'(e) / c)). Reductions
 * use a fixed order, so results are bitwise reproducible. The rooms, signals and lengths must
 * be those of the forward call whose output dy refers to. The source speed must
 * stay below c/2 on the output range (1 ms grid), else MSRC_ERR_UNSUPPORTED:
 * the dx scatter relies on consecutive samples of one image reading different
 * (Farrow segment, column) bins. */
msrc_status msrc_synthesize_backward(const msrc_room_t* rooms, int32_t n_rooms,
                                     const float* const* x_dev, const int64_t* n_in,
                                     const float* const* dy_dev, const int64_t* n_out,
                                     float* const* dx_dev, double* const* dparams_dev,
                                     double* const* dbeta_dev,
                                     void* workspace_dev, size_t workspace_bytes, void* stream);

/* msrc_synthesize_backward with one more output per room:
 *   darray_dev[r] (48 doubles, device, nullable): dL/d of the microphone
 *                 array's trajectory parameters (msrc_set_array_trajectory;
 *                 the microphones sit at their positions plus a(t) - a(0)),
 *                 laid out like those parameters; zeros for a room without
 *                 array motion.
 * The microphones' positions are inputs of Sec. II-A's distance; this is its
 * derivative through the array motion: dd/dm = -Delta / d at the knot time
 * (reception-time distances), through the upsampler's weights for band-limited
 * tiers, and dd/dm = -u / (1 + (sigma o u) . s'(e) / c) for emission-time
 * delays. Asking for it adds a second pass of the gradient kernel over the
 * linear tiers. Same workspace (msrc_workspace_size) and other arguments as
 * msrc_synthesize_backward, whose results it leaves unchanged. */
msrc_status msrc_synthesize_backward_ex(const msrc_room_t* rooms, int32_t n_rooms,
                                        const float* const* x_dev, const int64_t* n_in,
                                        const float* const* dy_dev, const int64_t* n_out,
                                        float* const* dx_dev, double* const* dparams_dev,
                                        double* const* dbeta_dev, double* const* darray_dev,
                                        void* workspace_dev, size_t workspace_bytes, void* stream);

/* Batched synthesis with a reusable plan. msrc_batch_create plans the call
 * (scene descriptors, work queue of (scene, microphone, image block, output
 * tile) items, workspace layout) and uploads the descriptors into the
 * workspace once, synchronising `stream`; the rooms' current trajectories,
 * walls and the signal / output pointers are bound at this point (re-create
 * the batch after changing them). msrc_batch_run enqueues only kernels on
 * `stream` (image enumeration and sort, knots, prefilter, one persistent
 * synthesis launch over all scenes, reduction); with use_graph != 0 the
 * first run captures them into a CUDA graph (the stream must not be the
 * legacy default stream) and later runs replay it. Arguments as for
 * msrc_synthesize; the workspace must stay allocated until the batch is
 * destroyed. msrc_batch_create runs in the process default tile configuration
 * at creation, msrc_batch_create_cfg in the one it is given (see
 * MSRC_TILE_DEFAULT); either is frozen for the life of the batch. */
typedef struct msrc_batch* msrc_batch_t;
msrc_status msrc_batch_create(const msrc_room_t* rooms, int32_t n_rooms,
                              const float* const* x_dev, const int64_t* n_in,
                              float* const* y_dev, const int64_t* n_out,
                              void* workspace_dev, size_t workspace_bytes, void* stream,
                              msrc_batch_t* out);
msrc_status msrc_batch_create_cfg(const msrc_room_t* rooms, int32_t n_rooms,
                                  const float* const* x_dev, const int64_t* n_in,
                                  float* const* y_dev, const int64_t* n_out, int32_t tile_config,
                                  void* workspace_dev, size_t workspace_bytes, void* stream,
                                  msrc_batch_t* out);
msrc_status msrc_batch_run(msrc_batch_t batch, int32_t use_graph, void* stream);
msrc_status msrc_batch_destroy(msrc_batch_t batch);

/* Autotuner of the synthesis launch: runs the given call (arguments as for
 * msrc_synthesize) in every tile configuration whose workspace fits, `reps`
 * times each after one warm-up, timed with CUDA events on `stream`; writes the
 * mean milliseconds per configuration into ms_per_config (msrc_tile_configs()
 * entries, -1 when skipped) and the fastest configuration's id into *best, for
 * the caller to pass to the _cfg entry points. No process-wide state changes.
 * Synchronises `stream`. */
msrc_status msrc_autotune(const msrc_room_t* rooms, int32_t n_rooms, const float* const* x_dev,
                          const int64_t* n_in, float* const* y_dev, const int64_t* n_out,
                          void* workspace_dev, size_t workspace_bytes, void* stream, int32_t reps,
                          double* ms_per_config, int32_t* best);

/* Reads (and clears) the device-side error word of a workspace used by the
 * calls above; synchronises `stream`. *flags receives a bit set:
 * 1 = a bounded wait gave up, 2 = a shared-memory window had to be clamped,
 * 4 = a block's band-limited knot scratch did not fit (its records were
 * skipped; the planner sizes blocks so that this does not happen). */
msrc_status msrc_workspace_errors(void* workspace_dev, void* stream, uint32_t* flags);

/* Test hook for the bounded waits. With bytes > 0 (a multiple of 16), every
 * shared-window staging of later synthesis and reverse-mode launches in this
 * process waits for `bytes` more than its copies deliver: the wait gives up
 * after about one second, the block records bit 1 in the error word and stops,
 * and the context stays usable (outputs of that launch are undefined).
 * 0 (the default) turns it off. Host only; INVALID_ARG for other sizes. */
msrc_status msrc_test_stall_window_copies(uint32_t bytes);

/* Measured ALU peaks of the current GPU: every thread of a full grid runs 16
 * independent fused multiply-add chains, FP32 and then FP64; best of 5 timed
 * launches after a warm-up, in TFLOP/s at 2 flops per FMA. These are the
 * measured counterparts of the unit-count peak (SMs x lanes x 2 x clock) that
 * the synthesis roofline is quoted against. scratch_dev: at least 16 bytes of
 * caller-owned device memory (never written in practice). Synchronises
 * `stream`; takes a few tens of milliseconds. */
msrc_status msrc_measure_alu_peaks(void* scratch_dev, void* stream, double* fp32_tflops, double* fp64_tflops);

/* Number of images of a room and, per tier, how many fall in it (host only).
 * per_tier: MSRC_MAX_TIERS entries, nullable. */
msrc_status msrc_room_image_count(msrc_room_t room, int64_t* count, int64_t* per_tier);

/* Maximum absolute error, over a dense grid of fractional delays, of the fitted
 * Farrow polynomials against the exact windowed sinc (host only). */
msrc_status msrc_room_fit_error(msrc_room_t room, double* max_abs_error);

/* The Farrow table the kernels use for this room (Sec. II-B, Eq. 3-5), as the
 * device receives it (host only). The fractional delay alpha in [0, 1) falls in
 * segment s = floor(4 alpha) with local variable w = 4 alpha - s - 1/2 in
 * [-1/2, 1/2), and tap k (k = -L/2 .. L/2 - 1, L = taps) weighs
 *   h(k; alpha) = sum_{q < P} out[(s * P + q) * L + k + L/2] w^q.
 * which = 0: the synthesis (and dx) table, P = 5; which = 1: the reverse-mode
 * gradient kernel's table, P = 6. out: 4 * P * L floats (host, caller-owned);
 * *n_powers receives P. */
msrc_status msrc_room_farrow_table(msrc_room_t room, int32_t which, float* out, int32_t* n_powers);

/* Process default tile configuration (MSRC_TILE_AUTO initially; an id or
 * MSRC_TILE_AUTO): the configuration of every call that names none
 * (msrc_synthesize, msrc_synthesize_host, msrc_workspace_size,
 * msrc_batch_create, msrc_synthesize_noalloc, or MSRC_TILE_DEFAULT);
 * msrc_tile_configs lists how many exist. Thread-safe. */
msrc_status msrc_set_tile_config(int32_t config_id);
int32_t msrc_tile_configs(void);

/* Per-phase timing with CUDA events recorded on the launching stream of every
 * subsequent msrc_synthesize call (at most 256 calls between reads).
 * msrc_profile_read synchronises on the recorded events and returns, summed
 * over the calls since the previous read, the milliseconds of the phases
 * ms[0] setup (image enumeration and sort, trajectory knots, delay records),
 * ms[1] prefilter, ms[2] synthesis (gather-accumulate), ms[3] reduction;
 * *n_calls receives the number of calls summed. */
msrc_status msrc_profile_enable(int32_t on);
msrc_status msrc_profile_read(double* ms, int32_t* n_calls);

/* Allocation-free forward synthesis. The paper has no counterpart: this is a
 * service of the library for callers that may not allocate device memory, such
 * as a plug-in whose host application owns every device buffer through its own
 * pool, or a real-time audio thread that must not enter the CUDA allocator.
 * Same result as msrc_synthesize for one room (x_dev: n_in floats, y_dev:
 * n_mics x n_out floats, both device memory owned by the caller), computed in a
 * scratch array of MSRC_NOALLOC_SCRATCH_BYTES that the library reserves in
 * device memory on every GPU where it is loaded, for the life of the process.
 * Rooms whose workspace (msrc_workspace_size) exceeds that size are rejected
 * with MSRC_ERR_WORKSPACE. The call makes no cudaMalloc or cudaFree. The array
 * is committed when the library's device code is loaded on a GPU; under lazy
 * module loading (the CUDA default) that is the first call on that device,
 * which also looks up the array's device address with the device current: make
 * that first call during set-up, before any stream capture. All calls share the
 * one array and its contents persist between calls: calls that may overlap on
 * the GPU (other streams or threads) race, so the caller serialises them.
 * Device-side anomalies of these calls (the error bits of msrc_workspace_errors)
 * are read with msrc_noalloc_errors. */
#define MSRC_NOALLOC_SCRATCH_BYTES (32u << 20)
msrc_status msrc_synthesize_noalloc(msrc_room_t room, const float* x_dev, int64_t n_in,
                                    float* y_dev, int64_t n_out, void* stream);

/* Reads and clears the device error word of the allocation-free calls on the
 * current device (the bit set of msrc_workspace_errors, for the scratch array
 * of msrc_synthesize_noalloc); synchronises `stream`. Returns
 * MSRC_ERR_TIMEOUT when bit 1 (a bounded wait gave up) is set. */
msrc_status msrc_noalloc_errors(void* stream, uint32_t* flags);

const char* msrc_status_string(msrc_status status);
const char* msrc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MSRC_H */
