/*
 * emppp.h -- C ABI of the GB300 EM-PP library (electromagnetic particle-particle bunch solver).
 *
 * One EM-PP step (arXiv 2605.05543, Sec. 2.1-2.3) advances N interacting electrons: every target i
 * sees every source j != i through the Lienard-Wiechert fields eq:LW_E / eq:LW_B evaluated at the
 * retarded time, which is bracketed in j's stored trajectory history and rebuilt by the linear
 * reconstruction eq:dt / eq:linear (eq:linear2 when it is older than the history); the summed self
 * fields plus a prescribed background B field (Sec. 2.6) drive a Higuera-Cary push (Sec. 2.3).
 *
 * Conventions for every call:
 *   - SI units: positions m, proper velocities u = gamma v in m/s, times s, fields V/m and T.
 *   - Vectors are interleaved per particle: x[3*i + c], c = 0,1,2 (x, y, z).
 *   - Pointers marked "host or device" are read as device pointers when is_device_ptr != 0, else as
 *     host pointers. Host arrays stay owned by the caller and are copied before the call returns;
 *     device arrays must stay valid until the call returns and are read on the handle's stream.
 *   - Every call returns an emppp_status. Calls never abort and never print. emppp_last_error()
 *     gives a text for the last failing call of this thread. A numeric fault found on the device
 *     (negative discriminant, |v| >= c, coincident particles, non-finite field) is reported as
 *     EMPPP_ERR_NUMERIC by the next call that synchronises (get_*, emppp_synchronize).
 *   - The library owns all device memory it allocates (cudaMalloc at create time; nothing is
 *     allocated by emppp_step).
 *   - A handle is not thread-safe: one thread at a time may use it.
 */
#ifndef EMPPP_H
#define EMPPP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define EMPPP_API __attribute__((visibility("default")))
#else
#define EMPPP_API
#endif

typedef struct emppp_ctx* emppp_handle;

typedef enum {
  EMPPP_OK = 0,
  EMPPP_ERR_ARG = -1,     /* bad handle, size, pointer or option */
  EMPPP_ERR_CUDA = -2,    /* a CUDA runtime call failed (text in emppp_last_error) */
  EMPPP_ERR_NUMERIC = -3, /* device-side numeric fault in a previous step */
  EMPPP_ERR_TIMEOUT = -4, /* a bounded device wait gave up: a warp's wait on its staged history window
                             (emppp_set_wait_limit); the fields of that step are still exact */
  EMPPP_ERR_STATE = -5,   /* call out of order (e.g. step before set_particles) */
  EMPPP_ERR_OOM = -6      /* device allocation failed */
} emppp_status;

/* Background magnetic field models (Sec. 2.6). NONE: B_ext = 0. UNIFORM: B_ext = b.
 * DIPOLE: centred dipole, B = mu0/(4 pi) [3 (M.rhat) rhat - M] / r^3 with M = m0 e_z and r measured
 * from `center`. B_ext is evaluated at the half-step position x^{n+1/2}. */
typedef enum { EMPPP_BEXT_NONE = 0, EMPPP_BEXT_UNIFORM = 1, EMPPP_BEXT_DIPOLE = 2 } emppp_bext_kind;

typedef struct {
  int32_t kind;     /* emppp_bext_kind */
  int32_t pad_;
  double b[3];      /* UNIFORM: field vector, T */
  double m0;        /* DIPOLE: moment along +z, A m^2 */
  double center[3]; /* DIPOLE: dipole position, m */
} emppp_bext;

/* Precision of the pair-field path.
 *   FP64:  every result of the pair path in FP64 (node tests decided in FP32 outside a guard band and
 *          in FP64 inside it, so the brackets are the FP64 ones); agrees with the FP64 oracle to ~1e-14.
 *   MIXED: pair geometry and fields in FP32 on hi/lo-split coordinates with compensated FP32
 *          sums; time stamps, the bracket decision and the push stay FP64. */
typedef enum { EMPPP_FP64 = 0, EMPPP_MIXED = 1 } emppp_precision;

/* First guess of the retarded-time search (Sec. 2.2). Every proposal ends in the same bracket
 * [t_k1, t_k1+1] as the plain search, because the bracket is the unique change of sign of the
 * node test and each guess is checked by it.
 *   BISECT:      the paper's search: out-of-history test, near-field shortcut, bisection.
 *   CLOSED_FORM: uniform-motion delay from the source's present state, then a guarded walk.
 *   MLP:         delay predicted by the 10-64-64-1 network set by emppp_set_proposal. */
typedef enum { EMPPP_PROPOSAL_BISECT = 0, EMPPP_PROPOSAL_CLOSED_FORM = 1, EMPPP_PROPOSAL_MLP = 2 } emppp_proposal;

/* Reconstruction of the retarded state inside the bracket [t_1, t_2] (Sec. 2.2).
 *   LINEAR:   the method's own: delta t from the quadratic eq:dt, then eq:linear.
 *   MIDPOINT: eq:mid, the earlier scheme the paper improves on, kept as an accuracy comparison:
 *             t_r = (t_1 + t_2) / 2, w = (w_1 + w_2) / 2, v = (v_1 + v_2) / 2, a = (v_2 - v_1) / (t_2 - t_1).
 *             Pairs older than the history keep eq:linear2. FP64 precision and a fixed dt only. */
typedef enum { EMPPP_RECON_LINEAR = 0, EMPPP_RECON_MIDPOINT = 1 } emppp_reconstruction;

/* Where a step evaluates the self fields (Sec. 2.3).
 *   PRESENT:   at the stored present positions x^n and time t_n (the method as built).
 *   HALF_STEP: at the pusher's half-step positions x^{n+1/2} = x^n + (dt/2) v^n and time t_n + dt/2,
 *              kept as a comparison. Before the pair evaluation every particle's history gains a
 *              provisional slot n+1 = (t_n + dt/2, x^{n+1/2}, v^n), which counts in the depth D; the push
 *              then replaces it with the real slot n+1 at t_n + dt. FP64 precision and a fixed dt only;
 *              emppp_fields is not affected. */
typedef enum { EMPPP_FIELD_PRESENT = 0, EMPPP_FIELD_HALF_STEP = 1 } emppp_field_point;

typedef struct {
  int32_t precision;   /* emppp_precision, default FP64 */
  int32_t proposal;    /* emppp_proposal, default BISECT */
  int32_t pair_fields; /* 1 (default): self fields on; 0: E = 0, B = B_ext (stage-2 transport, Sec. 2.7) */
  int32_t source_split;/* 0 (default): automatic; >0: number of source slices per target block */
  int32_t timing;      /* 1: record CUDA events around every pair evaluation and step (see emppp_stats) */
  int32_t graphs;      /* 1 (default): emppp_step with nsteps > 1 replays one captured CUDA graph per step
                          (only on a non-default stream and with timing off) */
  int32_t reconstruction; /* emppp_reconstruction, default LINEAR */
  int32_t field_point;    /* emppp_field_point, default PRESENT */
} emppp_options;

/* Counters accumulated over the steps since the last emppp_reset_stats (Sec. 2.2 branches). */
typedef struct {
  int64_t steps;           /* steps taken */
  int64_t pairs;           /* ordered pairs (i, j != i) evaluated: steps * N (N - 1) with pair fields on */
  int64_t out_of_history;  /* pairs with t_r older than the history (eq:linear2) */
  int64_t shortcut;        /* pairs bracketed by the near-field shortcut */
  int64_t bisection;       /* pairs bracketed by the search */
  int64_t node_tests;      /* evaluations of c (t - t_k) <= |r - w_k| over all pairs */
  int64_t guard_fallbacks; /* node tests decided in FP64 after an inconclusive FP32 test */
  int64_t kernel_launches; /* kernels launched by the library (cumulative since emppp_create) */
  double pair_ms;          /* device time of the pair evaluations (timing option on, else 0) */
  double step_ms;          /* device time of whole steps (timing option on, else 0) */
  int64_t timed_steps;     /* steps whose events were recorded (the event pool holds 4096 steps) */
  double dt_last;          /* step size of the last step (s) */
  double eta_min;          /* adaptive step: min |eta_ij| over the last step's pairs above the cutoff (m), else 0;
                              in a batch, of the bunch whose step is the smallest */
  double v_max;            /* adaptive step: max |v_i - v_j(t_r)| over the same pairs (m/s), else 0 */
} emppp_stats;

/* Work split and tile shape of the pair kernel: items_per_block work items (bunch, source chunk, target
 * tile) per resident block of 128 threads, which sets the sources per chunk; target_order 1 sorts the
 * targets spatially each step (both paths; the fields do not depend on it; a step of a system of at most
 * 2048 particles on the mixed path skips it). The tile shape: targets_per_block targets per work item and
 * thread block (64, 128 or 256; a mixed-path block stages half that many sources per tile) and, on the
 * mixed path, sources_per_sum sources per FP32 partial sum before the compensated addition (8, 16 or 32;
 * 16 and 32 only at 128 targets per block). The FP64 path ignores sources_per_sum. The shape changes the order
 * of each target's sum, so fields of different shapes agree within rounding, not bit for bit; the
 * adaptive time step and the comparison variants run the default shape (128, 8). history_window nonzero
 * (mixed path, shape (128, 32), closed-form or MLP proposal) has each warp copy, one source ahead, the
 * run of history slots its 32 targets' guessed brackets of the next source fall in (at most 32 slots) from
 * the FP32 ring into shared memory by bulk copy, and read those brackets' records there; it changes where
 * records are read, not the arithmetic or the work split, so its fields equal those of (128, 32) without
 * it bit for bit. Chosen by emppp_autotune or set with emppp_set_tuning. */
typedef struct {
  int32_t items_per_block;   /* default 16 */
  int32_t target_order;      /* default 1 */
  double ms;                 /* measured time of one field evaluation (emppp_autotune), else 0 */
  int32_t targets_per_block; /* default 128 (0 in emppp_set_tuning: 128) */
  int32_t sources_per_sum;   /* default 8 (0 in emppp_set_tuning: 8) */
  int32_t history_window;    /* default 0; slots of the staged window per warp and source when on */
} emppp_tuning;

typedef struct {
  int32_t ncand;           /* candidates timed */
  int32_t best;            /* index of the chosen one */
  emppp_tuning cand[32];
} emppp_tuning_report;

/* Fills *out with the defaults listed above. */
EMPPP_API void emppp_default_options(emppp_options* out);

/* Creates a solver for n particles with a history of `history_depth` slots (the present slot
 * included; depth >= 2) and fixed step dt > 0. opt may be NULL (defaults). cuda_stream is a
 * cudaStream_t (NULL: the legacy default stream). Allocates all device memory of the solver on the
 * current device. *out is NULL on failure; EMPPP_ERR_ARG for an unknown option value or for the
 * MIDPOINT reconstruction or HALF_STEP field point with MIXED precision. Sec. 2.2 (history), Sec. 2.3
 * (time step). */
EMPPP_API emppp_status emppp_create(int64_t n, int32_t history_depth, double dt, const emppp_options* opt,
                                    void* cuda_stream, emppp_handle* out);

/* Creates a solver for nbunch independent bunches (particles interact only within their own bunch)
 * with n_per_bunch[b] >= 1 particles each, sharing the history depth, the step dt and the time. All
 * per-particle arrays of the other calls then hold the bunches one after the other (bunch 0 first).
 * Every step evaluates all bunches in one persistent launch of the pair kernel whose work items are
 * (bunch, source chunk, target tile). emppp_create(n, ...) is the case nbunch = 1. */
EMPPP_API emppp_status emppp_create_batch(int32_t nbunch, const int64_t* n_per_bunch, int32_t history_depth,
                                          double dt, const emppp_options* opt, void* cuda_stream,
                                          emppp_handle* out);

/* Frees every device resource of the handle (NULL is ignored). */
EMPPP_API void emppp_destroy(emppp_handle h);

/* Sets the initial state at t = 0, step 0: positions x [3n], proper velocities u [3n] (host or
 * device) and optional macro-particle weights w [n] (charge -e w, mass m_e w; NULL: all 1). Resets
 * the history to the single slot 0 holding (x, v = u / gamma). Sec. 2.2, Sec. 2.5. */
EMPPP_API emppp_status emppp_set_particles(emppp_handle h, const double* x, const double* u, const double* w,
                                           int32_t is_device_ptr);

/* Restores a state with history (checkpoint resume, or a prepared history): the present step
 * index n >= 0, nslots = min(n + 1, depth) most recent slots k = n - nslots + 1 .. n with time
 * stamps T [nslots] (increasing), positions W [nslots][n_particles][3] and velocities
 * V [nslots][n_particles][3] (|V| < c), the present proper velocities u [3n] and optional weights
 * w [n] (NULL: all 1). Host or device. The present position is W[nslots - 1]. */
EMPPP_API emppp_status emppp_set_history(emppp_handle h, int64_t n, int32_t nslots, const double* T,
                                         const double* W, const double* V, const double* u, const double* w,
                                         int32_t is_device_ptr);

/* Copies the stored history out in the layout emppp_set_history takes. T [nslots], W, V
 * [nslots][n][3], u [3n] (host or device); *n_now and *nslots receive the present step and the
 * number of slots written (= min(n + 1, depth)); the arrays must hold `depth` slots. */
EMPPP_API emppp_status emppp_get_history(emppp_handle h, int64_t* n_now, int32_t* nslots, double* T, double* W,
                                         double* V, double* u, int32_t is_device_ptr);

/* Advances nsteps >= 0 steps (Sec. 2.1-2.3): self fields at (x^n, t_n), B_ext at x^{n+1/2},
 * Higuera-Cary push, append of slot n+1. bext may be NULL (NONE). Asynchronous on the handle's
 * stream: returns once the work is enqueued. */
EMPPP_API emppp_status emppp_step(emppp_handle h, int64_t nsteps, const emppp_bext* bext);

/* Stage-1 -> stage-2 handoff (Sec. 2.7): translates every bunch so that its weighted centroid sits at
 * center[3] (momenta kept) and restarts the history at the present slot. Used before
 * emppp_transport to start the field-dominated transport at a given place (e.g. 4 Earth radii on the
 * equator). Synchronises the stream. */
EMPPP_API emppp_status emppp_handoff(emppp_handle h, const double* center);

/* Stage-2 transport (Sec. 2.7): advances every particle nsteps >= 0 steps of dt > 0 with the pair
 * interaction off (E = 0, B = B_ext evaluated at x^{n+1/2}, the same Higuera-Cary step as
 * emppp_step), keeping no history on the way; afterwards the history holds only the present slot,
 * the step index has grown by nsteps and the time by nsteps * dt (accumulated step by step).
 * Particles are independent here, so each GPU thread keeps its particle in registers for up to 4096
 * steps per launch. Asynchronous. */
EMPPP_API emppp_status emppp_transport(emppp_handle h, int64_t nsteps, double dt, const emppp_bext* bext);

/* Present positions x [3n], proper velocities u [3n] (host or device, either may be NULL), time
 * and step index (either may be NULL). Synchronises the stream. */
EMPPP_API emppp_status emppp_get_state(emppp_handle h, double* x, double* u, double* t_now, int64_t* n_now,
                                       int32_t is_device_ptr);

/* Fields used by the last completed step: self E [3n] and B [3n] = self + B_ext(x^{n+1/2})
 * (host or device, either may be NULL). Synchronises the stream. */
EMPPP_API emppp_status emppp_get_fields(emppp_handle h, double* E, double* B, int32_t is_device_ptr);

/* Counters accumulated since the last emppp_reset_stats (or create / set_particles / set_history).
 * Synchronises the stream. */
EMPPP_API emppp_status emppp_get_stats(emppp_handle h, emppp_stats* out);

/* Zeroes the accumulated counters and recorded times (not kernel_launches). */
EMPPP_API emppp_status emppp_reset_stats(emppp_handle h);

/* Times the pair-field evaluation of the present state (slot tables, target order, pair kernel and
 * partial-sum reduction; the state is not advanced; one warm-up, best of two) for items_per_block in
 * {4, 8, 16, 32, 64}, with and without the spatial target order, at the default tile shape; then, with
 * the fastest of those and unless the adaptive time step is on, for the other tile shapes (targets per
 * block 64 and 256; on the mixed path also 16 and 32 sources per partial sum). Keeps the fastest candidate for
 * later steps of the current precision and proposal. report may be NULL. Synchronises the stream; resets
 * the stats; afterwards emppp_get_fields reports the fields of the last evaluation. */
EMPPP_API emppp_status emppp_autotune(emppp_handle h, emppp_tuning_report* report);

/* Bracket of the retarded-time search of every ordered pair of the present state (Sec. 2.2), for
 * checking the search pair by pair: one evaluation of the present state's self fields with the handle's
 * precision and proposal (the state does not advance; emppp_get_fields then reports this evaluation's
 * fields), whose pair kernel also writes, for target i and source j != i of one bunch,
 *   brackets[i * n + j] = 4 (k1 - k0) + branch   (branch 0 out of history, 1 near-field shortcut,
 *                                                 2 bisection; k1 the older node of the bracket),
 * and -1 for i == j and for pairs of different bunches. brackets: DEVICE array of n * n int32 (n the
 * particles of all bunches, at most 65536), owned by the caller. *k0 (host, may be NULL) receives the
 * absolute index of the earliest usable slot. Synchronises the stream and resets the stats; the library
 * allocates nothing.
 * EMPPP_ERR_STATE with pair fields off, with the half-step field point, or with the MLP proposal and no
 * network. */
EMPPP_API emppp_status emppp_bracket_dump(emppp_handle h, int32_t* brackets, int64_t* k0);

/* Sets the work split and tile shape directly (e.g. a tuning found earlier). items_per_block in 1..256,
 * targets_per_block in {0 (= 128), 64, 128, 256}, sources_per_sum in {0 (= 8), 8, 16, 32}, 16 and 32 only
 * with 128 targets per block, history_window nonzero only with (128, 32); EMPPP_ERR_ARG otherwise.
 * history_window on the FP64 path or with the bisection proposal reads the ring directly (no window). */
EMPPP_API emppp_status emppp_set_tuning(emppp_handle h, const emppp_tuning* tuning);

/* Probes of the bounded wait of a warp on its staged history window (history_window on; default 65536, each
 * probe suspending the thread for at most 1 us, so a wait gives up after at most about 65 ms). A wait that gives up leaves that warp
 * gathering the records from the ring for the rest of the launch, so the fields are unchanged, and the
 * device error word records it: the next call that reads it returns EMPPP_ERR_TIMEOUT. probes = 0 makes
 * every such wait give up at once (a test of that path). EMPPP_ERR_ARG for probes < 0. */
EMPPP_API emppp_status emppp_set_wait_limit(emppp_handle h, int32_t probes);

/* Replaces the options for later steps. EMPPP_ERR_STATE for a comparison variant (MIDPOINT, HALF_STEP)
 * while the adaptive time step is on. */
EMPPP_API emppp_status emppp_set_options(emppp_handle h, const emppp_options* opt);

/* Replaces the stream later calls enqueue on (cudaStream_t, NULL: legacy default stream). */
EMPPP_API emppp_status emppp_set_stream(emppp_handle h, void* cuda_stream);

/* Waits for the handle's stream and reports a pending device-side numeric fault. */
EMPPP_API emppp_status emppp_synchronize(emppp_handle h);

/* Self fields of n particles at the present slot of a history held by the caller, evaluated without
 * allocating any device memory. There is no counterpart in the paper: this entry point exists for
 * callers that own all device memory themselves (a framework whose caching allocator holds the GPU,
 * a service with a fixed device-memory budget, a loop where an allocation could stall or fail) and
 * so cannot let the library cudaMalloc its own buffers.
 *   T [nslots], W and V [nslots][n][3]: device pointers, the layout of emppp_set_history; slot
 *     nslots - 1 is the present one and every slot is usable (the history depth is nslots).
 *   w [n] optional weights (NULL: 1); E, B [n][3] device outputs (B is the self field only).
 *   cuda_stream: cudaStream_t the work is enqueued on (NULL: legacy default stream); asynchronous.
 * The FP64 path with the paper's search (out-of-history test, shortcut, bisection) is used. Its working
 * memory is one fixed 16 MiB device array inside the library (held by every GPU that loads the
 * library until the process exits), which limits n to 348160 and nslots to 4096: larger sizes are
 * rejected with EMPPP_ERR_ARG. All calls share that array, so calls whose work overlaps on the GPU
 * race with each other: serialise them. The first call on a device looks up the array's device
 * address (with that device current) and keeps it for the life of the process; make that first call
 * before any stream capture, and do not reset the device (cudaDeviceReset) between calls. The work runs
 * on the current device: T, W, V, w, E and B must be allocations of that device, and cuda_stream a stream
 * of it. A numeric fault of a pair (|v| >= c, coincident particles, a non-finite input) is not reported
 * through the status: that target's E and B come out NaN and the call returns EMPPP_OK. */
EMPPP_API emppp_status emppp_fields_noalloc(int64_t n, int32_t nslots, const double* T, const double* W,
                                            const double* V, const double* w, double* E, double* B,
                                            void* cuda_stream);

/* ---- Learned retarded-time proposal --------------------------------------------------------------
 * A 10-64-64-1 perceptron with SiLU activations predicts z = log(c (t - t_r) / |d|) for a target and a
 * source (d = r - w_n, the present separation); the search then starts at the slot the predicted
 * delay points at and finishes with the guarded search, so brackets and fields are those of the
 * paper's search whatever the network predicts (no counterpart in the paper: it is a proposal for
 * the bracketing of Sec. 2.2).
 * Features, per pair (FP32): d / |d| (3), |d| / L (1), beta_n (3), (beta_n - beta_{n-1}) D (3) with
 * L = c dt D, beta = v / c of the source at its present slot n and the slot before.
 * Parameters (FP32, EMPPP_MLP_NUM_PARAMS values): W1[10][64] (feature, unit), b1[64], W2[64][64] (in,
 * out), b2[64], w3[64], b3. Tensor-core passes round X, W1, silu(H1) and W2 to BF16 and accumulate in
 * FP32. */
#define EMPPP_MLP_NUM_PARAMS 4929

typedef struct {
  int32_t epochs;   /* passes over the data */
  int32_t batch;    /* rows per Adam step */
  float lr;         /* Adam step size */
  float beta1;      /* Adam first-moment decay (0.9) */
  float beta2;      /* Adam second-moment decay (0.999) */
  float eps;        /* Adam epsilon (1e-8) */
  float lr_final;   /* step size of the last Adam step: cosine decay from lr; 0 (or >= lr) keeps lr */
  int32_t reserved;
} emppp_mlp_config;

/* Training data from the method itself: for m (target, source) pairs (pairs[2k], pairs[2k+1], indices
 * into the present particles, target != source) at the present state, the features [m][10], the exact
 * retarded delay t - t_r [m] (FP64 bracket of Sec. 2.2 and the smaller root of eq:dt) and the training
 * target z = log(c (t - t_r) / |d|) [m]. All arrays host or device. */
EMPPP_API emppp_status emppp_sample_delays(emppp_handle h, const int32_t* pairs, int64_t m, float* features,
                                           double* delays, float* targets, int32_t is_device_ptr);

/* z [m] of the network with parameters params for features [m][10]. mode 0: the reference form that
 * training differentiates (FP32 SiLU, BF16 GEMM operands); mode 1: the inference form the pair kernels
 * evaluate (hidden layers scaled by 1/2, SiLU on packed BF16 pairs via tanh, output layer on the tensor
 * cores). Device pointers; synchronous. */
EMPPP_API emppp_status emppp_mlp_forward(const float* params, const float* features, int64_t m, float* z,
                                         int32_t mode, void* cuda_stream);

/* Loss sum_r (z_r - targets_r)^2 / m and its gradient grad [EMPPP_MLP_NUM_PARAMS] for one batch of m
 * rows. Device pointers (loss on the host); synchronous. */
EMPPP_API emppp_status emppp_mlp_gradient(const float* params, const float* features, const float* targets,
                                          int64_t m, float* grad, double* loss, void* cuda_stream);

/* Trains params (device, in place) with Adam on m rows of (features, targets) (device), in consecutive
 * batches of cfg->batch rows, cfg->epochs passes; loss_per_epoch [epochs] (host, may be NULL) receives
 * the mean loss of each pass. Synchronous. */
EMPPP_API emppp_status emppp_mlp_train(float* params, const float* features, const float* targets, int64_t m,
                                       const emppp_mlp_config* cfg, float* loss_per_epoch, void* cuda_stream);

/* ---- adaptive time step (Sec. 2.4) ------------------------------------------------------------------
 * With enable = 1 every stage-1 step chooses its own size from the retarded solve of its pair
 * evaluation: over ordered pairs i != j with |eta_ij| >= eta_allow (eta_ij = x_i^n - w_j(t_r)),
 * eta_min = min |eta_ij| and v_max = max |v_i(t_n) - v_j(t_r)|, and the push from n to n+1 uses
 * dt = min(dt_max, max(dt_min, c_dt eta_min / v_max)) (dt_max when no pair qualifies or v_max = 0).
 * The history then holds unevenly spaced slots, which the retarded-time search handles by their time
 * stamps. The mixed path forms eta_min and v_max in FP32. emppp_stats reports the last step's dt,
 * eta_min and v_max; emppp_get_state the accumulated time. enable = 0 (or cfg = NULL) returns to the
 * fixed dt of emppp_create. In a batch each bunch's step comes from its own pairs, and the step taken,
 * common to all bunches, is the smallest of them; with
 * pair fields off no pair qualifies and every step is dt_max. Returns EMPPP_ERR_ARG unless c_dt > 0,
 * eta_allow >= 0 and 0 < dt_min <= dt_max, all finite, and EMPPP_ERR_STATE when enabling it on a solver
 * created with the MIDPOINT reconstruction or the HALF_STEP field point. The setting is kept until
 * changed, across emppp_set_particles and emppp_set_history. */
typedef struct {
  int32_t enable;
  int32_t reserved;
  double c_dt;      /* safety factor C (0.05 in the paper) */
  double eta_allow; /* lower cutoff of |eta_ij| (m); the paper leaves it open */
  double dt_min;    /* 1e-15 s in the paper */
  double dt_max;    /* 1e-12 s in the paper */
} emppp_adaptive_dt;

EMPPP_API emppp_status emppp_set_adaptive_dt(emppp_handle h, const emppp_adaptive_dt* cfg);

/* ---- stage switch by the energy criterion (Sec. 2.7) -------------------------------------------------
 * With enable = 1, after every stage-1 step the device forms each bunch's mean kinetic energy per
 * electron, E(t) = sum_i w_i (gamma_i - 1) m_e c^2 / sum_i w_i, and its backward difference
 * dE/dt = (E_n - E_{n-1}) / (t_n - t_{n-1}). The criterion arms once |dE/dt| >= eps_E; the bunch's switch
 * step is then the first step at which |dE/dt| < eps_E has held for `hold` consecutive steps. Enabling
 * starts the record at the present state; emppp_set_particles and emppp_set_history restart it. The paper
 * takes eps_E = 30 keV/s or less: 30e3 * 1.602176634e-19 J/s. Returns EMPPP_ERR_ARG unless eps_E > 0 and
 * hold >= 1; enable = 0 (or cfg = NULL) turns the monitor off. */
typedef struct {
  int32_t enable;
  int32_t hold;
  double eps_E; /* J/s per electron */
} emppp_energy_monitor;

typedef struct {
  double ebar;      /* mean kinetic energy per electron at the present step (J) */
  double rate;      /* dE/dt over the last step (J/s); 0 right after the record starts */
  double t_sw;      /* time of the switch step (s), 0 before */
  int64_t n_sw;     /* switch step, -1 before */
  int32_t armed;    /* |dE/dt| has reached eps_E */
  int32_t switched; /* the criterion has held */
} emppp_energy_state;

EMPPP_API emppp_status emppp_set_energy_monitor(emppp_handle h, const emppp_energy_monitor* cfg);
/* Per-bunch record (out: one entry per bunch). EMPPP_ERR_STATE while the monitor is off. Synchronises. */
EMPPP_API emppp_status emppp_get_energy(emppp_handle h, emppp_energy_state* out);

/* The two-stage procedure of Sec. 2.7 on this handle:
 *   1. from the initial state (x0, u0, w0; host or device, as emppp_set_particles takes them) step the
 *      full EM-PP model with the energy monitor on, checking every check_every steps, until every bunch
 *      has met the criterion or max_stage1_steps have run. The threshold step n_th (time t_th, the
 *      paper's first crossing) is the latest of the bunches' criterion steps (max_stage1_steps when one
 *      never meets it);
 *   2. restart from the same initial state and step the full model past the threshold to the switch
 *      time t_sw = t_th + t_after (the paper keeps the coupled model on for some time after the first
 *      crossing: t_sw > t_th); the first n_th steps reproduce the monitoring run bit for bit;
 *   3. if do_handoff, translate each bunch so that its centroid sits at `center` (emppp_handoff); then
 *      push steps2 steps of dt2 in the background field bext2 alone (emppp_transport).
 * The adaptive time step, options and tuning of the handle apply to both stage-1 runs. The energy
 * monitor stays on afterwards with eps_E and hold. Returns the first failing status of the calls above. */
typedef struct {
  double eps_E;
  int32_t hold;
  int32_t do_handoff;
  int64_t max_stage1_steps;
  int64_t check_every;
  double t_after;     /* coupled time kept after the threshold (s, >= 0) */
  emppp_bext bext1;   /* stage-1 background field */
  double center[3];   /* handoff target of each bunch's centroid */
  double dt2;         /* stage-2 step (s) */
  int64_t steps2;
  emppp_bext bext2;   /* stage-2 background field (the dipole, Sec. 2.6) */
} emppp_two_stage_config;

typedef struct {
  int64_t n_th;                    /* threshold step (first crossing) */
  double t_th;                     /* its time (s) */
  int64_t n_sw;                    /* stage-1 steps of the re-run: the first step with t >= t_th + t_after */
  double t_sw;                     /* time at n_sw (s) */
  int64_t stage1_steps_first_run;  /* steps of the monitoring run */
  int32_t switched;                /* 1 if every bunch met the criterion before the cap */
  int32_t pad_;
} emppp_two_stage_report;

EMPPP_API emppp_status emppp_two_stage(emppp_handle h, const double* x0, const double* u0, const double* w0,
                                       int32_t is_device_ptr, const emppp_two_stage_config* cfg,
                                       emppp_two_stage_report* rep);

/* Sets the network used by EMPPP_PROPOSAL_MLP (params host or device, EMPPP_MLP_NUM_PARAMS values). On the
 * mixed path the network runs once per step in a kernel of its own, for every (group of 512 targets in the
 * spatial order, source) pair of each bunch, at the group's mean position; the first call allocates that
 * buffer of delay factors (sum over bunches of ceil(n / 512) n floats: 33.5 MB at n = 65536; EMPPP_ERR_ARG
 * if that sum exceeds 2^31 - 1, i.e. for bunches of more than about a million particles). On the FP64
 * path each warp evaluates it for 32 sources at a time at its own targets' mean position. */
EMPPP_API emppp_status emppp_set_proposal(emppp_handle h, const float* params, int32_t is_device_ptr);

/* ---- diagnostics ------------------------------------------------------------------------------------
 * Measured throughput of the plain ALU pipes that bound the pair kernels, at the clock the GPU runs at
 * during the call: every SM runs independent dependent chains of FP32 FMAs, FP64 FMAs and FP32 reciprocal
 * square roots (the multi-function unit); each rate is the operation count of one launch over its
 * event-timed duration (best of three after a warm-up). These are the measured denominators of the
 * benchmark's roofline fractions (no counterpart in the paper). Allocates and frees one scratch buffer
 * of 8 bytes per thread of the probe grid; synchronous on cuda_stream (NULL: legacy default stream). */
typedef struct {
  double fp32_flops; /* FP32 FMA: 2 flop per FMA, per second */
  double fp64_flops; /* FP64 FMA: 2 flop per FMA, per second */
  double mufu_ops;   /* FP32 reciprocal square roots per second */
  int32_t sms;       /* streaming multiprocessors of the device */
  int32_t launches;  /* kernels launched by the call */
} emppp_peaks;

EMPPP_API emppp_status emppp_measure_peaks(emppp_peaks* out, void* cuda_stream);

/* The FP64 pair kernel's reciprocal, y[k] = 1 / x[k] for n values (device pointers; synchronous on
 * cuda_stream): the hardware's approximate reciprocal refined by two Newton-Raphson steps, which the
 * kernel uses for 1 / (eta . v') and in the root of eq:dt. Exposed so that its error can be measured
 * against the correctly rounded quotient (within 2 units in the last place for finite x > 0 with
 * 2^-1022 < x < 2^1022; no counterpart in the paper). */
EMPPP_API emppp_status emppp_reciprocal_probe(const double* x, double* y, int64_t n, void* cuda_stream);

/* Text of the last failing call on this thread ("" if none). Valid until the next call. */
EMPPP_API const char* emppp_last_error(void);

/* Library version string. */
EMPPP_API const char* emppp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EMPPP_H */
