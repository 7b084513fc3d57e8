/*
 * esp.h — C ABI of the GB300 environment-electrostatic-potential library.
 *
 * The library evaluates, at many electron positions C, the electrostatic
 * potential of a fixed QM/MM environment:
 *
 *   V(C) = sum_beta Z_beta / |C - R_beta|                       (point charges)
 *        + sum_ab w_ab * int chi_a(r) chi_b(r) / |r - C| dr     (Gaussian pairs)
 *
 * with chi(r) = (x-Ax)^i (y-Ay)^j (z-Az)^k exp(-alpha |r-A|^2) an
 * unnormalised Cartesian primitive.  This is the field of Eq.
 * ElectrostaticField (Sec. II.B of "Acceleration of a QM/MM-QMC simulation
 * using GPU"), U_ES(r_new) = sum_m rho(r_m)/|r_new - r_m| - sum_beta
 * Z_beta/|r_new - R_beta|, with U_ES = -V for an electron: the paper's
 * discretised cells rho(r_m) are point charges of value -rho (pass them as
 * point charges), and a density given in a Gaussian basis is passed as
 * weighted primitive pairs.  Units: bohr in, hartree per elementary charge out.
 *
 * The split between esp_create (environment uploaded once, read-only on the
 * device) and esp_eval (positions in, potentials out, every Monte Carlo step)
 * follows the paper's data-residency design (Sec. III: the cell data is sent
 * to the GPU once; per step only r_new goes in and U_ES comes out).
 *
 * Conventions for every entry point:
 *  - No exception crosses the ABI and nothing aborts.  A failing call returns
 *    a non-zero esp_status and leaves its outputs untouched (for device
 *    outputs: not written by any kernel of this call); esp_last_error() then
 *    holds a one-line message for the calling thread.
 *  - Pointers named "host or device" may point to host memory (pageable or
 *    pinned) or to device memory of the context's device; all arrays passed
 *    to one call must live in the same space.  With host pointers the call is
 *    synchronous.  With device pointers the work is enqueued on the context's
 *    stream and the call returns without synchronising; the caller orders
 *    later reads on that stream or calls esp_synchronize.
 *  - The library copies every input it keeps; the caller may free its arrays
 *    as soon as a call returns (device inputs: once the stream has passed the
 *    call).
 *  - One context may be used by one host thread at a time; a call that finds
 *    the context busy returns ESP_ERR_STATE.
 */
#ifndef ESP_H
#define ESP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ESP_ABI_VERSION 1
#define ESP_MAX_L 4 /* largest la + lb of one primitive pair */

/* esp_options.flags: build the tiles on the host only, touch no GPU.  Such a
 * context serves esp_get_info and esp_debug_host_eval (test hooks); every
 * evaluation call on it returns ESP_ERR_STATE. */
#define ESP_FLAG_HOST_ONLY 1

typedef struct esp_ctx esp_ctx;

typedef enum {
    ESP_OK = 0,
    ESP_ERR_INVALID = 1,     /* bad argument: null pointer, non-finite value, exponent <= 0,
                                negative or too large angular momentum, n < 0, wrong memory space */
    ESP_ERR_OOM = 2,         /* a host or device allocation failed */
    ESP_ERR_CUDA = 3,        /* a CUDA runtime call failed (message in esp_last_error) */
    ESP_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out; the context stays usable */
    ESP_ERR_STATE = 5,       /* context busy in another thread, or destroyed */
    ESP_ERR_UNSUPPORTED = 6  /* valid request the library does not handle */
} esp_status;

/* A point charge: nucleus (Z > 0) or a discretised density cell (charge -rho).
 * Sec. II.B, Eq. ElectrostaticField: {Z_beta, R_beta} and {rho(r_m), r_m}. */
typedef struct {
    double xyz[3];
    double Z;
} esp_point_charge;

/* One product of two unnormalised Cartesian primitives (96 bytes).  lmn_a and
 * lmn_b are the Cartesian exponents (i, j, k); la + lb <= ESP_MAX_L where
 * la = i+j+k of A.  The density weight of the pair is passed separately. */
typedef struct {
    double A[3];
    double alpha;
    int32_t lmn_a[3];
    int32_t pad_a;
    double B[3];
    double beta;
    int32_t lmn_b[3];
    int32_t pad_b;
} esp_gauss_pair;

typedef enum {
    ESP_FP64 = 0,  /* every step in FP64: reference-accuracy path */
    ESP_FP32C = 1  /* bulk of the pair sum in FP32 with compensated accumulation;
                      point charges and near (position, tile) blocks in FP64 */
} esp_precision;

typedef struct {
    int32_t size;                  /* sizeof(esp_options); filled by esp_default_options */
    int32_t precision;             /* esp_precision; default ESP_FP32C */
    double screen_tol;             /* drop distributions whose absolute charge bound is below
                                      this; default 1e-12; 0 keeps every pair */
    double qm_center[3];           /* positions and centres are recentred here in FP64 */
    void *cuda_stream;             /* cudaStream_t for all work; NULL = the default stream */
    int32_t device;                /* CUDA device ordinal; -1 = the current device */
    int32_t tile_size;             /* distributions per tile: 32, 64, 128 or 256; 0 = 64 */
    int32_t threads_per_block;     /* 0 = tuned default; else 64, 128 or 256 */
    int32_t positions_per_thread;  /* 0 = tuned default; FP32C shapes built: 64x{2,4},
                                      128x{1,2,4}, 256x{1,2}; FP64 uses min(this, 2) */
    int32_t pair_splits;           /* tiles are dealt round-robin to this many splits per
                                      position block; 0 = chosen from the problem size */
    int32_t flags;                 /* ESP_FLAG_* bits; 0 for normal use */
    double near_radius;            /* FP32C: a (position, tile) block whose distance to the
                                      tile's bounding sphere is below this is evaluated in
                                      FP64, for tiles holding a distribution whose potential
                                      can exceed 2 Ha (a compact charge not merged into a
                                      point charge); < 0 = default (1.5 bohr), 0 = off */
    double point32_max_charge;     /* FP32C: point charges with |Z| at or below this (the paper's
                                      density cells) are summed in compensated FP32 like the
                                      distributions, larger ones (nuclei, merged monopoles) in
                                      FP64; < 0 = default (0.25), 0 = every point charge FP64 */
} esp_options;

/* Per-context facts, for reporting and for counting evaluations. */
typedef struct {
    int64_t n_point_charges;       /* point charges kept */
    int64_t n_pairs_in;            /* primitive pairs passed to esp_create */
    int64_t n_distributions;       /* Hermite distributions after folding and screening */
    int64_t n_screened;            /* distributions dropped by screen_tol */
    int64_t n_by_L[ESP_MAX_L + 1]; /* distributions per total angular momentum L */
    int64_t n_tiles;               /* tiles of distributions and of point charges */
    int64_t n_near_tiles;          /* tiles whose distributions may take the FP64 near path */
    int64_t device_bytes;          /* device memory held by the context */
    int32_t precision;
    int32_t tile_size;
    int32_t threads_per_block;
    int32_t positions_per_thread;
    int32_t pair_splits;
    int32_t device;
} esp_info;

/* Fill *opt with defaults (FP32C, screen 1e-12, centre origin, default stream,
 * current device, tuned launch shape). */
void esp_default_options(esp_options *opt);

/* Build a context: validate, fold pairs that share (A, alpha, B, beta) into one
 * Hermite distribution (McMurchie-Davidson expansion), screen, sort into tiles
 * and upload once (Sec. III, data residency).
 *   charges [n_charges]   host; may be NULL when n_charges == 0
 *   pairs   [n_pairs]     host; may be NULL when n_pairs == 0
 *   weights [n_pairs]     host; density weight w_ab of each pair
 *   opt                   NULL = defaults
 *   out                   receives the context; untouched on error
 * Errors: ESP_ERR_INVALID (bad input), ESP_ERR_OOM, ESP_ERR_CUDA. */
esp_status esp_create(const esp_point_charge *charges, int64_t n_charges,
                      const esp_gauss_pair *pairs, const double *weights, int64_t n_pairs,
                      const esp_options *opt, esp_ctx **out);

/* V[i] = potential at positions[i] (Eq. ElectrostaticField with U_ES = -V).
 *   positions [n][3] host or device, float64, row-major
 *   V_out     [n]    same space as positions, float64
 * Calls with at most 16 positions (the paper's one r_new per Metropolis move,
 * Sec. III) spread the environment's entries over the GPU's threads instead
 * of the positions and evaluate in FP64 whatever the precision setting.
 * n == 0 is a no-op.  Errors: ESP_ERR_INVALID, ESP_ERR_STATE, ESP_ERR_CUDA,
 * ESP_ERR_TIMEOUT, ESP_ERR_OOM. */
esp_status esp_eval(esp_ctx *ctx, const double *positions, int64_t n, double *V_out);

/* Walker-major positions [n_walkers][n_elec][3]; E_out[w] = sum_e U_ES(r_we) =
 * -sum_e V(r_we), reduced in FP64 on the device in a fixed order.  V_out may
 * be NULL.  Same memory-space rules as esp_eval. */
esp_status esp_eval_walkers(esp_ctx *ctx, const double *positions, int64_t n_walkers,
                            int64_t n_elec, double *V_out, double *E_out);

/* Largest n accepted by esp_eval_noalloc. */
#define ESP_NOALLOC_MAX_POSITIONS 65536

/* esp_eval without any device allocation (the paper has no counterpart; this
 * entry point exists for callers of this library that cannot call cudaMalloc:
 * code whose device memory is owned by another allocator, such as a
 * framework's caching allocator that already holds the GPU, and Monte Carlo
 * loops that must not pay cudaMalloc's implicit device-wide synchronisation).
 * The context must have been created beforehand by esp_create.
 *   positions [n][3] device memory of the context's device, float64
 *   V_out     [n]    device memory of the context's device, float64
 * Work is enqueued on the context's stream; the call returns without waiting.
 * The scratch (staged positions and per-split partial sums) lives in one
 * file-scope device array of fixed size inside the library, about 7 MiB for
 * ESP_NOALLOC_MAX_POSITIONS positions, which every GPU that loads the library
 * holds until the process exits.  Under CUDA's lazy module loading (the
 * default) the library's device module, and with it this array, is loaded on
 * a device by the first launch or symbol lookup there: the first call on each
 * device may therefore allocate device memory and synchronise; later calls do
 * not.  Every call looks up the array's device address (cudaGetSymbolAddress)
 * with the context's device current; make the first call on a device before
 * any stream capture.  All calls share the array and
 * it keeps the last call's contents: calls that overlap on the GPU (other
 * streams, other contexts, other threads) race on it, so order them on one
 * stream or synchronise between them.  The result equals esp_eval's within
 * FP32C rounding (the per-split partial count is capped at 8 here, and the
 * positions are neither spatially ordered nor routed to the few-position
 * path, which both need more scratch).
 * Errors: ESP_ERR_INVALID (n > ESP_NOALLOC_MAX_POSITIONS, host pointers, null
 * pointers), ESP_ERR_STATE, ESP_ERR_CUDA.  Calls no cudaMalloc or cudaFree. */
esp_status esp_eval_noalloc(esp_ctx *ctx, const double *positions, int64_t n, double *V_out);

/* ------------------------------------------------------------------------
 * The paper's call pattern as a replayed CUDA graph.  The paper evaluates one
 * electron position per call, once per Metropolis move (Sec. III,
 * Fig. codeStructure: r_new in, U_ES out).  esp_graph_create captures the
 * few-position evaluation of a fixed device position buffer into a fixed
 * device output once; each esp_graph_launch replays it on the context's
 * stream, so the caller writes the next positions into the same buffer (on
 * that stream, or before the launch) and reads V after it.  The precision is
 * the context's at creation (ESP_FP32C: small point charges in compensated
 * FP32, everything else FP64; ESP_FP64: all FP64).
 * ------------------------------------------------------------------------ */
#define ESP_GRAPH_MAX_POSITIONS 128
typedef struct esp_graph esp_graph;

/* positions [n][3] and V_out [n] float64, device memory of the context's
 * device, 1 <= n <= ESP_GRAPH_MAX_POSITIONS; both must stay allocated while
 * the graph exists, and the context must outlive the graph.  The graph owns
 * its scratch (partial sums).  Errors: ESP_ERR_INVALID, ESP_ERR_STATE,
 * ESP_ERR_UNSUPPORTED (empty environment), ESP_ERR_OOM, ESP_ERR_CUDA. */
esp_status esp_graph_create(esp_ctx *ctx, const double *positions, int64_t n, double *V_out, esp_graph **out);

/* V_out = potentials at the buffer's current positions; enqueued on the
 * context's stream, returns without waiting.  Errors: ESP_ERR_STATE,
 * ESP_ERR_CUDA. */
esp_status esp_graph_launch(esp_graph *g);

/* Waits for the context's stream and frees the graph.  NULL is a no-op. */
void esp_graph_destroy(esp_graph *g);

/* ------------------------------------------------------------------------
 * Several clients sharing one GPU context.  The paper runs one process per
 * core with a GPU each and proposes sharing one GPU among several processes
 * with OpenMP threads on the host (Introduction, Discussions).  A server owns
 * a context and one worker thread; any number of host threads submit their
 * positions and get a ticket; the worker takes every request queued when it
 * wakes, evaluates them together in one esp_eval (so small requests fill the
 * GPU together) and scatters the potentials back.  A client that does host
 * work between submit and wait overlaps it with the evaluation.
 * ------------------------------------------------------------------------ */
typedef struct esp_server esp_server;

/* Start a server on ctx with pinned staging for max_positions positions per
 * batch.  While the server exists its worker thread uses ctx: other calls on
 * ctx return ESP_ERR_STATE when they meet it busy.  Errors: ESP_ERR_INVALID,
 * ESP_ERR_STATE (host-only or invalid context), ESP_ERR_OOM, ESP_ERR_CUDA. */
esp_status esp_server_create(esp_ctx *ctx, int64_t max_positions, esp_server **out);

/* Queue positions [n][3] (host memory, 1 <= n <= max_positions) whose
 * potentials go to V_out [n] (host); both must stay valid until the wait for
 * the returned ticket returns.  Thread-safe, does not block on the GPU. */
esp_status esp_server_submit(esp_server *s, const double *positions, int64_t n, double *V_out, int64_t *ticket);

/* Block until the ticket's potentials are in its V_out.  Thread-safe.
 * Returns the batch's error if its evaluation failed. */
esp_status esp_server_wait(esp_server *s, int64_t ticket);

/* Batches evaluated and positions served so far (either pointer may be NULL). */
esp_status esp_server_stats(esp_server *s, int64_t *batches, int64_t *positions);

/* Finish the queued requests, stop the worker and free the server (not its
 * context).  NULL is a no-op. */
void esp_server_destroy(esp_server *s);

/* ------------------------------------------------------------------------
 * Batched evaluation of many independent systems (environment, positions).
 * An FMO calculation has many fragments and fragment pairs (Eq. FMO), each
 * with its own environment field, and QMC runs many walkers: the batch
 * evaluates all systems together with one persistent potential kernel that
 * takes (system, position block, pair split) work items, largest first, and
 * replays one captured CUDA graph per call.
 * ------------------------------------------------------------------------ */
typedef struct esp_batch esp_batch;

typedef struct {
    int32_t threads_per_block;    /* chosen launch shape */
    int32_t positions_per_thread;
    double split_scale;           /* chosen multiplier of the per-system split count */
    double best_ms;               /* time of one batched evaluation with that choice */
    int32_t n_tried;              /* candidates timed (<= 16) */
    int32_t tried_threads[16];
    int32_t tried_ppt[16];
    double tried_scale[16];
    double tried_ms[16];
} esp_tune_report;

/* Batch of n_sys existing contexts (kept by pointer: they must outlive the
 * batch).  All contexts must be on one device and use one precision.  Work
 * runs on cuda_stream (NULL = default stream).  Errors: ESP_ERR_INVALID,
 * ESP_ERR_STATE (host-only or invalid context), ESP_ERR_OOM, ESP_ERR_CUDA. */
esp_status esp_batch_create(esp_ctx *const *ctxs, int32_t n_sys, void *cuda_stream, esp_batch **out);

/* V_out[s][i] = potential of system s at positions[s][i].
 *   positions [n_sys] host array of device pointers, each [n[s]][3] float64
 *   n         [n_sys] host array of counts (0 allowed)
 *   V_out     [n_sys] host array of device pointers, each [n[s]] float64
 * Enqueued on the batch's stream; returns without waiting.  Scratch grows on
 * demand.  Errors: ESP_ERR_INVALID (host memory, bad counts), ESP_ERR_STATE,
 * ESP_ERR_OOM, ESP_ERR_CUDA. */
esp_status esp_batch_eval(esp_batch *b, const double *const *positions, const int64_t *n, double *const *V_out);

/* Time every built launch shape with split multipliers 0.5, 1 and 2 on the
 * given inputs (outputs are overwritten), keep the fastest and report all. */
esp_status esp_batch_autotune(esp_batch *b, const double *const *positions, const int64_t *n, double *const *V_out,
                              esp_tune_report *report);

/* Set the launch shape (FP32C: 128x4, 128x2, 256x2, 64x4; FP64: 128x2, 128x1,
 * 256x1) and split multiplier directly. */
esp_status esp_batch_set_shape(esp_batch *b, int32_t threads, int32_t ppt, double split_scale);

/* Wait for the last batched evaluation and return its device time (ms). */
esp_status esp_batch_last_ms(esp_batch *b, double *ms);

/* Free the batch (not its contexts).  NULL is a no-op. */
void esp_batch_destroy(esp_batch *b);

/* ------------------------------------------------------------------------
 * Learned surrogate of V over the QM region (the QM sphere of radius
 * qm_radius about the context's qm_center).  The environment is split once:
 * near tiles (any part closer to the centre than far_radius, or Gaussians
 * reaching into the sphere) are summed exactly on every call by the FP32C
 * kernel; the far tiles' potential, harmonic inside the sphere, is replaced by
 * its FP64 interior solid-harmonic expansion of degree `degree` (coefficients
 * projected from the exact far field on the sphere) plus a BF16 tensor-core
 * MLP on the remaining residual (64 Fourier features, 4 x 256 SiLU, scalar
 * out), trained by the library's own forward/backward kernels and Adam on
 * labels of the exact kernel over the far tiles.  The exact sum over all
 * tiles stays the fallback: positions in voxels whose validation error
 * exceeded tol/2, near point charges, or picked by the online probe are
 * evaluated exactly; a probe that misses tol withdraws its voxel, and the
 * call's other positions in that voxel are evaluated exactly before it
 * returns.  The paper has no surrogate; the exact sum it accelerates decides
 * the surrogate's error.
 * ------------------------------------------------------------------------ */
typedef struct esp_surrogate esp_surrogate;

typedef struct {
    int32_t size;              /* sizeof(esp_surrogate_cfg), set by esp_surrogate_default_cfg */
    int32_t n_train;           /* training positions (2^19) */
    int32_t n_valid;           /* validation positions for the trust map (2^17), plus one in every voxel */
    int32_t epochs;            /* passes over the training set (8) */
    int32_t batch;             /* mini-batch (8192) */
    int32_t degree;            /* degree L of the far field's interior expansion (12; <= 40) */
    double qm_radius;          /* radius of the QM sphere, bohr (6) */
    double position_sd;        /* sd of the walker law for half the samples (2) */
    double fourier_sigma;      /* sd of the Fourier frequencies, per unit radius (1) */
    double lr;                 /* Adam learning rate, cosine-decayed (1e-3) */
    double tol;                /* accepted error, Ha (2e-6): trust voxels at tol/2, probes at tol */
    double voxel;              /* trust-map voxel edge, bohr (0.25) */
    double nucleus_exclusion;  /* positions this close to a point charge fall back, bohr (0.5) */
    int32_t probe_stride;      /* every probe_stride-th position is also evaluated exactly (64; 0 off) */
    int32_t label_precision;   /* exact kernel of the training and validation labels (ESP_FP32C; or ESP_FP64) */
    uint64_t seed;             /* positions, frequencies and initial weights (1011) */
    double far_radius;         /* tiles wholly beyond this distance from the centre form the far field,
                                  bohr (10; >= qm_radius) */
    double far_penetration;    /* ... and only if p_min (d - qm_radius)^2 >= this for every Gaussian of
                                  the tile (d: distance of the tile's bounding sphere from the centre):
                                  30 keeps the non-harmonic tail inside the sphere below e^-30 of the
                                  charge; smaller values move more diffuse tiles to the far field, whose
                                  tails the network then has to absorb (30; >= 4) */
} esp_surrogate_cfg;

typedef struct {
    int64_t n_fallback;        /* positions of the last call evaluated exactly */
    int64_t n_probe_fail;      /* probes that missed tol (last call; total in esp_surrogate_info) */
    double surrogate_ms;       /* near sum + expansion + network time of the last call */
    double total_ms;           /* the whole last call, fallback included */
    double train_loss;         /* final training loss (normalised residual) */
    double valid_max_err;      /* largest validation error of expansion + network on the far field, Ha */
    double trusted_fraction;   /* share of visited voxels trusted */
    int64_t n_params;          /* network parameters */
    int64_t n_baseline;        /* expansion coefficients, (degree + 1)^2 */
    double valid_rms_err;      /* rms validation error of expansion + network, Ha */
    double baseline_max_err;   /* the same two errors of the expansion alone (without the network) */
    double baseline_rms_err;
    int64_t n_near_entries;    /* distributions + point charges summed exactly on every call */
    int64_t n_far_entries;     /* distributions + point charges replaced by expansion + network */
    double baseline_trusted_fraction; /* share of voxels the expansion alone (no network) would earn */
} esp_surrogate_stats;

void esp_surrogate_default_cfg(esp_surrogate_cfg *cfg);

/* Train a surrogate of ctx's potential (ctx stays in use for labels and
 * fallback; it must outlive the surrogate).  Synchronous.  Errors:
 * ESP_ERR_INVALID, ESP_ERR_STATE, ESP_ERR_UNSUPPORTED, ESP_ERR_OOM, ESP_ERR_CUDA. */
esp_status esp_surrogate_train(esp_ctx *ctx, const esp_surrogate_cfg *cfg, esp_surrogate **out);

/* V_out[i] for device positions [n][3]: surrogate where trusted, exact
 * elsewhere (see above).  Synchronous (one device->host read of the fallback
 * count).  stats may be NULL. */
esp_status esp_surrogate_eval(esp_surrogate *s, const double *positions, int64_t n, double *V_out,
                              esp_surrogate_stats *stats);

/* Baseline + network only (no fallback), device pointers; synchronous. */
esp_status esp_surrogate_predict(esp_surrogate *s, const double *positions, int64_t n, double *V_out);

esp_status esp_surrogate_info(const esp_surrogate *s, esp_surrogate_stats *stats);

/* Versioned binary file with a checksum: configuration, baseline, frequencies,
 * weights and trust map.  Loading binds the surrogate to ctx. */
esp_status esp_surrogate_save(const esp_surrogate *s, const char *path);
esp_status esp_surrogate_load(esp_ctx *ctx, const char *path, esp_surrogate **out);

/* Test hooks: one forward + backward pass on a host batch (positions [n][3],
 * normalised targets [n]) without updating; copies out the FP32 parameters,
 * the gradient of mean((y - t)^2) (flat layout W1 b1 W2 b2 W3 b3 W4 b4 w5 b5)
 * and the outputs y; and the Fourier frequencies [32][3] with
 * (centre x, y, z, 1/R). */
esp_status esp_surrogate_debug_step(esp_surrogate *s, const double *positions, const float *targets, int32_t n,
                                    float *params_out, float *grad_out, float *y_out);
esp_status esp_surrogate_features(const esp_surrogate *s, float *freq_out, double *centre_inv_r_out);
/* Test hook: add dc to the constant coefficient c_00 of the far-field
 * expansion (dc = 0: no change), then copy the first max_coef coefficients to
 * coef_out (esp_harmonics order).  Adding an offset plants a known error in
 * every surrogate value, which the probe must catch. */
esp_status esp_surrogate_debug_expansion(esp_surrogate *s, double dc, double *coef_out, int32_t max_coef);
/* Iterations of each bounded wait (mbarrier) of the network's tensor-core
 * kernels (fused inference and the training GEMMs) before it gives up: the
 * kernel then records an error, waits (with the default limit) for its own
 * copies and MMAs in flight, frees its tensor memory and returns, and the call
 * returns ESP_ERR_TIMEOUT with the context still usable.  limit < 0 restores the default (about one second); 0 makes
 * every first wait give up at once (used by the tests of that error path). */
esp_status esp_surrogate_set_wait_limit(esp_surrogate *s, int32_t limit);
/* Test hook: the network outputs y [n] (FP32 normalised residual, before the
 * baseline and scale are applied) of the fused tensor-core inference kernel
 * (tcgen05) at host positions [n][3], n <= 65536.  ESP_ERR_TIMEOUT if one of
 * the kernel's bounded waits gave up. */
esp_status esp_surrogate_debug_net(esp_surrogate *s, const double *positions, int32_t n, float *y_out);

void esp_surrogate_destroy(esp_surrogate *s);

/* Switch the arithmetic of later evaluations (ESP_FP64 or ESP_FP32C). */
esp_status esp_set_precision(esp_ctx *ctx, int32_t precision);

/* Fill *info.  Errors: ESP_ERR_INVALID. */
esp_status esp_get_info(const esp_ctx *ctx, esp_info *info);

/* Kernel timing.  With enable != 0, each later evaluation records CUDA events
 * on the context's stream around its potential kernel (the Eq.
 * ElectrostaticField sum) and around the whole device pipeline (staging,
 * potential, reductions).  esp_last_timing waits for the last evaluation and
 * returns both durations in milliseconds.  Errors: ESP_ERR_STATE when timing
 * is off or nothing was evaluated since it was enabled. */
esp_status esp_set_timing(esp_ctx *ctx, int32_t enable);
esp_status esp_last_timing(esp_ctx *ctx, double *potential_ms, double *pipeline_ms);

/* Wait for the context's stream. */
esp_status esp_synchronize(esp_ctx *ctx);

/* Free every resource of ctx.  NULL is a no-op. */
void esp_destroy(esp_ctx *ctx);

/* Static English name of a status code. */
const char *esp_status_string(esp_status s);

/* Message of the last failing call in this host thread ("" if none). */
const char *esp_last_error(void);

/* ABI version of the loaded library (ESP_ABI_VERSION). */
int32_t esp_abi_version(void);

/* Test hook, not part of the evaluation path: evaluate the Boys function
 * F_0..F_nmax(T) with the device algorithm of the given precision, run on the
 * host (nmax <= ESP_MAX_L).  Lets CPU tests check the tables and the Taylor
 * and asymptotic branches without a GPU. */
esp_status esp_debug_boys(int32_t precision, int32_t nmax, double T, double *F_out);

/* Test hook: 1 if the host-side fault injection names `what` ("alloc",
 * "upload" or "graph").  The environment variable ESP_FAULT (comma-separated
 * names, read on every use) makes the named operations fail as if their CUDA
 * call had failed: "alloc" every device allocation of the library (the call
 * returns ESP_ERR_OOM), "upload" the environment upload of esp_create
 * (ESP_ERR_CUDA), "graph" the instantiation of the batched driver's CUDA graph
 * (ESP_ERR_CUDA).  Clearing the variable lets the next call succeed; no GPU
 * fault is involved. */
int32_t esp_debug_fault_active(const char *what);

/* Test hook, not part of the evaluation path: the real regular solid
 * harmonics S_k(u), k < (L + 1)^2 (L <= 40), that the surrogate's far-field
 * expansion uses, evaluated on the host by the device code's recursion, at
 * the point u[3]; out gets (L + 1)^2 values in the order (l, 0), (l, 1, cos),
 * (l, 1, sin), ... for l = 0..L.  They are |u|^l times the real spherical
 * harmonics normalised to 4 pi over the unit sphere. */
esp_status esp_debug_solid_harmonics(int32_t L, const double *u, double *out);

/* Test hook, not part of the evaluation path: evaluate a built context's
 * tiles on the host with the kernels' own per-tile code, in the context's
 * precision (ESP_FP64: FP64; ESP_FP32C: the FP32-compensated arithmetic of
 * the kernel, emulated in IEEE single precision), so CPU tests can check the
 * pair builder and the error budget of the FP32 path without a GPU.
 * positions and V_out are host arrays.  esp_eval never calls this. */
esp_status esp_debug_host_eval(const esp_ctx *ctx, const double *positions, int64_t n,
                               double *V_out);

/* Largest sample accepted by esp_work_census. */
#define ESP_CENSUS_MAX_POSITIONS 4000

/* Work census of an evaluation at the host positions [n][3] (n <=
 * ESP_CENSUS_MAX_POSITIONS): every (distribution, position) term of the
 * context's environment, counted by the regime of its Boys argument
 * T = p |P - C|^2 (Sec. II.B, Eq. ElectrostaticField generalised to Hermite
 * Gaussian distributions; the regime decides which form of F_n(T) a term
 * needs and so its operation count).  counts (int64, 32 entries):
 *   counts[(L + 5 s) * 3 + b]  L = 0..4 total angular momentum, s = 1 for
 *                              distributions whose monopole sits in a point
 *                              charge (short-range remainder), b = 0: T < 30,
 *                              1: 30 <= T < 45, 2: T >= 45;
 *   counts[30]                 point-charge terms summed in FP64;
 *   counts[31]                 point-charge terms summed in FP32 (small charges).
 * Synchronous; allocates and frees a small device buffer.  Errors:
 * ESP_ERR_INVALID, ESP_ERR_STATE, ESP_ERR_CUDA, ESP_ERR_OOM. */
esp_status esp_work_census(esp_ctx *ctx, const double *positions, int64_t n, int64_t *counts);

/* ------------------------------------------------------------------------
 * The paper's coalescing study (Results: Eq. coalease vs Eq. incoalease,
 * Table Single Core performances; 6.0x kernel-only gain on its GPU), re-run
 * on this GPU as a measurement, not an evaluation path: the potential of the
 * context's point charges (cells and nuclei) at one position, by the paper's
 * kernel structure (blocks of 256 threads, n_loop iterations per thread,
 * shared-memory block sum) with the coalesced mapping (cell = l N_B N_th +
 * b N_th + j) or the incoalesced one (cell = (b N_th + j) n_loop + l), in FP64
 * or FP32 arithmetic (FP64 sums), over the point records as stored (32-byte
 * [x, y, z, Z]) or over separate x, y, z, Z arrays (soa_layout = 1).
 * ------------------------------------------------------------------------ */
/*   position   host [3] (bohr);  incoalesced: 0 or 1;  fp64: 0 (FP32) or 1;
 *   soa_layout 0: the 32-byte records; 1: separate arrays (FP64 or FP32 words);
 *   n_loop     iterations per thread (the paper used 9);  reps: timed launches;
 *   V_out      host: the sum;  ms_out (nullable): mean time of one launch pair
 *              (the block kernel and the final sum), CUDA events on the stream.
 * Synchronous.  Errors: ESP_ERR_INVALID, ESP_ERR_STATE, ESP_ERR_UNSUPPORTED (no
 * point charges), ESP_ERR_OOM, ESP_ERR_CUDA. */
esp_status esp_study_cell_sum(esp_ctx *ctx, const double *position, int32_t incoalesced, int32_t fp64,
                              int32_t soa_layout, int32_t n_loop, int32_t reps, double *V_out, double *ms_out);

/* ------------------------------------------------------------------------
 * Measured pipe peaks of the GPU: the denominators of the potential kernels'
 * rooflines.  The paper estimates its hardware's peaks from unit counts and
 * clocks (Sec. IV, Table performances) and sets its kernel against them; this
 * call measures them instead.  Each rate is instructions per second summed
 * over all lanes ("lane ops"; an FMA counts once), from kernels of independent
 * dependency chains on every SM (8 CTAs of 256 threads per SM), timed with
 * CUDA events on the default stream after one warm-up launch.
 * ------------------------------------------------------------------------ */
typedef struct {
    double fp32_fma_per_s;    /* FFMA lane ops / s */
    double fp32x2_fma_per_s;  /* FP32 FMA lane ops / s issued as packed pairs (FFMA2, two per instruction) */
    double fp64_fma_per_s;    /* DFMA lane ops / s */
    double mufu_rsqrt_per_s;  /* MUFU reciprocal square root, lane ops / s */
    double mufu_ex2_per_s;    /* MUFU base-2 exponential, lane ops / s */
    double fp32_ms, fp32x2_ms, fp64_ms, rsqrt_ms, ex2_ms; /* duration of one timed launch */
    int32_t num_sms;          /* cudaDevAttrMultiProcessorCount of the device */
    int32_t clock_khz;        /* cudaDevAttrClockRate (the rated, not the live clock) */
} esp_peaks;

/* Measure the peaks on `device` (< 0: the current device).  Synchronous; takes
 * tens of milliseconds; allocates (and frees) a few KB of device memory.
 * Errors: ESP_ERR_INVALID (out NULL), ESP_ERR_CUDA, ESP_ERR_OOM. */
esp_status esp_measure_peaks(int32_t device, esp_peaks *out);

#ifdef __cplusplus
}
#endif

#endif /* ESP_H */
