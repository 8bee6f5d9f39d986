/*
 * libreg -- GB300 (sm_103a) registration prefix scan for long electron
 * micrograph series.
 *
 * The method is the one of "Parallel Prefix Algorithms for the Registration of
 * Arbitrarily Long Electron Micrograph Series" (arXiv 1712.02533):
 *   - function A (Algorithm "Multilevel gradient flow for image registration"):
 *     register frame f_k to frame f_i by a multilevel L2 gradient flow on
 *     E[phi] = -NCC[f_i, f_k o phi] + lambda/2 int |D(phi - id)|^2
 *     (Section "Image registration for electron microscopy"), forward Euler
 *     steps with the Armijo rule with widening (Section "Gradient flow");
 *   - function B(phi_ij, phi_jk) = A(f_i, f_k, phi_jk o phi_ij) (Section
 *     "Registration for series of images");
 *   - image series registration (Definition "Image series registration"):
 *     preprocessing x_e = A(f_e, f_{e+1}, I), then the inclusive prefix scan
 *     phi_{0,e+1} = x_0 (.)_B ... (.)_B x_e (Section "Prefix sum for
 *     registration problem") with one of the paper's scan schedules.
 * All independent operator applications of one scan level run in one batched
 * device loop; every arithmetic step runs in this library's CUDA kernels.
 *
 * Units and layout.  A frame is side x side pixels, side = 2^L (32 <= side <=
 * 4096), row-major, row = x_1, column = x_0.  Level l of the pyramid is the
 * vertex grid of (2^l + 1)^2 nodes on Omega = [0,1]^2; the frame is embedded
 * on level L by repeating its last row and column.  Deformations are returned
 * as displacements u(x) = phi(x) - x in pixels, channel 0 along columns (x_0),
 * channel 1 along rows (x_1), with f_k(x + u(x)) ~ f_0(x).
 *
 * Errors.  Every call returns a reg_status; no C++ exception crosses the ABI.
 * A handle is not thread-safe: calls on one handle must be serialised by the
 * caller.  Work is enqueued on the stream given at creation; every call is
 * synchronous on return unless stated otherwise.
 */
#ifndef REG_H
#define REG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct reg_series *reg_series_t;

typedef enum reg_status {
    REG_OK = 0,
    REG_EINVAL = 1,   /* bad argument: size, index, chain mismatch, null pointer */
    REG_ENOMEM = 2,   /* device or host allocation failed */
    REG_ECUDA = 3,    /* a CUDA runtime call failed (message in reg_last_error) */
    REG_ESTATE = 4,   /* call not valid in the handle's current state */
    REG_ETIMEOUT = 5, /* a bounded device loop gave up (step budget exhausted) */
    REG_EKERNEL = 6   /* a kernel reported an internal error */
} reg_status;

/* Per-operator outcome (not a call error). */
typedef enum reg_op_status {
    REG_OP_CONVERGED = 0,     /* energy decrease below epsilon * max(1, |E|) */
    REG_OP_MAXITER = 1,       /* iter_max gradient steps on the finest level */
    REG_OP_LS_STALLED = 2,    /* Armijo search found no step >= tau_min */
    REG_OP_NONFINITE = 3,     /* an energy or slope was not finite on some level */
    REG_OP_ZERO_GRADIENT = 4  /* the slope g^T d was exactly zero */
} reg_op_status;

typedef enum reg_storage { REG_STORAGE_F32 = 0, REG_STORAGE_BF16 = 1 } reg_storage;

/* Optional device allocator (e.g. a framework's caching allocator).  When
 * alloc is NULL the library uses cudaMallocAsync/cudaFreeAsync on its stream. */
typedef struct reg_allocator {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, size_t bytes, void *stream, void *ctx);
    void *ctx;
} reg_allocator;

/* Method parameters.  n_levels: pyramid depth m1 - m0 + 1 with m1 = L
 * (Algorithm "Multilevel gradient flow"); iter_max and epsilon: stopping
 * criteria per level; lambda: regulariser weight; armijo_sigma, tau_*: step
 * rule (Section "Gradient flow").  trials_per_pass (1..8): how many step
 * sizes of the Armijo sequence one energy pass evaluates at once (does not
 * change the accepted step).  storage: pyramid storage precision.
 * init_levels: pyramid levels (the finest ones) that a preprocessing operator
 * runs when it starts from a learned initial displacement
 * (reg_cnn_init_series); 0 means n_levels.  The coarse levels exist to bring
 * a far start into the basin of the fine ones; a start that is already there
 * can skip them.  learned_fallback_px: the plain method judges a learned
 * start that skips levels by how far it moves it (mean |u_final - u_start|
 * over the finest nodes, x + y, px); an operator that moves it further is run
 * again from the identity on every level (reg_prefix_scan reports the count). */
typedef struct reg_params {
    int32_t n_levels;
    int32_t iter_max;
    double epsilon;
    double lambda;
    double armijo_sigma;
    double tau_init;
    double tau_max;
    double tau_min;
    int32_t storage;
    int32_t trials_per_pass;
    int32_t max_steps;        /* device step budget per batch; <= 0: automatic */
    int32_t flags;            /* REG_FLAG_* */
    int32_t init_levels;      /* 0 or 1..n_levels, see above */
    double learned_fallback_px; /* see above; 0: never fall back */
    reg_allocator allocator;
    double smooth;            /* H1-type smoother width s in grid spacings of each level; 0: lumped L2 flow */
} reg_params;

#define REG_FLAG_PROFILE 1    /* time kernel families with CUDA events */
/* Rigid variant (Definition "Rigid transformation": phi(x) = R(alpha) x + t,
 * rotation about the origin of Omega, t in Omega units).  A handle created
 * with this flag registers with the three-parameter operator: function A runs
 * gradient descent on theta = (alpha, t0, t1) (no smoother, Section "Gradient
 * flow") with the same Armijo rule on every pyramid level, carrying theta from
 * level to level unchanged (a rigid deformation is not restricted or
 * prolongated, Algorithm "Multilevel gradient flow"); the energy is E at
 * phi, whose regulariser is 2 lambda (1 - cos alpha) for a rigid map; function
 * B starts from the composition of the two rigid maps.  Slots hold the
 * parameters (reg_get_rigid / reg_set_rigid) and the field they define, so
 * reg_get_slot, reg_get_deformations and reg_average_series work unchanged.
 * The operator's iterations are driven from the host: each round launches one
 * evaluation over all active operators of the batch. */
#define REG_FLAG_RIGID 2

/* Replace the handle's reg_params.flags (REG_FLAG_*); takes effect at the next
 * batch.  With REG_FLAG_PROFILE the step kernels are launched one by one
 * between CUDA events instead of as the captured graph. */
reg_status reg_set_flags(reg_series_t s, int32_t flags);

/* The smoother A of the gradient flow d = -A^{-1} E'[phi] (Section "Gradient
 * flow": A is selected to smooth in the non-rigid registration).  smooth = 0:
 * A = diag(w), the lumped mass (an L2 flow; the default).  smooth = s > 0: A is
 * the tensor-product H1 Gram matrix M_s (x) M_s with M_s = M1 + (s h)^2 / 2 K1
 * (M1, K1 the 1D P1 mass and stiffness, h the level's grid spacing), whose
 * inverse is a tridiagonal solve along every row and then every column; two
 * more kernels per gradient step.  The diagnostic calls reg_eval_direction and
 * reg_eval_trials keep the lumped direction. */

/* Fills *p with the defaults: n_levels 3, iter_max 50, epsilon 1e-7,
 * lambda 10, sigma 0.5, tau_init 1, tau_max 1e4, tau_min 1e-12, F32 storage,
 * 4 trials per pass, init_levels 0, learned_fallback_px 2, smooth 0. */
void reg_default_params(reg_params *p);

/* One operator application (Section "Registration for series of images").
 * Registers frame_k (template) to frame_i (reference) of series `series`:
 *   left >= 0, right >= 0 : B = A(f_i, f_k, right o left)  (slots' fields)
 *   left >= 0, right <  0 : A(f_i, f_k, left)
 *   left <  0, right <  0 : A(f_i, f_k, I)
 * The result is written to slot dst of the same series.  All ops of one call
 * read their slots before any op writes (level-synchronous semantics). */
typedef struct reg_op_desc {
    int32_t series;
    int32_t left_slot;
    int32_t right_slot;
    int32_t dst_slot;
    int32_t frame_i;
    int32_t frame_k;
} reg_op_desc;

typedef enum reg_scan_kind {
    REG_SCAN_SERIAL = 0,      /* Algorithm "serial prefix sum" */
    REG_SCAN_SKLANSKY = 1,    /* Algorithm "Sklansky" (Ladner-Fischer) */
    REG_SCAN_KOGGE_STONE = 2, /* Algorithm "Kogge-Stone" (double-buffered) */
    REG_SCAN_BRENT_KUNG = 3,  /* Algorithm "Brent-Kung" */
    REG_SCAN_BLELLOCH = 4,    /* Algorithm "Blelloch" (exclusive, shifted) */
    REG_SCAN_CHUNKED = 5,     /* general strategy, Algorithm "Distributed parallel prefix sum" */
    REG_SCAN_CHUNKED_ALT = 6, /* alternative strategy (reduce-then-scan) */
    REG_SCAN_HAN_CARLSON = 7, /* Section "Other work": Brent-Kung/Kogge-Stone hybrid,
                                 parameter k (passed as `chunks`, k >= 1) */
    REG_SCAN_LADNER_FISCHER = 8 /* Section "Other work": Brent-Kung/Sklansky hybrid,
                                   parameter k (passed as `chunks`, k >= 0; 0 is Sklansky) */
} reg_scan_kind;

/* Create a handle holding `n_series` series (one segmented scan).
 * frames: the frames of all series back to back as rows of pitch_elems
 *   (>= max side) float32 elements: series s holds frames_per_series[s]
 *   frames of side_px[s] rows each (side_px[s] pixels used per row), so
 *   series s starts at row sum_{j<s} frames_per_series[j] * side_px[j].
 *   Host memory unless frames_on_device != 0 (then a device pointer; it is
 *   only read).
 * The library copies the frames, builds each frame's pyramid (restriction
 * with the 1/16 [1 2 1; 2 4 2; 1 2 1] stencil, Section "Multilevel") and
 * keeps it until reg_destroy_series.  cuda_stream: a cudaStream_t (NULL =
 * legacy default stream).  Errors: REG_EINVAL for a side that is not a power
 * of two in [32, 4096], fewer than 2 frames, or n_levels outside [1, L-3]. */
reg_status reg_create_series(const float *frames, int32_t n_series, const int32_t *frames_per_series,
                             const int32_t *side_px, int64_t pitch_elems, int32_t frames_on_device,
                             const reg_params *p, void *cuda_stream, reg_series_t *out);

/* Run a batch of independent operator applications in one device loop.
 * op_status_out, iters_out (nullable, n_ops entries, host memory): per-op
 * reg_op_status and total gradient steps over all levels.
 * Errors: REG_EINVAL for an out-of-range series/slot/frame, an identity slot
 * used as an operand, or a chain mismatch (left ends where right starts is
 * required: the slot holding phi_{a,b} and the one holding phi_{b,c}). */
reg_status reg_apply_operator_batch(reg_series_t s, int32_t n_ops, const reg_op_desc *ops,
                                    int32_t *op_status_out, int32_t *iters_out);

/* Image series registration: preprocessing (all A ops of all series in one
 * batch) followed by the prefix scan with the chosen schedule; each scan level
 * is one reg_apply_operator_batch over all series (segmented scan).  chunks:
 * the chunk count of the chunked strategies (1..64), or k of Han-Carlson
 * (1..30) and Ladner-Fischer (0..30) (values above log2 N give Brent-Kung);
 * global_kind: the chunked
 * strategies' global scan (a non-chunked kind up to Blelloch).  report_json_buf
 * (nullable): receives a NUL-terminated JSON summary (levels, op counts,
 * iterations, per-kernel timings when REG_FLAG_PROFILE is set). */
reg_status reg_prefix_scan(reg_series_t s, reg_scan_kind kind, int32_t chunks, reg_scan_kind global_kind,
                           char *report_json_buf, size_t buf_len);

/* Copy deformations phi_{0,k} - id, k = first .. first+count-1, of series
 * `series` into out (count x 2 x side x side float32, pixels; host memory
 * unless out_on_device).  phi_{0,0} is the identity (zeros).  Valid after
 * reg_prefix_scan. */
reg_status reg_get_deformations(reg_series_t s, int32_t series, int32_t first, int32_t count, float *out,
                                int32_t out_on_device);

/* Series averaging (Section "Introduction": the frames of a registered series,
 * deformed by phi_{0,i}, are averaged into one frame that holds the
 * information of the whole acquisition; Section "Registration for series of
 * images": the series averaging procedure repeats the registration to improve
 * it).  Valid after reg_prefix_scan.  The average is
 *   avg(x) = 1/N sum_{i=0}^{N-1} f_i(phi_i(x)),   phi_0 = id, phi_i = phi_{0,i},
 * on the finest vertex grid, each frame sampled by bilinear interpolation
 * (clamped to Omega) in its raw intensities (the stored normalisation undone).
 * Then `iterations` times: the average becomes the reference frame, every
 * frame f_i (f_0 included) is registered to it by function A started from
 * its current deformation (f_0 from the identity the first time) -- all N
 * operators in one batch -- and the average is formed again with the new
 * deformations.  After at least one iteration reg_get_deformations returns
 * these deformations from the average's frame to each frame (frame 0's
 * included) until the next reg_prefix_scan.  avg_out (nullable): side x side
 * float32, the average at the frame's pixels (host memory unless
 * out_on_device).  Errors: REG_ESTATE before a scan, REG_EINVAL for a bad
 * series or iterations outside [0, 1000]. */
reg_status reg_average_series(reg_series_t s, int32_t series, int32_t iterations, float *avg_out,
                              int32_t out_on_device);

/* Copy the finest-level field held in a slot and its (start, end) frame pair;
 * end < 0 marks the identity (zeros are written).  out: 2 x (side+1) x (side+1)
 * float32, pixels, the full vertex grid of level L (host unless
 * out_on_device).  Used by tests and by callers that drive
 * reg_apply_operator_batch themselves. */
reg_status reg_get_slot(reg_series_t s, int32_t series, int32_t slot, float *out, int32_t out_on_device,
                        int32_t *start_end);

/* Set a slot to phi_{start,end} given as a displacement field on the vertex
 * grid (2 x (side+1) x (side+1) float32, pixels, host or device) -- e.g. to
 * seed a scan with known neighbour deformations.  end < 0 marks the slot as
 * the identity (field ignored). */
reg_status reg_set_slot(reg_series_t s, int32_t series, int32_t slot, const float *field, int32_t on_device,
                        int32_t start, int32_t end);

/* Rigid handles (REG_FLAG_RIGID): the parameters (alpha in radians, t0, t1 in
 * Omega units) of the rigid map held in a slot, and its (start, end) pair;
 * reg_set_rigid sets a slot to phi_{start,end} given by its parameters (the
 * slot's field follows).  REG_ESTATE on a non-rigid handle. */
reg_status reg_get_rigid(reg_series_t s, int32_t series, int32_t slot, double *theta, int32_t *start_end);
reg_status reg_set_rigid(reg_series_t s, int32_t series, int32_t slot, const double *theta, int32_t start,
                         int32_t end);

/* Number of slots of a series (N-1 data slots for N frames plus the
 * auxiliary slots the largest schedule needs). */
reg_status reg_num_slots(reg_series_t s, int32_t series, int32_t *n_slots);

/* Diagnostic evaluation of the discrete energy of one frame pair at one level
 * for a given displacement (2 x n x n, grid units of that level, host memory):
 * fills parts[0..4] = {E, NCC, regulariser, T_bar, sigma_T}.  Used to check
 * the kernels against an independent implementation. */
reg_status reg_eval_energy(reg_series_t s, int32_t series, int32_t frame_i, int32_t frame_k, int32_t level,
                           const float *u_grid, double *parts);

/* Diagnostic evaluation of the gradient-flow direction d = -g / w (grid units)
 * and slope g^T d at a displacement (same conventions as reg_eval_energy). */
reg_status reg_eval_direction(reg_series_t s, int32_t series, int32_t frame_i, int32_t frame_k, int32_t level,
                              const float *u_grid, float *d_out, double *slope);

/* Diagnostic trial pass: at a displacement u (as for reg_eval_energy) one
 * gradient pass computes the direction d, then one trial pass evaluates the
 * energy change E(u + tau_j d) - E(u) of the Armijo search for the n_tau step
 * sizes taus[0..n_tau-1] (1 <= n_tau <= trials_per_pass), written to
 * dE_out[j] exactly as the operator state machine forms it (Section
 * "Optimization": gradient flow with a backtracking line search).  d_out
 * (2 x n x n, may be NULL) receives d.  Host buffers; returns when done. */
reg_status reg_eval_trials(reg_series_t s, int32_t series, int32_t frame_i, int32_t frame_k, int32_t level,
                           const float *u_grid, int32_t n_tau, const double *taus, float *d_out, double *dE_out);

/* ---------------------------------------------------------------------------
 * Learned initialiser (not in the paper: a coarse initial displacement for a
 * frame pair, predicted by a small convolutional network trained on
 * displacements the plain method computes; the plain gradient flow refines it).
 * Network: input 2 x S x S (channel 0 the reference frame, 1 the template,
 * normalised), six 3x3 convolutions with zero padding 1 -- 2->32 stride 2,
 * 32->32 stride 2, three 32->32 stride 1, 32->2 stride 1 -- with a ReLU after
 * every layer but the last; output 2 x S/4 x S/4, the displacement in input
 * pixels at input pixels (4i, 4j).  Loss: mean squared difference to a target.
 * Parameters: one flat float vector of reg_cnn_num_params() values, layer by
 * layer W (out x in x 3 x 3, row-major) then b.  All data pointers are device
 * pointers unless stated; calls return when the work is done.
 * ------------------------------------------------------------------------- */
typedef struct reg_cnn *reg_cnn_t;
int64_t reg_cnn_num_params(void);
/* A network for inputs of side x side (a multiple of 4, 16..4096) and batches
 * of up to max_batch pairs; parameters start at zero (set them). */
reg_status reg_cnn_create(int32_t side, int32_t max_batch, void *cuda_stream, reg_cnn_t *out);
/* Parameters from/to `theta` (host memory unless on_device); setting them also
 * resets the optimiser state. */
reg_status reg_cnn_set_params(reg_cnn_t h, const float *theta, int32_t on_device);
reg_status reg_cnn_get_params(reg_cnn_t h, float *theta, int32_t on_device);
/* y (batch x 2 x side/4 x side/4) = network(x (batch x 2 x side x side)).
 * tensor_cores != 0: the 32-channel layers on the tensor cores (BF16 operands,
 * FP32 accumulation), else every layer in FP32 on the CUDA cores. */
reg_status reg_cnn_forward(reg_cnn_t h, const float *x, int32_t batch, float *y, int32_t tensor_cores);
/* Loss against `target` (same shape as y) and its gradient (FP32, kept in the
 * handle for reg_cnn_adam_step; also copied to grad_out, host, if not NULL);
 * *loss (host) receives the mean squared error. */
reg_status reg_cnn_loss_grad(reg_cnn_t h, const float *x, const float *target, int32_t batch, double *loss,
                             float *grad_out);
/* reg_cnn_loss_grad with the training on the tensor cores: the forward of
 * the four 32-channel layers, their weight gradients and the data gradients
 * of the three stride-1 ones take BF16 operands with FP32 accumulation; the
 * first and last layers and the stride-2 layer's data gradient stay in FP32
 * on the CUDA cores; bias gradients sum the FP32 output gradients. */
reg_status reg_cnn_loss_grad_tc(reg_cnn_t h, const float *x, const float *target, int32_t batch, double *loss,
                                float *grad_out);
/* One Adam step (bias-corrected) with the last gradient. */
reg_status reg_cnn_adam_step(reg_cnn_t h, double lr, double beta1, double beta2, double eps);
reg_status reg_cnn_destroy(reg_cnn_t h);
/* Network inputs of `count` neighbour pairs (first_pair .. first_pair+count-1:
 * frames e and e+1) of a series, from its pyramid level of 257^2 nodes (the
 * first 256 rows and columns), into x (count x 2 x 256 x 256).  REG_EINVAL if
 * the pyramid has no such level. */
reg_status reg_cnn_pairs(reg_series_t s, int32_t series, int32_t first_pair, int32_t count, float *x);
/* Predict the initial displacement of every neighbour pair of a series with a
 * network for 256^2 inputs, upsample it (bilinear in the output grid, clamped)
 * onto the finest vertex grid in frame pixels, and store it in the pair's data
 * slot (reg_get_slot reads it back); the next reg_prefix_scan starts those
 * preprocessing operators from the slots instead of the identity, on the
 * finest reg_params.init_levels levels, and judges each start that skips
 * levels (reg_params.learned_fallback_px). */
reg_status reg_cnn_init_series(reg_series_t s, int32_t series, reg_cnn_t h, int32_t tensor_cores);

/* Tiles of the step kernels.  The gradient and trial passes walk strip tiles
 * of 30 node columns (gradient) or 31 cell columns (trial) by a number of rows
 * chosen per pyramid level l (2^l + 1 nodes per side); defaults 8 (l <= 6),
 * 16 (l <= 8), 32.  Rows must be 4, 8, 16, 32 or 64 (REG_EINVAL otherwise).
 * The rows change which FP32 partial sums are formed before the FP64 sum over
 * tiles, so results can differ at the rounding level. */
reg_status reg_set_tile_rows(reg_series_t s, int32_t level, int32_t grad_rows, int32_t trial_rows);
reg_status reg_get_tile_rows(reg_series_t s, int32_t level, int32_t *grad_rows, int32_t *trial_rows);
/* Tile autotuner: times a sample batch of function A on the neighbour pairs
 * 0..n_pairs-1 of `series` (best of `repeats` runs) and picks, level by level
 * from the finest (levels of at least 129 nodes), the gradient and trial tile
 * rows with the shortest time per device step, then the step sizes per trial
 * pass (2, 3, 4 or 8) with the shortest batch time; a change must gain 2%.  The
 * result stays in the handle (reg_get_tile_rows, and reg_params'
 * trials_per_pass as the handle uses it).  It overwrites the data slots
 * 0..n_pairs-1 (and drops a pending learned start): call it before
 * reg_prefix_scan, reg_set_slot or reg_cnn_init_series.  report (may be NULL):
 * a JSON object with the chosen table and the sample's time before and after. */
reg_status reg_autotune(reg_series_t s, int32_t series, int32_t n_pairs, int32_t repeats, char *report,
                        size_t buf_len);

/* Schedule export (host only, no GPU work): writes the op list of a schedule
 * over n elements as reg_schedule_op records (level index, kind, slots) into
 * buf (up to buf_len records), the total count into *n_out (call with buf NULL
 * to size) and the auxiliary slot count into *n_aux_slots.  Ops of one level
 * read the slots as they were before the level. */
typedef struct reg_schedule_op {
    int32_t level;
    int32_t kind;   /* 0 combine dst = a (.) b, 1 copy dst = a, 2 identity dst */
    int32_t dst;
    int32_t a;
    int32_t b;
} reg_schedule_op;
reg_status reg_schedule(reg_scan_kind kind, int32_t n, int32_t chunks, reg_scan_kind global_kind,
                        reg_schedule_op *buf, int64_t buf_len, int64_t *n_out, int32_t *n_aux_slots);

/* Per-kernel-family statistics accumulated since creation (or the last reset):
 * launches, device time (ms, CUDA events, only with REG_FLAG_PROFILE) and
 * algorithmic bytes (counted on the device per processed node).  Three more
 * records count nodes in `items`: "trial_exact_nodes", the trial-pass nodes
 * whose largest move left their cell (the exact path of the trial kernel);
 * "trial_seq_nodes", the sum over Armijo trials decided of the level's node
 * count (the trials of the one-at-a-time rule, however many step sizes a pass
 * evaluated); "trial_start_nodes", the nodes of level-start energy passes. */
typedef struct reg_kernel_stats {
    char name[24];
    int64_t launches;
    double ms;
    double bytes;
    int64_t items;
} reg_kernel_stats;
reg_status reg_get_kernel_stats(reg_series_t s, reg_kernel_stats *buf, int32_t buf_len, int32_t *n_out);
reg_status reg_reset_kernel_stats(reg_series_t s);

/* Diagnostic trace of every Armijo trial the device state machine decides:
 * reg_set_trace allocates room for `capacity` records (0 disables);
 * reg_get_trace copies up to cap records of 7 doubles
 * {op index in its batch, nodes per side of the level, iteration, tau,
 *  E(u + tau d) - E(u), sigma tau g^T d, accepted} and returns the number
 * recorded.  Records of one op appear in decision order. */
reg_status reg_set_trace(reg_series_t s, int64_t capacity);
reg_status reg_get_trace(reg_series_t s, double *out, int64_t cap, int64_t *n_out);

/* Lockstep replay (diagnostic).  The iteration of the gradient flow (Section
 * "Gradient flow": phi^{k+1} = phi^k - tau A^{-1} E'[phi^k], tau from the
 * Armijo rule) is chaotic on noisy frames: a decision whose margin is at the
 * rounding level sends two correct implementations down different paths.  In
 * lockstep the device takes a given sequence of accepted step sizes instead of
 * searching, so that its iterates can be compared step by step with another
 * implementation's.  After this call every reg_apply_operator_batch of exactly
 * n_ops operators (each with n_levels levels) runs in lockstep: operator o on
 * level k (0 = coarsest) makes counts[o * n_levels + k] gradient steps with
 * the step sizes taken in order from taus (operator-major, then level, then
 * iteration), then ends the level; the trace (reg_set_trace) records each
 * step's energy change and whether the Armijo test would have accepted it.
 * The per-op status is MAXITER.  Host arrays, copied.  n_ops = 0 switches
 * lockstep off.  Errors: REG_EINVAL for a negative count or a step size that
 * is not positive and finite; a later batch of another size or level count
 * fails with REG_EINVAL. */
reg_status reg_set_lockstep(reg_series_t s, int32_t n_ops, int32_t n_levels, const int32_t *counts,
                            const double *taus);

/* Energy of one frame pair at one grid level, allocating no memory at all.
 * The paper has no counterpart: this is a service for callers that must not
 * allocate device memory (for instance a plug-in inside an acquisition
 * pipeline whose host application reserved the device memory up front, or a
 * per-frame loop that cannot afford the synchronisation cudaMalloc implies).
 * It needs no handle.
 *   R, T      device pointers to the raw reference and template images of the
 *             level, n x n nodes (the vertex grid), row pitch `pitch` floats;
 *   u_grid    device pointer, displacement of the level in grid units, two
 *             planes of n x n floats (columns, then rows), dense;
 *   lambda    regulariser weight;
 *   parts_out {E, NCC, regulariser, T_bar, sigma_T} (5 doubles), host memory
 *             unless out_on_device;
 *   cuda_stream the stream to run on (NULL: legacy default stream); the call
 *             returns when the result is in parts_out.
 * Scratch: a file-scope device array sized for n <= REG_NOALLOC_MAX_NODES
 * (frames of 2048^2; about 192 KiB), held by every GPU that loads the library
 * until the process exits.  Its device address is looked up on the first
 * call on each device, so that first call should come before any stream
 * capture.  Every call shares the array and leaves its partial sums in it
 * (each call overwrites all it reads, so no clearing is needed); calls that
 * overlap on the GPU race and must be serialised by the caller.  The call
 * waits for its stream (cudaStreamSynchronize) before it returns.  The sums
 * are taken in two passes (FE means, then the moments of the centred images),
 * so raw frames whose mean is large against their spread keep their
 * precision.
 * Errors: REG_EINVAL for a null pointer, n < 3, n > REG_NOALLOC_MAX_NODES or
 * pitch < n; REG_ECUDA if a CUDA call fails.  Allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine. */
#define REG_NOALLOC_MAX_NODES 2049
reg_status reg_eval_energy_noalloc(const float *R, const float *T, int32_t n, int32_t pitch, const float *u_grid,
                                   double lambda, double *parts_out, int32_t out_on_device, void *cuda_stream);

reg_status reg_destroy_series(reg_series_t s);
const char *reg_status_string(reg_status st);
/* Message of the last error on this thread (empty if none). */
const char *reg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* REG_H */
