/*
 * kura.h -- C ABI of libkura: the Kuramoto model on graphs with localised
 * order parameters, integrated by classical RK4 on one NVIDIA GB300 GPU.
 *
 * Method: Boehle, Kuehn, Thalhammer, "On the reliable and efficient
 * numerical integration of the Kuramoto model and related dynamical systems
 * on graphs", arXiv 2102.07167.
 *
 *   theta'_m = omega_m + (K / calM_m) sum_l A_{m l} sin(theta_l - theta_m)
 *                                               (eq:KuramotoGraph, Sec. 3)
 *
 * The adjacency matrix is permuted so that communities are contiguous
 * (P A P^T, Sec. 3), every block (I, J) is classified by its zero fraction,
 * dense blocks are evaluated through the precomputed block sums
 * S_J = sum_{l in J} sin theta_l, C_J = sum_{l in J} cos theta_l minus the
 * sums over the block row's zeros, sparse blocks by direct summation over
 * their non-zeros (eq:KuramotoGraphApproach and the remark after it).
 *
 * Conventions for every entry point:
 *   - All vectors are in the caller's ("user") node order; the library
 *     applies and undoes its permutation at the boundary.
 *   - Phase/frequency vectors may be device pointers or host pointers
 *     (pinned or pageable); the library detects which.  With host pointers
 *     the call copies in and out and returns after the result is on the
 *     host.  With device pointers the call is asynchronous on the handle's
 *     stream.
 *   - Arrays passed to kura_create are copied; the caller keeps ownership of
 *     every pointer it passes.  The handle owns its internal buffers.
 *   - Every call returns a kura_status; nothing aborts or exits.  A failed
 *     call leaves a message in kura_last_error(handle).  Device-side
 *     conditions (non-finite phases, a bounded wait that gave up) latch in
 *     the handle and are reported by kura_sync and by any call that
 *     synchronises.
 *   - A handle is not thread-safe: one host thread at a time.
 */
#ifndef KURA_H
#define KURA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kura_ctx* kura_t;
typedef struct kura_plan_s* kura_plan_t;

typedef enum {
    KURA_OK = 0,
    KURA_EINVAL = 1,     /* invalid argument (bad CSR, label, size, pointer, h, ...) */
    KURA_ENOMEM = 2,     /* host or device allocation failed */
    KURA_ECUDA = 3,      /* CUDA runtime error (no device, launch failure, ...) */
    KURA_ESTATE = 4,     /* call not valid in the handle's state */
    KURA_ETIMEOUT = 5,   /* a bounded device-side wait gave up */
    KURA_ENUMERIC = 6    /* a non-finite value appeared in the state */
} kura_status;

enum { KURA_PREC_FP64 = 0, KURA_PREC_MIXED = 1 };
enum { KURA_SCALING_UNIFORM = 0, KURA_SCALING_DEGREE = 1 };

typedef struct {
    /* KURA_PREC_FP64: FP64 sin/cos, per-edge sums exact in 64-bit fixed
     *   point, FP64 epilogue and state.
     * KURA_PREC_MIXED: FP32 sin/cos of the phase reduced mod 2 pi (in 64-bit
     *   fixed point for 2^-10 <= |theta| < 2^21, else in FP64), FP32
     *   per-edge corrections, block sums exact in fixed point and rounded
     *   once to FP64, FP64 epilogue and state. */
    int32_t precision;
    /* calM_m of eq:KuramotoGraph: KURA_SCALING_UNIFORM (calM_m = N) or
     * KURA_SCALING_DEGREE (calM_m = sum_l A_{m l}; zero rows get theta' = omega). */
    int32_t scaling;
    /* block threshold: dense iff zero fraction < tau (Sec. 1, 3: precompute
     * when ones outnumber zeros); in [0, 1], default 0.5 */
    double tau;
    /* keep a host copy of the CSR (needed by kura_classify_blocks with a new
     * tau and by the direct-summation baseline); default 1 */
    int32_t keep_host_csr;
    /* tensor-core encoding of a community's dense-block zeros: a 0/1 mask over
     * 128-column blocks multiplied on the tensor cores (tcgen05, FP8 operands)
     * by the base-16 digits of the fixed-point (sin, cos) of those columns, so
     * that the subtracted sums are exact in fixed point.  Requires that the
     * community's dense columns span at most 4096 columns.  0: never; 1
     * (default): when the mask takes fewer bytes than the index lists; 2:
     * whenever possible. */
    int32_t tensor_cores;
    /* index encoding of a community's dense-block zeros (when not on the
     * tensor cores): a bitmap over the staged window when their fraction
     * exceeds this, else an index list; negative (default): index lists */
    double bitmap_zmin;
    /* batch handles: lanes that gather one row's listed entries, 32 (a warp
     * per row; default when 0), 16 or 8 (2 or 4 rows per warp) */
    int32_t row_lanes;
    /* single handles of small graphs (n <= 4096, n_comm <= 256, 0/1 matrix,
     * host CSR kept, at most 16 listed corrections per row on average):
     * 1 (default) kura_rk4_steps runs every step in one launch of one
     * thread-block cluster of 8 CTAs, the (sin, cos) table spread over their
     * shared memory and read through the cluster (not while kernel timing is
     * on); 0: always the CUDA-graph step loop */
    int32_t persistent_small;
    /* kura_rk4_steps on single handles: 1 (default) each RK4 stage's row
     * kernel also makes the next stage's (sin, cos) table, digits and
     * fixed-point block sums from the phases it writes, so a run of steps
     * needs one trig/block-sum launch in all (bit-identical results); 0: a
     * trig/block-sum launch before every stage */
    int32_t fused_trig;
    int32_t reserved;
} kura_opts;

typedef struct {
    int64_t n, nnz, self_loops;      /* nodes; edges as given; diagonal entries dropped */
    int32_t n_comm, q_bits;          /* communities; fixed-point fraction bits */
    double tau;
    int64_t dense_blocks, sparse_blocks, nonempty_blocks;
    int64_t missing_entries;         /* zeros of dense blocks stored (subtracted) */
    int64_t sparse_entries;          /* non-zeros of sparse blocks stored (added) */
    int64_t max_row_entries;
    int64_t tiles, max_window;
    /* Algorithmic bytes of one right-hand-side evaluation, split by kernel:
     * stream_bytes = correction streams + per-row metadata read by the row
     * kernel (with opts.fused_trig and tensor-core tiles, plus the digit
     * image it writes for the next stage); node_bytes_row = per-node traffic
     * of the row kernel in an RK4 stage (with opts.fused_trig, plus the next
     * stage's table entry); node_bytes_trig = per-node traffic of the
     * trig/block-sum kernel. */
    int64_t stream_bytes, node_bytes_row, node_bytes_trig;
    int64_t direct_edges;            /* edges summed by the direct baseline */
    int64_t tc_tiles, tc_rows;       /* tiles (and their rows) whose zeros are a tensor-core mask */
    int64_t tc_mask_bits;            /* mask bits of those tiles (128 x 128 blocks) */
} kura_block_stats;

/* Fills *opts with the defaults (FP64, uniform scaling, tau 0.5, host CSR kept,
 * tensor cores when smaller). */
void kura_default_opts(kura_opts* opts);

/* Library version (major*10000 + minor*100 + patch). */
int32_t kura_version(void);

/* Human-readable name of a status code (static string). */
const char* kura_status_string(kura_status s);

/* Creates a handle for the graph given in CSR (eq:KuramotoGraph).
 *   n               number of oscillators (M in the paper), >= 1
 *   row_ptr[n+1]    host, int64, row_ptr[0] = 0, non-decreasing
 *   col[nnz]        host, int32, row m lists the l with A_{m l} = 1,
 *                   strictly increasing within a row; diagonal entries are
 *                   dropped (they add sin 0 = 0, Sec. 2 remark)
 *   label[n]        host, community of each node in [0, n_comm) (the
 *                   partition of Sec. 3; communities may be empty)
 *   omega[n]        host, natural frequencies
 *   K               coupling constant (finite)
 *   opts            nullable (defaults)
 *   stream          cudaStream_t for all work of the handle (NULL: legacy
 *                   default stream)
 *   out             receives the handle
 * Permutes, classifies blocks with opts->tau and uploads.  Returns
 * KURA_EINVAL for malformed input, KURA_ECUDA if no usable GPU. */
kura_status kura_create(int64_t n, const int64_t* row_ptr, const int32_t* col,
                        const int32_t* label, int32_t n_comm, const double* omega,
                        double K, const kura_opts* opts, void* stream, kura_t* out);

/* Finite-valued adjacency (Sec. 1, "Generalisations": A_{ml} in {0, ..., J}):
 * as kura_create, with val[nnz] (host, int32, 1..127, parallel to col) the
 * value of each listed entry; n <= 2^24 - 2; uniform scaling only
 * (f_m = omega_m + (K/n) sum_l A_{ml} sin(theta_l - theta_m)).  Per block the
 * nonzero value of largest count v_IJ (ties: the smaller) is prevalent when
 * the fraction of entries different from it is below tau: the block then
 * contributes v_IJ (S_J, C_J) plus (A_{ml} - v_IJ)(sin, cos) theta_l over its
 * exceptions, else (sparse) A_{ml} (sin, cos) theta_l over its entries.  Both
 * corrections are index lists (no tensor cores, no bitmaps).  kura_rhs,
 * kura_rk4_steps, kura_integrate, kura_order_params, kura_classify_blocks and
 * kura_autotune apply; kura_adjoint, kura_potential and the direct baseline
 * return KURA_ESTATE. */
kura_status kura_create_valued(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* val,
                               const int32_t* label, int32_t n_comm, const double* omega, double K,
                               const kura_opts* opts, void* stream, kura_t* out);

/* Re-classifies the blocks with a new threshold tau in [0, 1] (pass a
 * negative tau to keep the current one) and rebuilds the streams (Sec. 3,
 * dense/sparse decision).  Needs the host CSR copy.  stats is nullable. */
kura_status kura_classify_blocks(kura_t h, double tau, kura_block_stats* stats);

/* Current classification statistics (host struct). */
kura_status kura_get_stats(kura_t h, kura_block_stats* stats);

/* One right-hand-side evaluation, dtheta = F(theta) (eq:KuramotoGraph by
 * eq:KuramotoGraphApproach).  theta[n], dtheta[n]: user order, device or
 * host, may not alias. */
kura_status kura_rhs(kura_t h, const double* theta, double* dtheta);

/* n_steps classical RK4 steps of size step on theta[n] in place (user
 * order, device or host).  step > 0 and finite; n_steps >= 0.  The step
 * loop runs as a CUDA graph (cached per (step, chunk)).  The phases are kept
 * unwrapped (eq:5c). */
kura_status kura_rk4_steps(kura_t h, double* theta, double step, int64_t n_steps);

enum { KURA_INT_RK4 = 0, KURA_INT_RK2 = 1, KURA_INT_IMPLICIT_MIDPOINT = 2 };

/* n_steps steps of a chosen integrator on theta[n] in place (user order,
 * device or host), with the block method as right-hand side:
 *   KURA_INT_RK4                as kura_rk4_steps (iters ignored);
 *   KURA_INT_RK2                explicit midpoint, Y = y + h/2 f(y), y' = y + h f(Y);
 *   KURA_INT_IMPLICIT_MIDPOINT  y' = 2 Z - y where Z = y + h/2 f(Z), the stage
 *                               found by `iters` (1..64) fixed-point sweeps from
 *                               the predictor y + h/2 f(y); a symmetric,
 *                               second-order geometric method.
 * The paper compares a second-order explicit Runge-Kutta method with a
 * second-order implicit one for the conserved quantity of eq:5c over long
 * times (Sec. 2, numerical results).  Steps run as cached CUDA graphs. */
kura_status kura_integrate(kura_t h, double* theta, double step, int64_t n_steps, int32_t method, int32_t iters);

/* Order parameters (eq:OrderParameter): r e^{i psi} = (1/n) sum_m e^{i theta_m}
 * of theta[n] (user order, device or host); r, psi: host scalars.  When
 * r_comm / psi_comm (host, n_comm entries each, nullable) are given, the
 * same quantity per community ("localised order parameters"); empty
 * communities give 0.  psi = 0 when r = 0.  Synchronises the stream. */
kura_status kura_order_params(kura_t h, const double* theta, double* r, double* psi,
                              double* r_comm, double* psi_comm);

/* Graph potential of eq:ExtendedPotentialConservation at theta[n] (user
 * order, device or host):
 *   V = -sum_m omega_m theta_m + (K/2) sum_m (1/calM_m) sum_l A_{ml} (1 - cos(theta_l - theta_m)),
 * rows without neighbours contributing no coupling term.  The inner sums use
 * the cosine identity sum_l A_{ml} cos(theta_l - theta_m) = cos theta_m
 * (A cos theta)_m + sin theta_m (A sin theta)_m, with the row sums of the
 * block method (one right-hand-side pass) and FP64 sin/cos of theta_m; the
 * reduction over m is FP64 in a fixed order (deterministic).  For symmetric
 * A and uniform scaling the flow is a gradient flow of V, so V does not
 * increase along trajectories.  *V: host.  Synchronises the stream. */
kura_status kura_potential(kura_t h, const double* theta, double* V);

/* eq:Means: (1/n) sum_m (theta_m(t) - theta_m(0) - t omega_m) of theta_t and
 * theta_0 (user order, device or host); zero at all t for symmetric A with
 * uniform scaling (the coupling terms cancel in pairs).  FP64, fixed-order
 * reduction.  *out: host.  Synchronises the stream. */
kura_status kura_mean_deviation(kura_t h, const double* theta_t, const double* theta_0, double t, double* out);

/* Gradient of a terminal loss of an RK4 trajectory by the discrete adjoint
 * of the classical RK4 step (backward sweep over the stage Jacobians of
 * eq:KuramotoGraph; the paper's integrator section, Sec. 2, extended to a
 * terminal loss, as in training):
 *   loss_kind 0: L = 1 - r(theta(T)) (eq:OrderParameter);
 *   loss_kind 1: L = 1/2 sum_m (theta_m(T) - target_m)^2 (target[n], user order).
 * theta0[n] (user order, device or host) is not modified.  The forward pass
 * keeps a checkpoint every ckpt_every steps; the backward pass recomputes one
 * segment at a time, keeping its stage inputs and stage row sums
 * (4 * ckpt_every * 24 bytes per node); segments of exactly ckpt_every
 * steps are replayed as one captured CUDA graph.  Outputs: *loss and *g_K
 * (host), g_omega[n] and g_theta0[n] (user order, device or host).  Needs a
 * handle created with KURA_PREC_MIXED (FP32 right-hand side, FP64 state and
 * accumulations) and the host CSR copy: KURA_ESTATE otherwise.  For a
 * directed A (checked once on the host CSR) the first call also plans A^T
 * (same labels, so the same permutation), over which the nu-weighted sums of
 * J^T w run; that plan keeps the options the handle had then.  Synchronises
 * the stream. */
kura_status kura_adjoint(kura_t h, const double* theta0, double step, int64_t n_steps,
                         int32_t ckpt_every, int32_t loss_kind, const double* target,
                         double* loss, double* g_omega, double* g_K, double* g_theta0);

/* One trajectory of a batch: its own graph (CSR as in kura_create), community
 * labels, natural frequencies and coupling constant.  row_ptr == NULL denotes
 * the complete graph without self-loops (the classical model, eq:Kuramoto):
 * col and label are ignored and n_comm must be 1. */
typedef struct {
    int64_t n;
    const int64_t* row_ptr;
    const int32_t* col;
    const int32_t* label;
    int32_t n_comm;
    const double* omega;
    double K;
} kura_graph_desc;

/* Creates a batch handle: n_traj independent trajectories (uneven sizes,
 * n_comm <= 1024 each), integrated together by one persistent launch per
 * kura_rk4_steps call: one CTA integrates a whole trajectory, all its steps,
 * with the trajectory's (sin, cos) table in shared memory; trajectories are
 * handed out longest first.  Each trajectory is planned as in kura_create
 * (eq:KuramotoGraphApproach with opts->tau, uniform scaling K/n).
 *   opts->precision  KURA_PREC_MIXED (1 <= n <= 16384 per trajectory) or
 *                    KURA_PREC_FP64 (1 <= n <= 8192: FP64 sin/cos, every sum
 *                    exact in 64-bit fixed point, FP64 epilogue and state)
 *   opts->tensor_cores (mixed only) 2: the dense-block zeros of a community
 *                    as a 0/1 mask multiplied on the tensor cores
 *                    (tcgen05.mma.kind::f16: BF16 mask, split BF16 hi + lo
 *                    (sin, cos), FP32 accumulation in tensor memory) wherever
 *                    the dense columns span <= 4096 columns; 0 or 1: index
 *                    lists.  With one graph per trajectory the product has 4
 *                    useful columns (N = 16) and touches every entry of a
 *                    dense block where the lists touch only its zeros, so the
 *                    lists are the default; kura_autotune may choose either
 *                    per size class.
 * On a batch handle kura_rk4_steps and kura_rhs take the phases (and the
 * right-hand side) of all trajectories concatenated in trajectory order
 * (user order within each); the other per-graph calls return KURA_ESTATE.
 * Host arrays are copied.  Errors as for kura_create. */
kura_status kura_batch_create(int32_t n_traj, const kura_graph_desc* graphs, const kura_opts* opts,
                              void* stream, kura_t* out);

/* Sizes of a batch: total oscillators and stored corrections (nullable outputs). */
kura_status kura_batch_stats(kura_t h, int64_t* n_total, int64_t* missing, int64_t* present);

typedef struct {
    int32_t n_traj, precision;
    int64_t n_total;             /* oscillators of all trajectories */
    int64_t missing_listed;      /* dense-block zeros given as index lists */
    int64_t present;             /* sparse-block non-zeros (index lists) */
    int32_t tc_traj;             /* trajectories with tensor-core tiles */
    int32_t pad;
    int64_t tc_tiles, tc_mask_bits;   /* tensor-core tiles (<= 128 rows each) and their mask bits */
} kura_batch_info_t;

/* Layout of a batch handle (host struct). */
kura_status kura_batch_info(kura_t h, kura_batch_info_t* out);

/* Plan choices of trajectory t of a batch handle: tau, encoding of the
 * dense-block zeros (as kura_opts.tensor_cores) and lanes per row (32, 16 or
 * 8); any output may be NULL. */
kura_status kura_batch_traj_params(kura_t h, int32_t t, double* tau, int32_t* tensor_cores, int32_t* row_lanes);

/* Host only (no device call): the cost the batch work queue would give each
 * of n_traj trajectories under opts, the same per-node, listed-entry and
 * tensor-core terms kura_batch_create sorts by.  Each trajectory is planned
 * as kura_batch_create would plan it (opts->precision, opts->tau,
 * opts->tensor_cores == 2); the planner's tile-size target uses the SM count
 * of the current device, else 152.  cost: host array of n_traj doubles,
 * caller-owned.  KURA_EINVAL for the trajectory errors of kura_batch_create
 * (message in kura_last_error(NULL)). */
kura_status kura_batch_costs(int32_t n_traj, const kura_graph_desc* graphs, const kura_opts* opts, double* cost);

/* Host only: longest-processing-time partition of n items over n_parts
 * parts, the rule by which independent trajectories shard across GPUs with
 * no collective.  Items are taken in decreasing cost (equal costs: lower
 * index first) and each goes to the part with the least load so far (equal
 * loads: lower part), so every process that calls it with the same costs
 * gets the same partition; the largest load is at most the mean load plus
 * the largest cost.  cost: n finite, non-negative doubles; part: n int32
 * outputs in [0, n_parts); load: n_parts outputs (nullable).  Host arrays,
 * caller-owned.  KURA_EINVAL for n < 0, n_parts < 1, NULL arrays or a
 * negative or non-finite cost. */
kura_status kura_partition_lpt(const double* cost, int32_t n, int32_t n_parts, int32_t* part, double* load);

/* Replaces omega (nullable; n entries, user order, device or host) and/or
 * K (nullable). */
kura_status kura_set_param(kura_t h, const double* omega, const double* K);

/* Direct-summation baseline: dtheta_m = omega_m + (K/calM_m) sum over the
 * CSR edges of sin(theta_l - theta_m), one sine per edge (eq:KuramotoGraph,
 * original formulation; the paper's straightforward summation).
 * precision: KURA_PREC_FP64 (FP64 sine per edge) or KURA_PREC_MIXED (FP32
 * sine of FP32 phases reduced mod 2 pi, FP32 row sums, FP64 epilogue). */
kura_status kura_direct_rhs(kura_t h, const double* theta, double* dtheta, int32_t precision);

/* n_steps RK4 steps with the direct-summation right-hand side. */
kura_status kura_direct_rk4_steps(kura_t h, double* theta, double step, int64_t n_steps,
                                  int32_t precision);

/* Enables (1) or disables (0) CUDA-event timing of every row-kernel launch
 * inside the captured RK4 graphs; kura_kernel_times then returns the
 * per-launch durations (ms) of the last replay, up to cap entries, and the
 * number available in *count. */
kura_status kura_set_timing(kura_t h, int32_t on);
kura_status kura_kernel_times(kura_t h, float* ms, int32_t cap, int32_t* count);

/* Ensemble of n_traj trajectories that share one graph (not in the paper:
 * its batched form).  n_traj must be a multiple of 16; the trajectories are
 * processed in groups of 16.
 *   omega   host, n_traj x n (trajectory-major, user order)
 *   K       host, n_traj (uniform scaling K / N per trajectory)
 * The graph arguments and opts->tau are as in kura_create; opts->tensor_cores
 * = 0 keeps index lists, any other value puts every dense community whose
 * dense columns span <= 4096 columns on the tensor cores.  The dense-block
 * product A_IJ [sin, cos] of eq:KuramotoGraphApproach is then a real matrix
 * product over the 16 trajectories of a group: the 0/1 mask (BF16, exact)
 * times the split BF16 hi + lo (sin, cos) of every trajectory, 64 columns,
 * FP32 accumulation in tensor memory (tcgen05.mma.kind::f16); listed entries
 * are gathered for all 16 trajectories at once.  FP32 sin/cos of phases
 * reduced mod 2 pi in FP64, FP64 block sums, epilogue and state.
 * kura_rhs and kura_rk4_steps then take theta (and dtheta) as n_traj x n
 * arrays, host or device; kura_get_stats, kura_sync, kura_set_stream,
 * kura_last_error and kura_destroy work as for single handles, every other
 * call returns KURA_ESTATE. */
kura_status kura_ensemble_create(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* label,
                                 int32_t n_comm, int32_t n_traj, const double* omega, const double* K,
                                 const kura_opts* opts, void* stream, kura_t* out);

/* Result of kura_autotune. */
typedef struct {
    double tau;              /* chosen dense/sparse threshold */
    int32_t tensor_cores;    /* chosen encoding of dense-block zeros (as kura_opts.tensor_cores) */
    int32_t candidates;      /* plans built and timed (the handle's own plan included) */
    int64_t tile_work;       /* chosen work target per tile (stored entries + per-row overhead) */
    double rhs_ms;           /* median time of one right-hand side with the chosen plan */
    double initial_rhs_ms;   /* the same with the plan the handle had on entry */
    double seconds;          /* wall time spent tuning */
} kura_tune_result;

/* Autotuner of the block plan (not in the paper: its tau = 0.5 is a cost
 * argument, Sec. 1 and 3).

 * On a batch handle (kura_batch_create with keep_host_csr = 1; theta is the
 * concatenated phases of all trajectories): the trajectories with a stored
 * graph are grouped by size class (ceil(log2 n)); per class, heaviest first
 * and within about budget_s seconds, one parameter at a time is moved from
 * the handle's choice -- the encoding of the dense-block zeros (index lists
 * or the tensor-core mask product, mixed precision only), the row tile
 * (32, 16 or 8 lanes gather one row's listed entries) and tau (0.35, 0.5,
 * 0.65) -- each candidate timed over 3 RK4 steps of a sub-batch of the class
 * (at most one trajectory per SM).  The fastest choice is kept for the class
 * and the batch is rebuilt.  out->rhs_ms and out->initial_rhs_ms are then
 * milliseconds per RK4 step of the whole batch (after and before), tau and
 * tensor_cores the choice of the heaviest class and tile_work its lanes per
 * row; kura_batch_traj_params gives every trajectory's choice.
 *
 * On a single handle:  Every plan computes the same right-hand side up
 * to rounding; only speed differs.  Times kura_rhs at theta (host or device,
 * user order, n values) for candidate plans, one parameter at a time
 * starting from the handle's own: the encoding of dense-block zeros
 * (tensor-core mask or index lists), the work per tile (x0.6, x1.6) and the
 * threshold tau (0.35, 0.65), within about budget_s seconds of wall time
 * (plan builds included).  The fastest plan is kept on the handle (cached
 * step graphs are dropped).  Needs the host CSR (keep_host_csr = 1), else
 * KURA_ESTATE.  Synchronous. */
kura_status kura_autotune(kura_t h, const double* theta, double budget_s, kura_tune_result* out);

/* Measurement for rooflines (not part of the method): the median rate, in
 * gathers per second, of random entry_bytes-byte (8 or 16) loads from a
 * table of table_entries entries (<= 2^30), as the row kernel makes for the
 * entries of sparse blocks.  Indices are counter-based hashes of the
 * position, uniform over the table; the table is L2-resident when it is
 * small enough.  gathers in [4096, 2^31] are made per run, four per 16-byte
 * index load, at full occupancy; one warm-up run, median of three timed
 * runs (CUDA events on stream).  Allocates and frees its own device memory;
 * synchronous.  KURA_EINVAL for sizes out of range. */
kura_status kura_measure_gather_rate(int64_t table_entries, int64_t gathers, int32_t entry_bytes, void* stream,
                                     double* gathers_per_s);

/* Measurement for rooflines (not part of the method): the read bandwidth, in
 * GB/s, of 16-byte loads streaming over a device buffer of `bytes` bytes
 * (1 MiB .. 1 GiB) 16 times; below the L2 size (126 MiB usable here) the
 * buffer stays in L2, so this is the L2 read bandwidth the L2-resident
 * workloads are bounded by.  One warm-up run, median of three (CUDA events on
 * stream).  Allocates and frees its own device memory; synchronous. */
kura_status kura_measure_l2_bandwidth(int64_t bytes, void* stream, double* gb_per_s);

/* Measurement (not part of the method): the time per kernel node, in
 * microseconds, of replaying a CUDA graph of `kernels` (1..4096) empty
 * dependent kernel launches `replays` (1..100000) times on stream: the launch
 * floor of a step loop captured as a graph.  Synchronous. */
kura_status kura_measure_graph_launch_floor(int32_t kernels, int32_t replays, void* stream, double* us_per_kernel);

/* Switches the handle to another stream (cached graphs stay valid). */
kura_status kura_set_stream(kura_t h, void* stream);

/* Waits for the handle's stream and reports latched device conditions
 * (KURA_ENUMERIC, KURA_ETIMEOUT), clearing them. */
kura_status kura_sync(kura_t h);

/* Last error message of the handle (or of the last failed kura_create when
 * h is NULL).  Static storage owned by the library. */
const char* kura_last_error(kura_t h);

/* Frees the handle and all its device and host memory.  NULL is a no-op. */
void kura_destroy(kura_t h);

/* Order parameters for callers that cannot allocate device memory.
 * The paper has no counterpart; this is a deployment convenience.  Some
 * callers may not call cudaMalloc at all: plug-ins inside a host application
 * that owns the whole device-memory budget and grants them none, and
 * real-time or watchdog-supervised loops in which the implicit device
 * synchronisation and unbounded latency of cudaMalloc/cudaFree are not
 * allowed.  Those callers pass their own input and output buffers; the
 * scratch this needs lives in a file-scope __device__ array of the library
 * (3 * 8 bytes per community plus two words, at most KURA_STATIC_MAX_COMM
 * communities, about 96 KB), which every GPU that loads the library holds
 * until process exit.
 *
 *   n                 number of oscillators, >= 1
 *   theta[n]          device, phases (any order)
 *   label[n]          device, community of each oscillator in [0, n_comm),
 *                     or NULL for one community (then n_comm must be 1)
 *   n_comm            1 .. KURA_STATIC_MAX_COMM; larger values -> KURA_EINVAL
 *   out[2 + 2 n_comm] device: out[0] = |(1/n) sum_m e^{i theta_m}| and
 *                     out[1] its argument (0 when the modulus is 0); then
 *                     out[2 + 2 J], out[3 + 2 J] the same mean over the
 *                     members of community J (0, 0 for an empty one)
 *   stream            cudaStream_t (NULL: legacy default stream)
 * Asynchronous on the stream.  It allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine.  The labels are device data, so
 * the host cannot check them: the kernel skips every oscillator whose label
 * lies outside [0, n_comm) and then writes NaN to every entry of out, so a
 * bad label never touches memory outside the scratch rows of this call.
 * Set-up: the first call in each CUDA context looks up the device address of
 * the scratch array (cudaGetSymbolAddress, with the device current) and
 * caches it with the context's id; after cudaDeviceReset the next call looks
 * it up again.  Make that first call on a device before any stream capture.
 * Every call on a device shares the one scratch array: calls that overlap on
 * the GPU (concurrent streams, or several host threads) race and give wrong
 * results, so serialise them.  Each call zeroes the part of the scratch it
 * uses before its kernel runs, and the kernel leaves it zeroed.  The sums are
 * exact 64-bit fixed-point sums of FP64 sin/cos, as in kura_order_params. */
#define KURA_STATIC_MAX_COMM 4096
kura_status kura_order_params_static(int64_t n, const double* theta, const int32_t* label,
                                     int32_t n_comm, double* out, void* stream);

/* ---------------------------------------------------------------------
 * Host-only block plan (no GPU needed): the permutation, classification and
 * correction streams that kura_create uploads, exposed for inspection.
 * Arguments as for kura_create (opts nullable: defaults); the layout follows
 * opts->precision, opts->tau and opts->bitmap_zmin.
 */
kura_status kura_plan_build(int64_t n, const int64_t* row_ptr, const int32_t* col,
                            const int32_t* label, int32_t n_comm, const kura_opts* opts,
                            kura_plan_t* out);
/* stats of the plan (the byte counts assume KURA_PREC_FP64) */
kura_status kura_plan_stats(kura_plan_t p, kura_block_stats* stats);
/* perm[n]: perm[new] = old; comm_off[n_comm + 1]: community boundaries in
 * the permuted order.  Either pointer may be NULL. */
kura_status kura_plan_perm(kura_plan_t p, int32_t* perm, int64_t* comm_off);
/* Correction streams of permuted row `row`: missing entries (zeros of its
 * dense blocks) and present entries (non-zeros of its sparse blocks), as
 * permuted column indices.  Writes up to cap entries to each array
 * (nullable) and the true counts to *n_missing, *n_present. */
kura_status kura_plan_row(kura_plan_t p, int64_t row, int32_t* missing, int64_t* n_missing,
                          int32_t* present, int64_t* n_present, int64_t cap);
/* Dense column blocks D(I) of row block I: up to cap entries, count in *count. */
kura_status kura_plan_dense_blocks(kura_plan_t p, int32_t I, int32_t* J, int32_t cap,
                                   int32_t* count);

/* Host-only plan of a finite-valued matrix (val as for kura_create_valued),
 * and the prevalent value of each dense block of row block I (in the order
 * of kura_plan_dense_blocks; 1 for 0/1 plans). */
kura_status kura_plan_build_valued(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* val,
                                   const int32_t* label, int32_t n_comm, const kura_opts* opts, kura_plan_t* out);
kura_status kura_plan_dense_values(kura_plan_t p, int32_t I, int32_t* v, int32_t cap, int32_t* count);
/* Read-only views of the packed correction data the row kernel consumes:
 * gstream (int32, *gstream_len entries), groups (*n_groups records of
 * {int64 off; int32 len; int32 first_subrow; int32 n_subrows; int32 pad}),
 * tiles (*n_tiles records of {int32 r0, r1, comm, wbeg, wlen, g0, g1,
 * first_subrow; int64 bitmap_off; int32 n_superwords, flags}), row_sub0
 * (n + 1 int32: first sub-row of each row) and the row bitmaps of tiles with
 * flag 1 (uint32, *bitmap_len words).  The pointers stay valid until
 * kura_plan_destroy.  Any output may be NULL. */
kura_status kura_plan_export(kura_plan_t p, const int32_t** gstream, int64_t* gstream_len,
                             const void** groups, int64_t* n_groups, const void** tiles,
                             int64_t* n_tiles, const int32_t** row_sub0, const uint32_t** bitmap,
                             int64_t* bitmap_len);
void kura_plan_destroy(kura_plan_t p);

#ifdef __cplusplus
}
#endif

#endif /* KURA_H */
