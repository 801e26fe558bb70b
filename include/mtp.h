/*
 * mtp.h -- C ABI of the GB300-native Model Tensor Planning (MTP) hot path.
 *
 * One planner iteration of MTP (arXiv 2505.01059, Alg. 2): sample paths
 * through a random M x N multipartite graph of control knots (Def. 1,
 * Alg. 1), interpolate them to H-step control trajectories (B-spline, Def. 2
 * and Eqs. 3-4; Akima, Def. 3 and Eqs. 5-7; or straight lines, Sec. 3.1),
 * mix them with local Gaussian samples around the current mean (beta-mixing,
 * Sec. 3.3), roll every candidate out through the dynamics with per-sample
 * randomised parameters and reduce its cost (Eq. 2), select the top-E elites
 * and apply the softmax-weighted CEM update (Alg. 2; Sec. 2.1 for the plain
 * CEM variant).
 *
 * Conventions for every entry point:
 *   - Return value: MTP_OK, or an error code; mtp_last_error() gives text.
 *   - Pointers named d_* are device pointers (any CUDA allocation on the
 *     handle's device), h_* are host pointers.  The caller owns them; the
 *     library reads/writes them stream-ordered on `stream` and keeps no
 *     reference after the call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously unless stated otherwise.
 *   - Logical layouts are the paper's, row-major: graph Z (M, N, n), path
 *     indices I (P, M), waypoints C (P, M, n), controls U (B, H, n), costs
 *     (B), mean/spread mu, sigma (H, n), state x (d).
 *   - Candidate rows of U (Alg. 2 stacking): [0, L) local Gaussian samples,
 *     [L, L+P) graph paths, row B-1 the nominal mean; P = min(floor(beta B),
 *     B-1), L = B-P-1.  Every control is clamped to [u_min, u_max].
 *   - Random draws are Philox4x32-10 (Salmon et al., SC'11) with key = the
 *     64-bit seed and counter = (index, sub-index/4, iteration, stream tag),
 *     so results depend only on (seed, iteration), never on launch shape.
 *   - No call traps the GPU; kernels report failures through return codes.
 */
#ifndef MTP_H
#define MTP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MTP_OK = 0,
  MTP_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter is out of range */
  MTP_ERR_OUT_OF_MEMORY = 2, /* a device or host allocation failed */
  MTP_ERR_CUDA = 3,          /* a CUDA runtime call failed (text in mtp_last_error) */
  MTP_ERR_ADMISSION = 4,     /* serving: over the memory budget, robot count or queue depth */
  MTP_ERR_TIMEOUT = 5,       /* a bounded wait ran out */
  MTP_ERR_NOT_READY = 6,     /* serving: the result is not there yet */
  MTP_ERR_UNSUPPORTED = 7    /* valid request the library does not implement */
} mtp_status;

typedef enum { MTP_DYN_POINTMASS = 0, MTP_DYN_CHAIN = 1, MTP_DYN_LEGGED = 2 } mtp_dyn;
typedef enum { MTP_INTERP_LINEAR = 0, MTP_INTERP_BSPLINE = 1, MTP_INTERP_AKIMA = 2 } mtp_interp;
/* Knot/evaluation-time reading of Defs. 2-3: VALID_SPAN maps the horizon onto
 * the span where the B-spline basis sums to one (and Akima's knots onto
 * [0, 1] with i/(M-1)); PAPER_LITERAL uses t_j = j/H as printed. */
typedef enum { MTP_TIME_VALID_SPAN = 0, MTP_TIME_PAPER_LITERAL = 1 } mtp_time_mapping;
/* SOFTMAX: Alg. 2's softmax-weighted mean/std with floor sigma_min.
 * PLAIN_CEM: Sec. 2.1's unweighted mean and 1/(E-1) variance. */
typedef enum { MTP_UPDATE_SOFTMAX = 0, MTP_UPDATE_PLAIN_CEM = 1 } mtp_update_rule;
/* Domain randomisation (Sec. 4): PER_SAMPLE gives every candidate its own
 * model scales; SHARED rolls every candidate out on R models and averages. */
typedef enum { MTP_DR_NONE = 0, MTP_DR_PER_SAMPLE = 1, MTP_DR_SHARED = 2 } mtp_dr_mode;

#define MTP_MAX_CTRL 32
#define MTP_MAX_LINKS 16
#define MTP_MAX_OBSTACLES 8

/* flags */
#define MTP_FLAG_NO_KAHAN 0x1u    /* plain FP32 cost sums instead of compensated ones */
#define MTP_FLAG_NO_GRAPH 0x2u    /* mtp_plan_step launches eagerly, no CUDA graph */
#define MTP_FLAG_BF16_BASIS 0x4u  /* B-spline contraction with BF16 operands: basis
                                     values and knots rounded to the nearest bfloat16
                                     (ties to even), exact products, FP32 sums.  B-spline
                                     only (MTP_ERR_UNSUPPORTED otherwise).  The graph rows
                                     are then a dense (H x M) by (M x paths*n) product on
                                     the tensor cores (tcgen05, BF16 x BF16 -> FP32) when
                                     H <= 256 and n <= 16, else a (p+1)-term sum on the
                                     FP32 pipe; such problems are not pipelined */
#define MTP_FLAG_COST_ENTROPY 0x10u /* every selection also computes the cost entropy of
                                       Sec. 4.1 over all B candidates (mtp_cost_entropy) */
#define MTP_FLAG_NO_PIPELINE 0x8u /* mtp_plan_step makes each iteration's candidates in
                                     full on the critical path instead of preparing parts
                                     of the next iteration's during the rollout (results
                                     are the same bits either way) */

/* One planning problem (Sec. 2.1 problem statement, Alg. 2 inputs, Table 3
 * hyper-parameters).  Plain data; mtp_create copies it. */
typedef struct mtp_problem {
  /* system and horizon (Sec. 2.1, Eq. 2) */
  int32_t dyn;        /* mtp_dyn */
  int32_t ctrl_dim;   /* n: point mass k, chain L, legged L-1 */
  int32_t state_dim;  /* d: point mass 2k, chain 2L, legged 2(L+2) */
  int32_t horizon;    /* H (the paper's T) */
  float dt;
  float u_min[MTP_MAX_CTRL], u_max[MTP_MAX_CTRL]; /* control box U (Def. 1) */
  /* planner (Alg. 2) */
  int32_t M, N;       /* graph layers and nodes per layer */
  int32_t B, E;       /* candidates and elites */
  double beta;        /* mixing rate in [0, 1] */
  double lambda;      /* softmax temperature > 0 */
  double alpha;       /* smoothing in [0, 1) */
  double sigma_min;   /* spread floor > 0 */
  double mu_init, sigma_init; /* initial mean and spread (constant over H, n) */
  int32_t interp;     /* mtp_interp */
  int32_t bspline_degree; /* p >= 0, M >= p + 1 */
  int32_t time_mapping;   /* mtp_time_mapping */
  int32_t update_rule;    /* mtp_update_rule */
  int32_t dr_mode;        /* mtp_dr_mode */
  int32_t R;              /* models for MTP_DR_SHARED (1..64) */
  float dr_lo, dr_hi;     /* randomisation scale range, e.g. 0.8 .. 1.2 */
  uint64_t seed;
  /* task model and cost */
  float target[MTP_MAX_CTRL]; /* point mass: goal (k); chain: reach target (x, y);
                                 legged: (height, forward velocity, pitch) */
  float w_target, w_obs, w_ctrl, w_term;
  int32_t n_obstacles;
  float obs_center[MTP_MAX_OBSTACLES][MTP_MAX_CTRL];
  float obs_radius[MTP_MAX_OBSTACLES];
  int32_t n_links;
  float link_mass[MTP_MAX_LINKS], link_length[MTP_MAX_LINKS];
  float gravity;
  float k_contact, c_contact, mu_friction, v_slip; /* legged ground contact */
  float w_height, w_pitch, w_vel;                  /* legged cost weights */
  uint32_t flags;     /* MTP_FLAG_* */
} mtp_problem;

typedef struct mtp_sizes {
  int32_t B, P, L, E, H, n, d, M, N;
  int32_t kernels_per_iteration; /* kernel launches of one mtp_plan_step iteration (after
                                    the first, when pipelined) */
  int32_t pipelined;             /* mtp_plan_step prepares each next iteration's graph rows
                                    (1) or graph rows and local draws (2) on the SMs its
                                    rollout leaves idle; 0: not pipelined */
} mtp_sizes;

/* Device buffers owned by a handle (valid until mtp_destroy).  After
 * mtp_plan_step they hold the last iteration's candidates and results.  A
 * pipelined handle alternates between two candidate buffers, so U is the
 * buffer of the latest iteration as of this call: query it again after each
 * mtp_plan_step. */
typedef struct mtp_buffers {
  float* U;        /* (B, H, n) */
  float* cost;     /* (B) */
  int32_t* elite;  /* (E), ascending cost, ties by index */
  double* weight;  /* (E) softmax weights */
  double* mu;      /* (H, n) FP64 mean */
  double* sigma;   /* (H, n) FP64 spread */
  float* ustar;    /* (n) */
  uint32_t* iter;  /* device iteration counter */
} mtp_buffers;

/* One planning problem's resident state.  A handle is used by one host
 * thread at a time (calls on it are not synchronised with one another), and
 * its work on the GPU is ordered by the streams the caller passes: calls on
 * different streams must be ordered by the caller.  Different handles are
 * independent. */
typedef struct mtp_handle mtp_handle;

/* sizeof(mtp_problem) as compiled into the library, so a binding can check
 * that its mirror of the struct has the same layout. */
size_t mtp_problem_bytes(void);

/* Validates and copies `problem`, allocates the handle's device state on the
 * current CUDA device (mean and spread initialised to mu_init / sigma_init,
 * iteration counter 0) and precomputes the interpolation tables.
 * Errors: MTP_ERR_INVALID_ARG (bad field; see mtp_last_error(NULL)),
 * MTP_ERR_OUT_OF_MEMORY, MTP_ERR_CUDA.  Synchronous. */
mtp_status mtp_create(const mtp_problem* problem, mtp_handle** out);

/* Frees everything the handle owns.  Synchronises the handle's device. */
mtp_status mtp_destroy(mtp_handle* h);

/* Text of the last error on this handle (or of the last failed mtp_create in
 * this thread when h is NULL).  Valid until the next call on the handle. */
const char* mtp_last_error(const mtp_handle* h);

mtp_status mtp_get_sizes(const mtp_handle* h, mtp_sizes* out);
mtp_status mtp_get_buffers(const mtp_handle* h, mtp_buffers* out);

/* Def. 1 and Alg. 1 (tensor sampling for iteration `iter`): writes the graph
 * d_Z (M, N, n), the path indices d_idx (P, M) and the gathered waypoints
 * d_C (P, M, n).  Any output may be NULL.  Indices are bit-exact functions of
 * (seed, iter). */
mtp_status mtp_sample_tensor(mtp_handle* h, uint32_t iter, float* d_Z, int32_t* d_idx,
                             float* d_C, void* stream);

/* Def. 2 / Def. 3 / straight lines: interpolates `P` waypoint sets d_C
 * (P, M, n) into d_U (P, H, n), clamped to the control box. */
mtp_status mtp_interpolate(mtp_handle* h, const float* d_C, int32_t P, float* d_U, void* stream);

/* Alg. 2 local sampling for iteration `iter`: writes rows [0, L) of d_U
 * (B, H, n) with mu + sigma * eps (eps standard normal, Box-Muller) and row
 * B-1 with mu, from the handle's current mean and spread; clamped. */
mtp_status mtp_sample_local(mtp_handle* h, uint32_t iter, float* d_U, void* stream);

/* Alg. 2 sampling in one launch: all B rows of d_U (B, H, n) for iteration
 * `iter` (local samples, interpolated graph paths, the mean), clamped. */
mtp_status mtp_generate_candidates(mtp_handle* h, uint32_t iter, float* d_U, void* stream);

/* Alg. 2 batch rollout and cost (Eq. 2) of candidates row0 .. row0+rows-1:
 * d_U points at row row0 of a (B, H, n) array, d_x0 is the start state (d),
 * d_cost receives `rows` costs.  Model randomisation uses (iter, candidate
 * index) so a candidate's cost does not depend on which rows are requested.
 * With MTP_DR_SHARED the cost is the mean over the R models.  Non-finite
 * costs are written as +inf. */
mtp_status mtp_rollout_cost(mtp_handle* h, uint32_t iter, const float* d_x0, const float* d_U,
                            int32_t row0, int32_t rows, float* d_cost, void* stream);

/* Like mtp_rollout_cost for one candidate `row`, also writing its state
 * trajectory d_X (H+1, d) in the paper's state coordinates. */
mtp_status mtp_rollout_states(mtp_handle* h, uint32_t iter, const float* d_x0,
                              const float* d_Urow, int32_t row, float* d_X, float* d_cost,
                              void* stream);

/* Alg. 2 elite selection and update: top-E of d_cost (B) in (cost, index)
 * order into d_elite (E, may be NULL), softmax weights, FP64 weighted mean
 * and spread of those rows of d_U (B, H, n), floor, smoothing; updates the
 * handle's mean and spread and writes u* = U[elite[0], 0, :] to d_ustar (n,
 * may be NULL). */
mtp_status mtp_elite_update(mtp_handle* h, const float* d_cost, const float* d_U,
                            int32_t* d_elite, float* d_ustar, void* stream);

/* `iters` full planner iterations (Alg. 2 loop body) from start state d_x0
 * (d) using and advancing the handle's iteration counter; writes the last
 * iteration's u* to d_ustar (n).  Replays a captured CUDA graph unless
 * MTP_FLAG_NO_GRAPH is set.  On a pipelined handle (mtp_sizes.pipelined)
 * each iteration also prepares the next iteration's graph rows (and, with
 * enough idle SMs, its local draws) on a second stream, on the SMs the
 * rollout leaves idle, and the next iteration (in this call or the next,
 * unless mtp_set_state or a batch run changed the iteration counter in
 * between) only makes or finishes its local rows and mean row.  The results
 * are the same bits as without the pipeline. */
mtp_status mtp_plan_step(mtp_handle* h, const float* d_x0, int32_t iters, float* d_ustar,
                         void* stream);

/* mtp_plan_step from host memory: copies h_x0 (d floats) to the device,
 * plans, copies u* back to h_ustar (n floats) and synchronises `stream`. */
mtp_status mtp_plan_step_host(mtp_handle* h, const float* h_x0, int32_t iters, float* h_ustar,
                              void* stream);

/* Warm start between control steps: shifts mean and spread k steps earlier
 * and repeats the last row (the paper leaves this open). */
mtp_status mtp_shift(mtp_handle* h, int32_t k, void* stream);

/* Sec. 4.1 rollout-cost entropy of the latest selection, a diagnostic of how
 * spread the candidates' costs are: H = -sum_b p_b log p_b over all B
 * candidates with p_b proportional to exp(-J_b / lambda) (the paper prints
 * exp(J_b); the sign is read so that low costs weigh most, as in the update).
 * Computed by the selection kernel (FP32 weights, FP64 sums) only for
 * problems created with MTP_FLAG_COST_ENTROPY, else MTP_ERR_INVALID_ARG.
 * Synchronises the device. */
mtp_status mtp_cost_entropy(mtp_handle* h, double* h_entropy);

/* Device-side failures since the last call: the rollouts stage their controls
 * through shared memory with bulk copies and wait for them with a bounded
 * wait (about two seconds); a wait that gives up marks the handle and scores
 * its candidates +inf instead of hanging the GPU.  Synchronises the device,
 * then returns MTP_ERR_TIMEOUT (and clears the mark) if that happened in any
 * of the handle's rollouts (alone or in a batch), else MTP_OK. */
mtp_status mtp_device_status(mtp_handle* h);

/* Self-test of the bounded device waits: one warp waits on an mbarrier whose
 * expected bytes never arrive, with a time limit of limit_s seconds (0 <
 * limit_s <= 10) of the GPU's global timer.  The wait can only end by giving
 * up, so a working library returns MTP_ERR_TIMEOUT after about limit_s, with
 * the device still usable; *waited_s (may be NULL) gets the host-measured
 * time.  MTP_OK would mean the wait saw bytes that were never sent;
 * MTP_ERR_CUDA a launch or copy failure.  Synchronises the device; allocates
 * 4 bytes of device memory for the result. */
mtp_status mtp_selftest_bounded_wait(double limit_s, double* waited_s);

/* Checkpoint / resume of the planner state: FP64 mean and spread (H, n) and
 * the iteration counter.  Synchronous. */
mtp_status mtp_get_state(mtp_handle* h, double* h_mu, double* h_sigma, uint32_t* h_iter);
mtp_status mtp_set_state(mtp_handle* h, const double* h_mu, const double* h_sigma,
                         uint32_t iter);

/* Per-stage device time: with profiling on, mtp_plan_step records CUDA
 * events around each stage (generate, rollout, select, update), inside the
 * captured graph unless MTP_FLAG_NO_GRAPH is set, and then waits for the
 * step so the events can be read.  mtp_stage_times returns the summed
 * milliseconds of the four stages and the number of iterations recorded
 * since the last read, then resets.  On a pipelined handle "generate" is the
 * part on the critical path (finishing the local rows and the mean row, or
 * the whole generation when the draws were not prepared); mtp_stage_times5
 * adds, fifth, the time of the next iteration's preparation, which runs on a
 * second stream during the rollout (0 when not pipelined). */
mtp_status mtp_set_profiling(mtp_handle* h, int32_t enable);
mtp_status mtp_stage_times(mtp_handle* h, double* ms4, int32_t* iterations);
mtp_status mtp_stage_times5(mtp_handle* h, double* ms5, int32_t* iterations);

/* Batched planning over many handles (uneven sizes, point masses and chains
 * mixed).  One iteration is one CUDA graph: the candidates of every
 * (dynamics, control dimension) group made on the group's own stream, the
 * rollouts either per group on those streams or in persistent launches over
 * the whole batch (mtp_batch_set_rollout_mode; the autotuner picks), one
 * selection block per instance, one update launch per group.  This is the GPU form of the paper's vectorised
 * planning of many model instances (Sec. 3.3, Sec. 4 practical settings);
 * each instance computes exactly what mtp_plan_step computes for it alone.
 * The handles must stay alive while the batch exists; their states advance. */
typedef struct mtp_batch mtp_batch;

/* Builds the device tables of a batch over `count` distinct handles that
 * live on the current device.  Errors: MTP_ERR_INVALID_ARG, MTP_ERR_CUDA,
 * MTP_ERR_OUT_OF_MEMORY (text in mtp_last_error(NULL)). */
mtp_status mtp_batch_create(mtp_handle* const* handles, int32_t count, mtp_batch** out);
mtp_status mtp_batch_destroy(mtp_batch* b);

/* Packed layouts: x0_offset[i] .. x0_offset[i+1] is instance i's start state
 * in the packed x0 vector, ustar_offset likewise for u*.  Each array has
 * count + 1 entries (the last is the total length). */
mtp_status mtp_batch_layout(const mtp_batch* b, int32_t* x0_offset, int32_t* ustar_offset);

/* A batch with device tables for up to `capacity` instances and none filled
 * yet: mtp_batch_fill gives it its instances, as often as needed, without
 * allocating.  Errors as mtp_batch_create. */
mtp_status mtp_batch_reserve(int32_t capacity, mtp_batch** out);

/* Replaces the batch's instances by `count` (1 .. capacity) distinct handles
 * on the batch's device: one host-to-device copy of the packed tables on
 * `stream`.  The handles must stay alive while they are in the batch.  Work
 * of this batch enqueued before the fill must be on `stream` too (or have
 * finished).  Errors: MTP_ERR_INVALID_ARG, MTP_ERR_CUDA. */
mtp_status mtp_batch_fill(mtp_batch* b, mtp_handle* const* handles, int32_t count, void* stream);

/* `iters` iterations of every instance from the packed start states d_x0;
 * writes the packed last-iteration u* to d_ustar.  Stream-ordered.  The
 * first call after a fill launches its kernels directly; later calls with
 * the same instances replay a captured CUDA graph. */
mtp_status mtp_batch_plan_step(mtp_batch* b, const float* d_x0, int32_t iters, float* d_ustar,
                               void* stream);

/* Picks the rollout tile of each (dynamics, dimension) group by timing its
 * rollout launch (best of three) for every choice: candidates per block (32,
 * 64 or 128) times the horizon chunk of the staged control loads (0: direct
 * loads; 4 or 8 steps of every candidate's controls copied at once into
 * shared memory by bulk copies, when every member's rows allow it: 16-byte
 * aligned, H * n a multiple of 4, one model per candidate), and for point
 * masses also two candidates per thread (64 per warp, direct loads).  The
 * legged group keeps its fixed tile.  Writes (dynamics, dimension, block,
 * chunk, candidates per thread) to tiles_out (5 * groups entries, may be
 * NULL) and the number of groups to n_groups.  Then it picks the rollout
 * mode (mtp_batch_set_rollout_mode) by timing whole iterations in each mode,
 * each captured as the CUDA graph that mtp_batch_plan_step replays (best of
 * three replays after one untimed one), with every instance's planner state
 * (mean, spread, iteration counter) saved before and restored after, so the
 * instances' next iteration is the one they would have run.  Synchronous;
 * overwrites the handles' candidate, cost, elite and u* buffers, and
 * allocates (and frees) device memory for the saved states.  Results do not
 * depend on the tile or the mode. */
mtp_status mtp_batch_autotune(mtp_batch* b, int32_t* tiles_out, int32_t* n_groups, void* stream);

/* How a batch runs its rollouts.
 * MTP_BATCH_ROLLOUT_GROUPS: each (dynamics, dimension) group's rollout is its
 *   own launch, in that group's chain of launches on its stream (groups
 *   overlap one another).
 * MTP_BATCH_ROLLOUT_PERSISTENT_STAGED / _DIRECT: the rollouts of every point
 *   mass (up to 16 axes) and every chain (up to 9 links) of the batch run in
 *   one persistent launch, after all instances' candidates are made: each
 *   warp takes warp tiles of 32 candidates of one instance from a device
 *   counter, group by group (the longest group first, within a group the
 *   longest expected rollout first: H times the group's time per step),
 *   with their controls staged through shared memory 4 steps at a
 *   time where the instance's rows allow it (_STAGED) or loaded directly
 *   (_DIRECT).  Legged robots and longer chains keep their own launches
 *   beside it.  The launch is counted as one kernel by mtp_batch_launches.
 * MTP_BATCH_ROLLOUT_PERSISTENT_SPLIT: the same with staged tiles, in two
 *   persistent launches split at a group boundary near 65 % of the expected
 *   rollout work: the first starts as soon as its groups' candidates are made
 *   (their generation on high-priority streams) and leaves one CTA per SM to
 *   the second part's generation, which overlaps it; the second starts when
 *   its own candidates are made.
 * Results are the same bits in every mode.  The mode takes effect at the
 * next mtp_batch_plan_step (captured graphs are dropped).  Errors:
 * MTP_ERR_INVALID_ARG for an unknown mode. */
#define MTP_BATCH_ROLLOUT_GROUPS 0
#define MTP_BATCH_ROLLOUT_PERSISTENT_STAGED 1
#define MTP_BATCH_ROLLOUT_PERSISTENT_DIRECT 2
#define MTP_BATCH_ROLLOUT_PERSISTENT_SPLIT 3
mtp_status mtp_batch_set_rollout_mode(mtp_batch* b, int32_t mode);

/* The batch's current rollout mode, and (ms4, 4 entries, one per mode, may
 * be NULL) the autotuner's iteration time of each mode in milliseconds (0
 * where it has not timed that mode; modes that cover no instance are not
 * timed). */
mtp_status mtp_batch_rollout_mode(const mtp_batch* b, int32_t* mode, double* ms4);

/* Device time of the persistent rollout launch alone (the covered groups'
 * rollouts, Alg. 2 rollout fused with the cost, Eq. 2) on `stream`, with
 * staged tiles unless the batch's mode is MTP_BATCH_ROLLOUT_PERSISTENT_DIRECT
 * (one launch over all covered instances in every mode), averaged over `reps` launches timed with CUDA
 * events: *ms (0 when the launch covers no instance).  *steps receives the
 * rollout steps (sum of B * H) it covers.  Synchronous; overwrites the
 * covered handles' cost buffers (with the same values). */
mtp_status mtp_batch_persistent_time(mtp_batch* b, int32_t reps, double* ms, int64_t* steps, void* stream);

/* mtp_shift(h, k) of every instance of the batch in one launch. */
mtp_status mtp_batch_shift(mtp_batch* b, int32_t k, void* stream);

/* Kernel launches one mtp_batch_plan_step(b, ..., iters, ...) issues: per
 * iteration, each (dynamics, dimension) group's graph, graph-path, local-row,
 * rollout, selection and update launches that have work (in a persistent
 * rollout mode the covered groups' rollouts count as one launch), plus the
 * scatter of the start states and the gather of u* once per call. */
mtp_status mtp_batch_launches(const mtp_batch* b, int32_t iters, int32_t* launches);

/* Device time of each group's rollout launch (Alg. 2 rollout fused with the
 * cost, Eq. 2) run alone on `stream` with its current tile, averaged over
 * `reps` launches timed with CUDA events: ms_out[g] (may be NULL).
 * info_out (8 per group, may be NULL): dynamics, dimension (point-mass axes
 * or links), candidates per block, instances, candidates (sum of B), rollout
 * steps (sum of B * H), the horizon chunk of staged control loads (0: direct
 * loads) and candidates per thread.  *n_groups is the group count; max_groups
 * must be at least that when an output array is given.  Synchronous;
 * overwrites the handles' cost buffers. */
mtp_status mtp_batch_rollout_times(mtp_batch* b, int32_t reps, double* ms_out, int32_t* info_out,
                                   int32_t max_groups, int32_t* n_groups, void* stream);

/* Device bytes a handle for `problem` uses, each allocation rounded up to
 * 512 bytes (the candidate tensor U dominates: B * H * n floats).  A
 * pipelined problem counts the second candidate buffer, which the first
 * single-instance mtp_plan_step allocates (a handle planned only in batches
 * never does; MTP_FLAG_NO_PIPELINE leaves it out).  The serving layer admits
 * robots against a memory budget with it, with the pipeline off.
 * MTP_ERR_INVALID_ARG when the problem does not validate. */
mtp_status mtp_problem_device_bytes(const mtp_problem* problem, uint64_t* bytes);

/* Re-planning server (continuous batching).  Robots are registered with
 * their planning problem; a client submits a robot's current state and polls
 * for its control.  A worker thread gathers up to max_batch robots that have
 * a queued request and no request in flight (a robot's next plan starts from
 * the state its previous one left), oldest request first, and runs them as
 * one batched planner cycle: iters_per_request iterations (Alg. 2), u* back
 * to pinned host memory, then the warm-start shift.  Two cycles may be in
 * flight on separate streams with disjoint robots.  Each request's u*, and
 * each robot's planner state after it, are exactly what mtp_plan_step
 * (and mtp_shift) give on the robot's handle alone. */
typedef struct mtp_server mtp_server;

typedef struct mtp_server_config {
  int32_t max_batch;          /* robots per cycle (>= 1) */
  int32_t iters_per_request;  /* planner iterations per request (>= 1) */
  int32_t shift_after;        /* warm-start shift k after each request (>= 0) */
  int32_t max_queue;          /* queued requests per robot before submits are refused (>= 1) */
  int32_t max_robots;         /* registrations before they are refused (>= 1) */
  uint64_t memory_budget;     /* device bytes the robots may take; 0: 90% of the
                                 free device memory when the server is created */
} mtp_server_config;

typedef struct mtp_server_stats {
  uint64_t submitted, completed, cycles, planned;  /* planned: robot-plans run */
  int32_t queued, in_flight, robots, failed;       /* failed: 1 after a device error */
  uint64_t bytes_admitted;
  double p50_latency_s, p99_latency_s;  /* submit -> result ready, completed requests */
} mtp_server_stats;

/* Creates the server on the current device and starts its worker thread.
 * Allocates everything a cycle needs now (tables, pinned staging).  Errors:
 * MTP_ERR_INVALID_ARG, MTP_ERR_OUT_OF_MEMORY, MTP_ERR_CUDA (text in
 * mtp_last_error(NULL)). */
mtp_status mtp_server_create(const mtp_server_config* cfg, mtp_server** out);

/* Stops the worker after the cycles in flight, drops queued requests and
 * frees everything, the robots' handles included.  No other thread may call
 * into the server during or after this call.  Every other server call may be
 * made from any thread. */
mtp_status mtp_server_destroy(mtp_server* srv);

/* Admits a robot: creates its planner handle when its footprint
 * (mtp_problem_device_bytes) fits the remaining budget and the robot count
 * is below max_robots; otherwise MTP_ERR_ADMISSION and nothing is
 * allocated.  Writes the robot's id (0, 1, ...). */
mtp_status mtp_server_register(mtp_server* srv, const mtp_problem* problem, int32_t* robot);

/* Queues a plan request for `robot` from host state h_x0 (state_dim
 * floats, copied) and writes its ticket (> 0).  MTP_ERR_ADMISSION when the
 * robot already has max_queue requests queued; MTP_ERR_CUDA after a device
 * error; MTP_ERR_INVALID_ARG for an unknown robot. */
mtp_status mtp_submit(mtp_server* srv, int32_t robot, const float* h_x0, uint64_t* ticket);

/* Result of a ticket: copies u* (ctrl_dim floats) to h_ustar and releases
 * the ticket (MTP_OK).  When it is not ready: waits up to timeout_s
 * seconds, then MTP_ERR_NOT_READY (timeout_s == 0) or MTP_ERR_TIMEOUT.
 * MTP_ERR_INVALID_ARG for a ticket never issued or already released;
 * MTP_ERR_CUDA if the server failed. */
mtp_status mtp_poll(mtp_server* srv, uint64_t ticket, float* h_ustar, double timeout_s);

/* mtp_submit for `count` requests in order: robots[i]'s start state follows
 * the previous request's in h_x0 (state_dim floats each).  Stops at the first
 * request refused; *accepted (may be NULL) is the number queued, whose
 * tickets are in tickets[0 .. accepted).  Returns that refusal's status, or
 * MTP_OK. */
mtp_status mtp_submit_many(mtp_server* srv, int32_t count, const int32_t* robots, const float* h_x0,
                           uint64_t* tickets, int32_t* accepted);

/* mtp_poll for `count` tickets, sharing one deadline timeout_s seconds
 * away: status[i] is ticket i's mtp_poll status and its u* goes to
 * h_ustar + i * stride (stride >= its ctrl_dim).  *ready (may be NULL) is
 * the number of MTP_OK entries.  Returns MTP_OK unless an argument is bad. */
mtp_status mtp_poll_many(mtp_server* srv, int32_t count, const uint64_t* tickets, float* h_ustar,
                         int32_t stride, double timeout_s, int32_t* status, int32_t* ready);

mtp_status mtp_server_get_stats(mtp_server* srv, mtp_server_stats* out);

/* Text of the server's last error (worker or call). */
const char* mtp_server_last_error(const mtp_server* srv);

/* Elite selection and update for callers that cannot allocate device memory.
 *
 * mtp_create allocates the handle's buffers with cudaMalloc.  Some callers
 * cannot do that: code that runs inside a memory pool or arena it does not
 * own, or a process whose device allocations are locked once it starts
 * serving.  This entry point does the same work as mtp_elite_update (top-E
 * of d_cost, softmax or plain-CEM weights, FP64 mean and spread of those rows
 * of d_U, floor, smoothing, u*) without a handle and without allocating:
 * the caller passes every input and output -- costs d_cost (B), candidates
 * d_U (B, H, n), the FP64 mean d_mu and spread d_sigma (H, n, updated in
 * place), and optionally d_elite (E) and d_ustar (n) -- and the intermediate
 * results live in one fixed array in device memory that every GPU loading
 * the library keeps until the process exits.  The paper has no counterpart;
 * this is a deployment convenience.
 *
 * Limits: E <= MTP_NOALLOC_MAX_ELITES, H * n <= MTP_NOALLOC_MAX_HN, and B as
 * for mtp_elite_update; larger requests return MTP_ERR_INVALID_ARG (text in
 * mtp_last_error(NULL)).  The first call on each device looks up the array's
 * device address and sets a kernel attribute; make that first call before
 * any stream capture.  All calls share the one array, so calls whose work
 * overlaps on the GPU (different streams, or threads without ordering) race
 * and must be serialised by the caller.  No call allocates or frees memory. */
#define MTP_NOALLOC_MAX_ELITES 2048
#define MTP_NOALLOC_MAX_HN 4096
mtp_status mtp_elite_update_noalloc(const float* d_cost, const float* d_U, int32_t B, int32_t E,
                                    int32_t H, int32_t n, double lambda, double alpha,
                                    double sigma_min, int32_t update_rule, double* d_mu,
                                    double* d_sigma, int32_t* d_elite, float* d_ustar,
                                    void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MTP_H */
