/*
 * stp.h - C ABI of the GB300 (sm_103a) batched space-time Extend library for
 * ST-pRRTC ("ST-pRRTC: Parallel Space-Time RRT-C with Adaptive Goal-Time
 * Forests").
 *
 * The library plans one single-goal query at a time (Sec. "Problem
 * Formulation": C subset of R^d with the Euclidean metric, velocity bound
 * v_max, horizon [0,H], moving obstacles with known trajectories) with the
 * interval-root planner (Algorithms 1-2) or the root-recycling planner
 * (Algorithm 3). Every step of a planning iteration runs in the library's CUDA
 * kernels; there is no CPU fallback: when no CUDA device is usable, every call
 * that would compute returns STP_ERR_CUDA.
 *
 * Conventions
 *   - All calls return an stp_status; none aborts the process.
 *   - Input arrays are read during the call and copied; the caller keeps
 *     ownership. Output buffers are owned by the caller.
 *   - Multi-dimensional arrays are row-major and contiguous.
 *   - Precision: stp_params.precision selects the arithmetic of the device
 *     path: 0 = FP32 (the fast path), 1 = FP64 (deterministic-parity mode).
 *     Arrays typed `const void *` below hold float in FP32 mode and double in
 *     FP64 mode.
 *   - A problem is not thread-safe; distinct problems may be used from
 *     distinct threads.
 */
#ifndef STP_H
#define STP_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stp_problem stp_problem; /* opaque, owned by the library */

typedef enum {
    STP_OK = 0,
    STP_ERR_INVALID = 1,   /* an argument violates the documented contract   */
    STP_ERR_CAPACITY = 2,  /* a tree arena or table would overflow           */
    STP_ERR_CUDA = 3,      /* no usable device, or a CUDA call failed         */
    STP_ERR_TIMEOUT = 4,   /* a bounded device wait gave up                   */
    STP_NO_SOLUTION = 5    /* budget exhausted without a solution (Alg. 2, 3) */
} stp_status;

/* Robot (Sec. "Problem Formulation": C subset of R^d, Euclidean D, v_max).
 *   dof        2..7. With arm = 0 the robot is a point (or sphere set) translated
 *              by q (q0, q1[, q2]) in the plane/space; with arm = 1 it is a
 *              serial chain in standard DH form.
 *   dh         [dof][4] rows (a, alpha, d, theta_offset); frame j+1 =
 *              frame j * Rz(q_j + theta_offset) Tz(d) Tx(a) Rx(alpha). NULL if
 *              arm = 0.
 *   q_lo,q_hi  [dof] configuration box; states outside it are in collision.
 *   spheres    [n_spheres][5]: frame index (0 = base, j = after joint j), local
 *              centre x, y, z, radius. 1 <= n_spheres <= 64.
 *   v_max      speed bound in the Euclidean metric of C (Eq. minimum-travel-time). */
typedef struct {
    int dof;
    int arm;
    const double *dh;
    const double *q_lo;
    const double *q_hi;
    int n_spheres;
    const double *spheres;
    double v_max;
} stp_robot;

/* Moving obstacles: spheres on piecewise-linear trajectories, positions
 * interpolated at each absolute query time (Sec. "Simulation Protocol");
 * before the first and after the last waypoint an obstacle holds that waypoint.
 *   n_obs      0..128, n_way 1..8.
 *   radius     [n_obs]
 *   way        [n_obs][n_way][4]: t, x, y, z (z = 0 for planar problems);
 *              times strictly increasing per obstacle.
 * Collision predicate: a robot sphere and an obstacle collide iff
 * |p - o|^2 < (r + r_o)^2 (touching is free). */
typedef struct {
    int n_obs;
    int n_way;
    const double *radius;
    const double *way;
} stp_obstacles;

/* Planner settings.
 *   variant        0 interval root (Algorithm 2), 1 root recycling (Algorithm 3),
 *                  2 no recycling (the paper's allocation ablation: the roots of
 *                  Algorithm 3's initialisation stay fixed; roots at T >= U turn
 *                  inactive and are never replaced).
 *   n_roots        N: interval-root groups or recycling slots, 1..128.
 *   ext_per_iter   W: GPU workers (one Extend each) per iteration, 1..8192.
 *   max_iters      iteration budget (>= 1). budget_ms > 0 adds a wall-clock
 *                  budget checked between graph launches.
 *   eta            range: steering step in rho (interval root, Algorithm 1) or
 *                  configuration step (root recycling, Eq. max-speed-extension).
 *   edge_res       check resolution: an edge is checked at
 *                  c = max(1, ceil(max(D, v_max |dt|) / edge_res - 1e-3))
 *                  points j/c, j = 1..c (the paper leaves the resolution rule
 *                  open; the 1e-3 slack keeps c stable when the length is an
 *                  exact multiple of edge_res, so the spacing may exceed
 *                  edge_res by at most 0.1 % of one step).
 *   env_dt         environment grid step dt for goal checks
 *                  (Eq. goal-time-lower-bound).
 *   p_new, p_guided  Sec. "Interval Root" (paper default 0.05 / 0.95).
 *   t_max          horizon H; arrival times lie in [0, H].
 *   seed, problem_id  Philox4x32-10 key and counter word 3.
 *   precision      0 FP32, 1 FP64.
 *   learned        0 plain sampling; 1 learned sampling branch: a proposal from
 *                  the proposal network (stp_set_proposal) guides 90 % of the
 *                  workers (the rest sample as with 0); stp_plan and
 *                  stp_batch_plan return STP_ERR_INVALID until one is set.
 *   capacity       nodes per tree arena; 0 = max_iters * ceil(W/2) + 2 (worst case).
 *   iters_per_graph  iterations captured per CUDA graph launch; 0 = 8.
 *   t_offset       absolute time of the query's local time 0 (>= 0): obstacle
 *                  trajectories are shifted by it, as when a goal sequence is
 *                  planned query by query (Sec. "Problem Formulation": a
 *                  query starts its own clock at zero, sees the obstacles
 *                  moved along by the absolute time at which it starts, and
 *                  gets what is left of the horizon, passed as t_max).
 *   continuous     0 discrete edge validation at edge_res; 1 closed-form
 *                  validation for point robots (arm = 0 only): between the
 *                  edge's end times and the obstacle waypoint times inside
 *                  them, robot spheres and obstacles move linearly, so the
 *                  exact minimum distance of every pair is the distance from
 *                  the origin to a segment. Not available in batches.
 *   self_collision 0 off; 1 (arms only) also test the robot's own spheres with
 *                  the same predicate: pairs on frames at least two apart,
 *                  except pairs that already overlap at q = 0 (treated as
 *                  permanent contacts). Not in the paper's queries.
 *   launch_mode    STP_LAUNCH_DEFAULT (0) = STP_LAUNCH_STEPS (1): one kernel
 *                  per step of the iteration, iterations captured into CUDA
 *                  graphs (iters_per_graph per graph); STP_LAUNCH_PERSISTENT
 *                  (2): the whole plan (every step of every iteration) in one
 *                  persistent, cooperative kernel launch whose steps are
 *                  separated by device-wide barriers (each wait bounded by 1 s).
 *                  Both run the same step code and take the same decisions.
 *                  Closed-form validation (continuous = 1) always uses steps.
 *   persist_ctas   CTAs of the persistent launch; 0 = every resident CTA
 *                  (SMs x CTAs per SM). */
#define STP_LAUNCH_DEFAULT 0
#define STP_LAUNCH_STEPS 1
#define STP_LAUNCH_PERSISTENT 2
typedef struct {
    int variant;
    int n_roots;
    int ext_per_iter;
    int max_iters;
    double budget_ms;
    double eta;
    double edge_res;
    double env_dt;
    double p_new;
    double p_guided;
    double t_max;
    unsigned long long seed;
    unsigned int problem_id;
    int precision;
    int learned;
    int capacity;
    int iters_per_graph;
    double t_offset;
    int continuous;
    int self_collision;
    int launch_mode;
    int persist_ctas;
} stp_params;

/* Per-call statistics filled by stp_plan. Times are GPU times (CUDA events /
 * device global timer), excluding problem upload (Sec. "Simulation Protocol"). */
typedef struct {
    int iterations;
    int first_solution_iter;      /* -1 if none */
    long long nodes;              /* inserted extensions (not counting roots) */
    long long edges_validated;    /* extension edges sent to edge validation */
    long long bridges_validated;  /* bridge edges sent to edge validation */
    long long root_checks;        /* sampled goal roots checked (interval root) */
    long long check_points;       /* check points evaluated (work counter: with early exit it
                                     depends on scheduling, not only on the inputs) */
    long long pair_tests;         /* robot-sphere / obstacle pair tests executed (same caveat) */
    double first_solution_ms;     /* device time from plan start to the first solution */
    double plan_ms;               /* device time of the whole plan */
    double U;
    double C;
    long long nn_evals;           /* NN scan: (query, vertex) key evaluations (Eq. space-time-metric) */
    long long nn_nodes;           /* NN scan: vertices of the scanned sets, once per set and iteration */
    long long bridge_evals;       /* bridge scan: (query, vertex) rank evaluations */
    long long bridge_nodes;       /* bridge scan: vertices of the scanned sets, once per set and iteration */
    double step_ms;               /* device time of every GPU operation of the call (state reset, all
                                     iterations, path extraction, statistics copy): CUDA events on the
                                     problem's stream around them, so host-side gaps after the work
                                     (synchronisation, return) are not counted; 0 without a plan */
} stp_stats;

/* Create a problem: validates and copies robot, obstacles, start, goal and
 * params to the device, runs the goal-time grid checks (Eq.
 * goal-time-lower-bound) and sizes the tree arenas.
 *   q_start, q_goal  [dof]. *out receives the handle (NULL on error).
 * Errors: STP_ERR_INVALID (bad sizes/values), STP_ERR_CUDA (no device or
 * allocation failed), STP_ERR_CAPACITY (arena size overflow). */
stp_status stp_create_problem(const stp_robot *robot, const stp_obstacles *obstacles,
                              const double *q_start, const double *q_goal,
                              const stp_params *params, stp_problem **out);

/* Run the planner from a fresh state (trees reset) for the configured budget.
 * Algorithm 2 ends early when L_g >= min(H, U). Outputs (any may be NULL):
 *   arrival_U, length_C  incumbent (U, C), lexicographic (Sec. "Space-Time
 *                        pRRTC"); +inf if none.
 *   path                 caller buffer [cap][dof+1] of (q..., t) states from
 *                        (q_s, 0) to (q_g, U); *n_path receives the count.
 * Returns STP_OK when a solution exists, STP_NO_SOLUTION when the budget ran
 * out without one (Algorithms 2, 3), STP_ERR_CAPACITY if path exceeds cap or
 * an arena overflowed, STP_ERR_TIMEOUT if a bounded device wait gave up. */
stp_status stp_plan(stp_problem *p, double *arrival_U, double *length_C, int *n_path, double *path,
                    int cap, stp_stats *stats);

/* Edge validation on its own (collision kernel; Sec. "Simulation Protocol":
 * obstacles interpolated at each absolute query time): for each edge
 * (qa[e], ta[e]) -> (qb[e], tb[e]) check points j/c, j = 1..c.
 *   qa, qb       [n_edges][dof], ta, tb [n_edges]; element type per precision.
 *   flags        bit 0 (STP_EDGES_DEVICE): all pointers (inputs and outputs) are
 *                device pointers; bit 1 (STP_EDGES_CLEARANCE): also compute the
 *                exact minimum clearance (no early exit); bit 2
 *                (STP_EDGES_NO_EARLY_EXIT): check every point even after a hit.
 *   verdict      [n_edges] output, 1 = collision-free, 0 = collides.
 *   min_clearance [n_edges] output (precision type) or NULL; requires bit 1.
 *   n_checks     [n_edges] int output or NULL: check points per edge.
 * Errors: STP_ERR_INVALID (n_edges < 0 or > 2^26, NULL arrays), STP_ERR_CUDA. */
#define STP_EDGES_DEVICE 1
#define STP_EDGES_CLEARANCE 2
#define STP_EDGES_NO_EARLY_EXIT 4
stp_status stp_check_edges(stp_problem *p, int n_edges, const void *qa, const void *ta, const void *qb,
                           const void *tb, int flags, unsigned char *verdict, void *min_clearance,
                           int *n_checks);

/* The collision-kernel launch inside the last stp_check_edges call on p:
 * device time in ms (CUDA events on the problem's stream), check points
 * evaluated and sphere-obstacle pair tests executed. Any output may be NULL. */
stp_status stp_last_validate(stp_problem *p, double *ms, long long *points, long long *pairs);

/* Kernel profiling of stp_plan. With on != 0 the captured iteration graphs
 * record a CUDA event before every kernel and after the last one, and stp_plan
 * accumulates the device time of each kernel kind over the iterations that
 * ran (the host waits after every graph launch while profiling is on). */
stp_status stp_set_profiling(stp_problem *p, int on);
/* Per-kernel totals of the last profiled stp_plan: for k < *n (at most cap):
 * names[k] (static strings), ms[k] total device time, launches[k]. */
stp_status stp_profile(stp_problem *p, int cap, const char **names, double *ms, long long *launches, int *n);

/* Decision trace of stp_plan (and of a batch created afterwards), for parity
 * tests and debugging: with max_iters > 0 every planned iteration k <
 * max_iters (clamped to the problem's max_iters) writes one record of
 * STP_TRACE_INTS ints per worker w at records[(k * W + w) * STP_TRACE_INTS]
 * describing that worker's decisions in the batch-synchronous iteration
 * (Algorithms 1-3):
 *   [0] flags: STP_TR_FWD forward worker ((w + k) even); STP_TR_SAMPLED
 *       interval root: the query-time window of Eq. conditional-query-time is
 *       non-empty, root recycling: the worker has a source tree;
 *       STP_TR_VIRTUAL the source is a new root (Algorithm 2); STP_TR_EMIT the
 *       extension edge was steered inside [0, H] and sent to validation;
 *       STP_TR_ROOT_HIT / STP_TR_EXT_HIT the sampled goal root / the extension
 *       collides (only meaningful with STP_TR_EMIT); STP_TR_INSERTED;
 *       STP_TR_BR_CAND an admissible bridge candidate exists; STP_TR_BR_EMIT it
 *       improves (U, C) and was validated; STP_TR_BR_HIT it collides;
 *       STP_TR_WINNER this worker's bridge was published; STP_TR_LEARNED the
 *       learned branch drew this worker; STP_TR_LEARNED_T its goal time came
 *       from the mixture; STP_TR_GUIDED interval root: the goal time came from
 *       the group's guided pieces (Sec. "Interval Root").
 *   [1] interval group, or recycling slot of a backward worker, else -1;
 *   [2] NN parent index (-1: virtual root or none); [3] extension check count;
 *   [4] bridge candidate arena (-1 forward tree, else backward group / slot);
 *   [5] candidate index in it; [6] bridge check count; [7] index of the
 *   inserted node (-1); [8] learned mixture component (-1); [9] interval root:
 *   the sampled goal time T as IEEE float bits, else 0.
 * max_iters = 0 turns the trace off. The buffer ([max_iters][W][10] ints) is
 * allocated here (cudaMalloc) and freed by stp_free; the next stp_plan
 * recaptures its graph. Errors: STP_ERR_INVALID, STP_ERR_CUDA. */
#define STP_TRACE_INTS 10
#define STP_TR_FWD 1
#define STP_TR_SAMPLED 2
#define STP_TR_VIRTUAL 4
#define STP_TR_EMIT 8
#define STP_TR_ROOT_HIT 16
#define STP_TR_EXT_HIT 32
#define STP_TR_INSERTED 64
#define STP_TR_BR_CAND 128
#define STP_TR_BR_EMIT 256
#define STP_TR_BR_HIT 512
#define STP_TR_WINNER 1024
#define STP_TR_LEARNED 2048
#define STP_TR_LEARNED_T 4096
#define STP_TR_GUIDED 8192
stp_status stp_set_trace(stp_problem *p, int max_iters);
/* Records of the last plan: *n_iters = iterations recorded; records may be
 * NULL (count only), else needs cap_iters >= *n_iters (STP_ERR_CAPACITY). */
stp_status stp_trace(stp_problem *p, int *records, int cap_iters, int *n_iters);

/* Edge validation that allocates nothing, for callers that cannot allocate
 * device memory while they run: for example a control loop that must not
 * block in the driver's allocator, or a host process whose device-memory
 * budget is fixed after start-up. The paper has no counterpart: this is the
 * collision batch of stp_check_edges with its per-call scratch (check counts,
 * offsets, hit flags, window counter, scan partials) taken from one static
 * device array built into the library, sized for STP_NOALLOC_MAX_EDGES edges
 * (about 1 MiB, held on every GPU that loads the library until the process
 * exits).
 *   qa, qb     [n_edges][dof] DEVICE pointers, ta, tb [n_edges] DEVICE
 *              pointers, element type per precision (as stp_check_edges).
 *   verdict    [n_edges] DEVICE output, 1 = collision-free, 0 = collides.
 * The work is queued on the problem's stream; the call does not wait for it.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) for the current device: make that first call before
 * any stream capture. Every call uses the same array, which keeps the last
 * call's contents; calls whose GPU work can overlap (other streams, threads
 * or problems without ordering between them) race on it, so the caller must
 * order them.
 * Errors: STP_ERR_INVALID (NULL pointers, n_edges < 0), STP_ERR_CAPACITY
 * (n_edges > STP_NOALLOC_MAX_EDGES), STP_ERR_CUDA. n_edges == 0 is a no-op. */
#define STP_NOALLOC_MAX_EDGES 65536
stp_status stp_check_edges_noalloc(stp_problem *p, int n_edges, const void *qa, const void *ta, const void *qb,
                                   const void *tb, unsigned char *verdict);

/* ---- Batched planning (many problems in one launch) -----------------------
 * A batch plans several FP32 problems together. STP_LAUNCH_DEFAULT (0) =
 * STP_LAUNCH_PERSISTENT (2): one persistent, cooperative kernel, captured in a
 * CUDA graph, whose CTAs form teams of team_ctas CTAs; each team takes the
 * next problem from a device work queue and plans it to the end (all
 * iterations, steps separated by team barriers), then takes the next.
 * STP_LAUNCH_STEPS (1): every kernel of an iteration covers all problems (one
 * CUDA grid dimension per problem) and iterations are captured into one CUDA
 * graph. Problems keep their own parameters (variant, N, W, budget, ...) and
 * arenas; they must stay alive while the batch exists. Problems whose start is
 * in collision, or whose start equals the goal, are resolved without
 * iterations as in stp_plan. */
typedef struct stp_batch stp_batch;
typedef struct {
    int nn_ctas;          /* steps: CTAs per problem for the NN and bridge scans; 0 = 8 */
    int validate_ctas;    /* steps: CTAs per problem for the collision kernel; 0 = 2 */
    int iters_per_graph;  /* steps: iterations per graph launch; 0 = 16 */
    int launch_mode;      /* STP_LAUNCH_DEFAULT / _PERSISTENT: work queue; STP_LAUNCH_STEPS: one kernel per step */
    int team_ctas;        /* persistent: CTAs per team (problems in flight = resident CTAs / team_ctas); 0 = 8 */
} stp_batch_params;
/* problems [n], n >= 1, all created with precision 0; params may be NULL. */
stp_status stp_batch_create(stp_problem *const *problems, int n, const stp_batch_params *params,
                            stp_batch **out);
/* Plan every problem from a fresh state. stats [n] (or NULL) receives each
 * problem's statistics (first_solution_ms is measured from the start of the
 * batch, so it includes the time a problem waited in the queue; plan_ms is
 * the problem's own plan from its start); *batch_ms the device time of the
 * whole batch. Returns STP_OK unless
 * a CUDA call failed or a problem overflowed (STP_ERR_CAPACITY). */
stp_status stp_batch_plan(stp_batch *b, stp_stats *stats, double *batch_ms);
/* Path of problem i after stp_batch_plan: [cap][dof+1]; *n_path = states. */
stp_status stp_batch_path(stp_batch *b, int i, double *path, int cap, int *n_path);
void stp_batch_free(stp_batch *b);

/* Release a problem. NULL is allowed. Waits for the problem's stream(s); its
 * device blocks, stream and executable iteration graph then go to a
 * per-process cache (up to 4 GiB of idle blocks, 8 idle graphs) that later
 * problems reuse, so short-lived problems cost no cudaMalloc/cudaFree, and a
 * later problem whose iteration graph has the same topology updates an idle
 * graph with its own kernel parameters instead of instantiating one. */
void stp_free(stp_problem *p);
/* Return every cached device block, stream and executable graph to the driver
 * (thread-safe; call when no problem created before it is still in use by
 * another thread). */
void stp_release_cached(void);

/* Use this CUDA stream (a cudaStream_t passed as void*) for every later call
 * on p; NULL selects the library's own stream. */
stp_status stp_set_stream(stp_problem *p, void *cuda_stream);

/* Failure-detection self-test (no paper counterpart): launches one kernel
 * that waits, with the library's bounded wait, on an mbarrier that nothing
 * ever arrives at, giving up after limit_ns nanoseconds (1 .. 1e10). Returns
 * STP_ERR_TIMEOUT (the status every library kernel reports when one of its
 * waits runs out) and the time waited in *waited_us (may be NULL); the CUDA
 * context stays usable. STP_ERR_CUDA without a device. Every wait inside the
 * library's kernels is bounded by 1 s the same way. */
stp_status stp_selftest_bounded_wait(unsigned long long limit_ns, int *waited_us);

/* Human-readable name of a status code (static string). */
const char *stp_status_string(stp_status s);

/* Last CUDA error text recorded by the library for p (static until the next
 * call on p); "" if none. */
const char *stp_last_error(const stp_problem *p);

/* ---- Inspection (tests and tooling) -------------------------------------
 * Arena -1 is the forward tree; arena i in [0, n_roots) is backward group i
 * (interval root) or slot i (root recycling, current generation only).
 * stp_tree_nodes writes n nodes: x [n][dof+1] (q..., t), parent (index in the
 * same arena, -1 for roots), troot (root/arrival time; 0 forward), cost
 * (configuration-space length to the root), tree (interval: backward tree id;
 * recycling: slot generation), iter (inserting iteration, -1 initial roots).
 * Any output pointer may be NULL. */
stp_status stp_tree_size(stp_problem *p, int arena, int *n);
stp_status stp_tree_nodes(stp_problem *p, int arena, double *x, int *parent, double *troot,
                          double *cost, int *tree, int *iter);
/* Incumbent arrival time after each iteration of the last stp_plan: U_hist[cap]. */
stp_status stp_history(stp_problem *p, double *U_hist, int cap, int *n);
/* Root-recycling slots after the last stp_plan: T, has_root, active, gen [n_roots]. */
stp_status stp_slots(stp_problem *p, double *T, int *has_root, int *active, int *gen);
/* Goal-time grid checks k = kmin..kmin+n-1 (free flags [cap]). */
stp_status stp_goal_grid(stp_problem *p, long *kmin, int *n, unsigned char *free_flags, int cap);

/* ---- Learned proposal network --------------------------------------------
 * The learned sampling branch of the method's GPU form: a 4-layer MLP of
 * width 256 (BF16 weights, FP32 accumulation on the tensor cores) maps a
 * problem summary x[STP_MLP_IN] to y[STP_MLP_OUT]: a mixture of 8 Gaussians
 * over the normalised arrival time tau = U/H (logits y[0:8], means y[8:16],
 * log standard deviations y[16:24], clamped to [-7, 2]) and 16 waypoints
 * (y[24 + 8 i + j]: joint j < 7 as an offset, in coordinates normalised to
 * [-1, 1] over the joint box, from the straight line (1 - f_i) u_s + f_i u_g
 * between the normalised start and goal, f_i = (i + 1) / 17; j = 7 the
 * waypoint time over H); y[152:160] is padding.
 *   x layout: q_s (7, normalised, zero padded), q_g (7), DOF one-hot (3: d = 2,
 *   6, 7), mean over obstacles of (first waypoint x, y, z, mean velocity x, y, z,
 *   radius) (7), H / 60, L_g / H with L_g = D(q_s, q_g) / v_max (2), zeros (6).
 *   Training targets t[STP_MLP_NTGT]: tau, 16 x 8 waypoint targets (same layout
 *   as the outputs), d. Loss per sample: mixture negative log-likelihood of tau
 *   plus the mean squared waypoint error over joints j < d and the time entry;
 *   the batch loss is the mean over samples. Optimiser: Adam (beta 0.9, 0.999,
 *   eps 1e-8) on FP32 master weights.
 * Parameters travel as STP_MLP_NPARAM floats in the order W1 [256][32], b1
 * [256], W2 [256][256], b2, W3 [256][256], b3, W4 [160][256], b4 [160]
 * (row-major, W maps inputs to outputs as y = W x + b); W4 rows 152..159 and
 * b4[152..159] must be zero.
 * Pointers are host memory unless flags has STP_MLP_DEVICE (device memory).
 * Every call is stream-ordered on the network's stream and returns after its
 * results are available. Errors: STP_ERR_INVALID for NULL or out-of-range
 * arguments, STP_ERR_CUDA for a CUDA failure, STP_ERR_TIMEOUT if a bounded
 * wait inside a tensor-core kernel ran out (results are then undefined). */
#define STP_MLP_IN 32
#define STP_MLP_OUT 160
#define STP_MLP_NTGT 130
#define STP_MLP_NPARAM 181152
#define STP_MLP_MAX_BATCH 65536
#define STP_MLP_DEVICE 1
typedef struct stp_mlp stp_mlp;
/* Device state for batches of up to max_batch samples; parameters start at 0. */
stp_status stp_mlp_create(int max_batch, stp_mlp **out);
void stp_mlp_free(stp_mlp *m);
stp_status stp_mlp_set_stream(stp_mlp *m, void *cuda_stream);
/* Load parameters (host, STP_MLP_NPARAM floats); resets the Adam state. */
stp_status stp_mlp_set_params(stp_mlp *m, const float *params);
stp_status stp_mlp_get_params(stp_mlp *m, float *params);
/* y [B][STP_MLP_OUT] from x [B][STP_MLP_IN]. */
stp_status stp_mlp_forward(stp_mlp *m, int B, const float *x, float *y, int flags);
/* Batch loss and its gradient (parameter order above) without an update. */
stp_status stp_mlp_gradients(stp_mlp *m, int B, const float *x, const float *targets, float *loss,
                             float *grads, int flags);
/* One Adam step at learning rate lr on the batch; *loss (may be NULL) gets
 * the batch loss before the step. */
stp_status stp_mlp_train_step(stp_mlp *m, int B, const float *x, const float *targets, float lr, float *loss,
                              int flags);
/* With profiling on, the forward chain of tensor-core GEMMs and the backward
 * pass's GEMMs are each bracketed by CUDA events (intervals that hold GEMM
 * launches only); stp_mlp_profile returns (and clears) their total time, FLOPs and
 * algorithmic HBM bytes, both over the layers' logical shapes (32 inputs,
 * 160 outputs, the batch without padding): operands read once, each output
 * written once in one layout. */
stp_status stp_mlp_set_profiling(stp_mlp *m, int on);
stp_status stp_mlp_profile(stp_mlp *m, double *gemm_ms, double *gemm_flops, double *gemm_bytes);
/* With profiling on, the device work of each stp_mlp_train_step and
 * stp_mlp_gradients call (input packing, forward chain, loss, backward pass,
 * gradient sums and parameter update; not the staging copies of x and the
 * targets, nor the loss read-back) is bracketed by CUDA events on the
 * network's stream; stp_mlp_profile_step returns (and clears) the total ms
 * and the number of steps. Either pointer may be NULL. */
stp_status stp_mlp_profile_step(stp_mlp *m, double *step_ms, int *steps);
const char *stp_mlp_last_error(const stp_mlp *m);

/* Training targets t[STP_MLP_NTGT] of the path found by the last stp_plan or
 * stp_batch_plan of p: tau = U/H; the path sampled at t_i = (i+1) U / 17,
 * i = 0..15, by linear interpolation in time (joints normalised to [-1, 1]
 * as offsets from the straight line between the path's end states, entry 7 =
 * t_i / H, unused joints 0); d. Computed on the device.
 * STP_NO_SOLUTION if there is no path of at least two states. */
stp_status stp_problem_targets(stp_problem *p, float *t);
/* Problem summary x[STP_MLP_IN] of p (layout above), from its FP64 inputs. */
stp_status stp_problem_features(const stp_problem *p, float *x);
/* Install the proposal for the learned branch from a network output
 * y[STP_MLP_OUT] (host, or device with flags = STP_MLP_DEVICE); host values
 * must be finite. The library keeps its own copy (the table is built on the
 * device in the problem's precision): mixture weights softmax(y[0:8]) as
 * cumulative sums, goal-time means y[8:16] H and standard deviations
 * exp(clamp(y[16:24], -7, 2)) H, waypoints q_lo + (clamp(y + line, -1, 1) +
 * 1)/2 (q_hi - q_lo) with line the straight-line point of the layout above.
 * A learned worker (Philox slot 12 below ceil(0.9 2^24)) draws
 * q_r uniformly within +-0.1 of each joint range around waypoint i (slot 13,
 * 16 equally likely), clipped to C; in interval root it also draws
 * T = mean_k + sd_k z (component k from the cumulative weights with slot 14,
 * z by Box-Muller from slots 15-16) and keeps T only inside the sampled
 * group's uniform interval. The paper's GPU form has a learned proposal but
 * fixes none of these choices. May be called again between plans. */
stp_status stp_set_proposal(stp_problem *p, const float *y, int flags);

#ifdef __cplusplus
}
#endif

#endif /* STP_H */
