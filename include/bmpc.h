/*
 * bmpc.h - C ABI of the B300 branch-MPC solver (multiple-shooting augmented-
 * Lagrangian iLQR over a scenario tree, arXiv 2506.13624).
 *
 * One call of bmpc_solve / bmpc_solve_batch runs the whole method of
 * Algorithm 1 on the GPU in one persistent kernel launch: per-node RK4
 * linearisation and Gauss-Newton quadratisation of the augmented Lagrangian
 * (Sec. IV-A, Eq. AL), the tree Riccati recursion that sums the children's
 * value functions at branch points (Sec. III-A, Eq. tree_Riccati and
 * Eq. tree_feedback_laws), the linear forward rollout along all root-to-leaf
 * paths, the merit line search over all step sizes (Eq. merit,
 * Eq. sufficient_decrease) and the BCL multiplier / penalty update (Sec. IV-B).
 *
 * Memory.  The library never allocates device memory.  The caller provides two
 * device arenas (any allocator: PyTorch tensors, cudaMalloc, ...) whose sizes
 * bmpc_batch_bytes reports: a data arena (problem tables, inputs, outputs,
 * statistics) and a scratch arena (per-node Jacobians, Riccati factors and
 * search directions).  Arenas must be 256-byte aligned and stay valid until
 * bmpc_destroy_batch.  Host staging memory for uploads/downloads may be passed
 * in (pinned memory gives asynchronous copies); with NULL the library uses
 * malloc.
 *
 * Streams.  Every device operation of a handle is issued on the handle's stream:
 * the one given at creation (a cudaStream_t passed as void*, NULL = legacy default
 * stream), or the one bmpc_set_stream set later.  bmpc_get_solutions synchronises
 * that stream.  Handles are not thread safe.
 *
 * Errors.  Every function returns a bmpc_status; negative values are errors.
 * After BMPC_ERR_CUDA the handle should be destroyed.
 */
#ifndef BMPC_H
#define BMPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BMPC_OK = 0,            /* converged: max(r_kkt, c) < eps_tol (Sec. IV-B)        */
    BMPC_MAX_ITER = 1,      /* iteration cap reached; the last iterate is returned   */
    BMPC_LS_FAIL = 2,       /* three consecutive line searches found no Armijo step  */
    BMPC_ERR_INVALID = -1,  /* bad argument, tree or size                            */
    BMPC_ERR_CUDA = -2,     /* a CUDA runtime call failed                            */
    BMPC_ERR_NUMERIC = -3,  /* non-positive-definite H_n or non-finite value         */
    BMPC_ERR_TIMEOUT = -4,  /* reserved: a bounded device wait expired               */
    BMPC_ERR_SPACE = -5     /* an arena or staging buffer is too small               */
} bmpc_status;

#define BMPC_MAX_OBS 8
#define BMPC_MAX_NX 6
#define BMPC_NU 2
#define BMPC_NUM_MODELS 4

/* Dynamics models (the ego vehicle's f_i of Eq. bmpc; discretised by RK4):
 *   0 kinematic bicycle, x = (X, Y, psi, v),          u = (a, delta), nx = 4
 *   1 dynamic bicycle (linear tyres, small steering), x = (X, Y, psi, vx, vy, r), nx = 6
 *   2 linear x+ = Alin x + Blin u,                     nx = 4
 *   3 unicycle, x = (X, Y, theta, v),                  u = (a, omega), nx = 4
 *     (X' = v cos theta, Y' = v sin theta, theta' = omega, v' = a; Sec. V-B's benchmark) */
typedef struct {
    int32_t num_nodes;      /* >= 2 */
    const int32_t *parent;  /* host [num_nodes]; parent[0] = -1; level order: nodes sorted by
                               stage, parent[i] < i and non-decreasing for i >= 1 (so the children
                               of a node are contiguous).  Copied at creation. */
    int32_t nx, nu, model;  /* nu must be 2 */
    int32_t n_obs;          /* obstacle ellipses per node, 0..BMPC_MAX_OBS */
    int32_t box_on;         /* input box rows on non-leaf nodes */
    int32_t lane_on;        /* lateral lane rows on non-root nodes */
    float dt;               /* discretisation step */
    float params[10];       /* L, m, Iz, lf, lr, Cf, Cr, vmin, veps, n_sub (RK4 substeps) */
    int32_t edge_dynamics;  /* 1: model 2 with its own (A_m, B_m) on every tree edge, x_m = A_m x_p(m) +
                               B_m u_p(m) (per-branch models, the mass-spring trees of Sec. V-A);
                               0: one model per node, shared by its children.  Per-edge problems
                               take sweep variants 0-2 (BMPC_ERR_INVALID otherwise), upload through
                               bmpc_set_problems (not the flat path) and have no device warm-start
                               shift or learned start. */
} bmpc_tree_desc;

/* Problem data of one tree (host pointers, copied by bmpc_set_problems).
 * Cost (Eq. bmpc):  l_i = w_i [1/2 (x-xref_i)' diag(Qw) (x-xref_i) + 1/2 u' diag(Rw) u],
 *                   l_f,i = w_i 1/2 (x-xref_i)' diag(QNw) (x-xref_i) at leaves.
 * Constraints g <= 0: u - u_hi, u_lo - u (non-leaf nodes); per obstacle the normalised
 * ellipse distance 1 - sqrt((d_par/a)^2 + (d_perp/b)^2 + 1e-6); Y - lane_hi, lane_lo - Y.
 * The root state is fixed to x0 and carries no state constraints. */
typedef struct {
    const float *x0;        /* [nx] measured state */
    const float *xref;      /* [num_nodes][nx] */
    const float *weight;    /* [num_nodes] node weights w_i, or NULL for all ones */
    float Qw[BMPC_MAX_NX], QNw[BMPC_MAX_NX], Rw[BMPC_NU];
    float u_lo[BMPC_NU], u_hi[BMPC_NU];
    float lane_lo, lane_hi;
    const float *obs;       /* [num_nodes][n_obs][5]: cx, cy, heading, a, b (may be NULL if n_obs = 0) */
    const float *Alin;      /* [nx][nx] row-major, model 2 only (not read with edge_dynamics) */
    const float *Blin;      /* [nx][nu] row-major, model 2 only (not read with edge_dynamics) */
    /* optional warm start; all four NULL = cold start of Sec. V-B (x linearly interpolated
       from x0 to the final reference of the node's first leaf, u = lam = y = 0) */
    const float *warm_x;    /* [num_nodes][nx] */
    const float *warm_u;    /* [num_nodes][nu] */
    const float *warm_lam;  /* [num_nodes][nx] */
    const float *warm_y;    /* [num_nodes][nc], nc = 2*nu*box_on + n_obs + 2*lane_on */
    const float *Aedge;     /* with edge_dynamics: [num_nodes][nx][nx], row m the edge into node m (row 0
                               unused); else NULL */
    const float *Bedge;     /* with edge_dynamics: [num_nodes][nx][nu], likewise */
} bmpc_problem;

/* Algorithm 1 constants (defaults: the values of Sec. V-B plus the readings of the oracle). */
typedef struct {
    int32_t max_iters;      /* cap on inner iterations (tree-LQR solves), default 50 */
    int32_t max_outer;      /* cap on outer iterations, default 60 */
    int32_t n_alpha;        /* step sizes alpha_i = 2^-i, i < n_alpha (<= 16), default 10 */
    float eps_tol;          /* 1e-5 */
    float tau;              /* 100 */
    float omega0, eta0;     /* 1, 0.1 */
    float a_omega, b_omega; /* 1, 1 */
    float a_eta, b_eta;     /* 0.1, 0.9 */
    float rho0, rho_max;    /* 10, 1e6 (the paper gives no cap; see cap_rule) */
    float mu0;              /* 1 */
    float beta;             /* Armijo constant, 1e-4 */
    float ls_rel_eps;       /* Armijo slack relative to |phi(0)|, 1e-6 */
    int32_t ls_chunk;       /* step sizes evaluated per parallel round (1..16), default 2; 0 = all.
                               The accepted step (the largest alpha_i meeting Armijo) does not
                               depend on it: it only trades parallel work for extra rounds. */
    int32_t block_threads;  /* threads per problem (32..512, multiple of 32); 0 = automatic */
    int32_t blocks_per_sm;  /* resident problems per SM; 0 = automatic */
    int32_t variant;        /* tree sweeps: 0 automatic by tree shape (2 when the tree has at most as many
                               scenario paths as threads per problem, else 1), 1 level-synchronous (one barrier per stage,
                               nodes of a stage in parallel), 2 per-scenario-path (one thread per
                               root-to-leaf path, barriers only at branch stages), 3 per-scenario-path
                               with 8 lanes per path (lane j owns column j of [A B], P and H),
                               4 scan sweeps (Sec. III-B): conditional value functions combined by
                               suffix scans along every non-branching segment (Eq. comb_rule), tree
                               Riccati steps at branch nodes, and pointer jumping over the closed-loop
                               maps (Eq. forward_comb_rule) forward, so that the sweeps' dependent
                               steps grow with log2 of the depth (a kernel instance of its own, up to
                               512 threads per problem), 5 the per-path backward sweep of 2 with the
                               pointer-jumping forward sweep of 4 (the fastest single solves of deep
                               paths); all compute the same search direction */
    int32_t warm_select;    /* 1: start from warm slot 0 only if its merit is not above that of the fallback
                               (warm slot 1 when set, else the cold start); default 0 */
    float select_mu;        /* defect penalty mu of the merit used by warm_select, default 100 */
    float select_rho;       /* constraint penalty rho of the merit used by warm_select, default 1e4: a start
                               that cuts through a keep-out region loses to one that does not */
    int32_t queue_order;    /* order in which the persistent blocks take problems: 1 (default) longest
                               predicted first, the prediction being nodes x (inner iterations of the
                               problem's previous solve in this batch + 1), sorted on the device before
                               each launch (so also inside a captured graph); 0 largest tree first.
                               The solutions do not depend on it. */
    int32_t block_threads_model[BMPC_NUM_MODELS]; /* threads per problem for the launch of one
                               dynamics model (0 kinematic, 1 dynamic, 2 linear, 3 unicycle) in a
                               mixed batch (32..512, multiple of
                               32); 0 = block_threads.  Each model has its own launch, so a mixed
                               batch can run, e.g., its kinematic problems two per SM and its large
                               dynamic ones one per SM. Default 0. */
    int32_t cap_rule;       /* what a failed outer step does (c > eta, Sec. IV-B):
                               0 (default) Algorithm 1: y kept, rho <- min(tau rho, rho_max);
                               1 the same below rho_max, but at rho_max the multiplier step
                               y <- max(0, y + rho g) instead, for a low cap (e.g. rho_max = 100):
                               with a plain FP32 iterate (compensated = 0) rho times the rounding of
                               g floors the relaxed KKT residual near 1e-5 once rho exceeds about
                               100, and this rule keeps the multipliers moving at such a cap. */
    float kkt_margin;       /* the kernel tests convergence (max(r_kkt, c) < tol) and floors omega and
                               eta at tol = kkt_margin * eps_tol, default 0.8, in (0, 1].  Its FP32
                               evaluation of r_kkt carries rounding of about 1e-6 (terms of size 1-10
                               at unit roundoff 6e-8), so a point it accepts at exactly eps_tol can
                               exceed eps_tol when evaluated in exact arithmetic; the margin keeps the
                               returned point within eps_tol. */
    int32_t compensated;    /* 1 (default): the iterate's positions (X, Y) and inputs are held as
                               pairs of floats (value and rounding remainder), every accepted step is
                               added without loss, and the constraint values that the penalty
                               multiplies by rho (input bounds, keep-out distances, lane bounds) are
                               formed from both parts, the keep-out distance in two-float arithmetic.
                               With plain FP32 iterates, rho times the rounding of an input resting on
                               its bound (or of a position on a keep-out boundary) floors the relaxed
                               KKT residual near 1e-5.  0: plain FP32 iterate. */
    int32_t hessian;        /* 0 (default): Gauss-Newton Hessian; 1: the exact Hessian of the
                               Lagrangian with eigenvalue modification (Sec. IV-A): every node's block
                               in (x, u) adds the RK4 map's second derivatives weighted by the
                               children's multipliers (hyper-dual arithmetic) and the curvature of the
                               active keep-out rows, and its eigenvalues are floored at 1e-6 max(1,
                               max |ev|) (Jacobi rotations when a Cholesky test shows one below).
                               Sweep variants 0-2 and 5 (3 and 4 assume the diagonal cost). */
} bmpc_opts;

typedef struct {
    int32_t status;         /* bmpc_status of this problem */
    int32_t inner_iters;    /* tree-LQR solves */
    int32_t outer_iters;
    int32_t ls_fail_total;
    int32_t ls_evals;       /* step sizes evaluated by the line search, summed over iterations */
    int32_t start_used;     /* starting point: 0 cold start, 1 warm slot 0, 2 warm slot 1 */
    float r_kkt, c, rho, mu;
    int64_t cycles_linearise, cycles_backward, cycles_forward, cycles_linesearch, cycles_total;
} bmpc_stats;

typedef struct bmpc_batch bmpc_batch;   /* opaque handle */

/* Fill *opts with the defaults listed above. */
void bmpc_default_opts(bmpc_opts *opts);

/* Bytes needed for n problems with the given tree descriptors: device data arena,
 * device scratch arena and host staging buffer.  Returns BMPC_ERR_INVALID on a bad tree. */
int bmpc_batch_bytes(const bmpc_tree_desc *descs, int32_t n, size_t *data_bytes, size_t *scratch_bytes,
                     size_t *staging_bytes);

/* Create a handle over caller-owned memory (see "Memory").  Validates every tree,
 * computes the device layout and uploads the tree tables on `stream`. */
int bmpc_create_batch(const bmpc_tree_desc *descs, int32_t n, void *dev_data, size_t data_bytes,
                      void *dev_scratch, size_t scratch_bytes, void *host_staging, size_t staging_bytes,
                      void *stream, bmpc_batch **out);

/* Copy the problem data of all n problems (host pointers) to the device: one packing
 * pass into the staging buffer and one host-to-device copy on the handle's stream. */
int bmpc_set_problems(bmpc_batch *b, const bmpc_problem *problems);

/* Run Algorithm 1 on every problem of the batch from its warm (or cold) start: one persistent
 * kernel launch per dynamics model present in the batch, on the handle's stream
 * (asynchronous).  opts may be NULL. */
int bmpc_solve_batch(bmpc_batch *b, const bmpc_opts *opts);

/* Same work captured once into a CUDA graph (queue reset + persistent kernel) and
 * replayed; the graph is rebuilt when opts change.  Asynchronous. */
int bmpc_solve_batch_graph(bmpc_batch *b, const bmpc_opts *opts);

/* Warm starts on the device.  Every problem has two warm-start slots: 0 (primary) and 1 (fallback).
 * bmpc_set_problems fills slot 0 from host arrays.  These calls fill a slot for every problem of the
 * batch on the handle's stream:
 *   bmpc_set_warm_start_device: from a device array, problem k at dev_start + k*stride floats, packed
 *     node-major x [n][nx] (absolute states) | u [n][nu] | lam [n][nx] | y [n][nc];
 *   bmpc_shift_warm_start: the receding-horizon shift of `prev`'s solution (same trees, same models):
 *     the node at stage k takes the previous solution at stage k+1 on the path of its first leaf,
 *     the last stage appends the last control and propagates the dynamics. */
int bmpc_set_warm_start_device(bmpc_batch *b, const float *dev_start, int64_t stride, int32_t slot);
int bmpc_shift_warm_start(bmpc_batch *next, const bmpc_batch *prev, int32_t slot);

/* Autotuner: solves the batch once per candidate launch configuration (threads per problem 32 / 64 /
 * 128 / 256 / 512, sweep variant 1 to 5, line-search chunk 1 / 2 / 4; the other fields from `base`,
 * NULL = defaults), timing each with CUDA events on the handle's stream, and returns in *best the
 * configuration with the most converged solves per second and in *best_us_per_solve its time per
 * problem.  The scan sweeps (variant 4) are candidates for single-problem batches only: they trade
 * work for depth, which only a problem solved alone can use.  Synchronises the stream; leaves the
 * last candidate's solution in the outputs. */
int bmpc_autotune(bmpc_batch *b, const bmpc_opts *base, bmpc_opts *best, float *best_us_per_solve);

/* Copy solutions back (synchronises the stream).  Host arrays, concatenated over problems
 * in batch order, node-major: x [sum n_i][nx_i], u [sum n_i][nu] (zero rows at leaves),
 * lam [sum n_i][nx_i] (row of each root zero), y [sum n_i][nc_i]; stats [n].
 * Any pointer may be NULL. */
int bmpc_get_solutions(bmpc_batch *b, float *x, float *u, float *lam, float *y, bmpc_stats *stats);

/* Device pointers of the output arrays of problem i (component-major [comp][npad]) and its
 * padded node count, for callers that keep results on the GPU.  The state array holds the
 * deviation x - xref of every node from its reference (the solver's coordinates). */
int bmpc_problem_device_outputs(const bmpc_batch *b, int32_t i, float **x, float **u, float **lam, float **y,
                                int32_t *npad);

/* Flat transfers for callers that keep the per-node data of the whole batch in three node-major
 * arrays, concatenated in problem order (best in pinned host memory or on the device; any
 * memory cudaMemcpy accepts):
 *   xref   [sum_k n_k * nx_k]       reference states;
 *   weight [sum_k n_k] or NULL      node probabilities (NULL: 1);
 *   obs    [sum_k n_k * n_obs_k * 5] obstacle ellipses (cx, cy, heading, a, b).
 * The per-problem scalars (x0, Q, R, Q_N, bounds, lane, linear model) still come from `probs`
 * (their array pointers and warm starts are ignored: this upload clears the warm-start slots).
 * One copy per array and a device kernel replace the host packing of bmpc_set_problems; the data
 * the solver sees are identical.  Asynchronous on the handle's stream; the caller keeps the
 * arrays unchanged until the stream has consumed them. */
int bmpc_set_problems_flat(bmpc_batch *b, const bmpc_problem *probs, const float *xref, const float *weight,
                           const float *obs);

/* Solutions as node-major arrays concatenated in problem order: x [sum n_k nx_k] (absolute
 * states), u [sum n_k nu], lam [sum n_k nx_k], y [sum n_k nc_k] (any may be NULL), packed on the
 * device and copied with one transfer each (fast into pinned memory), and per-problem statistics.
 * Synchronises the handle's stream.  Values equal bmpc_get_solutions'. */
int bmpc_get_solutions_flat(bmpc_batch *b, float *x, float *u, float *lam, float *y, bmpc_stats *stats);

/* Asynchronous form of bmpc_get_solutions_flat. It enqueues on the handle's stream the device
 * packing, one copy per array into x, u, lam, y (any may be NULL; pinned host memory for
 * asynchronous copies), and the copy of the statistics into the handle's staging area. It then
 * returns without waiting. The arrays hold the solutions once bmpc_wait_solutions has returned.
 * Two handles on two streams can overlap one batch's transfers with another batch's solve.
 * BMPC_ERR_INVALID on a null handle; BMPC_ERR_CUDA if a copy or launch is refused. */
int bmpc_get_solutions_flat_async(bmpc_batch *b, float *x, float *u, float *lam, float *y);

/* Waits for the handle's stream. With stats != NULL it fills the per-problem statistics that the
 * last bmpc_get_solutions_flat_async copied. The handle's next bmpc_set_problems_flat may
 * overwrite its staging area only after this wait. BMPC_ERR_CUDA on a failed stream. */
int bmpc_wait_solutions(bmpc_batch *b, bmpc_stats *stats);

/* Bytes one bmpc_set_problems_flat copies host to device (records, xref, weight, obs) and one
 * bmpc_get_solutions_flat copies device to host (x, u, lam, y, statistics). */
int bmpc_transfer_bytes_flat(const bmpc_batch *b, size_t *h2d, size_t *d2h);

/* Bytes one bmpc_set_problems copies host to device (cold starts: problem records and inputs;
 * with warm starts: plus the warm-start region) and one bmpc_get_solutions copies device to host
 * (outputs and statistics).  BMPC_ERR_INVALID on a null batch. */
int bmpc_transfer_bytes(const bmpc_batch *b, size_t *h2d_cold, size_t *h2d_warm, size_t *d2h);

/* Copies the work-queue order of the last solve to `order` (host, caller-allocated, n_problems
 * ints): problem ids grouped by model, in the order the persistent blocks took them.  Waits for
 * the batch's stream.  BMPC_ERR_INVALID on a null argument. */
int bmpc_get_queue_order(const bmpc_batch *b, int32_t *order);

void bmpc_destroy_batch(bmpc_batch *b);

/* ---- creation without a scratch arena (no counterpart in the paper) ----
 * For callers that cannot allocate device memory for the solver, e.g. a real-time control
 * loop that forbids allocation once running, or a plug-in whose host framework owns all device
 * buffers.  Same as bmpc_create_batch except that the solver scratch is a fixed array of
 * BMPC_STATIC_SCRATCH_BYTES (16 MiB) inside the library; the caller still provides the data
 * arena with the inputs and outputs, and drives the handle with the usual calls.
 *   - Allocates no device memory (no cudaMalloc, cudaFree or allocating library call).
 *   - Returns BMPC_ERR_SPACE when the batch needs more scratch than the array holds
 *     (bmpc_batch_bytes reports the need).
 *   - The first call on a device looks up the array's device address with that device current;
 *     make that first call before any stream capture starts.
 *   - Every handle made this way shares the one array: solves of such handles must not overlap
 *     on the GPU (they would race), e.g. issue them on one stream.  The array keeps the last
 *     solve's contents; no entry needs to start at zero. */
#define BMPC_STATIC_SCRATCH_BYTES (16u << 20)
int bmpc_create_batch_static(const bmpc_tree_desc *descs, int32_t n, void *dev_data, size_t data_bytes,
                             void *host_staging, size_t staging_bytes, void *stream, bmpc_batch **out);

/* Moves the handle to another stream (a cudaStream_t as void*, NULL = legacy default stream).
 * Every later call of the handle issues its work there.  Work already issued on the old stream
 * stays ordered before it: the new stream waits for an event recorded on the old one.  No
 * synchronisation with the host.  A captured graph (bmpc_solve_batch_graph) stays valid and is
 * launched on the new stream.  BMPC_ERR_INVALID on a null handle; BMPC_ERR_CUDA if the event
 * cannot be recorded or waited for. */
int bmpc_set_stream(bmpc_batch *b, void *stream);

/* ---- single-tree interface of the paper's problem statement (a batch of one) ----
 * The paper states one branch-MPC problem (Sec. II-B, Eq. bmpc): a scenario tree given by every
 * node's parent (tree notation of Sec. II-B), the measured state x-bar fixed at the root, node
 * costs l_i / l_f,i, dynamics x_i = f_p(i)(x_p(i), u_p(i)) and constraints g_i <= 0 per node, and
 * the initialisation of Sec. V-B.  These calls hold exactly one such problem; they are the batch
 * calls above with n = 1 (same arguments, layouts, ownership and errors). */
typedef bmpc_batch bmpc_tree;

/* Device and host bytes for one tree (Sec. II-B tree notation); as bmpc_batch_bytes with n = 1. */
int bmpc_tree_bytes(const bmpc_tree_desc *desc, size_t *data_bytes, size_t *scratch_bytes, size_t *staging_bytes);

/* The tree of Eq. (bmpc): desc->parent gives p(i) for every node in level order (Sec. II-B), with
 * the dynamics model f_i and the constraint families.  Caller-owned arenas as for
 * bmpc_create_batch; validates the tree (BMPC_ERR_INVALID), BMPC_ERR_SPACE on short arenas. */
int bmpc_create_tree(const bmpc_tree_desc *desc, void *dev_data, size_t data_bytes, void *dev_scratch,
                     size_t scratch_bytes, void *host_staging, size_t staging_bytes, void *stream, bmpc_tree **out);

/* The data of Eq. (bmpc) for the tree: x-bar (x_0 = x0), the stage and terminal costs l_i, l_f,i
 * (tracking references and weights), the constraint data of g_i, and an optional warm start; NULL
 * warm arrays give the cold start of Sec. V-B.  Host pointers, copied (bmpc_set_problems, n = 1). */
int bmpc_set_problem(bmpc_tree *t, const bmpc_problem *problem);

/* Solves the problem by the AL method of Algorithm 1 (Sec. IV): inner iLQR iterations on the
 * relaxed problem Eq. (relax_bmpc), each one linearisation, tree Riccati recursion
 * (Eq. tree_Riccati, Eq. tree_feedback_laws), linear rollout, merit line search (Eq. merit,
 * Eq. sufficient_decrease), and the BCL update of y_e and rho (Sec. IV-B).  opts NULL = defaults.
 * With stats != NULL it synchronises the stream, fills *stats and returns the problem's status
 * (BMPC_OK, BMPC_MAX_ITER, BMPC_LS_FAIL or BMPC_ERR_NUMERIC); otherwise it is asynchronous. */
int bmpc_solve(bmpc_tree *t, const bmpc_opts *opts, bmpc_stats *stats /* nullable; synchronises if given */);

/* The solution of Eq. (bmpc) (Algorithm 1's return value x, u, y_e, plus the dynamics multipliers
 * lambda of the Lagrangian of Sec. IV-A): host arrays, node-major x [n][nx] (absolute states),
 * u [n][nu] (zero rows at leaves), lam [n][nx] (root row zero), y [n][nc]; any may be NULL.
 * Synchronises the stream. */
int bmpc_get_solution(bmpc_tree *t, float *x, float *u, float *lam, float *y);
void bmpc_destroy_tree(bmpc_tree *t);

const char *bmpc_status_str(int status);
/* Library build string (architecture and version). */
const char *bmpc_version(void);

/* Test support: the device sine and cosine that the vehicle dynamics use (Cody-Waite reduction by
 * pi/2, Taylor polynomials on [-pi/4, pi/4]; about 1.5 ulp for |a| < 1e3) on n angles.  a, s, c
 * are device arrays of n floats; asynchronous on `stream`.  BMPC_ERR_INVALID on n < 0 or null
 * arrays, BMPC_ERR_CUDA if the launch fails. */
int bmpc_selftest_sincos(const float *a, float *s, float *c, int32_t n, void *stream);

/* Test support: the eigenvalue modification of the exact-Hessian option (Sec. IV-A; hessian = 1)
 * on `count` symmetric n x n matrices (n = 6 or 8, row-major, device array S of count n n floats,
 * modified in place): every eigenvalue below 1e-6 max(1, max |ev|) is raised to it; a matrix whose
 * Cholesky test shows none below is returned unchanged.  Asynchronous on `stream`.
 * BMPC_ERR_INVALID on a null array, another n or count < 1; BMPC_ERR_CUDA if the launch fails. */
int bmpc_selftest_eig_modify(float *S, int32_t n, int32_t count, void *stream);

/* Test support: the second derivatives of the exact-Hessian option (Sec. IV-A; hessian = 1):
 * H_k = sum_i mu_k,i d^2 f_i / dz dz of the discrete dynamics (RK4 with params[9] substeps of
 * dt / params[9], the model's right-hand side) at z = (x_k, u_k), by hyper-dual arithmetic, for
 * k < count.  params: host array of the 10 model constants (as bmpc_tree_desc.params); x, mu: device
 * [count][nx] (absolute states, nx = 6 for model 1 else 4); u: device [count][2]; H: device
 * [count][nx + 2][nx + 2], row-major in (x, u) order (zero for the linear model).  Asynchronous on
 * `stream`.  BMPC_ERR_INVALID on a model outside 0..3, null arrays, count < 1 or dt <= 0. */
int bmpc_selftest_dyn_hessian(int32_t model, const float *params, float dt, const float *x, const float *u,
                              const float *mu, float *H, int32_t count, void *stream);

/* Measurement support (no counterpart in the paper): the FP32 FMA peak of the device, against which
 * the solver's arithmetic rate is reported.  Launches `blocks` blocks of 256 threads; every thread
 * runs eight independent FMA chains of `iters` rounds and writes one float to out[thread] (out: a
 * device array of blocks * 256 floats).  The kernel performs 2 * 8 * iters * 256 * blocks FLOPs;
 * the caller times it (CUDA events on `stream`).  Asynchronous.  BMPC_ERR_INVALID on a null array or
 * a count below 1, BMPC_ERR_CUDA if the launch fails. */
int bmpc_selftest_fma(float *out, int32_t blocks, int32_t iters, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BMPC_H */
