/*
 * Device memory layout of a batch of branch-MPC problems.  Shared by the host
 * API (which builds the tables) and the solver kernel (which reads them).
 *
 * All per-node arrays are component-major, [component][npad] with npad = n
 * rounded up to a multiple of 32, so that the threads of a warp that work on
 * consecutive nodes of one stage read consecutive addresses.  Nodes are in
 * level order, so the nodes of a stage and the children of a node are
 * contiguous.
 */
#pragma once
#include <stdint.h>

namespace bmpc {

constexpr int NU = 2;
constexpr int NUM_MODELS = 4;   /* 0 kinematic bicycle, 1 dynamic bicycle, 2 linear, 3 unicycle */
constexpr int MAX_NX = 6;
constexpr int MAX_OBS = 8;
constexpr int MAX_NC = 2 * NU + MAX_OBS + 2;

__host__ __device__ constexpr int round_up(int v, int m) { return (v + m - 1) / m * m; }
__host__ __device__ constexpr int nsym(int nx) { return nx * (nx + 1) / 2; }

/* One record per problem; 16-byte aligned, plain data. */
struct alignas(16) ProbRec {
    int32_t n, npad, nx, nu, model, n_obs, nc, box_on, lane_on, n_stage, has_warm, n_paths;
    int32_t n_bstage, n_waves, edge_dyn, rsv2;  /* n_bstage: distinct stages holding branch nodes;
                                                  n_waves: waves of the segment scans (variant 4);
                                                  edge_dyn: linear dynamics per tree edge (model 2) */
    int64_t off_int;   /* int32 elements from the int region base      */
    int64_t off_in;    /* float elements from the input region base    */
    int64_t off_warm;  /* float elements from the warm-start region base */
    int64_t off_out;   /* float elements from the output region base   */
    int64_t off_scr;   /* float elements from the scratch arena base   */
    int64_t off_node, off_nx, off_nc, off_obs;   /* offsets in the node-major flat arrays of the batch:
                                                    sums of n, n*nx, n*nc, n*n_obs*5 over earlier problems */
    float dt, lane_lo, lane_hi, pad1;
    float params[10];  /* L, m, Iz, lf, lr, Cf, Cr, vmin, veps, n_sub  */
    float Qw[MAX_NX], QNw[MAX_NX], Rw[NU], u_lo[NU], u_hi[NU];
    float x0[MAX_NX];
    float Alin[16], Blin[8];
};

static_assert(sizeof(ProbRec) % 16 == 0, "the solver copies a record to shared memory in 16-byte words");

/* int region of one problem (int32 elements):
 *   node rows (npad each): parent, nchild, fchild (first child), stage, leaf (first leaf
 *   descendant), owner (index of the path of that leaf; the path that processes the node in
 *   the per-path sweeps), fnode, fend (the segment order of the scan sweeps, below);
 *   stage_start [n_stage + 1]   first node of every stage (level order);
 *   bstage      [n_bstage]      stages holding nodes with more than one child, descending;
 *   ptab        [n_paths][n_stage]  node of every root-to-leaf path at every stage (-1 past
 *                                   the path's leaf);
 *   pdepth, ptop [n_paths]      stage of the path's leaf, first stage the path owns;
 *   wave        [n_waves + 1] [n_waves]  first position of every wave in the segment order, then
 *                                   the longest segment of every wave (in nodes).
 * Segments (scan sweeps, Sec. III-B): a segment is a maximal chain of single-child nodes together
 * with the node that ends it (a leaf or a node with several children).  Its wave is 0 for a leaf's
 * segment, else one more than the largest wave among the segments of the end node's children.  The
 * segment order lists the nodes wave by wave, segment by segment, each segment from its top to its
 * end: fnode[f] is the node at position f, fend[f] the position of its segment's end.
 * Every block is padded to a multiple of 32 elements. */
struct IntOff {
    int64_t parent, nchild, fchild, stage, leaf, owner, fnode, fend, sstart, bstage, ptab, pdepth, ptop, wave, total;
};
__host__ __device__ inline IntOff int_off(int npad, int n_stage, int n_paths, int n_waves = 0) {
    IntOff o;
    o.parent = 0;
    o.nchild = npad;
    o.fchild = 2LL * npad;
    o.stage = 3LL * npad;
    o.leaf = 4LL * npad;
    o.owner = 5LL * npad;
    o.fnode = 6LL * npad;
    o.fend = 7LL * npad;
    o.sstart = 8LL * npad;
    o.bstage = o.sstart + round_up(n_stage + 1, 32);
    o.ptab = o.bstage + round_up(n_stage + 1, 32);
    o.pdepth = o.ptab + round_up(n_paths * n_stage, 32);
    o.ptop = o.pdepth + round_up(n_paths, 32);
    o.wave = o.ptop + round_up(n_paths, 32);
    o.total = o.wave + round_up(2 * n_waves + 1, 32);
    return o;
}

/* The stage and path tables (sstart .. ptop) are contiguous: the solver copies them into shared
 * memory per problem when they fit. */
__host__ __device__ inline int64_t table_ints(int npad, int n_stage, int n_paths) {
    const IntOff o = int_off(npad, n_stage, n_paths);
    return o.wave - o.sstart;
}

/* input region: xref[nx] weight[1] obs[6*n_obs] and, with per-edge dynamics, Ae[nx*nx] Be[nx*nu]
 * (rows of npad).  Per obstacle the rows hold the ellipse centre cx, cy, the cosine and sine of its
 * heading and 1/a^2, 1/b^2, converted once per upload on the device from the caller's cx, cy,
 * heading, a, b.  Ae, Be: the matrices of the edge into node m at column m (row-major entries,
 * one row each; column 0 unused), the layout of the scratch Jacobian rows A, B. */
constexpr int OBS_ROWS = 6;
struct InRows {
    int xref, weight, obs, edge, total;
};
__host__ __device__ inline InRows in_rows(int nx, int n_obs, int edge_dyn = 0) {
    InRows r;
    r.xref = 0;
    r.weight = nx;
    r.obs = r.weight + 1;
    r.edge = r.obs + OBS_ROWS * n_obs;
    r.total = r.edge + (edge_dyn ? nx * nx + nx * NU : 0);
    return r;
}

/* warm-start region: two slots per problem (slot 0 = primary start, slot 1 = fallback start), each
 * wx[nx] wu[nu] wl[nx] wy[nc]; has_warm bit s says slot s holds a start */
struct WarmRows {
    int wx, wu, wl, wy, total;
};
__host__ __device__ inline WarmRows warm_rows(int nx, int nc) {
    WarmRows r;
    r.wx = 0;
    r.wu = nx;
    r.wl = r.wu + NU;
    r.wy = r.wl + nx;
    r.total = r.wy + nc;
    return r;
}

/* output region: x[nx] u[nu] lam[nx] y[nc] */
struct OutRows {
    int x, u, lam, y, total;
};
__host__ __device__ inline OutRows out_rows(int nx, int nc) {
    OutRows r;
    r.x = 0;
    r.u = nx;
    r.lam = r.u + NU;
    r.y = r.lam + nx;
    r.total = r.y + nc;
    return r;
}

/* Rows of one conditional value function (CVF, Sec. III-B) element of the scan sweeps: A[nx*nx]
 * c[nx] C[nsym] P[nsym] p[nx] (C and P symmetric, packed). */
__host__ __device__ constexpr int cvf_rows(int nx) { return nx * nx + 2 * nx + 2 * nsym(nx); }

/* Floats per node of the node-major forward records (scratch region fr): K[nu*nx], the entries of
 * A and B that are not structurally fixed, k[nu], d[nx], padded to a multiple of 4 so that every
 * record starts on a 16-byte boundary.  The models with n_x = 6 (dynamic bicycle) store 32 entries of
 * [A B], those with n_x = 4 at most 12 (kinematic bicycle; the unicycle 10; the linear model keeps
 * no records): 52 and 28 floats, checked against each model's record at compile time. */
__host__ __device__ constexpr int fr_stride(int nx) { return nx == 6 ? 52 : 28; }

/* scratch: A[nx*nx] B[nx*nu] f[nx] d[nx] q[nx] r[nu] hq[3] hr[nu] K[nu*nx] k[nu] P[nsym] p[nx]
 *          dx[nx] du[nu] lq[nx] nv[3] xl[2] ul[nu] cv[2 * cvf_rows] ja[2] hs[nsym + nu*nx + 3]
 *          fr[fr_stride rows, node-major: fr_stride floats per node]
 * xl, ul: low-order parts of the compensated iterate (positions X, Y of the state deviation and the
 * inputs): the iterate is xi + xl, u + ul, each pair a float and its rounding remainder.
 * cv: two buffers of scan elements, indexed by position in the segment order (backward) or by node
 * (forward: closed-loop maps in the A, c rows); ja: two rows of ancestor indices (forward). */
struct ScrRows {
    int A, B, f, d, q, r, hq, hr, K, k, P, p, dx, du, lq, nv, xl, ul, cv, ja, hs, fr, total;
};
__host__ __device__ inline ScrRows scr_rows(int nx) {
    ScrRows s;
    s.A = 0;
    s.B = s.A + nx * nx;
    s.f = s.B + nx * NU;
    s.d = s.f + nx;
    s.q = s.d + nx;
    s.r = s.q + nx;
    s.hq = s.r + NU;
    s.hr = s.hq + 3;
    s.K = s.hr + NU;
    s.k = s.K + NU * nx;
    s.P = s.k + NU;
    s.p = s.P + nsym(nx);
    s.dx = s.p + nx;
    s.du = s.dx + nx;
    s.lq = s.du + NU;
    s.nv = s.lq + nx;
    s.xl = s.nv + 3;
    s.ul = s.xl + 2;
    s.cv = s.ul + NU;
    s.ja = s.cv + 2 * cvf_rows(nx);
    s.hs = s.ja + 2;   /* exact-Hessian option: the node's modified block Q (packed), M, R (packed) */
    s.fr = s.hs + nsym(nx) + NU * nx + 3;
    s.total = s.fr + fr_stride(nx);
    return s;
}

/* Kernel-side copy of the solver options (Algorithm 1 constants). */
struct KOpts {
    int32_t max_iters, max_outer, n_alpha, ls_chunk, variant, warm_select, cap_rule, compensated, hessian;
    float eps_tol, tau, omega0, eta0, a_omega, b_omega, a_eta, b_eta, rho0, rho_max, mu0, beta, ls_rel_eps, select_mu,
        select_rho;
};

/* Per-problem statistics, same layout as the public bmpc_stats. */
struct Stats {
    int32_t status, inner_iters, outer_iters, ls_fail_total, ls_evals, start_used;
    float r_kkt, c, rho, mu;
    int64_t cyc_lin, cyc_bwd, cyc_fwd, cyc_ls, cyc_total;
};

/* Node-major flat arrays of a batch in the raw region of the data arena.  Inputs: xref [T_nx] |
 * weight [T_n] | obs [T_obs] (caller layout, 5 values per obstacle); outputs: x [T_nx] (absolute
 * states) | u [2 T_n] | lam [T_nx] | y [T_nc]. */
struct FlatArgs {
    const ProbRec *recs;
    float *inbase;
    const float *outbase;
    float *raw;
    int64_t T_n, T_nx, T_nc, T_obs;
    int32_t has_weight;
};

/* Arguments of the warm-start kernels (device scatter and receding-horizon shift). */
struct WarmArgs {
    const ProbRec *recs, *prev_recs;
    const int32_t *ibase, *prev_ibase;
    const float *inbase, *prev_inbase, *prev_outbase;
    float *warmbase;
    const float *src;          /* device scatter: [problem][stride] packed x | u | lam | y (node-major) */
    int64_t stride;
    const int32_t *order;      /* problems of one model */
    int32_t n_problems, slot;
};

struct KernelArgs {
    const ProbRec *recs;
    const int32_t *order;     /* queue order of the problems of one model */
    int32_t n_problems;
    int32_t *queue;           /* work-queue counter, zeroed before each launch */
    const int32_t *ibase;
    const float *inbase;
    const float *warmbase;
    float *outbase;
    float *scr;
    Stats *stats;
    KOpts opts;
    int32_t tab_ints;         /* dynamic shared memory for the stage/path tables, in ints (0: none) */
    int32_t stg_ld;           /* path threads with sweep staging slots after the tables (0: no staging) */
};

/* Arguments of the warm-start glue kernels (features, targets, starts). */
struct GlueArgs {
    const ProbRec *recs;
    const int32_t *ibase;
    const float *inbase, *outbase;
    float *out;                 /* features / targets / starts, problem k at out + k*stride */
    int64_t stride;
    const float *pred, *mean, *std;
    int64_t ld_pred;
    int32_t n_scen, n_obs_max;
    const int32_t *order_base;  /* starts: problems of one model */
    int32_t y_sqrt;             /* targets / starts: AL multipliers in square-root form */
};

}  // namespace bmpc
