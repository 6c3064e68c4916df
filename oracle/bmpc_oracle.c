/*
 * FP64 CPU oracle for the multiple-shooting augmented-Lagrangian iLQR method
 * over a scenario tree (branch MPC), arXiv 2506.13624.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the CUDA path computes.  Only tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * constant or helper with the CUDA path.
 *
 * Passages followed (paper section / equation / algorithm):
 *   problem             Sec. II-B, Eq. (bmpc): node costs, x_i = f_p(i)(x_p(i), u_p(i)), g <= 0
 *   models              kinematic and dynamic bicycles (the planning scenes), linear (LQ pins),
 *                       unicycle (the constraint benchmark of Sec. V-B); dynamics per tree edge
 *                       (x_m = f_m(x_p(m), u_p(m)), the per-branch models of Sec. V-A) for the
 *                       linear model, per parent otherwise (every child of a node shares its f)
 *   tree LQR            Sec. III-A, Eq. (lqr_tree_approx), Eq. (tree_Riccati),
 *                       Eq. (tree_feedback_laws); forward rollout as in Sec. II-A
 *   tree LQR by scans   Sec. III-B, Eq. (sol_min), Eq. (comb_rule), Eq. (forward_comb_rule):
 *                       orc_tree_lqr_scan (CVF scans along the non-branching segments)
 *   augmented Lagr.     Sec. IV-A, Eq. (AL) (PHR penalty), Lagrangian with lambda,
 *                       Gauss-Newton Hessian of the PHR term
 *   linear rollout      Sec. IV-A "Search direction" (multiple shooting)
 *   merit, line search  Eq. (merit), Eq. (sufficient_decrease), Algorithm 1
 *   KKT residual        Sec. IV-A "Inner loop stopping criterion"
 *   outer loop (BCL)    Sec. IV-B, Algorithm 1, constants of Sec. V-B
 *
 * Readings where the paper is silent or garbled (kept identical on the CUDA side):
 *   - dynamics Jacobians A_n, B_n per parent node; defect c_m per child edge;
 *   - multiplier update y <- max(0, y + rho g) (standard PHR, Algorithm 1 drops y);
 *   - tolerance schedules omega <- omega rho^-b_omega, eta <- eta rho^-b_eta on success,
 *     omega <- omega0 rho^-a_omega, eta <- eta0 rho^-a_eta on failure, both floored at eps_tol;
 *   - a failed outer step keeps y and raises rho <- min(tau rho, rho_max) (Algorithm 1; the paper
 *     gives no cap, rho_max = 1e6 by default).  Option cap_rule = 1 is the FP32 product's rule
 *     instead: at rho = rho_max a failed outer step applies the multiplier update
 *     y <- max(0, y + rho g) (rho * FP32 rounding of g puts a floor under the KKT residual, so the
 *     GPU caps rho low, at 100); both sides implement both rules;
 *   - the merit uses J = L_a and moves (x, u, lambda) jointly; lambda_QP = P dx + p;
 *   - mu rule: phi'(0; mu) <= -1/2 dz'W dz, else mu <- max(mu, 2(phi'(0;0) + 1/2 dz'W dz)/|d|^2);
 *   - alpha_i = 2^-i; Armijo with an absolute slack ls_rel_eps*|phi(0)| for finite precision;
 *     no accepted alpha -> smallest alpha, three failures in a row -> LS_FAIL;
 *   - the root carries no state constraints (x_0 is fixed), leaves no input constraints;
 *   - cold start: x linearly interpolated from x0 to the node's final reference, u = 0,
 *     lambda = 0, y = 0 (Sec. V-B initialisation);
 *   - CVF combination signs follow Eq. (sol_min) (A = A2 E^-1 A1, c = A2 E^-1 (c1 - C1 p2) + c2,
 *     p = A1' E^-T (p2 + P2 c1) + p1); the separable tree form of Eq. (tree_CVF) is used only along
 *     non-branching segments, since a branch node's shared input couples its children.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* capacities of the fixed-size work arrays: state and input dimensions up to those of the
 * mass-spring chains of Sec. V-A (n_x = 2M = 30, n_u = M - 1 = 14) and a little beyond */
#define MAXX 32
#define MAXU 16
#define MAXN (MAXX + MAXU)
#define OBS_EPS 1e-6   /* smoothing of the normalised distance at the ellipse centre */

typedef struct {
    int n, nx, nu, model, n_obs, box_on, lane_on;
    const int *parent;
    double dt;
    const double *params;   /* [10]: L, m, Iz, lf, lr, Cf, Cr, vmin, veps, n_sub */
    const double *x0;       /* [nx] */
    const double *xref;     /* [n][nx] */
    const double *weight;   /* [n] */
    const double *Qw, *QNw; /* [nx] */
    const double *Rw;       /* [nu] */
    const double *u_lo, *u_hi;
    double lane_lo, lane_hi;
    const double *obs;      /* [n][n_obs][5] cx, cy, heading, a, b */
    const double *Alin, *Blin;
    const double *Aedge, *Bedge;   /* model 2 only, or NULL: per-edge dynamics [n][nx][nx], [n][nx][nu],
                                      row m the edge into node m (row 0 unused) */
} orc_problem;

/* Trace of a solve, for tests that check each decision of Algorithm 1 from outside.  kind 0 (one
 * call per inner iteration, after the line search and before the step is applied):
 *   info = [inner, outer, rho, mu before the update, mu, phi(0), phi'(0; mu), phi'(0; 0), dz'W dz,
 *           |d|^2, alpha, accepted, phi(alpha) (its merit), accepted only through the slack, r_kkt,
 *           omega], a0..a6 = x, u, lam, y, dx, du, dlam;
 * kind 1 (one call per outer update):
 *   info = [outer, branch (0 y updated, 1 rho raised and y kept, 2 multiplier step at the cap
 *           (cap_rule 1), 3 y kept at the cap), c, eta before, rho before, rho after, omega after,
 *           eta after, r_kkt, converged], a0..a4 = x, u, lam, y before, y after (a5, a6 NULL). */
typedef void (*orc_trace_fn)(void *user, int kind, const double *info, const double *a0, const double *a1,
                             const double *a2, const double *a3, const double *a4, const double *a5,
                             const double *a6);

typedef struct {
    int max_iters, max_outer, n_alpha;
    double eps_tol, tau, omega0, eta0, a_omega, b_omega, a_eta, b_eta;
    double rho0, rho_max, mu0, beta, ls_rel_eps;
    int lqr_scan;           /* 1: the search direction by the scans of Sec. III-B (orc_tree_lqr_scan) */
    int hessian;            /* 0: Gauss-Newton; 1: exact Hessian of the Lagrangian with eigenvalue
                               modification (Sec. IV-A), see exact_hessian */
    int cap_rule;           /* 0: Algorithm 1 (failure keeps y, rho <- min(tau rho, rho_max));
                               1: a failure at rho_max applies y <- max(0, y + rho g) */
    orc_trace_fn trace;     /* NULL: no trace */
    void *trace_user;
} orc_opts;

typedef struct {
    int status, inner_iters, outer_iters, ls_fail_total;
    double r_kkt, c, rho, mu, omega, eta;
} orc_stats;

enum { ORC_OK = 0, ORC_MAX_ITER = 1, ORC_LS_FAIL = 2, ORC_ERR_INVALID = -1, ORC_ERR_NUMERIC = -3 };

/* ------------------------------------------------------------ small dense algebra */
/* row-major: M[i*cols + j] */
static void matmul(int r, int k, int c, const double *A, const double *B, double *C) {
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < c; ++j) {
            double s = 0.0;
            for (int t = 0; t < k; ++t) s += A[i * k + t] * B[t * c + j];
            C[i * c + j] = s;
        }
}
/* C = A^T B with A (k x r), B (k x c) */
static void matTmul(int r, int k, int c, const double *A, const double *B, double *C) {
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < c; ++j) {
            double s = 0.0;
            for (int t = 0; t < k; ++t) s += A[t * r + i] * B[t * c + j];
            C[i * c + j] = s;
        }
}
/* y = A x, A (r x c) */
static void matvec(int r, int c, const double *A, const double *x, double *y) {
    for (int i = 0; i < r; ++i) {
        double s = 0.0;
        for (int j = 0; j < c; ++j) s += A[i * c + j] * x[j];
        y[i] = s;
    }
}
/* y = A^T x, A (r x c) */
static void matTvec(int r, int c, const double *A, const double *x, double *y) {
    for (int j = 0; j < c; ++j) {
        double s = 0.0;
        for (int i = 0; i < r; ++i) s += A[i * c + j] * x[i];
        y[j] = s;
    }
}
/* Cholesky H = L L^T (n x n), returns 0 if not positive definite. */
static int cholesky(int n, const double *H, double *L) {
    memset(L, 0, sizeof(double) * n * n);
    for (int j = 0; j < n; ++j) {
        double s = H[j * n + j];
        for (int t = 0; t < j; ++t) s -= L[j * n + t] * L[j * n + t];
        if (!(s > 0.0)) return 0;
        L[j * n + j] = sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double v = H[i * n + j];
            for (int t = 0; t < j; ++t) v -= L[i * n + t] * L[j * n + t];
            L[i * n + j] = v / L[j * n + j];
        }
    }
    return 1;
}
/* solve (L L^T) X = Bm for X (n x m) in place of Bm */
static void chol_solve(int n, int m, const double *L, double *Bm) {
    for (int col = 0; col < m; ++col) {
        for (int i = 0; i < n; ++i) {
            double v = Bm[i * m + col];
            for (int t = 0; t < i; ++t) v -= L[i * n + t] * Bm[t * m + col];
            Bm[i * m + col] = v / L[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double v = Bm[i * m + col];
            for (int t = i + 1; t < n; ++t) v -= L[t * n + i] * Bm[t * m + col];
            Bm[i * m + col] = v / L[i * n + i];
        }
    }
}

/* ------------------------------------------------------------ dynamics (Eq. bmpc, x_i = f_p(i)) */
/* Continuous-time right-hand side fc(s, u) and its Jacobians Jx (nx x nx), Ju (nx x nu). */
static void rhs(const orc_problem *P, const double *s, const double *u, double *f, double *Jx, double *Ju) {
    const double *prm = P->params;
    int nx = P->nx, nu = P->nu;
    memset(Jx, 0, sizeof(double) * nx * nx);
    memset(Ju, 0, sizeof(double) * nx * nu);
    if (P->model == 0) {
        /* kinematic bicycle: X' = v cos psi, Y' = v sin psi, psi' = v tan(delta)/L, v' = a */
        double L = prm[0], psi = s[2], v = s[3], a = u[0], d = u[1];
        double td = tan(d);
        f[0] = v * cos(psi);
        f[1] = v * sin(psi);
        f[2] = v * td / L;
        f[3] = a;
        Jx[0 * 4 + 2] = -v * sin(psi);
        Jx[0 * 4 + 3] = cos(psi);
        Jx[1 * 4 + 2] = v * cos(psi);
        Jx[1 * 4 + 3] = sin(psi);
        Jx[2 * 4 + 3] = td / L;
        Ju[2 * 2 + 1] = v * (1.0 + td * td) / L;
        Ju[3 * 2 + 0] = 1.0;
        return;
    }
    if (P->model == 3) {
        /* unicycle (Sec. V-B): X' = v cos th, Y' = v sin th, th' = omega, v' = a */
        double th = s[2], v = s[3];
        f[0] = v * cos(th);
        f[1] = v * sin(th);
        f[2] = u[1];
        f[3] = u[0];
        Jx[0 * 4 + 2] = -v * sin(th);
        Jx[0 * 4 + 3] = cos(th);
        Jx[1 * 4 + 2] = v * cos(th);
        Jx[1 * 4 + 3] = sin(th);
        Ju[2 * 2 + 1] = 1.0;
        Ju[3 * 2 + 0] = 1.0;
        return;
    }
    /* dynamic bicycle, linear tyres:
     *   slip alpha_f = atan((vy + lf r)/vb) - delta, alpha_r = atan((vy - lr r)/vb),
     *   vb = smooth max(vx, vmin), F_f = -Cf alpha_f, F_r = -Cr alpha_r,
     *   X' = vx cos psi - vy sin psi, Y' = vx sin psi + vy cos psi, psi' = r,
     *   vx' = a - F_f sin(delta)/m + r vy, vy' = (F_f cos(delta) + F_r)/m - r vx,
     *   r' = (lf F_f cos(delta) - lr F_r)/Iz                                    */
    double m = prm[1], Iz = prm[2], lf = prm[3], lr = prm[4], Cf = prm[5], Cr = prm[6];
    double vmin = prm[7], veps = prm[8];
    double psi = s[2], vx = s[3], vy = s[4], r = s[5], a = u[0], d = u[1];
    double w = sqrt((vx - vmin) * (vx - vmin) + veps * veps);
    double vb = 0.5 * (vx + vmin + w);
    double dvb = 0.5 * (1.0 + (vx - vmin) / w);
    double tf = (vy + lf * r) / vb, tr = (vy - lr * r) / vb;
    double af = atan(tf) - d, ar = atan(tr);
    double Ff = -Cf * af, Fr = -Cr * ar;
    double cp = cos(psi), sp = sin(psi);
    f[0] = vx * cp - vy * sp;
    f[1] = vx * sp + vy * cp;
    f[2] = r;
    f[3] = a + r * vy;
    f[4] = (Ff + Fr) / m - r * vx;
    f[5] = (lf * Ff - lr * Fr) / Iz;
    double gf = 1.0 / (1.0 + tf * tf), gr = 1.0 / (1.0 + tr * tr);
    /* partials of the slip angles */
    double daf_vx = gf * (-tf / vb) * dvb, daf_vy = gf / vb, daf_r = gf * lf / vb;
    double dar_vx = gr * (-tr / vb) * dvb, dar_vy = gr / vb, dar_r = -gr * lr / vb;
    double dFf_vx = -Cf * daf_vx, dFf_vy = -Cf * daf_vy, dFf_r = -Cf * daf_r, dFf_d = Cf;
    double dFr_vx = -Cr * dar_vx, dFr_vy = -Cr * dar_vy, dFr_r = -Cr * dar_r;
    /* row X */
    Jx[0 * 6 + 2] = -vx * sp - vy * cp;
    Jx[0 * 6 + 3] = cp;
    Jx[0 * 6 + 4] = -sp;
    /* row Y */
    Jx[1 * 6 + 2] = vx * cp - vy * sp;
    Jx[1 * 6 + 3] = sp;
    Jx[1 * 6 + 4] = cp;
    /* row psi */
    Jx[2 * 6 + 5] = 1.0;
    /* row vx */
    Jx[3 * 6 + 4] = r;
    Jx[3 * 6 + 5] = vy;
    Ju[3 * 2 + 0] = 1.0;
    /* row vy */
    Jx[4 * 6 + 3] = (dFf_vx + dFr_vx) / m - r;
    Jx[4 * 6 + 4] = (dFf_vy + dFr_vy) / m;
    Jx[4 * 6 + 5] = (dFf_r + dFr_r) / m - vx;
    Ju[4 * 2 + 1] = dFf_d / m;
    /* row r */
    Jx[5 * 6 + 3] = (lf * dFf_vx - lr * dFr_vx) / Iz;
    Jx[5 * 6 + 4] = (lf * dFf_vy - lr * dFr_vy) / Iz;
    Jx[5 * 6 + 5] = (lf * dFf_r - lr * dFr_r) / Iz;
    Ju[5 * 2 + 1] = lf * dFf_d / Iz;
}

/* Discrete dynamics x+ = f(x, u) and, if A/B are given, A = df/dx, B = df/du.
 * Models 0/1: n_sub classical RK4 steps of length dt/n_sub, Jacobians by the
 * forward-mode chain rule through every RK4 stage.  Model 2: x+ = Alin x + Blin u. */
int orc_dynamics(const orc_problem *P, const double *x, const double *u, double *xn, double *A, double *B) {
    int nx = P->nx, nu = P->nu, nz = nx + nu;
    if (P->model == 2) {
        double t[MAXX];
        matvec(nx, nx, P->Alin, x, xn);
        matvec(nx, nu, P->Blin, u, t);
        for (int i = 0; i < nx; ++i) xn[i] += t[i];
        if (A) memcpy(A, P->Alin, sizeof(double) * nx * nx);
        if (B) memcpy(B, P->Blin, sizeof(double) * nx * nu);
        return 0;
    }
    int n_sub = (int)P->params[9];
    if (n_sub < 1) n_sub = 1;
    double h = P->dt / n_sub;
    double S[MAXX * MAXN], Eu[MAXU * MAXN];          /* dz/d(x,u): state and input parts */
    memset(S, 0, sizeof S);
    memset(Eu, 0, sizeof Eu);
    for (int i = 0; i < nx; ++i) S[i * nz + i] = 1.0;
    for (int j = 0; j < nu; ++j) Eu[j * nz + nx + j] = 1.0;
    double z[MAXX];
    memcpy(z, x, sizeof(double) * nx);
    static const double cst[4] = {0.0, 0.5, 0.5, 1.0};
    static const double wts[4] = {1.0, 2.0, 2.0, 1.0};
    for (int sub = 0; sub < n_sub; ++sub) {
        double kprev[MAXX] = {0}, Dprev[MAXX * MAXN];
        memset(Dprev, 0, sizeof Dprev);
        double ksum[MAXX] = {0}, Dsum[MAXX * MAXN];
        memset(Dsum, 0, sizeof Dsum);
        for (int st = 0; st < 4; ++st) {
            double zs[MAXX], Ss[MAXX * MAXN], k[MAXX], D[MAXX * MAXN], Jx[MAXX * MAXX], Ju[MAXX * MAXU];
            for (int i = 0; i < nx; ++i) zs[i] = z[i] + cst[st] * h * kprev[i];
            for (int i = 0; i < nx * nz; ++i) Ss[i] = S[i] + cst[st] * h * Dprev[i];
            rhs(P, zs, u, k, Jx, Ju);
            for (int i = 0; i < nx; ++i) ksum[i] += wts[st] * k[i];
            memcpy(kprev, k, sizeof(double) * nx);
            if (!A && !B) continue;                    /* no Jacobian requested */
            double t1[MAXX * MAXN], t2[MAXX * MAXN];
            matmul(nx, nx, nz, Jx, Ss, t1);
            matmul(nx, nu, nz, Ju, Eu, t2);
            for (int i = 0; i < nx * nz; ++i) D[i] = t1[i] + t2[i];
            for (int i = 0; i < nx * nz; ++i) Dsum[i] += wts[st] * D[i];
            memcpy(Dprev, D, sizeof(double) * nx * nz);
        }
        for (int i = 0; i < nx; ++i) z[i] += h / 6.0 * ksum[i];
        for (int i = 0; i < nx * nz; ++i) S[i] += h / 6.0 * Dsum[i];
    }
    memcpy(xn, z, sizeof(double) * nx);
    if (A)
        for (int i = 0; i < nx; ++i)
            for (int j = 0; j < nx; ++j) A[i * nx + j] = S[i * nz + j];
    if (B)
        for (int i = 0; i < nx; ++i)
            for (int j = 0; j < nu; ++j) B[i * nu + j] = S[i * nz + nx + j];
    return 0;
}

/* Dynamics of the edge into node m from its parent's (x, u): the per-edge linear model when the
 * problem has one, else the parent's model (shared by all its children). */
static int edge_dynamics(const orc_problem *P, int m, const double *x, const double *u, double *xn, double *A,
                         double *B) {
    if (P->model == 2 && P->Aedge) {
        const int nx = P->nx, nu = P->nu;
        const double *Am = P->Aedge + (size_t)m * nx * nx, *Bm = P->Bedge + (size_t)m * nx * nu;
        double t[MAXX];
        matvec(nx, nx, Am, x, xn);
        matvec(nx, nu, Bm, u, t);
        for (int i = 0; i < nx; ++i) xn[i] += t[i];
        if (A) memcpy(A, Am, sizeof(double) * nx * nx);
        if (B) memcpy(B, Bm, sizeof(double) * nx * nu);
        return 0;
    }
    return orc_dynamics(P, x, u, xn, A, B);
}

/* ------------------------------------------------------------ tree helpers */
typedef struct {
    int n;
    int *first_child, *n_child, *child; /* children of i: child[first_child[i] .. +n_child[i]) ascending */
    int *stage;
} tree_t;

static int tree_build(const orc_problem *P, tree_t *T) {
    int n = P->n;
    T->n = n;
    T->first_child = (int *)calloc(n, sizeof(int));
    T->n_child = (int *)calloc(n, sizeof(int));
    T->child = (int *)calloc(n > 1 ? n - 1 : 1, sizeof(int));
    T->stage = (int *)calloc(n, sizeof(int));
    if (P->parent[0] != -1) return 0;
    for (int i = 1; i < n; ++i) {
        int p = P->parent[i];
        if (p < 0 || p >= i) return 0;
        T->n_child[p]++;
        T->stage[i] = T->stage[p] + 1;
    }
    int off = 0;
    for (int i = 0; i < n; ++i) { T->first_child[i] = off; off += T->n_child[i]; }
    int *fill = (int *)calloc(n, sizeof(int));
    for (int i = 1; i < n; ++i) {
        int p = P->parent[i];
        T->child[T->first_child[p] + fill[p]++] = i;
    }
    free(fill);
    return 1;
}
static void tree_free(tree_t *T) {
    free(T->first_child); free(T->n_child); free(T->child); free(T->stage);
}

/* number of constraint rows per node (same layout at every node) */
static int n_con(const orc_problem *P) { return 2 * P->nu * P->box_on + P->n_obs + 2 * P->lane_on; }

/* Constraint rows g(x, u) <= 0 of Eq. (bmpc) at node i, their Jacobians and existence flags.
 * Row layout: [u - u_hi (nu), u_lo - u (nu)] (box, non-leaf nodes), obstacle keep-out ellipses
 * as a normalised distance g = 1 - sqrt((d_par/a)^2 + (d_perp/b)^2 + eps) (non-root nodes),
 * lane [Y - hi, lo - Y] (non-root nodes). */
int orc_constraints(const orc_problem *P, int node, int is_leaf, const double *x, const double *u,
                    double *g, double *Jx, double *Ju, int *exists) {
    int nx = P->nx, nu = P->nu, nc = n_con(P), row = 0;
    memset(Jx, 0, sizeof(double) * nc * nx);
    memset(Ju, 0, sizeof(double) * nc * nu);
    for (int c = 0; c < nc; ++c) { g[c] = 0.0; exists[c] = 0; }
    if (P->box_on) {
        for (int j = 0; j < nu; ++j) {
            exists[row] = !is_leaf;
            g[row] = is_leaf ? 0.0 : u[j] - P->u_hi[j];
            Ju[row * nu + j] = 1.0;
            ++row;
        }
        for (int j = 0; j < nu; ++j) {
            exists[row] = !is_leaf;
            g[row] = is_leaf ? 0.0 : P->u_lo[j] - u[j];
            Ju[row * nu + j] = -1.0;
            ++row;
        }
    }
    for (int o = 0; o < P->n_obs; ++o) {
        const double *ob = P->obs + ((size_t)node * P->n_obs + o) * 5;
        double dx = x[0] - ob[0], dy = x[1] - ob[1];
        double ch = cos(ob[2]), sh = sin(ob[2]);
        double dpar = ch * dx + sh * dy, dper = -sh * dx + ch * dy;
        double a2 = ob[3] * ob[3], b2 = ob[4] * ob[4];
        double rr = sqrt(dpar * dpar / a2 + dper * dper / b2 + OBS_EPS);
        exists[row] = node != 0;
        g[row] = 1.0 - rr;
        Jx[row * nx + 0] = -(dpar / a2 * ch - dper / b2 * sh) / rr;
        Jx[row * nx + 1] = -(dpar / a2 * sh + dper / b2 * ch) / rr;
        ++row;
    }
    if (P->lane_on) {
        exists[row] = node != 0;
        g[row] = x[1] - P->lane_hi;
        Jx[row * nx + 1] = 1.0;
        ++row;
        exists[row] = node != 0;
        g[row] = P->lane_lo - x[1];
        Jx[row * nx + 1] = -1.0;
        ++row;
    }
    return row;
}

/* ------------------------------------------------------------ tree LQR (Sec. III-A) */
/* Solves the tree LQR problem of Eq. (lqr_tree_approx):
 *   min sum_i 1/2 dx'Q dx + du'M dx + 1/2 du'R du + q'dx + r'du   (leaves: Q, q only)
 *   s.t. dx_m = A_m dx_i + B_m du_i + c_m for m in ch(i), dx_0 = 0.
 * Backward: the modified Riccati recursion of Eq. (tree_Riccati) that sums the children's value
 * functions carried back through their edges (Q_xx = Q + sum A_m'P_m A_m, Q_ux = M + sum B_m'P_m A_m,
 * H = R + sum B_m'P_m B_m, q_x = q + sum A_m'(p_m + P_m c_m), q_u = r + sum B_m'(p_m + P_m c_m); with
 * the same A, B on every edge of a node this is the sum of P_m, p_m + P_m c_m first), with the
 * feedback law of Eq. (tree_feedback_laws); forward: the affine rollout along every root-to-leaf
 * path.  lam_m = P_m dx_m + p_m are the multipliers of the dynamics.
 * Arrays are per node, row-major: Q[n][nx][nx], M[n][nu][nx], R[n][nu][nu], q, r; A[n][nx][nx],
 * B[n][nx][nu], c[n][nx] of the edge into node m (row 0 unused). */
static int tree_lqr(const tree_t *T, int nx, int nu, const double *Q, const double *M, const double *R,
                    const double *q, const double *r, const double *A, const double *B, const double *c,
                    double *K, double *k, double *Pm, double *pv, double *dx, double *du, double *lam) {
    int n = T->n;
    for (int i = n - 1; i >= 0; --i) {       /* children always have larger index */
        double *Pi = Pm + (size_t)i * nx * nx, *pi = pv + (size_t)i * nx;
        if (T->n_child[i] == 0) {
            memcpy(Pi, Q + (size_t)i * nx * nx, sizeof(double) * nx * nx);
            memcpy(pi, q + (size_t)i * nx, sizeof(double) * nx);
            continue;
        }
        /* children's value functions through their edges */
        double Qxx[MAXX * MAXX] = {0}, Qux[MAXU * MAXX] = {0}, Quu[MAXU * MAXU] = {0}, qx[MAXX] = {0}, qu[MAXU] = {0};
        for (int t = 0; t < T->n_child[i]; ++t) {
            int m = T->child[T->first_child[i] + t];
            const double *Pc = Pm + (size_t)m * nx * nx, *pc = pv + (size_t)m * nx;
            const double *Am = A + (size_t)m * nx * nx, *Bm = B + (size_t)m * nx * nu;
            double pbar[MAXX], PA[MAXX * MAXX], PB[MAXX * MAXU], t1[MAXX * MAXX], t2[MAXU * MAXX], t3[MAXU * MAXU];
            double v1[MAXX], v2[MAXU];
            matvec(nx, nx, Pc, c + (size_t)m * nx, pbar);
            for (int e = 0; e < nx; ++e) pbar[e] += pc[e];
            matmul(nx, nx, nx, Pc, Am, PA);
            matmul(nx, nx, nu, Pc, Bm, PB);
            matTmul(nx, nx, nx, Am, PA, t1);
            matTmul(nu, nx, nx, Bm, PA, t2);
            matTmul(nu, nx, nu, Bm, PB, t3);
            matTvec(nx, nx, Am, pbar, v1);
            matTvec(nx, nu, Bm, pbar, v2);
            for (int e = 0; e < nx * nx; ++e) Qxx[e] += t1[e];
            for (int e = 0; e < nu * nx; ++e) Qux[e] += t2[e];
            for (int e = 0; e < nu * nu; ++e) Quu[e] += t3[e];
            for (int e = 0; e < nx; ++e) qx[e] += v1[e];
            for (int e = 0; e < nu; ++e) qu[e] += v2[e];
        }
        for (int e = 0; e < nx * nx; ++e) Qxx[e] += Q[(size_t)i * nx * nx + e];
        for (int e = 0; e < nu * nx; ++e) Qux[e] += M[(size_t)i * nu * nx + e];
        for (int e = 0; e < nu * nu; ++e) Quu[e] += R[(size_t)i * nu * nu + e];
        for (int e = 0; e < nx; ++e) qx[e] += q[(size_t)i * nx + e];
        for (int e = 0; e < nu; ++e) qu[e] += r[(size_t)i * nu + e];
        double L[MAXU * MAXU];
        if (!cholesky(nu, Quu, L)) return ORC_ERR_NUMERIC;
        double *Ki = K + (size_t)i * nu * nx, *ki = k + (size_t)i * nu;
        for (int e = 0; e < nu * nx; ++e) Ki[e] = -Qux[e];
        for (int e = 0; e < nu; ++e) ki[e] = -qu[e];
        chol_solve(nu, nx, L, Ki);
        chol_solve(nu, 1, L, ki);
        /* P = Qxx + Qux' K (symmetric in exact arithmetic; stored symmetrised), p = qx + Qux' k */
        double QK[MAXX * MAXX], Qk[MAXX];
        matTmul(nx, nu, nx, Qux, Ki, QK);
        matTvec(nu, nx, Qux, ki, Qk);
        for (int a = 0; a < nx; ++a)
            for (int b = 0; b < nx; ++b)
                Pi[a * nx + b] = 0.5 * ((Qxx[a * nx + b] + QK[a * nx + b]) + (Qxx[b * nx + a] + QK[b * nx + a]));
        for (int e = 0; e < nx; ++e) pi[e] = qx[e] + Qk[e];
    }
    /* forward sweep from the root (dx_0 = 0) */
    memset(dx, 0, sizeof(double) * nx);
    for (int i = 0; i < n; ++i) {
        if (T->n_child[i] == 0) { memset(du + (size_t)i * nu, 0, sizeof(double) * nu); continue; }
        const double *Ki = K + (size_t)i * nu * nx, *ki = k + (size_t)i * nu;
        double *dui = du + (size_t)i * nu;
        matvec(nu, nx, Ki, dx + (size_t)i * nx, dui);
        for (int e = 0; e < nu; ++e) dui[e] += ki[e];
        for (int t = 0; t < T->n_child[i]; ++t) {
            int m = T->child[T->first_child[i] + t];
            double Ax[MAXX], Bu[MAXX];
            matvec(nx, nx, A + (size_t)m * nx * nx, dx + (size_t)i * nx, Ax);
            matvec(nx, nu, B + (size_t)m * nx * nu, dui, Bu);
            for (int e = 0; e < nx; ++e) dx[(size_t)m * nx + e] = Ax[e] + Bu[e] + c[(size_t)m * nx + e];
        }
    }
    for (int i = 0; i < n; ++i) {
        double Pd[MAXX];
        matvec(nx, nx, Pm + (size_t)i * nx * nx, dx + (size_t)i * nx, Pd);
        for (int e = 0; e < nx; ++e) lam[(size_t)i * nx + e] = Pd[e] + pv[(size_t)i * nx + e];
    }
    return ORC_OK;
}

/* Per-edge copies of per-parent Jacobians: edge m takes the Jacobians of parent(m). */
static void parent_to_edge(int n, const int *parent, int nx, int nu, const double *A, const double *B, double *Ae,
                           double *Be) {
    memset(Ae, 0, sizeof(double) * nx * nx);
    memset(Be, 0, sizeof(double) * nx * nu);
    for (int m = 1; m < n; ++m) {
        memcpy(Ae + (size_t)m * nx * nx, A + (size_t)parent[m] * nx * nx, sizeof(double) * nx * nx);
        memcpy(Be + (size_t)m * nx * nu, B + (size_t)parent[m] * nx * nu, sizeof(double) * nx * nu);
    }
}

/* The tree LQR with A, B per parent (edge = 0: row i the Jacobians of node i's dynamics, shared by its
 * children) or per edge (edge = 1: row m the Jacobians of the edge into m). */
int orc_tree_lqr(int n, const int *parent, int nx, int nu, const double *Q, const double *M, const double *R,
                 const double *q, const double *r, const double *A, const double *B, const double *c,
                 double *K, double *k, double *Pm, double *pv, double *dx, double *du, double *lam, int edge) {
    if (nx > MAXX || nu > MAXU || n < 1) return ORC_ERR_INVALID;
    orc_problem P;
    memset(&P, 0, sizeof P);
    P.n = n;
    P.parent = parent;
    tree_t T;
    if (!tree_build(&P, &T)) { tree_free(&T); return ORC_ERR_INVALID; }
    double *Ae = NULL, *Be = NULL;
    if (!edge) {
        Ae = (double *)malloc(sizeof(double) * n * nx * nx);
        Be = (double *)malloc(sizeof(double) * n * nx * nu);
        parent_to_edge(n, parent, nx, nu, A, B, Ae, Be);
    }
    int st = tree_lqr(&T, nx, nu, Q, M, R, q, r, edge ? A : Ae, edge ? B : Be, c, K, k, Pm, pv, dx, du, lam);
    free(Ae); free(Be);
    tree_free(&T);
    return st;
}

/* ------------------------------------------------------------ tree LQR by scans (Sec. III-B) */
/* Conditional value function (CVF) of Eq. (sol_min) from a node x_k to one node x_i further down a
 * chain:  V(x_k, x_i) = max_lam  1/2 x_k' P x_k + p' x_k - 1/2 lam' C lam + lam' (x_i - A x_k - c)
 * (+ a constant).  An element with A = C = 0 and c = 0 is a plain value function 1/2 x'Px + p'x. */
typedef struct {
    double A[MAXX * MAXX], c[MAXX], C[MAXX * MAXX], p[MAXX], P[MAXX * MAXX];
} cvf_t;

/* Solves M X = Bm in place for m right-hand sides (n x n, Gaussian elimination with partial
 * pivoting); 0 if M is singular. */
static int lu_solve(int n, int m, const double *M, double *Bm) {
    double W[MAXX * MAXX];
    memcpy(W, M, sizeof(double) * n * n);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int i = col + 1; i < n; ++i)
            if (fabs(W[i * n + col]) > fabs(W[piv * n + col])) piv = i;
        if (W[piv * n + col] == 0.0) return 0;
        if (piv != col) {
            for (int j = 0; j < n; ++j) { double t = W[col * n + j]; W[col * n + j] = W[piv * n + j]; W[piv * n + j] = t; }
            for (int j = 0; j < m; ++j) { double t = Bm[col * m + j]; Bm[col * m + j] = Bm[piv * m + j]; Bm[piv * m + j] = t; }
        }
        for (int i = col + 1; i < n; ++i) {
            const double f = W[i * n + col] / W[col * n + col];
            for (int j = col; j < n; ++j) W[i * n + j] -= f * W[col * n + j];
            for (int j = 0; j < m; ++j) Bm[i * m + j] -= f * Bm[col * m + j];
        }
    }
    for (int i = n - 1; i >= 0; --i)
        for (int j = 0; j < m; ++j) {
            double v = Bm[i * m + j];
            for (int t = i + 1; t < n; ++t) v -= W[i * n + t] * Bm[t * m + j];
            Bm[i * m + j] = v / W[i * n + i];
        }
    return 1;
}

/* The associative operator of Eq. (V_ki_min): the CVF e1 from k to j followed by e2 from j to i,
 * minimised over x_j.  With E = I + C1 P2 (Eq. comb_rule):
 *   A = A2 E^-1 A1,  c = A2 E^-1 (c1 - C1 p2) + c2,  C = A2 E^-1 C1 A2' + C2,
 *   P = A1' E^-T P2 A1 + P1,  p = A1' E^-T (p2 + P2 c1) + p1.
 * The signs follow from the CVF form above (the printed equation's signs are not consistent with
 * one convention); the result equals the sequential Riccati recursion (tested). */
static int cvf_combine(int nx, const cvf_t *e1, const cvf_t *e2, cvf_t *out) {
    const int n = nx, m = 2 * nx + 1;
    double E[MAXX * MAXX], X[MAXX * (2 * MAXX + 1)];
    matmul(n, n, n, e1->C, e2->P, E);
    for (int i = 0; i < n; ++i) E[i * n + i] += 1.0;
    /* X = E^-1 [A1 | C1 A2' | c1 - C1 p2] */
    double C1A2t[MAXX * MAXX], C1p2[MAXX];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double v = 0.0;
            for (int t = 0; t < n; ++t) v += e1->C[i * n + t] * e2->A[j * n + t];
            C1A2t[i * n + j] = v;
        }
    matvec(n, n, e1->C, e2->p, C1p2);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            X[i * m + j] = e1->A[i * n + j];
            X[i * m + n + j] = C1A2t[i * n + j];
        }
        X[i * m + 2 * n] = e1->c[i] - C1p2[i];
    }
    if (!lu_solve(n, m, E, X)) return 0;
    /* F = E' = I + P2 C1; Y = F^-1 [P2 A1 | p2 + P2 c1] */
    double F[MAXX * MAXX], Y[MAXX * (MAXX + 1)], P2A1[MAXX * MAXX], P2c1[MAXX];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) F[i * n + j] = E[j * n + i];
    matmul(n, n, n, e2->P, e1->A, P2A1);
    matvec(n, n, e2->P, e1->c, P2c1);
    const int m2 = n + 1;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) Y[i * m2 + j] = P2A1[i * n + j];
        Y[i * m2 + n] = e2->p[i] + P2c1[i];
    }
    if (!lu_solve(n, m2, F, Y)) return 0;
    cvf_t r;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            double a = 0.0, cc = 0.0, pp = 0.0;
            for (int t = 0; t < n; ++t) {
                a += e2->A[i * n + t] * X[t * m + j];
                cc += e2->A[i * n + t] * X[t * m + n + j];
                pp += e1->A[t * n + i] * Y[t * m2 + j];
            }
            r.A[i * n + j] = a;
            r.C[i * n + j] = cc + e2->C[i * n + j];
            r.P[i * n + j] = pp + e1->P[i * n + j];
        }
        double cv = 0.0, pv = 0.0;
        for (int t = 0; t < n; ++t) {
            cv += e2->A[i * n + t] * X[t * m + 2 * n];
            pv += e1->A[t * n + i] * Y[t * m2 + n];
        }
        r.c[i] = cv + e2->c[i];
        r.p[i] = pv + e1->p[i];
    }
    *out = r;
    return 1;
}

/* One-step CVF of a node with a single child (Eq. sol_min for one stage): the stage cost
 * 1/2 x'Qx + q'x + 1/2 u'Ru + r'u + u'Mx minimised over u subject to x_m = A x + B u + c_m gives
 *   C = B R^-1 B',  A~ = A - B R^-1 M,  c~ = c_m - B R^-1 r,  P~ = Q - M' R^-1 M,  p~ = q - M' R^-1 r. */
static int cvf_step(int nx, int nu, const double *Q, const double *M, const double *R, const double *q,
                    const double *r, const double *A, const double *B, const double *cm, cvf_t *e) {
    double L[MAXU * MAXU], Z[MAXU * (2 * MAXX + 1)];
    if (!cholesky(nu, R, L)) return 0;
    const int m = 2 * nx + 1;   /* Z = R^-1 [B' | M | r] */
    for (int a = 0; a < nu; ++a) {
        for (int j = 0; j < nx; ++j) {
            Z[a * m + j] = B[j * nu + a];
            Z[a * m + nx + j] = M[a * nx + j];
        }
        Z[a * m + 2 * nx] = r[a];
    }
    chol_solve(nu, m, L, Z);
    for (int i = 0; i < nx; ++i) {
        for (int j = 0; j < nx; ++j) {
            double cc = 0.0, bm = 0.0, mm = 0.0;
            for (int a = 0; a < nu; ++a) {
                cc += B[i * nu + a] * Z[a * m + j];
                bm += B[i * nu + a] * Z[a * m + nx + j];
                mm += M[a * nx + i] * Z[a * m + nx + j];
            }
            e->C[i * nx + j] = cc;
            e->A[i * nx + j] = A[i * nx + j] - bm;
            e->P[i * nx + j] = Q[i * nx + j] - mm;
        }
        double br = 0.0, mr = 0.0;
        for (int a = 0; a < nu; ++a) {
            br += B[i * nu + a] * Z[a * m + 2 * nx];
            mr += M[a * nx + i] * Z[a * m + 2 * nx];
        }
        e->c[i] = cm[i] - br;
        e->p[i] = q[i] - mr;
    }
    return 1;
}

/* Feedback law of Eq. (tree_feedback_laws) at non-leaf node i from its children's value functions,
 * and its own value function (P_i, p_i). */
static int tree_law(const tree_t *T, int i, int nx, int nu, const double *Q, const double *M, const double *R,
                    const double *q, const double *r, const double *A, const double *B, const double *c,
                    const double *Pm, const double *pv, double *Ki, double *ki, double *Pi, double *pi) {
    double Qxx[MAXX * MAXX] = {0}, Qux[MAXU * MAXX] = {0}, Quu[MAXU * MAXU] = {0}, qx[MAXX] = {0}, qu[MAXU] = {0};
    for (int t = 0; t < T->n_child[i]; ++t) {   /* children through their edges (A, B, c of edge ch) */
        const int ch = T->child[T->first_child[i] + t];
        const double *Pc = Pm + (size_t)ch * nx * nx, *Am = A + (size_t)ch * nx * nx, *Bm = B + (size_t)ch * nx * nu;
        double pbar[MAXX], PA[MAXX * MAXX], PB[MAXX * MAXU], t1[MAXX * MAXX], t2[MAXU * MAXX], t3[MAXU * MAXU];
        double v1[MAXX], v2[MAXU];
        matvec(nx, nx, Pc, c + (size_t)ch * nx, pbar);
        for (int e = 0; e < nx; ++e) pbar[e] += pv[(size_t)ch * nx + e];
        matmul(nx, nx, nx, Pc, Am, PA);
        matmul(nx, nx, nu, Pc, Bm, PB);
        matTmul(nx, nx, nx, Am, PA, t1);
        matTmul(nu, nx, nx, Bm, PA, t2);
        matTmul(nu, nx, nu, Bm, PB, t3);
        matTvec(nx, nx, Am, pbar, v1);
        matTvec(nx, nu, Bm, pbar, v2);
        for (int e = 0; e < nx * nx; ++e) Qxx[e] += t1[e];
        for (int e = 0; e < nu * nx; ++e) Qux[e] += t2[e];
        for (int e = 0; e < nu * nu; ++e) Quu[e] += t3[e];
        for (int e = 0; e < nx; ++e) qx[e] += v1[e];
        for (int e = 0; e < nu; ++e) qu[e] += v2[e];
    }
    for (int e = 0; e < nx * nx; ++e) Qxx[e] += Q[(size_t)i * nx * nx + e];
    for (int e = 0; e < nu * nx; ++e) Qux[e] += M[(size_t)i * nu * nx + e];
    for (int e = 0; e < nu * nu; ++e) Quu[e] += R[(size_t)i * nu * nu + e];
    for (int e = 0; e < nx; ++e) qx[e] += q[(size_t)i * nx + e];
    for (int e = 0; e < nu; ++e) qu[e] += r[(size_t)i * nu + e];
    double L[MAXU * MAXU];
    if (!cholesky(nu, Quu, L)) return 0;
    for (int e = 0; e < nu * nx; ++e) Ki[e] = -Qux[e];
    for (int e = 0; e < nu; ++e) ki[e] = -qu[e];
    chol_solve(nu, nx, L, Ki);
    chol_solve(nu, 1, L, ki);
    if (Pi) {
        double QK[MAXX * MAXX], Qk[MAXX];
        matTmul(nx, nu, nx, Qux, Ki, QK);
        matTvec(nu, nx, Qux, ki, Qk);
        for (int a = 0; a < nx; ++a)
            for (int b = 0; b < nx; ++b)
                Pi[a * nx + b] = 0.5 * ((Qxx[a * nx + b] + QK[a * nx + b]) + (Qxx[b * nx + a] + QK[b * nx + a]));
        for (int e = 0; e < nx; ++e) pi[e] = qx[e] + Qk[e];
    }
    return 1;
}

/* The tree LQR of Eq. (lqr_tree_approx) the way Sec. III-B organises it, with the branch points
 * handled as follows (at a node with several children the one-step CVF couples the children, so
 * the separable combination of Eq. tree_comb_rule holds only along non-branching segments):
 *  1. every maximal chain of single-child nodes ending at a leaf or a branch node is a segment; the
 *     value function at its end (a leaf's terminal cost, or a branch node's tree Riccati step from
 *     its children) is the last element, and an inclusive suffix scan (Hillis-Steele, span doubling)
 *     of the one-step CVFs with cvf_combine gives the value function of every node of the segment;
 *     segments are processed from the deepest end upward;
 *  2. the feedback laws of Eq. (tree_feedback_laws) at every non-leaf node;
 *  3. along every root-to-leaf path, an inclusive prefix scan of the closed-loop affine maps
 *     x_m = (A_n + B_n K_n) x_n + (c_m + B_n k_n) (Eq. forward_comb_rule) from dx_0 = 0.
 * Outputs as orc_tree_lqr. */
static int tree_lqr_scan(const tree_t *Tp, const int *parent, int nx, int nu, const double *Q, const double *M,
                         const double *R, const double *q, const double *r, const double *A, const double *B,
                         const double *c, double *K, double *k, double *Pm, double *pv, double *dx, double *du,
                         double *lam) {
    const tree_t T = *Tp;
    const int n = T.n;
    int st = ORC_OK;
    int *chain = (int *)malloc(sizeof(int) * n);
    cvf_t *S = (cvf_t *)malloc(sizeof(cvf_t) * (n + 1)), *S2 = (cvf_t *)malloc(sizeof(cvf_t) * (n + 1));
    /* 1. backward: segments, deepest end first (children have larger indices) */
    for (int b = n - 1; b >= 0 && st == ORC_OK; --b) {
        if (T.n_child[b] == 1) continue;   /* not the end of a segment */
        double *Pb = Pm + (size_t)b * nx * nx, *pb = pv + (size_t)b * nx;
        if (T.n_child[b] == 0) {
            memcpy(Pb, Q + (size_t)b * nx * nx, sizeof(double) * nx * nx);
            memcpy(pb, q + (size_t)b * nx, sizeof(double) * nx);
        } else if (!tree_law(&T, b, nx, nu, Q, M, R, q, r, A, B, c, Pm, pv, K + (size_t)b * nu * nx,
                             k + (size_t)b * nu, Pb, pb)) {
            st = ORC_ERR_NUMERIC;
            break;
        }
        int L = 0;   /* single-child ancestors of b, top first */
        for (int a = b ? parent[b] : -1; a >= 0 && T.n_child[a] == 1; a = a ? parent[a] : -1) chain[L++] = a;
        for (int i = 0; i < L / 2; ++i) { int t = chain[i]; chain[i] = chain[L - 1 - i]; chain[L - 1 - i] = t; }
        if (L == 0) continue;
        for (int i = 0; i < L; ++i) {
            const int a = chain[i], ch = T.child[T.first_child[a]];
            if (!cvf_step(nx, nu, Q + (size_t)a * nx * nx, M + (size_t)a * nu * nx, R + (size_t)a * nu * nu,
                          q + (size_t)a * nx, r + (size_t)a * nu, A + (size_t)ch * nx * nx, B + (size_t)ch * nx * nu,
                          c + (size_t)ch * nx, &S[i])) {
                st = ORC_ERR_NUMERIC;
                break;
            }
        }
        if (st != ORC_OK) break;
        memset(&S[L], 0, sizeof(cvf_t));
        memcpy(S[L].P, Pb, sizeof(double) * nx * nx);
        memcpy(S[L].p, pb, sizeof(double) * nx);
        for (int d = 1; d <= L && st == ORC_OK; d *= 2) {
            for (int i = 0; i <= L; ++i) {
                if (i + d <= L) {
                    if (!cvf_combine(nx, &S[i], &S[i + d], &S2[i])) { st = ORC_ERR_NUMERIC; break; }
                } else {
                    S2[i] = S[i];
                }
            }
            cvf_t *t = S; S = S2; S2 = t;
        }
        for (int i = 0; i < L && st == ORC_OK; ++i) {
            memcpy(Pm + (size_t)chain[i] * nx * nx, S[i].P, sizeof(double) * nx * nx);
            memcpy(pv + (size_t)chain[i] * nx, S[i].p, sizeof(double) * nx);
        }
    }
    /* 2. feedback laws of the single-child nodes (branch nodes got theirs with their step) */
    for (int i = 0; i < n && st == ORC_OK; ++i)
        if (T.n_child[i] == 1 && !tree_law(&T, i, nx, nu, Q, M, R, q, r, A, B, c, Pm, pv, K + (size_t)i * nu * nx,
                                           k + (size_t)i * nu, NULL, NULL))
            st = ORC_ERR_NUMERIC;
    /* 3. forward: prefix scans of the closed-loop maps along every root-to-leaf path */
    double *GA = (double *)malloc(sizeof(double) * (n + 1) * nx * nx), *Gc = (double *)malloc(sizeof(double) * (n + 1) * nx);
    double *HA = (double *)malloc(sizeof(double) * (n + 1) * nx * nx), *Hc = (double *)malloc(sizeof(double) * (n + 1) * nx);
    for (int leaf = 0; leaf < n && st == ORC_OK; ++leaf) {
        if (T.n_child[leaf] != 0) continue;
        int D = 0;
        for (int a = leaf; a > 0; a = parent[a]) chain[D++] = a;   /* path without the root, leaf first */
        for (int i = 0; i < D / 2; ++i) { int t = chain[i]; chain[i] = chain[D - 1 - i]; chain[D - 1 - i] = t; }
        /* element j maps dx of parent(chain[j]) to dx of chain[j] */
        for (int j = 0; j < D; ++j) {
            const int m = chain[j], a = parent[m];
            const double *Ka = K + (size_t)a * nu * nx, *ka = k + (size_t)a * nu, *Ba = B + (size_t)m * nx * nu;
            for (int i = 0; i < nx; ++i) {
                for (int t = 0; t < nx; ++t) {
                    double v = A[(size_t)m * nx * nx + i * nx + t];
                    for (int s2 = 0; s2 < nu; ++s2) v += Ba[i * nu + s2] * Ka[s2 * nx + t];
                    GA[(size_t)j * nx * nx + i * nx + t] = v;
                }
                double v = c[(size_t)m * nx + i];
                for (int s2 = 0; s2 < nu; ++s2) v += Ba[i * nu + s2] * ka[s2];
                Gc[(size_t)j * nx + i] = v;
            }
        }
        for (int d = 1; d < D; d *= 2) {   /* inclusive prefix scan: G_j <- G_j o G_{j-d} */
            for (int j = 0; j < D; ++j) {
                if (j >= d) {
                    const double *A2 = GA + (size_t)j * nx * nx, *A1 = GA + (size_t)(j - d) * nx * nx;
                    matmul(nx, nx, nx, A2, A1, HA + (size_t)j * nx * nx);
                    matvec(nx, nx, A2, Gc + (size_t)(j - d) * nx, Hc + (size_t)j * nx);
                    for (int i = 0; i < nx; ++i) Hc[(size_t)j * nx + i] += Gc[(size_t)j * nx + i];
                } else {
                    memcpy(HA + (size_t)j * nx * nx, GA + (size_t)j * nx * nx, sizeof(double) * nx * nx);
                    memcpy(Hc + (size_t)j * nx, Gc + (size_t)j * nx, sizeof(double) * nx);
                }
            }
            double *t = GA; GA = HA; HA = t;
            t = Gc; Gc = Hc; Hc = t;
        }
        for (int j = 0; j < D; ++j) memcpy(dx + (size_t)chain[j] * nx, Gc + (size_t)j * nx, sizeof(double) * nx);
    }
    memset(dx, 0, sizeof(double) * nx);
    for (int i = 0; i < n && st == ORC_OK; ++i) {
        double *dui = du + (size_t)i * nu;
        if (T.n_child[i] == 0) {
            memset(dui, 0, sizeof(double) * nu);
        } else {
            matvec(nu, nx, K + (size_t)i * nu * nx, dx + (size_t)i * nx, dui);
            for (int e = 0; e < nu; ++e) dui[e] += k[(size_t)i * nu + e];
        }
        double Pd[MAXX];
        matvec(nx, nx, Pm + (size_t)i * nx * nx, dx + (size_t)i * nx, Pd);
        for (int e = 0; e < nx; ++e) lam[(size_t)i * nx + e] = Pd[e] + pv[(size_t)i * nx + e];
    }
    free(GA); free(Gc); free(HA); free(Hc);
    free(chain); free(S); free(S2);
    return st;
}

int orc_tree_lqr_scan(int n, const int *parent, int nx, int nu, const double *Q, const double *M, const double *R,
                      const double *q, const double *r, const double *A, const double *B, const double *c, double *K,
                      double *k, double *Pm, double *pv, double *dx, double *du, double *lam, int edge) {
    if (nx > MAXX || nu > MAXU || n < 1) return ORC_ERR_INVALID;
    orc_problem Pr;
    memset(&Pr, 0, sizeof Pr);
    Pr.n = n;
    Pr.parent = parent;
    tree_t T;
    if (!tree_build(&Pr, &T)) { tree_free(&T); return ORC_ERR_INVALID; }
    double *Ae = NULL, *Be = NULL;
    if (!edge) {
        Ae = (double *)malloc(sizeof(double) * n * nx * nx);
        Be = (double *)malloc(sizeof(double) * n * nx * nu);
        parent_to_edge(n, parent, nx, nu, A, B, Ae, Be);
    }
    const int st = tree_lqr_scan(&T, parent, nx, nu, Q, M, R, q, r, edge ? A : Ae, edge ? B : Be, c, K, k, Pm, pv, dx,
                                 du, lam);
    free(Ae); free(Be);
    tree_free(&T);
    return st;
}

/* ------------------------------------------------------------ exact second derivatives */
/* Hyper-dual numbers (Fike and Alonso, 2011): a + b e1 + c e2 + d e1 e2 with e1^2 = e2^2 = 0.
 * Evaluating a function at z + e1 v + e2 w gives its value in a, the directional derivatives
 * along v and w in b and c, and the second derivative v' H w in d, exactly (no truncation). */
typedef struct { double a, b, c, d; } hd;

static hd hd_c(double v) { hd r = {v, 0.0, 0.0, 0.0}; return r; }
static hd hd_add(hd x, hd y) { hd r = {x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d}; return r; }
static hd hd_sub(hd x, hd y) { hd r = {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d}; return r; }
static hd hd_scale(hd x, double s) { hd r = {s * x.a, s * x.b, s * x.c, s * x.d}; return r; }
static hd hd_mul(hd x, hd y) {
    hd r = {x.a * y.a, x.a * y.b + x.b * y.a, x.a * y.c + x.c * y.a, x.a * y.d + x.b * y.c + x.c * y.b + x.d * y.a};
    return r;
}
/* f(x) for a scalar function with value f0, first derivative f1 and second derivative f2 at x.a */
static hd hd_fn(hd x, double f0, double f1, double f2) {
    hd r = {f0, f1 * x.b, f1 * x.c, f1 * x.d + f2 * x.b * x.c};
    return r;
}
static hd hd_inv(hd x) { return hd_fn(x, 1.0 / x.a, -1.0 / (x.a * x.a), 2.0 / (x.a * x.a * x.a)); }
static hd hd_div(hd x, hd y) { return hd_mul(x, hd_inv(y)); }
static hd hd_sin(hd x) { return hd_fn(x, sin(x.a), cos(x.a), -sin(x.a)); }
static hd hd_cos(hd x) { return hd_fn(x, cos(x.a), -sin(x.a), -cos(x.a)); }
static hd hd_tan(hd x) {
    const double t = tan(x.a), s = 1.0 + t * t;
    return hd_fn(x, t, s, 2.0 * t * s);
}
static hd hd_atan(hd x) {
    const double s = 1.0 + x.a * x.a;
    return hd_fn(x, atan(x.a), 1.0 / s, -2.0 * x.a / (s * s));
}
static hd hd_sqrt(hd x) {
    const double r = sqrt(x.a);
    return hd_fn(x, r, 0.5 / r, -0.25 / (r * x.a));
}

/* The continuous right-hand side of rhs() in hyper-dual arithmetic (the same formulas). */
static void rhs_hd(const orc_problem *P, const hd *s, const hd *u, hd *f) {
    const double *prm = P->params;
    if (P->model == 0) {
        const double L = prm[0];
        f[0] = hd_mul(s[3], hd_cos(s[2]));
        f[1] = hd_mul(s[3], hd_sin(s[2]));
        f[2] = hd_scale(hd_mul(s[3], hd_tan(u[1])), 1.0 / L);
        f[3] = u[0];
        return;
    }
    if (P->model == 3) {
        f[0] = hd_mul(s[3], hd_cos(s[2]));
        f[1] = hd_mul(s[3], hd_sin(s[2]));
        f[2] = u[1];
        f[3] = u[0];
        return;
    }
    /* dynamic bicycle */
    const double m = prm[1], Iz = prm[2], lf = prm[3], lr = prm[4], Cf = prm[5], Cr = prm[6];
    const double vmin = prm[7], veps = prm[8];
    const hd psi = s[2], vx = s[3], vy = s[4], r = s[5], a = u[0], d = u[1];
    const hd dv = hd_sub(vx, hd_c(vmin));
    const hd w = hd_sqrt(hd_add(hd_mul(dv, dv), hd_c(veps * veps)));
    const hd vb = hd_scale(hd_add(hd_add(vx, hd_c(vmin)), w), 0.5);
    const hd tf = hd_div(hd_add(vy, hd_scale(r, lf)), vb), tr = hd_div(hd_sub(vy, hd_scale(r, lr)), vb);
    const hd af = hd_sub(hd_atan(tf), d), ar = hd_atan(tr);
    const hd Ff = hd_scale(af, -Cf), Fr = hd_scale(ar, -Cr);
    const hd cp = hd_cos(psi), sp = hd_sin(psi);
    f[0] = hd_sub(hd_mul(vx, cp), hd_mul(vy, sp));
    f[1] = hd_add(hd_mul(vx, sp), hd_mul(vy, cp));
    f[2] = r;
    f[3] = hd_add(a, hd_mul(r, vy));
    f[4] = hd_sub(hd_scale(hd_add(Ff, Fr), 1.0 / m), hd_mul(r, vx));
    f[5] = hd_scale(hd_sub(hd_scale(Ff, lf), hd_scale(Fr, lr)), 1.0 / Iz);
}

/* Second derivatives of the discrete dynamics: H[j][k] = sum_i mu_i d^2 f_i / dz_j dz_k with z = (x, u),
 * for the RK4 map of orc_dynamics (n_sub substeps) evaluated in hyper-dual arithmetic, one pair
 * (j, k) at a time.  The linear model has none. */
static void dyn_hessian(const orc_problem *P, const double *x, const double *u, const double *mu, double *H) {
    const int nx = P->nx, nu = P->nu, nz = nx + nu;
    memset(H, 0, sizeof(double) * nz * nz);
    if (P->model == 2) return;
    int n_sub = (int)P->params[9];
    if (n_sub < 1) n_sub = 1;
    const double h = P->dt / n_sub;
    static const double cst[4] = {0.0, 0.5, 0.5, 1.0};
    static const double wts[4] = {1.0, 2.0, 2.0, 1.0};
    for (int j = 0; j < nz; ++j)
        for (int k = j; k < nz; ++k) {
            hd z[MAXX], uu[MAXU];
            for (int i = 0; i < nx; ++i) z[i] = hd_c(x[i]);
            for (int i = 0; i < nu; ++i) uu[i] = hd_c(u[i]);
            hd *vj = j < nx ? &z[j] : &uu[j - nx], *vk = k < nx ? &z[k] : &uu[k - nx];
            vj->b = 1.0;
            vk->c = 1.0;
            for (int sub = 0; sub < n_sub; ++sub) {
                hd kp[MAXX], ks[MAXX];
                for (int i = 0; i < nx; ++i) { kp[i] = hd_c(0.0); ks[i] = hd_c(0.0); }
                for (int st = 0; st < 4; ++st) {
                    hd zs[MAXX], kk[MAXX];
                    for (int i = 0; i < nx; ++i) zs[i] = hd_add(z[i], hd_scale(kp[i], cst[st] * h));
                    rhs_hd(P, zs, uu, kk);
                    for (int i = 0; i < nx; ++i) { ks[i] = hd_add(ks[i], hd_scale(kk[i], wts[st])); kp[i] = kk[i]; }
                }
                for (int i = 0; i < nx; ++i) z[i] = hd_add(z[i], hd_scale(ks[i], h / 6.0));
            }
            double v = 0.0;
            for (int i = 0; i < nx; ++i) v += mu[i] * z[i].d;
            H[j * nz + k] = v;
            H[k * nz + j] = v;
        }
}

/* Second derivatives of the keep-out value g = 1 - sqrt((d_par/a)^2 + (d_perp/b)^2 + eps) in (X, Y),
 * hyper-dual like dyn_hessian: out = [gxx, gxy, gyy]. */
static void obs_hessian(const double *ob, double X, double Y, double *out) {
    const double ch = cos(ob[2]), sh = sin(ob[2]), a2 = ob[3] * ob[3], b2 = ob[4] * ob[4];
    const int pairs[3][2] = {{0, 0}, {0, 1}, {1, 1}};
    for (int t = 0; t < 3; ++t) {
        hd px = hd_c(X), py = hd_c(Y);
        hd *v1 = pairs[t][0] ? &py : &px, *v2 = pairs[t][1] ? &py : &px;
        v1->b = 1.0;
        v2->c = 1.0;
        const hd dx = hd_sub(px, hd_c(ob[0])), dy = hd_sub(py, hd_c(ob[1]));
        const hd dpar = hd_add(hd_scale(dx, ch), hd_scale(dy, sh)), dper = hd_sub(hd_scale(dy, ch), hd_scale(dx, sh));
        const hd q = hd_add(hd_add(hd_scale(hd_mul(dpar, dpar), 1.0 / a2), hd_scale(hd_mul(dper, dper), 1.0 / b2)),
                            hd_c(OBS_EPS));
        out[t] = -hd_sqrt(q).d;
    }
}

/* Eigen-decomposition of a symmetric n x n matrix by cyclic Jacobi rotations (Golub and Van Loan,
 * Sec. 8.5): S = V diag(ev) V'.  Sweeps until the off-diagonal mass is below 1e-30 of the total. */
static void jacobi_eig(int n, const double *S, double *ev, double *Vm) {
    double Aw[MAXN * MAXN];
    memcpy(Aw, S, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Vm[i * n + j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += Aw[i * n + j] * Aw[i * n + j];
                if (i != j) off += Aw[i * n + j] * Aw[i * n + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = Aw[p * n + q];
                if (apq == 0.0) continue;
                const double theta = (Aw[q * n + q] - Aw[p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {   /* A <- J' A J with the rotation in the (p, q) plane */
                    const double akp = Aw[k * n + p], akq = Aw[k * n + q];
                    Aw[k * n + p] = c * akp - s * akq;
                    Aw[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = Aw[p * n + k], aqk = Aw[q * n + k];
                    Aw[p * n + k] = c * apk - s * aqk;
                    Aw[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = Vm[k * n + p], vkq = Vm[k * n + q];
                    Vm[k * n + p] = c * vkp - s * vkq;
                    Vm[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) ev[i] = Aw[i * n + i];
}

/* Eigenvalue modification (Nocedal and Wright, Sec. 3.4): S <- V diag(max(ev, delta)) V' with
 * delta = EIG_FLOOR max(1, max |ev|), so that the modified block is positive definite. */
#define EIG_FLOOR 1e-6
static void eig_modify(int n, double *S) {
    double ev[MAXN], Vm[MAXN * MAXN], emax = 1.0;
    jacobi_eig(n, S, ev, Vm);
    for (int i = 0; i < n; ++i) if (fabs(ev[i]) > emax) emax = fabs(ev[i]);
    const double delta = EIG_FLOOR * emax;
    for (int i = 0; i < n; ++i) if (ev[i] < delta) ev[i] = delta;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double v = 0.0;
            for (int k = 0; k < n; ++k) v += Vm[i * n + k] * ev[k] * Vm[j * n + k];
            S[i * n + j] = v;
        }
}

/* ------------------------------------------------------------ AL quadratisation (Sec. IV-A) */
typedef struct {
    tree_t T;
    int nc;
    double *A, *B, *f;              /* per edge (row m: into node m): Jacobians and f_m(x_p(m), u_p(m)) */
    double *d;                      /* defect d_m = f_p(m) - x_m per node (row 0 zero) */
    double *Q, *M, *R, *q, *r;      /* GN quadratisation of L_a */
    double *g;                      /* constraint values [n][nc] */
    int *ex;                        /* existence flags [n][nc] */
    double *K, *k, *P, *p, *dx, *du, *lqp;
    double La;                      /* L_a value at the linearisation point */
} work_t;

static void work_alloc(work_t *W, const orc_problem *P) {
    int n = P->n, nx = P->nx, nu = P->nu, nc = n_con(P);
    W->nc = nc;
    W->A = (double *)calloc((size_t)n * nx * nx, sizeof(double));
    W->B = (double *)calloc((size_t)n * nx * nu, sizeof(double));
    W->f = (double *)calloc((size_t)n * nx, sizeof(double));
    W->d = (double *)calloc((size_t)n * nx, sizeof(double));
    W->Q = (double *)calloc((size_t)n * nx * nx, sizeof(double));
    W->M = (double *)calloc((size_t)n * nu * nx, sizeof(double));
    W->R = (double *)calloc((size_t)n * nu * nu, sizeof(double));
    W->q = (double *)calloc((size_t)n * nx, sizeof(double));
    W->r = (double *)calloc((size_t)n * nu, sizeof(double));
    W->g = (double *)calloc((size_t)n * (nc ? nc : 1), sizeof(double));
    W->ex = (int *)calloc((size_t)n * (nc ? nc : 1), sizeof(int));
    W->K = (double *)calloc((size_t)n * nu * nx, sizeof(double));
    W->k = (double *)calloc((size_t)n * nu, sizeof(double));
    W->P = (double *)calloc((size_t)n * nx * nx, sizeof(double));
    W->p = (double *)calloc((size_t)n * nx, sizeof(double));
    W->dx = (double *)calloc((size_t)n * nx, sizeof(double));
    W->du = (double *)calloc((size_t)n * nu, sizeof(double));
    W->lqp = (double *)calloc((size_t)n * nx, sizeof(double));
}
static void work_free(work_t *W) {
    free(W->A); free(W->B); free(W->f); free(W->d); free(W->Q); free(W->M); free(W->R);
    free(W->q); free(W->r); free(W->g); free(W->ex); free(W->K); free(W->k); free(W->P);
    free(W->p); free(W->dx); free(W->du); free(W->lqp);
    tree_free(&W->T);
}

/* Node cost l_i (stage) or l_f,i (leaf) of Eq. (bmpc): weighted quadratic tracking. */
static double node_cost(const orc_problem *P, int i, int leaf, const double *x, const double *u,
                        double *lx, double *lu) {
    int nx = P->nx, nu = P->nu;
    double w = P->weight ? P->weight[i] : 1.0, v = 0.0;
    const double *Qd = leaf ? P->QNw : P->Qw;
    for (int j = 0; j < nx; ++j) {
        double e = x[j] - P->xref[(size_t)i * nx + j];
        v += 0.5 * w * Qd[j] * e * e;
        if (lx) lx[j] = w * Qd[j] * e;
    }
    if (!leaf)
        for (int j = 0; j < nu; ++j) {
            v += 0.5 * w * P->Rw[j] * u[j] * u[j];
            if (lu) lu[j] = w * P->Rw[j] * u[j];
        }
    return v;
}

/* Evaluate everything the iteration needs at (x, u): dynamics, defects, the GN
 * quadratisation of L_a (Eq. AL) with fixed (y, rho), and L_a itself. */
static void linearise(const orc_problem *P, work_t *W, const double *x, const double *u, const double *y,
                      double rho) {
    int n = P->n, nx = P->nx, nu = P->nu, nc = W->nc;
    const tree_t *T = &W->T;
    double La = 0.0;
    for (int i = 0; i < n; ++i) {
        int leaf = T->n_child[i] == 0;
        const double *xi = x + (size_t)i * nx, *ui = u + (size_t)i * nu;
        double lx[MAXX] = {0}, lu[MAXU] = {0};
        La += node_cost(P, i, leaf, xi, ui, lx, lu);
        double *Qi = W->Q + (size_t)i * nx * nx, *Mi = W->M + (size_t)i * nu * nx, *Ri = W->R + (size_t)i * nu * nu;
        double *qi = W->q + (size_t)i * nx, *ri = W->r + (size_t)i * nu;
        double w = P->weight ? P->weight[i] : 1.0;
        memset(Qi, 0, sizeof(double) * nx * nx);
        memset(Mi, 0, sizeof(double) * nu * nx);
        memset(Ri, 0, sizeof(double) * nu * nu);
        for (int j = 0; j < nx; ++j) { Qi[j * nx + j] = w * (leaf ? P->QNw[j] : P->Qw[j]); qi[j] = lx[j]; }
        for (int j = 0; j < nu; ++j) { Ri[j * nu + j] = leaf ? 0.0 : w * P->Rw[j]; ri[j] = leaf ? 0.0 : lu[j]; }
        if (nc) {
            double Jx[64 * MAXX], Ju[64 * MAXU];
            double *gi = W->g + (size_t)i * nc;
            int *ei = W->ex + (size_t)i * nc;
            orc_constraints(P, i, leaf, xi, ui, gi, Jx, Ju, ei);
            for (int c = 0; c < nc; ++c) {
                if (!ei[c]) continue;
                double s = y[(size_t)i * nc + c] + rho * gi[c];
                if (s > 0.0) {
                    double pen = s / rho;     /* max(0, g + y/rho) */
                    La += 0.5 * rho * pen * pen;
                    for (int a = 0; a < nx; ++a) qi[a] += s * Jx[c * nx + a];
                    for (int a = 0; a < nu; ++a) ri[a] += s * Ju[c * nu + a];
                    for (int a = 0; a < nx; ++a)
                        for (int b = 0; b < nx; ++b) Qi[a * nx + b] += rho * Jx[c * nx + a] * Jx[c * nx + b];
                    for (int a = 0; a < nu; ++a)
                        for (int b = 0; b < nx; ++b) Mi[a * nx + b] += rho * Ju[c * nu + a] * Jx[c * nx + b];
                    for (int a = 0; a < nu; ++a)
                        for (int b = 0; b < nu; ++b) Ri[a * nu + b] += rho * Ju[c * nu + a] * Ju[c * nu + b];
                }
            }
        }
    }
    /* the dynamics of every edge (into node m, from its parent) and the defects d_m = f_m - x_m */
    memset(W->d, 0, sizeof(double) * nx);
    for (int m = 1; m < n; ++m) {
        int pnt = P->parent[m];
        edge_dynamics(P, m, x + (size_t)pnt * nx, u + (size_t)pnt * nu, W->f + (size_t)m * nx,
                      W->A + (size_t)m * nx * nx, W->B + (size_t)m * nx * nu);
        for (int j = 0; j < nx; ++j) W->d[(size_t)m * nx + j] = W->f[(size_t)m * nx + j] - x[(size_t)m * nx + j];
    }
    W->La = La;
}

/* The exact Hessian option of Sec. IV-A: every node's block [[Q, M'], [M, R]] of the Hessian of the
 * Lagrangian L_a + sum lam_m'(f_m - x_m) in (x_i, u_i), i.e. the Gauss-Newton block of linearise plus
 * the curvature of the active keep-out rows (s_c grad^2 g_c with s_c = y_c + rho g_c > 0) and the
 * dynamics' second derivatives weighted by the children's multipliers (sum_m lam_m' grad^2 f_m),
 * followed by the eigenvalue modification that makes it positive definite. */
static void exact_hessian(const orc_problem *P, work_t *W, const double *x, const double *u, const double *lam,
                          const double *y, double rho) {
    const int n = P->n, nx = P->nx, nu = P->nu, nc = W->nc;
    const tree_t *T = &W->T;
    for (int i = 0; i < n; ++i) {
        const int leaf = T->n_child[i] == 0, nz = leaf ? nx : nx + nu;
        double S[MAXN * MAXN];
        const double *Qi = W->Q + (size_t)i * nx * nx, *Mi = W->M + (size_t)i * nu * nx, *Ri = W->R + (size_t)i * nu * nu;
        for (int a = 0; a < nx; ++a)
            for (int b = 0; b < nx; ++b) S[a * nz + b] = Qi[a * nx + b];
        if (!leaf)
            for (int a = 0; a < nu; ++a) {
                for (int b = 0; b < nx; ++b) S[(nx + a) * nz + b] = S[b * nz + nx + a] = Mi[a * nx + b];
                for (int b = 0; b < nu; ++b) S[(nx + a) * nz + nx + b] = Ri[a * nu + b];
            }
        /* keep-out curvature (box and lane rows are linear) */
        const int row0 = 2 * nu * P->box_on;
        for (int o = 0; o < P->n_obs && i != 0; ++o) {
            const int c = row0 + o;
            const double sc = y[(size_t)i * nc + c] + rho * W->g[(size_t)i * nc + c];
            if (!(W->ex[(size_t)i * nc + c] && sc > 0.0)) continue;
            double hxy[3];
            obs_hessian(P->obs + ((size_t)i * P->n_obs + o) * 5, x[(size_t)i * nx], x[(size_t)i * nx + 1], hxy);
            S[0] += sc * hxy[0];
            S[1] += sc * hxy[1];
            S[nz] += sc * hxy[1];
            S[nz + 1] += sc * hxy[2];
        }
        /* the dynamics' curvature, weighted by the children's multipliers */
        if (!leaf) {
            double mu[MAXX] = {0}, H[MAXN * MAXN];
            for (int t = 0; t < T->n_child[i]; ++t) {
                const int m = T->child[T->first_child[i] + t];
                for (int e = 0; e < nx; ++e) mu[e] += lam[(size_t)m * nx + e];
            }
            dyn_hessian(P, x + (size_t)i * nx, u + (size_t)i * nu, mu, H);
            for (int e = 0; e < nz * nz; ++e) S[e] += H[e];
        }
        eig_modify(nz, S);
        double *Qw = W->Q + (size_t)i * nx * nx, *Mw = W->M + (size_t)i * nu * nx, *Rw = W->R + (size_t)i * nu * nu;
        for (int a = 0; a < nx; ++a)
            for (int b = 0; b < nx; ++b) Qw[a * nx + b] = S[a * nz + b];
        if (!leaf)
            for (int a = 0; a < nu; ++a) {
                for (int b = 0; b < nx; ++b) Mw[a * nx + b] = S[(nx + a) * nz + b];
                for (int b = 0; b < nu; ++b) Rw[a * nu + b] = S[(nx + a) * nz + nx + b];
            }
    }
}

/* KKT residual of the relaxed problem Eq. (relax_bmpc) at the linearisation point:
 * max(|grad_{x,u} Lagrangian|_inf, |d|_inf); the root state row is left out (x_0 fixed). */
static double kkt_relaxed(const orc_problem *P, const work_t *W, const double *lam) {
    int n = P->n, nx = P->nx, nu = P->nu;
    const tree_t *T = &W->T;
    double r = 0.0;
    for (int i = 0; i < n; ++i) {
        double Al[MAXX] = {0}, Bl[MAXU] = {0};   /* sum over children of A_m' lam_m, B_m' lam_m */
        for (int t = 0; t < T->n_child[i]; ++t) {
            int m = T->child[T->first_child[i] + t];
            double a1[MAXX], b1[MAXU];
            matTvec(nx, nx, W->A + (size_t)m * nx * nx, lam + (size_t)m * nx, a1);
            matTvec(nx, nu, W->B + (size_t)m * nx * nu, lam + (size_t)m * nx, b1);
            for (int e = 0; e < nx; ++e) Al[e] += a1[e];
            for (int e = 0; e < nu; ++e) Bl[e] += b1[e];
        }
        if (i != 0) {
            for (int e = 0; e < nx; ++e) {
                double gx = W->q[(size_t)i * nx + e] + Al[e] - lam[(size_t)i * nx + e];
                if (fabs(gx) > r) r = fabs(gx);
            }
            for (int e = 0; e < nx; ++e) if (fabs(W->d[(size_t)i * nx + e]) > r) r = fabs(W->d[(size_t)i * nx + e]);
        }
        if (T->n_child[i]) {
            for (int e = 0; e < nu; ++e) {
                double gu = W->r[(size_t)i * nu + e] + Bl[e];
                if (fabs(gu) > r) r = fabs(gu);
            }
        }
    }
    return r;
}

/* L_a + lambda'd + mu/2 |d|^2 at (x, u, lam): the merit of Eq. (merit) with J = L_a. */
static double merit_at(const orc_problem *P, const tree_t *T, int nc, const double *x, const double *u,
                       const double *lam, const double *y, double rho, double mu) {
    int n = P->n, nx = P->nx, nu = P->nu;
    double La = 0.0, ld = 0.0, dd = 0.0;
    for (int i = 0; i < n; ++i) {
        int leaf = T->n_child[i] == 0;
        const double *xi = x + (size_t)i * nx, *ui = u + (size_t)i * nu;
        La += node_cost(P, i, leaf, xi, ui, NULL, NULL);
        if (nc) {
            double g[64], Jx[64 * MAXX], Ju[64 * MAXU];
            int ex[64];
            orc_constraints(P, i, leaf, xi, ui, g, Jx, Ju, ex);
            for (int c = 0; c < nc; ++c) {
                if (!ex[c]) continue;
                double pen = g[c] + y[(size_t)i * nc + c] / rho;
                if (pen > 0.0) La += 0.5 * rho * pen * pen;
            }
        }
        if (!leaf) {
            for (int t = 0; t < T->n_child[i]; ++t) {
                int m = T->child[T->first_child[i] + t];
                double fx[MAXX];
                edge_dynamics(P, m, xi, ui, fx, NULL, NULL);
                for (int e = 0; e < nx; ++e) {
                    double dm = fx[e] - x[(size_t)m * nx + e];
                    ld += lam[(size_t)m * nx + e] * dm;
                    dd += dm * dm;
                }
            }
        }
    }
    return La + ld + 0.5 * mu * dd;
}

static int check_problem(const orc_problem *P) {
    if (!P || P->n < 1 || P->nx < 1 || P->nx > MAXX || P->nu < 1 || P->nu > MAXU) return 0;
    if (P->model < 0 || P->model > 3) return 0;
    if ((P->model == 0 || P->model == 3) && (P->nx != 4 || P->nu != 2)) return 0;
    if (P->model == 1 && (P->nx != 6 || P->nu != 2)) return 0;
    if (P->model != 2 && (P->nx < 2)) return 0;
    if (n_con(P) > 64) return 0;
    if ((P->Aedge != NULL) != (P->Bedge != NULL) || (P->Aedge && P->model != 2)) return 0;
    return 1;
}

/* Cold start of Sec. V-B: states linearly interpolated between x0 and the final reference
 * state of the node's first leaf descendant, u = 0, lambda = 0, y = 0. */
void orc_cold_start(const orc_problem *P, double *x, double *u, double *lam, double *y) {
    tree_t T;
    int n = P->n, nx = P->nx, nu = P->nu, nc = n_con(P);
    tree_build(P, &T);
    for (int i = 0; i < n; ++i) {
        int leaf = i;
        while (T.n_child[leaf]) leaf = T.child[T.first_child[leaf]];
        double s = T.stage[leaf] > 0 ? (double)T.stage[i] / T.stage[leaf] : 0.0;
        for (int j = 0; j < nx; ++j)
            x[(size_t)i * nx + j] = P->x0[j] + s * (P->xref[(size_t)leaf * nx + j] - P->x0[j]);
    }
    memset(u, 0, sizeof(double) * n * nu);
    memset(lam, 0, sizeof(double) * n * nx);
    if (nc) memset(y, 0, sizeof(double) * n * nc);
    tree_free(&T);
}

void orc_default_opts(orc_opts *o) {
    o->max_iters = 50;
    o->max_outer = 60;
    o->n_alpha = 10;
    o->eps_tol = 1e-5;
    o->tau = 100.0;
    o->omega0 = 1.0;
    o->eta0 = 0.1;
    o->a_omega = 1.0;
    o->b_omega = 1.0;
    o->a_eta = 0.1;
    o->b_eta = 0.9;
    o->rho0 = 10.0;
    o->rho_max = 1e6;
    o->mu0 = 1.0;
    o->beta = 1e-4;
    o->ls_rel_eps = 1e-6;
    o->lqr_scan = 0;
    o->hessian = 0;
    o->cap_rule = 0;
    o->trace = NULL;
    o->trace_user = NULL;
}

/* Directional data of one inner iteration at (x, u, lam) for fixed (y, rho, mu), with W
 * already linearised at (x, u): solves the tree LQR, and returns dx, du, dlam = lam_QP - lam,
 * phi(0), phi'(0) of the merit along (dx, du, dlam), dz'W dz and |d|^2. */
static int direction(const orc_problem *P, work_t *W, const double *x, const double *u, const double *lam,
                     const double *y, double rho, double mu, int scan, double *dlam, double out[6]) {
    int n = P->n, nx = P->nx, nu = P->nu;
    int st = scan ? tree_lqr_scan(&W->T, P->parent, nx, nu, W->Q, W->M, W->R, W->q, W->r, W->A, W->B, W->d, W->K,
                                  W->k, W->P, W->p, W->dx, W->du, W->lqp)
                  : tree_lqr(&W->T, nx, nu, W->Q, W->M, W->R, W->q, W->r, W->A, W->B, W->d, W->K, W->k, W->P, W->p,
                             W->dx, W->du, W->lqp);
    if (st) return st;
    double gd = 0.0, wq = 0.0, ld = 0.0, dd = 0.0;
    for (int i = 0; i < n; ++i) {
        const double *dxi = W->dx + (size_t)i * nx, *dui = W->du + (size_t)i * nu;
        double Qd[MAXX], Md[MAXU], Rd[MAXU];
        matvec(nx, nx, W->Q + (size_t)i * nx * nx, dxi, Qd);
        matvec(nu, nx, W->M + (size_t)i * nu * nx, dxi, Md);
        matvec(nu, nu, W->R + (size_t)i * nu * nu, dui, Rd);
        for (int e = 0; e < nx; ++e) { gd += W->q[(size_t)i * nx + e] * dxi[e]; wq += dxi[e] * Qd[e]; }
        for (int e = 0; e < nu; ++e) { gd += W->r[(size_t)i * nu + e] * dui[e]; wq += dui[e] * (2.0 * Md[e] + Rd[e]); }
        for (int e = 0; e < nx; ++e) {
            double dl = (i == 0) ? 0.0 : W->lqp[(size_t)i * nx + e] - lam[(size_t)i * nx + e];
            dlam[(size_t)i * nx + e] = dl;
            if (i) {
                double de = W->d[(size_t)i * nx + e];
                ld += (dl - lam[(size_t)i * nx + e]) * de;
                dd += de * de;
            }
        }
    }
    double phi0 = merit_at(P, &W->T, W->nc, x, u, lam, y, rho, mu);
    out[0] = phi0;
    out[1] = gd + ld - mu * dd;    /* phi'(0; mu) */
    out[2] = wq;
    out[3] = dd;
    out[4] = gd + ld;              /* phi'(0; 0) */
    out[5] = W->La;
    return ORC_OK;
}

/* ------------------------------------------------------------ the AL method (Algorithm 1) */
int orc_solve(const orc_problem *P, const orc_opts *O_in, const double *wx, const double *wu, const double *wlam,
              const double *wy, double *x, double *u, double *lam, double *y, orc_stats *S) {
    if (!check_problem(P)) return ORC_ERR_INVALID;
    orc_opts O;
    if (O_in) O = *O_in; else orc_default_opts(&O);
    int n = P->n, nx = P->nx, nu = P->nu;
    work_t W;
    if (!tree_build(P, &W.T)) { tree_free(&W.T); return ORC_ERR_INVALID; }
    work_alloc(&W, P);
    int nc = W.nc;
    if (wx) {
        memcpy(x, wx, sizeof(double) * n * nx);
        memcpy(u, wu, sizeof(double) * n * nu);
        memcpy(lam, wlam, sizeof(double) * n * nx);
        if (nc) memcpy(y, wy, sizeof(double) * n * nc);
    } else {
        orc_cold_start(P, x, u, lam, y);
    }
    memcpy(x, P->x0, sizeof(double) * nx);                        /* x_0 = x-bar */
    for (int i = 0; i < n; ++i)
        if (W.T.n_child[i] == 0) memset(u + (size_t)i * nu, 0, sizeof(double) * nu);
    memset(lam, 0, sizeof(double) * nx);

    double rho = O.rho0, mu = O.mu0, omega = O.omega0, eta = O.eta0;
    double r_kkt = INFINITY, cviol = INFINITY;
    int inner = 0, outer = 0, ls_fail = 0, ls_fail_total = 0, status = ORC_MAX_ITER;
    double *dlam = (double *)calloc((size_t)n * nx, sizeof(double));
    double *xt = (double *)calloc((size_t)n * nx, sizeof(double));
    double *ut = (double *)calloc((size_t)n * nu, sizeof(double));
    double *lt = (double *)calloc((size_t)n * nx, sizeof(double));
    double *ybefore = (double *)calloc((size_t)n * (nc ? nc : 1), sizeof(double));

    while (outer < O.max_outer) {
        ++outer;
        /* inner loop: iLQR steps on the relaxed problem until r_kkt <= omega */
        for (;;) {
            linearise(P, &W, x, u, y, rho);
            if (O.hessian) exact_hessian(P, &W, x, u, lam, y, rho);
            r_kkt = kkt_relaxed(P, &W, lam);
            if (r_kkt <= omega) break;
            if (inner >= O.max_iters) goto done;
            double info[6];
            int st = direction(P, &W, x, u, lam, y, rho, mu, O.lqr_scan, dlam, info);
            if (st) { status = st; goto done; }
            double wq = info[2], dd = info[3], dphi0 = info[4];
            const double mu_prev = mu;
            /* adaptive merit penalty (Gill et al. 1992 reading) */
            if (dd > 0.0 && dphi0 - mu * dd > -0.5 * wq) {
                double need = 2.0 * (dphi0 + 0.5 * wq) / dd;
                if (need > mu) mu = need;
            }
            double phi0 = merit_at(P, &W.T, nc, x, u, lam, y, rho, mu);
            double dphi = dphi0 - mu * dd;
            /* all step sizes alpha_i = 2^-i, take the largest satisfying Eq. (sufficient_decrease) */
            double alpha = ldexp(1.0, -(O.n_alpha - 1)), phi_alpha = NAN;
            int accepted = 0;
            for (int a = 0; a < O.n_alpha; ++a) {
                double al = ldexp(1.0, -a);
                for (int e = 0; e < n * nx; ++e) { xt[e] = x[e] + al * W.dx[e]; lt[e] = lam[e] + al * dlam[e]; }
                for (int e = 0; e < n * nu; ++e) ut[e] = u[e] + al * W.du[e];
                double phi = merit_at(P, &W.T, nc, xt, ut, lt, y, rho, mu);
                phi_alpha = phi;
                if (phi <= phi0 + O.beta * al * dphi + O.ls_rel_eps * fabs(phi0)) { alpha = al; accepted = 1; break; }
            }
            if (accepted) ls_fail = 0; else { ++ls_fail; ++ls_fail_total; }
            if (O.trace) {
                const double tinfo[16] = {(double)inner, (double)outer, rho, mu_prev, mu, phi0, dphi, dphi0, wq, dd,
                                          alpha, (double)accepted, phi_alpha,
                                          (double)(accepted && phi_alpha > phi0 + O.beta * alpha * dphi),
                                          r_kkt, omega};
                O.trace(O.trace_user, 0, tinfo, x, u, lam, y, W.dx, W.du, dlam);
            }
            for (int e = 0; e < n * nx; ++e) { x[e] += alpha * W.dx[e]; lam[e] += alpha * dlam[e]; }
            for (int e = 0; e < n * nu; ++e) u[e] += alpha * W.du[e];
            ++inner;
            if (ls_fail >= 3) { status = ORC_LS_FAIL; goto done; }
        }
        /* outer loop: BCL update of (y, rho) and the tolerance schedules */
        cviol = 0.0;
        for (int e = 0; e < n * nc; ++e) {
            if (!W.ex[e]) continue;
            double v = W.g[e] > -y[e] / rho ? W.g[e] : -y[e] / rho;
            if (fabs(v) > cviol) cviol = fabs(v);
        }
        const double eta_before = eta, rho_before = rho;
        int branch, converged = 0;
        if (nc) memcpy(ybefore, y, sizeof(double) * n * nc);
        if (cviol <= eta) {
            /* success: multiplier update, rho kept */
            branch = 0;
            for (int e = 0; e < n * nc; ++e) {
                if (!W.ex[e]) continue;
                double v = y[e] + rho * W.g[e];
                y[e] = v > 0.0 ? v : 0.0;
            }
            if ((r_kkt > cviol ? r_kkt : cviol) < O.eps_tol) {
                converged = 1;
            } else {
                omega = omega * pow(rho, -O.b_omega);
                eta = eta * pow(rho, -O.b_eta);
            }
        } else {
            if (O.cap_rule == 1 && rho >= O.rho_max) {
                /* product rule at the cap: first-order multiplier step instead of a larger rho */
                branch = 2;
                for (int e = 0; e < n * nc; ++e) {
                    if (!W.ex[e]) continue;
                    double v = y[e] + rho * W.g[e];
                    y[e] = v > 0.0 ? v : 0.0;
                }
            } else {
                /* Algorithm 1: y kept, rho <- tau rho (held at rho_max) */
                branch = rho >= O.rho_max ? 3 : 1;
                rho = O.tau * rho;
                if (rho > O.rho_max) rho = O.rho_max;
            }
            omega = O.omega0 * pow(rho, -O.a_omega);
            eta = O.eta0 * pow(rho, -O.a_eta);
        }
        if (!converged) {
            if (omega < O.eps_tol) omega = O.eps_tol;
            if (eta < O.eps_tol) eta = O.eps_tol;
        }
        if (O.trace) {
            const double tinfo[10] = {(double)outer, (double)branch, cviol, eta_before, rho_before, rho, omega, eta,
                                      r_kkt, (double)converged};
            O.trace(O.trace_user, 1, tinfo, x, u, lam, ybefore, y, NULL, NULL);
        }
        if (converged) { status = ORC_OK; goto done; }
    }
done:
    if (S) {
        S->status = status;
        S->inner_iters = inner;
        S->outer_iters = outer;
        S->ls_fail_total = ls_fail_total;
        S->r_kkt = r_kkt;
        S->c = cviol;
        S->rho = rho;
        S->mu = mu;
        S->omega = omega;
        S->eta = eta;
    }
    free(dlam); free(xt); free(ut); free(lt); free(ybefore);
    work_free(&W);
    return status;
}

/* ------------------------------------------------------------ evaluation entry points for tests */

/* KKT conditions of the original problem Eq. (bmpc) at (x, u, lam, y):
 * out[0] = |grad_{x,u} (sum l + y'g + lam'd)|_inf (root state row left out),
 * out[1] = |d|_inf, out[2] = |max(g, 0)|_inf, out[3] = |min(-g, y)|_inf, out[4] = |min(y, 0)|_inf. */
int orc_kkt(const orc_problem *P, const double *x, const double *u, const double *lam, const double *y,
            double *out) {
    if (!check_problem(P)) return ORC_ERR_INVALID;
    work_t W;
    if (!tree_build(P, &W.T)) { tree_free(&W.T); return ORC_ERR_INVALID; }
    work_alloc(&W, P);
    int n = P->n, nx = P->nx, nu = P->nu, nc = W.nc;
    /* y enters the stationarity directly: linearise with rho -> 0 penalty replaced by y'g */
    double *zero = (double *)calloc((size_t)n * (nc ? nc : 1), sizeof(double));
    linearise(P, &W, x, u, zero, 1.0);
    /* remove the PHR contribution (y = 0, rho = 1 activates g > 0 rows) and add y'g instead */
    for (int i = 0; i < n; ++i) {
        int leaf = W.T.n_child[i] == 0;
        double lx[MAXX] = {0}, lu[MAXU] = {0};
        node_cost(P, i, leaf, x + (size_t)i * nx, u + (size_t)i * nu, lx, lu);
        for (int e = 0; e < nx; ++e) W.q[(size_t)i * nx + e] = lx[e];
        for (int e = 0; e < nu; ++e) W.r[(size_t)i * nu + e] = leaf ? 0.0 : lu[e];
        if (nc) {
            double g[64], Jx[64 * MAXX], Ju[64 * MAXU];
            int ex[64];
            orc_constraints(P, i, leaf, x + (size_t)i * nx, u + (size_t)i * nu, g, Jx, Ju, ex);
            for (int c = 0; c < nc; ++c) {
                if (!ex[c]) continue;
                double yc = y[(size_t)i * nc + c];
                for (int a = 0; a < nx; ++a) W.q[(size_t)i * nx + a] += yc * Jx[c * nx + a];
                for (int a = 0; a < nu; ++a) W.r[(size_t)i * nu + a] += yc * Ju[c * nu + a];
            }
        }
    }
    double stat = 0.0, dmax = 0.0, inf = 0.0, comp = 0.0, neg = 0.0;
    for (int i = 0; i < n; ++i) {
        double Al[MAXX] = {0}, Bl[MAXU] = {0};   /* sum over children of A_m' lam_m, B_m' lam_m */
        for (int t = 0; t < W.T.n_child[i]; ++t) {
            int m = W.T.child[W.T.first_child[i] + t];
            double a1[MAXX], b1[MAXU];
            matTvec(nx, nx, W.A + (size_t)m * nx * nx, lam + (size_t)m * nx, a1);
            matTvec(nx, nu, W.B + (size_t)m * nx * nu, lam + (size_t)m * nx, b1);
            for (int e = 0; e < nx; ++e) Al[e] += a1[e];
            for (int e = 0; e < nu; ++e) Bl[e] += b1[e];
        }
        if (i) {
            for (int e = 0; e < nx; ++e) {
                double gx = W.q[(size_t)i * nx + e] + Al[e] - lam[(size_t)i * nx + e];
                if (fabs(gx) > stat) stat = fabs(gx);
                if (fabs(W.d[(size_t)i * nx + e]) > dmax) dmax = fabs(W.d[(size_t)i * nx + e]);
            }
        }
        if (W.T.n_child[i]) {
            for (int e = 0; e < nu; ++e) {
                double gu = W.r[(size_t)i * nu + e] + Bl[e];
                if (fabs(gu) > stat) stat = fabs(gu);
            }
        }
        for (int c = 0; c < nc; ++c) {
            if (!W.ex[(size_t)i * nc + c]) continue;
            double g = W.g[(size_t)i * nc + c], yc = y[(size_t)i * nc + c];
            if (g > inf) inf = g;
            double cm = fabs(-g < yc ? -g : yc);
            if (cm > comp) comp = cm;
            if (-yc > neg) neg = -yc;
        }
    }
    out[0] = stat; out[1] = dmax; out[2] = inf; out[3] = comp; out[4] = neg;
    free(zero);
    work_free(&W);
    return ORC_OK;
}

/* Merit phi = L_a + lam'd + mu/2 |d|^2 at a given point (Eq. merit with J = L_a). */
double orc_merit(const orc_problem *P, const double *x, const double *u, const double *lam, const double *y,
                 double rho, double mu) {
    tree_t T;
    if (!check_problem(P) || !tree_build(P, &T)) return NAN;
    double v = merit_at(P, &T, n_con(P), x, u, lam, y, rho, mu);
    tree_free(&T);
    return v;
}

/* One search direction at a given point (for tests): dx, du, dlam and
 * info = [phi(0), phi'(0; mu), dz'W dz, |d|^2, phi'(0; 0), L_a]. */
int orc_direction(const orc_problem *P, const double *x, const double *u, const double *lam, const double *y,
                  double rho, double mu, double *dx, double *du, double *dlam, double *info) {
    if (!check_problem(P)) return ORC_ERR_INVALID;
    work_t W;
    if (!tree_build(P, &W.T)) { tree_free(&W.T); return ORC_ERR_INVALID; }
    work_alloc(&W, P);
    linearise(P, &W, x, u, y, rho);
    int st = direction(P, &W, x, u, lam, y, rho, mu, 0, dlam, info);
    memcpy(dx, W.dx, sizeof(double) * P->n * P->nx);
    memcpy(du, W.du, sizeof(double) * P->n * P->nu);
    work_free(&W);
    return st;
}

/* KKT residual of the relaxed problem (Sec. IV-A) at (x, u, lam) for (y, rho). */
double orc_kkt_relaxed(const orc_problem *P, const double *x, const double *u, const double *lam,
                       const double *y, double rho) {
    if (!check_problem(P)) return NAN;
    work_t W;
    if (!tree_build(P, &W.T)) { tree_free(&W.T); return NAN; }
    work_alloc(&W, P);
    linearise(P, &W, x, u, y, rho);
    double r = kkt_relaxed(P, &W, lam);
    work_free(&W);
    return r;
}

/* L_a (Eq. AL) at (x, u) for (y, rho). */
double orc_aug_lagrangian(const orc_problem *P, const double *x, const double *u, const double *y, double rho) {
    if (!check_problem(P)) return NAN;
    work_t W;
    if (!tree_build(P, &W.T)) { tree_free(&W.T); return NAN; }
    work_alloc(&W, P);
    linearise(P, &W, x, u, y, rho);
    double v = W.La;
    work_free(&W);
    return v;
}

/* Test entry points of the exact-Hessian option: the dynamics' second derivatives weighted by mu
 * (H [nz][nz]), the keep-out curvature ([gxx, gxy, gyy] at X, Y of obstacle ob[5]), the Jacobi
 * eigen-decomposition and the eigenvalue modification of a symmetric n x n matrix (in place). */
int orc_dyn_hessian(const orc_problem *P, const double *x, const double *u, const double *mu, double *H) {
    if (!check_problem(P)) return ORC_ERR_INVALID;
    dyn_hessian(P, x, u, mu, H);
    return ORC_OK;
}
void orc_obs_hessian(const double *ob, double X, double Y, double *out) { obs_hessian(ob, X, Y, out); }
int orc_jacobi_eig(int n, const double *S, double *ev, double *Vm) {
    if (n < 1 || n > MAXN) return ORC_ERR_INVALID;
    jacobi_eig(n, S, ev, Vm);
    return ORC_OK;
}
int orc_eig_modify(int n, double *S) {
    if (n < 1 || n > MAXN) return ORC_ERR_INVALID;
    eig_modify(n, S);
    return ORC_OK;
}
