/* Tree LQR at general sizes with per-edge dynamics (B300, sm_103a).
 *
 * The linear-quadratic subproblem of the method, Eq. (lqr_tree_approx), solved by the tree Riccati
 * recursion of Eq. (tree_Riccati) with the feedback laws of Eq. (tree_feedback_laws) and the forward
 * sweep of Sec. III-A, for state and input dimensions beyond the solver's vehicle models: up to
 * n_x = 32 and n_u = 16, which covers the mass-spring chains of Sec. V-A (M masses: n_x = 2M,
 * n_u = M - 1; the paper uses n_x = 10 and 30).  Every edge carries its own dynamics (A_m, B_m, c_m),
 * as in Sec. V-A's trees, whose branches differ in the spring constant.  A batch of problems that
 * share one tree is solved in one sequence of launches (the batch LQR of Sec. V-A is a batch of
 * single-path trees).
 *
 * Problem t of the batch (0 <= t < batch), nodes i < n in level order (parent[0] = -1,
 * parent[i] < i, and stage(i) = stage(parent[i]) + 1 is nondecreasing in i):
 *
 *   minimise   sum_i [ 1/2 x_i' Q_i x_i + q_i' x_i ]
 *            + sum_{i not a leaf} [ u_i' M_i x_i + 1/2 u_i' R_i u_i + r_i' u_i ]
 *   subject to x_0 = x0,  x_m = A_m x_{p(m)} + B_m u_{p(m)} + c_m  for every node m > 0,
 *
 * where A_m, B_m, c_m belong to the edge into m.  Leaves have no input.  Returned: the laws
 * u_i = K_i x_i + k_i, the value functions V_i(x) = 1/2 x' P_i x + p_i' x + const (P_i symmetrised),
 * the solution x, u (leaf rows of u, K and k are 0) and the costates lam_i = P_i x_i + p_i.
 *
 * Layout: device arrays of float32, problem-major, then node-major, matrices row-major:
 *   Q, P [batch][n][nx][nx];  M, K [batch][n][nu][nx];  R [batch][n][nu][nu];
 *   q, p, c, x, lam [batch][n][nx];  r, k, u [batch][n][nu];
 *   A [batch][n][nx][nx];  B [batch][n][nx][nu];  x0 [batch][nx].
 * Row 0 of A, B and c is not read; M may be NULL (zero cross terms); Q, R are read as given (the
 * recursion uses the full matrices).  The caller owns every array; the handle owns only the tree
 * tables it copies at creation.
 *
 * The recursion needs every H_i = R_i + sum_m B_m' P_m B_m positive definite: a Cholesky pivot that
 * is not positive (or not finite) is recorded, the solve completes with undefined outputs and
 * bmpc_lqr_status returns BMPC_ERR_NUMERIC.
 */
#ifndef BMPC_LQR_H
#define BMPC_LQR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bmpc_lqr bmpc_lqr;

/* Validates the tree (n >= 1, parent[0] = -1, 0 <= parent[i] < i, stages nondecreasing in i) and
 * the sizes (1 <= nx <= 32, 1 <= nu <= 16, batch >= 1), copies the tree into per-node tables on the
 * device (child range, first child, parent) and binds the handle to `stream` (a cudaStream_t, NULL = the
 * default stream).  0 on success; BMPC_ERR_INVALID (-1) on a bad tree or size, BMPC_ERR_CUDA (-2)
 * if a device allocation or copy fails. */
int bmpc_lqr_create(int32_t n, const int32_t *parent, int32_t nx, int32_t nu, int32_t batch, void *stream,
                    bmpc_lqr **out);

/* One tree LQR solve of the whole batch, asynchronous on the handle's stream: the backward sweep,
 * leaves to root (one block per node step, each thread owning four entries of a row of the node's
 * matrix products), and the forward sweep, root to leaves (lane j of a warp on row j), on the
 * schedule of bmpc_lqr_set_schedule.  All pointers are device
 * pointers in the layout above; inputs are only read, the outputs K, k, P, p, x, u, lam written in
 * full.  0 on success, BMPC_ERR_INVALID on a NULL required pointer, BMPC_ERR_CUDA on a launch error.
 * The call is capturable into a CUDA graph. */
int bmpc_lqr_solve(bmpc_lqr *h, const float *Q, const float *M, const float *R, const float *q, const float *r,
                   const float *A, const float *B, const float *c, const float *x0, float *K, float *k, float *P,
                   float *p, float *x, float *u, float *lam);

/* Synchronises the handle's stream and returns BMPC_OK, or BMPC_ERR_NUMERIC if a solve since the
 * last call met a non-positive pivot (the record is cleared), or BMPC_ERR_CUDA. */
int bmpc_lqr_status(bmpc_lqr *h);

/* The stage count S of the tree (a solve makes 2 S launches on the per-stage schedule, 1 fused). */
int bmpc_lqr_stages(const bmpc_lqr *h);

/* The launch schedule of later solves: 0 (default) chooses by a cost model of the tree's stage
 * widths and the batch size; 1: one launch per stage and sweep, every node of a stage at once (wide
 * trees); 2: one block per problem walking its nodes in post-order backward and its stages forward,
 * one launch per solve (narrow trees, batches of single paths).  Both compute the same arithmetic in
 * the same order, so the results are bitwise equal.  BMPC_ERR_INVALID on a NULL handle or another value.  bmpc_lqr_fused returns 1
 * when solves run fused, 0 when per stage. */
int bmpc_lqr_set_schedule(bmpc_lqr *h, int32_t schedule);
int bmpc_lqr_fused(const bmpc_lqr *h);

void bmpc_lqr_destroy(bmpc_lqr *h);

#ifdef __cplusplus
}
#endif
#endif /* BMPC_LQR_H */
