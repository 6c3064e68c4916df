/*
 * Persistent FP32 solver kernel for branch MPC: the multiple-shooting
 * augmented-Lagrangian iLQR method of arXiv 2506.13624 (Algorithm 1) over a
 * scenario tree.  One thread block owns one problem at a time and takes the
 * next problem from a device work queue when it finishes, so a single launch
 * solves a whole batch of trees of uneven size.
 *
 * Per inner iteration the block runs, with a block barrier between phases:
 *   linearise   every node in parallel: RK4 increment with forward-mode Jacobians
 *               A_n, B_n, cost gradient, PHR penalty gradient and its
 *               Gauss-Newton Hessian (Sec. IV-A, Eq. AL);
 *   kkt         defects d_m = f_p(m) - x_m, KKT residual of the relaxed problem
 *               (Sec. IV-A stopping criterion) by a block max-reduction;
 *   backward    the tree Riccati recursion, level by level from the leaves:
 *               child value functions summed at branch points, then the
 *               feedback law of Eq. (tree_feedback_laws) (Sec. III-A);
 *   forward     the linear rollout, level by level from the root, and the
 *               QP multipliers lam_m = P_m dx_m + p_m;
 *   merit       phi(0), phi'(0) and the merit penalty mu (Eq. merit);
 *   line search all step sizes alpha_i = 2^-i of a chunk evaluated in
 *               parallel over (node, alpha), the largest one satisfying
 *               Eq. (sufficient_decrease) is taken (Algorithm 1);
 *   update      x, u, lam moved by alpha.
 * After the inner loop the block evaluates the constraint violation c and
 * applies the BCL update of (y_e, rho, omega, eta) (Sec. IV-B).
 *
 * State coordinates: the kernel iterates on the deviation xi = x - xref of every node
 * state from its reference, so that FP32 resolves states far from the origin; defects
 * are formed from reference increments, state deviations and RK4 increments without
 * subtracting two large absolute positions.  Absolute states are formed only on output.
 *
 * Scalar control (rho, mu, omega, eta, counters) is replicated in every
 * thread: block reductions return identical totals to all threads, so all
 * threads take the same branches.  Reductions use a fixed order and are
 * bitwise reproducible for a fixed block size.
 */
#include <algorithm>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bmpc_layout.h"

namespace bmpc {

/* Two instances of the solver per model: blocks of up to 256 threads, two per SM, for batches;
 * blocks of up to 512 threads, one per SM, for few large problems (single solves).  Both get at
 * most 128 registers per thread.  The shared reduction arrays are sized for the larger. */
constexpr int MAX_BLOCK = 512;
constexpr int BATCH_BLOCK = 256;
constexpr int MAX_WARPS = MAX_BLOCK / 32;
constexpr int MAX_CHUNK = 16;   /* at most 16 step sizes per line-search round */
/* The node loops load before they store (one or two batches of loads per node instead of one L2
 * round trip per stored component).  The linearisation does so only where the registers allow it:
 * the dynamic model's kernel is at its register limit, and hoisting there lengthens the live ranges
 * across the RK4 tangents into spills that cost more than the hoisting saves (measured), so it keeps
 * the load-compute-store order per row. */
template <int NX>
constexpr bool hoist_loads() { return NX <= 4; }

constexpr int GL = 8;   /* lanes per path in the cooperative sweeps (one per column of [A B], nx + nu <= 8) */

struct Shared {
    float red[MAX_WARPS][MAX_CHUNK + 1];
    float tr[MAX_BLOCK / GL][6][8];   /* per lane group: rows of P F, read back as columns */
    int flag;
};

/* ------------------------------------------------------------------ block reductions */
template <int K>
__device__ __forceinline__ void block_sum(float (&v)[K], Shared &sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sh.red[warp][k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float s = 0.f;
        for (int w = 0; w < nw; ++w) s += sh.red[w][k];
        v[k] = s;
    }
}

/* max of non-negative values; NaN is mapped to +inf so that it cannot vanish */
__device__ __forceinline__ float block_max(float v, Shared &sh) {
    if (!(v == v)) v = INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh.red[warp][0] = v;
    __syncthreads();
    float m = 0.f;
    for (int w = 0; w < nw; ++w) m = fmaxf(m, sh.red[w][0]);
    return m;
}

/* ------------------------------------------------------------------ packed symmetric index */
template <int NX>
__host__ __device__ constexpr int sidx(int a, int b) {
    return a <= b ? a * NX - a * (a - 1) / 2 + (b - a) : b * NX - b * (b - 1) / 2 + (a - b);
}

/* ------------------------------------------------------------------ dynamics */
/* sin and cos of an angle, accurate to about 1.5 ulp for |a| < 1e3 rad: Cody and Waite's reduction
 * a = q pi/2 + r with pi/2 split into three floats (P1 the float nearest pi/2, P2 and P3 the next
 * parts of the remainder), then the Taylor polynomials of sin r to r^9 and cos r to r^8 on
 * |r| <= pi/4 (truncation below 2e-9) in Horner form, and the quadrant's swap and signs.  Only
 * FMA-pipe arithmetic and no slow path: the dynamics evaluate it at every RK4 stage, and its
 * values and the analytic Jacobians built from them stay consistent to rounding, which the KKT
 * tolerance of 1e-5 in FP32 needs. */
__device__ __forceinline__ void sincos_cw(float a, float *s, float *c) {
    constexpr float TWO_OVER_PI = 0.636619772f;
    constexpr float P1 = 1.57079637f, P2 = -4.37113883e-8f, P3 = -1.71512451e-15f;
    const float qf = rintf(a * TWO_OVER_PI);
    const int q = (int)qf;
    const float r = fmaf(-qf, P3, fmaf(-qf, P2, fmaf(-qf, P1, a)));
    const float r2 = r * r;
    float ps = fmaf(r2, 1.f / 362880.f, -1.f / 5040.f);
    ps = fmaf(ps, r2, 1.f / 120.f);
    ps = fmaf(ps, r2, -1.f / 6.f);
    const float sr = fmaf(ps * r2, r, r);
    float pc = fmaf(r2, 1.f / 40320.f, -1.f / 720.f);
    pc = fmaf(pc, r2, 1.f / 24.f);
    pc = fmaf(pc, r2, -0.5f);
    const float cr = fmaf(pc, r2, 1.f);
    const float ss = (q & 1) ? cr : sr, cc = (q & 1) ? sr : cr;
    *s = (q & 2) ? -ss : ss;
    *c = ((q + 1) & 2) ? -cc : cc;
}

/* Reciprocal by the PTX approximate instruction (rcp.approx.ftz.f32: at most 1 ulp of error over
 * the normal range).  Unlike the IEEE-rounded reciprocal it has no slow path: a single SFU
 * operation on the Riccati critical path and in every RK4 stage. */
__device__ __forceinline__ float rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

/* 2^-k for 0 <= k <= 126, exactly (the step sizes alpha_i of the line search). */
__device__ __forceinline__ float pow2neg(int k) { return __int_as_float((127 - k) << 23); }

/* ------------------------------------------------------------------ compensated arithmetic */
/* Error-free transformations in round-to-nearest FP32 (Knuth's TwoSum; the FMA form of Dekker's
 * TwoProduct): s = fl(a + b) with a + b = s + e exactly, p = fl(a b) with a b = p + e exactly. */
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
    const float s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}
__device__ __forceinline__ float two_prod(float a, float b, float &e) {
    const float p = a * b;
    e = fmaf(a, b, -p);
    return p;
}

/* Low-order parts of the compensated iterate at one node: the state deviation's positions and the
 * inputs are held as pairs (hi, lo), hi the FP32 value and lo the remainder, so that an accepted
 * step smaller than an ulp of hi is not lost.  Near an active constraint the penalty multiplies
 * the constraint's value by rho; with the iterate rounded to FP32, rho times that rounding puts a
 * floor under the relaxed KKT residual (an input resting on its bound at 2.0 has ulp 2.4e-7, times
 * rho = 100: 2.4e-5).  The pairs remove that floor; everything else reads hi alone. */
struct Lo {
    float x[2], u[NU];
};

/* (hi, lo) += t, renormalised so that |lo| <= ulp(hi) / 2. */
__device__ __forceinline__ void comp_add(float &hi, float &lo, float t) {
    float e, e2;
    const float s = two_sum(hi, t, e);
    hi = two_sum(s, lo + e, e2);
    lo = e2;
}

/* Keep-out value g = 1 - sqrt(q2), q2 = (d_par/a)^2 + (d_perp/b)^2 + 1e-6, at the compensated
 * position (reference xr, yr plus deviation xh + xl, yh + yl) from the obstacle centre (cx, cy),
 * heading cosine ch and sine sh, ia2 = 1/a^2, ib2 = 1/b^2, in two-float arithmetic: near the boundary
 * q2 is close to 1, and in plain FP32 g would carry an absolute error of an ulp of 1 that the
 * penalty multiplies by rho.  Also returns the FP32 d_par, d_perp and 1/sqrt(q2) for the gradient,
 * where relative accuracy suffices. */
__device__ __forceinline__ float obs_g_comp(float xr, float yr, float cx, float cy, float xh, float xl, float yh,
                                            float yl, float ch, float sh, float ia2, float ib2, float &dpar,
                                            float &dper, float &irr) {
    float e1, e2, e3, e4;
    const float dxh = two_sum(two_sum(xr, -cx, e1), xh, e2);
    const float dxl = (e1 + e2) + xl;
    const float dyh = two_sum(two_sum(yr, -cy, e3), yh, e4);
    const float dyl = (e3 + e4) + yl;
    float f1, f2, f3, f4, f5, f6;
    const float p1 = two_prod(ch, dxh, f1), p2 = two_prod(sh, dyh, f2);
    const float parh = two_sum(p1, p2, f3);
    const float parl = ((f1 + f2) + f3) + (ch * dxl + sh * dyl);
    const float p3 = two_prod(-sh, dxh, f4), p4 = two_prod(ch, dyh, f5);
    const float perh = two_sum(p3, p4, f6);
    const float perl = ((f4 + f5) + f6) + (ch * dyl - sh * dxl);
    float g1, g2, g3, g4, g5, g6, g7;
    const float s1 = two_prod(parh, parh, g1);
    const float t1 = two_prod(ia2, s1, g2);
    const float t1l = g2 + ia2 * (g1 + 2.f * parh * parl);
    const float s2 = two_prod(perh, perh, g3);
    const float t2 = two_prod(ib2, s2, g4);
    const float t2l = g4 + ib2 * (g3 + 2.f * perh * perl);
    const float qb = two_sum(two_sum(t1, t2, g5), 1e-6f, g6);
    const float qh = two_sum(qb, ((g5 + g6) + t1l) + t2l, g7);
    /* sqrt(qh + g7) = r + (qh - r^2 + g7) / (2 r); qh - r^2 is exact through the FMA */
    const float r = sqrtf(qh);
    const float ir = rcp(r);
    const float res = fmaf(-r, r, qh) + g7;
    dpar = parh;
    dper = perh;
    irr = ir;
    return (1.f - r) - 0.5f * res * ir;
}

/* Per-call constants of a vehicle right-hand side: reciprocals of the model parameters that it
 * divides by, and tan(delta) of the kinematic model (the steering input is constant over an RK4
 * step).  Computed once per node instead of once per RK4 stage. */
struct ModelK {
    float iL, td, im, iIz;
};
template <int MODEL>
__device__ __forceinline__ ModelK model_k(const float *prm, float dl) {
    ModelK k{0.f, 0.f, 0.f, 0.f};
    if constexpr (MODEL == 0) {
        float sd, cd;
        sincos_cw(dl, &sd, &cd);
        k.iL = rcp(prm[0]);
        k.td = sd * rcp(cd);
    } else if constexpr (MODEL == 1) {
        k.im = rcp(prm[1]);
        k.iIz = rcp(prm[2]);
    }
    return k;
}

/* Continuous right-hand side and its Jacobians (dense arrays; compile-time zero
 * entries are folded away after unrolling).  MODEL 0: kinematic bicycle, 1: dynamic
 * bicycle with linear tyres and small steering angle, 3: unicycle (X' = v cos th,
 * Y' = v sin th, th' = omega, v' = a; the constraint benchmark of Sec. V-B). */
/* Structural nonzeros of the right-hand side's state Jacobian J = dF/dx as rhs_jac sets them (every
 * other entry stays 0).  The tangent propagation of dyn_lin skips the products with the structural
 * zeros: IEEE arithmetic does not let the compiler drop 0 * t itself, and acc + 0 * t = acc for
 * finite t, so the results are the same. */
template <int MODEL>
__host__ __device__ constexpr bool jac_nz(int i, int k) {
    if (MODEL == 0) return (i < 2 && (k == 2 || k == 3)) || (i == 2 && k == 3);
    if (MODEL == 3) return i < 2 && (k == 2 || k == 3);
    if (MODEL == 1)
        return (i < 2 && k >= 2 && k <= 4) || (i == 2 && k == 5) || (i == 3 && k >= 4) || (i >= 4 && k >= 3);
    return true;
}

template <int NX, int MODEL>
__device__ __forceinline__ void rhs_jac(const float *prm, const ModelK &mk, const float (&s)[NX], float a, float dl,
                                        float (&f)[NX], float (&J)[NX][NX], float (&Ju)[NX][NU]) {
#pragma unroll
    for (int i = 0; i < NX; ++i) {
#pragma unroll
        for (int j = 0; j < NX; ++j) J[i][j] = 0.f;
        Ju[i][0] = 0.f;
        Ju[i][1] = 0.f;
    }
    if constexpr (MODEL == 0) {
        float sp, cp;
        sincos_cw(s[2], &sp, &cp);
        const float td = mk.td, iL = mk.iL;
        const float v = s[3];
        f[0] = v * cp;
        f[1] = v * sp;
        f[2] = v * td * iL;
        f[3] = a;
        J[0][2] = -v * sp;
        J[0][3] = cp;
        J[1][2] = v * cp;
        J[1][3] = sp;
        J[2][3] = td * iL;
        Ju[2][1] = v * (1.f + td * td) * iL;
        Ju[3][0] = 1.f;
    } else if constexpr (MODEL == 1) {
        const float lf = prm[3], lr = prm[4], Cf = prm[5], Cr = prm[6];
        const float vmin = prm[7], veps = prm[8];
        const float im = mk.im, iIz = mk.iIz;
        const float psi = s[2], vx = s[3], vy = s[4], r = s[5];
        const float dv = vx - vmin;
        const float w2 = dv * dv + veps * veps;
        const float iw = rsqrtf(w2);   /* 1 / sqrt(dv^2 + veps^2) */
        const float vb = 0.5f * (vx + vmin + w2 * iw);
        const float dvb = 0.5f * (1.f + dv * iw);
        const float ivb = rcp(vb);
        const float tf = (vy + lf * r) * ivb, tr = (vy - lr * r) * ivb;
        const float af = atanf(tf) - dl, ar = atanf(tr);
        const float Ff = -Cf * af, Fr = -Cr * ar;
        float sp, cp;
        sincos_cw(psi, &sp, &cp);
        f[0] = vx * cp - vy * sp;
        f[1] = vx * sp + vy * cp;
        f[2] = r;
        f[3] = a + r * vy;
        f[4] = (Ff + Fr) * im - r * vx;
        f[5] = (lf * Ff - lr * Fr) * iIz;
        const float gf = rcp(1.f + tf * tf), gr = rcp(1.f + tr * tr);
        const float daf_vx = -gf * tf * ivb * dvb, daf_vy = gf * ivb, daf_r = gf * lf * ivb;
        const float dar_vx = -gr * tr * ivb * dvb, dar_vy = gr * ivb, dar_r = -gr * lr * ivb;
        const float dFf_vx = -Cf * daf_vx, dFf_vy = -Cf * daf_vy, dFf_r = -Cf * daf_r, dFf_d = Cf;
        const float dFr_vx = -Cr * dar_vx, dFr_vy = -Cr * dar_vy, dFr_r = -Cr * dar_r;
        J[0][2] = -vx * sp - vy * cp;
        J[0][3] = cp;
        J[0][4] = -sp;
        J[1][2] = vx * cp - vy * sp;
        J[1][3] = sp;
        J[1][4] = cp;
        J[2][5] = 1.f;
        J[3][4] = r;
        J[3][5] = vy;
        Ju[3][0] = 1.f;
        J[4][3] = (dFf_vx + dFr_vx) * im - r;
        J[4][4] = (dFf_vy + dFr_vy) * im;
        J[4][5] = (dFf_r + dFr_r) * im - vx;
        Ju[4][1] = dFf_d * im;
        J[5][3] = (lf * dFf_vx - lr * dFr_vx) * iIz;
        J[5][4] = (lf * dFf_vy - lr * dFr_vy) * iIz;
        J[5][5] = (lf * dFf_r - lr * dFr_r) * iIz;
        Ju[5][1] = lf * dFf_d * iIz;
    } else if constexpr (MODEL == 3) {
        float sp, cp;
        sincos_cw(s[2], &sp, &cp);
        const float v = s[3];
        f[0] = v * cp;
        f[1] = v * sp;
        f[2] = dl;
        f[3] = a;
        J[0][2] = -v * sp;
        J[0][3] = cp;
        J[1][2] = v * cp;
        J[1][3] = sp;
        Ju[2][1] = 1.f;
        Ju[3][0] = 1.f;
    }
}

template <int NX, int MODEL>
__device__ __forceinline__ void rhs(const float *prm, const ModelK &mk, const float (&s)[NX], float a, float dl,
                                    float (&f)[NX]) {
    if constexpr (MODEL == 0) {
        float sp, cp;
        sincos_cw(s[2], &sp, &cp);
        f[0] = s[3] * cp;
        f[1] = s[3] * sp;
        f[2] = s[3] * mk.td * mk.iL;
        f[3] = a;
    } else if constexpr (MODEL == 1) {
        const float lf = prm[3], lr = prm[4], Cf = prm[5], Cr = prm[6];
        const float vmin = prm[7], veps = prm[8];
        const float vx = s[3], vy = s[4], r = s[5];
        const float dv = vx - vmin;
        const float w2 = dv * dv + veps * veps;
        const float vb = 0.5f * (vx + vmin + w2 * rsqrtf(w2));
        const float ivb = rcp(vb);
        const float Ff = -Cf * (atanf((vy + lf * r) * ivb) - dl);
        const float Fr = -Cr * atanf((vy - lr * r) * ivb);
        float sp, cp;
        sincos_cw(s[2], &sp, &cp);
        f[0] = vx * cp - vy * sp;
        f[1] = vx * sp + vy * cp;
        f[2] = r;
        f[3] = a + r * vy;
        f[4] = (Ff + Fr) * mk.im - r * vx;
        f[5] = (lf * Ff - lr * Fr) * mk.iIz;
    } else if constexpr (MODEL == 3) {
        float sp, cp;
        sincos_cw(s[2], &sp, &cp);
        f[0] = s[3] * cp;
        f[1] = s[3] * sp;
        f[2] = dl;
        f[3] = a;
    }
}

/* Increment dlt = f(x, u) - x of the discrete dynamics with A = df/dx, B = df/du: n_sub
 * classical RK4 steps, Jacobians by the forward-mode chain rule through every stage (tangent
 * matrix S = dz/d(x, u)).  The increment is returned instead of f so that the defect
 * f(x_p, u_p) - x_m = (x_p - x_m) + dlt never subtracts two large absolute positions in FP32. */
template <int NX, int MODEL, typename Store>
__device__ __forceinline__ void dyn_lin(const ProbRec &R, const float (&x)[NX], const float (&u)[NU],
                                        float (&xn)[NX], Store store) {
    if constexpr (MODEL == 2) {
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < NX; ++j) {
                const float a = R.Alin[i * NX + j];
                store(i, j, a);
                s += (i == j ? a - 1.f : a) * x[j];
            }
#pragma unroll
            for (int j = 0; j < NU; ++j) {
                const float b = R.Blin[i * NU + j];
                store(i, NX + j, b);
                s += b * u[j];
            }
            xn[i] = s;
        }
    } else {
        /* The positions X, Y never enter the vehicle right-hand side, so their tangent columns
         * stay the unit vectors: only the columns of (psi, ..., a, delta) are propagated (forward
         * mode through every RK4 stage), and each entry is handed to `store` as soon as it is final. */
        constexpr int C0 = 2;
        constexpr int NZ = NX + NU;
        constexpr int GW = NZ - C0;   /* propagated tangent columns C0 .. NZ-1 */
        const int nsub = max(1, (int)R.params[9]);
        const float h = nsub == 1 ? R.dt : R.dt * rcp((float)nsub), h6 = h * (1.f / 6.f);
        const ModelK mk = model_k<MODEL>(R.params, u[1]);
        float S[NX][GW];
#pragma unroll
        for (int i = 0; i < NX; ++i)
#pragma unroll
            for (int j = 0; j < GW; ++j) S[i][j] = (i == C0 + j) ? 1.f : 0.f;
        float z[NX];   /* increment accumulated over the substeps */
#pragma unroll
        for (int i = 0; i < NX; ++i) z[i] = 0.f;
        for (int sub = 0; sub < nsub; ++sub) {
            float ks[NX], Ds[NX][GW], kp[NX], Dp[NX][GW];
#pragma unroll
            for (int i = 0; i < NX; ++i) {
                ks[i] = 0.f;
                kp[i] = 0.f;
#pragma unroll
                for (int j = 0; j < GW; ++j) {
                    Ds[i][j] = 0.f;
                    Dp[i][j] = 0.f;
                }
            }
#pragma unroll
            for (int st = 0; st < 4; ++st) {
                const float c = (st == 0) ? 0.f : (st == 3 ? 1.f : 0.5f);
                const float wg = (st == 0 || st == 3) ? 1.f : 2.f;
                float zs[NX];
#pragma unroll
                for (int i = 0; i < NX; ++i) zs[i] = x[i] + (z[i] + c * h * kp[i]);
                float f[NX], J[NX][NX], Ju[NX][NU];
                rhs_jac<NX, MODEL>(R.params, mk, zs, u[0], u[1], f, J, Ju);
#pragma unroll
                for (int j = 0; j < GW; ++j) {
                    const int jj = C0 + j;
                    float t[NX];
#pragma unroll
                    for (int k = C0; k < NX; ++k) t[k] = S[k][j] + c * h * Dp[k][j];
#pragma unroll
                    for (int i = 0; i < NX; ++i) {
                        float acc = (jj >= NX) ? Ju[i][jj - NX] : 0.f;
#pragma unroll
                        for (int k = C0; k < NX; ++k)
                            if (jac_nz<MODEL>(i, k)) acc += J[i][k] * t[k];
                        Ds[i][j] += wg * acc;
                        Dp[i][j] = acc;
                    }
                }
#pragma unroll
                for (int i = 0; i < NX; ++i) {
                    ks[i] += wg * f[i];
                    kp[i] = f[i];
                }
            }
#pragma unroll
            for (int i = 0; i < NX; ++i) {
                z[i] += h6 * ks[i];
#pragma unroll
                for (int j = 0; j < GW; ++j) S[i][j] += h6 * Ds[i][j];
            }
        }
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            xn[i] = z[i];
#pragma unroll
            for (int j = 0; j < GW; ++j) store(i, C0 + j, S[i][j]);
        }
    }
}

/* Increment f(x, u) - x of the discrete dynamics (no Jacobians). */
template <int NX, int MODEL>
__device__ __forceinline__ void dyn(const ProbRec &R, const float (&x)[NX], const float (&u)[NU], float (&xn)[NX]) {
    if constexpr (MODEL == 2) {
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < NX; ++j) s += (i == j ? R.Alin[i * NX + j] - 1.f : R.Alin[i * NX + j]) * x[j];
#pragma unroll
            for (int j = 0; j < NU; ++j) s += R.Blin[i * NU + j] * u[j];
            xn[i] = s;
        }
    } else {
        float z[NX];   /* increment */
#pragma unroll
        for (int i = 0; i < NX; ++i) z[i] = 0.f;
        const int nsub = max(1, (int)R.params[9]);
        const float h = nsub == 1 ? R.dt : R.dt * rcp((float)nsub), h6 = h * (1.f / 6.f);
        const ModelK mk = model_k<MODEL>(R.params, u[1]);
        for (int sub = 0; sub < nsub; ++sub) {
            float ks[NX], kp[NX];
#pragma unroll
            for (int i = 0; i < NX; ++i) {
                ks[i] = 0.f;
                kp[i] = 0.f;
            }
#pragma unroll
            for (int st = 0; st < 4; ++st) {
                const float c = (st == 0) ? 0.f : (st == 3 ? 1.f : 0.5f);
                const float wg = (st == 0 || st == 3) ? 1.f : 2.f;
                float zs[NX], f[NX];
#pragma unroll
                for (int i = 0; i < NX; ++i) zs[i] = x[i] + (z[i] + c * h * kp[i]);
                rhs<NX, MODEL>(R.params, mk, zs, u[0], u[1], f);
#pragma unroll
                for (int i = 0; i < NX; ++i) {
                    ks[i] += wg * f[i];
                    kp[i] = f[i];
                }
            }
#pragma unroll
            for (int i = 0; i < NX; ++i) z[i] += h6 * ks[i];
        }
#pragma unroll
        for (int i = 0; i < NX; ++i) xn[i] = z[i];
    }
}

/* Entries of the Jacobians A_n = df/dx and B_n = df/du that the model's structure fixes exactly:
 * 0 or 1 for a fixed entry, -1 for a computed one.  For the vehicle models the columns of the
 * positions X, Y are the unit vectors (positions do not enter the dynamics).  In the kinematic
 * bicycle and the unicycle (X, Y, heading, speed) the speed integrates the acceleration alone
 * (its row of A is e_3, its steering entry of B is 0), and the heading rate does not depend on the
 * heading (A[2][2] = 1); the unicycle's heading rate is its own input (A[2][3] = 0, B[2][0] = 0).
 * In the dynamic bicycle (X, Y, heading, v_x, v_y, r) only the positions' rates see the heading,
 * so its heading column is (*, *, 1, 0, 0, 0).
 * The forward-mode RK4 tangents produce these entries exactly (sums of exact zeros onto 1 or 0),
 * so reading them as constants changes no result; they are never loaded. */
template <int MODEL>
__host__ __device__ constexpr int a_fixed(int a, int b) {
    if (MODEL == 2) return -1;
    if (b < 2) return a == b ? 1 : 0;
    if (MODEL == 1) return b == 2 ? (a == 2 ? 1 : (a >= 3 ? 0 : -1)) : -1;   /* only X, Y see the heading */
    if (a == 2 && b == 2) return 1;
    if (a == 3) return b == 3 ? 1 : 0;
    if (MODEL == 3 && a == 2 && b == 3) return 0;
    return -1;
}
template <int MODEL>
__host__ __device__ constexpr int b_fixed(int a, int b) {
    if (MODEL != 0 && MODEL != 3) return -1;
    if (a == 3 && b == 1) return 0;
    if (MODEL == 3 && a == 2 && b == 0) return 0;
    return -1;
}
/* Index of row r of node i in a block of ROWS scratch rows.  The vehicle models' solver rows (A, B,
 * P, p, q, r, the penalty terms, the defects, dx, du, lam_QP, the merit terms) are tiled by 32
 * nodes, a tile's rows contiguous: ((i / 32) ROWS + r) 32 + i % 32.  Consecutive nodes stay
 * consecutive (coalesced node-parallel phases) and one node's rows sit at fixed offsets from one
 * address (the per-path sweeps).  The linear model keeps component-major rows: with per-edge
 * dynamics its A, B are input rows. */
template <int ROWS, int MODEL>
__device__ __forceinline__ size_t jrow(int np, int i, int r) {
    if constexpr (MODEL == 2) return (size_t)r * np + i;
    else return ((size_t)(i >> 5) * ROWS + r) * 32 + (i & 31);
}
template <int NX, int MODEL>
__device__ __forceinline__ float aload(const float *A, int np, int i, int a, int b) {
    if (a_fixed<MODEL>(a, b) >= 0) return (float)a_fixed<MODEL>(a, b);
    return A[jrow<NX * NX, MODEL>(np, i, a * NX + b)];
}
template <int NX, int MODEL>
__device__ __forceinline__ float bload(const float *B, int np, int i, int a, int b) {
    if (b_fixed<MODEL>(a, b) >= 0) return (float)b_fixed<MODEL>(a, b);
    return B[jrow<NX * NU, MODEL>(np, i, a * NU + b)];
}
/* ROWS consecutive scratch rows of node i (tiled like the Jacobian rows for the vehicle models). */
template <int ROWS, int MODEL>
__device__ __forceinline__ void ld_rows(const float *base, int np, int i, float (&v)[ROWS]) {
#pragma unroll
    for (int r = 0; r < ROWS; ++r) v[r] = base[jrow<ROWS, MODEL>(np, i, r)];
}
template <int ROWS, int MODEL>
__device__ __forceinline__ void st_rows(float *base, int np, int i, const float (&v)[ROWS]) {
#pragma unroll
    for (int r = 0; r < ROWS; ++r) base[jrow<ROWS, MODEL>(np, i, r)] = v[r];
}

/* ------------------------------------------------------------------ problem view */
template <int NX>
struct View {
    int n, np, nc, nobs;
    bool box, lane;
    /* int rows */
    const int32_t *parent, *nchild, *fchild, *stage, *leaf, *owner, *sstart, *bstage, *ptab, *pdepth, *ptop;
    const int32_t *fnode, *fend, *wave;   /* segment order of the scan sweeps */
    int64_t tab_off;
    /* inputs */
    const float *xref, *w, *obs, *wx, *wu, *wl, *wy;
    /* outputs */
    float *X, *U, *L, *Y;
    /* scratch */
    float *A, *B, *f, *d, *q, *r, *hq, *hr, *K, *k, *P, *p, *dx, *du, *lq, *nv, *XL, *UL;
    float *CV0, *CV1, *JA0, *JA1;   /* scan buffers (two of each) */
    bool comp;   /* compensated iterate (Lo parts) in use */
    bool edge;   /* per-edge linear dynamics: A, B point at the input rows, f and A, B are per edge */
    bool hess;   /* exact-Hessian option: the node blocks Q, M, R are the dense rows HS */
    float *HS;
    float *FR;   /* node-major forward records (fr_stride(NX) floats per node) */

    __device__ View(const ProbRec &R, const int32_t *ib, const float *fin, const float *fw, float *fout, float *fs) {
        n = R.n;
        np = R.npad;
        nc = R.nc;
        nobs = R.n_obs;
        box = R.box_on != 0;
        lane = R.lane_on != 0;
        const IntOff io = int_off(np, R.n_stage, R.n_paths, R.n_waves);
        fnode = ib + io.fnode;
        fend = ib + io.fend;
        wave = ib + io.wave;
        parent = ib + io.parent;
        nchild = ib + io.nchild;
        fchild = ib + io.fchild;
        stage = ib + io.stage;
        leaf = ib + io.leaf;
        owner = ib + io.owner;
        sstart = ib + io.sstart;
        bstage = ib + io.bstage;
        ptab = ib + io.ptab;
        pdepth = ib + io.pdepth;
        ptop = ib + io.ptop;
        tab_off = io.sstart;
        const InRows ir = in_rows(NX, nobs, R.edge_dyn);
        xref = fin + (size_t)ir.xref * np;
        w = fin + (size_t)ir.weight * np;
        obs = fin + (size_t)ir.obs * np;
        fwarm = fw;
        set_slot(0);
        const OutRows orw = out_rows(NX, nc);
        X = fout + (size_t)orw.x * np;
        U = fout + (size_t)orw.u * np;
        L = fout + (size_t)orw.lam * np;
        Y = fout + (size_t)orw.y * np;
        const ScrRows s = scr_rows(NX);
        A = fs + (size_t)s.A * np;
        B = fs + (size_t)s.B * np;
        f = fs + (size_t)s.f * np;
        d = fs + (size_t)s.d * np;
        q = fs + (size_t)s.q * np;
        r = fs + (size_t)s.r * np;
        hq = fs + (size_t)s.hq * np;
        hr = fs + (size_t)s.hr * np;
        K = fs + (size_t)s.K * np;
        k = fs + (size_t)s.k * np;
        P = fs + (size_t)s.P * np;
        p = fs + (size_t)s.p * np;
        dx = fs + (size_t)s.dx * np;
        du = fs + (size_t)s.du * np;
        lq = fs + (size_t)s.lq * np;
        nv = fs + (size_t)s.nv * np;
        XL = fs + (size_t)s.xl * np;
        UL = fs + (size_t)s.ul * np;
        edge = false;   /* set by the solver for the linear model (per-edge dynamics) */
        hess = false;
        HS = fs + (size_t)s.hs * np;
        FR = fs + (size_t)s.fr * np;
        CV0 = fs + (size_t)s.cv * np;
        CV1 = CV0 + (size_t)cvf_rows(NX) * np;
        JA0 = fs + (size_t)s.ja * np;
        JA1 = JA0 + np;
        comp = false;
    }
    const float *fwarm;
    /* point wx .. wy at warm-start slot s */
    __device__ __forceinline__ void set_slot(int s) {
        const WarmRows wr = warm_rows(NX, nc);
        const float *b = fwarm + (size_t)s * wr.total * np;
        wx = b + (size_t)wr.wx * np;
        wu = b + (size_t)wr.wu * np;
        wl = b + (size_t)wr.wl * np;
        wy = b + (size_t)wr.wy * np;
    }
    __device__ __forceinline__ void load_x(const float *base, int i, float (&v)[NX]) const {
#pragma unroll
        for (int j = 0; j < NX; ++j) v[j] = base[(size_t)j * np + i];
    }
    __device__ __forceinline__ void store_x(float *base, int i, const float (&v)[NX]) const {
#pragma unroll
        for (int j = 0; j < NX; ++j) base[(size_t)j * np + i] = v[j];
    }
    __device__ __forceinline__ void load_u(const float *base, int i, float (&v)[NU]) const {
        v[0] = base[i];
        v[1] = base[(size_t)np + i];
    }
    /* low-order parts of node i's iterate (zero when the iterate is not compensated) */
    __device__ __forceinline__ void load_lo(int i, Lo &lo) const {
        if (comp) {
            lo.x[0] = XL[i];
            lo.x[1] = XL[(size_t)np + i];
            lo.u[0] = UL[i];
            lo.u[1] = UL[(size_t)np + i];
        } else {
            lo.x[0] = lo.x[1] = lo.u[0] = lo.u[1] = 0.f;
        }
    }
    __device__ __forceinline__ void store_lo(int i, const Lo &lo) const {
        if (comp) {
            XL[i] = lo.x[0];
            XL[(size_t)np + i] = lo.x[1];
            UL[i] = lo.u[0];
            UL[(size_t)np + i] = lo.u[1];
        }
    }
    __device__ __forceinline__ void store_u(float *base, int i, const float (&v)[NU]) const {
        base[i] = v[0];
        base[(size_t)np + i] = v[1];
    }
};

/* ------------------------------------------------------------------ node cost + constraints */
/* Node part of L_a (Eq. AL) at (x, u) with multipliers y and penalty rho.  With grad != 0 also
 * the gradient (q, r) and the Gauss-Newton Hessian terms of the penalty: hq = (xx, xy, yy) on
 * the position block, hr on the input diagonal.  mode: 0 = value only. */
template <int NX, bool GRAD>
__device__ __forceinline__ float node_la(const ProbRec &R, const View<NX> &V, int i, bool is_leaf,
                                         const float (&x)[NX], const float (&u)[NU], const Lo &lo, float rho,
                                         float (&q)[NX], float (&r)[NU], float (&hq)[3], float (&hr)[NU]) {
    /* x is the deviation from the node's reference (the kernel's state coordinates) */
    const float w = V.w[i];
    const float *Qd = is_leaf ? R.QNw : R.Qw;
    const float irho = rcp(rho);
    float la = 0.f;
#pragma unroll
    for (int j = 0; j < NX; ++j) {
        const float e = x[j];
        la += 0.5f * w * Qd[j] * e * e;
        if (GRAD) q[j] = w * Qd[j] * e;
    }
#pragma unroll
    for (int j = 0; j < NU; ++j) {
        if (GRAD) {
            r[j] = 0.f;
            hr[j] = 0.f;
        }
        if (!is_leaf) {
            la += 0.5f * w * R.Rw[j] * u[j] * u[j];
            if (GRAD) r[j] = w * R.Rw[j] * u[j];
        }
    }
    if (GRAD) hq[0] = hq[1] = hq[2] = 0.f;
    int row = 0;
    if (V.box) {
        if (!is_leaf) {
#pragma unroll
            for (int j = 0; j < NU; ++j) {
#pragma unroll
                for (int sgn = 0; sgn < 2; ++sgn) {
                    const int rr = row + sgn * NU + j;
                    const float g = sgn == 0 ? (u[j] - R.u_hi[j]) + lo.u[j] : (R.u_lo[j] - u[j]) - lo.u[j];
                    const float s = V.Y[(size_t)rr * V.np + i] + rho * g;
                    if (s > 0.f) {
                        la += 0.5f * s * s * irho;
                        if (GRAD) {
                            r[j] += sgn == 0 ? s : -s;
                            hr[j] += rho;
                        }
                    }
                }
            }
        }
        row += 2 * NU;
    }
    if (i != 0) {
        for (int o = 0; o < V.nobs; ++o) {
            const float *ob = V.obs + (size_t)(OBS_ROWS * o) * V.np + i;
            const float cx = ob[0], cy = ob[V.np], ch = ob[2 * (size_t)V.np], sh = ob[3 * (size_t)V.np];
            const float ia2 = ob[4 * (size_t)V.np], ib2 = ob[5 * (size_t)V.np];
            float dpar, dper, irr, g;
            if (V.comp) {
                g = obs_g_comp(V.xref[i], V.xref[(size_t)V.np + i], cx, cy, x[0], lo.x[0], x[1], lo.x[1], ch, sh, ia2,
                               ib2, dpar, dper, irr);
            } else {
                const float dxo = (V.xref[i] - cx) + x[0], dyo = (V.xref[(size_t)V.np + i] - cy) + x[1];
                dpar = ch * dxo + sh * dyo;
                dper = -sh * dxo + ch * dyo;
                const float q2 = dpar * dpar * ia2 + dper * dper * ib2 + 1e-6f;
                irr = rsqrtf(q2);   /* 1 / rr2 */
                g = 1.f - q2 * irr;
            }
            const float s = V.Y[(size_t)(row + o) * V.np + i] + rho * g;
            if (s > 0.f) {
                la += 0.5f * s * s * irho;
                if (GRAD) {
                    const float gx = -(dpar * ia2 * ch - dper * ib2 * sh) * irr;
                    const float gy = -(dpar * ia2 * sh + dper * ib2 * ch) * irr;
                    q[0] += s * gx;
                    q[1] += s * gy;
                    hq[0] += rho * gx * gx;
                    hq[1] += rho * gx * gy;
                    hq[2] += rho * gy * gy;
                }
            }
        }
        row += V.nobs;
        if (V.lane) {
            const float yr = V.xref[(size_t)V.np + i];
            const float g0 = ((yr - R.lane_hi) + x[1]) + lo.x[1], g1 = ((R.lane_lo - yr) - x[1]) - lo.x[1];
            const float s0 = V.Y[(size_t)row * V.np + i] + rho * g0;
            const float s1 = V.Y[(size_t)(row + 1) * V.np + i] + rho * g1;
            if (s0 > 0.f) {
                la += 0.5f * s0 * s0 * irho;
                if (GRAD) {
                    q[1] += s0;
                    hq[2] += rho;
                }
            }
            if (s1 > 0.f) {
                la += 0.5f * s1 * s1 * irho;
                if (GRAD) {
                    q[1] -= s1;
                    hq[2] += rho;
                }
            }
        }
    }
    return la;
}

/* Constraint rows g (existing rows only, others skipped) at the deviation x: calls fn(row, g). */
template <int NX, typename Fn>
__device__ __forceinline__ void for_constraints(const ProbRec &R, const View<NX> &V, int i, bool is_leaf,
                                                const float (&x)[NX], const float (&u)[NU], const Lo &lo, Fn fn) {
    int row = 0;
    if (V.box) {
        if (!is_leaf) {
#pragma unroll
            for (int j = 0; j < NU; ++j) {
                fn(row + j, (u[j] - R.u_hi[j]) + lo.u[j]);
                fn(row + NU + j, (R.u_lo[j] - u[j]) - lo.u[j]);
            }
        }
        row += 2 * NU;
    }
    if (i != 0) {
        for (int o = 0; o < V.nobs; ++o) {
            const float *ob = V.obs + (size_t)(OBS_ROWS * o) * V.np + i;
            const float cx = ob[0], cy = ob[V.np], ch = ob[2 * (size_t)V.np], sh = ob[3 * (size_t)V.np];
            const float ia2 = ob[4 * (size_t)V.np], ib2 = ob[5 * (size_t)V.np];
            if (V.comp) {
                float dpar, dper, irr;
                fn(row + o, obs_g_comp(V.xref[i], V.xref[(size_t)V.np + i], cx, cy, x[0], lo.x[0], x[1], lo.x[1], ch,
                                       sh, ia2, ib2, dpar, dper, irr));
            } else {
                const float dxo = (V.xref[i] - cx) + x[0], dyo = (V.xref[(size_t)V.np + i] - cy) + x[1];
                const float dpar = ch * dxo + sh * dyo, dper = -sh * dxo + ch * dyo;
                const float q2 = dpar * dpar * ia2 + dper * dper * ib2 + 1e-6f;
                fn(row + o, 1.f - q2 * rsqrtf(q2));
            }
        }
        row += V.nobs;
        if (V.lane) {
            const float yr = V.xref[(size_t)V.np + i];
            fn(row, ((yr - R.lane_hi) + x[1]) + lo.x[1]);
            fn(row + 1, ((R.lane_lo - yr) - x[1]) - lo.x[1]);
        }
    }
}


/* Asynchronous 4-byte copy global -> shared (cp.async, cached in L1) and its group control. */
__device__ __forceinline__ void cp4(float *dst, const float *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

/* ------------------------------------------------------------------ tree Riccati step */
/* Terminal value function of a leaf: P = Q_N + penalty Hessian, p = q (stored and returned). */
template <int NX, int MODEL>
__device__ __forceinline__ void leaf_value(const ProbRec &R, const View<NX> &V, int i, float (&P)[nsym(NX)],
                                           float (&p)[NX]) {
    constexpr int NS = nsym(NX);
    const int np = V.np;
    const float w = V.w[i];
    const float hxx = V.hq[jrow<3, MODEL>(np, i, 0)], hxy = V.hq[jrow<3, MODEL>(np, i, 1)], hyy = V.hq[jrow<3, MODEL>(np, i, 2)];
#pragma unroll
    for (int a = 0; a < NX; ++a)
#pragma unroll
        for (int b = a; b < NX; ++b) {
            float v = (a == b) ? w * R.QNw[a] : 0.f;
            if (a == 0 && b == 0) v += hxx;
            if (a == 0 && b == 1) v += hxy;
            if (a == 1 && b == 1) v += hyy;
            if (V.hess) v = V.HS[(size_t)sidx<NX>(a, b) * np + i];
            P[sidx<NX>(a, b)] = v;
        }
#pragma unroll
    for (int e = 0; e < NS; ++e) V.P[jrow<NS, MODEL>(np, i, e)] = P[e];
#pragma unroll
    for (int a = 0; a < NX; ++a) {
        p[a] = V.q[jrow<NX, MODEL>(np, i, a)];
        V.p[jrow<NX, MODEL>(np, i, a)] = p[a];
    }
}

/* Stores an NX-vector as float2 pairs (dst 8-byte aligned). */
template <int NX>
__device__ __forceinline__ void put_pairs(float *dst, const float (&v)[NX]) {
#pragma unroll
    for (int j = 0; j < NX / 2; ++j) reinterpret_cast<float2 *>(dst)[j] = make_float2(v[2 * j], v[2 * j + 1]);
}

/* Adds the value function of child m to (Pb, pb): Pb += P_m, pb += p_m + P_m d_m, with
 * P_m, p_m, d_m read from memory (Eq. tree_Riccati, sum over ch(n)). */
template <int NX, int MODEL>
__device__ __forceinline__ void add_child_mem(const View<NX> &V, int m, float (&Pb)[nsym(NX)], float (&pb)[NX],
                                              float *dst = nullptr) {
    constexpr int NS = nsym(NX);
    const int np = V.np;
    float Pm[NS], dm[NX];
#pragma unroll
    for (int e = 0; e < NS; ++e) {
        Pm[e] = V.P[jrow<NS, MODEL>(np, m, e)];
        Pb[e] += Pm[e];
    }
    ld_rows<NX, MODEL>(V.d, V.np, m, dm);
    if (dst) put_pairs<NX>(dst, dm);   /* the child's defect into its forward record */
#pragma unroll
    for (int a = 0; a < NX; ++a) {
        float v = V.p[jrow<NX, MODEL>(np, m, a)];
#pragma unroll
        for (int b = 0; b < NX; ++b) v += Pm[sidx<NX>(a, b)] * dm[b];
        pb[a] += v;
    }
}

/* Inputs of the Riccati step at a node: Jacobians (with the constant position columns), cost
 * gradient q, r and the diagonal/penalty Hessian terms. */
template <int NX>
struct RicIn {
    float A[NX][NX], B[NX][NU], q[NX], r[NU], hq[3], hr[NU], w;
};

/* ja: the column of the Jacobians (node i's own for dynamics per node; the edge into its single
 * child for per-edge dynamics) */
template <int NX, int MODEL>
__device__ __forceinline__ void ric_load(const View<NX> &V, int i, RicIn<NX> &in, int ja = -1) {
    const int np = V.np;
    if (ja < 0) ja = i;
    in.w = V.w[i];
    ld_rows<NX, MODEL>(V.q, V.np, i, in.q);
#pragma unroll
    for (int a = 0; a < 3; ++a) in.hq[a] = V.hq[jrow<3, MODEL>(np, i, a)];
#pragma unroll
    for (int a = 0; a < NX; ++a) {
#pragma unroll
        for (int b = 0; b < NX; ++b) in.A[a][b] = aload<NX, MODEL>(V.A, np, ja, a, b);
#pragma unroll
        for (int b = 0; b < NU; ++b) in.B[a][b] = bload<NX, MODEL>(V.B, np, ja, a, b);
    }
#pragma unroll
    for (int a = 0; a < NU; ++a) {
        in.r[a] = V.r[jrow<NU, MODEL>(np, i, a)];
        in.hr[a] = V.hr[jrow<NU, MODEL>(np, i, a)];
    }
}

/* Staging of the per-path forward sweep: each path thread streams the rows of the nodes it visits
 * next into its own shared-memory slots (SWEEP_DEPTH buffers filled by cp.async), so that the loads
 * of the next stages overlap the arithmetic of the current one.  Slot (buffer, row, thread) lives
 * at stg[(buffer * rows + row) * ld + thread].  (The backward sweep loads directly: its Riccati
 * step is long enough that staging did not pay for its extra instructions.) */
constexpr int SWEEP_DEPTH = 3;
template <int NX, int MODEL>
__host__ __device__ constexpr int jac_stored() {   /* entries of A and B that are not fixed */
    int c = 0;
    for (int a = 0; a < NX; ++a) {
        for (int b = 0; b < NX; ++b) c += a_fixed<MODEL>(a, b) < 0;
        for (int b = 0; b < NU; ++b) c += b_fixed<MODEL>(a, b) < 0;
    }
    return c;
}
template <int NX, int MODEL>
__host__ __device__ constexpr int rows_stage() { return NX + jac_stored<NX, MODEL>() + NX * NU + NU; }

/* Position of the stored Jacobian entry (a, c) (column c < NX: A, else B) among the entries that
 * are not structurally fixed, in row-major order over [A B]. */
template <int NX, int MODEL>
__host__ __device__ constexpr int jac_slot(int a, int c) {
    int k = 0;
    for (int i = 0; i < NX; ++i)
        for (int j = 0; j < NX + NU; ++j) {
            if (i == a && j == c) return k;
            k += (j < NX ? a_fixed<MODEL>(i, j) : b_fixed<MODEL>(i, j - NX)) < 0;
        }
    return -1;
}

/* Models whose per-path forward sweep reads node-major records (not the linear model, whose A, B
 * may be per edge and live in the input rows). */
template <int MODEL>
__host__ __device__ constexpr bool frec_model() { return MODEL != 2; }

/* Node-major forward record of node i (the vehicle models; per-edge linear dynamics keep the rows):
 * K_i, the stored entries of A_i and B_i, k_i and d_i (the defect of the edge into i), written by the
 * tree Riccati step, the linearisation and the defect phase.  A per-path forward stage moves the
 * node's record with used/4 16-byte copies from one base address instead of one 4-byte copy per
 * row; the parent's A, B come from the record the stage before read. */
template <int NX, int MODEL>
struct Frec {
    static constexpr int K = 0, J = NU * NX, k = NU * NX + jac_stored<NX, MODEL>(), d = k + NU;
    static constexpr int used = (d + NX + 3) & ~3;
    static constexpr int stride = fr_stride(NX);
    static constexpr int ring = 4;                       /* records in flight per path thread */
    static constexpr int tstride = ring * used + 4;      /* floats per thread (spreads the banks) */
    static_assert(!frec_model<MODEL>() || used <= stride, "forward record larger than its allocation");
    static_assert(J % 4 == 0, "the Jacobian block must start on 16 bytes");
};

/* Riccati step of a non-leaf node n from the summed child value functions (Pb, pb):
 * H_n = R_n + B'Pb B, K_n = -H^-1 (M_n + B'Pb A), k_n = -H^-1 (r_n + B'pb) of
 * Eq. (tree_feedback_laws) (M_n = 0 here: no constraint couples x and u), then
 * P_n = Q_n + A'Pb A + Qux'K, p_n = q_n + A'pb + Qux'k.  Stores K, k, P, p; returns P, p. */
template <int NX, int MODEL, bool STORE_PV = true>
__device__ __forceinline__ void riccati_node(const ProbRec &R, const View<NX> &V, int i, const RicIn<NX> &in,
                                             const float (&Pb)[nsym(NX)], const float (&pb)[NX],
                                             float (&P)[nsym(NX)], float (&p)[NX], Shared &sh,
                                             float *rec = nullptr) {
    const int np = V.np;
    const float w = in.w;
    const float(&q)[NX] = in.q;
    const float hxx = in.hq[0], hxy = in.hq[1], hyy = in.hq[2];
    const float(&A)[NX][NX] = in.A;
    const float(&B)[NX][NU] = in.B;
    /* PA = Pbar A, PB = Pbar B */
    float PA[NX][NX], PB[NX][NU];
#pragma unroll
    for (int a = 0; a < NX; ++a) {
#pragma unroll
        for (int b = 0; b < NX; ++b) {
            float v = 0.f;
#pragma unroll
            for (int t = 0; t < NX; ++t) v += Pb[sidx<NX>(a, t)] * A[t][b];
            PA[a][b] = v;
        }
#pragma unroll
        for (int b = 0; b < NU; ++b) {
            float v = 0.f;
#pragma unroll
            for (int t = 0; t < NX; ++t) v += Pb[sidx<NX>(a, t)] * B[t][b];
            PB[a][b] = v;
        }
    }
    /* H blocks: Quu = R + B'PB, Qux = M + B'PA, qu = r + B'pbar, qx = q + A'pbar (M = 0 and R, Q
     * diagonal plus penalty terms for Gauss-Newton; the dense modified blocks of the exact option) */
    float Quu[NU][NU], Qux[NU][NX], qu[NU], qx[NX];
    const float *HSr = V.HS + nsym(NX) * (size_t)np + i;   /* M then R (packed) of the exact option */
#pragma unroll
    for (int a = 0; a < NU; ++a) {
#pragma unroll
        for (int b = 0; b < NU; ++b) {
            float v = V.hess ? HSr[(size_t)(NU * NX + (a + b)) * np] : ((a == b) ? w * R.Rw[a] + in.hr[a] : 0.f);
#pragma unroll
            for (int t = 0; t < NX; ++t) v += B[t][a] * PB[t][b];
            Quu[a][b] = v;
        }
#pragma unroll
        for (int b = 0; b < NX; ++b) {
            float v = V.hess ? HSr[(size_t)(a * NX + b) * np] : 0.f;
#pragma unroll
            for (int t = 0; t < NX; ++t) v += B[t][a] * PA[t][b];
            Qux[a][b] = v;
        }
        float v = in.r[a];
#pragma unroll
        for (int t = 0; t < NX; ++t) v += B[t][a] * pb[t];
        qu[a] = v;
    }
#pragma unroll
    for (int a = 0; a < NX; ++a) {
        float v = q[a];
#pragma unroll
        for (int t = 0; t < NX; ++t) v += A[t][a] * pb[t];
        qx[a] = v;
    }
    /* K = -H^-1 Qux, k = -H^-1 qu with the closed-form inverse of the 2x2 H_n (one reciprocal of
     * the determinant on the critical path; H_n must be positive definite) */
    const float h00 = Quu[0][0], h01 = Quu[1][0], h11 = Quu[1][1];
    const float det = h00 * h11 - h01 * h01;
    if (!(h00 > 0.f) || !(det > 0.f)) sh.flag = 1;
    const float idet = 1.f / det;   /* IEEE-rounded: the direction's accuracy sets the FP32 KKT floor */
    const float g00 = h11 * idet, g01 = -h01 * idet, g11 = h00 * idet;
    float Kn[NU][NX], kn[NU];
#pragma unroll
    for (int b = 0; b < NX + 1; ++b) {
        const float rhs0 = (b < NX) ? Qux[0][b] : qu[0];
        const float rhs1 = (b < NX) ? Qux[1][b] : qu[1];
        const float s0 = g00 * rhs0 + g01 * rhs1;
        const float s1 = g01 * rhs0 + g11 * rhs1;
        if (b < NX) {
            Kn[0][b] = -s0;
            Kn[1][b] = -s1;
        } else {
            kn[0] = -s0;
            kn[1] = -s1;
        }
    }
    /* P = Qxx + Qux'K with Qxx = Q + A'PA; p = qx + Qux'k */
#pragma unroll
    for (int a = 0; a < NX; ++a)
#pragma unroll
        for (int b = a; b < NX; ++b) {
            float v = (a == b) ? w * R.Qw[a] : 0.f;
            if (a == 0 && b == 0) v += hxx;
            if (a == 0 && b == 1) v += hxy;
            if (a == 1 && b == 1) v += hyy;
            if (V.hess) v = V.HS[(size_t)sidx<NX>(a, b) * np + i];
#pragma unroll
            for (int t = 0; t < NX; ++t) v += A[t][a] * PA[t][b];
#pragma unroll
            for (int t = 0; t < NU; ++t) v += Qux[t][a] * Kn[t][b];
            P[sidx<NX>(a, b)] = v;
            if (STORE_PV) V.P[jrow<nsym(NX), MODEL>(np, i, sidx<NX>(a, b))] = v;
        }
#pragma unroll
    for (int a = 0; a < NX; ++a) {
        float v = qx[a];
#pragma unroll
        for (int t = 0; t < NU; ++t) v += Qux[t][a] * kn[t];
        p[a] = v;
        if (STORE_PV) V.p[jrow<NX, MODEL>(np, i, a)] = v;
    }
    if constexpr (frec_model<MODEL>()) {
        if (rec) {   /* the node's forward record instead of the K, k rows: K, the stored A, B entries, k */
            using F = Frec<NX, MODEL>;
            constexpr int JS = F::k - F::J;
            float jv[JS];
#pragma unroll
            for (int a = 0; a < NX; ++a) {
#pragma unroll
                for (int b = 0; b < NX; ++b)
                    if (a_fixed<MODEL>(a, b) < 0) jv[jac_slot<NX, MODEL>(a, b)] = A[a][b];
#pragma unroll
                for (int b = 0; b < NU; ++b)
                    if (b_fixed<MODEL>(a, b) < 0) jv[jac_slot<NX, MODEL>(a, NX + b)] = B[a][b];
            }
            float4 *rK = reinterpret_cast<float4 *>(rec + F::K);
#pragma unroll
            for (int q = 0; q < NU * NX / 4; ++q) {
                const int e = 4 * q;
                rK[q] = make_float4(Kn[e / NX][e % NX], Kn[(e + 1) / NX][(e + 1) % NX], Kn[(e + 2) / NX][(e + 2) % NX],
                                    Kn[(e + 3) / NX][(e + 3) % NX]);
            }
            float4 *rJ = reinterpret_cast<float4 *>(rec + F::J);
#pragma unroll
            for (int q = 0; q < JS / 4; ++q) rJ[q] = make_float4(jv[4 * q], jv[4 * q + 1], jv[4 * q + 2], jv[4 * q + 3]);
            if constexpr (JS % 4 == 2)
                *reinterpret_cast<float2 *>(rec + F::k - 2) = make_float2(jv[JS - 2], jv[JS - 1]);
            *reinterpret_cast<float2 *>(rec + F::k) = make_float2(kn[0], kn[1]);
            return;
        }
    }
#pragma unroll
    for (int a = 0; a < NU; ++a) {
#pragma unroll
        for (int b = 0; b < NX; ++b) V.K[(size_t)(a * NX + b) * np + i] = Kn[a][b];
        V.k[(size_t)a * np + i] = kn[a];
    }
}

/* Per-edge linear dynamics: the increment f_m(x_p, u_p) - x_p = (A_m - I) xa + B_m u of the edge into
 * node m at the parent's absolute state xa and input u. */
template <int NX>
__device__ __forceinline__ void edge_increment(const View<NX> &V, int m, const float (&xa)[NX], const float (&u)[NU],
                                               float (&dl)[NX]) {
    const int np = V.np;
#pragma unroll
    for (int a = 0; a < NX; ++a) {
        float s = 0.f;
#pragma unroll
        for (int b = 0; b < NX; ++b) s += (V.A[(size_t)(a * NX + b) * np + m] - (a == b ? 1.f : 0.f)) * xa[b];
#pragma unroll
        for (int b = 0; b < NU; ++b) s += V.B[(size_t)(a * NU + b) * np + m] * u[b];
        dl[a] = s;
    }
}

/* Riccati step of a node with several children under per-edge dynamics (Eq. tree_Riccati with every
 * child carried back through its own edge): Qxx = Q + sum A_m'P_m A_m, Qux = sum B_m'P_m A_m,
 * H = R + sum B_m'P_m B_m, qx = q + sum A_m'(p_m + P_m d_m), qu = r + sum B_m'(p_m + P_m d_m); then
 * the law and the value function as in riccati_node.  Stores K, k, P, p; returns P, p. */
template <int NX>
__device__ void riccati_edges(const ProbRec &R, const View<NX> &V, int i, float (&P)[nsym(NX)], float (&p)[NX],
                              Shared &sh) {
    constexpr int NS = nsym(NX);
    const int np = V.np;
    float Qxx[NX][NX], Qux[NU][NX], Quu[NU][NU], qx[NX], qu[NU];
#pragma unroll
    for (int a = 0; a < NX; ++a) {
        qx[a] = 0.f;
#pragma unroll
        for (int b = 0; b < NX; ++b) Qxx[a][b] = 0.f;
    }
#pragma unroll
    for (int a = 0; a < NU; ++a) {
        qu[a] = 0.f;
#pragma unroll
        for (int b = 0; b < NX; ++b) Qux[a][b] = 0.f;
#pragma unroll
        for (int b = 0; b < NU; ++b) Quu[a][b] = 0.f;
    }
    const int fc = V.fchild[i], nch = V.nchild[i];
    for (int m = fc; m < fc + nch; ++m) {
        float Pm[NS], pbm[NX], Am[NX][NX], Bm[NX][NU], dm[NX];
#pragma unroll
        for (int e = 0; e < NS; ++e) Pm[e] = V.P[(size_t)e * np + m];
        V.load_x(V.d, m, dm);
#pragma unroll
        for (int a = 0; a < NX; ++a) {
            float v = V.p[(size_t)a * np + m];
#pragma unroll
            for (int b = 0; b < NX; ++b) v += Pm[sidx<NX>(a, b)] * dm[b];
            pbm[a] = v;
#pragma unroll
            for (int b = 0; b < NX; ++b) Am[a][b] = V.A[(size_t)(a * NX + b) * np + m];
#pragma unroll
            for (int b = 0; b < NU; ++b) Bm[a][b] = V.B[(size_t)(a * NU + b) * np + m];
        }
        float PA[NX][NX], PB[NX][NU];
#pragma unroll
        for (int a = 0; a < NX; ++a) {
#pragma unroll
            for (int b = 0; b < NX; ++b) {
                float v = 0.f;
#pragma unroll
                for (int t = 0; t < NX; ++t) v += Pm[sidx<NX>(a, t)] * Am[t][b];
                PA[a][b] = v;
            }
#pragma unroll
            for (int b = 0; b < NU; ++b) {
                float v = 0.f;
#pragma unroll
                for (int t = 0; t < NX; ++t) v += Pm[sidx<NX>(a, t)] * Bm[t][b];
                PB[a][b] = v;
            }
        }
#pragma unroll
        for (int a = 0; a < NX; ++a) {
#pragma unroll
            for (int b = a; b < NX; ++b) {
                float v = 0.f;
#pragma unroll
                for (int t = 0; t < NX; ++t) v += Am[t][a] * PA[t][b];
                Qxx[a][b] += v;
            }
            float v = 0.f;
#pragma unroll
            for (int t = 0; t < NX; ++t) v += Am[t][a] * pbm[t];
            qx[a] += v;
        }
#pragma unroll
        for (int j = 0; j < NU; ++j) {
#pragma unroll
            for (int b = 0; b < NX; ++b) {
                float v = 0.f;
#pragma unroll
                for (int t = 0; t < NX; ++t) v += Bm[t][j] * PA[t][b];
                Qux[j][b] += v;
            }
#pragma unroll
            for (int l = 0; l < NU; ++l) {
                float v = 0.f;
#pragma unroll
                for (int t = 0; t < NX; ++t) v += Bm[t][j] * PB[t][l];
                Quu[j][l] += v;
            }
            float v = 0.f;
#pragma unroll
            for (int t = 0; t < NX; ++t) v += Bm[t][j] * pbm[t];
            qu[j] += v;
        }
    }
    const float w = V.w[i];
    if (V.hess) {   /* the exact option's dense modified block: R and M here, Q below */
        const float *HSr = V.HS + nsym(NX) * (size_t)np + i;
#pragma unroll
        for (int a = 0; a < NU; ++a) {
#pragma unroll
            for (int b = 0; b < NU; ++b) Quu[a][b] += HSr[(size_t)(NU * NX + a + b) * np];
#pragma unroll
            for (int b = 0; b < NX; ++b) Qux[a][b] += HSr[(size_t)(a * NX + b) * np];
        }
    }
#pragma unroll
    for (int a = 0; a < NU; ++a) {
        if (!V.hess) Quu[a][a] += w * R.Rw[a] + V.hr[(size_t)a * np + i];
        qu[a] += V.r[(size_t)a * np + i];
    }
#pragma unroll
    for (int a = 0; a < NX; ++a) qx[a] += V.q[(size_t)a * np + i];
    const float h00 = Quu[0][0], h01 = 0.5f * (Quu[0][1] + Quu[1][0]), h11 = Quu[1][1];
    const float det = h00 * h11 - h01 * h01;
    if (!(h00 > 0.f) || !(det > 0.f)) sh.flag = 1;
    const float idet = 1.f / det;
    const float g00 = h11 * idet, g01 = -h01 * idet, g11 = h00 * idet;
    float Kn[NU][NX], kn[NU];
#pragma unroll
    for (int b = 0; b < NX + 1; ++b) {
        const float rhs0 = (b < NX) ? Qux[0][b] : qu[0];
        const float rhs1 = (b < NX) ? Qux[1][b] : qu[1];
        const float s0 = g00 * rhs0 + g01 * rhs1;
        const float s1 = g01 * rhs0 + g11 * rhs1;
        if (b < NX) {
            Kn[0][b] = -s0;
            Kn[1][b] = -s1;
        } else {
            kn[0] = -s0;
            kn[1] = -s1;
        }
    }
    const float hxx = V.hq[i], hxy = V.hq[(size_t)np + i], hyy = V.hq[2 * (size_t)np + i];
#pragma unroll
    for (int a = 0; a < NX; ++a)
#pragma unroll
        for (int b = a; b < NX; ++b) {
            float v = Qxx[a][b] + ((a == b) ? w * R.Qw[a] : 0.f);
            if (a == 0 && b == 0) v += hxx;
            if (a == 0 && b == 1) v += hxy;
            if (a == 1 && b == 1) v += hyy;
            if (V.hess) v = Qxx[a][b] + V.HS[(size_t)sidx<NX>(a, b) * np + i];
#pragma unroll
            for (int t = 0; t < NU; ++t) v += Qux[t][a] * Kn[t][b];
            P[sidx<NX>(a, b)] = v;
            V.P[(size_t)sidx<NX>(a, b) * np + i] = v;
        }
#pragma unroll
    for (int a = 0; a < NX; ++a) {
        float v = qx[a];
#pragma unroll
        for (int t = 0; t < NU; ++t) v += Qux[t][a] * kn[t];
        p[a] = v;
        V.p[(size_t)a * np + i] = v;
    }
#pragma unroll
    for (int a = 0; a < NU; ++a) {
#pragma unroll
        for (int b = 0; b < NX; ++b) V.K[(size_t)(a * NX + b) * np + i] = Kn[a][b];
        V.k[(size_t)a * np + i] = kn[a];
    }
}

/* Riccati step of non-leaf node i from its children's value functions in memory: the sum of Eq.
 * (tree_Riccati) and one step (dynamics per node, or a single child's edge), or the per-edge sum at
 * a node with several children. */
template <int NX, int MODEL>
__device__ __forceinline__ void riccati_from_children(const ProbRec &R, const View<NX> &V, int i, float (&P)[nsym(NX)],
                                                      float (&p)[NX], Shared &sh, bool rec = false) {
    constexpr int NS = nsym(NX);
    const int nch = V.nchild[i], fc = V.fchild[i];
    if constexpr (MODEL == 2) {
        if (V.edge && nch > 1) {
            riccati_edges<NX>(R, V, i, P, p, sh);
            return;
        }
    }
    float Pb[NS], pb[NX];
#pragma unroll
    for (int e = 0; e < NS; ++e) Pb[e] = 0.f;
#pragma unroll
    for (int a = 0; a < NX; ++a) pb[a] = 0.f;
    using F = Frec<NX, MODEL>;
    for (int m = fc; m < fc + nch; ++m)
        add_child_mem<NX, MODEL>(V, m, Pb, pb, rec ? V.FR + (size_t)m * F::stride + F::d : nullptr);
    RicIn<NX> in;
    ric_load<NX, MODEL>(V, i, in, (MODEL == 2 && V.edge) ? fc : i);
    riccati_node<NX, MODEL>(R, V, i, in, Pb, pb, P, p, sh, rec ? V.FR + (size_t)i * F::stride : nullptr);
}

/* Level-synchronous backward sweep: all nodes of a stage in parallel, one barrier per stage. */
template <int NX, int MODEL>
__device__ void backward_level(const ProbRec &R, const View<NX> &V, Shared &sh) {
    constexpr int NS = nsym(NX);
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int st = R.n_stage - 1; st >= 0; --st) {
        const int s0 = V.sstart[st], s1 = V.sstart[st + 1];
        for (int i = s0 + tid; i < s1; i += nt) {
            float P[NS], p[NX];
            if (V.nchild[i] == 0) {
                leaf_value<NX, MODEL>(R, V, i, P, p);
                continue;
            }
            riccati_from_children<NX, MODEL>(R, V, i, P, p, sh);
        }
        __syncthreads();
    }
}

/* Per-scenario-path backward sweep: path s walks up from its leaf through the nodes it owns
 * (the nodes whose first leaf descendant is its leaf), carrying the value function of the
 * child in registers; the block synchronises only before the stages that hold branch nodes,
 * where the children's value functions are summed from memory. */
template <int NX, int MODEL>
__device__ void backward_path(const ProbRec &R, const View<NX> &V, Shared &sh, bool rec = false) {
    using F = Frec<NX, MODEL>;
    constexpr int NS = nsym(NX);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int S = R.n_paths, ns = R.n_stage, nb = R.n_bstage;
    int hi = ns - 1;
    for (int ph = 0; ph <= nb; ++ph) {
        const int lo = (ph < nb) ? V.bstage[ph] : -1;    /* this phase covers stages (lo, hi] */
        for (int s = tid; s < S; s += nt) {
            const int depth = V.pdepth[s], top = V.ptop[s];
            const int khi = min(depth, hi), klo = max(top, lo + 1);
            if (khi < klo) continue;
            const int32_t *path = V.ptab + (size_t)s * ns;
            float P[NS], p[NX];
            int k = khi;
            {
                const int i = path[k];
                const int nch = V.nchild[i];
                if (nch == 0) leaf_value<NX, MODEL>(R, V, i, P, p);
                else riccati_from_children<NX, MODEL>(R, V, i, P, p, sh, rec);
            }
            for (k = khi - 1; k >= klo; --k) {
                const int i = path[k];   /* single child path[k+1], its value function in P, p */
                float dm[NX], Pb[NS], pb[NX];
                RicIn<NX> in;
                ld_rows<NX, MODEL>(V.d, V.np, path[k + 1], dm);
                ric_load<NX, MODEL>(V, i, in, (MODEL == 2 && V.edge) ? path[k + 1] : i);
                if (rec) put_pairs<NX>(V.FR + (size_t)path[k + 1] * F::stride + F::d, dm);
#pragma unroll
                for (int e = 0; e < NS; ++e) Pb[e] = 0.f + P[e];
#pragma unroll
                for (int a = 0; a < NX; ++a) {
                    float v = p[a];
#pragma unroll
                    for (int b = 0; b < NX; ++b) v += P[sidx<NX>(a, b)] * dm[b];
                    pb[a] = 0.f + v;
                }
                riccati_node<NX, MODEL>(R, V, i, in, Pb, pb, P, p, sh, rec ? V.FR + (size_t)i * F::stride : nullptr);
            }

        }
        hi = lo;
        __syncthreads();
    }
}

/* Inputs of the forward step at node i: its defect, the parent's Jacobians and its gains. */
template <int NX>
struct FwdIn {
    float d[NX], A[NX][NX], B[NX][NU], K[NU][NX], k[NU];
};

template <int NX, int MODEL>
__device__ __forceinline__ void fwd_load(const View<NX> &V, int i, int pa, FwdIn<NX> &in) {
    const int np = V.np;
#pragma unroll
    for (int a = 0; a < NX; ++a) {
        in.d[a] = V.d[jrow<NX, MODEL>(np, i, a)];
#pragma unroll
        for (int b = 0; b < NX; ++b) in.A[a][b] = aload<NX, MODEL>(V.A, np, pa, a, b);
#pragma unroll
        for (int b = 0; b < NU; ++b) in.B[a][b] = bload<NX, MODEL>(V.B, np, pa, a, b);
    }
#pragma unroll
    for (int a = 0; a < NU; ++a) {
        in.k[a] = V.k[(size_t)a * np + i];
#pragma unroll
        for (int b = 0; b < NX; ++b) in.K[a][b] = V.K[(size_t)(a * NX + b) * np + i];
    }
}

template <int NX, int MODEL>
__device__ __forceinline__ void fwd_issue(const View<NX> &V, int i, int pa, float *slot, int ld) {
    const int np = V.np;
    int j = 0;
#pragma unroll
    for (int a = 0; a < NX; ++a) {
        cp4(slot + (j++) * ld, V.d + jrow<NX, MODEL>(np, i, a));
#pragma unroll
        for (int b = 0; b < NX; ++b)
            if (a_fixed<MODEL>(a, b) < 0) cp4(slot + (j++) * ld, V.A + jrow<NX * NX, MODEL>(np, pa, a * NX + b));
#pragma unroll
        for (int b = 0; b < NU; ++b)
            if (b_fixed<MODEL>(a, b) < 0) cp4(slot + (j++) * ld, V.B + jrow<NX * NU, MODEL>(np, pa, a * NU + b));
    }
#pragma unroll
    for (int a = 0; a < NU; ++a) {
        cp4(slot + (j++) * ld, V.k + (size_t)a * np + i);
#pragma unroll
        for (int b = 0; b < NX; ++b) cp4(slot + (j++) * ld, V.K + (size_t)(a * NX + b) * np + i);
    }
}

template <int NX, int MODEL>
__device__ __forceinline__ void fwd_read(const float *slot, int ld, FwdIn<NX> &in) {
    int j = 0;
#pragma unroll
    for (int a = 0; a < NX; ++a) {
        in.d[a] = slot[(j++) * ld];
#pragma unroll
        for (int b = 0; b < NX; ++b) in.A[a][b] = a_fixed<MODEL>(a, b) >= 0 ? (float)a_fixed<MODEL>(a, b) : slot[(j++) * ld];
#pragma unroll
        for (int b = 0; b < NU; ++b) in.B[a][b] = b_fixed<MODEL>(a, b) >= 0 ? (float)b_fixed<MODEL>(a, b) : slot[(j++) * ld];
    }
#pragma unroll
    for (int a = 0; a < NU; ++a) {
        in.k[a] = slot[(j++) * ld];
#pragma unroll
        for (int b = 0; b < NX; ++b) in.K[a][b] = slot[(j++) * ld];
    }
}

/* Forward rollout at node i (parent pa, -1 at the root) given the parent's (dx, du):
 * dx_i = A_p dx_p + B_p du_p + d_i, du_i = K_i dx_i + k_i at non-leaves (stored when `own`). */
template <int NX, int MODEL>
__device__ __forceinline__ void forward_node(const View<NX> &V, int i, int pa, bool nonleaf, const FwdIn<NX> &in,
                                             const float (&dxp)[NX], const float (&dup)[NU], float (&dxv)[NX],
                                             float (&duv)[NU], bool own) {
    if (pa < 0) {
#pragma unroll
        for (int j = 0; j < NX; ++j) dxv[j] = 0.f;
    } else {
#pragma unroll
        for (int a = 0; a < NX; ++a) {
            float v = in.d[a];
#pragma unroll
            for (int b = 0; b < NX; ++b) v += in.A[a][b] * dxp[b];
#pragma unroll
            for (int b = 0; b < NU; ++b) v += in.B[a][b] * dup[b];
            dxv[a] = v;
        }
    }
    duv[0] = duv[1] = 0.f;
    if (nonleaf) {
#pragma unroll
        for (int a = 0; a < NU; ++a) {
            float v = in.k[a];
#pragma unroll
            for (int b = 0; b < NX; ++b) v += in.K[a][b] * dxv[b];
            duv[a] = v;
        }
    }
    if (own) {
        st_rows<NX, MODEL>(V.dx, V.np, i, dxv);
        st_rows<NU, MODEL>(V.du, V.np, i, duv);
    }
}

/* After the rollout, every node in parallel: QP multiplier lam_i = P_i dx_i + p_i and the
 * directional terms of the merit (grad'dz, dz'W dz, (dlam - lam)'d). */
template <int NX, int MODEL>
__device__ __forceinline__ void multipliers_and_directions(const ProbRec &R, const View<NX> &V, float (&dir)[3]) {
    const int tid = threadIdx.x, nt = blockDim.x, np = V.np;
    for (int i = tid; i < V.n; i += nt) {
        /* two batches of loads: the direction with the cost and penalty terms, then (after the
         * first merit terms) the value function, multipliers and defect for lam_QP */
        const int nch = V.nchild[i];
        float dxv[NX], duv[NU], qv[NX], rv[NU], hrv[NU];
        ld_rows<NX, MODEL>(V.dx, V.np, i, dxv);
        ld_rows<NU, MODEL>(V.du, V.np, i, duv);
        const float w = V.w[i];
        const float *Qd = nch ? R.Qw : R.QNw;
        const float hxx = V.hq[jrow<3, MODEL>(np, i, 0)], hxy = V.hq[jrow<3, MODEL>(np, i, 1)], hyy = V.hq[jrow<3, MODEL>(np, i, 2)];
        ld_rows<NX, MODEL>(V.q, V.np, i, qv);
        if (nch) {
            ld_rows<NU, MODEL>(V.r, V.np, i, rv);
            ld_rows<NU, MODEL>(V.hr, V.np, i, hrv);
        }
#pragma unroll
        for (int a = 0; a < NX; ++a) dir[0] += qv[a] * dxv[a];
        if (nch) {
#pragma unroll
            for (int a = 0; a < NU; ++a) dir[0] += rv[a] * duv[a];
        }
        if (!V.hess) {
#pragma unroll
            for (int a = 0; a < NX; ++a) dir[1] += w * Qd[a] * dxv[a] * dxv[a];
            dir[1] += hxx * dxv[0] * dxv[0] + 2.f * hxy * dxv[0] * dxv[1] + hyy * dxv[1] * dxv[1];
            if (nch) {
#pragma unroll
                for (int a = 0; a < NU; ++a) dir[1] += (w * R.Rw[a] + hrv[a]) * duv[a] * duv[a];
            }
        } else {   /* dz'W dz with the exact option's dense modified block */
#pragma unroll
            for (int a = 0; a < NX; ++a)
#pragma unroll
                for (int b = 0; b < NX; ++b) dir[1] += dxv[a] * V.HS[(size_t)sidx<NX>(a, b) * np + i] * dxv[b];
            if (nch) {
#pragma unroll
                for (int a = 0; a < NU; ++a) {
#pragma unroll
                    for (int b = 0; b < NX; ++b)
                        dir[1] += 2.f * duv[a] * V.HS[(size_t)(nsym(NX) + a * NX + b) * np + i] * dxv[b];
#pragma unroll
                    for (int b = 0; b < NU; ++b)
                        dir[1] += duv[a] * V.HS[(size_t)(nsym(NX) + NU * NX + a + b) * np + i] * duv[b];
                }
            }
        }
        if (i != 0) {
            float pv[NX], Pv[nsym(NX)], lv[NX], dv[NX], lqv[NX];
#pragma unroll
            for (int a = 0; a < NX; ++a) pv[a] = V.p[jrow<NX, MODEL>(np, i, a)];
#pragma unroll
            for (int e = 0; e < nsym(NX); ++e) Pv[e] = V.P[jrow<nsym(NX), MODEL>(np, i, e)];
            V.load_x(V.L, i, lv);
            ld_rows<NX, MODEL>(V.d, V.np, i, dv);
#pragma unroll
            for (int a = 0; a < NX; ++a) {
                float v = pv[a];
#pragma unroll
                for (int b = 0; b < NX; ++b) v += Pv[sidx<NX>(a, b)] * dxv[b];
                lqv[a] = v;
                const float lam = lv[a];
                dir[2] += ((v - lam) - lam) * dv[a];
            }
            st_rows<NX, MODEL>(V.lq, V.np, i, lqv);
        }
    }
}

/* Level-synchronous forward sweep: one barrier per stage, parents' (dx, du) read from memory. */
template <int NX, int MODEL>
__device__ void forward_level(const ProbRec &R, const View<NX> &V) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int st = 0; st < R.n_stage; ++st) {
        const int s0 = V.sstart[st], s1 = V.sstart[st + 1];
        for (int i = s0 + tid; i < s1; i += nt) {
            float dxp[NX], dup[NU] = {0.f, 0.f}, dxv[NX], duv[NU];
#pragma unroll
            for (int j = 0; j < NX; ++j) dxp[j] = 0.f;
            const int pa = i ? V.parent[i] : -1;
            if (pa >= 0) {
                ld_rows<NX, MODEL>(V.dx, V.np, pa, dxp);
                ld_rows<NU, MODEL>(V.du, V.np, pa, dup);
            }
            FwdIn<NX> in;
            /* Jacobians of the edge into i: the parent's, or i's own with per-edge dynamics */
            fwd_load<NX, MODEL>(V, i, (MODEL == 2 && V.edge) ? i : (pa < 0 ? 0 : pa), in);
            forward_node<NX, MODEL>(V, i, pa, V.nchild[i] != 0, in, dxp, dup, dxv, duv, true);
        }
        __syncthreads();
    }
}

/* Per-scenario-path forward sweep: path s rolls out from the root to its leaf with (dx, du) in
 * registers and no barrier; nodes shared by several paths are recomputed identically by each
 * and written only by their owner path.  The rows of the next nodes are streamed into shared
 * memory ahead of use (cp.async). */
template <int NX, int MODEL>
__device__ void forward_path(const ProbRec &R, const View<NX> &V, float *stg, int ld) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int S = R.n_paths, ns = R.n_stage;
    for (int s = tid; s < S; s += nt) {
        const int32_t *path = V.ptab + (size_t)s * ns;
        const int depth = V.pdepth[s], top = V.ptop[s];
        float dxp[NX], dup[NU] = {0.f, 0.f};
#pragma unroll
        for (int j = 0; j < NX; ++j) dxp[j] = 0.f;
        const int nst = depth + 1;
        float *slot = stg + tid;
        const int bs = rows_stage<NX, MODEL>() * ld;
        if (stg) {
#pragma unroll
            for (int q = 0; q < SWEEP_DEPTH - 1; ++q) {
                if (q < nst)
                    fwd_issue<NX, MODEL>(V, path[q], (MODEL == 2 && V.edge) ? path[q] : (q ? path[q - 1] : 0),
                                         slot + q * bs, ld);
                cp_commit();
            }
        }
        int pa = -1;
        for (int k = 0; k <= depth; ++k) {
            const int i = path[k];
            FwdIn<NX> in;
            if (stg) {
                const int q = k + SWEEP_DEPTH - 1;
                if (q < nst)
                    fwd_issue<NX, MODEL>(V, path[q], (MODEL == 2 && V.edge) ? path[q] : path[q - 1],
                                         slot + (q % SWEEP_DEPTH) * bs, ld);
                cp_commit();
                cp_wait<SWEEP_DEPTH - 1>();
                fwd_read<NX, MODEL>(slot + (k % SWEEP_DEPTH) * bs, ld, in);
            } else {
                fwd_load<NX, MODEL>(V, i, (MODEL == 2 && V.edge) ? i : (pa < 0 ? 0 : pa), in);
            }
            float dxv[NX], duv[NU];
            forward_node<NX, MODEL>(V, i, pa, k < depth, in, dxp, dup, dxv, duv, k >= top);
            pa = i;

#pragma unroll
            for (int j = 0; j < NX; ++j) dxp[j] = dxv[j];
            dup[0] = duv[0];
            dup[1] = duv[1];
        }
    }
    __syncthreads();
}


__device__ __forceinline__ void cp16(float *dst, const float *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

/* The per-path forward sweep on node-major records: stage k of path s copies node path[k + 2]'s
 * record into the thread's ring (four records, 16-byte copies), then takes node i = path[k] from
 * its own record (d_i, K_i, k_i) and its parent's (A, B, read the stage before):
 * dx_i = A_p dx_p + B_p du_p + d_i, du_i = K_i dx_i + k_i.  Thread t's ring lives at
 * stg[t * tstride], 16-byte aligned. */
template <int NX, int MODEL>
__device__ void forward_path_rec(const ProbRec &R, const View<NX> &V, float *stg) {
    using F = Frec<NX, MODEL>;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int S = R.n_paths, ns = R.n_stage;
    float *ring = stg + (size_t)tid * F::tstride;
    for (int s = tid; s < S; s += nt) {
        const int32_t *path = V.ptab + (size_t)s * ns;
        const int depth = V.pdepth[s], top = V.ptop[s];
        const int nst = depth + 1;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (q < nst) {
                const float *src = V.FR + (size_t)path[q] * F::stride;
#pragma unroll
                for (int c = 0; c < F::used / 4; ++c) cp16(ring + q * F::used + 4 * c, src + 4 * c);
            }
            cp_commit();
        }
        float dxp[NX], dup[NU] = {0.f, 0.f};
#pragma unroll
        for (int j = 0; j < NX; ++j) dxp[j] = 0.f;
        for (int k = 0; k <= depth; ++k) {
            const int i = path[k];
            {
                const int q = k + 2;
                if (q < nst) {
                    const float *src = V.FR + (size_t)path[q] * F::stride;
                    float *dst = ring + (q % F::ring) * F::used;
#pragma unroll
                    for (int c = 0; c < F::used / 4; ++c) cp16(dst + 4 * c, src + 4 * c);
                }
                cp_commit();
                cp_wait<2>();
            }
            const float *cur = ring + (k % F::ring) * F::used;
            const float *prv = ring + ((k + F::ring - 1) % F::ring) * F::used;
            float dxv[NX], duv[NU];
            if (k == 0) {
#pragma unroll
                for (int j = 0; j < NX; ++j) dxv[j] = 0.f;
            } else {
                float dv[NX];
#pragma unroll
                for (int j = 0; j < NX / 2; ++j) {
                    const float2 t2 = reinterpret_cast<const float2 *>(cur + F::d)[j];
                    dv[2 * j] = t2.x;
                    dv[2 * j + 1] = t2.y;
                }
                float jv[F::k - F::J];
#pragma unroll
                for (int c = 0; c < (F::k - F::J) / 4; ++c) {
                    const float4 t4 = reinterpret_cast<const float4 *>(prv + F::J)[c];
                    jv[4 * c] = t4.x;
                    jv[4 * c + 1] = t4.y;
                    jv[4 * c + 2] = t4.z;
                    jv[4 * c + 3] = t4.w;
                }
                if constexpr ((F::k - F::J) % 4 == 2) {
                    const float2 t2 = *reinterpret_cast<const float2 *>(prv + F::k - 2);
                    jv[F::k - F::J - 2] = t2.x;
                    jv[F::k - F::J - 1] = t2.y;
                }
#pragma unroll
                for (int a = 0; a < NX; ++a) {
                    float v = dv[a];
#pragma unroll
                    for (int b = 0; b < NX; ++b) {
                        const float ab = a_fixed<MODEL>(a, b) >= 0 ? (float)a_fixed<MODEL>(a, b)
                                                                   : jv[jac_slot<NX, MODEL>(a, b)];
                        v += ab * dxp[b];
                    }
#pragma unroll
                    for (int b = 0; b < NU; ++b) {
                        const float bb = b_fixed<MODEL>(a, b) >= 0 ? (float)b_fixed<MODEL>(a, b)
                                                                   : jv[jac_slot<NX, MODEL>(a, NX + b)];
                        v += bb * dup[b];
                    }
                    dxv[a] = v;
                }
            }
            duv[0] = duv[1] = 0.f;
            if (k < depth) {
                float kv[NU * NX + NU];
#pragma unroll
                for (int c = 0; c < NU * NX / 4; ++c) {
                    const float4 t4 = reinterpret_cast<const float4 *>(cur + F::K)[c];
                    kv[4 * c] = t4.x;
                    kv[4 * c + 1] = t4.y;
                    kv[4 * c + 2] = t4.z;
                    kv[4 * c + 3] = t4.w;
                }
                const float2 t2 = *reinterpret_cast<const float2 *>(cur + F::k);
                kv[NU * NX] = t2.x;
                kv[NU * NX + 1] = t2.y;
#pragma unroll
                for (int a = 0; a < NU; ++a) {
                    float v = kv[NU * NX + a];
#pragma unroll
                    for (int b = 0; b < NX; ++b) v += kv[a * NX + b] * dxv[b];
                    duv[a] = v;
                }
            }
            if (k >= top) {
                st_rows<NX, MODEL>(V.dx, V.np, i, dxv);
                st_rows<NU, MODEL>(V.du, V.np, i, duv);
            }
#pragma unroll
            for (int j = 0; j < NX; ++j) dxp[j] = dxv[j];
            dup[0] = duv[0];
            dup[1] = duv[1];
        }
    }
    __syncthreads();
}

/* ------------------------------------------------------------------ scan sweeps (Sec. III-B) */
/* The tree LQR of Sec. III-B with the sweeps' depth cut from N + 1 dependent steps to a logarithm
 * of it (sweep variant 4).  Backward: along every non-branching segment the value functions come
 * from an inclusive suffix scan of conditional value functions (CVFs, Eq. sol_min) with the
 * combination of Eq. (comb_rule); a node with several children takes the tree Riccati step of
 * Eq. (tree_Riccati) from its children (where the one-step CVF would couple the children, the
 * separable form of Eq. tree_CVF holds only along non-branching segments), and segments are
 * processed wave by wave from the leaves.  Forward: pointer jumping over the closed-loop affine
 * maps dx_m = (A_n + B_n K_n) dx_n + (d_m + B_n k_n) (Eq. forward_comb_rule) on the tree itself, so
 * that every node composes the maps of its ancestors in ceil(log2 depth) rounds. */

/* Row offsets of the fields of a CVF element: V(x_k, x_i) = max_lam 1/2 x_k'P x_k + p'x_k
 * - 1/2 lam'C lam + lam'(x_i - A x_k - c). */
template <int NX>
struct Cvf {
    static constexpr int A = 0, c = NX * NX, C = NX * NX + NX, P = NX * NX + NX + nsym(NX),
                         p = NX * NX + NX + 2 * nsym(NX);
};

/* One-step CVF of node i with the single child m, at position f of buffer S (M = 0 and a diagonal
 * R here): C = B R^-1 B', A~ = A, c~ = d_m - B R^-1 r, P~ = Q, p~ = q. */
template <int NX, int MODEL>
__device__ __forceinline__ void cvf_step(const ProbRec &R, const View<NX> &V, int i, int m, float *S, int f,
                                         Shared &sh) {
    const int np = V.np;
    RicIn<NX> in;
    ric_load<NX, MODEL>(V, i, in);
    float ir[NU];
#pragma unroll
    for (int a = 0; a < NU; ++a) {
        const float h = in.w * R.Rw[a] + in.hr[a];
        if (!(h > 0.f)) sh.flag = 1;
        ir[a] = 1.f / h;
    }
    float dm[NX];
    ld_rows<NX, MODEL>(V.d, V.np, m, dm);
#pragma unroll
    for (int a = 0; a < NX; ++a) {
#pragma unroll
        for (int b = a; b < NX; ++b) {
            float v = 0.f;
#pragma unroll
            for (int t = 0; t < NU; ++t) v += in.B[a][t] * ir[t] * in.B[b][t];
            S[(size_t)(Cvf<NX>::C + sidx<NX>(a, b)) * np + f] = v;
            float qv = (a == b) ? in.w * R.Qw[a] : 0.f;
            if (a == 0 && b == 0) qv += in.hq[0];
            if (a == 0 && b == 1) qv += in.hq[1];
            if (a == 1 && b == 1) qv += in.hq[2];
            S[(size_t)(Cvf<NX>::P + sidx<NX>(a, b)) * np + f] = qv;
        }
#pragma unroll
        for (int b = 0; b < NX; ++b) S[(size_t)(Cvf<NX>::A + a * NX + b) * np + f] = in.A[a][b];
        float cv = dm[a];
#pragma unroll
        for (int t = 0; t < NU; ++t) cv -= in.B[a][t] * ir[t] * in.r[t];
        S[(size_t)(Cvf<NX>::c + a) * np + f] = cv;
        S[(size_t)(Cvf<NX>::p + a) * np + f] = in.q[a];
    }
}

/* The element of a segment's end: the value function 1/2 x'Px + p'x itself (A = C = 0, c = 0). */
template <int NX>
__device__ __forceinline__ void cvf_end(const View<NX> &V, float *S, int f, const float (&P)[nsym(NX)],
                                        const float (&p)[NX]) {
    const int np = V.np;
#pragma unroll
    for (int e = 0; e < NX * NX + NX + nsym(NX); ++e) S[(size_t)e * np + f] = 0.f;
#pragma unroll
    for (int e = 0; e < nsym(NX); ++e) S[(size_t)(Cvf<NX>::P + e) * np + f] = P[e];
#pragma unroll
    for (int a = 0; a < NX; ++a) S[(size_t)(Cvf<NX>::p + a) * np + f] = p[a];
}

template <int NX>
__device__ __forceinline__ void cvf_copy(const View<NX> &V, const float *S, int f, float *O) {
    const int np = V.np;
#pragma unroll
    for (int e = 0; e < cvf_rows(NX); ++e) O[(size_t)e * np + f] = S[(size_t)e * np + f];
}

/* LU factors of an NX x NX matrix with partial pivoting, in registers (indices fixed at compile
 * time; the pivot choice only selects between register values). */
template <int NX>
struct Lu {
    float M[NX][NX], id[NX];
    int piv[NX];
    __device__ __forceinline__ bool factor() {
        bool ok = true;
#pragma unroll
        for (int k = 0; k < NX; ++k) {
            int pr = k;
            float best = fabsf(M[k][k]);
#pragma unroll
            for (int r = k + 1; r < NX; ++r) {
                const float v = fabsf(M[r][k]);
                if (v > best) {
                    best = v;
                    pr = r;
                }
            }
            piv[k] = pr;
#pragma unroll
            for (int r = k + 1; r < NX; ++r)
                if (pr == r) {
#pragma unroll
                    for (int c = 0; c < NX; ++c) {
                        const float t = M[k][c];
                        M[k][c] = M[r][c];
                        M[r][c] = t;
                    }
                }
            ok = ok && best > 0.f && best < INFINITY;
            id[k] = 1.f / M[k][k];
#pragma unroll
            for (int r = k + 1; r < NX; ++r) {
                const float l = M[r][k] * id[k];
                M[r][k] = l;
#pragma unroll
                for (int c = k + 1; c < NX; ++c) M[r][c] -= l * M[k][c];
            }
        }
        return ok;
    }
    /* x <- M^-1 x */
    __device__ __forceinline__ void solve(float (&x)[NX]) const {
#pragma unroll
        for (int k = 0; k < NX; ++k)
#pragma unroll
            for (int r = k + 1; r < NX; ++r)
                if (piv[k] == r) {
                    const float t = x[k];
                    x[k] = x[r];
                    x[r] = t;
                }
#pragma unroll
        for (int r = 1; r < NX; ++r)
#pragma unroll
            for (int c = 0; c < r; ++c) x[r] -= M[r][c] * x[c];
#pragma unroll
        for (int r = NX - 1; r >= 0; --r) {
#pragma unroll
            for (int c = r + 1; c < NX; ++c) x[r] -= M[r][c] * x[c];
            x[r] *= id[r];
        }
    }
    /* x <- M^-T x */
    __device__ __forceinline__ void solve_t(float (&x)[NX]) const {
#pragma unroll
        for (int r = 0; r < NX; ++r) {
#pragma unroll
            for (int c = 0; c < r; ++c) x[r] -= M[c][r] * x[c];
            x[r] *= id[r];
        }
#pragma unroll
        for (int r = NX - 2; r >= 0; --r)
#pragma unroll
            for (int c = r + 1; c < NX; ++c) x[r] -= M[c][r] * x[c];
#pragma unroll
        for (int k = NX - 1; k >= 0; --k)
#pragma unroll
            for (int r = k + 1; r < NX; ++r)
                if (piv[k] == r) {
                    const float t = x[k];
                    x[k] = x[r];
                    x[r] = t;
                }
    }
};

/* The combination of Eq. (comb_rule), e1 at position f1 (from x_k to x_j) followed by e2 at f2
 * (from x_j to x_i), written at position f1 of O; with E = I + C1 P2 and the signs of the CVF form of
 * Eq. (sol_min): A = A2 E^-1 A1, c = A2 E^-1 (c1 - C1 p2) + c2, C = A2 E^-1 C1 A2' + C2,
 * P = A1' E^-T P2 A1 + P1, p = A1' E^-T (p2 + P2 c1) + p1. */
template <int NX>
__device__ void cvf_combine(const View<NX> &V, const float *S, int f1, int f2, float *O, Shared &sh) {
    using F = Cvf<NX>;
    const int np = V.np;
    auto at = [&](int row, int f) { return S[(size_t)row * np + f]; };
    float C1[nsym(NX)], P2[nsym(NX)];
#pragma unroll
    for (int e = 0; e < nsym(NX); ++e) {
        C1[e] = at(F::C + e, f1);
        P2[e] = at(F::P + e, f2);
    }
    Lu<NX> E;
#pragma unroll
    for (int a = 0; a < NX; ++a)
#pragma unroll
        for (int b = 0; b < NX; ++b) {
            float v = (a == b) ? 1.f : 0.f;
#pragma unroll
            for (int t = 0; t < NX; ++t) v += C1[sidx<NX>(a, t)] * P2[sidx<NX>(t, b)];
            E.M[a][b] = v;
        }
    if (!E.factor()) sh.flag = 1;
    {
        float A2[NX][NX];
#pragma unroll
        for (int a = 0; a < NX; ++a)
#pragma unroll
            for (int b = 0; b < NX; ++b) A2[a][b] = at(F::A + a * NX + b, f2);
        /* A = A2 E^-1 A1, column by column */
#pragma unroll
        for (int j = 0; j < NX; ++j) {
            float x[NX];
#pragma unroll
            for (int a = 0; a < NX; ++a) x[a] = at(F::A + a * NX + j, f1);
            E.solve(x);
#pragma unroll
            for (int a = 0; a < NX; ++a) {
                float v = 0.f;
#pragma unroll
                for (int t = 0; t < NX; ++t) v += A2[a][t] * x[t];
                O[(size_t)(F::A + a * NX + j) * np + f1] = v;
            }
        }
        /* C = A2 E^-1 C1 A2' + C2, column j from C1 A2[j, :]' (upper triangle stored) */
#pragma unroll
        for (int j = 0; j < NX; ++j) {
            float x[NX];
#pragma unroll
            for (int a = 0; a < NX; ++a) {
                float v = 0.f;
#pragma unroll
                for (int t = 0; t < NX; ++t) v += C1[sidx<NX>(a, t)] * A2[j][t];
                x[a] = v;
            }
            E.solve(x);
#pragma unroll
            for (int a = 0; a <= j; ++a) {
                float v = at(F::C + sidx<NX>(a, j), f2);
#pragma unroll
                for (int t = 0; t < NX; ++t) v += A2[a][t] * x[t];
                O[(size_t)(F::C + sidx<NX>(a, j)) * np + f1] = v;
            }
        }
        /* c = A2 E^-1 (c1 - C1 p2) + c2 */
        float x[NX];
#pragma unroll
        for (int a = 0; a < NX; ++a) {
            float v = at(F::c + a, f1);
#pragma unroll
            for (int t = 0; t < NX; ++t) v -= C1[sidx<NX>(a, t)] * at(F::p + t, f2);
            x[a] = v;
        }
        E.solve(x);
#pragma unroll
        for (int a = 0; a < NX; ++a) {
            float v = at(F::c + a, f2);
#pragma unroll
            for (int t = 0; t < NX; ++t) v += A2[a][t] * x[t];
            O[(size_t)(F::c + a) * np + f1] = v;
        }
    }
    {
        float A1[NX][NX];
#pragma unroll
        for (int a = 0; a < NX; ++a)
#pragma unroll
            for (int b = 0; b < NX; ++b) A1[a][b] = at(F::A + a * NX + b, f1);
        /* P = A1' E^-T P2 A1 + P1, column j from P2 A1[:, j] (upper triangle stored) */
#pragma unroll
        for (int j = 0; j < NX; ++j) {
            float y[NX];
#pragma unroll
            for (int a = 0; a < NX; ++a) {
                float v = 0.f;
#pragma unroll
                for (int t = 0; t < NX; ++t) v += P2[sidx<NX>(a, t)] * A1[t][j];
                y[a] = v;
            }
            E.solve_t(y);
#pragma unroll
            for (int a = 0; a <= j; ++a) {
                float v = at(F::P + sidx<NX>(a, j), f1);
#pragma unroll
                for (int t = 0; t < NX; ++t) v += A1[t][a] * y[t];
                O[(size_t)(F::P + sidx<NX>(a, j)) * np + f1] = v;
            }
        }
        /* p = A1' E^-T (p2 + P2 c1) + p1 */
        float y[NX];
#pragma unroll
        for (int a = 0; a < NX; ++a) {
            float v = at(F::p + a, f2);
#pragma unroll
            for (int t = 0; t < NX; ++t) v += P2[sidx<NX>(a, t)] * at(F::c + t, f1);
            y[a] = v;
        }
        E.solve_t(y);
#pragma unroll
        for (int a = 0; a < NX; ++a) {
            float v = at(F::p + a, f1);
#pragma unroll
            for (int t = 0; t < NX; ++t) v += A1[t][a] * y[t];
            O[(size_t)(F::p + a) * np + f1] = v;
        }
    }
}

/* Backward sweep by scans (variant 4): wave by wave, the segments' end elements (a leaf's value or
 * a branch node's tree Riccati step), the one-step CVFs of the segment members, the inclusive suffix
 * scan by span doubling (Hillis-Steele), and the members' value functions; then the feedback laws of
 * the single-child nodes from their children's value functions, all nodes at once. */
template <int NX, int MODEL>
__device__ void backward_scan(const ProbRec &R, const View<NX> &V, Shared &sh) {
    constexpr int NS = nsym(NX);
    const int tid = threadIdx.x, nt = blockDim.x, W = R.n_waves, np = V.np;
    for (int w = 0; w < W; ++w) {
        const int f0 = V.wave[w], f1 = V.wave[w + 1], span = V.wave[W + 1 + w];
        for (int f = f0 + tid; f < f1; f += nt) {
            const int i = V.fnode[f];
            if (V.fend[f] == f) {
                float P[NS], p[NX];
                const int nch = V.nchild[i];
                if (nch == 0) {
                    leaf_value<NX, MODEL>(R, V, i, P, p);
                } else {
                    float Pb[NS], pb[NX];
#pragma unroll
                    for (int e = 0; e < NS; ++e) Pb[e] = 0.f;
#pragma unroll
                    for (int a = 0; a < NX; ++a) pb[a] = 0.f;
                    const int fc = V.fchild[i];
                    for (int m = fc; m < fc + nch; ++m) add_child_mem<NX, MODEL>(V, m, Pb, pb);
                    RicIn<NX> in;
                    ric_load<NX, MODEL>(V, i, in);
                    riccati_node<NX, MODEL>(R, V, i, in, Pb, pb, P, p, sh);
                }
                cvf_end<NX>(V, V.CV0, f, P, p);
            } else {
                cvf_step<NX, MODEL>(R, V, i, V.fchild[i], V.CV0, f, sh);
            }
        }
        __syncthreads();
        float *cur = V.CV0, *nxt = V.CV1;
        for (int d = 1; d < span; d *= 2) {
            for (int f = f0 + tid; f < f1; f += nt) {
                if (f + d <= V.fend[f]) cvf_combine<NX>(V, cur, f, f + d, nxt, sh);
                else cvf_copy<NX>(V, cur, f, nxt);
            }
            __syncthreads();
            float *t = cur;
            cur = nxt;
            nxt = t;
        }
        for (int f = f0 + tid; f < f1; f += nt) {
            if (V.fend[f] == f) continue;
            const int i = V.fnode[f];
#pragma unroll
            for (int e = 0; e < NS; ++e) V.P[jrow<NS, MODEL>(np, i, e)] = cur[(size_t)(Cvf<NX>::P + e) * np + f];
#pragma unroll
            for (int a = 0; a < NX; ++a) V.p[jrow<NX, MODEL>(np, i, a)] = cur[(size_t)(Cvf<NX>::p + a) * np + f];
        }
        __syncthreads();
    }
    for (int i = tid; i < V.n; i += nt) {
        if (V.nchild[i] != 1) continue;
        float Pb[NS], pb[NX], P[NS], p[NX];
#pragma unroll
        for (int e = 0; e < NS; ++e) Pb[e] = 0.f;
#pragma unroll
        for (int a = 0; a < NX; ++a) pb[a] = 0.f;
        add_child_mem<NX, MODEL>(V, V.fchild[i], Pb, pb);
        RicIn<NX> in;
        ric_load<NX, MODEL>(V, i, in);
        riccati_node<NX, MODEL, false>(R, V, i, in, Pb, pb, P, p, sh);
    }
}

/* Forward sweep by pointer jumping (variant 4): every non-root node m holds the closed-loop map
 * G_m: dx_a -> dx_m from an ancestor a (first its parent); each round composes G_m with G_a and
 * replaces a by a's ancestor, until every map starts at the root, where dx_0 = 0 and so dx_m = c_m.
 * Then du_n = K_n dx_n + k_n. */
template <int NX, int MODEL>
__device__ void forward_jump(const ProbRec &R, const View<NX> &V) {
    using F = Cvf<NX>;
    const int tid = threadIdx.x, nt = blockDim.x, np = V.np, n = V.n;
    for (int m = 1 + tid; m < n; m += nt) {
        const int a = V.parent[m];
        FwdIn<NX> in;
        fwd_load<NX, MODEL>(V, m, a, in);   /* d_m, A_a, B_a; K, k of m are not used here */
        float Ka[NU][NX], ka[NU];
#pragma unroll
        for (int t = 0; t < NU; ++t) {
            ka[t] = V.k[(size_t)t * np + a];
#pragma unroll
            for (int b = 0; b < NX; ++b) Ka[t][b] = V.K[(size_t)(t * NX + b) * np + a];
        }
#pragma unroll
        for (int r = 0; r < NX; ++r) {
#pragma unroll
            for (int b = 0; b < NX; ++b) {
                float v = in.A[r][b];
#pragma unroll
                for (int t = 0; t < NU; ++t) v += in.B[r][t] * Ka[t][b];
                V.CV0[(size_t)(F::A + r * NX + b) * np + m] = v;
            }
            float v = in.d[r];
#pragma unroll
            for (int t = 0; t < NU; ++t) v += in.B[r][t] * ka[t];
            V.CV0[(size_t)(F::c + r) * np + m] = v;
        }
        V.JA0[m] = __int_as_float(a);
    }
    __syncthreads();
    float *cur = V.CV0, *nxt = V.CV1, *jc = V.JA0, *jn = V.JA1;
    for (int span = 1; span < R.n_stage; span *= 2) {
        for (int m = 1 + tid; m < n; m += nt) {
            const int a = __float_as_int(jc[m]);
            if (a == 0) {
#pragma unroll
                for (int e = 0; e < NX * NX + NX; ++e) nxt[(size_t)e * np + m] = cur[(size_t)e * np + m];
                jn[m] = jc[m];
                continue;
            }
            float Am[NX][NX], cm[NX], Aa[NX][NX], ca[NX];
#pragma unroll
            for (int r = 0; r < NX; ++r) {
#pragma unroll
                for (int b = 0; b < NX; ++b) {
                    Am[r][b] = cur[(size_t)(F::A + r * NX + b) * np + m];
                    Aa[r][b] = cur[(size_t)(F::A + r * NX + b) * np + a];
                }
                cm[r] = cur[(size_t)(F::c + r) * np + m];
                ca[r] = cur[(size_t)(F::c + r) * np + a];
            }
#pragma unroll
            for (int r = 0; r < NX; ++r) {
#pragma unroll
                for (int b = 0; b < NX; ++b) {
                    float v = 0.f;
#pragma unroll
                    for (int t = 0; t < NX; ++t) v += Am[r][t] * Aa[t][b];
                    nxt[(size_t)(F::A + r * NX + b) * np + m] = v;
                }
                float v = cm[r];
#pragma unroll
                for (int t = 0; t < NX; ++t) v += Am[r][t] * ca[t];
                nxt[(size_t)(F::c + r) * np + m] = v;
            }
            jn[m] = jc[a];
        }
        __syncthreads();
        float *t = cur;
        cur = nxt;
        nxt = t;
        t = jc;
        jc = jn;
        jn = t;
    }
    for (int i = tid; i < n; i += nt) {
        float dxv[NX], du0 = 0.f, du1 = 0.f;
#pragma unroll
        for (int r = 0; r < NX; ++r) dxv[r] = i ? cur[(size_t)(F::c + r) * np + i] : 0.f;
        st_rows<NX, MODEL>(V.dx, V.np, i, dxv);
        if (V.nchild[i]) {
            du0 = V.k[i];
            du1 = V.k[(size_t)np + i];
#pragma unroll
            for (int b = 0; b < NX; ++b) {
                du0 += V.K[(size_t)b * np + i] * dxv[b];
                du1 += V.K[(size_t)(NX + b) * np + i] * dxv[b];
            }
        }
        V.du[jrow<NU, MODEL>(np, i, 0)] = du0;
        V.du[jrow<NU, MODEL>(np, i, 1)] = du1;
    }
}

/* ------------------------------------------------------------------ cooperative (8-lane) per-path sweeps */
/* A group of GL lanes handles one root-to-leaf path.  In the backward step lane j owns column j of
 * F = [A_n B_n], of the summed child value-function Hessian Pbar, of H = W + F' Pbar F and of the
 * new P; the gradient-side vectors (pbar, p) are replicated.  Rows of Pbar F are written to a small
 * shared tile and read back as columns; the u-block of H and its coupling columns are broadcast
 * with 8-lane shuffles.  The arithmetic is that of riccati_node (Eq. tree_feedback_laws). */
__device__ __forceinline__ float gshfl(float v, int src, unsigned mask) { return __shfl_sync(mask, v, src, GL); }

template <int NX, int MODEL>
__device__ __forceinline__ void coop_riccati(const ProbRec &R, const View<NX> &V, int i, const float (&Pbc)[NX],
                                             const float (&pb)[NX], float (&Pc)[NX], float (&p)[NX], int lane,
                                             unsigned gmask, float (*tr)[8], Shared &sh) {
    constexpr int NZ = NX + NU;
    const int np = V.np;
    const float w = V.w[i];
    float F[NX][NZ];
#pragma unroll
    for (int a = 0; a < NX; ++a) {
#pragma unroll
        for (int b = 0; b < NX; ++b) F[a][b] = aload<NX, MODEL>(V.A, np, i, a, b);
#pragma unroll
        for (int b = 0; b < NU; ++b) F[a][NX + b] = bload<NX, MODEL>(V.B, np, i, a, b);
    }
    /* row `lane` of Pbar F (Pbar symmetric: this lane's column is also its row) */
    if (lane < NX) {
#pragma unroll
        for (int c = 0; c < NZ; ++c) {
            float v = 0.f;
#pragma unroll
            for (int t = 0; t < NX; ++t) v += Pbc[t] * F[t][c];
            tr[lane][c] = v;
        }
    }
    __syncwarp(gmask);
    /* column `lane` of H = W + F' Pbar F and entry `lane` of g = [q; r] + F' pbar */
    float Hc[NZ], g = 0.f;
#pragma unroll
    for (int a = 0; a < NZ; ++a) Hc[a] = 0.f;
    if (lane < NZ) {
        float PFc[NX], Fc[NX];
#pragma unroll
        for (int t = 0; t < NX; ++t) {
            PFc[t] = tr[t][lane];
            Fc[t] = 0.f;
#pragma unroll
            for (int c = 0; c < NZ; ++c)
                if (c == lane) Fc[t] = F[t][c];
        }
#pragma unroll
        for (int a = 0; a < NZ; ++a) {
            float v = 0.f;
#pragma unroll
            for (int t = 0; t < NX; ++t) v += F[t][a] * PFc[t];
            Hc[a] = v;
        }
        const float hxx = V.hq[jrow<3, MODEL>(np, i, 0)], hxy = V.hq[jrow<3, MODEL>(np, i, 1)], hyy = V.hq[jrow<3, MODEL>(np, i, 2)];
#pragma unroll
        for (int a = 0; a < NZ; ++a) {
            if (a != lane) continue;
            if (a < NX) Hc[a] += w * R.Qw[a];
            else Hc[a] += w * R.Rw[a - NX] + V.hr[jrow<NU, MODEL>(np, i, a - NX)];
        }
        if (lane == 0) {
            Hc[0] += hxx;
            Hc[1] += hxy;
        } else if (lane == 1) {
            Hc[0] += hxy;
            Hc[1] += hyy;
        }
        g = lane < NX ? V.q[jrow<NX, MODEL>(np, i, lane)] : V.r[jrow<NU, MODEL>(np, i, lane - NX)];
#pragma unroll
        for (int t = 0; t < NX; ++t) g += Fc[t] * pb[t];
    }
    __syncwarp(gmask);
    /* 2x2 H_uu, g_u and the coupling columns H[:, nx], H[:, nx+1] to every lane */
    const float h00 = gshfl(Hc[NX], NX, gmask), h10 = gshfl(Hc[NX + 1], NX, gmask);
    const float h11 = gshfl(Hc[NX + 1], NX + 1, gmask);
    const float gu0 = gshfl(g, NX, gmask), gu1 = gshfl(g, NX + 1, gmask);
    float Hu0[NX], Hu1[NX], gx[NX];
#pragma unroll
    for (int a = 0; a < NX; ++a) {
        Hu0[a] = gshfl(Hc[a], NX, gmask);
        Hu1[a] = gshfl(Hc[a], NX + 1, gmask);
        gx[a] = gshfl(g, a, gmask);
    }
    /* K column `lane` and k: -H_uu^-1 (Qux column, qu), closed-form 2x2 inverse as in riccati_node */
    const float det = h00 * h11 - h10 * h10;
    if (!(h00 > 0.f) || !(det > 0.f)) sh.flag = 1;
    const float idet = 1.f / det;   /* IEEE-rounded: the direction's accuracy sets the FP32 KKT floor */
    const float g00 = h11 * idet, g01 = -h10 * idet, g11 = h00 * idet;
    const float K0 = -(g00 * Hc[NX] + g01 * Hc[NX + 1]);
    const float K1 = -(g01 * Hc[NX] + g11 * Hc[NX + 1]);
    const float k0 = -(g00 * gu0 + g01 * gu1);
    const float k1 = -(g01 * gu0 + g11 * gu1);
    /* new P column `lane` = H[0:nx, lane] + Qux' K[:, lane]; p = qx + Qux' k (replicated) */
#pragma unroll
    for (int a = 0; a < NX; ++a) {
        Pc[a] = Hc[a] + Hu0[a] * K0 + Hu1[a] * K1;
        p[a] = gx[a] + Hu0[a] * k0 + Hu1[a] * k1;
    }
    if (lane < NX) {
#pragma unroll
        for (int a = 0; a < NX; ++a)
            if (a <= lane) V.P[jrow<nsym(NX), MODEL>(np, i, sidx<NX>(a, lane))] = Pc[a];
        V.K[(size_t)lane * np + i] = K0;
        V.K[(size_t)(NX + lane) * np + i] = K1;
    } else if (lane == NX) {
#pragma unroll
        for (int a = 0; a < NX; ++a) V.p[jrow<NX, MODEL>(np, i, a)] = p[a];
        V.k[i] = k0;
        V.k[(size_t)np + i] = k1;
    }
}

/* pbar = p + P d (P distributed by columns over the lanes, p replicated): returns pbar replicated. */
template <int NX, int MODEL>
__device__ __forceinline__ void coop_pbar(const View<NX> &V, int c, const float (&Pc)[NX], const float (&p)[NX],
                                          float (&pb)[NX], int lane, unsigned gmask) {
    float dm[NX];
    ld_rows<NX, MODEL>(V.d, V.np, c, dm);
    float v = 0.f;
#pragma unroll
    for (int t = 0; t < NX; ++t) v += Pc[t] * dm[t];
#pragma unroll
    for (int a = 0; a < NX; ++a) pb[a] = p[a] + gshfl(v, a, gmask);
}

template <int NX, int MODEL>
__device__ void backward_coop(const ProbRec &R, const View<NX> &V, Shared &sh) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & (GL - 1), grp = tid / GL, ngrp = nt / GL;
    const unsigned gmask = 0xFFu << (tid & 31 & ~(GL - 1));
    float(*tr)[8] = sh.tr[grp];
    const int S = R.n_paths, ns = R.n_stage, nb = R.n_bstage;
    const int np = V.np;
    int hi = ns - 1;
    for (int ph = 0; ph <= nb; ++ph) {
        const int lo = (ph < nb) ? V.bstage[ph] : -1;
        for (int s = grp; s < S; s += ngrp) {
            const int depth = V.pdepth[s], top = V.ptop[s];
            const int khi = min(depth, hi), klo = max(top, lo + 1);
            if (khi < klo) continue;
            const int32_t *path = V.ptab + (size_t)s * ns;
            float Pc[NX], p[NX];
            {
                const int i = path[khi];
                const int nch = V.nchild[i];
                const int lc = min(lane, NX - 1);
                if (nch == 0) {
                    /* terminal value function of the leaf, column `lane` */
                    const float w = V.w[i];
#pragma unroll
                    for (int a = 0; a < NX; ++a) Pc[a] = (a == lc) ? w * R.QNw[a] : 0.f;
                    const float hxx = V.hq[jrow<3, MODEL>(np, i, 0)], hxy = V.hq[jrow<3, MODEL>(np, i, 1)], hyy = V.hq[jrow<3, MODEL>(np, i, 2)];
                    if (lc == 0) {
                        Pc[0] += hxx;
                        Pc[1] += hxy;
                    } else if (lc == 1) {
                        Pc[0] += hxy;
                        Pc[1] += hyy;
                    }
                    ld_rows<NX, MODEL>(V.q, V.np, i, p);
                    if (lane < NX) {
#pragma unroll
                        for (int a = 0; a < NX; ++a)
                            if (a <= lane) V.P[jrow<nsym(NX), MODEL>(np, i, sidx<NX>(a, lane))] = Pc[a];
                    } else if (lane == NX) {
#pragma unroll
                        for (int a = 0; a < NX; ++a) V.p[jrow<NX, MODEL>(np, i, a)] = p[a];
                    }
                } else {
                    /* children summed from memory: column `lane` of Pbar, pbar replicated */
                    float Pbc[NX], pb[NX];
                    float v = 0.f;
#pragma unroll
                    for (int a = 0; a < NX; ++a) {
                        Pbc[a] = 0.f;
                        pb[a] = 0.f;
                    }
                    const int fc = V.fchild[i];
                    for (int m = fc; m < fc + nch; ++m) {
                        float dm[NX];
                        ld_rows<NX, MODEL>(V.d, V.np, m, dm);
                        float vm = V.p[jrow<NX, MODEL>(np, m, lc)];
#pragma unroll
                        for (int a = 0; a < NX; ++a) {
                            const float Pa = V.P[jrow<nsym(NX), MODEL>(np, m, sidx<NX>(a, lc))];
                            Pbc[a] += Pa;
                            vm += Pa * dm[a];
                        }
                        v += vm;
                    }
#pragma unroll
                    for (int a = 0; a < NX; ++a) pb[a] = gshfl(v, a, gmask);
                    coop_riccati<NX, MODEL>(R, V, i, Pbc, pb, Pc, p, lane, gmask, tr, sh);
                }
            }
            for (int k = khi - 1; k >= klo; --k) {
                const int i = path[k], c = path[k + 1];
                float pb[NX];
                coop_pbar<NX, MODEL>(V, c, Pc, p, pb, lane, gmask);
                float Pbc[NX];
#pragma unroll
                for (int a = 0; a < NX; ++a) Pbc[a] = Pc[a];
                coop_riccati<NX, MODEL>(R, V, i, Pbc, pb, Pc, p, lane, gmask, tr, sh);
            }
        }
        hi = lo;
        __syncthreads();
    }
}

/* Cooperative forward rollout: lane a < nx computes dx[a], lanes 0..nu-1 compute du; the vectors
 * are replicated by 8-lane shuffles. */
template <int NX, int MODEL>
__device__ void forward_coop(const ProbRec &R, const View<NX> &V) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & (GL - 1), grp = tid / GL, ngrp = nt / GL;
    const unsigned gmask = 0xFFu << (tid & 31 & ~(GL - 1));
    const int S = R.n_paths, ns = R.n_stage, np = V.np;
    const int la = min(lane, NX - 1), lu = min(lane, NU - 1);
    for (int s = grp; s < S; s += ngrp) {
        const int32_t *path = V.ptab + (size_t)s * ns;
        const int depth = V.pdepth[s], top = V.ptop[s];
        float dx[NX], du[NU] = {0.f, 0.f};
#pragma unroll
        for (int j = 0; j < NX; ++j) dx[j] = 0.f;
        for (int k = 0; k <= depth; ++k) {
            const int i = path[k];
            if (i != 0) {
                const int pa = path[k - 1];
                float v = V.d[jrow<NX, MODEL>(np, i, la)];
#pragma unroll
                for (int b = 0; b < NX; ++b) v += aload<NX, MODEL>(V.A, np, pa, la, b) * dx[b];
#pragma unroll
                for (int b = 0; b < NU; ++b) v += bload<NX, MODEL>(V.B, np, pa, la, b) * du[b];
#pragma unroll
                for (int a = 0; a < NX; ++a) dx[a] = gshfl(v, a, gmask);
            }
            if (V.nchild[i]) {
                float v = V.k[(size_t)lu * np + i];
#pragma unroll
                for (int b = 0; b < NX; ++b) v += V.K[(size_t)(lu * NX + b) * np + i] * dx[b];
                du[0] = gshfl(v, 0, gmask);
                du[1] = gshfl(v, 1, gmask);
            } else {
                du[0] = du[1] = 0.f;
            }
            if (k >= top) {
                if (lane < NX) {
#pragma unroll
                    for (int a = 0; a < NX; ++a)
                        if (a == lane) V.dx[jrow<NX, MODEL>(np, i, a)] = dx[a];
                } else if (lane < NX + NU) {
#pragma unroll
                    for (int a = 0; a < NU; ++a)
                        if (a == lane - NX) V.du[jrow<NU, MODEL>(np, i, a)] = du[a];
                }
            }
        }
    }
    __syncthreads();
}

/* ------------------------------------------------------------------ starting points */
/* Fill the iterate (state deviation, u, lam, y) from start `which`: 0 the cold start of Sec. V-B
 * (x linearly interpolated from x0 to the final reference of the node's first leaf, u = lam = y
 * = 0), 1 warm-start slot 0, 2 warm-start slot 1.  The root state is x0 and its lam is zero. */
template <int NX>
__device__ void load_start(const ProbRec &R, View<NX> &V, int which) {
    const int tid = threadIdx.x, nt = blockDim.x, np = V.np, nc = V.nc;
    if (which > 0) V.set_slot(which - 1);
    for (int i = tid; i < V.n; i += nt) {
        const bool is_leaf = V.nchild[i] == 0;
        float x[NX], u[NU], l[NX];
        if (which > 0) {
            V.load_x(V.wx, i, x);
            V.load_u(V.wu, i, u);
            V.load_x(V.wl, i, l);
            for (int c = 0; c < nc; ++c) V.Y[(size_t)c * np + i] = V.wy[(size_t)c * np + i];
        } else {
            const int lf = V.leaf[i];
            const float s = V.stage[lf] > 0 ? (float)V.stage[i] * rcp((float)V.stage[lf]) : 0.f;
#pragma unroll
            for (int j = 0; j < NX; ++j) x[j] = R.x0[j] + s * (V.xref[(size_t)j * np + lf] - R.x0[j]);
            u[0] = u[1] = 0.f;
#pragma unroll
            for (int j = 0; j < NX; ++j) l[j] = 0.f;
            for (int c = 0; c < nc; ++c) V.Y[(size_t)c * np + i] = 0.f;
        }
        if (i == 0) {
#pragma unroll
            for (int j = 0; j < NX; ++j) {
                x[j] = R.x0[j];
                l[j] = 0.f;
            }
        }
        if (is_leaf) u[0] = u[1] = 0.f;
        Lo lo;
#pragma unroll
        for (int j = 0; j < NX; ++j) {   /* deviation coordinates; the positions keep the remainder */
            float e;
            x[j] = two_sum(x[j], -V.xref[(size_t)j * np + i], e);
            if (j < 2) lo.x[j] = e;
        }
        lo.u[0] = lo.u[1] = 0.f;
        V.store_x(V.X, i, x);
        V.store_u(V.U, i, u);
        V.store_x(V.L, i, l);
        V.store_lo(i, lo);
    }
}

/* Merit phi = L_a + lam'd + mu/2 |d|^2 (Eq. merit with J = L_a) at the current iterate. */
template <int NX, int MODEL>
__device__ float start_merit(const ProbRec &R, const View<NX> &V, float rho, float mu, Shared &sh) {
    const int tid = threadIdx.x, nt = blockDim.x, np = V.np;
    float acc[1] = {0.f};
    for (int i = tid; i < V.n; i += nt) {
        const int nch = V.nchild[i], fc = V.fchild[i];
        float x[NX], u[NU], qd[NX], rd[NU], hqd[3], hrd[NU];
        Lo lo;
        V.load_x(V.X, i, x);
        V.load_u(V.U, i, u);
        V.load_lo(i, lo);
        float v = node_la<NX, false>(R, V, i, nch == 0, x, u, lo, rho, qd, rd, hqd, hrd);
        if (nch) {
            float xa[NX], ft[NX];
#pragma unroll
            for (int j = 0; j < NX; ++j) xa[j] = V.xref[(size_t)j * np + i] + x[j];
            const bool per_edge = MODEL == 2 && V.edge;
            if (!per_edge) dyn<NX, MODEL>(R, xa, u, ft);
            for (int m = fc; m < fc + nch; ++m) {
                if constexpr (MODEL == 2) {
                    if (per_edge) edge_increment<NX>(V, m, xa, u, ft);
                }
#pragma unroll
                for (int j = 0; j < NX; ++j) {
                    const float dref = V.xref[(size_t)j * np + i] - V.xref[(size_t)j * np + m];
                    const float dm = (dref + (x[j] - V.X[(size_t)j * np + m])) + ft[j];
                    v += V.L[(size_t)j * np + m] * dm + 0.5f * mu * dm * dm;
                }
            }
        }
        acc[0] += v;
    }
    block_sum<1>(acc, sh);
    return acc[0];
}

/* The accepted step at node i: x += a dx, u += a du (in registers, caller stores) and, except at
 * the root, lam += a (lam_QP - lam) in memory (Algorithm 1, update after the line search). */
template <int NX, int MODEL>
__device__ __forceinline__ void apply_step(const View<NX> &V, int i, float a, float (&x)[NX], float (&u)[NU],
                                           float (&lam)[NX], Lo &lo) {
    /* every row is loaded before anything is computed or stored, so the loads go out together;
     * the caller stores x, u and (for i != 0) lam after the rest of its node work */
    float dxv[NX], duv[NU], lmv[NX], lqv[NX];
    ld_rows<NX, MODEL>(V.dx, V.np, i, dxv);
    ld_rows<NU, MODEL>(V.du, V.np, i, duv);
    if (i != 0) {
        V.load_x(V.L, i, lmv);
        ld_rows<NX, MODEL>(V.lq, V.np, i, lqv);
    }
    if (V.comp) {
        comp_add(x[0], lo.x[0], a * dxv[0]);
        comp_add(x[1], lo.x[1], a * dxv[1]);
#pragma unroll
        for (int j = 2; j < NX; ++j) x[j] += a * dxv[j];
#pragma unroll
        for (int j = 0; j < NU; ++j) comp_add(u[j], lo.u[j], a * duv[j]);
    } else {
#pragma unroll
        for (int j = 0; j < NX; ++j) x[j] += a * dxv[j];
#pragma unroll
        for (int j = 0; j < NU; ++j) u[j] += a * duv[j];
    }
    if (i != 0) {
#pragma unroll
        for (int j = 0; j < NX; ++j) lam[j] = lmv[j] + a * (lqv[j] - lmv[j]);
    }
}

/* The same step row by row, storing lam_i as it goes (the register-lean form; see hoist_loads). */
template <int NX, int MODEL>
__device__ __forceinline__ void apply_step_serial(const View<NX> &V, int i, float a, float (&x)[NX], float (&u)[NU],
                                                  Lo &lo) {
    const int np = V.np;
#pragma unroll
    for (int j = 0; j < NX; ++j) {
        const float t = a * V.dx[jrow<NX, MODEL>(np, i, j)];
        if (j < 2 && V.comp) comp_add(x[j], lo.x[j], t);
        else x[j] += t;
        if (i != 0) {
            const float lm = V.L[(size_t)j * np + i];
            V.L[(size_t)j * np + i] = lm + a * (V.lq[jrow<NX, MODEL>(np, i, j)] - lm);
        }
    }
#pragma unroll
    for (int j = 0; j < NU; ++j) {
        const float t = a * V.du[jrow<NU, MODEL>(np, i, j)];
        if (V.comp) comp_add(u[j], lo.u[j], t);
        else u[j] += t;
    }
}

/* ------------------------------------------------------------------ exact Hessian option (Sec. IV-A) */
/* Hyper-dual numbers (Fike and Alonso, 2011): a + b e1 + c e2 + d e1 e2 with e1^2 = e2^2 = 0; a
 * function evaluated at z + e1 v + e2 w returns w'H v in d exactly, without truncation error. */
struct Hd {
    float a, b, c, d;
};
__device__ __forceinline__ Hd hd_c(float v) { return Hd{v, 0.f, 0.f, 0.f}; }
__device__ __forceinline__ Hd operator+(Hd x, Hd y) { return Hd{x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d}; }
__device__ __forceinline__ Hd operator-(Hd x, Hd y) { return Hd{x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d}; }
__device__ __forceinline__ Hd operator*(Hd x, float s) { return Hd{x.a * s, x.b * s, x.c * s, x.d * s}; }
__device__ __forceinline__ Hd operator*(Hd x, Hd y) {
    return Hd{x.a * y.a, x.a * y.b + x.b * y.a, x.a * y.c + x.c * y.a, x.a * y.d + x.b * y.c + x.c * y.b + x.d * y.a};
}
/* f(x) from its value f0 and first and second derivatives f1, f2 at x.a */
__device__ __forceinline__ Hd hd_fn(Hd x, float f0, float f1, float f2) {
    return Hd{f0, f1 * x.b, f1 * x.c, f1 * x.d + f2 * x.b * x.c};
}
__device__ __forceinline__ void hd_sincos(Hd x, Hd &s, Hd &c) {
    float sv, cv;
    sincos_cw(x.a, &sv, &cv);
    s = hd_fn(x, sv, cv, -sv);
    c = hd_fn(x, cv, -sv, -cv);
}
__device__ __forceinline__ Hd hd_inv(Hd x) {
    const float i = 1.f / x.a;
    return hd_fn(x, i, -i * i, 2.f * i * i * i);
}
__device__ __forceinline__ Hd hd_atan(Hd x) {
    const float s = 1.f / (1.f + x.a * x.a);
    return hd_fn(x, atanf(x.a), s, -2.f * x.a * s * s);
}
__device__ __forceinline__ Hd hd_sqrt(Hd x) {
    const float r = sqrtf(x.a);
    return hd_fn(x, r, 0.5f / r, -0.25f / (r * x.a));
}

/* The vehicle right-hand sides of rhs() in hyper-dual arithmetic. */
template <int NX, int MODEL>
__device__ __forceinline__ void rhs_hd(const float *prm, const Hd (&s)[NX], const Hd (&u)[NU], Hd (&f)[NX]) {
    if constexpr (MODEL == 0 || MODEL == 3) {
        Hd sp, cp;
        hd_sincos(s[2], sp, cp);
        f[0] = s[3] * cp;
        f[1] = s[3] * sp;
        if constexpr (MODEL == 0) {
            Hd sd, cd;
            hd_sincos(u[1], sd, cd);
            f[2] = s[3] * (sd * hd_inv(cd)) * (1.f / prm[0]);
        } else {
            f[2] = u[1];
        }
        f[3] = u[0];
    } else if constexpr (MODEL == 1) {
        const float lf = prm[3], lr = prm[4], Cf = prm[5], Cr = prm[6], vmin = prm[7], veps = prm[8];
        const Hd vx = s[3], vy = s[4], r = s[5];
        const Hd dv = vx - hd_c(vmin);
        const Hd w = hd_sqrt(dv * dv + hd_c(veps * veps));
        const Hd ivb = hd_inv((vx + hd_c(vmin) + w) * 0.5f);
        const Hd Ff = (hd_atan((vy + r * lf) * ivb) - u[1]) * (-Cf);
        const Hd Fr = hd_atan((vy - r * lr) * ivb) * (-Cr);
        Hd sp, cp;
        hd_sincos(s[2], sp, cp);
        f[0] = vx * cp - vy * sp;
        f[1] = vx * sp + vy * cp;
        f[2] = r;
        f[3] = u[0] + r * vy;
        f[4] = (Ff + Fr) * (1.f / prm[1]) - r * vx;
        f[5] = (Ff * lf - Fr * lr) * (1.f / prm[2]);
    }
}

/* H = sum_i mu_i d^2 f_i / dz dz, z = (x, u), of the RK4 map (n_sub substeps) at absolute state xa,
 * one hyper-dual evaluation per pair (j, k); the positions X, Y do not enter the vehicle dynamics,
 * so their rows and columns are zero and skipped.  The linear model has none. */
template <int NX, int MODEL>
__device__ __forceinline__ void dyn_hessian(const ProbRec &R, const float (&xa)[NX], const float (&u)[NU],
                                            const float (&mu)[NX], float (&H)[NX + NU][NX + NU]) {
    constexpr int NZ = NX + NU;
#pragma unroll
    for (int j = 0; j < NZ; ++j)
#pragma unroll
        for (int k = 0; k < NZ; ++k) H[j][k] = 0.f;
    if constexpr (MODEL == 2) {
        return;
    } else {
        const int nsub = max(1, (int)R.params[9]);
        const float h = R.dt / (float)nsub;
        for (int j = 2; j < NZ; ++j)
            for (int k = j; k < NZ; ++k) {
                Hd z[NX], uu[NU];
#pragma unroll
                for (int i = 0; i < NX; ++i) z[i] = Hd{xa[i], i == j ? 1.f : 0.f, i == k ? 1.f : 0.f, 0.f};
#pragma unroll
                for (int i = 0; i < NU; ++i) uu[i] = Hd{u[i], NX + i == j ? 1.f : 0.f, NX + i == k ? 1.f : 0.f, 0.f};
                for (int sub = 0; sub < nsub; ++sub) {
                    Hd kp[NX], ks[NX];
#pragma unroll
                    for (int i = 0; i < NX; ++i) kp[i] = ks[i] = hd_c(0.f);
#pragma unroll
                    for (int st = 0; st < 4; ++st) {
                        const float c = (st == 0) ? 0.f : (st == 3 ? 1.f : 0.5f);
                        const float wg = (st == 0 || st == 3) ? 1.f : 2.f;
                        Hd zs[NX], kk[NX];
#pragma unroll
                        for (int i = 0; i < NX; ++i) zs[i] = z[i] + kp[i] * (c * h);
                        rhs_hd<NX, MODEL>(R.params, zs, uu, kk);
#pragma unroll
                        for (int i = 0; i < NX; ++i) {
                            ks[i] = ks[i] + kk[i] * wg;
                            kp[i] = kk[i];
                        }
                    }
#pragma unroll
                    for (int i = 0; i < NX; ++i) z[i] = z[i] + ks[i] * (h * (1.f / 6.f));
                }
                float v = 0.f;
#pragma unroll
                for (int i = 0; i < NX; ++i) v += mu[i] * z[i].d;
                H[j][k] = v;
                H[k][j] = v;
            }
    }
}

/* Eigenvalue modification of a symmetric n x n block (Nocedal and Wright, Sec. 3.4): eigenvalues
 * floored at delta = EIG_FLOOR max(1, max |ev|).  When a Cholesky factorisation of S - dF I
 * succeeds with dF = EIG_FLOOR max(1, |S|_F) >= delta, every eigenvalue already exceeds the floor
 * and S is kept; otherwise cyclic Jacobi sweeps (Golub and Van Loan, Sec. 8.5) decompose it. */
constexpr float EIG_FLOOR = 1e-6f;
template <int N>
__device__ __forceinline__ void eig_modify(float (&S)[N][N]) {
    float fro = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) fro += S[i][j] * S[i][j];
    const float dF = EIG_FLOOR * fmaxf(1.f, sqrtf(fro));
    {
        float L[N][N];
        bool pd = true;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            float s = S[j][j] - dF;
#pragma unroll
            for (int t = 0; t < j; ++t) s -= L[j][t] * L[j][t];
            pd = pd && s > 0.f;
            const float ljj = sqrtf(fmaxf(s, 1e-30f)), il = 1.f / ljj;
            L[j][j] = ljj;
#pragma unroll
            for (int i = j + 1; i < N; ++i) {
                float v = S[i][j];
#pragma unroll
                for (int t = 0; t < j; ++t) v -= L[i][t] * L[j][t];
                L[i][j] = v * il;
            }
        }
        if (pd) return;
    }
    float Vm[N][N];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) Vm[i][j] = i == j ? 1.f : 0.f;
    for (int sweep = 0; sweep < 12; ++sweep) {
        float off = 0.f;
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j)
                if (i != j) off += S[i][j] * S[i][j];
        if (!(off > 1e-14f * fro)) break;
#pragma unroll
        for (int p = 0; p < N - 1; ++p)
#pragma unroll
            for (int q = p + 1; q < N; ++q) {
                const float apq = S[p][q];
                if (apq == 0.f) continue;
                const float theta = (S[q][q] - S[p][p]) / (2.f * apq);
                const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
                const float c = rsqrtf(t * t + 1.f), s = t * c;
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const float akp = S[k][p], akq = S[k][q];
                    S[k][p] = c * akp - s * akq;
                    S[k][q] = s * akp + c * akq;
                }
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const float apk = S[p][k], aqk = S[q][k];
                    S[p][k] = c * apk - s * aqk;
                    S[q][k] = s * apk + c * aqk;
                }
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const float vkp = Vm[k][p], vkq = Vm[k][q];
                    Vm[k][p] = c * vkp - s * vkq;
                    Vm[k][q] = s * vkp + c * vkq;
                }
            }
    }
    float ev[N], emax = 1.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        ev[i] = S[i][i];
        emax = fmaxf(emax, fabsf(ev[i]));
    }
    const float delta = EIG_FLOOR * emax;
#pragma unroll
    for (int i = 0; i < N; ++i) ev[i] = fmaxf(ev[i], delta);
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            float v = 0.f;
#pragma unroll
            for (int k = 0; k < N; ++k) v += Vm[i][k] * ev[k] * Vm[j][k];
            S[i][j] = v;
        }
}

/* The exact-Hessian option at node i (called from the KKT pass, where mu, the sum of the children's
 * multipliers, is at hand): the node's block of the Hessian of the Lagrangian in (x_i, u_i) - the
 * Gauss-Newton block, the curvature of the active keep-out rows (s grad^2 g, s = y + rho g > 0) and
 * mu' grad^2 f of the dynamics - eigenvalue-modified and stored in the HS rows (Q packed, M, R
 * packed).  Not inlined: its registers stay out of the default path. */
template <int NX, int MODEL>
__device__ __noinline__ void node_exact_hessian(const ProbRec &R, const View<NX> &V, int i, const float (&mu)[NX],
                                                float rho) {
    constexpr int NZ = NX + NU;
    const int np = V.np;
    const bool leaf = V.nchild[i] == 0;
    const float w = V.w[i];
    const float *Qd = leaf ? R.QNw : R.Qw;
    float S[NZ][NZ];
#pragma unroll
    for (int a = 0; a < NZ; ++a)
#pragma unroll
        for (int b = 0; b < NZ; ++b) S[a][b] = 0.f;
#pragma unroll
    for (int a = 0; a < NX; ++a) S[a][a] = w * Qd[a];
    S[0][0] += V.hq[jrow<3, MODEL>(np, i, 0)];
    S[0][1] += V.hq[jrow<3, MODEL>(np, i, 1)];
    S[1][0] += V.hq[jrow<3, MODEL>(np, i, 1)];
    S[1][1] += V.hq[jrow<3, MODEL>(np, i, 2)];
#pragma unroll
    for (int a = 0; a < NU; ++a) S[NX + a][NX + a] = leaf ? 1.f : w * R.Rw[a] + V.hr[jrow<NU, MODEL>(np, i, a)];
    float x[NX], u[NU];
    Lo lo;
    V.load_x(V.X, i, x);
    V.load_u(V.U, i, u);
    V.load_lo(i, lo);
    if (i != 0) {
        const int row0 = V.box ? 2 * NU : 0;
        for (int o = 0; o < V.nobs; ++o) {
            const float *ob = V.obs + (size_t)(OBS_ROWS * o) * np + i;
            const float ch = ob[2 * (size_t)np], sh = ob[3 * (size_t)np];
            const float ia2 = ob[4 * (size_t)np], ib2 = ob[5 * (size_t)np];
            float dpar, dper, irr;
            const float g = obs_g_comp(V.xref[i], V.xref[(size_t)np + i], ob[0], ob[(size_t)np], x[0], lo.x[0], x[1],
                                       lo.x[1], ch, sh, ia2, ib2, dpar, dper, irr);
            const float s = V.Y[(size_t)(row0 + o) * np + i] + rho * g;
            if (!(s > 0.f)) continue;
            /* grad^2 g = -(Mq / r - v v' / r^3), Mq = Rot' diag(1/a^2, 1/b^2) Rot, v = Rot' diag(.) (d_par, d_perp) */
            const float m00 = ch * ch * ia2 + sh * sh * ib2, m01 = ch * sh * (ia2 - ib2), m11 = sh * sh * ia2 + ch * ch * ib2;
            const float v0 = ch * ia2 * dpar - sh * ib2 * dper, v1 = sh * ia2 * dpar + ch * ib2 * dper;
            const float i3 = irr * irr * irr;
            S[0][0] += s * (v0 * v0 * i3 - m00 * irr);
            S[0][1] += s * (v0 * v1 * i3 - m01 * irr);
            S[1][0] += s * (v0 * v1 * i3 - m01 * irr);
            S[1][1] += s * (v1 * v1 * i3 - m11 * irr);
        }
    }
    if (!leaf) {
        float xa[NX], H[NZ][NZ];
#pragma unroll
        for (int j = 0; j < NX; ++j) xa[j] = V.xref[(size_t)j * np + i] + x[j];
        dyn_hessian<NX, MODEL>(R, xa, u, mu, H);
#pragma unroll
        for (int a = 0; a < NZ; ++a)
#pragma unroll
            for (int b = 0; b < NZ; ++b) S[a][b] += H[a][b];
    }
    eig_modify<NZ>(S);
#pragma unroll
    for (int a = 0; a < NX; ++a)
#pragma unroll
        for (int b = a; b < NX; ++b) V.HS[(size_t)sidx<NX>(a, b) * np + i] = S[a][b];
#pragma unroll
    for (int a = 0; a < NU; ++a)
#pragma unroll
        for (int b = 0; b < NX; ++b) V.HS[(size_t)(nsym(NX) + a * NX + b) * np + i] = S[NX + a][b];
    V.HS[(size_t)(nsym(NX) + NU * NX) * np + i] = S[NX][NX];
    V.HS[(size_t)(nsym(NX) + NU * NX + 1) * np + i] = 0.5f * (S[NX][NX + 1] + S[NX + 1][NX]);
    V.HS[(size_t)(nsym(NX) + NU * NX + 2) * np + i] = S[NX + 1][NX + 1];
}

/* ------------------------------------------------------------------ the per-problem solver */
/* Kernel flavours: the plain sweeps (variants 1, 2, 3, 5), the scan sweeps (variant 4) and the
 * exact-Hessian option each have their own instances, so that the registers one needs leave the
 * others' alone. */
constexpr int FLAVOR_PLAIN = 0, FLAVOR_SCAN = 1, FLAVOR_HESS = 2;

template <int NX, int MODEL, int FLAVOR>
__device__ __forceinline__ void solve_problem(const ProbRec &R, const int32_t *ib, const float *fin, const float *fw, float *fout,
                              float *fs, Stats *stat, const KOpts &O, Shared &sh, int32_t *tab, int tab_cap,
                              float *stg, int stg_ld) {
    constexpr int NS = nsym(NX);
    constexpr bool HOIST_LOADS = hoist_loads<NX>();
    View<NX> V(R, ib, fin, fw, fout, fs);
    V.comp = O.compensated != 0;
    V.hess = FLAVOR == FLAVOR_HESS;
    constexpr bool SCAN = FLAVOR == FLAVOR_SCAN;
    if constexpr (MODEL == 2) {
        if (R.edge_dyn) {   /* per-edge matrices: inputs at the edge's column, never written by the solver */
            V.edge = true;
            V.A = const_cast<float *>(fin) + (size_t)in_rows(NX, R.n_obs, 1).edge * R.npad;
            V.B = V.A + (size_t)NX * NX * R.npad;
        }
    }
    /* stage and path tables into shared memory: the sweeps index through them at every stage */
    const int64_t tn = table_ints(R.npad, R.n_stage, R.n_paths);
    if (tn <= tab_cap) {
        const int32_t *src = ib + V.tab_off;
        for (int j = threadIdx.x; j < tn; j += blockDim.x) tab[j] = src[j];
        V.sstart = tab + (V.sstart - src);
        V.bstage = tab + (V.bstage - src);
        V.ptab = tab + (V.ptab - src);
        V.pdepth = tab + (V.pdepth - src);
        V.ptop = tab + (V.ptop - src);
        __syncthreads();
    }
    const int tid = threadIdx.x, nt = blockDim.x;
    const int n = V.n, np = V.np, nc = V.nc;
    long long t_start = clock64(), c_lin = 0, c_bwd = 0, c_fwd = 0, c_ls = 0;

    /* ---- initial iterate: a warm-start slot or the cold start of Sec. V-B.  With warm_select the
     * primary start is used only when its merit (penalties select_rho, select_mu) is not
     * above the fallback's (slot 1, or the cold start). */
    int start = (R.has_warm & 1) ? 1 : ((R.has_warm & 2) ? 2 : 0);
    if (O.warm_select && (R.has_warm & 1)) {
        const int fb = (R.has_warm & 2) ? 2 : 0;
        load_start<NX>(R, V, 1);
        __syncthreads();
        const float m1 = start_merit<NX, MODEL>(R, V, O.select_rho, O.select_mu, sh);
        load_start<NX>(R, V, fb);
        __syncthreads();
        const float m2 = start_merit<NX, MODEL>(R, V, O.select_rho, O.select_mu, sh);
        start = (m1 == m1 && !(m1 > m2)) ? 1 : fb;
    }
    load_start<NX>(R, V, start);
    __syncthreads();

    float rho = O.rho0, mu = O.mu0, omega = O.omega0, eta = O.eta0;
    float pending = 0.f;   /* step of the last line search, not yet applied to (x, u, lam) */
    /* f, A and B depend on (x, u) alone: after an outer update the point has not moved, so the
     * next linearisation keeps them and recomputes only the terms that see y and rho */
    bool lin_done = false;
    float r_kkt = INFINITY, cviol = INFINITY;
    int inner = 0, outer = 0, ls_fail = 0, ls_fail_total = 0, ls_evals = 0, status = 1 /* MAX_ITER */;
    const int G = (O.ls_chunk <= 0 || O.ls_chunk > MAX_CHUNK) ? min(O.n_alpha, MAX_CHUNK) : O.ls_chunk;
    /* sweeps: 1 level-synchronous, 2 (default) per-path with one thread per path, 3 per-path with 8 lanes */
    /* automatic choice by tree shape: one thread per scenario path while the paths fit the block,
     * else stage by stage (a thread would otherwise walk several paths one after another) */
    /* 4 (scan sweeps) has its own kernel instance, so that the registers its CVF combinations need
     * leave the others' alone; 5 is the per-path backward sweep with the pointer-jumping forward one */
    const int variant = SCAN ? 4
                        : (O.variant == 1 || O.variant == 3 || O.variant == 5) ? O.variant
                        : (O.variant == 2 || R.n_paths <= nt) ? 2 : 1;

    while (outer < O.max_outer) {
        ++outer;
        for (;;) {
            /* ===== linearise + quadratise at the current point (first applying the step of the
             * previous line search, node by node: x += a dx, u += a du, lam += a (lam_QP - lam)) */
            long long t0 = clock64();
            const bool relin = !lin_done || pending > 0.f;
            lin_done = true;
            for (int i = tid; i < n; i += nt) {
                if constexpr (HOIST_LOADS) {
                    /* loads first (the node's rows, the step, the constraint data), stores last: a
                     * store the compiler cannot prove distinct would hold back every later load */
                    const bool is_leaf = V.nchild[i] == 0;
                    float x[NX], u[NU], lam[NX], q[NX], r[NU], hq[3], hr[NU];
                    Lo lo;
                    V.load_x(V.X, i, x);
                    V.load_u(V.U, i, u);
                    V.load_lo(i, lo);
                    const bool step = pending > 0.f;
                    if (step) apply_step<NX, MODEL>(V, i, pending, x, u, lam, lo);
                    const float la = node_la<NX, true>(R, V, i, is_leaf, x, u, lo, rho, q, r, hq, hr);
                    float xa[NX];
                    if (!is_leaf && relin) {
    #pragma unroll
                        for (int j = 0; j < NX; ++j) xa[j] = V.xref[(size_t)j * np + i] + x[j];
                    }
                    if (step) {
                        V.store_x(V.X, i, x);
                        V.store_u(V.U, i, u);
                        V.store_lo(i, lo);
                        if (i != 0) V.store_x(V.L, i, lam);
                    }
                    st_rows<NX, MODEL>(V.q, V.np, i, q);
                    st_rows<NU, MODEL>(V.r, V.np, i, r);
                    V.hq[jrow<3, MODEL>(np, i, 0)] = hq[0];
                    V.hq[jrow<3, MODEL>(np, i, 1)] = hq[1];
                    V.hq[jrow<3, MODEL>(np, i, 2)] = hq[2];
                    st_rows<NU, MODEL>(V.hr, V.np, i, hr);
                    V.nv[jrow<3, MODEL>(np, i, 0)] = la;
                    if (!is_leaf && relin) {
                        bool done = false;
                        if constexpr (MODEL == 2) {
                            if (V.edge) {   /* per-edge dynamics: the increment of every child's edge */
                                for (int m = V.fchild[i]; m < V.fchild[i] + V.nchild[i]; ++m) {
                                    float dl[NX];
                                    edge_increment<NX>(V, m, xa, u, dl);
                                    V.store_x(V.f, m, dl);
                                }
                                done = true;
                            }
                        }
                        if (!done) {
                            float xn[NX];
                            /* Jacobian entries go straight to the scratch rows (column c < nx: A, else B) */
                            dyn_lin<NX, MODEL>(R, xa, u, xn, [&](int a, int c, float v) {
                                if (c < NX) {
                                    if (a_fixed<MODEL>(a, c) < 0) V.A[jrow<NX * NX, MODEL>(np, i, a * NX + c)] = v;
                                } else if (b_fixed<MODEL>(a, c - NX) < 0) {
                                    V.B[jrow<NX * NU, MODEL>(np, i, a * NU + (c - NX))] = v;
                                }
                            });
                            V.store_x(V.f, i, xn);
                        }
                    }
                } else {
                    const bool is_leaf = V.nchild[i] == 0;
                    float x[NX], u[NU], q[NX], r[NU], hq[3], hr[NU];
                    Lo lo;
                    V.load_x(V.X, i, x);
                    V.load_u(V.U, i, u);
                    V.load_lo(i, lo);
                    if (pending > 0.f) {
                        apply_step_serial<NX, MODEL>(V, i, pending, x, u, lo);
                        V.store_x(V.X, i, x);
                        V.store_u(V.U, i, u);
                        V.store_lo(i, lo);
                    }
                    const float la = node_la<NX, true>(R, V, i, is_leaf, x, u, lo, rho, q, r, hq, hr);
                    st_rows<NX, MODEL>(V.q, V.np, i, q);
                    st_rows<NU, MODEL>(V.r, V.np, i, r);
                    V.hq[jrow<3, MODEL>(np, i, 0)] = hq[0];
                    V.hq[jrow<3, MODEL>(np, i, 1)] = hq[1];
                    V.hq[jrow<3, MODEL>(np, i, 2)] = hq[2];
                    st_rows<NU, MODEL>(V.hr, V.np, i, hr);
                    V.nv[jrow<3, MODEL>(np, i, 0)] = la;
                    if (!is_leaf && relin) {
                        float xa[NX], xn[NX];
    #pragma unroll
                        for (int j = 0; j < NX; ++j) xa[j] = V.xref[(size_t)j * np + i] + x[j];
                        /* Jacobian entries go straight to the scratch rows (column c < nx: A, else B) */
                        dyn_lin<NX, MODEL>(R, xa, u, xn, [&](int a, int c, float v) {
                            if (c < NX) {
                                if (a_fixed<MODEL>(a, c) < 0) V.A[jrow<NX * NX, MODEL>(np, i, a * NX + c)] = v;
                            } else if (b_fixed<MODEL>(a, c - NX) < 0) {
                                V.B[jrow<NX * NU, MODEL>(np, i, a * NU + (c - NX))] = v;
                            }
                        });
                        V.store_x(V.f, i, xn);
                    }
                }
            }
            __syncthreads();
            pending = 0.f;
            /* ===== defects and the KKT residual of the relaxed problem */
            float rk = 0.f;
            float sums[3] = {0.f, 0.f, 0.f};   /* L_a, lam'd, |d|^2 */
            for (int i = tid; i < n; i += nt) {
                /* two batches of loads: the node's and its parent's rows with the children's
                 * multipliers (defect and the first gradient terms, then the stores of d and the
                 * merit terms), then the Jacobians A_i, B_i and r_i for the coupling terms */
                const int nch = V.nchild[i], fc = V.fchild[i];
                const int pa = i ? V.parent[i] : 0;
                const float la_i = V.nv[jrow<3, MODEL>(np, i, 0)];
                float lsum[NX];
#pragma unroll
                for (int j = 0; j < NX; ++j) lsum[j] = 0.f;
                for (int m = fc; m < fc + nch; ++m)
#pragma unroll
                    for (int j = 0; j < NX; ++j) lsum[j] += V.L[(size_t)j * np + m];
                float xi[NX], xri[NX], li[NX], qi[NX], xp[NX], xrp[NX], fp[NX];
                V.load_x(V.X, i, xi);
                V.load_x(V.xref, i, xri);
                V.load_x(V.L, i, li);
                ld_rows<NX, MODEL>(V.q, V.np, i, qi);
                V.load_x(V.X, pa, xp);
                V.load_x(V.xref, pa, xrp);
                V.load_x(V.f, (MODEL == 2 && V.edge) ? i : pa, fp);   /* the increment of the edge into i */
                float ld = 0.f, dd = 0.f, gx[NX];
                if (i != 0) {
                    float dv[NX];
#pragma unroll
                    for (int j = 0; j < NX; ++j) {
                        const float dref = xrp[j] - xri[j];
                        const float dj = (dref + (xp[j] - xi[j])) + fp[j];
                        dv[j] = dj;
                        const float lj = li[j];
                        ld += lj * dj;
                        dd += dj * dj;
                        rk = fmaxf(rk, fabsf(dj));
                        gx[j] = qi[j] - lj;
                    }
                    st_rows<NX, MODEL>(V.d, V.np, i, dv);
                }
                V.nv[jrow<3, MODEL>(np, i, 1)] = ld;
                V.nv[jrow<3, MODEL>(np, i, 2)] = dd;
                bool edge_done = false;
                if constexpr (MODEL == 2) {
                    if (nch && V.edge) {   /* per-edge: sum over children of A_m' lam_m and B_m' lam_m */
                        float gu[NU];
                        ld_rows<NU, MODEL>(V.r, V.np, i, gu);
                        for (int m = fc; m < fc + nch; ++m) {
                            float lm[NX];
                            V.load_x(V.L, m, lm);
#pragma unroll
                            for (int a = 0; a < NX; ++a) {
                                if (i != 0) {
#pragma unroll
                                    for (int b = 0; b < NX; ++b) gx[b] += V.A[(size_t)(a * NX + b) * np + m] * lm[a];
                                }
#pragma unroll
                                for (int b = 0; b < NU; ++b) gu[b] += bload<NX, MODEL>(V.B, np, m, a, b) * lm[a];
                            }
                        }
#pragma unroll
                        for (int b = 0; b < NU; ++b) rk = fmaxf(rk, fabsf(gu[b]));
                        edge_done = true;
                    }
                }
                if (nch && !edge_done) {
                    float Ai[NX][NX], Bi[NX][NU], ri[NU];
#pragma unroll
                    for (int a = 0; a < NX; ++a) {
#pragma unroll
                        for (int b = 0; b < NX; ++b) Ai[a][b] = aload<NX, MODEL>(V.A, np, i, a, b);
#pragma unroll
                        for (int b = 0; b < NU; ++b) Bi[a][b] = bload<NX, MODEL>(V.B, np, i, a, b);
                    }
                    ld_rows<NU, MODEL>(V.r, V.np, i, ri);
                    if (i != 0) {
#pragma unroll
                        for (int a = 0; a < NX; ++a)
#pragma unroll
                            for (int b = 0; b < NX; ++b) gx[b] += Ai[a][b] * lsum[a];
                    }
#pragma unroll
                    for (int b = 0; b < NU; ++b) {
                        float gu = ri[b];
#pragma unroll
                        for (int a = 0; a < NX; ++a) gu += Bi[a][b] * lsum[a];
                        rk = fmaxf(rk, fabsf(gu));
                    }
                }
                if (i != 0) {
#pragma unroll
                    for (int j = 0; j < NX; ++j) rk = fmaxf(rk, fabsf(gx[j]));
                }
                if constexpr (FLAVOR == FLAVOR_HESS) node_exact_hessian<NX, MODEL>(R, V, i, lsum, rho);
                if (!(rk == rk)) rk = INFINITY;
                sums[0] += la_i;
                sums[1] += ld;
                sums[2] += dd;
            }
            r_kkt = block_max(rk, sh);
            block_sum<3>(sums, sh);
            c_lin += clock64() - t0;
            if (!(r_kkt < INFINITY) || !(fabsf(sums[0]) < INFINITY)) {
                status = -3;
                goto done;
            }
            if (r_kkt <= omega) break;
            if (inner >= O.max_iters) goto done;

            /* ===== backward: tree Riccati recursion, leaves to root */
            t0 = clock64();
            if (tid == 0) sh.flag = 0;
            __syncthreads();
            if constexpr (SCAN) backward_scan<NX, MODEL>(R, V, sh);
            else if (variant == 3) backward_coop<NX, MODEL>(R, V, sh);
            else if (variant == 2 || variant == 5)   /* variant 2 with staging: forward records, no K, k rows */
                backward_path<NX, MODEL>(R, V, sh, frec_model<MODEL>() && variant == 2 && stg != nullptr);
            else backward_level<NX, MODEL>(R, V, sh);
            __syncthreads();
            c_bwd += clock64() - t0;
            if (sh.flag) {
                status = -3;
                goto done;
            }

            /* ===== forward: linear rollout from the root, QP multipliers */
            t0 = clock64();
            float dir[3] = {0.f, 0.f, 0.f};   /* grad'dz, dz'W dz, (dlam - lam)'d */
            if (SCAN || variant == 5) forward_jump<NX, MODEL>(R, V);
            else if (variant == 3) forward_coop<NX, MODEL>(R, V);
            else if (variant == 2) {
                if constexpr (frec_model<MODEL>()) {
                    if (stg) forward_path_rec<NX, MODEL>(R, V, stg);
                    else forward_path<NX, MODEL>(R, V, nullptr, 0);
                } else {
                    forward_path<NX, MODEL>(R, V, stg, stg_ld);
                }
            }
            else forward_level<NX, MODEL>(R, V);
            multipliers_and_directions<NX, MODEL>(R, V, dir);
            block_sum<3>(dir, sh);
            c_fwd += clock64() - t0;

            /* ===== merit penalty mu and phi(0), phi'(0) */
            t0 = clock64();
            const float La0 = sums[0], ld0 = sums[1], dd0 = sums[2];
            const float dphi0 = dir[0] + dir[2];
            if (dd0 > 0.f && dphi0 - mu * dd0 > -0.5f * dir[1]) {
                const float need = 2.f * (dphi0 + 0.5f * dir[1]) * rcp(dd0);
                if (need > mu) mu = need;
            }
            const float phi0 = La0 + ld0 + 0.5f * mu * dd0;
            const float dphi = dphi0 - mu * dd0;

            /* ===== line search over alpha_i = 2^-i in chunks of G evaluated in parallel */
            float alpha = pow2neg(O.n_alpha - 1);
            bool accepted = false;
            for (int a0 = 0; a0 < O.n_alpha && !accepted; a0 += G) {
                const int cnt = min(G, O.n_alpha - a0);
#pragma unroll 1
                for (int a = 0; a < cnt; ++a) {
                    const float al = pow2neg(a0 + a);
                    float acc = 0.f;
                    for (int i = tid; i < n; i += nt) {
                        const int nch = V.nchild[i], fc = V.fchild[i];
                        const bool is_leaf = nch == 0;
                        float x[NX], u[NU], dxv[NX], duv[NU];
                        V.load_x(V.X, i, x);
                        V.load_u(V.U, i, u);
                        ld_rows<NX, MODEL>(V.dx, V.np, i, dxv);
                        ld_rows<NU, MODEL>(V.du, V.np, i, duv);
                        float base = V.nv[jrow<3, MODEL>(np, i, 0)];
                        for (int m = fc; m < fc + nch; ++m)
                            base += V.nv[jrow<3, MODEL>(np, m, 1)] + 0.5f * mu * V.nv[jrow<3, MODEL>(np, m, 2)];
                        float xt[NX], ut[NU], qd[NX], rd[NU], hqd[3], hrd[NU];
                        Lo lt;
                        V.load_lo(i, lt);
#pragma unroll
                        for (int j = 0; j < NX; ++j) xt[j] = x[j] + al * dxv[j];
                        ut[0] = u[0] + al * duv[0];
                        ut[1] = u[1] + al * duv[1];
                        if (V.comp) {   /* the trial point's remainders */
                            float e;
#pragma unroll
                            for (int j = 0; j < 2; ++j) {
                                xt[j] = two_sum(x[j], al * dxv[j], e);
                                lt.x[j] += e;
                            }
#pragma unroll
                            for (int j = 0; j < NU; ++j) {
                                ut[j] = two_sum(u[j], al * duv[j], e);
                                lt.u[j] += e;
                            }
                        }
                        float v = node_la<NX, false>(R, V, i, is_leaf, xt, ut, lt, rho, qd, rd, hqd, hrd);
                        if (!is_leaf) {
                            float xa[NX], ft[NX];
#pragma unroll
                            for (int j = 0; j < NX; ++j) xa[j] = V.xref[(size_t)j * np + i] + xt[j];
                            const bool per_edge = MODEL == 2 && V.edge;
                            if (!per_edge) dyn<NX, MODEL>(R, xa, ut, ft);
                            for (int m = fc; m < fc + nch; ++m) {
                                if constexpr (MODEL == 2) {
                                    if (per_edge) edge_increment<NX>(V, m, xa, ut, ft);
                                }
#pragma unroll
                                for (int j = 0; j < NX; ++j) {
                                    const float lm = V.L[(size_t)j * np + m];
                                    const float ltj = lm + al * (V.lq[jrow<NX, MODEL>(np, m, j)] - lm);
                                    const float dref = V.xref[(size_t)j * np + i] - V.xref[(size_t)j * np + m];
                                    const float dm = (dref + ((x[j] - V.X[(size_t)j * np + m]) +
                                                              al * (dxv[j] - V.dx[jrow<NX, MODEL>(np, m, j)]))) + ft[j];
                                    v += ltj * dm + 0.5f * mu * dm * dm;
                                }
                            }
                        }
                        acc += v - base;
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if ((tid & 31) == 0) sh.red[tid >> 5][a] = acc;
                }
                __syncthreads();
                ls_evals += cnt;
                const int nw = nt >> 5;
                for (int a = 0; a < cnt && !accepted; ++a) {
                    float s = 0.f;
                    for (int w = 0; w < nw; ++w) s += sh.red[w][a];
                    const float al = pow2neg(a0 + a);
                    if (s <= O.beta * al * dphi + O.ls_rel_eps * fabsf(phi0)) {
                        alpha = al;
                        accepted = true;
                    }
                }
                __syncthreads();
            }
            if (accepted) ls_fail = 0;
            else {
                ++ls_fail;
                ++ls_fail_total;
            }
            /* ===== the step x, u, lam += alpha (...) is applied by the next linearisation */
            pending = alpha;
            c_ls += clock64() - t0;
            ++inner;
            if (ls_fail >= 3) {
                for (int i = tid; i < n; i += nt) {
                    float x[NX], u[NU];
                    Lo lo;
                    V.load_x(V.X, i, x);
                    V.load_u(V.U, i, u);
                    V.load_lo(i, lo);
                    apply_step_serial<NX, MODEL>(V, i, pending, x, u, lo);
                    V.store_x(V.X, i, x);
                    V.store_u(V.U, i, u);
                    V.store_lo(i, lo);
                }
                __syncthreads();
                status = 2;
                goto done;
            }
        }
        /* ===== outer loop: BCL update (Sec. IV-B, Algorithm 1) */
        {
            float cv = 0.f;
            for (int i = tid; i < n; i += nt) {
                const bool is_leaf = V.nchild[i] == 0;
                float x[NX], u[NU];
                Lo lo;
                V.load_x(V.X, i, x);
                V.load_u(V.U, i, u);
                V.load_lo(i, lo);
                for_constraints<NX>(R, V, i, is_leaf, x, u, lo, [&](int row, float g) {
                    const float yv = V.Y[(size_t)row * np + i];
                    cv = fmaxf(cv, fabsf(fmaxf(g, -yv * rcp(rho))));
                });
            }
            cviol = block_max(cv, sh);
            if (cviol <= eta) {
                for (int i = tid; i < n; i += nt) {
                    const bool is_leaf = V.nchild[i] == 0;
                    float x[NX], u[NU];
                    Lo lo;
                    V.load_x(V.X, i, x);
                    V.load_u(V.U, i, u);
                    V.load_lo(i, lo);
                    for_constraints<NX>(R, V, i, is_leaf, x, u, lo, [&](int row, float g) {
                        float *yp = V.Y + (size_t)row * np + i;
                        *yp = fmaxf(0.f, *yp + rho * g);
                    });
                }
                __syncthreads();
                if (fmaxf(r_kkt, cviol) < O.eps_tol) {
                    status = 0;
                    goto done;
                }
                omega = omega * powf(rho, -O.b_omega);
                eta = eta * powf(rho, -O.b_eta);
            } else {
                if (!(O.cap_rule == 1 && rho >= O.rho_max)) {
                    /* Algorithm 1: y kept, rho <- tau rho (held at rho_max) */
                    rho = fminf(O.tau * rho, O.rho_max);
                } else {
                    /* cap rule: at rho_max a first-order multiplier step instead of a larger rho */
                    for (int i = tid; i < n; i += nt) {
                        const bool is_leaf = V.nchild[i] == 0;
                        float x[NX], u[NU];
                        Lo lo;
                        V.load_x(V.X, i, x);
                        V.load_u(V.U, i, u);
                        V.load_lo(i, lo);
                        for_constraints<NX>(R, V, i, is_leaf, x, u, lo, [&](int row, float g) {
                            float *yp = V.Y + (size_t)row * np + i;
                            *yp = fmaxf(0.f, *yp + rho * g);
                        });
                    }
                    __syncthreads();
                }
                omega = O.omega0 * powf(rho, -O.a_omega);
                eta = O.eta0 * powf(rho, -O.a_eta);
            }
            omega = fmaxf(omega, O.eps_tol);
            eta = fmaxf(eta, O.eps_tol);
        }
    }
done:
    __syncthreads();
    if (tid == 0) {
        stat->status = status;
        stat->inner_iters = inner;
        stat->outer_iters = outer;
        stat->ls_fail_total = ls_fail_total;
        stat->ls_evals = ls_evals;
        stat->start_used = start;
        stat->r_kkt = r_kkt;
        stat->c = cviol;
        stat->rho = rho;
        stat->mu = mu;
        stat->cyc_lin = c_lin;
        stat->cyc_bwd = c_bwd;
        stat->cyc_fwd = c_fwd;
        stat->cyc_ls = c_ls;
        stat->cyc_total = clock64() - t_start;
    }
}

/* One kernel per dynamics model, so that each carries only its own code and registers. */
template <int MODEL, int BLOCK, int FLAVOR = FLAVOR_PLAIN>
__global__ void __launch_bounds__(BLOCK, BLOCK <= BATCH_BLOCK ? 2 : 1) bmpc_solve_kernel(KernelArgs args) {
    constexpr int NX = MODEL == 1 ? 6 : 4;
    __shared__ Shared sh;
    __shared__ int pid_s;
    __shared__ ProbRec rec_s;
    extern __shared__ __align__(16) int32_t tab_s[];   /* 16-byte aligned: the forward records are copied in 16-byte units */
    float *stg = reinterpret_cast<float *>(tab_s + ((args.tab_ints + 3) & ~3));
    for (;;) {
        if (threadIdx.x == 0) pid_s = atomicAdd(args.queue, 1);
        __syncthreads();
        const int slot = pid_s;
        __syncthreads();
        if (slot >= args.n_problems) break;
        const int pid = args.order[slot];
        /* the problem record in shared memory: its constants are read inside every node loop, and
         * from shared memory no global store can hold those reads back */
        {
            const int4 *src = reinterpret_cast<const int4 *>(args.recs + pid);
            int4 *dst = reinterpret_cast<int4 *>(&rec_s);
            for (int j = threadIdx.x; j < (int)(sizeof(ProbRec) / sizeof(int4)); j += blockDim.x) dst[j] = src[j];
        }
        __syncthreads();
        const ProbRec &R = rec_s;
        solve_problem<NX, MODEL, FLAVOR>(R, args.ibase + R.off_int, args.inbase + R.off_in, args.warmbase + R.off_warm,
                                 args.outbase + R.off_out, args.scr + R.off_scr, args.stats + pid, args.opts, sh,
                                 tab_s, args.tab_ints, args.stg_ld ? stg : nullptr, args.stg_ld);
    }
}


/* ------------------------------------------------------------------ work-queue order */
/* Longest-predicted-first order of the problems of one model (list scheduling of the persistent
 * blocks): the key is nodes x (previous inner iterations + 1), ties broken by problem id, so the
 * order is deterministic.  One block sorts a tile of ORDER_TILE entries of `order` in place
 * (bitonic sort in shared memory); batches longer than a tile are ordered tile by tile. */
constexpr int ORDER_TILE = 4096;

__global__ void __launch_bounds__(1024) bmpc_order_kernel(const ProbRec *recs, const Stats *stats, int32_t *order,
                                                          int cnt) {
    __shared__ unsigned long long key[ORDER_TILE];
    const int base = blockIdx.x * ORDER_TILE;
    const int m = min(ORDER_TILE, cnt - base);
    int P = 1;
    while (P < m) P <<= 1;
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        unsigned long long k = ~0ull;
        if (j < m) {
            const int pid = order[base + j];
            const int it = min(max(stats[pid].inner_iters, 0), 1 << 16);
            unsigned long long cost = (unsigned long long)recs[pid].n * (unsigned long long)(it + 1);
            if (cost > 0xFFFFFFFFull) cost = 0xFFFFFFFFull;
            k = ((0xFFFFFFFFull - cost) << 32) | (unsigned)pid;
        }
        key[j] = k;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int j = threadIdx.x; j < P / 2; j += blockDim.x) {
                const int lo = 2 * j - (j & (stride - 1)), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long a = key[lo], b = key[hi];
                if ((a > b) == up) {
                    key[lo] = b;
                    key[hi] = a;
                }
            }
            __syncthreads();
        }
    for (int j = threadIdx.x; j < m; j += blockDim.x) order[base + j] = (int32_t)(key[j] & 0xFFFFFFFFull);
}

cudaError_t launch_order(const ProbRec *recs, const Stats *stats, int32_t *order, int cnt, cudaStream_t stream) {
    if (cnt <= 1) return cudaSuccess;
    bmpc_order_kernel<<<(cnt + ORDER_TILE - 1) / ORDER_TILE, 1024, 0, stream>>>(recs, stats, order, cnt);
    return cudaGetLastError();
}

/* Device sin/cos of the dynamics on n angles (self-test of sincos_cw against its error bound). */
/* FP32 peak microbenchmark: every thread runs eight independent FMA chains (enough independent
 * instructions to cover the FMA latency at full occupancy), iters rounds each, and stores the sum so
 * that nothing is dead code.  FLOPs = 2 * 8 * iters * threads. */
__global__ void __launch_bounds__(256) bmpc_fma_kernel(float *out, int iters, float b, float c) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 1e-3f * threadIdx.x + (float)k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t launch_fma(float *out, int blocks, int iters, cudaStream_t stream) {
    bmpc_fma_kernel<<<blocks, 256, 0, stream>>>(out, iters, 0.999999f, 1e-7f);
    return cudaGetLastError();
}

__global__ void bmpc_sincos_kernel(const float *a, float *sn, float *cs, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) sincos_cw(a[i], sn + i, cs + i);
}

cudaError_t launch_sincos(const float *a, float *sn, float *cs, int n, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    bmpc_sincos_kernel<<<(n + 255) / 256 < 1184 ? (n + 255) / 256 : 1184, 256, 0, stream>>>(a, sn, cs, n);
    return cudaGetLastError();
}

/* Eigenvalue-modification self-test: eig_modify (the exact-Hessian option) on `count` symmetric
 * N x N matrices in place, one matrix per thread (N = 6 and 8: the stacked (x, u) blocks of the
 * n_x = 4 and n_x = 6 models). */
template <int N>
__global__ void bmpc_eig_kernel(float *S, int count) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    float M[N][N];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) M[i][j] = S[(size_t)k * N * N + i * N + j];
    eig_modify<N>(M);
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) S[(size_t)k * N * N + i * N + j] = M[i][j];
}

/* Second-derivative self-test: dyn_hessian (the exact-Hessian option's sum_i mu_i d^2 f_i / dz dz
 * of the RK4 map, z = (x, u)) at `count` points, one per thread; rows and columns in (x, u) order. */
struct Params10 {
    float v[10];
};

template <int MODEL>
__global__ void bmpc_dynhess_kernel(Params10 prm, float dt, const float *x, const float *u, const float *mu, float *H,
                                    int count) {
    constexpr int NX = MODEL == 1 ? 6 : 4, NZ = NX + NU;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    ProbRec R = {};
    R.dt = dt;
#pragma unroll
    for (int i = 0; i < 10; ++i) R.params[i] = prm.v[i];
    float xa[NX], uu[NU], m[NX], Hm[NZ][NZ];
#pragma unroll
    for (int i = 0; i < NX; ++i) {
        xa[i] = x[(size_t)k * NX + i];
        m[i] = mu[(size_t)k * NX + i];
    }
#pragma unroll
    for (int i = 0; i < NU; ++i) uu[i] = u[(size_t)k * NU + i];
    dyn_hessian<NX, MODEL>(R, xa, uu, m, Hm);
#pragma unroll
    for (int i = 0; i < NZ; ++i)
#pragma unroll
        for (int j = 0; j < NZ; ++j) H[(size_t)k * NZ * NZ + i * NZ + j] = Hm[i][j];
}

cudaError_t launch_dynhess(int model, const float *params, float dt, const float *x, const float *u, const float *mu,
                           float *H, int count, cudaStream_t stream) {
    Params10 p;
    for (int i = 0; i < 10; ++i) p.v[i] = params[i];
    const int blocks = (count + 127) / 128;
    if (model == 0) bmpc_dynhess_kernel<0><<<blocks, 128, 0, stream>>>(p, dt, x, u, mu, H, count);
    else if (model == 1) bmpc_dynhess_kernel<1><<<blocks, 128, 0, stream>>>(p, dt, x, u, mu, H, count);
    else if (model == 2) bmpc_dynhess_kernel<2><<<blocks, 128, 0, stream>>>(p, dt, x, u, mu, H, count);
    else bmpc_dynhess_kernel<3><<<blocks, 128, 0, stream>>>(p, dt, x, u, mu, H, count);
    return cudaGetLastError();
}

cudaError_t launch_eig(float *S, int n, int count, cudaStream_t stream) {
    const int blocks = (count + 127) / 128;
    if (n == 6) bmpc_eig_kernel<6><<<blocks, 128, 0, stream>>>(S, count);
    else bmpc_eig_kernel<8><<<blocks, 128, 0, stream>>>(S, count);
    return cudaGetLastError();
}

/* ------------------------------------------------------------------ input transfers */
/* Obstacle row values from the caller's heading and semi-axes: cos and sin of the heading and
 * 1/a^2, 1/b^2, each in double precision rounded once (one definition for both upload paths). */
__device__ __forceinline__ float obstacle_row(int c, float h, float ea, float eb) {
    if (c == 2) return (float)cos((double)h);
    if (c == 3) return (float)sin((double)h);
    const double s = c == 4 ? (double)ea : (double)eb;
    return (float)(1.0 / (s * s));
}

/* After bmpc_set_problems' copy: obstacle rows hold cx, cy, heading, -, a, b as packed by the
 * host; rows 2..5 become cos, sin, 1/a^2, 1/b^2 in place. */
__global__ void bmpc_obstacle_rows_kernel(FlatArgs a) {
    const ProbRec &R = a.recs[blockIdx.x];
    const int n = R.n, np = R.npad;
    float *ob = a.inbase + R.off_in + (size_t)in_rows(R.nx, R.n_obs).obs * np;
    for (int e = threadIdx.x; e < R.n_obs * n; e += blockDim.x) {
        const int o = e / n, i = e % n;
        float *r = ob + (size_t)(OBS_ROWS * o) * np + i;
        const float h = r[2 * (size_t)np], ea = r[4 * (size_t)np], eb = r[5 * (size_t)np];
        for (int c = 2; c < OBS_ROWS; ++c) r[(size_t)c * np] = obstacle_row(c, h, ea, eb);
    }
}

/* Inputs of problem blockIdx.x from the node-major flat arrays into its component-major input
 * region (the device side of bmpc_set_problems_flat), padding nodes zeroed. */
__global__ void bmpc_flat_in_kernel(FlatArgs a) {
    const ProbRec &R = a.recs[blockIdx.x];
    const int n = R.n, np = R.npad, nx = R.nx, no = R.n_obs;
    const InRows ir = in_rows(nx, no);
    float *base = a.inbase + R.off_in;
    const float *xr = a.raw + R.off_nx;
    const float *wt = a.raw + a.T_nx + R.off_node;
    const float *ob = a.raw + a.T_nx + a.T_n + R.off_obs;
    const int64_t total = (int64_t)ir.total * np;
    for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
        const int row = (int)(e / np), i = (int)(e % np);
        float v = 0.f;
        if (i < n) {
            if (row < ir.weight) v = xr[(size_t)i * nx + row];
            else if (row == ir.weight) v = a.has_weight ? wt[i] : 1.f;
            else {
                const int o = (row - ir.obs) / OBS_ROWS, c = (row - ir.obs) % OBS_ROWS;
                const float *q = ob + ((size_t)i * no + o) * 5;   /* cx, cy, heading, a, b */
                v = c < 2 ? q[c] : obstacle_row(c, q[2], q[3], q[4]);
            }
        }
        base[e] = v;
    }
}

/* Outputs of problem blockIdx.x into the node-major flat arrays (absolute states x = xref + xi,
 * the same sum as the host unpacking) for bmpc_get_solutions_flat. */
__global__ void bmpc_flat_out_kernel(FlatArgs a) {
    const ProbRec &R = a.recs[blockIdx.x];
    const int n = R.n, np = R.npad, nx = R.nx, nc = R.nc;
    const OutRows orw = out_rows(nx, nc);
    const InRows ir = in_rows(nx, R.n_obs);
    const float *o = a.outbase + R.off_out;
    const float *xref = a.inbase + R.off_in + (size_t)ir.xref * np;
    float *fx = a.raw + R.off_nx;
    float *fu = a.raw + a.T_nx + 2 * R.off_node;
    float *fl = a.raw + a.T_nx + 2 * a.T_n + R.off_nx;
    float *fy = a.raw + 2 * a.T_nx + 2 * a.T_n + R.off_nc;
    for (int e = threadIdx.x; e < n * nx; e += blockDim.x) {
        const int i = e / nx, j = e % nx;
        fx[e] = xref[(size_t)j * np + i] + o[(size_t)(orw.x + j) * np + i];
        fl[e] = o[(size_t)(orw.lam + j) * np + i];
    }
    for (int e = threadIdx.x; e < n * NU; e += blockDim.x) fu[e] = o[(size_t)(orw.u + e % NU) * np + e / NU];
    for (int e = threadIdx.x; e < n * nc; e += blockDim.x) fy[e] = o[(size_t)(orw.y + e % nc) * np + e / nc];
}

cudaError_t launch_flat(int which, const FlatArgs &a, int n_problems, cudaStream_t stream) {
    if (n_problems <= 0) return cudaSuccess;
    if (which == 0) bmpc_flat_in_kernel<<<n_problems, 256, 0, stream>>>(a);
    else if (which == 1) bmpc_flat_out_kernel<<<n_problems, 256, 0, stream>>>(a);
    else bmpc_obstacle_rows_kernel<<<n_problems, 256, 0, stream>>>(a);
    return cudaGetLastError();
}

/* ------------------------------------------------------------------ warm-start kernels */
/* Device scatter: problem `order[blockIdx.x]` takes its start from a dense device array, node-major
 * x | u | lam | y (absolute states), into warm-start slot `slot`. */
__global__ void bmpc_scatter_warm_kernel(WarmArgs a) {
    const int pid = a.order[blockIdx.x];
    const ProbRec &R = a.recs[pid];
    const int n = R.n, np = R.npad, nx = R.nx, nc = R.nc;
    const WarmRows wr = warm_rows(nx, nc);
    float *w = a.warmbase + R.off_warm + (size_t)a.slot * wr.total * np;
    const float *src = a.src + (size_t)pid * a.stride;
    const float *sx = src, *su = sx + (size_t)n * nx, *sl = su + (size_t)n * NU, *sy = sl + (size_t)n * nx;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        for (int j = 0; j < nx; ++j) {
            w[(size_t)(wr.wx + j) * np + i] = sx[(size_t)i * nx + j];
            w[(size_t)(wr.wl + j) * np + i] = sl[(size_t)i * nx + j];
        }
        for (int j = 0; j < NU; ++j) w[(size_t)(wr.wu + j) * np + i] = su[(size_t)i * NU + j];
        for (int c = 0; c < nc; ++c) w[(size_t)(wr.wy + c) * np + i] = sy[(size_t)i * nc + c];
    }
}

/* Receding-horizon shift of a previous solution on the same tree into warm-start slot `slot`:
 * the node at stage k takes the previous value at stage k+1 on the path of its first leaf (the
 * lowest-index scenario through it); the last stage appends the last control and propagates the
 * dynamics; u, lam and y are shifted the same way (input rows from the last non-leaf node). */
template <int MODEL>
__global__ void bmpc_shift_warm_kernel(WarmArgs a) {
    constexpr int NX = MODEL == 1 ? 6 : 4;
    const int pid = a.order[blockIdx.x];
    const ProbRec &R = a.recs[pid];
    const ProbRec &Q = a.prev_recs[pid];
    const int n = R.n, np = R.npad, nc = R.nc, ns = R.n_stage;
    const IntOff io = int_off(np, ns, R.n_paths);
    const int32_t *ib = a.ibase + R.off_int;
    const int32_t *owner = ib + io.owner, *stage = ib + io.stage, *ptab = ib + io.ptab, *pdepth = ib + io.pdepth;
    const IntOff qo = int_off(Q.npad, Q.n_stage, Q.n_paths);
    const int32_t *qparent = a.prev_ibase + Q.off_int + qo.parent;
    const InRows qi = in_rows(NX, Q.n_obs);
    const float *qxref = a.prev_inbase + Q.off_in + (size_t)qi.xref * np;
    const OutRows qr = out_rows(NX, nc);
    const float *qout = a.prev_outbase + Q.off_out;
    const float *qX = qout + (size_t)qr.x * np, *qU = qout + (size_t)qr.u * np;
    const float *qL = qout + (size_t)qr.lam * np, *qY = qout + (size_t)qr.y * np;
    const WarmRows wr = warm_rows(NX, nc);
    float *w = a.warmbase + R.off_warm + (size_t)a.slot * wr.total * np;
    const int box_rows = R.box_on ? 2 * NU : 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int s = owner[i], k = stage[i], depth = pdepth[s];
        const int32_t *path = ptab + (size_t)s * ns;
        const int jx = path[min(k + 1, depth)], ju = path[min(k + 1, max(depth - 1, 0))];
        float xa[NX];
#pragma unroll
        for (int j = 0; j < NX; ++j) xa[j] = qxref[(size_t)j * np + jx] + qX[(size_t)j * np + jx];
        if (k + 1 > depth) {       /* beyond the previous leaf: append the last control and propagate */
            const int jp = qparent[jx];
            float ua[NU] = {qU[jp], qU[(size_t)np + jp]}, dl[NX];
            dyn<NX, MODEL>(Q, xa, ua, dl);
#pragma unroll
            for (int j = 0; j < NX; ++j) xa[j] += dl[j];
        }
#pragma unroll
        for (int j = 0; j < NX; ++j) {
            w[(size_t)(wr.wx + j) * np + i] = xa[j];
            w[(size_t)(wr.wl + j) * np + i] = qL[(size_t)j * np + jx];
        }
        for (int j = 0; j < NU; ++j) w[(size_t)(wr.wu + j) * np + i] = qU[(size_t)j * np + ju];
        for (int c = 0; c < nc; ++c) {
            const int src = c < box_rows ? ju : jx;
            w[(size_t)(wr.wy + c) * np + i] = qY[(size_t)c * np + src];
        }
    }
}

cudaError_t launch_scatter_warm(const WarmArgs &a, cudaStream_t stream) {
    if (a.n_problems <= 0) return cudaSuccess;
    bmpc_scatter_warm_kernel<<<a.n_problems, 256, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_shift_warm(const WarmArgs &a, int model, cudaStream_t stream) {
    if (a.n_problems <= 0) return cudaSuccess;
    if (model == 0) bmpc_shift_warm_kernel<0><<<a.n_problems, 256, 0, stream>>>(a);
    else if (model == 1) bmpc_shift_warm_kernel<1><<<a.n_problems, 256, 0, stream>>>(a);
    else if (model == 2) bmpc_shift_warm_kernel<2><<<a.n_problems, 256, 0, stream>>>(a);
    else bmpc_shift_warm_kernel<3><<<a.n_problems, 256, 0, stream>>>(a);
    return cudaGetLastError();
}


/* ------------------------------------------------------------------ learned warm start: glue kernels */

/* Features: x0 without X, then per scenario and obstacle (cx - X0, cy) at the path's middle node
 * and (cx - X0, cy, heading) at its leaf. */
__global__ void bmpc_features_kernel(GlueArgs a) {
    const int pid = blockIdx.x;
    const ProbRec &R = a.recs[pid];
    const int np = R.npad, nx = R.nx;
    const IntOff io = int_off(np, R.n_stage, R.n_paths);
    const int32_t *ib = a.ibase + R.off_int;
    const InRows ir = in_rows(nx, R.n_obs);
    const float *obs = a.inbase + R.off_in + (size_t)ir.obs * np;
    float *f = a.out + (size_t)pid * a.stride;
    for (int j = threadIdx.x; j < a.stride; j += blockDim.x) f[j] = 0.f;
    __syncthreads();
    if (threadIdx.x < nx - 1) f[threadIdx.x] = R.x0[threadIdx.x + 1];
    const int S = min(a.n_scen, R.n_paths), O = min(a.n_obs_max, R.n_obs);
    for (int t = threadIdx.x; t < S * O; t += blockDim.x) {
        const int s = t / O, o = t % O;
        const int depth = ib[io.pdepth + s];
        const int32_t *path = ib + io.ptab + (size_t)s * R.n_stage;
        const int mid = path[depth / 2], leaf = path[depth];
        const float *ob = obs + (size_t)(OBS_ROWS * o) * np;
        float *g = f + (nx - 1) + 5 * (s * a.n_obs_max + o);
        g[0] = ob[mid] - R.x0[0];
        g[1] = ob[(size_t)np + mid];
        g[2] = ob[leaf] - R.x0[0];
        g[3] = ob[(size_t)np + leaf];
        g[4] = atan2f(ob[3 * (size_t)np + leaf], ob[2 * (size_t)np + leaf]);   /* heading */
    }
}

/* Targets: the current solution packed node-major x | u | lam | y, X0 subtracted from the X of
 * every state. */
__global__ void bmpc_targets_kernel(GlueArgs a) {
    const int pid = blockIdx.x;
    const ProbRec &R = a.recs[pid];
    const int n = R.n, np = R.npad, nx = R.nx, nc = R.nc;
    const InRows ir = in_rows(nx, R.n_obs);
    const float *xref = a.inbase + R.off_in + (size_t)ir.xref * np;
    const OutRows orw = out_rows(nx, nc);
    const float *o = a.outbase + R.off_out;
    float *t = a.out + (size_t)pid * a.stride;
    float *tx = t, *tu = tx + (size_t)n * nx, *tl = tu + (size_t)n * NU, *ty = tl + (size_t)n * nx;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        for (int j = 0; j < nx; ++j) {
            const float dv = o[(size_t)(orw.x + j) * np + i];
            tx[(size_t)i * nx + j] = j == 0 ? (xref[i] - R.x0[0]) + dv : xref[(size_t)j * np + i] + dv;
            tl[(size_t)i * nx + j] = o[(size_t)(orw.lam + j) * np + i];
        }
        for (int j = 0; j < NU; ++j) tu[(size_t)i * NU + j] = o[(size_t)(orw.u + j) * np + i];
        for (int c = 0; c < nc; ++c) {
            const float y = o[(size_t)(orw.y + c) * np + i];
            ty[(size_t)i * nc + c] = a.y_sqrt ? sqrtf(fmaxf(y, 0.f)) : y;
        }
    }
    const int64_t used = (int64_t)n * (2 * nx + NU + nc);
    for (int64_t j = used + threadIdx.x; j < a.stride; j += blockDim.x) t[j] = 0.f;
}

/* Starts from network outputs: mean + std * pred, X0 added back to the X of every state; then the
 * states are replaced by the rollout of the predicted controls from x0 through the tree (level by
 * level), so that the start satisfies the dynamics like the shifted start does. */
template <int MODEL>
__global__ void bmpc_starts_kernel(GlueArgs a) {
    constexpr int NX = MODEL == 1 ? 6 : 4;
    const int pid = a.order_base[blockIdx.x];
    const ProbRec &R = a.recs[pid];
    const int n = R.n;
    const int64_t used = (int64_t)n * (2 * NX + NU + R.nc);
    const float *p = a.pred + (size_t)pid * a.ld_pred;
    float *s = a.out + (size_t)pid * a.stride;
    for (int64_t j = threadIdx.x; j < used; j += blockDim.x) {
        float v = a.mean[j] + a.std[j] * p[j];
        if (j < (int64_t)n * NX && j % NX == 0) v += R.x0[0];
        if (j >= (int64_t)n * (2 * NX + NU)) {   /* AL multipliers are >= 0 */
            v = fmaxf(v, 0.f);
            if (a.y_sqrt) v *= v;
        }
        s[j] = v;
    }
    __syncthreads();
    const IntOff io = int_off(R.npad, R.n_stage, R.n_paths);
    const int32_t *ib = a.ibase + R.off_int;
    const int32_t *parent = ib + io.parent, *nchild = ib + io.nchild, *ss = ib + io.sstart;
    float *sx = s, *su = s + (size_t)n * NX;
    if (threadIdx.x < NX) sx[threadIdx.x] = R.x0[threadIdx.x];
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (!nchild[i]) su[(size_t)i * NU] = su[(size_t)i * NU + 1] = 0.f;
    __syncthreads();
    for (int st = 1; st < R.n_stage; ++st) {
        for (int i = ss[st] + threadIdx.x; i < ss[st + 1]; i += blockDim.x) {
            const int pa = parent[i];
            float xp[NX], up[NU] = {su[(size_t)pa * NU], su[(size_t)pa * NU + 1]}, dl[NX];
#pragma unroll
            for (int j = 0; j < NX; ++j) xp[j] = sx[(size_t)pa * NX + j];
            dyn<NX, MODEL>(R, xp, up, dl);
#pragma unroll
            for (int j = 0; j < NX; ++j) sx[(size_t)i * NX + j] = xp[j] + dl[j];
        }
        __syncthreads();
    }
}

cudaError_t launch_glue(int which, const GlueArgs &a, int n_problems, cudaStream_t stream, int model) {
    if (n_problems <= 0) return cudaSuccess;
    if (which == 0) bmpc_features_kernel<<<n_problems, 256, 0, stream>>>(a);
    else if (which == 1) bmpc_targets_kernel<<<n_problems, 256, 0, stream>>>(a);
    else if (model == 0) bmpc_starts_kernel<0><<<n_problems, 256, 0, stream>>>(a);
    else if (model == 1) bmpc_starts_kernel<1><<<n_problems, 256, 0, stream>>>(a);
    else if (model == 2) bmpc_starts_kernel<2><<<n_problems, 256, 0, stream>>>(a);
    else bmpc_starts_kernel<3><<<n_problems, 256, 0, stream>>>(a);
    return cudaGetLastError();
}

/* Launch helper used by the host API: `args.order` lists problems of `model` only. */
/* The kernel instance of a model for a block size. */
using SolveFn = void (*)(KernelArgs);
SolveFn solve_fn(int model, int block, int flavor = FLAVOR_PLAIN) {
    if (flavor == FLAVOR_SCAN) {   /* sweep variant 4: one instance per model, up to 512 threads per problem */
        if (model == 0) return bmpc_solve_kernel<0, MAX_BLOCK, FLAVOR_SCAN>;
        if (model == 1) return bmpc_solve_kernel<1, MAX_BLOCK, FLAVOR_SCAN>;
        if (model == 2) return bmpc_solve_kernel<2, MAX_BLOCK, FLAVOR_SCAN>;
        return bmpc_solve_kernel<3, MAX_BLOCK, FLAVOR_SCAN>;
    }
    if (flavor == FLAVOR_HESS) {   /* the exact-Hessian option: one instance per model */
        if (model == 0) return bmpc_solve_kernel<0, MAX_BLOCK, FLAVOR_HESS>;
        if (model == 1) return bmpc_solve_kernel<1, MAX_BLOCK, FLAVOR_HESS>;
        if (model == 2) return bmpc_solve_kernel<2, MAX_BLOCK, FLAVOR_HESS>;
        return bmpc_solve_kernel<3, MAX_BLOCK, FLAVOR_HESS>;
    }
    const bool big = block > BATCH_BLOCK;
    if (model == 0) return big ? bmpc_solve_kernel<0, MAX_BLOCK> : bmpc_solve_kernel<0, BATCH_BLOCK>;
    if (model == 1) return big ? bmpc_solve_kernel<1, MAX_BLOCK> : bmpc_solve_kernel<1, BATCH_BLOCK>;
    if (model == 2) return big ? bmpc_solve_kernel<2, MAX_BLOCK> : bmpc_solve_kernel<2, BATCH_BLOCK>;
    return big ? bmpc_solve_kernel<3, MAX_BLOCK> : bmpc_solve_kernel<3, BATCH_BLOCK>;
}

int solve_flavor(const KOpts &o) {
    return o.variant == 4 ? FLAVOR_SCAN : o.hessian ? FLAVOR_HESS : FLAVOR_PLAIN;
}

cudaError_t launch_solve(const KernelArgs &args, int model, int grid, int block, size_t smem, cudaStream_t stream) {
    solve_fn(model, block, solve_flavor(args.opts))<<<grid, block, smem, stream>>>(args);
    return cudaGetLastError();
}

int max_block_threads() { return MAX_BLOCK; }

/* Dynamic shared memory of a solve launch: the stage/path tables (tab_ints) and, when it fits in
 * 96 KB, the sweep staging of min(max_paths, block) path threads (*stg_ld, else 0). */
size_t solve_smem(int model, int tab_ints, int max_paths, int block, int *stg_ld) {
    /* floats per path thread: the ring of node-major records, or (per-edge dynamics) the row slots */
    const int per_thread = model == 0   ? Frec<4, 0>::tstride
                           : model == 1 ? Frec<6, 1>::tstride
                           : model == 2 ? SWEEP_DEPTH * rows_stage<4, 2>()
                                        : Frec<4, 3>::tstride;
    const int ld = std::min(max_paths, block);
    const size_t tab = sizeof(int32_t) * (size_t)((tab_ints + 3) & ~3);
    const size_t stg = sizeof(float) * (size_t)per_thread * ld;
    if (ld > 0 && tab + stg <= 96u * 1024u) {
        *stg_ld = ld;
        return tab + stg;
    }
    *stg_ld = 0;
    return sizeof(int32_t) * (size_t)tab_ints;
}

/* Raises the dynamic shared-memory limit of a model's kernels to at least `smem` (never lowers it,
 * so batches sharing the process keep theirs).  The attribute is always set: without it the 48 KB
 * default bounds static and dynamic shared memory together, and the kernels' static part (the
 * reduction arrays and the problem record) is about 14 KB. */
cudaError_t prepare_solve(int model, size_t smem) {
    static size_t granted[NUM_MODELS] = {0, 0, 0, 0};
    if (model < 0 || model >= NUM_MODELS || smem <= granted[model]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(solve_fn(model, BATCH_BLOCK), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(solve_fn(model, MAX_BLOCK), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int f = FLAVOR_SCAN; f <= FLAVOR_HESS && e == cudaSuccess; ++f)
        e = cudaFuncSetAttribute(solve_fn(model, MAX_BLOCK, f), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    if (e == cudaSuccess) granted[model] = smem;
    return e;
}

cudaError_t occupancy(int model, int block, size_t smem, int *blocks_per_sm, const KOpts &o) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, solve_fn(model, block, solve_flavor(o)), block,
                                                         smem);
}

}  // namespace bmpc
