/* Tree LQR at general sizes with per-edge dynamics: Eq. (lqr_tree_approx) by the tree Riccati
 * recursion of Eq. (tree_Riccati) and the feedback laws of Eq. (tree_feedback_laws), then the
 * forward sweep of Sec. III-A.  The C ABI and the problem statement are in include/bmpc_lqr.h.
 *
 * Layout of the work.  Backward, a block of NXP^2 / 4 threads (at least a warp) owns one node (of one
 * problem of the batch): thread l + NXP w owns entries (l, 4w .. 4w + 3) of the node's matrix products, so a
 * node step is a set of short dot products over shared-memory tiles, with the tree's depth as the
 * only sequential chain:
 *   per child edge m:  T1 = P_m A_m, T2 = P_m B_m, g = p_m + P_m c_m
 *                      S_xx += A_m' T1, S_xu += A_m' T2, S_uu += B_m' T2, s_x += A_m' g, s_u += B_m' g
 *   node:              H = R + S_uu, [K k] = -H^-1 [M + S_xu' | r + s_u] (thread c: right-hand side
 *                      c, factoring H in its own registers), P = Q + S_xx + S_ux' K, p = q + s_x + S_ux' k
 * Forward, lane j of a warp computes row j of x_m = A_m x_p + B_m u_p + c_m, then u and lam.
 * Two schedules: a launch per stage and sweep (a block per node backward, a warp per node forward),
 * or one block per problem that walks the nodes in post-order, keeping a node's P and p and the next
 * edge's data in shared memory from one step to the next.
 * Tiles are zero-padded to NXP x NXP (NXP in {8, 16, 32}) and NUP (in {4, 8, 16}) so that every
 * loop is unrolled at compile time; the tile rows that many threads read in common are fetched as
 * 16-byte broadcasts.  FP32 throughout (the paper's batch experiments run FP32 too). */
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "bmpc.h"
#include "bmpc_lqr.h"

namespace {

constexpr int LQR_WARPS = 4;   /* nodes per block of the forward sweep */

/* Threads of a node step's block: one per (row, group of four columns) of an NXP x NXP product
 * (NXP^2 / 4), at least one warp. */
template <int NXP>
__host__ __device__ constexpr int lqr_nt() { return NXP * NXP / 4 > 32 ? NXP * NXP / 4 : 32; }
constexpr unsigned FULL = 0xffffffffu;

struct LqrArgs {
    const float *Q, *M, *R, *q, *r, *A, *B, *c, *x0;
    float *K, *k, *P, *p, *x, *u, *lam;
    const int32_t *child_idx;
    const int4 *node4;   /* per node: first and end index into child_idx, first child (or -1), parent */
    int32_t *flag;
    int n, nx, nu, batch;
    int s0, cnt;   /* first node of the stage and its node count */
};

/* Shared tiles of one node step; row strides are multiples of 4 floats (16-byte rows for the
 * broadcast reads) and 4 more than the columns (16-byte stores or row reads by 8 lanes at a time
 * hit distinct banks).  The forward step of a single-node stage reuses A, B, PS and X. */
template <int NXP, int NUP>
struct LqrTiles {
    static constexpr int SX = NXP + 4, SU = NUP + 4;
    float A[NXP][SX];    /* the edge's A_m */
    float B[NXP][SU];    /* the edge's B_m */
    float PS[NXP][SX];   /* the child's P_m; the node's own P once its step ends (one block per problem) */
    float T1[NXP][SX];   /* P_m A_m; later the node's P before symmetrisation */
    float T2[NXP][SU];   /* P_m B_m */
    float H[NUP][SU];    /* H, then its Cholesky factor (lower triangle) */
    float X[NUP][SX];    /* [Q_ux | q_u] with q_u in column NXP, then [K | k]; forward: K_m */
    float QUX[NUP][SX];  /* Q_ux, kept for P and p */
    float g[NXP];        /* p_m + P_m c_m */
    float cv[NXP];       /* c_m */
    float pv[NXP];       /* the child's p_m; the node's own p once its step ends */
    float qx[NXP];       /* q + s_x */
    float xs[NXP];       /* forward: x of the stage's node */
    float id[NUP];       /* 1 / L_bb (0 past n_u) */
    float kv[NUP];       /* forward: k_m */
    float us[NUP];       /* forward: u of the stage's node */
};

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

/* This thread's share of one edge's A_m, B_m and c_m, and of a child's P_m and p_m, held in
 * registers between their loads and their stores into the zero-padded tiles: every load of a
 * staging is issued before its first store, so a staging costs one memory latency. */
template <int NXP, int NUP>
struct EdgeRegs {
    static constexpr int NT = lqr_nt<NXP>(), IA = (NXP * NXP + NT - 1) / NT, IB = (NXP * NUP + NT - 1) / NT;
    float va[IA], vb[IB], vc;
};
template <int NXP, int NUP>
struct ValueRegs {
    static constexpr int NT = lqr_nt<NXP>(), IA = (NXP * NXP + NT - 1) / NT;
    float vp[IA], vq;
};

template <int NXP, int NUP>
__device__ __forceinline__ void load_edge(EdgeRegs<NXP, NUP> &e, const LqrArgs &a, size_t cm, int tid) {
    using E = EdgeRegs<NXP, NUP>;
    const int nx = a.nx, nu = a.nu;
    const float *gA = a.A + cm * nx * nx, *gB = a.B + cm * nx * nu;
#pragma unroll
    for (int it = 0; it < E::IA; ++it) {
        const int idx = tid + it * E::NT, r = idx / NXP, c = idx % NXP;
        e.va[it] = (idx < NXP * NXP && r < nx && c < nx) ? gA[(size_t)r * nx + c] : 0.f;
    }
#pragma unroll
    for (int it = 0; it < E::IB; ++it) {
        const int idx = tid + it * E::NT, r = idx / NUP, c = idx % NUP;
        e.vb[it] = (idx < NXP * NUP && r < nx && c < nu) ? gB[(size_t)r * nu + c] : 0.f;
    }
    e.vc = tid < nx ? a.c[cm * nx + tid] : 0.f;
}

template <int NXP, int NUP>
__device__ __forceinline__ void store_edge(LqrTiles<NXP, NUP> *ts, const EdgeRegs<NXP, NUP> &e, int tid) {
    using E = EdgeRegs<NXP, NUP>;
#pragma unroll
    for (int it = 0; it < E::IA; ++it) {
        const int idx = tid + it * E::NT;
        if (idx < NXP * NXP) ts->A[idx / NXP][idx % NXP] = e.va[it];
    }
#pragma unroll
    for (int it = 0; it < E::IB; ++it) {
        const int idx = tid + it * E::NT;
        if (idx < NXP * NUP) ts->B[idx / NUP][idx % NUP] = e.vb[it];
    }
    if (tid < NXP) ts->cv[tid] = e.vc;
}

/* P_m is loaded by threads in rows; p_m by threads NXP .. 2 NXP - 1. */
template <int NXP, int NUP>
__device__ __forceinline__ void load_value(ValueRegs<NXP, NUP> &v, const LqrArgs &a, size_t cm, int tid) {
    using V = ValueRegs<NXP, NUP>;
    const int nx = a.nx, tq = tid - NXP;
    const float *gP = a.P + cm * nx * nx;
#pragma unroll
    for (int it = 0; it < V::IA; ++it) {
        const int idx = tid + it * V::NT, r = idx / NXP, c = idx % NXP;
        v.vp[it] = (idx < NXP * NXP && r < nx && c < nx) ? gP[(size_t)r * nx + c] : 0.f;
    }
    v.vq = (tq >= 0 && tq < nx) ? a.p[cm * nx + tq] : 0.f;
}

template <int NXP, int NUP>
__device__ __forceinline__ void store_value(LqrTiles<NXP, NUP> *ts, const ValueRegs<NXP, NUP> &v, int tid) {
    using V = ValueRegs<NXP, NUP>;
#pragma unroll
    for (int it = 0; it < V::IA; ++it) {
        const int idx = tid + it * V::NT;
        if (idx < NXP * NXP) ts->PS[idx / NXP][idx % NXP] = v.vp[it];
    }
    const int tq = tid - NXP;
    if (tq >= 0 && tq < NXP) ts->pv[tq] = v.vq;
}

__device__ __forceinline__ void fma4(float4 &acc, float s, const float4 v) {
    acc.x += s * v.x;
    acc.y += s * v.y;
    acc.z += s * v.z;
    acc.w += s * v.w;
}

/* acc += a . b term by term in index order (the order of the per-warp forward step) */
__device__ __forceinline__ void fma_row(float &acc, const float4 a, const float4 b) {
    acc += a.x * b.x;
    acc += a.y * b.y;
    acc += a.z * b.z;
    acc += a.w * b.w;
}

/* Backward step of node i of problem t by the whole block of lqr_nt<NXP>() threads; thread l + NXP w
 * owns entries (l, 4w .. 4w + 3) of the n_x-column products and, for w < NUP / 4, of the n_u-column
 * ones.  Every thread of the block calls it with the same arguments; nd = (first and end index into
 * child_idx, last child).  The children are taken from the last to the first.
 * FUSED (one block per problem, nodes in post-order): `prev` is the node stepped just before, which
 * left its P and p in PS and pv and, when this node is not a leaf, this node's first edge in A, B and
 * cv; this step leaves the same for the next one, whose first edge `pre_m` it loads at its start. */
template <int NXP, int NUP, bool REG_CHOL, bool FUSED>
__device__ __forceinline__ void backward_node(const LqrArgs &a, int t, int i, int4 nd, int prev, int pre_m) {
    constexpr int NW = NXP / 4, NWU = NUP / 4;
    extern __shared__ __align__(16) float lqr_smem[];
    using Tiles = LqrTiles<NXP, NUP>;
    Tiles *ts = reinterpret_cast<Tiles *>(lqr_smem);
    const int tid = threadIdx.x, nt = blockDim.x, l = tid % NXP, w = tid / NXP;
    const int j0 = 4 * w;     /* this thread's column group */
    /* threads past the NXP^2 / 4 product threads (a block of one warp at NXP = 8) idle in the products */
    const bool act = lqr_nt<NXP>() == NXP * NXP / 4 || w < NW;
    const int nx = a.nx, nu = a.nu;
    const size_t base = (size_t)t * a.n, node = base + i;
    const float *Qi = a.Q + node * nx * nx;
    float *Pi = a.P + node * nx * nx, *Ki = a.K + node * nu * nx;
    const int c0 = nd.x, c1 = nd.y;
    const bool row = l < nx && l < NXP;

    EdgeRegs<NXP, NUP> ahead;
    if (FUSED && pre_m >= 0) load_edge<NXP, NUP>(ahead, a, base + pre_m, tid);

    if (c0 == c1) {   /* leaf: P = sym(Q), p = q, no law */
        float ps[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int j = j0 + s;
            ps[s] = (row && j < nx) ? 0.5f * (Qi[(size_t)j * nx + l] + Qi[(size_t)l * nx + j]) : 0.f;
            if (row && j < nx) Pi[(size_t)j * nx + l] = ps[s];
        }
        const float qv = (w == 0 && row) ? a.q[node * nx + l] : 0.f;
        if (w == 0 && row) a.p[node * nx + l] = qv;
        for (int e = tid; e < nu * nx; e += nt) Ki[e] = 0.f;
        if (tid < nu) a.k[node * nu + tid] = 0.f;
        if constexpr (FUSED) {
            if (act) {
#pragma unroll
                for (int s = 0; s < 4; ++s) ts->PS[j0 + s][l] = ps[s];
                if (w == 0) ts->pv[l] = qv;
            }
            if (pre_m >= 0) store_edge<NXP, NUP>(ts, ahead, tid);
        }
        return;
    }

    /* the node's own data, loaded now so that its latency hides behind the children's products:
     * row l of Q at columns 4w .. 4w + 3, M and R at (4w .., l), q, r */
    float qr4[4], mv4[4], rv4[4];
#pragma unroll
    for (int s2 = 0; s2 < 4; ++s2) {
        const int b = j0 + s2;
        qr4[s2] = (row && b < nx) ? Qi[(size_t)l * nx + b] : 0.f;
        mv4[s2] = (a.M && w < NWU && row && b < nu) ? a.M[node * nu * nx + (size_t)b * nx + l] : 0.f;
        rv4[s2] = (w < NWU && l < nu && b < nu) ? a.R[node * nu * nu + (size_t)l * nu + b] : 0.f;
    }
    const float qv = (w == NW - 1 && row) ? a.q[node * nx + l] : 0.f;
    const float rv = (w == NW - 1 && l < nu) ? a.r[node * nu + l] : 0.f;

    float4 sxx = make_float4(0.f, 0.f, 0.f, 0.f), sxu = sxx, suu = sxx;
    float sx = 0.f, su = 0.f;
    for (int e = c1 - 1; e >= c0; --e) {
        const int m = e == c1 - 1 ? nd.z : a.child_idx[e];
        const size_t cm = base + m;
        const bool have_edge = FUSED && e == c1 - 1 && prev >= 0, have_value = FUSED && m == prev;
        if (e != c1 - 1) __syncthreads();   /* the previous child's tiles are no longer read */
        if (!have_edge || !have_value) {
            EdgeRegs<NXP, NUP> er;
            ValueRegs<NXP, NUP> vr;
            if (!have_edge) load_edge<NXP, NUP>(er, a, cm, tid);
            if (!have_value) load_value<NXP, NUP>(vr, a, cm, tid);
            if (!have_edge) store_edge<NXP, NUP>(ts, er, tid);
            if (!have_value) store_value<NXP, NUP>(ts, vr, tid);
            __syncthreads();
        }
        /* T1 = P_m A_m (and T2 = P_m B_m for w < NUP / 4): entries (l, 4w .. 4w + 3); g = p_m + P_m c_m */
        if (act) {
            float4 t1 = make_float4(0.f, 0.f, 0.f, 0.f), t2 = t1;
            float gl = 0.f;
#pragma unroll
            for (int k4 = 0; k4 < NXP; k4 += 4) {
                const float4 p4 = ld4(&ts->PS[l][k4]);
                const float pk[4] = {p4.x, p4.y, p4.z, p4.w};
                float4 a_[4], b_[4];
                float c_[4];
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    a_[s] = ld4(&ts->A[k4 + s][j0]);
                    if (w < NWU) b_[s] = ld4(&ts->B[k4 + s][j0]);
                    c_[s] = ts->cv[k4 + s];
                }
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    fma4(t1, pk[s], a_[s]);
                    if (w < NWU) fma4(t2, pk[s], b_[s]);
                    if (w == NW - 1) gl += pk[s] * c_[s];
                }
            }
            st4(&ts->T1[l][j0], t1);
            if (w < NWU) st4(&ts->T2[l][j0], t2);
            if (w == NW - 1) ts->g[l] = ts->pv[l] + gl;
        }
        __syncthreads();
        /* S_xx += A' T1, S_xu += A' T2, S_uu += B' T2 at (l, 4w ..); s_x += A' g, s_u += B' g (warp
         * NW - 1); the operands of four k at a time are loaded before their products */
        if (act) {
#pragma unroll
            for (int k4 = 0; k4 < NXP; k4 += 4) {
                float a_[4], b_[4], g_[4];
                float4 t1_[4], t2_[4];
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    a_[s] = ts->A[k4 + s][l];
                    t1_[s] = ld4(&ts->T1[k4 + s][j0]);
                    if (w < NWU) t2_[s] = ld4(&ts->T2[k4 + s][j0]);
                    b_[s] = l < NUP ? ts->B[k4 + s][l] : 0.f;
                    g_[s] = ts->g[k4 + s];
                }
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    fma4(sxx, a_[s], t1_[s]);
                    if (w < NWU) {
                        fma4(sxu, a_[s], t2_[s]);
                        fma4(suu, b_[s], t2_[s]);
                    }
                    if (w == NW - 1) {
                        sx += a_[s] * g_[s];
                        su += b_[s] * g_[s];
                    }
                }
            }
        }
    }

    /* the node's own terms: Q_xx (l, 4w ..) in registers; Q_ux into X and QUX, H, q_u, q_x (every
     * entry the later steps read is written, zeros past n_x and n_u, H the identity past n_u) */
    float4 qxx = sxx;
    qxx.x += qr4[0];
    qxx.y += qr4[1];
    qxx.z += qr4[2];
    qxx.w += qr4[3];
    if (w < NWU) {
        const float s4[4] = {sxu.x, sxu.y, sxu.z, sxu.w};
        const float h4[4] = {suu.x, suu.y, suu.z, suu.w};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int b = j0 + s;
            const float v = (row && b < nu) ? mv4[s] + s4[s] : 0.f;
            ts->X[b][l] = v;
            ts->QUX[b][l] = v;
            if (l < NUP) ts->H[l][b] = (l < nu && b < nu) ? rv4[s] + h4[s] : (l == b ? 1.f : 0.f);
        }
    }
    if (w == NW - 1) {
        ts->qx[l] = row ? qv + sx : 0.f;
        if (l < NUP) ts->X[l][NXP] = l < nu ? rv + su : 0.f;
    }
    __syncthreads();
    if (FUSED && pre_m >= 0) store_edge<NXP, NUP>(ts, ahead, tid);   /* A, B, cv are not read again */

    if constexpr (REG_CHOL) {
        /* H = L L' and [K k] = -H^-1 [Q_ux | q_u] with no exchange between threads: thread c (c <= n_x;
         * c = n_x is q_u, in column NXP) factors the whole of H in its own registers, then solves for
         * column c.  H is the identity past n_u, so the unrolled loops need no guards and the padded
         * part of L stays the identity; 1 / L_jj comes from one reciprocal square root. */
        if (tid <= nx) {
            const int col = tid < nx ? tid : NXP;
            float L[NUP * (NUP + 1) / 2], il[NUP], y[NUP];   /* packed rows: L_rc at r (r + 1) / 2 + c */
#pragma unroll
            for (int r = 0; r < NUP; ++r)
#pragma unroll
                for (int c4 = 0; c4 <= r; c4 += 4) {
                    const float4 v = ld4(&ts->H[r][c4]);
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int s = 0; s < 4; ++s)
                        if (c4 + s <= r) L[r * (r + 1) / 2 + c4 + s] = vv[s];
                }
#pragma unroll
            for (int b = 0; b < NUP; ++b) y[b] = ts->X[b][col];
            bool bad = false;
#pragma unroll
            /* right-looking factorisation with the column-oriented forward substitution L y = x taken
             * along (column j of L is final once scaled), then L' z = y */
            for (int j = 0; j < NUP; ++j) {
                const float d = L[j * (j + 1) / 2 + j];
                bad = bad || !(d > 0.f) || !isfinite(d);
                il[j] = rsqrtf(d);
#pragma unroll
                for (int r = j + 1; r < NUP; ++r) L[r * (r + 1) / 2 + j] *= il[j];
                y[j] *= il[j];
#pragma unroll
                for (int e = j + 1; e < NUP; ++e) y[e] -= L[e * (e + 1) / 2 + j] * y[j];
#pragma unroll
                for (int c = j + 1; c < NUP; ++c)
#pragma unroll
                    for (int r = c; r < NUP; ++r) L[r * (r + 1) / 2 + c] -= L[r * (r + 1) / 2 + j] * L[c * (c + 1) / 2 + j];
            }
#pragma unroll
            for (int b = NUP - 1; b >= 0; --b) {
                y[b] *= il[b];
#pragma unroll
                for (int e = 0; e < b; ++e) y[e] -= L[b * (b + 1) / 2 + e] * y[b];
            }
#pragma unroll
            for (int b = 0; b < NUP; ++b) ts->X[b][col] = -y[b];
            if (bad && tid == 0) atomicExch(a.flag, 1);
        }
        __syncthreads();
    } else {
    /* Cholesky H = L L' by warp 0 in registers: lane l holds row l, columns broadcast by shuffles
     * (H is the identity past n_u; pivots past n_u are skipped and 1 / L_bb is 0 there) */
    static_assert(NXP == 32, "the lane-parallel factorisation takes l as the lane");
    if (tid < 32) {
        float h[NUP], idl = 0.f;
#pragma unroll
        for (int b = 0; b < NUP; ++b) h[b] = l < NUP ? ts->H[l][b] : 0.f;
        bool bad = false;
#pragma unroll
        for (int j = 0; j < NUP; ++j) {
            if (j < nu) {
                const float d = __shfl_sync(FULL, h[j], j);
                bad = bad || !(d > 0.f) || !isfinite(d);
                const float il = rsqrtf(d);
                if (l == j) {
                    h[j] = d * il;
                    idl = il;
                } else if (l > j) {
                    h[j] *= il;
                }
#pragma unroll
                for (int b = j + 1; b < NUP; ++b) {
                    const float lbj = __shfl_sync(FULL, h[j], b);
                    if (l >= b) h[b] -= h[j] * lbj;
                }
            }
        }
        if (l < NUP) {
#pragma unroll
            for (int b = 0; b < NUP; ++b) ts->H[l][b] = b <= l ? h[b] : 0.f;
            ts->id[l] = l < nu ? idl : 0.f;
        }
        if (bad && l == 0) atomicExch(a.flag, 1);
    }
    __syncthreads();

    /* [K k] = -H^-1 [Q_ux | q_u]: thread c solves right-hand side c (c = nx is q_u, in column NXP);
     * the zero right-hand sides and 1 / L_bb = 0 past n_u make the unguarded substitutions exact */
    if (tid <= nx) {
        const int col = tid < nx ? tid : NXP;
        float y[NUP];
#pragma unroll
        for (int b = 0; b < NUP; ++b) y[b] = ts->X[b][col];
        /* column-oriented substitutions: each step scales one entry and updates the rest
         * independently, so the dependent chain is n_u steps long, not n_u^2 / 2 */
#pragma unroll
        for (int b = 0; b < NUP; ++b) {   /* L y = x */
            y[b] *= ts->id[b];
#pragma unroll
            for (int e = b + 1; e < NUP; ++e) y[e] -= ts->H[e][b] * y[b];
        }
#pragma unroll
        for (int b = NUP - 1; b >= 0; --b) {   /* L' z = y */
            y[b] *= ts->id[b];
#pragma unroll
            for (int e = 0; e < b; ++e) y[e] -= ts->H[b][e] * y[b];
        }
#pragma unroll
        for (int b = 0; b < NUP; ++b) ts->X[b][col] = -y[b];
    }
    __syncthreads();
    }

    /* P = Q_xx + Q_ux' K at (l, 4w ..) into T1; p = q_x + Q_ux' k (warp NW - 1) */
    if (act) {
        float4 pv4 = qxx;
        float pl = ts->qx[l];
#pragma unroll
        for (int b = 0; b < NUP; ++b) {
            const float qb = ts->QUX[b][l];
            fma4(pv4, qb, ld4(&ts->X[b][j0]));
            if (w == NW - 1) pl += qb * ts->X[b][NXP];
        }
        st4(&ts->T1[l][j0], pv4);
        if (w == NW - 1) {
            if (row) a.p[node * nx + l] = pl;
            if (FUSED) ts->pv[l] = pl;   /* 0 past n_x */
        }
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int j = j0 + s;
            const float v = 0.5f * (ts->T1[l][j] + ts->T1[j][l]);
            if (row && j < nx) Pi[(size_t)j * nx + l] = v;
            if (FUSED) ts->PS[j][l] = v;
        }
    }
    if (row && act)
        for (int b = w; b < nu; b += NW) Ki[(size_t)b * nx + l] = ts->X[b][l];
    if (tid < nu) a.k[node * nu + tid] = ts->X[tid][NXP];
}

/* One backward launch per stage: block b is node s0 + b % cnt of problem b / cnt. */
template <int NXP, int NUP, int MINB>
__global__ void __launch_bounds__(lqr_nt<NXP>(), MINB) lqr_backward_kernel(LqrArgs a) {
    const long long item = blockIdx.x;
    const int i = a.s0 + (int)(item % a.cnt);
    const int4 nd = a.node4[i];
    backward_node<NXP, NUP, (MINB == 1 || NUP < 16), false>(a, (int)(item / a.cnt), i, make_int4(nd.x, nd.y, nd.z, 0),
                                                           -1, -1);
}

/* Forward step of node m of problem t by one whole warp (lane j: row j). */
template <int NXP, int NUP>
__device__ __forceinline__ void forward_node(const LqrArgs &a, int t, int m, int lane) {
    const int nx = a.nx, nu = a.nu;
    const size_t node = (size_t)t * a.n + m;
    const bool row = lane < nx;
    const int4 nd = a.node4[m];
    const bool leaf = nd.x == nd.y;
    /* every row this lane needs, loaded at once: A_m, B_m (row `lane`), K_m (row `lane` < n_u) and
     * P_m (column `lane` = row, coalesced) */
    const float *Am = a.A + node * nx * nx + (size_t)lane * nx, *Bm = a.B + node * nx * nu + (size_t)lane * nu;
    const float *Km = a.K + node * nu * nx + (size_t)lane * nx, *Pm = a.P + node * nx * nx;
    float arow[NXP], brow[NUP], krow[NXP], prow[NXP];
#pragma unroll
    for (int k = 0; k < NXP; ++k) {
        arow[k] = (m > 0 && row && k < nx) ? __ldg(Am + k) : 0.f;
        krow[k] = (!leaf && lane < nu && k < nx) ? Km[k] : 0.f;
        prow[k] = (row && k < nx) ? Pm[(size_t)k * nx + lane] : 0.f;
    }
#pragma unroll
    for (int b = 0; b < NUP; ++b) brow[b] = (m > 0 && row && b < nu) ? __ldg(Bm + b) : 0.f;
    float xl = 0.f;
    if (m == 0) {
        xl = row ? a.x0[(size_t)t * nx + lane] : 0.f;
    } else {
        const size_t pa = (size_t)t * a.n + nd.w;
        const float xp = row ? a.x[pa * nx + lane] : 0.f;
        const float up = lane < nu ? a.u[pa * nu + lane] : 0.f;
        float v = row ? a.c[node * nx + lane] : 0.f;
#pragma unroll
        for (int k = 0; k < NXP; ++k) v += arow[k] * __shfl_sync(FULL, xp, k);
#pragma unroll
        for (int b = 0; b < NUP; ++b) v += brow[b] * __shfl_sync(FULL, up, b);
        xl = row ? v : 0.f;
    }
    /* u = K x + k (rows < n_u; 0 at leaves), lam = P x + p */
    float ul = (!leaf && lane < nu) ? a.k[node * nu + lane] : 0.f;
    float ll = row ? a.p[node * nx + lane] : 0.f;
#pragma unroll
    for (int j = 0; j < NXP; ++j) {
        const float xj = __shfl_sync(FULL, xl, j);
        ul += krow[j] * xj;
        ll += prow[j] * xj;
    }
    if (row) {
        a.x[node * nx + lane] = xl;
        a.lam[node * nx + lane] = ll;
    }
    if (lane < nu) a.u[node * nu + lane] = ul;
}

/* One forward launch per stage: warp w of block b is node s0 + item % cnt of problem item / cnt,
 * item = 4b + w. */
template <int NXP, int NUP>
__global__ void __launch_bounds__(32 * LQR_WARPS) lqr_forward_kernel(LqrArgs a) {
    const int w = threadIdx.x / 32, lane = threadIdx.x & 31;
    const long long item = (long long)blockIdx.x * LQR_WARPS + w;
    if (item >= (long long)a.cnt * a.batch) return;
    forward_node<NXP, NUP>(a, (int)(item / a.cnt), a.s0 + (int)(item % a.cnt), lane);
}

/* Forward step of the single node m of a stage (one block per problem): the whole block stages
 * A_m, B_m, K_m, P_m, c_m, k_m and p_m into the tiles (one memory latency), then warp 0 computes,
 * lane j on row j, x_m = A_m x_p + B_m u_p + c_m, u_m = K_m x_m + k_m and lam_m = P_m x_m + p_m.
 * x_p and u_p are in xs and us when the previous stage was a single node too (its step left them
 * there), else they are read back from memory.  Leaves have K = 0 and k = 0 in memory. */
template <int NXP, int NUP>
__device__ __forceinline__ void forward_single(const LqrArgs &a, int t, int m, bool par_smem) {
    extern __shared__ __align__(16) float lqr_smem[];
    using Tiles = LqrTiles<NXP, NUP>;
    Tiles *ts = reinterpret_cast<Tiles *>(lqr_smem);
    constexpr int NT = lqr_nt<NXP>(), IA = (NXP * NXP + NT - 1) / NT, IB = (NXP * NUP + NT - 1) / NT;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nx = a.nx, nu = a.nu;
    const size_t node = (size_t)t * a.n + m;
    const bool root = m == 0;
    const float *gA = a.A + node * nx * nx, *gB = a.B + node * nx * nu, *gK = a.K + node * nu * nx,
                *gP = a.P + node * nx * nx;
    float va[IA], vp[IA], vb[IB], vk[IB], vv = 0.f;
#pragma unroll
    for (int it = 0; it < IA; ++it) {
        const int idx = tid + it * NT, r = idx / NXP, c = idx % NXP;
        const bool ok = idx < NXP * NXP && r < nx && c < nx;
        va[it] = (ok && !root) ? gA[(size_t)r * nx + c] : 0.f;
        vp[it] = ok ? gP[(size_t)r * nx + c] : 0.f;
    }
#pragma unroll
    for (int it = 0; it < IB; ++it) {
        const int idx = tid + it * NT, rb = idx / NUP, cb = idx % NUP, rk = idx / NXP, ck = idx % NXP;
        vb[it] = (idx < NXP * NUP && rb < nx && cb < nu && !root) ? gB[(size_t)rb * nu + cb] : 0.f;
        vk[it] = (idx < NUP * NXP && rk < nu && ck < nx) ? gK[(size_t)rk * nx + ck] : 0.f;
    }
    const int v1 = tid - NXP, v2 = tid - NXP - NUP;   /* c_m: threads 0 .. NXP - 1, k_m next, then p_m */
    if (tid < NXP) vv = (tid < nx && !root) ? a.c[node * nx + tid] : 0.f;
    else if (v1 < NUP) vv = v1 < nu ? a.k[node * nu + v1] : 0.f;
    else if (v2 < NXP) vv = v2 < nx ? a.p[node * nx + v2] : 0.f;
#pragma unroll
    for (int it = 0; it < IA; ++it) {
        const int idx = tid + it * NT;
        if (idx < NXP * NXP) {
            ts->A[idx / NXP][idx % NXP] = va[it];
            ts->PS[idx / NXP][idx % NXP] = vp[it];
        }
    }
#pragma unroll
    for (int it = 0; it < IB; ++it) {
        const int idx = tid + it * NT;
        if (idx < NXP * NUP) {
            ts->B[idx / NUP][idx % NUP] = vb[it];
            ts->X[idx / NXP][idx % NXP] = vk[it];
        }
    }
    if (tid < NXP) ts->cv[tid] = vv;
    else if (v1 < NUP) ts->kv[v1] = vv;
    else if (v2 < NXP) ts->pv[v2] = vv;
    __syncthreads();
    if (tid < 32) {
        float xl;
        if (root) {
            xl = lane < nx ? a.x0[(size_t)t * nx + lane] : 0.f;
        } else {
            if (!par_smem) {
                const size_t pa = (size_t)t * a.n + a.node4[m].w;
                if (lane < NXP) ts->xs[lane] = lane < nx ? a.x[pa * nx + lane] : 0.f;
                if (lane < NUP) ts->us[lane] = lane < nu ? a.u[pa * nu + lane] : 0.f;
                __syncwarp();
            }
            float v = 0.f;
            if (lane < NXP) {
                v = ts->cv[lane];
#pragma unroll
                for (int k4 = 0; k4 < NXP; k4 += 4) fma_row(v, ld4(&ts->A[lane][k4]), ld4(&ts->xs[k4]));
#pragma unroll
                for (int b4 = 0; b4 < NUP; b4 += 4) fma_row(v, ld4(&ts->B[lane][b4]), ld4(&ts->us[b4]));
            }
            xl = lane < nx ? v : 0.f;
        }
        __syncwarp();
        if (lane < NXP) ts->xs[lane] = xl;
        __syncwarp();
        float ul = 0.f, ll = 0.f;
        if (lane < NUP) {
            ul = ts->kv[lane];
#pragma unroll
            for (int k4 = 0; k4 < NXP; k4 += 4) fma_row(ul, ld4(&ts->X[lane][k4]), ld4(&ts->xs[k4]));
        }
        if (lane < NXP) {
            ll = ts->pv[lane];
#pragma unroll
            for (int k4 = 0; k4 < NXP; k4 += 4) fma_row(ll, ld4(&ts->PS[lane][k4]), ld4(&ts->xs[k4]));
        }
        __syncwarp();
        if (lane < NUP) ts->us[lane] = ul;   /* 0 past n_u */
        if (lane < nx) {
            a.x[node * nx + lane] = xl;
            a.lam[node * nx + lane] = ll;
        }
        if (lane < nu) a.u[node * nu + lane] = ul;
    }
}

/* The whole solve of problem t = blockIdx.x in one block; no block waits on another.  Backward: the
 * nodes in post-order, plan[k] = (node, first and end index into child_idx, last child), so that a
 * node's last child is stepped just before it and leaves its P, p and the node's first edge in the
 * tiles; the plan is read two nodes ahead.  Forward: stage by stage, a single-node stage by the whole
 * block (forward_single), wider ones a warp per node.  For trees whose stages are narrow, where the
 * per-stage launches would leave the GPU idle between them. */
template <int NXP, int NUP>
__global__ void __launch_bounds__(lqr_nt<NXP>()) lqr_fused_kernel(LqrArgs a, const int4 *plan, const int32_t *sstart, int S) {
    constexpr int WARPS = lqr_nt<NXP>() / 32;
    const int t = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31, n = a.n;
    const int4 none = make_int4(-1, 0, 0, -1);
    int4 cur = plan[0], nxt = n > 1 ? plan[1] : none;
    int prev = -1;
    for (int k = 0; k < n; ++k) {
        const int4 after = k + 2 < n ? plan[k + 2] : none;
        const int pre_m = nxt.y != nxt.z ? nxt.w : -1;   /* the next node's first edge, if it has children */
        backward_node<NXP, NUP, true, true>(a, t, cur.x, make_int4(cur.y, cur.z, cur.w, 0), prev, pre_m);
        __syncthreads();   /* the node's P, p and the next edge reach the next step; the tiles are free again */
        prev = cur.x;
        cur = nxt;
        nxt = after;
    }
    int b0 = sstart[0], b1 = sstart[1];
    bool single_prev = false;
    for (int s = 0; s < S; ++s) {
        const int b2 = s + 2 <= S ? sstart[s + 2] : 0;
        if (b1 - b0 == 1) {
            forward_single<NXP, NUP>(a, t, b0, single_prev);
            single_prev = true;
        } else {
            for (int i = b0 + w; i < b1; i += WARPS) forward_node<NXP, NUP>(a, t, i, lane);
            single_prev = false;
        }
        __syncthreads();
        b0 = b1;
        b1 = b2;
    }
}

template <int NXP, int NUP>
size_t backward_smem() { return sizeof(LqrTiles<NXP, NUP>); }

using LqrKernel = void (*)(LqrArgs);
using FusedKernel = void (*)(LqrArgs, const int4 *, const int32_t *, int);
struct Instance {
    LqrKernel bwd, bwd_wide, fwd;   /* bwd_wide: two blocks per SM, for stages wider than the GPU */
    FusedKernel fused;
    size_t smem;
    int bwd_threads;   /* one block per node step: lqr_nt<NXP>() */
};

Instance instance(int nx, int nu) {
    if (nx <= 8 && nu <= 4)
        return {lqr_backward_kernel<8, 4, 1>, lqr_backward_kernel<8, 4, 8>, lqr_forward_kernel<8, 4>,
                lqr_fused_kernel<8, 4>, backward_smem<8, 4>(), lqr_nt<8>()};
    if (nx <= 16 && nu <= 8)
        return {lqr_backward_kernel<16, 8, 1>, lqr_backward_kernel<16, 8, 6>, lqr_forward_kernel<16, 8>,
                lqr_fused_kernel<16, 8>, backward_smem<16, 8>(), lqr_nt<16>()};
    return {lqr_backward_kernel<32, 16, 1>, lqr_backward_kernel<32, 16, 2>, lqr_forward_kernel<32, 16>,
            lqr_fused_kernel<32, 16>, backward_smem<32, 16>(), lqr_nt<32>()};
}

}  // namespace

struct bmpc_lqr {
    int n = 0, nx = 0, nu = 0, batch = 0;
    std::vector<int> sstart;   /* stage s holds nodes [sstart[s], sstart[s + 1]) */
    int32_t *d_child_idx = nullptr, *d_flag = nullptr, *d_sstart = nullptr;
    int4 *d_node4 = nullptr, *d_plan = nullptr;   /* d_plan: the post-order of the one-block-per-problem schedule */
    int schedule = 0;   /* 0: by the cost model, 1: a launch per stage and sweep, 2: one block per problem */
    int sm_count = 148;
    int occ_fused = 1, occ_wide = 1;   /* resident blocks per SM of the fused and the wide-stage kernels */
    cudaStream_t stream = nullptr;
    Instance inst{};
};

namespace {
/* The schedule: per-stage launches expose every node of a stage at once; one block per problem saves
 * the launches but walks each tree's nodes one after another.  Cost model in node-step units, a
 * launch worth half a node step, with the blocks each kernel keeps resident per SM (o_w for the
 * wide-stage backward kernel, o_f for the fused one):
 *   per stage:  sum_s (ceil(width_s * batch / (o_w SMs)) + 1/2),   fused:  ceil(batch / (o_f SMs)) * n. */
bool fused_schedule(const bmpc_lqr *h) {
    if (h->schedule) return h->schedule == 2;
    const double slots_w = (double)h->occ_wide * h->sm_count, slots_f = (double)h->occ_fused * h->sm_count;
    double staged = 0.0;
    for (size_t s = 0; s + 1 < h->sstart.size(); ++s)
        staged += std::ceil((double)(h->sstart[s + 1] - h->sstart[s]) * h->batch / slots_w) + 0.5;
    return std::ceil(h->batch / slots_f) * h->n <= staged;
}
}  // namespace

extern "C" {

int bmpc_lqr_create(int32_t n, const int32_t *parent, int32_t nx, int32_t nu, int32_t batch, void *stream,
                    bmpc_lqr **out) {
    if (!out) return BMPC_ERR_INVALID;
    *out = nullptr;
    if (n < 1 || !parent || nx < 1 || nx > 32 || nu < 1 || nu > 16 || batch < 1) return BMPC_ERR_INVALID;
    if ((long long)n * batch * 32 * 32 > (1ll << 40)) return BMPC_ERR_INVALID;
    if (parent[0] != -1) return BMPC_ERR_INVALID;
    std::vector<int> stage(n, 0), nchild(n, 0);
    for (int i = 1; i < n; ++i) {
        if (parent[i] < 0 || parent[i] >= i) return BMPC_ERR_INVALID;
        stage[i] = stage[parent[i]] + 1;
        if (stage[i] < stage[i - 1]) return BMPC_ERR_INVALID;   /* level order */
        ++nchild[parent[i]];
    }
    bmpc_lqr *h = new (std::nothrow) bmpc_lqr();
    if (!h) return BMPC_ERR_SPACE;
    h->n = n;
    h->nx = nx;
    h->nu = nu;
    h->batch = batch;
    h->stream = static_cast<cudaStream_t>(stream);
    const int S = stage[n - 1] + 1;
    h->sstart.assign(S + 1, n);
    for (int i = n - 1; i >= 0; --i) h->sstart[stage[i]] = i;
    std::vector<int32_t> off(n + 1, 0), idx(std::max(1, n - 1)), fill(n, 0);
    for (int i = 0; i < n; ++i) off[i + 1] = off[i] + nchild[i];
    for (int i = 1; i < n; ++i) idx[off[parent[i]] + fill[parent[i]]++] = i;   /* ascending child ids */
    h->inst = instance(nx, nu);
    std::vector<int4> node4(n);
    for (int i = 0; i < n; ++i) node4[i] = make_int4(off[i], off[i + 1], nchild[i] ? idx[off[i + 1] - 1] : -1, parent[i]);
    /* post-order, children in ascending order: a node comes right after its last child */
    std::vector<int4> plan;
    plan.reserve(n);
    std::vector<std::pair<int, int>> dfs{{0, off[0]}};
    while (!dfs.empty()) {
        const int v = dfs.back().first;
        if (dfs.back().second < off[v + 1]) {
            const int ch = idx[dfs.back().second++];
            dfs.push_back({ch, off[ch]});
        } else {
            plan.push_back(make_int4(v, node4[v].x, node4[v].y, node4[v].z));
            dfs.pop_back();
        }
    }
    bool ok = cudaMalloc(&h->d_node4, sizeof(int4) * n) == cudaSuccess &&
              cudaMalloc(&h->d_plan, sizeof(int4) * n) == cudaSuccess &&
              cudaMalloc(&h->d_sstart, sizeof(int32_t) * h->sstart.size()) == cudaSuccess &&
              cudaMalloc(&h->d_child_idx, sizeof(int32_t) * idx.size()) == cudaSuccess &&
              cudaMalloc(&h->d_flag, sizeof(int32_t)) == cudaSuccess;
    ok = ok && cudaMemcpy(h->d_node4, node4.data(), sizeof(int4) * n, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(h->d_plan, plan.data(), sizeof(int4) * n, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(h->d_sstart, h->sstart.data(), sizeof(int32_t) * h->sstart.size(), cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemcpy(h->d_child_idx, idx.data(), sizeof(int32_t) * idx.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(h->d_flag, 0, sizeof(int32_t)) == cudaSuccess;
    int dev = 0;
    ok = ok && cudaGetDevice(&dev) == cudaSuccess &&
         cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(h->inst.bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->inst.smem) ==
                   cudaSuccess;
    ok = ok && cudaFuncSetAttribute(h->inst.bwd_wide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)h->inst.smem) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(h->inst.fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->inst.smem) ==
                   cudaSuccess;
    ok = ok && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occ_fused, h->inst.fused, h->inst.bwd_threads,
                                                             h->inst.smem) == cudaSuccess &&
         cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occ_wide, h->inst.bwd_wide, h->inst.bwd_threads,
                                                       h->inst.smem) == cudaSuccess;
    h->occ_fused = std::max(1, h->occ_fused);
    h->occ_wide = std::max(1, h->occ_wide);
    if (!ok) {
        bmpc_lqr_destroy(h);
        return BMPC_ERR_CUDA;
    }
    *out = h;
    return BMPC_OK;
}

int bmpc_lqr_solve(bmpc_lqr *h, const float *Q, const float *M, const float *R, const float *q, const float *r,
                   const float *A, const float *B, const float *c, const float *x0, float *K, float *k, float *P,
                   float *p, float *x, float *u, float *lam) {
    if (!h || !Q || !R || !q || !r || !A || !B || !c || !x0 || !K || !k || !P || !p || !x || !u || !lam)
        return BMPC_ERR_INVALID;
    LqrArgs a{Q, M, R, q, r, A, B, c, x0, K, k, P, p, x, u, lam, h->d_child_idx, h->d_node4,
              h->d_flag, h->n, h->nx, h->nu, h->batch, 0, 0};
    const int S = (int)h->sstart.size() - 1;
    if (fused_schedule(h)) {
        h->inst.fused<<<(unsigned)h->batch, h->inst.bwd_threads, h->inst.smem, h->stream>>>(a, h->d_plan, h->d_sstart, S);
        return cudaGetLastError() == cudaSuccess ? BMPC_OK : BMPC_ERR_CUDA;
    }
    auto grid = [&](int cnt) { return (unsigned)(((long long)cnt * h->batch + LQR_WARPS - 1) / LQR_WARPS); };
    for (int s = S - 1; s >= 0; --s) {
        a.s0 = h->sstart[s];
        a.cnt = h->sstart[s + 1] - h->sstart[s];
        const long long blocks = (long long)a.cnt * h->batch;
        (blocks > h->sm_count ? h->inst.bwd_wide : h->inst.bwd)<<<(unsigned)blocks, h->inst.bwd_threads, h->inst.smem,
                                                                  h->stream>>>(a);
    }
    for (int s = 0; s < S; ++s) {
        a.s0 = h->sstart[s];
        a.cnt = h->sstart[s + 1] - h->sstart[s];
        h->inst.fwd<<<grid(a.cnt), 32 * LQR_WARPS, 0, h->stream>>>(a);
    }
    return cudaGetLastError() == cudaSuccess ? BMPC_OK : BMPC_ERR_CUDA;
}

int bmpc_lqr_status(bmpc_lqr *h) {
    if (!h) return BMPC_ERR_INVALID;
    int32_t f = 0;
    if (cudaMemcpyAsync(&f, h->d_flag, sizeof f, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->d_flag, 0, sizeof(int32_t), h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return BMPC_ERR_CUDA;
    return f ? BMPC_ERR_NUMERIC : BMPC_OK;
}

int bmpc_lqr_stages(const bmpc_lqr *h) { return h ? (int)h->sstart.size() - 1 : BMPC_ERR_INVALID; }

int bmpc_lqr_set_schedule(bmpc_lqr *h, int32_t schedule) {
    if (!h || schedule < 0 || schedule > 2) return BMPC_ERR_INVALID;
    h->schedule = schedule;
    return BMPC_OK;
}

int bmpc_lqr_fused(const bmpc_lqr *h) { return h ? (int)fused_schedule(h) : BMPC_ERR_INVALID; }

void bmpc_lqr_destroy(bmpc_lqr *h) {
    if (!h) return;
    cudaFree(h->d_node4);
    cudaFree(h->d_plan);
    cudaFree(h->d_sstart);
    cudaFree(h->d_child_idx);
    cudaFree(h->d_flag);
    delete h;
}

}  // extern "C"
