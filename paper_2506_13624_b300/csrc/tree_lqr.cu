/* Tree LQR at general sizes with per-edge dynamics: Eq. (lqr_tree_approx) by the tree Riccati
 * recursion of Eq. (tree_Riccati) and the feedback laws of Eq. (tree_feedback_laws), then the
 * forward sweep of Sec. III-A.  The C ABI and the problem statement are in include/bmpc_lqr.h.
 *
 * Layout of the work: one launch per stage and sweep.  Backward, a block of NXP / 4 warps owns one
 * node of the stage (of one problem of the batch): thread (lane l, warp w) owns entries
 * (l, 4w .. 4w + 3) of the node's matrix products, so a node step is a set of short dot products
 * over shared-memory tiles, with the tree's depth as the only sequential chain:
 *   per child edge m:  T1 = P_m A_m, T2 = P_m B_m, g = p_m + P_m c_m
 *                      S_xx += A_m' T1, S_xu += A_m' T2, S_uu += B_m' T2, s_x += A_m' g, s_u += B_m' g
 *   node:              H = R + S_uu (Cholesky by one warp), [K k] = -H^-1 [M + S_xu' | r + s_u]
 *                      (thread c: right-hand side c), P = Q + S_xx + S_ux' K, p = q + s_x + S_ux' k
 * Forward, one warp per node (lane j: row j of x_m = A_m x_p + B_m u_p + c_m, then u and lam).
 * Tiles are zero-padded to NXP x NXP (NXP in {8, 16, 32}) and NUP (in {4, 8, 16}) so that every
 * loop is unrolled at compile time; the tile rows that many threads read in common are fetched as
 * 16-byte broadcasts.  FP32 throughout (the paper's batch experiments run FP32 too). */
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "bmpc.h"
#include "bmpc_lqr.h"

namespace {

constexpr int LQR_WARPS = 4;   /* nodes per block of the forward sweep */
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
 * hit distinct banks). */
template <int NXP, int NUP>
struct LqrTiles {
    static constexpr int SX = NXP + 4, SU = NUP + 4;
    float A[NXP][SX];    /* the edge's A_m */
    float B[NXP][SU];    /* the edge's B_m */
    float PS[NXP][SX];   /* the child's P_m */
    float T1[NXP][SX];   /* P_m A_m; later the node's P before symmetrisation */
    float T2[NXP][SU];   /* P_m B_m */
    float H[NUP][SU];    /* H, then its Cholesky factor (lower triangle) */
    float X[NUP][SX];    /* [Q_ux | q_u] with q_u in column NXP, then [K | k] */
    float QUX[NUP][SX];  /* Q_ux, kept for P and p */
    float g[NXP];        /* p_m + P_m c_m */
    float cv[NXP];       /* c_m */
    float qx[NXP];       /* q + s_x */
    float id[NUP];       /* 1 / L_bb (0 past n_u) */
};

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

/* Stage a rows x cols row-major global matrix into a zero-padded tile of R x C (stride S), the
 * `nt` threads of the block striding over its entries. */
template <int R, int C, int S>
__device__ __forceinline__ void stage_tile(float (*T)[S], const float *g, int rows, int cols, int tid, int nt) {
    for (int idx = tid; idx < R * C; idx += nt) {
        const int a = idx / C, b = idx % C;
        T[a][b] = (a < rows && b < cols) ? g[(size_t)a * cols + b] : 0.f;
    }
}

/* The same with the thread count NT known at compile time: every load is issued before the first
 * store, so the tile costs one memory latency instead of one per round. */
template <int R, int C, int S, int NT>
__device__ __forceinline__ void stage_tile_nt(float (*T)[S], const float *g, int rows, int cols, int tid) {
    constexpr int IT = (R * C + NT - 1) / NT;
    float v[IT];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int idx = tid + it * NT, a = idx / C, b = idx % C;
        v[it] = (idx < R * C && a < rows && b < cols) ? g[(size_t)a * cols + b] : 0.f;
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int idx = tid + it * NT;
        if (idx < R * C) T[idx / C][idx % C] = v[it];
    }
}

__device__ __forceinline__ void fma4(float4 &acc, float s, const float4 v) {
    acc.x += s * v.x;
    acc.y += s * v.y;
    acc.z += s * v.z;
    acc.w += s * v.w;
}

/* Backward step of node i of problem t by the whole block: NXP / 4 warps; thread (lane l, warp w)
 * owns entries (l, 4w .. 4w + 3) of the n_x-column products and, for w < NUP / 4, of the n_u-column
 * ones.  Every thread of the block calls it with the same (t, i). */
template <int NXP, int NUP>
__device__ __forceinline__ void backward_node(const LqrArgs &a, int t, int i) {
    constexpr int NW = NXP / 4, NWU = NUP / 4;
    extern __shared__ __align__(16) float lqr_smem[];
    using Tiles = LqrTiles<NXP, NUP>;
    Tiles *ts = reinterpret_cast<Tiles *>(lqr_smem);
    const int tid = threadIdx.x, nt = blockDim.x, l = tid & 31, w = tid >> 5;
    const int j0 = 4 * w;   /* this thread's column group */
    const int nx = a.nx, nu = a.nu;
    const size_t node = (size_t)t * a.n + i;
    const float *Qi = a.Q + node * nx * nx;
    float *Pi = a.P + node * nx * nx, *Ki = a.K + node * nu * nx;
    const int4 nd = a.node4[i];   /* one load gives the child range and the first child */
    const int c0 = nd.x, c1 = nd.y;
    const bool row = l < nx && l < NXP;

    if (c0 == c1) {   /* leaf: P = sym(Q), p = q, no law */
        if (row)
            for (int j = j0; j < j0 + 4 && j < nx; ++j)
                Pi[(size_t)j * nx + l] = 0.5f * (Qi[(size_t)j * nx + l] + Qi[(size_t)l * nx + j]);
        if (w == 0 && row) a.p[node * nx + l] = a.q[node * nx + l];
        for (int e = tid; e < nu * nx; e += nt) Ki[e] = 0.f;
        if (tid < nu) a.k[node * nu + tid] = 0.f;
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
    for (int e = c0; e < c1; ++e) {
        const int m = e == c0 ? nd.z : a.child_idx[e];
        const size_t cm = (size_t)t * a.n + m;
        __syncthreads();   /* the previous child's tiles are no longer read */
        stage_tile_nt<NXP, NXP, Tiles::SX, 8 * NXP>(ts->A, a.A + cm * nx * nx, nx, nx, tid);
        stage_tile_nt<NXP, NUP, Tiles::SU, 8 * NXP>(ts->B, a.B + cm * nx * nu, nx, nu, tid);
        stage_tile_nt<NXP, NXP, Tiles::SX, 8 * NXP>(ts->PS, a.P + cm * nx * nx, nx, nx, tid);
        if (tid < NXP) ts->cv[tid] = tid < nx ? a.c[cm * nx + tid] : 0.f;
        __syncthreads();
        /* T1 = P_m A_m (and T2 = P_m B_m for w < NUP / 4): entries (l, 4w .. 4w + 3) */
        if (l < NXP) {
            float4 t1 = make_float4(0.f, 0.f, 0.f, 0.f), t2 = t1;
            float gl = 0.f;
#pragma unroll
            for (int k4 = 0; k4 < NXP; k4 += 4) {
                const float4 p4 = ld4(&ts->PS[l][k4]);
                const float pk[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    fma4(t1, pk[s], ld4(&ts->A[k4 + s][j0]));
                    if (w < NWU) fma4(t2, pk[s], ld4(&ts->B[k4 + s][j0]));
                    if (w == NW - 1) gl += pk[s] * ts->cv[k4 + s];
                }
            }
            st4(&ts->T1[l][j0], t1);
            if (w < NWU) st4(&ts->T2[l][j0], t2);
            if (w == NW - 1) ts->g[l] = (l < nx ? a.p[cm * nx + l] : 0.f) + gl;
        }
        __syncthreads();
        /* S_xx += A' T1, S_xu += A' T2, S_uu += B' T2 at (l, 4w ..); s_x += A' g, s_u += B' g (warp NW - 1) */
        if (l < NXP) {
#pragma unroll 8
            for (int kk = 0; kk < NXP; ++kk) {
                const float akl = ts->A[kk][l];
                fma4(sxx, akl, ld4(&ts->T1[kk][j0]));
                if (w < NWU) {
                    const float4 t2 = ld4(&ts->T2[kk][j0]);
                    fma4(sxu, akl, t2);
                    if (l < NUP) fma4(suu, ts->B[kk][l], t2);
                }
                if (w == NW - 1) {
                    sx += akl * ts->g[kk];
                    if (l < NUP) su += ts->B[kk][l] * ts->g[kk];
                }
            }
        }
    }
    __syncthreads();

    /* the node's own terms: Q_xx (l, 4w ..) in registers, Q_ux into X and QUX, H, q_u, q_x */
    for (int idx = tid; idx < NUP * Tiles::SX; idx += nt) (&ts->X[0][0])[idx] = 0.f;
    __syncthreads();
    float4 qxx = sxx;
    qxx.x += qr4[0];
    qxx.y += qr4[1];
    qxx.z += qr4[2];
    qxx.w += qr4[3];
    if (l < NXP && w < NWU) {
        const float s4[4] = {sxu.x, sxu.y, sxu.z, sxu.w};
        const float h4[4] = {suu.x, suu.y, suu.z, suu.w};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int b = j0 + s;
            const float v = (row && b < nu) ? mv4[s] + s4[s] : 0.f;
            ts->X[b][l] = v;
            ts->QUX[b][l] = v;
            if (l < NUP) ts->H[l][b] = (l < nu && b < nu) ? rv4[s] + h4[s] : 0.f;
        }
    }
    if (w == NW - 1 && l < NXP) {
        ts->qx[l] = row ? qv + sx : 0.f;
        if (l < nu) ts->X[l][NXP] = rv + su;
    }
    __syncthreads();

    /* Cholesky H = L L' by warp 0 in registers: lane l holds row l, columns broadcast by shuffles
     * (rows and columns past n_u are zero and stay zero) */
    if (w == 0) {
        float h[NUP];
#pragma unroll
        for (int b = 0; b < NUP; ++b) h[b] = l < NUP ? ts->H[l][b] : 0.f;
        bool bad = false;
#pragma unroll
        for (int j = 0; j < NUP; ++j) {
            if (j < nu) {
                const float d = __shfl_sync(FULL, h[j], j);
                bad = bad || !(d > 0.f) || !isfinite(d);
                const float ljj = sqrtf(d), il = 1.f / ljj;
                if (l == j) h[j] = ljj;
                else if (l > j) h[j] *= il;
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
            ts->id[l] = l < nu ? 1.f / h[l] : 0.f;
        }
        if (bad && l == 0) atomicExch(a.flag, 1);
    }
    __syncthreads();

    /* [K k] = -H^-1 [Q_ux | q_u]: thread c solves right-hand side c (c = nx is q_u, in column NXP);
     * the zero padding of L and 1/L_bb makes the unguarded substitutions exact past n_u */
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

    /* P = Q_xx + Q_ux' K at (l, 4w ..) into T1; p = q_x + Q_ux' k (warp NW - 1) */
    if (l < NXP) {
        float4 pv = qxx;
        float pl = ts->qx[l];
#pragma unroll
        for (int b = 0; b < NUP; ++b) {
            const float qb = ts->QUX[b][l];
            fma4(pv, qb, ld4(&ts->X[b][j0]));
            if (w == NW - 1) pl += qb * ts->X[b][NXP];
        }
        st4(&ts->T1[l][j0], pv);
        if (w == NW - 1 && row) a.p[node * nx + l] = pl;
    }
    __syncthreads();
    if (row)
        for (int j = j0; j < j0 + 4 && j < nx; ++j) Pi[(size_t)j * nx + l] = 0.5f * (ts->T1[l][j] + ts->T1[j][l]);
    if (row)
        for (int b = w; b < nu; b += NW) Ki[(size_t)b * nx + l] = ts->X[b][l];
    if (tid < nu) a.k[node * nu + tid] = ts->X[tid][NXP];
}

/* One backward launch per stage: block b is node s0 + b % cnt of problem b / cnt. */
template <int NXP, int NUP, int MINB>
__global__ void __launch_bounds__(8 * NXP, MINB) lqr_backward_kernel(LqrArgs a) {
    const long long item = blockIdx.x;
    backward_node<NXP, NUP>(a, (int)(item / a.cnt), a.s0 + (int)(item % a.cnt));
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

/* The whole solve of problem t = blockIdx.x in one block: the backward steps of all nodes, stage by
 * stage from the leaves (one node at a time, the block on each), then the forward steps (the warps
 * sharing each stage's nodes).  No block waits on another: problems are independent.  For trees
 * whose stages are narrow, where the per-stage launches would leave the GPU idle between them. */
template <int NXP, int NUP>
__global__ void __launch_bounds__(8 * NXP) lqr_fused_kernel(LqrArgs a, const int32_t *sstart, int S) {
    constexpr int NW = NXP / 4;
    const int t = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int s = S - 1; s >= 0; --s)
        for (int i = sstart[s]; i < sstart[s + 1]; ++i) {
            backward_node<NXP, NUP>(a, t, i);
            __syncthreads();   /* the node's P, p reach the parent's step; the tiles are free again */
        }
    for (int s = 0; s < S; ++s) {
        for (int i = sstart[s] + w; i < sstart[s + 1]; i += NW) forward_node<NXP, NUP>(a, t, i, lane);
        __syncthreads();
    }
}

template <int NXP, int NUP>
size_t backward_smem() { return sizeof(LqrTiles<NXP, NUP>); }

using LqrKernel = void (*)(LqrArgs);
using FusedKernel = void (*)(LqrArgs, const int32_t *, int);
struct Instance {
    LqrKernel bwd, bwd_wide, fwd;   /* bwd_wide: two blocks per SM, for stages wider than the GPU */
    FusedKernel fused;
    size_t smem;
    int bwd_threads;   /* one block per node: NXP / 4 warps */
};

Instance instance(int nx, int nu) {
    if (nx <= 8 && nu <= 4)
        return {lqr_backward_kernel<8, 4, 1>, lqr_backward_kernel<8, 4, 4>, lqr_forward_kernel<8, 4>,
                lqr_fused_kernel<8, 4>, backward_smem<8, 4>(), 64};
    if (nx <= 16 && nu <= 8)
        return {lqr_backward_kernel<16, 8, 1>, lqr_backward_kernel<16, 8, 3>, lqr_forward_kernel<16, 8>,
                lqr_fused_kernel<16, 8>, backward_smem<16, 8>(), 128};
    return {lqr_backward_kernel<32, 16, 1>, lqr_backward_kernel<32, 16, 2>, lqr_forward_kernel<32, 16>,
            lqr_fused_kernel<32, 16>, backward_smem<32, 16>(), 256};
}

}  // namespace

struct bmpc_lqr {
    int n = 0, nx = 0, nu = 0, batch = 0;
    std::vector<int> sstart;   /* stage s holds nodes [sstart[s], sstart[s + 1]) */
    int32_t *d_child_idx = nullptr, *d_flag = nullptr, *d_sstart = nullptr;
    int4 *d_node4 = nullptr;
    int schedule = 0;   /* 0: by the cost model, 1: a launch per stage and sweep, 2: one block per problem */
    int sm_count = 148;
    cudaStream_t stream = nullptr;
    Instance inst{};
};

namespace {
/* The schedule: per-stage launches expose every node of a stage at once; one block per problem saves
 * the launches but walks each tree's nodes one after another.  Cost model in node-step units, two
 * blocks resident per SM, a launch worth half a node step:
 *   per stage:  sum_s (ceil(width_s * batch / (2 SMs)) + 1/2),   fused:  ceil(batch / (2 SMs)) * n. */
bool fused_schedule(const bmpc_lqr *h) {
    if (h->schedule) return h->schedule == 2;
    const double slots = 2.0 * h->sm_count;
    double staged = 0.0;
    for (size_t s = 0; s + 1 < h->sstart.size(); ++s)
        staged += std::ceil((double)(h->sstart[s + 1] - h->sstart[s]) * h->batch / slots) + 0.5;
    return std::ceil(h->batch / slots) * h->n <= staged;
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
    for (int i = 0; i < n; ++i) node4[i] = make_int4(off[i], off[i + 1], nchild[i] ? idx[off[i]] : -1, parent[i]);
    bool ok = cudaMalloc(&h->d_node4, sizeof(int4) * n) == cudaSuccess &&
              cudaMalloc(&h->d_sstart, sizeof(int32_t) * h->sstart.size()) == cudaSuccess &&
              cudaMalloc(&h->d_child_idx, sizeof(int32_t) * idx.size()) == cudaSuccess &&
              cudaMalloc(&h->d_flag, sizeof(int32_t)) == cudaSuccess;
    ok = ok && cudaMemcpy(h->d_node4, node4.data(), sizeof(int4) * n, cudaMemcpyHostToDevice) == cudaSuccess &&
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
        h->inst.fused<<<(unsigned)h->batch, h->inst.bwd_threads, h->inst.smem, h->stream>>>(a, h->d_sstart, S);
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
    cudaFree(h->d_sstart);
    cudaFree(h->d_child_idx);
    cudaFree(h->d_flag);
    delete h;
}

}  // extern "C"
