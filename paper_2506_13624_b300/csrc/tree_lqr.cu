/* Tree LQR at general sizes with per-edge dynamics: Eq. (lqr_tree_approx) by the tree Riccati
 * recursion of Eq. (tree_Riccati) and the feedback laws of Eq. (tree_feedback_laws), then the
 * forward sweep of Sec. III-A.  The C ABI and the problem statement are in include/bmpc_lqr.h.
 *
 * Layout of the work: one launch per stage and sweep.  In a launch every warp owns one node of the
 * stage (of one problem of the batch); lane j owns row j of the node's n_x x n_x matrices (the
 * child value function P_m, the sums A'PA, and the new P), so a node step is a set of per-lane dot
 * products over shared-memory tiles:
 *   per child edge m:  T1 = P_m A_m, T2 = P_m B_m, g = p_m + P_m c_m           (lane j: row j)
 *                      S_xx += A_m' T1, S_xu += A_m' T2, S_uu += B_m' T2,
 *                      s_x += A_m' g, s_u += B_m' g                              (lane j: row j)
 *   node:              H = R + S_uu (Cholesky across the warp), [K k] = -H^-1 [M + S_xu' | r + s_u]
 *                      (lane c: right-hand side c), P = Q + S_xx + S_ux' K, p = q + s_x + S_ux' k
 * Tiles are zero-padded to NXP x NXP (NXP in {8, 16, 32}) and NUP (in {4, 8, 16}) so that every
 * loop is unrolled at compile time; the rows of the tiles that the lanes read in common are
 * fetched as 16-byte broadcasts.  FP32 throughout (the paper's batch experiments run FP32 too). */
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "bmpc.h"
#include "bmpc_lqr.h"

namespace {

constexpr int LQR_WARPS = 4;   /* nodes per block */
constexpr unsigned FULL = 0xffffffffu;

struct LqrArgs {
    const float *Q, *M, *R, *q, *r, *A, *B, *c, *x0;
    float *K, *k, *P, *p, *x, *u, *lam;
    const int32_t *parent, *child_off, *child_idx;
    int32_t *flag;
    int n, nx, nu, batch;
    int s0, cnt;   /* first node of the stage and its node count */
};

/* Per-warp shared tiles; row strides are multiples of 4 floats (16-byte rows for the broadcast
 * reads) and 4 more than the columns (stores of 16 bytes by 8 lanes at a time hit distinct banks). */
template <int NXP, int NUP>
struct LqrTiles {
    static constexpr int SX = NXP + 4, SU = NUP + 4;
    float A[NXP][SX];   /* the edge's A_m */
    float B[NXP][SU];   /* the edge's B_m */
    float T1[NXP][SX];  /* P_m A_m; later the node's P before symmetrisation */
    float T2[NXP][SU];  /* P_m B_m */
    float H[NUP][SU];   /* H, then its Cholesky factor (lower triangle) */
    float X[NUP][SX];   /* [Q_ux | q_u] with q_u in column NXP, then [K | k] */
    float g[NXP];       /* p_m + P_m c_m */
};

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float a, float b, float c, float d) {
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}

/* Stage a rows x cols row-major global matrix into a zero-padded tile of R x C (stride S). */
template <int R, int C, int S>
__device__ __forceinline__ void stage_tile(float (*T)[S], const float *g, int rows, int cols, int lane) {
    for (int idx = lane; idx < R * C; idx += 32) {
        const int a = idx / C, b = idx % C;
        T[a][b] = (a < rows && b < cols) ? g[(size_t)a * cols + b] : 0.f;
    }
}

template <int NXP, int NUP>
__global__ void __launch_bounds__(32 * LQR_WARPS) lqr_backward_kernel(LqrArgs a) {
    extern __shared__ __align__(16) float lqr_smem[];
    using Tiles = LqrTiles<NXP, NUP>;
    Tiles *ws = reinterpret_cast<Tiles *>(lqr_smem) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    const long long item = (long long)blockIdx.x * LQR_WARPS + threadIdx.x / 32;
    if (item >= (long long)a.cnt * a.batch) return;   /* the whole warp leaves together */
    const int t = (int)(item / a.cnt);
    const int i = a.s0 + (int)(item % a.cnt);
    const int nx = a.nx, nu = a.nu;
    const size_t node = (size_t)t * a.n + i;
    const float *Qi = a.Q + node * nx * nx;
    float *Pi = a.P + node * nx * nx, *Ki = a.K + node * nu * nx;
    const int c0 = a.child_off[i], c1 = a.child_off[i + 1];
    const bool row = lane < nx;

    if (c0 == c1) {   /* leaf: P = sym(Q), p = q, no law */
        if (row) {
            for (int j = 0; j < nx; ++j) Pi[(size_t)j * nx + lane] = 0.5f * (Qi[(size_t)j * nx + lane] + Qi[(size_t)lane * nx + j]);
            a.p[node * nx + lane] = a.q[node * nx + lane];
        }
        for (int e = lane; e < nu * nx; e += 32) Ki[e] = 0.f;
        if (lane < nu) a.k[node * nu + lane] = 0.f;
        return;
    }

    /* the k loops of the A'T sums are unrolled by 2 at n_x = 32: fully unrolled they spill */
    constexpr int KK_UNROLL = NXP > 16 ? 2 : NXP;
    float sxx[NXP], sxu[NUP], suu[NUP], sx = 0.f, su = 0.f;
#pragma unroll
    for (int j = 0; j < NXP; ++j) sxx[j] = 0.f;
#pragma unroll
    for (int j = 0; j < NUP; ++j) sxu[j] = suu[j] = 0.f;

    for (int e = c0; e < c1; ++e) {
        const int m = a.child_idx[e];
        const size_t cm = (size_t)t * a.n + m;
        __syncwarp();   /* the previous child's tiles are no longer read */
        stage_tile<NXP, NXP, Tiles::SX>(ws->A, a.A + cm * nx * nx, nx, nx, lane);
        stage_tile<NXP, NUP, Tiles::SU>(ws->B, a.B + cm * nx * nu, nx, nu, lane);
        /* row `lane` of P_m (symmetric: its column, read coalesced), p_m and c_m */
        const float *Pm = a.P + cm * nx * nx;
        float prow[NXP];
#pragma unroll
        for (int kk = 0; kk < NXP; ++kk) prow[kk] = (row && kk < nx) ? Pm[(size_t)kk * nx + lane] : 0.f;
        const float cl = row ? a.c[cm * nx + lane] : 0.f;
        float gl = row ? a.p[cm * nx + lane] : 0.f;
#pragma unroll
        for (int kk = 0; kk < NXP; ++kk) gl += prow[kk] * __shfl_sync(FULL, cl, kk);
        if (lane < NXP) ws->g[lane] = gl;
        __syncwarp();
        /* T1 = P_m A_m, T2 = P_m B_m: row `lane` */
        if (lane < NXP) {
#pragma unroll
            for (int j = 0; j < NXP; j += 4) {
                float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
#pragma unroll
                for (int kk = 0; kk < NXP; ++kk) {
                    const float4 a4 = ld4(&ws->A[kk][j]);
                    v0 += prow[kk] * a4.x;
                    v1 += prow[kk] * a4.y;
                    v2 += prow[kk] * a4.z;
                    v3 += prow[kk] * a4.w;
                }
                st4(&ws->T1[lane][j], v0, v1, v2, v3);
            }
#pragma unroll
            for (int j = 0; j < NUP; j += 4) {
                float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
#pragma unroll
                for (int kk = 0; kk < NXP; ++kk) {
                    const float4 b4 = ld4(&ws->B[kk][j]);
                    v0 += prow[kk] * b4.x;
                    v1 += prow[kk] * b4.y;
                    v2 += prow[kk] * b4.z;
                    v3 += prow[kk] * b4.w;
                }
                st4(&ws->T2[lane][j], v0, v1, v2, v3);
            }
        }
        __syncwarp();
        /* S_xx += A' T1, S_xu += A' T2, s_x += A' g (row `lane`); S_uu += B' T2, s_u += B' g (rows < NUP) */
        if (lane < NXP) {
#pragma unroll(KK_UNROLL)
            for (int kk = 0; kk < NXP; ++kk) {
                const float akl = ws->A[kk][lane];
#pragma unroll
                for (int j = 0; j < NXP; j += 4) {
                    const float4 t4 = ld4(&ws->T1[kk][j]);
                    sxx[j] += akl * t4.x;
                    sxx[j + 1] += akl * t4.y;
                    sxx[j + 2] += akl * t4.z;
                    sxx[j + 3] += akl * t4.w;
                }
#pragma unroll
                for (int j = 0; j < NUP; j += 4) {
                    const float4 t4 = ld4(&ws->T2[kk][j]);
                    sxu[j] += akl * t4.x;
                    sxu[j + 1] += akl * t4.y;
                    sxu[j + 2] += akl * t4.z;
                    sxu[j + 3] += akl * t4.w;
                }
                sx += akl * ws->g[kk];
            }
        }
        if (lane < NUP) {
#pragma unroll(KK_UNROLL)
            for (int kk = 0; kk < NXP; ++kk) {
                const float bkl = ws->B[kk][lane];
#pragma unroll
                for (int j = 0; j < NUP; j += 4) {
                    const float4 t4 = ld4(&ws->T2[kk][j]);
                    suu[j] += bkl * t4.x;
                    suu[j + 1] += bkl * t4.y;
                    suu[j + 2] += bkl * t4.z;
                    suu[j + 3] += bkl * t4.w;
                }
                su += bkl * ws->g[kk];
            }
        }
    }
    __syncwarp();

    /* the node's own terms: Q_xx (row `lane`), q_x; Q_ux column `lane` into X, H and q_u (rows < nu) */
    float qux[NUP];
#pragma unroll
    for (int b = 0; b < NUP; ++b) {
        const float mv = (a.M && row && b < nu) ? a.M[node * nu * nx + (size_t)b * nx + lane] : 0.f;
        qux[b] = (row && b < nu) ? mv + sxu[b] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < NXP; ++j) sxx[j] = (row && j < nx) ? Qi[(size_t)lane * nx + j] + sxx[j] : 0.f;
    const float qx = row ? a.q[node * nx + lane] + sx : 0.f;
    for (int idx = lane; idx < NUP * Tiles::SX; idx += 32) (&ws->X[0][0])[idx] = 0.f;
    __syncwarp();
    if (lane < NXP) {
#pragma unroll
        for (int b = 0; b < NUP; ++b) ws->X[b][lane] = qux[b];
    }
    if (lane < nu) {
        const float *Ri = a.R + node * nu * nu;
#pragma unroll
        for (int b = 0; b < NUP; ++b) ws->H[lane][b] = b < nu ? Ri[(size_t)lane * nu + b] + suu[b] : 0.f;
        ws->X[lane][NXP] = a.r[node * nu + lane] + su;
    }
    __syncwarp();

    /* Cholesky H = L L' in place (lower triangle), one column at a time across the warp */
    bool bad = false;
    for (int j = 0; j < nu; ++j) {
        const float d = ws->H[j][j];
        bad = bad || !(d > 0.f) || !isfinite(d);
        const float ljj = sqrtf(d), il = 1.f / ljj;
        __syncwarp();
        if (lane > j && lane < nu) ws->H[lane][j] *= il;
        if (lane == j) ws->H[j][j] = ljj;
        __syncwarp();
        if (lane > j && lane < nu) {
            const float lij = ws->H[lane][j];
            for (int b = j + 1; b <= lane; ++b) ws->H[lane][b] -= lij * ws->H[b][j];
        }
        __syncwarp();
    }
    if (bad && lane == 0) atomicExch(a.flag, 1);

    /* [K k] = -H^-1 [Q_ux | q_u]: lane c solves right-hand side c (c = nx is q_u, kept in column NXP) */
    for (int cidx = lane; cidx <= nx; cidx += 32) {
        const int col = cidx < nx ? cidx : NXP;
        float y[NUP];
#pragma unroll
        for (int b = 0; b < NUP; ++b) y[b] = b < nu ? ws->X[b][col] : 0.f;
#pragma unroll
        for (int b = 0; b < NUP; ++b)
            if (b < nu) {
                float s = y[b];
#pragma unroll
                for (int e = 0; e < b; ++e) s -= ws->H[b][e] * y[e];
                y[b] = s / ws->H[b][b];
            }
#pragma unroll
        for (int b = NUP - 1; b >= 0; --b)
            if (b < nu) {
                float s = y[b];
#pragma unroll
                for (int e = b + 1; e < NUP; ++e)
                    if (e < nu) s -= ws->H[e][b] * y[e];
                y[b] = s / ws->H[b][b];
            }
#pragma unroll
        for (int b = 0; b < NUP; ++b)
            if (b < nu) ws->X[b][col] = -y[b];
    }
    __syncwarp();

    /* P = Q_xx + Q_ux' K (row `lane`), p = q_x + Q_ux' k; symmetrised through T1 */
    float pl = qx;
    if (lane < NXP) {
#pragma unroll
        for (int j = 0; j < NXP; j += 4) {
            float v0 = sxx[j], v1 = sxx[j + 1], v2 = sxx[j + 2], v3 = sxx[j + 3];
#pragma unroll
            for (int b = 0; b < NUP; ++b) {
                const float4 k4 = ld4(&ws->X[b][j]);
                v0 += qux[b] * k4.x;
                v1 += qux[b] * k4.y;
                v2 += qux[b] * k4.z;
                v3 += qux[b] * k4.w;
            }
            st4(&ws->T1[lane][j], v0, v1, v2, v3);
        }
#pragma unroll
        for (int b = 0; b < NUP; ++b) pl += qux[b] * ws->X[b][NXP];
    }
    __syncwarp();
    if (row) {
        for (int j = 0; j < nx; ++j) Pi[(size_t)j * nx + lane] = 0.5f * (ws->T1[lane][j] + ws->T1[j][lane]);
        a.p[node * nx + lane] = pl;
        for (int b = 0; b < nu; ++b) Ki[(size_t)b * nx + lane] = ws->X[b][lane];
    }
    if (lane < nu) a.k[node * nu + lane] = ws->X[lane][NXP];
}

template <int NXP, int NUP>
__global__ void __launch_bounds__(32 * LQR_WARPS) lqr_forward_kernel(LqrArgs a) {
    __shared__ __align__(16) float sA[LQR_WARPS][NXP][NXP + 4];
    __shared__ __align__(16) float sB[LQR_WARPS][NXP][NUP + 4];
    const int w = threadIdx.x / 32, lane = threadIdx.x & 31;
    const long long item = (long long)blockIdx.x * LQR_WARPS + w;
    if (item >= (long long)a.cnt * a.batch) return;
    const int t = (int)(item / a.cnt);
    const int m = a.s0 + (int)(item % a.cnt);
    const int nx = a.nx, nu = a.nu;
    const size_t node = (size_t)t * a.n + m;
    const bool row = lane < nx;
    float xl = 0.f;
    if (m == 0) {
        xl = row ? a.x0[(size_t)t * nx + lane] : 0.f;
    } else {
        const size_t pa = (size_t)t * a.n + a.parent[m];
        stage_tile<NXP, NXP, NXP + 4>(sA[w], a.A + node * nx * nx, nx, nx, lane);
        stage_tile<NXP, NUP, NUP + 4>(sB[w], a.B + node * nx * nu, nx, nu, lane);
        const float xp = row ? a.x[pa * nx + lane] : 0.f;
        const float up = lane < nu ? a.u[pa * nu + lane] : 0.f;
        __syncwarp();
        float v = row ? a.c[node * nx + lane] : 0.f;
        const int r = lane % NXP;
#pragma unroll
        for (int kk = 0; kk < NXP; kk += 4) {
            const float4 a4 = ld4(&sA[w][r][kk]);
            v += a4.x * __shfl_sync(FULL, xp, kk) + a4.y * __shfl_sync(FULL, xp, kk + 1) +
                 a4.z * __shfl_sync(FULL, xp, kk + 2) + a4.w * __shfl_sync(FULL, xp, kk + 3);
        }
#pragma unroll
        for (int b = 0; b < NUP; b += 4) {
            const float4 b4 = ld4(&sB[w][r][b]);
            v += b4.x * __shfl_sync(FULL, up, b) + b4.y * __shfl_sync(FULL, up, b + 1) +
                 b4.z * __shfl_sync(FULL, up, b + 2) + b4.w * __shfl_sync(FULL, up, b + 3);
        }
        xl = row ? v : 0.f;
    }
    /* u = K x + k (rows < nu; 0 at leaves), lam = P x + p */
    const bool leaf = a.child_off[m] == a.child_off[m + 1];
    float ul = 0.f;
    const float *Km = a.K + node * nu * nx, *Pm = a.P + node * nx * nx;
    if (!leaf && lane < nu) ul = a.k[node * nu + lane];
    float ll = row ? a.p[node * nx + lane] : 0.f;
    for (int j = 0; j < nx; ++j) {
        const float xj = __shfl_sync(FULL, xl, j);
        if (!leaf && lane < nu) ul += Km[(size_t)lane * nx + j] * xj;
        if (row) ll += Pm[(size_t)j * nx + lane] * xj;
    }
    if (row) {
        a.x[node * nx + lane] = xl;
        a.lam[node * nx + lane] = ll;
    }
    if (lane < nu) a.u[node * nu + lane] = ul;
}

template <int NXP, int NUP>
size_t backward_smem() { return LQR_WARPS * sizeof(LqrTiles<NXP, NUP>); }

using LqrKernel = void (*)(LqrArgs);
struct Instance {
    LqrKernel bwd, fwd;
    size_t smem;
};

Instance instance(int nx, int nu) {
    if (nx <= 8 && nu <= 4) return {lqr_backward_kernel<8, 4>, lqr_forward_kernel<8, 4>, backward_smem<8, 4>()};
    if (nx <= 16 && nu <= 8) return {lqr_backward_kernel<16, 8>, lqr_forward_kernel<16, 8>, backward_smem<16, 8>()};
    return {lqr_backward_kernel<32, 16>, lqr_forward_kernel<32, 16>, backward_smem<32, 16>()};
}

}  // namespace

struct bmpc_lqr {
    int n = 0, nx = 0, nu = 0, batch = 0;
    std::vector<int> sstart;   /* stage s holds nodes [sstart[s], sstart[s + 1]) */
    int32_t *d_parent = nullptr, *d_child_off = nullptr, *d_child_idx = nullptr, *d_flag = nullptr;
    cudaStream_t stream = nullptr;
    Instance inst{};
};

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
    bool ok = cudaMalloc(&h->d_parent, sizeof(int32_t) * n) == cudaSuccess &&
              cudaMalloc(&h->d_child_off, sizeof(int32_t) * (n + 1)) == cudaSuccess &&
              cudaMalloc(&h->d_child_idx, sizeof(int32_t) * idx.size()) == cudaSuccess &&
              cudaMalloc(&h->d_flag, sizeof(int32_t)) == cudaSuccess;
    ok = ok && cudaMemcpy(h->d_parent, parent, sizeof(int32_t) * n, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(h->d_child_off, off.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(h->d_child_idx, idx.data(), sizeof(int32_t) * idx.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(h->d_flag, 0, sizeof(int32_t)) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(h->inst.bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->inst.smem) ==
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
    LqrArgs a{Q, M, R, q, r, A, B, c, x0, K, k, P, p, x, u, lam, h->d_parent, h->d_child_off, h->d_child_idx,
              h->d_flag, h->n, h->nx, h->nu, h->batch, 0, 0};
    const int S = (int)h->sstart.size() - 1;
    auto grid = [&](int cnt) { return (unsigned)(((long long)cnt * h->batch + LQR_WARPS - 1) / LQR_WARPS); };
    for (int s = S - 1; s >= 0; --s) {
        a.s0 = h->sstart[s];
        a.cnt = h->sstart[s + 1] - h->sstart[s];
        h->inst.bwd<<<grid(a.cnt), 32 * LQR_WARPS, h->inst.smem, h->stream>>>(a);
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

void bmpc_lqr_destroy(bmpc_lqr *h) {
    if (!h) return;
    cudaFree(h->d_parent);
    cudaFree(h->d_child_off);
    cudaFree(h->d_child_idx);
    cudaFree(h->d_flag);
    delete h;
}

}  // extern "C"
