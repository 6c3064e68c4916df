/*
 * Learned warm start: a multilayer perceptron with BF16 weights and activations, FP32
 * accumulation, trained and evaluated by the kernels in this file.
 *
 *   gemm_bf16<TA, TB, EPI>   C[M x N] = op(A)[M x K] op(B)[K x N] on the tensor cores
 *                            (mma.sync m16n8k16 bf16 -> f32), operands staged in shared memory by
 *                            cp.async with double buffering and read with ldmatrix; op(X) is X or
 *                            X^T.  Epilogues: plain f32 (weight gradients), + bias in f32 (output
 *                            layer), + bias then GELU in bf16 with the pre-activation kept (hidden
 *                            layers), times GELU'(pre) in bf16 (back-propagation through a hidden
 *                            layer).
 *   mse_grad                 loss and dL/dY of the mean squared error against bf16 targets.
 *   bias_grad                column sums of dL/dY.
 *   adamw                    AdamW on fp32 master weights, refreshing the bf16 copy.
 *   init                     uniform(-1/sqrt(in), 1/sqrt(in)) weights from a counter-based hash.
 *
 * Every matrix is row-major with dimensions that are multiples of 128 (the host pads).
 */
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace bmpc_mlp {

constexpr int BM = 128, BN = 128, BK = 32, THREADS = 256;
constexpr int LD_MK = BK + 8;     /* padded row length of a [128][32] tile (bf16) */
constexpr int LD_KM = BM + 8;     /* padded row length of a [32][128] tile (bf16) */
constexpr int TILE = 128 * LD_MK > BK * LD_KM ? 128 * LD_MK : BK * LD_KM;

enum Epi { EPI_F32 = 0, EPI_BIAS_F32 = 1, EPI_BIAS_GELU = 2, EPI_DGELU = 3 };

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void *s, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(s)), "l"(g));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

/* Copy one 128 x 32 (MK) or 32 x 128 (KM) bf16 tile from global into a padded shared tile. */
template <bool KM>
__device__ __forceinline__ void load_tile(__nv_bfloat16 *s, const __nv_bfloat16 *g, int ld, int r0, int c0) {
    const int t = threadIdx.x;
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {
        const int idx = t + rep * THREADS;          /* 512 chunks of 8 elements */
        if (!KM) {
            const int r = idx >> 2, c = (idx & 3) * 8;
            cp_async16(s + r * LD_MK + c, g + (size_t)(r0 + r) * ld + c0 + c);
        } else {
            const int r = idx >> 4, c = (idx & 15) * 8;
            cp_async16(s + r * LD_KM + c, g + (size_t)(r0 + r) * ld + c0 + c);
        }
    }
}

/* C = op(A) op(B).  TA: A is given transposed (stored K x M); TB: B is given transposed (stored
 * N x K).  lda/ldb are the row lengths of the stored matrices, ldc of C. */
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(THREADS) gemm_bf16(const __nv_bfloat16 *__restrict__ A, int lda,
                                                      const __nv_bfloat16 *__restrict__ B, int ldb, void *C, int ldc,
                                                      int K, const float *__restrict__ bias,
                                                      __nv_bfloat16 *__restrict__ pre) {
    __shared__ __align__(16) __nv_bfloat16 sA[2][TILE];
    __shared__ __align__(16) __nv_bfloat16 sB[2][TILE];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    auto load_stage = [&](int st, int k0) {
        if (!TA) load_tile<false>(sA[st], A, lda, m0, k0);     /* A[m][k] */
        else load_tile<true>(sA[st], A, lda, k0, m0);          /* A^T stored [k][m] */
        if (!TB) load_tile<true>(sB[st], B, ldb, k0, n0);      /* B[k][n] */
        else load_tile<false>(sB[st], B, ldb, n0, k0);         /* B^T stored [n][k] */
        cp_commit();
    };
    const int KT = K / BK;
    load_stage(0, 0);
    const int mat = lane >> 3, r8 = lane & 7;
    for (int kt = 0; kt < KT; ++kt) {
        if (kt + 1 < KT) {
            load_stage((kt + 1) & 1, (kt + 1) * BK);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        const __nv_bfloat16 *a = sA[kt & 1], *b = sB[kt & 1];
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[4][4], bf[2][4];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi) {
                const int mb = wm + mi * 16;
                if (!TA) {
                    const int m = mb + r8 + ((mat & 1) ? 8 : 0), k = kk + ((mat >= 2) ? 8 : 0);
                    ldsm_x4(af[mi], a + m * LD_MK + k);
                } else {
                    const int k = kk + r8 + ((mat >= 2) ? 8 : 0), m = mb + ((mat & 1) ? 8 : 0);
                    ldsm_x4_t(af[mi], a + k * LD_KM + m);
                }
            }
#pragma unroll
            for (int nj = 0; nj < 2; ++nj) {
                const int nb = wn + nj * 16;
                if (TB) {
                    const int n = nb + r8 + ((mat >= 2) ? 8 : 0), k = kk + ((mat & 1) ? 8 : 0);
                    ldsm_x4(bf[nj], b + n * LD_MK + k);
                } else {
                    const int k = kk + r8 + ((mat & 1) ? 8 : 0), n = nb + ((mat >= 2) ? 8 : 0);
                    ldsm_x4_t(bf[nj], b + k * LD_KM + n);
                }
            }
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
                    mma16816(acc[mi][ni], af[mi], bf[ni >> 1][(ni & 1) * 2], bf[ni >> 1][(ni & 1) * 2 + 1]);
        }
        __syncthreads();
    }
    /* epilogue */
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = m0 + wm + mi * 16 + (lane >> 2) + h * 8;
                const int c = n0 + wn + ni * 8 + (lane & 3) * 2;
                float v0 = acc[mi][ni][2 * h], v1 = acc[mi][ni][2 * h + 1];
                const size_t o = (size_t)r * ldc + c;
                if (EPI == EPI_F32) {
                    *reinterpret_cast<float2 *>(static_cast<float *>(C) + o) = make_float2(v0, v1);
                } else if (EPI == EPI_BIAS_F32) {
                    v0 += bias[c];
                    v1 += bias[c + 1];
                    *reinterpret_cast<float2 *>(static_cast<float *>(C) + o) = make_float2(v0, v1);
                } else if (EPI == EPI_BIAS_GELU) {
                    const __nv_bfloat162 pz = __floats2bfloat162_rn(v0 + bias[c], v1 + bias[c + 1]);
                    *reinterpret_cast<__nv_bfloat162 *>(pre + o) = pz;
                    const float2 pf = __bfloat1622float2(pz);
                    *reinterpret_cast<__nv_bfloat162 *>(static_cast<__nv_bfloat16 *>(C) + o) =
                        __floats2bfloat162_rn(gelu(pf.x), gelu(pf.y));
                } else {   /* EPI_DGELU: dX = (dY W^T) * gelu'(pre) */
                    const float2 pf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(pre + o));
                    *reinterpret_cast<__nv_bfloat162 *>(static_cast<__nv_bfloat16 *>(C) + o) =
                        __floats2bfloat162_rn(v0 * gelu_grad(pf.x), v1 * gelu_grad(pf.y));
                }
            }
}

/* loss = mean (pred - target)^2 over rows x cols; dY = 2 (pred - target) / (rows cols) in bf16. */
__global__ void mse_grad(const float *__restrict__ pred, const __nv_bfloat16 *__restrict__ tgt, __nv_bfloat16 *dy,
                         int64_t count, float scale, float *loss) {
    float s = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = pred[i] - __bfloat162float(tgt[i]);
        s += e * e;
        dy[i] = __float2bfloat16_rn(2.f * e * scale);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        atomicAdd(loss, t * scale);
    }
}

/* db[c] = sum_r dY[r][c] */
__global__ void bias_grad(const __nv_bfloat16 *__restrict__ dy, int rows, int cols, float *db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += __bfloat162float(dy[(size_t)r * cols + c]);
    db[c] = s;
}

/* AdamW step on fp32 master weights; refreshes the bf16 copy when given. */
__global__ void adamw(float *w, float *m, float *v, const float *g, __nv_bfloat16 *wb, int64_t count, float lr,
                      float b1, float b2, float eps, float wd, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * w[i]);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16_rn(wi);
    }
}

/* SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator: uniform in [-a, a). */
__device__ __forceinline__ float hash_uniform(uint64_t seed, uint64_t i, float a) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return a * (2.f * (float)(z >> 40) * (1.f / 16777216.f) - 1.f);
}

__global__ void init_layer(float *w, __nv_bfloat16 *wb, float *m, float *v, int64_t count, float a, uint64_t seed,
                           float *b, float *bm, float *bv, int nb) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = hash_uniform(seed, (uint64_t)i, a);
        w[i] = x;
        wb[i] = __float2bfloat16_rn(x);
        m[i] = 0.f;
        v[i] = 0.f;
        if (i < nb) {
            b[i] = 0.f;
            bm[i] = 0.f;
            bv[i] = 0.f;
        }
    }
}

__global__ void standardize(const float *__restrict__ raw, const float *__restrict__ mean,
                            const float *__restrict__ std, __nv_bfloat16 *out, int64_t count, int dim) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % dim);
        out[i] = __float2bfloat16_rn((raw[i] - mean[j]) / std[j]);
    }
}

}  // namespace bmpc_mlp

/* ------------------------------------------------------------------ host entry points */
#include "../../include/bmpc_mlp.h"

namespace {
using namespace bmpc_mlp;

bool dims_ok(int M, int N, int K) { return M > 0 && N > 0 && K > 0 && M % BM == 0 && N % BN == 0 && K % BK == 0; }

template <bool TA, bool TB, int EPI>
cudaError_t gemm(const void *A, int lda, const void *B, int ldb, void *C, int ldc, int M, int N, int K, const float *bias,
                 void *pre, cudaStream_t s) {
    dim3 grid(N / BN, M / BM);
    gemm_bf16<TA, TB, EPI><<<grid, THREADS, 0, s>>>(static_cast<const __nv_bfloat16 *>(A), lda,
                                                    static_cast<const __nv_bfloat16 *>(B), ldb, C, ldc, K, bias,
                                                    static_cast<__nv_bfloat16 *>(pre));
    return cudaGetLastError();
}

int check_layers(const bmpc_mlp_layer *L, int n) {
    if (!L || n < 1 || n > BMPC_MLP_MAX_LAYERS) return -1;
    for (int l = 0; l < n; ++l) {
        if (L[l].in % 128 || L[l].out % 128 || L[l].in <= 0 || L[l].out <= 0) return -1;
        if (l > 0 && L[l].in != L[l - 1].out) return -1;
    }
    return 0;
}

int grid_for(int64_t count) { return (int)((count + 255) / 256 > 4096 ? 4096 : (count + 255) / 256); }

int forward(const bmpc_mlp_layer *L, int n, const uint16_t *x, int batch, const bmpc_mlp_work *w, cudaStream_t s) {
    const void *in = x;
    for (int l = 0; l < n; ++l) {
        cudaError_t e;
        if (l + 1 < n)
            e = gemm<false, false, EPI_BIAS_GELU>(in, L[l].in, L[l].w_bf16, L[l].out, w->act[l], L[l].out, batch,
                                                  L[l].out, L[l].in, L[l].b, w->pre[l], s);
        else
            e = gemm<false, false, EPI_BIAS_F32>(in, L[l].in, L[l].w_bf16, L[l].out, w->pred, L[l].out, batch,
                                                 L[l].out, L[l].in, L[l].b, nullptr, s);
        if (e != cudaSuccess) return -2;
        in = w->act[l];
    }
    return 0;
}
}  // namespace

extern "C" {

int bmpc_mlp_init(const bmpc_mlp_layer *L, int32_t n, uint64_t seed, void *stream) {
    if (check_layers(L, n)) return -1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int l = 0; l < n; ++l) {
        const int64_t cnt = (int64_t)L[l].in * L[l].out;
        init_layer<<<grid_for(cnt), 256, 0, s>>>(L[l].w, reinterpret_cast<__nv_bfloat16 *>(L[l].w_bf16), L[l].w_m,
                                                 L[l].w_v, cnt, 1.f / sqrtf((float)L[l].in), seed + 7919ull * l,
                                                 L[l].b, L[l].b_m, L[l].b_v, L[l].out);
        if (cudaGetLastError() != cudaSuccess) return -2;
    }
    return 0;
}

int bmpc_mlp_forward(const bmpc_mlp_layer *L, int32_t n, const uint16_t *x, int32_t batch, const bmpc_mlp_work *w,
                     void *stream) {
    if (check_layers(L, n) || !w || !x || batch % 128 || batch <= 0) return -1;
    return forward(L, n, x, batch, w, static_cast<cudaStream_t>(stream));
}

int bmpc_mlp_train_step(const bmpc_mlp_layer *L, int32_t n, const uint16_t *x, const uint16_t *target, int32_t batch,
                        float lr, float weight_decay, int32_t step, const bmpc_mlp_work *w, void *stream) {
    if (check_layers(L, n) || !w || !x || !target || batch % 128 || batch <= 0 || step < 1) return -1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (forward(L, n, x, batch, w, s)) return -2;
    const int out = L[n - 1].out;
    const int64_t cnt = (int64_t)batch * out;
    if (cudaMemsetAsync(w->loss, 0, sizeof(float), s) != cudaSuccess) return -2;
    mse_grad<<<grid_for(cnt), 256, 0, s>>>(w->pred, reinterpret_cast<const __nv_bfloat16 *>(target),
                                           reinterpret_cast<__nv_bfloat16 *>(w->dy0), cnt, 1.f / (float)cnt, w->loss);
    uint16_t *g = w->dy0, *gn = w->dy1;
    for (int l = n - 1; l >= 0; --l) {
        const void *in = l == 0 ? static_cast<const void *>(x) : static_cast<const void *>(w->act[l - 1]);
        /* dW = in^T g, db = column sums of g */
        if (gemm<true, false, EPI_F32>(in, L[l].in, g, L[l].out, L[l].dw, L[l].out, L[l].in, L[l].out, batch, nullptr,
                                       nullptr, s) != cudaSuccess)
            return -2;
        bias_grad<<<(L[l].out + 255) / 256, 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(g), batch, L[l].out,
                                                         L[l].db);
        if (l > 0) {   /* g_prev = (g W^T) * gelu'(pre_{l-1}) */
            if (gemm<false, true, EPI_DGELU>(g, L[l].out, L[l].w_bf16, L[l].out, gn, L[l].in, batch, L[l].in,
                                             L[l].out, nullptr, w->pre[l - 1], s) != cudaSuccess)
                return -2;
            uint16_t *t = g;
            g = gn;
            gn = t;
        }
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    for (int l = 0; l < n; ++l) {
        const int64_t cw = (int64_t)L[l].in * L[l].out;
        adamw<<<grid_for(cw), 256, 0, s>>>(L[l].w, L[l].w_m, L[l].w_v, L[l].dw,
                                           reinterpret_cast<__nv_bfloat16 *>(L[l].w_bf16), cw, lr, b1, b2, eps,
                                           weight_decay, c1, c2);
        adamw<<<grid_for(L[l].out), 256, 0, s>>>(L[l].b, L[l].b_m, L[l].b_v, L[l].db, nullptr, L[l].out, lr, b1, b2,
                                                 eps, 0.f, c1, c2);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int bmpc_mlp_standardize(const float *raw, const float *mean, const float *std, uint16_t *out, int64_t rows,
                         int32_t dim, void *stream) {
    if (!raw || !mean || !std || !out || rows <= 0 || dim <= 0) return -1;
    const int64_t cnt = rows * dim;
    standardize<<<grid_for(cnt), 256, 0, static_cast<cudaStream_t>(stream)>>>(raw, mean, std,
                                                                          reinterpret_cast<__nv_bfloat16 *>(out), cnt,
                                                                          dim);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int bmpc_mlp_gemm(const uint16_t *A, int32_t lda, int32_t trans_a, const uint16_t *B, int32_t ldb, int32_t trans_b,
                  float *C, int32_t ldc, int32_t M, int32_t N, int32_t K, void *stream) {
    if (!dims_ok(M, N, K) || !A || !B || !C) return -1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (!trans_a && !trans_b) e = gemm<false, false, EPI_F32>(A, lda, B, ldb, C, ldc, M, N, K, nullptr, nullptr, s);
    else if (trans_a && !trans_b) e = gemm<true, false, EPI_F32>(A, lda, B, ldb, C, ldc, M, N, K, nullptr, nullptr, s);
    else if (!trans_a && trans_b) e = gemm<false, true, EPI_F32>(A, lda, B, ldb, C, ldc, M, N, K, nullptr, nullptr, s);
    else e = gemm<true, true, EPI_F32>(A, lda, B, ldb, C, ldc, M, N, K, nullptr, nullptr, s);
    return e == cudaSuccess ? 0 : -2;
}

}  // extern "C"
