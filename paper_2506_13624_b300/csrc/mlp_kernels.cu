/*
 * Learned warm start: a multilayer perceptron with BF16 weights and activations, FP32
 * accumulation, trained and evaluated by the kernels in this file.
 *
 *   gemm_tc<TA, TB, EPI, WN> C[M x N] = op(A)[M x K] op(B)[K x N] on the 5th-generation tensor
 *                            cores: tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) issued by one
 *                            thread from shared-memory descriptors, the 128 x WN accumulator
 *                            (WN = 128, or 256 when N allows) in tensor memory (TMEM), operand tiles
 *                            loaded by TMA (cp.async.bulk.tensor, 128-byte swizzle) into a 4-stage
 *                            ring of full/empty mbarriers; the epilogue reads TMEM with tcgen05.ld.
 *                            op(X) is X or X^T: K-major and MN-major operands use the matching
 *                            swizzled descriptor layouts.
 *                            Epilogues: plain f32 (weight gradients), + bias in f32 (output
 *                            layer), + bias then GELU in bf16 with the pre-activation kept (hidden
 *                            layers), times GELU'(pre) in bf16 (back-propagation through a hidden
 *                            layer).
 *   mse_grad                 loss and dL/dY of the mean squared error against bf16 targets.
 *   bias_grad                column sums of dL/dY.
 *   adamw                    AdamW on fp32 master weights, refreshing the bf16 copy.
 *   init                     uniform(-1/sqrt(in), 1/sqrt(in)) weights from a counter-based hash.
 *
 * Every matrix is row-major; M and N are multiples of 128 and K of 64 (the host pads).
 */
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

namespace bmpc_mlp {

constexpr int BM = 128, BN = 128, BK = 64, NSTAGE = 4;   /* BN: the narrow tile (N a multiple of 128) */
constexpr int THREADS = 192;                                   /* warp 0 TMA, warp 1 MMA, warps 2-5 epilogue */
constexpr int TILE_BYTES = 128 * BK * 2;                       /* one 128 x 64 bf16 operand tile (16 KB) */
constexpr int OUT_BUF = 32 * 32 * 4;                           /* one 32 x 32 FP32 chunk of C for a TMA store */
constexpr int OUT_BYTES = 4 * 2 * OUT_BUF;                     /* two buffers per epilogue warp */
constexpr int GROUP_M = 16;                                    /* m-tiles per group of the tile order */

/* Output tiles of 128 x WN, WN = 128 or 256 (N a multiple of 256): the wide tile reads 3/4 of the
 * operand bytes per product of the narrow one.  Per k-step the A slice is 16 KB and the B slice
 * WN x 64 bf16; two FP32 accumulators of 128 lanes x WN columns fill 256 or all 512 TMEM columns. */
template <int WN>
struct GemmCfg {
    static constexpr int STAGE = TILE_BYTES + WN * BK * 2;                  /* A and B slices of one k-step */
    static constexpr int SMEM = NSTAGE * STAGE + OUT_BYTES + 1024;           /* 161 or 225 KB with the slack */
    static constexpr int TMEM = 2 * WN;
};

enum Epi { EPI_F32 = 0, EPI_BIAS_F32 = 1, EPI_BIAS_GELU = 2, EPI_DGELU = 3 };

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

/* ------------------------------------------------------------------ tcgen05 GEMM */
__device__ int g_gemm_timeout;   /* set when an mbarrier wait of a GEMM gave up (read by bmpc_mlp_status) */

/* Shared-memory matrix descriptor (tcgen05) of an operand tile in the 128-byte-swizzled layout
 * TMA writes with CU_TENSOR_MAP_SWIZZLE_128B: start address, leading and stride byte offsets,
 * descriptor version 1, layout code 2 (128-byte swizzle).
 *   K-major tile (128 rows x 64 k, one 128-byte row per tile row, 8-row atoms of 1024 bytes):
 *     stride offset 1024 between 8-row atoms; the leading offset is unused; the MMA of k-slice j
 *     (16 k) starts 32 j bytes into the tile.
 *   M/N-major tile (64 k rows x 128 mn, two 64-wide halves of 8 KB): leading offset 8192 between
 *     the halves, stride offset 1024 between 8-row groups of k; k-slice j starts 2048 j bytes in. */
__device__ __forceinline__ uint64_t tile_desc(uint32_t addr, bool mn_major) {
    const uint64_t lbo = mn_major ? 8192 : 16, sbo = 1024;
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46) | (2ull << 61);
}
__device__ __forceinline__ uint32_t slice_offset(int j, bool mn_major) { return mn_major ? 2048u * j : 32u * j; }

/* Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5), BF16 A and B
 * (bits 7-9, 10-12), A and B majors (bit 15, 16: 0 K-major, 1 M/N-major), N/8 (bits 17-22),
 * M/16 (bits 24-28); M = 128, N = WN. */
template <int WN>
__host__ __device__ constexpr uint32_t mma_idesc(bool a_mn, bool b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
           ((uint32_t)(WN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

/* One 2-D TMA load (one thread) with 128-byte swizzle into `dst` (1024-byte aligned), completing
 * on `bar`: the box at coordinates (x, y) of the operand's map; x, the innermost coordinate, is a
 * multiple of 64 elements (128 bytes). */
__device__ __forceinline__ void tma_box(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

/* TMA store (one thread) of a 32 x 32 FP32 chunk from shared memory (128-byte-swizzled rows) to
 * C at (x, y, z) of the output map; x, the column, is a multiple of 32 elements (128 bytes). */
__device__ __forceinline__ void tma_store_chunk(const CUtensorMap *map, const void *src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(map), "r"(x),
                 "r"(y), "r"(z), "r"(smem_addr(src))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

/* The operand slice of k-step t for a tile of ROWS rows (128 or 256): K-major, one box of 64 k x ROWS
 * rows (the map's box); M/N-major, ROWS / 64 boxes of 64 mn x 64 k, 8 KB apart. */
template <bool KMAJ, int ROWS>
__device__ __forceinline__ void load_slice(unsigned char *dst, const CUtensorMap *map, int k0, int r0, uint64_t *bar) {
    if (KMAJ) {
        tma_box(dst, map, k0, r0, bar);
    } else {
#pragma unroll
        for (int h = 0; h < ROWS / 64; ++h) tma_box(dst + 8192 * h, map, r0 + 64 * h, k0, bar);
    }
}

constexpr long long WAIT_CYCLES = 4000000000ll;   /* about 2 s of SM clock */

/* Waits (at most `limit` SM cycles) for the phase of `bar` with the given parity; 0 on timeout. */
__device__ __forceinline__ int mbar_wait(uint64_t *bar, uint32_t parity, long long limit = WAIT_CYCLES) {
    const uint32_t a = smem_addr(bar);
    const long long t0 = clock64();
    do {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, q;\n\t}"
                     : "=r"(ok)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (ok) return 1;
    } while (clock64() - t0 < limit);
    return 0;
}

/* mbar_wait that also gives up (returning 0) as soon as another role of the block has set *abort. */
__device__ __forceinline__ int mbar_wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort) {
    const uint32_t a = smem_addr(bar);
    const long long t0 = clock64();
    do {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, q;\n\t}"
                     : "=r"(ok)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (ok) return 1;
        if (*abort) return 0;
    } while (clock64() - t0 < WAIT_CYCLES);
    *abort = 1;
    return 0;
}

/* 32 consecutive accumulator columns of this thread's TMEM lane. */
__device__ __forceinline__ void tmem_ld32(uint32_t (&r)[32], uint32_t taddr) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

/* C = op(A) op(B), persistent and warp-specialised.  TA: A is given transposed (stored K x M);
 * TB: B is given transposed (stored N x K); amap/bmap are their TMA views and ldc the row length of
 * C.  The grid's blocks take the 128 x WN output tiles t = blockIdx.x, + gridDim.x, ... of the
 * S x MT x NT tile space: split z slowest, then groups of GROUP_M m-tiles, inside a group the m-tile
 * fastest, so that the blocks that run together share each B tile and a panel of GROUP_M A tiles
 * in L2; split z covers k-steps [z kps, min(K/BK, (z+1) kps)) and, for EPI_F32, writes its partial
 * product to C + z c_split.
 *   warp 0, one thread: TMA producer over an NSTAGE ring of operand stages (full/empty mbarriers);
 *   warp 1, one thread: issues the MMAs of each k-step once its stage has landed, commits them to
 *     the stage's empty barrier, and after a tile's last k-step to tmem_full of its accumulator;
 *     two TMEM accumulators alternate between tiles, so the MMAs of tile i+1 overlap the epilogue
 *     of tile i;
 *   warps 2-5: the epilogue.  Warp w reads TMEM lanes 32 (w mod 4) .. + 31 (rows of C), applies
 *     the epilogue, and releases the accumulator on tmem_empty.
 * Every wait is bounded; on a timeout the block records it in g_gemm_timeout, every role stops,
 * the producer waits for its loads in flight, the MMA thread for its MMAs, and TMEM is freed. */
template <bool TA, bool TB, int EPI, int WN>
__global__ void __launch_bounds__(THREADS) gemm_tc(const __grid_constant__ CUtensorMap amap,
                                                    const __grid_constant__ CUtensorMap bmap,
                                                    const __grid_constant__ CUtensorMap cmap, void *C, int ldc, int K,
                                                    const float *__restrict__ bias, __nv_bfloat16 *__restrict__ pre,
                                                    int kps, int64_t c_split, int MT, int NT, int T) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[NSTAGE], empty[NSTAGE], tmem_full[2], tmem_empty[2], drain;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(GemmCfg<WN>::TMEM));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < NSTAGE; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&empty[s])));
        }
        for (int a = 0; a < 2; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&tmem_full[a])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_addr(&tmem_empty[a])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&drain)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const int KT_all = K / BK;
    auto tile_of = [&](int t, int &m0, int &n0, int &kbeg, int &KT, int &z) {
        const int per = MT * NT, r = t % per, g = r / (GROUP_M * NT), first = g * GROUP_M;
        const int gm = min(MT - first, GROUP_M), w = r - g * GROUP_M * NT;
        z = t / per;
        m0 = (first + w % gm) * BM;
        n0 = (w / gm) * WN;
        kbeg = z * kps;
        KT = min(KT_all - kbeg, kps);
    };
    if (warp == 0) {
        if (lane == 0) {
            uint32_t g = 0;
            for (int t = blockIdx.x; t < T && !abort_flag; t += gridDim.x) {
                int m0, n0, kbeg, KT, z;
                tile_of(t, m0, n0, kbeg, KT, z);
                for (int kt = 0; kt < KT; ++kt, ++g) {
                    const int s = g % NSTAGE;
                    if (!mbar_wait_or_abort(&empty[s], ((g / NSTAGE) & 1) ^ 1, &abort_flag)) break;
                    unsigned char *sa = smem + s * GemmCfg<WN>::STAGE;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&full[s])),
                                 "r"(GemmCfg<WN>::STAGE)
                                 : "memory");
                    load_slice<!TA, BM>(sa, &amap, (kbeg + kt) * BK, m0, &full[s]);
                    load_slice<TB, WN>(sa + TILE_BYTES, &bmap, (kbeg + kt) * BK, n0, &full[s]);
                }
            }
            if (abort_flag) {   /* the last loads of every stage land before the block frees its memory */
                for (uint32_t q = (g > NSTAGE ? g - NSTAGE : 0); q < g; ++q)
                    mbar_wait(&full[q % NSTAGE], (q / NSTAGE) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = mma_idesc<WN>(TA, !TB);
            uint32_t g = 0;
            int i = 0;
            for (int t = blockIdx.x; t < T && !abort_flag; t += gridDim.x, ++i) {
                int m0, n0, kbeg, KT, z;
                tile_of(t, m0, n0, kbeg, KT, z);
                const int acc = i & 1;
                if (!mbar_wait_or_abort(&tmem_empty[acc], ((i >> 1) & 1) ^ 1, &abort_flag)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(acc * WN);
                bool fail = false;
                for (int kt = 0; kt < KT; ++kt, ++g) {
                    const int s = g % NSTAGE;
                    if (!mbar_wait_or_abort(&full[s], (g / NSTAGE) & 1, &abort_flag)) {
                        fail = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = smem_addr(smem + s * GemmCfg<WN>::STAGE), sb = sa + TILE_BYTES;
#pragma unroll
                    for (int j = 0; j < BK / 16; ++j) {
                        const uint64_t da = tile_desc(sa + slice_offset(j, TA), TA);
                        const uint64_t db = tile_desc(sb + slice_offset(j, !TB), !TB);
                        const uint32_t accumulate = (kt | j) != 0;
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                                     "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_addr(&empty[s]))
                                 : "memory");
                }
                if (fail) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_addr(&tmem_full[acc]))
                             : "memory");
            }
            if (abort_flag) {   /* every MMA issued so far completes before TMEM is freed */
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_addr(&drain))
                             : "memory");
                mbar_wait(&drain, 0);
            }
        }
    } else {
        const int q = warp & 3;   /* TMEM lane quarter this warp may access */
        unsigned char *obuf = smem + NSTAGE * GemmCfg<WN>::STAGE;   /* 1024-byte aligned output chunk buffers */
        int nst = 0;                                          /* TMA stores issued by this warp */
        int i = 0;
        for (int t = blockIdx.x; t < T; t += gridDim.x, ++i) {
            int m0, n0, kbeg, KT, z;
            tile_of(t, m0, n0, kbeg, KT, z);
            const int acc = i & 1;
            if (!mbar_wait_or_abort(&tmem_full[acc], (i >> 1) & 1, &abort_flag)) break;
            __syncwarp();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            void *Cz = EPI == EPI_F32 ? static_cast<void *>(static_cast<float *>(C) + z * c_split) : C;
            const int r = m0 + q * 32 + lane;
#pragma unroll 1
            for (int cc = 0; cc < WN / 32; ++cc) {
                uint32_t v[32];
                tmem_ld32(v, tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * WN + cc * 32));
                const int c0 = n0 + cc * 32;
                const size_t o = (size_t)r * ldc + c0;
                if (EPI == EPI_F32 || EPI == EPI_BIAS_F32) {
                    /* the warp's 32 x 32 chunk goes through one of its two shared buffers and leaves by
                     * one TMA store; lane l writes row l with its 16-byte pieces in the 128-byte
                     * swizzle order (piece k at position k ^ (l mod 8)), free of bank conflicts */
                    unsigned char *buf = obuf + (size_t)(((warp - 2) * 2 + (nst & 1)) * OUT_BUF);
                    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                    __syncwarp();
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq) {
                        float4 f = make_float4(__uint_as_float(v[4 * qq]), __uint_as_float(v[4 * qq + 1]),
                                               __uint_as_float(v[4 * qq + 2]), __uint_as_float(v[4 * qq + 3]));
                        if (EPI == EPI_BIAS_F32) {
                            f.x += bias[c0 + 4 * qq];
                            f.y += bias[c0 + 4 * qq + 1];
                            f.z += bias[c0 + 4 * qq + 2];
                            f.w += bias[c0 + 4 * qq + 3];
                        }
                        *reinterpret_cast<float4 *>(buf + lane * 128 + ((qq ^ (lane & 7)) << 4)) = f;
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) tma_store_chunk(&cmap, buf, c0, m0 + q * 32, EPI == EPI_F32 ? z : 0);
                    ++nst;
                } else if (EPI == EPI_BIAS_GELU) {
                    uint4 *dp = reinterpret_cast<uint4 *>(pre + o);
                    uint4 *dc = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(Cz) + o);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        uint32_t pz[4], az[4];
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const int j = 8 * qq + 2 * h;
                            pz[h] = pack_bf16(__uint_as_float(v[j]) + bias[c0 + j],
                                              __uint_as_float(v[j + 1]) + bias[c0 + j + 1]);
                            const float2 pf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&pz[h]));
                            az[h] = pack_bf16(gelu(pf.x), gelu(pf.y));
                        }
                        dp[qq] = make_uint4(pz[0], pz[1], pz[2], pz[3]);
                        dc[qq] = make_uint4(az[0], az[1], az[2], az[3]);
                    }
                } else {   /* EPI_DGELU: dX = (dY W^T) * gelu'(pre) */
                    const uint4 *sp = reinterpret_cast<const uint4 *>(pre + o);
                    uint4 *dc = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(Cz) + o);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        const uint4 pq = sp[qq];
                        const uint32_t pw[4] = {pq.x, pq.y, pq.z, pq.w};
                        uint32_t oz[4];
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const int j = 8 * qq + 2 * h;
                            const float2 pf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&pw[h]));
                            oz[h] = pack_bf16(__uint_as_float(v[j]) * gelu_grad(pf.x),
                                              __uint_as_float(v[j + 1]) * gelu_grad(pf.y));
                        }
                        dc[qq] = make_uint4(oz[0], oz[1], oz[2], oz[3]);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&tmem_empty[acc])) : "memory");
        }
        if ((EPI == EPI_F32 || EPI == EPI_BIAS_F32) && lane == 0)   /* the stores complete before exit */
            asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        __syncwarp();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (abort_flag && tid == 0) atomicExch(&g_gemm_timeout, 1);
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GemmCfg<WN>::TMEM));
}

/* Self-test of the bounded wait: one thread waits for the first phase of an mbarrier that nothing
 * arrives on, for at most `cycles` SM cycles, and records the timeout as a GEMM does. */
__global__ void wait_selftest_kernel(long long cycles) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!mbar_wait(&bar, 0, cycles)) atomicExch(&g_gemm_timeout, 1);
    }
}

/* Split-K reduction: C = epilogue(sum over the S partial products in ws, in split order). */
template <int EPI>
__global__ void splitk_reduce(const float *__restrict__ ws, int S, int M, int N, void *C, int ldc,
                              const float *__restrict__ bias, __nv_bfloat16 *__restrict__ pre) {
    const int64_t pairs = (int64_t)M * N / 2;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < pairs; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = 2 * p;
        const int r = (int)(e / N), c = (int)(e % N);
        float v0 = 0.f, v1 = 0.f;
        for (int z = 0; z < S; ++z) {
            const float2 w = *reinterpret_cast<const float2 *>(ws + (int64_t)z * M * N + e);
            v0 += w.x;
            v1 += w.y;
        }
        const size_t o = (size_t)r * ldc + c;
        if (EPI == EPI_F32) {
            *reinterpret_cast<float2 *>(static_cast<float *>(C) + o) = make_float2(v0, v1);
        } else if (EPI == EPI_BIAS_F32) {
            *reinterpret_cast<float2 *>(static_cast<float *>(C) + o) = make_float2(v0 + bias[c], v1 + bias[c + 1]);
        } else if (EPI == EPI_BIAS_GELU) {
            const uint32_t pz = pack_bf16(v0 + bias[c], v1 + bias[c + 1]);
            *reinterpret_cast<uint32_t *>(pre + o) = pz;
            const float2 pf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&pz));
            *reinterpret_cast<uint32_t *>(static_cast<__nv_bfloat16 *>(C) + o) = pack_bf16(gelu(pf.x), gelu(pf.y));
        } else {
            const float2 pf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(pre + o));
            *reinterpret_cast<uint32_t *>(static_cast<__nv_bfloat16 *>(C) + o) =
                pack_bf16(v0 * gelu_grad(pf.x), v1 * gelu_grad(pf.y));
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

/* The output tile width for N columns: 256 when N is a multiple of 256, else 128. */
int gemm_wn(int N) { return N % 256 == 0 ? 256 : BN; }

/* K-steps per split for a GEMM with few output tiles: enough splits to give every SM about two
 * blocks, at least 8 k-steps each; returns K/BK (one split) when splitting does not pay. */
int split_kps(int M, int N, int K) {
    const int tiles = (M / BM) * (N / gemm_wn(N)), KT = K / BK;
    if (tiles >= 148) return KT;
    int S = std::min((2 * 148 + tiles - 1) / tiles, KT / 8);
    if (S < 2) return KT;
    return (KT + S - 1) / S;
}

int64_t split_floats(int M, int N, int K) {
    const int kps = split_kps(M, N, K), KT = K / BK;
    return kps >= KT ? 0 : (int64_t)((KT + kps - 1) / kps) * M * N;
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

/* cuTensorMapEncodeTiled from the driver, looked up once through the runtime. */
EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

/* TMA view of a GEMM operand for gemm_tc (see load_slice): a 2-D map of the stored matrix with
 * 128-byte swizzle.  kmajor: stored [mn][ld] with K along a row, boxes of 64 k x `rows` rows (the
 * operand tile's 128 or 256); else stored [k][ld] with MN along a row, boxes of 64 mn x 64 k.  mn and
 * k are the operand's extents (multiples of the tile and of BK), ld the stored row length in
 * elements (a multiple of 8: 16-byte rows). */
bool make_operand_map(CUtensorMap *m, const void *ptr, int mn, int k, int ld, bool kmajor, int rows) {
    const EncodeTiled enc = encoder();
    if (!enc) return false;
    cuuint64_t dim[2], str[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2], es[2] = {1, 1};
    if (kmajor) {
        dim[0] = (cuuint64_t)k;
        dim[1] = (cuuint64_t)mn;
        box[0] = 64;
        box[1] = (cuuint32_t)rows;
    } else {
        dim[0] = (cuuint64_t)mn;
        dim[1] = (cuuint64_t)k;
        box[0] = 64;
        box[1] = 64;
    }
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dim, str, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

/* TMA view of an FP32 output for the GEMM's stores: C [S][M][ldc] (S partial products c_split
 * floats apart), boxes of 32 columns x 32 rows x 1 with 128-byte swizzle. */
bool make_output_map(CUtensorMap *m, void *C, int M, int N, int ldc, int S, int64_t c_split) {
    const EncodeTiled enc = encoder();
    if (!enc) return false;
    cuuint64_t dim[3] = {(cuuint64_t)N, (cuuint64_t)M, (cuuint64_t)S};
    cuuint64_t str[2] = {(cuuint64_t)ldc * 4, (cuuint64_t)(S > 1 ? c_split : (int64_t)M * ldc) * 4};
    cuuint32_t box[3] = {32, 32, 1}, es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, C, dim, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

template <bool TA, bool TB, int EPI, int WN>
cudaError_t set_smem() {
    static bool done = false;   /* 161 or 225 KB of dynamic shared memory need the opt-in, once per instance */
    if (done) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(gemm_tc<TA, TB, EPI, WN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               GemmCfg<WN>::SMEM);
    done = e == cudaSuccess;
    return e;
}

/* Persistent blocks for T output tiles: one per SM (the shared-memory ring allows one block per
 * SM), fewer when there are fewer tiles. */
int gemm_grid(int T) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || sms < 1)
            sms = 1;
    }
    return std::max(1, std::min(T, sms));
}

/* C = epilogue(op(A) op(B)) with output tiles of 128 x WN; GEMMs with few output tiles and a long K
 * are split along K into the workspace ws (ws_floats floats, may be 0) and reduced in split order by
 * splitk_reduce. */
template <bool TA, bool TB, int EPI, int WN>
cudaError_t gemm_w(const void *A, int lda, const void *B, int ldb, void *C, int ldc, int M, int N, int K,
                   const float *bias, void *pre, cudaStream_t s, float *ws, int64_t ws_floats) {
    constexpr int SMEM = GemmCfg<WN>::SMEM;
    const int KT = K / BK, kps = split_kps(M, N, K), S = (KT + kps - 1) / kps;
    const int MT = M / BM, NT = N / WN;
    CUtensorMap am, bm;
    if (!make_operand_map(&am, A, M, K, lda, !TA, BM) || !make_operand_map(&bm, B, N, K, ldb, TB, WN))
        return cudaErrorInvalidValue;
    if (S > 1 && ws && (int64_t)S * M * N <= ws_floats) {
        cudaError_t e = set_smem<TA, TB, EPI_F32, WN>();
        if (e != cudaSuccess) return e;
        const int T = S * MT * NT;
        CUtensorMap cm;
        if (!make_output_map(&cm, ws, M, N, N, S, (int64_t)M * N)) return cudaErrorInvalidValue;
        gemm_tc<TA, TB, EPI_F32, WN><<<gemm_grid(T), THREADS, SMEM, s>>>(am, bm, cm, ws, N, K, nullptr, nullptr, kps,
                                                                         (int64_t)M * N, MT, NT, T);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int64_t pairs = (int64_t)M * N / 2;
        const int grid = (int)std::min<int64_t>((pairs + 255) / 256, 4096);
        splitk_reduce<EPI><<<grid, 256, 0, s>>>(ws, S, M, N, C, ldc, bias, static_cast<__nv_bfloat16 *>(pre));
        return cudaGetLastError();
    }
    const cudaError_t e = set_smem<TA, TB, EPI, WN>();
    if (e != cudaSuccess) return e;
    CUtensorMap cm;
    if (EPI == EPI_F32 || EPI == EPI_BIAS_F32) {
        if (!make_output_map(&cm, C, M, N, ldc, 1, 0)) return cudaErrorInvalidValue;
    } else {
        cm = am;   /* unused by the bf16 epilogues */
    }
    gemm_tc<TA, TB, EPI, WN><<<gemm_grid(MT * NT), THREADS, SMEM, s>>>(am, bm, cm, C, ldc, K, bias,
                                                                      static_cast<__nv_bfloat16 *>(pre), KT, 0, MT,
                                                                      NT, MT * NT);
    return cudaGetLastError();
}

template <bool TA, bool TB, int EPI>
cudaError_t gemm(const void *A, int lda, const void *B, int ldb, void *C, int ldc, int M, int N, int K, const float *bias,
                 void *pre, cudaStream_t s, float *ws = nullptr, int64_t ws_floats = 0) {
    return gemm_wn(N) == 256 ? gemm_w<TA, TB, EPI, 256>(A, lda, B, ldb, C, ldc, M, N, K, bias, pre, s, ws, ws_floats)
                             : gemm_w<TA, TB, EPI, BN>(A, lda, B, ldb, C, ldc, M, N, K, bias, pre, s, ws, ws_floats);
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
                                                  L[l].out, L[l].in, L[l].b, w->pre[l], s, w->splitk, w->splitk_floats);
        else
            e = gemm<false, false, EPI_BIAS_F32>(in, L[l].in, L[l].w_bf16, L[l].out, w->pred, L[l].out, batch,
                                                 L[l].out, L[l].in, L[l].b, nullptr, s, w->splitk, w->splitk_floats);
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
                                       nullptr, s, w->splitk, w->splitk_floats) != cudaSuccess)
            return -2;
        bias_grad<<<(L[l].out + 255) / 256, 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(g), batch, L[l].out,
                                                         L[l].db);
        if (l > 0) {   /* g_prev = (g W^T) * gelu'(pre_{l-1}) */
            if (gemm<false, true, EPI_DGELU>(g, L[l].out, L[l].w_bf16, L[l].out, gn, L[l].in, batch, L[l].in,
                                             L[l].out, nullptr, w->pre[l - 1], s, w->splitk, w->splitk_floats) !=
                cudaSuccess)
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
    /* 16-byte rows for the cp.async staging and the vector stores of the epilogue */
    if (!dims_ok(M, N, K) || !A || !B || !C || lda % 8 || ldb % 8 || ldc % 8) return -1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (!trans_a && !trans_b) e = gemm<false, false, EPI_F32>(A, lda, B, ldb, C, ldc, M, N, K, nullptr, nullptr, s);
    else if (trans_a && !trans_b) e = gemm<true, false, EPI_F32>(A, lda, B, ldb, C, ldc, M, N, K, nullptr, nullptr, s);
    else if (!trans_a && trans_b) e = gemm<false, true, EPI_F32>(A, lda, B, ldb, C, ldc, M, N, K, nullptr, nullptr, s);
    else e = gemm<true, true, EPI_F32>(A, lda, B, ldb, C, ldc, M, N, K, nullptr, nullptr, s);
    return e == cudaSuccess ? 0 : -2;
}

int64_t bmpc_mlp_workspace_floats(const bmpc_mlp_layer *L, int32_t n, int32_t batch) {
    if (check_layers(L, n) || batch <= 0 || batch % 128) return -1;
    int64_t f = 0;
    for (int l = 0; l < n; ++l) {
        f = std::max(f, split_floats(batch, L[l].out, L[l].in));        /* forward */
        f = std::max(f, split_floats(L[l].in, L[l].out, batch));        /* dW = in^T g */
        if (l > 0) f = std::max(f, split_floats(batch, L[l].in, L[l].out));   /* g W^T */
    }
    return f;
}

int bmpc_mlp_selftest_wait(int64_t cycles, void *stream) {
    if (cycles < 1 || cycles > 100000000) return -1;
    wait_selftest_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>((long long)cycles);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int bmpc_mlp_status(void *stream) {
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return -2;
    int flag = 0;
    if (cudaMemcpyFromSymbol(&flag, g_gemm_timeout, sizeof flag) != cudaSuccess) return -2;
    if (!flag) return 0;
    const int zero = 0;
    cudaMemcpyToSymbol(g_gemm_timeout, &zero, sizeof zero);
    return -4;
}

}  // extern "C"
