// Learned Metropolis-Hastings proposal: a MADE autoregressive Bernoulli network
// n -> H -> H -> n (ReLU), BF16 operands with FP32 accumulation on the tensor
// cores, trained by AdamW on chain samples, sampled bit by bit.
//
// Precision: FP32 master weights; the GEMMs read BF16 (round-to-nearest-even)
// copies of the masked weights and BF16 activations H1, H2 and backward signals
// dZ3, dZ2, dZ1; accumulation, biases, logits and gradients are FP32.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <vector>

#include <algorithm>

#include "lrs_device.cuh"

typedef __nv_bfloat16 bf16;

struct lrs_mlp {
    int device = 0;
    int n = 0, NP = 64, H = 0;
    // FP32 master parameters and AdamW moments (device)
    float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr, *W3 = nullptr, *b3 = nullptr;
    int gemm = 0;                         // LRS_MLP_GEMM_TCGEN05 or LRS_MLP_GEMM_MMA_SYNC
    int* err = nullptr;                   // device [2]: a tensor-core wait gave up; test request
    int* err_h = nullptr;                 // pinned host copy of err[0], refreshed after every call
    float *mW = nullptr, *vW = nullptr;   // moments for all parameters, packed
    float *grad = nullptr;                // gradients, packed like the parameters
    float *mask = nullptr;                // MADE masks, packed like the weights (1 for biases)
    int64_t n_params = 0;
    int64_t off[6] = {0};                 // offsets of W1 b1 W2 b2 W3 b3 in the packed arrays
    int64_t step = 0;
    // BF16 masked copies used by the GEMMs
    bf16 *W1b = nullptr;   // [H][NP]
    bf16 *W2b = nullptr;   // [H][H]
    bf16 *W3b = nullptr;   // [NP][H]   (rows >= n are zero)
    bf16 *W2t = nullptr;   // [H][H]    W2b transposed
    bf16 *W3t = nullptr;   // [H][NP]   W3b transposed
    // activations / workspace (grown on demand)
    void* ws = nullptr;
    size_t ws_bytes = 0;
};

namespace {

// ------------------------------------------------------------------------------------
// mma.sync BF16 GEMM: C[M x N] = A[M x K] . B[N x K]^T, both operands K-contiguous,
// K a multiple of 32, FP32 accumulation, fused epilogue.
// ------------------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void* smem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t b0,
                                         const uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <class Epi>
__global__ void __launch_bounds__(128) k_gemm_tn(const bf16* __restrict__ A, int lda,
                                                 const bf16* __restrict__ B, int ldb, int M, int N,
                                                 int K, Epi epi) {
    __shared__ __align__(16) bf16 sA[2][GBM][GBK + GPAD];
    __shared__ __align__(16) bf16 sB[2][GBN][GBK + GPAD];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    auto load = [&](int stage, int k0) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int chunk = tid + i * 128;
            const int r = chunk >> 2, c = (chunk & 3) * 8;
            const int gm = m0 + r, gn = n0 + r;
            cp_async16(&sA[stage][r][c], A + (size_t)(gm < M ? gm : M - 1) * lda + k0 + c, gm < M ? 16 : 0);
            cp_async16(&sB[stage][r][c], B + (size_t)(gn < N ? gn : N - 1) * ldb + k0 + c, gn < N ? 16 : 0);
        }
        cp_async_commit();
    };
    const int nk = K / GBK;
    load(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        if (kt + 1 < nk) {
            load((kt + 1) & 1, (kt + 1) * GBK);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int st = kt & 1;
#pragma unroll
        for (int kk = 0; kk < GBK; kk += 16) {
            uint32_t af[2][4], bq[2][4];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int r = wm * 32 + mi * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
                const int c = kk + (lane >> 4) * 8;
                ldmatrix_x4(af[mi], &sA[st][r][c]);
            }
#pragma unroll
            for (int nj = 0; nj < 2; ++nj) {
                const int r = wn * 32 + nj * 16 + (lane & 7) + (lane >> 4) * 8;
                const int c = kk + ((lane >> 3) & 1) * 8;
                ldmatrix_x4(bq[nj], &sB[st][r][c]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
                    mma_bf16(acc[mi][ni], af[mi], bq[ni >> 1][(ni & 1) * 2], bq[ni >> 1][(ni & 1) * 2 + 1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int row = m0 + wm * 32 + mi * 16 + (lane >> 2) + 8 * (e >> 1);
                const int col = n0 + wn * 32 + ni * 8 + (lane & 3) * 2 + (e & 1);
                if (row < M && col < N) epi(row, col, acc[mi][ni][e]);
            }
}

// ------------------------------------------------------------------------------------
// tcgen05 (5th-generation tensor core) GEMM: C[M x N] = A[M x K] . B[N x K]^T, BF16
// operands, FP32 accumulator in tensor memory.  One CTA computes a 128 x TN tile:
//   warp 0, lane 0   TMA producer: 128 x 64 and TN x 64 boxes (128-byte swizzle) into
//                    a ring of ST shared-memory stages, completion counted in bytes on
//                    full[s]; a stage is refilled after the MMAs that read it arrive on
//                    empty[s]
//   warp 1, lane 0   MMA issuer: four tcgen05.mma (K = 16 each) per stage, then
//                    tcgen05.commit -> empty[s]; after the last stage -> done
//   all four warps   epilogue: tcgen05.ld of their 32 accumulator lanes (rows),
//                    fused element-wise output
// Every wait is bounded in time; a wait that gives up sets *err and the tile is not
// written.  Rows >= M read as zero (TMA out-of-bounds fill).  N % TN == 0, K % 64 == 0.
// ------------------------------------------------------------------------------------
constexpr int TC_M = 128, TC_BK = 64;
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;   // 1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for the phase with the given parity to complete; false after TC_WAIT_NS.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
    if (mbar_try(addr, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try(addr, parity))
        if (global_ns() - t0 > TC_WAIT_NS) return false;
    return true;
}

// Shared-memory matrix descriptor for a K-major operand stored as 128-byte rows with
// the 128-byte swizzle (the layout a TMA box of 64 BF16 x rows with that swizzle
// writes): start address, stride between 8-row groups 1024 bytes, descriptor
// version 1, swizzle mode 2 (128 B).  The leading offset is unused for this layout.
__device__ __forceinline__ uint64_t tc_desc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Descriptor for an MN-major operand: the stage holds 64 x 64 boxes (64 consecutive
// M (or N) values = one 128-byte swizzled row per K index); 8-row K groups 1024
// bytes apart, 64-wide MN blocks 8192 bytes apart.
__device__ __forceinline__ uint64_t tc_desc_mn_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(8192 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, N >> 3, M >> 4; both
// operands K-major, or (mn) both MN-major.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N, bool mn = false) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (mn ? (1u << 15) | (1u << 16) : 0u) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

template <int TN, int ST>
struct TcShape {
    static constexpr int A_BYTES = TC_M * TC_BK * 2;
    static constexpr int B_BYTES = TN * TC_BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;        // a multiple of 1024
    static constexpr int SMEM = ST * STAGE + 1024;          // + alignment slack
};

template <int TN, int ST, bool MN, class Epi>
__global__ void __launch_bounds__(128) k_gemm_tc(const __grid_constant__ CUtensorMap tmA,
                                                 const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
                                                 Epi epi, int* err) {
    using S = TcShape<TN, ST>;
    extern __shared__ uint8_t tc_dyn[];
    __shared__ __align__(8) uint64_t full[ST], empty[ST], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag, consumed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * TN;
    const int nk = K / TC_BK;
    const uint32_t sbase = (smem_u32(tc_dyn) + 1023u) & ~1023u;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "n"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 32) {
        for (int i = 0; i < ST; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[i])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty[i])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        abort_flag = 0;
        consumed = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;

    int issued = 0;
    if (warp == 0 && lane == 0) {
        // TMA producer.  err[1] is a one-shot test request (lrs_mlp_debug_inject_wait_timeout):
        // block (0, 0) takes it and makes its first stage expect 16 bytes that no copy
        // delivers, so the MMA issuer's bounded wait on that stage runs out.
        const uint32_t extra = (blockIdx.x == 0 && blockIdx.y == 0 && atomicExch(&err[1], 0) != 0) ? 16u : 0u;
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % ST;
            if (kt >= ST && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((kt / ST) - 1) & 1u)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            if (*(volatile int*)&abort_flag) break;
            const uint32_t fb = smem_u32(&full[s]);
            const uint32_t sa = sbase + (uint32_t)(s * S::STAGE), sb = sa + (uint32_t)S::A_BYTES;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb),
                         "r"((uint32_t)S::STAGE + (kt == 0 ? extra : 0u))
                         : "memory");
            if constexpr (!MN) {
                tma_load_2d(sa, &tmA, kt * TC_BK, m0, fb);
                tma_load_2d(sb, &tmB, kt * TC_BK, n0, fb);
            } else {
#pragma unroll
                for (int h = 0; h < TC_M / 64; ++h) tma_load_2d(sa + h * 8192, &tmA, m0 + 64 * h, kt * TC_BK, fb);
#pragma unroll
                for (int j = 0; j < TN / 64; ++j) tma_load_2d(sb + j * 8192, &tmB, n0 + 64 * j, kt * TC_BK, fb);
            }
            issued = kt + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = tc_idesc(TC_M, TN, MN);
        int kt = 0;
        for (; kt < nk; ++kt) {
            const int s = kt % ST;
            if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(kt / ST) & 1u)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t sa = sbase + (uint32_t)(s * S::STAGE), sb = sa + (uint32_t)S::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                const uint64_t da = MN ? tc_desc_mn_sw128(sa + kk * 2048) : tc_desc_sw128(sa + kk * 32);
                const uint64_t db = MN ? tc_desc_mn_sw128(sb + kk * 2048) : tc_desc_sw128(sb + kk * 32);
                const uint32_t accum = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(accum)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        consumed = kt;
        // arrives once every MMA issued above has completed (also after an abort)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         smem_u32(&done))
                     : "memory");
    }
    __syncwarp();
    bool ok = mbar_wait(smem_u32(&done), 0u);
    ok = __syncthreads_and(ok && !*(volatile int*)&abort_flag) != 0;
    if (!ok) {
        if (tid == 32) mbar_wait(smem_u32(&done), 0u);   // the MMAs issued so far have finished
        if (tid == 0) {
            atomicExch(err, 1);
            // let the producer's copies that no MMA waited for land before the CTA exits
            // (each stage's wait is bounded; a stage whose wait runs out does not stop the
            // drain of the later ones)
            for (int kt = consumed; kt < issued; ++kt) mbar_wait(smem_u32(&full[kt % ST]), (uint32_t)(kt / ST) & 1u);
        }
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const int row = m0 + warp * 32 + lane;
#pragma unroll
        for (int c0 = 0; c0 < TN; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (row < M) {
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
                epi.row16(row, n0 + c0, v);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(TN) : "memory");
}

// Persistent variant for products with several k-steps.  A grid of at most one CTA
// per SM slot walks the output tiles (tile t, t + gridDim.x, ...); 192 threads:
//   warp 0, lane 0   TMA producer for every tile; k-steps are counted across tiles, so
//                    the ring of ST stages runs on from one tile into the next
//   warp 1, lane 0   MMA issuer; tile j accumulates into tensor-memory buffer j & 1
//                    (2 TN columns in all) and commits to accf[j & 1]
//   warps 2-5        epilogue: wait accf[b], read the 32 lanes of their quadrant
//                    (warp & 3), run the fused epilogue, release the buffer (acce[b])
// so a tile's epilogue overlaps the next tile's loads and MMAs.  Every wait is bounded
// (1 s); a wait that gives up stops all roles, the MMAs and copies in flight are waited
// for, and *err is set.
template <int TN, int ST, bool MN, class Epi>
__global__ void __launch_bounds__(192, 1) k_gemm_tcp(const __grid_constant__ CUtensorMap tmA,
                                                     const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
                                                     int ksplit, Epi epi, int* err) {
    using S = TcShape<TN, ST>;
    extern __shared__ uint8_t tc_dyn[];
    __shared__ __align__(8) uint64_t full[ST], empty[ST], accf[2], acce[2], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag, s_issued, s_consumed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // work unit u: output tile u % tiles, k-steps [kc (u / tiles), kc (u / tiles + 1))
    const int tiles_n = N / TN;
    const int tiles = tiles_n * ((M + TC_M - 1) / TC_M);
    const int units = tiles * ksplit;
    const int nk = K / TC_BK / ksplit;
    const uint32_t sbase = (smem_u32(tc_dyn) + 1023u) & ~1023u;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "n"(2 * TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 32) {
        for (int i = 0; i < ST; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[i])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty[i])) : "memory");
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&accf[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(smem_u32(&acce[b])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        abort_flag = 0;
        s_issued = 0;
        s_consumed = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer (block 0 takes a pending one-shot test request, as in k_gemm_tc)
        const uint32_t extra = (blockIdx.x == 0 && atomicExch(&err[1], 0) != 0) ? 16u : 0u;
        int g = 0;
        for (int u = blockIdx.x; u < units; u += gridDim.x) {
            const int t = u % tiles, k0 = (u / tiles) * nk;
            const int m0 = (t / tiles_n) * TC_M, n0 = (t % tiles_n) * TN;
            bool ok = true;
            for (int kt = k0; kt < k0 + nk; ++kt, ++g) {
                const int s = g % ST;
                if (g >= ST && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((g / ST) - 1) & 1u)) {
                    atomicExch(&abort_flag, 1);
                    ok = false;
                    break;
                }
                if (*(volatile int*)&abort_flag) {
                    ok = false;
                    break;
                }
                const uint32_t fb = smem_u32(&full[s]);
                const uint32_t sa = sbase + (uint32_t)(s * S::STAGE), sb = sa + (uint32_t)S::A_BYTES;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb),
                             "r"((uint32_t)S::STAGE + (g == 0 ? extra : 0u))
                             : "memory");
                if constexpr (!MN) {
                    tma_load_2d(sa, &tmA, kt * TC_BK, m0, fb);
                    tma_load_2d(sb, &tmB, kt * TC_BK, n0, fb);
                } else {
#pragma unroll
                    for (int h = 0; h < TC_M / 64; ++h) tma_load_2d(sa + h * 8192, &tmA, m0 + 64 * h, kt * TC_BK, fb);
#pragma unroll
                    for (int jj = 0; jj < TN / 64; ++jj) tma_load_2d(sb + jj * 8192, &tmB, n0 + 64 * jj, kt * TC_BK, fb);
                }
                s_issued = g + 1;
            }
            if (!ok) break;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = tc_idesc(TC_M, TN, MN);
        int g = 0, j = 0;
        for (int u = blockIdx.x; u < units; u += gridDim.x, ++j) {
            const int b = j & 1;
            if (j >= 2 && !mbar_wait(smem_u32(&acce[b]), (uint32_t)((j >> 1) - 1) & 1u)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t acc = tmem + (uint32_t)(b * TN);
            bool ok = true;
            for (int kt = 0; kt < nk; ++kt, ++g) {
                const int s = g % ST;
                if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(g / ST) & 1u)) {
                    atomicExch(&abort_flag, 1);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t sa = sbase + (uint32_t)(s * S::STAGE), sb = sa + (uint32_t)S::A_BYTES;
#pragma unroll
                for (int kk = 0; kk < TC_BK / 16; ++kk) {
                    const uint64_t da = MN ? tc_desc_mn_sw128(sa + kk * 2048) : tc_desc_sw128(sa + kk * 32);
                    const uint64_t db = MN ? tc_desc_mn_sw128(sb + kk * 2048) : tc_desc_sw128(sb + kk * 32);
                    const uint32_t accum = (kt > 0 || kk > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc),
                        "l"(da), "l"(db), "r"(idesc), "r"(accum)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 smem_u32(&empty[s]))
                             : "memory");
                s_consumed = g + 1;
            }
            if (!ok) break;
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&accf[b]))
                         : "memory");
        }
        // arrives once every MMA issued above has completed (also after an abort)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         smem_u32(&done))
                     : "memory");
    } else if (warp >= 2) {
        // epilogue: lanes 32 q .. 32 q + 31 of the accumulator
        const int q = warp & 3;
        int j = 0;
        for (int u = blockIdx.x; u < units; u += gridDim.x, ++j) {
            const int t = u % tiles;
            const int b = j & 1;
            const bool ok = mbar_wait(smem_u32(&accf[b]), (uint32_t)(j >> 1) & 1u);
            if (!__all_sync(0xffffffffu, ok)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const int m0 = (t / tiles_n) * TC_M, n0 = (t % tiles_n) * TN;
            const int row = m0 + q * 32 + lane;
#pragma unroll 1
            for (int c0 = 0; c0 < TN; c0 += 16) {
                uint32_t r[16];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * TN + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(taddr)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                if (row < M) {
                    float v[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
                    epi.row16(row, n0 + c0, v);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&acce[b])) : "memory");
        }
    }
    __syncwarp();
    __syncthreads();
    // every MMA issued has completed before the accumulators are freed
    const bool mma_done = mbar_wait(smem_u32(&done), 0u);
    if (tid == 0 && (*(volatile int*)&abort_flag || !mma_done)) {
        atomicExch(err, 1);
        // let the producer's copies that no MMA waited for land before the CTA exits
        for (int g = s_consumed; g < s_issued; ++g) mbar_wait(smem_u32(&full[g % ST]), (uint32_t)(g / ST) & 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(2 * TN) : "memory");
}

// Host side: cuTensorMapEncodeTiled through the runtime's driver entry point.
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (PFN_cuTensorMapEncodeTiled_v12000)p;
    }();
    return fn;
}

// 2-D map of a row-major BF16 matrix [rows][cols] (row stride ld elements), boxes of
// 64 columns x box_rows rows, 128-byte swizzle, zero fill outside.
lrs_status tmap_2d(CUtensorMap* tm, const bf16* ptr, int rows, int cols, int ld, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return lrs_fail(LRS_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    if (((uintptr_t)ptr & 15u) || (ld * 2) % 16 || cols % TC_BK)
        return lrs_fail(LRS_ERR_ARG, "gemm operand not 16-byte aligned (ld=%d, cols=%d)", ld, cols);
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)ptr, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return lrs_fail(LRS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return LRS_OK;
}

// MN = false: A [M][lda], B [N][ldb] (K contiguous).  MN = true: A [K][lda] holds
// A^T and B [K][ldb] holds B^T (M and N contiguous), so C = A . B^T needs no
// transposed copies.
template <int TN, int ST, bool MN, class Epi>
lrs_status launch_gemm_tc(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, Epi epi, int* err,
                          cudaStream_t st) {
    CUtensorMap ta, tb;
    lrs_status rc;
    if (!MN) {
        if ((rc = tmap_2d(&ta, A, M, K, lda, TC_M)) != LRS_OK) return rc;
        if ((rc = tmap_2d(&tb, B, N, K, ldb, TN)) != LRS_OK) return rc;
    } else {
        if ((rc = tmap_2d(&ta, A, K, M, lda, 64)) != LRS_OK) return rc;
        if ((rc = tmap_2d(&tb, B, K, N, ldb, 64)) != LRS_OK) return rc;
    }
    constexpr int smem = TcShape<TN, ST>::SMEM;
    LRS_CUDA(cudaFuncSetAttribute(k_gemm_tc<TN, ST, MN, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    dim3 grid(N / TN, (M + TC_M - 1) / TC_M);
    k_gemm_tc<TN, ST, MN, Epi><<<grid, 128, smem, st>>>(ta, tb, M, N, K, epi, err);
    LRS_LAUNCH_CHECK("tcgen05 gemm");
    return LRS_OK;
}

// Persistent launch: grid = resident CTAs (at most one per tile).
template <int TN, int ST, bool MN, class Epi>
lrs_status launch_gemm_tcp(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, Epi epi, int* err,
                           cudaStream_t st, int ksplit = 1) {
    CUtensorMap ta, tb;
    lrs_status rc;
    if (!MN) {
        if ((rc = tmap_2d(&ta, A, M, K, lda, TC_M)) != LRS_OK) return rc;
        if ((rc = tmap_2d(&tb, B, N, K, ldb, TN)) != LRS_OK) return rc;
    } else {
        if ((rc = tmap_2d(&ta, A, K, M, lda, 64)) != LRS_OK) return rc;
        if ((rc = tmap_2d(&tb, B, K, N, ldb, 64)) != LRS_OK) return rc;
    }
    constexpr int smem = TcShape<TN, ST>::SMEM;
    LRS_CUDA(cudaFuncSetAttribute(k_gemm_tcp<TN, ST, MN, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int dev = 0, sms = 0, per_sm = 0;
    LRS_CUDA(cudaGetDevice(&dev));
    LRS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LRS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemm_tcp<TN, ST, MN, Epi>, 192, smem));
    if (per_sm < 1) per_sm = 1;
    if (per_sm * 2 * TN > 512) per_sm = 512 / (2 * TN);   // tensor memory: 512 columns per SM
    const int units = (N / TN) * ((M + TC_M - 1) / TC_M) * ksplit;
    const int grid = std::min(units, sms * per_sm);
    k_gemm_tcp<TN, ST, MN, Epi><<<grid, 192, smem, st>>>(ta, tb, M, N, K, ksplit, epi, err);
    LRS_LAUNCH_CHECK("persistent tcgen05 gemm");
    return LRS_OK;
}

// Tile width for an M x N output: the widest of 256, 128, 64 that divides N and still
// gives every SM a tile; a single k-step takes a one-stage ring.
template <bool MN, class Epi>
lrs_status gemm_tc(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, Epi epi, int* err,
                   cudaStream_t st) {
    if (K % TC_BK != 0 || N % 64 != 0 || (MN && M % 64 != 0))
        return lrs_fail(LRS_ERR_ARG, "gemm: M=%d, N=%d, K=%d not multiples of 64", M, N, K);
    const int64_t mt = (M + TC_M - 1) / TC_M;
    if (K == TC_BK) {
        // one k-step: the tile is all epilogue, so a one-stage ring lets several CTAs
        // share an SM and overlap their stores
        if (N % 128 == 0) return launch_gemm_tc<128, 1, MN>(A, lda, B, ldb, M, N, K, epi, err, st);
        return launch_gemm_tc<64, 1, MN>(A, lda, B, ldb, M, N, K, epi, err, st);
    }
    if (N % 256 == 0 && mt * (N / 256) >= 148) return launch_gemm_tcp<256, 4, MN>(A, lda, B, ldb, M, N, K, epi, err, st);
    if (N % 128 == 0 && mt * (N / 128) >= 148) return launch_gemm_tcp<128, 3, MN>(A, lda, B, ldb, M, N, K, epi, err, st);
    return launch_gemm_tcp<64, 4, MN>(A, lda, B, ldb, M, N, K, epi, err, st);
}

// Weight gradients: C[M x N] = A . B^T with K = the batch (MN-major operands), few
// output tiles and many k-steps.  The k-steps are split over up to 16 chunks so that
// up to four work units per SM exist; the chunks' partial products are added into
// the output, which is zeroed first.  Uses the persistent kernel.
template <class EpiAdd>
lrs_status gemm_tc_splitk(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, float* out, int ldo,
                          int* err, cudaStream_t st) {
    if (K % TC_BK != 0 || N % 64 != 0 || M % 64 != 0)
        return lrs_fail(LRS_ERR_ARG, "gemm: M=%d, N=%d, K=%d not multiples of 64", M, N, K);
    LRS_CUDA(cudaMemsetAsync(out, 0, (size_t)M * ldo * sizeof(float), st));
    const int64_t mt = (M + TC_M - 1) / TC_M;
    const int tn = (N % 128 == 0 && mt * (N / 128) >= 64) ? 128 : 64;
    const int tiles = (int)(mt * (N / tn));
    const int nk = K / TC_BK;
    int ks = 1;
    while (ks < 16 && tiles * ks * 2 <= 4 * 152 && nk % (ks * 2) == 0 && nk / (ks * 2) >= 4) ks *= 2;
    const EpiAdd e{out, ldo};
    if (tn == 128) return launch_gemm_tcp<128, 3, true>(A, lda, B, ldb, M, N, K, e, err, st, ks);
    return launch_gemm_tcp<64, 4, true>(A, lda, B, ldb, M, N, K, e, err, st, ks);
}

// ---- epilogues ------------------------------------------------------------------------
// operator() takes one element (mma.sync kernel); row16 takes 16 consecutive columns
// c0..c0+15 of one row (tcgen05 kernel: one accumulator lane, c0 % 16 == 0, row
// strides multiples of 64 elements, so every access below is a 16-byte vector).
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

struct EpiBiasReluBf16 {     // out = bf16(relu(acc + bias))
    const float* bias;
    bf16* out;
    int ldo;
    __device__ __forceinline__ void operator()(int r, int c, float v) const {
        out[(size_t)r * ldo + c] = __float2bfloat16_rn(fmaxf(v + bias[c], 0.f));
    }
    __device__ __forceinline__ void row16(int r, int c0, const float (&v)[16]) const {
        uint32_t p[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 b = __ldg(reinterpret_cast<const float4*>(bias + c0) + q);
            p[2 * q] = pack_bf16x2(fmaxf(v[4 * q] + b.x, 0.f), fmaxf(v[4 * q + 1] + b.y, 0.f));
            p[2 * q + 1] = pack_bf16x2(fmaxf(v[4 * q + 2] + b.z, 0.f), fmaxf(v[4 * q + 3] + b.w, 0.f));
        }
        uint4* o = reinterpret_cast<uint4*>(out + (size_t)r * ldo + c0);
        o[0] = make_uint4(p[0], p[1], p[2], p[3]);
        o[1] = make_uint4(p[4], p[5], p[6], p[7]);
    }
};
struct EpiBiasF32 {          // out = acc + bias (columns >= nvalid get 0)
    const float* bias;
    float* out;
    int ldo, nvalid;
    __device__ __forceinline__ void operator()(int r, int c, float v) const {
        out[(size_t)r * ldo + c] = c < nvalid ? v + bias[c] : 0.f;
    }
    __device__ __forceinline__ void row16(int r, int c0, const float (&v)[16]) const {
        float4* o = reinterpret_cast<float4*>(out + (size_t)r * ldo + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float t[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = c0 + 4 * q + e;
                t[e] = c < nvalid ? v[4 * q + e] + __ldg(bias + c) : 0.f;   // bias has nvalid entries
            }
            o[q] = make_float4(t[0], t[1], t[2], t[3]);
        }
    }
};
struct EpiReluGrad {         // dZ = acc * [H > 0]; FP32 and BF16 copies
    const bf16* act;
    int lda;
    float* out32;
    bf16* out16;
    int ldo;
    __device__ __forceinline__ void operator()(int r, int c, float v) const {
        const float d = __bfloat162float(act[(size_t)r * lda + c]) > 0.f ? v : 0.f;
        out32[(size_t)r * ldo + c] = d;
        out16[(size_t)r * ldo + c] = __float2bfloat16_rn(d);
    }
    __device__ __forceinline__ void row16(int r, int c0, const float (&v)[16]) const {
        const uint4* a4 = reinterpret_cast<const uint4*>(act + (size_t)r * lda + c0);
        uint4 ar[2] = {a4[0], a4[1]};
        const bf16* a = reinterpret_cast<const bf16*>(ar);
        float d[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) d[j] = __bfloat162float(a[j]) > 0.f ? v[j] : 0.f;
        float4* o32 = reinterpret_cast<float4*>(out32 + (size_t)r * ldo + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) o32[q] = make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]);
        uint32_t p[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) p[q] = pack_bf16x2(d[2 * q], d[2 * q + 1]);
        uint4* o16 = reinterpret_cast<uint4*>(out16 + (size_t)r * ldo + c0);
        o16[0] = make_uint4(p[0], p[1], p[2], p[3]);
        o16[1] = make_uint4(p[4], p[5], p[6], p[7]);
    }
};
struct EpiAddF32 {           // out += acc (split-K partial products into a zeroed output)
    float* out;
    int ldo;
    __device__ __forceinline__ void operator()(int r, int c, float v) const { atomicAdd(out + (size_t)r * ldo + c, v); }
    __device__ __forceinline__ void row16(int r, int c0, const float (&v)[16]) const {
        float* o = out + (size_t)r * ldo + c0;
#pragma unroll
        for (int q = 0; q < 16; ++q) atomicAdd(o + q, v[q]);
    }
};
struct EpiStoreF32 {
    float* out;
    int ldo;
    __device__ __forceinline__ void operator()(int r, int c, float v) const { out[(size_t)r * ldo + c] = v; }
    __device__ __forceinline__ void row16(int r, int c0, const float (&v)[16]) const {
        float4* o = reinterpret_cast<float4*>(out + (size_t)r * ldo + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
};

// C = A . B^T with the network's GEMM kernel: tcgen05 (128 x 256, 128 x 128 or 128 x 64
// tiles, K in steps of 64) or mma.sync (64 x 64 tiles, K in steps of 32).  Every product of the network
// has N and K multiples of 64.
template <class Epi>
lrs_status gemm_tn(const lrs_mlp* m, const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K,
                   Epi epi, cudaStream_t st) {
    if (m->gemm == LRS_MLP_GEMM_TCGEN05) {
        return gemm_tc<false>(A, lda, B, ldb, M, N, K, epi, m->err, st);
    }
    if (K % GBK != 0) return lrs_fail(LRS_ERR_ARG, "gemm: K=%d not a multiple of %d", K, GBK);
    dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
    k_gemm_tn<Epi><<<grid, 128, 0, st>>>(A, lda, B, ldb, M, N, K, epi);
    LRS_LAUNCH_CHECK("mma gemm");
    return LRS_OK;
}

// ---- elementwise kernels ----------------------------------------------------------------
// bitstrings -> X [Mp][NP] bf16 (rows >= M zero)
__global__ void k_expand_bits(const uint64_t* __restrict__ xs, int M, int Mp, int n, int NP, bf16* X) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)Mp * NP) return;
    const int r = (int)(i / NP), c = (int)(i % NP);
    const float v = (r < M && c < n) ? (float)((xs[r] >> c) & 1ull) : 0.f;
    X[i] = __float2bfloat16_rn(v);
}

// out[c][r] = in[r][c] for an R x C bf16 matrix
__global__ void k_transpose_bf16(const bf16* __restrict__ in, int R, int C, bf16* __restrict__ out) {
    __shared__ bf16 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int r = r0 + j, c = c0 + threadIdx.x;
        tile[j][threadIdx.x] = (r < R && c < C) ? in[(size_t)r * C + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int c = c0 + j, r = r0 + threadIdx.x;
        if (c < C && r < R) out[(size_t)c * R + r] = tile[threadIdx.x][j];
    }
}

// dZ3 = (sigmoid(z) - x) / M for valid rows / columns; per-row NLL
__global__ void k_logit_grad(const float* __restrict__ logits, const uint64_t* __restrict__ xs, int M,
                             int Mp, int n, int NP, float* d32, bf16* d16, float* nll_rows) {
    const int r = blockIdx.x;
    const int c = threadIdx.x;   // NP threads
    float d = 0.f, l = 0.f;
    if (r < M && c < n) {
        const float z = logits[(size_t)r * NP + c];
        const float x = (float)((xs[r] >> c) & 1ull);
        const float s = 1.f / (1.f + expf(-z));
        d = (s - x) / (float)M;
        l = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))) - x * z;   // softplus(z) - x z
    }
    d32[(size_t)r * NP + c] = d;
    d16[(size_t)r * NP + c] = __float2bfloat16_rn(d);
    // row NLL
    __shared__ float red[64];
    red[c] = l;
    __syncthreads();
    for (int off = 32; off > 0; off >>= 1) {
        if (c < off) red[c] += red[c + off];
        __syncthreads();
    }
    if (c == 0 && nll_rows && r < M) nll_rows[r] = red[0];
}

// column sums of an FP32 [rows][ld] matrix -> out[c] (first `cols` columns), in two
// deterministic passes: block (x, y) sums rows y*chunk .. (y+1)*chunk - 1 of 64
// columns into part[y][c] (4 row lanes, then a fixed-order combine); then each
// column adds its COLSUM_CHUNKS partials in order.
constexpr int COLSUM_CHUNKS = 128;

__global__ void __launch_bounds__(256) k_colsum_part(const float* __restrict__ a, int rows, int ld, int cols,
                                                     float* __restrict__ part) {
    __shared__ float red[4][64];
    const int cx = threadIdx.x & 63, ry = threadIdx.x >> 6;
    const int c = blockIdx.x * 64 + cx;
    const int chunk = (rows + COLSUM_CHUNKS - 1) / COLSUM_CHUNKS;
    const int r0 = blockIdx.y * chunk, r1 = min(rows, r0 + chunk);
    float s = 0.f;
    if (c < cols)
        for (int r = r0 + ry; r < r1; r += 4) s += a[(size_t)r * ld + c];
    red[ry][cx] = s;
    __syncthreads();
    if (ry == 0 && c < cols) part[(size_t)blockIdx.y * cols + c] = (red[0][cx] + red[1][cx]) + (red[2][cx] + red[3][cx]);
}

__global__ void k_colsum_fin(const float* __restrict__ part, int cols, float* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int y = 0; y < COLSUM_CHUNKS; ++y) s += part[(size_t)y * cols + c];
    out[c] = s;
}

__global__ void k_mean(const float* __restrict__ v, int m, float* out) {
    __shared__ float red[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < m; i += 256) s += v[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0] / (float)m;
}

// copy a padded FP32 gradient block into the packed gradient array
__global__ void k_copy_grad(const float* __restrict__ src, int rows, int cols, int lds, float* dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    dst[i] = src[(size_t)(i / cols) * lds + (i % cols)];
}

__global__ void k_apply_mask(float* __restrict__ g, const float* __restrict__ mask, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) g[i] *= mask[i];
}

// AdamW on the packed parameters (masked gradients)
__global__ void k_adamw(float* __restrict__ p, const float* __restrict__ g, const float* __restrict__ mask,
                        float* __restrict__ m, float* __restrict__ v, int64_t count, float lr, float b1,
                        float b2, float eps, float wd, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i] * mask[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    p[i] = p[i] - lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
}

// BF16 masked copies (and transposes) of the weights
__global__ void k_refresh_bf16(const float* __restrict__ W1, const float* __restrict__ W2,
                               const float* __restrict__ W3, const float* __restrict__ mask, int64_t o1,
                               int64_t o2, int64_t o3, int n, int NP, int H, bf16* W1b, bf16* W2b,
                               bf16* W3b, bf16* W2t, bf16* W3t) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n1 = (int64_t)H * NP, n2 = (int64_t)H * H, n3 = (int64_t)NP * H;
    if (i < n1) {
        const int k = (int)(i / NP), c = (int)(i % NP);
        const float w = c < n ? W1[(int64_t)k * n + c] * mask[o1 + (int64_t)k * n + c] : 0.f;
        W1b[i] = __float2bfloat16_rn(w);
    } else if (i < n1 + n2) {
        const int64_t j = i - n1;
        const int k2 = (int)(j / H), k1 = (int)(j % H);
        const bf16 w = __float2bfloat16_rn(W2[j] * mask[o2 + j]);
        W2b[j] = w;
        W2t[(int64_t)k1 * H + k2] = w;
    } else if (i < n1 + n2 + n3) {
        const int64_t j = i - n1 - n2;
        const int r = (int)(j / H), k = (int)(j % H);
        const float wv = r < n ? W3[(int64_t)r * H + k] * mask[o3 + (int64_t)r * H + k] : 0.f;
        const bf16 w = __float2bfloat16_rn(wv);
        W3b[j] = w;
        W3t[(int64_t)k * NP + r] = w;
    }
}

// log q(x) per row from logits: -sum_i softplus(z_i) - x_i z_i
__global__ void k_logq(const float* __restrict__ logits, const uint64_t* __restrict__ xs, int M, int n,
                       int NP, float* out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    float s = 0.f;
    for (int c = 0; c < n; ++c) {
        const float z = logits[(size_t)r * NP + c];
        const float x = (float)((xs[r] >> c) & 1ull);
        s += fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))) - x * z;
    }
    out[r] = -s;
}

// ---- autoregressive sampling ---------------------------------------------------------------
// Z1 [M][H] fp32 starts at b1; H1 = bf16(relu(Z1)); y = 0, logq = 0.
__global__ void k_sample_init(const float* __restrict__ b1, int Mp, int H, int count, float* Z1, bf16* H1,
                              uint64_t* y, float* logq) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (int64_t)Mp * H) {
        const float z = b1[i % H];
        Z1[i] = z;
        H1[i] = __float2bfloat16_rn(fmaxf(z, 0.f));
    }
    if (i < count) {
        y[i] = 0ull;
        logq[i] = 0.f;
    }
}

// bit i of every sample: logit_i = H2[r] . W3b[i] + b3[i]; y_i = [u < sigmoid];
// then Z1 += y_i W1b[:, i] and H1 = bf16(relu(Z1)).  One warp per row.
__global__ void k_sample_bit(const bf16* __restrict__ H2, const bf16* __restrict__ W3b,
                             const float* __restrict__ b3, const bf16* __restrict__ W1b, int M, int H,
                             int NP, int i, uint64_t seed, int64_t sid0, float* Z1, bf16* H1, uint64_t* y,
                             float* logq) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= M) return;
    const int r = warp;
    float s = 0.f;
    for (int k = lane; k < H; k += 32)
        s += __bfloat162float(H2[(size_t)r * H + k]) * __bfloat162float(W3b[(size_t)i * H + k]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const float z = s + b3[i];
    const float p = 1.f / (1.f + expf(-z));
    // uniform draw: rand64(seed, 2^40 + sample id, bit i)
    const double u = sm64_unit(sm64_at(sm64_key(seed, (1ull << 40) + (uint64_t)(sid0 + r)), (uint64_t)i));
    const int bit = (float)u < p ? 1 : 0;
    if (lane == 0) {
        if (bit) y[r] |= 1ull << i;
        logq[r] += -(fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))) - (float)bit * z);
    }
    if (bit) {
        for (int k = lane; k < H; k += 32) {
            const float zz = Z1[(size_t)r * H + k] + __bfloat162float(W1b[(size_t)k * NP + i]);
            Z1[(size_t)r * H + k] = zz;
            H1[(size_t)r * H + k] = __float2bfloat16_rn(fmaxf(zz, 0.f));
        }
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct MlpWS {   // workspace views for a batch of Mp rows
    bf16 *X, *H1, *H2, *D3, *D2, *D1, *T1, *T2;
    float *logits, *d3f, *d2f, *d1f, *gW, *nll, *Z1;
    uint64_t* ybuf;
    float* lqbuf;
    float* colp;   // [COLSUM_CHUNKS][H] column-sum partials
};

lrs_status mlp_ws(lrs_mlp* m, int Mp, MlpWS& w) {
    const size_t NP = m->NP, H = m->H;
    size_t sz[] = {Mp * NP * 2, Mp * H * 2, Mp * H * 2, Mp * NP * 2, Mp * H * 2, Mp * H * 2,
                   H * (size_t)Mp * 2, H * (size_t)Mp * 2, Mp * NP * 4, Mp * NP * 4, Mp * H * 4,
                   Mp * H * 4, H * H * 4, (size_t)Mp * 4, Mp * H * 4, (size_t)Mp * 8, (size_t)Mp * 4,
                   (size_t)COLSUM_CHUNKS * H * 4};
    size_t total = 0;
    for (size_t s : sz) total += align256(s);
    lrs_status rc = lrs_ensure(&m->ws, &m->ws_bytes, total);
    if (rc != LRS_OK) return rc;
    char* p = (char*)m->ws;
    void* ptrs[18];
    for (int i = 0; i < 18; ++i) {
        ptrs[i] = p;
        p += align256(sz[i]);
    }
    w.X = (bf16*)ptrs[0]; w.H1 = (bf16*)ptrs[1]; w.H2 = (bf16*)ptrs[2]; w.D3 = (bf16*)ptrs[3];
    w.D2 = (bf16*)ptrs[4]; w.D1 = (bf16*)ptrs[5]; w.T1 = (bf16*)ptrs[6]; w.T2 = (bf16*)ptrs[7];
    w.logits = (float*)ptrs[8]; w.d3f = (float*)ptrs[9]; w.d2f = (float*)ptrs[10]; w.d1f = (float*)ptrs[11];
    w.gW = (float*)ptrs[12]; w.nll = (float*)ptrs[13]; w.Z1 = (float*)ptrs[14];
    w.ybuf = (uint64_t*)ptrs[15]; w.lqbuf = (float*)ptrs[16]; w.colp = (float*)ptrs[17];
    return LRS_OK;
}

int pad64(int64_t M) { return (int)((M + 63) / 64 * 64); }

lrs_status mlp_forward(lrs_mlp* m, const uint64_t* xs, int M, const MlpWS& w, cudaStream_t st) {
    const int Mp = pad64(M), NP = m->NP, H = m->H;
    const int64_t tot = (int64_t)Mp * NP;
    k_expand_bits<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(xs, M, Mp, m->n, NP, w.X);
    LRS_LAUNCH_CHECK("expand bits");
    lrs_status rc;
    if ((rc = gemm_tn(m, w.X, NP, m->W1b, NP, Mp, H, NP, EpiBiasReluBf16{m->b1, w.H1, H}, st)) != LRS_OK) return rc;
    if ((rc = gemm_tn(m, w.H1, H, m->W2b, H, Mp, H, H, EpiBiasReluBf16{m->b2, w.H2, H}, st)) != LRS_OK) return rc;
    return gemm_tn(m, w.H2, H, m->W3b, H, Mp, NP, H, EpiBiasF32{m->b3, w.logits, NP, m->n}, st);
}

void colsum(const float* a, int rows, int ld, int cols, float* part, float* out, cudaStream_t st) {
    k_colsum_part<<<dim3((cols + 63) / 64, COLSUM_CHUNKS), 256, 0, st>>>(a, rows, ld, cols, part);
    k_colsum_fin<<<(cols + 127) / 128, 128, 0, st>>>(part, cols, out);
}

void transpose(const bf16* in, int R, int C, bf16* out, cudaStream_t st) {
    dim3 grid((C + 31) / 32, (R + 31) / 32), blk(32, 8);
    k_transpose_bf16<<<grid, blk, 0, st>>>(in, R, C, out);
}

// forward + backward into m->grad; loss (mean NLL) to loss_dev
lrs_status mlp_backward(lrs_mlp* m, const uint64_t* xs, int M, const MlpWS& w, float* loss_dev,
                        cudaStream_t st) {
    const int Mp = pad64(M), NP = m->NP, H = m->H, n = m->n;
    lrs_status rc = mlp_forward(m, xs, M, w, st);
    if (rc != LRS_OK) return rc;
    k_logit_grad<<<Mp, NP, 0, st>>>(w.logits, xs, M, Mp, n, NP, w.d3f, w.D3, w.nll);
    LRS_LAUNCH_CHECK("logit grad");
    if (loss_dev) {
        k_mean<<<1, 256, 0, st>>>(w.nll, M, loss_dev);
        LRS_LAUNCH_CHECK("mean");
    }
    float* g = m->grad;
    // weight gradient D^T Hin (D [Mp][Mo], Hin [Mp][No]): the tcgen05 kernel reads both
    // operands MN-major straight from the activations; mma.sync goes through transposes
    auto dW = [&](const bf16* D, int Mo, const bf16* Hin, int No, EpiStoreF32 e) -> lrs_status {
        if (m->gemm == LRS_MLP_GEMM_TCGEN05)
            return gemm_tc_splitk<EpiAddF32>(D, Mo, Hin, No, Mo, No, Mp, e.out, e.ldo, m->err, st);
        transpose(D, Mp, Mo, w.T1, st);
        transpose(Hin, Mp, No, w.T2, st);
        return gemm_tn(m, w.T1, Mp, w.T2, Mp, Mo, No, Mp, e, st);
    };
    // dW3 = dZ3^T H2   [NP x H]
    if ((rc = dW(w.D3, NP, w.H2, H, EpiStoreF32{w.gW, H})) != LRS_OK) return rc;
    k_copy_grad<<<(n * H + 255) / 256, 256, 0, st>>>(w.gW, n, H, H, g + m->off[4]);
    colsum(w.d3f, Mp, NP, n, w.colp, g + m->off[5], st);
    // dZ2 = (dZ3 W3) * [H2 > 0]
    if ((rc = gemm_tn(m, w.D3, NP, m->W3t, NP, Mp, H, NP, EpiReluGrad{w.H2, H, w.d2f, w.D2, H}, st)) != LRS_OK)
        return rc;
    // dW2 = dZ2^T H1   [H x H]
    if ((rc = dW(w.D2, H, w.H1, H, EpiStoreF32{g + m->off[2], H})) != LRS_OK) return rc;
    colsum(w.d2f, Mp, H, H, w.colp, g + m->off[3], st);
    // dZ1 = (dZ2 W2) * [H1 > 0]
    if ((rc = gemm_tn(m, w.D2, H, m->W2t, H, Mp, H, H, EpiReluGrad{w.H1, H, w.d1f, w.D1, H}, st)) != LRS_OK)
        return rc;
    // dW1 = dZ1^T X   [H x NP] -> packed [H x n]
    if ((rc = dW(w.D1, H, w.X, NP, EpiStoreF32{w.gW, NP})) != LRS_OK) return rc;
    k_copy_grad<<<(H * n + 255) / 256, 256, 0, st>>>(w.gW, H, n, NP, g + m->off[0]);
    colsum(w.d1f, Mp, H, H, w.colp, g + m->off[1], st);
    k_apply_mask<<<(unsigned)((m->n_params + 255) / 256), 256, 0, st>>>(g, m->mask, m->n_params);
    LRS_LAUNCH_CHECK("backward");
    return LRS_OK;
}

lrs_status refresh_bf16(lrs_mlp* m, cudaStream_t st) {
    const int64_t tot = (int64_t)m->H * m->NP * 2 + (int64_t)m->H * m->H;
    k_refresh_bf16<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
        m->W1, m->W2, m->W3, m->mask, m->off[0], m->off[2], m->off[4], m->n, m->NP, m->H, m->W1b, m->W2b,
        m->W3b, m->W2t, m->W3t);
    LRS_LAUNCH_CHECK("refresh bf16 weights");
    return LRS_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------
extern "C" lrs_status lrs_mlp_create(int32_t device, int32_t n, int32_t hidden, lrs_mlp** out) {
    if (!out) return lrs_fail(LRS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 2 || n > 64) return lrs_fail(LRS_ERR_ARG, "MADE needs 2 <= n <= 64 (got %d)", n);
    if (hidden < 64 || hidden > 4096 || hidden % 64) return lrs_fail(LRS_ERR_ARG, "hidden must be a multiple of 64 in 64..4096");
    LRS_CUDA(cudaSetDevice(device));
    lrs_mlp* m = new lrs_mlp();
    m->device = device;
    m->n = n;
    m->H = hidden;
    const int64_t H = hidden;
    const int64_t sizes[6] = {H * n, H, H * H, H, (int64_t)n * H, n};
    int64_t o = 0;
    for (int i = 0; i < 6; ++i) {
        m->off[i] = o;
        o += sizes[i];
    }
    m->n_params = o;
    const size_t pb = (size_t)o * sizeof(float);
    cudaError_t e = cudaSuccess;
    float* params = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&params, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->mW, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->vW, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->grad, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->mask, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->W1b, (size_t)H * 64 * 2);
    if (e == cudaSuccess) e = cudaMalloc(&m->W2b, (size_t)H * H * 2);
    if (e == cudaSuccess) e = cudaMalloc(&m->W3b, (size_t)64 * H * 2);
    if (e == cudaSuccess) e = cudaMalloc(&m->W2t, (size_t)H * H * 2);
    if (e == cudaSuccess) e = cudaMalloc(&m->W3t, (size_t)H * 64 * 2);
    if (e == cudaSuccess) e = cudaMalloc(&m->err, 2 * sizeof(int));   // flag, one-shot test request
    if (e == cudaSuccess) e = cudaMemset(m->err, 0, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&m->err_h, sizeof(int), cudaHostAllocDefault);
    if (e == cudaSuccess) *m->err_h = 0;
    if (e != cudaSuccess) {
        delete m;
        return lrs_cuda_check(e, "mlp storage");
    }
    m->W1 = params + m->off[0]; m->b1 = params + m->off[1]; m->W2 = params + m->off[2];
    m->b2 = params + m->off[3]; m->W3 = params + m->off[4]; m->b3 = params + m->off[5];
    // MADE masks: input degree i+1, hidden m(k) = (k mod (n-1)) + 1
    std::vector<float> mk((size_t)o, 1.f);
    for (int64_t k = 0; k < H; ++k) {
        const int mk1 = (int)(k % (n - 1)) + 1;
        for (int i = 0; i < n; ++i) mk[(size_t)(m->off[0] + k * n + i)] = mk1 >= i + 1 ? 1.f : 0.f;
        for (int64_t k1 = 0; k1 < H; ++k1) {
            const int m1 = (int)(k1 % (n - 1)) + 1;
            mk[(size_t)(m->off[2] + k * H + k1)] = mk1 >= m1 ? 1.f : 0.f;
        }
    }
    for (int i = 0; i < n; ++i)
        for (int64_t k = 0; k < H; ++k) {
            const int m2 = (int)(k % (n - 1)) + 1;
            mk[(size_t)(m->off[4] + i * H + k)] = (i + 1) > m2 ? 1.f : 0.f;
        }
    LRS_CUDA(cudaMemcpy(m->mask, mk.data(), pb, cudaMemcpyHostToDevice));
    LRS_CUDA(cudaMemset(params, 0, pb));
    LRS_CUDA(cudaMemset(m->mW, 0, pb));
    LRS_CUDA(cudaMemset(m->vW, 0, pb));
    LRS_CUDA(cudaMemset(m->grad, 0, pb));
    *out = m;
    lrs_status rc = refresh_bf16(m, 0);
    if (rc != LRS_OK) return rc;
    LRS_CUDA(cudaDeviceSynchronize());
    return LRS_OK;
}

extern "C" lrs_status lrs_mlp_destroy(lrs_mlp* m) {
    if (!m) return LRS_OK;
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    cudaFree(m->W1);   // start of the packed parameters
    cudaFree(m->mW); cudaFree(m->vW); cudaFree(m->grad); cudaFree(m->mask);
    cudaFree(m->W1b); cudaFree(m->W2b); cudaFree(m->W3b); cudaFree(m->W2t); cudaFree(m->W3t);
    cudaFree(m->err);
    cudaFreeHost(m->err_h);
    cudaFree(m->ws);
    delete m;
    return LRS_OK;
}

extern "C" lrs_status lrs_mlp_set_params(lrs_mlp* m, const float* params_host) {
    if (!m || !params_host) return lrs_fail(LRS_ERR_ARG, "NULL argument");
    LRS_CUDA(cudaSetDevice(m->device));
    const size_t pb = (size_t)m->n_params * sizeof(float);
    LRS_CUDA(cudaMemcpy(m->W1, params_host, pb, cudaMemcpyHostToDevice));
    LRS_CUDA(cudaMemset(m->mW, 0, pb));
    LRS_CUDA(cudaMemset(m->vW, 0, pb));
    m->step = 0;
    lrs_status rc = refresh_bf16(m, 0);
    if (rc != LRS_OK) return rc;
    LRS_CUDA(cudaDeviceSynchronize());
    return LRS_OK;
}

// Reads (and clears) the device flag that a tcgen05 GEMM sets when its completion
// wait gives up; the caller has synchronised the device.
static lrs_status mlp_check_err(lrs_mlp* m) {
    int flag = 0;
    LRS_CUDA(cudaMemcpy(&flag, m->err, sizeof(int), cudaMemcpyDeviceToHost));
    *(volatile int*)m->err_h = 0;
    if (flag) {
        LRS_CUDA(cudaMemset(m->err, 0, sizeof(int)));
        return lrs_fail(LRS_ERR_TIMEOUT, "a tcgen05 GEMM gave up waiting for its MMAs; results are invalid");
    }
    return LRS_OK;
}

// Every enqueuing call ends by copying the device flag into the pinned host word
// (4 bytes, asynchronous) and starts by reading that word: a wait that gave up in an
// earlier call is reported by a later one without synchronising in the common case.
static void mlp_post_err(lrs_mlp* m, cudaStream_t st) {
    cudaMemcpyAsync(m->err_h, m->err, sizeof(int), cudaMemcpyDeviceToHost, st);
}
static lrs_status mlp_poll_err(lrs_mlp* m) {
    if (*(volatile int*)m->err_h == 0) return LRS_OK;
    LRS_CUDA(cudaDeviceSynchronize());   // no copy of the flag is left in flight
    return mlp_check_err(m);
}

extern "C" lrs_status lrs_mlp_debug_inject_wait_timeout(lrs_mlp* m) {
    if (!m) return lrs_fail(LRS_ERR_ARG, "NULL argument");
    LRS_CUDA(cudaSetDevice(m->device));
    const int one = 1;
    LRS_CUDA(cudaMemcpy(m->err + 1, &one, sizeof(int), cudaMemcpyHostToDevice));
    return LRS_OK;
}

extern "C" lrs_status lrs_mlp_get_params(lrs_mlp* m, float* params_host, float* grads_host) {
    if (!m) return lrs_fail(LRS_ERR_ARG, "NULL argument");
    LRS_CUDA(cudaSetDevice(m->device));
    LRS_CUDA(cudaDeviceSynchronize());
    lrs_status rc = mlp_check_err(m);
    if (rc != LRS_OK) return rc;
    const size_t pb = (size_t)m->n_params * sizeof(float);
    if (params_host) LRS_CUDA(cudaMemcpy(params_host, m->W1, pb, cudaMemcpyDeviceToHost));
    if (grads_host) LRS_CUDA(cudaMemcpy(grads_host, m->grad, pb, cudaMemcpyDeviceToHost));
    return LRS_OK;
}

extern "C" lrs_status lrs_mlp_set_gemm(lrs_mlp* m, int32_t kind) {
    if (!m) return lrs_fail(LRS_ERR_ARG, "NULL argument");
    if (kind != LRS_MLP_GEMM_TCGEN05 && kind != LRS_MLP_GEMM_MMA_SYNC)
        return lrs_fail(LRS_ERR_ARG, "unknown GEMM kernel %d", kind);
    LRS_CUDA(cudaSetDevice(m->device));
    LRS_CUDA(cudaDeviceSynchronize());
    lrs_status rc = mlp_check_err(m);
    m->gemm = kind;
    return rc;
}

extern "C" lrs_status lrs_mlp_get_gemm(const lrs_mlp* m, int32_t* kind) {
    if (!m || !kind) return lrs_fail(LRS_ERR_ARG, "NULL argument");
    *kind = m->gemm;
    return LRS_OK;
}

extern "C" lrs_status lrs_mlp_info(const lrs_mlp* m, int32_t* n, int32_t* hidden, int64_t* n_params) {
    if (!m) return lrs_fail(LRS_ERR_ARG, "NULL argument");
    if (n) *n = m->n;
    if (hidden) *hidden = m->H;
    if (n_params) *n_params = m->n_params;
    return LRS_OK;
}

extern "C" lrs_status lrs_mlp_forward(lrs_mlp* m, const uint64_t* x, int64_t batch, float* logits,
                                      float* logq, void* stream) {
    if (!m || batch < 0 || (batch > 0 && !x)) return lrs_fail(LRS_ERR_ARG, "bad arguments");
    if (batch == 0) return LRS_OK;
    if (batch > (1 << 24)) return lrs_fail(LRS_ERR_ARG, "batch too large");
    LRS_CUDA(cudaSetDevice(m->device));
    cudaStream_t st = (cudaStream_t)stream;
    lrs_status rc = mlp_poll_err(m);
    if (rc != LRS_OK) return rc;
    MlpWS w;
    if ((rc = mlp_ws(m, pad64(batch), w)) != LRS_OK) return rc;
    if ((rc = mlp_forward(m, x, (int)batch, w, st)) != LRS_OK) return rc;
    if (logits)
        LRS_CUDA(cudaMemcpy2DAsync(logits, (size_t)m->n * 4, w.logits, (size_t)m->NP * 4, (size_t)m->n * 4,
                                   (size_t)batch, cudaMemcpyDeviceToDevice, st));
    if (logq) {
        k_logq<<<(unsigned)((batch + 127) / 128), 128, 0, st>>>(w.logits, x, (int)batch, m->n, m->NP, logq);
        LRS_LAUNCH_CHECK("logq");
    }
    mlp_post_err(m, st);
    return LRS_OK;
}

extern "C" lrs_status lrs_mlp_backward(lrs_mlp* m, const uint64_t* x, int64_t batch, float* loss,
                                       void* stream) {
    if (!m || batch < 1 || !x) return lrs_fail(LRS_ERR_ARG, "bad arguments");
    if (batch > (1 << 24)) return lrs_fail(LRS_ERR_ARG, "batch too large");
    LRS_CUDA(cudaSetDevice(m->device));
    lrs_status rc = mlp_poll_err(m);
    if (rc != LRS_OK) return rc;
    MlpWS w;
    if ((rc = mlp_ws(m, pad64(batch), w)) != LRS_OK) return rc;
    if ((rc = mlp_backward(m, x, (int)batch, w, loss, (cudaStream_t)stream)) != LRS_OK) return rc;
    mlp_post_err(m, (cudaStream_t)stream);
    return LRS_OK;
}

extern "C" lrs_status lrs_mlp_train_step(lrs_mlp* m, const uint64_t* x, int64_t batch, float lr,
                                         float beta1, float beta2, float eps, float wd, float* loss,
                                         void* stream) {
    lrs_status rc = lrs_mlp_backward(m, x, batch, loss, stream);
    if (rc != LRS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    m->step += 1;
    const float c1 = 1.f - powf(beta1, (float)m->step), c2 = 1.f - powf(beta2, (float)m->step);
    k_adamw<<<(unsigned)((m->n_params + 255) / 256), 256, 0, st>>>(m->W1, m->grad, m->mask, m->mW, m->vW,
                                                                    m->n_params, lr, beta1, beta2, eps, wd,
                                                                    c1, c2);
    LRS_LAUNCH_CHECK("adamw");
    return refresh_bf16(m, st);
}

extern "C" lrs_status lrs_mlp_sample(lrs_mlp* m, int64_t count, uint64_t seed, int64_t sample0,
                                     uint64_t* y, float* logq, void* stream) {
    if (!m || count < 0 || (count > 0 && (!y || !logq))) return lrs_fail(LRS_ERR_ARG, "bad arguments");
    if (count == 0) return LRS_OK;
    if (count > (1 << 24)) return lrs_fail(LRS_ERR_ARG, "count too large");
    LRS_CUDA(cudaSetDevice(m->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int M = (int)count, Mp = pad64(count), H = m->H;
    MlpWS w;
    lrs_status rc = mlp_ws(m, Mp, w);
    if (rc != LRS_OK) return rc;
    if ((rc = mlp_poll_err(m)) != LRS_OK) return rc;
    const int64_t tot = (int64_t)Mp * H;
    k_sample_init<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(m->b1, Mp, H, M, w.Z1, w.H1, y, logq);
    LRS_LAUNCH_CHECK("sample init");
    for (int i = 0; i < m->n; ++i) {
        if ((rc = gemm_tn(m, w.H1, H, m->W2b, H, Mp, H, H, EpiBiasReluBf16{m->b2, w.H2, H}, st)) != LRS_OK) return rc;
        k_sample_bit<<<(unsigned)((M * 32 + 127) / 128), 128, 0, st>>>(w.H2, m->W3b, m->b3, m->W1b, M, H, m->NP,
                                                                     i, seed, sample0, w.Z1, w.H1, y, logq);
        LRS_LAUNCH_CHECK("sample bit");
    }
    mlp_post_err(m, st);
    return LRS_OK;
}
