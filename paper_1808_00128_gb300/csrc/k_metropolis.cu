// Metropolis chains with the incremental Pauli update of Sec. 4.2.
//
// State per (chain c, term alpha): Q = i^mu X(u) Z(w) = U_C^{-1} X(x_c) U_C,
// packed in 12 bytes for n <= 40 and 16 bytes up to n = 62 (q_store), layout
// [chain][term].
// A step proposes y = x ^ e_j; every term updates Q_y = Q_x P_j with
// P_j = U_C^{-1} X_j U_C = i^{gamma_j} X(F_j) Z(M_j):
//     mu += gamma_j + 2 parity(w & F_j);  u ^= F_j;  w ^= M_j
// and contributes b <0|Q_y U_H|s> (Eq. (amplitude1)).  Q is written back only
// for accepted moves, lazily, at the start of the next step.  The accept test
// is done in FP64 per chain by a separate small kernel.
#include <string.h>

#include "lrs_device.cuh"

namespace {

constexpr int MC_TPB = 128;   // threads per block
constexpr int MC_TPT = 2;     // terms per thread
constexpr int MC_TERMS = MC_TPB * MC_TPT;   // terms per block (cap is a multiple of 256)
constexpr int MC_CG = 64;     // chains per block (grid.y groups)

__device__ __forceinline__ float2 block_sum(float2 v, float2 (*red)[MC_TPB / 32], int slot) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    if ((threadIdx.x & 31) == 0) red[slot][threadIdx.x >> 5] = v;
    return v;
}

// b e^{i pi k/4} 2^{-e/2} times i^m (m = mu + 2 sign): the Z8 factor of a term at a
// string, with the term's part (coefficient, phase k, |v| + h) folded in once.
__device__ __forceinline__ float2 times_i_pow(float2 z, uint32_t m) {
    const float2 r = (m & 1u) ? make_float2(-z.y, z.x) : z;
    return (m & 2u) ? make_float2(-r.x, -r.y) : r;
}

// ---- bulk-copy pipeline helpers (1-D cp.async.bulk completing on an mbarrier) ----------
constexpr unsigned long long MC_WAIT_NS = 1000000000ull;   // 1 s
__device__ __forceinline__ uint32_t mc_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long mc_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mc_bar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mc_bar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mc_bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ bool mc_bar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for the phase of the given parity; false after MC_WAIT_NS.
__device__ __forceinline__ bool mc_bar_wait(uint32_t bar, uint32_t parity) {
    if (mc_bar_try(bar, parity)) return true;
    const unsigned long long t0 = mc_ns();
    while (!mc_bar_try(bar, parity))
        if (mc_ns() - t0 > MC_WAIT_NS) return false;
    return true;
}

// One chain's inputs for the block's MC_TERMS terms: its Pauli states and the rows
// F_j, M_j of its proposal and F_p, M_p of its pending accepted flip.
// At most MC_ST chains in flight per block; the launch takes nst <= MC_ST stages
// (a tuning knob: two stages, 24 KB, leave room for eight blocks per SM at n = 40,
// four suit the n = 50 workload).
constexpr int MC_ST = 4;
struct McStage {
    // the chain's Pauli states: MC_TERMS 16-byte pairs, or (compact) MC_TERMS 64-bit
    // words followed by MC_TERMS 32-bit words
    __align__(16) unsigned char q[MC_TERMS * 16];
    uint64_t fj[MC_TERMS], mj[MC_TERMS], fp[MC_TERMS], mp[MC_TERMS];
};

// One proposal: apply the pending accepted flip, then form the amplitude of y.
// The block owns MC_TERMS consecutive terms; for each of its chains thread 0 copies
// the 4 KB of Q and the 2 KB row segments (coalesced [row][term] layout) into a
// shared stage with cp.async.bulk, nst chains ahead, so the HBM stream does not
// depend on how many loads the threads keep in flight.  Q is written back only
// where a pending flip is committed.  Each thread owns MC_TPT terms
// (tid + k * MC_TPB) and sums them before the block reduction.  A stage wait that
// gives up (1 s) sets *err, stops the block and leaves its partial sums unwritten.
template <bool CQ>
__global__ void __launch_bounds__(MC_TPB) k_metro_propose(TermsView T, int64_t C, void* __restrict__ Q,
                                                          const int32_t* __restrict__ pend,
                                                          const int32_t* __restrict__ jprop,
                                                          float2* __restrict__ partial, int64_t n_tiles,
                                                          int cg, int nst, int* err, int groups_fast) {
    extern __shared__ __align__(128) unsigned char mc_dyn[];
    McStage* stage = reinterpret_cast<McStage*>(mc_dyn);
    __shared__ float2 red[MC_CG][MC_TPB / 32];
    __shared__ int32_t spj[MC_CG], spq[MC_CG], sj[MC_CG];
    __shared__ __align__(8) uint64_t full[MC_ST];
    __shared__ int abort_flag;
    const int tid = threadIdx.x;
    // groups_fast: blockIdx.x is the chain group, so the blocks that read the same
    // term tile's rows F_j, M_j run together and share them through L2
    const int64_t tile = groups_fast ? blockIdx.y : blockIdx.x;
    const int64_t c0 = (int64_t)(groups_fast ? blockIdx.x : blockIdx.y) * cg;
    const int nc = (int)(C - c0 < cg ? C - c0 : cg);
    const int64_t a0 = tile * MC_TERMS;
    const int64_t pairs = C * T.cap;   // entries of the Pauli-state arrays
    if (tid < nc) {
        spj[tid] = pend[c0 + tid];
        spq[tid] = pend[C + c0 + tid];
        sj[tid] = jprop[c0 + tid];
    }
    if (tid < MC_ST) mc_bar_init(mc_smem(&full[tid]));
    if (tid == 0) abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    // err[1] is a one-shot test request (lrs_debug_inject_wait_timeout): block (0, 0)
    // takes it and makes its first stage expect 16 bytes that no copy delivers, so the
    // stage's bounded wait runs out
    uint32_t extra = 0;
    if (tid == 0 && blockIdx.x == 0 && blockIdx.y == 0 && *(volatile int*)&err[1] != 0) {
        *(volatile int*)&err[1] = 0;
        extra = 16;
    }
    auto issue = [&](int ci, int si) {   // thread 0: chain ci into stage si
        McStage& S = stage[si];
        const uint32_t bar = mc_smem(&full[si]);
        const int pj = spj[ci], j = sj[ci];
        const int64_t c = c0 + ci;
        const uint32_t qb = CQ ? MC_TERMS * 12 : MC_TERMS * 16;
        mc_bar_expect(bar, (uint32_t)(qb + 2 * sizeof(S.fj) + (pj >= 0 ? 2 * sizeof(S.fp) : 0)) + (ci == 0 ? extra : 0u));
        if (CQ) {
            mc_bulk_load(mc_smem(S.q), reinterpret_cast<const uint64_t*>(Q) + c * T.cap + a0, MC_TERMS * 8, bar);
            mc_bulk_load(mc_smem(S.q + MC_TERMS * 8),
                         reinterpret_cast<const uint32_t*>(reinterpret_cast<const uint64_t*>(Q) + pairs) + c * T.cap + a0,
                         MC_TERMS * 4, bar);
        } else {
            mc_bulk_load(mc_smem(S.q), reinterpret_cast<const ulonglong2*>(Q) + c * T.cap + a0, MC_TERMS * 16, bar);
        }
        mc_bulk_load(mc_smem(S.fj), T.F + (int64_t)j * T.cap + a0, sizeof(S.fj), bar);
        mc_bulk_load(mc_smem(S.mj), T.M + (int64_t)j * T.cap + a0, sizeof(S.mj), bar);
        if (pj >= 0) {
            mc_bulk_load(mc_smem(S.fp), T.F + (int64_t)pj * T.cap + a0, sizeof(S.fp), bar);
            mc_bulk_load(mc_smem(S.mp), T.M + (int64_t)pj * T.cap + a0, sizeof(S.mp), bar);
        }
    };
    if (tid == 0)
        for (int ci = 0; ci < nc && ci < nst; ++ci) issue(ci, ci);

    int tl[MC_TPT];
    uint64_t glo[MC_TPT], ghi[MC_TPT], s[MC_TPT], nv[MC_TPT], sv[MC_TPT];
    float2 base[MC_TPT];
    bool live[MC_TPT];
#pragma unroll
    for (int k = 0; k < MC_TPT; ++k) {
        tl[k] = tid + k * MC_TPB;
        const int64_t a = a0 + tl[k];
        glo[k] = T.glo[a];
        ghi[k] = T.ghi[a];
        const uint64_t v = T.v[a];
        s[k] = T.s[a];
        nv[k] = ~v & T.nmask;
        sv[k] = s[k] & v;
        const uint32_t om = T.omega[a];
        live[k] = ((om >> 3) & 1u) == 0u;
        base[k] = z8_scale(T.coef[a], (int)(om & 7u), __popcll(v) + (int)(om >> 8));
    }
    int ci = 0, si = 0;       // chain, its stage
    uint32_t ph = 0;          // parity of the stage's current phase
    for (; ci < nc; ++ci) {
        const McStage& S = stage[si];
        if (!mc_bar_wait(mc_smem(&full[si]), ph)) abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;   // uniform: read after the barrier
        const int64_t c = c0 + ci;
        const int pj = spj[ci], pq = spq[ci], j = sj[ci];
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < MC_TPT; ++k) {
            uint64_t u, w;
            uint32_t mu;
            if (CQ)
                q_unpack<true>(reinterpret_cast<const uint64_t*>(S.q)[tl[k]],
                               reinterpret_cast<const uint32_t*>(S.q + MC_TERMS * 8)[tl[k]], u, w, mu);
            else
                q_unpack<false>(reinterpret_cast<const ulonglong2*>(S.q)[tl[k]].x,
                                reinterpret_cast<const ulonglong2*>(S.q)[tl[k]].y, u, w, mu);
            if (pj >= 0) {   // commit the flip accepted at the previous step
                const uint64_t Fp = S.fp[tl[k]];
                mu = (mu + (uint32_t)(getb(glo[k], pj) | (getb(ghi[k], pj) << 1)) + 2u * par64(w & Fp)) & 3u;
                u ^= Fp;
                w ^= S.mp[tl[k]];
            }
            if (pq >= 0) {   // the second flip of a two-step pass (rows from global memory)
                const uint64_t Fq = T.F[(int64_t)pq * T.cap + a0 + tl[k]];
                mu = (mu + (uint32_t)(getb(glo[k], pq) | (getb(ghi[k], pq) << 1)) + 2u * par64(w & Fq)) & 3u;
                u ^= Fq;
                w ^= T.M[(int64_t)pq * T.cap + a0 + tl[k]];
            }
            if (pj >= 0 || pq >= 0) q_store<CQ>(Q, pairs, c * T.cap + a0 + tl[k], u, w, mu);
            const uint64_t Fj = S.fj[tl[k]];
            const uint32_t muy =
                (mu + (uint32_t)(getb(glo[k], j) | (getb(ghi[k], j) << 1)) + 2u * par64(w & Fj)) & 3u;
            const uint64_t uy = u ^ Fj, wy = w ^ S.mj[tl[k]];
            if (live[k] && ((uy ^ s[k]) & nv[k]) == 0) {
                const uint32_t sign = par64(uy & wy) ^ par64(uy & sv[k]);
                const float2 t = times_i_pow(base[k], muy + 2u * sign);
                acc.x += t.x;
                acc.y += t.y;
            }
        }
        block_sum(acc, red, ci);
        __syncthreads();   // every thread is done with this stage
        if (tid == 0 && ci + nst < nc) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(ci + nst, si);
        }
        if (++si == nst) {
            si = 0;
            ph ^= 1u;
        }
    }
    if (ci < nc) {
        // gave up: wait (bounded) for the copies still in flight into this block's
        // stages, report, and leave the partial sums unwritten
        if (tid == 0) {
            for (int cj = ci; cj < nc && cj < ci + nst; ++cj) {
                mc_bar_wait(mc_smem(&full[si]), ph);
                if (++si == nst) {
                    si = 0;
                    ph ^= 1u;
                }
            }
            atomicExch(err, 1);
        }
        return;
    }
    if (tid < nc) {
        float2 acc = red[tid][0];
        for (int w2 = 1; w2 < MC_TPB / 32; ++w2) { acc.x += red[tid][w2].x; acc.y += red[tid][w2].y; }
        partial[(c0 + tid) * n_tiles + tile] = acc;
    }
}

// Two steps per pass over the Pauli states.  The proposals j1 = j_t and j2 = j_{t+1}
// are drawn from the counter RNG and do not depend on the chain, so one pass can form
// <y|psi> for every string step t + 1 may propose: y1 = x ^ e_j1 (step t), y1 ^ e_j2
// (step t + 1 after an accepted move) and x ^ e_j2 (after a rejected one), with
// Q_y1 = Q_x P_j1, Q_y1 P_j2 and Q_x P_j2.  The accept kernel then takes both
// decisions in order.  Each term's contribution to each sum is the one a single step
// would add for the same string, in the same order, so the chains are bit-identical to
// single steps; the pass reads Q once per two steps instead of once per step.
// Pending flips: both accepted flips of the previous pass, committed in order.
struct McStage2 {
    __align__(16) unsigned char q[MC_TERMS * 16];
    uint64_t f1[MC_TERMS], m1[MC_TERMS], f2[MC_TERMS], m2[MC_TERMS];   // rows F, M of j1, j2
    uint64_t fp[MC_TERMS], mp[MC_TERMS], fq[MC_TERMS], mq[MC_TERMS];   // rows of the pending flips
};

// b i^m <0|X(u) Z(w) U_H|s> contribution of one term to a sum over terms (Eq. (amplitude1)).
__device__ __forceinline__ void mc_add(float2& acc, float2 base, uint64_t s, uint64_t nv, uint64_t sv,
                                       uint32_t mu, uint64_t u, uint64_t w) {
    if (((u ^ s) & nv) == 0) {
        const uint32_t sign = par64(u & w) ^ par64(u & sv);
        const float2 t = times_i_pow(base, mu + 2u * sign);
        acc.x += t.x;
        acc.y += t.y;
    }
}

template <bool CQ>
__global__ void __launch_bounds__(MC_TPB) k_metro_propose2(TermsView T, int64_t C, void* __restrict__ Q,
                                                           const int32_t* __restrict__ pend,
                                                           const int32_t* __restrict__ jprop,
                                                           float2* __restrict__ partial, int64_t n_tiles,
                                                           int cg, int nst, int* err, int groups_fast) {
    extern __shared__ __align__(128) unsigned char mc_dyn[];
    McStage2* stage = reinterpret_cast<McStage2*>(mc_dyn);
    __shared__ float2 red[3 * MC_CG][MC_TPB / 32];
    __shared__ int32_t sp1[MC_CG], sp2[MC_CG], sj1[MC_CG], sj2[MC_CG];
    __shared__ __align__(8) uint64_t full[MC_ST];
    __shared__ int abort_flag;
    const int tid = threadIdx.x;
    const int64_t tile = groups_fast ? blockIdx.y : blockIdx.x;
    const int64_t c0 = (int64_t)(groups_fast ? blockIdx.x : blockIdx.y) * cg;
    const int nc = (int)(C - c0 < cg ? C - c0 : cg);
    const int64_t a0 = tile * MC_TERMS;
    const int64_t pairs = C * T.cap;
    if (tid < nc) {
        sp1[tid] = pend[c0 + tid];
        sp2[tid] = pend[C + c0 + tid];
        sj1[tid] = jprop[c0 + tid];
        sj2[tid] = jprop[C + c0 + tid];
    }
    if (tid < MC_ST) mc_bar_init(mc_smem(&full[tid]));
    if (tid == 0) abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    // one-shot test request, as in k_metro_propose
    uint32_t extra = 0;
    if (tid == 0 && blockIdx.x == 0 && blockIdx.y == 0 && *(volatile int*)&err[1] != 0) {
        *(volatile int*)&err[1] = 0;
        extra = 16;
    }
    auto issue = [&](int ci, int si) {   // thread 0: chain ci into stage si
        McStage2& S = stage[si];
        const uint32_t bar = mc_smem(&full[si]);
        const int p1 = sp1[ci], p2 = sp2[ci], j1 = sj1[ci], j2 = sj2[ci];
        const int64_t c = c0 + ci;
        const uint32_t qb = CQ ? MC_TERMS * 12 : MC_TERMS * 16;
        const uint32_t rb = (uint32_t)sizeof(S.f1);
        mc_bar_expect(bar, qb + 4 * rb + (p1 >= 0 ? 2 * rb : 0u) + (p2 >= 0 ? 2 * rb : 0u) + (ci == 0 ? extra : 0u));
        if (CQ) {
            mc_bulk_load(mc_smem(S.q), reinterpret_cast<const uint64_t*>(Q) + c * T.cap + a0, MC_TERMS * 8, bar);
            mc_bulk_load(mc_smem(S.q + MC_TERMS * 8),
                         reinterpret_cast<const uint32_t*>(reinterpret_cast<const uint64_t*>(Q) + pairs) + c * T.cap + a0,
                         MC_TERMS * 4, bar);
        } else {
            mc_bulk_load(mc_smem(S.q), reinterpret_cast<const ulonglong2*>(Q) + c * T.cap + a0, MC_TERMS * 16, bar);
        }
        mc_bulk_load(mc_smem(S.f1), T.F + (int64_t)j1 * T.cap + a0, rb, bar);
        mc_bulk_load(mc_smem(S.m1), T.M + (int64_t)j1 * T.cap + a0, rb, bar);
        mc_bulk_load(mc_smem(S.f2), T.F + (int64_t)j2 * T.cap + a0, rb, bar);
        mc_bulk_load(mc_smem(S.m2), T.M + (int64_t)j2 * T.cap + a0, rb, bar);
        if (p1 >= 0) {
            mc_bulk_load(mc_smem(S.fp), T.F + (int64_t)p1 * T.cap + a0, rb, bar);
            mc_bulk_load(mc_smem(S.mp), T.M + (int64_t)p1 * T.cap + a0, rb, bar);
        }
        if (p2 >= 0) {
            mc_bulk_load(mc_smem(S.fq), T.F + (int64_t)p2 * T.cap + a0, rb, bar);
            mc_bulk_load(mc_smem(S.mq), T.M + (int64_t)p2 * T.cap + a0, rb, bar);
        }
    };
    if (tid == 0)
        for (int ci = 0; ci < nc && ci < nst; ++ci) issue(ci, ci);

    int tl[MC_TPT];
    uint64_t glo[MC_TPT], ghi[MC_TPT], s[MC_TPT], nv[MC_TPT], sv[MC_TPT];
    float2 base[MC_TPT];
    bool live[MC_TPT];
#pragma unroll
    for (int k = 0; k < MC_TPT; ++k) {
        tl[k] = tid + k * MC_TPB;
        const int64_t a = a0 + tl[k];
        glo[k] = T.glo[a];
        ghi[k] = T.ghi[a];
        const uint64_t v = T.v[a];
        s[k] = T.s[a];
        nv[k] = ~v & T.nmask;
        sv[k] = s[k] & v;
        const uint32_t om = T.omega[a];
        live[k] = ((om >> 3) & 1u) == 0u;
        base[k] = z8_scale(T.coef[a], (int)(om & 7u), __popcll(v) + (int)(om >> 8));
    }
    int ci = 0, si = 0;
    uint32_t ph = 0;
    for (; ci < nc; ++ci) {
        const McStage2& S = stage[si];
        if (!mc_bar_wait(mc_smem(&full[si]), ph)) abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;   // uniform: read after the barrier
        const int64_t c = c0 + ci;
        const int p1 = sp1[ci], p2 = sp2[ci], j1 = sj1[ci], j2 = sj2[ci];
        float2 acc1 = make_float2(0.f, 0.f), acc2a = acc1, acc2r = acc1;
#pragma unroll
        for (int k = 0; k < MC_TPT; ++k) {
            uint64_t u, w;
            uint32_t mu;
            if (CQ)
                q_unpack<true>(reinterpret_cast<const uint64_t*>(S.q)[tl[k]],
                               reinterpret_cast<const uint32_t*>(S.q + MC_TERMS * 8)[tl[k]], u, w, mu);
            else
                q_unpack<false>(reinterpret_cast<const ulonglong2*>(S.q)[tl[k]].x,
                                reinterpret_cast<const ulonglong2*>(S.q)[tl[k]].y, u, w, mu);
            if (p1 >= 0) {   // commit the flips accepted in the previous pass, in order
                const uint64_t Fp = S.fp[tl[k]];
                mu = (mu + (uint32_t)(getb(glo[k], p1) | (getb(ghi[k], p1) << 1)) + 2u * par64(w & Fp)) & 3u;
                u ^= Fp;
                w ^= S.mp[tl[k]];
            }
            if (p2 >= 0) {
                const uint64_t Fq = S.fq[tl[k]];
                mu = (mu + (uint32_t)(getb(glo[k], p2) | (getb(ghi[k], p2) << 1)) + 2u * par64(w & Fq)) & 3u;
                u ^= Fq;
                w ^= S.mq[tl[k]];
            }
            if (p1 >= 0 || p2 >= 0) q_store<CQ>(Q, pairs, c * T.cap + a0 + tl[k], u, w, mu);
            if (!live[k]) continue;
            const uint64_t F1 = S.f1[tl[k]], M1 = S.m1[tl[k]], F2 = S.f2[tl[k]], M2 = S.m2[tl[k]];
            const uint32_t g1 = (uint32_t)(getb(glo[k], j1) | (getb(ghi[k], j1) << 1));
            const uint32_t g2 = (uint32_t)(getb(glo[k], j2) | (getb(ghi[k], j2) << 1));
            // y1 = x ^ e_j1
            const uint32_t mu1 = (mu + g1 + 2u * par64(w & F1)) & 3u;
            const uint64_t u1 = u ^ F1, w1 = w ^ M1;
            mc_add(acc1, base[k], s[k], nv[k], sv[k], mu1, u1, w1);
            // y1 ^ e_j2 (step t accepted)
            mc_add(acc2a, base[k], s[k], nv[k], sv[k], (mu1 + g2 + 2u * par64(w1 & F2)) & 3u, u1 ^ F2, w1 ^ M2);
            // x ^ e_j2 (step t rejected)
            mc_add(acc2r, base[k], s[k], nv[k], sv[k], (mu + g2 + 2u * par64(w & F2)) & 3u, u ^ F2, w ^ M2);
        }
        block_sum(acc1, red, 3 * ci);
        block_sum(acc2a, red, 3 * ci + 1);
        block_sum(acc2r, red, 3 * ci + 2);
        __syncthreads();   // every thread is done with this stage
        if (tid == 0 && ci + nst < nc) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(ci + nst, si);
        }
        if (++si == nst) {
            si = 0;
            ph ^= 1u;
        }
    }
    if (ci < nc) {
        // gave up: wait (bounded) for the copies still in flight, report, and leave the
        // partial sums unwritten
        if (tid == 0) {
            for (int cj = ci; cj < nc && cj < ci + nst; ++cj) {
                mc_bar_wait(mc_smem(&full[si]), ph);
                if (++si == nst) {
                    si = 0;
                    ph ^= 1u;
                }
            }
            atomicExch(err, 1);
        }
        return;
    }
    for (int e = tid; e < 3 * nc; e += MC_TPB) {   // sum r of chain cc: [r][chain][tile]
        const int cc = e / 3, r = e - 3 * cc;
        float2 acc = red[e][0];
        for (int w2 = 1; w2 < MC_TPB / 32; ++w2) { acc.x += red[e][w2].x; acc.y += red[e][w2].y; }
        partial[((int64_t)r * C + c0 + cc) * n_tiles + tile] = acc;
    }
}

__device__ __forceinline__ double chain_reduce(const float2* __restrict__ partial, int64_t c,
                                               int64_t n_tiles) {
    double re = 0.0, im = 0.0;
    for (int64_t t = threadIdx.x; t < n_tiles; t += blockDim.x) {
        const float2 p = partial[c * n_tiles + t];
        re += (double)p.x;
        im += (double)p.y;
    }
    __shared__ double sre[256], sim[256];
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            sre[threadIdx.x] += sre[threadIdx.x + off];
            sim[threadIdx.x] += sim[threadIdx.x + off];
        }
        __syncthreads();
    }
    return sre[0] * sre[0] + sim[0] * sim[0];
}

__device__ __forceinline__ int draw_j(uint64_t seed, int64_t c, int64_t step, int n) {
    const uint64_t r = sm64_at(sm64_key(seed, (uint64_t)c), (uint64_t)(2 * step));
    return (int)(((r >> 32) * (uint64_t)n) >> 32);
}

__global__ void k_chains_set(const double* __restrict__ amp, int64_t C, const uint64_t* xs, uint64_t nmask,
                             uint64_t* cx, double* cp, int32_t* pend) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const double re = amp[2 * c], im = amp[2 * c + 1];
    cx[c] = xs[c] & nmask;
    cp[c] = re * re + im * im;
    pend[c] = -1;
    pend[C + c] = -1;
}

// Per-call parameters live in device memory so that a captured graph of steps
// can be replayed: step t of a launch uses global step P->step0 + t.
__global__ void k_mc_set(McParams* P, uint64_t seed, int64_t step0) {
    P->seed = seed;
    P->step0 = step0;
}
__global__ void k_mc_advance(McParams* P, int64_t by) { P->step0 += by; }

__global__ void k_metro_first(int64_t C, const McParams* __restrict__ P, int n, int32_t* jprop, int32_t* jprop2) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    jprop[c] = draw_j(P->seed, c, P->step0, n);
    if (jprop2) jprop2[c] = draw_j(P->seed, c, P->step0 + 1, n);
}

// FP64 accept test (Sec. 4.2) and the proposal index of the next step.
__global__ void k_metro_accept(const float2* __restrict__ partial, int64_t n_tiles,
                               const McParams* __restrict__ P, int64_t t, int n, uint64_t* cx, double* cp,
                               int32_t* pend, int32_t* jprop, uint64_t* trace, int64_t C) {
    const int64_t c = blockIdx.x;
    const double py = chain_reduce(partial, c, n_tiles);
    const uint64_t seed = P->seed;
    const int64_t step = P->step0 + t;
    if (threadIdx.x == 0) {
        const double px = cp[c];
        const int j = jprop[c];
        bool acc;
        if (py >= px) {
            acc = true;
        } else {
            const double r = sm64_unit(sm64_at(sm64_key(seed, (uint64_t)c), (uint64_t)(2 * step + 1)));
            acc = r < py / px;
        }
        if (acc) {
            cx[c] ^= 1ull << j;
            cp[c] = py;
            pend[c] = j;
        } else {
            pend[c] = -1;
        }
        pend[C + c] = -1;
        if (trace) trace[c] = cx[c];
        jprop[c] = draw_j(seed, c, step + 1, n);
    }
}

// The two decisions of a two-step pass (steps t and t + 1), each the FP64 test of
// k_metro_accept with the same draws: step t + 1 compares the sum of the string it
// proposes from the state step t left.  Sums in partial: [0] y1, [1] y1 ^ e_j2,
// [2] x ^ e_j2; proposals j1 = jprop[c], j2 = jprop[C + c].
__global__ void k_metro_accept2(const float2* __restrict__ partial, int64_t n_tiles,
                                const McParams* __restrict__ P, int64_t t, int n, uint64_t* cx, double* cp,
                                int32_t* pend, int32_t* jprop, uint64_t* trace, int64_t C) {
    const int64_t c = blockIdx.x;
    const double p1 = chain_reduce(partial, c, n_tiles);
    __syncthreads();   // every thread has read the first result before the shared sums are reused
    const double p2a = chain_reduce(partial + C * n_tiles, c, n_tiles);
    __syncthreads();
    const double p2r = chain_reduce(partial + 2 * C * n_tiles, c, n_tiles);
    if (threadIdx.x == 0) {
        const uint64_t seed = P->seed;
        const uint64_t key = sm64_key(seed, (uint64_t)c);
        const int64_t step = P->step0 + t;
        const int j1 = jprop[c], j2 = jprop[C + c];
        uint64_t x = cx[c];
        double px = cp[c];
        bool a1;
        if (p1 >= px) a1 = true;
        else a1 = sm64_unit(sm64_at(key, (uint64_t)(2 * step + 1))) < p1 / px;
        if (a1) {
            x ^= 1ull << j1;
            px = p1;
        }
        if (trace) trace[c] = x;
        const double py = a1 ? p2a : p2r;
        bool a2;
        if (py >= px) a2 = true;
        else a2 = sm64_unit(sm64_at(key, (uint64_t)(2 * (step + 1) + 1))) < py / px;
        if (a2) {
            x ^= 1ull << j2;
            px = py;
        }
        if (trace) trace[C + c] = x;
        cx[c] = x;
        cp[c] = px;
        pend[c] = a1 ? j1 : -1;
        pend[C + c] = a2 ? j2 : -1;
        jprop[c] = draw_j(seed, c, step + 2, n);
        jprop[C + c] = draw_j(seed, c, step + 3, n);
    }
}

// Metropolis-Hastings with an independent learned proposal q: accept y with
// probability min(1, P(y) q(x) / (P(x) q(y))), FP64; the uniform of step t of
// chain c is uniform(seed, c, t).
__global__ void k_mh_accept(const double* __restrict__ ampy, const uint64_t* __restrict__ y,
                            const float* __restrict__ lqy, uint64_t seed, int64_t step, int64_t C,
                            uint64_t* cx, double* cp, float* lqx, uint64_t* trace, int64_t* accepts) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const double py = ampy[2 * c] * ampy[2 * c] + ampy[2 * c + 1] * ampy[2 * c + 1];
    const double px = cp[c];
    bool acc;
    if (px <= 0.0) {
        acc = true;
    } else {
        const double ratio = (py / px) * exp((double)lqx[c] - (double)lqy[c]);
        const double r = sm64_unit(sm64_at(sm64_key(seed, (uint64_t)c), (uint64_t)step));
        acc = ratio >= 1.0 || r < ratio;
    }
    if (acc) {
        cx[c] = y[c];
        cp[c] = py;
        lqx[c] = lqy[c];
        if (accepts) accepts[c] += 1;
    }
    if (trace) trace[c] = cx[c];
}

// Term-sharded steps: the FP64 sum over tiles of each chain's partial <y|psi_shard>
// (not squared: the shards' sums add before P(y) is formed).
__global__ void k_metro_partial_out(const float2* __restrict__ partial, int64_t n_tiles, double* __restrict__ amp) {
    const int64_t c = blockIdx.x;
    double re = 0.0, im = 0.0;
    for (int64_t t = threadIdx.x; t < n_tiles; t += blockDim.x) {
        const float2 p = partial[c * n_tiles + t];
        re += (double)p.x;
        im += (double)p.y;
    }
    __shared__ double sre[256], sim[256];
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            sre[threadIdx.x] += sre[threadIdx.x + off];
            sim[threadIdx.x] += sim[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        amp[2 * c] = sre[0];
        amp[2 * c + 1] = sim[0];
    }
}

// The FP64 accept test of step `step` (Sec. 4.2) on the summed amplitudes of the
// proposals: the same rule and draws as k_metro_accept.
__global__ void k_metro_accept_amp(const double* __restrict__ amp, int64_t C, uint64_t seed, int64_t step,
                                   const int32_t* __restrict__ jprop, uint64_t* cx, double* cp, int32_t* pend,
                                   uint64_t* trace) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const double py = amp[2 * c] * amp[2 * c] + amp[2 * c + 1] * amp[2 * c + 1];
    const double px = cp[c];
    const int j = jprop[c];
    bool acc;
    if (py >= px) {
        acc = true;
    } else {
        const double r = sm64_unit(sm64_at(sm64_key(seed, (uint64_t)c), (uint64_t)(2 * step + 1)));
        acc = r < py / px;
    }
    if (acc) {
        cx[c] ^= 1ull << j;
        cp[c] = py;
        pend[c] = j;
    } else {
        pend[c] = -1;
    }
    pend[C + c] = -1;
    if (trace) trace[c] = cx[c];
}

__global__ void k_chains_set_prob(const double* __restrict__ amp, int64_t C, double* cp) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < C) cp[c] = amp[2 * c] * amp[2 * c] + amp[2 * c + 1] * amp[2 * c + 1];
}

__global__ void k_metro_out(int64_t C, const uint64_t* cx, const double* cp, uint64_t* x_out,
                            double* p_out) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    if (x_out) x_out[c] = cx[c];
    if (p_out) p_out[c] = cp[c];
}

}  // namespace

lrs_status launch_chains_init(lrs_ctx* ctx, const uint64_t* x, cudaStream_t st) {
    // Q of every (chain, term) and <x_c|psi> by the amplitude kernel (Four-Russians
    // tables of the Pauli accumulator), then the chain scalars
    const int64_t C = ctx->n_chains;
    double* amp = nullptr;
    lrs_status rc = launch_amplitude_q(ctx, x, C, ctx->Q, &amp, st);
    if (rc != LRS_OK) return rc;
    k_chains_set<<<(unsigned)((C + 127) / 128), 128, 0, st>>>(amp, C, x, ctx->nmask, ctx->cx, ctx->cp, ctx->pend);
    LRS_LAUNCH_CHECK("chains_set kernel");
    return LRS_OK;
}

// Enqueue steps t0 .. t0 + count - 1 (relative to P->step0) of the flip chains.
static lrs_status enqueue_steps(lrs_ctx* ctx, int64_t t0, int64_t count, float2* partial, int32_t* jprop,
                                uint64_t* trace, cudaStream_t st) {
    const int64_t C = ctx->n_chains;
    const int64_t n_tiles = ctx->cap / MC_TERMS;
    const int cg = (int)ctx->tune_mc_cg;
    // chain groups fastest (the rows of a tile are read from DRAM once per step, not once
    // per group); tiles along x when they exceed the grid's y limit
    const int64_t groups = (C + cg - 1) / cg;
    const int gf = n_tiles <= 65535 ? 1 : 0;
    dim3 grid = gf ? dim3((unsigned)groups, (unsigned)n_tiles) : dim3((unsigned)n_tiles, (unsigned)groups);
    const int nst = (int)ctx->tune_mc_stages;
    int64_t t = t0;
    if (ctx->tune_mc_lookahead == 2) {
        for (; t + 1 < t0 + count; t += 2) {
            if (q_compact(ctx->n))
                k_metro_propose2<true><<<grid, MC_TPB, nst * sizeof(McStage2), st>>>(
                    ctx->view(), C, ctx->Q, ctx->pend, jprop, partial, n_tiles, cg, nst, ctx->mc_err_d, gf);
            else
                k_metro_propose2<false><<<grid, MC_TPB, nst * sizeof(McStage2), st>>>(
                    ctx->view(), C, ctx->Q, ctx->pend, jprop, partial, n_tiles, cg, nst, ctx->mc_err_d, gf);
            LRS_LAUNCH_CHECK("metropolis two-step propose kernel");
            k_metro_accept2<<<(unsigned)C, 256, 0, st>>>(partial, n_tiles, ctx->mc_par, t, ctx->n, ctx->cx,
                                                          ctx->cp, ctx->pend, jprop,
                                                          trace ? trace + t * C : nullptr, C);
            LRS_LAUNCH_CHECK("metropolis two-step accept kernel");
        }
    }
    for (; t < t0 + count; ++t) {
        if (q_compact(ctx->n))
            k_metro_propose<true><<<grid, MC_TPB, nst * sizeof(McStage), st>>>(
                ctx->view(), C, ctx->Q, ctx->pend, jprop, partial, n_tiles, cg, nst, ctx->mc_err_d, gf);
        else
            k_metro_propose<false><<<grid, MC_TPB, nst * sizeof(McStage), st>>>(
                ctx->view(), C, ctx->Q, ctx->pend, jprop, partial, n_tiles, cg, nst, ctx->mc_err_d, gf);
        LRS_LAUNCH_CHECK("metropolis propose kernel");
        k_metro_accept<<<(unsigned)C, 256, 0, st>>>(partial, n_tiles, ctx->mc_par, t, ctx->n, ctx->cx,
                                                     ctx->cp, ctx->pend, jprop,
                                                     trace ? trace + t * C : nullptr, C);
        LRS_LAUNCH_CHECK("metropolis accept kernel");
    }
    return LRS_OK;
}

// One CUDA graph holding LRS_MC_GRAPH_STEPS steps followed by step0 += steps;
// rebuilt whenever the buffers it was captured with change.
static lrs_status mc_graph(lrs_ctx* ctx, float2* partial, int32_t* jprop, cudaGraphExec_t* out) {
    const void* key[6] = {partial, jprop, ctx->Q, ctx->F,
                          (void*)(intptr_t)(((ctx->n_chains * 128 + ctx->tune_mc_cg) * 8 + ctx->tune_mc_stages) * 4 +
                                            ctx->tune_mc_lookahead),
                          (void*)(intptr_t)ctx->cap};
    if (ctx->mc_exec && memcmp(key, ctx->mc_key, sizeof(key)) == 0) {
        *out = (cudaGraphExec_t)ctx->mc_exec;
        return LRS_OK;
    }
    if (ctx->mc_exec) cudaGraphExecDestroy((cudaGraphExec_t)ctx->mc_exec);
    ctx->mc_exec = nullptr;
    if (!ctx->cap_stream) LRS_CUDA(cudaStreamCreateWithFlags((cudaStream_t*)&ctx->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = (cudaStream_t)ctx->cap_stream;
    LRS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    lrs_status rc = enqueue_steps(ctx, 0, LRS_MC_GRAPH_STEPS, partial, jprop, nullptr, cs);
    if (rc == LRS_OK) {
        k_mc_advance<<<1, 1, 0, cs>>>(ctx->mc_par, LRS_MC_GRAPH_STEPS);
        if (cudaGetLastError() != cudaSuccess) rc = lrs_fail(LRS_ERR_CUDA, "graph advance kernel");
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (rc != LRS_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return lrs_cuda_check(e, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return lrs_cuda_check(e, "cudaGraphInstantiate");
    ctx->mc_exec = ex;
    memcpy(ctx->mc_key, key, sizeof(key));
    *out = ex;
    return LRS_OK;
}

// The mapped host words of the propose kernels: [0] a stage wait gave up, [1] a
// one-shot test request (lrs_debug_inject_wait_timeout).
lrs_status mc_flags(lrs_ctx* ctx) {
    if (ctx->mc_err_h) return LRS_OK;
    LRS_CUDA(cudaHostAlloc((void**)&ctx->mc_err_h, 2 * sizeof(int), cudaHostAllocMapped));
    ctx->mc_err_h[0] = 0;
    ctx->mc_err_h[1] = 0;
    LRS_CUDA(cudaHostGetDevicePointer((void**)&ctx->mc_err_d, ctx->mc_err_h, 0));
    return LRS_OK;
}

lrs_status launch_metropolis(lrs_ctx* ctx, int64_t steps, uint64_t seed, int64_t step0,
                             uint64_t* x_out, double* p_out, uint64_t* trace, cudaStream_t st) {
    const int64_t C = ctx->n_chains;
    const int64_t n_tiles = ctx->cap / MC_TERMS;
    void* scr = nullptr;
    // partial sums: three per chain and tile for two-step passes; proposals j_t, j_{t+1}
    const size_t part_bytes = 3 * (size_t)C * n_tiles * sizeof(float2);
    lrs_status rc = lrs_scratch(ctx, part_bytes + 2 * (size_t)C * sizeof(int32_t) + 256, &scr);
    if (rc != LRS_OK) return rc;
    if (!ctx->mc_par) LRS_CUDA(cudaMalloc(&ctx->mc_par, sizeof(McParams)));
    lrs_status rf = mc_flags(ctx);
    if (rf != LRS_OK) return rf;
    if (*(volatile int*)ctx->mc_err_h) {   // set by an earlier propose launch that gave up waiting
        *(volatile int*)ctx->mc_err_h = 0;
        return lrs_fail(LRS_ERR_TIMEOUT, "a Metropolis propose kernel gave up waiting for its copies");
    }
    // inside a graph capture: the attributes were set by an earlier uncaptured call, and
    // the steps are captured as plain launches (no nested graph)
    const bool capturing = lrs_capturing(st);
    if (!capturing) {
        LRS_CUDA(cudaFuncSetAttribute(k_metro_propose<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(MC_ST * sizeof(McStage))));
        LRS_CUDA(cudaFuncSetAttribute(k_metro_propose<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(MC_ST * sizeof(McStage))));
        LRS_CUDA(cudaFuncSetAttribute(k_metro_propose2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(MC_ST * sizeof(McStage2))));
        LRS_CUDA(cudaFuncSetAttribute(k_metro_propose2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(MC_ST * sizeof(McStage2))));
    }
    float2* partial = (float2*)scr;
    int32_t* jprop = (int32_t*)((char*)scr + ((part_bytes + 255) & ~(size_t)255));
    k_mc_set<<<1, 1, 0, st>>>(ctx->mc_par, seed, step0);
    k_metro_first<<<(unsigned)((C + 127) / 128), 128, 0, st>>>(C, ctx->mc_par, ctx->n, jprop, jprop + C);
    LRS_LAUNCH_CHECK("metropolis first kernel");
    int64_t done = 0;
    if (!trace && !capturing && steps >= LRS_MC_GRAPH_STEPS) {
        // replay a captured graph of LRS_MC_GRAPH_STEPS steps (one launch instead of 2 per step)
        cudaGraphExec_t ex = nullptr;
        rc = mc_graph(ctx, partial, jprop, &ex);
        if (rc != LRS_OK) return rc;
        for (; done + LRS_MC_GRAPH_STEPS <= steps; done += LRS_MC_GRAPH_STEPS)
            LRS_CUDA(cudaGraphLaunch(ex, st));
    }
    rc = enqueue_steps(ctx, trace ? 0 : 0, steps - done, partial, jprop, trace, st);
    if (rc != LRS_OK) return rc;
    k_metro_out<<<(unsigned)((C + 127) / 128), 128, 0, st>>>(C, ctx->cx, ctx->cp, x_out, p_out);
    LRS_LAUNCH_CHECK("metropolis out kernel");
    return LRS_OK;
}

// One term-sharded proposal: every chain's partial amplitude of its proposal y over
// this context's terms (the pending flip of the previous step is applied to Q first).
lrs_status launch_metropolis_propose(lrs_ctx* ctx, uint64_t seed, int64_t step, double* amp, cudaStream_t st) {
    const int64_t C = ctx->n_chains;
    const int64_t n_tiles = ctx->cap / MC_TERMS;
    void* scr = nullptr;
    lrs_status rc = lrs_scratch(ctx, (size_t)C * n_tiles * sizeof(float2), &scr);
    if (rc != LRS_OK) return rc;
    if (!ctx->mc_par) LRS_CUDA(cudaMalloc(&ctx->mc_par, sizeof(McParams)));
    size_t have = ctx->jbuf_bytes;
    if ((rc = lrs_ensure((void**)&ctx->jbuf, &have, (size_t)C * sizeof(int32_t))) != LRS_OK) return rc;
    ctx->jbuf_bytes = have;
    if ((rc = mc_flags(ctx)) != LRS_OK) return rc;
    if (*(volatile int*)ctx->mc_err_h) {
        *(volatile int*)ctx->mc_err_h = 0;
        return lrs_fail(LRS_ERR_TIMEOUT, "a Metropolis propose kernel gave up waiting for its copies");
    }
    if (!lrs_capturing(st)) {
        LRS_CUDA(cudaFuncSetAttribute(k_metro_propose<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(MC_ST * sizeof(McStage))));
        LRS_CUDA(cudaFuncSetAttribute(k_metro_propose<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(MC_ST * sizeof(McStage))));
    }
    k_mc_set<<<1, 1, 0, st>>>(ctx->mc_par, seed, step);
    k_metro_first<<<(unsigned)((C + 127) / 128), 128, 0, st>>>(C, ctx->mc_par, ctx->n, ctx->jbuf, nullptr);
    LRS_LAUNCH_CHECK("metropolis first kernel");
    const int cg = (int)ctx->tune_mc_cg;
    const int64_t groups = (C + cg - 1) / cg;
    const int gf = n_tiles <= 65535 ? 1 : 0;
    dim3 grid = gf ? dim3((unsigned)groups, (unsigned)n_tiles) : dim3((unsigned)n_tiles, (unsigned)groups);
    const int nst = (int)ctx->tune_mc_stages;
    float2* partial = (float2*)scr;
    if (q_compact(ctx->n))
        k_metro_propose<true><<<grid, MC_TPB, nst * sizeof(McStage), st>>>(
            ctx->view(), C, ctx->Q, ctx->pend, ctx->jbuf, partial, n_tiles, cg, nst, ctx->mc_err_d, gf);
    else
        k_metro_propose<false><<<grid, MC_TPB, nst * sizeof(McStage), st>>>(
            ctx->view(), C, ctx->Q, ctx->pend, ctx->jbuf, partial, n_tiles, cg, nst, ctx->mc_err_d, gf);
    LRS_LAUNCH_CHECK("metropolis propose kernel");
    k_metro_partial_out<<<(unsigned)C, 256, 0, st>>>(partial, n_tiles, amp);
    LRS_LAUNCH_CHECK("metropolis partial amplitude kernel");
    return LRS_OK;
}

lrs_status launch_metropolis_accept(lrs_ctx* ctx, const double* amp, uint64_t seed, int64_t step, uint64_t* trace,
                                    cudaStream_t st) {
    const int64_t C = ctx->n_chains;
    k_metro_accept_amp<<<(unsigned)((C + 127) / 128), 128, 0, st>>>(amp, C, seed, step, ctx->jbuf, ctx->cx, ctx->cp,
                                                                     ctx->pend, trace);
    LRS_LAUNCH_CHECK("metropolis accept kernel");
    return LRS_OK;
}

lrs_status launch_chains_set_prob(lrs_ctx* ctx, const double* amp, cudaStream_t st) {
    const int64_t C = ctx->n_chains;
    k_chains_set_prob<<<(unsigned)((C + 127) / 128), 128, 0, st>>>(amp, C, ctx->cp);
    LRS_LAUNCH_CHECK("chain probability kernel");
    return LRS_OK;
}

lrs_status launch_metropolis_learned(lrs_ctx* ctx, lrs_mlp* mlp, int64_t steps, uint64_t seed, int64_t step0,
                                     uint64_t* x_out, double* p_out, uint64_t* trace, int64_t* accepts,
                                     cudaStream_t st) {
    const int64_t C = ctx->n_chains;
    if (C > ctx->mh_cap) {
        cudaFree(ctx->ybuf); cudaFree(ctx->lqy); cudaFree(ctx->lqx); cudaFree(ctx->ampy);
        ctx->ybuf = nullptr; ctx->lqy = nullptr; ctx->lqx = nullptr; ctx->ampy = nullptr;
        ctx->mh_cap = 0;
        LRS_CUDA(cudaMalloc(&ctx->ybuf, (size_t)C * sizeof(uint64_t)));
        LRS_CUDA(cudaMalloc(&ctx->lqy, (size_t)C * sizeof(float)));
        LRS_CUDA(cudaMalloc(&ctx->lqx, (size_t)C * sizeof(float)));
        LRS_CUDA(cudaMalloc(&ctx->ampy, (size_t)C * 2 * sizeof(double)));
        ctx->mh_cap = C;
    }
    // log q of the current states under the current network
    lrs_status rc = lrs_mlp_forward(mlp, ctx->cx, C, nullptr, ctx->lqx, st);
    if (rc != LRS_OK) return rc;
    for (int64_t t = 0; t < steps; ++t) {
        const int64_t step = step0 + t;
        rc = lrs_mlp_sample(mlp, C, seed, step * C, ctx->ybuf, ctx->lqy, st);
        if (rc != LRS_OK) return rc;
        rc = launch_amplitude(ctx, ctx->ybuf, C, ctx->ampy, nullptr, st);
        if (rc != LRS_OK) return rc;
        k_mh_accept<<<(unsigned)((C + 127) / 128), 128, 0, st>>>(ctx->ampy, ctx->ybuf, ctx->lqy, seed, step, C,
                                                                  ctx->cx, ctx->cp, ctx->lqx,
                                                                  trace ? trace + t * C : nullptr, accepts);
        LRS_LAUNCH_CHECK("learned MH accept kernel");
    }
    ctx->q_stale = true;
    k_metro_out<<<(unsigned)((C + 127) / 128), 128, 0, st>>>(C, ctx->cx, ctx->cp, x_out, p_out);
    LRS_LAUNCH_CHECK("metropolis out kernel");
    return LRS_OK;
}

// Rebuild Q for the chains' current strings (after learned moves).  The strings are
// copied into the learned proposal's buffer (free at this point) because chains_set
// rewrites cx.
lrs_status launch_chains_refresh(lrs_ctx* ctx, cudaStream_t st) {
    const int64_t C = ctx->n_chains;
    if (!ctx->ybuf || ctx->mh_cap < C) return lrs_fail(LRS_ERR_STATE, "chain refresh without a learned-move buffer");
    LRS_CUDA(cudaMemcpyAsync(ctx->ybuf, ctx->cx, (size_t)C * 8, cudaMemcpyDeviceToDevice, st));
    double* amp = nullptr;
    lrs_status rc = launch_amplitude_q(ctx, ctx->ybuf, C, ctx->Q, &amp, st);
    if (rc != LRS_OK) return rc;
    k_chains_set<<<(unsigned)((C + 127) / 128), 128, 0, st>>>(amp, C, ctx->ybuf, ctx->nmask, ctx->cx, ctx->cp,
                                                            ctx->pend);
    LRS_LAUNCH_CHECK("chains refresh set kernel");
    ctx->q_stale = false;
    return LRS_OK;
}
