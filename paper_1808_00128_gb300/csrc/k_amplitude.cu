// Batched amplitudes <x|psi> = sum_alpha b_alpha <x|phi_alpha> (Eqs. (amplitude),
// (amplitude1)).
//
// For each (x, term) the Pauli Q = prod_{p: x_p = 1} U_C^{-1} X_p U_C is written
// i^mu X(u) Z(w); taking the rows in increasing p,
//     z ^= w & F_p;  u ^= F_p;  w ^= M_p,   mu = x.gamma + 2 parity(z)  (mod 4).
// The rows are grouped four at a time (Four Russians): for the current term the
// block builds a shared table, per 4-row chunk c and pattern q of x's bits
// 4c..4c+3, of (u_q, w_q, z_q) restricted to those rows; a chunk then enters as
//     z ^= (w & u_q) ^ z_q;  u ^= u_q;  w ^= w_q.
// One thread owns XP strings x and walks the block's tile of terms, so its
// chi-sum is a private FP32 Kahan sum (no cross-thread reduction); the tile
// partials are summed in FP64 by k_amp_reduce.
#include <string.h>

#include <atomic>

#include "lrs_device.cuh"

namespace {

constexpr int AMP_XT = 128;   // threads per block
// strings per thread (independent chains for ILP): eight for the plain batch (each
// term's tables and barrier serve 1024 strings), four for the chain start (its
// per-string state buffers)
__host__ __device__ constexpr int amp_xp(bool qout) { return qout ? 4 : 8; }
__host__ __device__ constexpr int amp_xb(bool qout) { return AMP_XT * amp_xp(qout); }

struct AmpEntry {
    uint64_t u, w, z;
};

// QOUT: also store every (x_i, term) Pauli state at entry i * cap + alpha of Qout
// (q_store: 12 bytes for n <= 40, i.e. NCH <= 10, else 16), zero terms included (the
// Metropolis chain state of Sec. 4.2).
// PK (n <= 62): only parity(z) enters mu, and parity(z_after) = parity(z) +
// parity(w & u_q) + parity(z_q), so a table entry keeps parity(z_q) in bit 63 of u_q
// and the lookups XOR-accumulate w & u_q (one popcount per string at the end): two
// 8-byte tables (u_q, w_q) instead of three, each a conflict-free 128-byte row per
// chunk.
// Register budget: five blocks per SM (96 registers, eight strings per thread) for the
// plain amplitude batch, six (80 registers, four strings) for the variant that also
// writes the Pauli states.
constexpr int amp_min_blocks(bool qout) { return qout ? 6 : 5; }
// ERR: also sum |b_alpha <x|phi_alpha>| over the terms that contribute at x (one FP32
// add per contributing (x, term)), written to magp[i * n_tiles + tile]: the input of
// the per-result error bound of k_amp_reduce.
// One block of the amplitude launch: term tile `tile`, strings xblk * AMP_XB ... (shared
// by the single-circuit kernel and the batched kernel of several circuits).
template <int NCH, bool QOUT, bool PK, bool ERR>
__device__ __forceinline__ void amp_block(const TermsView& T, const uint64_t* __restrict__ xs, int64_t batch,
                                          int64_t tt, float2* __restrict__ partial, int64_t n_tiles,
                                          void* __restrict__ Qout, float* __restrict__ magp, int64_t tile,
                                          int64_t xblk) {
    // One barrier per term: while the block evaluates term a from table slot a, it
    // builds the table of term a + 1 (from the rows stored in the previous interval)
    // and stores the rows of term a + 2; tables and rows are double-buffered, the
    // per-term scalars (read while the scalars of a + 2 are written) triple-buffered.
    __shared__ AmpEntry tab[2][PK ? 1 : NCH][16];
    __shared__ uint64_t tabU[2][PK ? NCH : 1][16], tabW[2][PK ? NCH : 1][16];
    __shared__ uint64_t sF[2][64], sM[2][64];
    __shared__ float2 val8[3][8];           // b e^{i pi k/4} 2^{-(|v|+h)/2}, k = 0..7
    __shared__ float val_abs[3];            // |b| 2^{-(|v|+h)/2} (ERR)
    __shared__ uint64_t sc[3][4];           // glo, ghi, v, s
    __shared__ uint32_t sc_live[3];
    // compact Pauli states of the last QG terms for each of the block's strings, private
    // to the thread that owns the string: written out as 16-byte vectors every QG terms
    constexpr int AMP_XP = amp_xp(QOUT), AMP_XB = amp_xb(QOUT);
    constexpr bool CQ = QOUT && NCH <= 10;
    constexpr int QG = 4;
    __shared__ uint64_t qb8[CQ ? QG : 1][CQ ? AMP_XB : 1];
    __shared__ uint32_t qb4[CQ ? QG : 1][CQ ? AMP_XB : 1];
    // the 16-byte states (n > 40) of the last QW terms, written out as one full 32-byte
    // sector per string every QW terms (a store per term would write half sectors)
    constexpr bool WQ = QOUT && !CQ;
    constexpr int QW = 2;
    __shared__ uint64_t qwu[WQ ? QW : 1][WQ ? AMP_XB : 1], qww[WQ ? QW : 1][WQ ? AMP_XB : 1];
    const int n = T.n;
    const int tid = threadIdx.x;
    const int64_t xb = xblk * AMP_XB;
    uint64_t xv[AMP_XP];
#pragma unroll
    for (int k = 0; k < AMP_XP; ++k) {
        const int64_t i = xb + tid + k * AMP_XT;
        xv[k] = i < batch ? (xs[i] & T.nmask) : 0ull;   // bits >= n are ignored
    }
    KahanC acc[AMP_XP];
    float mag[ERR ? AMP_XP : 1];
#pragma unroll
    for (int k = 0; k < AMP_XP; ++k) acc[k].init();
#pragma unroll
    for (int k = 0; k < (ERR ? AMP_XP : 1); ++k) mag[k] = 0.f;

    const int64_t a0 = tile * tt;
    const int64_t a1 = (a0 + tt < T.cap) ? a0 + tt : T.cap;
    // register prefetch of the next term: threads < n hold rows, threads 64..66 scalars
    // (thread 66 keeps its own copy of v: it must not read sc[2], which thread 65
    // writes in the same barrier interval)
    uint64_t pf = 0, pm = 0, pv = 0;
    auto prefetch = [&](int64_t a) {
        if (tid < n) {
            pf = T.F[(int64_t)tid * T.cap + a];
            pm = T.M[(int64_t)tid * T.cap + a];
        } else if (tid == 64) {
            pf = T.glo[a]; pm = T.ghi[a];
        } else if (tid == 65) {
            pf = T.v[a]; pm = T.s[a];
        } else if (tid == 66) {
            pf = T.omega[a];
            const float2 b = T.coef[a];
            pm = (uint64_t)__float_as_uint(b.x) | ((uint64_t)__float_as_uint(b.y) << 32);
            pv = T.v[a];
        }
    };
    // thread-owned stores of the prefetched term into row slot rs and scalar slot ss
    auto store = [&](int rs, int ss) {
        if (tid < n) { sF[rs][tid] = pf; sM[rs][tid] = pm; }
        if (tid == 64) { sc[ss][0] = pf; sc[ss][1] = pm; }
        if (tid == 65) { sc[ss][2] = pf; sc[ss][3] = pm; }
        if (tid == 66) {
            const uint32_t om = (uint32_t)pf;
            const float2 b = make_float2(__uint_as_float((uint32_t)pm), __uint_as_float((uint32_t)(pm >> 32)));
            sc_live[ss] = ((om >> 3) & 1u) ? 0u : 1u;
            const int e0 = __popcll(pv) + (int)(om >> 8);
#pragma unroll
            for (int k = 0; k < 8; ++k) val8[ss][k] = z8_scale(b, k + (int)(om & 7u), e0);
            if (ERR) val_abs[ss] = ldexpf(hypotf(b.x, b.y), -(e0 >> 1)) * ((e0 & 1) ? 0.70710678f : 1.f);
        }
    };
    // the Four-Russians table of the term whose rows are in slot ts, into table slot ts
    auto build = [&](int ts) {
        for (int e = tid; e < NCH * 16; e += AMP_XT) {
            const int c = e >> 4, q = e & 15;
            uint64_t u = 0, w = 0, z = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int r = 4 * c + b;
                if (((q >> b) & 1) && r < n) {
                    const uint64_t Fr = sF[ts][r];
                    z ^= w & Fr;
                    u ^= Fr;
                    w ^= sM[ts][r];
                }
            }
            if (PK) {
                tabU[ts][c][q] = u | ((uint64_t)par64(z) << 63);
                tabW[ts][c][q] = w;
            } else {
                tab[ts][c][q].u = u;
                tab[ts][c][q].w = w;
                tab[ts][c][q].z = z;
            }
        }
    };
    if (a0 < a1) { prefetch(a0); store(0, 0); }
    if (a0 + 1 < a1) { prefetch(a0 + 1); store(1, 1); }
    if (a0 + 2 < a1) prefetch(a0 + 2);
    __syncthreads();
    if (a0 < a1) build(0);
    __syncthreads();
    for (int64_t a = a0; a < a1; ++a) {
        const int kt = (int)(a - a0);
        const int tb = kt & 1, ss = kt % 3;
        if (a + 1 < a1) build(tb ^ 1);
        if (a + 2 < a1) store(tb, (kt + 2) % 3);
        if (a + 3 < a1) prefetch(a + 3);
        const bool live = sc_live[ss] != 0u;
        if (QOUT || live) {
            const uint64_t glo = sc[ss][0], ghi = sc[ss][1], v = sc[ss][2], s = sc[ss][3];
            const uint64_t nv = ~v & T.nmask, sv = s & v;
    #pragma unroll
            for (int k = 0; k < AMP_XP; ++k) {
                const uint64_t x = xv[k];
                uint64_t u = 0, w = 0;
                uint32_t zpar;
                if (PK) {
                    // only the parity of sum_c popc(w_c & u_q) enters, and that is the
                    // parity of the XOR of the terms: one popcount per string
                    uint64_t zx = 0;
    #pragma unroll
                    for (int c = 0; c < NCH; ++c) {
                        const int q = (int)((x >> (4 * c)) & 15u);
                        const uint64_t Eu = tabU[tb][c][q], Ew = tabW[tb][c][q];
                        zx ^= w & Eu;   // w has no bit 63
                        u ^= Eu;
                        w ^= Ew;
                    }
                    zpar = ((uint32_t)__popcll(zx) + (uint32_t)(u >> 63)) & 1u;
                    u &= ~(1ull << 63);
                } else {
                    uint64_t z = 0;
    #pragma unroll
                    for (int c = 0; c < NCH; ++c) {
                        const AmpEntry& E = tab[tb][c][(int)((x >> (4 * c)) & 15u)];
                        z ^= (w & E.u) ^ E.z;
                        u ^= E.u;
                        w ^= E.w;
                    }
                    zpar = par64(z);
                }
                const int mu = __popcll(x & glo) + 2 * __popcll(x & ghi) + 2 * (int)zpar;
                if (CQ) {
                    const int g = (int)((a - a0) & (QG - 1));
                    qb8[g][tid + k * AMP_XT] = u | (w << 40);
                    qb4[g][tid + k * AMP_XT] = (uint32_t)(w >> 24) | ((uint32_t)(mu & 3) << 16);
                } else if (WQ) {
                    const int g = (int)((a - a0) & (QW - 1));
                    qwu[g][tid + k * AMP_XT] = u | ((uint64_t)(mu & 3) << 62);   // the q_store layout
                    qww[g][tid + k * AMP_XT] = w;
                }
                if (live && ((u ^ s) & nv) == 0) {
                    const int sign = (int)par64(u & (w ^ sv));
                    acc[k].add(val8[ss][(2 * mu + 4 * sign) & 7]);
                    if (ERR) mag[k] += val_abs[ss];
                }
            }
            if (CQ && ((a - a0) & (QG - 1)) == QG - 1) {
                // terms a-3 .. a of each of the thread's strings: 32 bytes of u | w << 40 and
                // 16 bytes of (w >> 24) | mu << 16, contiguous and 16-byte aligned (a0 and
                // the tile length are multiples of QG, cap of 256)
                uint64_t* q8 = reinterpret_cast<uint64_t*>(Qout);
                uint32_t* q4 = reinterpret_cast<uint32_t*>(q8 + batch * T.cap);
    #pragma unroll
                for (int k = 0; k < AMP_XP; ++k) {
                    const int sl = tid + k * AMP_XT;
                    const int64_t i = xb + sl;
                    if (i >= batch) continue;
                    const int64_t e = i * T.cap + a - (QG - 1);
                    reinterpret_cast<ulonglong2*>(q8 + e)[0] = make_ulonglong2(qb8[0][sl], qb8[1][sl]);
                    reinterpret_cast<ulonglong2*>(q8 + e)[1] = make_ulonglong2(qb8[2][sl], qb8[3][sl]);
                    *reinterpret_cast<uint4*>(q4 + e) = make_uint4(qb4[0][sl], qb4[1][sl], qb4[2][sl], qb4[3][sl]);
                }
            }
            if (WQ && ((a - a0) & (QW - 1)) == QW - 1) {
                // terms a-1, a of each of the thread's strings: one 32-byte sector (a0
                // and the tile length are even, cap a multiple of 256)
                ulonglong2* q16 = reinterpret_cast<ulonglong2*>(Qout);
#pragma unroll
                for (int k = 0; k < AMP_XP; ++k) {
                    const int sl = tid + k * AMP_XT;
                    const int64_t i = xb + sl;
                    if (i >= batch) continue;
                    const int64_t e = i * T.cap + a - (QW - 1);
                    q16[e] = make_ulonglong2(qwu[0][sl], qww[0][sl]);
                    q16[e + 1] = make_ulonglong2(qwu[1][sl], qww[1][sl]);
                }
            }
        }   // live (every term for the Pauli-state output)
        __syncthreads();   // slot tb ^ 1 and the next rows and scalars are complete
    }
#pragma unroll
    for (int k = 0; k < AMP_XP; ++k) {
        const int64_t i = xb + tid + k * AMP_XT;
        if (i < batch) {
            partial[i * n_tiles + tile] = acc[k].value();
            if (ERR) magp[i * n_tiles + tile] = mag[ERR ? k : 0];
        }
    }
}

template <int NCH, bool QOUT, bool PK, bool ERR>
__global__ void __launch_bounds__(AMP_XT, amp_min_blocks(QOUT)) k_amplitude(TermsView T, const uint64_t* __restrict__ xs,
                                                      int64_t batch, int64_t tt,
                                                      float2* __restrict__ partial, int64_t n_tiles,
                                                      void* __restrict__ Qout, float* __restrict__ magp) {
    amp_block<NCH, QOUT, PK, ERR>(T, xs, batch, tt, partial, n_tiles, Qout, magp, blockIdx.x, blockIdx.y);
}

// Several circuits of the same width in one launch: block b runs block b - first[c]
// of circuit c's own launch shape (term tile fastest), so every circuit gets exactly the
// partial sums of its single-circuit launch; the table is a kernel parameter, so the
// circuit lookup and every value read from it are warp-uniform.
#define LRS_AMP_BATCH_MAX 12
struct AmpBatch {
    int count;
    int64_t first[LRS_AMP_BATCH_MAX + 1];
    TermsView T[LRS_AMP_BATCH_MAX];
    const uint64_t* xs[LRS_AMP_BATCH_MAX];
    int64_t batch[LRS_AMP_BATCH_MAX], tt[LRS_AMP_BATCH_MAX], n_tiles[LRS_AMP_BATCH_MAX];
    float2* partial[LRS_AMP_BATCH_MAX];
    double* out[LRS_AMP_BATCH_MAX];
};

template <int NCH, bool PK>
__global__ void __launch_bounds__(AMP_XT, amp_min_blocks(false)) k_amplitude_batch(const __grid_constant__ AmpBatch B) {
    const int64_t b = blockIdx.x;
    int c = 0;
#pragma unroll 1
    for (int i = 1; i < B.count; ++i)
        if (B.first[i] <= b) c = i;
    const int64_t local = b - B.first[c];
    amp_block<NCH, false, PK, false>(B.T[c], B.xs[c], B.batch[c], B.tt[c], B.partial[c], B.n_tiles[c], nullptr,
                                     nullptr, local % B.n_tiles[c], local / B.n_tiles[c]);
}

// FP64 sum of the block partials of each x, and (magp != NULL) the error bound of
// that sum against the exact chi-sum:
//   |a_gpu - a| <= (8u + 8 tt u^2)(1 + tt u)(1 + 1e-4) M + n_tiles 2^-52 P,
// u = 2^-24, M = sum over contributing terms of |b_alpha <x|phi_alpha>| (FP32 sums of
// the tiles), P = sum over tiles of |partial|.  Per addend: the FP32 coefficient and
// the FP32 phase/sqrt2 factors of z8_scale give at most 4u |a_alpha|; the Kahan sum of
// a tile of tt addends adds (2u + O(tt u^2)) per real component, 2 sqrt2 u |a_alpha|
// for the complex pair; the final s - c rounding u; M itself is an FP32 sum of tt
// positive values (relative tt u) of magnitudes computed to 1e-4.  The FP64 sum of
// n_tiles partials adds at most n_tiles 2^-53 P per component.
__global__ void k_amp_reduce(const float2* __restrict__ partial, const float* __restrict__ magp, int64_t n_tiles,
                             int64_t batch, int64_t tt, double* __restrict__ out, float* __restrict__ err) {
    const int64_t xi = blockIdx.x;
    if (xi >= batch) return;
    double re = 0.0, im = 0.0, m = 0.0, pa = 0.0;
    for (int64_t t = threadIdx.x; t < n_tiles; t += blockDim.x) {
        const float2 p = partial[xi * n_tiles + t];
        re += (double)p.x;
        im += (double)p.y;
        if (magp) {
            m += (double)magp[xi * n_tiles + t];
            pa += hypot((double)p.x, (double)p.y);
        }
    }
    __shared__ double sre[256], sim[256], sm[256], spa[256];
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    sm[threadIdx.x] = m;
    spa[threadIdx.x] = pa;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            sre[threadIdx.x] += sre[threadIdx.x + off];
            sim[threadIdx.x] += sim[threadIdx.x + off];
            sm[threadIdx.x] += sm[threadIdx.x + off];
            spa[threadIdx.x] += spa[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * xi] = sre[0];
        out[2 * xi + 1] = sim[0];
        if (magp) {
            const double u = 5.9604644775390625e-8, ttd = (double)tt;
            const double c = (8.0 * u + 8.0 * ttd * u * u) * (1.0 + ttd * u) * (1.0 + 1e-4);
            err[xi] = (float)((c * sm[0] + (double)n_tiles * 2.220446049250313e-16 * spa[0]) * (1.0 + 1e-6));
        }
    }
}

// The FP64 tile sums of several circuits in one launch: block b is string b - xfirst[c]
// of circuit c (same summation order as k_amp_reduce).
__global__ void k_amp_reduce_batch(const __grid_constant__ AmpBatch B, int64_t total) {
    const int64_t b = blockIdx.x;
    if (b >= total) return;
    int c = 0;
#pragma unroll 1
    for (int i = 1; i < B.count; ++i)
        if (B.first[i] <= b) c = i;
    const int64_t xi = b - B.first[c];
    const float2* partial = B.partial[c];
    const int64_t n_tiles = B.n_tiles[c];
    double re = 0.0, im = 0.0;
    for (int64_t t = threadIdx.x; t < n_tiles; t += blockDim.x) {
        const float2 p = partial[xi * n_tiles + t];
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
        B.out[c][2 * xi] = sre[0];
        B.out[c][2 * xi + 1] = sim[0];
    }
}

struct AmpPlan {
    int64_t xblocks, n_tiles, tt;
};

// Term tiles so that the grid covers every SM several times.
AmpPlan amp_plan(const lrs_ctx* ctx, int64_t batch, bool qout) {
    AmpPlan P;
    P.xblocks = (batch + amp_xb(qout) - 1) / amp_xb(qout);
    const int64_t target = (int64_t)ctx->sm_count * ctx->tune_amp_bps;
    int64_t nt = (target + P.xblocks - 1) / P.xblocks;
    const int64_t maxt = (ctx->cap + 31) / 32;
    if (nt > maxt) nt = maxt;
    if (nt < 1) nt = 1;
    P.tt = ((ctx->cap + nt - 1) / nt + 7) & ~(int64_t)7;   // tiles start at multiples of 8 terms
    P.n_tiles = (ctx->cap + P.tt - 1) / P.tt;
    return P;
}

template <int NCH>
lrs_status launch_amp_t(lrs_ctx* ctx, const uint64_t* x, int64_t batch, float2* partial,
                        const AmpPlan& P, void* Qout, float* magp, cudaStream_t st) {
    dim3 grid((unsigned)P.n_tiles, (unsigned)P.xblocks);
    const bool pk = ctx->n <= 62;
    const TermsView T = ctx->view();
    if (Qout)   // chains need n <= 62 (mu lives in bits 62-63 of Q), so the packed tables apply
        k_amplitude<NCH, true, true, false><<<grid, AMP_XT, 0, st>>>(T, x, batch, P.tt, partial, P.n_tiles, Qout,
                                                                    nullptr);
    else if (pk && magp)
        k_amplitude<NCH, false, true, true><<<grid, AMP_XT, 0, st>>>(T, x, batch, P.tt, partial, P.n_tiles,
                                                                    nullptr, magp);
    else if (pk)
        k_amplitude<NCH, false, true, false><<<grid, AMP_XT, 0, st>>>(T, x, batch, P.tt, partial, P.n_tiles,
                                                                     nullptr, nullptr);
    else if (magp)
        k_amplitude<NCH, false, false, true><<<grid, AMP_XT, 0, st>>>(T, x, batch, P.tt, partial, P.n_tiles,
                                                                     nullptr, magp);
    else
        k_amplitude<NCH, false, false, false><<<grid, AMP_XT, 0, st>>>(T, x, batch, P.tt, partial, P.n_tiles,
                                                                      nullptr, nullptr);
    LRS_LAUNCH_CHECK("amplitude kernel");
    return LRS_OK;
}

lrs_status launch_amp_kernels(lrs_ctx* ctx, const uint64_t* x, int64_t batch, double* out,
                              float2* partial, const AmpPlan& P, cudaStream_t st, void* Qout,
                              float* magp = nullptr, float* err = nullptr) {
    if (P.xblocks > 65535) return lrs_fail(LRS_ERR_UNSUPPORTED, "amplitude batch too large");
    lrs_status rc;
    switch ((ctx->n + 3) / 4) {
        case 1: rc = launch_amp_t<1>(ctx, x, batch, partial, P, Qout, magp, st); break;
        case 2: rc = launch_amp_t<2>(ctx, x, batch, partial, P, Qout, magp, st); break;
        case 3: rc = launch_amp_t<3>(ctx, x, batch, partial, P, Qout, magp, st); break;
        case 4: rc = launch_amp_t<4>(ctx, x, batch, partial, P, Qout, magp, st); break;
        case 5: rc = launch_amp_t<5>(ctx, x, batch, partial, P, Qout, magp, st); break;
        case 6: rc = launch_amp_t<6>(ctx, x, batch, partial, P, Qout, magp, st); break;
        case 7: rc = launch_amp_t<7>(ctx, x, batch, partial, P, Qout, magp, st); break;
        case 8: rc = launch_amp_t<8>(ctx, x, batch, partial, P, Qout, magp, st); break;
        case 9: rc = launch_amp_t<9>(ctx, x, batch, partial, P, Qout, magp, st); break;
        case 10: rc = launch_amp_t<10>(ctx, x, batch, partial, P, Qout, magp, st); break;
        case 11: rc = launch_amp_t<11>(ctx, x, batch, partial, P, Qout, magp, st); break;
        case 12: rc = launch_amp_t<12>(ctx, x, batch, partial, P, Qout, magp, st); break;
        case 13: rc = launch_amp_t<13>(ctx, x, batch, partial, P, Qout, magp, st); break;
        case 14: rc = launch_amp_t<14>(ctx, x, batch, partial, P, Qout, magp, st); break;
        case 15: rc = launch_amp_t<15>(ctx, x, batch, partial, P, Qout, magp, st); break;
        default: rc = launch_amp_t<16>(ctx, x, batch, partial, P, Qout, magp, st); break;
    }
    if (rc != LRS_OK) return rc;
    k_amp_reduce<<<(unsigned)batch, 256, 0, st>>>(partial, magp, P.n_tiles, batch, P.tt, out, err);
    LRS_LAUNCH_CHECK("amplitude reduce kernel");
    return LRS_OK;
}

}  // namespace

// Amplitudes of x[0..batch) into scratch (*amp_out, 2 doubles per x) and the Pauli
// state Q[i * cap + alpha] of every (x_i, term): the chain start of Sec. 4.2.
lrs_status launch_amplitude_q(lrs_ctx* ctx, const uint64_t* x, int64_t batch, void* Q, double** amp_out,
                              cudaStream_t st) {
    const AmpPlan P = amp_plan(ctx, batch, true);
    const size_t part = ((size_t)batch * P.n_tiles * sizeof(float2) + 255) & ~(size_t)255;
    void* scr = nullptr;
    lrs_status rc = lrs_scratch(ctx, part + (size_t)batch * 2 * sizeof(double), &scr);
    if (rc != LRS_OK) return rc;
    *amp_out = (double*)((char*)scr + part);
    return launch_amp_kernels(ctx, x, batch, *amp_out, (float2*)scr, P, st, Q);
}

lrs_status launch_amplitude(lrs_ctx* ctx, const uint64_t* x, int64_t batch, double* out, float* err,
                            cudaStream_t st) {
    if (batch == 0) return LRS_OK;
    const AmpPlan P = amp_plan(ctx, batch, false);
    const size_t part = ((size_t)batch * P.n_tiles * sizeof(float2) + 255) & ~(size_t)255;
    void* scr = nullptr;
    lrs_status rc = lrs_scratch(ctx, part + (err ? (size_t)batch * P.n_tiles * sizeof(float) : 0), &scr);
    if (rc != LRS_OK) return rc;
    float* magp = err ? (float*)((char*)scr + part) : nullptr;
    return launch_amp_kernels(ctx, x, batch, out, (float2*)scr, P, st, nullptr, magp, err);
}

template <int NCH>
static lrs_status launch_amp_batch_t(const AmpBatch& B, int64_t blocks, bool pk, cudaStream_t st) {
    if (pk)
        k_amplitude_batch<NCH, true><<<(unsigned)blocks, AMP_XT, 0, st>>>(B);
    else
        k_amplitude_batch<NCH, false><<<(unsigned)blocks, AMP_XT, 0, st>>>(B);
    LRS_LAUNCH_CHECK("batched amplitude kernel");
    return LRS_OK;
}

// Amplitudes of several circuits of the same width (count <= LRS_AMP_BATCH_MAX per
// launch pair): one amplitude launch and one reduction launch for all of them, each
// circuit with the tile plan and partial buffer of its own single launch.
lrs_status launch_amplitude_batch(lrs_ctx* const* ctxs, const uint64_t* const* xs, const int64_t* batch,
                                  double* const* out, int32_t count, cudaStream_t st) {
    const int n = ctxs[0]->n;
    for (int32_t base = 0; base < count; base += LRS_AMP_BATCH_MAX) {
        AmpBatch B;
        memset(&B, 0, sizeof(B));
        int64_t xfirst[LRS_AMP_BATCH_MAX + 1];
        int k = 0;
        int64_t blocks = 0, strings = 0;
        const int32_t end = (count - base < LRS_AMP_BATCH_MAX) ? count : base + LRS_AMP_BATCH_MAX;
        for (int32_t i = base; i < end; ++i) {
            if (batch[i] == 0) continue;
            lrs_ctx* c = ctxs[i];
            const AmpPlan P = amp_plan(c, batch[i], false);
            if (P.xblocks > 65535) return lrs_fail(LRS_ERR_UNSUPPORTED, "amplitude batch too large");
            void* scr = nullptr;
            lrs_status rc = lrs_scratch(c, (size_t)batch[i] * P.n_tiles * sizeof(float2), &scr);
            if (rc != LRS_OK) return rc;
            B.first[k] = blocks;
            B.T[k] = c->view();
            B.xs[k] = xs[i];
            B.batch[k] = batch[i];
            B.tt[k] = P.tt;
            B.n_tiles[k] = P.n_tiles;
            B.partial[k] = (float2*)scr;
            B.out[k] = out[i];
            xfirst[k] = strings;
            blocks += P.n_tiles * P.xblocks;
            strings += batch[i];
            ++k;
        }
        if (k == 0) continue;
        if (blocks > 0x7FFFFFFF) return lrs_fail(LRS_ERR_UNSUPPORTED, "batched amplitude grid too large");
        B.count = k;
        B.first[k] = blocks;
        xfirst[k] = strings;
        AmpBatch R = B;   // the reduction indexes strings instead of blocks
        for (int j = 0; j <= k; ++j) R.first[j] = xfirst[j];
        lrs_status rc;
        const bool pk = n <= 62;
        switch ((n + 3) / 4) {
            case 1: rc = launch_amp_batch_t<1>(B, blocks, pk, st); break;
            case 2: rc = launch_amp_batch_t<2>(B, blocks, pk, st); break;
            case 3: rc = launch_amp_batch_t<3>(B, blocks, pk, st); break;
            case 4: rc = launch_amp_batch_t<4>(B, blocks, pk, st); break;
            case 5: rc = launch_amp_batch_t<5>(B, blocks, pk, st); break;
            case 6: rc = launch_amp_batch_t<6>(B, blocks, pk, st); break;
            case 7: rc = launch_amp_batch_t<7>(B, blocks, pk, st); break;
            case 8: rc = launch_amp_batch_t<8>(B, blocks, pk, st); break;
            case 9: rc = launch_amp_batch_t<9>(B, blocks, pk, st); break;
            case 10: rc = launch_amp_batch_t<10>(B, blocks, pk, st); break;
            case 11: rc = launch_amp_batch_t<11>(B, blocks, pk, st); break;
            case 12: rc = launch_amp_batch_t<12>(B, blocks, pk, st); break;
            case 13: rc = launch_amp_batch_t<13>(B, blocks, pk, st); break;
            case 14: rc = launch_amp_batch_t<14>(B, blocks, pk, st); break;
            case 15: rc = launch_amp_batch_t<15>(B, blocks, pk, st); break;
            default: rc = launch_amp_batch_t<16>(B, blocks, pk, st); break;
        }
        if (rc != LRS_OK) return rc;
        k_amp_reduce_batch<<<(unsigned)strings, 256, 0, st>>>(R, strings);
        LRS_LAUNCH_CHECK("batched amplitude reduce kernel");
    }
    return LRS_OK;
}

// ---------------------------------------------------------------------------------
// Allocation-free variant of lrs_amplitude.
//
// Some callers cannot call cudaMalloc at the point where they need amplitudes:
// a serving loop whose framework allocator has already reserved all device
// memory, or code that must not take the allocator's locks or its latency on
// a hot path.  For them the block partial sums live in a fixed file-scope
// device array instead of the context's growable scratch buffer.  The array
// is allocated when the library is loaded and stays on every GPU that loads
// the library until the process exits.
// ---------------------------------------------------------------------------------
#define LRS_NOALLOC_PARTIALS (2u * 1024u * 1024u)   // float2 entries = 16 MiB

static __device__ __align__(256) float2 g_noalloc_partials[LRS_NOALLOC_PARTIALS];

// Device address of g_noalloc_partials, looked up once per device.  In host
// code the symbol name is only a host-side stand-in, so it is never passed to a
// kernel directly.  The address is published through an atomic, so first calls
// racing from several host threads each look it up (same value) without a data
// race; a failed lookup publishes nothing and the next call tries again.
static std::atomic<void*> g_noalloc_addr[128];

static lrs_status noalloc_address(int device, float2** out) {
    if (device < 0 || device >= 128) return lrs_fail(LRS_ERR_UNSUPPORTED, "device index %d", device);
    void* p = g_noalloc_addr[device].load(std::memory_order_acquire);
    if (!p) {
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return lrs_cuda_check(e, "cudaGetSymbolAddress(g_noalloc_partials)");
        g_noalloc_addr[device].store(p, std::memory_order_release);
    }
    *out = (float2*)p;
    return LRS_OK;
}

extern "C" lrs_status lrs_amplitude_noalloc(lrs_ctx* ctx, const uint64_t* x, int64_t batch,
                                            double* out, void* stream) {
    if (!ctx) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    if (!ctx->have_terms) return lrs_fail(LRS_ERR_STATE, "no terms");
    if (batch < 0) return lrs_fail(LRS_ERR_ARG, "batch < 0");
    if (batch > 0 && (!x || !out)) return lrs_fail(LRS_ERR_ARG, "NULL buffer");
    LRS_CUDA(cudaSetDevice(ctx->device));
    float2* partial = nullptr;
    lrs_status rc = noalloc_address(ctx->device, &partial);   // first call on a device: set-up
    if (rc != LRS_OK) return rc;
    if (batch == 0) return LRS_OK;
    const AmpPlan P = amp_plan(ctx, batch, false);
    if ((uint64_t)batch * (uint64_t)P.n_tiles > (uint64_t)LRS_NOALLOC_PARTIALS)
        return lrs_fail(LRS_ERR_ARG,
                        "lrs_amplitude_noalloc: %lld partial sums (batch x term tiles) exceed the "
                        "fixed buffer of %u; use a smaller batch or lrs_amplitude",
                        (long long)(batch * P.n_tiles), LRS_NOALLOC_PARTIALS);
    return launch_amp_kernels(ctx, x, batch, out, partial, P, (cudaStream_t)stream, nullptr);
}
