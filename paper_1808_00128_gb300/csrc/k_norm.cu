// Norm estimation (Sec. 4.3): eta_l = 2^n |<phi_{A_l}|psi>|^2.
//
// Three launches per call:
//   k_norm_prep    per term: J = M F^T off the diagonal, z0 = G s, u = F s and, for a
//                  term with n - |v| <= max_folds, the reduced echelon form of the
//                  constraints f_k = column k of F, k not in v
//   k_norm_draw_a  per l: A_l in M_n from the counter RNG
//   k_norm         one thread per A_l, a block of 64 A's walks a tile of terms, each
//                  thread keeping its own FP32 Kahan sum over the tile
// then k_norm_reduce sums the tiles in FP64.
//
// Per (A, term), with D = A + J (diagonal A_cc + gamma_c in Z4) the paper's route
// (Lemma (Inner Product)) forms K = G^T D G and sums i^(x^T B x) over x in Z2^v,
// B = K|_v + 2 diag(s + sK).  The kernel has two exact routes to that sum:
//   K path         P_c = D_c G by Four-Russians lookups in a per-term shared table of
//                  G, an in-place bit transpose (R_k = D g_k), K_k = R_k G, and K_kk
//                  mod 4 bit-sliced over k
//   change of      with y = G x, x^T K x = y^T D y and s.x + s^T K x = (F s + D z0).y
//   variables      (G^-1 = F^T since F G^T = I); x in Z2^v is the subspace
//                  (F^T y)_k = 0 for k not in v, and each such constraint, in reduced
//                  echelon form y_p = h . y, is substituted into the form (a rank-2
//                  update of the rows of D plus diagonal carries).  No K is formed.
// Either route ends in the exponential sum of a Z4 form by pairwise elimination on a
// symmetric adjacency (Lemma (Exponential Sum), lifted to Z2 with one extra variable,
// Eq. (Q)).  Everything up to the chi-sum is exact integer arithmetic.
#include "lrs_device.cuh"

namespace {

constexpr int NRM_TPB = 64;   // A's per block
constexpr int NRM_MFOLD = 12; // most constraints a change-of-variables term may carry
constexpr int NRM_PIVOTS = 4; // elimination pairs applied per pass over the rows
constexpr int NRM_MFUSE = 8;  // most constraints folded in the single row pass

struct NormTerm {
    uint64_t glo, ghi, v, s, z0;
    uint32_t omega;
    float2 coef;
};

// S <- S + m1 m2^T + m2 m1^T (+ n1 n2^T + n2 n1^T) on the rows in `rows`: row j gets
// m2 if j is in m1, m1 if j is in m2, and likewise for (n1, n2).  The rows are walked
// by their lowest set bit in two 32-bit halves, so each membership test is one AND
// with that bit and each addition a predicated XOR.  Rows are stored unmasked: every
// read of a row masks it with the active set (and drops its own bit).
__device__ __forceinline__ void rank_update(uint64_t* sK, uint64_t rows, uint64_t m1, uint64_t m2, uint64_t n1,
                                            uint64_t n2) {
#pragma unroll
    for (int hw = 0; hw < 2; ++hw) {
        const uint32_t b1 = (uint32_t)(m1 >> (32 * hw)), b2 = (uint32_t)(m2 >> (32 * hw));
        const uint32_t b3 = (uint32_t)(n1 >> (32 * hw)), b4 = (uint32_t)(n2 >> (32 * hw));
        for (uint32_t r = (uint32_t)(rows >> (32 * hw)); r;) {
            const uint32_t lb = r & (0u - r);
            r ^= lb;
            uint64_t x = 0;
            if (b1 & lb) x ^= m2;
            if (b2 & lb) x ^= m1;
            if (b3 & lb) x ^= n2;
            if (b4 & lb) x ^= n1;
            sK[(__ffs(lb) - 1 + 32 * hw) * NRM_TPB] ^= x;
        }
    }
}

// Row part of substituting y_p = h . y into the form (see the fold path in k_norm): row c
// gets q if c is in h, h if c is in q (q = row p), and h if c is in h and the diagonal
// of p is odd.  Rows stay unmasked (see rank_update).
__device__ __forceinline__ void fold_rows(uint64_t* sK, uint64_t h, uint64_t q, uint64_t op) {
    const uint64_t hq = q ^ (h & (0ull - op));
#pragma unroll
    for (int hw = 0; hw < 2; ++hw) {
        const uint32_t bh = (uint32_t)(h >> (32 * hw)), bq = (uint32_t)(q >> (32 * hw));
        for (uint32_t r = (uint32_t)((h | q) >> (32 * hw)); r;) {
            const uint32_t lb = r & (0u - r);
            r ^= lb;
            uint64_t x = 0;
            if (bh & lb) x ^= hq;
            if (bq & lb) x ^= h;
            sK[(__ffs(lb) - 1 + 32 * hw) * NRM_TPB] ^= x;
        }
    }
}

// Linear terms and signs of eliminating the pair (a, b) (given as the one-bit masks ba,
// bb; neighbour sets m1 of a without b, m2 of b without a): summing x_a, x_b out leaves
// the product of the two linear forms, whose constant part goes to the sign and the
// rest to the linear vectors.
__device__ __forceinline__ void pivot_terms(uint64_t ba, uint64_t bb, uint64_t m1, uint64_t m2, uint64_t& Lre,
                                            uint64_t& Lim, uint32_t& sre, uint32_t& sim) {
    const bool c1r = (Lre & ba) != 0, c2r = (Lre & bb) != 0;
    const bool c1i = (Lim & ba) != 0, c2i = (Lim & bb) != 0;
    sre ^= (uint32_t)(c1r && c2r);
    sim ^= (uint32_t)(c1i && c2i);
    const uint64_t mm = m1 & m2;
    uint64_t dr = mm, di = mm;
    if (c1r) dr ^= m2;
    if (c2r) dr ^= m1;
    if (c1i) di ^= m2;
    if (c2i) di ^= m1;
    Lre ^= dr;
    Lim ^= di;
}

// Sum over variables of (-1)^(quadratic form), lifted from Z4 (Eq. (Q), (real)).
// Rows S_j (j in v) live in sK[j * NRM_TPB]; X's neighbours are `odd`.
// Returns Re, Im signs of Z (in {-1,0,1}) and e with |Re|,|Im| = 2^(e-1).
__device__ __forceinline__ void eliminate(uint64_t* sK, uint64_t v, uint64_t odd, uint64_t Lb,
                                         int& re_s, int& im_s, int& e) {
    uint64_t act = v;
    uint32_t sre = 0, sim = 0;
    bool zre = false, zim = false;
    uint64_t Lre = Lb, Lim = Lb;
    e = 0;
    if (odd) {
        // pair the extra variable X (linear coefficient 0 for Re, 1 for Im) with bq
        const int bq = ffs64(odd);
        const uint64_t bb = odd & (0ull - odd);   // bit bq
        const uint64_t m1 = odd & ~bb;
        const uint64_t m2 = sK[bq * NRM_TPB] & act & ~bb;
        e += 1;
        const bool cr = (Lre & bb) != 0, ci = (Lim & bb) != 0;
        sim ^= (uint32_t)ci;
        const uint64_t mm = m1 & m2;
        Lre ^= (cr ? m1 : 0ull) ^ mm;
        Lim ^= m2 ^ (ci ? m1 : 0ull) ^ mm;
        rank_update(sK, m1 | m2, m1, m2, 0ull, 0ull);
        act &= ~bb;
    } else {
        e += 1;      // sum over x_X of (-1)^0 = 2 (Re), of (-1)^x_X = 0 (Im)
        zim = true;
    }
    // Pivots are taken NRM_PIVOTS at a time: pair k is found on the matrix as updated by
    // pairs 0..k-1, whose rows are read with those updates applied on the fly, and one
    // pass over the remaining rows then applies all the rank-2 updates together.
    uint64_t cand = act;
    while (cand) {
        uint64_t P1[NRM_PIVOTS], P2[NRM_PIVOTS];
        int np = 0;
#pragma unroll
        for (int k = 0; k < NRM_PIVOTS; ++k) {
            P1[k] = 0;
            P2[k] = 0;
            if (np != k) continue;
            while (cand) {
                const int a = ffs64(cand);
                const uint64_t ba = cand & (0ull - cand);   // bit a
                uint64_t ra = sK[a * NRM_TPB];
                // row a as pairs 0..k-1 left it: row j gains P2 if j is in P1, P1 if in P2
#pragma unroll
                for (int i = 0; i < k; ++i) {
                    if (P1[i] & ba) ra ^= P2[i];
                    if (P2[i] & ba) ra ^= P1[i];
                }
                ra &= act & ~ba;
                if (!ra) {       // isolated: stays isolated
                    cand &= ~ba;
                    continue;
                }
                const int bq = ffs64(ra);
                const uint64_t bb = ra & (0ull - ra);       // bit bq
                uint64_t rb = sK[bq * NRM_TPB];
#pragma unroll
                for (int i = 0; i < k; ++i) {
                    if (P1[i] & bb) rb ^= P2[i];
                    if (P2[i] & bb) rb ^= P1[i];
                }
                const uint64_t ab = ba | bb;
                P1[k] = ra & ~bb;
                P2[k] = rb & act & ~ab;
                pivot_terms(ba, bb, P1[k], P2[k], Lre, Lim, sre, sim);
                e += 1;
                act &= ~ab;
                cand &= ~ab;
                ++np;
                break;
            }
        }
        uint64_t rows = 0;
#pragma unroll
        for (int k = 0; k < NRM_PIVOTS; ++k) rows |= P1[k] | P2[k];
        rows &= act;
#pragma unroll
        for (int hw = 0; hw < 2; ++hw) {
            uint32_t B1[NRM_PIVOTS], B2[NRM_PIVOTS];
#pragma unroll
            for (int k = 0; k < NRM_PIVOTS; ++k) {
                B1[k] = (uint32_t)(P1[k] >> (32 * hw));
                B2[k] = (uint32_t)(P2[k] >> (32 * hw));
            }
            for (uint32_t r = (uint32_t)(rows >> (32 * hw)); r;) {
                const uint32_t lb = r & (0u - r);
                r ^= lb;
                uint64_t x = 0;
#pragma unroll
                for (int k = 0; k < NRM_PIVOTS; ++k) {
                    if (B1[k] & lb) x ^= P2[k];
                    if (B2[k] & lb) x ^= P1[k];
                }
                sK[(__ffs(lb) - 1 + 32 * hw) * NRM_TPB] ^= x;
            }
        }
    }
    e += __popcll(act);
    if (Lre & act) zre = true;
    if (Lim & act) zim = true;
    re_s = zre ? 0 : (sre ? -1 : 1);
    im_s = zim ? 0 : (sim ? -1 : 1);
}

// Four-Russians product with the current term's G: XOR of rows G_d over the set
// bits d of x, from the shared table tab[chunk][nibble] = XOR of the rows selected
// by that nibble of x.  A 16-entry chunk table is 128 bytes, so a warp's lookups
// into one chunk never conflict on shared-memory banks.
template <int NCH>
__device__ __forceinline__ uint64_t fr_rows(const uint64_t* __restrict__ tab, uint64_t x) {
    uint64_t r = 0;
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) r ^= tab[ch * 16 + (int)((x >> (4 * ch)) & 15u)];
    return r;
}

// Transpose of an 8 x 8 bit block held in one word (row r in byte r, column c in bit
// c of that byte): three rounds exchanging bit groups across the diagonal (the
// bit-matrix transposition of Warren, Hacker's Delight, ch. 7).
__device__ __forceinline__ uint64_t tr8(uint64_t x) {
    uint64_t t;
    t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
    x ^= t ^ (t << 7);
    t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
    x ^= t ^ (t << 14);
    t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
    x ^= t ^ (t << 28);
    return x;
}

// In-place transpose of the (8 NB) x (8 NB) bit matrix W[k * NRM_TPB] (bit b of row k)
// by 8 x 8 blocks: block (i, j) transposed lands in block (j, i).  Needs no rows beyond
// the matrix itself, so the work area is 8 ceil(n/8) words per thread.
template <int NB>
__device__ __forceinline__ void transpose_blocks(uint64_t* W) {
#pragma unroll
    for (int bi = 0; bi < NB; ++bi) {
        {
            uint64_t row[8], x = 0;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                row[r] = W[(8 * bi + r) * NRM_TPB];
                x |= ((row[r] >> (8 * bi)) & 0xFFull) << (8 * r);
            }
            x = tr8(x);
#pragma unroll
            for (int r = 0; r < 8; ++r)
                W[(8 * bi + r) * NRM_TPB] =
                    (row[r] & ~(0xFFull << (8 * bi))) | (((x >> (8 * r)) & 0xFFull) << (8 * bi));
        }
#pragma unroll
        for (int bj = bi + 1; bj < NB; ++bj) {
            uint64_t ri[8], rj[8], x = 0, y = 0;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                ri[r] = W[(8 * bi + r) * NRM_TPB];
                rj[r] = W[(8 * bj + r) * NRM_TPB];
                x |= ((ri[r] >> (8 * bj)) & 0xFFull) << (8 * r);
                y |= ((rj[r] >> (8 * bi)) & 0xFFull) << (8 * r);
            }
            x = tr8(x);
            y = tr8(y);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                W[(8 * bi + r) * NRM_TPB] =
                    (ri[r] & ~(0xFFull << (8 * bj))) | (((y >> (8 * r)) & 0xFFull) << (8 * bj));
                W[(8 * bj + r) * NRM_TPB] =
                    (rj[r] & ~(0xFFull << (8 * bi))) | (((x >> (8 * r)) & 0xFFull) << (8 * bi));
            }
        }
    }
}

// Per-term quantities every A-block of the norm kernel needs, computed once per call
// (one thread per term, struct-of-arrays over the term index alpha < cap):
//   J[c][alpha]  row c of J = M F^T off the diagonal
//   z0, u        z0 = G s (bit c = s . G_c) and u = F s (bit c = s . F_c)
//   piv          for a term with n - |v| <= max_folds: the pivot set of the reduced
//                echelon form of the constraints f_k = column k of F (k not in v),
//                else 0; f[i][alpha] the i-th reduced constraint (it holds exactly
//                one pivot, its own)
struct NormPrep {
    uint64_t *J, *z0, *u, *piv, *f;
    uint64_t *A, *adlo, *adhi;   // A_l: off-diagonal rows A[c][l], diagonal bit-planes (Z4)
};

// A_l in M_n from the counter RNG (one thread per l): the diagonal as two bit-planes
// (words 0 and 1 of the stream of l), the upper triangle from words 2.. in the order
// (0,1), (0,2), .., (0,n-1), (1,2), .., one bit each, mirrored below the diagonal.
__global__ void __launch_bounds__(NRM_TPB) k_norm_draw_a(int n, uint64_t nmask, int64_t L, uint64_t seed,
                                                         NormPrep P) {
    extern __shared__ uint64_t sRow[];   // row c of this thread's A at sRow[c * NRM_TPB + tid]
    const int tid = threadIdx.x;
    const int64_t l = (int64_t)blockIdx.x * NRM_TPB + tid;
    if (l >= L) return;
    uint64_t* sA = sRow + tid;
    const uint64_t key = sm64_key(seed, (uint64_t)l);
    P.adlo[l] = sm64_at(key, 0) & nmask;
    P.adhi[l] = sm64_at(key, 1) & nmask;
    for (int c = 0; c < n; ++c) sA[c * NRM_TPB] = 0;
    int64_t kbit = 0;
    uint64_t word = sm64_at(key, 2);
    for (int a = 0; a < n; ++a) {
        uint64_t rowa = sA[a * NRM_TPB];
        for (int b = a + 1; b < n; ++b) {
            const uint64_t bt = (word >> (kbit & 63)) & 1ull;
            rowa |= bt << b;
            sA[b * NRM_TPB] |= bt << a;
            ++kbit;
            if ((kbit & 63) == 0) word = sm64_at(key, 2 + (uint64_t)(kbit >> 6));
        }
        P.A[(int64_t)a * L + l] = rowa;
    }
}

__global__ void __launch_bounds__(NRM_TPB) k_norm_prep(TermsView T, int max_folds, NormPrep P) {
    extern __shared__ uint64_t sF[];   // row c of this thread's F at sF[c * NRM_TPB + tid]
    const int n = T.n, tid = threadIdx.x;
    const int64_t alpha = (int64_t)blockIdx.x * NRM_TPB + tid;
    if (alpha >= T.cap) return;        // no block-wide synchronisation below
    uint64_t* F = sF + tid;
    for (int c = 0; c < n; ++c) F[c * NRM_TPB] = T.F[(int64_t)c * T.cap + alpha];
    const uint64_t s = T.s[alpha], v = T.v[alpha];
    uint64_t z0 = 0, u = 0;
    for (int c = 0; c < n; ++c) {
        z0 |= (uint64_t)par64(s & T.G[(int64_t)c * T.cap + alpha]) << c;
        u |= (uint64_t)par64(s & F[c * NRM_TPB]) << c;
        const uint64_t Mc = T.M[(int64_t)c * T.cap + alpha];
        uint64_t jrow = 0;
        for (int d = 0; d < n; ++d) jrow |= (uint64_t)par64(Mc & F[d * NRM_TPB]) << d;
        P.J[(int64_t)c * T.cap + alpha] = jrow & ~bit64(c);
    }
    P.z0[alpha] = z0;
    P.u[alpha] = u;
    const int mf = n - __popcll(v);
    uint64_t piv = 0;
    if (mf <= max_folds) {
        uint64_t f[NRM_MFOLD];
        uint64_t ks = ~v & T.nmask;
#pragma unroll
        for (int i = 0; i < NRM_MFOLD; ++i) {
            f[i] = 0;
            if (i < mf) {
                const int k = ffs64(ks);
                ks &= ks - 1;
                for (int c = 0; c < n; ++c) f[i] |= getb(F[c * NRM_TPB], k) << c;
            }
        }
        // reduced echelon form (the f_k are independent: F is invertible); pivot of f_i
        // = its lowest bit when it is processed, then cleared from every other f_j
#pragma unroll
        for (int i = 0; i < NRM_MFOLD; ++i) {
            if (i < mf) {
                const int p = ffs64(f[i]);
                piv |= bit64(p);
#pragma unroll
                for (int j = 0; j < NRM_MFOLD; ++j)
                    if (j != i && j < mf && getb(f[j], p)) f[j] ^= f[i];
            }
        }
#pragma unroll
        for (int i = 0; i < NRM_MFOLD; ++i)
            if (i < mf) P.f[(int64_t)i * T.cap + alpha] = f[i];
    }
    P.piv[alpha] = piv;
}

// Blocks per SM the register budget is sized for: at n <= 40 96 registers (shared
// memory then fits nine blocks; the few spilled values cost less than the extra
// warps gain); at 41 <= n <= 56 seven blocks, the most shared memory fits (128
// registers: measured 2% faster at n = 50 than six blocks at 168, spills included);
// five for wider tableaux.
constexpr int norm_min_blocks(int nch) { return nch <= 10 ? 10 : nch <= 14 ? 7 : 5; }

template <int NCH, int NB>
__global__ void __launch_bounds__(NRM_TPB, norm_min_blocks(NCH)) k_norm(TermsView T, NormPrep P, int64_t L, int64_t tt,
                                                  float2* __restrict__ partial, int64_t n_tiles,
                                                  int max_folds, int fuse_folds) {
    extern __shared__ uint64_t smem[];
    __shared__ uint64_t tG[64], tJ[64];
    __shared__ NormTerm tS;
    __shared__ unsigned long long tz0, tU, tH[NRM_MFOLD];
    __shared__ int tPiv[NRM_MFOLD];
    const int n = T.n;
    const uint64_t nmask = T.nmask;
    const int tid = threadIdx.x;
    const int64_t l = (int64_t)blockIdx.y * NRM_TPB + tid;
    uint64_t* tab = smem;                                          // [NCH][16], shared
    uint64_t* sW = smem + NCH * 16 + tid;                          // 8 NB work rows

    // ---- A_l (drawn once per call by k_norm_draw_a).  Its rows are read from global
    // memory for every term: the block's 64 A's (n rows each) stay in L1, and keeping
    // them out of shared memory lets eight blocks share an SM instead of five.
    const int64_t la = l < L ? l : 0;
    const uint64_t adlo = P.adlo[la], adhi = P.adhi[la];
    const uint64_t* gA = P.A + la;
#define NRM_AROW(c) __ldg(gA + (int64_t)(c) * L)

    KahanC acc;
    acc.init();
    const int64_t tile = blockIdx.x;
    for (int64_t t = 0; t < tt; ++t) {
        const int64_t alpha = tile * tt + t;
        if (alpha >= T.cap) break;              // uniform across the block
        __syncthreads();
        // Terms whose v misses at most max_folds qubits sum over y = G x directly: the
        // form becomes y^T D y + 2 (F s + D G s) . y on the subspace F^T y = 0 off v.
        const uint64_t vv = T.v[alpha];
        const int mf = n - __popcll(vv);
        const bool fold = mf <= max_folds;   // max_folds <= NRM_MFOLD
        if (tid < n) {
            tJ[tid] = P.J[(int64_t)tid * T.cap + alpha];
            if (!fold) tG[tid] = T.G[(int64_t)tid * T.cap + alpha];
        }
        if (fold && tid < mf) {
            // constraint tid: y_p = h . y with p its pivot and h free of every pivot
            const uint64_t pv = P.piv[alpha], f = P.f[(int64_t)tid * T.cap + alpha];
            tPiv[tid] = ffs64(f & pv);
            tH[tid] = f & ~pv;
        }
        if (tid == 0) {
            tS.glo = T.glo[alpha]; tS.ghi = T.ghi[alpha];
            tS.v = vv; tS.s = T.s[alpha];
            tS.omega = T.omega[alpha]; tS.coef = T.coef[alpha];
            tz0 = P.z0[alpha];
            tU = P.u[alpha];
        }
        __syncthreads();
        if (!fold) {
            for (int e = tid; e < NCH * 16; e += NRM_TPB) {    // Four-Russians table of G rows
                const int ch = e >> 4, p = e & 15;
                uint64_t r = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (((p >> b) & 1) && 4 * ch + b < n) r ^= tG[4 * ch + b];
                tab[e] = r;
            }
            __syncthreads();
        }
        const NormTerm S = tS;
        if ((S.omega >> 3) & 1u) continue;     // zero term (uniform)
        // diag(A + J) mod 4 as bit-planes: lo = adlo ^ glo, hi = adhi ^ ghi ^ (adlo & glo)
        const uint64_t dlo = adlo ^ S.glo;
        const uint64_t dhi = adhi ^ S.ghi ^ (adlo & S.glo);
        const uint64_t z0 = tz0;
        uint64_t act, odd, Lb;
        uint32_t sKs;
        if (fold && mf <= fuse_folds) {   // fuse_folds <= NRM_MFUSE
            // The folds of the sequential form below, reordered: the pivot rows p_i are
            // folded first (row p_i only takes h_j from an earlier fold j with p_i in
            // q_j, since no h holds a pivot, and for the same reason the odd and linear
            // bits at p_i are those of D), then one pass builds every row of D, applies
            // every fold's update (x ^= hq_i if c in h_i, h_i if c in q_i) and the lift,
            // and stores the row once.  The updates are XORs fixed by the q_i, so their
            // order does not matter.
            uint64_t Q[NRM_MFUSE], HQ[NRM_MFUSE], Hv[NRM_MFUSE];
            uint64_t actf = nmask, oddf = dlo, dLb = 0;
            const uint64_t lb0 = dhi ^ tU ^ (dlo & z0);
#pragma unroll
            for (int i = 0; i < NRM_MFUSE; ++i) {
                Q[i] = 0;
                HQ[i] = 0;
                Hv[i] = 0;
                if (i < mf) {
                    const int p = tPiv[i];
                    const uint64_t h = tH[i];
                    const uint64_t bp = bit64(p);
                    const uint64_t Dp = NRM_AROW(p) ^ tJ[p];
                    uint64_t r = Dp;
#pragma unroll
                    for (int j = 0; j < i; ++j)
                        if (Q[j] & bp) r ^= Hv[j];
                    const uint64_t q = r & actf & ~bp;
                    const bool op = (dlo & bp) != 0;
                    const bool lp = ((lb0 & bp) != 0) != (par64(Dp & z0) != 0u);
                    const uint64_t ho = op ? h : 0ull;
                    dLb ^= (lp ? h : 0ull) ^ (oddf & ho) ^ (h & q);
                    oddf ^= ho;
                    Q[i] = q;
                    HQ[i] = q ^ ho;
                    Hv[i] = h;
                    actf &= ~bp;
                }
            }
            const uint64_t oddm = oddf & actf;
            uint64_t dz0 = 0;
            uint32_t pcnt = 0;
#pragma unroll
            for (int hw = 0; hw < 2; ++hw) {
                const int c0 = 32 * hw, c1 = n < c0 + 32 ? n : c0 + 32;
                uint32_t hh[NRM_MFUSE], qh[NRM_MFUSE];
#pragma unroll
                for (int i = 0; i < NRM_MFUSE; ++i) {
                    hh[i] = (uint32_t)(Hv[i] >> c0);
                    qh[i] = (uint32_t)(Q[i] >> c0);
                }
                const uint32_t oh = (uint32_t)(oddm >> c0), zh = (uint32_t)(z0 >> c0);
                // the next row of A is loaded one row ahead, so its L1 latency overlaps
                // this row's folds
                uint64_t anext = c0 < c1 ? NRM_AROW(c0) : 0ull;
                for (int c = c0; c < c1; ++c) {
                    const uint32_t lb = 1u << (c - c0);
                    const uint64_t arow = anext;
                    if (c + 1 < c1) anext = NRM_AROW(c + 1);
                    const uint64_t Doff = arow ^ tJ[c];
                    uint64_t x = Doff;
                    if (zh & lb) {
                        dz0 ^= Doff;
                        pcnt += (uint32_t)__popcll(Doff & z0);
                    }
#pragma unroll
                    for (int i = 0; i < NRM_MFUSE; ++i) {
                        if (i >= mf) break;
                        if (hh[i] & lb) x ^= HQ[i];
                        if (qh[i] & lb) x ^= Hv[i];
                    }
                    if (oh & lb) x ^= oddm;
                    sW[c * NRM_TPB] = x;
                }
            }
            dz0 ^= dlo & z0;
            sKs = ((uint32_t)__popcll(z0 & dlo) + 2u * (uint32_t)__popcll(z0 & dhi) + pcnt) & 3u;
            odd = oddm;
            Lb = (dhi ^ tU ^ dz0 ^ dLb) & actf;
            act = actf;
        } else if (fold) {
            // rows of D off the diagonal, D z0 (mod 2), and sum_{c in z0} |D_c & z0| =
            // twice the number of pairs of z0 joined in D
            uint64_t dz0 = 0, zs = z0;
            uint32_t pcnt = 0;
            for (int c = 0; c < n; ++c) {
                const uint64_t Doff = NRM_AROW(c) ^ tJ[c];
                sW[c * NRM_TPB] = Doff;
                if (zs & 1ull) {
                    dz0 ^= Doff;
                    pcnt += (uint32_t)__popcll(Doff & z0);
                }
                zs >>= 1;
            }
            dz0 ^= dlo & z0;
            sKs = ((uint32_t)__popcll(z0 & dlo) + 2u * (uint32_t)__popcll(z0 & dhi) + pcnt) & 3u;
            // Z4 form on y: diagonal D_cc + 2 (u + D z0)_c, off-diagonal D (mod 2)
            odd = dlo;
            Lb = dhi ^ tU ^ dz0;
            act = nmask;
            for (int i = 0; i < mf; ++i) {
                // substitute y_p = h . y (h free of pivots): with y_p = sum_h y - 2 sum_pairs
                // (mod 4), the diagonal of p spreads over h (with carry) and onto the
                // pairs of h, and the row q of p couples h with q
                const int p = tPiv[i];
                const uint64_t h = tH[i];
                const uint64_t q = sW[p * NRM_TPB] & act & ~bit64(p);
                const uint64_t op = getb(odd, p), lp = getb(Lb, p);
                Lb ^= h & ((0ull - lp) ^ (odd & (0ull - op)) ^ q);
                odd ^= h & (0ull - op);
                fold_rows(sW, h, q, op);
                act &= ~bit64(p);
            }
            // lift: S_c = Q_c + odd_c odd (rows stay unmasked, see rank_update)
            odd &= act;
            Lb &= act;
            for (uint64_t r = odd; r; r &= r - 1) sW[ffs64(r) * NRM_TPB] ^= odd;
        } else {
        // P = D G row by row (D = (A + J) mod 2 with its diagonal), the pair
        // parities sum_{c<d in g_k} D_cd for every k at once, and those of z0.
        uint64_t pacc = 0, pz = 0, clo = 0, chi = 0;
        for (int c = 0; c < n; ++c) {
            const uint64_t Doff = NRM_AROW(c) ^ tJ[c];
            const uint64_t above = (c == 63) ? 0ull : (~0ull << (c + 1));
            const uint64_t Gc = tG[c];
            sW[c * NRM_TPB] = fr_rows<NCH>(tab, Doff ^ (getb(dlo, c) << c));
            pacc ^= Gc & fr_rows<NCH>(tab, Doff & above);
            if (getb(z0, c)) pz ^= Doff & z0 & above;
            // sum over c in g_k of diag(A+J)_cc (mod 4), bit-sliced over k
            const uint64_t m1 = 0ull - getb(dlo, c), m2 = 0ull - getb(dhi, c);
            chi ^= clo & Gc & m1;
            clo ^= Gc & m1;
            chi ^= Gc & m2;
        }
        for (int c = n; c < 8 * NB; ++c) sW[c * NRM_TPB] = 0;
        transpose_blocks<NB>(sW);              // sW[k] = column k of P = D g_k
        const uint64_t kdlo = clo;             // K_kk mod 2
        const uint64_t kdhi = chi ^ pacc;      // bit 1 of K_kk
        uint64_t lin = 0;
        for (uint64_t vr = S.v; vr; vr &= vr - 1) {
            const int k = ffs64(vr);
            const uint64_t Kr = fr_rows<NCH>(tab, sW[k * NRM_TPB]);   // row k of K (mod 2)
            sW[k * NRM_TPB] = Kr;
            lin |= (getb(S.s, k) ^ (uint64_t)par64(S.s & Kr)) << k;
        }
        sKs = ((uint32_t)__popcll(z0 & dlo) + 2u * (uint32_t)__popcll(z0 & dhi) + 2u * par64(pz)) & 3u;
        // B = K|_v + 2 diag(s + sK); lifted Z2 form: S_jk = B_jk + odd_j odd_k, X adjacent to odd
        odd = kdlo & S.v;
        Lb = (kdhi ^ lin) & S.v;
        act = S.v;
        for (uint64_t vr = S.v; vr; vr &= vr - 1) {
            const int k = ffs64(vr);
            const uint64_t Kr = sW[k * NRM_TPB];
            sW[k * NRM_TPB] = (Kr ^ (getb(odd, k) ? odd : 0ull)) & S.v & ~bit64(k);
        }
        }
        int re_s, im_s, e;
        eliminate(sW, act, odd, Lb, re_s, im_s, e);
        if (re_s == 0 && im_s == 0) continue;
        // zeta = re_s + i im_s as sqrt2^{both} e^{i pi phz / 4}
        int phz;
        if (im_s == 0) phz = re_s > 0 ? 0 : 4;
        else if (re_s == 0) phz = im_s > 0 ? 2 : 6;
        else if (re_s > 0) phz = im_s > 0 ? 1 : 7;
        else phz = im_s > 0 ? 3 : 5;
        const int both = (re_s != 0 && im_s != 0) ? 1 : 0;
        const int vw = __popcll(S.v);
        const int h = (int)(S.omega >> 8);
        const int ph = (int)(S.omega & 7u) - 2 * (int)sKs + 4 * __popcll(S.s & S.v) - phz;
        const int E = vw + h - 2 * (e - 1) - both;
        acc.add(z8_scale(S.coef, ph, E));
    }
    if (l < L) partial[l * n_tiles + tile] = acc.value();
}

// ov (may be NULL) receives the FP64 sums themselves, 2^{n/2} <phi_{A_l}|psi> (the
// per-term values carry the 2^{n/2}), for term-sharded estimates; eta (may be NULL)
// their squared magnitude.
__global__ void k_norm_reduce(const float2* __restrict__ partial, int64_t n_tiles, int64_t L,
                              double* __restrict__ eta, double* __restrict__ ov) {
    const int64_t l = blockIdx.x;
    if (l >= L) return;
    double re = 0.0, im = 0.0;
    for (int64_t t = threadIdx.x; t < n_tiles; t += blockDim.x) {
        const float2 p = partial[l * n_tiles + t];
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
        if (eta) eta[l] = sre[0] * sre[0] + sim[0] * sim[0];
        if (ov) {
            ov[2 * l] = sre[0];
            ov[2 * l + 1] = sim[0];
        }
    }
}

__global__ void k_norm_eta(const double* __restrict__ ov, int64_t L, double* __restrict__ eta) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l < L) eta[l] = ov[2 * l] * ov[2 * l] + ov[2 * l + 1] * ov[2 * l + 1];
}

}  // namespace

template <int NCH>
static lrs_status launch_norm_t(lrs_ctx* ctx, const NormPrep& P, int64_t L, int64_t tt,
                                float2* partial, int64_t n_tiles, cudaStream_t st) {
    constexpr int NB = (NCH + 1) / 2;   // 8 x 8 blocks per side of the transposed matrix
    const size_t smem = ((size_t)NCH * 16 + (size_t)(8 * NB) * NRM_TPB) * sizeof(uint64_t);
    if (!lrs_capturing(st))
        LRS_CUDA(cudaFuncSetAttribute(k_norm<NCH, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t lblocks = (L + NRM_TPB - 1) / NRM_TPB;
    dim3 grid((unsigned)n_tiles, (unsigned)lblocks);
    k_norm<NCH, NB><<<grid, NRM_TPB, smem, st>>>(ctx->view(), P, L, tt, partial, n_tiles,
                                                  (int)ctx->tune_norm_folds,
                                                  (int)(ctx->tune_norm_fuse < NRM_MFUSE ? ctx->tune_norm_fuse
                                                                                        : NRM_MFUSE));
    LRS_LAUNCH_CHECK("norm kernel");
    return LRS_OK;
}

lrs_status launch_norm_eta(const double* ov, int64_t L, double* eta, cudaStream_t st) {
    k_norm_eta<<<(unsigned)((L + 255) / 256), 256, 0, st>>>(ov, L, eta);
    LRS_LAUNCH_CHECK("norm eta kernel");
    return LRS_OK;
}

lrs_status launch_norm_estimate(lrs_ctx* ctx, int64_t L, uint64_t seed, double* eta, double* ov,
                                cudaStream_t st) {
    // tile of terms per block: keep the partial buffer at <= 2048 tiles per A
    int64_t tt = 32;
    while ((ctx->cap + tt - 1) / tt > ctx->tune_norm_tiles) tt *= 2;
    const int64_t n_tiles = (ctx->cap + tt - 1) / tt;
    void* scr = nullptr;
    // scratch: partial sums, then the per-term prep arrays
    const size_t part_bytes = ((size_t)L * n_tiles * sizeof(float2) + 255) & ~(size_t)255;
    const size_t words = (size_t)ctx->cap * (size_t)(ctx->n + 3 + NRM_MFOLD) + (size_t)L * (size_t)(ctx->n + 2);
    lrs_status rc = lrs_scratch(ctx, part_bytes + words * sizeof(uint64_t), &scr);
    if (rc != LRS_OK) return rc;
    float2* partial = (float2*)scr;
    NormPrep P;
    P.J = (uint64_t*)((char*)scr + part_bytes);
    P.z0 = P.J + (size_t)ctx->n * ctx->cap;
    P.u = P.z0 + ctx->cap;
    P.piv = P.u + ctx->cap;
    P.f = P.piv + ctx->cap;
    P.A = P.f + (size_t)NRM_MFOLD * ctx->cap;
    P.adlo = P.A + (size_t)ctx->n * L;
    P.adhi = P.adlo + L;
    const int max_folds = (int)ctx->tune_norm_folds;
    k_norm_prep<<<(unsigned)((ctx->cap + NRM_TPB - 1) / NRM_TPB), NRM_TPB,
                  (size_t)ctx->n * NRM_TPB * sizeof(uint64_t), st>>>(ctx->view(), max_folds, P);
    LRS_LAUNCH_CHECK("norm prep kernel");
    k_norm_draw_a<<<(unsigned)((L + NRM_TPB - 1) / NRM_TPB), NRM_TPB, (size_t)ctx->n * NRM_TPB * sizeof(uint64_t),
                    st>>>(ctx->n, ctx->nmask, L, seed, P);
    LRS_LAUNCH_CHECK("equatorial state kernel");
    if ((L + NRM_TPB - 1) / NRM_TPB > 65535) return lrs_fail(LRS_ERR_UNSUPPORTED, "L too large");
    switch ((ctx->n + 3) / 4) {
        case 1: rc = launch_norm_t<1>(ctx, P, L, tt, partial, n_tiles, st); break;
        case 2: rc = launch_norm_t<2>(ctx, P, L, tt, partial, n_tiles, st); break;
        case 3: rc = launch_norm_t<3>(ctx, P, L, tt, partial, n_tiles, st); break;
        case 4: rc = launch_norm_t<4>(ctx, P, L, tt, partial, n_tiles, st); break;
        case 5: rc = launch_norm_t<5>(ctx, P, L, tt, partial, n_tiles, st); break;
        case 6: rc = launch_norm_t<6>(ctx, P, L, tt, partial, n_tiles, st); break;
        case 7: rc = launch_norm_t<7>(ctx, P, L, tt, partial, n_tiles, st); break;
        case 8: rc = launch_norm_t<8>(ctx, P, L, tt, partial, n_tiles, st); break;
        case 9: rc = launch_norm_t<9>(ctx, P, L, tt, partial, n_tiles, st); break;
        case 10: rc = launch_norm_t<10>(ctx, P, L, tt, partial, n_tiles, st); break;
        case 11: rc = launch_norm_t<11>(ctx, P, L, tt, partial, n_tiles, st); break;
        case 12: rc = launch_norm_t<12>(ctx, P, L, tt, partial, n_tiles, st); break;
        case 13: rc = launch_norm_t<13>(ctx, P, L, tt, partial, n_tiles, st); break;
        case 14: rc = launch_norm_t<14>(ctx, P, L, tt, partial, n_tiles, st); break;
        case 15: rc = launch_norm_t<15>(ctx, P, L, tt, partial, n_tiles, st); break;
        default: rc = launch_norm_t<16>(ctx, P, L, tt, partial, n_tiles, st); break;
    }
    if (rc != LRS_OK) return rc;
    k_norm_reduce<<<(unsigned)L, 256, 0, st>>>(partial, n_tiles, L, eta, ov);
    LRS_LAUNCH_CHECK("norm reduce kernel");
    return LRS_OK;
}
