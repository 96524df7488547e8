// Norm estimation (Sec. 4.3): eta_l = 2^n |<phi_{A_l}|psi>|^2.
//
// One thread per equatorial state A_l; a block walks a tile of terms, so each
// thread keeps its own FP32 Kahan sum over terms and no cross-thread reduction
// is needed inside the tile.  Per (A, term), with g_k = column k of G and
// D = (A + J) mod 2 (J_cd = (M F^T)_cd off the diagonal):
//   R_k   = D g_k^T  (XOR of the rows D_d, d in g_k, plus the diagonal parity)
//   K_k   = XOR of rows G_c over c in R_k       -> row k of K = G^T (A+J) G mod 2
//   K_kk  = sum_{c in g_k} (A_cc + gamma_c) + 2 #{c<d in g_k : D_cd = 1}  (mod 4)
// for k in v only (Lemma (Inner Product)), then the exponential sum of
// B = K|_v + 2 diag(s + sK) by pairwise elimination on a symmetric adjacency
// (Lemma (Exponential Sum), lifted to Z2 with one extra variable, Eq. (Q)).
// Everything up to the chi-sum is exact integer arithmetic.
#include "lrs_device.cuh"

namespace {

constexpr int NRM_TPB = 64;   // A's per block

struct NormTerm {
    uint64_t glo, ghi, v, s, z0;
    uint32_t omega;
    float2 coef;
};

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
        const uint64_t m1 = odd & ~bit64(bq);
        const uint64_t m2 = sK[bq * NRM_TPB] & act & ~bit64(bq);
        e += 1;
        sim ^= (uint32_t)getb(Lim, bq);
        const uint64_t mm = m1 & m2;
        Lre ^= (getb(Lre, bq) ? m1 : 0ull) ^ mm;
        Lim ^= m2 ^ (getb(Lim, bq) ? m1 : 0ull) ^ mm;
        for (uint64_t r = m1; r; r &= r - 1) sK[ffs64(r) * NRM_TPB] ^= m2;
        for (uint64_t r = m2; r; r &= r - 1) sK[ffs64(r) * NRM_TPB] ^= m1;
        act &= ~bit64(bq);
    } else {
        e += 1;      // sum over x_X of (-1)^0 = 2 (Re), of (-1)^x_X = 0 (Im)
        zim = true;
    }
    uint64_t cand = act;
    while (cand) {
        const int a = ffs64(cand);
        const uint64_t ra = sK[a * NRM_TPB] & act & ~bit64(a);
        if (!ra) {           // isolated: stays isolated
            cand &= ~bit64(a);
            continue;
        }
        const int bq = ffs64(ra);
        const uint64_t ab = bit64(a) | bit64(bq);
        const uint64_t m1 = ra & ~bit64(bq);
        const uint64_t m2 = sK[bq * NRM_TPB] & act & ~ab;
        const uint64_t c1r = getb(Lre, a), c2r = getb(Lre, bq);
        const uint64_t c1i = getb(Lim, a), c2i = getb(Lim, bq);
        e += 1;
        sre ^= (uint32_t)(c1r & c2r);
        sim ^= (uint32_t)(c1i & c2i);
        const uint64_t mm = m1 & m2;
        Lre ^= (m2 & (0ull - c1r)) ^ (m1 & (0ull - c2r)) ^ mm;
        Lim ^= (m2 & (0ull - c1i)) ^ (m1 & (0ull - c2i)) ^ mm;
        for (uint64_t r = m1; r; r &= r - 1) sK[ffs64(r) * NRM_TPB] ^= m2;
        for (uint64_t r = m2; r; r &= r - 1) sK[ffs64(r) * NRM_TPB] ^= m1;
        act &= ~ab;
        cand &= ~ab;
    }
    e += __popcll(act);
    if (Lre & act) zre = true;
    if (Lim & act) zim = true;
    re_s = zre ? 0 : (sre ? -1 : 1);
    im_s = zim ? 0 : (sim ? -1 : 1);
}

__global__ void __launch_bounds__(NRM_TPB) k_norm(TermsView T, int64_t L, uint64_t seed, int64_t tt,
                                                  float2* __restrict__ partial, int64_t n_tiles) {
    extern __shared__ uint64_t smem[];
    __shared__ uint64_t tG[64], tGT[64], tJ[64], tF[64], tM[64];
    __shared__ NormTerm tS;
    __shared__ unsigned long long tz0;
    const int n = T.n;
    const uint64_t nmask = T.nmask;
    const int tid = threadIdx.x;
    const int64_t l = (int64_t)blockIdx.y * NRM_TPB + tid;
    uint64_t* sA = smem + tid;                     // A_c at sA[c * NRM_TPB]
    uint64_t* sK = smem + (int64_t)n * NRM_TPB + tid;

    // ---- A_l in M_n from the counter RNG
    const uint64_t key = sm64_key(seed, (uint64_t)(l < L ? l : 0));
    const uint64_t adlo = sm64_at(key, 0) & nmask;
    const uint64_t adhi = sm64_at(key, 1) & nmask;
    for (int c = 0; c < n; ++c) sA[c * NRM_TPB] = 0;
    {
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
            sA[a * NRM_TPB] = rowa;
        }
    }

    KahanC acc;
    acc.init();
    const int64_t tile = blockIdx.x;
    for (int64_t t = 0; t < tt; ++t) {
        const int64_t alpha = tile * tt + t;
        if (alpha >= T.cap) break;              // uniform across the block
        __syncthreads();
        if (tid < n) {
            tG[tid] = T.G[(int64_t)tid * T.cap + alpha];
            tF[tid] = T.F[(int64_t)tid * T.cap + alpha];
            tM[tid] = T.M[(int64_t)tid * T.cap + alpha];
        }
        if (tid == 0) {
            tS.glo = T.glo[alpha]; tS.ghi = T.ghi[alpha];
            tS.v = T.v[alpha]; tS.s = T.s[alpha];
            tS.omega = T.omega[alpha]; tS.coef = T.coef[alpha];
            tz0 = 0ull;
        }
        __syncthreads();
        if (tid < n) {
            // column tid of G, row tid of J = (M F^T) off the diagonal, bit tid of z0 = s G^T
            uint64_t col = 0, jrow = 0;
            const uint64_t Mc = tM[tid];
            for (int c = 0; c < n; ++c) {
                col |= getb(tG[c], tid) << c;
                if (c != tid) jrow |= (uint64_t)par64(Mc & tF[c]) << c;
            }
            tGT[tid] = col;
            tJ[tid] = jrow;
            if (par64(tS.s & tG[tid])) atomicOr(&tz0, 1ull << tid);
        }
        __syncthreads();
        const NormTerm S = tS;
        if ((S.omega >> 3) & 1u) continue;     // zero term (uniform)
        // diag(A + J) mod 4 as bit-planes: lo = adlo ^ glo, hi = adhi ^ ghi ^ (adlo & glo)
        const uint64_t dlo = adlo ^ S.glo;
        const uint64_t dhi = adhi ^ S.ghi ^ (adlo & S.glo);
        uint64_t kdlo = 0, kdhi = 0;
        for (uint64_t vr = S.v; vr; vr &= vr - 1) {
            const int k = ffs64(vr);
            const uint64_t gk = tGT[k];
            uint64_t R = 0, pacc = 0;
            for (uint64_t gr = gk; gr;) {
                const int d = ffs64(gr);
                gr &= gr - 1;                       // gr = bits of g_k above d
                const uint64_t D = sA[d * NRM_TPB] ^ tJ[d];
                R ^= D;
                pacc ^= D & gr;
            }
            R ^= gk & dlo;
            uint64_t Kr = 0;
            for (uint64_t rr = R; rr; rr &= rr - 1) Kr ^= tG[ffs64(rr)];
            const uint32_t d4 = ((uint32_t)__popcll(gk & dlo) + 2u * (uint32_t)__popcll(gk & dhi) +
                                 2u * par64(pacc)) & 3u;
            sK[k * NRM_TPB] = Kr;
            kdlo |= (uint64_t)(d4 & 1u) << k;
            kdhi |= (uint64_t)(d4 >> 1) << k;
        }
        // s K s^T = q_{A+J}(z0) mod 4
        const uint64_t z0 = tz0;
        uint64_t pz = 0;
        for (uint64_t zr = z0; zr;) {
            const int c = ffs64(zr);
            zr &= zr - 1;
            pz ^= (sA[c * NRM_TPB] ^ tJ[c]) & zr;
        }
        const uint32_t sKs = ((uint32_t)__popcll(z0 & dlo) + 2u * (uint32_t)__popcll(z0 & dhi) +
                              2u * par64(pz)) & 3u;
        // B = K|_v + 2 diag(s + sK); lifted Z2 form: S_jk = B_jk + odd_j odd_k, X adjacent to odd
        uint64_t lin = 0;
        for (uint64_t vr = S.v; vr; vr &= vr - 1) {
            const int k = ffs64(vr);
            lin |= (getb(S.s, k) ^ (uint64_t)par64(S.s & sK[k * NRM_TPB])) << k;
        }
        const uint64_t odd = kdlo;                 // B_jj mod 2 = K_jj mod 2
        const uint64_t Lb = (kdhi ^ lin) & S.v;    // bit 1 of B_jj
        for (uint64_t vr = S.v; vr; vr &= vr - 1) {
            const int k = ffs64(vr);
            const uint64_t Kr = sK[k * NRM_TPB];
            sK[k * NRM_TPB] = (Kr ^ (getb(odd, k) ? odd : 0ull)) & S.v & ~bit64(k);
        }
        int re_s, im_s, e;
        eliminate(sK, S.v, odd, Lb, re_s, im_s, e);
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

__global__ void k_norm_reduce(const float2* __restrict__ partial, int64_t n_tiles, int64_t L,
                              double* __restrict__ eta) {
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
    if (threadIdx.x == 0) eta[l] = sre[0] * sre[0] + sim[0] * sim[0];
}

}  // namespace

lrs_status launch_norm_estimate(lrs_ctx* ctx, int64_t L, uint64_t seed, double* eta,
                                cudaStream_t st) {
    // tile of terms per block: keep the partial buffer at <= 2048 tiles per A
    int64_t tt = 32;
    while (ctx->cap / tt > 2048) tt *= 2;
    const int64_t n_tiles = (ctx->cap + tt - 1) / tt;
    void* scr = nullptr;
    lrs_status rc = lrs_scratch(ctx, (size_t)L * n_tiles * sizeof(float2), &scr);
    if (rc != LRS_OK) return rc;
    float2* partial = (float2*)scr;
    const size_t smem = (size_t)2 * ctx->n * NRM_TPB * sizeof(uint64_t);
    LRS_CUDA(cudaFuncSetAttribute(k_norm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  2 * 64 * NRM_TPB * (int)sizeof(uint64_t)));
    const int64_t lblocks = (L + NRM_TPB - 1) / NRM_TPB;
    if (lblocks > 65535) return lrs_fail(LRS_ERR_UNSUPPORTED, "L too large");
    dim3 grid((unsigned)n_tiles, (unsigned)lblocks);
    k_norm<<<grid, NRM_TPB, smem, st>>>(ctx->view(), L, seed, tt, partial, n_tiles);
    LRS_LAUNCH_CHECK("norm kernel");
    k_norm_reduce<<<(unsigned)L, 256, 0, st>>>(partial, n_tiles, L, eta);
    LRS_LAUNCH_CHECK("norm reduce kernel");
    return LRS_OK;
}
