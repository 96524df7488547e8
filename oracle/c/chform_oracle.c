/*
 * Plain C restatement of the CPU oracle (test infrastructure only; no GPU, no code
 * shared with the CUDA library).  It follows the same paper passages and readings as
 * the Python oracle (oracle/chform.py, oracle/estimators.py, oracle/expsum.py,
 * oracle/decomp.py, oracle/exact.py) and exists to run them at the benchmark's full
 * sizes: every term is built from |0^n> on the fly, its contribution to the requested
 * amplitudes and equatorial overlaps is added to exact integer sums, and the term is
 * dropped, so memory stays O(1) per thread.  The Python wrapper is oracle/fast.py;
 * the tests pin this file against the Python oracle and the dense state vector.
 *
 * CH-form (Sec. 4.1, Eqs. (phi), (tableaux), (Htype)): rows F[p], G[p], M[p] as bit
 * vectors (bit j = column j), gamma[p] in Z4, v, s, and omega = zero ? 0 :
 * e^{i pi k/4} 2^{-h/2}.  Readings as in the Python oracle: the rules of one gate are
 * simultaneous, the incoming omega multiplies Eqs. (H1)/(H7), "the first qubit" of V_b
 * is the lowest index, the single-qubit rewrite is found by brute force with a = 0
 * tried first.
 *
 * Exact sums (the exact Z[zeta8] accumulation of the Python oracle): a term contributes
 * sgn * zeta^K * 2^{-e/2} times a factor common to all terms (zeta = e^{i pi/4}); the
 * sum is kept as four 128-bit integer coordinates over 1, zeta, zeta^2, zeta^3 at the
 * scale 2^-EX_S (zeta^4 = -1; an odd e uses 2^{-1/2} = 2^{-1}(zeta + zeta^7)).
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* gate codes of the wrapper (oracle/fast.py) */
enum { G_H = 0, G_S = 1, G_SDG = 2, G_Z = 3, G_X = 4, G_CX = 5, G_CZ = 6, G_P0 = 7, G_P1 = 8, G_SLOT = 9 };

#define EX_S 100   /* exact sums are integers at scale 2^-EX_S */
#define MAXQ 64

typedef __int128 i128;

typedef struct {
    int n;
    uint64_t mask;
    uint64_t F[MAXQ], G[MAXQ], M[MAXQ];
    int gamma[MAXQ];
    uint64_t v, s;
    int zero, k, h;
} chf;

static int bitof(uint64_t x, int j) { return (int)((x >> j) & 1u); }
static int parity(uint64_t x) { return __builtin_popcountll(x) & 1; }
static int popc(uint64_t x) { return __builtin_popcountll(x); }

static void ch_init(chf* c, int n) {
    memset(c, 0, sizeof(*c));
    c->n = n;
    c->mask = n == 64 ? ~0ull : ((1ull << n) - 1);
    for (int p = 0; p < n; ++p) c->F[p] = c->G[p] = 1ull << p;
}

/* ---- left multiplications U_C <- Gamma U_C (Sec. 4.1) ---------------------------- */
static void left_S(chf* c, int q) {
    c->M[q] ^= c->G[q];
    c->gamma[q] = (c->gamma[q] + 3) & 3;
}
static void left_CZ(chf* c, int q, int r) {
    const uint64_t Gq = c->G[q], Gr = c->G[r];
    c->M[q] ^= Gr;
    c->M[r] ^= Gq;
}
static void left_CX(chf* c, int q, int r) {
    const int g = (c->gamma[q] + c->gamma[r] + 2 * parity(c->M[q] & c->F[r])) & 3;
    const uint64_t Gq = c->G[q], Fr = c->F[r], Mr = c->M[r];
    c->G[r] ^= Gq;
    c->F[q] ^= Fr;
    c->M[q] ^= Mr;
    c->gamma[q] = g;
}

/* ---- right multiplications U_C <- U_C Gamma (Sec. 4.1) --------------------------- */
static void right_S(chf* c, int q) {
    for (int p = 0; p < c->n; ++p) {
        const int f = bitof(c->F[p], q);
        c->M[p] ^= (uint64_t)f << q;
        c->gamma[p] = (c->gamma[p] - f + 4) & 3;
    }
}
static void right_CZ(chf* c, int q, int r) {
    for (int p = 0; p < c->n; ++p) {
        const int fq = bitof(c->F[p], q), fr = bitof(c->F[p], r);
        c->M[p] ^= ((uint64_t)fr << q) ^ ((uint64_t)fq << r);
        c->gamma[p] = (c->gamma[p] + 2 * fq * fr) & 3;
    }
}
static void right_CX(chf* c, int q, int r) {
    for (int p = 0; p < c->n; ++p) {
        c->G[p] ^= (uint64_t)bitof(c->G[p], r) << q;
        c->F[p] ^= (uint64_t)bitof(c->F[p], q) << r;
        c->M[p] ^= (uint64_t)bitof(c->M[p], r) << q;
    }
}

/* k with z = e^{i pi k/4} for a unit complex z on the 8th roots of unity */
static int phase_index(double complex z) {
    const double a = carg(z) / (M_PI / 4);
    const int k = (int)lround(a);
    return ((k % 8) + 8) % 8;
}

/* (a, b, c, k1) with H^vq (|yq> + i^d |zq>) = sqrt2 e^{i pi k1/4} S^a H^b |c>, by brute
 * force over the eight forms, a = 0 first (proof of Prop. (prop:H)). */
static void single_qubit_form(int vq, int yq, int zq, int d, int* a_out, int* b_out, int* c_out, int* k_out) {
    const double r2 = 1.0 / sqrt(2.0);
    double complex vec[2] = {0, 0};
    vec[yq] += 1;
    vec[zq] += cpow(I, d);
    if (vq) {
        const double complex v0 = r2 * (vec[0] + vec[1]), v1 = r2 * (vec[0] - vec[1]);
        vec[0] = v0;
        vec[1] = v1;
    }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int cc = 0; cc < 2; ++cc) {
                double complex cand[2] = {cc == 0 ? 1 : 0, cc == 1 ? 1 : 0};
                if (b) {
                    const double complex w0 = r2 * (cand[0] + cand[1]), w1 = r2 * (cand[0] - cand[1]);
                    cand[0] = w0;
                    cand[1] = w1;
                }
                if (a) cand[1] *= I;
                const double complex inner = vec[0] * conj(cand[0]) + vec[1] * conj(cand[1]);
                const double complex r0 = vec[0] - inner * cand[0], r1 = vec[1] - inner * cand[1];
                if (cabs(r0) < 1e-12 && cabs(r1) < 1e-12) {
                    *a_out = a;
                    *b_out = b;
                    *c_out = cc;
                    *k_out = phase_index(inner / cabs(inner));
                    return;
                }
            }
    abort();   /* unreachable: some form always exists */
}

/* Prop. (prop:H): U_H(|t> + i^delta |u>) = sqrt2 e^{i pi k1/4} W_C W_H |s'>, t != u;
 * returns k1 and updates U_C <- U_C W_C, v, s. */
static int prop_H(chf* c, uint64_t t, uint64_t u, int delta) {
    const uint64_t d = t ^ u;
    const uint64_t V0 = d & ~c->v & c->mask, V1 = d & c->v;
    int q;
    if (V0) {
        q = __builtin_ctzll(V0);
        for (int i = 0; i < c->n; ++i)
            if (bitof(V0, i) && i != q) right_CX(c, q, i);
        for (int i = 0; i < c->n; ++i)
            if (bitof(V1, i)) right_CZ(c, q, i);
    } else {
        q = __builtin_ctzll(V1);
        for (int i = 0; i < c->n; ++i)
            if (bitof(V1, i) && i != q) right_CX(c, i, q);
    }
    uint64_t y, z;
    if (bitof(t, q)) {
        y = u ^ (1ull << q);
        z = u;
    } else {
        y = t;
        z = t ^ (1ull << q);
    }
    int a, b, cc, k1;
    single_qubit_form(bitof(c->v, q), bitof(y, q), bitof(z, q), delta, &a, &b, &cc, &k1);
    if (a) right_S(c, q);
    c->v = (c->v & ~(1ull << q)) | ((uint64_t)b << q);
    c->s = (y & ~(1ull << q)) | ((uint64_t)cc << q);
    return k1;
}

/* Hadamard on qubit p (Eqs. (H1)-(H7)) */
static void apply_H(chf* c, int p) {
    if (c->zero) return;
    const uint64_t nv = ~c->v & c->mask;
    const uint64_t t = c->s ^ (c->G[p] & c->v);
    const uint64_t u = c->s ^ (c->F[p] & nv) ^ (c->M[p] & c->v);
    const int alpha = parity(c->G[p] & nv & c->s);
    const int beta = parity((c->M[p] & nv & c->s) ^ (c->F[p] & c->v & (c->M[p] ^ c->s)));
    const int g = c->gamma[p];
    if (t == u) {
        /* omega' = 2^{-1/2} [(-1)^alpha + i^g (-1)^beta] omega, a unit phase here */
        const double complex f = (alpha ? -1.0 : 1.0) + cpow(I, g) * (beta ? -1.0 : 1.0);
        c->k += phase_index(f / cabs(f));
        c->s = t;
        return;
    }
    const int delta = (g + 2 * (alpha + beta)) & 3;
    c->k += 4 * alpha;
    c->k += prop_H(c, t, u, delta);
}

/* projective gate (I + (-1)^sigma Z_j)/2 (Sec. 4.1, end) */
static void apply_proj(chf* c, int j, int sigma) {
    if (c->zero) return;
    const uint64_t nv = ~c->v & c->mask;
    const uint64_t t = c->s ^ (c->G[j] & c->v);
    const int sign = (sigma + parity(c->G[j] & nv & c->s)) & 1;
    if (t == c->s) {
        if (sign) c->zero = 1;
        return;
    }
    c->k += prop_H(c, c->s, t, 2 * sign);
    c->h += 1;
}

static void apply_gate(chf* c, int op, int q, int r) {
    switch (op) {
        case G_H: apply_H(c, q); break;
        case G_S: left_S(c, q); break;
        case G_SDG: left_S(c, q); left_S(c, q); left_S(c, q); break;
        case G_Z: left_S(c, q); left_S(c, q); break;
        case G_X: apply_H(c, q); left_S(c, q); left_S(c, q); apply_H(c, q); break;
        case G_CX: left_CX(c, q, r); break;
        case G_CZ: left_CZ(c, q, r); break;
        case G_P0: apply_proj(c, q, 0); break;
        case G_P1: apply_proj(c, q, 1); break;
        default: abort();
    }
}

/* ---- counter RNG (SplitMix64 output function in counter mode, published
 * definition: Steele, Lea and Flood 2014) ---------------------------------------- */
static uint64_t mix64(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}
static double uniform01(uint64_t seed, uint64_t stream, uint64_t i) {
    const uint64_t G = 0x9E3779B97F4A7C15ull;
    const uint64_t key = mix64(seed ^ mix64(stream + G));
    return (double)(mix64(key + (i + 1) * G) >> 11) * (1.0 / 9007199254740992.0);
}

/* ---- the circuit as the wrapper passes it ---------------------------------------- */
typedef struct {
    int n;
    int64_t n_gates;
    const int32_t* gates;      /* [n_gates][3]: op, q, r (r = slot index for G_SLOT) */
    int64_t n_slots;
    const int32_t* n_choices;  /* [n_slots] */
    const int32_t* k_off;      /* [n_slots][8] into kgates */
    const int32_t* k_len;      /* [n_slots][8] */
    const int32_t* kgates;     /* [*][3] */
    const int32_t* phase_m;    /* [n_slots][8]: c_j = r_j g_p zeta^{m_j} */
    const int32_t* e_shift;    /* [n_slots][8]: r_j = r_ref 2^{-e_shift/2} */
    const double* cdf;         /* [n_slots][8]: cumulative |c_j| / ||c||_1 (sparsify) */
    const int32_t* nonzero;    /* [n_slots][8]: c_j != 0 */
    int mode;                  /* 0 exact, 1 sparsify */
    uint64_t seed;
} circuit_t;

/* Slot choices of term alpha: exact mixed-radix digits over the nonzero choices
 * (slot 0 least significant), or the first j with u < cdf_j, u = uniform(seed, alpha,
 * p) (Lemma (Sparsification)). */
static void term_choices(const circuit_t* C, int64_t alpha, int* ch) {
    int64_t rem = alpha;
    for (int64_t p = 0; p < C->n_slots; ++p) {
        const int nc = C->n_choices[p];
        if (C->mode == 0) {
            int nzc = 0;
            for (int j = 0; j < nc; ++j) nzc += C->nonzero[p * 8 + j];
            int digit = (int)(rem % nzc);
            rem /= nzc;
            for (int j = 0; j < nc; ++j)
                if (C->nonzero[p * 8 + j]) {
                    if (digit == 0) {
                        ch[p] = j;
                        break;
                    }
                    --digit;
                }
        } else {
            const double u = uniform01(C->seed, (uint64_t)alpha, (uint64_t)p);
            int pick = -1, last = 0;
            for (int j = 0; j < nc; ++j) {
                if (!C->nonzero[p * 8 + j]) continue;
                last = j;
                if (pick < 0 && u < C->cdf[p * 8 + j]) pick = j;
            }
            ch[p] = pick < 0 ? last : pick;
        }
    }
}

/* Build term alpha; returns its coefficient's phase index M and e-shift (b_alpha =
 * common * zeta^M * 2^{-eshift/2}). */
static void build_term(const circuit_t* C, int64_t alpha, int* ch, chf* c, int* M_out, int* eshift_out) {
    term_choices(C, alpha, ch);
    ch_init(c, C->n);
    int M = 0, es = 0;
    for (int64_t i = 0; i < C->n_gates; ++i) {
        const int32_t* g = C->gates + 3 * i;
        if (g[0] == G_SLOT) {
            const int p = g[2], j = ch[p];
            M += C->phase_m[p * 8 + j];
            es += C->e_shift[p * 8 + j];
            const int off = C->k_off[p * 8 + j], len = C->k_len[p * 8 + j];
            for (int e = 0; e < len; ++e) {
                const int32_t* k = C->kgates + 3 * (off + e);
                apply_gate(c, k[0], k[1], k[2]);
            }
        } else {
            apply_gate(c, g[0], g[1], g[2]);
        }
    }
    *M_out = M;
    *eshift_out = es;
}

/* ---- exact Z[zeta8] accumulation ------------------------------------------------ */
static void z8_put(i128* acc, int K, i128 val) {
    K = ((K % 8) + 8) % 8;
    if (K >= 4) {
        val = -val;
        K -= 4;
    }
    acc[K] += val;
}
/* acc += s * zeta^K * 2^{-e/2} at scale 2^-EX_S */
static void z8_add(i128* acc, int K, int e, int64_t s) {
    if (s == 0) return;
    if ((e & 1) == 0) {
        const int sh = EX_S - e / 2;
        if (sh < 0 || sh > 120) abort();
        z8_put(acc, K, (i128)s << sh);
    } else {
        const int sh = EX_S - (e + 1) / 2;
        if (sh < 0 || sh > 120) abort();
        z8_put(acc, K + 1, (i128)s << sh);
        z8_put(acc, K - 1, (i128)s << sh);
    }
}

/* <x|phi> parts (Eqs. (amplitude), (amplitude1)): returns 0 if the term vanishes at
 * x, else 1 with <x|phi> = zeta^K 2^{-e/2} (omega included). */
static int amplitude_parts(const chf* c, uint64_t x, int* K, int* e) {
    if (c->zero) return 0;
    int mu = 0;
    uint64_t uu = 0, ww = 0;
    for (int p = 0; p < c->n; ++p)
        if (bitof(x, p)) {
            mu = (mu + c->gamma[p] + 2 * popc(ww & c->F[p])) & 3;
            uu ^= c->F[p];
            ww ^= c->M[p];
        }
    const uint64_t nv = ~c->v & c->mask;
    if ((uu ^ c->s) & nv) return 0;
    const int sign = popc(uu & ww) + popc(uu & c->s & c->v);
    *K = 2 * mu + 4 * sign + c->k;
    *e = popc(c->v) + c->h;
    return 1;
}

/* ---- exponential sums (Lemma (Exponential Sum)) --------------------------------- */
typedef unsigned __int128 u128;

/* sum over x in {0,1}^m of (-1)^{sum_{a<b} S_ab x_a x_b + L.x} for a symmetric
 * adjacency S on the variables 0..nvar-1 (rows as bit masks, no diagonal), by pairwise
 * elimination
 * (Eqs. (Zreal), (eq1partialsum), (identity), (eq5)): returns sign in {-1, 0, 1} and
 * sets *pow2 with |sum| = 2^pow2. */
static int expsum_z2(u128* S, u128 L, u128 act, int nvar, int* pow2) {
    int sgn = 1, e = 0;
    for (;;) {
        int a = -1, b = -1;
        for (int i = 0; i < nvar && a < 0; ++i)
            if ((act >> i) & 1) {
                const u128 nb = S[i] & act & ~((u128)1 << i);
                if (nb) {
                    a = i;
                    for (b = 0; !((nb >> b) & 1); ++b) {
                    }
                }
            }
        if (a < 0) break;
        const u128 ab = ((u128)1 << a) | ((u128)1 << b);
        const u128 m1 = S[a] & act & ~ab, m2 = S[b] & act & ~ab;
        const int c1 = (int)((L >> a) & 1), c2 = (int)((L >> b) & 1);
        /* sum over x_a, x_b of (-1)^{x_a x_b + (c1 + m1.y) x_a + (c2 + m2.y) x_b}
         * = 2 (-1)^{(c1 + m1.y)(c2 + m2.y)} */
        for (int i = 0; i < nvar; ++i) {
            if (!((act >> i) & 1) || ((ab >> i) & 1)) continue;
            u128 add = 0;
            if ((m1 >> i) & 1) add ^= m2;
            if ((m2 >> i) & 1) add ^= m1;
            S[i] ^= add & ~((u128)1 << i);
        }
        L ^= (c1 ? m2 : 0) ^ (c2 ? m1 : 0) ^ (m1 & m2);
        if (c1 & c2) sgn = -sgn;
        e += 1;
        act &= ~ab;
    }
    /* what is left has no quadratic part: 2^{|act|} if L vanishes on it, else 0 */
    if (L & act) return 0;
    int m = 0;
    for (int i = 0; i < nvar; ++i) m += (int)((act >> i) & 1);
    *pow2 = e + m;
    return sgn;
}

/* Z(B) = sum_x i^{x B x^T} for B symmetric (off-diagonal mod 2, diagonal mod 4), lifted
 * to a Z2 form on one more variable (Eq. (Q)); *re, *im in {0, +-2^p}. */
static void expsum_z4(int m, const int* B, int64_t* re, int64_t* im) {
    u128 S[MAXQ + 1];
    memset(S, 0, sizeof(S));
    u128 L = 0, act = 0;
    int K[64];
    for (int a = 0; a < m; ++a) {
        K[a] = B[a * m + a] & 1;
        if ((B[a * m + a] & 3) >> 1) L |= (u128)1 << a;
        act |= (u128)1 << a;
    }
    for (int a = 0; a < m; ++a)
        for (int b = a + 1; b < m; ++b)
            if (((B[a * m + b] + K[a] * K[b]) & 1) != 0) {
                S[a] |= (u128)1 << b;
                S[b] |= (u128)1 << a;
            }
    const int X = m;   /* the extra variable */
    for (int a = 0; a < m; ++a)
        if (K[a]) {
            S[a] |= (u128)1 << X;
            S[X] |= (u128)1 << a;
        }
    act |= (u128)1 << X;
    int64_t part[2];
    for (int w = 0; w < 2; ++w) {
        u128 S2[MAXQ + 1];
        memcpy(S2, S, sizeof(S));
        const u128 Lw = w ? (L | ((u128)1 << X)) : L;
        int p2 = 0;
        const int sg = expsum_z2(S2, Lw, act, m + 1, &p2);
        part[w] = sg ? (int64_t)sg << p2 : 0;
    }
    /* Eq. (real): the Z2 sums are twice Re Z and Im Z */
    *re = part[0] / 2;
    *im = part[1] / 2;
}

/* <phi|phi_A> parts for the omega = 1 part of c (Lemma (Inner Product)):
 * 2^{-(n+|v|)/2} i^{sKs} (-1)^{s.v} Z(B), K = G^T (A+J) G over the integers. */
static void inner_parts(const chf* c, const int8_t* A, int* sKs, int* sv, int* nvars, int64_t* re, int64_t* im) {
    const int n = c->n;
    static __thread int D[MAXQ * MAXQ], Gm[MAXQ * MAXQ], T[MAXQ * MAXQ], Km[MAXQ * MAXQ], Bm[MAXQ * MAXQ];
    /* D = A + J: J_ab = (M F^T)_ab mod 2 off the diagonal, gamma on it; Gm = G as a 0/1
     * integer matrix */
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            D[a * n + b] = A[a * n + b] + (a == b ? c->gamma[a] : parity(c->M[a] & c->F[b]));
            Gm[a * n + b] = bitof(c->G[a], b);
        }
    /* T = D G, then K = G^T T (integer matrix products) */
    for (int a = 0; a < n; ++a) {
        int* Ta = T + a * n;
        for (int j = 0; j < n; ++j) Ta[j] = 0;
        for (int b = 0; b < n; ++b) {
            const int d = D[a * n + b];
            const int* Gb = Gm + b * n;
            for (int j = 0; j < n; ++j) Ta[j] += d * Gb[j];
        }
    }
    for (int i = 0; i < n; ++i) {
        int* Ki = Km + i * n;
        for (int j = 0; j < n; ++j) Ki[j] = 0;
        for (int a = 0; a < n; ++a) {
            const int g = Gm[a * n + i];
            const int* Ta = T + a * n;
            for (int j = 0; j < n; ++j) Ki[j] += g * Ta[j];
        }
    }
    int sk = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) sk += bitof(c->s, i) * Km[i * n + j] * bitof(c->s, j);
    *sKs = ((sk % 4) + 4) % 4;
    /* B = (K + 2 diag(s + sK)) restricted to v */
    int idx[MAXQ], m = 0;
    for (int j = 0; j < n; ++j)
        if (bitof(c->v, j)) idx[m++] = j;
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
            int val = Km[idx[a] * n + idx[b]];
            if (a == b) {
                int lin = bitof(c->s, idx[a]);
                for (int i = 0; i < n; ++i) lin += bitof(c->s, i) * Km[i * n + idx[a]];
                val += 2 * (lin & 1);
                val = ((val % 4) + 4) % 4;
            } else {
                val = ((val % 2) + 2) % 2;
            }
            Bm[a * m + b] = val;
        }
    *sv = parity(c->s & c->v);
    *nvars = m;
    expsum_z4(m, Bm, re, im);
}

/* ---- the threaded sweep over terms ----------------------------------------------- */
typedef struct {
    const circuit_t* C;
    int64_t a0, a1;
    const uint64_t* xs;
    int64_t nx;
    const int8_t* As;   /* [nA][n][n] */
    int64_t nA;
    i128* acc;          /* [(nx + nA) * 4] this worker's sums */
} job_t;

static void* worker(void* arg) {
    job_t* J = (job_t*)arg;
    const circuit_t* C = J->C;
    const int n = C->n;
    int* ch = (int*)malloc(sizeof(int) * (size_t)(C->n_slots > 0 ? C->n_slots : 1));
    chf c;
    for (int64_t alpha = J->a0; alpha < J->a1; ++alpha) {
        int M = 0, es = 0;
        build_term(C, alpha, ch, &c, &M, &es);
        if (c.zero) continue;
        for (int64_t i = 0; i < J->nx; ++i) {
            int K, e;
            if (amplitude_parts(&c, J->xs[i], &K, &e)) z8_add(J->acc + 4 * i, K + M, e + es, 1);
        }
        for (int64_t l = 0; l < J->nA; ++l) {
            int sKs, sv, nv;
            int64_t re, im;
            inner_parts(&c, J->As + l * n * n, &sKs, &sv, &nv, &re, &im);
            /* b omega conj(<phi'|phi_A>): zeta^{M + k - 2 sKs + 4 sv} 2^{-(h + n + |v|)/2}
             * (re - i im) */
            const int K = M + c.k - 2 * sKs + 4 * sv, e = c.h + n + nv + es;
            i128* acc = J->acc + 4 * (J->nx + l);
            z8_add(acc, K, e, re);
            z8_add(acc, K + 6, e, im);
        }
    }
    free(ch);
    return 0;
}

/* Exact sums over the terms [alpha0, alpha0 + count) of the decomposition: for each x_i
 * the coordinates of sum_alpha (b_alpha / common) <x_i|phi_alpha>, then for each A_l
 * those of sum_alpha (b_alpha / common) omega_alpha conj(<phi'_alpha|phi_{A_l}>), as
 * four 128-bit integers each (low and high 64-bit halves, out[8 r + 2 j], out[8 r + 2
 * j + 1]) at the scale 2^-EX_S.  Returns 0, or -1 for bad arguments. */
int oracle_sums(int n, int64_t n_gates, const int32_t* gates, int64_t n_slots, const int32_t* n_choices,
                const int32_t* k_off, const int32_t* k_len, const int32_t* kgates, const int32_t* phase_m,
                const int32_t* e_shift, const double* cdf, const int32_t* nonzero, int mode, uint64_t seed,
                int64_t alpha0, int64_t count, const uint64_t* xs, int64_t nx, const int8_t* As, int64_t nA,
                int threads, int64_t* out) {
    if (n < 1 || n > MAXQ || count < 0 || threads < 1 || nx < 0 || nA < 0) return -1;
    circuit_t C = {n, n_gates, gates, n_slots, n_choices, k_off, k_len, kgates, phase_m, e_shift, cdf, nonzero,
                   mode, seed};
    const int64_t rows = nx + nA;
    if (threads > count && count > 0) threads = (int)count;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
    job_t* jobs = (job_t*)calloc((size_t)threads, sizeof(job_t));
    for (int t = 0; t < threads; ++t) {
        jobs[t].C = &C;
        jobs[t].a0 = alpha0 + count * t / threads;
        jobs[t].a1 = alpha0 + count * (t + 1) / threads;
        jobs[t].xs = xs;
        jobs[t].nx = nx;
        jobs[t].As = As;
        jobs[t].nA = nA;
        jobs[t].acc = (i128*)calloc((size_t)(4 * (rows > 0 ? rows : 1)), sizeof(i128));
        pthread_create(&th[t], 0, worker, &jobs[t]);
    }
    i128* tot = (i128*)calloc((size_t)(4 * (rows > 0 ? rows : 1)), sizeof(i128));
    for (int t = 0; t < threads; ++t) {
        pthread_join(th[t], 0);
        for (int64_t i = 0; i < 4 * rows; ++i) tot[i] += jobs[t].acc[i];
        free(jobs[t].acc);
    }
    for (int64_t i = 0; i < 4 * rows; ++i) {
        const unsigned __int128 u = (unsigned __int128)tot[i];
        out[2 * i] = (int64_t)(uint64_t)u;
        out[2 * i + 1] = (int64_t)(uint64_t)(u >> 64);
    }
    free(tot);
    free(jobs);
    free(th);
    return 0;
}

/* Tableau of one term (bit-exact comparisons with the Python oracle):
 * F, G, M [n] each, gamma [n], then v, s, zero, k mod 8, h. */
int oracle_term(int n, int64_t n_gates, const int32_t* gates, int64_t n_slots, const int32_t* n_choices,
                const int32_t* k_off, const int32_t* k_len, const int32_t* kgates, const int32_t* phase_m,
                const int32_t* e_shift, const double* cdf, const int32_t* nonzero, int mode, uint64_t seed,
                int64_t alpha, uint64_t* rows_out, int32_t* gamma_out, int64_t* scal_out) {
    if (n < 1 || n > MAXQ) return -1;
    circuit_t C = {n, n_gates, gates, n_slots, n_choices, k_off, k_len, kgates, phase_m, e_shift, cdf, nonzero,
                   mode, seed};
    int* ch = (int*)malloc(sizeof(int) * (size_t)(n_slots > 0 ? n_slots : 1));
    chf c;
    int M, es;
    build_term(&C, alpha, ch, &c, &M, &es);
    free(ch);
    for (int p = 0; p < n; ++p) {
        rows_out[p] = c.F[p];
        rows_out[n + p] = c.G[p];
        rows_out[2 * n + p] = c.M[p];
        gamma_out[p] = c.gamma[p];
    }
    scal_out[0] = (int64_t)c.v;
    scal_out[1] = (int64_t)c.s;
    scal_out[2] = c.zero;
    scal_out[3] = ((c.k % 8) + 8) % 8;
    scal_out[4] = c.h;
    scal_out[5] = M;
    scal_out[6] = es;
    return 0;
}
