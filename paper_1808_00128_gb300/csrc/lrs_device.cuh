// Device helpers: counter RNG, bit utilities, Z8 phases, CH-form gate rules.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lrs_internal.h"

// ---- SplitMix64 in counter mode (Steele, Lea, Flood 2014) ------------------------
__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}
__host__ __device__ __forceinline__ uint64_t sm64_key(uint64_t seed, uint64_t stream) {
    return sm64_mix(seed ^ sm64_mix(stream + 0x9E3779B97F4A7C15ull));
}
__host__ __device__ __forceinline__ uint64_t sm64_at(uint64_t key, uint64_t i) {
    return sm64_mix(key + (i + 1) * 0x9E3779B97F4A7C15ull);
}
__host__ __device__ __forceinline__ double sm64_unit(uint64_t r) {
    return (double)(r >> 11) * (1.0 / 9007199254740992.0);
}

// ---- bits ----------------------------------------------------------------------
__device__ __forceinline__ uint32_t par64(uint64_t x) {
    return __popc((uint32_t)x ^ (uint32_t)(x >> 32)) & 1u;
}
__device__ __forceinline__ int ffs64(uint64_t x) {  // index of lowest set bit, x != 0
    return __ffsll((long long)x) - 1;
}
__device__ __forceinline__ uint64_t bit64(int j) { return 1ull << j; }
__device__ __forceinline__ uint64_t getb(uint64_t x, int j) { return (x >> j) & 1ull; }

// ---- exact Z8 phase times power of sqrt2, rounded once to FP32 -------------------
// returns b * exp(i pi ph / 4) * 2^(-e/2)  (ph any int, e any int)
__device__ __forceinline__ float2 z8_scale(float2 b, int ph, int e) {
    ph &= 7;
    // odd e: 2^(-1/2) factor; odd ph: (1+i)/sqrt2 factor.  Both odd: (1+i)/2 exact.
    const float r2 = 0.70710678118654752440f;
    float2 z = b;
    int halfe;
    if (e >= 0) halfe = e >> 1; else halfe = -((-e + 1) >> 1);   // floor(e/2)
    bool oddE = (e - 2 * halfe) != 0;                             // e = 2 halfe + oddE
    if (ph & 1) {
        // multiply by (1+i): (x - y) + i (x + y)
        float2 t = make_float2(z.x - z.y, z.x + z.y);
        if (oddE) {
            z = make_float2(t.x * 0.5f, t.y * 0.5f);       // (1+i)/2 = e^{i pi/4} / sqrt2
        } else {
            z = make_float2(t.x * r2, t.y * r2);           // (1+i)/sqrt2
        }
    } else if (oddE) {
        z = make_float2(z.x * r2, z.y * r2);
    }
    // remaining i^(ph >> 1)
    switch ((ph >> 1) & 3) {
        case 1: z = make_float2(-z.y, z.x); break;
        case 2: z = make_float2(-z.x, -z.y); break;
        case 3: z = make_float2(z.y, -z.x); break;
        default: break;
    }
    return make_float2(ldexpf(z.x, -halfe), ldexpf(z.y, -halfe));
}

// ---- compensated FP32 complex accumulation (Kahan) ------------------------------
struct KahanC {
    float2 s, c;
    __device__ __forceinline__ void init() { s = make_float2(0.f, 0.f); c = s; }
    __device__ __forceinline__ void add(float2 x) {
        float yx = x.x - c.x, yy = x.y - c.y;
        float tx = s.x + yx, ty = s.y + yy;
        c.x = (tx - s.x) - yx;
        c.y = (ty - s.y) - yy;
        s.x = tx; s.y = ty;
    }
    __device__ __forceinline__ float2 value() const { return make_float2(s.x - c.x, s.y - c.y); }
};

// ---- CH-form state in registers, rows behind an accessor ------------------------
struct TermRegs {
    uint64_t glo, ghi, v, s;
    uint32_t k;     // omega phase (mod 8 in use)
    uint32_t h;     // omega = 2^(-h/2) ...
    uint32_t zero;  // omega = 0
};

__device__ __forceinline__ uint32_t gamma_get(const TermRegs& t, int p) {
    return (uint32_t)(getb(t.glo, p) | (getb(t.ghi, p) << 1));
}
__device__ __forceinline__ void gamma_set(TermRegs& t, int p, uint32_t g) {
    uint64_t m = bit64(p);
    t.glo = (t.glo & ~m) | ((uint64_t)(g & 1u) << p);
    t.ghi = (t.ghi & ~m) | ((uint64_t)((g >> 1) & 1u) << p);
}

// Single-qubit rewrite H^{vq}(|yq> + i^d |1-yq>) = sqrt2 e^{i pi dk/4} S^a H^b |c>,
// after mapping yq = 1 to yq = 0 (k += 2d, d -> -d).  Entry = a | b<<1 | c<<2 | dk<<3,
// indexed [vq*4 + d].  For b = 0 the entry takes a = 0.
__device__ __forceinline__ uint32_t sq_entry(int vq, int d) {
    // vq=0: d0 (0,1,0,0) d1 (1,1,0,0) d2 (0,1,1,0) d3 (1,1,1,0)
    // vq=1: d0 (0,0,0,0) d1 (1,1,1,1) d2 (0,0,1,0) d3 (1,1,0,7)
    const uint32_t tab[8] = {0x2u, 0x3u, 0x6u, 0x7u, 0x0u, 0x7u | (1u << 3), 0x4u, 0x3u | (7u << 3)};
    return tab[vq * 4 + d];
}

// Row pass of the Hadamard fan-out (proof of Prop. (prop:H)) followed by R[S_q]^a.
// With V0 = d \ v nonempty (q = min V0, mA = V0 \ q, m1 = V1):
//   R[CX_{q,i}], i in mA:  G[p,q] ^= G[p,i]; F[p,i] ^= F[p,q]; M[p,q] ^= M[p,i]
//   R[CZ_{q,i}], i in m1:  M[p,q] ^= F[p,i]; M[p,i] ^= F[p,q]; gamma_p += 2 F[p,q] F[p,i]
// otherwise (q = min V1, mB = V1 \ q):
//   R[CX_{i,q}], i in mB:  G[p,i] ^= G[p,q]; F[p,q] ^= F[p,i]; M[p,i] ^= M[p,q]
// and then, when a = 1,    R[S_q]: M[p,q] ^= F[p,q]; gamma_p -= F[p,q].
// Both fan-outs have one matrix X that takes a parity into column q (G, resp. F) and
// one matrix Y that copies its column q out over the mask (F, resp. G), so each term
// works on X and Y through row pointers chosen once per gate, and only M differs:
// parity over mA plus the CZ terms (first case) or a copy of M[p,q] over mB (second).
// Rows are worked on as 32-bit halves: bit q of a row is taken from the half that holds
// it (sign-extended to a whole-word mask), a parity is placed at q through the one-bit
// masks qml/qmh, and the bits of add2 / sub1 are shifted in from the top row down.
struct HRowMasks {
    uint32_t qs, sh, qml, qmh, aql, aqh, a;
    uint32_t ml, mh;     // mA or mB
    uint32_t m1l, m1h;   // m1 (0 in the second case)
    uint32_t mPl, mPh;   // parity mask of M: mA (0 in the second case)
    uint32_t mFl, mFh;   // mask of the copy into M: m1, or mB
    bool qh, first;      // q >= 32; the first case
};

template <bool FAN, class Rows, class Mat>
__device__ __forceinline__ void prop_h_row(Rows& R, const Mat& X, const Mat& Y, const Mat& Mm, int p,
                                           const HRowMasks& k, uint64_t Xp, uint64_t Yp, uint64_t Mp,
                                           uint32_t& add2, uint32_t& sub1) {
    const uint32_t Xl = (uint32_t)Xp, Xh = (uint32_t)(Xp >> 32);
    const uint32_t Yl = (uint32_t)Yp, Yh = (uint32_t)(Yp >> 32);
    const uint32_t Ml = (uint32_t)Mp, Mh = (uint32_t)(Mp >> 32);
    uint32_t Xnl = Xl, Xnh = Xh, Ynl = Yl, Ynh = Yh, Mnl = Ml, Mnh = Mh;
    uint32_t f2 = 0;
    if (FAN) {
        const uint32_t my = (uint32_t)((int32_t)((k.qh ? Yh : Yl) << k.sh) >> 31);   // Y[p,q]
        const uint32_t mm = (uint32_t)((int32_t)((k.qh ? Mh : Ml) << k.sh) >> 31);   // M[p,q]
        const uint32_t c1 = __popc((Yl & k.m1l) ^ (Yh & k.m1h));
        const uint32_t tx = __popc((Xl & k.ml) ^ (Xh & k.mh)) << k.qs;
        const uint32_t tm = (__popc((Ml & k.mPl) ^ (Mh & k.mPh)) ^ c1) << k.qs;
        const uint32_t ms = k.first ? my : mm;
        Xnl ^= tx & k.qml;
        Xnh ^= tx & k.qmh;
        Ynl ^= k.ml & my;
        Ynh ^= k.mh & my;
        Mnl ^= (tm & k.qml) ^ (k.mFl & ms);
        Mnh ^= (tm & k.qmh) ^ (k.mFh & ms);
        f2 = c1 & my & 1u;
    }
    // a F'[p,q]: F is Y in the first case (column q unchanged), X in the second
    const uint32_t fl = k.first ? Ynl : Xnl, fh = k.first ? Ynh : Xnh;
    const uint32_t fs = ((k.qh ? fh : fl) >> k.qs) & k.a;
    Mnl ^= fl & k.aql;
    Mnh ^= fh & k.aqh;
    add2 = (add2 << Rows::kStep) + f2;   // own rows are kStep apart
    sub1 = (sub1 << Rows::kStep) + fs;
    if (FAN) {
        R.set(X, p, ((uint64_t)Xnh << 32) | Xnl);
        R.set(Y, p, ((uint64_t)Ynh << 32) | Ynl);
    }
    R.set(Mm, p, ((uint64_t)Mnh << 32) | Mnl);
}

// Rows p, p - ST, .., p - (U - 1) ST (all >= lo): the 3U row loads are issued before
// the first row is rewritten, so the loads of a group overlap one another and the
// rewrites of its rows are independent chains.  (The row accessors order every shared
// access after the previous store, so a load placed after a store waits for it.)
template <int U, bool FAN, class Rows, class Mat>
__device__ __forceinline__ void prop_h_group(Rows& R, const Mat& X, const Mat& Y, const Mat& Mm, int p,
                                             const HRowMasks& k, uint32_t& add2, uint32_t& sub1) {
    constexpr int ST = Rows::kStep;
    uint64_t xs[U], ys[U], ms[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        xs[u] = R.get(X, p - u * ST);
        ys[u] = R.get(Y, p - u * ST);
        ms[u] = R.get(Mm, p - u * ST);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) prop_h_row<FAN>(R, X, Y, Mm, p - u * ST, k, xs[u], ys[u], ms[u], add2, sub1);
}

// This lane's rows from p down to lo (p = lo mod ST), top row first, in groups of
// Rows::kRowUnroll.
template <bool FAN, class Rows, class Mat>
__device__ __forceinline__ void prop_h_span(Rows& R, const Mat& X, const Mat& Y, const Mat& Mm, int p, int lo,
                                            const HRowMasks& k, uint32_t& add2, uint32_t& sub1) {
    constexpr int ST = Rows::kStep, U = Rows::kRowUnroll;
    for (; p - (U - 1) * ST >= lo; p -= U * ST) prop_h_group<U, FAN>(R, X, Y, Mm, p, k, add2, sub1);
    for (; p >= lo; p -= ST) prop_h_group<1, FAN>(R, X, Y, Mm, p, k, add2, sub1);
}

// QLO: q < 32 for every term of the warp (the usual case: q is the lowest bit of a
// mask), so column q lies in the low halves and the high halves only take part in the
// parities and the fan-out copies.
// SECOND: every term of the warp has V0 empty (e.g. all of v set, as after a layer of
// Hadamards on |0>), so no CZ part and no parity into M.
template <bool FAN, bool QLO, bool SECOND, class Rows>
__device__ __forceinline__ void prop_h_rows(Rows& R, int n, const HRowMasks& k0, uint64_t& add2, uint64_t& sub1) {
    HRowMasks k = k0;
    if (QLO) {
        k.qh = false;
        k.qmh = 0u;
        k.aqh = 0u;
    }
    if (SECOND) {
        k.first = false;
        k.m1l = k.m1h = k.mPl = k.mPh = 0u;
        k.mFl = k.ml;
        k.mFh = k.mh;
    }
    const auto X = k.first ? R.matG() : R.matF();
    const auto Y = k.first ? R.matF() : R.matG();
    const auto Mm = R.matM();
    uint32_t ah = 0, sh = 0, al = 0, sl = 0;
    // this lane's rows: p = part (mod kStep), walked downwards in each 32-row half; the
    // bit of row p lands at p - (lowest own row of the half) and is shifted into place
    constexpr int ST = Rows::kStep;
    const int part = R.part();
    const int top = n - 1 - ((n - 1 - part) & (ST - 1));
    prop_h_span<FAN>(R, X, Y, Mm, top, 32, k, ah, sh);
    const int lt = (n < 32 ? n : 32) - 1;
    prop_h_span<FAN>(R, X, Y, Mm, lt - ((lt - part) & (ST - 1)), 0, k, al, sl);
    add2 = R.combine(((uint64_t)(ah << part) << 32) | (al << part));
    sub1 = R.combine(((uint64_t)(sh << part) << 32) | (sl << part));
}

// Prop. (prop:H): U_H(|t> + i^delta |u>) = sqrt2 e^{i pi k1/4} W_C W_H |s'> for t != u.
// Applies U_C <- U_C W_C to every row (fused fan-out of right multiplications,
// then R[S_q] when a = 1), updates v, s and adds k1 to the phase.
template <class Rows>
__device__ __forceinline__ void prop_h(Rows& R, TermRegs& T, int n, uint64_t t, uint64_t u,
                                       uint32_t delta) {
    const uint64_t d = t ^ u;
    const uint64_t V0 = d & ~T.v;
    const uint64_t V1 = d & T.v;
    // V_C = prod_{i in V0\q} CX_{q,i} prod_{i in V1} CZ_{q,i} when V0 is nonempty,
    // else prod_{i in V1\q} CX_{i,q}
    const bool first = V0 != 0;
    const int q = ffs64(first ? V0 : V1);
    const uint64_t m = (first ? V0 : V1) & ~bit64(q);
    const uint64_t m1 = first ? V1 : 0ull;
    uint64_t y;
    if (getb(t, q)) y = u ^ bit64(q); else y = t;
    const int yq = (int)getb(y, q);
    const int vq = (int)getb(T.v, q);
    uint32_t dd = delta & 3u;
    if (yq) {
        T.k += 2u * dd;
        dd = (4u - dd) & 3u;
    }
    const uint32_t e = sq_entry(vq, (int)dd);
    const uint64_t a = e & 1u, b = (e >> 1) & 1u, c = (e >> 2) & 1u;
    T.k += e >> 3;

    HRowMasks k;
    k.qs = (uint32_t)q & 31u;
    k.sh = 31u - k.qs;
    k.qh = q >= 32;
    k.first = first;
    k.qml = k.qh ? 0u : (1u << k.qs);
    k.qmh = k.qh ? (1u << k.qs) : 0u;
    k.a = (uint32_t)a;
    k.aql = a ? k.qml : 0u;
    k.aqh = a ? k.qmh : 0u;
    k.ml = (uint32_t)m; k.mh = (uint32_t)(m >> 32);
    k.m1l = (uint32_t)m1; k.m1h = (uint32_t)(m1 >> 32);
    k.mPl = first ? k.ml : 0u; k.mPh = first ? k.mh : 0u;
    k.mFl = first ? k.m1l : k.ml; k.mFh = first ? k.m1h : k.mh;
    uint64_t add2 = 0, sub1 = 0;
    R.sync();   // every lane of the term has read the rows the row pass rewrites
    // The warp skips the fan-out when no active term has one (e.g. H on |0>), and the
    // row pass altogether when no term needs R[S_q] either.
    const unsigned am = __activemask();
    if (__any_sync(am, (m | m1) != 0)) {
        if (__all_sync(am, q < 32)) {
            if (__all_sync(am, !first)) prop_h_rows<true, true, true>(R, n, k, add2, sub1);
            else prop_h_rows<true, true, false>(R, n, k, add2, sub1);
        } else {
            prop_h_rows<true, false, false>(R, n, k, add2, sub1);
        }
    } else if (__any_sync(am, a != 0)) {
        prop_h_rows<false, false, false>(R, n, k, add2, sub1);
    }
    // gamma += 2 add2, then gamma -= sub1 (bit-plane Z4 arithmetic)
    T.ghi ^= add2;
    T.ghi ^= sub1 & ~T.glo;
    T.glo ^= sub1;
    T.v = (T.v & ~bit64(q)) | (b << q);
    T.s = (y & ~bit64(q)) | (c << q);
}

// Hadamard on qubit p (Eqs. (H1)-(H7)).
template <class Rows>
__device__ __forceinline__ void gate_h(Rows& R, TermRegs& T, int n, uint64_t nmask, int p) {
    if (T.zero) return;
    const uint64_t Gp = R.G(p), Fp = R.F(p), Mp = R.M(p);
    const uint64_t nv = ~T.v & nmask;
    const uint64_t t = T.s ^ (Gp & T.v);
    const uint64_t u = T.s ^ (Fp & nv) ^ (Mp & T.v);
    const uint32_t alpha = par64(Gp & nv & T.s);
    const uint32_t beta = par64((Mp & nv & T.s) ^ (Fp & T.v & (Mp ^ T.s)));
    const uint32_t delta = (gamma_get(T, p) + 2u * (alpha + beta)) & 3u;
    T.k += 4u * alpha;
    if (t == u) {
        // 2^{-1/2}(1 + i^delta), delta odd: e^{+-i pi/4}
        T.k += (delta == 1u) ? 1u : 7u;
        T.s = t;
        return;
    }
    prop_h(R, T, n, t, u, delta);
}

// Projector (I + (-1)^sigma Z_j)/2 (Sec. 4.1, projective gates).
template <class Rows>
__device__ __forceinline__ void gate_proj(Rows& R, TermRegs& T, int n, uint64_t nmask, int j,
                                          uint32_t sigma) {
    if (T.zero) return;
    const uint64_t Gj = R.G(j);
    const uint64_t nv = ~T.v & nmask;
    const uint64_t t = T.s ^ (Gj & T.v);
    const uint32_t sg = (sigma + par64(Gj & nv & T.s)) & 1u;
    if (t == T.s) {
        if (sg) T.zero = 1u;
        return;
    }
    prop_h(R, T, n, T.s, t, 2u * sg);
    T.h += 1u;
}

// Left multiplications (Sec. 4.1 update rules).
// With several lanes per term (Rows::kStep > 1) every lane keeps the same scalars and
// only the owner of a row writes it; apply_gate starts each gate with R.sync().
template <class Rows>
__device__ __forceinline__ void gate_s(Rows& R, TermRegs& T, int q, uint32_t dg) {
    // S: dg = 3 (gamma_q -= 1); S^dagger: dg = 1; both M_q ^= G_q.
    if (R.own(q)) R.setM(q, R.M(q) ^ R.G(q));
    gamma_set(T, q, (gamma_get(T, q) + dg) & 3u);
}
template <class Rows>
__device__ __forceinline__ void gate_z(Rows& R, TermRegs& T, int q) {
    (void)R;
    T.ghi ^= bit64(q);
}
// Every row a gate reads is loaded before its first store (q != r, so no load reads a
// row the gate writes): the row accessors keep shared accesses in program order, and a
// load placed after a store would wait for the stored value's whole dependency chain.
template <class Rows>
__device__ __forceinline__ void gate_cz(Rows& R, TermRegs& T, int q, int r) {
    (void)T;
    const uint64_t Gq = R.G(q), Gr = R.G(r), Mq = R.M(q), Mr = R.M(r);
    R.sync();   // every lane has read M_q, M_r before their owners rewrite them
    if (R.own(q)) R.setM(q, Mq ^ Gr);
    if (R.own(r)) R.setM(r, Mr ^ Gq);
}
template <class Rows>
__device__ __forceinline__ void gate_cx(Rows& R, TermRegs& T, int q, int r) {
    const uint64_t Mq = R.M(q), Fr = R.F(r), Gr = R.G(r), Gq = R.G(q), Fq = R.F(q), Mr = R.M(r);
    const uint32_t g = (gamma_get(T, q) + gamma_get(T, r) + 2u * par64(Mq & Fr)) & 3u;
    gamma_set(T, q, g);
    R.sync();   // every lane has read the pre-gate rows before their owners rewrite them
    if (R.own(r)) R.setG(r, Gr ^ Gq);
    if (R.own(q)) {
        R.setF(q, Fq ^ Fr);
        R.setM(q, Mq ^ Mr);
    }
}

template <class Rows>
__device__ __forceinline__ void apply_gate(Rows& R, TermRegs& T, int n, uint64_t nmask, lrs_gate g) {
    R.sync();   // rows written by the term's other lanes in the previous gate are visible
    switch (g.op) {
        case LRS_OP_H: gate_h(R, T, n, nmask, g.q); break;
        case LRS_OP_S: gate_s(R, T, g.q, 3u); break;
        case LRS_OP_SDG: gate_s(R, T, g.q, 1u); break;
        case LRS_OP_Z: gate_z(R, T, g.q); break;
        case LRS_OP_CX: gate_cx(R, T, g.q, g.r); break;
        case LRS_OP_CZ: gate_cz(R, T, g.q, g.r); break;
        case LRS_OP_P0: gate_proj(R, T, n, nmask, g.q, 0u); break;
        case LRS_OP_P1: gate_proj(R, T, n, nmask, g.q, 1u); break;
        default: break;
    }
}

// Pauli state Q = i^mu X(u) Z(w) of a (chain, term) pair (Sec. 4.2), entry idx of
// `pairs` entries.  For n <= 40 it takes 12 bytes: the 64-bit word u | w << 40 in an
// array of pairs words, followed by an array of 32-bit words (w >> 24) | mu << 16;
// wider registers (n <= 62) take 16 bytes, (u | mu << 62, w).
__host__ __device__ constexpr bool q_compact(int n) { return n <= 40; }
__host__ __device__ constexpr size_t q_bytes(int n) { return q_compact(n) ? 12 : 16; }
template <bool CQ>
__device__ __forceinline__ void q_store(void* Q, int64_t pairs, int64_t idx, uint64_t u, uint64_t w, uint32_t mu) {
    if (CQ) {
        reinterpret_cast<uint64_t*>(Q)[idx] = u | (w << 40);
        reinterpret_cast<uint32_t*>(reinterpret_cast<uint64_t*>(Q) + pairs)[idx] =
            (uint32_t)(w >> 24) | ((mu & 3u) << 16);
    } else {
        reinterpret_cast<ulonglong2*>(Q)[idx] = make_ulonglong2(u | ((uint64_t)(mu & 3u) << 62), w);
    }
}
// Unpack from the two words (compact) or the 16-byte pair.
template <bool CQ>
__device__ __forceinline__ void q_unpack(uint64_t a, uint64_t b, uint64_t& u, uint64_t& w, uint32_t& mu) {
    if (CQ) {   // a = u | w << 40, b = (w >> 24) | mu << 16
        u = a & ((1ull << 40) - 1);
        w = (a >> 40) | ((b & 0xFFFFull) << 24);
        mu = (uint32_t)(b >> 16) & 3u;
    } else {
        u = a & ((1ull << 62) - 1);
        w = b;
        mu = (uint32_t)(a >> 62);
    }
}

__host__ __device__ __forceinline__ uint32_t omega_pack(uint32_t k, uint32_t zero, uint32_t h) {
    return (k & 7u) | ((zero & 1u) << 3) | (h << 8);
}
