// Term initialisation (exact enumeration / sparsification) and the fused
// Clifford-circuit kernel.
#include <string.h>

#include <algorithm>

#include <vector>

#include "lrs_device.cuh"

namespace {

// ---- init_terms: one thread per term ---------------------------------------------
__global__ void k_init_terms(TermsView T, int32_t mode, uint64_t seed, double scale) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= T.cap) return;
    const int n = T.n;
    // reset to |0^n>: G = F = I, M = 0, gamma = v = s = 0, omega = 1
    for (int p = 0; p < n; ++p) {
        T.F[(int64_t)p * T.cap + a] = 1ull << p;
        T.G[(int64_t)p * T.cap + a] = 1ull << p;
        T.M[(int64_t)p * T.cap + a] = 0ull;
    }
    T.glo[a] = 0; T.ghi[a] = 0; T.v[a] = 0; T.s[a] = 0;
    T.omega[a] = 0u;
    if (a >= T.chi) {  // padding term: valid state, zero weight
        for (int64_t p = 0; p < T.n_slots; ++p) T.choice[p * T.cap + a] = 0;
        T.coef[a] = make_float2(0.f, 0.f);
        return;
    }
    double bre, bim;
    if (mode == LRS_MODE_EXACT) {
        bre = 1.0; bim = 0.0;
        int64_t rem = T.alpha0 + a;
        for (int64_t p = 0; p < T.n_slots; ++p) {
            const DevSlot& S = T.slots[p];
            const int64_t r = S.n_nonzero;
            const int d = (int)(rem % r);
            rem /= r;
            const int j = S.nz_idx[d];
            T.choice[p * T.cap + a] = (uint8_t)j;
            const double xr = bre * S.c_re[j] - bim * S.c_im[j];
            const double xi = bre * S.c_im[j] + bim * S.c_re[j];
            bre = xr; bim = xi;
        }
    } else {
        bre = scale; bim = 0.0;
        const uint64_t key = sm64_key(seed, (uint64_t)(T.alpha0 + a));
        for (int64_t p = 0; p < T.n_slots; ++p) {
            const DevSlot& S = T.slots[p];
            const double u = sm64_unit(sm64_at(key, (uint64_t)p));
            int j = -1, last = 0;
            for (int c = 0; c < S.n_choices; ++c) {
                if (S.c_re[c] == 0.0 && S.c_im[c] == 0.0) continue;
                last = c;
                if (j < 0 && u < S.cdf[c]) j = c;
            }
            if (j < 0) j = last;
            T.choice[p * T.cap + a] = (uint8_t)j;
            const double xr = bre * S.ph_re[j] - bim * S.ph_im[j];
            const double xi = bre * S.ph_im[j] + bim * S.ph_re[j];
            bre = xr; bim = xi;
        }
    }
    T.coef[a] = make_float2((float)bre, (float)bim);
}

// ---- apply_clifford: TPT lanes per term, tableau rows in shared memory ------------
// Shared layout [row][term] makes every per-lane row index conflict-free.  For
// n <= 48 a row is kept as its low 32 bits plus its next HB bits (0, 8 or 16; bits at
// or above n are zero in every row): a 40-qubit tableau takes 15n bytes per term
// instead of 24n, so five 64-term blocks fit on an SM instead of three.  Wider
// tableaux keep each row as one 64-bit word (HB = 64): at n = 50 one 64-bit access
// per row beats a 16 + 8-bit split of the high word (three accesses per row for the
// same three blocks per SM).
// The Hadamard row pass reads F and G through per-term pointers; the narrow high rows
// of G and M are padded so that a warp reading row p of F for some terms and of G for
// others hits other banks.
// A block holds APPLY_TERMS terms.  With TPT lanes per term (the wide layout), the
// lanes of a term sit 32/TPT apart in one warp, keep identical scalars (gamma, v, s,
// omega) and split the rows: lane `part` owns the rows p = part (mod TPT), loads,
// stores and rewrites only those, and the Hadamard / projector row pass -- the bulk of
// the work -- runs on each lane's own rows; the column-q parities of the row pass are
// merged with shuffles.  A term's tableau stays in shared memory, so the split gives
// TPT times the warps per SM (latency hiding) at the same shared-memory footprint.
constexpr int APPLY_TERMS = 64;
// Launch-internal gate codes (never in the public gate lists): a slot whose choice 0 is
// the identity and whose choice 1 is one S (S^dagger) on q -- every T and RZ slot of the
// lowering -- so that a term needs its choice byte only, not the slot table and K-gate
// list behind it (two dependent global loads fewer per slot).
constexpr uint8_t APPLY_OP_SLOT_S = 16, APPLY_OP_SLOT_SDG = 17;

template <int HB> struct HiWord { typedef uint32_t T; };
template <> struct HiWord<8> { typedef uint8_t T; };
template <> struct HiWord<16> { typedef uint16_t T; };

// Elements of padding after the F rows of an array of esz-byte entries, so that
// row p of G starts 16 banks away from row p of F (the warp's entries of one row
// cover at most 16 banks when esz < 4; 4-byte entries are conflict-free anyway).
__host__ __device__ __forceinline__ int rows_pad(int n, int esz) {
    if (esz >= 4) return 0;
    const int offw = (n * APPLY_TERMS * esz / 4) & 31;
    return ((16 - offw) & 31) * 4 / esz;
}

// The lanes of one term: TPT lanes 32/TPT apart; `part` selects the owned rows.
template <int TPT>
struct TermLanes {
    static constexpr int kStep = TPT;
    int part_, col_;
    unsigned mask_;
    __device__ __forceinline__ TermLanes() {
        const int lane = threadIdx.x & 31, span = 32 / TPT;
        part_ = lane / span;
        col_ = (int)(threadIdx.x >> 5) * span + lane % span;
        unsigned m = 0;
#pragma unroll
        for (int i = 0; i < TPT; ++i) m |= 1u << (lane % span + i * span);
        mask_ = m;
    }
    __device__ __forceinline__ int part() const { return TPT == 1 ? 0 : part_; }
    __device__ __forceinline__ int col() const { return col_; }
    __device__ __forceinline__ bool own(int p) const { return TPT == 1 || (p & (TPT - 1)) == part_; }
    __device__ __forceinline__ void sync() const {
        if (TPT > 1) __syncwarp(mask_);
    }
    // OR over the term's lanes (their row bits are disjoint)
    __device__ __forceinline__ uint64_t combine(uint64_t v) const {
#pragma unroll
        for (int off = 32 / TPT; off < 32; off <<= 1) v |= __shfl_xor_sync(mask_, v, off);
        return v;
    }
};

template <int HB, int TPT = 1>
struct SmemRows : TermLanes<TPT> {
    static_assert(TPT == 1, "narrow row layouts take one lane per term");
    typedef typename HiWord<HB>::T Hi;
    static constexpr int kRowUnroll = 4;   // rows per load group of the Hadamard row pass
    struct Mat {
        uint32_t* lo;
        Hi* hi;
    };
    Mat f, g, m;
    __device__ __forceinline__ SmemRows(uint64_t* smem, int n) {
        const int rows = 3 * n * APPLY_TERMS;
        const int hp = HB > 0 ? rows_pad(n, (int)sizeof(Hi)) : 0;
        uint32_t* lo = reinterpret_cast<uint32_t*>(smem) + this->col();
        Hi* hi = reinterpret_cast<Hi*>(reinterpret_cast<uint32_t*>(smem) + rows) + this->col();
        f = Mat{lo, hi};
        g = Mat{lo + n * APPLY_TERMS, hi + n * APPLY_TERMS + hp};
        m = Mat{lo + 2 * n * APPLY_TERMS, hi + 2 * n * APPLY_TERMS + hp};
    }
    __device__ __forceinline__ uint64_t get(const Mat& x, int p) const {
        uint64_t v = x.lo[p * APPLY_TERMS];
        if (HB > 0) v |= (uint64_t)x.hi[p * APPLY_TERMS] << 32;
        return v;
    }
    __device__ __forceinline__ void set(const Mat& x, int p, uint64_t v) {
        x.lo[p * APPLY_TERMS] = (uint32_t)v;
        if (HB > 0) x.hi[p * APPLY_TERMS] = (Hi)(v >> 32);
    }
    __device__ __forceinline__ Mat matF() const { return f; }
    __device__ __forceinline__ Mat matG() const { return g; }
    __device__ __forceinline__ Mat matM() const { return m; }
    __device__ __forceinline__ uint64_t F(int p) const { return get(f, p); }
    __device__ __forceinline__ uint64_t G(int p) const { return get(g, p); }
    __device__ __forceinline__ uint64_t M(int p) const { return get(m, p); }
    __device__ __forceinline__ void setF(int p, uint64_t x) { set(f, p, x); }
    __device__ __forceinline__ void setG(int p, uint64_t x) { set(g, p, x); }
    __device__ __forceinline__ void setM(int p, uint64_t x) { set(m, p, x); }
    static size_t bytes(int n) {
        const size_t rows = (size_t)3 * n * APPLY_TERMS;
        size_t b = rows * 4;
        if (HB > 0) b += (rows + rows_pad(n, (int)sizeof(Hi))) * sizeof(Hi);
        return b;
    }
};

// Rows kept whole as one 64-bit word ([row][term], one 64-bit shared access each),
// addressed by 32-bit shared-space addresses with explicit shared loads and stores
// (4% faster at n = 50 than generic pointers).  A warp's access to one row of 32 / TPT
// terms for each of its TPT row sets is 256 bytes in two wavefronts, as for one row
// of 32 terms.
template <int TPT>
struct SmemRows<64, TPT> : TermLanes<TPT> {
    static constexpr int kRowUnroll = 4;   // rows per load group (2, 3, 6 and 8 measured slower)
    struct Mat {
        uint32_t a;
    };
    Mat f, g, m;
    __device__ __forceinline__ SmemRows(uint64_t* smem, int n) {
        const uint32_t b = (uint32_t)__cvta_generic_to_shared(smem + this->col());
        f = Mat{b};
        g = Mat{b + (uint32_t)(n * APPLY_TERMS * 8)};
        m = Mat{b + (uint32_t)(2 * n * APPLY_TERMS * 8)};
    }
    __device__ __forceinline__ uint64_t get(const Mat& x, int p) const {
        uint32_t lo, hi;
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(lo), "=r"(hi) : "r"(x.a + (uint32_t)(p * APPLY_TERMS * 8))
                     : "memory");
        return ((uint64_t)hi << 32) | lo;
    }
    __device__ __forceinline__ void set(const Mat& x, int p, uint64_t v) {
        asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(x.a + (uint32_t)(p * APPLY_TERMS * 8)), "r"((uint32_t)v),
                     "r"((uint32_t)(v >> 32))
                     : "memory");
    }
    __device__ __forceinline__ Mat matF() const { return f; }
    __device__ __forceinline__ Mat matG() const { return g; }
    __device__ __forceinline__ Mat matM() const { return m; }
    __device__ __forceinline__ uint64_t F(int p) const { return get(f, p); }
    __device__ __forceinline__ uint64_t G(int p) const { return get(g, p); }
    __device__ __forceinline__ uint64_t M(int p) const { return get(m, p); }
    __device__ __forceinline__ void setF(int p, uint64_t x) { set(f, p, x); }
    __device__ __forceinline__ void setG(int p, uint64_t x) { set(g, p, x); }
    __device__ __forceinline__ void setM(int p, uint64_t x) { set(m, p, x); }
    static size_t bytes(int n) { return (size_t)3 * n * APPLY_TERMS * 8; }
};

// Row layout for n qubits.
inline int apply_hb(int n) { return n <= 32 ? 0 : n <= 40 ? 8 : n <= 48 ? 16 : 64; }

// One tile of APPLY_TERMS terms through the whole gate list.
template <int HB, int TPT, class Gates>
__device__ __forceinline__ void apply_tile(const TermsView T, const Gates gates, int64_t n_gates, int64_t tile,
                                           uint64_t* smem) {
    const int n = T.n;
    SmemRows<HB, TPT> R(smem, n);
    const int64_t a = tile * APPLY_TERMS + R.col();   // cap % APPLY_TERMS == 0
    for (int p = R.part(); p < n; p += TPT) {
        R.setF(p, T.F[(int64_t)p * T.cap + a]);
        R.setG(p, T.G[(int64_t)p * T.cap + a]);
        R.setM(p, T.M[(int64_t)p * T.cap + a]);
    }
    TermRegs S;
    S.glo = T.glo[a]; S.ghi = T.ghi[a]; S.v = T.v[a]; S.s = T.s[a];
    const uint32_t om = T.omega[a];
    S.k = om & 7u; S.zero = (om >> 3) & 1u; S.h = om >> 8;
    const uint64_t nmask = T.nmask;
    for (int64_t i = 0; i < n_gates; ++i) {
        const lrs_gate g = gates[i];
        if (g.op == LRS_OP_SLOT) {
            const DevSlot& sl = T.slots[g.r];
            const int j = T.choice[(int64_t)g.r * T.cap + a];
            const int off = sl.k_off[j], len = sl.k_len[j];
            for (int e = 0; e < len; ++e) apply_gate(R, S, n, nmask, T.kgates[off + e]);
        } else if (g.op == APPLY_OP_SLOT_S || g.op == APPLY_OP_SLOT_SDG) {
            // two-choice slot K_0 = I, K_1 = S (or S^dagger) on q: one choice load
            R.sync();
            if (T.choice[(int64_t)g.r * T.cap + a] != 0) gate_s(R, S, g.q, g.op == APPLY_OP_SLOT_S ? 3u : 1u);
        } else {
            apply_gate(R, S, n, nmask, g);
        }
    }
    R.sync();
    for (int p = R.part(); p < n; p += TPT) {   // a lane's own rows were last written by it
        T.F[(int64_t)p * T.cap + a] = R.F(p);
        T.G[(int64_t)p * T.cap + a] = R.G(p);
        T.M[(int64_t)p * T.cap + a] = R.M(p);
    }
    if (R.part() == 0) {
        T.glo[a] = S.glo; T.ghi[a] = S.ghi; T.v[a] = S.v; T.s[a] = S.s;
        T.omega[a] = omega_pack(S.k, S.zero, S.h);
    }
}

// The gate list of one launch is a kernel parameter (at most APPLY_PARAM_GATES gates;
// longer lists take several launches): every thread reads the same gate, which the
// parameter space serves from the constant cache without a global-memory round trip.
constexpr int APPLY_PARAM_GATES = 7680;
struct GateList {
    lrs_gate g[APPLY_PARAM_GATES];
};
struct GatesParam {
    const GateList* p;
    __device__ __forceinline__ lrs_gate operator[](int64_t i) const { return p->g[i]; }
};
struct GatesGlobal {
    const lrs_gate* __restrict__ p;
    __device__ __forceinline__ lrs_gate operator[](int64_t i) const { return p[i]; }
};

template <int HB, int TPT>
__global__ void __launch_bounds__(APPLY_TERMS * TPT) k_apply_clifford(TermsView T, const __grid_constant__ GateList G,
                                                                      int n_gates) {
    extern __shared__ uint64_t smem[];
    apply_tile<HB, TPT>(T, GatesParam{&G}, n_gates, blockIdx.x, smem);
}

// Several circuits of uneven chi in one launch: block b runs global tile b; the
// circuit table is a kernel parameter, so the circuit lookup and every value read
// from it are warp-uniform (as in the single-circuit kernel).  The hardware block
// scheduler balances the uneven circuits.
#define LRS_APPLY_BATCH_MAX 12
struct ApplyBatch {
    int count;
    int64_t first_tile[LRS_APPLY_BATCH_MAX + 1];
    TermsView T[LRS_APPLY_BATCH_MAX];
    const lrs_gate* gates[LRS_APPLY_BATCH_MAX];
    int64_t n_gates[LRS_APPLY_BATCH_MAX];
};

template <int HB, int TPT>
__global__ void __maxnreg__(168)
    k_apply_clifford_batch(const __grid_constant__ ApplyBatch B) {
    extern __shared__ uint64_t smem[];
    const int64_t tile = blockIdx.x;
    int c = 0;
#pragma unroll 1
    for (int i = 1; i < B.count; ++i)
        if (B.first_tile[i] <= tile) c = i;
    apply_tile<HB, TPT>(B.T[c], GatesGlobal{B.gates[c]}, B.n_gates[c], tile - B.first_tile[c], smem);
}

// ---- sample x from single terms (Sec. 4.1, "Simulating measurements") --------------
__global__ void k_sample_terms(TermsView T, int64_t count, uint64_t seed, uint64_t* x_out,
                               int64_t* alpha_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint64_t key = sm64_key(seed, (uint64_t)i);
    const uint64_t r0 = sm64_at(key, 0), r1 = sm64_at(key, 1);
    const int64_t a = (int64_t)__umul64hi(r0, (uint64_t)T.chi);
    const uint64_t w = T.s[a] ^ (r1 & T.v[a]);
    uint64_t x = 0;
    for (int j = 0; j < T.n; ++j) x |= (uint64_t)par64(w & T.G[(int64_t)j * T.cap + a]) << j;
    x_out[i] = x;
    if (alpha_out) alpha_out[i] = a;
}

// Prefix sharing: terms [R, Rn) become copies of term (alpha mod R) -- the state of
// their common choice prefix (exact mode, slot 0 the least significant digit).
__global__ void k_expand_terms(TermsView T, int64_t R, int64_t Rn) {
    const int64_t a = R + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= Rn) return;
    const int64_t src = a % R;
    for (int p = 0; p < T.n; ++p) {
        T.F[(int64_t)p * T.cap + a] = T.F[(int64_t)p * T.cap + src];
        T.G[(int64_t)p * T.cap + a] = T.G[(int64_t)p * T.cap + src];
        T.M[(int64_t)p * T.cap + a] = T.M[(int64_t)p * T.cap + src];
    }
    T.glo[a] = T.glo[src]; T.ghi[a] = T.ghi[src];
    T.v[a] = T.v[src]; T.s[a] = T.s[src];
    T.omega[a] = T.omega[src];
}

}  // namespace

lrs_status launch_expand_terms(lrs_ctx* ctx, int64_t R, int64_t Rn, cudaStream_t st) {
    if (Rn <= R) return LRS_OK;
    const int tpb = 256;
    k_expand_terms<<<(unsigned)((Rn - R + tpb - 1) / tpb), tpb, 0, st>>>(ctx->view(), R, Rn);
    LRS_LAUNCH_CHECK("expand terms kernel");
    return LRS_OK;
}

lrs_status launch_init_terms(lrs_ctx* ctx, int32_t mode, uint64_t seed, double scale,
                             cudaStream_t st) {
    const int tpb = 256;
    const int64_t blocks = (ctx->cap + tpb - 1) / tpb;
    k_init_terms<<<(unsigned)blocks, tpb, 0, st>>>(ctx->view(), mode, seed, scale);
    LRS_LAUNCH_CHECK("init_terms kernel");
    return LRS_OK;
}

lrs_status launch_apply_clifford(lrs_ctx* ctx, const lrs_gate* gates_host, int64_t n_gates, cudaStream_t st) {
    return launch_apply_clifford_range(ctx, gates_host, n_gates, ctx->cap, st);
}

// The launch-internal code of gate g (APPLY_OP_SLOT_S / _SDG for a slot of the form
// {I, S_q} or {I, S^dagger_q} with both coefficients nonzero; g itself otherwise).
static lrs_gate specialise_gate(const lrs_ctx* ctx, lrs_gate g) {
    if (g.op != LRS_OP_SLOT || (size_t)g.r >= ctx->slots_host.size()) return g;
    const lrs_slot& sl = ctx->slots_host[g.r];
    if (sl.n_choices != 2 || sl.k_len[0] != 0 || sl.k_len[1] != 1) return g;
    if ((sl.c_re[0] == 0.0 && sl.c_im[0] == 0.0) || (sl.c_re[1] == 0.0 && sl.c_im[1] == 0.0)) return g;
    const lrs_gate k = ctx->kgates_host[(size_t)sl.k_off[1]];
    if (k.op != LRS_OP_S && k.op != LRS_OP_SDG) return g;
    lrs_gate o;
    o.op = k.op == LRS_OP_S ? APPLY_OP_SLOT_S : APPLY_OP_SLOT_SDG;
    o.q = k.q;
    o.r = g.r;
    return o;
}

void specialise_gates(const lrs_ctx* ctx, const lrs_gate* in, int64_t n, lrs_gate* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = specialise_gate(ctx, in[i]);
}

template <int HB, int TPT>
static lrs_status launch_apply_hb(lrs_ctx* ctx, const lrs_gate* gates_host, int64_t n_gates, int64_t blocks,
                                  cudaStream_t st) {
    if (!lrs_capturing(st))
        LRS_CUDA(cudaFuncSetAttribute(k_apply_clifford<HB, TPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)SmemRows<HB, TPT>::bytes(64)));
    static thread_local GateList G;
    for (int64_t i0 = 0; i0 < n_gates; i0 += APPLY_PARAM_GATES) {
        const int len = (int)std::min<int64_t>(APPLY_PARAM_GATES, n_gates - i0);
        specialise_gates(ctx, gates_host + i0, len, G.g);
        k_apply_clifford<HB, TPT><<<(unsigned)blocks, APPLY_TERMS * TPT, SmemRows<HB, TPT>::bytes(ctx->n), st>>>(
            ctx->view(), G, len);
        LRS_LAUNCH_CHECK("apply_clifford kernel");
    }
    return LRS_OK;
}

// The gate list (host memory, read before return) on the terms of the first
// ceil(n_terms / APPLY_TERMS) tiles only.
lrs_status launch_apply_clifford_range(lrs_ctx* ctx, const lrs_gate* gates_host, int64_t n_gates, int64_t n_terms,
                                       cudaStream_t st) {
    if (n_terms > ctx->cap) n_terms = ctx->cap;
    const int64_t blocks = (n_terms + APPLY_TERMS - 1) / APPLY_TERMS;
    if (blocks == 0 || n_gates == 0) return LRS_OK;
    switch (apply_hb(ctx->n)) {
        case 0: return launch_apply_hb<0, 1>(ctx, gates_host, n_gates, blocks, st);
        case 8: return launch_apply_hb<8, 1>(ctx, gates_host, n_gates, blocks, st);
        case 16: return launch_apply_hb<16, 1>(ctx, gates_host, n_gates, blocks, st);
        default:
            switch (ctx->tune_apply_lanes) {
                case 1: return launch_apply_hb<64, 1>(ctx, gates_host, n_gates, blocks, st);
                case 4: return launch_apply_hb<64, 4>(ctx, gates_host, n_gates, blocks, st);
                default: return launch_apply_hb<64, 2>(ctx, gates_host, n_gates, blocks, st);
            }
    }
}

lrs_status launch_sample_terms(lrs_ctx* ctx, int64_t count, uint64_t seed, uint64_t* x,
                               int64_t* alpha, cudaStream_t st) {
    if (count == 0) return LRS_OK;
    const int tpb = 128;
    k_sample_terms<<<(unsigned)((count + tpb - 1) / tpb), tpb, 0, st>>>(ctx->view(), count, seed, x,
                                                                        alpha);
    LRS_LAUNCH_CHECK("sample_terms kernel");
    return LRS_OK;
}

// The circuits of one batch share the layout of the widest one (a narrower tableau
// keeps zero high bits) and the lane split of the first context.
template <int HB, int TPT>
static lrs_status launch_apply_batch_hb(const ApplyBatch& B, int64_t tiles, int nmax, cudaStream_t st) {
    if (!lrs_capturing(st))
        LRS_CUDA(cudaFuncSetAttribute(k_apply_clifford_batch<HB, TPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)SmemRows<HB, TPT>::bytes(64)));
    k_apply_clifford_batch<HB, TPT><<<(unsigned)tiles, APPLY_TERMS * TPT, SmemRows<HB, TPT>::bytes(nmax), st>>>(B);
    LRS_LAUNCH_CHECK("batched apply_clifford kernel");
    return LRS_OK;
}

lrs_status launch_apply_clifford_batch(lrs_ctx* const* ctxs, int32_t count, cudaStream_t st,
                                       void** dev_buf, size_t* dev_buf_bytes) {
    (void)dev_buf;
    (void)dev_buf_bytes;
    for (int32_t base = 0; base < count; base += LRS_APPLY_BATCH_MAX) {
        ApplyBatch B;
        memset(&B, 0, sizeof(B));
        B.count = (count - base < LRS_APPLY_BATCH_MAX) ? count - base : LRS_APPLY_BATCH_MAX;
        int64_t tiles = 0;
        int nmax = 1;
        for (int i = 0; i < B.count; ++i) {
            const lrs_ctx* c = ctxs[base + i];
            B.T[i] = c->view();
            B.gates[i] = c->gates_dev;
            B.n_gates[i] = c->batch_n_gates;
            B.first_tile[i] = tiles;
            tiles += c->cap / APPLY_TERMS;
            if (c->n > nmax) nmax = c->n;
        }
        B.first_tile[B.count] = tiles;
        lrs_status rc;
        switch (apply_hb(nmax)) {
            case 0: rc = launch_apply_batch_hb<0, 1>(B, tiles, nmax, st); break;
            case 8: rc = launch_apply_batch_hb<8, 1>(B, tiles, nmax, st); break;
            case 16: rc = launch_apply_batch_hb<16, 1>(B, tiles, nmax, st); break;
            default:
                switch (ctxs[base]->tune_apply_lanes) {
                    case 1: rc = launch_apply_batch_hb<64, 1>(B, tiles, nmax, st); break;
                    case 4: rc = launch_apply_batch_hb<64, 4>(B, tiles, nmax, st); break;
                    default: rc = launch_apply_batch_hb<64, 2>(B, tiles, nmax, st); break;
                }
        }
        if (rc != LRS_OK) return rc;
    }
    return LRS_OK;
}
