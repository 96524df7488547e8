// Host side of the C ABI: argument checks, storage, slot tables, lowering.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "lrs_device.cuh"
#include "lrs_internal.h"

static thread_local char g_err[512] = "";

lrs_status lrs_fail(lrs_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

lrs_status lrs_cuda_check(cudaError_t e, const char* what) {
    return lrs_fail(e == cudaErrorMemoryAllocation ? LRS_ERR_OOM : LRS_ERR_CUDA, "%s: %s", what,
                    cudaGetErrorString(e));
}

extern "C" const char* lrs_last_error(void) { return g_err; }

lrs_status lrs_ensure(void** ptr, size_t* have, size_t bytes) {
    if (*have >= bytes && *ptr) return LRS_OK;
    if (*ptr) {
        cudaFree(*ptr);
        *ptr = nullptr;
        *have = 0;
    }
    if (bytes == 0) return LRS_OK;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return lrs_cuda_check(e, "cudaMalloc");
    }
    *have = bytes;
    return LRS_OK;
}

lrs_status lrs_scratch(lrs_ctx* ctx, size_t bytes, void** out) {
    lrs_status rc = lrs_ensure(&ctx->scratch, &ctx->scratch_bytes, bytes);
    *out = ctx->scratch;
    return rc;
}

static cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

bool lrs_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();   // the query's own error is not the next launch's
        return false;
    }
    return cs == cudaStreamCaptureStatusActive;
}

// ---------------------------------------------------------------------------------
// Lowering (Sec. 2.3.2): T and RZ(theta) -> 2-term slot (Eq. (Rtheta)); CCZ ->
// projector form I - 2 P1 P1 P1, or the 8-term form of Eq. (CCZ_decomposition)
// with prefactor 1/6.
// ---------------------------------------------------------------------------------
namespace {
struct Lowering {
    std::vector<lrs_gate> gates;
    std::vector<lrs_slot> slots;
    std::vector<lrs_gate> kg;
    void add_choice(lrs_slot& s, double re, double im, std::initializer_list<lrs_gate> k) {
        const int j = s.n_choices++;
        s.c_re[j] = re;
        s.c_im[j] = im;
        s.k_off[j] = (int32_t)kg.size();
        s.k_len[j] = (int32_t)k.size();
        for (const lrs_gate& g : k) kg.push_back(g);
    }
};
lrs_gate mk(int op, int q, int r = 0) {
    lrs_gate g;
    g.op = (uint8_t)op;
    g.q = (uint8_t)q;
    g.r = (uint16_t)r;
    return g;
}
}  // namespace

// The sum-over-Cliffords slot of one non-Clifford op acting on qubits q[0..t) (the
// op's own qubits, or its gadget's ancillas), every coefficient times `scale`.
static void push_slot(Lowering& L, const lrs_circuit_op& o, const int* q, int32_t ccz_mode, double scale) {
    lrs_slot s;
    memset(&s, 0, sizeof(s));
    if (o.kind == LRS_C_T || o.kind == LRS_C_RZ) {
        // R(theta) = (cos(th/2) - sin(th/2)) I + sqrt2 e^{-i pi/4} sin(th/2) S, th >= 0;
        // conjugate on (I, S^dagger) for theta < 0.  T = e^{i pi/8} R(pi/4).
        const double theta = (o.kind == LRS_C_T) ? M_PI / 4 : o.theta;
        const double th = fabs(theta);
        const double c0 = cos(th / 2) - sin(th / 2);
        const double sn = sin(th / 2);
        // sqrt2 e^{-i pi/4} = 1 - i
        const double c1re = sn, c1im = (theta >= 0) ? -sn : sn;
        double g_re = 1.0, g_im = 0.0;
        if (o.kind == LRS_C_T) { g_re = cos(M_PI / 8); g_im = sin(M_PI / 8); }
        L.add_choice(s, scale * (g_re * c0), scale * (g_im * c0), {});
        L.add_choice(s, scale * (g_re * c1re - g_im * c1im), scale * (g_re * c1im + g_im * c1re),
                     {mk(theta >= 0 ? LRS_OP_S : LRS_OP_SDG, q[0])});
    } else {
        const int a = q[0], b = q[1], c = q[2];
        if (ccz_mode == LRS_CCZ_PROJECTOR) {
            L.add_choice(s, scale * 1.0, 0.0, {});
            L.add_choice(s, scale * -2.0, 0.0, {mk(LRS_OP_P1, a), mk(LRS_OP_P1, b), mk(LRS_OP_P1, c)});
        } else {
            const double w = scale * (1.0 / 6.0);
            L.add_choice(s, w, 0, {});
            L.add_choice(s, w, 0, {mk(LRS_OP_CZ, a, b)});
            L.add_choice(s, w, 0, {mk(LRS_OP_CZ, a, c)});
            L.add_choice(s, w, 0, {mk(LRS_OP_CZ, b, c)});
            L.add_choice(s, w, 0, {mk(LRS_OP_CZ, a, b), mk(LRS_OP_CZ, a, c), mk(LRS_OP_Z, a)});
            L.add_choice(s, w, 0, {mk(LRS_OP_CZ, a, b), mk(LRS_OP_CZ, b, c), mk(LRS_OP_Z, b)});
            L.add_choice(s, w, 0, {mk(LRS_OP_CZ, a, c), mk(LRS_OP_CZ, b, c), mk(LRS_OP_Z, c)});
            L.add_choice(s, -w, 0,
                         {mk(LRS_OP_CZ, a, b), mk(LRS_OP_CZ, a, c), mk(LRS_OP_CZ, b, c), mk(LRS_OP_Z, a),
                          mk(LRS_OP_Z, b), mk(LRS_OP_Z, c)});
        }
    }
    L.gates.push_back(mk(LRS_OP_SLOT, 0, (int)L.slots.size()));
    L.slots.push_back(s);
}

static lrs_status check_ops(int32_t n, const lrs_circuit_op* ops, int64_t n_ops) {
    if (n < 1 || n > 64) return lrs_fail(LRS_ERR_ARG, "n_qubits must be in 1..64 (got %d)", n);
    if (n_ops < 0 || (n_ops > 0 && !ops)) return lrs_fail(LRS_ERR_ARG, "bad ops array");
    for (int64_t i = 0; i < n_ops; ++i) {
        const lrs_circuit_op& o = ops[i];
        if (o.kind < LRS_C_H || o.kind > LRS_C_CCZ)
            return lrs_fail(LRS_ERR_ARG, "op %lld: unknown kind %d", (long long)i, o.kind);
        const int nq = (o.kind == LRS_C_CX || o.kind == LRS_C_CZ) ? 2 : (o.kind == LRS_C_CCZ ? 3 : 1);
        for (int t = 0; t < nq; ++t) {
            if (o.q[t] < 0 || o.q[t] >= n)
                return lrs_fail(LRS_ERR_ARG, "op %lld: qubit %d out of range", (long long)i, o.q[t]);
            for (int t2 = 0; t2 < t; ++t2)
                if (o.q[t] == o.q[t2])
                    return lrs_fail(LRS_ERR_ARG, "op %lld: repeated qubit %d", (long long)i, o.q[t]);
        }
    }
    return LRS_OK;
}

static lrs_status emit(const Lowering& L, lrs_gate* gates, int64_t gates_cap, int64_t* n_gates, lrs_slot* slots,
                       int64_t slots_cap, int64_t* n_slots, lrs_gate* k_gates, int64_t k_cap, int64_t* n_k_gates) {
    if (L.slots.size() > 65535) return lrs_fail(LRS_ERR_ARG, "more than 65535 slots");
    if (n_gates) *n_gates = (int64_t)L.gates.size();
    if (n_slots) *n_slots = (int64_t)L.slots.size();
    if (n_k_gates) *n_k_gates = (int64_t)L.kg.size();
    if ((int64_t)L.gates.size() > gates_cap || (int64_t)L.slots.size() > slots_cap ||
        (int64_t)L.kg.size() > k_cap)
        return lrs_fail(LRS_ERR_ARG, "output capacity too small (need %zu gates, %zu slots, %zu k_gates)",
                        L.gates.size(), L.slots.size(), L.kg.size());
    if (!L.gates.empty()) memcpy(gates, L.gates.data(), L.gates.size() * sizeof(lrs_gate));
    if (!L.slots.empty()) memcpy(slots, L.slots.data(), L.slots.size() * sizeof(lrs_slot));
    if (!L.kg.empty()) memcpy(k_gates, L.kg.data(), L.kg.size() * sizeof(lrs_gate));
    return LRS_OK;
}

extern "C" lrs_status lrs_lower_gadget(int32_t n, const lrs_circuit_op* ops, int64_t n_ops, int32_t ccz_mode,
                                       int32_t* n_total, lrs_gate* gates, int64_t gates_cap, int64_t* n_gates,
                                       lrs_slot* slots, int64_t slots_cap, int64_t* n_slots, lrs_gate* k_gates,
                                       int64_t k_cap, int64_t* n_k_gates) {
    lrs_status rc = check_ops(n, ops, n_ops);
    if (rc != LRS_OK) return rc;
    if (ccz_mode != LRS_CCZ_PROJECTOR && ccz_mode != LRS_CCZ_SUM8)
        return lrs_fail(LRS_ERR_ARG, "unknown ccz_mode %d", ccz_mode);
    // ancillas from qubit n on, in the order of the non-Clifford ops
    int64_t tau = 0;
    for (int64_t i = 0; i < n_ops; ++i)
        tau += ops[i].kind == LRS_C_CCZ ? 3 : ((ops[i].kind == LRS_C_T || ops[i].kind == LRS_C_RZ) ? 1 : 0);
    if (n + tau > 64)
        return lrs_fail(LRS_ERR_ARG, "gadget form needs %lld qubits (more than 64)", (long long)(n + tau));
    if (n_total) *n_total = (int32_t)(n + tau);
    Lowering L;
    // magic states |V_j> = V_j |+^t>: H on the ancillas, then V_j's slot on them with its
    // coefficients times 2^{t/2} (the post-selection renormalisation of Eq. (Uidentity))
    int a = n;
    for (int64_t i = 0; i < n_ops; ++i) {
        const lrs_circuit_op& o = ops[i];
        const int t = o.kind == LRS_C_CCZ ? 3 : ((o.kind == LRS_C_T || o.kind == LRS_C_RZ) ? 1 : 0);
        if (t == 0) continue;
        const int anc[3] = {a, a + 1, a + 2};
        for (int k = 0; k < t; ++k) L.gates.push_back(mk(LRS_OP_H, anc[k]));
        push_slot(L, o, anc, ccz_mode, (t == 1) ? sqrt(2.0) : 2.0 * sqrt(2.0));
        a += t;
    }
    // the circuit with V_j replaced by CX(q_k, a_k), then post-selection on 0^tau
    a = n;
    for (int64_t i = 0; i < n_ops; ++i) {
        const lrs_circuit_op& o = ops[i];
        switch (o.kind) {
            case LRS_C_H: L.gates.push_back(mk(LRS_OP_H, o.q[0])); break;
            case LRS_C_S: L.gates.push_back(mk(LRS_OP_S, o.q[0])); break;
            case LRS_C_SDG: L.gates.push_back(mk(LRS_OP_SDG, o.q[0])); break;
            case LRS_C_Z: L.gates.push_back(mk(LRS_OP_Z, o.q[0])); break;
            case LRS_C_CX: L.gates.push_back(mk(LRS_OP_CX, o.q[0], o.q[1])); break;
            case LRS_C_CZ: L.gates.push_back(mk(LRS_OP_CZ, o.q[0], o.q[1])); break;
            case LRS_C_T:
            case LRS_C_RZ: L.gates.push_back(mk(LRS_OP_CX, o.q[0], a)); a += 1; break;
            case LRS_C_CCZ:
                for (int k = 0; k < 3; ++k) L.gates.push_back(mk(LRS_OP_CX, o.q[k], a + k));
                a += 3;
                break;
        }
    }
    for (int q = n; q < a; ++q) L.gates.push_back(mk(LRS_OP_P0, q));
    return emit(L, gates, gates_cap, n_gates, slots, slots_cap, n_slots, k_gates, k_cap, n_k_gates);
}

extern "C" lrs_status lrs_lower_circuit(int32_t n, const lrs_circuit_op* ops, int64_t n_ops,
                                        int32_t ccz_mode, lrs_gate* gates, int64_t gates_cap,
                                        int64_t* n_gates, lrs_slot* slots, int64_t slots_cap,
                                        int64_t* n_slots, lrs_gate* k_gates, int64_t k_cap,
                                        int64_t* n_k_gates) {
    lrs_status rc = check_ops(n, ops, n_ops);
    if (rc != LRS_OK) return rc;
    if (ccz_mode != LRS_CCZ_PROJECTOR && ccz_mode != LRS_CCZ_SUM8)
        return lrs_fail(LRS_ERR_ARG, "unknown ccz_mode %d", ccz_mode);
    Lowering L;
    for (int64_t i = 0; i < n_ops; ++i) {
        const lrs_circuit_op& o = ops[i];
        switch (o.kind) {
            case LRS_C_H: L.gates.push_back(mk(LRS_OP_H, o.q[0])); break;
            case LRS_C_S: L.gates.push_back(mk(LRS_OP_S, o.q[0])); break;
            case LRS_C_SDG: L.gates.push_back(mk(LRS_OP_SDG, o.q[0])); break;
            case LRS_C_Z: L.gates.push_back(mk(LRS_OP_Z, o.q[0])); break;
            case LRS_C_CX: L.gates.push_back(mk(LRS_OP_CX, o.q[0], o.q[1])); break;
            case LRS_C_CZ: L.gates.push_back(mk(LRS_OP_CZ, o.q[0], o.q[1])); break;
            default: {
                const int q[3] = {o.q[0], o.q[1], o.q[2]};
                push_slot(L, o, q, ccz_mode, 1.0);
                break;
            }
        }
        if (L.slots.size() > 65535) return lrs_fail(LRS_ERR_ARG, "more than 65535 slots");
    }
    return emit(L, gates, gates_cap, n_gates, slots, slots_cap, n_slots, k_gates, k_cap, n_k_gates);
}

extern "C" lrs_status lrs_decomposition_stats(const lrs_slot* slots, int64_t n_slots, double* l1_norm,
                                              int64_t* exact_chi, double* log2_exact_chi) {
    if (n_slots < 0 || (n_slots > 0 && !slots)) return lrs_fail(LRS_ERR_ARG, "bad slot table");
    double l1 = 1.0, lg = 0.0;
    bool fits = true;
    int64_t chi = 1;
    for (int64_t p = 0; p < n_slots; ++p) {
        const lrs_slot& sl = slots[p];
        if (sl.n_choices < 1 || sl.n_choices > LRS_MAX_CHOICES)
            return lrs_fail(LRS_ERR_ARG, "slot %lld: n_choices %d", (long long)p, sl.n_choices);
        double norm = 0.0;
        int64_t nz = 0;
        for (int j = 0; j < sl.n_choices; ++j) {
            norm += hypot(sl.c_re[j], sl.c_im[j]);
            nz += (sl.c_re[j] != 0.0 || sl.c_im[j] != 0.0) ? 1 : 0;
        }
        l1 *= norm;
        lg += log2((double)(nz > 0 ? nz : 1));
        if (nz == 0) chi = 0;
        else if (fits && chi > ((int64_t)1 << 62) / nz) fits = false;
        else if (fits) chi *= nz;
    }
    if (l1_norm) *l1_norm = l1;
    if (exact_chi) *exact_chi = fits ? chi : -1;
    if (log2_exact_chi) *log2_exact_chi = lg;
    return LRS_OK;
}

// ---------------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------------
static void free_terms(lrs_ctx* c) {
    cudaFree(c->F); cudaFree(c->G); cudaFree(c->M);
    cudaFree(c->glo); cudaFree(c->ghi); cudaFree(c->v); cudaFree(c->s);
    cudaFree(c->omega); cudaFree(c->coef); cudaFree(c->choice);
    c->F = c->G = c->M = c->glo = c->ghi = c->v = c->s = nullptr;
    c->omega = nullptr; c->coef = nullptr; c->choice = nullptr;
    c->cap = 0; c->chi = 0; c->choice_slots_cap = 0; c->have_terms = false;
}

static void free_chains(lrs_ctx* c) {
    cudaFree(c->Q); cudaFree(c->cx); cudaFree(c->cp); cudaFree(c->pend);
    c->Q = nullptr; c->cx = nullptr; c->cp = nullptr; c->pend = nullptr;
    c->Q_bytes = 0; c->chains_cap = 0; c->n_chains = 0;
    cudaFree(c->ybuf); cudaFree(c->lqy); cudaFree(c->lqx); cudaFree(c->ampy);
    c->ybuf = nullptr; c->lqy = nullptr; c->lqx = nullptr; c->ampy = nullptr; c->mh_cap = 0;
}

extern "C" lrs_status lrs_create(int32_t device, int32_t n_qubits, const lrs_options* opts, lrs_ctx** out) {
    if (!out) return lrs_fail(LRS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > 64)
        return lrs_fail(LRS_ERR_ARG, "n_qubits must be in 1..64 (got %d)", n_qubits);
    if (opts && opts->size < (int32_t)sizeof(lrs_options))
        return lrs_fail(LRS_ERR_ARG, "lrs_options.size %d is smaller than %d", opts->size, (int)sizeof(lrs_options));
    int count = 0;
    LRS_CUDA(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return lrs_fail(LRS_ERR_ARG, "bad device %d", device);
    LRS_CUDA(cudaSetDevice(device));
    int sms = 0;
    LRS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    lrs_ctx* c = new lrs_ctx();
    c->device = device;
    c->sm_count = sms;
    c->n = n_qubits;
    c->nmask = n_qubits == 64 ? ~0ull : ((1ull << n_qubits) - 1);
    if (opts) {
        for (int i = 0; i < LRS_OPTIONS_TUNING; ++i) {
            if (!((opts->tuning_mask >> i) & 1u)) continue;
            const lrs_status rc = lrs_set_tuning(c, i, opts->tuning[i]);
            if (rc != LRS_OK) {
                delete c;
                return rc;
            }
        }
    }
    *out = c;
    return LRS_OK;
}

extern "C" lrs_status lrs_destroy(lrs_ctx* c) {
    if (!c) return LRS_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    free_terms(c);
    free_chains(c);
    cudaFree(c->slots_dev); cudaFree(c->kgates_dev); cudaFree(c->gates_dev); cudaFree(c->scratch);
    cudaFree(c->mc_par);
    cudaFree(c->batch_buf);
    cudaFree(c->eta_buf);
    cudaFree(c->jbuf);
    if (c->mc_exec) cudaGraphExecDestroy((cudaGraphExec_t)c->mc_exec);
    if (c->cap_stream) cudaStreamDestroy((cudaStream_t)c->cap_stream);
    if (c->mc_err_h) cudaFreeHost(c->mc_err_h);
    delete c;
    return LRS_OK;
}

extern "C" lrs_status lrs_info(const lrs_ctx* c, int64_t* chi, int32_t* n, int64_t* n_slots) {
    if (!c) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    if (chi) *chi = c->chi;
    if (n) *n = c->n;
    if (n_slots) *n_slots = c->n_slots;
    return LRS_OK;
}

// Term storage for `cap` terms and `n_slots` slot choices (reused when it fits the
// same capacity; chains are dropped when it is reallocated).
static lrs_status ensure_terms(lrs_ctx* c, int64_t cap, int64_t n_slots) {
    if (cap == c->cap && n_slots <= c->choice_slots_cap) return LRS_OK;
    free_terms(c);
    free_chains(c);
    const size_t rows = (size_t)c->n * cap * sizeof(uint64_t);
    const size_t vec = (size_t)cap * sizeof(uint64_t);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&c->F, rows);
    if (e == cudaSuccess) e = cudaMalloc(&c->G, rows);
    if (e == cudaSuccess) e = cudaMalloc(&c->M, rows);
    if (e == cudaSuccess) e = cudaMalloc(&c->glo, vec);
    if (e == cudaSuccess) e = cudaMalloc(&c->ghi, vec);
    if (e == cudaSuccess) e = cudaMalloc(&c->v, vec);
    if (e == cudaSuccess) e = cudaMalloc(&c->s, vec);
    if (e == cudaSuccess) e = cudaMalloc(&c->omega, (size_t)cap * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->coef, (size_t)cap * sizeof(float2));
    const int64_t cs = std::max<int64_t>(n_slots, 1);
    if (e == cudaSuccess) e = cudaMalloc(&c->choice, (size_t)cs * cap);
    if (e != cudaSuccess) {
        free_terms(c);
        return lrs_cuda_check(e, "term storage");
    }
    c->cap = cap;
    c->choice_slots_cap = cs;
    return LRS_OK;
}

static lrs_status check_gate(const lrs_ctx* c, const lrs_gate& g, int64_t n_slots, bool allow_slot,
                             int64_t idx, const char* what) {
    if (g.op > LRS_OP_SLOT) return lrs_fail(LRS_ERR_ARG, "%s %lld: unknown op %d", what, (long long)idx, g.op);
    if (g.op == LRS_OP_SLOT) {
        if (!allow_slot) return lrs_fail(LRS_ERR_ARG, "%s %lld: nested slot", what, (long long)idx);
        if ((int64_t)g.r >= n_slots)
            return lrs_fail(LRS_ERR_ARG, "%s %lld: slot %d out of range (%lld slots)", what, (long long)idx,
                            g.r, (long long)n_slots);
        return LRS_OK;
    }
    if (g.q >= c->n) return lrs_fail(LRS_ERR_ARG, "%s %lld: qubit %d >= n", what, (long long)idx, g.q);
    if (g.op == LRS_OP_CX || g.op == LRS_OP_CZ) {
        if (g.r >= c->n) return lrs_fail(LRS_ERR_ARG, "%s %lld: qubit %d >= n", what, (long long)idx, g.r);
        if (g.r == g.q) return lrs_fail(LRS_ERR_ARG, "%s %lld: q == r", what, (long long)idx);
    }
    return LRS_OK;
}

extern "C" lrs_status lrs_init_terms(lrs_ctx* c, const lrs_slot* slots, int64_t n_slots,
                                     const lrs_gate* k_gates, int64_t n_k_gates, int64_t chi_total,
                                     int64_t alpha0, int64_t chi, int32_t mode, uint64_t seed,
                                     void* stream) {
    if (!c) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    if (chi < 1) return lrs_fail(LRS_ERR_ARG, "chi must be >= 1 (got %lld)", (long long)chi);
    if (alpha0 < 0 || chi_total < 1 || alpha0 + chi > chi_total)
        return lrs_fail(LRS_ERR_ARG, "term range [%lld, %lld) outside chi_total = %lld", (long long)alpha0,
                        (long long)(alpha0 + chi), (long long)chi_total);
    if (chi > (1ll << 34)) return lrs_fail(LRS_ERR_ARG, "chi too large");
    if (mode != LRS_MODE_EXACT && mode != LRS_MODE_SPARSIFY)
        return lrs_fail(LRS_ERR_ARG, "unknown mode %d", mode);
    if (n_slots < 0 || (n_slots > 0 && !slots) || n_k_gates < 0 || (n_k_gates > 0 && !k_gates))
        return lrs_fail(LRS_ERR_ARG, "bad slot tables");
    if (n_slots > 65535) return lrs_fail(LRS_ERR_ARG, "too many slots");
    LRS_CUDA(cudaSetDevice(c->device));
    // validate tables and build the device copies
    std::vector<DevSlot> ds((size_t)n_slots);
    double l1 = 1.0;
    long double exact_chi = 1.0L;
    for (int64_t p = 0; p < n_slots; ++p) {
        const lrs_slot& s = slots[p];
        if (s.n_choices < 1 || s.n_choices > LRS_MAX_CHOICES)
            return lrs_fail(LRS_ERR_ARG, "slot %lld: n_choices %d", (long long)p, s.n_choices);
        DevSlot& d = ds[(size_t)p];
        memset(&d, 0, sizeof(d));
        d.n_choices = s.n_choices;
        double norm = 0.0;
        for (int j = 0; j < s.n_choices; ++j) {
            if (s.k_len[j] < 0 || s.k_off[j] < 0 || (int64_t)s.k_off[j] + s.k_len[j] > n_k_gates)
                return lrs_fail(LRS_ERR_ARG, "slot %lld choice %d: bad gate range", (long long)p, j);
            for (int e = 0; e < s.k_len[j]; ++e) {
                lrs_status rc = check_gate(c, k_gates[s.k_off[j] + e], 0, false, s.k_off[j] + e, "k_gate");
                if (rc != LRS_OK) return rc;
            }
            d.k_off[j] = s.k_off[j];
            d.k_len[j] = s.k_len[j];
            d.c_re[j] = s.c_re[j];
            d.c_im[j] = s.c_im[j];
            norm += hypot(s.c_re[j], s.c_im[j]);
            if (s.c_re[j] != 0.0 || s.c_im[j] != 0.0) d.nz_idx[d.n_nonzero++] = j;
        }
        if (d.n_nonzero == 0) return lrs_fail(LRS_ERR_ARG, "slot %lld: all coefficients zero", (long long)p);
        double acc = 0.0;
        for (int j = 0; j < s.n_choices; ++j) {
            const double a = hypot(s.c_re[j], s.c_im[j]);
            acc += a / norm;
            d.cdf[j] = acc;
            d.ph_re[j] = a > 0 ? s.c_re[j] / a : 0.0;
            d.ph_im[j] = a > 0 ? s.c_im[j] / a : 0.0;
        }
        l1 *= norm;
        exact_chi *= d.n_nonzero;
    }
    if (mode == LRS_MODE_EXACT && (exact_chi > 1e18L || (int64_t)exact_chi != chi_total))
        return lrs_fail(LRS_ERR_ARG, "EXACT mode needs chi_total = %.0Lf (got %lld)", exact_chi,
                        (long long)chi_total);

    // (re)allocate term storage
    const int64_t cap = (chi + LRS_TERM_ALIGN - 1) / LRS_TERM_ALIGN * LRS_TERM_ALIGN;
    lrs_status rs = ensure_terms(c, cap, n_slots);
    if (rs != LRS_OK) return rs;
    c->chi = chi;
    c->alpha0 = alpha0;
    c->chi_total = chi_total;
    c->n_chains = 0;
    // slot tables
    size_t have = (size_t)c->slots_cap * sizeof(DevSlot);
    lrs_status rc = lrs_ensure((void**)&c->slots_dev, &have, std::max<size_t>(1, ds.size()) * sizeof(DevSlot));
    if (rc != LRS_OK) return rc;
    c->slots_cap = (int64_t)(have / sizeof(DevSlot));
    have = (size_t)c->kgates_cap * sizeof(lrs_gate);
    rc = lrs_ensure((void**)&c->kgates_dev, &have, std::max<int64_t>(1, n_k_gates) * sizeof(lrs_gate));
    if (rc != LRS_OK) return rc;
    c->kgates_cap = (int64_t)(have / sizeof(lrs_gate));
    cudaStream_t st = as_stream(stream);
    if (n_slots > 0)
        LRS_CUDA(cudaMemcpyAsync(c->slots_dev, ds.data(), ds.size() * sizeof(DevSlot),
                                 cudaMemcpyHostToDevice, st));
    if (n_k_gates > 0)
        LRS_CUDA(cudaMemcpyAsync(c->kgates_dev, k_gates, (size_t)n_k_gates * sizeof(lrs_gate),
                                 cudaMemcpyHostToDevice, st));
    LRS_CUDA(cudaStreamSynchronize(st));   // host tables may be freed on return
    c->n_slots = n_slots;
    c->slots_host.assign(slots, slots + n_slots);
    c->kgates_host.assign(k_gates, k_gates + n_k_gates);
    c->init_scale = l1 / (double)chi_total;
    rc = launch_init_terms(c, mode, seed, c->init_scale, st);
    if (rc != LRS_OK) return rc;
    c->have_terms = true;
    c->mode = mode;
    c->fresh = true;
    return LRS_OK;
}

extern "C" lrs_status lrs_reinit_terms(lrs_ctx* c, uint64_t seed, void* stream) {
    if (!c) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    if (c->cap == 0 || c->init_scale == 0.0) return lrs_fail(LRS_ERR_STATE, "lrs_init_terms has not been called");
    LRS_CUDA(cudaSetDevice(c->device));
    lrs_status rc = launch_init_terms(c, c->mode, seed, c->init_scale, as_stream(stream));
    if (rc != LRS_OK) return rc;
    c->have_terms = true;
    c->fresh = true;
    c->n_chains = 0;
    return LRS_OK;
}

extern "C" lrs_status lrs_apply_clifford(lrs_ctx* c, const lrs_gate* gates, int64_t n_gates,
                                         void* stream) {
    if (!c) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    if (!c->have_terms) return lrs_fail(LRS_ERR_STATE, "lrs_init_terms has not been called");
    if (n_gates < 0 || (n_gates > 0 && !gates)) return lrs_fail(LRS_ERR_ARG, "bad gate array");
    if (n_gates == 0) return LRS_OK;
    for (int64_t i = 0; i < n_gates; ++i) {
        lrs_status rc = check_gate(c, gates[i], c->n_slots, true, i, "gate");
        if (rc != LRS_OK) return rc;
    }
    LRS_CUDA(cudaSetDevice(c->device));
    c->n_chains = 0;                        // chain states refer to the old terms
    c->fresh = false;
    return launch_apply_clifford(c, gates, n_gates, as_stream(stream));   // gates go in as launch parameters
}

extern "C" lrs_status lrs_apply_circuit_shared(lrs_ctx* c, const lrs_gate* gates, int64_t n_gates, void* stream) {
    if (!c) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    if (!c->have_terms) return lrs_fail(LRS_ERR_STATE, "lrs_init_terms has not been called");
    if (!c->fresh) return lrs_fail(LRS_ERR_STATE, "terms are not as lrs_init_terms left them");
    if (c->mode != LRS_MODE_EXACT || c->alpha0 != 0 || c->chi != c->chi_total)
        return lrs_fail(LRS_ERR_STATE, "prefix sharing needs the whole exact decomposition in one context");
    if (n_gates < 0 || (n_gates > 0 && !gates)) return lrs_fail(LRS_ERR_ARG, "bad gate array");
    // Nonzero choices of the slot that gate i names: its digit's radix.
    auto radix = [&](int64_t i) {
        const lrs_slot& sl = c->slots_host[(size_t)gates[i].r];
        int64_t r = 0;
        for (int j = 0; j < sl.n_choices; ++j) r += (sl.c_re[j] != 0.0 || sl.c_im[j] != 0.0) ? 1 : 0;
        return r;
    };
    int64_t next_slot = 0, prod = 1;
    for (int64_t i = 0; i < n_gates; ++i) {
        lrs_status rc = check_gate(c, gates[i], c->n_slots, true, i, "gate");
        if (rc != LRS_OK) return rc;
        if (gates[i].op == LRS_OP_SLOT) {
            if (gates[i].r != next_slot)
                return lrs_fail(LRS_ERR_ARG, "gate %lld: slots must appear once each, in order 0..%lld",
                                (long long)i, (long long)c->n_slots - 1);
            ++next_slot;
            const int64_t r = radix(i);
            if (r < 1 || prod > c->chi / r)
                return lrs_fail(LRS_ERR_STATE, "gate %lld: slot radices give more than %lld terms", (long long)i,
                                (long long)c->chi);
            prod *= r;
        }
    }
    if (next_slot != c->n_slots) return lrs_fail(LRS_ERR_ARG, "the gate list misses slots");
    if (prod != c->chi)
        return lrs_fail(LRS_ERR_STATE, "slot radices give %lld terms, not %lld", (long long)prod, (long long)c->chi);
    LRS_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = as_stream(stream);
    c->n_chains = 0;
    c->fresh = false;
    // Term alpha has digit j_p = (alpha / R_p) mod r_p over the nonzero choices of slot
    // p (R_p = r_0 ... r_{p-1}), so the R_p distinct states before slot p are terms
    // 0..R_p-1.  Each Clifford segment runs on those only; at a run of consecutive
    // slots the R_p states are copied out to R_{p+k} terms at once, and the run's slots
    // (each term its own choices) go into the same launch as the segment after them.
    int64_t R = 1, start = 0, i = 0;
    lrs_status rc;
    while (i < n_gates) {
        if (gates[i].op != LRS_OP_SLOT) { ++i; continue; }
        if ((rc = launch_apply_clifford_range(c, gates + start, i - start, R, st)) != LRS_OK) return rc;
        int64_t Rn = R;
        start = i;
        for (; i < n_gates && gates[i].op == LRS_OP_SLOT; ++i) Rn *= radix(i);
        if ((rc = launch_expand_terms(c, R, Rn, st)) != LRS_OK) return rc;
        R = Rn;
    }
    return launch_apply_clifford_range(c, gates + start, n_gates - start, R, st);
}

extern "C" lrs_status lrs_apply_clifford_batch(lrs_ctx* const* ctxs, const lrs_gate* const* gates,
                                               const int64_t* n_gates, int32_t count, void* stream) {
    if (!ctxs || !gates || !n_gates || count < 1) return lrs_fail(LRS_ERR_ARG, "bad batch arguments");
    const int dev = ctxs[0] ? ctxs[0]->device : -1;
    for (int32_t i = 0; i < count; ++i) {
        lrs_ctx* c = ctxs[i];
        if (!c) return lrs_fail(LRS_ERR_ARG, "ctx %d is NULL", i);
        if (c->device != dev) return lrs_fail(LRS_ERR_ARG, "contexts on different devices");
        if (!c->have_terms) return lrs_fail(LRS_ERR_STATE, "ctx %d has no terms", i);
        for (int32_t j = 0; j < i; ++j)
            if (ctxs[j] == c) return lrs_fail(LRS_ERR_ARG, "ctx %d repeated", i);
        if (n_gates[i] < 0 || (n_gates[i] > 0 && !gates[i])) return lrs_fail(LRS_ERR_ARG, "bad gate array %d", i);
        for (int64_t g = 0; g < n_gates[i]; ++g) {
            lrs_status rc = check_gate(c, gates[i][g], c->n_slots, true, g, "gate");
            if (rc != LRS_OK) return rc;
        }
    }
    LRS_CUDA(cudaSetDevice(dev));
    cudaStream_t st = as_stream(stream);
    for (int32_t i = 0; i < count; ++i) {
        lrs_ctx* c = ctxs[i];
        std::vector<lrs_gate> sg((size_t)n_gates[i]);
        specialise_gates(c, gates[i], n_gates[i], sg.data());
        // upload only a list that is not resident already (so that a repeated batch,
        // e.g. one being captured into a CUDA graph, makes no copy and no host wait)
        const bool resident = sg.size() == c->gates_resident.size() &&
                              (sg.empty() || memcmp(sg.data(), c->gates_resident.data(), sg.size() * sizeof(lrs_gate)) == 0);
        if (!resident) {
            size_t have = (size_t)c->gates_cap * sizeof(lrs_gate);
            lrs_status rc = lrs_ensure((void**)&c->gates_dev, &have, std::max<size_t>(1, sg.size()) * sizeof(lrs_gate));
            if (rc != LRS_OK) return rc;
            c->gates_cap = (int64_t)(have / sizeof(lrs_gate));
            c->gates_resident.clear();
            if (!sg.empty()) {
                LRS_CUDA(cudaMemcpyAsync(c->gates_dev, sg.data(), sg.size() * sizeof(lrs_gate), cudaMemcpyHostToDevice,
                                         st));
                LRS_CUDA(cudaStreamSynchronize(st));   // the staging vector is freed on return
            }
            c->gates_resident.swap(sg);
        }
        c->batch_n_gates = n_gates[i];
        c->n_chains = 0;
        c->fresh = false;
    }
    return launch_apply_clifford_batch(ctxs, count, st, &ctxs[0]->batch_buf, &ctxs[0]->batch_buf_bytes);
}

extern "C" lrs_status lrs_amplitude(lrs_ctx* c, const uint64_t* x, int64_t batch, double* out,
                                    float* err_est, void* stream) {
    if (!c) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    if (!c->have_terms) return lrs_fail(LRS_ERR_STATE, "no terms");
    if (batch < 0) return lrs_fail(LRS_ERR_ARG, "batch < 0");
    if (batch > 0 && (!x || !out)) return lrs_fail(LRS_ERR_ARG, "NULL buffer");
    LRS_CUDA(cudaSetDevice(c->device));
    return launch_amplitude(c, x, batch, out, err_est, as_stream(stream));
}

extern "C" lrs_status lrs_amplitude_batch(lrs_ctx* const* ctxs, const uint64_t* const* x, const int64_t* batch,
                                          double* const* out, int32_t count, void* stream) {
    if (!ctxs || !x || !batch || !out || count < 1) return lrs_fail(LRS_ERR_ARG, "bad batch arguments");
    const lrs_ctx* c0 = ctxs[0];
    if (!c0) return lrs_fail(LRS_ERR_ARG, "ctx 0 is NULL");
    for (int32_t i = 0; i < count; ++i) {
        const lrs_ctx* c = ctxs[i];
        if (!c) return lrs_fail(LRS_ERR_ARG, "ctx %d is NULL", i);
        if (c->device != c0->device || c->n != c0->n)
            return lrs_fail(LRS_ERR_ARG, "contexts differ in device or qubit count");
        if (!c->have_terms) return lrs_fail(LRS_ERR_STATE, "ctx %d has no terms", i);
        for (int32_t j = 0; j < i; ++j)
            if (ctxs[j] == c) return lrs_fail(LRS_ERR_ARG, "ctx %d repeated", i);
        if (batch[i] < 0 || (batch[i] > 0 && (!x[i] || !out[i]))) return lrs_fail(LRS_ERR_ARG, "bad buffers %d", i);
    }
    LRS_CUDA(cudaSetDevice(c0->device));
    return launch_amplitude_batch(ctxs, x, batch, out, count, as_stream(stream));
}

extern "C" lrs_status lrs_norm_estimate(lrs_ctx* c, int64_t L, uint64_t seed, double* eta,
                                        double* mean_host, void* stream) {
    if (!c) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    if (!c->have_terms) return lrs_fail(LRS_ERR_STATE, "no terms");
    if (L < 1) return lrs_fail(LRS_ERR_ARG, "L must be >= 1");
    if (!eta) return lrs_fail(LRS_ERR_ARG, "eta is NULL");
    LRS_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = as_stream(stream);
    lrs_status rc = launch_norm_estimate(c, L, seed, eta, nullptr, st);
    if (rc != LRS_OK) return rc;
    if (mean_host) {
        std::vector<double> h((size_t)L);
        LRS_CUDA(cudaMemcpyAsync(h.data(), eta, (size_t)L * sizeof(double), cudaMemcpyDeviceToHost, st));
        LRS_CUDA(cudaStreamSynchronize(st));
        double m = 0.0;
        for (double x : h) m += x;
        *mean_host = m / (double)L;
    }
    return LRS_OK;
}

extern "C" lrs_status lrs_norm_overlaps(lrs_ctx* c, int64_t L, uint64_t seed, double* ov, void* stream) {
    if (!c) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    if (!c->have_terms) return lrs_fail(LRS_ERR_STATE, "no terms");
    if (L < 1) return lrs_fail(LRS_ERR_ARG, "L must be >= 1");
    if (!ov) return lrs_fail(LRS_ERR_ARG, "ov is NULL");
    LRS_CUDA(cudaSetDevice(c->device));
    return launch_norm_estimate(c, L, seed, nullptr, ov, as_stream(stream));
}

extern "C" lrs_status lrs_norm_eta_from_overlaps(lrs_ctx* c, int64_t L, const double* ov, double* eta,
                                                 void* stream) {
    if (!c || !ov || !eta) return lrs_fail(LRS_ERR_ARG, "NULL argument");
    if (L < 1) return lrs_fail(LRS_ERR_ARG, "L must be >= 1");
    LRS_CUDA(cudaSetDevice(c->device));
    return launch_norm_eta(ov, L, eta, as_stream(stream));
}

extern "C" lrs_status lrs_copy_terms(lrs_ctx* dst, const lrs_ctx* src, void* stream) {
    if (!dst || !src) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    if (dst == src) return LRS_OK;
    if (!src->have_terms) return lrs_fail(LRS_ERR_STATE, "source has no terms");
    if (dst->n != src->n || dst->device != src->device)
        return lrs_fail(LRS_ERR_ARG, "contexts differ in qubit count or device");
    LRS_CUDA(cudaSetDevice(dst->device));
    cudaStream_t st = as_stream(stream);
    lrs_status rc = ensure_terms(dst, src->cap, src->n_slots);
    if (rc != LRS_OK) return rc;
    const size_t rows = (size_t)src->n * src->cap * sizeof(uint64_t), vec = (size_t)src->cap * sizeof(uint64_t);
    const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
    LRS_CUDA(cudaMemcpyAsync(dst->F, src->F, rows, dd, st));
    LRS_CUDA(cudaMemcpyAsync(dst->G, src->G, rows, dd, st));
    LRS_CUDA(cudaMemcpyAsync(dst->M, src->M, rows, dd, st));
    LRS_CUDA(cudaMemcpyAsync(dst->glo, src->glo, vec, dd, st));
    LRS_CUDA(cudaMemcpyAsync(dst->ghi, src->ghi, vec, dd, st));
    LRS_CUDA(cudaMemcpyAsync(dst->v, src->v, vec, dd, st));
    LRS_CUDA(cudaMemcpyAsync(dst->s, src->s, vec, dd, st));
    LRS_CUDA(cudaMemcpyAsync(dst->omega, src->omega, (size_t)src->cap * sizeof(uint32_t), dd, st));
    LRS_CUDA(cudaMemcpyAsync(dst->coef, src->coef, (size_t)src->cap * sizeof(float2), dd, st));
    if (src->n_slots > 0)
        LRS_CUDA(cudaMemcpyAsync(dst->choice, src->choice, (size_t)src->n_slots * src->cap, dd, st));
    size_t have = (size_t)dst->slots_cap * sizeof(DevSlot);
    rc = lrs_ensure((void**)&dst->slots_dev, &have, std::max<size_t>(1, (size_t)src->n_slots) * sizeof(DevSlot));
    if (rc != LRS_OK) return rc;
    dst->slots_cap = (int64_t)(have / sizeof(DevSlot));
    have = (size_t)dst->kgates_cap * sizeof(lrs_gate);
    rc = lrs_ensure((void**)&dst->kgates_dev, &have, std::max<size_t>(1, src->kgates_host.size()) * sizeof(lrs_gate));
    if (rc != LRS_OK) return rc;
    dst->kgates_cap = (int64_t)(have / sizeof(lrs_gate));
    if (src->n_slots > 0)
        LRS_CUDA(cudaMemcpyAsync(dst->slots_dev, src->slots_dev, (size_t)src->n_slots * sizeof(DevSlot), dd, st));
    if (!src->kgates_host.empty())
        LRS_CUDA(cudaMemcpyAsync(dst->kgates_dev, src->kgates_dev, src->kgates_host.size() * sizeof(lrs_gate), dd, st));
    dst->n_slots = src->n_slots;
    dst->slots_host = src->slots_host;
    dst->kgates_host = src->kgates_host;
    dst->chi = src->chi;
    dst->alpha0 = src->alpha0;
    dst->chi_total = src->chi_total;
    dst->n_chains = 0;
    dst->have_terms = true;
    dst->mode = src->mode;
    dst->init_scale = src->init_scale;
    dst->fresh = src->fresh;
    return LRS_OK;
}

// Median of the K means of consecutive groups of L values (even K: mean of the two
// middle means).
static double median_of_means(const double* eta, int64_t L, int32_t K) {
    std::vector<double> m((size_t)K);
    for (int32_t g = 0; g < K; ++g) {
        double acc = 0.0;
        for (int64_t l = 0; l < L; ++l) acc += eta[(size_t)g * L + l];
        m[(size_t)g] = acc / (double)L;
    }
    std::sort(m.begin(), m.end());
    return (K & 1) ? m[(size_t)K / 2] : 0.5 * (m[(size_t)K / 2 - 1] + m[(size_t)K / 2]);
}

static lrs_status norm_mom(lrs_ctx* c, int64_t L, int32_t K, uint64_t seed, double* out, cudaStream_t st) {
    const int64_t LK = L * K;
    size_t have = c->eta_bytes;
    lrs_status rc = lrs_ensure((void**)&c->eta_buf, &have, (size_t)LK * sizeof(double));
    if (rc != LRS_OK) return rc;
    c->eta_bytes = have;
    rc = launch_norm_estimate(c, LK, seed, c->eta_buf, nullptr, st);
    if (rc != LRS_OK) return rc;
    std::vector<double> h((size_t)LK);
    LRS_CUDA(cudaMemcpyAsync(h.data(), c->eta_buf, (size_t)LK * sizeof(double), cudaMemcpyDeviceToHost, st));
    LRS_CUDA(cudaStreamSynchronize(st));
    *out = median_of_means(h.data(), L, K);
    return LRS_OK;
}

extern "C" lrs_status lrs_norm_median_of_means(lrs_ctx* c, int64_t L, int32_t K, uint64_t seed,
                                               double* estimate_host, void* stream) {
    if (!c || !estimate_host) return lrs_fail(LRS_ERR_ARG, "NULL argument");
    if (!c->have_terms) return lrs_fail(LRS_ERR_STATE, "no terms");
    if (L < 1 || K < 1 || L * (int64_t)K > (1ll << 22)) return lrs_fail(LRS_ERR_ARG, "need L, K >= 1 and L K <= 2^22");
    LRS_CUDA(cudaSetDevice(c->device));
    return norm_mom(c, L, K, seed, estimate_host, as_stream(stream));
}

extern "C" lrs_status lrs_sparsification_certificate(lrs_ctx* c, int64_t L, int32_t K, uint64_t seed,
                                                      lrs_certificate* out, void* stream) {
    if (!c || !out) return lrs_fail(LRS_ERR_ARG, "NULL argument");
    if (!c->have_terms) return lrs_fail(LRS_ERR_STATE, "no terms");
    if (L < 1 || K < 1 || L * (int64_t)K > (1ll << 22)) return lrs_fail(LRS_ERR_ARG, "need L, K >= 1 and L K <= 2^22");
    LRS_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = as_stream(stream);
    double mom = 0.0;
    lrs_status rc = norm_mom(c, L, K, seed, &mom, st);   // leaves the L K values in eta_buf
    if (rc != LRS_OK) return rc;
    const int64_t LK = L * K;
    std::vector<double> h((size_t)LK);
    LRS_CUDA(cudaMemcpy(h.data(), c->eta_buf, (size_t)LK * sizeof(double), cudaMemcpyDeviceToHost));
    double mean = 0.0;
    for (double x : h) mean += x;
    mean /= (double)LK;
    double var = 0.0;
    for (double x : h) var += (x - mean) * (x - mean);
    const double se = LK > 1 ? sqrt(var / (double)(LK - 1) / (double)LK) : INFINITY;
    double l1 = 1.0;
    rc = lrs_decomposition_stats(c->slots_host.data(), (int64_t)c->slots_host.size(), &l1, nullptr, nullptr);
    if (rc != LRS_OK) return rc;
    memset(out, 0, sizeof(*out));
    out->omega_norm2 = mom;
    out->stderr_mean = se;
    out->delta2 = l1 * l1 / (double)c->chi_total;
    out->bound = mom - 1.0 + out->delta2;
    out->bound_upper = mom + 2.0 * se - 1.0 + out->delta2;
    out->conclusive = (2.0 * se < out->delta2) ? 1 : 0;
    return LRS_OK;
}

extern "C" lrs_status lrs_marginal_sample(lrs_ctx* c, lrs_ctx* work0, lrs_ctx* work1, const int32_t* qubits,
                                          int32_t w, int64_t L, int32_t K, uint64_t seed, uint8_t* bits_host,
                                          double* probs_host, void* stream) {
    if (!c || !work0 || !work1 || (w > 0 && (!qubits || !bits_host))) return lrs_fail(LRS_ERR_ARG, "NULL argument");
    if (work0 == work1 || work0 == c || work1 == c) return lrs_fail(LRS_ERR_ARG, "contexts must be distinct");
    if (!c->have_terms) return lrs_fail(LRS_ERR_STATE, "no terms");
    if (w < 0 || w > c->n) return lrs_fail(LRS_ERR_ARG, "w must be in 0..n");
    if (L < 1 || K < 1 || L * (int64_t)K > (1ll << 22)) return lrs_fail(LRS_ERR_ARG, "need L, K >= 1 and L K <= 2^22");
    for (int32_t i = 0; i < w; ++i) {
        if (qubits[i] < 0 || qubits[i] >= c->n) return lrs_fail(LRS_ERR_ARG, "qubit %d out of range", qubits[i]);
        for (int32_t j = 0; j < i; ++j)
            if (qubits[j] == qubits[i]) return lrs_fail(LRS_ERR_ARG, "qubit %d listed twice", qubits[i]);
    }
    LRS_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = as_stream(stream);
    lrs_status rc = lrs_copy_terms(work0, c, stream);      // prefix Pi_{x_<i} psi
    if (rc != LRS_OK) return rc;
    lrs_ctx* pref = work0;
    lrs_ctx* alt = work1;
    for (int32_t i = 0; i < w; ++i) {
        // both branches from the prefix, the same equatorial states for both
        if ((rc = lrs_copy_terms(alt, pref, stream)) != LRS_OK) return rc;
        lrs_gate g0, g1;
        g0.op = LRS_OP_P0; g0.q = (uint8_t)qubits[i]; g0.r = 0;
        g1.op = LRS_OP_P1; g1.q = (uint8_t)qubits[i]; g1.r = 0;
        if ((rc = lrs_apply_clifford(alt, &g0, 1, stream)) != LRS_OK) return rc;
        if ((rc = lrs_apply_clifford(pref, &g1, 1, stream)) != LRS_OK) return rc;
        const uint64_t s_i = sm64_at(sm64_key(seed, (1ull << 41) + (uint64_t)i), 0);
        double p0 = 0.0, p1 = 0.0;
        if ((rc = norm_mom(alt, L, K, s_i, &p0, st)) != LRS_OK) return rc;
        if ((rc = norm_mom(pref, L, K, s_i, &p1, st)) != LRS_OK) return rc;
        const double u = sm64_unit(sm64_at(sm64_key(seed, (1ull << 42) + (uint64_t)i), 0));
        const double tot = p0 + p1;
        const int x = (tot > 0.0 && u < p1 / tot) ? 1 : 0;
        bits_host[i] = (uint8_t)x;
        if (probs_host) {
            probs_host[2 * i] = p0;
            probs_host[2 * i + 1] = p1;
        }
        if (x == 0) std::swap(pref, alt);   // the prefix holds the chosen branch
    }
    return LRS_OK;
}

extern "C" lrs_status lrs_sample_terms(lrs_ctx* c, int64_t count, uint64_t seed, uint64_t* x,
                                       int64_t* alpha, void* stream) {
    if (!c) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    if (!c->have_terms) return lrs_fail(LRS_ERR_STATE, "no terms");
    if (count < 0 || (count > 0 && !x)) return lrs_fail(LRS_ERR_ARG, "bad output");
    LRS_CUDA(cudaSetDevice(c->device));
    return launch_sample_terms(c, count, seed, x, alpha, as_stream(stream));
}

extern "C" lrs_status lrs_chains_init(lrs_ctx* c, int64_t n_chains, const uint64_t* x, void* stream) {
    if (!c) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    if (!c->have_terms) return lrs_fail(LRS_ERR_STATE, "no terms");
    if (c->n > 62) return lrs_fail(LRS_ERR_UNSUPPORTED, "Metropolis needs n <= 62");
    if (n_chains < 1 || !x) return lrs_fail(LRS_ERR_ARG, "bad chains");
    if (n_chains > 65535) return lrs_fail(LRS_ERR_ARG, "at most 65535 chains");
    LRS_CUDA(cudaSetDevice(c->device));
    const size_t qb = (size_t)n_chains * c->cap * q_bytes(c->n);
    lrs_status rc = lrs_ensure((void**)&c->Q, &c->Q_bytes, qb);
    if (rc != LRS_OK) return rc;
    if (n_chains > c->chains_cap) {
        cudaFree(c->cx); cudaFree(c->cp); cudaFree(c->pend);
        c->cx = nullptr; c->cp = nullptr; c->pend = nullptr;
        c->chains_cap = 0;
        LRS_CUDA(cudaMalloc(&c->cx, (size_t)n_chains * sizeof(uint64_t)));
        LRS_CUDA(cudaMalloc(&c->cp, (size_t)n_chains * sizeof(double)));
        LRS_CUDA(cudaMalloc(&c->pend, 2 * (size_t)n_chains * sizeof(int32_t)));
        c->chains_cap = n_chains;
    }
    c->n_chains = n_chains;
    c->q_stale = false;
    c->split_step = -1;
    return launch_chains_init(c, x, as_stream(stream));
}

extern "C" lrs_status lrs_metropolis_step(lrs_ctx* c, int64_t steps, uint64_t seed, int64_t step0,
                                          uint64_t* x_out, double* p_out, uint64_t* trace, void* stream) {
    if (!c) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    if (c->n_chains < 1) return lrs_fail(LRS_ERR_STATE, "chains not initialised");
    if (steps < 0 || step0 < 0) return lrs_fail(LRS_ERR_ARG, "steps < 0");
    LRS_CUDA(cudaSetDevice(c->device));
    if (c->q_stale) {
        lrs_status rc = launch_chains_refresh(c, as_stream(stream));
        if (rc != LRS_OK) return rc;
    }
    return launch_metropolis(c, steps, seed, step0, x_out, p_out, trace, as_stream(stream));
}

extern "C" lrs_status lrs_chains_set_amplitude(lrs_ctx* c, const double* amp, void* stream) {
    if (!c || !amp) return lrs_fail(LRS_ERR_ARG, "NULL argument");
    if (c->n_chains < 1) return lrs_fail(LRS_ERR_STATE, "chains not initialised");
    LRS_CUDA(cudaSetDevice(c->device));
    return launch_chains_set_prob(c, amp, as_stream(stream));
}

extern "C" lrs_status lrs_metropolis_propose(lrs_ctx* c, uint64_t seed, int64_t step, double* amp, void* stream) {
    if (!c || !amp) return lrs_fail(LRS_ERR_ARG, "NULL argument");
    if (c->n_chains < 1) return lrs_fail(LRS_ERR_STATE, "chains not initialised");
    if (step < 0) return lrs_fail(LRS_ERR_ARG, "step < 0");
    if (c->q_stale) return lrs_fail(LRS_ERR_STATE, "chains moved by learned proposals: re-initialise them");
    LRS_CUDA(cudaSetDevice(c->device));
    lrs_status rc = launch_metropolis_propose(c, seed, step, amp, as_stream(stream));
    if (rc == LRS_OK) c->split_step = step;
    return rc;
}

extern "C" lrs_status lrs_metropolis_accept(lrs_ctx* c, const double* amp, uint64_t seed, int64_t step,
                                            uint64_t* trace, void* stream) {
    if (!c || !amp) return lrs_fail(LRS_ERR_ARG, "NULL argument");
    if (c->n_chains < 1) return lrs_fail(LRS_ERR_STATE, "chains not initialised");
    if (c->split_step != step) return lrs_fail(LRS_ERR_STATE, "no lrs_metropolis_propose of step %lld", (long long)step);
    LRS_CUDA(cudaSetDevice(c->device));
    lrs_status rc = launch_metropolis_accept(c, amp, seed, step, trace, as_stream(stream));
    c->split_step = -1;
    return rc;
}

extern "C" lrs_status lrs_metropolis_learned(lrs_ctx* c, lrs_mlp* mlp, int64_t steps, uint64_t seed,
                                             int64_t step0, uint64_t* x_out, double* p_out,
                                             uint64_t* trace, int64_t* accepts, void* stream) {
    if (!c || !mlp) return lrs_fail(LRS_ERR_ARG, "NULL argument");
    if (c->n_chains < 1) return lrs_fail(LRS_ERR_STATE, "chains not initialised");
    if (steps < 0 || step0 < 0) return lrs_fail(LRS_ERR_ARG, "steps < 0");
    int32_t mn = 0;
    lrs_mlp_info(mlp, &mn, nullptr, nullptr);
    if (mn != c->n) return lrs_fail(LRS_ERR_ARG, "network width %d != n = %d", mn, c->n);
    LRS_CUDA(cudaSetDevice(c->device));
    return launch_metropolis_learned(c, mlp, steps, seed, step0, x_out, p_out, trace, accepts,
                                     as_stream(stream));
}

extern "C" lrs_status lrs_debug_inject_wait_timeout(lrs_ctx* c) {
    if (!c) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    LRS_CUDA(cudaSetDevice(c->device));
    lrs_status rc = mc_flags(c);
    if (rc != LRS_OK) return rc;
    *(volatile int*)&c->mc_err_h[1] = 1;
    return LRS_OK;
}

extern "C" lrs_status lrs_export_terms(lrs_ctx* c, int64_t first, int64_t count, uint64_t* F,
                                       uint64_t* G, uint64_t* M, uint8_t* gamma, uint64_t* v,
                                       uint64_t* s, int32_t* omega, float* coef, uint8_t* choice) {
    if (!c) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    if (!c->have_terms) return lrs_fail(LRS_ERR_STATE, "no terms");
    if (first < 0 || count < 0 || first + count > c->chi) return lrs_fail(LRS_ERR_ARG, "bad range");
    if (count == 0) return LRS_OK;
    LRS_CUDA(cudaSetDevice(c->device));
    LRS_CUDA(cudaDeviceSynchronize());
    const int n = c->n;
    std::vector<uint64_t> buf((size_t)count);
    auto rows = [&](const uint64_t* src, uint64_t* dst) -> lrs_status {
        for (int p = 0; p < n; ++p) {
            LRS_CUDA(cudaMemcpy(buf.data(), src + (int64_t)p * c->cap + first, (size_t)count * 8,
                                cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < count; ++i) dst[i * n + p] = buf[(size_t)i];
        }
        return LRS_OK;
    };
    lrs_status rc;
    if (F && (rc = rows(c->F, F)) != LRS_OK) return rc;
    if (G && (rc = rows(c->G, G)) != LRS_OK) return rc;
    if (M && (rc = rows(c->M, M)) != LRS_OK) return rc;
    if (gamma) {
        std::vector<uint64_t> lo((size_t)count), hi((size_t)count);
        LRS_CUDA(cudaMemcpy(lo.data(), c->glo + first, (size_t)count * 8, cudaMemcpyDeviceToHost));
        LRS_CUDA(cudaMemcpy(hi.data(), c->ghi + first, (size_t)count * 8, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < count; ++i)
            for (int p = 0; p < n; ++p)
                gamma[i * n + p] = (uint8_t)(((lo[(size_t)i] >> p) & 1) | (((hi[(size_t)i] >> p) & 1) << 1));
    }
    if (v) LRS_CUDA(cudaMemcpy(v, c->v + first, (size_t)count * 8, cudaMemcpyDeviceToHost));
    if (s) LRS_CUDA(cudaMemcpy(s, c->s + first, (size_t)count * 8, cudaMemcpyDeviceToHost));
    if (omega) LRS_CUDA(cudaMemcpy(omega, c->omega + first, (size_t)count * 4, cudaMemcpyDeviceToHost));
    if (coef) LRS_CUDA(cudaMemcpy(coef, c->coef + first, (size_t)count * 8, cudaMemcpyDeviceToHost));
    if (choice && c->n_slots > 0) {
        std::vector<uint8_t> cb((size_t)count);
        for (int64_t p = 0; p < c->n_slots; ++p) {
            LRS_CUDA(cudaMemcpy(cb.data(), c->choice + p * c->cap + first, (size_t)count,
                                cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < count; ++i) choice[i * c->n_slots + p] = cb[(size_t)i];
        }
    }
    return LRS_OK;
}

extern "C" lrs_status lrs_set_tuning(lrs_ctx* c, int32_t param, int64_t value) {
    if (!c) return lrs_fail(LRS_ERR_ARG, "ctx is NULL");
    switch (param) {
        case LRS_TUNE_AMP_BLOCKS_PER_SM:
            if (value < 1 || value > 64) return lrs_fail(LRS_ERR_ARG, "amp blocks per SM in 1..64");
            c->tune_amp_bps = value;
            return LRS_OK;
        case LRS_TUNE_NORM_MAX_TILES:
            if (value < 1 || value > (1 << 20)) return lrs_fail(LRS_ERR_ARG, "norm tiles in 1..2^20");
            c->tune_norm_tiles = value;
            return LRS_OK;
        case LRS_TUNE_MC_CHAINS_PER_BLOCK:
            if (value < 1 || value > 64) return lrs_fail(LRS_ERR_ARG, "chains per block in 1..64");
            c->tune_mc_cg = value;
            return LRS_OK;
        case LRS_TUNE_MC_STAGES:
            if (value < 1 || value > 4) return lrs_fail(LRS_ERR_ARG, "Metropolis stages in 1..4");
            c->tune_mc_stages = value;
            return LRS_OK;
        case LRS_TUNE_NORM_MAX_FOLDS:
            if (value < -1 || value > 12) return lrs_fail(LRS_ERR_ARG, "norm max folds in -1..12");
            c->tune_norm_folds = value;
            return LRS_OK;
        case LRS_TUNE_APPLY_LANES:
            if (value != 1 && value != 2 && value != 4) return lrs_fail(LRS_ERR_ARG, "apply lanes per term: 1, 2 or 4");
            c->tune_apply_lanes = value;
            return LRS_OK;
        case LRS_TUNE_NORM_FUSE_FOLDS:
            if (value < 0 || value > 8) return lrs_fail(LRS_ERR_ARG, "norm fused folds in 0..8");
            c->tune_norm_fuse = value;
            return LRS_OK;
        case LRS_TUNE_MC_LOOKAHEAD:
            if (value != 1 && value != 2) return lrs_fail(LRS_ERR_ARG, "Metropolis steps per pass: 1 or 2");
            c->tune_mc_lookahead = value;
            return LRS_OK;
        default:
            return lrs_fail(LRS_ERR_ARG, "unknown tuning parameter %d", param);
    }
}

extern "C" lrs_status lrs_get_tuning(const lrs_ctx* c, int32_t param, int64_t* value) {
    if (!c || !value) return lrs_fail(LRS_ERR_ARG, "NULL argument");
    switch (param) {
        case LRS_TUNE_AMP_BLOCKS_PER_SM: *value = c->tune_amp_bps; return LRS_OK;
        case LRS_TUNE_NORM_MAX_TILES: *value = c->tune_norm_tiles; return LRS_OK;
        case LRS_TUNE_MC_CHAINS_PER_BLOCK: *value = c->tune_mc_cg; return LRS_OK;
        case LRS_TUNE_MC_STAGES: *value = c->tune_mc_stages; return LRS_OK;
        case LRS_TUNE_NORM_MAX_FOLDS: *value = c->tune_norm_folds; return LRS_OK;
        case LRS_TUNE_APPLY_LANES: *value = c->tune_apply_lanes; return LRS_OK;
        case LRS_TUNE_NORM_FUSE_FOLDS: *value = c->tune_norm_fuse; return LRS_OK;
        case LRS_TUNE_MC_LOOKAHEAD: *value = c->tune_mc_lookahead; return LRS_OK;
        default: return lrs_fail(LRS_ERR_ARG, "unknown tuning parameter %d", param);
    }
}
