/*
 * lrstab.h -- C ABI of the GB300 low-rank stabilizer-decomposition simulator.
 *
 * The library holds chi CH-form stabilizer states (F, G, M, gamma, v, s,
 * omega) of one n-qubit circuit, n <= 64 (Sec. 4.1, Eqs. (phi), (tableaux),
 * (Htype) of Bravyi et al., arXiv:1808.00128), together with their
 * coefficients b_alpha, so that psi = sum_alpha b_alpha phi_alpha
 * (Eq. (approxU1)).  Its calls follow the paper's problem statement
 * (Sec. 2.3: a circuit U = D_m V_m ... V_1 D_0 on |0^n>, tasks (a) sampling
 * and (b) norm estimation):
 *
 *   lrs_lower_circuit   split a circuit into Clifford gates and
 *                       sum-over-Cliffords slots (Sec. 2.3.2, Eq. (Rtheta),
 *                       Eq. (CCZ_decomposition)); host only
 *   lrs_init_terms      choose every term's slot choices (exact enumeration
 *                       or Lemma (Sparsification), Sec. 5.2), set b_alpha and
 *                       reset every CH-form to |0^n>
 *   lrs_apply_clifford  push every term through a gate list (Sec. 4.1 update
 *                       rules, Eqs. (H1)-(H7), Prop. (prop:H), projectors)
 *   lrs_amplitude       <x|psi> for a batch of x (Eqs. (amplitude),
 *                       (amplitude1))
 *   lrs_norm_estimate   eta_l = 2^n |<phi_{A_l}|psi>|^2 for L random
 *                       equatorial states (Sec. 4.3, Lemmas (Norm
 *                       Estimation), (Inner Product), (Exponential Sum))
 *   lrs_chains_init / lrs_metropolis_step
 *                       single-flip Metropolis chains with the incremental
 *                       Pauli update Q_y = (U_C^-1 X_j U_C) Q_x (Sec. 4.2)
 *
 * Conventions
 *   - Every function returns lrs_status; nothing throws across the ABI.  On
 *     error lrs_last_error() returns a message (thread-local, valid until the
 *     next call on the same thread).
 *   - A basis string x is a uint64 with bit j holding qubit j; bits >= n must
 *     be zero.
 *   - Pointers named *_dev are device pointers (cudaMalloc'ed or from a
 *     framework allocator) owned by the caller; *_host are host pointers owned
 *     by the caller.  The library owns the term storage inside lrs_ctx.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Device-side
 *     calls are stream-ordered and asynchronous; they return after enqueuing
 *     unless stated otherwise.  A context must not be used from two host
 *     threads at once.
 *   - Graph capture: lrs_reinit_terms, lrs_apply_clifford (a gate list of at
 *     most 7680 gates), lrs_apply_clifford_batch (the gate lists of its previous
 *     call), lrs_amplitude, lrs_amplitude_batch, lrs_norm_estimate (mean_host
 *     NULL), lrs_sample_terms, lrs_chains_init and lrs_metropolis_step enqueue
 *     only kernel launches and device copies once a first, uncaptured call of the
 *     same sizes has sized the context's buffers and set its kernels' attributes,
 *     so a stream that runs them can be captured into one CUDA graph (Metropolis
 *     steps are then captured as plain launches).  The graph keeps the device
 *     addresses of the context's buffers: replay it only while no later call on
 *     those contexts has needed larger buffers (more strings, chains, L or terms),
 *     and before lrs_destroy.  Scalars (seeds, step0) are fixed at capture.
 *   - Random numbers are drawn on the device from SplitMix64 in counter mode
 *     (Steele, Lea and Flood 2014):
 *        mix(z) = z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
 *                 z *= 0x94D049BB133111EB; z ^= z>>31
 *        rand64(seed, stream, i) = mix(mix(seed ^ mix(stream + G)) + (i+1) G),
 *        G = 0x9E3779B97F4A7C15; uniform double = (rand64 >> 11) * 2^-53.
 */
#ifndef LRSTAB_H
#define LRSTAB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lrs_ctx lrs_ctx;

typedef enum {
    LRS_OK = 0,
    LRS_ERR_ARG = -1,         /* invalid argument (message says which)          */
    LRS_ERR_OOM = -2,         /* device allocation failed                       */
    LRS_ERR_CUDA = -3,        /* a CUDA runtime call or launch failed           */
    LRS_ERR_TIMEOUT = -4,     /* a device-side wait gave up                     */
    LRS_ERR_STATE = -5,       /* call out of order (e.g. no terms initialised)  */
    LRS_ERR_UNSUPPORTED = -6  /* valid request outside what this build supports */
} lrs_status;

/* ---- lowered gates (what the device executes) ------------------------------- */
enum {
    LRS_OP_H = 0,    /* Hadamard on q                                          */
    LRS_OP_S = 1,    /* S = diag(1, i) on q                                    */
    LRS_OP_SDG = 2,  /* S^dagger on q                                          */
    LRS_OP_Z = 3,    /* Z on q                                                 */
    LRS_OP_CX = 4,   /* CX, control q, target r                                */
    LRS_OP_CZ = 5,   /* CZ on q, r                                             */
    LRS_OP_P0 = 6,   /* projector (I + Z_q)/2                                  */
    LRS_OP_P1 = 7,   /* projector (I - Z_q)/2                                  */
    LRS_OP_SLOT = 8  /* non-Clifford slot number r: each term applies its K_j  */
};

typedef struct {
    uint8_t op;   /* LRS_OP_*                                   */
    uint8_t q;    /* first qubit                                */
    uint16_t r;   /* second qubit (CX, CZ) or slot index (SLOT) */
} lrs_gate;

#define LRS_MAX_CHOICES 8

/* V = sum_j c_j K_j for one non-Clifford gate; K_j is the gate sub-list
 * k_gates[k_off[j] .. k_off[j] + k_len[j]) (Clifford or projector gates only). */
typedef struct {
    int32_t n_choices;                 /* 1..LRS_MAX_CHOICES */
    int32_t k_off[LRS_MAX_CHOICES];
    int32_t k_len[LRS_MAX_CHOICES];
    double c_re[LRS_MAX_CHOICES];
    double c_im[LRS_MAX_CHOICES];
} lrs_slot;

/* ---- circuit description (host) --------------------------------------------- */
enum {
    LRS_C_H = 0, LRS_C_S = 1, LRS_C_SDG = 2, LRS_C_Z = 3, LRS_C_CX = 4, LRS_C_CZ = 5,
    LRS_C_T = 6,    /* diag(1, e^{i pi/4})                       */
    LRS_C_RZ = 7,   /* exp(-i theta Z / 2)                       */
    LRS_C_CCZ = 8   /* doubly controlled Z on q[0], q[1], q[2]   */
};

/* How a CCZ is decomposed (Sec. 2.3.2). */
enum {
    LRS_CCZ_PROJECTOR = 0,  /* exact 2-term form CCZ = I - 2 P1 P1 P1           */
    LRS_CCZ_SUM8 = 1        /* 8-term Clifford form with xi = 16/9 (Eq.
                               (CCZ_decomposition), prefactor 1/6)            */
};

typedef struct {
    int32_t kind;      /* LRS_C_*                    */
    int32_t q[3];      /* qubits (unused ones ignored) */
    double theta;      /* LRS_C_RZ angle             */
} lrs_circuit_op;

/* Lower a circuit to Clifford gates plus LRS_OP_SLOT entries and slot tables
 * (Sec. 2.3.2).  T and RZ(theta) use the optimal 2-term form of Eq. (Rtheta)
 * ((cos - sin) I + sqrt2 e^{-i pi/4} sin S for theta >= 0, its conjugate on
 * (I, S^dagger) for theta < 0; T carries its global phase e^{i pi/8}).
 * Host only, no GPU needed.  Output arrays are caller-owned with the given
 * capacities; the used counts are written to *n_gates, *n_slots, *n_k_gates.
 * Errors: LRS_ERR_ARG for a bad op, qubit >= n_qubits, or a capacity too small
 * (the counts then hold the sizes needed).                                    */
lrs_status lrs_lower_circuit(int32_t n_qubits, const lrs_circuit_op* ops_host, int64_t n_ops,
                             int32_t ccz_mode,
                             lrs_gate* gates_host, int64_t gates_cap, int64_t* n_gates,
                             lrs_slot* slots_host, int64_t slots_cap, int64_t* n_slots,
                             lrs_gate* k_gates_host, int64_t k_cap, int64_t* n_k_gates);

/* Fixed-sample gadget form of the same circuit (Sec. 2.3.1, Eqs. (singlegate),
 * (Uidentity)): each non-Clifford op V_j on t_j qubits (T, RZ: 1; CCZ: 3) gets t_j
 * ancillas, numbered from n on in the order of the ops, prepared in the magic state
 * V_j |+^t_j> (H on each ancilla, then V_j's sum-over-Cliffords slot on the
 * ancillas with every coefficient times 2^{t_j/2}); V_j itself becomes
 * CX(q_k, a_k) for its qubits q_k and ancillas a_k; at the end every ancilla is
 * post-selected on 0 by the projector (I + Z)/2.  The state on *n_total = n + tau
 * <= 64 qubits is then exactly (U|0^n>) (x) |0^tau> (ancilla bits of x are 0).
 * Outputs as lrs_lower_circuit.                                                  */
lrs_status lrs_lower_gadget(int32_t n_qubits, const lrs_circuit_op* ops_host, int64_t n_ops, int32_t ccz_mode,
                            int32_t* n_total, lrs_gate* gates_host, int64_t gates_cap, int64_t* n_gates,
                            lrs_slot* slots_host, int64_t slots_cap, int64_t* n_slots,
                            lrs_gate* k_gates_host, int64_t k_cap, int64_t* n_k_gates);

/* Sizes of the decomposition a slot table defines (Sec. 2.3.2, Lemma
 * (Sparsification)), host only: *l1_norm = ||c||_1 = prod_p sum_j |c_j^(p)| (the
 * sparsification error is delta^2 = ||c||_1^2 / k for k sampled terms) and
 * *exact_chi = prod_p (number of nonzero c_j^(p)), the number of terms of the
 * exact enumeration, or -1 when it exceeds 2^62; *log2_exact_chi its base-2
 * logarithm (any output may be NULL).
 * Errors: LRS_ERR_ARG (n_slots < 0, NULL table, n_choices out of range).     */
lrs_status lrs_decomposition_stats(const lrs_slot* slots_host, int64_t n_slots, double* l1_norm,
                                   int64_t* exact_chi, double* log2_exact_chi);

/* ---- context ------------------------------------------------------------------ */
/* Options of a new context (no counterpart in the paper).  `size` must be
 * sizeof(lrs_options) as the caller compiled it (later versions may append fields);
 * bit i of `tuning_mask` gives launch knob i (an LRS_TUNE_* value) the initial value
 * tuning[i], exactly as lrs_set_tuning would; other knobs keep their defaults.
 * Everything else a call needs travels with the call.                          */
#define LRS_OPTIONS_TUNING 16
typedef struct {
    int32_t size;
    uint32_t tuning_mask;
    int64_t tuning[LRS_OPTIONS_TUNING];
} lrs_options;

/* Create a context for n_qubits (1..64) on CUDA device `device`; opts may be NULL
 * (every knob at its default, which suits a GB300).  *out is owned by the caller
 * and released with lrs_destroy.
 * Errors: LRS_ERR_ARG (n out of range, opts->size smaller than the fields read, a
 * tuning value lrs_set_tuning rejects; no context is created), LRS_ERR_CUDA (bad
 * device).                                                                   */
lrs_status lrs_create(int32_t device, int32_t n_qubits, const lrs_options* opts, lrs_ctx** out);

/* Free all device storage of the context.  Synchronises the device.  NULL ok. */
lrs_status lrs_destroy(lrs_ctx* ctx);

const char* lrs_last_error(void);

/* ---- terms ------------------------------------------------------------------- */
enum { LRS_MODE_EXACT = 0, LRS_MODE_SPARSIFY = 1 };

/* Allocate (or reuse) storage for the chi terms with global indices
 * alpha = alpha0 .. alpha0 + chi - 1 of a decomposition with chi_total terms,
 * and initialise them (a context may hold a contiguous shard of the terms).
 * EXACT: chi_total must equal prod_p (number of nonzero c_j of slot p); term
 *   alpha takes the mixed-radix digits of alpha over each slot's nonzero
 *   choices (slot 0 least significant) and b_alpha = prod_p c_{j_p}.
 * SPARSIFY (Lemma (Sparsification)): slot p of term alpha takes the first j
 *   with u < sum_{i<=j} |c_i| / ||c^(p)||_1, u = uniform(seed, alpha, p);
 *   b_alpha = (||c||_1 / chi_total) prod_p c_{j_p} / |c_{j_p}|,
 *   ||c||_1 = prod_p ||c^(p)||_1.
 * Every CH-form is reset to |0^n> (G = F = I, M = 0, gamma = v = s = 0,
 * omega = 1).  b_alpha is stored as FP32 complex.  Slots and k_gates are
 * copied; host arrays may be freed on return.  Blocks until the tables are
 * uploaded, then runs asynchronously on `stream`.
 * Errors: LRS_ERR_ARG (chi < 1, alpha0 < 0, alpha0 + chi > chi_total, bad
 * slot tables, qubit >= n, EXACT chi_total mismatch), LRS_ERR_OOM.           */
lrs_status lrs_init_terms(lrs_ctx* ctx, const lrs_slot* slots_host, int64_t n_slots,
                          const lrs_gate* k_gates_host, int64_t n_k_gates,
                          int64_t chi_total, int64_t alpha0, int64_t chi, int32_t mode,
                          uint64_t seed, void* stream);

/* Re-initialise the terms of the last lrs_init_terms (or lrs_copy_terms) call from
 * the slot tables already on the device: the same term range, mode and b_alpha
 * scale, the choices of SPARSIFY drawn again with `seed` (Lemma (Sparsification)),
 * every CH-form reset to |0^n>.  One kernel launch, no copy and no host wait, so
 * it can be captured into a CUDA graph (see "Graph capture" above).  Chains are
 * dropped (lrs_chains_init again).
 * Errors: LRS_ERR_STATE (no earlier lrs_init_terms), LRS_ERR_CUDA.            */
lrs_status lrs_reinit_terms(lrs_ctx* ctx, uint64_t seed, void* stream);

/* Apply the lowered gate list to every term (left multiplications for
 * S, S^dagger, Z, CX, CZ; Eqs. (H1)-(H7) with Prop. (prop:H) for H; the
 * projective-gate rule of Sec. 4.1 for P0/P1; each term's own K_j for
 * LRS_OP_SLOT).  The gate list is read before return (it travels as kernel launch
 * parameters, 7680 gates per launch); the work runs asynchronously on `stream`.
 * Readings: rules of one gate are simultaneous; "the first qubit" of V_b is
 * the lowest index; the single-qubit rewrite takes a = 0 when b = 0.
 * Errors: LRS_ERR_ARG (qubit >= n, q == r, unknown op, slot index out of
 * range), LRS_ERR_STATE (no terms).                                          */
lrs_status lrs_apply_clifford(lrs_ctx* ctx, const lrs_gate* gates_host, int64_t n_gates,
                              void* stream);

/* The same as lrs_apply_clifford with the lowered circuit on freshly initialised
 * EXACT-mode terms (the whole decomposition, alpha0 = 0), sharing the work of common
 * choice prefixes: term alpha takes choice digit j_p = (alpha / R_p) mod r_p of slot p
 * (r_q its number of nonzero choices, R_p = r_0 ... r_{p-1}; the enumeration of
 * lrs_init_terms), so before slot p only R_p distinct states exist.  Each Clifford
 * segment runs on those R_p states; at a run of consecutive slots p..p+k-1 they are
 * copied out to R_{p+k} terms, which take the run's slots and the next segment in
 * one launch.  The gate list must hold every slot exactly once, in order 0, 1, ..
 * The resulting terms equal lrs_apply_clifford's bit for bit; the work of segment p
 * falls from chi to R_p terms (the paper applies each term's gates separately).
 * LRS_ERR_STATE if the terms are not fresh EXACT-mode terms of the whole
 * decomposition or the slots' radices do not multiply to chi (checked before any
 * launch).  The gate list is read before return; the work runs asynchronously.      */
lrs_status lrs_apply_circuit_shared(lrs_ctx* ctx, const lrs_gate* gates_host, int64_t n_gates, void* stream);

/* Batched form of lrs_apply_clifford for several circuits (contexts on one
 * device, e.g. decompositions of uneven chi): context i receives gate list i
 * (copied before return).  All tiles of all circuits run in one launch (up to
 * 12 circuits per launch); each block finds its circuit from its block index.
 * Same rules and errors
 * as lrs_apply_clifford, plus LRS_ERR_ARG for repeated contexts or contexts
 * on different devices.                                                      */
lrs_status lrs_apply_clifford_batch(lrs_ctx* const* ctxs, const lrs_gate* const* gates_host,
                                    const int64_t* n_gates, int32_t count, void* stream);

/* out_dev[2i], out_dev[2i+1] = Re, Im of <x_i|psi> = sum_alpha b_alpha
 * <x_i|phi_alpha> for i < batch (Eq. (amplitude1) per term).  Per-term values
 * are exact Z8 phases times powers of sqrt2 times b_alpha; the chi-sum is a
 * per-thread compensated (Kahan) FP32 sum over a tile of terms, then an FP64
 * tree sum across tiles.
 * err_est_dev (may be NULL; device, batch floats): a rigorous bound on
 * |out_i - exact chi-sum of the stored coefficients|,
 *   err_i = (8u + 8 t u^2)(1 + t u)(1 + 1e-4) M_i + n_tiles 2^-52 P_i,
 * u = 2^-24, t the tile length, M_i = sum over the terms that contribute at x_i of
 * |b_alpha <x_i|phi_alpha>|, P_i = sum of the tiles' |FP32 partial sum|: 4u per
 * addend (FP32 coefficient and phase factors), 2 sqrt2 u for the Kahan sum of a
 * complex tile, u for its final rounding, the FP64 tile sum.  It is a worst case,
 * linear in M_i: where the terms cancel (sparsified states, M_i >> |out_i|) the
 * observed error is far below it.  Asking for it costs one FP32 add per
 * contributing (x, term) and an extra FP32 partial per (x, tile).
 * x_dev: batch uint64 basis strings.  batch = 0 is a no-op.
 * Errors: LRS_ERR_ARG (batch < 0, NULL pointers), LRS_ERR_STATE.            */
lrs_status lrs_amplitude(lrs_ctx* ctx, const uint64_t* x_dev, int64_t batch, double* out_dev,
                         float* err_est_dev, void* stream);

/* lrs_amplitude for several circuits (contexts with the same qubit count on one
 * device, e.g. decompositions of uneven chi) in two launches: one amplitude launch
 * covering every circuit's term tiles (at most 12 circuits per launch; more take
 * further launches) and one FP64 reduction for all their strings.  Circuit i gets
 * batch[i] strings x_dev[i] and writes out_dev[i] (2 batch[i] doubles), with the tile
 * plan of its own lrs_amplitude call, so its values equal that call's bit for bit.
 * Errors: LRS_ERR_ARG (NULL or repeated contexts, different devices or widths),
 * LRS_ERR_STATE (a context without terms).                                       */
lrs_status lrs_amplitude_batch(lrs_ctx* const* ctxs, const uint64_t* const* x_dev, const int64_t* batch,
                               double* const* out_dev, int32_t count, void* stream);

/* Same result as lrs_amplitude, but the call allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc when they need amplitudes (for example a serving
 * loop whose framework allocator already holds the device memory, or code
 * that must avoid the allocator's latency and locks).  The partial sums go to
 * a fixed 16 MiB array in the library's device memory (2^21 float2 entries),
 * present on every GPU that loads the library until the process exits.
 * Limit: batch * n_tiles <= 2^21 partial sums, where n_tiles, the number of
 * term tiles the kernel uses, is at most min(ceil(b * SMs / ceil(batch / 1024)),
 * ceil(chi_padded / 32)) with b = LRS_TUNE_AMP_BLOCKS_PER_SM (default 8: 304
 * tiles for batch 4096 on a 152-SM GPU; tiles are whole multiples of 8 terms);
 * larger requests return LRS_ERR_ARG.
 * Any batch above 2^21 is rejected.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the one array and each call overwrites every entry it
 * reads, so nothing needs clearing; calls that overlap on the GPU (for
 * example on two streams, or from two contexts) race on the array and must be
 * serialised by the caller.
 * Errors: as lrs_amplitude, plus LRS_ERR_ARG when the batch is too large.   */
lrs_status lrs_amplitude_noalloc(lrs_ctx* ctx, const uint64_t* x_dev, int64_t batch,
                                 double* out_dev, void* stream);

/* eta_dev[l] = 2^n |<phi_{A_l}|psi>|^2 for l < L (Lemma (Norm Estimation)),
 * A_l in M_n drawn from rand64(seed, l, i): word 0 = low bits of diag(A),
 * word 1 = high bits, words 2.. = strict upper triangle in row-major order.
 * Each <phi_{A_l}|phi_alpha> is exact (Lemma (Inner Product) with the exact
 * exponential sum of Lemma (Exponential Sum)); the chi-sum is FP32 then FP64;
 * eta is FP64.  If mean_host is not NULL the call synchronises `stream` and
 * writes the mean of the L values.
 * Errors: LRS_ERR_ARG (L < 1), LRS_ERR_STATE.                                */
lrs_status lrs_norm_estimate(lrs_ctx* ctx, int64_t L, uint64_t seed, double* eta_dev,
                             double* mean_host, void* stream);

/* Term-sharded norm estimation (Sec. 4.3: <phi_A|psi> is a sum over terms).
 *   lrs_norm_overlaps           ov_dev[2l], ov_dev[2l+1] = Re, Im of
 *                               2^{n/2} <phi_{A_l}|psi_ctx> over ctx's terms, the same
 *                               A_l and sums as lrs_norm_estimate (ov_dev: 2 L doubles)
 *   lrs_norm_eta_from_overlaps  eta_dev[l] = |ov_dev[l]|^2 for overlaps summed over the
 *                               shards (2^n |<phi_{A_l}|psi>|^2, as lrs_norm_estimate)
 * Both are stream-ordered.  Errors: LRS_ERR_ARG (L < 1, NULL), LRS_ERR_STATE.    */
lrs_status lrs_norm_overlaps(lrs_ctx* ctx, int64_t L, uint64_t seed, double* ov_dev, void* stream);
lrs_status lrs_norm_eta_from_overlaps(lrs_ctx* ctx, int64_t L, const double* ov_dev, double* eta_dev,
                                      void* stream);

/* Draw count basis strings from the terms (Sec. 4.1, "Simulating
 * measurements"): term alpha = floor(rand64(seed, i, 0) * chi / 2^64)
 * (uniform), w = s ^ (rand64(seed, i, 1) & v), x = w G^T.  Writes x_dev[i]
 * and, if alpha_dev is not NULL, alpha_dev[i].                               */
lrs_status lrs_sample_terms(lrs_ctx* ctx, int64_t count, uint64_t seed, uint64_t* x_dev,
                            int64_t* alpha_dev, void* stream);

/* ---- Metropolis (Sec. 4.2) ------------------------------------------------------ */
/* Start n_chains chains at x_dev[c]: computes Q_x for every (chain, term) and
 * P(x) = |<x|psi>|^2.  Needs n <= 62 (Q = i^mu X(u) Z(w) is packed in 12 bytes for
 * n <= 40, 16 bytes above).  Storage is n_chains * chi_padded * 12 (or 16) bytes,
 * owned by the context.
 * Errors: LRS_ERR_ARG, LRS_ERR_STATE, LRS_ERR_UNSUPPORTED (n > 62), LRS_ERR_OOM. */
lrs_status lrs_chains_init(lrs_ctx* ctx, int64_t n_chains, const uint64_t* x_dev, void* stream);

/* Run `steps` Metropolis steps on every chain.  Step t (global index
 * step0 + t) of chain c proposes y = x ^ e_j with j = (hi32(rand64(seed, c,
 * 2t)) * n) >> 32 and accepts if P(y) >= P(x), else iff
 * uniform(seed, c, 2t+1) < P(y)/P(x) (FP64).  Optional outputs (device, may
 * be NULL): x_out_dev[c] and p_out_dev[c] after the last step, trace_dev
 * [t * n_chains + c] = x after step t.  Runs asynchronously on `stream`.
 * Errors: LRS_ERR_ARG (steps < 0), LRS_ERR_STATE (chains not initialised),
 * LRS_ERR_TIMEOUT (an earlier call's propose kernel gave up waiting, after 1 s, for
 * the copies of its inputs into shared memory; that call's results are invalid).  */
lrs_status lrs_metropolis_step(lrs_ctx* ctx, int64_t steps, uint64_t seed, int64_t step0,
                               uint64_t* x_out_dev, double* p_out_dev, uint64_t* trace_dev,
                               void* stream);

/* Term-sharded Metropolis.  Every estimator of Sec. 4 is a sum over terms, so a
 * decomposition can be split into contiguous term ranges (lrs_init_terms' alpha0 /
 * chi_total), one per context (one per GPU of a job).  The chain step then has one
 * exchange: each shard forms its partial amplitudes of the proposals, the caller sums
 * them over the shards (an all-reduce of 2 C doubles), and every shard takes the same
 * FP64 decision from the same draws.
 *   lrs_chains_set_amplitude  after lrs_chains_init on every shard with the same
 *                             strings: P(x_c) = |amp_dev[c]|^2 from the summed
 *                             amplitudes (amp_dev: 2 C doubles, Re/Im; device)
 *   lrs_metropolis_propose    step `step` (global index) of lrs_metropolis_step's draws:
 *                             applies the previous step's accepted flips to the Pauli
 *                             states, draws j, writes the shard's sum over its terms of
 *                             b <y_c|phi> into amp_dev (2 C doubles, not squared)
 *   lrs_metropolis_accept     the FP64 accept rule of lrs_metropolis_step on the summed
 *                             amp_dev of the same step; trace_dev (may be NULL) gets x
 *                             after the step
 * Steps alternate propose, accept; lrs_metropolis_step may follow on the same chains.
 * Errors: LRS_ERR_STATE (no chains, or an accept without the propose of its step),
 * LRS_ERR_ARG, LRS_ERR_TIMEOUT (as lrs_metropolis_step).                        */
lrs_status lrs_chains_set_amplitude(lrs_ctx* ctx, const double* amp_dev, void* stream);
lrs_status lrs_metropolis_propose(lrs_ctx* ctx, uint64_t seed, int64_t step, double* amp_dev, void* stream);
lrs_status lrs_metropolis_accept(lrs_ctx* ctx, const double* amp_dev, uint64_t seed, int64_t step,
                                 uint64_t* trace_dev, void* stream);

/* ---- median of means and marginal sampling (end of Sec. 4.3) ------------------ */
/* Copy the terms of src (tableaux, gamma, v, s, omega, coefficients, slot choices
 * and slot tables) into dst, which must have the same qubit count and device;
 * dst's storage is reallocated when its capacity differs, and its chains are
 * dropped.  Stream-ordered.                                                     */
lrs_status lrs_copy_terms(lrs_ctx* dst, const lrs_ctx* src, void* stream);
/* ||psi||^2 estimated as the median of K empirical means of eta_A, group g using
 * the equatorial states l = g L .. g L + L - 1 of lrs_norm_estimate's stream
 * `seed` (the median of an even K is the mean of the two middle means).  L, K >= 1,
 * L K <= 2^22.  Writes *estimate_host; synchronises the stream.                  */
lrs_status lrs_norm_median_of_means(lrs_ctx* ctx, int64_t L, int32_t K, uint64_t seed,
                                    double* estimate_host, void* stream);
/* Sparsification certificate (Lemma (Sparsification tail bound), Sec. 5.2): for the
 * sparsified state Omega held by ctx (chi_total sampled terms of the decomposition its
 * slot tables define), ||psi - Omega||^2 <= <Omega|Omega> - 1 + delta^2 with high
 * probability, delta^2 = ||c||_1^2 / chi_total.  <Omega|Omega> is estimated as
 * lrs_norm_median_of_means(L, K, seed).  The bound is informative only when the
 * estimate's own error is well below delta^2: `conclusive` is 1 when twice the
 * standard error of the mean of the L K values eta_l is below delta^2.  Writes
 * *out_host; synchronises the stream.  Errors: as lrs_norm_median_of_means.     */
typedef struct {
    double omega_norm2;   /* median of K means of L eta values: <Omega|Omega>      */
    double stderr_mean;   /* standard error of the mean of the L K eta values       */
    double delta2;        /* ||c||_1^2 / chi_total                                  */
    double bound;         /* omega_norm2 - 1 + delta2                               */
    double bound_upper;   /* omega_norm2 + 2 stderr_mean - 1 + delta2               */
    int32_t conclusive;   /* 2 stderr_mean < delta2                                 */
    int32_t reserved;
} lrs_certificate;
lrs_status lrs_sparsification_certificate(lrs_ctx* ctx, int64_t L, int32_t K, uint64_t seed,
                                          lrs_certificate* out_host, void* stream);

/* Chain-rule sample of the bits on qubits[0..w) by norm estimation: step i fixes
 * the bits drawn so far by the projectors (I + (-1)^x Z_q)/2 (Sec. 4.1, projective
 * gates), estimates both branches p_b = ||Pi_{x_<i, b} psi||^2 by
 * lrs_norm_median_of_means(L, K, seed_i) with seed_i = rand64(seed, 2^41 + i, 0)
 * (the same equatorial states for both branches), and sets bits_host[i] = 1 iff
 * uniform(seed, 2^42 + i, 0) < p_1 / (p_0 + p_1) (0 when p_0 + p_1 <= 0).
 * probs_host (may be NULL) receives p_0, p_1 of every step.  work0 and work1 are
 * two further contexts with the same qubit count (their terms are overwritten);
 * ctx is not modified.  Distinct qubits, 0 <= w <= n.  Synchronises the stream. */
lrs_status lrs_marginal_sample(lrs_ctx* ctx, lrs_ctx* work0, lrs_ctx* work1, const int32_t* qubits_host,
                               int32_t w, int64_t L, int32_t K, uint64_t seed, uint8_t* bits_host,
                               double* probs_host, void* stream);

/* ---- learned proposal (MADE network; the paper proposes single flips only) ----- */
/* The paper's Metropolis chain (Sec. 4.2) uses single bit flips and notes that
 * its mixing time is generally unknown.  These calls add an independent
 * proposal y ~ q learned from chain samples: q(x) = prod_i q(x_i | x_<i), a
 * masked autoencoder (MADE) n -> H -> H -> n with ReLU hidden layers and
 * Bernoulli outputs; input degree i+1, hidden degree m(k) = (k mod (n-1)) + 1,
 * masks W1[k,i]: m(k) >= i+1, W2[k2,k1]: m(k2) >= m(k1), W3[i,k]: i+1 > m(k).
 * Products run on the tensor cores with BF16 operands (round-to-nearest-even
 * copies of FP32 master weights, BF16 activations and backward signals) and
 * FP32 accumulation; biases, logits, gradients and AdamW state are FP32.
 * Parameters are packed as W1 [H][n], b1 [H], W2 [H][H], b2 [H], W3 [n][H],
 * b3 [n] (row-major, FP32).                                                    */
typedef struct lrs_mlp lrs_mlp;

/* 2 <= n <= 64, hidden a multiple of 64 in 64..4096.  Parameters start at 0. */
lrs_status lrs_mlp_create(int32_t device, int32_t n, int32_t hidden, lrs_mlp** out);
lrs_status lrs_mlp_destroy(lrs_mlp* mlp);
lrs_status lrs_mlp_info(const lrs_mlp* mlp, int32_t* n, int32_t* hidden, int64_t* n_params);
/* GEMM kernel used by every product of the network (default TCGEN05):
 *   LRS_MLP_GEMM_TCGEN05   5th-generation tensor cores: one thread issues
 *                          tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) on
 *                          128 x 64 tiles from shared memory, the accumulator
 *                          lives in tensor memory, completion arrives on an
 *                          mbarrier whose wait is bounded (a wait that gives
 *                          up sets a flag that lrs_mlp_get_params and
 *                          lrs_mlp_set_gemm report as LRS_ERR_TIMEOUT, and so
 *                          does the first forward, backward, train or sample
 *                          call that starts after the call that set it has
 *                          completed: each copies the flag to the host,
 *                          asynchronously, when it has enqueued its work)
 *   LRS_MLP_GEMM_MMA_SYNC  warp-level mma.sync m16n8k16 on 64 x 64 tiles
 * Both accumulate exact BF16 products in FP32; results differ only in the
 * order of the FP32 additions.  Synchronises the device.                       */
enum { LRS_MLP_GEMM_TCGEN05 = 0, LRS_MLP_GEMM_MMA_SYNC = 1 };
lrs_status lrs_mlp_set_gemm(lrs_mlp* mlp, int32_t kind);
lrs_status lrs_mlp_get_gemm(const lrs_mlp* mlp, int32_t* kind);
/* Upload packed FP32 parameters (host, n_params floats); resets AdamW state. */
lrs_status lrs_mlp_set_params(lrs_mlp* mlp, const float* params_host);
/* Download packed parameters and/or the last gradients (host, may be NULL).
 * Synchronises the device.                                                     */
lrs_status lrs_mlp_get_params(lrs_mlp* mlp, float* params_host, float* grads_host);
/* logits_dev [batch][n] (may be NULL) and log q(x) per row (may be NULL) for
 * basis strings x_dev[batch].                                                  */
lrs_status lrs_mlp_forward(lrs_mlp* mlp, const uint64_t* x_dev, int64_t batch, float* logits_dev,
                           float* logq_dev, void* stream);
/* Gradients of the mean negative log-likelihood over x_dev[batch] (kept in the
 * network; read with lrs_mlp_get_params); *loss_dev = mean NLL (may be NULL). */
lrs_status lrs_mlp_backward(lrs_mlp* mlp, const uint64_t* x_dev, int64_t batch, float* loss_dev,
                            void* stream);
/* lrs_mlp_backward followed by one AdamW step (decoupled weight decay wd,
 * bias-corrected moments) on the masked gradients.                            */
lrs_status lrs_mlp_train_step(lrs_mlp* mlp, const uint64_t* x_dev, int64_t batch, float lr,
                              float beta1, float beta2, float eps, float wd, float* loss_dev,
                              void* stream);
/* count samples y ~ q, bit by bit in qubit order: bit i of sample k is
 * [u < sigmoid(logit_i)] with u = uniform(seed, 2^40 + sample0 + k, i)
 * (FP32 compare); logq_dev[k] = log q(y_k).                                   */
lrs_status lrs_mlp_sample(lrs_mlp* mlp, int64_t count, uint64_t seed, int64_t sample0,
                          uint64_t* y_dev, float* logq_dev, void* stream);

/* Metropolis-Hastings with the learned independent proposal on the chains of
 * lrs_chains_init: step t (global step0 + t) draws y_c ~ q (sample index
 * t * n_chains + c), evaluates P(y) = |<y|psi>|^2 exactly by lrs_amplitude's
 * kernels, and accepts with probability min(1, P(y) q(x) / (P(x) q(y))) (FP64;
 * uniform(seed, c, t)); a chain at P(x) = 0 always accepts.  Outputs as
 * lrs_metropolis_step; accepts_dev[c] (may be NULL) is incremented per accepted
 * move.  A later lrs_metropolis_step first rebuilds the single-flip state.     */
lrs_status lrs_metropolis_learned(lrs_ctx* ctx, lrs_mlp* mlp, int64_t steps, uint64_t seed,
                                  int64_t step0, uint64_t* x_out_dev, double* p_out_dev,
                                  uint64_t* trace_dev, int64_t* accepts_dev, void* stream);

/* ---- failure-path test support (no counterpart in the paper) ------------------- */
/* Every device-side wait of the library is bounded (1 s); a kernel whose wait runs out
 * records it in a flag, waits (bounded) for the copies it has in flight, frees what it
 * holds and returns, and the next synchronising call reports LRS_ERR_TIMEOUT.  These
 * calls let a test make one such wait run out without faulting anything: each sets a
 * one-shot request that the next launch of the kernel concerned takes in one block,
 * whose first shared-memory stage then expects 16 bytes more than its copies deliver.
 *   lrs_debug_inject_wait_timeout      the next Metropolis propose kernel of ctx: that
 *                                      launch ends about 2 s later with one block's
 *                                      partial sums unwritten; the next
 *                                      lrs_metropolis_step returns LRS_ERR_TIMEOUT
 *                                      (re-initialise the chains after it)
 *   lrs_mlp_debug_inject_wait_timeout  the next tcgen05 GEMM of mlp: one output tile is
 *                                      not written; lrs_mlp_get_params or
 *                                      lrs_mlp_set_gemm then returns LRS_ERR_TIMEOUT
 * A later call of the same kind runs normally.                                       */
lrs_status lrs_debug_inject_wait_timeout(lrs_ctx* ctx);
lrs_status lrs_mlp_debug_inject_wait_timeout(lrs_mlp* mlp);

/* ---- export (checkpoint / bit-exact parity) ----------------------------------- */
/* Copy local terms [first, first + count) (global index alpha0 + first ..) to host arrays (each may be NULL):
 *   F, G, M: count * n uint64, term-major (row p of term i at [i*n + p]);
 *   gamma: count * n bytes (0..3); v, s: count uint64;
 *   omega: count int32 = k | zero << 3 | h << 8 (omega = 0 if zero else
 *          e^{i pi k/4} 2^{-h/2});
 *   coef: count * 2 float (Re, Im of b_alpha);
 *   choice: count * n_slots bytes (choice j_p of slot p at [i*n_slots + p]).
 * Synchronises the device.                                                   */
lrs_status lrs_export_terms(lrs_ctx* ctx, int64_t first, int64_t count, uint64_t* F_host,
                            uint64_t* G_host, uint64_t* M_host, uint8_t* gamma_host,
                            uint64_t* v_host, uint64_t* s_host, int32_t* omega_host,
                            float* coef_host, uint8_t* choice_host);

/* ---- measurement support ----------------------------------------------------- */
/* Integer-pipe probe (no counterpart in the paper): runs a kernel of
 * independent 32-bit LOP3 dependency chains on every SM of `device` for
 * `iters` iterations per thread and writes the sustained rate in 32-bit
 * logic operations per second to *ops_per_s (host).  Synchronises the device.
 * Used as the ALU roofline denominator next to the unit-count derivation.   */
lrs_status lrs_alu_probe(int32_t device, int64_t iters, double* ops_per_s);

/* Launch-shape knobs of a context, chosen by timing (the package's autotuner);
 * they change speed and the grouping of the FP32 partial sums, not the
 * per-term exact values.  The paper has no counterpart.
 *   LRS_TUNE_AMP_BLOCKS_PER_SM    amplitude grid target, blocks per SM (1..64, 8)
 *   LRS_TUNE_NORM_MAX_TILES       norm estimate, maximum term tiles (1..2^20, 2048)
 *   LRS_TUNE_MC_CHAINS_PER_BLOCK  Metropolis chains per block (1..64, 64)
 *   LRS_TUNE_NORM_MAX_FOLDS       norm estimate: a term with n - |v| <= this
 *                                 value (-1..12, 12) evaluates its exponential
 *                                 sum over y = G x, i.e. the form y^T (A+J) y
 *                                 plus 2 (F s + (A+J) G s) . y restricted to the
 *                                 n - |v| constraints (F^T y)_k = 0, k not in v,
 *                                 instead of forming K = G^T (A+J) G; -1 forms
 *                                 K for every term.  Both give the same exact
 *                                 per-term value.
 *   LRS_TUNE_MC_STAGES            Metropolis: chains whose inputs a block keeps
 *                                 in flight in shared memory (1..4, 1; 12 KB each
 *                                 for one step per pass, 20 KB for two: one stage
 *                                 leaves room for the most blocks per SM)
 *   LRS_TUNE_APPLY_LANES          apply_clifford for n > 48 (64-bit rows): lanes
 *                                 per term (1, 2 or 4; default 1).  The lanes of a
 *                                 term share its tableau in shared memory and split
 *                                 its rows, so more warps share an SM, at the cost of
 *                                 repeating the per-gate scalar work in every lane;
 *                                 results are bit-identical for every value.
 *                                 Narrower tableaux take one lane per term.
 *   LRS_TUNE_NORM_FUSE_FOLDS      norm estimate: a term that takes the y = G x
 *                                 route with n - |v| <= this value (0..8, 8) folds
 *                                 its constraints into the rows of A+J while the
 *                                 rows are formed (one pass), above it one pass
 *                                 per constraint.  Same exact per-term value.
 *   LRS_TUNE_MC_LOOKAHEAD         Metropolis flip chains: steps per pass over the
 *                                 chains' Pauli states (1 or 2, default 2).  With 2
 *                                 one pass forms <y|psi> for step t's proposal and
 *                                 for both strings step t + 1 may propose (after an
 *                                 accepted or a rejected move; proposals do not
 *                                 depend on the chain), then both decisions are taken
 *                                 in order: the same chains, bit for bit, as one step
 *                                 per pass, with half the Pauli-state reads.
 */
enum {
    LRS_TUNE_AMP_BLOCKS_PER_SM = 0,
    LRS_TUNE_NORM_MAX_TILES = 1,
    LRS_TUNE_MC_CHAINS_PER_BLOCK = 2,
    LRS_TUNE_NORM_MAX_FOLDS = 3,
    LRS_TUNE_MC_STAGES = 4,
    LRS_TUNE_APPLY_LANES = 5,
    LRS_TUNE_NORM_FUSE_FOLDS = 6,
    LRS_TUNE_MC_LOOKAHEAD = 7
};
lrs_status lrs_set_tuning(lrs_ctx* ctx, int32_t param, int64_t value);
lrs_status lrs_get_tuning(const lrs_ctx* ctx, int32_t param, int64_t* value);

/* Number of terms, qubits and slots of the context (any pointer may be NULL). */
lrs_status lrs_info(const lrs_ctx* ctx, int64_t* chi, int32_t* n_qubits, int64_t* n_slots);

#ifdef __cplusplus
}
#endif
#endif /* LRSTAB_H */
