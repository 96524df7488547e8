// Internal declarations shared by the library's translation units.
// Not part of the public ABI (see include/lrstab.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lrstab.h"

// Term storage is padded to a multiple of this many terms; padding terms are
// valid |0^n> CH-forms with b = 0, so kernels need no tail checks.
#define LRS_TERM_ALIGN 256

// Per-call parameters of the flip-chain kernels (device memory, so a captured
// graph of steps can be replayed with new values).
struct McParams {
    uint64_t seed;
    int64_t step0;
};
#define LRS_MC_GRAPH_STEPS 16

// Device copy of one slot table.
struct DevSlot {
    int32_t n_choices;
    int32_t n_nonzero;                 // radix in exact mode
    int32_t nz_idx[LRS_MAX_CHOICES];   // nonzero choices in index order
    int32_t k_off[LRS_MAX_CHOICES];
    int32_t k_len[LRS_MAX_CHOICES];
    double cdf[LRS_MAX_CHOICES];       // cumulative |c_j| / ||c||_1 (sparsify)
    double c_re[LRS_MAX_CHOICES], c_im[LRS_MAX_CHOICES];     // c_j (exact)
    double ph_re[LRS_MAX_CHOICES], ph_im[LRS_MAX_CHOICES];   // c_j / |c_j| (sparsify)
};

// Plain view of the term arrays passed to kernels by value.
struct TermsView {
    int32_t n;          // qubits
    uint64_t nmask;     // low n bits set
    int64_t chi;        // number of real terms held
    int64_t alpha0;     // global index of local term 0
    int64_t cap;        // allocated (multiple of LRS_TERM_ALIGN), row stride
    uint64_t* F;        // [n][cap]
    uint64_t* G;        // [n][cap]
    uint64_t* M;        // [n][cap]
    uint64_t* glo;      // [cap] gamma bit-plane 0 (bit p = bit 0 of gamma_p)
    uint64_t* ghi;      // [cap] gamma bit-plane 1
    uint64_t* v;        // [cap]
    uint64_t* s;        // [cap]
    uint32_t* omega;    // [cap] k | zero << 3 | h << 8
    float2* coef;       // [cap] b_alpha
    uint8_t* choice;    // [n_slots][cap]
    int64_t n_slots;
    const DevSlot* slots;
    const lrs_gate* kgates;
};

struct lrs_ctx {
    int device = 0;
    int sm_count = 0;
    int n = 0;
    uint64_t nmask = 0;
    int64_t chi = 0;
    int64_t alpha0 = 0;
    int64_t chi_total = 0;
    int64_t cap = 0;
    bool have_terms = false;
    int32_t mode = -1;              // lrs_init_terms mode of the current terms
    bool fresh = false;             // terms as lrs_init_terms left them (|0^n>, no gate applied)
    double init_scale = 0.0;        // ||c||_1 / chi_total of the last lrs_init_terms (term weights)

    uint64_t *F = nullptr, *G = nullptr, *M = nullptr;
    uint64_t *glo = nullptr, *ghi = nullptr, *v = nullptr, *s = nullptr;
    uint32_t* omega = nullptr;
    float2* coef = nullptr;
    uint8_t* choice = nullptr;
    int64_t choice_slots_cap = 0;

    int64_t n_slots = 0;
    DevSlot* slots_dev = nullptr;
    int64_t slots_cap = 0;
    lrs_gate* kgates_dev = nullptr;
    int64_t kgates_cap = 0;
    std::vector<lrs_slot> slots_host;
    std::vector<lrs_gate> kgates_host;

    lrs_gate* gates_dev = nullptr;
    int64_t gates_cap = 0;
    std::vector<lrs_gate> gates_resident;   // the specialised gate list now in gates_dev
    int64_t batch_n_gates = 0;      // gate count uploaded for a batched launch

    // scratch for partial sums
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    // launch-shape tuning (lrs_set_tuning)
    int64_t tune_amp_bps = 8;       // amplitude: target blocks per SM
    int64_t tune_norm_tiles = 2048; // norm: maximum term tiles per A-block column
    int64_t tune_mc_cg = 64;        // Metropolis: chains per block (1..64)
    int64_t tune_mc_stages = 1;     // Metropolis: chains in flight per block (1..4)
    int64_t tune_mc_lookahead = 2;  // Metropolis: steps per pass over the Pauli states (1, 2)
    int64_t tune_norm_folds = 12;   // norm: terms with n - |v| <= this sum over y = G x (-1..12)
    int64_t tune_norm_fuse = 8;     // norm: of those, n - |v| <= this fold while forming the rows (0..8)
    int64_t tune_apply_lanes = 1;   // apply_clifford, 64-bit rows (n > 48): lanes per term (1, 2, 4)
    // equatorial samples of median-of-means estimates
    double* eta_buf = nullptr;
    size_t eta_bytes = 0;
    // work table of batched launches led by this context
    void* batch_buf = nullptr;
    size_t batch_buf_bytes = 0;

    // Metropolis chains
    int64_t n_chains = 0;
    void* Q = nullptr;              // [chain][cap] Pauli states (q_store layout)
    size_t Q_bytes = 0;
    uint64_t* cx = nullptr;         // [chain] current x
    double* cp = nullptr;           // [chain] P(x) (unnormalised)
    int32_t* pend = nullptr;        // [2][chain] pending accepted flips, committed in order (-1 none)
    int64_t chains_cap = 0;
    bool q_stale = false;           // x moved by learned proposals: Q must be rebuilt
    McParams* mc_par = nullptr;     // device parameters of the flip-chain kernels
    int* mc_err_h = nullptr;        // mapped host [2]: a propose kernel gave up waiting; test request
    int* mc_err_d = nullptr;        // its device address
    void* mc_exec = nullptr;        // cudaGraphExec_t of LRS_MC_GRAPH_STEPS steps
    const void* mc_key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    void* cap_stream = nullptr;     // cudaStream_t used for graph capture
    // learned-proposal Metropolis-Hastings buffers
    uint64_t* ybuf = nullptr;       // [chain] proposals
    float* lqy = nullptr;           // [chain] log q(y)
    float* lqx = nullptr;           // [chain] log q(x)
    double* ampy = nullptr;         // [chain][2] <y|psi>
    int64_t mh_cap = 0;
    // proposals of a term-sharded step (lrs_metropolis_propose -> lrs_metropolis_accept)
    int32_t* jbuf = nullptr;
    size_t jbuf_bytes = 0;
    int64_t split_step = -1;        // step of the proposal awaiting its accept

    TermsView view() const {
        TermsView t;
        t.n = n; t.nmask = nmask; t.chi = chi; t.alpha0 = alpha0; t.cap = cap;
        t.F = F; t.G = G; t.M = M; t.glo = glo; t.ghi = ghi; t.v = v; t.s = s;
        t.omega = omega; t.coef = coef; t.choice = choice; t.n_slots = n_slots;
        t.slots = slots_dev; t.kgates = kgates_dev;
        return t;
    }
};

// ---- error reporting -----------------------------------------------------------
lrs_status lrs_fail(lrs_status st, const char* fmt, ...);
lrs_status lrs_cuda_check(cudaError_t e, const char* what);
#define LRS_CUDA(call)                                              \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return lrs_cuda_check(e_, #call);    \
    } while (0)
#define LRS_LAUNCH_CHECK(what)                                      \
    do {                                                            \
        cudaError_t e_ = cudaGetLastError();                        \
        if (e_ != cudaSuccess) return lrs_cuda_check(e_, what);     \
    } while (0)

// Grow a device buffer to at least `bytes` (contents not kept).
lrs_status lrs_ensure(void** ptr, size_t* have, size_t bytes);
lrs_status lrs_scratch(lrs_ctx* ctx, size_t bytes, void** out);
// True while `st` is being captured into a CUDA graph: launches then skip the one-time
// function-attribute calls (made by an earlier uncaptured call) and nested graphs.
bool lrs_capturing(cudaStream_t st);

// ---- launchers implemented in the kernel translation units --------------------
lrs_status launch_init_terms(lrs_ctx* ctx, int32_t mode, uint64_t seed, double scale,
                             cudaStream_t st);
// Gate lists are host arrays, read before the call returns (passed to the kernel as
// launch parameters).
lrs_status launch_apply_clifford(lrs_ctx* ctx, const lrs_gate* gates_host, int64_t n_gates, cudaStream_t st);
lrs_status launch_apply_clifford_range(lrs_ctx* ctx, const lrs_gate* gates_host, int64_t n_gates, int64_t n_terms,
                                       cudaStream_t st);
lrs_status launch_expand_terms(lrs_ctx* ctx, int64_t R, int64_t Rn, cudaStream_t st);
// err (may be NULL): per-result bound on |out - exact chi-sum| (see k_amp_reduce).
lrs_status launch_amplitude(lrs_ctx* ctx, const uint64_t* x, int64_t batch, double* out, float* err,
                            cudaStream_t st);
lrs_status launch_amplitude_q(lrs_ctx* ctx, const uint64_t* x, int64_t batch, void* Q, double** amp_out,
                              cudaStream_t st);
// eta and ov may each be NULL (ov: 2^{n/2} <phi_{A_l}|psi> as Re, Im pairs)
lrs_status launch_norm_estimate(lrs_ctx* ctx, int64_t L, uint64_t seed, double* eta, double* ov,
                                cudaStream_t st);
lrs_status launch_norm_eta(const double* ov, int64_t L, double* eta, cudaStream_t st);
lrs_status launch_sample_terms(lrs_ctx* ctx, int64_t count, uint64_t seed, uint64_t* x,
                               int64_t* alpha, cudaStream_t st);
lrs_status launch_chains_init(lrs_ctx* ctx, const uint64_t* x, cudaStream_t st);
lrs_status launch_metropolis(lrs_ctx* ctx, int64_t steps, uint64_t seed, int64_t step0,
                             uint64_t* x_out, double* p_out, uint64_t* trace, cudaStream_t st);
lrs_status launch_metropolis_learned(lrs_ctx* ctx, lrs_mlp* mlp, int64_t steps, uint64_t seed,
                                     int64_t step0, uint64_t* x_out, double* p_out, uint64_t* trace,
                                     int64_t* accepts, cudaStream_t st);
lrs_status launch_chains_refresh(lrs_ctx* ctx, cudaStream_t st);
lrs_status mc_flags(lrs_ctx* ctx);
lrs_status launch_metropolis_propose(lrs_ctx* ctx, uint64_t seed, int64_t step, double* amp, cudaStream_t st);
lrs_status launch_metropolis_accept(lrs_ctx* ctx, const double* amp, uint64_t seed, int64_t step, uint64_t* trace,
                                    cudaStream_t st);
lrs_status launch_chains_set_prob(lrs_ctx* ctx, const double* amp, cudaStream_t st);
lrs_status launch_amplitude_batch(lrs_ctx* const* ctxs, const uint64_t* const* xs, const int64_t* batch,
                                  double* const* out, int32_t count, cudaStream_t st);
// Gate list with the launch-internal slot codes of the apply kernels (k_terms.cu).
void specialise_gates(const lrs_ctx* ctx, const lrs_gate* in, int64_t n, lrs_gate* out);
lrs_status launch_apply_clifford_batch(lrs_ctx* const* ctxs, int32_t count, cudaStream_t st,
                                       void** dev_buf, size_t* dev_buf_bytes);
