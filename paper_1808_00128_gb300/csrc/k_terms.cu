// Term initialisation (exact enumeration / sparsification) and the fused
// Clifford-circuit kernel.
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

// ---- apply_clifford: one thread per term, tableau rows in shared memory -----------
// Shared layout [row][thread] makes every per-thread row index conflict-free.
struct SmemRows {
    uint64_t* base;
    int n;
    __device__ __forceinline__ uint64_t& F(int p) { return base[(p) * APPLY_TPB_STRIDE]; }
    __device__ __forceinline__ uint64_t& G(int p) { return base[(n + p) * APPLY_TPB_STRIDE]; }
    __device__ __forceinline__ uint64_t& M(int p) { return base[(2 * n + p) * APPLY_TPB_STRIDE]; }
    static constexpr int APPLY_TPB_STRIDE = 64;
};
constexpr int APPLY_TPB = SmemRows::APPLY_TPB_STRIDE;

// One tile of APPLY_TPB terms through the whole gate list.
__device__ __forceinline__ void apply_tile(const TermsView& T, const lrs_gate* __restrict__ gates,
                                           int64_t n_gates, int64_t tile, uint64_t* smem) {
    const int n = T.n;
    const int64_t a = tile * APPLY_TPB + threadIdx.x;   // cap % APPLY_TPB == 0
    SmemRows R{smem + threadIdx.x, n};
    for (int p = 0; p < n; ++p) {
        R.F(p) = T.F[(int64_t)p * T.cap + a];
        R.G(p) = T.G[(int64_t)p * T.cap + a];
        R.M(p) = T.M[(int64_t)p * T.cap + a];
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
        } else {
            apply_gate(R, S, n, nmask, g);
        }
    }
    for (int p = 0; p < n; ++p) {
        T.F[(int64_t)p * T.cap + a] = R.F(p);
        T.G[(int64_t)p * T.cap + a] = R.G(p);
        T.M[(int64_t)p * T.cap + a] = R.M(p);
    }
    T.glo[a] = S.glo; T.ghi[a] = S.ghi; T.v[a] = S.v; T.s[a] = S.s;
    T.omega[a] = omega_pack(S.k, S.zero, S.h);
}

__global__ void __launch_bounds__(APPLY_TPB) k_apply_clifford(TermsView T, const lrs_gate* __restrict__ gates,
                                                              int64_t n_gates) {
    extern __shared__ uint64_t smem[];
    apply_tile(T, gates, n_gates, blockIdx.x, smem);
}

// Several circuits of uneven chi in one persistent launch: blocks pull global
// tile indices from an atomic counter; circuit c owns tiles [first[c], first[c+1]).
struct ApplyItem {
    TermsView T;
    const lrs_gate* gates;
    int64_t n_gates;
    int64_t first_tile;
};

__global__ void __launch_bounds__(APPLY_TPB) k_apply_clifford_batch(const ApplyItem* __restrict__ items,
                                                                    int count, int64_t total_tiles,
                                                                    unsigned long long* counter) {
    extern __shared__ uint64_t smem[];
    __shared__ long long s_idx;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_idx = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const int64_t idx = s_idx;
        if (idx >= total_tiles) break;
        int lo = 0, hi = count - 1;          // last item with first_tile <= idx
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (items[mid].first_tile <= idx) lo = mid; else hi = mid - 1;
        }
        const ApplyItem& it = items[lo];
        apply_tile(it.T, it.gates, it.n_gates, idx - it.first_tile, smem);
    }
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

}  // namespace

lrs_status launch_init_terms(lrs_ctx* ctx, int32_t mode, uint64_t seed, double scale,
                             cudaStream_t st) {
    const int tpb = 256;
    const int64_t blocks = (ctx->cap + tpb - 1) / tpb;
    k_init_terms<<<(unsigned)blocks, tpb, 0, st>>>(ctx->view(), mode, seed, scale);
    LRS_LAUNCH_CHECK("init_terms kernel");
    return LRS_OK;
}

lrs_status launch_apply_clifford(lrs_ctx* ctx, const lrs_gate* gates_dev, int64_t n_gates,
                                 cudaStream_t st) {
    const size_t smem = (size_t)3 * ctx->n * APPLY_TPB * sizeof(uint64_t);
    static int configured_dev = -1;
    if (configured_dev != ctx->device) {
        LRS_CUDA(cudaFuncSetAttribute(k_apply_clifford, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      3 * 64 * APPLY_TPB * (int)sizeof(uint64_t)));
        configured_dev = ctx->device;
    }
    const int64_t blocks = ctx->cap / APPLY_TPB;
    k_apply_clifford<<<(unsigned)blocks, APPLY_TPB, smem, st>>>(ctx->view(), gates_dev, n_gates);
    LRS_LAUNCH_CHECK("apply_clifford kernel");
    return LRS_OK;
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

lrs_status launch_apply_clifford_batch(lrs_ctx* const* ctxs, int32_t count, cudaStream_t st,
                                       void** dev_buf, size_t* dev_buf_bytes) {
    std::vector<ApplyItem> items((size_t)count);
    int64_t tiles = 0;
    int nmax = 1;
    for (int32_t i = 0; i < count; ++i) {
        items[(size_t)i].T = ctxs[i]->view();
        items[(size_t)i].gates = ctxs[i]->gates_dev;
        items[(size_t)i].n_gates = ctxs[i]->batch_n_gates;
        items[(size_t)i].first_tile = tiles;
        tiles += ctxs[i]->cap / APPLY_TPB;
        if (ctxs[i]->n > nmax) nmax = ctxs[i]->n;
    }
    const size_t bytes = 256 + items.size() * sizeof(ApplyItem);
    lrs_status rc = lrs_ensure(dev_buf, dev_buf_bytes, bytes);
    if (rc != LRS_OK) return rc;
    unsigned long long* counter = (unsigned long long*)*dev_buf;
    ApplyItem* ditems = (ApplyItem*)((char*)*dev_buf + 256);
    LRS_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    LRS_CUDA(cudaMemcpyAsync(ditems, items.data(), items.size() * sizeof(ApplyItem), cudaMemcpyHostToDevice, st));
    LRS_CUDA(cudaStreamSynchronize(st));   // host item table may go out of scope
    const size_t smem = (size_t)3 * nmax * APPLY_TPB * sizeof(uint64_t);
    LRS_CUDA(cudaFuncSetAttribute(k_apply_clifford_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  3 * 64 * APPLY_TPB * (int)sizeof(uint64_t)));
    int per_sm = 0;
    LRS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_clifford_batch, APPLY_TPB, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)ctxs[0]->sm_count * per_sm;
    if (grid > tiles) grid = tiles;
    k_apply_clifford_batch<<<(unsigned)grid, APPLY_TPB, smem, st>>>(ditems, count, tiles, counter);
    LRS_LAUNCH_CHECK("batched apply_clifford kernel");
    return LRS_OK;
}
