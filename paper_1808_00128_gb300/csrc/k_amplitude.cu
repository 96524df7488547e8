// Batched amplitudes <x|psi> = sum_alpha b_alpha <x|phi_alpha> (Eqs. (amplitude),
// (amplitude1)).
//
// One thread per term, x uniform across the block: the set bits of x drive a
// uniform loop over rows, so there is no divergence and every shared-memory
// access ([row][thread] layout) is conflict-free.  Per set bit p of x the
// Pauli accumulator i^mu X(u) Z(w) absorbs U_C^{-1} X_p U_C:
//     z ^= w & F_p;  u ^= F_p;  w ^= M_p
// and the phase is mu = x.gamma + 2 parity(z) (mod 4) at the end, so the loop
// body is pure LOP3 work.  The block's 128 term values are summed pairwise in
// FP32 (warp shuffles, then across warps); block partials are summed in FP64.
#include "lrs_device.cuh"

namespace {

constexpr int AMP_TPB = 128;   // terms per block
constexpr int AMP_XB = 64;     // x values per block

__global__ void __launch_bounds__(AMP_TPB) k_amplitude(TermsView T, const uint64_t* __restrict__ xs,
                                                       int64_t batch, float2* __restrict__ partial,
                                                       int64_t n_tiles) {
    extern __shared__ uint64_t smem[];
    __shared__ float2 red[AMP_TPB / 32][AMP_XB];
    const int n = T.n;
    const int tid = threadIdx.x;
    const int64_t tile = blockIdx.x;
    const int64_t a = tile * AMP_TPB + tid;
    uint64_t* sF = smem + tid;
    uint64_t* sM = smem + (int64_t)n * AMP_TPB + tid;
    for (int p = 0; p < n; ++p) {
        sF[p * AMP_TPB] = T.F[(int64_t)p * T.cap + a];
        sM[p * AMP_TPB] = T.M[(int64_t)p * T.cap + a];
    }
    const uint64_t glo = T.glo[a], ghi = T.ghi[a], v = T.v[a], s = T.s[a];
    const uint32_t om = T.omega[a];
    const uint64_t nv = ~v & T.nmask;
    const uint64_t sv = s & v;
    const bool live = ((om >> 3) & 1u) == 0u;
    const int k0 = (int)(om & 7u);
    const int e0 = __popcll(v) + (int)(om >> 8);   // 2^{-(|v| + h)/2}
    const float2 b = T.coef[a];

    const int64_t x0 = (int64_t)blockIdx.y * AMP_XB;
    const int nx = (int)(batch - x0 < AMP_XB ? batch - x0 : AMP_XB);
    const int lane = tid & 31, warp = tid >> 5;
    for (int xi = 0; xi < nx; ++xi) {
        const uint64_t x = xs[x0 + xi] & T.nmask;   // bits >= n are ignored
        uint64_t u = 0, w = 0, z = 0, xr = x;
        while (xr) {
            const int p = ffs64(xr);
            xr &= xr - 1;
            const uint64_t Fp = sF[p * AMP_TPB];
            z ^= w & Fp;
            u ^= Fp;
            w ^= sM[p * AMP_TPB];
        }
        float2 val = make_float2(0.f, 0.f);
        if (live && ((u ^ s) & nv) == 0) {
            const int mu = __popcll(x & glo) + 2 * __popcll(x & ghi) + 2 * (int)par64(z);
            const int sign = (int)(par64(u & w) ^ par64(u & sv));
            val = z8_scale(b, 2 * mu + 4 * sign + k0, e0);
        }
        // pairwise FP32 reduction over the block's terms
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            val.x += __shfl_xor_sync(0xffffffffu, val.x, off);
            val.y += __shfl_xor_sync(0xffffffffu, val.y, off);
        }
        if (lane == 0) red[warp][xi] = val;
    }
    __syncthreads();
    if (tid < nx) {
        float2 acc = red[0][tid];
#pragma unroll
        for (int w2 = 1; w2 < AMP_TPB / 32; ++w2) {
            acc.x += red[w2][tid].x;
            acc.y += red[w2][tid].y;
        }
        partial[(x0 + tid) * n_tiles + tile] = acc;
    }
}

// FP64 sum of the block partials of each x.
__global__ void k_amp_reduce(const float2* __restrict__ partial, int64_t n_tiles, int64_t batch,
                             double* __restrict__ out) {
    const int64_t xi = blockIdx.x;
    if (xi >= batch) return;
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
        out[2 * xi] = sre[0];
        out[2 * xi + 1] = sim[0];
    }
}

}  // namespace

lrs_status launch_amplitude(lrs_ctx* ctx, const uint64_t* x, int64_t batch, double* out,
                            cudaStream_t st) {
    if (batch == 0) return LRS_OK;
    const int64_t n_tiles = ctx->cap / AMP_TPB;
    void* scr = nullptr;
    lrs_status rc = lrs_scratch(ctx, (size_t)batch * n_tiles * sizeof(float2), &scr);
    if (rc != LRS_OK) return rc;
    float2* partial = (float2*)scr;
    const size_t smem = (size_t)2 * ctx->n * AMP_TPB * sizeof(uint64_t);
    LRS_CUDA(cudaFuncSetAttribute(k_amplitude, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  2 * 64 * AMP_TPB * (int)sizeof(uint64_t)));
    const int64_t xblocks = (batch + AMP_XB - 1) / AMP_XB;
    if (xblocks > 65535) return lrs_fail(LRS_ERR_UNSUPPORTED, "amplitude batch too large (max %d)",
                                         65535 * AMP_XB);
    dim3 grid((unsigned)n_tiles, (unsigned)xblocks);
    k_amplitude<<<grid, AMP_TPB, smem, st>>>(ctx->view(), x, batch, partial, n_tiles);
    LRS_LAUNCH_CHECK("amplitude kernel");
    k_amp_reduce<<<(unsigned)batch, 256, 0, st>>>(partial, n_tiles, batch, out);
    LRS_LAUNCH_CHECK("amplitude reduce kernel");
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
// kernel directly.
static void* g_noalloc_addr[128];
static bool g_noalloc_ready[128];

static lrs_status noalloc_address(int device, float2** out) {
    if (device < 0 || device >= 128) return lrs_fail(LRS_ERR_UNSUPPORTED, "device index %d", device);
    if (!g_noalloc_ready[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return lrs_cuda_check(e, "cudaGetSymbolAddress(g_noalloc_partials)");
        g_noalloc_addr[device] = p;
        g_noalloc_ready[device] = true;
    }
    *out = (float2*)g_noalloc_addr[device];
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
    const int64_t n_tiles = ctx->cap / AMP_TPB;
    if ((uint64_t)batch * (uint64_t)n_tiles > (uint64_t)LRS_NOALLOC_PARTIALS)
        return lrs_fail(LRS_ERR_ARG,
                        "lrs_amplitude_noalloc: batch * ceil(chi/128) = %lld exceeds the fixed "
                        "buffer of %u partial sums; use a smaller batch or lrs_amplitude",
                        (long long)(batch * n_tiles), LRS_NOALLOC_PARTIALS);
    const int64_t xblocks = (batch + AMP_XB - 1) / AMP_XB;
    if (xblocks > 65535) return lrs_fail(LRS_ERR_UNSUPPORTED, "amplitude batch too large");
    const size_t smem = (size_t)2 * ctx->n * AMP_TPB * sizeof(uint64_t);
    LRS_CUDA(cudaFuncSetAttribute(k_amplitude, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  2 * 64 * AMP_TPB * (int)sizeof(uint64_t)));
    cudaStream_t st = (cudaStream_t)stream;
    dim3 grid((unsigned)n_tiles, (unsigned)xblocks);
    k_amplitude<<<grid, AMP_TPB, smem, st>>>(ctx->view(), x, batch, partial, n_tiles);
    LRS_LAUNCH_CHECK("amplitude kernel (no-alloc)");
    k_amp_reduce<<<(unsigned)batch, 256, 0, st>>>(partial, n_tiles, batch, out);
    LRS_LAUNCH_CHECK("amplitude reduce kernel (no-alloc)");
    return LRS_OK;
}
