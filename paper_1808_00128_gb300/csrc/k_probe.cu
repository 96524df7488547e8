// Integer-pipe throughput probe: independent LOP3 chains, 8 per thread.
#include "lrs_device.cuh"

namespace {
__global__ void k_alu_probe(int64_t iters, uint32_t seed, uint32_t* sink) {
    uint32_t a0 = seed ^ threadIdx.x, a1 = a0 * 3u, a2 = a0 * 5u, a3 = a0 * 7u;
    uint32_t a4 = a0 * 11u, a5 = a0 * 13u, a6 = a0 * 17u, a7 = a0 * 19u;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            // each line is one three-input LOP3: a ^= b & c
            a0 ^= a1 & a2;
            a1 ^= a2 & a3;
            a2 ^= a3 & a4;
            a3 ^= a4 & a5;
            a4 ^= a5 & a6;
            a5 ^= a6 & a7;
            a6 ^= a7 & a0;
            a7 ^= a0 & a1;
        }
    }
    const uint32_t r = a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7;
    if (r == 0x12345678u) sink[0] = r;   // keeps the chains live
}
}  // namespace

extern "C" lrs_status lrs_alu_probe(int32_t device, int64_t iters, double* ops_per_s) {
    if (iters < 1 || !ops_per_s) return lrs_fail(LRS_ERR_ARG, "bad probe arguments");
    LRS_CUDA(cudaSetDevice(device));
    int sms = 0;
    LRS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    uint32_t* sink = nullptr;
    LRS_CUDA(cudaMalloc(&sink, 4));
    const int tpb = 256, blocks = sms * 8;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_alu_probe<<<blocks, tpb>>>(iters / 8 + 1, 1u, sink);   // warm-up
    cudaEventRecord(e0);
    k_alu_probe<<<blocks, tpb>>>(iters, 12345u, sink);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return lrs_cuda_check(e, "alu probe");
    LRS_LAUNCH_CHECK("alu probe");
    // 8 chains x 16 unrolled x 1 LOP3 each per iteration per thread
    const double ops = (double)blocks * tpb * (double)iters * 16.0 * 8.0;
    *ops_per_s = ops / (ms * 1e-3);
    return LRS_OK;
}
