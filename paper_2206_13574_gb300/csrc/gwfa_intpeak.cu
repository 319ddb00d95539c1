// gwfa_intpeak.cu -- integer-pipe throughput ceiling of this GPU (measurement only).
//
// The alignment kernels do integer scan, hash and graph work with no dense
// contraction, so their compute ceiling is the integer ALU pipe, not the tensor
// cores.  This kernel measures that ceiling: every thread runs kChains independent
// chains of 3-input logic operations (one lop3.b32 each, an ALU-pipe instruction
// with no memory traffic), enough warps per SM and enough independent chains per
// warp that the pipe, not latency, bounds the rate.  The count of lop3 warp
// instructions is known by construction (threads / 32 x iterations x kChains x
// kUnroll); a profiler's ALU-pipe instruction counter on this kernel checks it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gwfa_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 8;
constexpr int kThreads = 1024;

__device__ uint32_t g_intpeak_sink;

__global__ void __launch_bounds__(kThreads) int_peak_kernel(uint32_t iters, uint32_t b, uint32_t c) {
    uint32_t x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (blockIdx.x * blockDim.x + threadIdx.x) * (2 * i + 1);
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int i = 0; i < kChains; ++i)
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[i]) : "r"(b), "r"(c));
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc ^= x[i];
    if (acc == 0x9E3779B9u) g_intpeak_sink = acc;   // keeps the chains live
}

}  // namespace

extern "C" int gwfa_measure_int_peak(int device, uint32_t blocks_per_sm, uint32_t iters, float *ms_out,
                                     uint64_t *warp_insts_out) {
    if (!ms_out || !warp_insts_out || iters == 0) return GWFA_ERR_INVALID;
    if (blocks_per_sm == 0) blocks_per_sm = 2;
    if (cudaSetDevice(device) != cudaSuccess) return GWFA_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return GWFA_ERR_CUDA;
    const uint32_t blocks = (uint32_t)sms * blocks_per_sm;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = GWFA_OK;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        st = GWFA_ERR_CUDA;
    float best = 0.f;
    for (int rep = 0; rep < 4 && !st; ++rep) {   // the first run warms up; best of the others
        cudaEventRecord(e0, s);
        int_peak_kernel<<<blocks, kThreads, 0, s>>>(iters, 0x12345678u, 0x0F0F0F0Fu);
        cudaEventRecord(e1, s);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            st = GWFA_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (st) return st;
    *ms_out = best;
    *warp_insts_out = (uint64_t)blocks * (kThreads / 32) * iters * kChains * kUnroll;
    return GWFA_OK;
}
