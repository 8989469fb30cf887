// Microbenchmarks for the non-HBM ceilings of the samplers: shared-memory
// load bandwidth, shared 32-bit atomic throughput and LOP3 (integer ALU)
// throughput of the current device. The samplers move GF(2) bit words, so
// their co-bounds are the shared-memory pipe and the integer pipe; the
// profile summaries divide the kernels' measured rates by these peaks.
//
// Every kernel is compute-only over its own shared memory; the only global
// write is one word per thread of a caller-invisible sink that keeps the
// compiler from removing the work.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "tmcs_internal.h"

namespace tmcs {

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakSmemWords = 8192;  // 32 KB per CTA
constexpr int kPeakIters = 4096;

// Shared memory is 256 rows of 32 words. Each warp-wide access reads one
// row at (row * 32 + lane): 32 consecutive words, one wavefront, no bank
// conflict. Row bases are multiples of 8 below 256 and j < 8, so every index
// stays below 256 * 32.
__device__ __forceinline__ uint32_t peak_row_base(int it, uint32_t warp) {
    return ((uint32_t(it) * 8u + warp * 8u) & 255u) * 32u;
}

__global__ void __launch_bounds__(kPeakThreads) peak_smem_load(uint32_t *sink) {
    __shared__ uint32_t buf[kPeakSmemWords];
    for (int i = threadIdx.x; i < kPeakSmemWords; i += blockDim.x) buf[i] = uint32_t(i) * 2654435761u;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int it = 0; it < kPeakIters; it++) {
        const uint32_t *r = buf + peak_row_base(it, warp) + lane;
#pragma unroll
        for (int j = 0; j < 8; j++) acc[j] ^= r[32 * j];
    }
    uint32_t v = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) v ^= acc[j];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = v;
}

// 32-bit shared atomic XORs with the same conflict-free pattern.
__global__ void __launch_bounds__(kPeakThreads) peak_smem_atomic(uint32_t *sink) {
    __shared__ uint32_t buf[kPeakSmemWords];
    for (int i = threadIdx.x; i < kPeakSmemWords; i += blockDim.x) buf[i] = 0u;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (int it = 0; it < kPeakIters / 8; it++) {
        uint32_t *r = buf + peak_row_base(it, warp) + lane;
#pragma unroll
        for (int j = 0; j < 8; j++) atomicXor(r + 32 * j, uint32_t(it + j) | 1u);
    }
    __syncthreads();
    sink[blockIdx.x * blockDim.x + threadIdx.x] = buf[threadIdx.x];
}

// Eight independent chains of lop3.b32 (a ^ (b & c)) per thread: chain j
// depends only on its own previous value, so the pipe, not the latency,
// bounds the rate.
__device__ __forceinline__ uint32_t lop3_xor_and(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x6a;" : "=r"(d) : "r"(a), "r"(b), "r"(c));  // a ^ (b & c)
    return d;
}

__global__ void __launch_bounds__(kPeakThreads) peak_lop3(uint32_t *sink, uint32_t seed) {
    uint32_t a0 = seed ^ threadIdx.x, a1 = a0 * 3u, a2 = a0 * 5u, a3 = a0 * 7u;
    uint32_t a4 = a0 * 11u, a5 = a0 * 13u, a6 = a0 * 17u, a7 = a0 * 19u;
    const uint32_t b = seed * 2654435761u, c = ~seed;
    for (int it = 0; it < kPeakIters; it++) {
        a0 = lop3_xor_and(a0, b, c);
        a1 = lop3_xor_and(a1, c, b);
        a2 = lop3_xor_and(a2, b, ~c);
        a3 = lop3_xor_and(a3, ~b, c);
        a4 = lop3_xor_and(a4, b ^ 1u, c);
        a5 = lop3_xor_and(a5, c ^ 2u, b);
        a6 = lop3_xor_and(a6, b ^ 4u, c);
        a7 = lop3_xor_and(a7, c ^ 8u, b);
    }
    sink[blockIdx.x * blockDim.x + threadIdx.x] = a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7;
}

}  // namespace

}  // namespace tmcs

using namespace tmcs;

extern "C" int tmcs_measure_peaks(tmcs_peaks *out) {
    if (!out) return fail(TMCS_E_INVALID, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    int dev = 0, sms = 0, clk_khz = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    if (e != cudaSuccess) return fail(TMCS_E_CUDA, std::string("device query: ") + cudaGetErrorString(e));
    // one full wave per kernel: the CTAs that are resident at once
    int occ[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], peak_smem_load, kPeakThreads, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], peak_smem_atomic, kPeakThreads, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[2], peak_lop3, kPeakThreads, 0);
    if (e != cudaSuccess) return fail(TMCS_E_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
    int blocks_k[3];
    for (int k = 0; k < 3; k++) blocks_k[k] = sms * (occ[k] > 0 ? occ[k] : 1);
    const int blocks = std::max(blocks_k[0], std::max(blocks_k[1], blocks_k[2]));
    uint32_t *sink = nullptr;
    if ((e = cudaMalloc(&sink, size_t(blocks) * kPeakThreads * 4)) != cudaSuccess) {
        cudaGetLastError();
        return fail(TMCS_E_OOM, std::string("cudaMalloc of the benchmark sink: ") + cudaGetErrorString(e));
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms[3] = {0, 0, 0};
    for (int k = 0; k < 3 && e == cudaSuccess; k++) {
        for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {  // first run warms up
            cudaEventRecord(e0);
            if (k == 0) peak_smem_load<<<blocks_k[0], kPeakThreads>>>(sink);
            if (k == 1) peak_smem_atomic<<<blocks_k[1], kPeakThreads>>>(sink);
            if (k == 2) peak_lop3<<<blocks_k[2], kPeakThreads>>>(sink, 0x9E3779B9u);
            cudaEventRecord(e1);
            e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[k], e0, e1);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return fail(TMCS_E_CUDA, std::string("peak benchmark: ") + cudaGetErrorString(e));
    double threads[3];
    for (int k = 0; k < 3; k++) threads[k] = double(blocks_k[k]) * kPeakThreads;
    const double loads = threads[0] / 32.0 * kPeakIters * 8.0;  // warp-wide 32-bit loads = wavefronts
    out->smem_load_wavefronts_per_s = loads / (ms[0] * 1e-3);
    out->smem_load_bytes_per_s = out->smem_load_wavefronts_per_s * 128.0;
    out->smem_atomic_lanes_per_s = threads[1] * (kPeakIters / 8) * 8.0 / (ms[1] * 1e-3);
    out->lop3_lanes_per_s = threads[2] * kPeakIters * 8.0 / (ms[2] * 1e-3);
    out->lop3_warp_inst_per_s = out->lop3_lanes_per_s / 32.0;
    out->sms = sms;
    out->sm_clock_mhz = clk_khz / 1000.0;
    set_error("");
    return TMCS_OK;
}
