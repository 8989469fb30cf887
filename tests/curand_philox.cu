// Test helper (not part of the library): cuRAND's device Philox4x32-10 on
// caller-given counter/key pairs, for comparison with the CPU oracle's
// generator. Built by tests/test_gpu_rng.py with nvcc.
#include <cuda_runtime.h>
#include <curand_kernel.h>

#include <cstdint>

__global__ void curand_philox_kernel(const uint4 *ctr, const uint2 *key, uint4 *out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

// ctr: 4n words, key: 2n words, out: 4n words (host memory). Returns 0 or a
// cudaError_t value.
extern "C" int curand_philox_batch(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int n) {
    if (n <= 0) return 0;
    uint4 *dc = nullptr, *dout = nullptr;
    uint2 *dk = nullptr;
    cudaError_t e = cudaMalloc(&dc, sizeof(uint4) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dk, sizeof(uint2) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(uint4) * n);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, key, sizeof(uint2) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        curand_philox_kernel<<<(n + 255) / 256, 256>>>(dc, dk, dout, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    return int(e);
}
