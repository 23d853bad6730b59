// Test helper: runs the library's device Philox4x32-10 and the independent
// implementation in CUDA's curand header on the same (counter, key) inputs.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <cstdint>

#include "../../paper_1611_06684_gb300/csrc/philox.cuh"

__global__ void k_philox_pair(const uint4* ctr, uint2 key, uint4* mine, uint4* ref, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    mine[i] = mrfk::philox4x32_10(ctr[i], key);
    ref[i] = curand_Philox4x32_10(ctr[i], key);
}

extern "C" int philox_pair(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* mine, uint32_t* ref, int n) {
    uint4 *dc = nullptr, *dm = nullptr, *dr = nullptr;
    const size_t bytes = (size_t)n * sizeof(uint4);
    if (cudaMalloc(&dc, bytes) || cudaMalloc(&dm, bytes) || cudaMalloc(&dr, bytes)) return 1;
    cudaMemcpy(dc, ctr, bytes, cudaMemcpyHostToDevice);
    k_philox_pair<<<(n + 255) / 256, 256>>>(dc, make_uint2(k0, k1), dm, dr, n);
    cudaMemcpy(mine, dm, bytes, cudaMemcpyDeviceToHost);
    cudaMemcpy(ref, dr, bytes, cudaMemcpyDeviceToHost);
    const int err = cudaGetLastError() != cudaSuccess;
    cudaFree(dc); cudaFree(dm); cudaFree(dr);
    return err;
}
