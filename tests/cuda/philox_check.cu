// Test helper: runs the library's device Philox4x32-10 forms and the
// independent implementation in CUDA's curand header on the same (counter,
// key) inputs.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <cstdint>

#include "../../paper_1611_06684_gb300/csrc/philox.cuh"

// mode 0: philox4x32_10; mode 1: philox4x32_10_rk (precomputed round keys)
__global__ void k_philox_pair(const uint4* ctr, uint2 key, mrfk::RoundKeys rk, int mode, uint4* mine, uint4* ref,
                              int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    mine[i] = mode == 0 ? mrfk::philox4x32_10(ctr[i], key) : mrfk::philox4x32_10_rk(ctr[i], rk);
    ref[i] = curand_Philox4x32_10(ctr[i], key);
}

// draw_rk_subs<4>: four calls (index, sweep, chain, phase << 24 | s), s = 0..3,
// sharing their first rounds; item i takes counter words 0..2 and phase from ctr[i]
__global__ void k_philox_subs(const uint4* ctr, uint2 key, mrfk::RoundKeys rk, uint4* mine, uint4* ref, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = ctr[i];
    const uint32_t phase = c.w & 0xFFu;
    uint4 out[4];
    mrfk::draw_rk_subs<4>(c.x, c.y, c.z, phase, rk, out);
    for (int s = 0; s < 4; ++s) {
        mine[4 * i + s] = out[s];
        ref[4 * i + s] = curand_Philox4x32_10(make_uint4(c.x, c.y, c.z, (phase << 24) | (uint32_t)s), key);
    }
}

static int run(int which, const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* mine, uint32_t* ref, int n) {
    const int per = which == 2 ? 4 : 1;
    uint4 *dc = nullptr, *dm = nullptr, *dr = nullptr;
    const size_t bytes = (size_t)n * sizeof(uint4);
    if (cudaMalloc(&dc, bytes) || cudaMalloc(&dm, bytes * per) || cudaMalloc(&dr, bytes * per)) return 1;
    cudaMemcpy(dc, ctr, bytes, cudaMemcpyHostToDevice);
    const uint2 key = make_uint2(k0, k1);
    const mrfk::RoundKeys rk = mrfk::round_keys(key);
    if (which == 2)
        k_philox_subs<<<(n + 255) / 256, 256>>>(dc, key, rk, dm, dr, n);
    else
        k_philox_pair<<<(n + 255) / 256, 256>>>(dc, key, rk, which, dm, dr, n);
    cudaMemcpy(mine, dm, bytes * per, cudaMemcpyDeviceToHost);
    cudaMemcpy(ref, dr, bytes * per, cudaMemcpyDeviceToHost);
    const int err = cudaGetLastError() != cudaSuccess;
    cudaFree(dc); cudaFree(dm); cudaFree(dr);
    return err;
}

extern "C" int philox_pair(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* mine, uint32_t* ref, int n) {
    return run(0, ctr, k0, k1, mine, ref, n);
}
extern "C" int philox_rk_pair(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* mine, uint32_t* ref, int n) {
    return run(1, ctr, k0, k1, mine, ref, n);
}
// mine and ref hold 4 n uint4
extern "C" int philox_subs_pair(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* mine, uint32_t* ref, int n) {
    return run(2, ctr, k0, k1, mine, ref, n);
}
