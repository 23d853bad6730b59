// Device-side CSR incidence build, used after edits so that a dynamic model
// never round-trips its edge list through the host.  The result is identical
// to the host build: within a site, incidences in increasing edge slot order
// (a site is never both ends of one edge), code = slot * 2 + side.
//   1. degree of every site over live edges (atomics)
//   2. exclusive scan of the degrees into inc_ptr (block scans, one CTA over the block sums)
//   3. scatter of every live edge's two incidences (atomic cursors)
//   4. per-site insertion sort by code (restores the deterministic order)
#include "common.cuh"

namespace mrfk {

__global__ void k_csr_degree(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t E,
                             int32_t* __restrict__ deg) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int s = src[e];
        if (s < 0) continue;
        atomicAdd(&deg[s], 1);
        atomicAdd(&deg[dst[e]], 1);
    }
}

// Block-local exclusive scan of 1024 values per block; block totals to sums[].
__global__ void k_scan_blocks(const int32_t* __restrict__ in, int64_t n, int64_t* __restrict__ out,
                              int64_t* __restrict__ sums) {
    __shared__ int64_t warp_tot[32];
    const int64_t i = blockIdx.x * 1024ll + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = warp_tot[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(0xFFFFFFFFu, t, d);
            if (lane >= d) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    const int64_t incl = x + (w > 0 ? warp_tot[w - 1] : 0);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == 1023) sums[blockIdx.x] = incl;
}

// One CTA of 1024 threads: exclusive scan of the block totals in place, each
// thread over a contiguous chunk; the grand total to *total.
__global__ void __launch_bounds__(1024) k_scan_sums(int64_t* sums, int64_t nb, int64_t* total) {
    __shared__ int64_t warp_tot[32];
    const int64_t chunk = (nb + 1023) / 1024;
    const int64_t b0 = threadIdx.x * chunk < nb ? threadIdx.x * chunk : nb;
    const int64_t b1 = b0 + chunk < nb ? b0 + chunk : nb;
    int64_t v = 0;
    for (int64_t b = b0; b < b1; ++b) v += sums[b];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = warp_tot[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(0xFFFFFFFFu, t, d);
            if (lane >= d) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    int64_t run = x - v + (w > 0 ? warp_tot[w - 1] : 0);
    for (int64_t b = b0; b < b1; ++b) {
        const int64_t t = sums[b];
        sums[b] = run;
        run += t;
    }
    if (threadIdx.x == 1023) *total = warp_tot[31];
}

__global__ void k_scan_add(int64_t* out, int64_t n, const int64_t* __restrict__ sums, const int64_t* total) {
    const int64_t i = blockIdx.x * 1024ll + threadIdx.x;
    if (i < n) out[i] += sums[blockIdx.x];
    if (i == n) out[n] = *total;     // inc_ptr[N]
}

__global__ void k_csr_fill(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t E,
                           const int64_t* __restrict__ ptr, int32_t* __restrict__ cursor, int2* __restrict__ inc) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int s = src[e];
        if (s < 0) continue;
        const int t = dst[e];
        inc[ptr[s] + atomicAdd(&cursor[s], 1)] = make_int2((int)(e * 2 + 0), t);
        inc[ptr[t] + atomicAdd(&cursor[t], 1)] = make_int2((int)(e * 2 + 1), s);
    }
}

// Insertion sort of each site's incidences by code; sites with more than
// max_deg incidences are left unsorted and counted (a host-side edit then
// rebuilds the lists on the host; a queue round sorts them with one CTA per
// site, k_csr_sort_long).
__global__ void k_csr_sort(const int64_t* __restrict__ ptr, int2* __restrict__ inc, int N, int max_deg,
                           unsigned long long* too_long) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    const int64_t p0 = ptr[v], p1 = ptr[v + 1];
    if (p1 - p0 > max_deg) { atomicAdd(too_long, 1ull); return; }
    for (int64_t i = p0 + 1; i < p1; ++i) {
        const int2 key = inc[i];
        int64_t j = i - 1;
        while (j >= p0 && inc[j].x > key.x) { inc[j + 1] = inc[j]; --j; }
        inc[j + 1] = key;
    }
}

// src[slot] / dst[slot] updates of an edit (removals carry src = dst = -1).
__global__ void k_scatter_edges(const int64_t* __restrict__ slots, const int32_t* __restrict__ s,
                                const int32_t* __restrict__ t, int64_t n, int32_t* src, int32_t* dst) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    src[slots[i]] = s[i];
    dst[slots[i]] = t[i];
}

cudaError_t launch_scatter_edges(const int64_t* slots, const int32_t* s, const int32_t* t, int64_t n, int32_t* src,
                                 int32_t* dst, cudaStream_t st) {
    if (n > 0) k_scatter_edges<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(slots, s, t, n, src, dst);
    return cudaGetLastError();
}

// Largest incidence count of a site: atomicMax of ptr[v + 1] - ptr[v] into *out (zeroed by the caller).
__global__ void k_max_degree(const int64_t* __restrict__ ptr, int N, unsigned* out) {
    unsigned m = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        const int64_t d = ptr[v + 1] - ptr[v];
        const unsigned du = d > 0x7FFFFFFF ? 0x7FFFFFFFu : (unsigned)d;
        m = du > m ? du : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned y = __shfl_xor_sync(0xFFFFFFFFu, m, o);
        m = y > m ? y : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

cudaError_t launch_max_degree(const int64_t* ptr, int N, unsigned* out, cudaStream_t s) {
    if (N > 0) k_max_degree<<<std::min(1216, (N + 255) / 256), 256, 0, s>>>(ptr, N, out);
    return cudaGetLastError();
}

// work: int32 [2N + 2] scratch (degrees, cursors); sums: int64 [ceil((N+1)/1024) + 1].
cudaError_t build_csr_device(const int32_t* src, const int32_t* dst, int64_t E, int N, int64_t* ptr, int2* inc,
                             int32_t* work, int64_t* sums, unsigned long long* too_long, int max_deg, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(work, 0, sizeof(int32_t) * 2 * (size_t)N, s)) != cudaSuccess) return e;
    int32_t* deg = work;
    int32_t* cursor = work + N;
    const unsigned eb = (unsigned)std::min<int64_t>((E + 255) / 256 + 1, 1216 * 4);
    if (E > 0) k_csr_degree<<<eb, 256, 0, s>>>(src, dst, E, deg);
    const int64_t nb = ((int64_t)N + 1 + 1023) / 1024;
    k_scan_blocks<<<(unsigned)nb, 1024, 0, s>>>(deg, N, ptr, sums);
    k_scan_sums<<<1, 1024, 0, s>>>(sums, nb, sums + nb);
    k_scan_add<<<(unsigned)nb, 1024, 0, s>>>(ptr, N, sums, sums + nb);
    if (E > 0) k_csr_fill<<<eb, 256, 0, s>>>(src, dst, E, ptr, cursor, inc);
    k_csr_sort<<<(N + 127) / 128, 128, 0, s>>>(ptr, inc, N, max_deg, too_long);
    return cudaGetLastError();
}

}  // namespace mrfk
