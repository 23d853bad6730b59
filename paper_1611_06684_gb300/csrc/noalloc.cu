// Allocation-free plain sweep.  Same dual and primal half-steps as the
// handle's plain sweep, but the bit-packed dual variables (the sweep's scratch)
// live in a fixed, file-scope device array instead of a buffer the library
// allocates, and the labels are read from and written to buffers the caller
// owns.  The paper has no counterpart; this exists for callers that cannot
// allocate device memory when they sweep.
//
// The array is loaded with the library and held by every GPU that loads it
// until the process exits.  Host code must not use the array's name as a
// device address (in host code it names a host-side stand-in); the device
// address is looked up once per device with cudaGetSymbolAddress, below.
#include "sweep_impl.cuh"

#include <mutex>

namespace mrfk {

// words [0, kNoallocCtlWords): control block (boundary counter); then theta.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoallocCtlWords + MRF_NOALLOC_THETA_WORDS];

namespace {
std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
uint32_t* g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
cudaError_t noalloc_scratch(uint32_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

__global__ void k_noalloc_reset(Ctl* ctl) { ctl->boundary = 0; }

template <int L, int LAYOUT>
__global__ void __launch_bounds__(256, 4) k_dual_noalloc(SweepArgs a, const uint8_t* __restrict__ xin, uint32_t sweep) {
    using E = Ent<L, LAYOUT>;
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (uint64_t)a.E * a.C) return;
    const uint32_t e = a.fdC.div(g);
    const uint32_t c = g - e * (uint32_t)a.C;
    uint32_t bits[E::W];
    const int s = a.src[e];
    if (s >= 0) {
        const int t = a.dst[e];
        dual_bits<L, LAYOUT>(e, c, xin[(int64_t)s * a.C + c], xin[(int64_t)t * a.C + c],
                             a.tpl + (int64_t)e * E::PW, a.thr + (int64_t)e * E::M, sweep, a.rk, bits);
    } else {
#pragma unroll
        for (int w = 0; w < E::W; ++w) bits[w] = 0;
    }
    uint32_t* out = a.theta + (int64_t)g * E::W;
#pragma unroll
    for (int w = 0; w < E::W; ++w) out[w] = bits[w];
}

template <int L, int LAYOUT>
__global__ void __launch_bounds__(256, 4) k_primal_noalloc(SweepArgs a, uint8_t* __restrict__ xout, uint32_t sweep) {
    using E = Ent<L, LAYOUT>;
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (uint64_t)a.N * a.C) return;
    const uint32_t v = a.fdC.div(g), c = g - v * (uint32_t)a.C;
    float acc[L], hi[L], lo[L];
#pragma unroll
    for (int x = 0; x < L; ++x) { acc[x] = 0.0f; hi[x] = 0.0f; lo[x] = 0.0f; }
    int chunk = 0;
    bool flushed = false;
    for (int64_t p = a.inc_ptr[v]; p < a.inc_ptr[v + 1]; ++p) {
        const int2 ic = a.inc[p];
        const int64_t e = ic.x >> 1;
        uint32_t bits[E::W];
        const uint32_t* th = a.theta + (e * a.C + c) * E::W;
#pragma unroll
        for (int w = 0; w < E::W; ++w) bits[w] = th[w];
        add_side<L, LAYOUT>(bits, a.tau + e * E::MP, ic.x & 1, acc);
        if (++chunk == 32) {
#pragma unroll
            for (int x = 0; x < L; ++x) { two_sum_add(hi[x], lo[x], acc[x]); acc[x] = 0.0f; }
            chunk = 0;
            flushed = true;
        }
    }
    float F[L];
    const float* uf = a.utf + (int64_t)v * L;
#pragma unroll
    for (int x = 0; x < L; ++x) {
        if (flushed) two_sum_add(hi[x], lo[x], acc[x]);
        F[x] = flushed ? __ldg(uf + x) + (hi[x] + lo[x]) : __ldg(uf + x) + acc[x];
    }
    xout[g] = (uint8_t)draw_label<L>(F, v, c, sweep, a.rk, PH_PRIMAL, nullptr, a.ctl);
}

#define MRF_DISPATCH_L3(L_, ...)                                                  \
    switch (L_) {                                                                 \
        case 2: { constexpr int LL = 2; __VA_ARGS__; } break;                     \
        case 3: { constexpr int LL = 3; __VA_ARGS__; } break;                     \
        case 4: { constexpr int LL = 4; __VA_ARGS__; } break;                     \
        case 5: { constexpr int LL = 5; __VA_ARGS__; } break;                     \
        case 6: { constexpr int LL = 6; __VA_ARGS__; } break;                     \
        case 7: { constexpr int LL = 7; __VA_ARGS__; } break;                     \
        case 8: { constexpr int LL = 8; __VA_ARGS__; } break;                     \
        case 9: { constexpr int LL = 9; __VA_ARGS__; } break;                     \
        case 10: { constexpr int LL = 10; __VA_ARGS__; } break;                   \
        case 11: { constexpr int LL = 11; __VA_ARGS__; } break;                   \
        case 12: { constexpr int LL = 12; __VA_ARGS__; } break;                   \
        case 13: { constexpr int LL = 13; __VA_ARGS__; } break;                   \
        case 14: { constexpr int LL = 14; __VA_ARGS__; } break;                   \
        case 15: { constexpr int LL = 15; __VA_ARGS__; } break;                   \
        case 16: { constexpr int LL = 16; __VA_ARGS__; } break;                   \
        default: return cudaErrorInvalidValue;                                    \
    }

// One plain sweep with theta in the static array: a.theta and a.ctl must point
// into it (noalloc_scratch), the caller has checked E * C * W against its size.
cudaError_t launch_sweep_noalloc(const SweepArgs& a, int layout, const uint8_t* xin, uint8_t* xout, uint32_t sweep,
                                 cudaStream_t s) {
    k_noalloc_reset<<<1, 1, 0, s>>>(a.ctl);
    const unsigned bd = (unsigned)(((uint64_t)a.E * a.C + 255) / 256);
    const unsigned bp = (unsigned)(((uint64_t)a.N * a.C + 255) / 256);
    if (layout == MRF_LAYOUT_PIVOT) {
        MRF_DISPATCH_L3(a.L, if (bd) (k_dual_noalloc<LL, MRF_LAYOUT_PIVOT><<<bd, 256, 0, s>>>(a, xin, sweep));
                        (k_primal_noalloc<LL, MRF_LAYOUT_PIVOT><<<bp, 256, 0, s>>>(a, xout, sweep)));
    } else {
        MRF_DISPATCH_L3(a.L, if (bd) (k_dual_noalloc<LL, MRF_LAYOUT_DIAG><<<bd, 256, 0, s>>>(a, xin, sweep));
                        (k_primal_noalloc<LL, MRF_LAYOUT_DIAG><<<bp, 256, 0, s>>>(a, xout, sweep)));
    }
    return cudaGetLastError();
}

}  // namespace mrfk
