// Sweep driver kernels (initial labels, count accumulation, sweep counter) and
// the dispatch from the runtime (L, layout) to the templated half-step kernels
// of sweep_impl.cuh, instantiated in sweep_la.cu, sweep_lb.cu and sweep_lc.cu.
#include "common.cuh"

namespace mrfk {

template <int L, int LAYOUT> cudaError_t run_dual(const SweepArgs& a, cudaStream_t s);
template <int L, int LAYOUT, bool FUSED> cudaError_t run_primal(const SweepArgs& a, cudaStream_t s);
template <int L, int LAYOUT> cudaError_t run_primal_cta(const SweepArgs& a, cudaStream_t s);
template <int L, int LAYOUT> cudaError_t run_sweep_partial(const SweepArgs& a, int step, cudaStream_t s);

__global__ void k_init_labels(SweepArgs a) {
    const int64_t n = (int64_t)a.N * a.C;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)(g / a.C), c = (uint32_t)(g % a.C);
        const uint32_t U = draw(v, 0, c, PH_INIT, 0, a.key).x >> 8;
        a.x[g] = (uint8_t)(((uint64_t)U * (uint32_t)a.L) >> 24);
    }
}

// counts[v][a] += #{c : x_new[v][c] = a} for counted sweeps.  Per-label
// counts of up to 255 chains per pass are kept as sixteen 8-bit lanes of two
// 64-bit registers (label x adds 1 << 8x to the low or high word).
__global__ void k_accumulate(SweepArgs a) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.N) return;
    const unsigned long long t = a.ctl->sweep;
    if (t < a.ctl->count_from) return;
    const uint8_t* xo = a.x + (size_t)((t + 1) & 1) * a.N * a.C + (int64_t)v * a.C;
    uint32_t tot[kMaxLabels];
#pragma unroll
    for (int x = 0; x < kMaxLabels; ++x) tot[x] = 0;
    for (int c0 = 0; c0 < a.C; c0 += 255) {
        const int c1 = min(a.C, c0 + 255);
        unsigned long long lo = 0, hi = 0;
        int c = c0;
        if (((a.C | c0) & 3) == 0) {
            for (; c + 4 <= c1; c += 4) {
                const uint32_t w = *reinterpret_cast<const uint32_t*>(xo + c);
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const uint32_t x = (w >> (8 * b)) & 15u;
                    lo += x < 8 ? 1ull << (8 * x) : 0ull;
                    hi += x >= 8 ? 1ull << (8 * (x - 8)) : 0ull;
                }
            }
        }
        for (; c < c1; ++c) {
            const uint32_t x = xo[c] & 15u;
            lo += x < 8 ? 1ull << (8 * x) : 0ull;
            hi += x >= 8 ? 1ull << (8 * (x - 8)) : 0ull;
        }
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            tot[x] += (uint32_t)((lo >> (8 * x)) & 0xFF);
            tot[x + 8] += (uint32_t)((hi >> (8 * x)) & 0xFF);
        }
    }
    uint32_t* cnt = a.counts + (int64_t)v * a.L;
#pragma unroll
    for (int x = 0; x < kMaxLabels; ++x)
        if (x < a.L && tot[x]) cnt[x] += tot[x];
}

__global__ void k_advance(Ctl* ctl) { ctl->sweep += 1; }

// Label layout conversion between the internal x[v][c] (chain-innermost) and
// the ABI view y[c][v], through 32x32 shared-memory tiles.
__global__ void k_labels_to_abi(const uint8_t* __restrict__ x, uint8_t* __restrict__ y, int N, int C) {
    __shared__ uint8_t tile[32][33];
    const int v0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int v = v0 + r, c = c0 + threadIdx.x;
        if (v < N && c < C) tile[r][threadIdx.x] = x[(int64_t)v * C + c];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int c = c0 + r, v = v0 + threadIdx.x;
        if (v < N && c < C) y[(int64_t)c * N + v] = tile[threadIdx.x][r];
    }
}

__global__ void k_labels_from_abi(const uint8_t* __restrict__ y, uint8_t* __restrict__ x, int N, int C) {
    __shared__ uint8_t tile[32][33];
    const int v0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int c = c0 + r, v = v0 + threadIdx.x;
        if (v < N && c < C) tile[r][threadIdx.x] = y[(int64_t)c * N + v];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int v = v0 + r, c = c0 + threadIdx.x;
        if (v < N && c < C) x[(int64_t)v * C + c] = tile[threadIdx.x][r];
    }
}

__global__ void k_count_ge(const uint8_t* __restrict__ y, int64_t n, int L, unsigned long long* bad) {
    unsigned long long cnt = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        cnt += y[i] >= L;
    if (cnt) atomicAdd(bad, cnt);
}

cudaError_t launch_labels_to_abi(const uint8_t* x, uint8_t* y, int N, int C, cudaStream_t s) {
    k_labels_to_abi<<<dim3((N + 31) / 32, (C + 31) / 32), dim3(32, 8), 0, s>>>(x, y, N, C);
    return cudaGetLastError();
}

cudaError_t launch_labels_from_abi(const uint8_t* y, uint8_t* x, int N, int C, cudaStream_t s) {
    k_labels_from_abi<<<dim3((N + 31) / 32, (C + 31) / 32), dim3(32, 8), 0, s>>>(y, x, N, C);
    return cudaGetLastError();
}

cudaError_t launch_count_ge(const uint8_t* y, int64_t n, int L, unsigned long long* bad, cudaStream_t s) {
    k_count_ge<<<1216, 256, 0, s>>>(y, n, L, bad);
    return cudaGetLastError();
}

// Philox4x32-10 throughput probe: every thread runs `calls` independent calls
// (counters distinct across threads and calls, four in flight) and folds the
// outputs into one word so that nothing is optimised away.
__global__ void __launch_bounds__(256) k_philox_rate(RoundKeys rk, int calls, uint32_t* sink) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int i = 0; i < calls; i += 4) {
        const uint4 a = draw_rk(g, (uint32_t)i, 0, PH_DUAL, 0, rk);
        const uint4 b = draw_rk(g, (uint32_t)i + 1, 0, PH_DUAL, 0, rk);
        const uint4 c = draw_rk(g, (uint32_t)i + 2, 0, PH_DUAL, 0, rk);
        const uint4 d = draw_rk(g, (uint32_t)i + 3, 0, PH_DUAL, 0, rk);
        acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
    }
    if (acc == 0x12345678u) sink[g & 1023] = acc;    // practically never; keeps the work live
}

cudaError_t launch_philox_rate(uint64_t threads, int calls, uint32_t* sink, cudaStream_t s) {
    k_philox_rate<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(round_keys(make_uint2(1u, 2u)), calls, sink);
    return cudaGetLastError();
}

// log V of Section 5.2 for every chain after a plain sweep (a.lpv recorded by
// the primal step): out[c] += sum_v (u~_v(x_v) - log p(x_v | theta))
//                            + sum_e psi_e(x_s, x_t),
// psi = w - fold_s - fold_t the exact edge tables (so that sum_v u~ + sum_e psi
// = sum_v u + sum_e w = log p~(x)).  The item stride is a multiple of C, so a
// thread always sums one chain; per-chain partials meet in shared memory
// (float64) and then in out[c].
__global__ void k_log_v(SweepArgs a, const double* __restrict__ ut, double* __restrict__ out, int64_t stride) {
    extern __shared__ double s_acc[];
    const bool use_smem = a.C <= 4096;
    if (use_smem) {
        for (int i = threadIdx.x; i < a.C; i += blockDim.x) s_acc[i] = 0.0;
        __syncthreads();
    }
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int c = (int)(g % a.C);
    const uint8_t* x = a.x + (size_t)((uint32_t)a.ctl->sweep & 1u) * a.N * a.C;
    double acc = 0.0;
    const int64_t nsite = (int64_t)a.N * a.C, nedge = a.E * a.C;
    for (int64_t i = g; i < nsite; i += stride) {
        const int64_t v = i / a.C;
        acc += ut[v * a.L + x[i]] - (double)a.lpv[i];
    }
    for (int64_t i = g; i < nedge; i += stride) {
        const int64_t e = i / a.C;
        const int s = a.src[e];
        if (s < 0) continue;
        const int t = a.dst[e];
        acc += (double)a.resid[(e * a.L + x[(int64_t)s * a.C + c]) * a.L + x[(int64_t)t * a.C + c]];
    }
    if (use_smem) {
        atomicAdd(&s_acc[c], acc);
        __syncthreads();
        for (int i = threadIdx.x; i < a.C; i += blockDim.x) atomicAdd(&out[i], s_acc[i]);
    } else {
        atomicAdd(&out[c], acc);
    }
}

static int64_t gcd64(int64_t p, int64_t q) {
    while (q) { const int64_t r = p % q; p = q; q = r; }
    return p;
}

cudaError_t launch_log_v(const SweepArgs& a, const double* ut, double* out, cudaStream_t s) {
    // blocks * 256 must be a multiple of C; about four blocks per SM
    const int64_t unit = a.C / gcd64(256, a.C);                   // blocks per stride unit
    int64_t blocks = unit * std::max<int64_t>(1, (152 * 4 + unit - 1) / unit);
    blocks = std::min<int64_t>(blocks, std::max<int64_t>(unit, unit * ((((int64_t)a.N + a.E) * a.C / 256 + unit) / unit)));
    const size_t smem = a.C <= 4096 ? (size_t)a.C * sizeof(double) : 0;
    k_log_v<<<(unsigned)blocks, 256, smem, s>>>(a, ut, out, blocks * 256);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- dispatch

#define MRF_DISPATCH_L(L_, ...)                                                   \
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


cudaError_t launch_init_labels(const SweepArgs& a, cudaStream_t s) {
    k_init_labels<<<1216, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <int L, int LAYOUT> cudaError_t run_sweep_small(const SweepArgs&, int, cudaStream_t);

// Small models: the smem need of k_sweep_small (theta of all items) in bytes.
int64_t sweep_small_smem(const SweepArgs& a) { return a.E * a.C * (int64_t)a.W * 4; }

cudaError_t launch_sweep_small(const SweepArgs& a, int layout, int n_sweeps, cudaStream_t s) {
    if (layout == MRF_LAYOUT_PIVOT) {
        MRF_DISPATCH_L(a.L, return (run_sweep_small<LL, MRF_LAYOUT_PIVOT>(a, n_sweeps, s)));
    } else {
        MRF_DISPATCH_L(a.L, return (run_sweep_small<LL, MRF_LAYOUT_DIAG>(a, n_sweeps, s)));
    }
    return cudaGetLastError();
}

template <int L, int LAYOUT> cudaError_t run_em(const SweepArgs&, const uint8_t*, uint8_t*, cudaStream_t);
template <int L, int LAYOUT> cudaError_t run_mf(const SweepArgs&, const float*, float*, cudaStream_t);
template <int L, int LAYOUT> cudaError_t run_em_pot(const SweepArgs&, const uint8_t*, cudaStream_t);
template <int L, int LAYOUT> cudaError_t run_mf_pot(const SweepArgs&, const float*, cudaStream_t);

cudaError_t launch_mf_pot(const SweepArgs& a, int layout, const float* qin, cudaStream_t s) {
    if (layout == MRF_LAYOUT_PIVOT) {
        MRF_DISPATCH_L(a.L, return (run_mf_pot<LL, MRF_LAYOUT_PIVOT>(a, qin, s)));
    } else {
        MRF_DISPATCH_L(a.L, return (run_mf_pot<LL, MRF_LAYOUT_DIAG>(a, qin, s)));
    }
    return cudaGetLastError();
}

cudaError_t launch_em_pot(const SweepArgs& a, int layout, const uint8_t* xin, cudaStream_t s) {
    if (layout == MRF_LAYOUT_PIVOT) {
        MRF_DISPATCH_L(a.L, return (run_em_pot<LL, MRF_LAYOUT_PIVOT>(a, xin, s)));
    } else {
        MRF_DISPATCH_L(a.L, return (run_em_pot<LL, MRF_LAYOUT_DIAG>(a, xin, s)));
    }
    return cudaGetLastError();
}

cudaError_t launch_em(const SweepArgs& a, int layout, const uint8_t* xin, uint8_t* xout, cudaStream_t s) {
    if (layout == MRF_LAYOUT_PIVOT) {
        MRF_DISPATCH_L(a.L, return (run_em<LL, MRF_LAYOUT_PIVOT>(a, xin, xout, s)));
    } else {
        MRF_DISPATCH_L(a.L, return (run_em<LL, MRF_LAYOUT_DIAG>(a, xin, xout, s)));
    }
    return cudaGetLastError();
}

cudaError_t launch_mf(const SweepArgs& a, int layout, const float* qin, float* qout, cudaStream_t s) {
    if (layout == MRF_LAYOUT_PIVOT) {
        MRF_DISPATCH_L(a.L, return (run_mf<LL, MRF_LAYOUT_PIVOT>(a, qin, qout, s)));
    } else {
        MRF_DISPATCH_L(a.L, return (run_mf<LL, MRF_LAYOUT_DIAG>(a, qin, qout, s)));
    }
    return cudaGetLastError();
}

// marginals [C][N][L] (interface) <-> [N][L][C] (kernels)
__global__ void k_marg_layout(const float* __restrict__ in, float* __restrict__ out, int N, int L, int C, int to_abi) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)N * L * C) return;
    const int c = (int)(i % C);
    const int64_t vl = i / C;                          // v * L + a
    const int64_t j = (int64_t)c * N * L + vl;         // [c][v][a]
    if (to_abi) out[j] = in[i]; else out[i] = in[j];
}

cudaError_t launch_marg_layout(const float* in, float* out, int N, int L, int C, bool to_abi, cudaStream_t s) {
    const int64_t n = (int64_t)N * L * C;
    if (n > 0) k_marg_layout<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, N, L, C, to_abi ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_dual(const SweepArgs& a, int layout, cudaStream_t s) {
    const int64_t n = a.E * a.C;
    if (n == 0) return cudaSuccess;
    if (layout == MRF_LAYOUT_PIVOT) {
        MRF_DISPATCH_L(a.L, return (run_dual<LL, MRF_LAYOUT_PIVOT>(a, s)));
    } else {
        MRF_DISPATCH_L(a.L, return (run_dual<LL, MRF_LAYOUT_DIAG>(a, s)));
    }
    return cudaGetLastError();
}

cudaError_t launch_sweep_partial(const SweepArgs& a, int layout, int step, cudaStream_t s) {
    if (layout == MRF_LAYOUT_PIVOT) {
        MRF_DISPATCH_L(a.L, return (run_sweep_partial<LL, MRF_LAYOUT_PIVOT>(a, step, s)));
    } else {
        MRF_DISPATCH_L(a.L, return (run_sweep_partial<LL, MRF_LAYOUT_DIAG>(a, step, s)));
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_primal(const SweepArgs& a, int layout, int schedule, cudaStream_t s) {
    if (schedule == 2) {
        if (layout == MRF_LAYOUT_PIVOT) {
            MRF_DISPATCH_L(a.L, return (run_primal_cta<LL, MRF_LAYOUT_PIVOT>(a, s)));
        } else {
            MRF_DISPATCH_L(a.L, return (run_primal_cta<LL, MRF_LAYOUT_DIAG>(a, s)));
        }
    }
    if (layout == MRF_LAYOUT_PIVOT) {
        MRF_DISPATCH_L(a.L, return (run_primal<LL, MRF_LAYOUT_PIVOT, false>(a, s)));
    } else {
        MRF_DISPATCH_L(a.L, return (run_primal<LL, MRF_LAYOUT_DIAG, false>(a, s)));
    }
    return cudaGetLastError();
}

cudaError_t launch_fused(const SweepArgs& a, int layout, int schedule, cudaStream_t s) {
    (void)schedule;
    const int64_t n = (int64_t)a.N * a.C;
    if (layout == MRF_LAYOUT_PIVOT) {
        MRF_DISPATCH_L(a.L, return (run_primal<LL, MRF_LAYOUT_PIVOT, true>(a, s)));
    } else {
        MRF_DISPATCH_L(a.L, return (run_primal<LL, MRF_LAYOUT_DIAG, true>(a, s)));
    }
    return cudaGetLastError();
}

cudaError_t launch_accumulate(const SweepArgs& a, cudaStream_t s) {
    k_accumulate<<<(a.N + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_advance(const SweepArgs& a, cudaStream_t s) {
    k_advance<<<1, 1, 0, s>>>(a.ctl);
    return cudaGetLastError();
}

}  // namespace mrfk
