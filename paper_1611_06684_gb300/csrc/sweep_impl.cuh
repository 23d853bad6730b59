// The two half-steps of the primal-dual sweep (Section 5.1) for sm_103a.
//
//   dual step    theta_ek ~ Bernoulli(sigmoid(q + beta1 [x_s = i_k] + beta2 [x_t = j_k]))
//                for every edge slot e, dualised entry k and chain c    (k_dual)
//   primal step  x_v ~ softmax_a F_v(a),
//                F_v(a) = u~_v(a) + sum over incident edges of the beta terms of
//                the set dual bits whose entry row (source side) or column
//                (destination side) is a                                 (k_primal)
//   fused form   both in one vertex-centric kernel: each endpoint regenerates
//                the dual bits of its incident edges from the counter-based
//                RNG (identical at both ends), so theta is never stored (k_fused)
//
// Labels are stored chain-innermost, x[buf][v][c], so that lanes of a warp
// working on consecutive chains of one site or edge read consecutive bytes and
// share the edge's table row (one broadcast load per entry for the warp).
// The dual bits of one (edge, chain) are packed into W = ceil(m/32) words,
// theta[e][c][w].  Both kernels read the sweep index from device memory (Ctl),
// so one sweep can be captured once as a CUDA graph and replayed.
#pragma once
#include "common.cuh"

namespace mrfk {

// ---------------------------------------------------------------------------- dual bits

// Threshold of entry word `w` for the dual-logit case (y, z): logit is -tau, 0
// or +tau; 0 marks an entry without a dual bit.
__device__ __forceinline__ uint32_t case_threshold(uint32_t w, int y, int z) {
    const uint32_t tp = w & 0x1FFFFFFu;
    const uint32_t tm = (1u << 24) - tp + ((w >> 25) & 3u) - 1u;
    const int lvl = (w >> 31) ? (z - y + 1) : (y + z);      // 0: -tau, 1: 0, 2: +tau
    const uint32_t t = lvl == 0 ? tm : (lvl == 1 ? (1u << 23) : tp);
    return w ? t : 0u;
}

// Dual bits of edge e, chain c, given the endpoint labels (xs, xt).  The 8-bit
// prefix of each uniform decides unless it equals the threshold's prefix; only
// then are the low 16 bits drawn (the comparison result is the same as with
// the full 24-bit uniform).
template <int L, int LAYOUT>
__device__ __forceinline__ void dual_bits(uint32_t e, uint32_t c, int xs, int xt, const uint32_t* __restrict__ thr_e,
                                          uint32_t sweep, uint2 key, uint32_t (&bits)[Ent<L, LAYOUT>::W]) {
    using E = Ent<L, LAYOUT>;
#pragma unroll
    for (int w = 0; w < E::W; ++w) bits[w] = 0;
#pragma unroll
    for (int kb = 0; kb < (E::M + 15) / 16; ++kb) {
        const uint4 r = draw(e, sweep, c, PH_DUAL, (uint32_t)kb, key);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const int k = kb * 16 + kk;
            if (k < E::M) {
                const uint32_t t = case_threshold(__ldg(thr_e + k), xs == E::i(k), xt == E::j(k));
                const uint32_t pre = (word_of(r, kk >> 2) >> (8 * (kk & 3))) & 0xFFu;
                const uint32_t th = t >> 16;
                uint32_t bit = pre < th;
                if (pre == th && (t & 0xFFFFu)) bit = dual_low16(e, sweep, c, k, key) < (t & 0xFFFFu);
                bits[k >> 5] |= bit << (k & 31);
            }
        }
    }
}

// ---------------------------------------------------------------------------- label draw

// Draw x_v from exp(F)/Z by the inverse CDF with u from Philox (phase `phase`);
// optionally record log p.  Counts draws within 1e-6 of a CDF boundary.
template <int L>
__device__ __forceinline__ int draw_label(const double (&F)[L], uint32_t v, uint32_t c, uint32_t sweep, uint2 key,
                                          uint32_t phase, float* __restrict__ logp_out, Ctl* ctl) {
    double mx = F[0];
#pragma unroll
    for (int a = 1; a < L; ++a) mx = fmax(mx, F[a]);
    float d[L], ex[L];
    float s = 0.0f;
#pragma unroll
    for (int a = 0; a < L; ++a) {
        d[a] = (float)(F[a] - mx);
        ex[a] = expf(d[a]);
        s += ex[a];
    }
    const float inv = 1.0f / s;
    if (logp_out) {
        const float ls = logf(s);
#pragma unroll
        for (int a = 0; a < L; ++a) logp_out[a] = d[a] - ls;
    }
    const uint32_t U = draw(v, sweep, c, phase, 0, key).x >> 8;
    const double u = ((double)U + 0.5) * (1.0 / 16777216.0);
    float cdf = 0.0f;
    int lab = -1, last_pos = 0;
    bool near = false;
#pragma unroll
    for (int a = 0; a < L; ++a) {
        const float p = ex[a] * inv;
        cdf += p;
        if (p > 0.0f) last_pos = a;
        if (lab < 0 && u < (double)cdf) lab = a;
        near |= fabs(u - (double)cdf) < 1e-6;
    }
    if (near) atomicAdd(&ctl->boundary, 1ull);
    return lab < 0 ? last_pos : lab;
}

// ---------------------------------------------------------------------------- kernels

template <int L, int LAYOUT>
__global__ void __launch_bounds__(256) k_dual(SweepArgs a) {
    using E = Ent<L, LAYOUT>;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= a.E * a.C) return;
    const int64_t e = g / a.C;
    const uint32_t c = (uint32_t)(g % a.C);
    const uint32_t sweep = (uint32_t)a.ctl->sweep;
    const uint8_t* xin = a.x + (size_t)(sweep & 1) * a.N * a.C;
    uint32_t bits[E::W];
    const int s = a.src[e];
    if (s >= 0) {
        const int t = a.dst[e];
        dual_bits<L, LAYOUT>((uint32_t)e, c, xin[(int64_t)s * a.C + c], xin[(int64_t)t * a.C + c],
                             a.thr + e * E::M, sweep, a.key, bits);
    } else {
#pragma unroll
        for (int w = 0; w < E::W; ++w) bits[w] = 0;
    }
    uint32_t* out = a.theta + g * E::W;
#pragma unroll
    for (int w = 0; w < E::W; ++w) out[w] = bits[w];
}

// Accumulate the beta terms of edge e's set dual bits for one endpoint side.
template <int L, int LAYOUT>
__device__ __forceinline__ void add_side(const uint32_t (&bits)[Ent<L, LAYOUT>::W], const float* __restrict__ tau_e,
                                         int side, float (&acc)[L]) {
    using E = Ent<L, LAYOUT>;
    if (side == 0) {
#pragma unroll
        for (int k = 0; k < E::M; ++k)
            if ((bits[k >> 5] >> (k & 31)) & 1u) acc[E::i(k)] += __ldg(tau_e + k);
    } else {
#pragma unroll
        for (int k = 0; k < E::M; ++k)
            if ((bits[k >> 5] >> (k & 31)) & 1u) acc[E::j(k)] += fabsf(__ldg(tau_e + k));
    }
}

// FUSED = false: read theta written by k_dual.  FUSED = true: regenerate it.
template <int L, int LAYOUT, bool FUSED>
__global__ void __launch_bounds__(256) k_primal(SweepArgs a) {
    using E = Ent<L, LAYOUT>;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)a.N * a.C) return;
    const uint32_t v = (uint32_t)(g / a.C), c = (uint32_t)(g % a.C);
    const uint32_t sweep = (uint32_t)a.ctl->sweep;
    const uint8_t* xin = a.x + (size_t)(sweep & 1) * a.N * a.C;
    uint8_t* xout = a.x + (size_t)((sweep + 1) & 1) * a.N * a.C;
    double F[L];
    float acc[L];
#pragma unroll
    for (int x = 0; x < L; ++x) { F[x] = a.ut[(int64_t)v * L + x]; acc[x] = 0.0f; }
    int xv = 0;
    if (FUSED) xv = xin[g];
    const int64_t p0 = a.inc_ptr[v], p1 = a.inc_ptr[v + 1];
    int chunk = 0;
    for (int64_t p = p0; p < p1; ++p) {
        const int2 ic = a.inc[p];
        const int64_t e = ic.x >> 1;
        const int side = ic.x & 1;
        uint32_t bits[E::W];
        if (FUSED) {
            const int xn = xin[(int64_t)ic.y * a.C + c];
            dual_bits<L, LAYOUT>((uint32_t)e, c, side == 0 ? xv : xn, side == 0 ? xn : xv, a.thr + e * E::M, sweep,
                                 a.key, bits);
        } else {
            const uint32_t* th = a.theta + (e * a.C + c) * E::W;
#pragma unroll
            for (int w = 0; w < E::W; ++w) bits[w] = th[w];
        }
        add_side<L, LAYOUT>(bits, a.tau + e * E::M, side, acc);
        if (++chunk == 16) {            // fp32 partial sums per 16 edges, fp64 across chunks
#pragma unroll
            for (int x = 0; x < L; ++x) { F[x] += acc[x]; acc[x] = 0.0f; }
            chunk = 0;
        }
    }
#pragma unroll
    for (int x = 0; x < L; ++x) F[x] += acc[x];
    float* lp = a.logp ? a.logp + ((int64_t)c * a.N + v) * L : nullptr;
    xout[g] = (uint8_t)draw_label<L>(F, v, c, sweep, a.key, PH_PRIMAL, lp, a.ctl);
}

static inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

template <int L, int LAYOUT>
cudaError_t run_dual(const SweepArgs& a, cudaStream_t s) {
    const int64_t n = a.E * a.C;
    if (n > 0) k_dual<L, LAYOUT><<<blocks_for(n, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <int L, int LAYOUT, bool FUSED>
cudaError_t run_primal(const SweepArgs& a, cudaStream_t s) {
    const int64_t n = (int64_t)a.N * a.C;
    if (n > 0) k_primal<L, LAYOUT, FUSED><<<blocks_for(n, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

#define MRF_INSTANTIATE_SWEEP(L)                                                                 \
    template cudaError_t run_dual<L, MRF_LAYOUT_PIVOT>(const SweepArgs&, cudaStream_t);           \
    template cudaError_t run_dual<L, MRF_LAYOUT_DIAG>(const SweepArgs&, cudaStream_t);            \
    template cudaError_t run_primal<L, MRF_LAYOUT_PIVOT, false>(const SweepArgs&, cudaStream_t);  \
    template cudaError_t run_primal<L, MRF_LAYOUT_DIAG, false>(const SweepArgs&, cudaStream_t);   \
    template cudaError_t run_primal<L, MRF_LAYOUT_PIVOT, true>(const SweepArgs&, cudaStream_t);   \
    template cudaError_t run_primal<L, MRF_LAYOUT_DIAG, true>(const SweepArgs&, cudaStream_t);

}  // namespace mrfk
