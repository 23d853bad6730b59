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
//                RNG (identical at both ends), so theta is never stored
//
// Labels are stored chain-innermost, x[buf][v][c], so that lanes of a warp
// working on consecutive chains of one site or edge read consecutive bytes and
// share the edge's table row (one broadcast load per word for the warp).
// The dual bits of one (edge, chain) are packed into W = ceil(m/32) words,
// theta[e][c][w].  The kernels read the sweep index from device memory (Ctl),
// so one sweep can be captured once as a CUDA graph and replayed.
#pragma once
#include "common.cuh"

namespace mrfk {

// ---------------------------------------------------------------------------- entry masks

// Bits [lo, hi) of a 32-bit word (lo, hi relative to the word, clipped).
__device__ __forceinline__ uint32_t range_mask(int lo, int hi) {
    lo = max(lo, 0);
    hi = min(hi, 32);
    if (hi <= lo) return 0u;
    const uint32_t upto = hi == 32 ? 0xFFFFFFFFu : ((1u << hi) - 1u);
    return upto & ~((1u << lo) - 1u);
}

// Word g of the PIVOT column-1 pattern: entries k = r (L-1), r = 0..L-2.
__host__ __device__ constexpr uint32_t col_pattern_word(int L, int g) {
    uint32_t w = 0;
    for (int r = 0; r < L - 1; ++r) {
        const int k = r * (L - 1) - 32 * g;
        if (k >= 0 && k < 32) w |= 1u << k;
    }
    return w;
}

__host__ __device__ constexpr uint32_t valid_word(int M, int g) {
    return M - 32 * g >= 32 ? 0xFFFFFFFFu : (M - 32 * g <= 0 ? 0u : ((1u << (M - 32 * g)) - 1u));
}

// Entries of group g whose row is label a (y = 1) and whose column is b (z = 1).
template <int L, int LAYOUT>
__device__ __forceinline__ uint32_t row_mask(int a, int g) {
    if (LAYOUT == MRF_LAYOUT_DIAG) return (a >> 5) == g ? (1u << (a & 31)) : 0u;
    if (a == 0) return 0u;
    const int lo = (a - 1) * (L - 1) - 32 * g;
    return range_mask(lo, lo + L - 1);
}

template <int L, int LAYOUT>
__device__ __forceinline__ uint32_t col_mask(int b, int g) {
    if (LAYOUT == MRF_LAYOUT_DIAG) return (b >> 5) == g ? (1u << (b & 31)) : 0u;
    if (b == 0) return 0u;
    const uint32_t hi = col_pattern_word(L, g);
    const uint32_t lo = g > 0 ? col_pattern_word(L, g - 1) : 0u;
    return __funnelshift_l(lo, hi, (unsigned)(b - 1));
}

// ---------------------------------------------------------------------------- blocked sweep

// Offset (ox, oy, oz) of the block grid of the current blocked sweep.
__device__ __forceinline__ void splash_offset(const Ctl* ctl, int& ox, int& oy, int& oz) {
    const uint32_t o = (uint32_t)ctl->splash_offset;
    ox = o & 0xFF; oy = (o >> 8) & 0xFF; oz = (o >> 16) & 0xFF;
}

// Lowest coordinate of the (clipped) 4-block containing coordinate x.
__device__ __forceinline__ int block_lo(int x, int o) { return max(0, ((x + o) >> 2) * 4 - o); }

// Is lattice edge slot e an edge of the comb forest of the current blocked
// sweep?  x-edges inside a block always are; y-edges when both ends have
// local x = 0; z-edges when both ends have local x = y = 0.
__device__ __forceinline__ bool is_tree_edge(const SweepArgs& a, uint32_t e) {
    int ox, oy, oz;
    splash_offset(a.ctl, ox, oy, oz);
    if (e < (uint64_t)a.nxe) {
        const uint32_t r = a.fdX1.div(e);
        const int x = (int)(e - r * (uint32_t)(a.grid_nx - 1));
        return ((x + ox) >> 2) == ((x + 1 + ox) >> 2);
    }
    if (e < (uint64_t)(a.nxe + a.nye)) {
        const uint32_t f = e - (uint32_t)a.nxe;
        const uint32_t r = a.fdX.div(f);
        const int x = (int)(f - r * (uint32_t)a.grid_nx);
        const uint32_t r2 = a.fdY1.div(r);
        const int y = (int)(r - r2 * (uint32_t)(a.grid_ny - 1));
        return x == block_lo(x, ox) && ((y + oy) >> 2) == ((y + 1 + oy) >> 2);
    }
    const uint32_t f = e - (uint32_t)(a.nxe + a.nye);
    const uint32_t r = a.fdX.div(f);
    const int x = (int)(f - r * (uint32_t)a.grid_nx);
    const uint32_t z = a.fdY.div(r);
    const int y = (int)(r - z * (uint32_t)a.grid_ny);
    return x == block_lo(x, ox) && y == block_lo(y, oy) && ((int(z) + oz) >> 2) == ((int(z) + 1 + oz) >> 2);
}

// ---------------------------------------------------------------------------- dual bits

// Row and column masks of the entries of a PIVOT table with at most 64
// entries as 64-bit words: entries (xs, j) and (i, xt).
template <int L>
__device__ __forceinline__ void pivot_masks64(int xs, int xt, uint64_t& Y, uint64_t& Z) {
    constexpr int R = L - 1;
    constexpr uint64_t row = (1ull << R) - 1ull;
    uint64_t col = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) col |= 1ull << (R * r);
    Y = xs ? row << (R * (xs - 1)) : 0ull;
    Z = xt ? col << (xt - 1) : 0ull;
}

// Dual bits of edge e, chain c, given the endpoint labels (xs, xt).
// Bit-sliced: the 8-bit prefixes of 32 uniforms arrive as 8 bit planes (two
// Philox calls per group of 32 entries; one call, two planes per word, when
// the table has at most 16 entries).  An entry's dual logit q + beta1 y +
// beta2 z sits at one of three levels, fixed by its sign s = [l < 0] and its
// case y = [x_s = i_k], z = [x_t = j_k]:
//   s = 0: level y + z,   s = 1: level z - y + 1   (0: -tau, 1: 0, 2: +tau)
// so with X = S ^ Y over a group's masks:
//   L0 = Act & ~Z & ~X,   L2 = Act & Z & X,   L1 = Act & ~(L0 | L2).
// Level 1 is p = 1/2 exactly (T = 2^23): its bit is the complement of the
// prefix's top bit.  For levels 0 and 2 the planes of the matching threshold
// prefix, t = B ^ (AB & L0) (k_build_planes), are compared with the random
// planes least significant first:
//   lt = (~r & t) | (~(r ^ t) & lt)        prefix <  threshold prefix
//   le = (~r & t) | (~(r ^ t) & le)        prefix <= threshold prefix
// Returns lt in bits, the ties le & ~lt (probability 1/256 per entry) in ties
// and the level-2 mask in lev2; a tie is decided by the low 16 bits of its
// uniform against the exact threshold of its level (resolve_tie).
template <int L, int LAYOUT>
__device__ __forceinline__ void dual_prefix_bits(uint32_t e, uint32_t c, int xs, int xt,
                                                 const uint32_t* __restrict__ tpl_e, uint32_t sweep,
                                                 const RoundKeys& key, uint32_t (&bits)[Ent<L, LAYOUT>::W],
                                                 uint32_t (&ties)[Ent<L, LAYOUT>::W],
                                                 uint32_t (&lev2)[Ent<L, LAYOUT>::W]) {
    using E = Ent<L, LAYOUT>;
    const uint4* tp = reinterpret_cast<const uint4*>(tpl_e);
    if constexpr (E::M <= 16) {
        // one Philox call: word p = plane p (bits 0..15) and plane p + 4 (bits
        // 16..31); the low halves compare the prefix's high nibble, the high
        // halves its low nibble, combined at the end
        const uint4 r4 = draw_rk(e, sweep, c, PH_DUAL, 0u, key);
        const uint32_t R[4] = {r4.x, r4.y, r4.z, r4.w};
        const uint4 qa = __ldg(tp), qb = __ldg(tp + 1);
        const uint32_t sa = __ldg(tpl_e + 8);
        const uint32_t AB[4] = {qa.x, qa.y, qa.z, qa.w}, B[4] = {qb.x, qb.y, qb.z, qb.w};
        const uint32_t Y = row_mask<L, LAYOUT>(xs, 0), Z = col_mask<L, LAYOUT>(xt, 0);
        const uint32_t X = (sa & 0xFFFFu) ^ Y, act = sa >> 16;
        const uint32_t l0 = act & ~Z & ~X, l2 = act & Z & X, l02 = l0 | l2;
        const uint32_t L0 = l0 | (l0 << 16);
        uint32_t lt = 0u, le = 0xFFFFFFFFu;
#pragma unroll
        for (int p = 3; p >= 0; --p) {
            const uint32_t t = B[p] ^ (AB[p] & L0), r = R[p];
            lt = (~r & t) | (~(r ^ t) & lt);
            le = (~r & t) | (~(r ^ t) & le);
        }
        const uint32_t eq = le & ~lt;
        bits[0] = ((lt | (eq & (lt >> 16))) & l02) | (~R[0] & act & ~l02);
        ties[0] = eq & (eq >> 16) & l02;
        lev2[0] = l2;
        return;
    }
    constexpr bool M64 = LAYOUT == MRF_LAYOUT_PIVOT && E::M <= 64;
    uint64_t Y64 = 0, Z64 = 0;
    if constexpr (M64) pivot_masks64<L>(xs, xt, Y64, Z64);
    // the first two groups' four Philox calls share their first rounds and are in flight together
    constexpr int GA = E::W < 2 ? E::W : 2;
    uint4 RA[2 * GA];
    draw_rk_subs<2 * GA>(e, sweep, c, PH_DUAL, key, RA);
#pragma unroll
    for (int g = 0; g < E::W; ++g) {
        uint4 r0, r1;
        if (g < GA) {
            r0 = RA[2 * (g < GA ? g : 0)];
            r1 = RA[2 * (g < GA ? g : 0) + 1];
        } else {
            r0 = draw_rk(e, sweep, c, PH_DUAL, 2u * g, key);
            r1 = draw_rk(e, sweep, c, PH_DUAL, 2u * g + 1u, key);
        }
        const uint32_t Rg[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
        const uint4* tg = tp + 5 * g;
        const uint4 sq = __ldg(tg + 4);                    // {S, Act}
        uint32_t Y, Z;
        if constexpr (M64) {
            Y = (uint32_t)(Y64 >> (32 * g));
            Z = (uint32_t)(Z64 >> (32 * g));
        } else {
            Y = row_mask<L, LAYOUT>(xs, g);
            Z = col_mask<L, LAYOUT>(xt, g);
        }
        const uint32_t X = sq.x ^ Y;
        const uint32_t L0 = sq.y & ~Z & ~X, L2 = sq.y & Z & X, L02 = L0 | L2;
        uint32_t lt = 0u, le = 0xFFFFFFFFu;
#pragma unroll
        for (int h = 3; h >= 0; --h) {
            const uint4 q = __ldg(tg + h);                 // {AB_2h, B_2h, AB_2h+1, B_2h+1}
            uint32_t t = q.w ^ (q.z & L0), r = Rg[2 * h + 1];
            lt = (~r & t) | (~(r ^ t) & lt);
            le = (~r & t) | (~(r ^ t) & le);
            t = q.y ^ (q.x & L0); r = Rg[2 * h];
            lt = (~r & t) | (~(r ^ t) & lt);
            le = (~r & t) | (~(r ^ t) & le);
        }
        bits[g] = (lt & L02) | (~Rg[0] & sq.y & ~L02);
        ties[g] = le & ~lt & L02;
        lev2[g] = L2;
    }
}

// Decision of a tie at entry k (its 8-bit prefix equals the prefix of the
// threshold T of its level): low 16 bits of the uniform < T - (prefix << 16).
__device__ __forceinline__ bool resolve_tie(uint32_t e, uint32_t c, bool lev2, int k, uint32_t thr_word,
                                            uint32_t sweep, const RoundKeys& key) {
    const uint32_t t = level_threshold(thr_word, lev2);
    const uint32_t rem = t - (threshold_prefix(t) << 16);      // in [0, 65536]
    return rem && dual_low16(e, sweep, c, k, key) < rem;
}

// Dual bits with the ties decided by the thread itself, one after another.
template <int L, int LAYOUT>
__device__ __forceinline__ void dual_bits(uint32_t e, uint32_t c, int xs, int xt, const uint32_t* __restrict__ tpl_e,
                                          const uint32_t* __restrict__ thr_e, uint32_t sweep, const RoundKeys& key,
                                          uint32_t (&bits)[Ent<L, LAYOUT>::W]) {
    using E = Ent<L, LAYOUT>;
    uint32_t ties[E::W], lev2[E::W];
    dual_prefix_bits<L, LAYOUT>(e, c, xs, xt, tpl_e, sweep, key, bits, ties, lev2);
#pragma unroll 1
    for (int g = 0; g < E::W; ++g) {
        uint32_t tg = ties[g];
        while (tg) {
            const int b = __ffs(tg) - 1;
            tg &= tg - 1u;
            const int k = 32 * g + b;
            if (resolve_tie(e, c, (lev2[g] >> b) & 1u, k, __ldg(thr_e + k), sweep, key)) bits[g] |= 1u << b;
        }
    }
}

// ---------------------------------------------------------------------------- label draw

// Draw x_v from exp(F)/Z by the inverse CDF with the 23-bit uniform u of
// Philox phase `phase` (u is exact in float32); optionally record log p.
// Counts draws within 1e-6 of a CDF boundary.
// lp_drawn (optional) receives log p of the drawn label.
template <int L>
__device__ __forceinline__ int draw_label(const float (&F)[L], uint32_t v, uint32_t c, uint32_t sweep,
                                          const RoundKeys& key, uint32_t phase, float* __restrict__ logp_out, Ctl* ctl,
                                          float* __restrict__ lp_drawn = nullptr) {
    float mx = F[0];
#pragma unroll
    for (int a = 1; a < L; ++a) mx = fmaxf(mx, F[a]);
    float ex[L];
    float s = 0.0f;
#pragma unroll
    for (int a = 0; a < L; ++a) {
        ex[a] = expf(F[a] - mx);
        s += ex[a];
    }
    const float inv = 1.0f / s;
    if (logp_out) {
        const float ls = logf(s);
#pragma unroll
        for (int a = 0; a < L; ++a) logp_out[a] = (F[a] - mx) - ls;
    }
    const uint32_t U = draw_rk(v, sweep, c, phase, 0, key).x >> 9;
    const float u = ((float)U + 0.5f) * (1.0f / 8388608.0f);
    float cdf = 0.0f;
    int lab = -1, last_pos = 0;
    bool near = false;
#pragma unroll
    for (int a = 0; a < L; ++a) {
        const float p = ex[a] * inv;
        cdf += p;
        if (p > 0.0f) last_pos = a;
        if (lab < 0 && u < cdf) lab = a;
        near |= fabsf(u - cdf) < 1e-6f;
    }
    if (near) atomicAdd(&ctl->boundary, 1ull);
    const int pick = lab < 0 ? last_pos : lab;
    if (lp_drawn) {
        float fp = F[0];
#pragma unroll
        for (int a = 1; a < L; ++a) fp = a == pick ? F[a] : fp;
        *lp_drawn = (fp - mx) - logf(s);
    }
    return pick;
}

// ---------------------------------------------------------------------------- kernels

// Dual step.  A warp takes NG consecutive groups of 32 (edge, chain) items
// (item g = e C + c, one item per lane).  A tie needs one more Philox call and
// a scattered threshold word; deciding it in the owning lane would hold the
// whole warp for a few lanes.  Instead the warp stages its dual words in
// shared memory and queues every nonzero tie word of a lane as one entry
// {group, lane, word | tie mask | level-2 mask}; after its NG groups the warp
// decides the queued entries with one entry per lane per round and ORs the
// won bits into the staged words, which are then stored.  Ties of a lane
// whose entry does not fit the queue are decided by the lane itself.
template <int M, int W>
struct DualTile {
    static constexpr int WARPS = 8;                                         // 256 threads
    static constexpr int NG = W >= 4 ? 2 : (M >= 32 ? 4 : (M >= 8 ? 8 : 16));
    // nonzero tie words expected per warp: NG 32 W (1 - (1 - 1/256)^32) <= NG 32 M / 256;
    // capacity twice that plus 32, in whole rounds of 32
    static constexpr int Q = ((NG * 32 * M * 2 / 256 + 32) + 31) / 32 * 32;
};

// FEW: the launch bounds of the form for fewer than 32 chains (run_dual).
template <int L, int LAYOUT, bool FEW = false>
__global__ void __launch_bounds__(256, FEW ? 2 : 4) k_dual(SweepArgs a) {
    using E = Ent<L, LAYOUT>;
    using T = DualTile<E::M, E::W>;
    constexpr int W = E::W, NG = T::NG, Q = T::Q;
    constexpr uint32_t FULL = 0xFFFFFFFFu;
    __shared__ uint32_t s_th[T::WARPS][NG * W][32];        // staged dual words, [group, word][lane]
    __shared__ uint4 s_q[T::WARPS][Q];                     // queued tie words
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    const uint64_t n_items = (uint64_t)a.E * a.C;          // < 2^32 (checked by the host)
    const uint64_t base = ((uint64_t)blockIdx.x * T::WARPS + warp) * (NG * 32);
    const uint32_t sweep = (uint32_t)a.ctl->sweep;
    const uint8_t* xin = a.x + (size_t)(sweep & 1) * a.N * a.C;
    int nq = 0;                                            // entries queued (warp-uniform)
#pragma unroll 1
    for (int j = 0; j < NG; ++j) {
        const uint64_t g64 = base + 32 * j + lane;
        const uint32_t g = (uint32_t)g64;
        const bool in_range = g64 < n_items;
        const uint32_t e = in_range ? a.fdC.div(g) : 0u;
        const uint32_t c = g - e * (uint32_t)a.C;
        uint32_t bits[W], ties[W], lev2[W];
        const int s = in_range ? a.src[e] : -1;
        if (s >= 0 && !(a.splash && is_tree_edge(a, e)) && !(a.skip && a.skip[e])) {
            const int t = a.dst[e];
            const int xs = xin[(int64_t)s * a.C + c], xt = xin[(int64_t)t * a.C + c];
            dual_prefix_bits<L, LAYOUT>(e, c, xs, xt, a.tpl + (int64_t)e * E::PW, sweep, a.rk, bits, ties, lev2);
        } else {
#pragma unroll
            for (int w = 0; w < W; ++w) { bits[w] = 0u; ties[w] = 0u; lev2[w] = 0u; }
        }
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const bool has = ties[w] != 0u;
            const uint32_t bal = __ballot_sync(FULL, has);
            const int pos = nq + __popc(bal & below);
            nq += __popc(bal);
            if (has) {
                if (pos < Q) {
                    s_q[warp][pos] = make_uint4((uint32_t)(j * W + w) | ((uint32_t)lane << 8), ties[w], lev2[w] & ties[w], 0u);
                } else {
                    uint32_t tw = ties[w];                 // queue full: decide here
                    while (tw) {
                        const int b = __ffs(tw) - 1;
                        tw &= tw - 1u;
                        const int k = 32 * w + b;
                        if (resolve_tie(e, c, (lev2[w] >> b) & 1u, k, __ldg(a.thr + (int64_t)e * E::M + k), sweep, a.rk))
                            bits[w] |= 1u << b;
                    }
                }
            }
            s_th[warp][j * W + w][lane] = bits[w];
        }
    }
    __syncwarp();
    const int nres = nq < Q ? nq : Q;
#pragma unroll 1
    for (int r = lane; r < nres; r += 32) {
        const uint4 q = s_q[warp][r];
        const int jw = (int)(q.x & 0xFFu), l = (int)(q.x >> 8), j = jw / W, w = jw - j * W;
        const uint32_t g = (uint32_t)(base + 32 * j + l);
        const uint32_t e = a.fdC.div(g), c = g - e * (uint32_t)a.C;
        uint32_t tw = q.y, won = 0u;
        while (tw) {
            const int b = __ffs(tw) - 1;
            tw &= tw - 1u;
            const int k = 32 * w + b;
            if (resolve_tie(e, c, (q.z >> b) & 1u, k, __ldg(a.thr + (int64_t)e * E::M + k), sweep, a.rk)) won |= 1u << b;
        }
        if (won) atomicOr(&s_th[warp][jw][l], won);
    }
    __syncwarp();
#pragma unroll 1
    for (int j = 0; j < NG; ++j) {
        const uint64_t g64 = base + 32 * j + lane;
        if (g64 >= n_items) break;
        uint32_t* out = a.theta + g64 * W;
        if (W % 2 == 0) {
#pragma unroll
            for (int w = 0; w < W; w += 2)
                *reinterpret_cast<uint2*>(out + w) = make_uint2(s_th[warp][j * W + w][lane], s_th[warp][j * W + (w + 1 < W ? w + 1 : w)][lane]);
        } else {
#pragma unroll
            for (int w = 0; w < W; ++w) out[w] = s_th[warp][j * W + w][lane];
        }
    }
}

// Accumulate the beta terms of edge e's set dual bits for one endpoint side
// (tau row loaded as 16-byte vectors; beta1 = tau_signed, beta2 = |tau_signed|).
// GLOBAL: the row is in global memory (read-only path); else in shared memory.
template <int L, int LAYOUT, bool GLOBAL = true>
__device__ __forceinline__ void add_side(const uint32_t (&bits)[Ent<L, LAYOUT>::W], const float* __restrict__ tau_e,
                                         int side, float (&acc)[L]) {
    using E = Ent<L, LAYOUT>;
    const float4* t4 = reinterpret_cast<const float4*>(tau_e);
    if (side == 0) {
#pragma unroll
        for (int k4 = 0; k4 < E::MP / 4; ++k4) {
            const float4 q = GLOBAL ? __ldg(t4 + k4) : t4[k4];
            const float tv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = 4 * k4 + u;
                if (k < E::M && ((bits[k >> 5] >> (k & 31)) & 1u)) acc[E::i(k)] += tv[u];
            }
        }
    } else {
#pragma unroll
        for (int k4 = 0; k4 < E::MP / 4; ++k4) {
            const float4 q = GLOBAL ? __ldg(t4 + k4) : t4[k4];
            const float tv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = 4 * k4 + u;
                if (k < E::M && ((bits[k >> 5] >> (k & 31)) & 1u)) acc[E::j(k)] += fabsf(tv[u]);
            }
        }
    }
}

// Compensated (two-sum) flush of a float32 partial sum into a hi/lo pair, used
// every 32 incident edges so that high-degree sites keep ~double precision.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

// FUSED = false: read theta written by k_dual.  FUSED = true: regenerate it.
// POT = true (blocked sweep): write the node potentials F to a.pot instead of
// drawing labels.
// Four blocks per SM even where the field arrays of wide tables spill at 64
// registers (L = 9: 354 B, L = 16: 702 B): fewer blocks measured slower (L = 8,
// one chain: 0.403 vs 0.386 ms; L = 10, 8 chains: 0.68 vs 0.60 ms; L = 12, 16
// chains: 0.39 vs 0.26 ms; L = 16, 8 chains: 2.22 vs 1.34 ms).
template <int L, int LAYOUT, bool FUSED, bool POT = false>
__global__ void __launch_bounds__(256, FUSED ? 2 : 4) k_primal(SweepArgs a) {
    using E = Ent<L, LAYOUT>;
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;     // N * C < 2^32 (checked by the host)
    if (g >= (uint64_t)a.N * a.C) return;
    const uint32_t v = a.fdC.div(g), c = g - v * (uint32_t)a.C;
    const uint32_t sweep = (uint32_t)a.ctl->sweep;
    const uint8_t* xin = a.x + (size_t)(sweep & 1) * a.N * a.C;
    uint8_t* xout = a.x + (size_t)((sweep + 1) & 1) * a.N * a.C;
    float acc[L], hi[L], lo[L];
#pragma unroll
    for (int x = 0; x < L; ++x) { acc[x] = 0.0f; hi[x] = 0.0f; lo[x] = 0.0f; }
    int xv = 0;
    if (FUSED) xv = xin[g];
    const int64_t p0 = a.inc_ptr[v], p1 = a.inc_ptr[v + 1];
    int chunk = 0;
    bool flushed = false;
    // Incidences in batches of B: all incidence records and (plain form) all
    // theta words of a batch are loaded before any is used, so the dependent
    // loads of B edges are in flight together.
    constexpr int B = FUSED ? 1 : 4;
    for (int64_t base = p0; base < p1; base += B) {
        int2 ic[B];
        uint32_t bits[B][E::W];
#pragma unroll
        for (int u = 0; u < B; ++u) ic[u] = base + u < p1 ? __ldg(&a.inc[base + u]) : make_int2(-1, 0);
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int64_t e = ic[u].x >> 1;
            if (ic[u].x < 0) {
#pragma unroll
                for (int w = 0; w < E::W; ++w) bits[u][w] = 0;
            } else if (FUSED) {
                const int side = ic[u].x & 1;
                const int xn = xin[(int64_t)ic[u].y * a.C + c];
                dual_bits<L, LAYOUT>((uint32_t)e, c, side == 0 ? xv : xn, side == 0 ? xn : xv, a.tpl + e * E::PW,
                                     a.thr + e * E::M, sweep, a.rk, bits[u]);
            } else {
                const uint32_t* th = a.theta + (e * a.C + c) * E::W;
                if (E::W % 2 == 0) {
#pragma unroll
                    for (int w = 0; w < E::W; w += 2) {
                        const uint2 q = __ldcs(reinterpret_cast<const uint2*>(th + w));
                        bits[u][w] = q.x;
                        bits[u][w + 1 < E::W ? w + 1 : w] = q.y;
                    }
                } else {
#pragma unroll
                    for (int w = 0; w < E::W; ++w) bits[u][w] = __ldcs(th + w);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
            if (ic[u].x < 0) continue;
            add_side<L, LAYOUT>(bits[u], a.tau + (ic[u].x >> 1) * (int64_t)E::MP, ic[u].x & 1, acc);
            if (++chunk == 32) {
#pragma unroll
                for (int x = 0; x < L; ++x) { two_sum_add(hi[x], lo[x], acc[x]); acc[x] = 0.0f; }
                chunk = 0;
                flushed = true;
            }
        }
    }
    float F[L];
    const float* uf = a.utf + (int64_t)v * L;
    if (flushed) {
#pragma unroll
        for (int x = 0; x < L; ++x) { two_sum_add(hi[x], lo[x], acc[x]); F[x] = __ldg(uf + x) + (hi[x] + lo[x]); }
    } else {
#pragma unroll
        for (int x = 0; x < L; ++x) F[x] = __ldg(uf + x) + acc[x];
    }
    if (POT) {
        float* pv = a.pot + (int64_t)v * L * a.C + c;
#pragma unroll
        for (int x = 0; x < L; ++x) pv[(int64_t)x * a.C] = F[x];
        return;
    }
    float* lp = a.logp ? a.logp + ((int64_t)c * a.N + v) * L : nullptr;
    xout[g] = (uint8_t)draw_label<L>(F, v, c, sweep, a.rk, PH_PRIMAL, lp, a.ctl, a.lpv ? a.lpv + g : nullptr);
}

// Warp-per-site form of the plain primal step (chains a multiple of 32, so a
// warp is one site and 32 of its chains).  BATCH (chosen by the host when no
// site has more than KB incidences, e.g. every lattice): one batch per site --
// the lanes load the incidence records in parallel, every lane issues the
// theta loads of all incidences at once, the incidences' tau rows are staged
// in shared memory (one row per incidence, shared by the 32 chains), then the
// field is summed.  Otherwise chunks of K incidences (same pattern, a two-sum
// flush of the partial sums every 32 incidences).  Both keep k_primal's order
// of additions.
template <int L, int LAYOUT>
struct PrimalWarp {
    static constexpr int MP = Ent<L, LAYOUT>::MP;
    static constexpr int W = Ent<L, LAYOUT>::W;
    static constexpr int K = 2;                          // incidences per chunk of the general path
    static constexpr int KB = W >= 8 ? 2 : (W >= 4 ? 4 : 8);   // one-batch path: degree <= KB
    static constexpr int WARPS = 8;                      // 256 threads
};

template <int L, int LAYOUT, bool POT = false, bool BATCH = false>
__global__ void __launch_bounds__(256, 4) k_primal_warp(SweepArgs a) {
    using E = Ent<L, LAYOUT>;
    using PW = PrimalWarp<L, LAYOUT>;
    constexpr int K = PW::K, KB = PW::KB, MP = PW::MP, Q = MP / 4;    // float4 per tau row
    constexpr uint32_t FULL = 0xFFFFFFFFu;
    __shared__ __align__(16) float4 s_tau[PW::WARPS][KB > K ? KB : K][Q];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;     // N * C < 2^32, C % 32 == 0 (host)
    if (g >= (uint64_t)a.N * a.C) return;                         // whole warps only
    const uint32_t v = a.fdC.div(g), c = g - v * (uint32_t)a.C;
    const uint32_t sweep = (uint32_t)a.ctl->sweep;
    uint8_t* xout = a.x + (size_t)((sweep + 1) & 1) * a.N * a.C;
    const int64_t p0 = a.inc_ptr[v], p1 = a.inc_ptr[v + 1];
    const float4* tau4 = reinterpret_cast<const float4*>(a.tau);
    float F[L];
    const float* uf = a.utf + (int64_t)v * L;
    if constexpr (BATCH) {                                        // every site has at most KB incidences
        const int deg = (int)(p1 - p0);
        float acc[L];
#pragma unroll
        for (int x = 0; x < L; ++x) acc[x] = 0.0f;
        const int code_l = lane < deg ? __ldg(&a.inc[p0 + lane]).x : 0;
        uint32_t bits[KB][E::W];
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            const int cu = __shfl_sync(FULL, code_l, u);
            if (u < deg) {
                const uint32_t* th = a.theta + ((int64_t)(cu >> 1) * a.C + c) * E::W;
                if (E::W % 2 == 0) {
#pragma unroll
                    for (int w = 0; w < E::W; w += 2) {
                        const uint2 q = __ldcs(reinterpret_cast<const uint2*>(th + w));
                        bits[u][w] = q.x;
                        bits[u][w + 1 < E::W ? w + 1 : w] = q.y;
                    }
                } else {
#pragma unroll
                    for (int w = 0; w < E::W; ++w) bits[u][w] = __ldcs(th + w);
                }
            }
        }
#pragma unroll
        for (int i0 = 0; i0 < KB * Q; i0 += 32) {
            const int i = i0 + lane;
            const int u = i / Q;
            const int cu = __shfl_sync(FULL, code_l, u < KB ? u : 0);
            if (i < KB * Q && u < deg) s_tau[warp][u][i - u * Q] = __ldg(tau4 + (int64_t)(cu >> 1) * Q + (i - u * Q));
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            if (u >= deg) break;
            const int cu = __shfl_sync(FULL, code_l, u);
            add_side<L, LAYOUT, false>(bits[u], reinterpret_cast<const float*>(&s_tau[warp][u][0]), cu & 1, acc);
        }
#pragma unroll
        for (int x = 0; x < L; ++x) F[x] = __ldg(uf + x) + acc[x];
    } else {
        float acc[L], hi[L], lo[L];
    #pragma unroll
        for (int x = 0; x < L; ++x) { acc[x] = 0.0f; hi[x] = 0.0f; lo[x] = 0.0f; }
        int chunk = 0;
        bool flushed = false;
        for (int64_t base = p0; base < p1; base += K) {              // warp-uniform
            const int cnt = p1 - base < K ? (int)(p1 - base) : K;
            const int code_l = lane < cnt ? __ldg(&a.inc[base + lane]).x : 0;
            // tau rows of the chunk -> shared memory (uniform trip count; lanes split the float4s)
    #pragma unroll
            for (int i0 = 0; i0 < K * Q; i0 += 32) {
                const int i = i0 + lane;
                const int u = i / Q;
                const int cu = __shfl_sync(FULL, code_l, u < K ? u : 0);
                if (i < K * Q && u < cnt) s_tau[warp][u][i - u * Q] = __ldg(tau4 + (int64_t)(cu >> 1) * Q + (i - u * Q));
            }
            uint32_t bits[K][E::W];
            int code[K];
    #pragma unroll
            for (int u = 0; u < K; ++u) {
                code[u] = __shfl_sync(FULL, code_l, u);
                if (u < cnt) {
                    const uint32_t* th = a.theta + ((int64_t)(code[u] >> 1) * a.C + c) * E::W;
                    if (E::W % 2 == 0) {
    #pragma unroll
                        for (int w = 0; w < E::W; w += 2) {
                            const uint2 q = __ldcs(reinterpret_cast<const uint2*>(th + w));
                            bits[u][w] = q.x;
                            bits[u][w + 1 < E::W ? w + 1 : w] = q.y;
                        }
                    } else {
    #pragma unroll
                        for (int w = 0; w < E::W; ++w) bits[u][w] = __ldcs(th + w);
                    }
                }
            }
            __syncwarp();
    #pragma unroll
            for (int u = 0; u < K; ++u) {
                if (u >= cnt) break;
                add_side<L, LAYOUT, false>(bits[u], reinterpret_cast<const float*>(&s_tau[warp][u][0]), code[u] & 1, acc);
                if (++chunk == 32) {
    #pragma unroll
                    for (int x = 0; x < L; ++x) { two_sum_add(hi[x], lo[x], acc[x]); acc[x] = 0.0f; }
                    chunk = 0;
                    flushed = true;
                }
            }
            __syncwarp();                                              // rows consumed before the next chunk
        }
        if (flushed) {
    #pragma unroll
            for (int x = 0; x < L; ++x) { two_sum_add(hi[x], lo[x], acc[x]); F[x] = __ldg(uf + x) + (hi[x] + lo[x]); }
        } else {
    #pragma unroll
            for (int x = 0; x < L; ++x) F[x] = __ldg(uf + x) + acc[x];
        }
    }
    if (POT) {
        float* pv = a.pot + (int64_t)v * L * a.C + c;
#pragma unroll
        for (int x = 0; x < L; ++x) pv[(int64_t)x * a.C] = F[x];
        return;
    }
    float* lp = a.logp ? a.logp + ((int64_t)c * a.N + v) * L : nullptr;
    xout[g] = (uint8_t)draw_label<L>(F, v, c, sweep, a.rk, PH_PRIMAL, lp, a.ctl, a.lpv ? a.lpv + g : nullptr);
}

// CTA-per-site schedule of the plain primal step for high-degree sites: a CTA
// of 256 threads covers one site and CG = min(C, 32) chains; its CG x S threads
// (S = 256 / CG incidence slices) each sum a strided share of the incidence
// list for one chain, the S partial sums are combined in shared memory with
// the two-sum pair, and the first slice draws the labels.
template <int L, int LAYOUT>
__global__ void __launch_bounds__(256) k_primal_cta(SweepArgs a, int CG) {
    using E = Ent<L, LAYOUT>;
    __shared__ float red_hi[256][L];
    __shared__ float red_lo[256][L];
    const int S = 256 / CG;
    const int lane = threadIdx.x % CG, slice = threadIdx.x / CG;
    const int groups = (a.C + CG - 1) / CG;
    const uint32_t v = blockIdx.x / groups;
    const int c = (blockIdx.x % groups) * CG + lane;
    const bool active = slice < S && c < a.C;
    const uint32_t sweep = (uint32_t)a.ctl->sweep;
    float acc[L], hi[L], lo[L];
#pragma unroll
    for (int x = 0; x < L; ++x) { acc[x] = 0.0f; hi[x] = 0.0f; lo[x] = 0.0f; }
    if (active) {
        const int64_t p0 = a.inc_ptr[v], p1 = a.inc_ptr[v + 1];
        int chunk = 0;
        // B incidences of the slice per iteration, their records and theta words
        // loaded before any is added (same order of additions)
        // (8 for one word: 62 registers, 1.40 vs 1.12 ms at N = 4096; staging a site's records in
        // shared memory first: 1.14 ms, no gain)
        constexpr int B = E::W <= 2 ? 4 : 2;
        for (int64_t p = p0 + slice; p < p1; p += (int64_t)B * S) {
            int2 ic[B];
            uint32_t bits[B][E::W];
#pragma unroll
            for (int u = 0; u < B; ++u) ic[u] = p + (int64_t)u * S < p1 ? __ldg(&a.inc[p + (int64_t)u * S]) : make_int2(-1, 0);
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const uint32_t* th = a.theta + ((int64_t)(ic[u].x >> 1) * a.C + c) * E::W;
#pragma unroll
                for (int w = 0; w < E::W; ++w) bits[u][w] = ic[u].x >= 0 ? __ldcs(th + w) : 0u;
            }
#pragma unroll
            for (int u = 0; u < B; ++u) {
                if (ic[u].x < 0) continue;
                add_side<L, LAYOUT>(bits[u], a.tau + (int64_t)(ic[u].x >> 1) * E::MP, ic[u].x & 1, acc);
                if (++chunk == 32) {
#pragma unroll
                    for (int x = 0; x < L; ++x) { two_sum_add(hi[x], lo[x], acc[x]); acc[x] = 0.0f; }
                    chunk = 0;
                }
            }
        }
#pragma unroll
        for (int x = 0; x < L; ++x) two_sum_add(hi[x], lo[x], acc[x]);
    }
#pragma unroll
    for (int x = 0; x < L; ++x) { red_hi[threadIdx.x][x] = hi[x]; red_lo[threadIdx.x][x] = lo[x]; }
    __syncthreads();
    if (slice == 0 && c < a.C) {
#pragma unroll
        for (int x = 0; x < L; ++x) {
            float h = 0.0f, l = 0.0f;
            for (int q = 0; q < S; ++q) {
                two_sum_add(h, l, red_hi[q * CG + lane][x]);
                l += red_lo[q * CG + lane][x];
            }
            hi[x] = h; lo[x] = l;
        }
        float F[L];
        const float* uf = a.utf + (int64_t)v * L;
#pragma unroll
        for (int x = 0; x < L; ++x) F[x] = __ldg(uf + x) + (hi[x] + lo[x]);
        uint8_t* xout = a.x + (size_t)((sweep + 1) & 1) * a.N * a.C;
        float* lp = a.logp ? a.logp + ((int64_t)c * a.N + v) * L : nullptr;
        xout[(int64_t)v * a.C + c] = (uint8_t)draw_label<L>(F, v, (uint32_t)c, sweep, a.rk, PH_PRIMAL, lp, a.ctl,
                                                            a.lpv ? a.lpv + (int64_t)v * a.C + c : nullptr);
    }
}

// ---------------------------------------------------------------------------- few chains, many entries

// Plain sweep for few chains (C <= 4) and tables with more than 16 entries,
// where a thread per (site, chain) would read every incident entry's weight
// row on its own.  After the dual step (k_dual), one warp per edge reads the
// edge's signed weights once (lane b: entries k = 32 g + b, coalesced) and,
// per chain, its dual bit words, and writes the edge's two partial fields:
// over the set bits, the row sums of the signed weights (source side, beta1)
// and the column sums of their magnitudes (destination side, beta2), each in
// entry order.  The primal step (k_primal_partial) then adds the partial
// fields of a site's incidences in incidence order (two-sum flush every 32,
// as k_primal) and draws the label.
template <int L, int LAYOUT>
__global__ void __launch_bounds__(256) k_edge_partial(SweepArgs a) {
    using E = Ent<L, LAYOUT>;
    constexpr int M = E::M, W = E::W, MP = E::MP;
    static_assert(M > 16 && L <= 16, "edge-partial form: more than 16 entries, at most 16 labels");
    __shared__ float s_t[8][W * 32];                       // weights of the set bits, per warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t e = blockIdx.x * 8ll + warp;
    if (e >= a.E || a.src[e] < 0) return;                  // whole warps; a free slot has no incidences
    const int C = a.C;
    float tv[W];
#pragma unroll
    for (int g = 0; g < W; ++g) {
        const int k = 32 * g + lane;
        tv[g] = k < M ? __ldg(a.tau + e * MP + k) : 0.0f;
    }
    for (int c = 0; c < C; ++c) {
        const uint32_t* th = a.theta + (e * C + c) * W;
        uint32_t bw[W];
        if constexpr (W % 4 == 0) {                        // the edge-chain's words in 16-byte loads
#pragma unroll
            for (int g = 0; g < W; g += 4) {
                const uint4 q = __ldcs(reinterpret_cast<const uint4*>(th + g));
                bw[g] = q.x; bw[g + 1] = q.y; bw[g + 2] = q.z; bw[g + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int g = 0; g < W; ++g) bw[g] = __ldcs(th + g);
        }
#pragma unroll
        for (int g = 0; g < W; ++g) s_t[warp][32 * g + lane] = ((bw[g] >> lane) & 1u) ? tv[g] : 0.0f;
        __syncwarp();
        float* pe = a.part + ((e * C + c) * 2) * L;
        if (lane < L) {                                    // row `lane`: source side
            float sum = 0.0f;
            if (LAYOUT == MRF_LAYOUT_PIVOT) {
                if (lane >= 1)
#pragma unroll
                    for (int jj = 1; jj < L; ++jj) sum += s_t[warp][(lane - 1) * (L - 1) + (jj - 1)];
            } else {
                sum = s_t[warp][lane];
            }
            pe[lane] = sum;
        } else if (lane >= 16 && lane < 16 + L) {          // column `lane - 16`: destination side
            const int x = lane - 16;
            float sum = 0.0f;
            if (LAYOUT == MRF_LAYOUT_PIVOT) {
                if (x >= 1)
#pragma unroll
                    for (int ii = 1; ii < L; ++ii) sum += fabsf(s_t[warp][(ii - 1) * (L - 1) + (x - 1)]);
            } else {
                sum = fabsf(s_t[warp][x]);
            }
            pe[L + x] = sum;
        }
        __syncwarp();
    }
}

template <int L>
__global__ void __launch_bounds__(256, 3) k_primal_partial(SweepArgs a) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;     // N * C < 2^32 (checked by the host)
    if (g >= (uint64_t)a.N * a.C) return;
    const uint32_t v = a.fdC.div(g), c = g - v * (uint32_t)a.C;
    const uint32_t sweep = (uint32_t)a.ctl->sweep;
    uint8_t* xout = a.x + (size_t)((sweep + 1) & 1) * a.N * a.C;
    float acc[L], hi[L], lo[L];
#pragma unroll
    for (int x = 0; x < L; ++x) { acc[x] = 0.0f; hi[x] = 0.0f; lo[x] = 0.0f; }
    const int64_t p0 = a.inc_ptr[v], p1 = a.inc_ptr[v + 1];
    int chunk = 0;
    bool flushed = false;
    constexpr int B = 4;                                   // incidence records loaded together
    for (int64_t base = p0; base < p1; base += B) {
        int code[B];
#pragma unroll
        for (int u = 0; u < B; ++u) code[u] = base + u < p1 ? __ldg(&a.inc[base + u]).x : -1;
#pragma unroll
        for (int u = 0; u < B; ++u) {
            if (code[u] < 0) continue;
            const float* pe = a.part + (((int64_t)(code[u] >> 1) * a.C + c) * 2 + (code[u] & 1)) * L;
            if constexpr (L % 4 == 0) {
#pragma unroll
                for (int x4 = 0; x4 < L / 4; ++x4) {
                    const float4 q = __ldcs(reinterpret_cast<const float4*>(pe) + x4);
                    acc[4 * x4] += q.x; acc[4 * x4 + 1] += q.y; acc[4 * x4 + 2] += q.z; acc[4 * x4 + 3] += q.w;
                }
            } else {
#pragma unroll
                for (int x = 0; x < L; ++x) acc[x] += __ldcs(pe + x);
            }
            if (++chunk == 32) {
#pragma unroll
                for (int x = 0; x < L; ++x) { two_sum_add(hi[x], lo[x], acc[x]); acc[x] = 0.0f; }
                chunk = 0;
                flushed = true;
            }
        }
    }
    float F[L];
    const float* uf = a.utf + (int64_t)v * L;
    if (flushed) {
#pragma unroll
        for (int x = 0; x < L; ++x) { two_sum_add(hi[x], lo[x], acc[x]); F[x] = __ldg(uf + x) + (hi[x] + lo[x]); }
    } else {
#pragma unroll
        for (int x = 0; x < L; ++x) F[x] = __ldg(uf + x) + acc[x];
    }
    float* lp = a.logp ? a.logp + ((int64_t)c * a.N + v) * L : nullptr;
    xout[g] = (uint8_t)draw_label<L>(F, v, c, sweep, a.rk, PH_PRIMAL, lp, a.ctl, a.lpv ? a.lpv + g : nullptr);
}

template <int L, int LAYOUT>
cudaError_t run_sweep_partial(const SweepArgs& a, int step, cudaStream_t s) {
    if constexpr (Ent<L, LAYOUT>::M > 16) {
        const int64_t n = (int64_t)a.N * a.C;
        if (step == 0 && a.E > 0) k_edge_partial<L, LAYOUT><<<(unsigned)((a.E + 7) / 8), 256, 0, s>>>(a);
        if (step == 1 && n > 0) k_primal_partial<L><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------- small models

// n_sweeps whole plain sweeps of a small model in one CTA (sizes where launch
// latency, not work, sets the time): dual half-step into shared memory,
// primal half-step, marginal counts and the sweep advance, separated by CTA
// barriers only.  The draws and the order of every addition are those of
// k_dual / k_primal, so the chain is the same bit for bit.
template <int L, int LAYOUT>
__global__ void __launch_bounds__(1024) k_sweep_small(SweepArgs a, int n_sweeps) {
    using E = Ent<L, LAYOUT>;
    extern __shared__ uint32_t s_theta[];                          // [E][C][W]
    const int64_t ne = a.E * a.C, nv = (int64_t)a.N * a.C;
    uint32_t sweep = (uint32_t)a.ctl->sweep;
    const unsigned long long count_from = a.ctl->count_from;
    for (int it = 0; it < n_sweeps; ++it, ++sweep) {
        const uint8_t* xin = a.x + (size_t)(sweep & 1) * a.N * a.C;
        uint8_t* xout = a.x + (size_t)((sweep + 1) & 1) * a.N * a.C;
        for (int64_t g = threadIdx.x; g < ne; g += blockDim.x) {
            const uint32_t e = a.fdC.div((uint32_t)g), c = (uint32_t)g - e * (uint32_t)a.C;
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
#pragma unroll
            for (int w = 0; w < E::W; ++w) s_theta[g * E::W + w] = bits[w];
        }
        __syncthreads();
        for (int64_t g = threadIdx.x; g < nv; g += blockDim.x) {
            const uint32_t v = a.fdC.div((uint32_t)g), c = (uint32_t)g - v * (uint32_t)a.C;
            float acc[L], hi[L], lo[L];
#pragma unroll
            for (int x = 0; x < L; ++x) { acc[x] = 0.0f; hi[x] = 0.0f; lo[x] = 0.0f; }
            int chunk = 0;
            bool flushed = false;
            for (int64_t p = a.inc_ptr[v]; p < a.inc_ptr[v + 1]; ++p) {
                const int2 ic = __ldg(&a.inc[p]);
                const int64_t e = ic.x >> 1;
                uint32_t bits[E::W];
#pragma unroll
                for (int w = 0; w < E::W; ++w) bits[w] = s_theta[(e * a.C + c) * E::W + w];
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
            if (flushed) {
#pragma unroll
                for (int x = 0; x < L; ++x) { two_sum_add(hi[x], lo[x], acc[x]); F[x] = __ldg(uf + x) + (hi[x] + lo[x]); }
            } else {
#pragma unroll
                for (int x = 0; x < L; ++x) F[x] = __ldg(uf + x) + acc[x];
            }
            float* lp = a.logp ? a.logp + ((int64_t)c * a.N + v) * L : nullptr;
            xout[g] = (uint8_t)draw_label<L>(F, v, c, sweep, a.rk, PH_PRIMAL, lp, a.ctl);
        }
        __syncthreads();
        if (sweep >= count_from) {
            for (int64_t v = threadIdx.x; v < a.N; v += blockDim.x) {
                uint32_t tot[L];
#pragma unroll
                for (int x = 0; x < L; ++x) tot[x] = 0;
                for (int c = 0; c < a.C; ++c) {
                    const int x = xout[v * a.C + c];
#pragma unroll
                    for (int y = 0; y < L; ++y) tot[y] += x == y ? 1u : 0u;
                }
#pragma unroll
                for (int x = 0; x < L; ++x) a.counts[v * L + x] += tot[x];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) a.ctl->sweep = sweep;
}

// ---------------------------------------------------------------------------- EM and mean field

// Theta-update of Section 5.3's primal-dual EM / mean field for one incident
// edge: with eta_y,k and eta_z,k the (expected) indicators of the entry's row
// and column labels, pi_k = sigmoid(q_k + beta1 eta_y + beta2 eta_z),
// q = -max(tau, 0), beta1 = tau, beta2 = |tau| (tau signed), and its beta pi
// is added to the field of this endpoint (row i_k on the source side, column
// j_k on the destination side).  ey / ez give eta for label a of the source /
// destination endpoint.
template <int L, int LAYOUT, typename EtaS, typename EtaT>
__device__ __forceinline__ void add_side_mean(const float* __restrict__ tau_e, int side, EtaS ey, EtaT ez,
                                              float (&acc)[L]) {
    using E = Ent<L, LAYOUT>;
    const float4* t4 = reinterpret_cast<const float4*>(tau_e);
#pragma unroll
    for (int k4 = 0; k4 < E::MP / 4; ++k4) {
        const float4 qv = __ldg(t4 + k4);
        const float tv[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = 4 * k4 + u;
            if (k >= E::M) continue;
            const float ts = tv[u], b2 = fabsf(ts);
            const float logit = -fmaxf(ts, 0.0f) + ts * ey(E::i(k)) + b2 * ez(E::j(k));
            const float pi = 1.0f / (1.0f + expf(-logit));
            if (side == 0) acc[E::i(k)] += ts * pi;
            else acc[E::j(k)] += b2 * pi;
        }
    }
}

// EM (local MAP): x' = argmax of the field of the expected duals given x.
template <int L, int LAYOUT>
__global__ void __launch_bounds__(256) k_em(SweepArgs a, const uint8_t* __restrict__ xin, uint8_t* __restrict__ xout) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (uint64_t)a.N * a.C) return;
    const uint32_t v = a.fdC.div(g), c = g - v * (uint32_t)a.C;
    const int xv = xin[g];
    float acc[L];
#pragma unroll
    for (int x = 0; x < L; ++x) acc[x] = 0.0f;
    for (int64_t p = a.inc_ptr[v]; p < a.inc_ptr[v + 1]; ++p) {
        const int2 ic = __ldg(&a.inc[p]);
        const int side = ic.x & 1;
        const int xu = xin[(int64_t)ic.y * a.C + c];
        const int xs = side == 0 ? xv : xu, xt = side == 0 ? xu : xv;
        add_side_mean<L, LAYOUT>(a.tau + (int64_t)(ic.x >> 1) * Ent<L, LAYOUT>::MP, side,
                                 [&](int i) { return xs == i ? 1.0f : 0.0f; }, [&](int j) { return xt == j ? 1.0f : 0.0f; }, acc);
    }
    const float* uf = a.utf + (int64_t)v * L;
    int best = 0;
    float fb = __ldg(uf) + acc[0];
#pragma unroll
    for (int x = 1; x < L; ++x) {
        const float f = __ldg(uf + x) + acc[x];
        if (f > fb) { fb = f; best = x; }
    }
    xout[g] = (uint8_t)best;
}

// Blocked EM, potentials: F_v = u~_v + the beta pi of the expected duals of
// v's incident non-tree edges (the comb forest of the current block offset),
// written to a.pot ([N][L][C]) for the tree MAP.
template <int L, int LAYOUT>
__global__ void __launch_bounds__(256) k_em_pot(SweepArgs a, const uint8_t* __restrict__ xin) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (uint64_t)a.N * a.C) return;
    const uint32_t v = a.fdC.div(g), c = g - v * (uint32_t)a.C;
    const int xv = xin[g];
    float acc[L];
#pragma unroll
    for (int x = 0; x < L; ++x) acc[x] = 0.0f;
    for (int64_t p = a.inc_ptr[v]; p < a.inc_ptr[v + 1]; ++p) {
        const int2 ic = __ldg(&a.inc[p]);
        if (is_tree_edge(a, (uint32_t)(ic.x >> 1))) continue;
        const int side = ic.x & 1;
        const int xu = xin[(int64_t)ic.y * a.C + c];
        const int xs = side == 0 ? xv : xu, xt = side == 0 ? xu : xv;
        add_side_mean<L, LAYOUT>(a.tau + (int64_t)(ic.x >> 1) * Ent<L, LAYOUT>::MP, side,
                                 [&](int i) { return xs == i ? 1.0f : 0.0f; }, [&](int j) { return xt == j ? 1.0f : 0.0f; }, acc);
    }
    const float* uf = a.utf + (int64_t)v * L;
    float* pv = a.pot + (int64_t)v * L * a.C + c;
#pragma unroll
    for (int x = 0; x < L; ++x) pv[(int64_t)x * a.C] = __ldg(uf + x) + acc[x];
}

// Mean field: q' = softmax of the field of the expected duals given the site
// marginals q ([N][L][C], chain innermost).
template <int L, int LAYOUT>
__global__ void __launch_bounds__(256) k_mf(SweepArgs a, const float* __restrict__ qin, float* __restrict__ qout) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (uint64_t)a.N * a.C) return;
    const uint32_t v = a.fdC.div(g), c = g - v * (uint32_t)a.C;
    const int64_t C = a.C;
    float qv[L], acc[L];
#pragma unroll
    for (int x = 0; x < L; ++x) { qv[x] = qin[((int64_t)v * L + x) * C + c]; acc[x] = 0.0f; }
    for (int64_t p = a.inc_ptr[v]; p < a.inc_ptr[v + 1]; ++p) {
        const int2 ic = __ldg(&a.inc[p]);
        const int side = ic.x & 1;
        float qu[L];
#pragma unroll
        for (int x = 0; x < L; ++x) qu[x] = qin[((int64_t)ic.y * L + x) * C + c];
        const float* tau_e = a.tau + (int64_t)(ic.x >> 1) * Ent<L, LAYOUT>::MP;
        if (side == 0)
            add_side_mean<L, LAYOUT>(tau_e, 0, [&](int i) { return qv[i]; }, [&](int j) { return qu[j]; }, acc);
        else
            add_side_mean<L, LAYOUT>(tau_e, 1, [&](int i) { return qu[i]; }, [&](int j) { return qv[j]; }, acc);
    }
    const float* uf = a.utf + (int64_t)v * L;
    float F[L], mx = -INFINITY;
#pragma unroll
    for (int x = 0; x < L; ++x) { F[x] = __ldg(uf + x) + acc[x]; mx = fmaxf(mx, F[x]); }
    float s = 0.0f;
#pragma unroll
    for (int x = 0; x < L; ++x) { F[x] = expf(F[x] - mx); s += F[x]; }
    const float inv = 1.0f / s;
#pragma unroll
    for (int x = 0; x < L; ++x) qout[((int64_t)v * L + x) * C + c] = F[x] * inv;
}

// Blocked (tree) mean field, potentials: F_v = u~_v + the beta pi of the
// expected duals of v's incident non-forest edges given the site marginals q
// ([N][L][C]), written to a.pot for the forest's sum-product pass.
template <int L, int LAYOUT>
__global__ void __launch_bounds__(256) k_mf_pot(SweepArgs a, const float* __restrict__ qin) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (uint64_t)a.N * a.C) return;
    const uint32_t v = a.fdC.div(g), c = g - v * (uint32_t)a.C;
    const int64_t C = a.C;
    float qv[L], acc[L];
#pragma unroll
    for (int x = 0; x < L; ++x) { qv[x] = qin[((int64_t)v * L + x) * C + c]; acc[x] = 0.0f; }
    for (int64_t p = a.inc_ptr[v]; p < a.inc_ptr[v + 1]; ++p) {
        const int2 ic = __ldg(&a.inc[p]);
        if (is_tree_edge(a, (uint32_t)(ic.x >> 1))) continue;
        const int side = ic.x & 1;
        float qu[L];
#pragma unroll
        for (int x = 0; x < L; ++x) qu[x] = qin[((int64_t)ic.y * L + x) * C + c];
        const float* tau_e = a.tau + (int64_t)(ic.x >> 1) * Ent<L, LAYOUT>::MP;
        if (side == 0)
            add_side_mean<L, LAYOUT>(tau_e, 0, [&](int i) { return qv[i]; }, [&](int j) { return qu[j]; }, acc);
        else
            add_side_mean<L, LAYOUT>(tau_e, 1, [&](int i) { return qu[i]; }, [&](int j) { return qv[j]; }, acc);
    }
    const float* uf = a.utf + (int64_t)v * L;
    float* pv = a.pot + (int64_t)v * L * C + c;
#pragma unroll
    for (int x = 0; x < L; ++x) pv[(int64_t)x * C] = __ldg(uf + x) + acc[x];
}

static inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

template <int L, int LAYOUT>
cudaError_t run_primal_cta(const SweepArgs& a, cudaStream_t s) {
    const int CG = a.C >= 32 ? 32 : a.C;
    const int64_t blocks = (int64_t)a.N * ((a.C + CG - 1) / CG);
    if (blocks > 0) k_primal_cta<L, LAYOUT><<<(unsigned)blocks, 256, 0, s>>>(a, CG);
    return cudaGetLastError();
}

template <int L, int LAYOUT>
cudaError_t run_dual(const SweepArgs& a, cudaStream_t s) {
    using T = DualTile<Ent<L, LAYOUT>::M, Ent<L, LAYOUT>::W>;
    const int64_t n = a.E * a.C;
    if (n <= 0) return cudaSuccess;
    // few chains and wide tables (two groups per warp): 128 registers and two blocks per SM; at 64
    // registers the 8-word form spills (224 B); with one chain on 25.2 M edges of L = 16 (the
    // 2,000-graph batch's largest class) it measured 5.14 vs 4.12 ms per sweep
    if (a.C < 32 && T::NG <= 2)
        k_dual<L, LAYOUT, true><<<blocks_for(n, 32 * T::NG * T::WARPS), 32 * T::WARPS, 0, s>>>(a);
    else
        k_dual<L, LAYOUT><<<blocks_for(n, 32 * T::NG * T::WARPS), 32 * T::WARPS, 0, s>>>(a);
    return cudaGetLastError();
}

template <int L, int LAYOUT, bool FUSED>
cudaError_t run_primal(const SweepArgs& a, cudaStream_t s) {
    const int64_t n = (int64_t)a.N * a.C;
    if (n <= 0) return cudaSuccess;
    if (!FUSED && a.C % 32 == 0) {
        if (a.max_deg <= PrimalWarp<L, LAYOUT>::KB)
            k_primal_warp<L, LAYOUT, false, true><<<blocks_for(n, 256), 256, 0, s>>>(a);
        else
            k_primal_warp<L, LAYOUT><<<blocks_for(n, 256), 256, 0, s>>>(a);
    } else
        k_primal<L, LAYOUT, FUSED><<<blocks_for(n, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <int L, int LAYOUT>
cudaError_t run_potential(const SweepArgs& a, cudaStream_t s) {
    const int64_t n = (int64_t)a.N * a.C;
    if (n <= 0) return cudaSuccess;
    if (a.C % 32 == 0) {
        if (a.max_deg <= PrimalWarp<L, LAYOUT>::KB)
            k_primal_warp<L, LAYOUT, true, true><<<blocks_for(n, 256), 256, 0, s>>>(a);
        else
            k_primal_warp<L, LAYOUT, true><<<blocks_for(n, 256), 256, 0, s>>>(a);
    } else
        k_primal<L, LAYOUT, false, true><<<blocks_for(n, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <int L, int LAYOUT>
cudaError_t run_em(const SweepArgs& a, const uint8_t* xin, uint8_t* xout, cudaStream_t s) {
    const int64_t n = (int64_t)a.N * a.C;
    if (n > 0) k_em<L, LAYOUT><<<blocks_for(n, 256), 256, 0, s>>>(a, xin, xout);
    return cudaGetLastError();
}

template <int L, int LAYOUT>
cudaError_t run_mf(const SweepArgs& a, const float* qin, float* qout, cudaStream_t s) {
    const int64_t n = (int64_t)a.N * a.C;
    if (n > 0) k_mf<L, LAYOUT><<<blocks_for(n, 256), 256, 0, s>>>(a, qin, qout);
    return cudaGetLastError();
}

template <int L, int LAYOUT>
cudaError_t run_sweep_small(const SweepArgs& a, int n_sweeps, cudaStream_t s) {
    const size_t smem = (size_t)a.E * a.C * Ent<L, LAYOUT>::W * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep_small<L, LAYOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_sweep_small<L, LAYOUT><<<1, 1024, smem, s>>>(a, n_sweeps);
    return cudaGetLastError();
}

template <int L, int LAYOUT>
cudaError_t run_mf_pot(const SweepArgs& a, const float* qin, cudaStream_t s) {
    const int64_t n = (int64_t)a.N * a.C;
    if (n > 0) k_mf_pot<L, LAYOUT><<<blocks_for(n, 256), 256, 0, s>>>(a, qin);
    return cudaGetLastError();
}

template <int L, int LAYOUT>
cudaError_t run_em_pot(const SweepArgs& a, const uint8_t* xin, cudaStream_t s) {
    const int64_t n = (int64_t)a.N * a.C;
    if (n > 0) k_em_pot<L, LAYOUT><<<blocks_for(n, 256), 256, 0, s>>>(a, xin);
    return cudaGetLastError();
}

#define MRF_INSTANTIATE_SWEEP(L)                                                                 \
    template cudaError_t run_mf_pot<L, MRF_LAYOUT_PIVOT>(const SweepArgs&, const float*, cudaStream_t); \
    template cudaError_t run_mf_pot<L, MRF_LAYOUT_DIAG>(const SweepArgs&, const float*, cudaStream_t);  \
    template cudaError_t run_em_pot<L, MRF_LAYOUT_PIVOT>(const SweepArgs&, const uint8_t*, cudaStream_t); \
    template cudaError_t run_em_pot<L, MRF_LAYOUT_DIAG>(const SweepArgs&, const uint8_t*, cudaStream_t);  \
    template cudaError_t run_sweep_small<L, MRF_LAYOUT_PIVOT>(const SweepArgs&, int, cudaStream_t); \
    template cudaError_t run_sweep_small<L, MRF_LAYOUT_DIAG>(const SweepArgs&, int, cudaStream_t);  \
    template cudaError_t run_em<L, MRF_LAYOUT_PIVOT>(const SweepArgs&, const uint8_t*, uint8_t*, cudaStream_t); \
    template cudaError_t run_em<L, MRF_LAYOUT_DIAG>(const SweepArgs&, const uint8_t*, uint8_t*, cudaStream_t);  \
    template cudaError_t run_mf<L, MRF_LAYOUT_PIVOT>(const SweepArgs&, const float*, float*, cudaStream_t);     \
    template cudaError_t run_mf<L, MRF_LAYOUT_DIAG>(const SweepArgs&, const float*, float*, cudaStream_t);      \
    template cudaError_t run_primal_cta<L, MRF_LAYOUT_PIVOT>(const SweepArgs&, cudaStream_t);     \
    template cudaError_t run_primal_cta<L, MRF_LAYOUT_DIAG>(const SweepArgs&, cudaStream_t);      \
    template cudaError_t run_potential<L, MRF_LAYOUT_PIVOT>(const SweepArgs&, cudaStream_t);      \
    template cudaError_t run_potential<L, MRF_LAYOUT_DIAG>(const SweepArgs&, cudaStream_t);       \
    template cudaError_t run_sweep_partial<L, MRF_LAYOUT_PIVOT>(const SweepArgs&, int, cudaStream_t); \
    template cudaError_t run_sweep_partial<L, MRF_LAYOUT_DIAG>(const SweepArgs&, int, cudaStream_t);  \
    template cudaError_t run_dual<L, MRF_LAYOUT_PIVOT>(const SweepArgs&, cudaStream_t);           \
    template cudaError_t run_dual<L, MRF_LAYOUT_DIAG>(const SweepArgs&, cudaStream_t);            \
    template cudaError_t run_primal<L, MRF_LAYOUT_PIVOT, false>(const SweepArgs&, cudaStream_t);  \
    template cudaError_t run_primal<L, MRF_LAYOUT_DIAG, false>(const SweepArgs&, cudaStream_t);   \
    template cudaError_t run_primal<L, MRF_LAYOUT_PIVOT, true>(const SweepArgs&, cudaStream_t);   \
    template cudaError_t run_primal<L, MRF_LAYOUT_DIAG, true>(const SweepArgs&, cudaStream_t);

}  // namespace mrfk
