// Swendsen-Wang sweep as a degenerate duality (Section 4.3).
//
// For a ferromagnetic Potts-type table exp(l_x [x_s = x_t]) with l_x >= 0 the
// dual variable of an edge is one bond bit: given x it is 1 with probability
// 1 - e^{-l_{x_s}} when x_s = x_t (never otherwise); given the bonds, the
// bonds' connected components (clusters) take one label each, cluster K
// label x with weight exp(sum_{v in K} u_v(x) + sum_{bonds in K} log(e^{l_x} - 1)).
//
// One sweep on the device, items (site or edge, chain) with the chain
// innermost so that a warp works on one site or edge for 32 chains.  Between
// sweeps every site is its own tree (parent[v][c] = v), its ban word is 0 and
// its weight row lw[v][.][c] is 0; a sweep touches only what its bonds reach
// and restores that state:
//   k_sw_bond     bond draws into a bitmap (one ballot word per warp)
//   k_sw_union    a thread per bitmap word: each bond unions its endpoints'
//                 trees, adds its label weights to its source site's row and
//                 marks both endpoints bonded (dense work: the sparse bonds no
//                 longer hold whole warps of non-bonded lanes)
//   k_sw_flatten  every bonded site records its root (the smallest site of its
//                 cluster) and adds its unaries and row into the root's row
//   k_sw_draw     every root (bonded or not) draws its cluster's label from
//                 its unaries plus its row
//   k_sw_assign   bonded non-roots copy the root's label; rows, parents and
//                 ban words of bonded sites are reset.
// Unaries enter as fixed-point values precomputed once per factor change.
// Higdon's partial Swendsen-Wang (k_hg_*) runs the same kernels with its own
// bond tables and per-chain potentials in place of the unaries; small models
// run whole Swendsen-Wang sweeps in one single-CTA launch (k_sw_small).
// The union-find is lock-free: a link always points from a root to a smaller
// site (atomicCAS on the root's entry), so every walk visits strictly
// decreasing sites and ends within N steps; a walk that exceeds that bound
// sets the error flag instead of looping (the host then resets the state).
// The forest of a chain is its own column of parent[][], so chains never
// contend.
#include "sweep_impl.cuh"   // draw_label

namespace mrfk {

namespace {

__device__ __forceinline__ int64_t pidx(int32_t v, int32_t c, int32_t C) { return (int64_t)v * C + c; }

// Root of v, halving the path on the way (loads bypass L1: other threads
// rewrite entries meanwhile).  A halving store replaces a non-root's parent by
// one of its ancestors, so it never meets a link (links only rewrite roots)
// and any interleaving of halving stores leaves a forest with the same roots.
// Roots found by k_sw_flatten go to a separate array, not into parent[][]: a
// halving store landing after such a write would leave a non-root there.
// Returns -1 when the step bound is exceeded.
__device__ __forceinline__ int32_t sw_find(int32_t* __restrict__ par, int32_t v, int32_t c, int32_t C, int32_t N) {
    for (int32_t step = 0; step <= N; ++step) {
        const int32_t p = __ldcg(par + pidx(v, c, C));
        if (p == v) return v;
        const int32_t gp = __ldcg(par + pidx(p, c, C));
        if (gp != p) par[pidx(v, c, C)] = gp;
        v = gp;
    }
    return -1;
}

// Union of the trees of a and b: the larger root is linked to the smaller one.
// A failed link means that root was linked meanwhile; the retry starts from
// roots strictly smaller than before, so at most N retries happen.
__device__ __forceinline__ bool sw_union(int32_t* __restrict__ par, int32_t a, int32_t b, int32_t c, int32_t C,
                                         int32_t N) {
    for (int32_t step = 0; step <= N; ++step) {
        a = sw_find(par, a, c, C, N);
        b = sw_find(par, b, c, C, N);
        if (a < 0 || b < 0) return false;
        if (a == b) return true;
        if (a < b) { const int32_t t = a; a = b; b = t; }
        if (atomicCAS(par + pidx(a, c, C), a, b) == a) return true;
    }
    return false;
}

__device__ __forceinline__ void red_add_s64(int64_t* p, int64_t v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

}  // namespace

// sw_fix of a float32 value without float64 arithmetic: the value is
// m 2^(e - 150) with a 24-bit mantissa m, so its fixed-point form m 2^(e - 118)
// is a shift of m (rounded half away from zero when it drops bits; |f| < 2^30
// is guaranteed by the model check).
__device__ __forceinline__ int64_t fix_from_float(float f) {
    const uint32_t bits = __float_as_uint(f);
    const int e = (int)((bits >> 23) & 0xFFu);
    if (e == 0) return 0;                                          // zero and subnormals (|f| < 2^-126)
    const int64_t m = (int64_t)((bits & 0x7FFFFFu) | 0x800000u);
    const int sh = e - 118;
    int64_t v;
    if (sh >= 0) v = m << (sh < 38 ? sh : 38);
    else if (sh > -25) v = (m + ((int64_t)1 << (-sh - 1))) >> (-sh);
    else v = 0;
    return (bits >> 31) ? -v : v;
}

// Unary term of label x of item (v, c): the fixed-point unary, or the
// per-chain potential of Higdon's sweep.
template <int L>
__device__ __forceinline__ int64_t sw_unary(const SwArgs& a, int32_t v, int32_t c, int x) {
    return a.pot ? fix_from_float(a.pot[((int64_t)v * L + x) * a.C + c]) : __ldg(a.ufix + (int64_t)v * L + x);
}

// float of a fixed-point weight difference d <= 0 (two 32-bit conversions:
// GB300's 64-bit conversions run on its slow FP64 path).
__device__ __forceinline__ float sw_float(int64_t d) {
    return (float)(int32_t)(d >> 32) + (float)(uint32_t)d * (1.0f / 4294967296.0f);
}

// State between sweeps: parent[v][c] = v, ban[v][c] = 0, lw = 0 (the kernels
// below restore it); this kernel sets parent and ban, the host zeroes lw.
__global__ void __launch_bounds__(256) k_sw_reset(SwArgs a) {
    const int64_t n = (int64_t)a.N * a.C;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        a.parent[g] = (int32_t)a.fdC.div((uint32_t)g);
        a.ban[g] = 0u;
    }
}

// Bond draws, one item per (edge, chain), items g = e C + c.  A warp's 32
// lanes hold 32 consecutive items (the grid stride is a multiple of 32), so
// its bonds form one 32-bit word of the bond bitmap, bits[g / 32], written by
// one lane; every word is written every sweep.
__global__ void __launch_bounds__(256) k_sw_bond(SwArgs a) {
    const int64_t n = a.E * a.C;
    const unsigned long long t = a.ctl->sweep;
    const uint8_t* __restrict__ xin = a.x + (size_t)(t & 1) * a.N * a.C;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g - lane < n; g += stride) {
        bool bond = false;
        if (g < n) {
            const int64_t e = a.fdC.div((uint32_t)g);
            const int32_t c = (int32_t)(g - e * a.C);
            const int32_t s = a.src[e];
            if (s >= 0) {
                const int xs = xin[pidx(s, c, a.C)];
                if (xs == xin[pidx(a.dst[e], c, a.C)]) {
                    const uint32_t T = a.thr[e * a.L + xs];
                    bond = T != 0u && (draw_rk((uint32_t)e, (uint32_t)t, (uint32_t)c, PH_BOND, 0, a.rk).x >> 9) < T;
                }
            }
        }
        const uint32_t word = __ballot_sync(0xffffffffu, bond);
        if (lane == 0) a.bits[(g - lane) >> 5] = word;
    }
}

// Unions of the bonds: one bitmap word per thread, its set bits in order.
// Each bond links its endpoints' trees, adds its label weights to its source
// site's row unless they are equal for every label (then they would shift all
// of a cluster's exact sums alike and leave its draw unchanged: Potts tables
// with one coupling per edge, every two-label table), and marks both
// endpoints bonded.
template <int L>
__global__ void __launch_bounds__(256) k_sw_union(SwArgs a) {
    const int64_t n = a.E * a.C;
    const int64_t words = (n + 31) >> 5;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t word = a.bits[i];
        while (word) {
            const int bit = __ffs(word) - 1;
            word &= word - 1u;
            const int64_t g = i * 32 + bit;
            const int64_t e = a.fdC.div((uint32_t)g);
            const int32_t c = (int32_t)(g - e * a.C);
            const int32_t s = a.src[e], d = a.dst[e];
            if (!sw_union(a.parent, s, d, c, a.C, a.N)) { atomicOr(a.err, 1u); continue; }
            // every load before the first atomic (the compiler cannot move a
            // load above an atomic to a possibly aliasing address)
            int64_t wv[L];
#pragma unroll
            for (int x = 0; x < L; ++x) wv[x] = __ldg(a.lwe + e * L + x);
            bool uniform = wv[0] != kSwNoLabel;
#pragma unroll
            for (int x = 1; x < L; ++x) uniform &= wv[x] == wv[0];
            uint32_t flags = kSwBonded;
            if (!uniform) {
                flags |= kSwRow;
#pragma unroll
                for (int x = 0; x < L; ++x) {
                    if (wv[x] == kSwNoLabel) flags |= 1u << x;
                    else red_add_s64(a.lw + ((int64_t)s * L + x) * a.C + c, wv[x]);
                }
            }
            atomicOr(a.ban + pidx(s, c, a.C), flags);
            atomicOr(a.ban + pidx(d, c, a.C), kSwBonded);
        }
    }
}

// Bonded sites only (a site without a bond is its own cluster).  The forest
// is final once k_sw_bond has finished: every bonded site records its root
// (the smallest site of its cluster), and a non-root adds its unaries and the
// weights of the bonds it is the source of into its root's row.  Only roots'
// rows and ban words are written here, and only non-roots' are read.
template <int L>
__global__ void __launch_bounds__(256) k_sw_flatten(SwArgs a) {
    const int64_t n = (int64_t)a.N * a.C;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = a.ban[g];
        if (!(b & kSwBonded)) continue;
        const int32_t v = (int32_t)a.fdC.div((uint32_t)g), c = (int32_t)(g - (int64_t)v * a.C);
        const int32_t r = sw_find(a.parent, v, c, a.C, a.N);
        if (r < 0) { atomicOr(a.err, 1u); continue; }
        a.root[g] = r;
        if (r == v) continue;
        int64_t w[L];
#pragma unroll
        for (int x = 0; x < L; ++x) w[x] = sw_unary<L>(a, v, c, x);
        if (b & kSwRow) {
            const int64_t* row = a.lw + (int64_t)v * L * a.C + c;
#pragma unroll
            for (int x = 0; x < L; ++x) w[x] += row[(int64_t)x * a.C];
        }
#pragma unroll
        for (int x = 0; x < L; ++x) red_add_s64(a.lw + ((int64_t)r * L + x) * a.C + c, w[x]);
        if (b & kSwLabelMask) atomicOr(a.ban + pidx(r, c, a.C), b & kSwLabelMask);
    }
}

// Label of every cluster, drawn at its root r by the inverse CDF with the
// uniform of Philox(r, t, c, CLUSTER): weights are the root's unaries plus its
// row (bonded sites), the differences to the largest are exact in fixed point
// and then rounded to float for the softmax.  Nothing but the label is written
// here: a store right behind the loads of the same row stalled the kernel
// several-fold, so k_sw_assign clears rows and ban words.
template <int L>
__global__ void __launch_bounds__(256) k_sw_draw(SwArgs a) {
    const int64_t n = (int64_t)a.N * a.C;
    const unsigned long long t = a.ctl->sweep;
    uint8_t* __restrict__ xout = a.x + (size_t)((t + 1) & 1) * a.N * a.C;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = (int32_t)a.fdC.div((uint32_t)g), c = (int32_t)(g - (int64_t)v * a.C);
        const uint32_t b = a.ban[g];
        const bool bonded = (b & kSwBonded) != 0u;
        if (bonded && a.root[g] != v) {                     // labelled by k_sw_assign
            if (a.lpv) a.lpv[g] = 0.0f;
            continue;
        }
        int64_t w[L];
#pragma unroll
        for (int x = 0; x < L; ++x) w[x] = sw_unary<L>(a, v, c, x);
        if (bonded) {
            const int64_t* row = a.lw + (int64_t)v * L * a.C + c;
#pragma unroll
            for (int x = 0; x < L; ++x) w[x] += row[(int64_t)x * a.C];
        }
        int64_t mx = 0;
        bool any = false;
#pragma unroll
        for (int x = 0; x < L; ++x)
            if (!((b >> x) & 1u) && (!any || w[x] > mx)) { mx = w[x]; any = true; }
        float F[L];
#pragma unroll
        for (int x = 0; x < L; ++x)
            F[x] = ((b >> x) & 1u) ? -INFINITY : sw_float(w[x] - mx);
        xout[g] = (uint8_t)draw_label<L>(F, (uint32_t)v, (uint32_t)c, (uint32_t)t, a.rk, PH_CLUSTER, nullptr, a.ctl,
                                         a.lpv ? a.lpv + g : nullptr);
    }
}

// Bonded sites return to the between-sweeps state: non-roots copy their
// root's label; a root's row (its cluster's sums) and a bond source's row are
// cleared; parent and ban words are reset.  (Clearing whole 32-byte sectors
// whenever any lane of a warp clears its entries wrote more than the merged
// 8-byte writes cost: measured slower.)
template <int L>
__global__ void __launch_bounds__(256) k_sw_assign(SwArgs a) {
    const int64_t n = (int64_t)a.N * a.C;
    const unsigned long long t = a.ctl->sweep;
    uint8_t* __restrict__ xout = a.x + (size_t)((t + 1) & 1) * a.N * a.C;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = a.ban[g];
        if (!(b & kSwBonded)) continue;
        const int32_t v = (int32_t)a.fdC.div((uint32_t)g), c = (int32_t)(g - (int64_t)v * a.C);
        const int32_t r = a.root[g];
        if (r != v) xout[g] = xout[pidx(r, c, a.C)];
        if (r == v || (b & kSwRow)) {
            int64_t* row = a.lw + (int64_t)v * L * a.C + c;
#pragma unroll
            for (int x = 0; x < L; ++x) row[(int64_t)x * a.C] = 0;
        }
        a.parent[g] = v;
        a.ban[g] = 0u;
    }
}

// Small models: n_sweeps whole Swendsen-Wang sweeps in one launch of a single
// 1024-thread CTA (launch latency dominates there), the union-find state in
// shared memory: parent, root and ban words [N][C], weight rows [N][L][C].
// The same draws, exact sums and rules as the kernels above, phases separated
// by CTA barriers, hence the same chain bit for bit; marginal counts and the
// sweep counter are advanced here too.
__device__ __forceinline__ int32_t sws_find(volatile int32_t* par, int32_t v, int32_t c, int32_t C, int32_t N) {
    for (int32_t step = 0; step <= N; ++step) {
        const int32_t p = par[pidx(v, c, C)];
        if (p == v) return v;
        const int32_t gp = par[pidx(p, c, C)];
        if (gp != p) par[pidx(v, c, C)] = gp;
        v = gp;
    }
    return -1;
}

template <int L>
__global__ void __launch_bounds__(1024) k_sw_small(SwArgs a, int n_sweeps) {
    extern __shared__ int64_t s_lw[];                                  // [N][L][C]
    const int64_t nv = (int64_t)a.N * a.C, ne = a.E * a.C;
    int32_t* s_par = reinterpret_cast<int32_t*>(s_lw + nv * L);       // [N][C]
    int32_t* s_root = s_par + nv;                                     // [N][C]
    uint32_t* s_ban = reinterpret_cast<uint32_t*>(s_root + nv);       // [N][C]
    volatile int32_t* vpar = s_par;
    for (int64_t g = threadIdx.x; g < nv; g += blockDim.x) {
        s_par[g] = (int32_t)a.fdC.div((uint32_t)g);
        s_ban[g] = 0u;
    }
    for (int64_t i = threadIdx.x; i < nv * L; i += blockDim.x) s_lw[i] = 0;
    __syncthreads();
    uint32_t sweep = (uint32_t)a.ctl->sweep;
    const unsigned long long count_from = a.ctl->count_from;
    for (int it = 0; it < n_sweeps; ++it, ++sweep) {
        const uint8_t* xin = a.x + (size_t)(sweep & 1) * a.N * a.C;
        uint8_t* xout = a.x + (size_t)((sweep + 1) & 1) * a.N * a.C;
        // bonds and unions
        for (int64_t g = threadIdx.x; g < ne; g += blockDim.x) {
            const int64_t e = a.fdC.div((uint32_t)g);
            const int32_t c = (int32_t)(g - e * a.C);
            const int32_t s = a.src[e];
            if (s < 0) continue;
            const int32_t d = a.dst[e];
            const int xs = xin[pidx(s, c, a.C)];
            if (xs != xin[pidx(d, c, a.C)]) continue;
            const uint32_t T = a.thr[e * L + xs];
            if (T == 0u || (draw_rk((uint32_t)e, sweep, (uint32_t)c, PH_BOND, 0, a.rk).x >> 9) >= T) continue;
            int32_t ra = s, rb = d;
            bool linked = false;
            for (int32_t step = 0; step <= a.N && !linked; ++step) {
                ra = sws_find(vpar, ra, c, a.C, a.N);
                rb = sws_find(vpar, rb, c, a.C, a.N);
                if (ra < 0 || rb < 0) break;
                if (ra == rb) { linked = true; break; }
                if (ra < rb) { const int32_t t2 = ra; ra = rb; rb = t2; }
                linked = atomicCAS(s_par + pidx(ra, c, a.C), ra, rb) == ra;
            }
            if (!linked) { atomicOr(a.err, 1u); continue; }
            int64_t wv[L];
#pragma unroll
            for (int x = 0; x < L; ++x) wv[x] = __ldg(a.lwe + e * L + x);
            bool uniform = wv[0] != kSwNoLabel;
#pragma unroll
            for (int x = 1; x < L; ++x) uniform &= wv[x] == wv[0];
            uint32_t flags = kSwBonded;
            if (!uniform) {
                flags |= kSwRow;
#pragma unroll
                for (int x = 0; x < L; ++x) {
                    if (wv[x] == kSwNoLabel) flags |= 1u << x;
                    else atomicAdd(reinterpret_cast<unsigned long long*>(s_lw + ((int64_t)s * L + x) * a.C + c),
                                   (unsigned long long)wv[x]);
                }
            }
            atomicOr(s_ban + pidx(s, c, a.C), flags);
            atomicOr(s_ban + pidx(d, c, a.C), kSwBonded);
        }
        __syncthreads();
        // roots and cluster sums
        for (int64_t g = threadIdx.x; g < nv; g += blockDim.x) {
            const uint32_t b = s_ban[g];
            if (!(b & kSwBonded)) continue;
            const int32_t v = (int32_t)a.fdC.div((uint32_t)g), c = (int32_t)(g - (int64_t)v * a.C);
            const int32_t r = sws_find(vpar, v, c, a.C, a.N);
            if (r < 0) { atomicOr(a.err, 1u); s_root[g] = v; continue; }
            s_root[g] = r;
            if (r == v) continue;
#pragma unroll
            for (int x = 0; x < L; ++x) {
                int64_t w = __ldg(a.ufix + (int64_t)v * L + x);
                if (b & kSwRow) w += s_lw[((int64_t)v * L + x) * a.C + c];
                atomicAdd(reinterpret_cast<unsigned long long*>(s_lw + ((int64_t)r * L + x) * a.C + c),
                          (unsigned long long)w);
            }
            if (b & kSwLabelMask) atomicOr(s_ban + pidx(r, c, a.C), b & kSwLabelMask);
        }
        __syncthreads();
        // labels of the roots
        for (int64_t g = threadIdx.x; g < nv; g += blockDim.x) {
            const int32_t v = (int32_t)a.fdC.div((uint32_t)g), c = (int32_t)(g - (int64_t)v * a.C);
            const uint32_t b = s_ban[g];
            const bool bonded = (b & kSwBonded) != 0u;
            if (bonded && s_root[g] != v) continue;
            int64_t w[L];
#pragma unroll
            for (int x = 0; x < L; ++x) {
                w[x] = __ldg(a.ufix + (int64_t)v * L + x);
                if (bonded) w[x] += s_lw[((int64_t)v * L + x) * a.C + c];
            }
            int64_t mx = 0;
            bool any = false;
#pragma unroll
            for (int x = 0; x < L; ++x)
                if (!((b >> x) & 1u) && (!any || w[x] > mx)) { mx = w[x]; any = true; }
            float F[L];
#pragma unroll
            for (int x = 0; x < L; ++x) F[x] = ((b >> x) & 1u) ? -INFINITY : sw_float(w[x] - mx);
            xout[g] = (uint8_t)draw_label<L>(F, (uint32_t)v, (uint32_t)c, sweep, a.rk, PH_CLUSTER, nullptr, a.ctl);
        }
        __syncthreads();
        // labels of the other sites, state reset
        for (int64_t g = threadIdx.x; g < nv; g += blockDim.x) {
            const uint32_t b = s_ban[g];
            if (!(b & kSwBonded)) continue;
            const int32_t v = (int32_t)a.fdC.div((uint32_t)g), c = (int32_t)(g - (int64_t)v * a.C);
            const int32_t r = s_root[g];
            if (r != v) xout[g] = xout[pidx(r, c, a.C)];
            if (r == v || (b & kSwRow)) {
#pragma unroll
                for (int x = 0; x < L; ++x) s_lw[((int64_t)v * L + x) * a.C + c] = 0;
            }
            s_par[g] = v;
            s_ban[g] = 0u;
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

// Higdon's partial Swendsen-Wang (Section 4.3): per edge and label a with
// coupling l (float64), alpha = rho (e^l - 1) and the remainder
// A = exp(l' [a = b]), l' = log(1 + (1 - rho)(e^l - 1)), dualised by
// entry_dual (diagonal layout, entry k = label k).  Written per edge: the bond
// threshold of rho (1 - e^{-l}), the bond weight log alpha - alpha1 - alpha2
// in fixed point, A's dual weights, thresholds and unary terms, and the
// edge's bound for the range check.
__global__ void k_hg_tables(const int32_t* __restrict__ src, const double* __restrict__ ell, int64_t E, int L,
                            double rho, HigdonTables t) {
    const int MP = pad4(L);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        double bound_w = 0.0, bound_tau = 0.0;
        for (int x = 0; x < L; ++x) {
            const double l = src[e] >= 0 ? ell[e * L + x] : 0.0;
            const double alpha = rho * expm1(l);
            const double lp = log1p((1.0 - rho) * expm1(l));
            uint32_t T = 0;
            if (l > 0.0 && rho > 0.0) T = (uint32_t)ceil(rho * -expm1(-l) * 8388608.0 - 0.5);
            float tau_s = 0.0f;
            uint32_t word = 0;
            double a12 = 0.0;
            if (lp != 0.0) {
                const EntryDual d = entry_dual(lp);
                tau_s = d.tau_s; word = d.word; a12 = d.alpha1 + d.alpha2;
                t.fold[(e * 2 + 0) * L + x] = d.alpha1;
                t.fold[(e * 2 + 1) * L + x] = d.alpha2;
            } else {
                t.fold[(e * 2 + 0) * L + x] = 0.0;
                t.fold[(e * 2 + 1) * L + x] = 0.0;
            }
            int64_t lw = kSwNoLabel;
            if (alpha > 0.0) {
                const double w = log(alpha) - a12;
                lw = sw_fix(w);
                bound_w = fmax(bound_w, fabs(w));
            }
            bound_tau = fmax(bound_tau, fabs((double)tau_s));
            t.bond_thr[e * L + x] = T;
            t.bond_lw[e * L + x] = lw;
            t.tau[e * MP + x] = tau_s;
            t.thr[e * L + x] = word;
        }
        for (int x = L; x < MP; ++x) t.tau[e * MP + x] = 0.0f;
        t.bound[e] = src[e] >= 0 ? bound_w + 2.0 * bound_tau : 0.0;
    }
}

// out[0] += sum over sites of max_x |ut_v(x)| + sum over live edges of their bound.
__global__ void k_hg_check(const double* __restrict__ ut, int N, int L, const int32_t* __restrict__ src,
                           const double* __restrict__ bound, int64_t E, double* out) {
    double acc = 0.0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        double m = 0.0;
        for (int x = 0; x < L; ++x) m = fmax(m, fabs(ut[v * L + x]));
        acc += m;
    }
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x)
        if (src[e] >= 0) acc += bound[e];
    if (acc != 0.0) atomicAdd(out, acc);
}

// A bond carries no bits of A: clear the dual bits of every bonded (edge,
// chain) item (one dual word per item: the diagonal layout with L <= 16).
__global__ void k_hg_clear(const uint32_t* __restrict__ bits, uint32_t* __restrict__ theta, int64_t items) {
    const int64_t words = (items + 31) >> 5;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t word = bits[i];
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1u;
            theta[i * 32 + b] = 0u;
        }
    }
}

// Small models, Higdon's sweep: n_sweeps whole sweeps in one single-CTA
// launch, the remainder's dual bits, the union-find state and the cluster
// rows in shared memory.  The bonds, bits (the dual contract of k_dual,
// decided by dual_bits), potentials (summed in the incidence order of the
// primal kernels, flushed every 32 incidences) and exact cluster sums are
// those of the launch-per-step path, hence the same chain bit for bit.
template <int L>
__global__ void __launch_bounds__(1024) k_hg_small(SweepArgs d, SwArgs a, int n_sweeps) {
    using En = Ent<L, MRF_LAYOUT_DIAG>;
    extern __shared__ int64_t s_lw[];                                  // [N][L][C]
    const int64_t nv = (int64_t)a.N * a.C, ne = a.E * a.C;
    int32_t* s_par = reinterpret_cast<int32_t*>(s_lw + nv * L);       // [N][C]
    int32_t* s_root = s_par + nv;                                     // [N][C]
    uint32_t* s_ban = reinterpret_cast<uint32_t*>(s_root + nv);       // [N][C]
    uint32_t* s_theta = s_ban + nv;                                   // [E][C] remainder's bits
    volatile int32_t* vpar = s_par;
    for (int64_t g = threadIdx.x; g < nv; g += blockDim.x) {
        s_par[g] = (int32_t)a.fdC.div((uint32_t)g);
        s_ban[g] = 0u;
    }
    for (int64_t i = threadIdx.x; i < nv * L; i += blockDim.x) s_lw[i] = 0;
    __syncthreads();
    uint32_t sweep = (uint32_t)a.ctl->sweep;
    const unsigned long long count_from = a.ctl->count_from;
    for (int it = 0; it < n_sweeps; ++it, ++sweep) {
        const uint8_t* xin = a.x + (size_t)(sweep & 1) * a.N * a.C;
        uint8_t* xout = a.x + (size_t)((sweep + 1) & 1) * a.N * a.C;
        // bonds (with their unions) or the remainder's bits, per (edge, chain)
        for (int64_t g = threadIdx.x; g < ne; g += blockDim.x) {
            const int64_t e = a.fdC.div((uint32_t)g);
            const int32_t c = (int32_t)(g - e * a.C);
            const int32_t s = a.src[e];
            s_theta[g] = 0u;
            if (s < 0) continue;
            const int32_t t = a.dst[e];
            const int xs = xin[pidx(s, c, a.C)], xt = xin[pidx(t, c, a.C)];
            bool bond = false;
            if (xs == xt) {
                const uint32_t T = a.thr[e * L + xs];
                bond = T != 0u && (draw_rk((uint32_t)e, sweep, (uint32_t)c, PH_BOND, 0, a.rk).x >> 9) < T;
            }
            if (!bond) {
                uint32_t bits[En::W];
                dual_bits<L, MRF_LAYOUT_DIAG>((uint32_t)e, (uint32_t)c, xs, xt, d.tpl + e * En::PW, d.thr + e * En::M,
                                              sweep, d.rk, bits);
                s_theta[g] = bits[0];
                continue;
            }
            int32_t ra = s, rb = t;
            bool linked = false;
            for (int32_t step = 0; step <= a.N && !linked; ++step) {
                ra = sws_find(vpar, ra, c, a.C, a.N);
                rb = sws_find(vpar, rb, c, a.C, a.N);
                if (ra < 0 || rb < 0) break;
                if (ra == rb) { linked = true; break; }
                if (ra < rb) { const int32_t t2 = ra; ra = rb; rb = t2; }
                linked = atomicCAS(s_par + pidx(ra, c, a.C), ra, rb) == ra;
            }
            if (!linked) { atomicOr(a.err, 1u); continue; }
            int64_t wv[L];
#pragma unroll
            for (int x = 0; x < L; ++x) wv[x] = __ldg(a.lwe + e * L + x);
            bool uniform = wv[0] != kSwNoLabel;
#pragma unroll
            for (int x = 1; x < L; ++x) uniform &= wv[x] == wv[0];
            uint32_t flags = kSwBonded;
            if (!uniform) {
                flags |= kSwRow;
#pragma unroll
                for (int x = 0; x < L; ++x) {
                    if (wv[x] == kSwNoLabel) flags |= 1u << x;
                    else atomicAdd(reinterpret_cast<unsigned long long*>(s_lw + ((int64_t)s * L + x) * a.C + c),
                                   (unsigned long long)wv[x]);
                }
            }
            atomicOr(s_ban + pidx(s, c, a.C), flags);
            atomicOr(s_ban + pidx(t, c, a.C), kSwBonded);
        }
        __syncthreads();
        // potentials of every site, moved into the rows of the cluster roots
        for (int64_t g = threadIdx.x; g < nv; g += blockDim.x) {
            const int32_t v = (int32_t)a.fdC.div((uint32_t)g), c = (int32_t)(g - (int64_t)v * a.C);
            float acc[L], hi[L], lo[L];
#pragma unroll
            for (int x = 0; x < L; ++x) { acc[x] = 0.0f; hi[x] = 0.0f; lo[x] = 0.0f; }
            int chunk = 0;
            bool flushed = false;
            for (int64_t p = d.inc_ptr[v]; p < d.inc_ptr[v + 1]; ++p) {
                const int2 ic = __ldg(&d.inc[p]);
                const int64_t e = ic.x >> 1;
                const uint32_t bits[En::W] = {s_theta[e * a.C + c]};
                add_side<L, MRF_LAYOUT_DIAG>(bits, d.tau + e * En::MP, ic.x & 1, acc);
                if (++chunk == 32) {
#pragma unroll
                    for (int x = 0; x < L; ++x) { two_sum_add(hi[x], lo[x], acc[x]); acc[x] = 0.0f; }
                    chunk = 0;
                    flushed = true;
                }
            }
            int64_t w[L];
            const float* uf = d.utf + (int64_t)v * L;
#pragma unroll
            for (int x = 0; x < L; ++x) {
                float F;
                if (flushed) { two_sum_add(hi[x], lo[x], acc[x]); F = __ldg(uf + x) + (hi[x] + lo[x]); }
                else F = __ldg(uf + x) + acc[x];
                w[x] = fix_from_float(F);
            }
            const uint32_t b = s_ban[g];
            int32_t r = v;
            if (b & kSwBonded) {
                r = sws_find(vpar, v, c, a.C, a.N);
                if (r < 0) { atomicOr(a.err, 1u); r = v; }
                s_root[g] = r;
                if (r != v && (b & kSwRow)) {
#pragma unroll
                    for (int x = 0; x < L; ++x) w[x] += s_lw[((int64_t)v * L + x) * a.C + c];
                }
                if (r != v && (b & kSwLabelMask)) atomicOr(s_ban + pidx(r, c, a.C), b & kSwLabelMask);
            }
#pragma unroll
            for (int x = 0; x < L; ++x)
                atomicAdd(reinterpret_cast<unsigned long long*>(s_lw + ((int64_t)r * L + x) * a.C + c),
                          (unsigned long long)w[x]);
        }
        __syncthreads();
        // labels of the roots
        for (int64_t g = threadIdx.x; g < nv; g += blockDim.x) {
            const int32_t v = (int32_t)a.fdC.div((uint32_t)g), c = (int32_t)(g - (int64_t)v * a.C);
            const uint32_t b = s_ban[g];
            if ((b & kSwBonded) && s_root[g] != v) continue;
            int64_t w[L];
#pragma unroll
            for (int x = 0; x < L; ++x) w[x] = s_lw[((int64_t)v * L + x) * a.C + c];
            int64_t mx = 0;
            bool any = false;
#pragma unroll
            for (int x = 0; x < L; ++x)
                if (!((b >> x) & 1u) && (!any || w[x] > mx)) { mx = w[x]; any = true; }
            float F[L];
#pragma unroll
            for (int x = 0; x < L; ++x) F[x] = ((b >> x) & 1u) ? -INFINITY : sw_float(w[x] - mx);
            xout[g] = (uint8_t)draw_label<L>(F, (uint32_t)v, (uint32_t)c, sweep, a.rk, PH_CLUSTER, nullptr, a.ctl);
        }
        __syncthreads();
        // labels of the other sites, state reset (every root's row holds sums now)
        for (int64_t g = threadIdx.x; g < nv; g += blockDim.x) {
            const int32_t v = (int32_t)a.fdC.div((uint32_t)g), c = (int32_t)(g - (int64_t)v * a.C);
            const uint32_t b = s_ban[g];
            const int32_t r = (b & kSwBonded) ? s_root[g] : v;
            if (r != v) xout[g] = xout[pidx(r, c, a.C)];
            if (r == v || (b & kSwRow)) {
#pragma unroll
                for (int x = 0; x < L; ++x) s_lw[((int64_t)v * L + x) * a.C + c] = 0;
            }
            s_par[g] = v;
            s_ban[g] = 0u;
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

// Model check before the first Swendsen-Wang sweep after the factors change:
// out[0] = dual weights tau < 0 on live edges (antiferromagnetic entries; with
// two labels the one pivot entry's tau has the sign of l),
// out[1] = sum over live edges of max_x |log(e^{l_x} - 1)| over bondable labels,
// out[2] = sum over sites of max_x |u_v(x)| (the unaries the sweep uses).
// out[1] + out[2] bounds the magnitude of every partial sum of a cluster weight.
__global__ void k_sw_check(const int32_t* src, const float* tau, int64_t E, int M, const int64_t* lwe, int L,
                           const float* unary, const double* unary_d, int N, double* out) {
    double neg = 0.0, se = 0.0, su = 0.0;
    const int MP = pad4(M);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        if (src[e] < 0) continue;
        double m = 0.0;
        for (int k = 0; k < M; ++k) neg += tau[e * MP + k] < 0.0f;
        for (int x = 0; x < L; ++x) {
            const int64_t w = lwe[e * L + x];
            if (w != kSwNoLabel) m = fmax(m, fabs((double)w / kSwFixScale));
        }
        se += m;
    }
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        double m = 0.0;
        for (int x = 0; x < L; ++x) m = fmax(m, fabs(unary_d ? unary_d[v * L + x] : (double)unary[v * L + x]));
        su += m;
    }
    if (neg != 0.0) atomicAdd(out + 0, neg);
    if (se != 0.0) atomicAdd(out + 1, se);
    if (su != 0.0) atomicAdd(out + 2, su);
}

#define MRF_DISPATCH_LSW(L_, ...)                                                 \
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

static inline unsigned sw_blocks(int64_t n) {
    // grid-stride loops over at most 8 resident blocks of 256 threads per SM
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8);
}

cudaError_t launch_sw_check(const int32_t* src, const float* tau, int64_t E, int M, const int64_t* lwe, int L,
                            const float* unary, const double* unary_d, int N, double* out, cudaStream_t s) {
    k_sw_check<<<sw_blocks(E > N ? E : N), 256, 0, s>>>(src, tau, E, M, lwe, L, unary, unary_d, N, out);
    return cudaGetLastError();
}

// Fixed-point unaries ufix[v][x] = sw_fix(u_v(x)) (once per factor change).
__global__ void k_sw_fix_unary(const float* unary, const double* unary_d, int64_t n, int64_t* ufix) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        ufix[i] = sw_fix(unary_d ? unary_d[i] : (double)unary[i]);
}

cudaError_t launch_hg_tables(const int32_t* src, const double* ell, int64_t E, int L, double rho, HigdonTables t,
                             cudaStream_t s) {
    if (E > 0) k_hg_tables<<<sw_blocks(E), 256, 0, s>>>(src, ell, E, L, rho, t);
    return cudaGetLastError();
}

cudaError_t launch_hg_check(const double* ut, int N, int L, const int32_t* src, const double* bound, int64_t E,
                            double* out, cudaStream_t s) {
    k_hg_check<<<sw_blocks(E > N ? E : N), 256, 0, s>>>(ut, N, L, src, bound, E, out);
    return cudaGetLastError();
}

cudaError_t launch_hg_clear(const uint32_t* bits, uint32_t* theta, int64_t items, cudaStream_t s) {
    if (items > 0) k_hg_clear<<<sw_blocks((items + 31) / 32), 256, 0, s>>>(bits, theta, items);
    return cudaGetLastError();
}

cudaError_t launch_sw_fix_unary(const float* unary, const double* unary_d, int64_t n, int64_t* ufix, cudaStream_t s) {
    if (n > 0) k_sw_fix_unary<<<sw_blocks(n), 256, 0, s>>>(unary, unary_d, n, ufix);
    return cudaGetLastError();
}

cudaError_t launch_sw_reset(const SwArgs& a, cudaStream_t s) {
    const int64_t n = (int64_t)a.N * a.C;
    if (n > 0) {
        k_sw_reset<<<sw_blocks(n), 256, 0, s>>>(a);
        const cudaError_t e = cudaMemsetAsync(a.lw, 0, (size_t)n * a.L * sizeof(int64_t), s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_sw_bond(const SwArgs& a, cudaStream_t s) {
    const int64_t n = a.E * a.C;
    if (n <= 0) return cudaSuccess;
    k_sw_bond<<<sw_blocks(n), 256, 0, s>>>(a);
    MRF_DISPATCH_LSW(a.L, (k_sw_union<LL><<<sw_blocks((n + 31) / 32), 256, 0, s>>>(a)));
    return cudaGetLastError();
}

cudaError_t launch_sw_flatten(const SwArgs& a, cudaStream_t s) {
    const int64_t n = (int64_t)a.N * a.C;
    if (n <= 0) return cudaSuccess;
    MRF_DISPATCH_LSW(a.L, (k_sw_flatten<LL><<<sw_blocks(n), 256, 0, s>>>(a)));
    return cudaGetLastError();
}

int64_t sw_small_smem(const SwArgs& a) { return (int64_t)a.N * a.C * (12 + 8 * a.L); }

cudaError_t launch_sw_small(const SwArgs& a, int n_sweeps, cudaStream_t s) {
    if (!a.counts || !a.ufix || !a.err || !a.ctl || !a.x || (a.E > 0 && (!a.src || !a.dst || !a.thr || !a.lwe)))
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)sw_small_smem(a);
    MRF_DISPATCH_LSW(a.L, ({
        if (smem > 48 * 1024) {
            const cudaError_t e = cudaFuncSetAttribute(k_sw_small<LL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_sw_small<LL><<<1, 1024, smem, s>>>(a, n_sweeps);
    }));
    return cudaGetLastError();
}

int64_t hg_small_smem(const SwArgs& a) { return (int64_t)a.N * a.C * (12 + 8 * a.L) + a.E * a.C * 4; }

cudaError_t launch_hg_small(const SweepArgs& d, const SwArgs& a, int n_sweeps, cudaStream_t s) {
    if (!a.counts || !a.ufix || !a.err || !a.ctl || !a.x || !d.utf || !d.inc_ptr ||
        (a.E > 0 && (!a.src || !a.dst || !a.thr || !a.lwe || !d.tau || !d.thr || !d.tpl || !d.inc)))
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)hg_small_smem(a);
    MRF_DISPATCH_LSW(a.L, ({
        if (smem > 48 * 1024) {
            const cudaError_t e = cudaFuncSetAttribute(k_hg_small<LL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_hg_small<LL><<<1, 1024, smem, s>>>(d, a, n_sweeps);
    }));
    return cudaGetLastError();
}

cudaError_t launch_sw_draw(const SwArgs& a, cudaStream_t s) {
    const int64_t n = (int64_t)a.N * a.C;
    if (n <= 0) return cudaSuccess;
    MRF_DISPATCH_LSW(a.L, (k_sw_draw<LL><<<sw_blocks(n), 256, 0, s>>>(a)));
    MRF_DISPATCH_LSW(a.L, (k_sw_assign<LL><<<sw_blocks(n), 256, 0, s>>>(a)));
    return cudaGetLastError();
}

}  // namespace mrfk
