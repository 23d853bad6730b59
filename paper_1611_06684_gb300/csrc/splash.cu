// Blocked sweep of Section 5.4 on a lattice (Figure 1: blocking with respect
// to a tree).  Every sweep draws an offset o in [0,4)^3 for a grid of 4x4x4
// blocks (clipped at the lattice boundary).  Inside each block the dual
// variables of a "comb" spanning tree are kept exact:
//   parent(lx>0, ly, lz) = (lx-1, ly, lz), parent(0, ly>0, lz) = (0, ly-1, lz),
//   parent(0, 0, lz>0) = (0, 0, lz-1), root (0, 0, 0),
// all other duals are drawn (k_dual with the tree edges masked), node
// potentials phi_v = u~_v + sum of the drawn beta terms are gathered
// (k_primal in potential mode), and x | theta_1 is sampled exactly per block
// and chain by forward filtering / backward sampling (k_ffbs) with the exact
// tree-edge potentials psi_e(a, b) = w_e(a, b) - fold_s(a) - fold_t(b).
#include "common.cuh"

namespace mrfk {

template <int L, int LAYOUT> cudaError_t run_potential(const SweepArgs& a, cudaStream_t s);

// Offset of the block grid for blocked sweep t (t = the sweep index) or, for
// blocked EM, iteration t (iter >= 0).
__global__ void k_splash_offset(SweepArgs a, int64_t iter) {
    const uint32_t t = iter >= 0 ? (uint32_t)iter : (uint32_t)a.ctl->sweep;
    const uint4 r = draw(0, t, 0, PH_SPLASH, 0, a.key);
    a.ctl->splash_offset = (r.x >> 30) | ((r.y >> 30) << 8) | ((r.z >> 30) << 16);
}

// out[b] = log sum_a exp(bel[a] + psi[b][a]) - max_b(...)  (message to the
// parent with label b).  Subtracting the maximum over b keeps beliefs of the
// size of one node's potentials however large the subtree; a constant shift
// of a message changes no conditional.  psi rows are read as 16-byte vectors
// when L is a multiple of 4.
template <int L>
__device__ __forceinline__ void tree_message(const float (&bel)[L], const float* __restrict__ psi, float (&out)[L]) {
    float top = -INFINITY;
#pragma unroll
    for (int b = 0; b < L; ++b) {
        float t[L];
        if (L % 4 == 0) {
            const float4* r4 = reinterpret_cast<const float4*>(psi + b * L);
#pragma unroll
            for (int q = 0; q < L / 4; ++q) {
                const float4 v = __ldg(r4 + q);
                t[4 * q + 0] = bel[4 * q + 0] + v.x;
                t[4 * q + 1] = bel[4 * q + 1] + v.y;
                t[4 * q + 2] = bel[4 * q + 2] + v.z;
                t[4 * q + 3] = bel[4 * q + 3] + v.w;
            }
        } else {
#pragma unroll
            for (int x = 0; x < L; ++x) t[x] = bel[x] + __ldg(psi + b * L + x);
        }
        float mx = -INFINITY;
#pragma unroll
        for (int x = 0; x < L; ++x) mx = fmaxf(mx, t[x]);
        float s = 0.0f;
#pragma unroll
        for (int x = 0; x < L; ++x) s += expf(t[x] - mx);
        out[b] = mx + logf(s);
        top = fmaxf(top, out[b]);
    }
#pragma unroll
    for (int b = 0; b < L; ++b) out[b] -= top;
}

// Max-product counterpart: out[b] = max_a (bel[a] + psi[b][a]) - max_b(...).
template <int L>
__device__ __forceinline__ void tree_message_max(const float (&bel)[L], const float* __restrict__ psi, float (&out)[L]) {
    float top = -INFINITY;
#pragma unroll
    for (int b = 0; b < L; ++b) {
        float mx = -INFINITY;
#pragma unroll
        for (int x = 0; x < L; ++x) mx = fmaxf(mx, bel[x] + __ldg(psi + b * L + x));
        out[b] = mx;
        top = fmaxf(top, mx);
    }
#pragma unroll
    for (int b = 0; b < L; ++b) out[b] -= top;
}

template <int L>
__device__ __forceinline__ void label_draw_ffbs(const float (&F)[L], uint32_t v, uint32_t c, uint32_t sweep, uint2 key,
                                                float* logp_out, Ctl* ctl, int& lab) {
    float mx = F[0];
#pragma unroll
    for (int x = 1; x < L; ++x) mx = fmaxf(mx, F[x]);
    float ex[L];
    float s = 0.0f;
#pragma unroll
    for (int x = 0; x < L; ++x) { ex[x] = expf(F[x] - mx); s += ex[x]; }
    const float inv = 1.0f / s;
    if (logp_out) {
        const float ls = logf(s);
#pragma unroll
        for (int x = 0; x < L; ++x) logp_out[x] = (F[x] - mx) - ls;
    }
    const uint32_t U = draw(v, sweep, c, PH_FFBS, 0, key).x >> 9;
    const float u = ((float)U + 0.5f) * (1.0f / 8388608.0f);
    float cdf = 0.0f;
    int pick = -1, last_pos = 0;
    bool near = false;
#pragma unroll
    for (int x = 0; x < L; ++x) {
        const float p = ex[x] * inv;
        cdf += p;
        if (p > 0.0f) last_pos = x;
        if (pick < 0 && u < cdf) pick = x;
        near |= fabsf(u - cdf) < 1e-6f;
    }
    if (near) atomicAdd(&ctl->boundary, 1ull);
    lab = pick < 0 ? last_pos : pick;
}

// Downward sum-product message to a child: out[a] = log sum_b exp(B[b] +
// psi[b][a]), B the parent's belief without the child's own message.
template <int L>
__device__ __forceinline__ void tree_message_down(const float (&B)[L], const float* __restrict__ psi, float (&out)[L]) {
#pragma unroll
    for (int x = 0; x < L; ++x) {
        float t[L], mx = -INFINITY;
#pragma unroll
        for (int b = 0; b < L; ++b) { t[b] = B[b] + __ldg(psi + b * L + x); mx = fmaxf(mx, t[b]); }
        float s = 0.0f;
#pragma unroll
        for (int b = 0; b < L; ++b) s += expf(t[b] - mx);
        out[x] = mx + logf(s);
    }
}

enum FfbsMode { FFBS_SAMPLE = 0, FFBS_MAP = 1, FFBS_MARGINALS = 2 };

// One thread per (block, chain); lanes are consecutive chains of one block.
// MODE = FFBS_SAMPLE: forward filtering / backward sampling (blocked sweep).
// MODE = FFBS_MAP (blocked EM): max-product messages and argmax labels (first
// maximum) written to xmap.  MODE = FFBS_MARGINALS (tree mean field):
// sum-product messages up, then down (each child's message from its parent's
// full belief minus the child's own upward message), site marginals written
// to qmarg ([N][L][C]).
template <int L, int MODE = FFBS_SAMPLE>
__global__ void __launch_bounds__(128) k_ffbs(SweepArgs a, uint8_t* __restrict__ xmap = nullptr,
                                              float* __restrict__ qmarg = nullptr) {
    constexpr bool MAP = MODE == FFBS_MAP;
    int ox, oy, oz;
    {
        const uint32_t o = (uint32_t)a.ctl->splash_offset;
        ox = o & 0xFF; oy = (o >> 8) & 0xFF; oz = (o >> 16) & 0xFF;
    }
    const int nx = a.grid_nx, ny = a.grid_ny, nz = a.grid_nz;
    const int nbx = (nx + ox + 3) >> 2, nby = (ny + oy + 3) >> 2, nbz = (nz + oz + 3) >> 2;
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (uint64_t)nbx * nby * nbz * a.C) return;
    const uint32_t b = a.fdC.div(g), c = g - b * (uint32_t)a.C;
    const int bx = (int)(b % (uint32_t)nbx), by = (int)((b / (uint32_t)nbx) % (uint32_t)nby);
    const int bz = (int)(b / ((uint32_t)nbx * nby));
    const int x0 = max(0, 4 * bx - ox), x1 = min(nx, 4 * bx + 4 - ox);
    const int y0 = max(0, 4 * by - oy), y1 = min(ny, 4 * by + 4 - oy);
    const int z0 = max(0, 4 * bz - oz), z1 = min(nz, 4 * bz + 4 - oz);
    const int sx = x1 - x0, sy = y1 - y0, sz = z1 - z0;
    const uint32_t sweep = (uint32_t)a.ctl->sweep;
    uint8_t* xout = MAP ? xmap : a.x + (size_t)((sweep + 1) & 1) * a.N * a.C;
    const int64_t C = a.C;
    auto site = [&](int x, int y, int z) -> int64_t { return x + (int64_t)nx * (y + (int64_t)ny * z); };
    auto xedge = [&](int x, int y, int z) -> int64_t { return ((int64_t)z * ny + y) * (nx - 1) + x; };
    auto yedge = [&](int x, int y, int z) -> int64_t { return a.nxe + ((int64_t)z * (ny - 1) + y) * nx + x; };
    auto zedge = [&](int x, int y, int z) -> int64_t { return a.nxe + a.nye + ((int64_t)z * ny + y) * nx + x; };

    // upward pass: beliefs bel_v = phi_v + messages of the children, stored in
    // place.  Nodes in reverse order i = n-1 .. 0 (i = lx + sx (ly + sy lz));
    // the next node's potentials are loaded before the current node's message
    // is computed, so their latency overlaps it.
    float xm[L], ym[L], zm[L];
#pragma unroll
    for (int x = 0; x < L; ++x) { xm[x] = 0.0f; ym[x] = 0.0f; zm[x] = 0.0f; }
    const int n_nodes = sx * sy * sz;
    float nxt[L];
    {
        const float* pv = a.pot + site(x1 - 1, y1 - 1, z1 - 1) * L * C + c;
#pragma unroll
        for (int x = 0; x < L; ++x) nxt[x] = pv[x * C];
    }
    int lx = sx - 1, ly = sy - 1, lz = sz - 1;
    for (int i = n_nodes - 1; i >= 0; --i) {
        float bel[L];
#pragma unroll
        for (int x = 0; x < L; ++x) bel[x] = nxt[x];
        const int X = x0 + lx, Y = y0 + ly, Z = z0 + lz;
        // coordinates of node i - 1
        int px = lx - 1, py = ly, pz = lz;
        if (px < 0) { px = sx - 1; if (--py < 0) { py = sy - 1; --pz; } }
        if (i > 0) {
            const float* pn = a.pot + site(x0 + px, y0 + py, z0 + pz) * L * C + c;
#pragma unroll
            for (int x = 0; x < L; ++x) nxt[x] = pn[x * C];
        }
        float* pv = a.pot + site(X, Y, Z) * L * C + c;
#pragma unroll
        for (int x = 0; x < L; ++x) {
            float f = bel[x];
            if (lx + 1 < sx) f += xm[x];
            if (lx == 0 && ly + 1 < sy) f += ym[x];
            if (lx == 0 && ly == 0 && lz + 1 < sz) f += zm[x];
            bel[x] = f;
            pv[x * C] = f;
        }
        auto send = [&](const float* pe, float (&msg)[L]) {
            if (MAP) tree_message_max<L>(bel, pe, msg);
            else tree_message<L>(bel, pe, msg);
        };
        if (lx > 0) send(a.resid + xedge(X - 1, Y, Z) * L * L, xm);
        else if (ly > 0) send(a.resid + yedge(X, Y - 1, Z) * L * L, ym);
        else if (lz > 0) send(a.resid + zedge(X, Y, Z - 1) * L * L, zm);
        lx = px; ly = py; lz = pz;
    }
    if constexpr (MODE == FFBS_MARGINALS) {
        // downward pass: total belief (upward belief + message from the parent)
        // of the last node of the x-chain, of the first node of the row and of
        // the first node of the plane, each shifted to maximum 0
        float xT[L], yT[L], zT[L];
#pragma unroll
        for (int x = 0; x < L; ++x) { xT[x] = 0.0f; yT[x] = 0.0f; zT[x] = 0.0f; }
        for (int lz = 0; lz < sz; ++lz)
            for (int ly = 0; ly < sy; ++ly)
                for (int lx = 0; lx < sx; ++lx) {
                    const int X = x0 + lx, Y = y0 + ly, Z = z0 + lz;
                    const int64_t v = site(X, Y, Z);
                    const float* pv = a.pot + v * L * C + c;
                    float bel[L], tot[L];
#pragma unroll
                    for (int x = 0; x < L; ++x) bel[x] = pv[x * C];
                    const float* psi = nullptr;
                    const float* PT = nullptr;
                    if (lx > 0) { psi = a.resid + xedge(X - 1, Y, Z) * L * L; PT = xT; }
                    else if (ly > 0) { psi = a.resid + yedge(X, Y - 1, Z) * L * L; PT = yT; }
                    else if (lz > 0) { psi = a.resid + zedge(X, Y, Z - 1) * L * L; PT = zT; }
                    if (psi) {
                        float up[L], B[L], dn[L];
                        tree_message<L>(bel, psi, up);          // the message this node sent up
#pragma unroll
                        for (int x = 0; x < L; ++x) B[x] = PT[x] - up[x];
                        tree_message_down<L>(B, psi, dn);
#pragma unroll
                        for (int x = 0; x < L; ++x) tot[x] = bel[x] + dn[x];
                    } else {
#pragma unroll
                        for (int x = 0; x < L; ++x) tot[x] = bel[x];
                    }
                    float mx = -INFINITY;
#pragma unroll
                    for (int x = 0; x < L; ++x) mx = fmaxf(mx, tot[x]);
                    float ex[L], sum = 0.0f;
#pragma unroll
                    for (int x = 0; x < L; ++x) { tot[x] -= mx; ex[x] = expf(tot[x]); sum += ex[x]; }
                    const float inv = 1.0f / sum;
                    float* qv = qmarg + v * L * C + c;
#pragma unroll
                    for (int x = 0; x < L; ++x) qv[x * C] = ex[x] * inv;
#pragma unroll
                    for (int x = 0; x < L; ++x) {
                        xT[x] = tot[x];
                        if (lx == 0) {
                            yT[x] = tot[x];
                            if (ly == 0) zT[x] = tot[x];
                        }
                    }
                }
        return;
    }
    // downward pass: root, then every child given its parent's label
    int xl = 0, yl = 0, zl = 0;
    for (int lz = 0; lz < sz; ++lz)
        for (int ly = 0; ly < sy; ++ly)
            for (int lx = 0; lx < sx; ++lx) {
                const int X = x0 + lx, Y = y0 + ly, Z = z0 + lz;
                const int64_t v = site(X, Y, Z);
                const float* pv = a.pot + v * L * C + c;
                const float* psi = nullptr;
                int pl = 0;
                if (lx > 0) { psi = a.resid + xedge(X - 1, Y, Z) * L * L; pl = xl; }
                else if (ly > 0) { psi = a.resid + yedge(X, Y - 1, Z) * L * L; pl = yl; }
                else if (lz > 0) { psi = a.resid + zedge(X, Y, Z - 1) * L * L; pl = zl; }
                float F[L];
#pragma unroll
                for (int x = 0; x < L; ++x) F[x] = pv[x * C] + (psi ? __ldg(psi + pl * L + x) : 0.0f);
                int lab = 0;
                if (MAP) {
                    float fb = F[0];
#pragma unroll
                    for (int x = 1; x < L; ++x)
                        if (F[x] > fb) { fb = F[x]; lab = x; }
                } else {
                    float* lp = a.logp ? a.logp + ((int64_t)c * a.N + v) * L : nullptr;
                    label_draw_ffbs<L>(F, (uint32_t)v, c, sweep, a.key, lp, a.ctl, lab);
                }
                xout[v * C + c] = (uint8_t)lab;
                xl = lab;
                if (lx == 0) {
                    yl = lab;
                    if (ly == 0) zl = lab;
                }
            }
}

#define MRF_DISPATCH_L2(L_, ...)                                                  \
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

cudaError_t launch_splash_offset(const SweepArgs& a, cudaStream_t s, int64_t iter) {
    k_splash_offset<<<1, 1, 0, s>>>(a, iter);
    return cudaGetLastError();
}

cudaError_t launch_potential(const SweepArgs& a, int layout, cudaStream_t s) {
    if (layout == MRF_LAYOUT_PIVOT) {
        MRF_DISPATCH_L2(a.L, return (run_potential<LL, MRF_LAYOUT_PIVOT>(a, s)));
    } else {
        MRF_DISPATCH_L2(a.L, return (run_potential<LL, MRF_LAYOUT_DIAG>(a, s)));
    }
    return cudaGetLastError();
}

cudaError_t launch_tree_map(const SweepArgs& a, uint8_t* xout, cudaStream_t s) {
    const int64_t nb = (int64_t)(a.grid_nx / 4 + 2) * (a.grid_ny / 4 + 2) * (a.grid_nz / 4 + 2);
    const int64_t n = nb * a.C;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    MRF_DISPATCH_L2(a.L, (k_ffbs<LL, FFBS_MAP><<<blocks, 128, 0, s>>>(a, xout)));
    return cudaGetLastError();
}

cudaError_t launch_tree_marginals(const SweepArgs& a, float* qout, cudaStream_t s) {
    const int64_t nb = (int64_t)(a.grid_nx / 4 + 2) * (a.grid_ny / 4 + 2) * (a.grid_nz / 4 + 2);
    const int64_t n = nb * a.C;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    MRF_DISPATCH_L2(a.L, (k_ffbs<LL, FFBS_MARGINALS><<<blocks, 128, 0, s>>>(a, nullptr, qout)));
    return cudaGetLastError();
}

cudaError_t launch_ffbs(const SweepArgs& a, cudaStream_t s) {
    // upper bound on blocks for any offset: (ceil(n/4) + 1) per axis
    const int64_t nb = (int64_t)(a.grid_nx / 4 + 2) * (a.grid_ny / 4 + 2) * (a.grid_nz / 4 + 2);
    const int64_t n = nb * a.C;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    MRF_DISPATCH_L2(a.L, (k_ffbs<LL><<<blocks, 128, 0, s>>>(a)));
    return cudaGetLastError();
}

cudaError_t launch_splash(const SweepArgs& a, int layout, cudaStream_t s) {
    SweepArgs b = a;
    b.splash = 1;
    cudaError_t e = launch_splash_offset(b, s);
    if (e == cudaSuccess) e = launch_dual(b, layout, s);
    if (e == cudaSuccess) e = launch_potential(b, layout, s);
    if (e == cudaSuccess) e = launch_ffbs(b, s);
    return e;
}

}  // namespace mrfk
