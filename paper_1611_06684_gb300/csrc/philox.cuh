// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) for the device, and the
// sampler's draw contract.  Written from the published definition: ten rounds,
// each multiplying counter words 0 and 2 by the two round multipliers,
// exchanging the halves with xor of the key, then bumping the key by the two
// Weyl constants.
//
// Draw contract: key = (seed lo, seed hi); counter = (index, sweep, chain,
// phase << 24 | sub).  See mrf.h for the draws that use each phase.
#pragma once
#include <cstdint>

namespace mrfk {

enum Phase : uint32_t {
    PH_DUAL = 1,      // bit planes of the 8-bit prefixes of dual-bit uniforms
    PH_DUAL_LO = 2,   // low 16 bits of dual-bit uniforms (8 per call)
    PH_PRIMAL = 3,    // label draw of the plain sweep (word 0)
    PH_INIT = 4,      // initial labels (word 0)
    PH_FFBS = 5,      // label draw inside a tree block (word 0)
    PH_SPLASH = 6,    // block-grid offset of a blocked sweep (words 0..2)
    PH_PROPOSAL = 7,
    PH_ACCEPT = 8,
    PH_BOND = 9,      // Swendsen-Wang bond of (edge, chain) (word 0, 23-bit uniform)
    PH_CLUSTER = 10,  // Swendsen-Wang cluster label, index = the cluster's smallest site (word 0)
};

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
    constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(kMul0, c.x), lo0 = kMul0 * c.x;
        const uint32_t hi1 = __umulhi(kMul1, c.z), lo1 = kMul1 * c.z;
#else
        const uint64_t p0 = (uint64_t)kMul0 * c.x, p1 = (uint64_t)kMul1 * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += kWeyl0;
        k.y += kWeyl1;
    }
    return c;
}

// The ten round keys of a key (k + r * Weyl, r = 0..9), precomputed once on
// the host and passed as kernel parameters, so a call executes no key updates.
struct RoundKeys {
    uint32_t k0[10], k1[10];
};

__host__ __device__ inline RoundKeys round_keys(uint2 k) {
    RoundKeys rk{};
    for (int r = 0; r < 10; ++r) {
        rk.k0[r] = k.x + (uint32_t)r * 0x9E3779B9u;
        rk.k1[r] = k.y + (uint32_t)r * 0xBB67AE85u;
    }
    return rk;
}

// Same function as philox4x32_10 with precomputed round keys; each product is
// one 32x32 -> 64-bit multiply.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const RoundKeys& rk) {
    constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)kMul0 * c.x;
        const uint64_t p1 = (uint64_t)kMul1 * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk.k0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk.k1[r],
                       (uint32_t)p0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw_rk(uint32_t index, uint32_t sweep, uint32_t chain, uint32_t phase, uint32_t sub,
                                         const RoundKeys& rk) {
    return philox4x32_10_rk(make_uint4(index, sweep, chain, (phase << 24) | sub), rk);
}

// NC calls draw_rk(index, sweep, chain, phase, s, rk) for s = 0 .. NC-1 (NC <= 256).
// The counters differ only in the low bits of word 3, which enters round 1
// only through the new word 2; so the round-1 products, the round-2 product
// of word 0 and the round-3 product of word 2 are the same for every call and
// are computed once.
template <int NC>
__device__ __forceinline__ void draw_rk_subs(uint32_t index, uint32_t sweep, uint32_t chain, uint32_t phase,
                                             const RoundKeys& rk, uint4 (&out)[NC]) {
    constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
    const uint64_t pa = (uint64_t)kMul0 * index, pb = (uint64_t)kMul1 * chain;
    const uint32_t x1 = (uint32_t)(pb >> 32) ^ sweep ^ rk.k0[0], y1 = (uint32_t)pb;
    const uint32_t z1b = (uint32_t)(pa >> 32) ^ (phase << 24) ^ rk.k1[0], w1 = (uint32_t)pa;
    const uint64_t pc = (uint64_t)kMul0 * x1;
    const uint32_t z2 = (uint32_t)(pc >> 32) ^ w1 ^ rk.k1[1], w2 = (uint32_t)pc;
    const uint64_t pd = (uint64_t)kMul1 * z2;
    const uint32_t y3 = (uint32_t)pd, h3 = (uint32_t)(pd >> 32);
#pragma unroll
    for (int s = 0; s < NC; ++s) {
        const uint64_t p1 = (uint64_t)kMul1 * (z1b ^ (uint32_t)s);
        const uint32_t x2 = (uint32_t)(p1 >> 32) ^ y1 ^ rk.k0[1], y2 = (uint32_t)p1;
        const uint64_t p0 = (uint64_t)kMul0 * x2;
        uint4 c = make_uint4(h3 ^ y2 ^ rk.k0[2], y3, (uint32_t)(p0 >> 32) ^ w2 ^ rk.k1[2], (uint32_t)p0);
#pragma unroll
        for (int r = 3; r < 10; ++r) {
            const uint64_t q0 = (uint64_t)kMul0 * c.x, q1 = (uint64_t)kMul1 * c.z;
            c = make_uint4((uint32_t)(q1 >> 32) ^ c.y ^ rk.k0[r], (uint32_t)q1, (uint32_t)(q0 >> 32) ^ c.w ^ rk.k1[r],
                           (uint32_t)q0);
        }
        out[s] = c;
    }
}

__host__ __device__ __forceinline__ uint2 seed_key(uint64_t seed) {
    return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

__host__ __device__ __forceinline__ uint4 draw(uint32_t index, uint32_t sweep, uint32_t chain,
                                               uint32_t phase, uint32_t sub, uint2 key) {
    return philox4x32_10(make_uint4(index, sweep, chain, (phase << 24) | sub), key);
}

__device__ __forceinline__ uint32_t word_of(const uint4& r, int w) {
    return w == 0 ? r.x : (w == 1 ? r.y : (w == 2 ? r.z : r.w));
}

// Low 16 bits of the uniform of dual entry k (drawn only when the prefix byte
// ties with the threshold's prefix).
__device__ __forceinline__ uint32_t dual_low16(uint32_t e, uint32_t sweep, uint32_t c, int k, const RoundKeys& rk) {
    const uint4 r = draw_rk(e, sweep, c, PH_DUAL_LO, (uint32_t)k >> 3, rk);
    const uint32_t w = word_of(r, (k & 7) >> 1);
    return (w >> (16 * (k & 1))) & 0xFFFFu;
}

}  // namespace mrfk
