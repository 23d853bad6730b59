/*
 * One primal-dual sweep (Section 5.1) in float32 on the host cores, OpenMP.
 *
 * Test infrastructure and the CPU baseline of the benchmark: only the tests,
 * the smoke check and the benchmark's CPU legs use it.  It is a plain
 * multi-threaded statement of the same chain as oracle/sampler.py, with the
 * arithmetic in float32 instead of float64:
 *   dual step    theta_ek = [u_ek < sigmoid(q_ek + beta1_ek [x_s = i_k] + beta2_ek [x_t = j_k])]
 *                with u = (U24 + 1/2) / 2^24 and U24 the 24-bit integer of the
 *                draw contract (8-bit prefix from the bit planes of the DUAL
 *                phase, 16 low bits from the DUAL_LO phase);
 *   primal step  F_v(a) = u~_v(a) + sum over incident edges of the beta terms
 *                of the set dual bits in row a (source side) or column a
 *                (destination side); x_v = the first label whose cumulative
 *                softmax probability exceeds u = ((U >> 9) + 1/2) / 2^23 of the
 *                PRIMAL phase (the largest label with p > 0 if none does).
 * Philox4x32-10 is written here from Salmon, Moraes, Dror and Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32 ->
 * 64-bit products with the key bumped by the two Weyl constants.
 * Parallel over edges in the dual step and over sites in the primal step;
 * chains innermost.
 *
 * Pin (tests/test_oracle_cpu_sweep.py): dual bits and labels equal those of
 * oracle/sampler.py on the same inputs except draws within 1e-6 of their
 * decision boundary.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { PH_DUAL = 1, PH_DUAL_LO = 2, PH_PRIMAL = 3 };

static void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = (uint32_t)p1;
        c[2] = n2;
        c[3] = (uint32_t)p0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

static void draw(uint32_t out[4], uint32_t index, uint32_t sweep, uint32_t chain, uint32_t phase, uint32_t sub,
                 uint64_t seed) {
    out[0] = index;
    out[1] = sweep;
    out[2] = chain;
    out[3] = (phase << 24) | sub;
    philox(out, (uint32_t)seed, (uint32_t)(seed >> 32));
}

/* 24-bit integer uniforms U24[m] of the dual draws of (edge e, chain c). */
static void dual_u24(uint32_t e, uint32_t c, uint32_t sweep, uint64_t seed, int m, uint32_t* u24) {
    uint32_t w[4];
    for (int k = 0; k < m; ++k) u24[k] = 0;
    if (m <= 16) {
        draw(w, e, sweep, c, PH_DUAL, 0, seed);
        for (int p = 0; p < 8; ++p)
            for (int k = 0; k < m; ++k) u24[k] |= ((w[p % 4] >> (16 * (p / 4) + k)) & 1u) << (23 - p);
    } else {
        for (int g = 0; 32 * g < m; ++g)
            for (int half = 0; half < 2; ++half) {
                draw(w, e, sweep, c, PH_DUAL, (uint32_t)(2 * g + half), seed);
                for (int q = 0; q < 4; ++q) {
                    const int p = 4 * half + q;
                    for (int b = 0; b < 32 && 32 * g + b < m; ++b) u24[32 * g + b] |= ((w[q] >> b) & 1u) << (23 - p);
                }
            }
    }
    for (int k8 = 0; 8 * k8 < m; ++k8) {
        draw(w, e, sweep, c, PH_DUAL_LO, (uint32_t)k8, seed);
        for (int h = 0; h < 8 && 8 * k8 + h < m; ++h) u24[8 * k8 + h] |= (w[h >> 1] >> (16 * (h & 1))) & 0xFFFFu;
    }
}

/*
 * One sweep.  Arrays (row-major):
 *   src, dst [E]; q, beta1, beta2 [E][m] float32; active [E][m] (0/1);
 *   i_pos, j_pos [m]; utilde [N][L] float32;
 *   inc_ptr [N+1], inc_edge [2E], inc_side [2E] (0: the site is the source);
 *   x_in, x_out [C][N]; theta [E][C][W] uint32 workspace, W = ceil(m / 32).
 * Returns 0.
 */
int cpu_sweep(int N, int L, int C, int64_t E, int m, const int32_t* src, const int32_t* dst, const float* q,
              const float* beta1, const float* beta2, const uint8_t* active, const int32_t* i_pos,
              const int32_t* j_pos, const float* utilde, const int64_t* inc_ptr, const int64_t* inc_edge,
              const uint8_t* inc_side, const uint8_t* x_in, uint8_t* x_out, uint32_t* theta, uint32_t sweep,
              uint64_t seed, int n_threads) {
    const int W = (m + 31) / 32;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
#pragma omp parallel
    {
        uint32_t* u24 = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
#pragma omp for schedule(static)
        for (int64_t e = 0; e < E; ++e) {
            const int s = src[e], t = dst[e];
            for (int c = 0; c < C; ++c) {
                uint32_t* th = theta + ((size_t)e * C + c) * W;
                for (int w = 0; w < W; ++w) th[w] = 0;
                dual_u24((uint32_t)e, (uint32_t)c, sweep, seed, m, u24);
                const int xs = x_in[(size_t)c * N + s], xt = x_in[(size_t)c * N + t];
                for (int k = 0; k < m; ++k) {
                    if (!active[e * m + k]) continue;
                    const float logit = q[e * m + k] + (xs == i_pos[k] ? beta1[e * m + k] : 0.0f) +
                                        (xt == j_pos[k] ? beta2[e * m + k] : 0.0f);
                    const float p = 1.0f / (1.0f + expf(-logit));
                    const float u = ((float)u24[k] + 0.5f) * (1.0f / 16777216.0f);
                    if (u < p) th[k >> 5] |= 1u << (k & 31);
                }
            }
        }
        free(u24);
        float* F = (float*)malloc(sizeof(float) * (size_t)L);
#pragma omp for schedule(static)
        for (int v = 0; v < N; ++v) {
            for (int c = 0; c < C; ++c) {
                for (int a = 0; a < L; ++a) F[a] = utilde[(size_t)v * L + a];
                for (int64_t p = inc_ptr[v]; p < inc_ptr[v + 1]; ++p) {
                    const int64_t e = inc_edge[p];
                    const uint32_t* th = theta + ((size_t)e * C + c) * W;
                    for (int k = 0; k < m; ++k) {
                        if (!((th[k >> 5] >> (k & 31)) & 1u)) continue;
                        if (inc_side[p] == 0) F[i_pos[k]] += beta1[e * m + k];
                        else F[j_pos[k]] += beta2[e * m + k];
                    }
                }
                float mx = F[0];
                for (int a = 1; a < L; ++a) mx = F[a] > mx ? F[a] : mx;
                float sum = 0.0f;
                for (int a = 0; a < L; ++a) sum += expf(F[a] - mx);
                uint32_t r[4];
                draw(r, (uint32_t)v, sweep, (uint32_t)c, PH_PRIMAL, 0, seed);
                const float u = ((float)(r[0] >> 9) + 0.5f) * (1.0f / 8388608.0f);
                float cdf = 0.0f;
                int pick = -1, last = 0;
                for (int a = 0; a < L; ++a) {
                    const float pa = expf(F[a] - mx) / sum;
                    cdf += pa;
                    if (pa > 0.0f) last = a;
                    if (pick < 0 && u < cdf) pick = a;
                }
                x_out[(size_t)c * N + v] = (uint8_t)(pick < 0 ? last : pick);
            }
        }
        free(F);
    }
    return 0;
}
