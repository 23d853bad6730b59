// Learned block proposal with Metropolis-Hastings correction (no counterpart in
// the paper; it builds on Section 5.4's blocking with respect to arbitrary
// subgraphs).  Per sweep:
//   1. dual bits of the cut edges only (k_dual with the intra-block edges masked),
//   2. node potentials phi = u~ + cut beta terms (k_primal in potential mode),
//   3. features of every (block, chain): centred phi of the <= 16 members and
//      the block's static pair couplings (k_learned_features, bf16),
//   4. MLP logits with tensor cores: two GEMM + bias + ReLU layers and a GEMM +
//      bias output layer (k_gemm_nt: mma.sync m16n8k16 bf16 -> fp32),
//   5. one independence MH step per (block, chain) against the exact block
//      conditional with intra-block factors psi = w - folds (k_learned_mh).
// Training (maximum likelihood of harvested plain-chain samples) uses float32
// SIMT kernels for the forward and backward passes and Adam on float32 master
// weights; the bf16 copies are what the proposal uses.
#include "common.cuh"

#include <cuda_bf16.h>

namespace mrfk {

using bf16 = __nv_bfloat16;

// ============================================================================ features

// Per-chain features: centred potentials of the members, Kx columns (the
// block's pair couplings enter the first layer as a per-block bias instead).
__global__ void k_learned_features(const LearnedArgs a, FastDiv fdC, const float* __restrict__ pot, int C) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (uint64_t)a.nb * C) return;
    const uint32_t b = fdC.div(r), c = r - b * (uint32_t)C;
    const int L = a.L, n = a.nmem[b];
    uint4* x = reinterpret_cast<uint4*>(a.X + (int64_t)r * a.Kx);
    uint32_t pk[4];
    int fill = 0, q16 = 0;
    auto push = [&](float v0, float v1) {
        __nv_bfloat162 t = __floats2bfloat162_rn(v0, v1);
        pk[fill++] = *reinterpret_cast<uint32_t*>(&t);
        if (fill == 4) { x[q16++] = make_uint4(pk[0], pk[1], pk[2], pk[3]); fill = 0; }
    };
    float pend = 0.0f;
    bool have = false;
    for (int i = 0; i < kLearnBlock; ++i) {
        float phi[kMaxLabels];
        float mean = 0.0f;
        if (i < n) {
            const int v = a.members[b * kLearnBlock + i];
            for (int q = 0; q < L; ++q) { phi[q] = pot[((int64_t)v * L + q) * C + c]; mean += phi[q]; }
            mean /= (float)L;
        } else {
            for (int q = 0; q < L; ++q) phi[q] = 0.0f;
        }
        for (int q = 0; q < L; ++q) {
            const float val = phi[q] - mean;
            if (have) { push(pend, val); have = false; } else { pend = val; have = true; }
        }
    }
    for (int col = kLearnBlock * L; col < a.Kx; ++col) {
        if (have) { push(pend, 0.0f); have = false; } else { pend = 0.0f; have = true; }
    }
}

// Pair couplings kappa_e = mean_a psi(a,a) - mean_{a != b} psi(a,b) of every
// intra-block edge (psi = w - folds has the same kappa as w), summed per pair.
__global__ void k_learned_couplings(LearnedArgs a, const float* __restrict__ resid, float* cf) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.nb) return;
    const int L = a.L;
    for (int p = 0; p < kLearnPairs; ++p) cf[(int64_t)b * kLearnPairs + p] = 0.0f;
    for (int64_t q = a.intra_ptr[b]; q < a.intra_ptr[b + 1]; ++q) {
        const int4 ie = a.intra[q];
        const float* ps = resid + (int64_t)ie.x * L * L;
        float dsum = 0.0f, tot = 0.0f;
        for (int u = 0; u < L; ++u)
            for (int w = 0; w < L; ++w) {
                tot += ps[u * L + w];
                if (u == w) dsum += ps[u * L + w];
            }
        const float kappa = dsum / L - (tot - dsum) / (L * (L - 1));
        const int i = min(ie.y, ie.z), j = max(ie.y, ie.z);
        cf[(int64_t)b * kLearnPairs + i * (2 * kLearnBlock - i - 1) / 2 + (j - i - 1)] += kappa;
    }
    for (int p = 0; p < kLearnPairs; ++p) a.cfb[(int64_t)b * kLearnPairs + p] = __float2bfloat16_rn(cf[(int64_t)b * kLearnPairs + p]);
}

// ============================================================================ tensor-core GEMM

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C[M][N] = act(A[M][K] W[N][K]^T + bias[N]); A, W bf16 row-major; K % 32 == 0,
// N even.  CTA tile 128 x 64 x 32, 8 warps (4 along M x 2 along N), warp
// tile 32 x 32 = 2 x 4 mma tiles, cp.async double buffering, ldmatrix fragments.
constexpr int kBM = 128, kBN = 64, kBK = 32, kPad = 8;

template <bool RELU, bool OUT_BF16>
__global__ void __launch_bounds__(256) k_gemm_nt(const bf16* __restrict__ A, const bf16* __restrict__ W,
                                                 const float* __restrict__ bias, void* __restrict__ Cout, int M, int N,
                                                 int K, const float* __restrict__ rowbias, FastDiv rows_per_bias) {
    __shared__ __align__(16) bf16 As[2][kBM][kBK + kPad];
    __shared__ __align__(16) bf16 Bs[2][kBN][kBK + kPad];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = warp & 3, wn = warp >> 2;
    const int64_t m0 = (int64_t)blockIdx.x * kBM;
    const int n0 = blockIdx.y * kBN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;

    auto load_tile = [&](int stage, int k0) {
        // A: 128 rows x 32 cols = 512 chunks of 8 bf16
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int ch = tid + u * 256;
            const int row = ch >> 2, cc = (ch & 3) * 8;
            const int64_t gr = m0 + row;
            const bool ok = gr < M;
            cp_async16(&As[stage][row][cc], A + (ok ? gr : 0) * K + k0 + cc, ok);
        }
        {
            const int row = tid >> 2, cc = (tid & 3) * 8;
            const int gn = n0 + row;
            const bool ok = gn < N;
            cp_async16(&Bs[stage][row][cc], W + (int64_t)(ok ? gn : 0) * K + k0 + cc, ok);
        }
        cp_async_commit();
    };

    const int nk = K / kBK;
    load_tile(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        cp_async_wait_all();
        __syncthreads();
        if (kt + 1 < nk) load_tile(st ^ 1, (kt + 1) * kBK);
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            uint32_t af[2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int row = wm * 32 + i * 16 + (lane & 15);
                const int col = kk + (lane >> 4) * 8;
                ldmatrix_x4(af[i], &As[st][row][col]);
            }
            uint32_t bfr[4][2];
#pragma unroll
            for (int j2 = 0; j2 < 2; ++j2) {
                uint32_t r[4];
                const int row = wn * 32 + j2 * 16 + (lane & 7) + ((lane >> 4) << 3);
                const int col = kk + ((lane >> 3) & 1) * 8;
                ldmatrix_x4(r, &Bs[st][row][col]);
                bfr[2 * j2][0] = r[0]; bfr[2 * j2][1] = r[1];
                bfr[2 * j2 + 1][0] = r[2]; bfr[2 * j2 + 1][1] = r[3];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j][0], bfr[j][1]);
        }
        __syncthreads();
    }
    // epilogue
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = n0 + wn * 32 + j * 8 + 2 * t;
            if (col >= N) continue;
            float b0 = bias ? bias[col] : 0.0f, b1 = bias ? bias[col + 1] : 0.0f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t row = m0 + wm * 32 + i * 16 + g + h * 8;
                if (row >= M) continue;
                if (rowbias) {
                    const float* rb = rowbias + (int64_t)rows_per_bias.div((uint32_t)row) * N;
                    b0 = rb[col]; b1 = rb[col + 1];
                }
                float v0 = acc[i][j][2 * h] + b0, v1 = acc[i][j][2 * h + 1] + b1;
                if (RELU) { v0 = fmaxf(v0, 0.0f); v1 = fmaxf(v1, 0.0f); }
                if (OUT_BF16) {
                    *reinterpret_cast<__nv_bfloat162*>(static_cast<bf16*>(Cout) + row * N + col) =
                        __floats2bfloat162_rn(v0, v1);
                } else {
                    *reinterpret_cast<float2*>(static_cast<float*>(Cout) + row * N + col) = make_float2(v0, v1);
                }
            }
        }
}

cudaError_t launch_gemm_nt(const bf16* A, const bf16* W, const float* bias, void* C, int M, int N, int K, bool relu,
                           bool out_bf16, cudaStream_t s, const float* rowbias = nullptr, int rows_per_bias = 1) {
    if (M <= 0) return cudaSuccess;
    if (K % kBK || N % 2) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + kBN - 1) / kBN));
    const FastDiv rpb = FastDiv::make((uint32_t)rows_per_bias);
    if (relu && out_bf16) k_gemm_nt<true, true><<<grid, 256, 0, s>>>(A, W, bias, C, M, N, K, rowbias, rpb);
    else if (relu) k_gemm_nt<true, false><<<grid, 256, 0, s>>>(A, W, bias, C, M, N, K, rowbias, rpb);
    else if (out_bf16) k_gemm_nt<false, true><<<grid, 256, 0, s>>>(A, W, bias, C, M, N, K, rowbias, rpb);
    else k_gemm_nt<false, false><<<grid, 256, 0, s>>>(A, W, bias, C, M, N, K, rowbias, rpb);
    return cudaGetLastError();
}

// ============================================================================ MH step

__device__ __forceinline__ float site_u23(uint32_t index, uint32_t sweep, uint32_t c, uint32_t phase, uint2 key) {
    const uint32_t U = draw(index, sweep, c, phase, 0, key).x >> 9;
    return ((float)U + 0.5f) * (1.0f / 8388608.0f);
}

// One independence MH step per (block, chain) row r = b*C + c.
__global__ void k_learned_mh(const LearnedArgs a, SweepArgs s) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    const int C = s.C, L = s.L;
    if (r >= (uint64_t)a.nb * C) return;
    const uint32_t b = s.fdC.div(r), c = r - b * (uint32_t)C;
    const uint32_t sweep = (uint32_t)s.ctl->sweep;
    const uint8_t* xin = s.x + (size_t)(sweep & 1) * s.N * C;
    uint8_t* xout = s.x + (size_t)((sweep + 1) & 1) * s.N * C;
    const int n = a.nmem[b];
    const int* mem = a.members + b * kLearnBlock;
    const float* z = a.Z + (int64_t)r * a.O;
    uint8_t cur[kLearnBlock], prop[kLearnBlock];
    float lq_cur = 0.0f, lq_new = 0.0f, lp_cur = 0.0f, lp_new = 0.0f;
    bool near = false;
    for (int i = 0; i < n; ++i) {
        const int v = mem[i];
        const int xc = xin[(int64_t)v * C + c];
        cur[i] = (uint8_t)xc;
        float mx = -INFINITY;
        for (int q = 0; q < L; ++q) mx = fmaxf(mx, z[i * L + q]);
        float ssum = 0.0f;
        for (int q = 0; q < L; ++q) ssum += expf(z[i * L + q] - mx);
        const float lse = mx + logf(ssum);
        const float u = site_u23((uint32_t)v, sweep, c, PH_PROPOSAL, s.key);
        float cdf = 0.0f;
        int pick = -1, last_pos = 0;
        for (int q = 0; q < L; ++q) {
            const float p = expf(z[i * L + q] - lse);
            cdf += p;
            if (p > 0.0f) last_pos = q;
            if (pick < 0 && u < cdf) pick = q;
            near |= fabsf(u - cdf) < 1e-6f;
        }
        if (pick < 0) pick = last_pos;
        prop[i] = (uint8_t)pick;
        lq_cur += z[i * L + xc] - lse;
        lq_new += z[i * L + pick] - lse;
        const float* pv = s.pot + (int64_t)v * L * C + c;
        lp_cur += pv[(int64_t)xc * C];
        lp_new += pv[(int64_t)pick * C];
    }
    for (int64_t q = a.intra_ptr[b]; q < a.intra_ptr[b + 1]; ++q) {
        const int4 ie = a.intra[q];
        const float* ps = s.resid + (int64_t)ie.x * L * L;
        lp_cur += ps[cur[ie.y] * L + cur[ie.z]];
        lp_new += ps[prop[ie.y] * L + prop[ie.z]];
    }
    const float log_alpha = (lp_new - lp_cur) + (lq_cur - lq_new);
    const float ua = site_u23(b, sweep, c, PH_ACCEPT, s.key);
    const float alpha = expf(fminf(0.0f, log_alpha));
    const bool acc = ua < alpha;
    near |= fabsf(ua - alpha) < 1e-6f;
    if (near) atomicAdd(&s.ctl->boundary, 1ull);
    if (acc) atomicAdd(a.n_accepted, 1ull);
    for (int i = 0; i < n; ++i) xout[(int64_t)mem[i] * C + c] = acc ? prop[i] : cur[i];
}

// ============================================================================ training (float32 SIMT)

// C[i][j] = sum_k A(i,k) B(k,j) (+ bias[j]) (relu), A(i,k) = A[i*a0 + k*a1],
// B(k,j) = B[k*b0 + j*b1], C[i*ldc + j]; TA/TB are float or bf16.
template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_gemm_f32(int M, int N, int K, const TA* __restrict__ A, int64_t a0, int64_t a1,
                                                  const TB* __restrict__ B, int64_t b0, int64_t b1, float* __restrict__ Cm,
                                                  int64_t ldc, const float* __restrict__ bias, int relu) {
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int q = threadIdx.x; q < 16 * 64; q += 256) {
            const int kk = q >> 6, ii = q & 63;
            const int gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi < M && gk < K) ? (float)A[gi * a0 + gk * a1] : 0.0f;
            const int gj = j0 + ii;
            Bs[kk][ii] = (gj < N && gk < K) ? (float)B[gk * b0 + gj * b1] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { av[u] = As[kk][ty * 4 + u]; bv[u] = Bs[kk][tx * 4 + u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] = fmaf(av[u], bv[w], acc[u][w]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int gi = i0 + ty * 4 + u, gj = j0 + tx * 4 + w;
            if (gi < M && gj < N) {
                float v = acc[u][w] + (bias ? bias[gj] : 0.0f);
                if (relu) v = fmaxf(v, 0.0f);
                Cm[gi * ldc + gj] = v;
            }
        }
}

template <typename TA, typename TB>
static cudaError_t gemm_f32(int M, int N, int K, const TA* A, int64_t a0, int64_t a1, const TB* B, int64_t b0, int64_t b1,
                            float* Cm, int64_t ldc, const float* bias, bool relu, cudaStream_t s) {
    dim3 grid((unsigned)((M + 63) / 64), (unsigned)((N + 63) / 64));
    k_gemm_f32<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, a0, a1, B, b0, b1, Cm, ldc, bias, relu ? 1 : 0);
    return cudaGetLastError();
}

// dz = (softmax(z_i) - onehot(y_i)) [i < nmem] / R per row; loss accumulated (double).
__global__ void k_ce_grad(const float* __restrict__ z, const uint8_t* __restrict__ y, const uint8_t* __restrict__ nmem,
                          int R, int L, float* __restrict__ dz, double* loss) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int O = kLearnBlock * L;
    double l = 0.0;
    for (int i = 0; i < kLearnBlock; ++i) {
        const float* zi = z + (int64_t)r * O + i * L;
        float* di = dz + (int64_t)r * O + i * L;
        if (i >= nmem[r]) {
            for (int q = 0; q < L; ++q) di[q] = 0.0f;
            continue;
        }
        float mx = -INFINITY;
        for (int q = 0; q < L; ++q) mx = fmaxf(mx, zi[q]);
        float ssum = 0.0f;
        for (int q = 0; q < L; ++q) ssum += expf(zi[q] - mx);
        const float lse = mx + logf(ssum);
        const int yi = y[(int64_t)r * kLearnBlock + i];
        l -= (double)(zi[yi] - lse);
        for (int q = 0; q < L; ++q) di[q] = (expf(zi[q] - lse) - (q == yi ? 1.0f : 0.0f)) / (float)R;
    }
    atomicAdd(loss, l / R);
}

__global__ void k_relu_mask(float* __restrict__ d, const float* __restrict__ h, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && !(h[i] > 0.0f)) d[i] = 0.0f;
}

__global__ void k_colsum(const float* __restrict__ d, int R, int N, float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float s = 0.0f;
    for (int r = 0; r < R; ++r) s += d[(int64_t)r * N + j];
    out[j] = s;
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps); weight blocks also
// refresh their bf16 copy.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi; v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_to_bf16(const float* __restrict__ src, bf16* __restrict__ dst, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

// Rows r with r % stride == phase of the current features and labels go to the
// dataset at slot base + (r - phase) / stride (bounded by cap).
__global__ void k_learned_harvest(const LearnedArgs a, SweepArgs s, int stride, int phase, int64_t base, int64_t cap) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    const int C = s.C;
    if (r >= (uint64_t)a.nb * C || (int)(r % (uint32_t)stride) != phase) return;
    const int64_t slot = base + (r - phase) / stride;
    if (slot >= cap) return;
    const uint32_t b = s.fdC.div(r), c = r - b * (uint32_t)C;
    const uint8_t* xcur = s.x + (size_t)(((uint32_t)s.ctl->sweep) & 1) * s.N * C;
    // full feature row: per-chain part from X, the block's couplings, zero padding
    const int fx = kLearnBlock * a.L;
    for (int q = 0; q < a.Dp; ++q) {
        bf16 v = __float2bfloat16_rn(0.0f);
        if (q < fx) v = a.X[(int64_t)r * a.Kx + q];
        else if (q < fx + kLearnPairs) v = a.cfb[(int64_t)b * kLearnPairs + (q - fx)];
        a.ds_X[slot * a.Dp + q] = v;
    }
    const int n = a.nmem[b];
    for (int i = 0; i < kLearnBlock; ++i)
        a.ds_y[slot * kLearnBlock + i] = i < n ? xcur[(int64_t)a.members[b * kLearnBlock + i] * C + c] : 0;
    a.ds_n[slot] = (uint8_t)n;
}

__global__ void k_gather_rows(const int32_t* __restrict__ idx, int R, const LearnedArgs a, bf16* __restrict__ X,
                              uint8_t* __restrict__ y, uint8_t* __restrict__ nm) {
    const int r = blockIdx.x;
    if (r >= R) return;
    const int64_t src = idx[r];
    for (int q = threadIdx.x; q < a.Dp; q += blockDim.x) X[(int64_t)r * a.Dp + q] = a.ds_X[src * a.Dp + q];
    for (int i = threadIdx.x; i < kLearnBlock; i += blockDim.x) y[(int64_t)r * kLearnBlock + i] = a.ds_y[src * kLearnBlock + i];
    if (threadIdx.x == 0) nm[r] = a.ds_n[src];
}

// ============================================================================ launchers

cudaError_t launch_learned_features(const LearnedArgs& a, const SweepArgs& s, cudaStream_t st) {
    const int64_t n = (int64_t)a.nb * s.C;
    if (n > 0) k_learned_features<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(a, s.fdC, s.pot, s.C);
    return cudaGetLastError();
}

cudaError_t launch_learned_couplings(const LearnedArgs& a, const float* resid, float* cf, cudaStream_t st) {
    if (a.nb > 0) k_learned_couplings<<<(a.nb + 127) / 128, 128, 0, st>>>(a, resid, cf);
    return cudaGetLastError();
}

cudaError_t launch_learned_mlp(const LearnedArgs& a, int64_t rows, const bf16* X, cudaStream_t st) {
    cudaError_t e = launch_gemm_nt(X, a.W1b, a.b1, a.H1, (int)rows, a.H, a.Dp, true, true, st);
    if (e == cudaSuccess) e = launch_gemm_nt(a.H1, a.W2b, a.b2, a.H2, (int)rows, a.H, a.H, true, true, st);
    if (e == cudaSuccess) e = launch_gemm_nt(a.H2, a.W3b, a.b3, a.Zm, (int)rows, a.O, a.H, false, false, st);
    return e;
}

// Sweep path: layer 1 on the per-chain features only (K = Kx) with the
// per-block bias b1 + cf_b W1_cf^T, then layers 2 and 3.
cudaError_t launch_learned_mlp_blocks(const LearnedArgs& a, cudaStream_t st) {
    const int rows = a.nb * a.C;
    cudaError_t e = launch_gemm_nt(a.X, a.W1xb, nullptr, a.H1, rows, a.H, a.Kx, true, true, st, a.rowbias, a.C);
    if (e == cudaSuccess) e = launch_gemm_nt(a.H1, a.W2b, a.b2, a.H2, rows, a.H, a.H, true, true, st);
    if (e == cudaSuccess) e = launch_gemm_nt(a.H2, a.W3b, a.b3, a.Zm, rows, a.O, a.H, false, false, st);
    return e;
}

__global__ void k_copy_cols_bf16(const bf16* __restrict__ src, int64_t src_ld, int cols, bf16* __restrict__ dst,
                                 int dst_ld, int rows) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * dst_ld) return;
    const int64_t r = i / dst_ld;
    const int c = (int)(i % dst_ld);
    dst[i] = c < cols ? src[r * src_ld + c] : __float2bfloat16_rn(0.0f);
}

// rowbias[b][h] = b1[h] + sum_p bf16(cf[b][p]) W1b[h][16L + p]   (float32)
cudaError_t learned_rowbias(const LearnedArgs& a, cudaStream_t s) {
    cudaError_t e = gemm_f32(a.nb, a.H, kLearnPairs, (const bf16*)a.cfb, kLearnPairs, 1,
                             (const bf16*)(a.W1b + kLearnBlock * a.L), 1, a.Dp, a.rowbias, a.H, a.b1, false, s);
    return e;
}

cudaError_t launch_learned_mh(const LearnedArgs& a, const SweepArgs& s, cudaStream_t st) {
    const int64_t n = (int64_t)a.nb * s.C;
    if (n > 0) k_learned_mh<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(a, s);
    return cudaGetLastError();
}

cudaError_t launch_learned_harvest(const LearnedArgs& a, const SweepArgs& s, int stride, int phase, int64_t base,
                                   int64_t cap, cudaStream_t st) {
    const int64_t n = (int64_t)a.nb * s.C;
    if (n > 0) k_learned_harvest<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(a, s, stride, phase, base, cap);
    return cudaGetLastError();
}

// One training step (or a gradient evaluation when lr == 0 and grads are kept):
// forward in float32 on the bf16 weights, cross-entropy, backward into
// a.grad, then Adam (when step > 0).  Rows X/y/nm are already gathered.
cudaError_t learned_forward_backward(const LearnedArgs& a, int R, const bf16* X, const uint8_t* y, const uint8_t* nm,
                                     double* loss, cudaStream_t s) {
    const int Dp = a.Dp, H = a.H, O = a.O;
    float *h1 = a.t_h1, *h2 = a.t_h2, *zz = a.t_z, *dz = a.t_dz, *d2 = a.t_d2, *d1 = a.t_d1;
    float* g = a.grad;
    float* gW1 = g;                       float* gb1 = gW1 + (int64_t)H * Dp;
    float* gW2 = gb1 + H;                 float* gb2 = gW2 + (int64_t)H * H;
    float* gW3 = gb2 + H;                 float* gb3 = gW3 + (int64_t)O * H;
    cudaError_t e;
    // forward: h1 = relu(X W1^T + b1), h2 = relu(h1 W2^T + b2), z = h2 W3^T + b3
    if ((e = gemm_f32(R, H, Dp, X, Dp, 1, a.W1b, 1, Dp, h1, H, a.b1, true, s))) return e;
    if ((e = gemm_f32(R, H, H, (const float*)h1, H, 1, a.W2b, 1, H, h2, H, a.b2, true, s))) return e;
    if ((e = gemm_f32(R, O, H, (const float*)h2, H, 1, a.W3b, 1, H, zz, O, a.b3, false, s))) return e;
    if ((e = cudaMemsetAsync(loss, 0, sizeof(double), s))) return e;
    k_ce_grad<<<(R + 127) / 128, 128, 0, s>>>(zz, y, nm, R, a.L, dz, loss);
    // backward
    if ((e = gemm_f32(O, H, R, (const float*)dz, 1, O, (const float*)h2, H, 1, gW3, H, nullptr, false, s))) return e;
    k_colsum<<<(O + 127) / 128, 128, 0, s>>>(dz, R, O, gb3);
    if ((e = gemm_f32(R, H, O, (const float*)dz, O, 1, a.W3b, H, 1, d2, H, nullptr, false, s))) return e;
    k_relu_mask<<<(unsigned)(((int64_t)R * H + 255) / 256), 256, 0, s>>>(d2, h2, (int64_t)R * H);
    if ((e = gemm_f32(H, H, R, (const float*)d2, 1, H, (const float*)h1, H, 1, gW2, H, nullptr, false, s))) return e;
    k_colsum<<<(H + 127) / 128, 128, 0, s>>>(d2, R, H, gb2);
    if ((e = gemm_f32(R, H, H, (const float*)d2, H, 1, a.W2b, H, 1, d1, H, nullptr, false, s))) return e;
    k_relu_mask<<<(unsigned)(((int64_t)R * H + 255) / 256), 256, 0, s>>>(d1, h1, (int64_t)R * H);
    if ((e = gemm_f32(H, Dp, R, (const float*)d1, 1, H, X, Dp, 1, gW1, Dp, nullptr, false, s))) return e;
    k_colsum<<<(H + 127) / 128, 128, 0, s>>>(d1, R, H, gb1);
    return cudaGetLastError();
}

cudaError_t learned_adam(const LearnedArgs& a, int64_t n_params, float lr, int step, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_adam<<<(unsigned)((n_params + 255) / 256), 256, 0, s>>>(a.w32, a.grad, a.adam_m, a.adam_v, n_params, lr, b1, b2,
                                                               eps, c1, c2);
    return learned_sync_bf16(a, s);
}

// bf16 copies of the three weight matrices from the float32 master parameters.
cudaError_t learned_sync_bf16(const LearnedArgs& a, cudaStream_t s) {
    const int64_t n1 = (int64_t)a.H * a.Dp, n2 = (int64_t)a.H * a.H, n3 = (int64_t)a.O * a.H;
    const float* w1 = a.w32;
    const float* w2 = w1 + n1 + a.H;
    const float* w3 = w2 + n2 + a.H;
    k_to_bf16<<<(unsigned)((n1 + 255) / 256), 256, 0, s>>>(w1, a.W1b, n1);
    k_to_bf16<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(w2, a.W2b, n2);
    k_to_bf16<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(w3, a.W3b, n3);
    if (a.W1xb) {
        const int64_t nx = (int64_t)a.H * a.Kx;
        k_copy_cols_bf16<<<(unsigned)((nx + 255) / 256), 256, 0, s>>>(a.W1b, a.Dp, kLearnBlock * a.L, a.W1xb, a.Kx, a.H);
        if (a.wimg) {
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            return launch_mlp_images(a, s);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* src, bf16* dst, int64_t n, cudaStream_t s) {
    if (n > 0) k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t learned_gather(const LearnedArgs& a, const int32_t* idx, int R, bf16* X, uint8_t* y, uint8_t* nm,
                           cudaStream_t s) {
    if (R > 0) k_gather_rows<<<R, 128, 0, s>>>(idx, R, a, X, y, nm);
    return cudaGetLastError();
}

}  // namespace mrfk
