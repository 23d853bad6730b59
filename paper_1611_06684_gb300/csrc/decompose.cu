// Factor decomposition of Sections 4.1-4.2 on the device (setup and edits).
//
// For every edge e with log-table w (L x L, row = label of the source):
//  * PIVOT layout: l(i,j) = w(i,j) - w(i,0) - w(0,j) + w(0,0) for i, j >= 1;
//    offsets w(a,0) - w(0,0) fold into the source unary, w(0,b) - w(0,0) into
//    the destination unary, w(0,0) into the log constant.
//  * DIAG layout (Potts-type tables, Section 4.2): l(a,a) = w(a,a), no offsets.
// Every entry with l != 0 gets one dual bit (Section 4.2: none for 1-entries).
// Its one-hot 2x2 factor [[1,1],[1,e^l]] factors as in Lemmas 2-4 and Theorem 2;
// in closed form, with tau = 2 arccosh(e^{|l|/2}) evaluated stably as
// tau = |l| + 2 log1p(sqrt(-expm1(-|l|))):
//    l > 0:  q = -tau, beta1 = beta2 = tau, alpha1 = alpha2 = (l - tau)/2
//    l < 0:  q = 0, beta1 = -tau, beta2 = tau, alpha1 = (l + tau)/2, alpha2 = (l - tau)/2
// so the dual logit q + beta1 y + beta2 z takes one of {-tau, 0, +tau}.
//
// Stored per entry: tau_signed (= beta1; beta2 = |tau_signed|) as float, and a
// packed threshold word: T+ = ceil(sigmoid(tau) 2^24 - 1/2) in bits 0..24,
// d = T+ + T- - (2^24 - 1) in bits 25..26 (T- from sigmoid(-tau)), the sign of
// l in bit 31; 0 marks an entry without a dual bit.  A draw with 24-bit
// integer uniform U sets theta iff U < T for the case's threshold, which is
// exactly u = (U + 1/2) / 2^24 < p.  All of this runs in float64.
#include "common.cuh"

#include <cmath>

namespace mrfk {

__global__ void k_check_finite(const float* p, int64_t n, unsigned long long* bad) {
    unsigned long long cnt = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        cnt += !isfinite(p[i]);
    if (cnt) atomicAdd(bad, cnt);
}

__global__ void k_count_offdiag(const float* pair, int64_t n_edges, int L, unsigned long long* nz) {
    const int64_t n = n_edges * L * L;
    unsigned long long cnt = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)((i / L) % L), c = (int)(i % L);
        cnt += (r != c) && (pair[i] != 0.0f);
    }
    if (cnt) atomicAdd(nz, cnt);
}

__global__ void k_decompose(DecompArgs a) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n || (a.n_dev && i >= *a.n_dev) || (a.status && (*a.status & kQFatal))) return;
    const int L = a.L, M = a.M;
    const int64_t e = a.slots ? a.slots[i] : a.first_slot + i;
    const float* w = a.pair + (a.pair_off ? a.pair_off[i] : i * L * L);
    double fs[kMaxLabels], ft[kMaxLabels];
    double cst = 0.0;
    if (a.layout == MRF_LAYOUT_PIVOT) {
        const double w00 = w[0];
        for (int x = 0; x < L; ++x) {
            fs[x] = (double)w[x * L] - w00;
            ft[x] = (double)w[x] - w00;
        }
        cst = w00;
    } else {
        for (int x = 0; x < L; ++x) fs[x] = ft[x] = 0.0;
    }
    for (int k = 0; k < M; ++k) {
        int ii, jj;
        double l;
        if (a.layout == MRF_LAYOUT_PIVOT) {
            ii = 1 + k / (L - 1); jj = 1 + k % (L - 1);
            l = (double)w[ii * L + jj] - (double)w[ii * L] - (double)w[jj] + (double)w[0];
        } else {
            ii = jj = k;
            l = (double)w[k * L + k];
        }
        float tau_s = 0.0f;
        uint32_t word = 0;
        if (l != 0.0) {
            const EntryDual d = entry_dual(l);
            word = d.word;
            tau_s = d.tau_s;
            fs[ii] += d.alpha1;
            ft[jj] += d.alpha2;
            cst += d.log_norm;   // -log(1 + e^q)
        }
        a.tau[e * pad4(M) + k] = tau_s;
        a.thr[e * M + k] = word;
    }
    for (int k = M; k < pad4(M); ++k) a.tau[e * pad4(M) + k] = 0.0f;
    for (int x = 0; x < L; ++x) {
        a.fold[(e * 2 + 0) * L + x] = fs[x];
        a.fold[(e * 2 + 1) * L + x] = ft[x];
    }
    a.cst[e] = cst;
    if (a.sw_thr && (a.layout == MRF_LAYOUT_DIAG || L == 2)) {
        // Swendsen-Wang tables (Section 4.3): the table as
        // c + f(a) + g(b) + l_a [a = b] -- diagonal tables: l_x = w(x,x), f = g = 0;
        // two labels: l = (w00 + w11 - w01 - w10) / 2 for both labels,
        // f(1) = w10 - w00 + l, g(1) = w01 - w00 + l (folded into the SW unaries).
        // Per label x: bond probability 1 - e^{-l_x} as the exact 23-bit threshold
        // T = ceil(p 2^23 - 1/2) (a draw U bonds iff U < T, i.e. (U + 1/2) / 2^23 < p),
        // and the bond's label weight log(e^{l_x} - 1) in fixed point (sw_fix);
        // l <= 0: no bond (T = 0) and the label is excluded when bonded (kSwNoLabel).
        double lx[kMaxLabels];
        if (L == 2) {
            const double k2 = 0.5 * ((double)w[0] + (double)w[3] - (double)w[1] - (double)w[2]);
            lx[0] = lx[1] = k2;
            if (a.sw_fold) {
                a.sw_fold[(e * 2 + 0) * 2 + 0] = 0.0;
                a.sw_fold[(e * 2 + 0) * 2 + 1] = (double)w[2] - (double)w[0] + k2;
                a.sw_fold[(e * 2 + 1) * 2 + 0] = 0.0;
                a.sw_fold[(e * 2 + 1) * 2 + 1] = (double)w[1] - (double)w[0] + k2;
            }
        } else {
            for (int x = 0; x < L; ++x) lx[x] = (double)w[x * L + x];
        }
        for (int x = 0; x < L; ++x) {
            const double l = lx[x];
            uint32_t T = 0;
            int64_t lw = kSwNoLabel;
            if (l > 0.0) {
                T = (uint32_t)ceil(-expm1(-l) * 8388608.0 - 0.5);
                lw = sw_fix(log(expm1(l)));
            }
            a.sw_thr[e * L + x] = T;
            a.sw_lw[e * L + x] = lw;
            if (a.sw_ell) a.sw_ell[e * L + x] = l;
        }
    }
    if (a.resid) {
        // exact pairwise potential in the folded representation (tree edges of
        // the blocked sweep): w(a,b) - fold_s(a) - fold_t(b)
        for (int x = 0; x < L; ++x)
            for (int y = 0; y < L; ++y)
                a.resid[(e * L + x) * L + y] = (float)((double)w[x * L + y] - fs[x] - ft[y]);
    }
}

// Threshold prefix planes of the bit-sliced dual draw, per edge and group of
// 32 entries (entry 32g + b at bit b).  An entry's dual logit is at one of
// three levels: 0 (-tau, threshold T-), 1 (logit 0, T = 2^23) or 2 (+tau, T+);
// which one depends on its sign and its case (see dual_prefix_bits).  Stored:
// the 8 bit planes of the 8-bit prefix of T+ (B_p: bit 7 - p of the prefix),
// the planes of the difference between the prefixes of T- and T+
// (AB_p = A_p ^ B_p, A_p the planes of T-'s prefix), the sign mask and the mask
// of entries with a dual bit:
//   uint4 {AB_p, B_p, AB_p+1, B_p+1} for p = 0, 2, 4, 6,   uint4 {S, Act, 0, 0}
// 20 words per group.  A chain whose level-0 entries are L0 reads its
// threshold plane as B_p ^ (AB_p & L0).  Tables with at most 16 entries pack
// two planes per word (plane p in bits 0..15, plane p + 4 in bits 16..31), 12
// words per edge:
//   uint4 {AB_0|AB_4<<16, .., AB_3|AB_7<<16}, uint4 {B likewise}, uint4 {S | Act << 16, 0, 0, 0}.
__global__ void k_build_planes(const uint32_t* thr, int64_t n, const int64_t* slots, int64_t first_slot, int M,
                               uint32_t* tpl, const int64_t* n_dev, const uint32_t* status) {
    const int G = (M + 31) / 32;
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= n * G) return;
    const int64_t i = gid / G;
    if ((n_dev && i >= *n_dev) || (status && (*status & kQFatal))) return;
    const int g = (int)(gid % G);
    const int64_t e = slots ? slots[i] : first_slot + i;
    uint32_t A[8] = {0, 0, 0, 0, 0, 0, 0, 0}, B[8] = {0, 0, 0, 0, 0, 0, 0, 0}, S = 0, Act = 0;
    for (int b = 0; b < 32; ++b) {
        const int k = 32 * g + b;
        if (k >= M) break;
        const uint32_t w = thr[e * M + k];
        const uint32_t pa = threshold_prefix(level_threshold(w, false));
        const uint32_t pb = threshold_prefix(level_threshold(w, true));
        for (int p = 0; p < 8; ++p) {
            A[p] |= ((pa >> (7 - p)) & 1u) << b;
            B[p] |= ((pb >> (7 - p)) & 1u) << b;
        }
        S |= (w >> 31) << b;
        Act |= (w != 0u ? 1u : 0u) << b;
    }
    uint4* out = reinterpret_cast<uint4*>(tpl + e * (int64_t)plane_words(M) + 20 * g);
    for (int p = 0; p < 8; ++p) A[p] ^= B[p];
    if (M <= 16) {
        out[0] = make_uint4(A[0] | A[4] << 16, A[1] | A[5] << 16, A[2] | A[6] << 16, A[3] | A[7] << 16);
        out[1] = make_uint4(B[0] | B[4] << 16, B[1] | B[5] << 16, B[2] | B[6] << 16, B[3] | B[7] << 16);
        out[2] = make_uint4(S | Act << 16, 0u, 0u, 0u);
        return;
    }
    for (int p = 0; p < 8; p += 2) out[p / 2] = make_uint4(A[p], B[p], A[p + 1], B[p + 1]);
    out[4] = make_uint4(S, Act, 0u, 0u);
}

__global__ void k_fold_unary(const float* unary, const double* unary_d, const double* fold, const int64_t* inc_ptr,
                             const int2* inc, int N, int L, double* ut, float* utf) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    double acc[kMaxLabels];
    for (int x = 0; x < L; ++x) acc[x] = unary_d ? unary_d[(int64_t)v * L + x] : (double)unary[(int64_t)v * L + x];
    for (int64_t p = inc_ptr[v]; p < inc_ptr[v + 1]; ++p) {
        const int code = inc[p].x;
        const int64_t e = code >> 1;
        const double* f = fold + (e * 2 + (code & 1)) * L;
        for (int x = 0; x < L; ++x) acc[x] += f[x];
    }
    for (int x = 0; x < L; ++x) {
        ut[(int64_t)v * L + x] = acc[x];
        if (utf) utf[(int64_t)v * L + x] = (float)acc[x];
    }
}

cudaError_t launch_check_finite(const float* p, int64_t n, unsigned long long* bad, cudaStream_t s) {
    if (n > 0) k_check_finite<<<1216, 256, 0, s>>>(p, n, bad);
    return cudaGetLastError();
}

cudaError_t launch_count_offdiag(const float* pair, int64_t n_edges, int L, unsigned long long* nz, cudaStream_t s) {
    if (n_edges > 0) k_count_offdiag<<<1216, 256, 0, s>>>(pair, n_edges, L, nz);
    return cudaGetLastError();
}

cudaError_t launch_decompose(const DecompArgs& a, cudaStream_t s) {
    if (a.n > 0) k_decompose<<<(unsigned)((a.n + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fold_unary(const float* unary, const double* fold, const int64_t* inc_ptr, const int2* inc,
                              int N, int L, double* ut, float* utf, cudaStream_t s, const double* unary_d) {
    if (N > 0) k_fold_unary<<<(N + 127) / 128, 128, 0, s>>>(unary, unary_d, fold, inc_ptr, inc, N, L, ut, utf);
    return cudaGetLastError();
}

cudaError_t launch_build_planes(const uint32_t* thr, int64_t n, const int64_t* slots, int64_t first_slot, int M,
                                uint32_t* tpl, cudaStream_t s, const int64_t* n_dev, const uint32_t* status) {
    const int64_t work = n * ((M + 31) / 32);
    if (work > 0)
        k_build_planes<<<(unsigned)((work + 127) / 128), 128, 0, s>>>(thr, n, slots, first_slot, M, tpl, n_dev, status);
    return cudaGetLastError();
}

}  // namespace mrfk
