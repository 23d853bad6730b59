// Internal declarations shared by the CUDA translation units of libmrf.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/mrf.h"
#include "philox.cuh"

namespace mrfk {

constexpr int kMaxLabels = 16;

// Swendsen-Wang cluster log weights are summed in 64-bit fixed point with 32
// fraction bits, so that the sum is exact and independent of the order of the
// atomic adds (every run draws the same clusters' labels).  Terms are clamped
// to +-kSwFixMax; the sweep refuses a model whose summed term magnitudes could
// reach it, which keeps every partial sum far inside the int64 range.
constexpr double kSwFixScale = 4294967296.0;               // 2^32
constexpr double kSwFixMax = 1073741824.0;                 // 2^30
constexpr int64_t kSwNoLabel = (int64_t)(-0x7fffffffffffffffLL - 1);   // bonded: label excluded
// Swendsen-Wang ban word of a (site, chain): bits 0..15 labels the cluster
// may not take, kSwBonded = the site has a bond in this sweep, kSwRow = its
// weight row holds bond weights (it is the source of a bond).
constexpr uint32_t kSwLabelMask = 0xFFFFu;
constexpr uint32_t kSwRow = 1u << 30;
constexpr uint32_t kSwBonded = 1u << 31;
__host__ __device__ inline int64_t sw_fix(double x) {
    x = x > kSwFixMax ? kSwFixMax : (x < -kSwFixMax ? -kSwFixMax : x);
    return (int64_t)llrint(x * kSwFixScale);
}

// Control block in device memory, read by every sweep kernel so that a
// captured CUDA graph of one sweep can be replayed: the sweep index decides
// the RNG counter and which half of the label double buffer is current.
struct Ctl {
    unsigned long long sweep;          // index t of the sweep being run / next
    unsigned long long count_from;     // sweeps with t >= count_from are counted
    unsigned long long boundary;       // draws within 1e-6 of a decision boundary
    unsigned long long splash_offset;  // packed (ox | oy << 8 | oz << 16) of the last blocked sweep
};

// Division by a fixed 32-bit divisor d via a multiply (Granlund & Montgomery,
// "Division by invariant integers using multiplication", 1994):
// q = (umulhi(m, n) + n) >> l with l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1.
struct FastDiv {
    uint32_t d, m, l;
    static FastDiv make(uint32_t d) {
        if (d == 0) d = 1;
        uint32_t l = 0;
        while ((1ull << l) < d) ++l;
        const uint64_t m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
        return FastDiv{d, (uint32_t)m, l};
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const {
        return (uint32_t)(((uint64_t)__umulhi(m, n) + n) >> l);
    }
};

// Dualised-entry layout: entry k <-> table position (i_k, j_k).  Rows of the
// tau table are padded to MP = M rounded up to 4 floats (16-byte loads).
__host__ __device__ constexpr int pad4(int m) { return (m + 3) & ~3; }

// 32-bit words of threshold planes per edge (see k_build_planes): 20 per
// group of 32 entries, 12 for tables with at most 16 entries (two planes per word).
__host__ __device__ constexpr int plane_words(int m) { return m <= 16 ? 12 : 20 * ((m + 31) / 32); }

template <int L, int LAYOUT>
struct Ent {
    static constexpr int M = (LAYOUT == MRF_LAYOUT_PIVOT) ? (L - 1) * (L - 1) : L;
    static constexpr int MP = pad4(M);
    static constexpr int W = (M + 31) / 32;
    static constexpr int PW = plane_words(M);
    __host__ __device__ static constexpr int i(int k) { return LAYOUT == MRF_LAYOUT_PIVOT ? 1 + k / (L - 1) : k; }
    __host__ __device__ static constexpr int j(int k) { return LAYOUT == MRF_LAYOUT_PIVOT ? 1 + k % (L - 1) : k; }
};

__host__ __device__ inline int n_entries(int L, int layout) {
    return layout == MRF_LAYOUT_PIVOT ? (L - 1) * (L - 1) : L;
}

// Exact 24-bit threshold of a dual draw at logit level 0 (-tau, lev2 = 0) or
// level 2 (+tau, lev2 = 1) from the packed entry word; 0 for an entry without
// a dual bit.  (Level 1, logit 0, is T = 2^23 and never needs the low bits.)
__host__ __device__ __forceinline__ uint32_t level_threshold(uint32_t w, bool lev2) {
    const uint32_t tp = w & 0x1FFFFFFu;
    const uint32_t tm = (1u << 24) - tp + ((w >> 25) & 3u) - 1u;
    return w ? (lev2 ? tp : tm) : 0u;
}

// 8-bit prefix of a threshold (255 stands for T = 2^24, decided by the low bits).
__host__ __device__ __forceinline__ uint32_t threshold_prefix(uint32_t t) { return t >= (1u << 24) ? 255u : (t >> 16); }

// Everything a sweep kernel needs, passed by value.
struct SweepArgs {
    int32_t N, C, L, M, W;     // W = G = ceil(M/32) groups of 32 entries
    int64_t E;                 // edge slots
    const int32_t* src;        // [E] (-1 = free slot)
    const int32_t* dst;        // [E]
    const float* tau;          // [E][MP] signed dual weight (rows padded to 4)
    const uint32_t* thr;       // [E][M] packed thresholds
    const uint32_t* tpl;       // [E][plane_words(M)] threshold prefix planes (k_build_planes)
    const float* utf;          // [N][L] folded unaries, float32
    const float* resid;        // [E][L][L] exact tree-edge potentials (blocked sweep)
    const int64_t* inc_ptr;    // [N+1]
    int32_t max_deg;           // largest incidence count of a site (selects the primal kernels' one-batch form)
    const int2* inc;           // [2E] {edge*2 + side, neighbour}
    const double* ut;          // [N][L] folded unaries
    uint8_t* x;                // [2][N][C] label double buffer
    uint32_t* theta;           // [E][C][W]
    uint32_t* counts;          // [N][L]
    float* logp;               // [C][N][L] or null
    float* lpv;                // [N][C] log p of each drawn label (log-partition estimator) or null
    Ctl* ctl;
    uint2 key;
    RoundKeys rk;              // Philox round keys of `key`
    FastDiv fdC;               // division by the chain count
    int32_t grid_nx, grid_ny, grid_nz;
    // blocked sweep (lattice): tree edges of the sweep's comb forest get theta = 0
    int32_t splash;            // 1 while running a blocked sweep
    int64_t nxe, nye;          // numbers of x- and y-edges (canonical lattice order)
    FastDiv fdX1, fdX, fdY1, fdY;   // division by nx-1, nx, ny-1, ny
    float* pot;                // [N][L][C] node potentials / beliefs of the blocked sweep
    const uint8_t* skip;       // [E] 1 = edge kept exact (no dual bit) in a learned sweep; null otherwise
    float* part;               // [E][C][2][L] partial fields of the edge-partial plain sweep, or null
};

// One dualised entry of log-value l != 0 (Lemma 2-4 and Theorem 2 in closed
// form, float64): tau = 2 arccosh(e^{|l|/2}) = |l| + 2 log1p(sqrt(-expm1(-|l|))),
// the packed threshold word of its dual draw (T+ = ceil(sigmoid(tau) 2^24 - 1/2)
// in bits 0..24, d = T+ + T- - (2^24 - 1) in bits 25..26, the sign of l in bit
// 31), the signed tau, the Theorem-2 terms alpha1, alpha2 folded into the
// source and destination unaries, and -log(1 + e^q) for the log constant.
struct EntryDual {
    float tau_s;
    uint32_t word;
    double alpha1, alpha2, log_norm;
};
//
// With a = |l|, s = sqrt(1 - e^-a) and b = (1 + s)^2: tau = a + 2 log1p(s) and
// e^-tau = e^-a / b, so sigmoid(+tau) = b / (b + e^-a), sigmoid(-tau) = e^-a / (b + e^-a)
// and, for l > 0 (q = -tau), -log(1 + e^q) = -log1p(e^-a / b): four float64
// transcendentals per entry (expm1, exp, two log1p) and one division.
__host__ __device__ inline EntryDual entry_dual(double l) {
    const double al = fabs(l);
    const double s = sqrt(-expm1(-al));
    const double tau = al + 2.0 * log1p(s);
    const double ea = exp(-al), b = (1.0 + s) * (1.0 + s);
    const double inv = 1.0 / (b + ea);
    const double pp = b * inv;                   // sigmoid(+tau)
    const double pm = ea * inv;                  // sigmoid(-tau)
    const uint32_t tp = (uint32_t)ceil(pp * 16777216.0 - 0.5), tm = (uint32_t)ceil(pm * 16777216.0 - 0.5);
    const uint32_t d = tp + tm - ((1u << 24) - 1u);   // in {0,1,2}
    EntryDual r;
    r.word = tp | (d << 25) | (l < 0 ? 0x80000000u : 0u);
    r.tau_s = (float)(l > 0 ? tau : -tau);
    r.alpha1 = l > 0 ? 0.5 * (l - tau) : 0.5 * (l + tau);
    r.alpha2 = 0.5 * (l - tau);
    r.log_norm = l > 0 ? -log1p(ea / b) : -0.69314718055994530942;   // q = -tau, or q = 0: -log 2
    return r;
}

// Swendsen-Wang sweep (sw.cu): bonds, union-find and cluster labels.
struct SwArgs {
    int32_t N, C, L;
    int64_t E;                 // edge slots
    const int32_t* src;        // [E] (-1 = free slot)
    const int32_t* dst;        // [E]
    const uint32_t* thr;       // [E][L] 23-bit bond thresholds
    const int64_t* lwe;        // [E][L] fixed-point bond log weights (kSwNoLabel: label excluded)
    const int64_t* ufix;       // [N][L] fixed-point unaries (two labels: offsets folded in)
    const float* pot;          // [N][L][C] per-chain unaries instead of ufix (Higdon's sweep), or null
    uint8_t* x;                // [2][N][C] label double buffer
    int32_t* parent;           // [N][C] union-find forest, links to smaller sites only
    int32_t* root;             // [N][C] root of a bonded site (written by k_sw_flatten)
    uint32_t* bits;            // [ceil(E C / 32)] bond bitmap of the sweep, bit g of item g = e C + c
    uint32_t* ban;             // [N][C] labels a cluster may not take (bit per label)
    int64_t* lw;               // [N][L][C] fixed-point bond weights, then cluster weights at roots
    unsigned* err;             // set when a union-find walk exceeded its step bound
    float* lpv;                // [N][C] log p of each root's drawn label, 0 at other sites (estimator) or null
    uint32_t* counts;          // [N][L] marginal counts (k_sw_small accumulates them itself)
    Ctl* ctl;
    RoundKeys rk;
    FastDiv fdC;
};

// Learned block proposal (learned.cu).
constexpr int kLearnBlock = 16;                                   // sites per block (max)
constexpr int kLearnPairs = kLearnBlock * (kLearnBlock - 1) / 2;  // pair-coupling features

struct LearnedArgs {
    int32_t nb, L, Dp, H, O;            // blocks, labels, padded feature width, hidden, 16*L
    int32_t Kx, C;                      // width of the per-chain feature part (16 L padded to 32), chains
    const int32_t* members;             // [nb][16] site ids (sorted, -1 padding)
    const int32_t* nmem;                // [nb]
    const int64_t* intra_ptr;           // [nb+1]
    const int4* intra;                  // {edge slot, member index of src, of dst, 0}
    const float* cf;                    // [nb][120] pair couplings
    __nv_bfloat16* X;                   // [R][Dp] features, R = nb * C
    __nv_bfloat16* H1;                  // [R][H]
    __nv_bfloat16* H2;                  // [R][H]
    float* Zm;                          // [R][O] logits
    const float* Z;                     // = Zm
    float* w32;                         // flat float32 parameters W1,b1,W2,b2,W3,b3
    const float* b1; const float* b2; const float* b3;
    __nv_bfloat16* W1b; __nv_bfloat16* W2b; __nv_bfloat16* W3b;
    __nv_bfloat16* W1xb;                // [H][Kx] first 16 L columns of W1 (zero padded)
    __nv_bfloat16* cfb;                 // [nb][120] pair couplings rounded to bf16
    float* rowbias;                     // [nb][H] b1 + cf_b W1[:, 16L:16L+120]^T (per block)
    float* grad; float* adam_m; float* adam_v;
    float* t_h1; float* t_h2; float* t_z; float* t_dz; float* t_d2; float* t_d1;   // training scratch
    __nv_bfloat16* ds_X; uint8_t* ds_y; uint8_t* ds_n;                               // dataset
    unsigned long long* n_accepted;
    uint8_t* wimg;                      // swizzled bf16 images of W1x, W2, W3 for the tensor-core MLP
    unsigned* tc_err;                   // set by the tensor-core MLP when a wait timed out
    int32_t tc_inject_timeout;          // test hook: the next tensor-core MLP launch waits on a completion never signalled
};

// Kernel launchers (sweep.cu, splash.cu, decompose.cu).  All return cudaGetLastError().
cudaError_t launch_init_labels(const SweepArgs& a, cudaStream_t s);
cudaError_t launch_dual(const SweepArgs& a, int layout, cudaStream_t s);
cudaError_t launch_primal(const SweepArgs& a, int layout, int schedule, cudaStream_t s);
// Plain sweep in the edge-partial form (few chains, more than 16 entries per
// edge), after the dual step: step 0 the per-edge partial fields, step 1 the labels.
cudaError_t launch_sweep_partial(const SweepArgs& a, int layout, int step, cudaStream_t s);
constexpr int kPartialMaxChains = 4;
constexpr int kPartialMinEntries = 100;
cudaError_t launch_fused(const SweepArgs& a, int layout, int schedule, cudaStream_t s);
cudaError_t launch_accumulate(const SweepArgs& a, cudaStream_t s);
cudaError_t launch_philox_rate(uint64_t threads, int calls, uint32_t* sink, cudaStream_t s);
cudaError_t launch_log_v(const SweepArgs& a, const double* ut, double* out, cudaStream_t s);
cudaError_t launch_em(const SweepArgs& a, int layout, const uint8_t* xin, uint8_t* xout, cudaStream_t s);
int64_t sweep_small_smem(const SweepArgs& a);
cudaError_t launch_sweep_small(const SweepArgs& a, int layout, int n_sweeps, cudaStream_t s);
cudaError_t launch_mf(const SweepArgs& a, int layout, const float* qin, float* qout, cudaStream_t s);
cudaError_t launch_marg_layout(const float* in, float* out, int N, int L, int C, bool to_abi, cudaStream_t s);
// Tensor-core MLP (mlp_tc.cu)
bool mlp_tc_supported(const LearnedArgs& a);
int64_t mlp_tc_image_bytes(int H, int O, int Kx);
cudaError_t launch_mlp_images(const LearnedArgs& a, cudaStream_t s);
cudaError_t launch_learned_mlp_tc(const LearnedArgs& a, cudaStream_t s);
cudaError_t launch_advance(const SweepArgs& a, cudaStream_t s);
cudaError_t launch_splash(const SweepArgs& a, int layout, cudaStream_t s);
cudaError_t launch_splash_offset(const SweepArgs& a, cudaStream_t s, int64_t iter = -1);
cudaError_t launch_tree_map(const SweepArgs& a, uint8_t* xout, cudaStream_t s);
cudaError_t launch_tree_marginals(const SweepArgs& a, float* qout, cudaStream_t s);
cudaError_t launch_mf_pot(const SweepArgs& a, int layout, const float* qin, cudaStream_t s);
cudaError_t launch_em_pot(const SweepArgs& a, int layout, const uint8_t* xin, cudaStream_t s);
cudaError_t launch_potential(const SweepArgs& a, int layout, cudaStream_t s);
cudaError_t launch_ffbs(const SweepArgs& a, cudaStream_t s);
cudaError_t launch_max_degree(const int64_t* ptr, int N, unsigned* out, cudaStream_t s);
cudaError_t build_csr_device(const int32_t* src, const int32_t* dst, int64_t E, int N, int64_t* ptr, int2* inc,
                             int32_t* work, int64_t* sums, unsigned long long* too_long, int max_deg, cudaStream_t s);
cudaError_t launch_scatter_edges(const int64_t* slots, const int32_t* s, const int32_t* t, int64_t n, int32_t* src,
                                 int32_t* dst, cudaStream_t st);
cudaError_t launch_learned_features(const LearnedArgs& a, const SweepArgs& s, cudaStream_t st);
cudaError_t launch_learned_couplings(const LearnedArgs& a, const float* resid, float* cf, cudaStream_t st);
cudaError_t launch_learned_mlp(const LearnedArgs& a, int64_t rows, const __nv_bfloat16* X, cudaStream_t st);
cudaError_t launch_learned_mh(const LearnedArgs& a, const SweepArgs& s, cudaStream_t st);
cudaError_t launch_learned_harvest(const LearnedArgs& a, const SweepArgs& s, int stride, int phase, int64_t base,
                                   int64_t cap, cudaStream_t st);
cudaError_t learned_forward_backward(const LearnedArgs& a, int R, const __nv_bfloat16* X, const uint8_t* y,
                                     const uint8_t* nm, double* loss, cudaStream_t s);
cudaError_t learned_adam(const LearnedArgs& a, int64_t n_params, float lr, int step, cudaStream_t s);
cudaError_t learned_sync_bf16(const LearnedArgs& a, cudaStream_t s);
cudaError_t learned_rowbias(const LearnedArgs& a, cudaStream_t s);
cudaError_t launch_learned_mlp_blocks(const LearnedArgs& a, cudaStream_t st);
cudaError_t learned_gather(const LearnedArgs& a, const int32_t* idx, int R, __nv_bfloat16* X, uint8_t* y, uint8_t* nm,
                           cudaStream_t s);
cudaError_t launch_to_bf16(const float* src, __nv_bfloat16* dst, int64_t n, cudaStream_t s);
// Layout of the allocation-free sweep's scratch array (noalloc.cu): words
// [0, kNoallocCtlWords) hold its control block, the dual bits follow.
constexpr size_t kNoallocCtlWords = 64;
static_assert(sizeof(Ctl) <= kNoallocCtlWords * sizeof(uint32_t), "control block larger than its reserved words");
cudaError_t noalloc_scratch(uint32_t** out);
cudaError_t launch_sweep_noalloc(const SweepArgs& a, int layout, const uint8_t* xin, uint8_t* xout, uint32_t sweep,
                                 cudaStream_t s);
// Swendsen-Wang (sw.cu)
cudaError_t launch_sw_check(const int32_t* src, const float* tau, int64_t E, int M, const int64_t* lwe, int L,
                            const float* unary, const double* unary_d, int N, double* out, cudaStream_t s);
// Higdon's partial Swendsen-Wang (sw.cu)
struct HigdonTables {
    uint32_t* bond_thr;        // [E][L] 23-bit thresholds of rho (1 - e^{-l})
    int64_t* bond_lw;          // [E][L] fixed-point log alpha - alpha1 - alpha2 (kSwNoLabel where alpha = 0)
    float* tau;                // [E][pad4(L)] signed dual weights of the remainder A
    uint32_t* thr;             // [E][L] packed thresholds of A's bits
    double* fold;              // [E][2][L] A's Theorem-2 terms for the unaries
    double* bound;             // [E] max |bond weight| + 2 max tau of the edge (range check)
};
cudaError_t launch_hg_tables(const int32_t* src, const double* ell, int64_t E, int L, double rho, HigdonTables t,
                             cudaStream_t s);
cudaError_t launch_hg_check(const double* ut, int N, int L, const int32_t* src, const double* bound, int64_t E,
                            double* out, cudaStream_t s);
cudaError_t launch_hg_clear(const uint32_t* bits, uint32_t* theta, int64_t items, cudaStream_t s);
cudaError_t launch_sw_fix_unary(const float* unary, const double* unary_d, int64_t n, int64_t* ufix, cudaStream_t s);
cudaError_t launch_sw_reset(const SwArgs& a, cudaStream_t s);
cudaError_t launch_sw_bond(const SwArgs& a, cudaStream_t s);
cudaError_t launch_sw_flatten(const SwArgs& a, cudaStream_t s);
cudaError_t launch_sw_draw(const SwArgs& a, cudaStream_t s);
int64_t sw_small_smem(const SwArgs& a);
cudaError_t launch_sw_small(const SwArgs& a, int n_sweeps, cudaStream_t s);
int64_t hg_small_smem(const SwArgs& a);
cudaError_t launch_hg_small(const SweepArgs& d, const SwArgs& a, int n_sweeps, cudaStream_t s);
cudaError_t launch_labels_to_abi(const uint8_t* x, uint8_t* y, int N, int C, cudaStream_t s);
cudaError_t launch_labels_from_abi(const uint8_t* y, uint8_t* x, int N, int C, cudaStream_t s);
cudaError_t launch_count_ge(const uint8_t* y, int64_t n, int L, unsigned long long* bad, cudaStream_t s);

struct DecompArgs {
    int32_t L, M, layout;
    int64_t n;                 // edges to decompose
    const int64_t* slots;      // [n] slot of each edge (null: slot = first_slot + i)
    int64_t first_slot;
    const float* pair;         // [n][L][L] raw log tables
    float* tau;                // [E][MP]
    uint32_t* thr;             // [E][M]
    double* fold;              // [E][2][L]
    double* cst;               // [E] per-edge log constant
    float* resid;              // [E][L][L] or null
    uint32_t* sw_thr;          // [E][L] Swendsen-Wang bond thresholds (diagonal layout) or null
    int64_t* sw_lw;            // [E][L] Swendsen-Wang bond log weights, fixed point, or null
    double* sw_fold;           // [E][2][L] Swendsen-Wang unary offsets (two labels) or null
    double* sw_ell;            // [E][L] Swendsen-Wang couplings l_x (float64) or null
    // device edit queue (all null elsewhere): the edge count is min(n, *n_dev),
    // edge i's table starts at pair + pair_off[i], and nothing is written while
    // *status holds a bit of kQFatal
    const int64_t* n_dev;
    const int64_t* pair_off;
    const uint32_t* status;
};
cudaError_t launch_check_finite(const float* p, int64_t n, unsigned long long* bad, cudaStream_t s);
cudaError_t launch_count_offdiag(const float* pair, int64_t n_edges, int L, unsigned long long* nz, cudaStream_t s);
cudaError_t launch_decompose(const DecompArgs& a, cudaStream_t s);
cudaError_t launch_build_planes(const uint32_t* thr, int64_t n, const int64_t* slots, int64_t first_slot, int M,
                                uint32_t* tpl, cudaStream_t s, const int64_t* n_dev = nullptr,
                                const uint32_t* status = nullptr);
cudaError_t launch_fold_unary(const float* unary, const double* fold, const int64_t* inc_ptr, const int2* inc,
                              int N, int L, double* ut, float* utf, cudaStream_t s,
                              const double* unary_d = nullptr);

// Device edit queue of a batch (queue.cu).  Status bits of a round: the
// first ten cancel its edit, kQUnsorted reports a site whose incidence list
// was too long to sort on the device (its sums then run in another order).
enum : uint32_t {
    kQCount = MRF_Q_COUNT, kQGraph = MRF_Q_GRAPH, kQVertex = MRF_Q_VERTEX, kQLoop = MRF_Q_LOOP,
    kQSlot = MRF_Q_SLOT, kQDup = MRF_Q_DUP, kQFinite = MRF_Q_NONFINITE, kQDiag = MRF_Q_OFFDIAG,
    kQPair = MRF_Q_PAIR, kQSlots = MRF_Q_SLOTS, kQFatal = 1023u, kQUnsorted = MRF_Q_UNSORTED
};
// One label class as the queue kernels see it.
struct QClass {
    int32_t* src;              // [E_res] endpoints of the class's slots (-1: free)
    int32_t* dst;
    uint32_t* mark;            // [E_res] removal marks, zero between rounds
    uint8_t* touched;          // [N] sites whose folded unaries are stale
    int64_t E_res;             // slots the class holds (used, free and reserved)
    int32_t N, L, layout, pad;
    int64_t* rm;               // [cap_rm] removed slots of the round
    int64_t* add_slot;         // [cap_add] slot given to each added edge
    int64_t* add_idx;          // [cap_add] position of the addition in the queue
    int64_t* add_poff;         // [cap_add] offset of its table in the queue's table buffer
    int32_t* add_s;            // [cap_add] endpoints (class site ids)
    int32_t* add_t;
    int64_t* cnt;              // [3] removals and additions of the round, live edges
    int64_t* fsum;             // [ceil(E_res / 1024)] free slots per block of 1024 slots
};
struct QArgs {
    const int32_t* rm_graph;   // [cap_rm]
    const int64_t* rm_slot;    // [cap_rm] class slots
    const int32_t* add_graph;  // [cap_add]
    const int32_t* add_src;    // [cap_add] graph site ids
    const int32_t* add_dst;
    const float* pair;         // [cap_pair] the additions' tables, packed in queue order
    int64_t* counts;           // [3] removals, additions, table floats (zeroed after the edit)
    int64_t* out_slot;         // [cap_add] class slot of each added edge, -1 if the edit failed
    uint32_t* status;
    int64_t cap_rm, cap_add, cap_pair;
    int32_t G, K;
    const int32_t* g_cls;      // [G] class of each graph
    const int32_t* g_off;      // [G] first class site of each graph
    const int32_t* g_n;        // [G] sites of each graph
    const int32_t* g_L;        // [G] labels of each graph
    const QClass* cls;         // [K] in device memory
    int64_t* blk;              // [nblk][2K + 1] per-block counts of the routing
    int64_t nblk;              // ceil(max(cap_rm, cap_add) / 1024)
};
constexpr int kCsrSortLongSmem = 200 * 1024;
cudaError_t launch_queue_route(const QArgs& q, cudaStream_t s);
cudaError_t launch_queue_apply(const QArgs& q, const QClass& c, cudaStream_t s);
cudaError_t launch_queue_finish(const QArgs& q, cudaStream_t s);
cudaError_t launch_fold_touched(const float* unary, const double* fold, const int64_t* inc_ptr, const int2* inc,
                                int N, int L, uint8_t* touched, double* ut, float* utf, cudaStream_t s);
int csr_sort_long_cap();
cudaError_t init_csr_sort_long();
cudaError_t launch_csr_sort_long(const int64_t* ptr, int2* inc, int N, int min_deg, uint32_t* status, cudaStream_t s);

}  // namespace mrfk
