// Device edit queue of a batch: a round of factor insertions and deletions
// (the dynamic networks of the abstract and Section 6) applied by kernels
// alone, so that {edit, sweeps} replays as one captured CUDA graph.
//
// The queue holds up to cap_rm removals (graph, slot) and cap_add additions
// (graph, src, dst, L_g x L_g log table, tables packed in queue order); the
// counts live in device memory and are read by every kernel, whose grids are
// sized by the capacities.  A round:
//   route    per block of 1024 queue items, the count of removals and
//            additions of every label class and the table floats; one CTA
//            scans the block counts; a stable route of every item to its
//            class's lists (warp match + block offsets) with all checks
//            (graph and vertex ids, self-loops, live and distinct removed
//            slots, finite tables, diagonal tables in a diagonal-layout
//            class, free slots); removal marks are cleared.
//   apply    per class, unless a check failed: removed slots freed; added
//            edge j takes the j-th free slot in increasing slot order (the
//            host edit's rule: freed slots first, then fresh ones, since the
//            reserved fresh slots lie above every used one); endpoints
//            placed, decomposition and bit planes of the new slots, incidence
//            lists rebuilt, folded unaries of the touched sites recomputed.
// A failed check cancels the whole edit (nothing is written, the added
// edges' output slots are -1) and leaves its bits in the status word; the
// sweeps of the round still run on the unchanged model.
#include "common.cuh"

#include <algorithm>

namespace mrfk {

namespace {

constexpr int QB = 1024;                    // queue items per routing block
constexpr uint32_t FULL = 0xFFFFFFFFu;

__device__ __forceinline__ bool q_counts_ok(const QArgs& q, int64_t& n_rm, int64_t& n_add) {
    n_rm = q.counts[0];
    n_add = q.counts[1];
    return n_rm >= 0 && n_rm <= q.cap_rm && n_add >= 0 && n_add <= q.cap_add;
}

// Exclusive prefix over the 1024 threads of a CTA (every thread calls it).
__device__ int64_t cta_exclusive_1024(int64_t v, int64_t* s_warp, int64_t& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += y;
    }
    __syncthreads();
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = s_warp[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, t, d);
            if (lane >= d) t += y;
        }
        s_warp[lane] = t;
    }
    __syncthreads();
    total = s_warp[31];
    return x - v + (w > 0 ? s_warp[w - 1] : 0);
}

// In-place exclusive scan of n values a[0], a[stride], ... by one CTA of 1024
// threads, each summing a contiguous chunk; returns the total to every thread.
__device__ int64_t cta_scan_strided(int64_t* a, int64_t n, int64_t stride, int64_t* s_warp) {
    const int64_t chunk = (n + QB - 1) / QB;
    const int64_t b0 = threadIdx.x * chunk, b1 = b0 + chunk < n ? b0 + chunk : n;
    int64_t sum = 0;
    for (int64_t b = b0; b < b1; ++b) sum += a[b * stride];
    int64_t total = 0;
    int64_t run = cta_exclusive_1024(sum, s_warp, total);
    for (int64_t b = b0; b < b1; ++b) {
        const int64_t t = a[b * stride];
        a[b * stride] = run;
        run += t;
    }
    return total;
}

__global__ void __launch_bounds__(QB) k_q_count(QArgs q) {
    __shared__ unsigned long long s_c[2 * kMaxLabels + 1];
    const int K = q.K, cols = 2 * K + 1;
    if (threadIdx.x < cols) s_c[threadIdx.x] = 0ull;
    __syncthreads();
    int64_t n_rm, n_add;
    const int64_t i = blockIdx.x * (int64_t)QB + threadIdx.x;
    if (q_counts_ok(q, n_rm, n_add)) {
        if (i < n_rm) {
            const int g = q.rm_graph[i];
            if (g >= 0 && g < q.G) atomicAdd(&s_c[q.g_cls[g]], 1ull);
        }
        if (i < n_add) {
            const int g = q.add_graph[i];
            if (g >= 0 && g < q.G) {
                atomicAdd(&s_c[K + q.g_cls[g]], 1ull);
                atomicAdd(&s_c[2 * K], (unsigned long long)(q.g_L[g] * q.g_L[g]));
            }
        }
    } else if (i == 0) {
        atomicOr(q.status, kQCount);
    }
    __syncthreads();
    if (threadIdx.x < cols) q.blk[blockIdx.x * cols + threadIdx.x] = (int64_t)s_c[threadIdx.x];
}

// One CTA: block offsets of every column, class totals, capacity checks.
__global__ void __launch_bounds__(QB) k_q_scan(QArgs q) {
    __shared__ int64_t s_warp[32];
    __shared__ int64_t s_tot[2 * kMaxLabels + 1];
    const int K = q.K, cols = 2 * K + 1;
    for (int c = 0; c < cols; ++c) {
        const int64_t t = cta_scan_strided(q.blk + c, q.nblk, cols, s_warp);
        if (threadIdx.x == 0) s_tot[c] = t;
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    int64_t n_rm, n_add;
    const bool ok = q_counts_ok(q, n_rm, n_add);
    uint32_t bad = 0;
    if (ok && (s_tot[2 * K] != q.counts[2] || s_tot[2 * K] > q.cap_pair)) bad |= kQPair;
    for (int k = 0; k < K; ++k) {
        const QClass& c = q.cls[k];
        const int64_t r = ok ? s_tot[k] : 0, a = ok ? s_tot[K + k] : 0;
        c.cnt[0] = r;
        c.cnt[1] = a;
        if (c.E_res - c.cnt[2] + r < a) bad |= kQSlots;
    }
    if (bad) atomicOr(q.status, bad);
}

__global__ void __launch_bounds__(QB) k_q_route(QArgs q) {
    __shared__ int s_wc[32][2 * kMaxLabels];        // per-warp counts, then offsets, of each class column
    __shared__ int64_t s_l2[32];                    // per-warp table floats, then offsets
    int64_t n_rm, n_add;
    if (!q_counts_ok(q, n_rm, n_add)) return;       // block-uniform
    const int K = q.K, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t below = (1u << lane) - 1u;
    const int64_t i = blockIdx.x * (int64_t)QB + threadIdx.x;
    int kr = -1, ka = -1, ga = -1;
    if (i < n_rm) {
        const int g = q.rm_graph[i];
        if (g >= 0 && g < q.G) kr = q.g_cls[g];
        else atomicOr(q.status, kQGraph);
    }
    int64_t l2 = 0;
    if (i < n_add) {
        ga = q.add_graph[i];
        if (ga >= 0 && ga < q.G) { ka = q.g_cls[ga]; l2 = (int64_t)q.g_L[ga] * q.g_L[ga]; }
        else atomicOr(q.status, kQGraph);
    }
    for (int t = threadIdx.x; t < 32 * 2 * kMaxLabels; t += QB) (&s_wc[0][0])[t] = 0;
    __syncthreads();
    const unsigned mr = __match_any_sync(FULL, kr), ma = __match_any_sync(FULL, ka);
    const int rank_r = __popc(mr & below), rank_a = __popc(ma & below);
    if (kr >= 0 && rank_r == 0) s_wc[warp][kr] = __popc(mr);
    if (ka >= 0 && rank_a == 0) s_wc[warp][K + ka] = __popc(ma);
    int64_t x = l2;                                 // inclusive warp prefix of the table floats
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_l2[warp] = x;
    __syncthreads();
    if (threadIdx.x < 2 * K) {
        int run = 0;
        for (int w = 0; w < 32; ++w) { const int c = s_wc[w][threadIdx.x]; s_wc[w][threadIdx.x] = run; run += c; }
    } else if (threadIdx.x == QB - 1) {
        int64_t run = 0;
        for (int w = 0; w < 32; ++w) { const int64_t c = s_l2[w]; s_l2[w] = run; run += c; }
    }
    __syncthreads();
    const int64_t* bo = q.blk + blockIdx.x * (int64_t)(2 * K + 1);
    if (kr >= 0) {
        const QClass& c = q.cls[kr];
        const int64_t pos = bo[kr] + s_wc[warp][kr] + rank_r;
        const int64_t slot = q.rm_slot[i];
        if (slot < 0 || slot >= c.E_res || c.src[slot] < 0) atomicOr(q.status, kQSlot);
        else if (atomicAdd(&c.mark[slot], 1u) != 0u) atomicOr(q.status, kQDup);
        c.rm[pos] = slot;
    }
    if (ka >= 0) {
        const QClass& c = q.cls[ka];
        const int64_t pos = bo[K + ka] + s_wc[warp][K + ka] + rank_a;
        const int64_t poff = bo[2 * K] + s_l2[warp] + (x - l2);
        const int L = q.g_L[ga], n = q.g_n[ga], off = q.g_off[ga];
        const int s = q.add_src[i], t = q.add_dst[i];
        uint32_t bad = 0;
        if (s < 0 || s >= n || t < 0 || t >= n) bad |= kQVertex;
        else if (s == t) bad |= kQLoop;
        if (poff + (int64_t)L * L > q.cap_pair) {
            bad |= kQPair;
        } else {
            const float* w = q.pair + poff;
            for (int e = 0; e < L * L; ++e) {
                const float v = w[e];
                if (!isfinite(v)) bad |= kQFinite;
                else if (c.layout == MRF_LAYOUT_DIAG && e / L != e % L && v != 0.0f) bad |= kQDiag;
            }
        }
        if (bad) atomicOr(q.status, bad);
        c.add_s[pos] = s + off;
        c.add_t[pos] = t + off;
        c.add_idx[pos] = i;
        c.add_poff[pos] = poff;
    }
}

// Clear the removal marks; on a failed check, every added edge's slot is -1.
__global__ void __launch_bounds__(QB) k_q_unmark(QArgs q) {
    int64_t n_rm, n_add;
    if (!q_counts_ok(q, n_rm, n_add)) return;
    const int64_t i = blockIdx.x * (int64_t)QB + threadIdx.x;
    if (i < n_rm) {
        const int g = q.rm_graph[i];
        if (g >= 0 && g < q.G) {
            const QClass& c = q.cls[q.g_cls[g]];
            const int64_t slot = q.rm_slot[i];
            if (slot >= 0 && slot < c.E_res) c.mark[slot] = 0u;
        }
    }
    if (i < n_add && (*q.status & kQFatal)) q.out_slot[i] = -1;
}

__global__ void k_q_remove(QClass c, int64_t cap, const uint32_t* status) {
    if (*status & kQFatal) return;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= cap || j >= c.cnt[0]) return;
    const int64_t slot = c.rm[j];
    c.touched[c.src[slot]] = 1;
    c.touched[c.dst[slot]] = 1;
    c.src[slot] = -1;
    c.dst[slot] = -1;
}

// Free slots per block of 1024 slots (after the removals).
__global__ void __launch_bounds__(QB) k_q_free_count(QClass c, const uint32_t* status) {
    if ((*status & kQFatal) || c.cnt[1] == 0) return;
    const int64_t e = blockIdx.x * (int64_t)QB + threadIdx.x;
    const int n = __syncthreads_count(e < c.E_res && c.src[e] < 0);
    if (threadIdx.x == 0) c.fsum[blockIdx.x] = n;
}

__global__ void __launch_bounds__(QB) k_q_free_scan(QClass c, int64_t nb, const uint32_t* status) {
    __shared__ int64_t s_warp[32];
    if ((*status & kQFatal) || c.cnt[1] == 0) return;
    cta_scan_strided(c.fsum, nb, 1, s_warp);
}

// Added edge j takes the j-th free slot in increasing slot order.
__global__ void __launch_bounds__(QB) k_q_assign(QClass c, const uint32_t* status) {
    __shared__ int s_w[32];
    const int64_t n_add = c.cnt[1];
    if ((*status & kQFatal) || n_add == 0) return;
    const int64_t base = c.fsum[blockIdx.x];
    if (base >= n_add) return;                      // block-uniform
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t e = blockIdx.x * (int64_t)QB + threadIdx.x;
    const bool fr = e < c.E_res && c.src[e] < 0;
    const unsigned bal = __ballot_sync(FULL, fr);
    if (lane == 0) s_w[warp] = __popc(bal);
    __syncthreads();
    int off = 0;
    for (int w = 0; w < warp; ++w) off += s_w[w];
    const int64_t rank = base + off + __popc(bal & ((1u << lane) - 1u));
    if (fr && rank < n_add) c.add_slot[rank] = e;
}

__global__ void k_q_place(QClass c, int64_t cap, int64_t* out_slot, uint32_t* status_w) {
    if (*status_w & kQFatal) return;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n_add = c.cnt[1];
    if (j == 0) c.cnt[2] += n_add - c.cnt[0];
    if (j >= cap || j >= n_add) return;
    const int64_t slot = c.add_slot[j];
    if (slot < 0 || slot >= c.E_res) {             // not assigned: cannot happen while the live count is exact
        atomicOr(status_w, kQSlots);
        return;
    }
    const int s = c.add_s[j], t = c.add_t[j];
    c.src[slot] = s;
    c.dst[slot] = t;
    c.touched[s] = 1;
    c.touched[t] = 1;
    out_slot[c.add_idx[j]] = slot;
}

// Folded unaries (Sections 4.1-4.2 offsets of every incident edge) of the
// sites an edit touched, in incidence order as in the full fold.
__global__ void k_fold_touched(const float* unary, const double* fold, const int64_t* inc_ptr, const int2* inc,
                               int N, int L, uint8_t* touched, double* ut, float* utf) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N || !touched[v]) return;
    touched[v] = 0;
    double acc[kMaxLabels];
    for (int x = 0; x < L; ++x) acc[x] = (double)unary[(int64_t)v * L + x];
    for (int64_t p = inc_ptr[v]; p < inc_ptr[v + 1]; ++p) {
        const int code = inc[p].x;
        const double* f = fold + ((int64_t)(code >> 1) * 2 + (code & 1)) * L;
        for (int x = 0; x < L; ++x) acc[x] += f[x];
    }
    for (int x = 0; x < L; ++x) {
        ut[(int64_t)v * L + x] = acc[x];
        utf[(int64_t)v * L + x] = (float)acc[x];
    }
}

__global__ void k_q_finish(QArgs q) {
    if (threadIdx.x < 3) q.counts[threadIdx.x] = 0;
}

// Sites with more than min_deg incidences (left unsorted by k_csr_sort): one
// CTA per site sorts the list by code, each incidence's position being the
// number of smaller codes (codes are distinct), from a copy in shared memory.
__global__ void __launch_bounds__(256) k_csr_sort_long(const int64_t* __restrict__ ptr, int2* __restrict__ inc, int N,
                                                       int min_deg, int cap, uint32_t* status) {
    extern __shared__ int2 s_inc[];
    __shared__ int s_list[256];
    __shared__ int s_n;
    for (int64_t v0 = (int64_t)blockIdx.x * 256; v0 < N; v0 += (int64_t)gridDim.x * 256) {
        if (threadIdx.x == 0) s_n = 0;
        __syncthreads();
        const int64_t v = v0 + threadIdx.x;
        if (v < N && ptr[v + 1] - ptr[v] > min_deg) s_list[atomicAdd(&s_n, 1)] = (int)v;
        __syncthreads();
        const int n = s_n;
        for (int l = 0; l < n; ++l) {
            const int u = s_list[l];
            const int64_t p0 = ptr[u];
            const int d = (int)(ptr[u + 1] - p0);
            if (d > cap) {
                if (threadIdx.x == 0) atomicOr(status, kQUnsorted);
                continue;
            }
            for (int i = threadIdx.x; i < d; i += 256) s_inc[i] = inc[p0 + i];
            __syncthreads();
            for (int i = threadIdx.x; i < d; i += 256) {
                const int key = s_inc[i].x;
                int r = 0;
                for (int j = 0; j < d; ++j) r += s_inc[j].x < key;
                inc[p0 + r] = s_inc[i];
            }
            __syncthreads();
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_queue_route(const QArgs& q, cudaStream_t s) {
    const unsigned nb = (unsigned)q.nblk;
    k_q_count<<<nb, QB, 0, s>>>(q);
    k_q_scan<<<1, QB, 0, s>>>(q);
    k_q_route<<<nb, QB, 0, s>>>(q);
    k_q_unmark<<<nb, QB, 0, s>>>(q);
    return cudaGetLastError();
}

cudaError_t launch_queue_apply(const QArgs& q, const QClass& c, cudaStream_t s) {
    if (q.cap_rm > 0) k_q_remove<<<(unsigned)((q.cap_rm + 255) / 256), 256, 0, s>>>(c, q.cap_rm, q.status);
    const int64_t nb = (c.E_res + QB - 1) / QB;
    if (nb > 0 && q.cap_add > 0) {
        k_q_free_count<<<(unsigned)nb, QB, 0, s>>>(c, q.status);
        k_q_free_scan<<<1, QB, 0, s>>>(c, nb, q.status);
        k_q_assign<<<(unsigned)nb, QB, 0, s>>>(c, q.status);
    }
    k_q_place<<<(unsigned)((std::max<int64_t>(q.cap_add, 1) + 255) / 256), 256, 0, s>>>(c, q.cap_add, q.out_slot, q.status);
    return cudaGetLastError();
}

cudaError_t launch_fold_touched(const float* unary, const double* fold, const int64_t* inc_ptr, const int2* inc,
                                int N, int L, uint8_t* touched, double* ut, float* utf, cudaStream_t s) {
    if (N > 0) k_fold_touched<<<(N + 255) / 256, 256, 0, s>>>(unary, fold, inc_ptr, inc, N, L, touched, ut, utf);
    return cudaGetLastError();
}

cudaError_t launch_queue_finish(const QArgs& q, cudaStream_t s) {
    k_q_finish<<<1, 32, 0, s>>>(q);
    return cudaGetLastError();
}

int csr_sort_long_cap() { return kCsrSortLongSmem / (int)sizeof(int2); }

// Opt-in to the large dynamic shared memory of k_csr_sort_long (outside any
// stream capture; idempotent).
cudaError_t init_csr_sort_long() {
    return cudaFuncSetAttribute(k_csr_sort_long, cudaFuncAttributeMaxDynamicSharedMemorySize, kCsrSortLongSmem);
}

cudaError_t launch_csr_sort_long(const int64_t* ptr, int2* inc, int N, int min_deg, uint32_t* status, cudaStream_t s) {
    if (N > 0) {
        const int blocks = (int)std::min<int64_t>(((int64_t)N + 255) / 256, 2 * 152);
        k_csr_sort_long<<<blocks, 256, kCsrSortLongSmem, s>>>(ptr, inc, N, min_deg, csr_sort_long_cap(), status);
    }
    return cudaGetLastError();
}

}  // namespace mrfk
