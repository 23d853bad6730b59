// Host side of the C ABI declared in include/mrf.h: handle life cycle,
// argument checks, device buffers, CSR incidence build, edits, and the sweep
// driver (optionally replayed as a captured CUDA graph).
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>

using namespace mrfk;

struct mrf {
    int32_t N = 0, L = 0, C = 0, layout = MRF_LAYOUT_PIVOT, M = 0, W = 0;
    int64_t E_live = 0, E_slots = 0, E_cap = 0;
    uint64_t seed = 0;
    uint2 key{};
    cudaStream_t stream = nullptr;
    mrf_options opt{};
    bool has_factors = false;
    // device buffers
    float* d_unary = nullptr;
    double* d_ut = nullptr;
    int32_t* d_src = nullptr;
    int32_t* d_dst = nullptr;
    float* d_tau = nullptr;
    uint32_t* d_thr = nullptr;
    uint32_t* d_tpl = nullptr;         // [E][W][32] threshold prefix planes
    float* d_utf = nullptr;            // [N][L] folded unaries, float32
    double* d_fold = nullptr;
    double* d_cst = nullptr;
    float* d_resid = nullptr;
    int64_t* d_inc_ptr = nullptr;
    int2* d_inc = nullptr;
    uint8_t* d_x = nullptr;
    uint32_t* d_theta = nullptr;
    uint32_t* d_counts = nullptr;
    float* d_logp = nullptr;
    Ctl* d_ctl = nullptr;
    unsigned long long* d_flag = nullptr;
    // host mirrors
    std::vector<int32_t> h_src, h_dst;
    std::vector<int64_t> free_slots;   // sorted ascending
    int64_t sweep_host = 0, count_from_host = 0;
    double log_const = NAN;
    std::string err;
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
    uint8_t* d_stage = nullptr;        // [C][N] staging for the ABI label view
    float* d_pot = nullptr;            // [N][L][C] node potentials of the blocked sweep
    // kernel timing (options.kernel_timing)
    struct Rec { int id; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
};

namespace {

mrf_status fail(mrf_t* h, mrf_status st, const std::string& msg) {
    if (h) h->err = msg;
    return st;
}

#define MRF_CUDA(h, call)                                                                       \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            cudaGetLastError();                                                                 \
            return fail(h, e_ == cudaErrorMemoryAllocation ? MRF_ENOMEM : MRF_ECUDA,            \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                    \
        }                                                                                       \
    } while (0)

template <class T>
void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

template <class T>
cudaError_t dalloc(T*& p, size_t n) {
    dfree(p);
    if (n == 0) n = 1;
    return cudaMalloc((void**)&p, n * sizeof(T));
}

cudaEvent_t take_event(mrf_t* h) {
    if (!h->pool.empty()) { cudaEvent_t e = h->pool.back(); h->pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch fn() on the handle's stream, bracketed by CUDA events when timing is on.
template <class Fn>
cudaError_t timed(mrf_t* h, int id, Fn fn) {
    if (!h->opt.kernel_timing) return fn();
    mrf_t::Rec r{id, take_event(h), take_event(h)};
    cudaEventRecord(r.a, h->stream);
    cudaError_t e = fn();
    cudaEventRecord(r.b, h->stream);
    h->pending.push_back(r);
    return e;
}

void drop_graphs(mrf_t* h) {
    for (auto& g : h->graph)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
}

SweepArgs make_args(const mrf_t* h) {
    SweepArgs a{};
    a.N = h->N; a.C = h->C; a.L = h->L; a.M = h->M; a.W = h->W;
    a.E = h->E_slots;
    a.src = h->d_src; a.dst = h->d_dst; a.tau = h->d_tau; a.thr = h->d_thr; a.resid = h->d_resid;
    a.tpl = h->d_tpl; a.utf = h->d_utf;
    a.inc_ptr = h->d_inc_ptr; a.inc = h->d_inc; a.ut = h->d_ut;
    a.x = h->d_x; a.theta = h->d_theta; a.counts = h->d_counts; a.logp = h->d_logp;
    a.ctl = h->d_ctl; a.key = h->key;
    a.fdC = FastDiv::make((uint32_t)h->C);
    const int nx = h->opt.grid_nx, ny = h->opt.grid_ny, nz = h->opt.grid_nz;
    if (nx > 0) {
        a.nxe = (int64_t)(nx - 1) * ny * nz;
        a.nye = (int64_t)nx * (ny - 1) * nz;
        a.fdX1 = FastDiv::make((uint32_t)(nx - 1)); a.fdX = FastDiv::make((uint32_t)nx);
        a.fdY1 = FastDiv::make((uint32_t)(ny - 1)); a.fdY = FastDiv::make((uint32_t)ny);
    }
    a.pot = h->d_pot;
    a.grid_nx = h->opt.grid_nx; a.grid_ny = h->opt.grid_ny; a.grid_nz = h->opt.grid_nz;
    return a;
}

// Copy n elements of T from a host or device pointer to host.
template <class T>
cudaError_t to_host(std::vector<T>& out, const T* p, int64_t n, int ptr_kind, cudaStream_t s) {
    out.resize((size_t)n);
    if (n == 0) return cudaSuccess;
    if (ptr_kind == MRF_PTR_HOST) {
        std::memcpy(out.data(), p, (size_t)n * sizeof(T));
        return cudaSuccess;
    }
    cudaError_t e = cudaMemcpyAsync(out.data(), p, (size_t)n * sizeof(T), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

template <class T>
cudaError_t to_device(T* dst, const T* p, int64_t n, int ptr_kind, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, p, (size_t)n * sizeof(T),
                           ptr_kind == MRF_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s);
}

// CSR incidence of live edges; within a site, incidences in increasing slot order.
cudaError_t build_csr(mrf_t* h) {
    const int64_t E = h->E_slots;
    std::vector<int64_t> ptr((size_t)h->N + 1, 0);
    for (int64_t e = 0; e < E; ++e) {
        if (h->h_src[e] < 0) continue;
        ptr[h->h_src[e] + 1]++;
        ptr[h->h_dst[e] + 1]++;
    }
    for (int v = 0; v < h->N; ++v) ptr[v + 1] += ptr[v];
    std::vector<int2> inc((size_t)ptr[h->N]);
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t e = 0; e < E; ++e) {
        const int s = h->h_src[e];
        if (s < 0) continue;
        const int t = h->h_dst[e];
        inc[fill[s]++] = make_int2((int)(e * 2 + 0), t);
        inc[fill[t]++] = make_int2((int)(e * 2 + 1), s);
    }
    cudaError_t err;
    if ((err = dalloc(h->d_inc_ptr, ptr.size())) != cudaSuccess) return err;
    if ((err = dalloc(h->d_inc, std::max<size_t>(inc.size(), 1))) != cudaSuccess) return err;
    if ((err = cudaMemcpyAsync(h->d_inc_ptr, ptr.data(), ptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                               h->stream)) != cudaSuccess)
        return err;
    if (!inc.empty() && (err = cudaMemcpyAsync(h->d_inc, inc.data(), inc.size() * sizeof(int2),
                                               cudaMemcpyHostToDevice, h->stream)) != cudaSuccess)
        return err;
    return cudaStreamSynchronize(h->stream);   // host vectors go out of scope
}

bool lattice_ok(const mrf_t* h) {
    const int nx = h->opt.grid_nx, ny = h->opt.grid_ny, nz = h->opt.grid_nz;
    if ((int64_t)nx * ny * nz != h->N) return false;
    int64_t e = 0;
    auto site = [&](int x, int y, int z) { return x + nx * (y + ny * z); };
    for (int axis = 0; axis < 3; ++axis) {
        const int lim[3] = {nx, ny, nz};
        if (lim[axis] <= 1) continue;
        for (int z = 0; z < nz - (axis == 2); ++z)
            for (int y = 0; y < ny - (axis == 1); ++y)
                for (int x = 0; x < nx - (axis == 0); ++x, ++e) {
                    if (e >= h->E_slots) return false;
                    const int s = site(x, y, z);
                    const int t = site(x + (axis == 0), y + (axis == 1), z + (axis == 2));
                    if (h->h_src[e] != s || h->h_dst[e] != t) return false;
                }
    }
    return e == h->E_slots;
}

mrf_status check_finite_device(mrf_t* h, const float* d, int64_t n, const char* what) {
    MRF_CUDA(h, cudaMemsetAsync(h->d_flag, 0, sizeof(unsigned long long), h->stream));
    MRF_CUDA(h, launch_check_finite(d, n, h->d_flag, h->stream));
    unsigned long long bad = 0;
    MRF_CUDA(h, cudaMemcpyAsync(&bad, h->d_flag, sizeof(bad), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (bad) return fail(h, MRF_ENONFINITE, std::string(what) + ": " + std::to_string(bad) + " non-finite values");
    return MRF_OK;
}

}  // namespace

extern "C" {

void mrf_default_options(mrf_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->use_graphs = 1;
}

const char* mrf_status_string(mrf_status s) {
    switch (s) {
        case MRF_OK: return "ok";
        case MRF_EINVAL: return "invalid argument";
        case MRF_ENONFINITE: return "non-finite log-potential";
        case MRF_ENOMEM: return "out of device memory";
        case MRF_ECUDA: return "CUDA error";
        case MRF_ERANGE: return "index out of range";
        case MRF_ETIMEOUT: return "device wait timed out";
        case MRF_ESTATE: return "invalid state";
    }
    return "unknown";
}

const char* mrf_last_error(const mrf_t* h) { return h ? h->err.c_str() : "null handle"; }

mrf_status mrf_kernel_times(mrf_t* h, double* ms, int64_t* launches) {
    if (!h || !ms || !launches) return MRF_EINVAL;
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < MRF_K_COUNT; ++i) { ms[i] = 0.0; launches[i] = 0; }
    for (auto& r : h->pending) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) { ms[r.id] += t; launches[r.id] += 1; }
        h->pool.push_back(r.a); h->pool.push_back(r.b);
    }
    cudaGetLastError();
    h->pending.clear();
    return MRF_OK;
}

mrf_status mrf_create(mrf_t** out, int32_t n_vars, int32_t n_labels, int32_t n_chains, uint64_t seed,
                      const mrf_options* opt, void* cuda_stream) {
    if (!out) return MRF_EINVAL;
    *out = nullptr;
    if (n_vars <= 0 || n_chains <= 0) return MRF_EINVAL;
    if (n_labels < 2 || n_labels > kMaxLabels) return MRF_ERANGE;
    if ((int64_t)n_vars * n_chains >= (int64_t)1 << 32) return MRF_ERANGE;
    mrf_t* h = new mrf_t();
    h->N = n_vars; h->L = n_labels; h->C = n_chains; h->seed = seed; h->key = seed_key(seed);
    h->stream = (cudaStream_t)cuda_stream;
    if (opt) h->opt = *opt; else mrf_default_options(&h->opt);
    auto bail = [&](mrf_status st) { mrf_destroy(h); return st; };
    const size_t NL = (size_t)n_vars * n_labels, NC = (size_t)n_vars * n_chains;
    if (dalloc(h->d_unary, NL) || dalloc(h->d_ut, NL) || dalloc(h->d_utf, NL) || dalloc(h->d_x, 2 * NC) || dalloc(h->d_counts, NL) ||
        dalloc(h->d_ctl, 1) || dalloc(h->d_flag, 1)) {
        cudaGetLastError();
        return bail(MRF_ENOMEM);
    }
    if (h->opt.record_logp && dalloc(h->d_logp, NC * n_labels)) { cudaGetLastError(); return bail(MRF_ENOMEM); }
    Ctl c0{0, 0, 0, 0};
    if (cudaMemcpyAsync(h->d_ctl, &c0, sizeof(c0), cudaMemcpyHostToDevice, h->stream) ||
        cudaMemsetAsync(h->d_unary, 0, NL * sizeof(float), h->stream) ||
        cudaMemsetAsync(h->d_ut, 0, NL * sizeof(double), h->stream) ||
        cudaMemsetAsync(h->d_counts, 0, NL * sizeof(uint32_t), h->stream)) {
        cudaGetLastError();
        return bail(MRF_ECUDA);
    }
    SweepArgs a = make_args(h);
    if (launch_init_labels(a, h->stream) != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        return bail(MRF_ECUDA);
    }
    *out = h;
    return MRF_OK;
}

void mrf_destroy(mrf_t* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
    drop_graphs(h);
    dfree(h->d_unary); dfree(h->d_ut); dfree(h->d_utf); dfree(h->d_tpl); dfree(h->d_src); dfree(h->d_dst); dfree(h->d_tau); dfree(h->d_thr);
    dfree(h->d_fold); dfree(h->d_cst); dfree(h->d_resid); dfree(h->d_inc_ptr); dfree(h->d_inc); dfree(h->d_x);
    dfree(h->d_theta); dfree(h->d_counts); dfree(h->d_logp); dfree(h->d_ctl); dfree(h->d_flag); dfree(h->d_stage); dfree(h->d_pot);
    for (auto& r : h->pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : h->pool) cudaEventDestroy(e);
    delete h;
}

mrf_status mrf_set_factors(mrf_t* h, const float* unary_log, int64_t n_edges, const int32_t* src,
                           const int32_t* dst, const float* pair_log, int32_t ptr_kind) {
    if (!h) return MRF_EINVAL;
    if (!unary_log || n_edges < 0 || (n_edges > 0 && (!src || !dst || !pair_log)))
        return fail(h, MRF_EINVAL, "null pointer or negative edge count");
    if (ptr_kind != MRF_PTR_HOST && ptr_kind != MRF_PTR_DEVICE) return fail(h, MRF_EINVAL, "bad ptr_kind");
    if (n_edges >= ((int64_t)1 << 30)) return fail(h, MRF_ERANGE, "too many edges (limit 2^30)");
    drop_graphs(h);
    const int L = h->L, N = h->N;
    // indices: host-side checks
    MRF_CUDA(h, to_host(h->h_src, src, n_edges, ptr_kind, h->stream));
    MRF_CUDA(h, to_host(h->h_dst, dst, n_edges, ptr_kind, h->stream));
    for (int64_t e = 0; e < n_edges; ++e) {
        const int s = h->h_src[e], t = h->h_dst[e];
        if (s < 0 || s >= N || t < 0 || t >= N) return fail(h, MRF_ERANGE, "edge " + std::to_string(e) + ": vertex id out of range");
        if (s == t) return fail(h, MRF_ERANGE, "edge " + std::to_string(e) + ": self-loop");
    }
    // potentials: copy, then check on the device
    MRF_CUDA(h, to_device(h->d_unary, unary_log, (int64_t)N * L, ptr_kind, h->stream));
    mrf_status st = check_finite_device(h, h->d_unary, (int64_t)N * L, "unary_log");
    if (st != MRF_OK) return st;
    float* d_pair = nullptr;
    MRF_CUDA(h, dalloc(d_pair, (size_t)n_edges * L * L));
    struct Guard { float*& p; ~Guard() { dfree(p); } } guard{d_pair};
    MRF_CUDA(h, to_device(d_pair, pair_log, n_edges * L * L, ptr_kind, h->stream));
    st = check_finite_device(h, d_pair, n_edges * L * L, "pair_log");
    if (st != MRF_OK) return st;
    // layout: DIAG when L >= 3 and every off-diagonal entry is exactly zero
    MRF_CUDA(h, cudaMemsetAsync(h->d_flag, 0, sizeof(unsigned long long), h->stream));
    MRF_CUDA(h, launch_count_offdiag(d_pair, n_edges, L, h->d_flag, h->stream));
    unsigned long long offdiag = 0;
    MRF_CUDA(h, cudaMemcpyAsync(&offdiag, h->d_flag, sizeof(offdiag), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    h->layout = (L >= 3 && n_edges > 0 && offdiag == 0) ? MRF_LAYOUT_DIAG : MRF_LAYOUT_PIVOT;
    h->M = n_entries(L, h->layout);
    h->W = (h->M + 31) / 32;
    h->E_live = h->E_slots = h->E_cap = n_edges;
    h->free_slots.clear();
    const bool want_resid = h->opt.grid_nx > 0;
    if (want_resid && !lattice_ok(h)) {
        h->has_factors = false;
        return fail(h, MRF_EINVAL, "options.grid set but the edges are not the lattice's in canonical order");
    }
    const size_t E = (size_t)n_edges;
    MRF_CUDA(h, dalloc(h->d_src, E)); MRF_CUDA(h, dalloc(h->d_dst, E));
    if ((uint64_t)E * h->C >= (1ull << 32)) return fail(h, MRF_ERANGE, "edges x chains must be below 2^32");
    MRF_CUDA(h, dalloc(h->d_tau, E * pad4(h->M))); MRF_CUDA(h, dalloc(h->d_thr, E * h->M));
    MRF_CUDA(h, dalloc(h->d_tpl, E * h->W * 32));
    MRF_CUDA(h, dalloc(h->d_fold, E * 2 * L)); MRF_CUDA(h, dalloc(h->d_cst, E));
    if (want_resid) MRF_CUDA(h, dalloc(h->d_resid, E * L * L)); else dfree(h->d_resid);
    MRF_CUDA(h, dalloc(h->d_theta, E * h->C * h->W));
    MRF_CUDA(h, to_device(h->d_src, h->h_src.data(), n_edges, MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, to_device(h->d_dst, h->h_dst.data(), n_edges, MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, build_csr(h));
    DecompArgs d{};
    d.L = L; d.M = h->M; d.layout = h->layout; d.n = n_edges; d.slots = nullptr; d.first_slot = 0;
    d.pair = d_pair; d.tau = h->d_tau; d.thr = h->d_thr; d.fold = h->d_fold; d.cst = h->d_cst; d.resid = h->d_resid;
    MRF_CUDA(h, launch_decompose(d, h->stream));
    MRF_CUDA(h, launch_build_planes(h->d_thr, n_edges, nullptr, 0, h->M, h->d_tpl, h->stream));
    MRF_CUDA(h, launch_fold_unary(h->d_unary, h->d_fold, h->d_inc_ptr, h->d_inc, N, L, h->d_ut, h->d_utf, h->stream));
    // log constant (for log-partition estimates): sum of per-edge constants
    std::vector<double> cst((size_t)n_edges);
    if (n_edges) MRF_CUDA(h, cudaMemcpyAsync(cst.data(), h->d_cst, E * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    h->log_const = std::accumulate(cst.begin(), cst.end(), 0.0);
    h->has_factors = true;
    return MRF_OK;
}

mrf_status mrf_edit_factors(mrf_t* h, int64_t n_remove, const int64_t* edge_ids, int64_t n_add,
                            const int32_t* src, const int32_t* dst, const float* pair_log, int64_t* out_new_ids,
                            int32_t ptr_kind) {
    if (!h) return MRF_EINVAL;
    if (!h->has_factors) return fail(h, MRF_ESTATE, "mrf_set_factors first");
    if (n_remove < 0 || n_add < 0 || (n_remove && !edge_ids) || (n_add && (!src || !dst || !pair_log || !out_new_ids)))
        return fail(h, MRF_EINVAL, "bad edit arguments");
    if (h->opt.grid_nx > 0) return fail(h, MRF_ESTATE, "edits are not available on a lattice handle");
    const int L = h->L, N = h->N;
    std::vector<int64_t> rem;
    std::vector<int32_t> as, at;
    MRF_CUDA(h, to_host(rem, edge_ids, n_remove, ptr_kind, h->stream));
    MRF_CUDA(h, to_host(as, src, n_add, ptr_kind, h->stream));
    MRF_CUDA(h, to_host(at, dst, n_add, ptr_kind, h->stream));
    {
        std::vector<int64_t> sorted = rem;
        std::sort(sorted.begin(), sorted.end());
        for (size_t i = 0; i < sorted.size(); ++i) {
            const int64_t e = sorted[i];
            if (e < 0 || e >= h->E_slots || h->h_src[e] < 0 || (i && sorted[i - 1] == e))
                return fail(h, MRF_ERANGE, "edit: slot " + std::to_string(e) + " is not a live edge");
        }
    }
    for (int64_t i = 0; i < n_add; ++i) {
        if (as[i] < 0 || as[i] >= N || at[i] < 0 || at[i] >= N) return fail(h, MRF_ERANGE, "edit: vertex id out of range");
        if (as[i] == at[i]) return fail(h, MRF_ERANGE, "edit: self-loop");
    }
    float* d_pair = nullptr;
    MRF_CUDA(h, dalloc(d_pair, (size_t)n_add * L * L));
    struct Guard { float*& p; ~Guard() { dfree(p); } } guard{d_pair};
    MRF_CUDA(h, to_device(d_pair, pair_log, n_add * L * L, ptr_kind, h->stream));
    mrf_status st = check_finite_device(h, d_pair, n_add * L * L, "pair_log");
    if (st != MRF_OK) return st;
    if (h->layout == MRF_LAYOUT_DIAG) {
        MRF_CUDA(h, cudaMemsetAsync(h->d_flag, 0, sizeof(unsigned long long), h->stream));
        MRF_CUDA(h, launch_count_offdiag(d_pair, n_add, L, h->d_flag, h->stream));
        unsigned long long offdiag = 0;
        MRF_CUDA(h, cudaMemcpyAsync(&offdiag, h->d_flag, sizeof(offdiag), cudaMemcpyDeviceToHost, h->stream));
        MRF_CUDA(h, cudaStreamSynchronize(h->stream));
        if (offdiag) return fail(h, MRF_EINVAL, "edit: handle uses the diagonal layout; new tables must be diagonal");
    }
    drop_graphs(h);
    // free removed slots
    for (int64_t e : rem) { h->h_src[e] = -1; h->h_dst[e] = -1; }
    std::vector<int64_t> pool = h->free_slots;
    pool.insert(pool.end(), rem.begin(), rem.end());
    std::sort(pool.begin(), pool.end());
    // new edges: freed slots in increasing order, then fresh slots
    std::vector<int64_t> slots((size_t)n_add);
    size_t used = 0;
    int64_t next = h->E_slots;
    for (int64_t i = 0; i < n_add; ++i) slots[i] = used < pool.size() ? pool[used++] : next++;
    h->free_slots.assign(pool.begin() + used, pool.end());
    const int64_t new_slots = next;
    if (new_slots > h->E_cap) {
        // grow every per-slot buffer (x1.25 slack)
        const int64_t cap = std::max<int64_t>(new_slots, h->E_cap + h->E_cap / 4 + 1024);
        auto grow = [&](auto*& p, size_t per) -> cudaError_t {
            using T = std::remove_reference_t<decltype(*p)>;
            T* q = nullptr;
            cudaError_t e = cudaMalloc((void**)&q, (size_t)cap * per * sizeof(T));
            if (e != cudaSuccess) return e;
            if (h->E_slots) e = cudaMemcpyAsync(q, p, (size_t)h->E_slots * per * sizeof(T), cudaMemcpyDeviceToDevice, h->stream);
            if (e != cudaSuccess) { cudaFree(q); return e; }
            cudaStreamSynchronize(h->stream);
            dfree(p);
            p = q;
            return cudaSuccess;
        };
        MRF_CUDA(h, grow(h->d_src, 1)); MRF_CUDA(h, grow(h->d_dst, 1));
        if ((uint64_t)cap * h->C >= (1ull << 32)) return fail(h, MRF_ERANGE, "edges x chains must be below 2^32");
        MRF_CUDA(h, grow(h->d_tau, pad4(h->M))); MRF_CUDA(h, grow(h->d_thr, h->M)); MRF_CUDA(h, grow(h->d_tpl, h->W * 32));
        MRF_CUDA(h, grow(h->d_fold, 2 * L)); MRF_CUDA(h, grow(h->d_cst, 1));
        MRF_CUDA(h, dalloc(h->d_theta, (size_t)cap * h->C * h->W));
        h->E_cap = cap;
    }
    h->h_src.resize(new_slots, -1); h->h_dst.resize(new_slots, -1);
    for (int64_t i = 0; i < n_add; ++i) { h->h_src[slots[i]] = as[i]; h->h_dst[slots[i]] = at[i]; }
    h->E_slots = new_slots;
    h->E_live += n_add - n_remove;
    MRF_CUDA(h, to_device(h->d_src, h->h_src.data(), new_slots, MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, to_device(h->d_dst, h->h_dst.data(), new_slots, MRF_PTR_HOST, h->stream));
    int64_t* d_slots = nullptr;
    MRF_CUDA(h, dalloc(d_slots, (size_t)n_add));
    struct Guard2 { int64_t*& p; ~Guard2() { dfree(p); } } guard2{d_slots};
    MRF_CUDA(h, to_device(d_slots, slots.data(), n_add, MRF_PTR_HOST, h->stream));
    DecompArgs d{};
    d.L = L; d.M = h->M; d.layout = h->layout; d.n = n_add; d.slots = d_slots;
    d.pair = d_pair; d.tau = h->d_tau; d.thr = h->d_thr; d.fold = h->d_fold; d.cst = h->d_cst; d.resid = nullptr;
    MRF_CUDA(h, launch_decompose(d, h->stream));
    MRF_CUDA(h, launch_build_planes(h->d_thr, n_add, d_slots, 0, h->M, h->d_tpl, h->stream));
    MRF_CUDA(h, build_csr(h));
    MRF_CUDA(h, launch_fold_unary(h->d_unary, h->d_fold, h->d_inc_ptr, h->d_inc, N, L, h->d_ut, h->d_utf, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    std::copy(slots.begin(), slots.end(), out_new_ids);
    return MRF_OK;
}

static mrf_status enqueue_sweep(mrf_t* h, int mode) {
    SweepArgs a = make_args(h);
    cudaStream_t s = h->stream;
    cudaError_t e = cudaSuccess;
    if (mode == MRF_MODE_PLAIN) {
        e = timed(h, MRF_K_DUAL, [&] { return launch_dual(a, h->layout, s); });
        if (e == cudaSuccess) e = timed(h, MRF_K_PRIMAL, [&] { return launch_primal(a, h->layout, h->opt.schedule, s); });
    } else if (mode == MRF_MODE_FUSED) {
        e = timed(h, MRF_K_FUSED, [&] { return launch_fused(a, h->layout, h->opt.schedule, s); });
    } else {
        a.splash = 1;
        e = launch_splash_offset(a, s);
        if (e == cudaSuccess) e = timed(h, MRF_K_DUAL, [&] { return launch_dual(a, h->layout, s); });
        if (e == cudaSuccess) e = timed(h, MRF_K_POTENTIAL, [&] { return launch_potential(a, h->layout, s); });
        if (e == cudaSuccess) e = timed(h, MRF_K_FFBS, [&] { return launch_ffbs(a, s); });
    }
    if (e == cudaSuccess) e = timed(h, MRF_K_ACCUMULATE, [&] { return launch_accumulate(a, s); });
    if (e == cudaSuccess) e = launch_advance(a, s);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(h, MRF_ECUDA, std::string("sweep launch: ") + cudaGetErrorString(e)); }
    return MRF_OK;
}

mrf_status mrf_sweep(mrf_t* h, int32_t n_sweeps, int32_t mode) {
    if (!h) return MRF_EINVAL;
    if (!h->has_factors) return fail(h, MRF_ESTATE, "mrf_set_factors first");
    if (n_sweeps < 0 || mode < MRF_MODE_PLAIN || mode > MRF_MODE_SPLASH) return fail(h, MRF_EINVAL, "bad sweep count or mode");
    if (mode == MRF_MODE_SPLASH && h->opt.grid_nx <= 0) return fail(h, MRF_ESTATE, "splash mode needs options.grid");
    if (mode == MRF_MODE_SPLASH && !h->d_pot) {
        drop_graphs(h);
        MRF_CUDA(h, dalloc(h->d_pot, (size_t)h->N * h->L * h->C));
    }
    const bool graphs = h->opt.use_graphs && h->stream != nullptr && !h->opt.kernel_timing;
    if (graphs && !h->graph[mode] && n_sweeps > 0) {
        cudaGraph_t g = nullptr;
        MRF_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        mrf_status st = enqueue_sweep(h, mode);
        cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
        if (st != MRF_OK) { if (g) cudaGraphDestroy(g); return st; }
        MRF_CUDA(h, ce);
        ce = cudaGraphInstantiate(&h->graph[mode], g, 0);
        cudaGraphDestroy(g);
        MRF_CUDA(h, ce);
    }
    for (int i = 0; i < n_sweeps; ++i) {
        if (graphs) {
            MRF_CUDA(h, cudaGraphLaunch(h->graph[mode], h->stream));
        } else {
            mrf_status st = enqueue_sweep(h, mode);
            if (st != MRF_OK) return st;
        }
    }
    h->sweep_host += n_sweeps;
    return MRF_OK;
}

mrf_status mrf_get_counts(mrf_t* h, uint32_t* out, int32_t ptr_kind) {
    if (!h || !out) return MRF_EINVAL;
    const size_t n = (size_t)h->N * h->L;
    MRF_CUDA(h, cudaMemcpyAsync(out, h->d_counts, n * sizeof(uint32_t),
                                ptr_kind == MRF_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    return MRF_OK;
}

mrf_status mrf_marginals(mrf_t* h, float* out, int64_t* n_samples, int32_t ptr_kind) {
    if (!h || !out) return MRF_EINVAL;
    const size_t n = (size_t)h->N * h->L;
    std::vector<uint32_t> cnt(n);
    mrf_status st = mrf_get_counts(h, cnt.data(), MRF_PTR_HOST);
    if (st != MRF_OK) return st;
    const int64_t ns = std::max<int64_t>(0, h->sweep_host - h->count_from_host) * h->C;
    std::vector<float> m(n);
    for (size_t i = 0; i < n; ++i) m[i] = ns ? (float)((double)cnt[i] / (double)ns) : 0.0f;
    if (n_samples) *n_samples = ns;
    if (ptr_kind == MRF_PTR_HOST) std::memcpy(out, m.data(), n * sizeof(float));
    else {
        MRF_CUDA(h, cudaMemcpyAsync(out, m.data(), n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    return MRF_OK;
}

mrf_status mrf_reset_marginals(mrf_t* h, int32_t burn_in_sweeps) {
    if (!h || burn_in_sweeps < 0) return MRF_EINVAL;
    h->count_from_host = h->sweep_host + burn_in_sweeps;
    unsigned long long cf = (unsigned long long)h->count_from_host;
    MRF_CUDA(h, cudaMemsetAsync(h->d_counts, 0, (size_t)h->N * h->L * sizeof(uint32_t), h->stream));
    MRF_CUDA(h, cudaMemcpyAsync(&h->d_ctl->count_from, &cf, sizeof(cf), cudaMemcpyHostToDevice, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    return MRF_OK;
}

// Labels live in buffer (t & 1) of x[2][N][C]; the ABI view is [C][N].  The
// layout change runs on the device through a [C][N] staging buffer.
mrf_status mrf_get_labels(mrf_t* h, uint8_t* out, int32_t ptr_kind) {
    if (!h || !out) return MRF_EINVAL;
    const size_t NC = (size_t)h->N * h->C;
    if (!h->d_stage) MRF_CUDA(h, dalloc(h->d_stage, NC));
    MRF_CUDA(h, launch_labels_to_abi(h->d_x + (h->sweep_host & 1) * NC, h->d_stage, h->N, h->C, h->stream));
    MRF_CUDA(h, cudaMemcpyAsync(out, h->d_stage, NC,
                                ptr_kind == MRF_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    return MRF_OK;
}

mrf_status mrf_set_labels(mrf_t* h, const uint8_t* in, int32_t ptr_kind) {
    if (!h || !in) return MRF_EINVAL;
    const size_t NC = (size_t)h->N * h->C;
    if (!h->d_stage) MRF_CUDA(h, dalloc(h->d_stage, NC));
    MRF_CUDA(h, to_device(h->d_stage, in, (int64_t)NC, ptr_kind, h->stream));
    MRF_CUDA(h, cudaMemsetAsync(h->d_flag, 0, sizeof(unsigned long long), h->stream));
    MRF_CUDA(h, launch_count_ge(h->d_stage, (int64_t)NC, h->L, h->d_flag, h->stream));
    unsigned long long bad = 0;
    MRF_CUDA(h, cudaMemcpyAsync(&bad, h->d_flag, sizeof(bad), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (bad) return fail(h, MRF_ERANGE, "label out of range");
    MRF_CUDA(h, launch_labels_from_abi(h->d_stage, h->d_x + (h->sweep_host & 1) * NC, h->N, h->C, h->stream));
    return MRF_OK;
}

mrf_status mrf_set_sweep_index(mrf_t* h, int64_t t) {
    if (!h || t < 0 || t >= ((int64_t)1 << 32)) return MRF_EINVAL;
    const size_t NC = (size_t)h->N * h->C;
    if ((t & 1) != (h->sweep_host & 1))
        MRF_CUDA(h, cudaMemcpyAsync(h->d_x + (t & 1) * NC, h->d_x + (h->sweep_host & 1) * NC, NC,
                                    cudaMemcpyDeviceToDevice, h->stream));
    unsigned long long tt = (unsigned long long)t;
    MRF_CUDA(h, cudaMemcpyAsync(&h->d_ctl->sweep, &tt, sizeof(tt), cudaMemcpyHostToDevice, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    h->count_from_host += t - h->sweep_host;   // keep the burn-in window relative
    unsigned long long cf = (unsigned long long)std::max<int64_t>(0, h->count_from_host);
    MRF_CUDA(h, cudaMemcpyAsync(&h->d_ctl->count_from, &cf, sizeof(cf), cudaMemcpyHostToDevice, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    h->sweep_host = t;
    return MRF_OK;
}

mrf_status mrf_get_info(const mrf_t* h, mrf_info* out) {
    if (!h || !out) return MRF_EINVAL;
    out->n_vars = h->N; out->n_labels = h->L; out->n_chains = h->C; out->layout = h->layout; out->n_entries = h->M;
    out->n_edges = h->E_live; out->n_edge_slots = h->E_slots; out->sweep_index = h->sweep_host;
    out->n_samples = std::max<int64_t>(0, h->sweep_host - h->count_from_host) * h->C;
    out->log_const = h->log_const;
    return MRF_OK;
}

mrf_status mrf_debug_tables(mrf_t* h, float* tau, uint32_t* thr, double* utilde) {
    if (!h) return MRF_EINVAL;
    if (!h->has_factors) return fail(h, MRF_ESTATE, "no factors");
    const size_t EM = (size_t)h->E_slots * h->M;
    if (tau) MRF_CUDA(h, cudaMemcpy2DAsync(tau, h->M * sizeof(float), h->d_tau, pad4(h->M) * sizeof(float),
                                           h->M * sizeof(float), (size_t)h->E_slots, cudaMemcpyDeviceToHost, h->stream));
    if (thr) MRF_CUDA(h, cudaMemcpyAsync(thr, h->d_thr, EM * sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
    if (utilde) MRF_CUDA(h, cudaMemcpyAsync(utilde, h->d_ut, (size_t)h->N * h->L * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    return MRF_OK;
}

mrf_status mrf_debug_logp(mrf_t* h, float* out, uint64_t* boundary_draws) {
    if (!h) return MRF_EINVAL;
    if (out) {
        if (!h->d_logp) return fail(h, MRF_ESTATE, "create the handle with options.record_logp = 1");
        MRF_CUDA(h, cudaMemcpyAsync(out, h->d_logp, (size_t)h->C * h->N * h->L * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    }
    unsigned long long b = 0;
    MRF_CUDA(h, cudaMemcpyAsync(&b, &h->d_ctl->boundary, sizeof(b), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (boundary_draws) *boundary_draws = b;
    return MRF_OK;
}

mrf_status mrf_debug_theta(mrf_t* h, uint32_t* out) {
    if (!h || !out) return MRF_EINVAL;
    if (!h->has_factors) return fail(h, MRF_ESTATE, "no factors");
    MRF_CUDA(h, cudaMemcpyAsync(out, h->d_theta, (size_t)h->E_slots * h->C * h->W * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    return MRF_OK;
}

mrf_status mrf_sweep_noalloc(mrf_t* h, const uint8_t* labels_in, uint8_t* labels_out, int64_t sweep_index) {
    if (!h) return MRF_EINVAL;
    if (!h->has_factors) return fail(h, MRF_ESTATE, "mrf_set_factors first");
    if (!labels_in || !labels_out) return fail(h, MRF_EINVAL, "null label buffer");
    const uint64_t NC = (uint64_t)h->N * h->C;
    if (labels_in < labels_out + NC && labels_out < labels_in + NC) return fail(h, MRF_EINVAL, "label buffers overlap");
    if (sweep_index < 0 || sweep_index >= ((int64_t)1 << 32)) return fail(h, MRF_EINVAL, "sweep index out of range");
    const uint64_t words = (uint64_t)h->E_slots * h->C * h->W;
    if (words > MRF_NOALLOC_THETA_WORDS)
        return fail(h, MRF_ERANGE, "edge slots x chains x ceil(m/32) = " + std::to_string(words) +
                                       " words exceeds the static scratch of " +
                                       std::to_string(MRF_NOALLOC_THETA_WORDS) + " words");
    uint32_t* scratch = nullptr;
    MRF_CUDA(h, noalloc_scratch(&scratch));
    SweepArgs a = make_args(h);
    a.ctl = reinterpret_cast<Ctl*>(scratch);
    a.theta = scratch + 64;
    a.logp = nullptr;
    MRF_CUDA(h, launch_sweep_noalloc(a, h->layout, labels_in, labels_out, (uint32_t)sweep_index, h->stream));
    return MRF_OK;
}

}  // extern "C"
