// Host side of the C ABI declared in include/mrf.h: handle life cycle,
// argument checks, device buffers, CSR incidence build, edits, and the sweep
// driver (optionally replayed as a captured CUDA graph).
#include "common.cuh"

#include <algorithm>
#include <iterator>
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
    int32_t max_deg = 0;               // largest incidence count of a site
    int2* d_inc = nullptr;
    uint8_t* d_x = nullptr;
    uint32_t* d_theta = nullptr;
    uint8_t* d_em = nullptr;           // [2][N][C] labels of the EM iterations
    float* d_mfq = nullptr;            // [2][N][L][C] marginals of the mean-field iterations
    float* d_mfs = nullptr;            // [C][N][L] staging of the mean-field interface
    float* d_lpv = nullptr;            // [N][C] log p of the drawn labels (log-partition estimator)
    double* d_logv = nullptr;          // [sweeps][C] log V of the estimator
    int64_t logv_cap = 0;
    bool lpv_on = false;
    uint32_t* d_counts = nullptr;
    float* d_logp = nullptr;
    Ctl* d_ctl = nullptr;
    unsigned long long* d_flag = nullptr;
    // host mirrors
    std::vector<int32_t> h_src, h_dst;
    std::vector<int64_t> free_slots;   // sorted ascending
    bool mirror_stale = false;         // device edits (a batch's edit queue) changed the endpoints since
    bool dyn_degree = false;           // captured sweeps must not assume the current largest degree
    const int64_t* d_live_ext = nullptr;   // device count of live edges kept by a batch's edit queue
    int64_t sweep_host = 0, count_from_host = 0;
    double log_const = NAN;
    std::string err;
    cudaGraphExec_t graph[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    uint8_t* d_stage = nullptr;        // [C][N] staging for the ABI label view
    // Swendsen-Wang (diagonal layout): per-edge tables and per-sweep union-find state
    uint32_t* d_swt = nullptr;         // [E][L] 23-bit bond thresholds
    int64_t* d_swl = nullptr;          // [E][L] fixed-point bond log weights
    double* d_swfold = nullptr;        // [E][2][L] two-label unary offsets
    double* d_swut = nullptr;          // [N][L] two-label unaries with the offsets folded in
    int32_t* d_swpar = nullptr;        // [N][C] union-find parents
    int32_t* d_swroot = nullptr;       // [N][C] roots of bonded sites
    uint32_t* d_swbits = nullptr;      // bond bitmap, one bit per (edge slot, chain)
    int64_t swbits_cap = 0;            // words of d_swbits
    uint32_t* d_swban = nullptr;       // [N][C] excluded labels of a cluster
    int64_t* d_swlw = nullptr;         // [N][L][C] fixed-point cluster log weights
    unsigned* d_swerr = nullptr;       // union-find step bound exceeded
    int64_t* d_swufix = nullptr;       // [N][L] fixed-point unaries of the Swendsen-Wang sweep
    double* d_swchk = nullptr;         // [3] model check sums (k_sw_check)
    double* d_swell = nullptr;         // [E][L] couplings l_x of the Swendsen-Wang form (float64)
    // Higdon's partial Swendsen-Wang: tables of the split at hg_rho (rebuilt after factor changes)
    double hg_rho = 0.5;
    bool hg_ready = false;
    int64_t hg_cap = 0;                // edge slots the tables below hold
    uint32_t* d_hgT = nullptr; int64_t* d_hglb = nullptr; float* d_hgtau = nullptr; uint32_t* d_hgthr = nullptr;
    uint32_t* d_hgtpl = nullptr; double* d_hgfold = nullptr; double* d_hgbound = nullptr;
    double* d_hgut = nullptr; float* d_hgutf = nullptr;
    bool sw_checked = false;           // the model passed the check since the factors last changed
    float* d_pot = nullptr;            // [N][L][C] node potentials of the blocked sweep
    float* d_part = nullptr;           // [E_cap][C][2][L] partial fields of the edge-partial plain sweep
    int64_t part_cap = 0;              // edge slots d_part holds
    int schedule = 0;                  // primal schedule in use (1 thread, 2 CTA); 0 = not tuned yet
    int32_t* d_csr_work = nullptr;     // [2N] degrees and cursors of the device CSR build
    int64_t* d_csr_sums = nullptr;     // block sums of the device scan
    int64_t inc_cap = 0;               // capacity of d_inc (incidences)
    int64_t n_device_csr = 0, n_host_csr = 0;   // CSR builds after edits, by path
    // edit staging (grow-only, so that an edit allocates nothing in steady state)
    float* d_ed_pair = nullptr; int64_t ed_pair_cap = 0;
    int64_t* d_ed_slots = nullptr; int64_t* d_ed_new = nullptr; int32_t* d_ed_s = nullptr; int32_t* d_ed_t = nullptr;
    int64_t ed_cap = 0;
    // learned block proposal
    bool learned = false;
    LearnedArgs la{};
    int64_t n_params = 0;
    int32_t* d_members = nullptr; int32_t* d_nmem = nullptr; int64_t* d_intra_ptr = nullptr; int4* d_intra = nullptr;
    float* d_cf = nullptr; uint8_t* d_skip = nullptr;
    __nv_bfloat16* d_X = nullptr; __nv_bfloat16* d_H1 = nullptr; __nv_bfloat16* d_H2 = nullptr; float* d_Z = nullptr;
    float* d_w32 = nullptr; __nv_bfloat16* d_Wb = nullptr; float* d_grad = nullptr; float* d_m = nullptr; float* d_v = nullptr;
    float* d_train = nullptr; int64_t train_rows = 0;
    int32_t* d_bidx = nullptr; __nv_bfloat16* d_bX = nullptr; uint8_t* d_by = nullptr; uint8_t* d_bn = nullptr;
    __nv_bfloat16* d_dsX = nullptr; uint8_t* d_dsy = nullptr; uint8_t* d_dsn = nullptr;
    int64_t ds_cap = 0, ds_rows = 0;
    double* d_loss = nullptr; int64_t loss_cap = 0;
    __nv_bfloat16* d_W1x = nullptr; __nv_bfloat16* d_cfb = nullptr; float* d_rowbias = nullptr;
    uint8_t* d_wimg = nullptr; unsigned* d_tc_err = nullptr;    // tensor-core MLP weight images, error flag
    bool mlp_unusable = false;         // a timed-out tensor-core MLP did not drain: no further learned sweeps
    bool rowbias_dirty = true;
    unsigned long long* d_acc = nullptr;
    uint64_t proposed = 0;
    int adam_step = 0;
    float tune_ms[2] = {0.0f, 0.0f};   // autotuner timings (thread, CTA) per primal launch
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
    a.inc_ptr = h->d_inc_ptr; a.inc = h->d_inc; a.ut = h->d_ut; a.max_deg = h->dyn_degree ? 0x7FFFFFFF : h->max_deg;
    a.x = h->d_x; a.theta = h->d_theta; a.counts = h->d_counts; a.logp = h->d_logp;
    a.lpv = h->lpv_on ? h->d_lpv : nullptr;
    a.ctl = h->d_ctl; a.key = h->key;
    a.rk = round_keys(h->key);
    a.fdC = FastDiv::make((uint32_t)h->C);
    const int nx = h->opt.grid_nx, ny = h->opt.grid_ny, nz = h->opt.grid_nz;
    if (nx > 0) {
        a.nxe = (int64_t)(nx - 1) * ny * nz;
        a.nye = (int64_t)nx * (ny - 1) * nz;
        a.fdX1 = FastDiv::make((uint32_t)(nx - 1)); a.fdX = FastDiv::make((uint32_t)nx);
        a.fdY1 = FastDiv::make((uint32_t)(ny - 1)); a.fdY = FastDiv::make((uint32_t)ny);
    }
    a.pot = h->d_pot;
    a.part = h->d_part;
    a.grid_nx = h->opt.grid_nx; a.grid_ny = h->opt.grid_ny; a.grid_nz = h->opt.grid_nz;
    return a;
}

// The plain sweep takes the edge-partial form (k_edge_partial) for few chains
// and large tables: there it replaces reading each incident edge's whole
// weight row per (site, chain).  On 1-chain Erdos-Renyi classes it took the
// L = 16 class (225 entries) from 18.5 to 12.9 ms per sweep, while L = 8 (49
// entries, 4 words of weights per lane-pass) went from 2.7 to 4.8 ms: hence
// at least kPartialMinEntries entries.
bool use_partial(const mrf_t* h) { return h->C <= kPartialMaxChains && h->M >= kPartialMinEntries; }

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
    int64_t md = 0;
    for (int v = 0; v < h->N; ++v) { md = std::max(md, ptr[v + 1]); ptr[v + 1] += ptr[v]; }
    h->max_deg = (int32_t)std::min<int64_t>(md, 0x7FFFFFFF);
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
    h->inc_cap = (int64_t)inc.size();
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

// Grow every per-slot buffer to hold new_slots slots (x1.25 slack); the first
// E_slots slots keep their contents.
mrf_status grow_slots(mrf_t* h, int64_t new_slots) {
    if (new_slots <= h->E_cap) return MRF_OK;
    const int L = h->L;
    const int64_t cap = std::max<int64_t>(new_slots, h->E_cap + h->E_cap / 4 + 1024);
    if ((uint64_t)cap * h->C >= (1ull << 32)) return fail(h, MRF_ERANGE, "edges x chains must be below 2^32");
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
    MRF_CUDA(h, grow(h->d_tau, pad4(h->M))); MRF_CUDA(h, grow(h->d_thr, h->M)); MRF_CUDA(h, grow(h->d_tpl, plane_words(h->M)));
    MRF_CUDA(h, grow(h->d_fold, 2 * L)); MRF_CUDA(h, grow(h->d_cst, 1));
    if (h->d_swt) { MRF_CUDA(h, grow(h->d_swt, L)); MRF_CUDA(h, grow(h->d_swl, L)); MRF_CUDA(h, grow(h->d_swell, L)); }
    if (h->d_swfold) MRF_CUDA(h, grow(h->d_swfold, 2 * L));
    MRF_CUDA(h, dalloc(h->d_theta, (size_t)cap * h->C * h->W));
    if (use_partial(h)) MRF_CUDA(h, dalloc(h->d_part, (size_t)cap * h->C * 2 * L));
    h->E_cap = cap;
    return MRF_OK;
}

// Fresh free slots up to E_new: device endpoints -1, free in the host mirror.
mrf_status reserve_slots(mrf_t* h, int64_t E_new) {
    if (E_new <= h->E_slots) return MRF_OK;
    mrf_status st = grow_slots(h, E_new);
    if (st != MRF_OK) return st;
    const size_t n = (size_t)(E_new - h->E_slots);
    MRF_CUDA(h, cudaMemsetAsync(h->d_src + h->E_slots, 0xFF, n * sizeof(int32_t), h->stream));
    MRF_CUDA(h, cudaMemsetAsync(h->d_dst + h->E_slots, 0xFF, n * sizeof(int32_t), h->stream));
    h->h_src.resize((size_t)E_new, -1);
    h->h_dst.resize((size_t)E_new, -1);
    for (int64_t e = h->E_slots; e < E_new; ++e) h->free_slots.push_back(e);
    h->E_slots = E_new;
    h->sw_checked = false;
    h->hg_ready = false;
    drop_graphs(h);
    return MRF_OK;
}

// After device edits: endpoints, free slots, live count and largest degree of
// the host mirror read back from the device.
mrf_status sync_mirror(mrf_t* h) {
    if (!h->mirror_stale) return MRF_OK;
    const size_t E = (size_t)h->E_slots;
    h->h_src.resize(E);
    h->h_dst.resize(E);
    if (E) {
        MRF_CUDA(h, cudaMemcpyAsync(h->h_src.data(), h->d_src, E * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
        MRF_CUDA(h, cudaMemcpyAsync(h->h_dst.data(), h->d_dst, E * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    }
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    h->free_slots.clear();
    std::vector<int32_t> deg((size_t)h->N, 0);
    int64_t live = 0;
    for (size_t e = 0; e < E; ++e) {
        if (h->h_src[e] < 0) { h->free_slots.push_back((int64_t)e); continue; }
        ++live;
        ++deg[h->h_src[e]];
        ++deg[h->h_dst[e]];
    }
    h->E_live = live;
    h->max_deg = deg.empty() ? 0 : *std::max_element(deg.begin(), deg.end());
    h->mirror_stale = false;
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

mrf_status mrf_philox_rate(uint64_t threads, int32_t calls, void* cuda_stream, double* calls_per_s) {
    if (!threads || calls <= 0 || calls % 4 || !calls_per_s) return MRF_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    uint32_t* sink = nullptr;
    if (cudaMalloc(&sink, 1024 * sizeof(uint32_t)) != cudaSuccess) { cudaGetLastError(); return MRF_ENOMEM; }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0); cudaEventCreate(&e1);
    launch_philox_rate(threads, calls, sink, s);                 // warm
    cudaEventRecord(e0, s);
    launch_philox_rate(threads, calls, sink, s);
    cudaEventRecord(e1, s);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0); cudaEventDestroy(e1); cudaFree(sink);
    if (err != cudaSuccess) { cudaGetLastError(); return MRF_ECUDA; }
    *calls_per_s = (double)threads * calls / (ms / 1e3);
    return MRF_OK;
}

mrf_status mrf_set_kernel_timing(mrf_t* h, int32_t on) {
    if (!h) return MRF_EINVAL;
    h->opt.kernel_timing = on ? 1 : 0;
    return MRF_OK;
}

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
    dfree(h->d_theta); dfree(h->d_counts); dfree(h->d_lpv); dfree(h->d_logv); dfree(h->d_em); dfree(h->d_mfq); dfree(h->d_mfs); dfree(h->d_logp); dfree(h->d_ctl); dfree(h->d_flag); dfree(h->d_stage); dfree(h->d_pot); dfree(h->d_part);
    dfree(h->d_swt); dfree(h->d_swl); dfree(h->d_swfold); dfree(h->d_swut); dfree(h->d_swpar); dfree(h->d_swroot); dfree(h->d_swbits); dfree(h->d_swban); dfree(h->d_swlw); dfree(h->d_swerr); dfree(h->d_swchk);
    dfree(h->d_swufix); dfree(h->d_swell);
    dfree(h->d_hgT); dfree(h->d_hglb); dfree(h->d_hgtau); dfree(h->d_hgthr); dfree(h->d_hgtpl); dfree(h->d_hgfold);
    dfree(h->d_hgbound); dfree(h->d_hgut); dfree(h->d_hgutf);
    dfree(h->d_csr_work); dfree(h->d_csr_sums);
    dfree(h->d_ed_pair); dfree(h->d_ed_slots); dfree(h->d_ed_new); dfree(h->d_ed_s); dfree(h->d_ed_t);
    dfree(h->d_members); dfree(h->d_nmem); dfree(h->d_intra_ptr); dfree(h->d_intra); dfree(h->d_cf); dfree(h->d_skip);
    dfree(h->d_X); dfree(h->d_H1); dfree(h->d_H2); dfree(h->d_Z); dfree(h->d_w32); dfree(h->d_Wb); dfree(h->d_grad);
    dfree(h->d_m); dfree(h->d_v); dfree(h->d_train); dfree(h->d_bidx); dfree(h->d_bX); dfree(h->d_by); dfree(h->d_bn);
    dfree(h->d_dsX); dfree(h->d_dsy); dfree(h->d_dsn); dfree(h->d_loss); dfree(h->d_acc);
    dfree(h->d_W1x); dfree(h->d_cfb); dfree(h->d_rowbias); dfree(h->d_wimg); dfree(h->d_tc_err);
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
    h->mirror_stale = false;
    h->free_slots.clear();
    const bool want_resid = h->opt.grid_nx > 0 || h->opt.exact_edges;
    if (h->opt.grid_nx > 0 && !lattice_ok(h)) {
        h->has_factors = false;
        return fail(h, MRF_EINVAL, "options.grid set but the edges are not the lattice's in canonical order");
    }
    const size_t E = (size_t)n_edges;
    MRF_CUDA(h, dalloc(h->d_src, E)); MRF_CUDA(h, dalloc(h->d_dst, E));
    if ((uint64_t)E * h->C >= (1ull << 32)) return fail(h, MRF_ERANGE, "edges x chains must be below 2^32");
    MRF_CUDA(h, dalloc(h->d_tau, E * pad4(h->M))); MRF_CUDA(h, dalloc(h->d_thr, E * h->M));
    MRF_CUDA(h, dalloc(h->d_tpl, E * plane_words(h->M)));
    MRF_CUDA(h, dalloc(h->d_fold, E * 2 * L)); MRF_CUDA(h, dalloc(h->d_cst, E));
    if (want_resid) MRF_CUDA(h, dalloc(h->d_resid, E * L * L)); else dfree(h->d_resid);
    if (h->layout == MRF_LAYOUT_DIAG || L == 2) {
        MRF_CUDA(h, dalloc(h->d_swt, E * L)); MRF_CUDA(h, dalloc(h->d_swl, E * L)); MRF_CUDA(h, dalloc(h->d_swell, E * L));
    } else {
        dfree(h->d_swt); dfree(h->d_swl); dfree(h->d_swell);
    }
    h->hg_ready = false;
    if (L == 2) {
        MRF_CUDA(h, dalloc(h->d_swfold, E * 2 * L)); MRF_CUDA(h, dalloc(h->d_swut, (size_t)N * L));
    } else {
        dfree(h->d_swfold); dfree(h->d_swut);
    }
    h->sw_checked = false;
    MRF_CUDA(h, dalloc(h->d_theta, E * h->C * h->W));
    if (use_partial(h)) MRF_CUDA(h, dalloc(h->d_part, E * h->C * 2 * h->L));
    MRF_CUDA(h, to_device(h->d_src, h->h_src.data(), n_edges, MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, to_device(h->d_dst, h->h_dst.data(), n_edges, MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, build_csr(h));
    DecompArgs d{};
    d.L = L; d.M = h->M; d.layout = h->layout; d.n = n_edges; d.slots = nullptr; d.first_slot = 0;
    d.pair = d_pair; d.tau = h->d_tau; d.thr = h->d_thr; d.fold = h->d_fold; d.cst = h->d_cst; d.resid = h->d_resid;
    d.sw_thr = h->d_swt; d.sw_lw = h->d_swl; d.sw_fold = h->d_swfold; d.sw_ell = h->d_swell;
    MRF_CUDA(h, launch_decompose(d, h->stream));
    MRF_CUDA(h, launch_build_planes(h->d_thr, n_edges, nullptr, 0, h->M, h->d_tpl, h->stream));
    MRF_CUDA(h, launch_fold_unary(h->d_unary, h->d_fold, h->d_inc_ptr, h->d_inc, N, L, h->d_ut, h->d_utf, h->stream));
    if (h->d_swut)
        MRF_CUDA(h, launch_fold_unary(h->d_unary, h->d_swfold, h->d_inc_ptr, h->d_inc, N, L, h->d_swut, nullptr, h->stream));
    // log constant (for log-partition estimates): sum of per-edge constants
    std::vector<double> cst((size_t)n_edges);
    if (n_edges) MRF_CUDA(h, cudaMemcpyAsync(cst.data(), h->d_cst, E * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    h->log_const = std::accumulate(cst.begin(), cst.end(), 0.0);
    h->has_factors = true;
    h->schedule = 0;
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
    if (h->learned) return fail(h, MRF_ESTATE, "edits are not available once the learned proposal is set up");
    if (h->d_resid) return fail(h, MRF_ESTATE, "edits are not available with exact edge tables");
    mrf_status sst = sync_mirror(h);
    if (sst != MRF_OK) return sst;
    const int L = h->L, N = h->N;
    std::vector<int64_t> rem;
    std::vector<int32_t> as, at;
    MRF_CUDA(h, to_host(rem, edge_ids, n_remove, ptr_kind, h->stream));
    MRF_CUDA(h, to_host(as, src, n_add, ptr_kind, h->stream));
    MRF_CUDA(h, to_host(at, dst, n_add, ptr_kind, h->stream));
    std::vector<int64_t> rem_sorted = rem;
    std::sort(rem_sorted.begin(), rem_sorted.end());
    for (size_t i = 0; i < rem_sorted.size(); ++i) {
        const int64_t e = rem_sorted[i];
        if (e < 0 || e >= h->E_slots || h->h_src[e] < 0 || (i && rem_sorted[i - 1] == e))
            return fail(h, MRF_ERANGE, "edit: slot " + std::to_string(e) + " is not a live edge");
    }
    for (int64_t i = 0; i < n_add; ++i) {
        if (as[i] < 0 || as[i] >= N || at[i] < 0 || at[i] >= N) return fail(h, MRF_ERANGE, "edit: vertex id out of range");
        if (as[i] == at[i]) return fail(h, MRF_ERANGE, "edit: self-loop");
    }
    if (n_add * L * L > h->ed_pair_cap) {
        const int64_t cap = std::max<int64_t>(n_add * L * L, h->ed_pair_cap * 2);
        MRF_CUDA(h, dalloc(h->d_ed_pair, (size_t)cap));
        h->ed_pair_cap = cap;
    }
    float* d_pair = h->d_ed_pair;
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
    std::vector<int64_t> pool(h->free_slots.size() + rem_sorted.size());      // both sorted: merge
    std::merge(h->free_slots.begin(), h->free_slots.end(), rem_sorted.begin(), rem_sorted.end(), pool.begin());
    // new edges: freed slots in increasing order, then fresh slots
    std::vector<int64_t> slots((size_t)n_add);
    size_t used = 0;
    int64_t next = h->E_slots;
    for (int64_t i = 0; i < n_add; ++i) slots[i] = used < pool.size() ? pool[used++] : next++;
    h->free_slots.assign(pool.begin() + used, pool.end());
    const int64_t new_slots = next;
    if (new_slots > h->E_cap) {
        mrf_status gst = grow_slots(h, new_slots);
        if (gst != MRF_OK) return gst;
    }
    h->h_src.resize(new_slots, -1); h->h_dst.resize(new_slots, -1);
    for (int64_t i = 0; i < n_add; ++i) { h->h_src[slots[i]] = as[i]; h->h_dst[slots[i]] = at[i]; }
    // device: every touched slot gets its final endpoints from the host mirror
    // (a removed slot is usually reused by an added edge of the same edit)
    // (removed slots and new slots are both ascending: their union by a merge)
    std::vector<int64_t> upd_slot;
    upd_slot.reserve(rem_sorted.size() + slots.size());
    std::set_union(rem_sorted.begin(), rem_sorted.end(), slots.begin(), slots.end(), std::back_inserter(upd_slot));
    std::vector<int32_t> upd_s(upd_slot.size()), upd_t(upd_slot.size());
    for (size_t i = 0; i < upd_slot.size(); ++i) { upd_s[i] = h->h_src[upd_slot[i]]; upd_t[i] = h->h_dst[upd_slot[i]]; }
    const int64_t n_upd = (int64_t)upd_slot.size();
    if (n_upd > h->ed_cap || n_add > h->ed_cap) {
        const int64_t cap = std::max<int64_t>(std::max(n_upd, n_add), h->ed_cap * 2);
        MRF_CUDA(h, dalloc(h->d_ed_slots, (size_t)cap)); MRF_CUDA(h, dalloc(h->d_ed_new, (size_t)cap));
        MRF_CUDA(h, dalloc(h->d_ed_s, (size_t)cap)); MRF_CUDA(h, dalloc(h->d_ed_t, (size_t)cap));
        h->ed_cap = cap;
    }
    int64_t* d_slots = h->d_ed_slots;
    int64_t* d_new = h->d_ed_new;
    int32_t* d_us = h->d_ed_s;
    int32_t* d_ut2 = h->d_ed_t;
    MRF_CUDA(h, to_device(d_slots, upd_slot.data(), n_upd, MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, to_device(d_new, slots.data(), n_add, MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, to_device(d_us, upd_s.data(), n_upd, MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, to_device(d_ut2, upd_t.data(), n_upd, MRF_PTR_HOST, h->stream));
    if (new_slots > h->E_slots) {     // fresh slots start free on the device too
        std::vector<int32_t> neg((size_t)(new_slots - h->E_slots), -1);
        MRF_CUDA(h, to_device(h->d_src + h->E_slots, neg.data(), new_slots - h->E_slots, MRF_PTR_HOST, h->stream));
        MRF_CUDA(h, to_device(h->d_dst + h->E_slots, neg.data(), new_slots - h->E_slots, MRF_PTR_HOST, h->stream));
    }
    MRF_CUDA(h, launch_scatter_edges(d_slots, d_us, d_ut2, n_upd, h->d_src, h->d_dst, h->stream));
    h->E_slots = new_slots;
    h->E_live += n_add - n_remove;
    DecompArgs d{};
    d.L = L; d.M = h->M; d.layout = h->layout; d.n = n_add; d.slots = d_new;
    d.pair = d_pair; d.tau = h->d_tau; d.thr = h->d_thr; d.fold = h->d_fold; d.cst = h->d_cst; d.resid = nullptr;
    d.sw_thr = h->d_swt; d.sw_lw = h->d_swl; d.sw_fold = h->d_swfold; d.sw_ell = h->d_swell;
    h->sw_checked = false;
    h->hg_ready = false;
    MRF_CUDA(h, launch_decompose(d, h->stream));
    MRF_CUDA(h, launch_build_planes(h->d_thr, n_add, d_new, 0, h->M, h->d_tpl, h->stream));
    // incidence lists rebuilt on the device (host build if a site is very long)
    if (2 * h->E_live > h->inc_cap) {
        MRF_CUDA(h, dalloc(h->d_inc, (size_t)(2 * h->E_live + h->E_live / 4 + 64)));
        h->inc_cap = 2 * h->E_live + h->E_live / 4 + 64;
    }
    if (!h->d_csr_work) {
        MRF_CUDA(h, dalloc(h->d_csr_work, 2 * (size_t)N + 2));
        MRF_CUDA(h, dalloc(h->d_csr_sums, (size_t)((N + 1 + 1023) / 1024 + 2)));
    }
    MRF_CUDA(h, cudaMemsetAsync(h->d_flag, 0, sizeof(unsigned long long), h->stream));
    MRF_CUDA(h, build_csr_device(h->d_src, h->d_dst, h->E_slots, N, h->d_inc_ptr, h->d_inc, h->d_csr_work,
                                 h->d_csr_sums, h->d_flag, 512, h->stream));
    unsigned long long too_long = 0;
    MRF_CUDA(h, cudaMemcpyAsync(&too_long, h->d_flag, sizeof(too_long), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (too_long) {
        MRF_CUDA(h, build_csr(h));
        h->n_host_csr++;
    } else {
        h->n_device_csr++;
        unsigned md = 0;
        MRF_CUDA(h, cudaMemsetAsync(h->d_flag, 0, sizeof(unsigned long long), h->stream));
        MRF_CUDA(h, launch_max_degree(h->d_inc_ptr, N, reinterpret_cast<unsigned*>(h->d_flag), h->stream));
        MRF_CUDA(h, cudaMemcpyAsync(&md, h->d_flag, sizeof(md), cudaMemcpyDeviceToHost, h->stream));
        MRF_CUDA(h, cudaStreamSynchronize(h->stream));
        h->max_deg = (int32_t)md;
    }
    MRF_CUDA(h, launch_fold_unary(h->d_unary, h->d_fold, h->d_inc_ptr, h->d_inc, N, L, h->d_ut, h->d_utf, h->stream));
    if (h->d_swut)
        MRF_CUDA(h, launch_fold_unary(h->d_unary, h->d_swfold, h->d_inc_ptr, h->d_inc, N, L, h->d_swut, nullptr, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    std::copy(slots.begin(), slots.end(), out_new_ids);
    return MRF_OK;
}

// Autotuner for the plain primal schedule: with theta of the coming sweep in
// place, time the thread-per-(site, chain) and CTA-per-site kernels (each only
// rewrites the next label buffer from the same theta, so the chain state is
// unchanged) and keep the faster.  The boundary counter is restored after.
static mrf_status tune_schedule(mrf_t* h) {
    if (h->opt.schedule == 1 || h->opt.schedule == 2) { h->schedule = h->opt.schedule; return MRF_OK; }
    if (use_partial(h)) { h->schedule = 1; return MRF_OK; }         // one primal form only
    SweepArgs a = make_args(h);
    a.logp = nullptr;
    unsigned long long bnd = 0;
    MRF_CUDA(h, cudaMemcpyAsync(&bnd, &h->d_ctl->boundary, sizeof(bnd), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, launch_dual(a, h->layout, h->stream));
    cudaEvent_t e0 = take_event(h), e1 = take_event(h);
    for (int sched = 1; sched <= 2; ++sched) {
        // first (warm-up) launch timed alone: a schedule already 2x slower than
        // the thread schedule is not timed further
        float ms = 0.0f;
        MRF_CUDA(h, cudaEventRecord(e0, h->stream));
        MRF_CUDA(h, launch_primal(a, h->layout, sched, h->stream));
        MRF_CUDA(h, cudaEventRecord(e1, h->stream));
        MRF_CUDA(h, cudaEventSynchronize(e1));
        MRF_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
        if (sched == 2 && ms > 2.0f * h->tune_ms[0]) { h->tune_ms[1] = ms; break; }
        MRF_CUDA(h, cudaEventRecord(e0, h->stream));
        for (int r = 0; r < 3; ++r) MRF_CUDA(h, launch_primal(a, h->layout, sched, h->stream));
        MRF_CUDA(h, cudaEventRecord(e1, h->stream));
        MRF_CUDA(h, cudaEventSynchronize(e1));
        MRF_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
        h->tune_ms[sched - 1] = ms / 3.0f;
    }
    h->pool.push_back(e0); h->pool.push_back(e1);
    MRF_CUDA(h, cudaMemcpyAsync(&h->d_ctl->boundary, &bnd, sizeof(bnd), cudaMemcpyHostToDevice, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    h->schedule = h->tune_ms[1] < 0.9f * h->tune_ms[0] ? 2 : 1;
    return MRF_OK;
}

static bool use_mlp_tc(const mrf_t* h) { return h->opt.mlp_path == 0 && mlp_tc_supported(h->la); }

// Models small enough for k_sweep_small: at most 2^16 (site, chain) and
// (edge, chain) items, theta of all items within 200 KB of shared memory.
// Small models run several plain sweeps in one single-CTA launch (k_sweep_small,
// the additions of k_primal); handles on the edge-partial form keep it for
// every sweep, so that a chain does not depend on the sweeps per call.
static bool small_model(const mrf_t* h) {
    const int64_t nv = (int64_t)h->N * h->C, ne = h->E_slots * h->C;
    return nv <= 65536 && ne <= 65536 && ne * h->W * 4 <= 200 * 1024 && !use_partial(h);
}

static SwArgs make_sw_args(const mrf_t* h) {
    SwArgs w{};
    w.N = h->N; w.C = h->C; w.L = h->L; w.E = h->E_slots;
    w.src = h->d_src; w.dst = h->d_dst; w.thr = h->d_swt; w.lwe = h->d_swl; w.ufix = h->d_swufix;
    w.x = h->d_x; w.parent = h->d_swpar; w.root = h->d_swroot; w.bits = h->d_swbits; w.ban = h->d_swban; w.lw = h->d_swlw; w.err = h->d_swerr;
    w.ctl = h->d_ctl; w.rk = round_keys(h->key); w.fdC = FastDiv::make((uint32_t)h->C);
    w.lpv = h->lpv_on ? h->d_lpv : nullptr;
    w.counts = h->d_counts;
    return w;
}

// Before Swendsen-Wang sweeps: the model must have Potts-type (diagonal)
// tables with every l >= 0, and cluster weights must fit the fixed-point sum
// (checked once per factor change); the union-find buffers are allocated on
// first use.
static mrf_status sw_prepare(mrf_t* h) {
    {
        const mrf_status sst = sync_mirror(h);
        if (sst != MRF_OK) return sst;
    }
    // (a model without live edges has no tables to check: every cluster is one site)
    if (!h->d_swt && h->E_live > 0)
        return fail(h, MRF_EINVAL, "Swendsen-Wang sweeps need two labels or Potts-type tables (diagonal layout)");
    if (!h->sw_checked) {
        if (!h->d_swchk) MRF_CUDA(h, dalloc(h->d_swchk, 3));
        MRF_CUDA(h, cudaMemsetAsync(h->d_swchk, 0, 3 * sizeof(double), h->stream));
        MRF_CUDA(h, launch_sw_check(h->d_src, h->d_tau, h->E_slots, h->M, h->d_swl, h->L, h->d_unary, h->d_swut, h->N,
                                    h->d_swchk, h->stream));
        double chk[3] = {0.0, 0.0, 0.0};
        MRF_CUDA(h, cudaMemcpyAsync(chk, h->d_swchk, sizeof(chk), cudaMemcpyDeviceToHost, h->stream));
        MRF_CUDA(h, cudaStreamSynchronize(h->stream));
        if (chk[0] > 0.0) return fail(h, MRF_EINVAL, "Swendsen-Wang sweeps need ferromagnetic tables (w(x,x) >= 0)");
        if (chk[1] + chk[2] >= kSwFixMax)
            return fail(h, MRF_ERANGE, "Swendsen-Wang: summed |log weights| exceed the fixed-point range (2^30)");
        if (!h->d_swufix) { drop_graphs(h); MRF_CUDA(h, dalloc(h->d_swufix, (size_t)h->N * h->L)); }
        MRF_CUDA(h, launch_sw_fix_unary(h->d_unary, h->d_swut, (int64_t)h->N * h->L, h->d_swufix, h->stream));
        h->sw_checked = true;
    }
    const int64_t words = (h->E_slots * h->C + 31) / 32;       // edge slots grow with edits
    if (words > h->swbits_cap) {
        drop_graphs(h);
        MRF_CUDA(h, dalloc(h->d_swbits, (size_t)std::max<int64_t>(words, 1)));
        h->swbits_cap = words;
    }
    if (!h->d_swpar) {
        drop_graphs(h);
        const size_t NC = (size_t)h->N * h->C;
        MRF_CUDA(h, dalloc(h->d_swpar, NC)); MRF_CUDA(h, dalloc(h->d_swroot, NC)); MRF_CUDA(h, dalloc(h->d_swban, NC));
        MRF_CUDA(h, dalloc(h->d_swlw, NC * h->L)); MRF_CUDA(h, dalloc(h->d_swerr, 1));
        MRF_CUDA(h, cudaMemsetAsync(h->d_swerr, 0, sizeof(unsigned), h->stream));
        MRF_CUDA(h, launch_sw_reset(make_sw_args(h), h->stream));
    }
    return MRF_OK;
}

// After Swendsen-Wang sweeps: a union-find walk that exceeded its step bound
// left the between-sweeps state unrestored; it is reset and reported.
static mrf_status sw_check_error(mrf_t* h) {
    unsigned err = 0;
    MRF_CUDA(h, cudaMemcpyAsync(&err, h->d_swerr, sizeof(err), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (err) {
        MRF_CUDA(h, cudaMemsetAsync(h->d_swerr, 0, sizeof(unsigned), h->stream));
        MRF_CUDA(h, launch_sw_reset(make_sw_args(h), h->stream));
        return fail(h, MRF_ETIMEOUT, "Swendsen-Wang: a union-find walk exceeded its step bound");
    }
    return MRF_OK;
}

// Before Higdon sweeps: the Swendsen-Wang prerequisites, then the tables of
// the split at hg_rho (once per factor or rho change), the remainder's folded
// unaries and the range check that now includes the bits' fields.
static mrf_status hg_prepare(mrf_t* h) {
    {
        const mrf_status sst = sync_mirror(h);
        if (sst != MRF_OK) return sst;
    }
    mrf_status st = sw_prepare(h);
    if (st != MRF_OK) return st;
    if (!h->d_pot) { drop_graphs(h); MRF_CUDA(h, dalloc(h->d_pot, (size_t)h->N * h->L * h->C)); }
    if (h->hg_ready) return MRF_OK;
    if (h->E_live > 0 && !h->d_swell) return fail(h, MRF_EINVAL, "Higdon sweeps need two labels or Potts-type tables");
    const int L = h->L;
    const int64_t E = h->E_slots;
    if (h->hg_cap < E || !h->d_hgut) {
        drop_graphs(h);
        const size_t cap = (size_t)std::max<int64_t>(E, 1);
        MRF_CUDA(h, dalloc(h->d_hgT, cap * L)); MRF_CUDA(h, dalloc(h->d_hglb, cap * L));
        MRF_CUDA(h, dalloc(h->d_hgtau, cap * pad4(L))); MRF_CUDA(h, dalloc(h->d_hgthr, cap * L));
        MRF_CUDA(h, dalloc(h->d_hgtpl, cap * plane_words(L))); MRF_CUDA(h, dalloc(h->d_hgfold, cap * 2 * L));
        MRF_CUDA(h, dalloc(h->d_hgbound, cap));
        MRF_CUDA(h, dalloc(h->d_hgut, (size_t)h->N * L)); MRF_CUDA(h, dalloc(h->d_hgutf, (size_t)h->N * L));
        h->hg_cap = (int64_t)cap;
    }
    HigdonTables t{h->d_hgT, h->d_hglb, h->d_hgtau, h->d_hgthr, h->d_hgfold, h->d_hgbound};
    MRF_CUDA(h, launch_hg_tables(h->d_src, h->d_swell, E, L, h->hg_rho, t, h->stream));
    MRF_CUDA(h, launch_build_planes(h->d_hgthr, E, nullptr, 0, L, h->d_hgtpl, h->stream));
    // the remainder's unaries: the Swendsen-Wang unaries plus A's Theorem-2 terms of every edge
    MRF_CUDA(h, launch_fold_unary(h->d_unary, h->d_hgfold, h->d_inc_ptr, h->d_inc, h->N, L, h->d_hgut, h->d_hgutf,
                                  h->stream, h->d_swut));
    MRF_CUDA(h, cudaMemsetAsync(h->d_swchk, 0, sizeof(double), h->stream));
    MRF_CUDA(h, launch_hg_check(h->d_hgut, h->N, L, h->d_src, h->d_hgbound, E, h->d_swchk, h->stream));
    double bound = 0.0;
    MRF_CUDA(h, cudaMemcpyAsync(&bound, h->d_swchk, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (bound >= kSwFixMax)
        return fail(h, MRF_ERANGE, "Higdon: summed |log weights| exceed the fixed-point range (2^30)");
    h->hg_ready = true;
    return MRF_OK;
}

// Arguments of Higdon's sweep: the remainder's tables in the dual and
// potential kernels, the bond tables and per-chain potentials in the cluster
// kernels.
static void make_hg_args(const mrf_t* h, SweepArgs& d, SwArgs& w) {
    w = make_sw_args(h);
    w.thr = h->d_hgT; w.lwe = h->d_hglb; w.pot = h->d_pot;
    d = make_args(h);
    d.M = h->L; d.W = 1; d.tau = h->d_hgtau; d.thr = h->d_hgthr; d.tpl = h->d_hgtpl;
    d.utf = h->d_hgutf; d.ut = h->d_hgut; d.logp = nullptr; d.lpv = nullptr;
    d.pot = h->d_pot;
}

static mrf_status enqueue_sweep(mrf_t* h, int mode) {
    SweepArgs a = make_args(h);
    cudaStream_t s = h->stream;
    cudaError_t e = cudaSuccess;
    if (mode == MRF_MODE_PLAIN && use_partial(h)) {
        e = timed(h, MRF_K_DUAL, [&] { return launch_dual(a, h->layout, s); });
        if (e == cudaSuccess) e = timed(h, MRF_K_PARTIAL, [&] { return launch_sweep_partial(a, h->layout, 0, s); });
        if (e == cudaSuccess) e = timed(h, MRF_K_PRIMAL, [&] { return launch_sweep_partial(a, h->layout, 1, s); });
    } else if (mode == MRF_MODE_PLAIN) {
        e = timed(h, MRF_K_DUAL, [&] { return launch_dual(a, h->layout, s); });
        if (e == cudaSuccess) e = timed(h, MRF_K_PRIMAL, [&] { return launch_primal(a, h->layout, h->schedule, s); });
    } else if (mode == MRF_MODE_FUSED) {
        e = timed(h, MRF_K_FUSED, [&] { return launch_fused(a, h->layout, h->opt.schedule, s); });
    } else if (mode == MRF_MODE_SW) {
        const SwArgs w = make_sw_args(h);
        e = timed(h, MRF_K_SW_BOND, [&] { return launch_sw_bond(w, s); });
        if (e == cudaSuccess) e = timed(h, MRF_K_SW_FLATTEN, [&] { return launch_sw_flatten(w, s); });
        if (e == cudaSuccess) e = timed(h, MRF_K_SW_DRAW, [&] { return launch_sw_draw(w, s); });
    } else if (mode == MRF_MODE_HIGDON) {
        // bonds (and their unions), A's bits of the other edges, the bits'
        // potentials, then the clusters as in the Swendsen-Wang sweep
        SweepArgs d;
        SwArgs w;
        make_hg_args(h, d, w);
        e = timed(h, MRF_K_SW_BOND, [&] { return launch_sw_bond(w, s); });
        if (e == cudaSuccess) e = timed(h, MRF_K_DUAL, [&] {
            const cudaError_t e2 = launch_dual(d, MRF_LAYOUT_DIAG, s);
            return e2 != cudaSuccess ? e2 : launch_hg_clear(w.bits, d.theta, h->E_slots * h->C, s);
        });
        if (e == cudaSuccess) e = timed(h, MRF_K_POTENTIAL, [&] { return launch_potential(d, MRF_LAYOUT_DIAG, s); });
        if (e == cudaSuccess) e = timed(h, MRF_K_SW_FLATTEN, [&] { return launch_sw_flatten(w, s); });
        if (e == cudaSuccess) e = timed(h, MRF_K_SW_DRAW, [&] { return launch_sw_draw(w, s); });
    } else if (mode == MRF_MODE_LEARNED) {
        a.skip = h->d_skip;
        e = timed(h, MRF_K_DUAL, [&] { return launch_dual(a, h->layout, s); });
        if (e == cudaSuccess) e = timed(h, MRF_K_POTENTIAL, [&] { return launch_potential(a, h->layout, s); });
        if (e == cudaSuccess) e = timed(h, MRF_K_FEATURES, [&] { return launch_learned_features(h->la, a, s); });
        if (e == cudaSuccess)
            e = timed(h, MRF_K_MLP, [&] {
                return use_mlp_tc(h) ? launch_learned_mlp_tc(h->la, s) : launch_learned_mlp_blocks(h->la, s);
            });
        if (e == cudaSuccess) e = timed(h, MRF_K_MH, [&] { return launch_learned_mh(h->la, a, s); });
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
    if (n_sweeps < 0 || mode < MRF_MODE_PLAIN || mode > MRF_MODE_HIGDON) return fail(h, MRF_EINVAL, "bad sweep count or mode");
    if (mode == MRF_MODE_HIGDON) {
        mrf_status st = hg_prepare(h);
        if (st != MRF_OK) return st;
        // small models: all the sweeps in one single-CTA launch, state and bits in shared memory
        SweepArgs d;
        SwArgs w;
        make_hg_args(h, d, w);
        if (n_sweeps >= 2 && (int64_t)h->N * h->C <= 65536 && h->E_slots * h->C <= 65536 &&
            hg_small_smem(w) <= 200 * 1024) {
            MRF_CUDA(h, timed(h, MRF_K_SW_SMALL, [&] { return launch_hg_small(d, w, n_sweeps, h->stream); }));
            h->sweep_host += n_sweeps;
            return sw_check_error(h);
        }
    }
    if (mode == MRF_MODE_SW) {
        mrf_status st = sw_prepare(h);
        if (st != MRF_OK) return st;
        // small models: all the sweeps in one single-CTA launch, state in shared memory
        const SwArgs w = make_sw_args(h);
        if (n_sweeps >= 2 && (int64_t)h->N * h->C <= 65536 && h->E_slots * h->C <= 65536 &&
            sw_small_smem(w) <= 200 * 1024) {
            MRF_CUDA(h, timed(h, MRF_K_SW_SMALL, [&] { return launch_sw_small(w, n_sweeps, h->stream); }));
            h->sweep_host += n_sweeps;
            return sw_check_error(h);
        }
    }
    if (mode == MRF_MODE_LEARNED && !h->learned) return fail(h, MRF_ESTATE, "learned mode needs mrf_learned_setup");
    if (mode == MRF_MODE_LEARNED && h->mlp_unusable)
        return fail(h, MRF_ESTATE, "tensor-core MLP did not drain after a timeout; recreate the handle");
    if (mode == MRF_MODE_LEARNED && h->rowbias_dirty) {      // per-block first-layer bias of the current weights
        MRF_CUDA(h, learned_rowbias(h->la, h->stream));
        h->rowbias_dirty = false;
    }
    if (mode == MRF_MODE_SPLASH && h->opt.grid_nx <= 0) return fail(h, MRF_ESTATE, "splash mode needs options.grid");
    if (mode == MRF_MODE_SPLASH && !h->d_pot) {
        drop_graphs(h);
        MRF_CUDA(h, dalloc(h->d_pot, (size_t)h->N * h->L * h->C));
    }
    if (mode == MRF_MODE_PLAIN && h->schedule == 0 && n_sweeps > 0) {
        mrf_status st = tune_schedule(h);
        if (st != MRF_OK) return st;
    }
    // small models: all the sweeps in one single-CTA launch (launch latency dominates there)
    if (mode == MRF_MODE_PLAIN && n_sweeps >= 2 && small_model(h)) {
        const SweepArgs a = make_args(h);
        MRF_CUDA(h, timed(h, MRF_K_SMALL, [&] { return launch_sweep_small(a, h->layout, n_sweeps, h->stream); }));
        h->sweep_host += n_sweeps;
        return MRF_OK;
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
    if ((mode == MRF_MODE_SW || mode == MRF_MODE_HIGDON) && n_sweeps > 0) {
        mrf_status st = sw_check_error(h);
        if (st != MRF_OK) return st;
    }
    if (mode == MRF_MODE_LEARNED) {
        h->proposed += (uint64_t)n_sweeps * h->la.nb * h->C;
        if (use_mlp_tc(h) && n_sweeps > 0) {                 // a bounded wait of the tensor-core MLP gave up
            unsigned err = 0;
            MRF_CUDA(h, cudaMemcpyAsync(&err, h->d_tc_err, sizeof(err), cudaMemcpyDeviceToHost, h->stream));
            MRF_CUDA(h, cudaStreamSynchronize(h->stream));
            if (h->la.tc_inject_timeout) { h->la.tc_inject_timeout = 0; drop_graphs(h); }
            if (err & 2u) {
                h->mlp_unusable = true;
                return fail(h, MRF_ESTATE, "tensor-core MLP: a wait timed out and its work did not drain; "
                                           "recreate the handle");
            }
            if (err) {
                MRF_CUDA(h, cudaMemsetAsync(h->d_tc_err, 0, sizeof(unsigned), h->stream));
                return fail(h, MRF_ETIMEOUT, "tensor-core MLP: a wait timed out");
            }
        }
    }
    return MRF_OK;
}

static mrf_status estimate_log_partition(mrf_t* h, int32_t n_sweeps, int mode, double* log_v) {
    if (!h || n_sweeps < 0 || (n_sweeps > 0 && !log_v)) return MRF_EINVAL;
    if (!h->has_factors) return fail(h, MRF_ESTATE, "mrf_set_factors first");
    if (!h->d_resid) return fail(h, MRF_ESTATE, "the estimator needs exact edge tables (options.grid or options.exact_edges)");
    if (n_sweeps == 0) return MRF_OK;
    if (mode == MRF_MODE_SW || mode == MRF_MODE_HIGDON) {
        mrf_status st = mode == MRF_MODE_SW ? sw_prepare(h) : hg_prepare(h);
        if (st != MRF_OK) return st;
    } else if (h->schedule == 0) {
        mrf_status st = tune_schedule(h);
        if (st != MRF_OK) return st;
    }
    if (!h->d_lpv) MRF_CUDA(h, dalloc(h->d_lpv, (size_t)h->N * h->C));
    if ((int64_t)n_sweeps * h->C > h->logv_cap) {
        MRF_CUDA(h, dalloc(h->d_logv, (size_t)n_sweeps * h->C));
        h->logv_cap = (int64_t)n_sweeps * h->C;
    }
    MRF_CUDA(h, cudaMemsetAsync(h->d_logv, 0, sizeof(double) * (size_t)n_sweeps * h->C, h->stream));
    h->lpv_on = true;
    mrf_status st = MRF_OK;
    for (int i = 0; i < n_sweeps && st == MRF_OK; ++i) {
        st = enqueue_sweep(h, mode);                            // not from a graph: the launches carry lpv
        if (st == MRF_OK) {
            cudaError_t e = launch_log_v(make_args(h), h->d_ut, h->d_logv + (int64_t)i * h->C, h->stream);
            if (e != cudaSuccess) { cudaGetLastError(); st = fail(h, MRF_ECUDA, std::string("log V: ") + cudaGetErrorString(e)); }
        }
        if (st == MRF_OK) h->sweep_host++;
    }
    h->lpv_on = false;
    if (st != MRF_OK) return st;
    MRF_CUDA(h, cudaMemcpyAsync(log_v, h->d_logv, sizeof(double) * (size_t)n_sweeps * h->C, cudaMemcpyDeviceToHost,
                                h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (mode == MRF_MODE_SW || mode == MRF_MODE_HIGDON) return sw_check_error(h);
    return MRF_OK;
}

mrf_status mrf_set_higdon(mrf_t* h, double rho) {
    if (!h) return MRF_EINVAL;
    if (!(rho >= 0.0 && rho <= 1.0)) return fail(h, MRF_EINVAL, "Higdon's fraction rho must lie in [0, 1]");
    if (rho != h->hg_rho) { h->hg_rho = rho; h->hg_ready = false; drop_graphs(h); }
    return MRF_OK;
}

mrf_status mrf_estimate_log_partition(mrf_t* h, int32_t n_sweeps, double* log_v) {
    return estimate_log_partition(h, n_sweeps, MRF_MODE_PLAIN, log_v);
}

mrf_status mrf_estimate_log_partition_sw(mrf_t* h, int32_t n_sweeps, double* log_v) {
    return estimate_log_partition(h, n_sweeps, MRF_MODE_SW, log_v);
}

mrf_status mrf_estimate_log_partition_higdon(mrf_t* h, int32_t n_sweeps, double* log_v) {
    return estimate_log_partition(h, n_sweeps, MRF_MODE_HIGDON, log_v);
}

mrf_status mrf_map_em(mrf_t* h, int32_t n_iters, uint8_t* labels, int32_t ptr_kind) {
    if (!h || !labels || n_iters < 0) return MRF_EINVAL;
    if (!h->has_factors) return fail(h, MRF_ESTATE, "mrf_set_factors first");
    const size_t NC = (size_t)h->N * h->C;
    if (!h->d_stage) MRF_CUDA(h, dalloc(h->d_stage, NC));
    if (!h->d_em) MRF_CUDA(h, dalloc(h->d_em, 2 * NC));
    MRF_CUDA(h, to_device(h->d_stage, labels, (int64_t)NC, ptr_kind, h->stream));
    MRF_CUDA(h, cudaMemsetAsync(h->d_flag, 0, sizeof(unsigned long long), h->stream));
    MRF_CUDA(h, launch_count_ge(h->d_stage, (int64_t)NC, h->L, h->d_flag, h->stream));
    unsigned long long bad = 0;
    MRF_CUDA(h, cudaMemcpyAsync(&bad, h->d_flag, sizeof(bad), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (bad) return fail(h, MRF_ERANGE, "label out of range");
    MRF_CUDA(h, launch_labels_from_abi(h->d_stage, h->d_em, h->N, h->C, h->stream));
    const SweepArgs a = make_args(h);
    for (int i = 0; i < n_iters; ++i)
        MRF_CUDA(h, launch_em(a, h->layout, h->d_em + (i & 1) * NC, h->d_em + ((i + 1) & 1) * NC, h->stream));
    MRF_CUDA(h, launch_labels_to_abi(h->d_em + (n_iters & 1) * NC, h->d_stage, h->N, h->C, h->stream));
    MRF_CUDA(h, cudaMemcpyAsync(labels, h->d_stage, NC,
                                ptr_kind == MRF_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    return MRF_OK;
}

mrf_status mrf_map_em_blocked(mrf_t* h, int32_t n_iters, uint8_t* labels, int32_t ptr_kind) {
    if (!h || !labels || n_iters < 0) return MRF_EINVAL;
    if (!h->has_factors) return fail(h, MRF_ESTATE, "mrf_set_factors first");
    if (h->opt.grid_nx <= 0 || !h->d_resid) return fail(h, MRF_ESTATE, "blocked EM needs options.grid");
    const size_t NC = (size_t)h->N * h->C;
    if (!h->d_stage) MRF_CUDA(h, dalloc(h->d_stage, NC));
    if (!h->d_em) MRF_CUDA(h, dalloc(h->d_em, 2 * NC));
    if (!h->d_pot) { drop_graphs(h); MRF_CUDA(h, dalloc(h->d_pot, (size_t)h->N * h->L * h->C)); }
    MRF_CUDA(h, to_device(h->d_stage, labels, (int64_t)NC, ptr_kind, h->stream));
    MRF_CUDA(h, cudaMemsetAsync(h->d_flag, 0, sizeof(unsigned long long), h->stream));
    MRF_CUDA(h, launch_count_ge(h->d_stage, (int64_t)NC, h->L, h->d_flag, h->stream));
    unsigned long long bad = 0;
    MRF_CUDA(h, cudaMemcpyAsync(&bad, h->d_flag, sizeof(bad), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (bad) return fail(h, MRF_ERANGE, "label out of range");
    MRF_CUDA(h, launch_labels_from_abi(h->d_stage, h->d_em, h->N, h->C, h->stream));
    SweepArgs a = make_args(h);
    a.splash = 1;
    for (int i = 0; i < n_iters; ++i) {
        // block offset of iteration i, potentials from the expected non-tree duals, tree MAP
        MRF_CUDA(h, launch_splash_offset(a, h->stream, i));
        MRF_CUDA(h, launch_em_pot(a, h->layout, h->d_em + (i & 1) * NC, h->stream));
        MRF_CUDA(h, launch_tree_map(a, h->d_em + ((i + 1) & 1) * NC, h->stream));
    }
    MRF_CUDA(h, launch_labels_to_abi(h->d_em + (n_iters & 1) * NC, h->d_stage, h->N, h->C, h->stream));
    MRF_CUDA(h, cudaMemcpyAsync(labels, h->d_stage, NC,
                                ptr_kind == MRF_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    return MRF_OK;
}

mrf_status mrf_mean_field(mrf_t* h, int32_t n_iters, float* marginals, int32_t ptr_kind) {
    if (!h || !marginals || n_iters < 0) return MRF_EINVAL;
    if (!h->has_factors) return fail(h, MRF_ESTATE, "mrf_set_factors first");
    const size_t n = (size_t)h->N * h->L * h->C;
    if (!h->d_mfq) MRF_CUDA(h, dalloc(h->d_mfq, 2 * n));
    if (!h->d_mfs) MRF_CUDA(h, dalloc(h->d_mfs, n));
    MRF_CUDA(h, to_device(h->d_mfs, marginals, (int64_t)n, ptr_kind, h->stream));
    mrf_status st = check_finite_device(h, h->d_mfs, (int64_t)n, "marginals");
    if (st != MRF_OK) return st;
    MRF_CUDA(h, launch_marg_layout(h->d_mfs, h->d_mfq, h->N, h->L, h->C, false, h->stream));
    const SweepArgs a = make_args(h);
    for (int i = 0; i < n_iters; ++i)
        MRF_CUDA(h, launch_mf(a, h->layout, h->d_mfq + (i & 1) * n, h->d_mfq + ((i + 1) & 1) * n, h->stream));
    MRF_CUDA(h, launch_marg_layout(h->d_mfq + (n_iters & 1) * n, h->d_mfs, h->N, h->L, h->C, true, h->stream));
    MRF_CUDA(h, cudaMemcpyAsync(marginals, h->d_mfs, n * sizeof(float),
                                ptr_kind == MRF_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    return MRF_OK;
}

mrf_status mrf_mean_field_blocked(mrf_t* h, int32_t n_iters, float* marginals, int32_t ptr_kind) {
    if (!h || !marginals || n_iters < 0) return MRF_EINVAL;
    if (!h->has_factors) return fail(h, MRF_ESTATE, "mrf_set_factors first");
    if (h->opt.grid_nx <= 0 || !h->d_resid) return fail(h, MRF_ESTATE, "blocked mean field needs options.grid");
    const size_t n = (size_t)h->N * h->L * h->C;
    if (!h->d_mfq) MRF_CUDA(h, dalloc(h->d_mfq, 2 * n));
    if (!h->d_mfs) MRF_CUDA(h, dalloc(h->d_mfs, n));
    if (!h->d_pot) { drop_graphs(h); MRF_CUDA(h, dalloc(h->d_pot, (size_t)h->N * h->L * h->C)); }
    MRF_CUDA(h, to_device(h->d_mfs, marginals, (int64_t)n, ptr_kind, h->stream));
    mrf_status st = check_finite_device(h, h->d_mfs, (int64_t)n, "marginals");
    if (st != MRF_OK) return st;
    MRF_CUDA(h, launch_marg_layout(h->d_mfs, h->d_mfq, h->N, h->L, h->C, false, h->stream));
    SweepArgs a = make_args(h);
    a.splash = 1;
    for (int i = 0; i < n_iters; ++i) {
        // block offset of iteration i, potentials of the expected non-forest duals, forest marginals
        MRF_CUDA(h, launch_splash_offset(a, h->stream, i));
        MRF_CUDA(h, launch_mf_pot(a, h->layout, h->d_mfq + (i & 1) * n, h->stream));
        MRF_CUDA(h, launch_tree_marginals(a, h->d_mfq + ((i + 1) & 1) * n, h->stream));
    }
    MRF_CUDA(h, launch_marg_layout(h->d_mfq + (n_iters & 1) * n, h->d_mfs, h->N, h->L, h->C, true, h->stream));
    MRF_CUDA(h, cudaMemcpyAsync(marginals, h->d_mfs, n * sizeof(float),
                                ptr_kind == MRF_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    return MRF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------- checkpoints

namespace {

constexpr char kCkptMagic[8] = {'M', 'R', 'F', 'C', 'K', 'P', 'T', '2'};   // 2: Swendsen-Wang tables

struct CkptHeader {
    int32_t N, L, C, layout, M, W;
    int64_t E_live, E_slots, n_free, sweep_host, count_from_host;
    uint64_t seed;
    double log_const;
    int32_t has_resid, has_sw;
    double hg_rho;                     // fraction of Higdon's sweep
    mrf_options opt;
    Ctl ctl;
};

template <typename T>
bool write_dev(FILE* f, const T* d, size_t n, std::vector<uint8_t>& buf, cudaStream_t s) {
    if (n == 0) return true;
    buf.resize(n * sizeof(T));
    if (cudaMemcpyAsync(buf.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
    if (cudaStreamSynchronize(s) != cudaSuccess) return false;
    return fwrite(buf.data(), 1, buf.size(), f) == buf.size();
}

template <typename T>
bool read_dev(FILE* f, T* d, size_t n, std::vector<uint8_t>& buf, cudaStream_t s) {
    if (n == 0) return true;
    buf.resize(n * sizeof(T));
    if (fread(buf.data(), 1, buf.size(), f) != buf.size()) return false;
    if (cudaMemcpyAsync(d, buf.data(), buf.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) return false;
    return cudaStreamSynchronize(s) == cudaSuccess;
}

}  // namespace

extern "C" {

mrf_status mrf_save(mrf_t* h, const char* path) {
    if (!h || !path) return MRF_EINVAL;
    if (!h->has_factors) return fail(h, MRF_ESTATE, "mrf_set_factors first");
    mrf_status sst = sync_mirror(h);
    if (sst != MRF_OK) return sst;
    CkptHeader hd{};
    hd.N = h->N; hd.L = h->L; hd.C = h->C; hd.layout = h->layout; hd.M = h->M; hd.W = h->W;
    hd.E_live = h->E_live; hd.E_slots = h->E_slots; hd.n_free = (int64_t)h->free_slots.size();
    hd.sweep_host = h->sweep_host; hd.count_from_host = h->count_from_host; hd.seed = h->seed; hd.log_const = h->log_const;
    hd.has_resid = h->d_resid ? 1 : 0;
    hd.has_sw = (h->d_swt ? 1 : 0) | (h->d_swfold ? 2 : 0);
    hd.hg_rho = h->hg_rho;
    hd.opt = h->opt;
    MRF_CUDA(h, cudaMemcpyAsync(&hd.ctl, h->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    FILE* f = fopen(path, "wb");
    if (!f) return fail(h, MRF_EINVAL, std::string("cannot open ") + path + " for writing");
    const size_t NL = (size_t)h->N * h->L, E = (size_t)h->E_slots, L = (size_t)h->L;
    std::vector<uint8_t> buf;
    bool ok = fwrite(kCkptMagic, 1, 8, f) == 8 && fwrite(&hd, sizeof(hd), 1, f) == 1;
    ok = ok && write_dev(f, h->d_unary, NL, buf, h->stream) && write_dev(f, h->d_ut, NL, buf, h->stream) &&
         write_dev(f, h->d_utf, NL, buf, h->stream);
    ok = ok && (E == 0 || (fwrite(h->h_src.data(), sizeof(int32_t), E, f) == E && fwrite(h->h_dst.data(), sizeof(int32_t), E, f) == E));
    ok = ok && write_dev(f, h->d_tau, E * pad4(h->M), buf, h->stream) && write_dev(f, h->d_thr, E * h->M, buf, h->stream) &&
         write_dev(f, h->d_tpl, E * plane_words(h->M), buf, h->stream) && write_dev(f, h->d_fold, E * 2 * L, buf, h->stream) &&
         write_dev(f, h->d_cst, E, buf, h->stream);
    if (hd.has_resid) ok = ok && write_dev(f, h->d_resid, E * L * L, buf, h->stream);
    if (hd.has_sw & 1) ok = ok && write_dev(f, h->d_swt, E * L, buf, h->stream) && write_dev(f, h->d_swl, E * L, buf, h->stream) &&
                          write_dev(f, h->d_swell, E * L, buf, h->stream);
    if (hd.has_sw & 2) ok = ok && write_dev(f, h->d_swfold, E * 2 * L, buf, h->stream);
    ok = ok && write_dev(f, h->d_x, 2 * (size_t)h->N * h->C, buf, h->stream) && write_dev(f, h->d_counts, NL, buf, h->stream);
    ok = ok && (hd.n_free == 0 || fwrite(h->free_slots.data(), sizeof(int64_t), (size_t)hd.n_free, f) == (size_t)hd.n_free);
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(h, MRF_ECUDA, std::string("writing ") + path + " failed");
    return MRF_OK;
}

mrf_status mrf_load(mrf_t** out, const char* path, void* cuda_stream) {
    if (!out || !path) return MRF_EINVAL;
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return MRF_EINVAL;
    char magic[8];
    CkptHeader hd{};
    if (fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kCkptMagic, 8) != 0 || fread(&hd, sizeof(hd), 1, f) != 1 ||
        hd.E_slots < 0 || hd.E_live < 0 || hd.E_live > hd.E_slots || hd.n_free < 0 || hd.M != n_entries(hd.L, hd.layout)) {
        fclose(f);
        return MRF_EINVAL;
    }
    mrf_t* h = nullptr;
    mrf_status st = mrf_create(&h, hd.N, hd.L, hd.C, hd.seed, &hd.opt, cuda_stream);
    if (st != MRF_OK) { fclose(f); return st; }
    auto bail = [&](mrf_status code) { fclose(f); mrf_destroy(h); return code; };
    h->layout = hd.layout; h->M = hd.M; h->W = hd.W;
    h->E_live = hd.E_live; h->E_slots = h->E_cap = hd.E_slots;
    h->mirror_stale = false;
    const size_t NL = (size_t)h->N * h->L, E = (size_t)hd.E_slots, L = (size_t)h->L;
    if ((uint64_t)E * h->C >= (1ull << 32)) return bail(MRF_ERANGE);
    std::vector<uint8_t> buf;
    bool ok = read_dev(f, h->d_unary, NL, buf, h->stream) && read_dev(f, h->d_ut, NL, buf, h->stream) &&
              read_dev(f, h->d_utf, NL, buf, h->stream);
    h->h_src.resize(E); h->h_dst.resize(E);
    ok = ok && (E == 0 || (fread(h->h_src.data(), sizeof(int32_t), E, f) == E && fread(h->h_dst.data(), sizeof(int32_t), E, f) == E));
    for (size_t e = 0; ok && e < E; ++e)
        if (h->h_src[e] >= h->N || h->h_dst[e] >= h->N || (h->h_src[e] < 0) != (h->h_dst[e] < 0)) ok = false;
    if (!ok) return bail(MRF_EINVAL);
    if (dalloc(h->d_src, E) || dalloc(h->d_dst, E) || dalloc(h->d_tau, E * pad4(h->M)) || dalloc(h->d_thr, E * h->M) ||
        dalloc(h->d_tpl, E * plane_words(h->M)) || dalloc(h->d_fold, E * 2 * L) || dalloc(h->d_cst, E) ||
        (hd.has_resid && dalloc(h->d_resid, E * L * L)) || ((hd.has_sw & 1) && (dalloc(h->d_swt, E * L) || dalloc(h->d_swl, E * L) || dalloc(h->d_swell, E * L))) ||
        ((hd.has_sw & 2) && (dalloc(h->d_swfold, E * 2 * L) || dalloc(h->d_swut, NL))) ||
        dalloc(h->d_theta, E * h->C * h->W) || (use_partial(h) && dalloc(h->d_part, E * h->C * 2 * L))) {
        cudaGetLastError();
        return bail(MRF_ENOMEM);
    }
    ok = to_device(h->d_src, h->h_src.data(), (int64_t)E, MRF_PTR_HOST, h->stream) == cudaSuccess &&
         to_device(h->d_dst, h->h_dst.data(), (int64_t)E, MRF_PTR_HOST, h->stream) == cudaSuccess;
    ok = ok && read_dev(f, h->d_tau, E * pad4(h->M), buf, h->stream) && read_dev(f, h->d_thr, E * h->M, buf, h->stream) &&
         read_dev(f, h->d_tpl, E * plane_words(h->M), buf, h->stream) && read_dev(f, h->d_fold, E * 2 * L, buf, h->stream) &&
         read_dev(f, h->d_cst, E, buf, h->stream);
    if (hd.has_resid) ok = ok && read_dev(f, h->d_resid, E * L * L, buf, h->stream);
    if (hd.has_sw & 1) ok = ok && read_dev(f, h->d_swt, E * L, buf, h->stream) && read_dev(f, h->d_swl, E * L, buf, h->stream) &&
                          read_dev(f, h->d_swell, E * L, buf, h->stream);
    if (hd.has_sw & 2) ok = ok && read_dev(f, h->d_swfold, E * 2 * L, buf, h->stream);
    ok = ok && read_dev(f, h->d_x, 2 * (size_t)h->N * h->C, buf, h->stream) && read_dev(f, h->d_counts, NL, buf, h->stream);
    h->free_slots.resize((size_t)hd.n_free);
    ok = ok && (hd.n_free == 0 || fread(h->free_slots.data(), sizeof(int64_t), (size_t)hd.n_free, f) == (size_t)hd.n_free);
    if (!ok) return bail(MRF_EINVAL);
    fclose(f);
    if (build_csr(h) != cudaSuccess ||
        (h->d_swut && launch_fold_unary(h->d_unary, h->d_swfold, h->d_inc_ptr, h->d_inc, h->N, h->L, h->d_swut,
                                        nullptr, h->stream) != cudaSuccess)) {
        cudaGetLastError();
        mrf_destroy(h);
        return MRF_ECUDA;
    }
    // labels index per-label tables in every kernel: a file with a label >= L is rejected
    unsigned long long bad_labels = 1;
    if (cudaMemsetAsync(h->d_flag, 0, sizeof(unsigned long long), h->stream) != cudaSuccess ||
        launch_count_ge(h->d_x, 2 * (int64_t)h->N * h->C, h->L, h->d_flag, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(&bad_labels, h->d_flag, sizeof(bad_labels), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        mrf_destroy(h);
        return MRF_ECUDA;
    }
    if (bad_labels) { mrf_destroy(h); return MRF_EINVAL; }
    if (cudaMemcpyAsync(h->d_ctl, &hd.ctl, sizeof(Ctl), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        mrf_destroy(h);
        return MRF_ECUDA;
    }
    h->sweep_host = hd.sweep_host;
    h->count_from_host = hd.count_from_host;
    h->hg_rho = (hd.hg_rho >= 0.0 && hd.hg_rho <= 1.0) ? hd.hg_rho : 0.5;
    h->log_const = hd.log_const;
    h->has_factors = true;
    h->schedule = 0;
    *out = h;
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
    if (h->mirror_stale && h->d_live_ext) {        // live edges after device edits, from the device counter
        int64_t live = 0;
        if (cudaMemcpyAsync(&live, h->d_live_ext, sizeof(live), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess) {
            cudaGetLastError();
            return MRF_ECUDA;
        }
        out->n_edges = live;
    }
    out->n_samples = std::max<int64_t>(0, h->sweep_host - h->count_from_host) * h->C;
    out->log_const = h->log_const;
    out->schedule = h->schedule;
    out->tune_ms_thread = h->tune_ms[0];
    out->tune_ms_cta = h->tune_ms[1];
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
    a.theta = scratch + kNoallocCtlWords;
    a.logp = nullptr;
    MRF_CUDA(h, launch_sweep_noalloc(a, h->layout, labels_in, labels_out, (uint32_t)sweep_index, h->stream));
    return MRF_OK;
}

}  // extern "C"

// ============================================================================ batches

struct mrf_batch {
    int32_t G = 0, C = 0;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    mrf_options opt{};
    std::vector<int32_t> n_vars, n_labels, cls, site_off;
    std::vector<int64_t> edge_off;
    std::vector<int32_t> class_L, class_N;
    std::vector<std::vector<int32_t>> class_graphs;
    std::vector<mrf_t*> h;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    std::string err;
    // per-class edit staging, kept across edits (capacity reused)
    std::vector<std::vector<int64_t>> ed_rm, ed_idx, ed_ids;
    std::vector<std::vector<int32_t>> ed_s, ed_t;
    std::vector<std::vector<float>> ed_p;
    // device edit queue (mrf_batch_queue_create): buffers, per-class lists and
    // the round graph {edit, n sweeps}
    bool q_on = false;
    int64_t q_cap_rm = 0, q_cap_add = 0, q_cap_pair = 0, q_extra = 0;
    int32_t* dq_rm_graph = nullptr; int64_t* dq_rm_slot = nullptr;
    int32_t* dq_add_graph = nullptr; int32_t* dq_add_src = nullptr; int32_t* dq_add_dst = nullptr;
    float* dq_pair = nullptr;
    int64_t* dq_counts = nullptr; int64_t* dq_out = nullptr; uint32_t* dq_status = nullptr;
    int64_t* dq_blk = nullptr; int64_t q_nblk = 0;
    unsigned long long* dq_toolong = nullptr;
    int32_t* dq_g = nullptr;               // [4][G]: class, first class site, sites, labels of each graph
    QClass* dq_cls = nullptr;              // [K]
    std::vector<QClass> qc;                // host copies
    std::vector<int64_t> qc_mark_cap, qc_fsum_cap;
    bool q_ready = false;                  // per-class state matches the class handles
    cudaGraphExec_t round_graph = nullptr;
    int32_t round_n = -1, round_mode = -1;
};

namespace {

mrf_status bfail(mrf_batch_t* b, mrf_status st, const std::string& msg) {
    if (b) b->err = msg;
    return st;
}

void drop_batch_graphs(mrf_batch_t* b) {
    for (auto& g : b->graph)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    if (b->round_graph) { cudaGraphExecDestroy(b->round_graph); b->round_graph = nullptr; }
    b->q_ready = false;
}

// Frees the queue; with keep_mirror, the class handles' host mirrors are read
// back first (the live-edge counter they would report goes away).
void free_queue(mrf_batch_t* b, bool keep_mirror = true) {
    if (keep_mirror)
        for (mrf_t* hk : b->h)
            if (hk->mirror_stale && sync_mirror(hk) != MRF_OK) hk->err.clear();
    dfree(b->dq_rm_graph); dfree(b->dq_rm_slot); dfree(b->dq_add_graph); dfree(b->dq_add_src); dfree(b->dq_add_dst);
    dfree(b->dq_pair); dfree(b->dq_counts); dfree(b->dq_out); dfree(b->dq_status); dfree(b->dq_blk);
    dfree(b->dq_toolong); dfree(b->dq_g); dfree(b->dq_cls);
    for (QClass& c : b->qc) {
        dfree(c.mark); dfree(c.touched); dfree(c.rm); dfree(c.add_slot); dfree(c.add_idx); dfree(c.add_poff);
        dfree(c.add_s); dfree(c.add_t); dfree(c.cnt); dfree(c.fsum);
    }
    for (mrf_t* hk : b->h) hk->d_live_ext = nullptr;
    b->qc.clear(); b->qc_mark_cap.clear(); b->qc_fsum_cap.clear();
    b->q_on = false;
    b->q_ready = false;
}

mrf_status class_status(mrf_batch_t* b, int k, mrf_status st) {
    if (st != MRF_OK) b->err = "class L=" + std::to_string(b->class_L[k]) + ": " + b->h[k]->err;
    return st;
}

}  // namespace

extern "C" {

mrf_status mrf_batch_create(mrf_batch_t** out, int32_t n_graphs, const int32_t* n_vars, const int32_t* n_labels,
                            int32_t n_chains, uint64_t seed, const mrf_options* opt, void* cuda_stream) {
    if (!out || n_graphs <= 0 || !n_vars || !n_labels || n_chains <= 0) return MRF_EINVAL;
    *out = nullptr;
    mrf_batch_t* b = new mrf_batch_t();
    b->G = n_graphs; b->C = n_chains; b->seed = seed; b->stream = (cudaStream_t)cuda_stream;
    if (opt) b->opt = *opt; else mrf_default_options(&b->opt);
    b->n_vars.assign(n_vars, n_vars + n_graphs);
    b->n_labels.assign(n_labels, n_labels + n_graphs);
    for (int g = 0; g < n_graphs; ++g) {
        if (n_vars[g] <= 0) { delete b; return MRF_EINVAL; }
        if (n_labels[g] < 2 || n_labels[g] > kMaxLabels) { delete b; return MRF_ERANGE; }
    }
    std::vector<int32_t> Ls(b->n_labels);
    std::sort(Ls.begin(), Ls.end());
    Ls.erase(std::unique(Ls.begin(), Ls.end()), Ls.end());
    b->class_L = Ls;
    b->class_N.assign(Ls.size(), 0);
    b->class_graphs.assign(Ls.size(), {});
    b->cls.assign(n_graphs, 0);
    b->site_off.assign(n_graphs, 0);
    b->edge_off.assign(n_graphs, 0);
    for (int g = 0; g < n_graphs; ++g) {
        const int k = (int)(std::lower_bound(Ls.begin(), Ls.end(), n_labels[g]) - Ls.begin());
        b->cls[g] = k;
        if ((int64_t)b->class_N[k] + n_vars[g] >= (1ll << 31)) { delete b; return MRF_ERANGE; }
        b->site_off[g] = b->class_N[k];
        b->class_N[k] += n_vars[g];
        b->class_graphs[k].push_back(g);
    }
    mrf_options copt = b->opt;
    copt.use_graphs = 0;          // the batch captures all classes together
    copt.grid_nx = copt.grid_ny = copt.grid_nz = 0;
    for (size_t k = 0; k < Ls.size(); ++k) {
        mrf_t* hk = nullptr;
        const uint64_t ks = seed + (uint64_t)Ls[k] * 0x9E3779B97F4A7C15ull;
        mrf_status st = mrf_create(&hk, b->class_N[k], Ls[k], n_chains, ks, &copt, cuda_stream);
        if (st != MRF_OK) { mrf_batch_destroy(b); return st; }
        b->h.push_back(hk);
    }
    *out = b;
    return MRF_OK;
}

void mrf_batch_destroy(mrf_batch_t* b) {
    if (!b) return;
    drop_batch_graphs(b);
    free_queue(b, false);
    for (auto* hk : b->h) mrf_destroy(hk);
    delete b;
}

const char* mrf_batch_last_error(const mrf_batch_t* b) { return b ? b->err.c_str() : "null batch"; }
int32_t mrf_batch_n_classes(const mrf_batch_t* b) { return b ? (int32_t)b->h.size() : 0; }
mrf_t* mrf_batch_class(mrf_batch_t* b, int32_t k) { return (b && k >= 0 && k < (int)b->h.size()) ? b->h[k] : nullptr; }

mrf_status mrf_batch_graph(const mrf_batch_t* b, int32_t g, mrf_batch_graph_info* out) {
    if (!b || !out || g < 0 || g >= b->G) return MRF_EINVAL;
    out->n_vars = b->n_vars[g]; out->n_labels = b->n_labels[g]; out->class_index = b->cls[g];
    out->site_offset = b->site_off[g]; out->first_edge_slot = b->edge_off[g];
    return MRF_OK;
}

mrf_status mrf_batch_set_factors(mrf_batch_t* b, const float* unary_log, const int64_t* n_edges, const int32_t* src,
                                 const int32_t* dst, const float* pair_log) {
    if (!b || !unary_log || !n_edges) return MRF_EINVAL;
    drop_batch_graphs(b);
    const int G = b->G, K = (int)b->h.size();
    std::vector<int64_t> u_off(G + 1, 0), e_off(G + 1, 0), p_off(G + 1, 0);
    for (int g = 0; g < G; ++g) {
        if (n_edges[g] < 0) return bfail(b, MRF_EINVAL, "negative edge count");
        const int64_t L = b->n_labels[g];
        u_off[g + 1] = u_off[g] + (int64_t)b->n_vars[g] * L;
        e_off[g + 1] = e_off[g] + n_edges[g];
        p_off[g + 1] = p_off[g] + n_edges[g] * L * L;
    }
    if (e_off[G] > 0 && (!src || !dst || !pair_log)) return bfail(b, MRF_EINVAL, "null edge arrays");
    for (int k = 0; k < K; ++k) {
        const int L = b->class_L[k];
        std::vector<float> u, p;
        std::vector<int32_t> s, t;
        int64_t ne = 0;
        for (int g : b->class_graphs[k]) ne += n_edges[g];
        u.reserve((size_t)b->class_N[k] * L); s.reserve(ne); t.reserve(ne); p.reserve((size_t)ne * L * L);
        int64_t slot = 0;
        for (int g : b->class_graphs[k]) {
            u.insert(u.end(), unary_log + u_off[g], unary_log + u_off[g + 1]);
            b->edge_off[g] = slot;
            for (int64_t e = e_off[g]; e < e_off[g + 1]; ++e) {
                const int32_t a = src[e], c = dst[e];
                if (a < 0 || a >= b->n_vars[g] || c < 0 || c >= b->n_vars[g])
                    return bfail(b, MRF_ERANGE, "graph " + std::to_string(g) + ": vertex id out of range");
                s.push_back(a + b->site_off[g]);
                t.push_back(c + b->site_off[g]);
            }
            p.insert(p.end(), pair_log + p_off[g], pair_log + p_off[g + 1]);
            slot += n_edges[g];
        }
        mrf_status st = mrf_set_factors(b->h[k], u.data(), ne, s.data(), t.data(), p.data(), MRF_PTR_HOST);
        if (st != MRF_OK) return class_status(b, k, st);
    }
    return MRF_OK;
}

mrf_status mrf_batch_edit_factors(mrf_batch_t* b, int64_t n_remove, const int32_t* remove_graph,
                                  const int64_t* remove_slot, int64_t n_add, const int32_t* add_graph,
                                  const int32_t* src, const int32_t* dst, const float* pair_log, int64_t* out_slots) {
    if (!b || n_remove < 0 || n_add < 0) return MRF_EINVAL;
    if ((n_remove && (!remove_graph || !remove_slot)) || (n_add && (!add_graph || !src || !dst || !pair_log || !out_slots)))
        return bfail(b, MRF_EINVAL, "null edit arrays");
    drop_batch_graphs(b);
    const int K = (int)b->h.size();
    b->ed_rm.resize(K); b->ed_idx.resize(K); b->ed_ids.resize(K);
    b->ed_s.resize(K); b->ed_t.resize(K); b->ed_p.resize(K);
    std::vector<int64_t> n_rm(K, 0), n_ad(K, 0), n_fl(K, 0);
    for (int64_t i = 0; i < n_remove; ++i) {
        const int g = remove_graph[i];
        if (g < 0 || g >= b->G) return bfail(b, MRF_ERANGE, "edit: graph id out of range");
        n_rm[b->cls[g]]++;
    }
    for (int64_t i = 0; i < n_add; ++i) {
        const int g = add_graph[i];
        if (g < 0 || g >= b->G) return bfail(b, MRF_ERANGE, "edit: graph id out of range");
        if (src[i] < 0 || src[i] >= b->n_vars[g] || dst[i] < 0 || dst[i] >= b->n_vars[g])
            return bfail(b, MRF_ERANGE, "edit: vertex id out of range");
        const int k = b->cls[g];
        n_ad[k]++;
        n_fl[k] += (int64_t)b->n_labels[g] * b->n_labels[g];
    }
    for (int k = 0; k < K; ++k) {
        b->ed_rm[k].clear(); b->ed_rm[k].reserve(n_rm[k]);
        b->ed_idx[k].clear(); b->ed_idx[k].reserve(n_ad[k]);
        b->ed_s[k].clear(); b->ed_s[k].reserve(n_ad[k]);
        b->ed_t[k].clear(); b->ed_t[k].reserve(n_ad[k]);
        b->ed_p[k].resize(n_fl[k]);
        b->ed_ids[k].resize(n_ad[k]);
    }
    for (int64_t i = 0; i < n_remove; ++i) b->ed_rm[b->cls[remove_graph[i]]].push_back(remove_slot[i]);
    std::vector<int64_t> pos(K, 0);
    int64_t poff = 0;
    for (int64_t i = 0; i < n_add; ++i) {
        const int g = add_graph[i];
        const int k = b->cls[g];
        const int64_t LL = (int64_t)b->n_labels[g] * b->n_labels[g];
        b->ed_idx[k].push_back(i);
        b->ed_s[k].push_back(src[i] + b->site_off[g]);
        b->ed_t[k].push_back(dst[i] + b->site_off[g]);
        std::memcpy(b->ed_p[k].data() + pos[k], pair_log + poff, (size_t)LL * sizeof(float));
        pos[k] += LL;
        poff += LL;
    }
    for (int k = 0; k < K; ++k) {
        if (b->ed_rm[k].empty() && b->ed_idx[k].empty()) continue;
        std::vector<int64_t>& ids = b->ed_ids[k];
        mrf_status st = mrf_edit_factors(b->h[k], (int64_t)b->ed_rm[k].size(), b->ed_rm[k].data(),
                                         (int64_t)b->ed_idx[k].size(), b->ed_s[k].data(), b->ed_t[k].data(),
                                         b->ed_p[k].data(), ids.data(), MRF_PTR_HOST);
        if (st != MRF_OK) return class_status(b, k, st);
        for (size_t j = 0; j < ids.size(); ++j) out_slots[b->ed_idx[k][j]] = ids[j];
    }
    return MRF_OK;
}

mrf_status mrf_batch_sweep(mrf_batch_t* b, int32_t n_sweeps, int32_t mode) {
    if (!b) return MRF_EINVAL;
    const int K = (int)b->h.size();
    if (n_sweeps >= 0 && (mode == MRF_MODE_SW || mode == MRF_MODE_HIGDON)) {
        // cluster sweeps (Section 4.3): each class as its own handle would run them
        for (int k = 0; k < K; ++k) {
            if (!b->h[k]->has_factors) return bfail(b, MRF_ESTATE, "mrf_batch_set_factors first");
            mrf_status st = mrf_sweep(b->h[k], n_sweeps, mode);
            if (st != MRF_OK) return class_status(b, k, st);
        }
        return MRF_OK;
    }
    if (n_sweeps < 0 || (mode != MRF_MODE_PLAIN && mode != MRF_MODE_FUSED)) return bfail(b, MRF_EINVAL, "bad sweep count or mode");
    for (int k = 0; k < K; ++k) {
        if (!b->h[k]->has_factors) return bfail(b, MRF_ESTATE, "mrf_batch_set_factors first");
        if (mode == MRF_MODE_PLAIN && b->h[k]->schedule == 0 && n_sweeps > 0) {
            mrf_status st = tune_schedule(b->h[k]);
            if (st != MRF_OK) return class_status(b, k, st);
        }
    }
    const bool graphs = b->opt.use_graphs && b->stream != nullptr && !b->opt.kernel_timing;
    if (graphs && !b->graph[mode] && n_sweeps > 0) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return bfail(b, MRF_ECUDA, "stream capture failed");
        mrf_status st = MRF_OK;
        for (int k = 0; k < K && st == MRF_OK; ++k) st = enqueue_sweep(b->h[k], mode);
        cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
        if (st != MRF_OK || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return bfail(b, st != MRF_OK ? st : MRF_ECUDA, "batch graph capture failed");
        }
        ce = cudaGraphInstantiate(&b->graph[mode], g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) { cudaGetLastError(); return bfail(b, MRF_ECUDA, "batch graph instantiate failed"); }
    }
    for (int i = 0; i < n_sweeps; ++i) {
        if (graphs) {
            if (cudaGraphLaunch(b->graph[mode], b->stream) != cudaSuccess) { cudaGetLastError(); return bfail(b, MRF_ECUDA, "graph launch"); }
        } else {
            for (int k = 0; k < K; ++k) {
                mrf_status st = enqueue_sweep(b->h[k], mode);
                if (st != MRF_OK) return class_status(b, k, st);
            }
        }
    }
    for (int k = 0; k < K; ++k) b->h[k]->sweep_host += n_sweeps;
    return MRF_OK;
}

namespace {

// Per-class queue state matching the class handles: free slots reserved,
// lists, removal marks, live counts and incidence capacity.  Runs before a
// round is captured (a new queue, or after set_factors or host edits).
mrf_status queue_prepare(mrf_batch_t* b) {
    if (b->q_ready) return MRF_OK;
    const int K = (int)b->h.size();
    for (auto& g : b->graph)                     // sweep graphs captured before the reserve
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    if (b->round_graph) { cudaGraphExecDestroy(b->round_graph); b->round_graph = nullptr; }
    if ((int)b->qc.size() != K) {
        b->qc.assign(K, QClass{});
        b->qc_mark_cap.assign(K, 0);
        b->qc_fsum_cap.assign(K, 0);
    }
    for (int k = 0; k < K; ++k) {
        mrf_t* h = b->h[k];
        if (!h->has_factors) return bfail(b, MRF_ESTATE, "mrf_batch_set_factors first");
        mrf_status st = sync_mirror(h);
        if (st == MRF_OK) st = reserve_slots(h, std::max(h->E_slots, h->E_live + b->q_extra));
        if (st != MRF_OK) return class_status(b, k, st);
        h->dyn_degree = true;
        drop_graphs(h);
        QClass& c = b->qc[k];
        auto ok = [&](cudaError_t e) {
            if (e != cudaSuccess) { cudaGetLastError(); b->err = std::string("queue buffers: ") + cudaGetErrorString(e); }
            return e == cudaSuccess;
        };
        if (!c.cnt) {
            if (!ok(dalloc(c.rm, (size_t)b->q_cap_rm)) || !ok(dalloc(c.add_slot, (size_t)b->q_cap_add)) ||
                !ok(dalloc(c.add_idx, (size_t)b->q_cap_add)) || !ok(dalloc(c.add_poff, (size_t)b->q_cap_add)) ||
                !ok(dalloc(c.add_s, (size_t)b->q_cap_add)) || !ok(dalloc(c.add_t, (size_t)b->q_cap_add)) ||
                !ok(dalloc(c.touched, (size_t)h->N)) || !ok(dalloc(c.cnt, 3)) ||
                !ok(cudaMemsetAsync(c.touched, 0, (size_t)h->N, b->stream)) ||
                !ok(cudaMemsetAsync(c.add_slot, 0xFF, (size_t)std::max<int64_t>(b->q_cap_add, 1) * sizeof(int64_t), b->stream)) ||
                !ok(cudaMemsetAsync(c.cnt, 0, 3 * sizeof(int64_t), b->stream)))
                return MRF_ENOMEM;
        }
        if (b->qc_mark_cap[k] < h->E_slots) {
            if (!ok(dalloc(c.mark, (size_t)h->E_slots)) ||
                !ok(cudaMemsetAsync(c.mark, 0, (size_t)h->E_slots * sizeof(uint32_t), b->stream)))
                return MRF_ENOMEM;
            b->qc_mark_cap[k] = h->E_slots;
        }
        const int64_t nb = (h->E_slots + 1023) / 1024;
        if (b->qc_fsum_cap[k] < nb + 1) {
            if (!ok(dalloc(c.fsum, (size_t)nb + 1))) return MRF_ENOMEM;
            b->qc_fsum_cap[k] = nb + 1;
        }
        if (h->inc_cap < 2 * h->E_slots) {       // every slot may be live; the current lists are kept
            int2* inc = nullptr;
            if (!ok(cudaMalloc((void**)&inc, (size_t)(2 * h->E_slots) * sizeof(int2)))) return MRF_ENOMEM;
            if (!ok(cudaMemcpyAsync(inc, h->d_inc, (size_t)h->inc_cap * sizeof(int2), cudaMemcpyDeviceToDevice, b->stream)) ||
                !ok(cudaStreamSynchronize(b->stream))) {
                cudaFree(inc);
                return MRF_ECUDA;
            }
            dfree(h->d_inc);
            h->d_inc = inc;
            h->inc_cap = 2 * h->E_slots;
        }
        if (!h->d_csr_work) {
            if (!ok(dalloc(h->d_csr_work, 2 * (size_t)h->N + 2)) ||
                !ok(dalloc(h->d_csr_sums, (size_t)((h->N + 1 + 1023) / 1024 + 2))))
                return MRF_ENOMEM;
        }
        c.src = h->d_src; c.dst = h->d_dst; c.E_res = h->E_slots;
        c.N = h->N; c.L = h->L; c.layout = h->layout;
        const int64_t live = h->E_live;
        if (!ok(cudaMemcpyAsync(c.cnt + 2, &live, sizeof(live), cudaMemcpyHostToDevice, b->stream)) ||
            !ok(cudaStreamSynchronize(b->stream)))
            return MRF_ECUDA;
        h->d_live_ext = c.cnt + 2;
    }
    if (cudaMemcpyAsync(b->dq_cls, b->qc.data(), (size_t)K * sizeof(QClass), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, MRF_ECUDA, "queue class table upload");
    }
    b->q_ready = true;
    return MRF_OK;
}

QArgs make_qargs(const mrf_batch_t* b) {
    QArgs q{};
    q.rm_graph = b->dq_rm_graph; q.rm_slot = b->dq_rm_slot;
    q.add_graph = b->dq_add_graph; q.add_src = b->dq_add_src; q.add_dst = b->dq_add_dst; q.pair = b->dq_pair;
    q.counts = b->dq_counts; q.out_slot = b->dq_out; q.status = b->dq_status;
    q.cap_rm = b->q_cap_rm; q.cap_add = b->q_cap_add; q.cap_pair = b->q_cap_pair;
    q.G = b->G; q.K = (int32_t)b->h.size();
    q.g_cls = b->dq_g; q.g_off = b->dq_g + b->G; q.g_n = b->dq_g + 2 * (size_t)b->G; q.g_L = b->dq_g + 3 * (size_t)b->G;
    q.cls = b->dq_cls; q.blk = b->dq_blk; q.nblk = b->q_nblk;
    return q;
}

// The kernels of one round on the batch's stream (captured or launched).
mrf_status enqueue_round(mrf_batch_t* b, int n_sweeps, int mode) {
    const QArgs q = make_qargs(b);
    cudaStream_t s = b->stream;
    cudaError_t e = cudaMemsetAsync(b->dq_status, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = launch_queue_route(q, s);
    for (int k = 0; k < (int)b->h.size() && e == cudaSuccess; ++k) {
        mrf_t* h = b->h[k];
        const QClass& c = b->qc[k];
        e = launch_queue_apply(q, c, s);
        DecompArgs d{};
        d.L = h->L; d.M = h->M; d.layout = h->layout; d.n = b->q_cap_add; d.slots = c.add_slot;
        d.pair = b->dq_pair; d.pair_off = c.add_poff; d.n_dev = c.cnt + 1; d.status = b->dq_status;
        d.tau = h->d_tau; d.thr = h->d_thr; d.fold = h->d_fold; d.cst = h->d_cst; d.resid = nullptr;
        d.sw_thr = h->d_swt; d.sw_lw = h->d_swl; d.sw_fold = h->d_swfold; d.sw_ell = h->d_swell;
        if (e == cudaSuccess) e = launch_decompose(d, s);
        if (e == cudaSuccess)
            e = launch_build_planes(h->d_thr, b->q_cap_add, c.add_slot, 0, h->M, h->d_tpl, s, c.cnt + 1, b->dq_status);
        if (e == cudaSuccess)
            e = build_csr_device(h->d_src, h->d_dst, h->E_slots, h->N, h->d_inc_ptr, h->d_inc, h->d_csr_work,
                                 h->d_csr_sums, b->dq_toolong, 512, s);
        if (e == cudaSuccess) e = launch_csr_sort_long(h->d_inc_ptr, h->d_inc, h->N, 512, b->dq_status, s);
        if (e == cudaSuccess && h->d_swut)
            e = launch_fold_unary(h->d_unary, h->d_swfold, h->d_inc_ptr, h->d_inc, h->N, h->L, h->d_swut, nullptr, s);
        if (e == cudaSuccess)
            e = launch_fold_touched(h->d_unary, h->d_fold, h->d_inc_ptr, h->d_inc, h->N, h->L, c.touched, h->d_ut,
                                    h->d_utf, s);
    }
    if (e == cudaSuccess) e = launch_queue_finish(q, s);
    if (e != cudaSuccess) { cudaGetLastError(); return bfail(b, MRF_ECUDA, std::string("round launch: ") + cudaGetErrorString(e)); }
    for (int i = 0; i < n_sweeps; ++i)
        for (int k = 0; k < (int)b->h.size(); ++k) {
            mrf_status st = enqueue_sweep(b->h[k], mode);
            if (st != MRF_OK) return class_status(b, k, st);
        }
    return MRF_OK;
}

}  // namespace

mrf_status mrf_batch_set_kernel_timing(mrf_batch_t* b, int32_t on) {
    if (!b) return MRF_EINVAL;
    b->opt.kernel_timing = on ? 1 : 0;
    for (mrf_t* h : b->h) h->opt.kernel_timing = on ? 1 : 0;
    return MRF_OK;
}

mrf_status mrf_batch_queue_create(mrf_batch_t* b, int64_t max_remove, int64_t max_add, int64_t max_pair_floats,
                                  int64_t extra_slots) {
    if (!b) return MRF_EINVAL;
    if (max_remove < 0 || max_add < 0 || max_pair_floats < 0 || extra_slots < 0)
        return bfail(b, MRF_EINVAL, "negative queue size");
    drop_batch_graphs(b);
    free_queue(b);
    const int G = b->G, K = (int)b->h.size();
    b->q_cap_rm = max_remove; b->q_cap_add = max_add; b->q_cap_pair = max_pair_floats; b->q_extra = extra_slots;
    b->q_nblk = (std::max<int64_t>({max_remove, max_add, 1}) + 1023) / 1024;
    std::vector<int32_t> gt(4 * (size_t)G);
    for (int g = 0; g < G; ++g) {
        gt[g] = b->cls[g]; gt[G + g] = b->site_off[g]; gt[2 * G + g] = b->n_vars[g]; gt[3 * G + g] = b->n_labels[g];
    }
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess) { cudaGetLastError(); b->err = std::string("queue buffers: ") + cudaGetErrorString(e); }
        return e == cudaSuccess;
    };
    if (!ok(dalloc(b->dq_rm_graph, (size_t)max_remove)) || !ok(dalloc(b->dq_rm_slot, (size_t)max_remove)) ||
        !ok(dalloc(b->dq_add_graph, (size_t)max_add)) || !ok(dalloc(b->dq_add_src, (size_t)max_add)) ||
        !ok(dalloc(b->dq_add_dst, (size_t)max_add)) || !ok(dalloc(b->dq_pair, (size_t)max_pair_floats)) ||
        !ok(dalloc(b->dq_counts, 3)) || !ok(dalloc(b->dq_out, (size_t)max_add)) || !ok(dalloc(b->dq_status, 1)) ||
        !ok(dalloc(b->dq_blk, (size_t)(b->q_nblk * (2 * K + 1)))) || !ok(dalloc(b->dq_toolong, 1)) ||
        !ok(dalloc(b->dq_g, gt.size())) || !ok(dalloc(b->dq_cls, (size_t)K)) ||
        !ok(cudaMemsetAsync(b->dq_counts, 0, 3 * sizeof(int64_t), b->stream)) ||
        !ok(cudaMemsetAsync(b->dq_status, 0, sizeof(uint32_t), b->stream)) ||
        !ok(cudaMemcpyAsync(b->dq_g, gt.data(), gt.size() * sizeof(int32_t), cudaMemcpyHostToDevice, b->stream)) ||
        !ok(cudaStreamSynchronize(b->stream)) || !ok(init_csr_sort_long())) {
        free_queue(b);
        return MRF_ENOMEM;
    }
    b->q_on = true;
    return MRF_OK;
}

mrf_status mrf_batch_queue_load(mrf_batch_t* b, int64_t n_remove, const int32_t* remove_graph,
                                const int64_t* remove_slot, int64_t n_add, const int32_t* add_graph,
                                const int32_t* src, const int32_t* dst, int64_t n_pair, const float* pair_log,
                                int32_t ptr_kind) {
    if (!b) return MRF_EINVAL;
    if (!b->q_on) return bfail(b, MRF_ESTATE, "mrf_batch_queue_create first");
    if (ptr_kind != MRF_PTR_HOST && ptr_kind != MRF_PTR_DEVICE) return bfail(b, MRF_EINVAL, "bad ptr_kind");
    if (n_remove < 0 || n_add < 0 || n_pair < 0) return bfail(b, MRF_EINVAL, "negative count");
    if (n_remove > b->q_cap_rm || n_add > b->q_cap_add || n_pair > b->q_cap_pair)
        return bfail(b, MRF_ERANGE, "edit larger than the queue's capacities");
    if ((n_remove && (!remove_graph || !remove_slot)) || (n_add && (!add_graph || !src || !dst)) || (n_pair && !pair_log))
        return bfail(b, MRF_EINVAL, "null edit arrays");
    const cudaMemcpyKind kind = ptr_kind == MRF_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaStream_t s = b->stream;
    const int64_t counts[3] = {n_remove, n_add, n_pair};
    cudaError_t e = cudaSuccess;
    auto cp = [&](void* d, const void* p, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(d, p, bytes, kind, s);
    };
    cp(b->dq_rm_graph, remove_graph, (size_t)n_remove * sizeof(int32_t));
    cp(b->dq_rm_slot, remove_slot, (size_t)n_remove * sizeof(int64_t));
    cp(b->dq_add_graph, add_graph, (size_t)n_add * sizeof(int32_t));
    cp(b->dq_add_src, src, (size_t)n_add * sizeof(int32_t));
    cp(b->dq_add_dst, dst, (size_t)n_add * sizeof(int32_t));
    cp(b->dq_pair, pair_log, (size_t)n_pair * sizeof(float));
    // counts[] is pageable: the copy stages it before returning
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->dq_counts, counts, sizeof(counts), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { cudaGetLastError(); return bfail(b, MRF_ECUDA, std::string("queue load: ") + cudaGetErrorString(e)); }
    return MRF_OK;
}

mrf_status mrf_batch_round(mrf_batch_t* b, int32_t n_sweeps, int32_t mode) {
    if (!b) return MRF_EINVAL;
    if (!b->q_on) return bfail(b, MRF_ESTATE, "mrf_batch_queue_create first");
    if (n_sweeps < 0 || (mode != MRF_MODE_PLAIN && mode != MRF_MODE_FUSED)) return bfail(b, MRF_EINVAL, "bad sweep count or mode");
    mrf_status st = queue_prepare(b);
    if (st != MRF_OK) return st;
    const int K = (int)b->h.size();
    for (int k = 0; k < K; ++k)
        if (mode == MRF_MODE_PLAIN && b->h[k]->schedule == 0 && n_sweeps > 0) {
            st = tune_schedule(b->h[k]);
            if (st != MRF_OK) return class_status(b, k, st);
        }
    const bool graphs = b->opt.use_graphs && b->stream != nullptr && !b->opt.kernel_timing;
    if (graphs && b->round_graph && (b->round_n != n_sweeps || b->round_mode != mode)) {
        cudaGraphExecDestroy(b->round_graph);
        b->round_graph = nullptr;
    }
    if (graphs && !b->round_graph) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, MRF_ECUDA, "stream capture failed");
        }
        st = enqueue_round(b, n_sweeps, mode);
        cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
        if (st != MRF_OK || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return st != MRF_OK ? st : bfail(b, MRF_ECUDA, "round graph capture failed");
        }
        ce = cudaGraphInstantiate(&b->round_graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) { cudaGetLastError(); b->round_graph = nullptr; return bfail(b, MRF_ECUDA, "round graph instantiate failed"); }
        b->round_n = n_sweeps;
        b->round_mode = mode;
    }
    if (graphs) {
        if (cudaGraphLaunch(b->round_graph, b->stream) != cudaSuccess) { cudaGetLastError(); return bfail(b, MRF_ECUDA, "graph launch"); }
    } else {
        st = enqueue_round(b, n_sweeps, mode);
        if (st != MRF_OK) return st;
    }
    for (mrf_t* h : b->h) {
        h->sweep_host += n_sweeps;
        h->mirror_stale = true;
        h->sw_checked = false;
        h->hg_ready = false;
    }
    return MRF_OK;
}

mrf_status mrf_batch_queue_result(mrf_batch_t* b, uint32_t* status, int64_t n, int64_t* out_slots) {
    if (!b || !status || n < 0 || (n > 0 && !out_slots)) return MRF_EINVAL;
    if (!b->q_on) return bfail(b, MRF_ESTATE, "mrf_batch_queue_create first");
    if (n > b->q_cap_add) return bfail(b, MRF_ERANGE, "more slots than the queue's max_add");
    cudaError_t e = cudaMemcpyAsync(status, b->dq_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(out_slots, b->dq_out, (size_t)n * sizeof(int64_t), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) { cudaGetLastError(); return bfail(b, MRF_ECUDA, std::string("queue result: ") + cudaGetErrorString(e)); }
    return MRF_OK;
}

mrf_status mrf_batch_reset_marginals(mrf_batch_t* b, int32_t burn_in_sweeps) {
    if (!b) return MRF_EINVAL;
    for (int k = 0; k < (int)b->h.size(); ++k) {
        mrf_status st = mrf_reset_marginals(b->h[k], burn_in_sweeps);
        if (st != MRF_OK) return class_status(b, k, st);
    }
    return MRF_OK;
}

mrf_status mrf_batch_get_counts(mrf_batch_t* b, int32_t g, uint32_t* out) {
    if (!b || !out || g < 0 || g >= b->G) return MRF_EINVAL;
    mrf_t* h = b->h[b->cls[g]];
    const size_t L = (size_t)b->n_labels[g];
    if (cudaMemcpyAsync(out, h->d_counts + (size_t)b->site_off[g] * L, (size_t)b->n_vars[g] * L * sizeof(uint32_t),
                        cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, MRF_ECUDA, "copy counts");
    }
    return MRF_OK;
}

mrf_status mrf_batch_get_labels(mrf_batch_t* b, int32_t g, uint8_t* out) {
    if (!b || !out || g < 0 || g >= b->G) return MRF_EINVAL;
    mrf_t* h = b->h[b->cls[g]];
    const size_t n = (size_t)b->n_vars[g], C = (size_t)h->C;
    std::vector<uint8_t> buf(n * C);
    const uint8_t* src = h->d_x + (h->sweep_host & 1) * (size_t)h->N * C + (size_t)b->site_off[g] * C;
    if (cudaMemcpyAsync(buf.data(), src, n * C, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, MRF_ECUDA, "copy labels");
    }
    for (size_t v = 0; v < n; ++v)
        for (size_t c = 0; c < C; ++c) out[c * n + v] = buf[v * C + c];
    return MRF_OK;
}

}  // extern "C"

// ============================================================================ learned proposal

namespace {

// splitmix64 (Steele, Lea, Flood 2014): seeding and shuffling on the host.
uint64_t splitmix64(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

mrf_status learned_train_buffers(mrf_t* h, int64_t rows) {
    if (rows <= h->train_rows) return MRF_OK;
    const int64_t H = h->la.H, O = h->la.O, Dp = h->la.Dp;
    MRF_CUDA(h, dalloc(h->d_train, (size_t)rows * (4 * H + 2 * O)));
    MRF_CUDA(h, dalloc(h->d_bidx, (size_t)rows));
    MRF_CUDA(h, dalloc(h->d_bX, (size_t)rows * Dp));
    MRF_CUDA(h, dalloc(h->d_by, (size_t)rows * kLearnBlock));
    MRF_CUDA(h, dalloc(h->d_bn, (size_t)rows));
    float* t = h->d_train;
    h->la.t_h1 = t; t += rows * H;
    h->la.t_h2 = t; t += rows * H;
    h->la.t_d2 = t; t += rows * H;
    h->la.t_d1 = t; t += rows * H;
    h->la.t_z = t; t += rows * O;
    h->la.t_dz = t;
    h->train_rows = rows;
    return MRF_OK;
}

}  // namespace

extern "C" {

int64_t mrf_learned_param_count(const mrf_t* h) { return h && h->learned ? h->n_params : 0; }

mrf_status mrf_learned_setup(mrf_t* h, const int32_t* block_of_site, int32_t hidden, uint64_t init_seed) {
    if (!h || !block_of_site) return MRF_EINVAL;
    if (!h->has_factors) return fail(h, MRF_ESTATE, "mrf_set_factors first");
    if (!h->d_resid) return fail(h, MRF_ESTATE, "create the handle with options.exact_edges = 1");
    if (hidden < 64 || hidden % 64) return fail(h, MRF_EINVAL, "hidden width must be a positive multiple of 64");
    const int N = h->N, L = h->L, C = h->C;
    int nb = 0;
    for (int v = 0; v < N; ++v) {
        if (block_of_site[v] < 0) return fail(h, MRF_ERANGE, "every site needs a block");
        nb = std::max(nb, block_of_site[v] + 1);
    }
    std::vector<std::vector<int32_t>> mem(nb);
    for (int v = 0; v < N; ++v) mem[block_of_site[v]].push_back(v);
    std::vector<int32_t> members((size_t)nb * kLearnBlock, -1), nmem(nb), pos(N);
    for (int b = 0; b < nb; ++b) {
        if (mem[b].empty() || mem[b].size() > (size_t)kLearnBlock)
            return fail(h, MRF_ERANGE, "block " + std::to_string(b) + " has " + std::to_string(mem[b].size()) + " sites");
        nmem[b] = (int32_t)mem[b].size();
        for (size_t i = 0; i < mem[b].size(); ++i) { members[(size_t)b * kLearnBlock + i] = mem[b][i]; pos[mem[b][i]] = (int32_t)i; }
    }
    std::vector<int64_t> iptr(nb + 1, 0);
    std::vector<uint8_t> skip((size_t)h->E_slots, 0);
    for (int64_t e = 0; e < h->E_slots; ++e) {
        const int s = h->h_src[e];
        if (s >= 0 && block_of_site[s] == block_of_site[h->h_dst[e]]) { iptr[block_of_site[s] + 1]++; skip[e] = 1; }
    }
    for (int b = 0; b < nb; ++b) iptr[b + 1] += iptr[b];
    std::vector<int4> intra((size_t)iptr[nb]);
    std::vector<int64_t> fill(iptr.begin(), iptr.end() - 1);
    for (int64_t e = 0; e < h->E_slots; ++e) {
        if (!skip[e]) continue;
        const int s = h->h_src[e], t = h->h_dst[e];
        intra[fill[block_of_site[s]]++] = make_int4((int)e, pos[s], pos[t], 0);
    }
    LearnedArgs& a = h->la;
    a = LearnedArgs{};
    a.nb = nb; a.L = L; a.H = hidden; a.O = kLearnBlock * L;
    a.Dp = (kLearnBlock * L + kLearnPairs + 31) / 32 * 32;
    a.Kx = (kLearnBlock * L + 31) / 32 * 32;
    a.C = C;
    const int64_t H = hidden, Dp = a.Dp, O = a.O;
    h->n_params = H * Dp + H + H * H + H + O * H + O;
    const int64_t R = (int64_t)nb * C;
    MRF_CUDA(h, dalloc(h->d_members, members.size())); MRF_CUDA(h, dalloc(h->d_nmem, (size_t)nb));
    MRF_CUDA(h, dalloc(h->d_intra_ptr, (size_t)nb + 1)); MRF_CUDA(h, dalloc(h->d_intra, std::max<size_t>(intra.size(), 1)));
    MRF_CUDA(h, dalloc(h->d_cf, (size_t)nb * kLearnPairs)); MRF_CUDA(h, dalloc(h->d_skip, (size_t)h->E_slots));
    MRF_CUDA(h, dalloc(h->d_X, (size_t)R * a.Kx)); MRF_CUDA(h, dalloc(h->d_H1, (size_t)R * H));
    MRF_CUDA(h, dalloc(h->d_W1x, (size_t)H * a.Kx)); MRF_CUDA(h, dalloc(h->d_cfb, (size_t)nb * kLearnPairs));
    MRF_CUDA(h, dalloc(h->d_rowbias, (size_t)nb * H));
    MRF_CUDA(h, dalloc(h->d_H2, (size_t)R * H)); MRF_CUDA(h, dalloc(h->d_Z, (size_t)R * O));
    MRF_CUDA(h, dalloc(h->d_w32, (size_t)h->n_params)); MRF_CUDA(h, dalloc(h->d_grad, (size_t)h->n_params));
    MRF_CUDA(h, dalloc(h->d_m, (size_t)h->n_params)); MRF_CUDA(h, dalloc(h->d_v, (size_t)h->n_params));
    MRF_CUDA(h, dalloc(h->d_Wb, (size_t)(H * Dp + H * H + O * H)));
    MRF_CUDA(h, dalloc(h->d_acc, 1));
    MRF_CUDA(h, dalloc(h->d_wimg, (size_t)mlp_tc_image_bytes(H, O, a.Kx)));
    MRF_CUDA(h, dalloc(h->d_tc_err, 1));
    MRF_CUDA(h, cudaMemsetAsync(h->d_tc_err, 0, sizeof(unsigned), h->stream));
    if (!h->d_pot) MRF_CUDA(h, dalloc(h->d_pot, (size_t)N * L * C));
    MRF_CUDA(h, to_device(h->d_members, members.data(), (int64_t)members.size(), MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, to_device(h->d_nmem, nmem.data(), nb, MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, to_device(h->d_intra_ptr, iptr.data(), nb + 1, MRF_PTR_HOST, h->stream));
    if (!intra.empty()) MRF_CUDA(h, to_device(h->d_intra, intra.data(), (int64_t)intra.size(), MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, to_device(h->d_skip, skip.data(), h->E_slots, MRF_PTR_HOST, h->stream));
    // He-uniform weights, zero biases (host generator, then float32 master copy)
    std::vector<float> w((size_t)h->n_params, 0.0f);
    uint64_t st = init_seed;
    auto uni = [&]() { return (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0); };
    auto fill_w = [&](int64_t off, int64_t rows, int64_t cols) {
        const double lim = std::sqrt(6.0 / (double)cols);
        for (int64_t i = 0; i < rows * cols; ++i) w[off + i] = (float)((2.0 * uni() - 1.0) * lim);
    };
    fill_w(0, H, Dp);
    fill_w(H * Dp + H, H, H);
    fill_w(H * Dp + H + H * H + H, O, H);
    MRF_CUDA(h, to_device(h->d_w32, w.data(), h->n_params, MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, cudaMemsetAsync(h->d_m, 0, sizeof(float) * h->n_params, h->stream));
    MRF_CUDA(h, cudaMemsetAsync(h->d_v, 0, sizeof(float) * h->n_params, h->stream));
    MRF_CUDA(h, cudaMemsetAsync(h->d_acc, 0, sizeof(unsigned long long), h->stream));
    a.members = h->d_members; a.nmem = h->d_nmem; a.intra_ptr = h->d_intra_ptr; a.intra = h->d_intra; a.cf = h->d_cf;
    a.X = h->d_X; a.H1 = h->d_H1; a.H2 = h->d_H2; a.Zm = h->d_Z; a.Z = h->d_Z;
    a.w32 = h->d_w32;
    a.b1 = h->d_w32 + H * Dp; a.b2 = h->d_w32 + H * Dp + H + H * H; a.b3 = h->d_w32 + H * Dp + H + H * H + H + O * H;
    a.W1b = h->d_Wb; a.W2b = h->d_Wb + H * Dp; a.W3b = h->d_Wb + H * Dp + H * H;
    a.grad = h->d_grad; a.adam_m = h->d_m; a.adam_v = h->d_v; a.n_accepted = h->d_acc;
    a.ds_X = h->d_dsX; a.ds_y = h->d_dsy; a.ds_n = h->d_dsn;
    a.W1xb = h->d_W1x; a.cfb = h->d_cfb; a.rowbias = h->d_rowbias;
    a.wimg = h->d_wimg; a.tc_err = h->d_tc_err;
    MRF_CUDA(h, learned_sync_bf16(a, h->stream));
    MRF_CUDA(h, launch_learned_couplings(a, h->d_resid, h->d_cf, h->stream));
    h->rowbias_dirty = true;
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    h->learned = true;
    h->adam_step = 0;
    h->proposed = 0;
    return MRF_OK;
}

mrf_status mrf_learned_set_params(mrf_t* h, const float* params, int64_t n) {
    if (!h || !params) return MRF_EINVAL;
    if (!h->learned) return fail(h, MRF_ESTATE, "mrf_learned_setup first");
    if (n != h->n_params) return fail(h, MRF_EINVAL, "parameter count " + std::to_string(n) + " != " + std::to_string(h->n_params));
    MRF_CUDA(h, to_device(h->d_w32, params, n, MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, learned_sync_bf16(h->la, h->stream));
    h->rowbias_dirty = true;
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    return MRF_OK;
}

mrf_status mrf_learned_get_params(mrf_t* h, float* params, int64_t n) {
    if (!h || !params) return MRF_EINVAL;
    if (!h->learned) return fail(h, MRF_ESTATE, "mrf_learned_setup first");
    if (n != h->n_params) return fail(h, MRF_EINVAL, "parameter count mismatch");
    MRF_CUDA(h, cudaMemcpyAsync(params, h->d_w32, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    return MRF_OK;
}

mrf_status mrf_learned_harvest(mrf_t* h, int32_t n_sweeps, int32_t stride, int64_t max_rows, int64_t* rows) {
    if (!h || n_sweeps < 0 || stride <= 0 || max_rows <= 0) return MRF_EINVAL;
    if (!h->learned) return fail(h, MRF_ESTATE, "mrf_learned_setup first");
    if (max_rows > h->ds_cap) {
        if (h->ds_rows) return fail(h, MRF_ESTATE, "the training set cannot grow once filled");
        MRF_CUDA(h, dalloc(h->d_dsX, (size_t)max_rows * h->la.Dp));
        MRF_CUDA(h, dalloc(h->d_dsy, (size_t)max_rows * kLearnBlock));
        MRF_CUDA(h, dalloc(h->d_dsn, (size_t)max_rows));
        h->ds_cap = max_rows;
        h->la.ds_X = h->d_dsX; h->la.ds_y = h->d_dsy; h->la.ds_n = h->d_dsn;
    }
    const int64_t R = (int64_t)h->la.nb * h->C;
    for (int i = 0; i < n_sweeps && h->ds_rows < h->ds_cap; ++i) {
        if (h->schedule == 0) { mrf_status st = tune_schedule(h); if (st != MRF_OK) return st; }
        mrf_status st = enqueue_sweep(h, MRF_MODE_PLAIN);
        if (st != MRF_OK) return st;
        h->sweep_host += 1;
        SweepArgs a = make_args(h);
        a.skip = h->d_skip;
        const int phase = (int)(h->sweep_host % stride);
        MRF_CUDA(h, launch_dual(a, h->layout, h->stream));
        MRF_CUDA(h, launch_potential(a, h->layout, h->stream));
        MRF_CUDA(h, launch_learned_features(h->la, a, h->stream));
        MRF_CUDA(h, launch_learned_harvest(h->la, a, stride, phase, h->ds_rows, h->ds_cap, h->stream));
        const int64_t k = phase < R ? (R - phase + stride - 1) / stride : 0;
        h->ds_rows = std::min(h->ds_cap, h->ds_rows + k);
    }
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (rows) *rows = h->ds_rows;
    return MRF_OK;
}

mrf_status mrf_learned_train(mrf_t* h, int32_t steps, int32_t batch, float lr, uint64_t shuffle_seed, float* loss_trace) {
    if (!h || steps < 0 || batch <= 0) return MRF_EINVAL;
    if (!h->learned) return fail(h, MRF_ESTATE, "mrf_learned_setup first");
    if (h->ds_rows <= 0) return fail(h, MRF_ESTATE, "harvest a training set first");
    mrf_status st = learned_train_buffers(h, batch);
    if (st != MRF_OK) return st;
    if (steps > h->loss_cap) { MRF_CUDA(h, dalloc(h->d_loss, (size_t)steps)); h->loss_cap = steps; }
    std::vector<int32_t> idx((size_t)batch);
    uint64_t rs = shuffle_seed;
    for (int s = 0; s < steps; ++s) {
        for (int j = 0; j < batch; ++j) idx[j] = (int32_t)(splitmix64(rs) % (uint64_t)h->ds_rows);
        MRF_CUDA(h, to_device(h->d_bidx, idx.data(), batch, MRF_PTR_HOST, h->stream));
        MRF_CUDA(h, learned_gather(h->la, h->d_bidx, batch, h->d_bX, h->d_by, h->d_bn, h->stream));
        MRF_CUDA(h, learned_forward_backward(h->la, batch, h->d_bX, h->d_by, h->d_bn, h->d_loss + s, h->stream));
        h->adam_step += 1;
        MRF_CUDA(h, learned_adam(h->la, h->n_params, lr, h->adam_step, h->stream));
    }
    std::vector<double> losses((size_t)steps);
    if (steps) MRF_CUDA(h, cudaMemcpyAsync(losses.data(), h->d_loss, sizeof(double) * steps, cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    h->rowbias_dirty = true;
    if (loss_trace) for (int s = 0; s < steps; ++s) loss_trace[s] = (float)losses[s];
    return MRF_OK;
}

mrf_status mrf_learned_grad(mrf_t* h, const float* X, const uint8_t* y, const uint8_t* nmem, int32_t rows, float* grads,
                            double* loss) {
    if (!h || !X || !y || !nmem || rows <= 0 || !grads) return MRF_EINVAL;
    if (!h->learned) return fail(h, MRF_ESTATE, "mrf_learned_setup first");
    mrf_status st = learned_train_buffers(h, rows);
    if (st != MRF_OK) return st;
    const int64_t Dp = h->la.Dp;
    float* d_xf = nullptr;
    MRF_CUDA(h, dalloc(d_xf, (size_t)rows * Dp));
    struct G { float*& p; ~G() { dfree(p); } } guard{d_xf};
    MRF_CUDA(h, to_device(d_xf, X, rows * Dp, MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, launch_to_bf16(d_xf, h->d_bX, rows * Dp, h->stream));
    MRF_CUDA(h, to_device(h->d_by, y, (int64_t)rows * kLearnBlock, MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, to_device(h->d_bn, nmem, rows, MRF_PTR_HOST, h->stream));
    if (h->loss_cap < 1) { MRF_CUDA(h, dalloc(h->d_loss, 1)); h->loss_cap = 1; }
    MRF_CUDA(h, learned_forward_backward(h->la, rows, h->d_bX, h->d_by, h->d_bn, h->d_loss, h->stream));
    MRF_CUDA(h, cudaMemcpyAsync(grads, h->d_grad, sizeof(float) * h->n_params, cudaMemcpyDeviceToHost, h->stream));
    double l = 0.0;
    MRF_CUDA(h, cudaMemcpyAsync(&l, h->d_loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (loss) *loss = l;
    return MRF_OK;
}

mrf_status mrf_learned_forward(mrf_t* h, const float* X, int32_t rows, float* z) {
    if (!h || !X || !z || rows <= 0) return MRF_EINVAL;
    if (!h->learned) return fail(h, MRF_ESTATE, "mrf_learned_setup first");
    if ((int64_t)rows > (int64_t)h->la.nb * h->C) return fail(h, MRF_ERANGE, "at most n_blocks x chains rows");
    const int64_t Dp = h->la.Dp;
    float* d_xf = nullptr;
    __nv_bfloat16* d_xb = nullptr;
    MRF_CUDA(h, dalloc(d_xf, (size_t)rows * Dp));
    MRF_CUDA(h, dalloc(d_xb, (size_t)rows * Dp));
    struct G { float*& p; __nv_bfloat16*& q; ~G() { dfree(p); dfree(q); } } guard{d_xf, d_xb};
    MRF_CUDA(h, to_device(d_xf, X, rows * Dp, MRF_PTR_HOST, h->stream));
    MRF_CUDA(h, launch_to_bf16(d_xf, d_xb, rows * Dp, h->stream));
    MRF_CUDA(h, launch_learned_mlp(h->la, rows, d_xb, h->stream));
    MRF_CUDA(h, cudaMemcpyAsync(z, h->d_Z, sizeof(float) * rows * h->la.O, cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    return MRF_OK;
}

mrf_status mrf_learned_stats(mrf_t* h, uint64_t* proposed, uint64_t* accepted) {
    if (!h) return MRF_EINVAL;
    if (!h->learned) return fail(h, MRF_ESTATE, "mrf_learned_setup first");
    unsigned long long acc = 0;
    MRF_CUDA(h, cudaMemcpyAsync(&acc, h->d_acc, sizeof(acc), cudaMemcpyDeviceToHost, h->stream));
    MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (proposed) *proposed = h->proposed;
    if (accepted) *accepted = acc;
    return MRF_OK;
}

mrf_status mrf_debug_mlp_timeout(mrf_t* h, int32_t on) {
    if (!h) return MRF_EINVAL;
    if (!h->learned) return fail(h, MRF_ESTATE, "mrf_learned_setup first");
    if (!use_mlp_tc(h)) return fail(h, MRF_ESTATE, "the tensor-core MLP is not in use on this handle");
    h->la.tc_inject_timeout = on ? 1 : 0;
    drop_graphs(h);                                         // captured launches carry the hook's old value
    return MRF_OK;
}

mrf_status mrf_learned_debug(mrf_t* h, float* X, float* z) {
    if (!h) return MRF_EINVAL;
    if (!h->learned) return fail(h, MRF_ESTATE, "mrf_learned_setup first");
    const int64_t R = (int64_t)h->la.nb * h->C;
    if (X) {
        const int Kx = h->la.Kx, Dp = h->la.Dp, fx = kLearnBlock * h->L;
        std::vector<__nv_bfloat16> xb((size_t)(R * Kx)), cb((size_t)h->la.nb * kLearnPairs);
        MRF_CUDA(h, cudaMemcpyAsync(xb.data(), h->d_X, sizeof(__nv_bfloat16) * xb.size(), cudaMemcpyDeviceToHost, h->stream));
        MRF_CUDA(h, cudaMemcpyAsync(cb.data(), h->d_cfb, sizeof(__nv_bfloat16) * cb.size(), cudaMemcpyDeviceToHost, h->stream));
        MRF_CUDA(h, cudaStreamSynchronize(h->stream));
        for (int64_t r = 0; r < R; ++r) {
            const int64_t b = r / h->C;
            for (int q = 0; q < Dp; ++q) {
                float v = 0.0f;
                if (q < fx) v = __bfloat162float(xb[r * Kx + q]);
                else if (q < fx + kLearnPairs) v = __bfloat162float(cb[b * kLearnPairs + (q - fx)]);
                X[r * Dp + q] = v;
            }
        }
    }
    if (z) {
        MRF_CUDA(h, cudaMemcpyAsync(z, h->d_Z, sizeof(float) * R * h->la.O, cudaMemcpyDeviceToHost, h->stream));
        MRF_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    return MRF_OK;
}

}  // extern "C"
