/*
 * mrf.h -- C ABI of the GB300 primal-dual Gibbs sampler (libmrf.so).
 *
 * Method: "Probabilistic Duality for Parallel Gibbs Sampling without Graph
 * Coloring" (Mescheder, Nowozin, Geiger).  A discrete pairwise MRF with
 * strictly positive factors (abstract; Section 4, Hammersley-Clifford form)
 *
 *     p(x) ~ exp( sum_v u_v(x_v) + sum_e w_e(x_s(e), x_t(e)) ),  x_v in {0..L-1}
 *
 * is sampled by the two-block Gibbs sampler of Section 5.1 on the dual
 * representation of Sections 4.1-4.2: every dualised entry of every pairwise
 * table gets one binary dual variable theta; one sweep draws all theta | x
 * (fully parallel over edges) and then all x | theta (fully parallel over
 * sites), without any graph coloring.  Section 5.4's blocked variant keeps a
 * spanning forest of every lattice block exact and samples it by
 * forward-filtering/backward-sampling.
 *
 * Conventions for every entry point
 *  - Return value: MRF_OK or an error status; nothing aborts the process.
 *    mrf_last_error() returns a text for the last failing call on a handle.
 *  - ptr_kind: MRF_PTR_HOST for host memory, MRF_PTR_DEVICE for device
 *    memory of the handle's device.  Inputs are copied; the caller keeps
 *    ownership of every buffer it passes.
 *  - All device work is ordered on the stream given to mrf_create; calls
 *    that return data to a host pointer synchronise that stream.  A handle is
 *    not thread-safe.
 *  - Layouts are row-major, innermost index last.
 *  - Random draws follow a fixed counter-based Philox4x32-10 contract keyed
 *    by (seed, chain, sweep, site or edge slot), so results do not depend on
 *    launch shapes and a run resumed at sweep t repeats the original run.
 */
#ifndef MRF_H
#define MRF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mrf mrf_t;

typedef enum {
    MRF_OK = 0,
    MRF_EINVAL = 1,      /* bad argument (null pointer, size, mode, state)      */
    MRF_ENONFINITE = 2,  /* a log-potential is NaN or infinite (factor not > 0) */
    MRF_ENOMEM = 3,      /* device allocation failed                             */
    MRF_ECUDA = 4,       /* a CUDA call failed                                   */
    MRF_ERANGE = 5,      /* index out of range, self-loop, L out of [2,16]       */
    MRF_ETIMEOUT = 6,    /* a bounded device wait gave up                        */
    MRF_ESTATE = 7       /* call not valid in the handle's current state         */
} mrf_status;

enum { MRF_PTR_HOST = 0, MRF_PTR_DEVICE = 1 };

/* Sweep modes (mrf_sweep). */
enum {
    MRF_MODE_PLAIN = 0,  /* Section 5.1: dual kernel writes bit-packed theta,
                            primal kernel gathers it over the CSR incidence  */
    MRF_MODE_FUSED = 1,  /* same chain, theta regenerated at both endpoints
                            from the counter-based RNG (never stored)        */
    MRF_MODE_SPLASH = 2, /* Section 5.4 blocked sweep on a lattice (needs
                            mrf_options.grid); 4x4x4 blocks, comb trees      */
    MRF_MODE_LEARNED = 3,/* cut-edge duals, then one Metropolis-Hastings step
                            per block with the learned proposal (needs
                            mrf_learned_setup)                               */
    MRF_MODE_SW = 4,     /* Section 4.3: Swendsen-Wang as a degenerate
                            duality (two labels or Potts-type tables, l >= 0)  */
    MRF_MODE_HIGDON = 5  /* Section 4.3: Higdon's partial Swendsen-Wang with
                            three-state duals (mrf_set_higdon)               */
};

/* Dualised table layout chosen by mrf_set_factors (mrf_info.layout). */
enum { MRF_LAYOUT_PIVOT = 0, MRF_LAYOUT_DIAG = 1 };

typedef struct {
    int32_t grid_nx, grid_ny, grid_nz; /* lattice shape (site v = x + nx*(y + ny*z))
                                          for MRF_MODE_SPLASH; 0 = not a lattice  */
    int32_t record_logp;               /* 1: keep the last sweep's log p(x_v|.)
                                          [C][N][L] for mrf_debug_logp            */
    int32_t use_graphs;                /* 1 (default): replay sweeps as a CUDA graph */
    int32_t schedule;                  /* primal schedule: 0 auto, 1 thread/site,
                                          2 CTA/site (high degree)               */
    int32_t kernel_timing;             /* 1: bracket every sweep kernel with CUDA
                                          events (graphs off); see mrf_kernel_times */
    int32_t exact_edges;               /* 1: keep every edge's exact folded table
                                          (needed by mrf_learned_setup)          */
    int32_t mlp_path;                  /* learned proposal MLP: 0 = fused tensor-core
                                          (tcgen05) kernel when its shapes allow
                                          (hidden % 64 == 0, <= 256), else 1;
                                          1 = three mma.sync GEMMs             */
    int32_t reserved[5];
} mrf_options;

typedef struct {
    int32_t n_vars, n_labels, n_chains, layout, n_entries;  /* m = dual bits per edge */
    int64_t n_edges;        /* live edges                                         */
    int64_t n_edge_slots;   /* slots (live + free), the RNG index space of edges  */
    int64_t sweep_index;    /* index t of the next sweep                          */
    int64_t n_samples;      /* label samples accumulated per site (sweeps x chains) */
    double log_const;       /* log p~(x) = log sum_theta p~(x,theta) + log_const  */
    int32_t schedule;       /* primal schedule picked by the autotuner: 1 thread per
                               (site, chain), 2 CTA per site; 0 before the first sweep */
    float tune_ms_thread, tune_ms_cta;   /* the autotuner's timings per launch      */
} mrf_info;

/* Fill *opt with defaults (no lattice, no logp record, graphs on, auto schedule). */
void mrf_default_options(mrf_options* opt);

/* Create a sampler for n_vars sites with n_labels in [2,16] labels and
 * n_chains independent chains, keyed by seed.  cuda_stream is a
 * cudaStream_t (0 = legacy default stream) on the current device.
 * Initial labels are drawn from the contract (uniform over labels). */
mrf_status mrf_create(mrf_t** out, int32_t n_vars, int32_t n_labels, int32_t n_chains,
                      uint64_t seed, const mrf_options* opt, void* cuda_stream);

/* Set the model (Section 4): unary_log [n_vars][L]; n_edges pairwise factors
 * (src[e], dst[e]) with pair_log [n_edges][L][L], row = label of src.  Every
 * value must be finite (strict positivity, abstract).  Duplicate (s,t) pairs
 * are allowed and multiply (Theorem 1).  Runs the Section 4.1-4.2
 * decomposition on the device: per dualised entry the dual weight tau and its
 * sampling thresholds, and the folded unaries.  Edge e gets slot e.
 * Errors: MRF_ENONFINITE, MRF_ERANGE (ids, self-loops), MRF_ENOMEM. */
mrf_status mrf_set_factors(mrf_t* h, const float* unary_log, int64_t n_edges,
                           const int32_t* src, const int32_t* dst, const float* pair_log,
                           int32_t ptr_kind);

/* Dynamic model (abstract, Section 6: factors added and removed between
 * sweeps): remove the edges in slots edge_ids[0..n_remove) and add n_add new
 * factors.  New edges take the freed slots in increasing slot order, then
 * fresh slots; their slot ids are written to out_new_ids (host memory).
 * Only the touched edges are re-decomposed; no coloring is maintained.
 * Errors: MRF_ERANGE for a slot that is not live, MRF_ENONFINITE. */
mrf_status mrf_edit_factors(mrf_t* h, int64_t n_remove, const int64_t* edge_ids,
                            int64_t n_add, const int32_t* src, const int32_t* dst,
                            const float* pair_log, int64_t* out_new_ids, int32_t ptr_kind);

/* Run n_sweeps sweeps (Section 5.1 or 5.4) and accumulate label counts for
 * sweeps with index >= burn-in.  Asynchronous on the handle's stream.  Plain
 * sweeps of a small model (at most 2^16 site x chain and edge x chain items)
 * with n_sweeps >= 2 run in one single-CTA launch (the same chain, bit for
 * bit, as one sweep at a time).
 *
 * MRF_MODE_SW (Section 4.3): every table is read as c + f(x_s) + g(x_t) +
 * l_{x_s} [x_s = x_t] with f, g folded into the unaries -- Potts-type tables
 * (diagonal layout): l_x = w(x,x), f = g = 0; two labels, any table:
 * l = (w00 + w11 - w01 - w10) / 2, f(1) = w10 - w00 + l, g(1) = w01 - w00 + l --
 * and needs every l >= 0.  Every edge whose endpoints agree on label x is
 * bonded with probability
 * 1 - e^{-l_x} (draw: 23-bit uniform of Philox(edge slot, t, chain, BOND)
 * compared with the exact threshold); every connected component of the
 * bonds (cluster) takes one label, label x with weight
 * exp(sum_{v in cluster} u_v(x) + sum_{bonds in cluster} log(e^{l_x} - 1))
 * (u with the offsets folded in)
 * (a bond with l_x = 0 excludes x), drawn by the inverse CDF with the 23-bit
 * uniform of Philox(smallest site of the cluster, t, chain, CLUSTER).
 * A model without live edges is accepted with any layout.  Cluster weights
 * are summed exactly in 64-bit fixed point (2^-32), so runs
 * are reproducible.  Errors: MRF_EINVAL when L >= 3 and the tables are not
 * diagonal, or some l < 0; MRF_ERANGE when sum_v max_x |u_v(x)| + sum_e max_x
 * |log(e^{l_x} - 1)| reaches 2^30; MRF_ETIMEOUT if a union-find walk
 * exceeded its bound of n_vars steps (cannot happen for a consistent forest).
 * The call synchronises the stream at its end to read that flag.  As for
 * plain sweeps, n_sweeps >= 2 sweeps of a small model (at most 2^16 site x
 * chain and edge x chain items, union-find state within 200 KB) run in one
 * single-CTA launch with the state in shared memory (the same chain, bit for
 * bit).
 * mrf_debug_logp and the log-partition estimator do not cover this mode. */
mrf_status mrf_sweep(mrf_t* h, int32_t n_sweeps, int32_t mode);

/* Fraction rho in [0, 1] of MRF_MODE_HIGDON (default 0.5).  Section 4.3:
 * with the Swendsen-Wang form 1 + (e^{l_a} - 1)[a = b] of every table, the
 * factor splits into a bond part alpha_a [a = b], alpha_a = rho (e^{l_a} - 1),
 * and a remainder A = exp(l'_a [a = b]), l'_a = log(1 + (1 - rho)(e^{l_a} - 1)),
 * that is dualised as in Sections 4.1-4.2 (one bit per label with l' != 0).
 * A sweep draws, given x, each edge's bond (probability rho (1 - e^{-l_a})
 * when both ends have label a; 23-bit uniform of Philox(edge slot, t, chain,
 * BOND)) and, for every edge that is not a bond, A's bits (the plain sweep's
 * dual-bit contract); then every cluster of the bonds takes one label with
 * weight exp(sum_{v in cluster} F_v(a) + sum_{bonds} (log alpha_a - alpha1_a -
 * alpha2_a)), F the primal field of A's bits with A's folded unaries and
 * alpha1, alpha2 the Theorem-2 terms of A's entry a, drawn as in
 * MRF_MODE_SW.  rho = 1 is Swendsen-Wang, rho = 0 a plain dual sweep of the
 * Potts form.  The fields enter the exact fixed-point cluster sums from
 * float32 (per-site rounding 2^-24 relative).  Errors as for MRF_MODE_SW;
 * MRF_ERANGE also when the fields' bound reaches 2^30; MRF_EINVAL for rho
 * outside [0, 1]. */
mrf_status mrf_set_higdon(mrf_t* h, double rho);

/* Estimated marginals out[n_vars][L] = counts / n_samples (float32) and the
 * number of samples per site.  Synchronises. */
mrf_status mrf_marginals(mrf_t* h, float* out, int64_t* n_samples, int32_t ptr_kind);

/* Raw label counts [n_vars][L] (uint32) summed over chains.  Synchronises. */
mrf_status mrf_get_counts(mrf_t* h, uint32_t* out, int32_t ptr_kind);

/* Zero the counts; sweeps with index < sweep_index + burn_in_sweeps are not counted. */
mrf_status mrf_reset_marginals(mrf_t* h, int32_t burn_in_sweeps);

/* Labels of all chains, [n_chains][n_vars] uint8.  get synchronises. */
mrf_status mrf_get_labels(mrf_t* h, uint8_t* out, int32_t ptr_kind);
mrf_status mrf_set_labels(mrf_t* h, const uint8_t* in, int32_t ptr_kind);

/* Index t of the next sweep (the RNG's sweep counter); set it to resume or
 * to replay one sweep from a given state. */
mrf_status mrf_set_sweep_index(mrf_t* h, int64_t t);

mrf_status mrf_get_info(const mrf_t* h, mrf_info* out);

/* Debug/parity views (host pointers; synchronise):
 * tau [slots][m] signed dual weight (+tau for l>0, -tau for l<0, 0 inactive),
 * thr [slots][m] packed thresholds, utilde [n_vars][L] folded unaries (float64). */
mrf_status mrf_debug_tables(mrf_t* h, float* tau, uint32_t* thr, double* utilde);
/* log p(x_v = a | .) of the last sweep [C][N][L] (needs record_logp) and the
 * number of draws the device saw within 1e-6 of a decision boundary. */
mrf_status mrf_debug_logp(mrf_t* h, float* out, uint64_t* boundary_draws);
/* Bit-packed theta of the last PLAIN/SPLASH sweep [slots][C][ceil(m/32)] uint32. */
mrf_status mrf_debug_theta(mrf_t* h, uint32_t* out);

/* Kernel ids of mrf_kernel_times. */
enum { MRF_K_DUAL = 0, MRF_K_PRIMAL = 1, MRF_K_FUSED = 2, MRF_K_POTENTIAL = 3, MRF_K_FFBS = 4,
       MRF_K_ACCUMULATE = 5, MRF_K_FEATURES = 6, MRF_K_MLP = 7, MRF_K_MH = 8,
       MRF_K_SMALL = 9,    /* whole plain sweeps of a small model in one launch (see mrf_sweep) */
       MRF_K_SW_BOND = 10, MRF_K_SW_FLATTEN = 11,
       MRF_K_SW_DRAW = 12, /* Swendsen-Wang: label draw of every cluster and the copy to its sites */
       MRF_K_SW_SMALL = 13,/* whole Swendsen-Wang sweeps of a small model in one launch */
       MRF_K_PARTIAL = 14, /* per-edge partial fields of the plain sweep for few chains and
                              tables with more than 16 entries (then MRF_K_PRIMAL adds them) */
       MRF_K_COUNT = 15 };
/* With options.kernel_timing: total device milliseconds ms[MRF_K_COUNT] and
 * launch counts launches[MRF_K_COUNT] of every sweep kernel since the last
 * call (CUDA events on the handle's stream); resets the totals.  Synchronises. */
mrf_status mrf_kernel_times(mrf_t* h, double* ms, int64_t* launches);
/* Throughput of the device's Philox4x32-10 (calls per second) measured by a
 * kernel that does nothing else: `threads` threads x `calls` calls, timed with
 * CUDA events on `cuda_stream` (0 = default stream).  A diagnostic for the
 * integer-ALU roof of the dual step. */
mrf_status mrf_philox_rate(uint64_t threads, int32_t calls, void* cuda_stream, double* calls_per_s);

/* Estimator of the log-partition function (Section 5.2).  Runs n_sweeps plain
 * sweeps from the current state and, after each, writes for every chain c
 *   log_v[i * C + c] = log p~(x) - sum_v log p(x_v | theta)
 * = log V(x, theta) of the sweep's duals theta and new labels x, with p~ the
 * model's unnormalised density exp(sum u + sum w).  At stationarity
 * E[V] = Z and E[log V] <= log Z (the gap is the mutual information of x and
 * theta): the mean of log_v is a lower bound on log Z and log(mean(exp(log_v)))
 * an unbiased-in-Z estimate.  log_v: host float64 [n_sweeps][C].  Needs the
 * exact edge tables (options.grid or options.exact_edges), else MRF_ESTATE.
 * The sweeps advance the chains and the marginal counts like mrf_sweep. */
mrf_status mrf_estimate_log_partition(mrf_t* h, int32_t n_sweeps, double* log_v);

/* The same estimator on the Swendsen-Wang duality (Sections 4.3 and 5.2):
 * n_sweeps MRF_MODE_SW sweeps, after each
 *   log_v[i * C + c] = log p~(x) - sum_clusters log p(x_cluster | theta),
 * which for the Ising model without fields is C(theta) log 2 + log p~(x)
 * (C = number of clusters).  The joint of x and the bonds is zero wherever a
 * bond joins unequal labels, so here E[V] = Z (p(x) p(theta))(support) < Z:
 * exp(log_v) is biased low, while E[log V] = log Z - I(x; theta) remains a
 * lower bound on log Z.  Same requirements as MRF_MODE_SW and
 * mrf_estimate_log_partition. */
mrf_status mrf_estimate_log_partition_sw(mrf_t* h, int32_t n_sweeps, double* log_v);

/* The same estimator on Higdon's duality (MRF_MODE_HIGDON sweeps at the
 * fraction of mrf_set_higdon): log V = log p~(x) - sum_clusters
 * log p(x_cluster | bonds, remainder's bits).  The joint is again zero where
 * a bond joins unequal labels (for rho > 0), so E[log V] = log Z - I(x; theta)
 * is the lower bound to use.  Requirements as for mrf_estimate_log_partition_sw. */
mrf_status mrf_estimate_log_partition_higdon(mrf_t* h, int32_t n_sweeps, double* log_v);

/* Primal-dual EM (local MAP, Section 5.3): n_iters iterations of
 *   xi = E[r(theta) | x]  (pi_k = sigmoid(q_k + beta1_k [x_s = i_k] + beta2_k [x_t = j_k]))
 *   x  = argmax_x h(x) exp(<s(x), xi>)  (per site: the first label of largest field)
 * from labels[C][N] (in/out, uint8, host or device per ptr_kind).  Every
 * iteration does not decrease log p~(x).  The sampler's state is untouched. */
mrf_status mrf_map_em(mrf_t* h, int32_t n_iters, uint8_t* labels, int32_t ptr_kind);

/* Blocked EM on a lattice handle (options.grid; Sections 5.3 and 5.4): the
 * duals of the comb forest of 4x4x4 blocks are not introduced; each iteration
 * i takes the block offset from the SPLASH draw with index i, the expected
 * duals of all other edges given the labels, and sets the labels to the exact
 * MAP of the resulting tree MRF (max-product, first maximum).  labels[C][N]
 * in/out as for mrf_map_em.  Every iteration does not decrease log p~(x). */
mrf_status mrf_map_em_blocked(mrf_t* h, int32_t n_iters, uint8_t* labels, int32_t ptr_kind);

/* Primal-dual mean field (Section 5.3): n_iters iterations of
 *   xi = E[r(theta) | eta],  eta = E[s(x)] from the site marginals q
 *   q_v = softmax of the field of xi
 * from marginals[C][N][L] (in/out, float32, host or device per ptr_kind; each
 * row a distribution over labels).  The sampler's state is untouched. */
mrf_status mrf_mean_field(mrf_t* h, int32_t n_iters, float* marginals, int32_t ptr_kind);

/* Tree (blocked) mean field on a lattice handle (options.grid; Sections 5.3
 * and 5.4, Figure 1 caption: the blocked EM with sum-product in place of
 * max-product).  Each iteration i takes the comb forest of the block offset
 * of the SPLASH draw with index i, the expected duals of all other edges
 * given the site marginals (theta-update), and replaces the marginals by the
 * exact site marginals of the resulting tree MRF (sum-product up and down
 * the forest; x-update).  marginals[C][N][L] in/out as for mrf_mean_field.
 * With a fixed forest neither half-step increases KL(q_x q_theta || p(x,
 * theta)) (the forest's duals summed out).  MRF_ESTATE without options.grid;
 * MRF_ENONFINITE for non-finite marginals.  The sampler's state is untouched. */
mrf_status mrf_mean_field_blocked(mrf_t* h, int32_t n_iters, float* marginals, int32_t ptr_kind);

/* Checkpoint of a handle to a file: the model's device tables (unaries,
 * edge slots, decomposition and Swendsen-Wang tables), Higdon's fraction,
 * the labels of every chain, the marginal counts and the sweep index, so
 * that mrf_load resumes the same chains: the
 * sweeps after a load are the ones the saved handle would have run, bit for
 * bit.  The learned proposal is not saved (set it up again after a load).
 * Errors: MRF_ESTATE before mrf_set_factors, MRF_EINVAL if the file cannot be
 * written / read or is not a checkpoint. */
mrf_status mrf_save(mrf_t* h, const char* path);
/* A new handle from a checkpoint, on `cuda_stream`; *out = NULL on error. */
mrf_status mrf_load(mrf_t** out, const char* path, void* cuda_stream);

/* Switch options.kernel_timing on (1) or off (0) for later sweeps. */
mrf_status mrf_set_kernel_timing(mrf_t* h, int32_t on);

/* ---- Batches of uneven graphs (dynamic-network workloads) --------------------
 * Many independent graphs, each with its own size and label count, sampled
 * together.  Graphs with the same L form one class; a class is the disjoint
 * union of its graphs and is swept by the same kernels as a single model, so
 * a batch sweep is a handful of launches (one dual and one primal kernel per
 * class) replayed as one CUDA graph, independent of the number of graphs.
 * Random draws of class L use the key of seed + L * 0x9E3779B97F4A7C15 and the
 * class-union site and edge-slot indices. */
typedef struct mrf_batch mrf_batch_t;

typedef struct {
    int32_t n_vars, n_labels;
    int32_t class_index;       /* class (sorted by L) that holds the graph            */
    int32_t site_offset;       /* first site of the graph in its class union          */
    int64_t first_edge_slot;   /* slot of the graph's edge 0 after mrf_batch_set_factors */
} mrf_batch_graph_info;

/* n_graphs graphs with n_vars[g] sites and n_labels[g] in [2,16] labels; every
 * graph gets n_chains chains. */
mrf_status mrf_batch_create(mrf_batch_t** out, int32_t n_graphs, const int32_t* n_vars, const int32_t* n_labels,
                            int32_t n_chains, uint64_t seed, const mrf_options* opt, void* cuda_stream);

/* All graphs at once, host memory, concatenated in graph order: unary_log
 * (graph g: [n_vars[g]][L_g]), n_edges[g], src/dst (graph-local site ids), and
 * pair_log (graph g's edges: [L_g][L_g] each).  Same checks as mrf_set_factors. */
mrf_status mrf_batch_set_factors(mrf_batch_t* b, const float* unary_log, const int64_t* n_edges,
                                 const int32_t* src, const int32_t* dst, const float* pair_log);

/* One edit of many graphs (host memory): remove the edges (remove_graph[i],
 * remove_slot[i]) -- slots are class-union slots as reported by
 * mrf_batch_graph_info and earlier edits -- and add edges (add_graph[i],
 * src[i], dst[i]) with graph-local ids and tables pair_log (L_g x L_g each,
 * concatenated).  Slots of the added edges go to out_slots.  Per class the
 * freed slots are reused in increasing order (mrf_edit_factors). */
mrf_status mrf_batch_edit_factors(mrf_batch_t* b, int64_t n_remove, const int32_t* remove_graph,
                                  const int64_t* remove_slot, int64_t n_add, const int32_t* add_graph,
                                  const int32_t* src, const int32_t* dst, const float* pair_log, int64_t* out_slots);

/* n_sweeps sweeps of every graph: MRF_MODE_PLAIN or MRF_MODE_FUSED (one CUDA
 * graph per sweep with options.use_graphs and a stream), or the cluster sweeps
 * MRF_MODE_SW / MRF_MODE_HIGDON, run class by class as mrf_sweep runs them on
 * one handle (same requirements: two labels or Potts-type tables; the failing
 * class is named in mrf_batch_last_error). */
mrf_status mrf_batch_sweep(mrf_batch_t* b, int32_t n_sweeps, int32_t mode);

/* ---- Device edit queue of a batch (dynamic networks: abstract, Section 6) ----
 * The edits of a round are staged in device buffers and applied by kernels
 * inside the round {edit, n sweeps}, which replays as one CUDA graph: the
 * route of every removal and addition to its class, the checks, the slot
 * rule of mrf_batch_edit_factors (freed slots reused in increasing order,
 * then fresh ones), the decomposition (Sections 4.1-4.2) of the new tables,
 * the incidence lists and the folded unaries, then the sweeps.  A rejected
 * edit changes nothing (the sweeps still run); its reasons are status bits: */
enum {
    MRF_Q_COUNT = 1,          /* staged counts above the queue's capacities           */
    MRF_Q_GRAPH = 2,          /* graph id out of range                                */
    MRF_Q_VERTEX = 4,         /* vertex id out of range                               */
    MRF_Q_LOOP = 8,           /* self-loop                                            */
    MRF_Q_SLOT = 16,          /* removed slot is not a live edge of the graph's class */
    MRF_Q_DUP = 32,           /* slot removed twice                                   */
    MRF_Q_NONFINITE = 64,     /* non-finite table value                               */
    MRF_Q_OFFDIAG = 128,      /* off-diagonal value in a diagonal-layout class        */
    MRF_Q_PAIR = 256,         /* table floats differ from n_pair or exceed capacity   */
    MRF_Q_SLOTS = 512,        /* a class has too few free slots for its additions     */
    MRF_Q_UNSORTED = 1024     /* (edit applied) a site with more than 25,600 incidences
                                 kept an unsorted incidence list: its field sums run
                                 in another order                                      */
};

/* Queue of at most max_remove removals, max_add additions and max_pair_floats
 * table floats per round.  Every class keeps extra_slots free edge slots
 * beyond its live edges (reserved when a round is first prepared and after
 * each host-side change); a round whose additions need more free slots in a
 * class than it has fails with MRF_Q_SLOTS.  Creating a queue again replaces
 * the previous one.  MRF_EINVAL for negative sizes, MRF_ENOMEM. */
mrf_status mrf_batch_queue_create(mrf_batch_t* b, int64_t max_remove, int64_t max_add, int64_t max_pair_floats,
                                  int64_t extra_slots);

/* Stage the next round's edit: the arrays of mrf_batch_edit_factors and
 * n_pair, the floats of pair_log (the sum over additions of L_g^2), copied on
 * the batch's stream from host or device memory (ptr_kind).  Pinned host or
 * device buffers are read when the copy runs: keep them unchanged until the
 * round has started.  MRF_ERANGE above the capacities, MRF_ESTATE without a
 * queue. */
mrf_status mrf_batch_queue_load(mrf_batch_t* b, int64_t n_remove, const int32_t* remove_graph,
                                const int64_t* remove_slot, int64_t n_add, const int32_t* add_graph,
                                const int32_t* src, const int32_t* dst, int64_t n_pair, const float* pair_log,
                                int32_t ptr_kind);

/* One round: the staged edit (none if nothing was staged since the previous
 * round), then n_sweeps sweeps of every graph (MRF_MODE_PLAIN or
 * MRF_MODE_FUSED).  With options.use_graphs and a stream it is one CUDA graph
 * launch (captured on the first round with this n_sweeps and mode); else the
 * same kernels are launched one by one.  Asynchronous: read the edit's
 * outcome with mrf_batch_queue_result.  MRF_ESTATE without a queue or
 * factors. */
mrf_status mrf_batch_round(mrf_batch_t* b, int32_t n_sweeps, int32_t mode);

/* Waits for the batch's stream; *status = the MRF_Q_* bits of the last round's
 * edit (0: applied) and out_slots[0..n) = the class slots of its first n
 * added edges, -1 if the edit was rejected (out_slots may be null when n = 0).
 * MRF_ERANGE if n exceeds the queue's max_add. */
mrf_status mrf_batch_queue_result(mrf_batch_t* b, uint32_t* status, int64_t n, int64_t* out_slots);
mrf_status mrf_batch_reset_marginals(mrf_batch_t* b, int32_t burn_in_sweeps);
/* Counts [n_vars[g]][L_g] and labels [n_chains][n_vars[g]] of graph g (host). */
mrf_status mrf_batch_get_counts(mrf_batch_t* b, int32_t graph, uint32_t* out);
mrf_status mrf_batch_get_labels(mrf_batch_t* b, int32_t graph, uint8_t* out);
mrf_status mrf_batch_graph(const mrf_batch_t* b, int32_t graph, mrf_batch_graph_info* out);
/* Kernel timing of every class (as mrf_set_kernel_timing; batch sweeps and
 * rounds then launch without graphs): read per class with mrf_kernel_times
 * on mrf_batch_class(b, k). */
mrf_status mrf_batch_set_kernel_timing(mrf_batch_t* b, int32_t on);
/* Number of classes and the mrf_t of class k (for info, timing and debug views;
 * owned by the batch). */
int32_t mrf_batch_n_classes(const mrf_batch_t* b);
mrf_t* mrf_batch_class(mrf_batch_t* b, int32_t k);
const char* mrf_batch_last_error(const mrf_batch_t* b);
void mrf_batch_destroy(mrf_batch_t* b);

/* ---- Learned block proposal (no counterpart in the paper) ---------------------
 * Blocks of at most 16 sites (Section 5.4 allows blocking with respect to
 * arbitrary subgraphs).  A learned sweep draws the duals of the cut edges
 * (between blocks), then gives every (block, chain) one independence
 * Metropolis-Hastings step: an MLP (features -> hidden -> hidden -> 16 x L
 * logits, bf16 weights, fp32 accumulation) proposes all the block's labels at
 * once; the step accepts with min(1, pi(x') q(x) / (pi(x) q(x'))) under the
 * exact block conditional pi (intra-block factors kept exact), so the chain
 * keeps the target whatever the weights.  Features per (block, chain):
 * centred node potentials of the members (sorted site ids) and the block's
 * pair couplings kappa_e = mean_a w(a,a) - mean_{a!=b} w(a,b); width
 * 16 L + 120 padded to a multiple of 32.  Parameters (float32, flat):
 * W1 [H][Dp], b1 [H], W2 [H][H], b2 [H], W3 [16L][H], b3 [16L]. */

/* Partition into blocks (block_of_site[v] in [0, n_blocks), host memory, at
 * most 16 sites each), hidden width H (multiple of 64), He-uniform weights from
 * init_seed.  Needs mrf_options.exact_edges.  Errors: MRF_ERANGE for a block
 * over 16 sites, MRF_ESTATE without factors or exact edges. */
mrf_status mrf_learned_setup(mrf_t* h, const int32_t* block_of_site, int32_t hidden, uint64_t init_seed);
int64_t mrf_learned_param_count(const mrf_t* h);
/* Parameters to / from host float32 (weights are used rounded to bf16). */
mrf_status mrf_learned_set_params(mrf_t* h, const float* params, int64_t n);
mrf_status mrf_learned_get_params(mrf_t* h, float* params, int64_t n);
/* Run n_sweeps plain sweeps; after each, compute the cut duals and features
 * of the new state and keep every stride-th (block, chain) row (features and
 * the block's labels) in the on-device training set (at most max_rows rows).
 * Returns the number of rows held in *rows. */
mrf_status mrf_learned_harvest(mrf_t* h, int32_t n_sweeps, int32_t stride, int64_t max_rows, int64_t* rows);
/* steps Adam steps (lr, betas 0.9/0.999, eps 1e-8) on minibatches of `batch`
 * rows drawn with replacement by a generator seeded with shuffle_seed; the
 * cross-entropy of every step goes to loss_trace[steps] (host, may be null). */
mrf_status mrf_learned_train(mrf_t* h, int32_t steps, int32_t batch, float lr, uint64_t shuffle_seed,
                             float* loss_trace);
/* Gradient of the mean cross-entropy on given rows (host): X [rows][Dp]
 * float32 (used as bf16), y [rows][16], nmem [rows]; grads [param_count]. */
mrf_status mrf_learned_grad(mrf_t* h, const float* X, const uint8_t* y, const uint8_t* nmem, int32_t rows,
                            float* grads, double* loss);
/* Logits z [rows][16 L] of the tensor-core forward pass on given features. */
mrf_status mrf_learned_forward(mrf_t* h, const float* X, int32_t rows, float* z);
/* Proposals made and accepted by learned sweeps so far. */
mrf_status mrf_learned_stats(mrf_t* h, uint64_t* proposed, uint64_t* accepted);
/* Features [n_blocks * C][Dp] and logits [n_blocks * C][16 L] of the last learned
 * sweep (host float32; rows b * C + c). */
mrf_status mrf_learned_debug(mrf_t* h, float* X, float* z);
/* Test hook for the bounded waits of the tensor-core MLP: with on = 1 the
 * next learned sweep's MLP kernel does not signal the completion of its first
 * layer, so its waits run out (after roughly a second); the kernel then
 * records the timeout, lets its own copies and MMAs finish, frees its tensor
 * memory and returns, and mrf_sweep returns MRF_ETIMEOUT.  The handle stays
 * usable.  The hook disarms itself after that sweep.  (Should the kernel's
 * own copies and MMAs not finish within the bound either, mrf_sweep returns
 * MRF_ESTATE instead and refuses further learned sweeps on the handle, which
 * must then be recreated.) */
mrf_status mrf_debug_mlp_timeout(mrf_t* h, int32_t on);

/* Capacity, in 32-bit words, of the fixed device array that holds the dual
 * bits of mrf_sweep_noalloc (16 MiB). */
#define MRF_NOALLOC_THETA_WORDS (1u << 22)

/* One plain sweep that allocates no device memory.  The paper has no
 * counterpart: this is for callers that cannot allocate device memory at the
 * moment they sweep, such as code running under a framework that forbids
 * allocation at that point, or code that keeps all device memory inside its
 * own fixed pool and wants to push several label sets of its own through one
 * loaded model.
 *   h           a handle after mrf_set_factors (its tables are the inputs)
 *   labels_in   device pointer, [n_vars][n_chains] uint8 labels (chain
 *               innermost), the state before the sweep; not modified
 *   labels_out  device pointer, [n_vars][n_chains] uint8, receives the new
 *               labels; must not overlap labels_in
 *   sweep_index index t of the sweep in the random-draw contract
 * The result equals that of mrf_sweep(h, 1, MRF_MODE_PLAIN) from the same
 * labels at sweep index t.  The handle's own labels, sweep index and counts
 * are neither read nor changed.  The dual bits go to a file-scope device array
 * of MRF_NOALLOC_THETA_WORDS words instead of a buffer of the handle; every GPU
 * that loads the library holds that array until the process exits.  The first
 * call on a device looks up the array's device address (once per device, with
 * that device current); make that first call before any stream capture.  All
 * calls share the one array and each overwrites it, so calls whose work
 * overlaps on the GPU (other streams, other threads) race.  Work is enqueued
 * on the handle's stream; the call returns without synchronising.  These
 * sweeps do not report draws within 1e-6 of a decision boundary (their
 * counter lives in the shared array and is not read back).
 * Errors: MRF_ERANGE when edge slots x chains x ceil(m/32) exceeds
 * MRF_NOALLOC_THETA_WORDS; MRF_EINVAL for null or overlapping buffers;
 * MRF_ESTATE before mrf_set_factors. */
mrf_status mrf_sweep_noalloc(mrf_t* h, const uint8_t* labels_in, uint8_t* labels_out, int64_t sweep_index);

const char* mrf_last_error(const mrf_t* h);
const char* mrf_status_string(mrf_status s);
void mrf_destroy(mrf_t* h);

#ifdef __cplusplus
}
#endif
#endif /* MRF_H */
