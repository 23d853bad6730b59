"""CPU FP64 oracle for the primal-dual Gibbs sampler (test infrastructure).

This package is the plain, slow, obviously-correct statement of what the
sampler computes, written from the paper ("Probabilistic Duality for
Parallel Gibbs Sampling without Graph Coloring", Mescheder, Nowozin,
Geiger) in numpy float64.  It is test infrastructure only: the tests, the
smoke check and the benchmark's CPU-baseline leg may use it; the library
never does.  It shares no code with the CUDA path; the only module both
sides import is the seeded input generator (paper_1611_06684_gb300.workloads),
which contains none of the sampler's arithmetic.

Modules
  philox       counter-based RNG (Salmon et al., SC'11) and the draw contract
  decompose    Section 4.1/4.2 factor decomposition (literal and closed form)
  sampler      Section 5.1 two-block sweep: theta | x, then x | theta
  blocked      Section 5.4 blocking: exact forward-filter/backward-sample on trees
  learned      MLP block proposal with Metropolis-Hastings correction
  brute        enumeration of p(x), p(x, theta) and the sweep kernel (tiny models)
  diagnostics  TV distance, ESS (Geyer), PSRF (Gelman-Rubin)

Parity status per function is stated in each module's header.
"""
