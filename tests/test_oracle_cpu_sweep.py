"""Pin of the OpenMP float32 CPU sweep (oracle/cpu_sweep.c) against the float64
numpy oracle: the same dual bits and labels away from decision boundaries."""
import numpy as np
import pytest

from oracle import cpu_sweep, decompose as dc, philox as ph, sampler
from paper_1611_06684_gb300 import workloads as wl

CASES = [
    (lambda: wl.potts_grid3d(7, 6, 5, L=8, seed=1), 8),       # PIVOT, 49 entries (two groups)
    (lambda: wl.tiny_potts(200, 4, 700, seed=2), 5),           # DIAG, 4 entries (packed planes)
    (lambda: wl.ising_grid(12, 10, seed=3), 3),                # L = 2, one entry
    (lambda: wl.random_graph(80, k=2, L=16, seed=4, w_std=0.3), 2),   # 225 entries (eight groups)
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_cpu_sweep_matches_oracle(case):
    model, C = CASES[case][0](), CASES[case][1]
    dec = dc.decompose(model)
    seed, t = 99, 3
    x0 = ph.init_labels(model.n_vars, model.n_labels, C, seed)
    cs = cpu_sweep.CpuSweep(dec, C, seed, threads=2)
    x1 = cs.sweep(x0, t)
    ref = sampler.sweep(dec, x0, t, seed)
    dual_b, site_b = sampler.boundary_draws(ref["p_dual"], ref["u_dual"], ref["cdf"], ref["u_site"])
    th = cs.theta_bits()
    bad_theta = (th != ref["theta"]) & ~dual_b
    assert not bad_theta.any(), int(bad_theta.sum())
    exempt = site_b.copy()
    for c_, e_ in zip(*np.nonzero(((th != ref["theta"]) | (dual_b & dec.active[None])).any(axis=2))):
        exempt[c_, dec.src[e_]] = True
        exempt[c_, dec.dst[e_]] = True
    bad = (x1 != ref["x"]) & ~exempt
    assert not bad.any(), int(bad.sum())


def test_cpu_sweep_threads_agree():
    model = wl.potts_grid3d(6, 5, 4, L=4, seed=5)
    dec = dc.decompose(model)
    x0 = ph.init_labels(model.n_vars, model.n_labels, 4, 7)
    a = cpu_sweep.CpuSweep(dec, 4, 7, threads=1).sweep(x0, 1)
    b = cpu_sweep.CpuSweep(dec, 4, 7, threads=3).sweep(x0, 1)
    assert np.array_equal(a, b)
