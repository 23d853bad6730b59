"""GPU parity of the Swendsen-Wang sweep (Section 4.3: Swendsen-Wang as a
degenerate duality) against the CPU oracle, through the C ABI.

Bond decisions are exact on both sides (the device compares the 23-bit draw
with a threshold computed in float64 from the same l).  Cluster weights are
exact sums on the device (fixed point, 2^-32 per term) and the label draw
rounds to float32 as the plain sweep does: a cluster whose uniform lies within
1e-6 of a CDF boundary may differ, and all its sites are exempt.
"""
import numpy as np
import pytest

from oracle import brute, swendsen_wang as sw
from paper_1611_06684_gb300 import workloads as wl
from paper_1611_06684_gb300 import mrf as M
from tests.gpu_helpers import make_handle, BOUNDARY_EPS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_06684_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _no_edges():
    rng = np.random.default_rng(31)
    return wl.Model(n_vars=37, n_labels=3, unary=rng.normal(size=(37, 3)).astype(np.float32),
                    src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32), pair=np.zeros((0, 3, 3), np.float32),
                    name="no_edges")


def _two_labels(N=300, E=900, seed=17):
    """Two labels, arbitrary tables made ferromagnetic (w00 + w11 >= w01 + w10),
    off-diagonal entries nonzero: the folded unary offsets matter."""
    m = wl.tiny_random(N, 2, E, seed=seed)
    w = m.pair.astype(np.float64)
    k = 0.5 * (w[:, 0, 0] + w[:, 1, 1] - w[:, 0, 1] - w[:, 1, 0])
    w[:, 1, 1] += np.where(k < 0, -2 * k + 0.05, 0.0)
    return wl.Model(m.n_vars, 2, m.unary, m.src, m.dst, w.astype(np.float32), name="two_labels")


CASES = {
    # the paper's Ising example: 2-D grid, L = 2, one chain
    "ising32_C1": (lambda: wl.ising_grid(32, 32, seed=0), 1),
    "ising64_strong_C64": (lambda: wl.ising_grid(64, 64, j_lo=0.4, j_hi=0.9, seed=18), 64),
    "two_labels_C33": (_two_labels, 33),
    # label-dependent couplings, ragged chain count
    "graph_L4_C37": (lambda: wl.ferro_potts_graph(300, 4, 900, seed=1), 37),
    # the lattice shape of the Swendsen-Wang benchmark, small
    "ferro3d_L8_C64": (lambda: wl.ferro_potts_grid3d(13, 11, 9, L=8, seed=2), 64),
    # strong couplings: clusters spanning most of the graph
    "strong_L3_C32": (lambda: wl.ferro_potts_graph(500, 3, 1500, beta_lo=1.0, beta_hi=3.0, seed=3), 32),
    # some l_x = 0: a bond at another label excludes x from its cluster
    "zero_entries_L5_C33": (lambda: wl.ferro_potts_graph(200, 5, 700, p_zero=0.3, seed=4), 33),
    "L16_C32": (lambda: wl.ferro_potts_graph(60, 16, 150, seed=5), 32),
    "isolated_sites_L4_C7": (lambda: wl.ferro_potts_graph(80, 4, 30, seed=6), 7),
    "no_edges_C4": (_no_edges, 4),
    # every coupling zero: no bond can form, each site is its own cluster
    "zero_couplings_L3_C32": (lambda: wl.ferro_potts_graph(150, 3, 400, beta_lo=0.0, beta_hi=0.0, seed=8), 32),
}


def compare_sw(ref, x_gpu):
    """Labels of one sweep; returns the number of exempt (chain, site) pairs."""
    C, N = x_gpu.shape
    near = np.any(np.abs(ref["u_cluster"][..., None] - ref["cdf_cluster"]) < BOUNDARY_EPS, axis=-1)
    exempt = near[np.arange(C)[:, None], ref["roots"]]
    # a bond draw exactly at its threshold (both sides decide in float64): the chain is exempt
    exempt |= (np.abs(ref["u_bond"] - ref["p_bond"]) < 1e-12).any(axis=1)[:, None]
    bad = (x_gpu != ref["x"]) & ~exempt
    assert not bad.any(), f"{int(bad.sum())} of {bad.size} labels differ away from boundaries"
    return int(exempt.sum())


def test_sw_tables_match_oracle():
    """Per-edge bond thresholds are the oracle's probabilities, and cluster
    weights use the oracle's folded unaries: checked through one sweep from a
    state where every edge agrees, on both table forms."""
    for model in (_two_labels(60, 150, 19), wl.ferro_potts_graph(60, 5, 150, seed=20)):
        C, seed = 32, 47
        h = make_handle(model, C, seed)
        x0 = np.zeros((C, model.n_vars), np.uint8)
        h.set_labels(x0)
        h.set_sweep_index(9)
        h.sweep(1, M.MODE_SW)
        ref = sw.sw_sweep(model, x0.astype(np.int64), 9, seed)
        compare_sw(ref, h.get_labels())
        h.close()


@pytest.mark.parametrize("name", list(CASES))
def test_sw_sweeps_match_oracle(name):
    model, C = CASES[name][0](), CASES[name][1]
    seed = 41
    tables = sw.sw_tables(model)
    h = make_handle(model, C, seed)
    h.sweep(2, M.MODE_PLAIN)                       # a state reached by the plain sampler
    exempt = 0
    for _ in range(3):
        t = h.info().sweep_index
        x0 = h.get_labels().astype(np.int64)
        h.sweep(1, M.MODE_SW)
        ref = sw.sw_sweep(model, x0, t, seed, tables=tables)
        exempt += compare_sw(ref, h.get_labels())
    h.close()
    assert exempt < 0.01 * 3 * C * model.n_vars


def test_sw_alternates_with_plain_sweeps():
    model = wl.ferro_potts_graph(250, 4, 800, seed=7)
    C, seed = 32, 42
    from oracle import decompose as dc, sampler
    dec = dc.decompose(model)
    h = make_handle(model, C, seed)
    from tests.gpu_helpers import compare_sweep
    for mode in (M.MODE_SW, M.MODE_PLAIN, M.MODE_SW, M.MODE_FUSED, M.MODE_SW):
        t = h.info().sweep_index
        x0 = h.get_labels().astype(np.int64)
        h.sweep(1, mode)
        if mode == M.MODE_SW:
            compare_sw(sw.sw_sweep(model, x0, t, seed), h.get_labels())
        else:
            compare_sweep(dec, sampler.sweep(dec, x0, t, seed), h.get_labels())
    assert h.info().sweep_index == 5
    h.close()


@pytest.mark.parametrize("L", [4, 2])
def test_sw_after_edits_uses_slot_ids(L):
    model = wl.ferro_potts_graph(300, 4, 1000, seed=8) if L == 4 else _two_labels(300, 1000, 21)
    C, seed = 16, 43
    h = make_handle(model, C, seed)
    h.sweep(1, M.MODE_SW)
    rng = np.random.default_rng(3)
    rem = np.sort(rng.choice(model.n_edges, size=120, replace=False))
    # fewer additions than removals: some slots stay free
    add = wl.ferro_potts_graph(300, 4, 80, seed=9) if L == 4 else _two_labels(300, 80, 22)
    ids = h.edit_factors(rem, add.src, add.dst, add.pair)
    live = np.ones(model.n_edges, bool); live[rem] = False
    live[ids] = True
    src = model.src.copy(); dst = model.dst.copy(); pair = model.pair.copy()
    src[ids] = add.src; dst[ids] = add.dst; pair[ids] = add.pair
    slots = np.nonzero(live)[0]
    edited = wl.Model(model.n_vars, L, model.unary, src[slots], dst[slots], pair[slots])
    for _ in range(2):
        t = h.info().sweep_index
        x0 = h.get_labels().astype(np.int64)
        h.sweep(1, M.MODE_SW)
        compare_sw(sw.sw_sweep(edited, x0, t, seed, edge_ids=slots), h.get_labels())
    h.close()


def test_sw_is_reproducible_and_graph_replay_identical():
    import torch
    model = wl.ferro_potts_graph(400, 6, 1600, beta_lo=0.5, beta_hi=2.0, seed=10)
    C, seed = 64, 44
    s = torch.cuda.Stream()
    out = []
    for graphs in (True, False, True):
        h = make_handle(model, C, seed, use_graphs=graphs, stream=s.cuda_stream)
        h.sweep(6, M.MODE_SW)
        out.append(h.get_labels())
        h.close()
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_sw_marginals_match_exact():
    model = wl.ferro_potts_graph(6, 3, 9, beta_lo=0.3, beta_hi=1.5, seed=11)
    exact, _ = brute.exact_marginals(model)
    h = make_handle(model, 4096, 45)
    h.sweep(10, M.MODE_SW)
    h.reset_marginals(0)
    h.sweep(100, M.MODE_SW)
    est, ns = h.marginals()
    h.close()
    assert ns == 4096 * 100
    # 409600 samples, autocorrelated over a few sweeps at most: std < 0.002
    assert np.abs(est - exact).max() < 0.01, np.abs(est - exact).max()


def test_sw_errors():
    # full tables (pivot layout)
    m = wl.tiny_random(20, 3, 30, seed=12)
    h = make_handle(m, 4, 0)
    with pytest.raises(M.MrfError) as e:
        h.sweep(1, M.MODE_SW)
    assert e.value.status == M.MRF_EINVAL
    h.close()
    # two labels, antiferromagnetic coupling
    m = wl.ising_grid(8, 8, j_lo=-0.5, j_hi=-0.1, seed=13)
    h = make_handle(m, 4, 0)
    with pytest.raises(M.MrfError) as e:
        h.sweep(1, M.MODE_SW)
    assert e.value.status == M.MRF_EINVAL
    h.close()
    # an antiferromagnetic diagonal entry
    m = wl.ferro_potts_graph(30, 3, 40, seed=14)
    m.pair[5, 1, 1] = -0.5
    h = make_handle(m, 4, 0)
    with pytest.raises(M.MrfError) as e:
        h.sweep(1, M.MODE_SW)
    assert e.value.status == M.MRF_EINVAL
    h.close()
    # cluster weights beyond the fixed-point range
    m = wl.ferro_potts_graph(30, 3, 40, seed=15)
    m.unary[3, 0] = 2.0e9
    h = make_handle(m, 4, 0)
    with pytest.raises(M.MrfError) as e:
        h.sweep(1, M.MODE_SW)
    assert e.value.status == M.MRF_ERANGE
    # the handle stays usable: fix the unary and sweep
    m.unary[3, 0] = 0.0
    h.set_factors(m.unary, m.src, m.dst, m.pair)
    h.sweep(2, M.MODE_SW)
    h.close()


def test_sw_full_size_lattice_sampled_chains():
    """The Swendsen-Wang benchmark workload (ferromagnetic 3-D Potts 128^3,
    L = 8, 64 chains, CUDA graph replay): whole chains 0, 29 and 63 of the
    third sweep against the oracle."""
    import torch
    model = wl.ferro_potts_grid3d(128, L=8, seed=0)
    C, seed = 64, 0
    s = torch.cuda.Stream()
    h = M.MRF(model.n_vars, model.n_labels, C, seed=seed, stream=s.cuda_stream, grid=model.grid)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    h.sweep(2, M.MODE_SW)
    t = h.info().sweep_index
    x0 = h.get_labels()
    h.sweep(1, M.MODE_SW)
    x1 = h.get_labels()
    h.close()
    chains = np.array([0, 29, 63])
    ref = sw.sw_sweep(model, x0[chains].astype(np.int64), t, seed, chain_ids=chains)
    n_ex = compare_sw(ref, x1[chains])
    assert n_ex < 0.01 * x1[chains].size


def test_sw_resumes_from_checkpoint(tmp_path):
    model = wl.ferro_potts_graph(300, 5, 900, seed=16)
    C, seed = 32, 46
    h = make_handle(model, C, seed)
    h.sweep(3, M.MODE_SW)
    path = str(tmp_path / "sw.ckpt")
    h.save(path)
    h.sweep(4, M.MODE_SW)
    want = h.get_labels()
    h.close()
    g = M.MRF.load(path)
    g.sweep(4, M.MODE_SW)
    assert np.array_equal(g.get_labels(), want)
    g.close()


@pytest.mark.parametrize("which", ["ferro3d_L4", "ising_L2"])
def test_sw_log_v_of_one_sweep_matches_oracle(which):
    """Section 5.2's estimator on the Swendsen-Wang duality: log V per chain of
    one sweep from a common state, within the summed per-cluster float32
    tolerance of the drawn labels' log-probabilities."""
    from oracle.sampler import log_softmax
    if which == "ferro3d_L4":
        model = wl.ferro_potts_grid3d(7, 6, 5, L=4, seed=23)
    else:
        model = wl.ising_grid(12, 10, j_lo=0.2, j_hi=0.8, seed=24)
    C, seed, t = 32, 48, 13
    x0 = np.random.default_rng(5).integers(0, model.n_labels, size=(C, model.n_vars))
    h = M.MRF(model.n_vars, model.n_labels, C, seed=seed, grid=model.grid)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    h.set_labels(x0.astype(np.uint8))
    h.set_sweep_index(t)
    lv = h.estimate_log_partition(1, M.MODE_SW)[0]
    x1 = h.get_labels()
    h.close()
    tables = sw.sw_tables(model)
    res = sw.sw_sweep(model, x0, t, seed, tables=tables)
    ref = sw.log_v(model, res["x"], res["bonds"], tables)
    near = np.any(np.abs(res["u_cluster"][..., None] - res["cdf_cluster"]) < BOUNDARY_EPS, axis=-1)
    clean = (x1 == res["x"]).all(axis=1) & ~(near & (res["roots"] == np.arange(model.n_vars)[None, :])).any(axis=1)
    assert clean.sum() >= C // 2
    tol = np.zeros(C)
    for c in range(C):
        root = res["roots"][c]
        rs = np.unique(root)
        lw = sw.cluster_log_weights(tables[1], tables[0], model.src, root, res["bonds"][c])
        lp = log_softmax(lw[rs])[np.arange(rs.size), res["x"][c][rs]]
        tol[c] = 1e-5 * np.maximum(1.0, np.abs(lp)).sum() + 1e-6 * (model.n_vars + model.n_edges)
    err = np.abs(lv - ref)
    assert (err[clean] <= tol[clean]).all(), (err[clean].max(), tol[clean].min())


def test_sw_estimator_moments_match_enumeration():
    """Many chains of a tiny model at stationarity: the mean of log V over
    Swendsen-Wang sweeps matches the exact E[log V] = log Z - I(x; theta)."""
    model = wl.ferro_potts_graph(5, 3, 6, beta_lo=0.2, beta_hi=1.2, seed=25)
    e_logv, logZ, mi = sw.exact_moments(model)
    C = 8192
    h = M.MRF(model.n_vars, 3, C, seed=26, exact_edges=True)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    h.sweep(20, M.MODE_SW)
    lv = h.estimate_log_partition(16, M.MODE_SW).ravel()
    h.close()
    n_eff = lv.size / 4                                               # consecutive sweeps are correlated
    se_mean = lv.std() / np.sqrt(n_eff)
    assert abs(lv.mean() - e_logv) < 4 * se_mean + 1e-6, (lv.mean(), e_logv, se_mean)
    assert e_logv < logZ and mi > 0


SMALL = {
    "ising32_C1": (lambda: wl.ising_grid(32, 32, seed=0), 1),
    "graph_L4_C37": (lambda: wl.ferro_potts_graph(80, 4, 200, seed=1), 37),
    "zero_entries_L5_C33": (lambda: wl.ferro_potts_graph(60, 5, 150, p_zero=0.3, seed=4), 33),
}


@pytest.mark.parametrize("name", list(SMALL))
def test_sw_small_model_kernel_is_the_same_chain(name):
    """n >= 2 sweeps of a small model run in one single-CTA launch; the chain,
    counts and sweep index equal those of one sweep per call."""
    model, C = SMALL[name][0](), SMALL[name][1]
    seed = 49
    one = make_handle(model, C, seed)
    many = make_handle(model, C, seed, kernel_timing=True)
    for h in (one, many):
        h.reset_marginals(2)
    for _ in range(7):
        one.sweep(1, M.MODE_SW)
    many.sweep(7, M.MODE_SW)
    assert "k_sw_small" in many.kernel_times()                     # the single-CTA kernel ran
    assert np.array_equal(one.get_labels(), many.get_labels())
    assert np.array_equal(one.counts(), many.counts())
    assert one.info().sweep_index == many.info().sweep_index == 7
    assert many.boundary_draws() == one.boundary_draws()
    one.close(); many.close()
