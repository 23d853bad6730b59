"""GPU parity of Higdon's partial Swendsen-Wang sweep (Section 4.3, three-state
duals) against the CPU oracle, through the C ABI.

Bonds are decided exactly on both sides (float64 thresholds).  The remainder's
dual bits follow the plain sweep's contract: a bit whose uniform lies within
1e-6 of its probability may differ, and the clusters of its endpoints are
exempt.  Cluster weights sum float32 potentials on the device (float64 in the
oracle): a cluster whose uniform lies within 1e-6 + 5e-7 sum_v max_a |F_v(a)|
of a CDF boundary is exempt.
"""
import numpy as np
import pytest

from oracle import brute, higdon as hg
from paper_1611_06684_gb300 import workloads as wl
from paper_1611_06684_gb300 import mrf as M
from tests.gpu_helpers import make_handle
from tests.test_gpu_sw import _two_labels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_06684_gb300 import build
    build.build()
    torch.cuda.set_device(0)


CASES = {
    "ferro3d_L8_C64_rho0.5": (lambda: wl.ferro_potts_grid3d(13, 11, 9, L=8, seed=2), 64, 0.5),
    "graph_L4_C37_rho0.3": (lambda: wl.ferro_potts_graph(300, 4, 900, seed=1), 37, 0.3),
    "two_labels_C33_rho0.7": (lambda: _two_labels(300, 900, 31), 33, 0.7),
    "ising_C32_rho0.9": (lambda: wl.ising_grid(24, 20, j_lo=0.2, j_hi=0.9, seed=32), 32, 0.9),
    "zero_entries_L5_C33_rho0.6": (lambda: wl.ferro_potts_graph(200, 5, 700, p_zero=0.3, seed=4), 33, 0.6),
    "graph_L4_C32_rho0": (lambda: wl.ferro_potts_graph(250, 4, 800, seed=7), 32, 0.0),
    "graph_L3_C32_rho1": (lambda: wl.ferro_potts_graph(500, 3, 1500, beta_lo=1.0, beta_hi=3.0, seed=3), 32, 1.0),
}


def compare_higdon(model, ref, x_gpu):
    """Labels of one sweep; returns the number of exempt (chain, site) pairs."""
    C, N = x_gpu.shape
    roots = ref["roots"]
    # A's bits at their decision boundary: the clusters of both endpoints are exempt
    near_bit = (np.abs(ref["u_dual"] - ref["p_dual"]) < 1e-6).any(axis=2) & ~ref["bonds"]   # [C][E]
    bad_root = np.zeros((C, N), bool)
    for c, e in zip(*np.nonzero(near_bit)):
        bad_root[c, roots[c, model.src[e]]] = True
        bad_root[c, roots[c, model.dst[e]]] = True
    # cluster draws within the float32 tolerance of a CDF boundary
    scale = np.abs(ref["field"]).max(axis=2)                                                 # [C][N]
    for c in range(C):
        s = np.zeros(N)
        np.add.at(s, roots[c], scale[c])
        tol = 1e-6 + 5e-7 * s
        d = np.abs(ref["u_cluster"][c][:, None] - ref["cdf_cluster"][c]).min(axis=1)
        is_root = roots[c] == np.arange(N)
        bad_root[c] |= is_root & (d < tol)
    exempt = bad_root[np.arange(C)[:, None], roots]
    exempt |= (np.abs(ref["u_bond"] - ref["p_bond"]) < 1e-12).any(axis=1)[:, None]
    bad = (x_gpu != ref["x"]) & ~exempt
    assert not bad.any(), f"{int(bad.sum())} of {bad.size} labels differ away from boundaries"
    return int(exempt.sum())


@pytest.mark.parametrize("name", list(CASES))
def test_higdon_sweeps_match_oracle(name):
    make, C, rho = CASES[name]
    model = make()
    seed = 51
    split = hg.higdon_split(model, rho)
    h = make_handle(model, C, seed)
    h.set_higdon(rho)
    h.sweep(2, M.MODE_PLAIN)
    exempt = 0
    for _ in range(3):
        t = h.info().sweep_index
        x0 = h.get_labels().astype(np.int64)
        h.sweep(1, M.MODE_HIGDON)
        ref = hg.higdon_sweep(model, x0, rho, t, seed, split=split)
        exempt += compare_higdon(model, ref, h.get_labels())
    h.close()
    assert exempt < 0.05 * 3 * C * model.n_vars


def test_higdon_at_rho_one_is_the_swendsen_wang_chain():
    model = wl.ferro_potts_graph(400, 6, 1600, beta_lo=0.5, beta_hi=2.0, seed=10)
    C, seed = 64, 52
    a = make_handle(model, C, seed)
    b = make_handle(model, C, seed)
    b.set_higdon(1.0)
    for _ in range(4):
        a.sweep(1, M.MODE_SW)
        b.sweep(1, M.MODE_HIGDON)
        assert np.array_equal(a.get_labels(), b.get_labels())
    a.close(); b.close()


def test_higdon_rho_change_rebuilds_tables():
    model = wl.ferro_potts_graph(200, 4, 600, seed=53)
    C, seed = 32, 54
    h = make_handle(model, C, seed)
    for rho in (0.2, 0.8):
        h.set_higdon(rho)
        t = h.info().sweep_index
        x0 = h.get_labels().astype(np.int64)
        h.sweep(1, M.MODE_HIGDON)
        compare_higdon(model, hg.higdon_sweep(model, x0, rho, t, seed), h.get_labels())
    h.close()


def test_higdon_marginals_match_exact():
    model = wl.ferro_potts_graph(6, 3, 9, beta_lo=0.3, beta_hi=1.5, seed=11)
    exact, _ = brute.exact_marginals(model)
    h = make_handle(model, 4096, 55)
    h.set_higdon(0.5)
    h.sweep(10, M.MODE_HIGDON)
    h.reset_marginals(0)
    h.sweep(100, M.MODE_HIGDON)
    est, ns = h.marginals()
    h.close()
    assert ns == 4096 * 100
    assert np.abs(est - exact).max() < 0.01, np.abs(est - exact).max()


def test_higdon_errors():
    m = wl.ferro_potts_graph(30, 3, 40, seed=14)
    h = make_handle(m, 4, 0)
    for bad in (-0.1, 1.5, float("nan")):
        with pytest.raises(M.MrfError) as e:
            h.set_higdon(bad)
        assert e.value.status == M.MRF_EINVAL
    h.close()
    m = wl.tiny_random(20, 3, 30, seed=12)                          # full L = 3 tables
    h = make_handle(m, 4, 0)
    with pytest.raises(M.MrfError) as e:
        h.sweep(1, M.MODE_HIGDON)
    assert e.value.status == M.MRF_EINVAL
    h.close()


def test_higdon_resumes_from_checkpoint(tmp_path):
    model = wl.ferro_potts_graph(300, 5, 900, seed=56)
    C, seed = 32, 57
    h = make_handle(model, C, seed)
    h.set_higdon(0.35)
    h.sweep(2, M.MODE_HIGDON)
    path = str(tmp_path / "hg.ckpt")
    h.save(path)
    h.sweep(3, M.MODE_HIGDON)
    want = h.get_labels()
    h.close()
    g = M.MRF.load(path)                                            # the fraction travels with the checkpoint
    g.sweep(3, M.MODE_HIGDON)
    assert np.array_equal(g.get_labels(), want)
    g.close()


@pytest.mark.parametrize("L", [4, 2])
def test_higdon_after_edits_uses_slot_ids(L):
    """Edits grow the edge slots past the tables' capacity and leave free slots;
    the split is rebuilt and the RNG index of an edge is its slot."""
    model = wl.ferro_potts_graph(300, 4, 1000, seed=58) if L == 4 else _two_labels(300, 1000, 59)
    C, seed, rho = 16, 60, 0.6
    h = make_handle(model, C, seed)
    h.set_higdon(rho)
    h.sweep(1, M.MODE_HIGDON)
    rng = np.random.default_rng(4)
    rem = np.sort(rng.choice(model.n_edges, size=100, replace=False))
    add = wl.ferro_potts_graph(300, 4, 400, seed=61) if L == 4 else _two_labels(300, 400, 62)
    ids = h.edit_factors(rem, add.src, add.dst, add.pair)           # 300 fresh slots beyond the first 1000
    src = np.concatenate([model.src, np.zeros(300, model.src.dtype)])
    dst = np.concatenate([model.dst, np.zeros(300, model.dst.dtype)])
    pair = np.concatenate([model.pair, np.zeros((300,) + model.pair.shape[1:], model.pair.dtype)])
    src[ids] = add.src; dst[ids] = add.dst; pair[ids] = add.pair
    live = np.ones(src.size, bool); live[rem] = False; live[ids] = True
    slots = np.nonzero(live)[0]
    edited = wl.Model(model.n_vars, L, model.unary, src[slots], dst[slots], pair[slots])
    for _ in range(2):
        t = h.info().sweep_index
        x0 = h.get_labels().astype(np.int64)
        h.sweep(1, M.MODE_HIGDON)
        compare_higdon(edited, hg.higdon_sweep(edited, x0, rho, t, seed, edge_ids=slots), h.get_labels())
    h.close()


SMALL = {
    "ising_C4": (lambda: wl.ising_grid(24, 20, j_lo=0.2, j_hi=0.9, seed=32), 4, 0.9),
    "graph_L4_C37": (lambda: wl.ferro_potts_graph(80, 4, 200, seed=1), 37, 0.3),
    "zero_entries_L5_C33": (lambda: wl.ferro_potts_graph(60, 5, 150, p_zero=0.3, seed=4), 33, 0.6),
}


@pytest.mark.parametrize("name", list(SMALL))
def test_higdon_small_model_kernel_is_the_same_chain(name):
    """n >= 2 Higdon sweeps of a small model run in one single-CTA launch; the
    chain, counts and sweep index equal those of one sweep per call."""
    make, C, rho = SMALL[name]
    model = make()
    seed = 63
    one = make_handle(model, C, seed)
    many = make_handle(model, C, seed, kernel_timing=True)
    for h in (one, many):
        h.set_higdon(rho)
        h.reset_marginals(2)
    for _ in range(7):
        one.sweep(1, M.MODE_HIGDON)
    many.sweep(7, M.MODE_HIGDON)
    assert "k_sw_small" in many.kernel_times()                     # the single-CTA kernel ran
    assert np.array_equal(one.get_labels(), many.get_labels())
    assert np.array_equal(one.counts(), many.counts())
    assert one.info().sweep_index == many.info().sweep_index == 7
    one.close(); many.close()


def test_higdon_log_v_of_one_sweep_matches_oracle():
    """Section 5.2's estimator on Higdon's duality: log V per chain of one sweep
    from a common state, within the float32 tolerance of the fields and of the
    drawn clusters' log-probabilities."""
    from oracle.sampler import log_softmax
    model = wl.ferro_potts_grid3d(7, 6, 5, L=4, seed=23)
    C, seed, t, rho = 32, 64, 13, 0.5
    x0 = np.random.default_rng(6).integers(0, model.n_labels, size=(C, model.n_vars))
    h = M.MRF(model.n_vars, model.n_labels, C, seed=seed, grid=model.grid)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    h.set_higdon(rho)
    h.set_labels(x0.astype(np.uint8))
    h.set_sweep_index(t)
    lv = h.estimate_log_partition(1, M.MODE_HIGDON)[0]
    x1 = h.get_labels()
    h.close()
    split = hg.higdon_split(model, rho)
    res = hg.higdon_sweep(model, x0, rho, t, seed, split=split)
    ref = hg.log_v(model, res["x"], res["bonds"], res["theta"], split)
    # chains whose labels agree and whose remainder's bits were all decided away
    # from their boundaries (a flipped bit changes the fields, hence log V)
    near_bit = ((np.abs(res["u_dual"] - res["p_dual"]) < 1e-6) & ~res["bonds"][:, :, None]).any(axis=(1, 2))
    clean = (x1 == res["x"]).all(axis=1) & ~near_bit
    assert clean.sum() >= C // 2
    tol = np.zeros(C)
    for c in range(C):
        root, lw = hg.cluster_log_weights(model, split, res["bonds"][c], res["field"][c])
        rs = np.unique(root)
        lp = log_softmax(lw[rs])[np.arange(rs.size), res["x"][c][rs]]
        tol[c] = 1e-5 * np.maximum(1.0, np.abs(lp)).sum() + 5e-7 * np.abs(res["field"][c]).max(axis=1).sum() \
            + 1e-6 * (model.n_vars + model.n_edges)
    err = np.abs(lv - ref)
    assert (err[clean] <= tol[clean]).all(), (err[clean].max(), tol[clean].min())
