"""Pins of the oracle's sweep (Section 5.1) by brute-force enumeration:
Theorem 1 (the joint marginalises to p(x)), Lemma 1 (the conditionals), and
stationarity of the sweep kernel; plus a Monte-Carlo check of the sampled
marginals against exact ones."""
import numpy as np
import pytest

from oracle import brute, decompose as dc, sampler, philox as ph
from paper_1611_06684_gb300 import workloads as wl


def _tiny_models():
    return [
        wl.tiny_random(4, 2, 5, seed=1),                     # L=2 pivot, m=1
        wl.tiny_random(3, 3, 3, seed=2),                     # L=3 pivot, m=4, M=12
        wl.tiny_potts(4, 3, 4, seed=3),                      # L=3 diag, m=3, M=12
        wl.tiny_random(4, 2, 6, seed=4, allow_duplicates=True),   # repeated factors multiply
        wl.ising_grid(2, 3, seed=5),                         # grid, L=2
    ]


@pytest.mark.parametrize("model", _tiny_models(), ids=lambda m: m.name)
def test_theorem1_joint_marginalises_to_target(model):
    dec = dc.decompose(model)
    X = brute.all_labelings(model.n_vars, model.n_labels)
    M = int(dec.active.sum())
    assert M <= 18
    jl = brute.joint_log(dec, X, brute.all_dual_configs(M))
    marg = np.logaddexp.reduce(jl, axis=1)
    np.testing.assert_allclose(marg, brute.log_ptilde(model, X), rtol=0, atol=1e-11)


@pytest.mark.parametrize("model", _tiny_models(), ids=lambda m: m.name)
def test_lemma1_conditionals(model):
    """p(theta | x) and p(x | theta) of the sweep equal the enumerated joint's."""
    dec = dc.decompose(model)
    X = brute.all_labelings(model.n_vars, model.n_labels)
    ent = brute.active_entries(dec)
    Th = brute.all_dual_configs(ent.shape[0])
    jl = brute.joint_log(dec, X, Th)
    # p(theta | x)
    cond_t = jl - np.logaddexp.reduce(jl, axis=1, keepdims=True)
    pa = sampler.dual_probs(dec, X)[:, ent[:, 0], ent[:, 1]]
    mine = (np.log(pa)[:, None, :] * Th[None] + np.log1p(-pa)[:, None, :] * (1 - Th[None])).sum(-1)
    np.testing.assert_allclose(mine, cond_t, atol=1e-11)
    # p(x | theta)
    cond_x = jl - np.logaddexp.reduce(jl, axis=0, keepdims=True)
    E, m = dec.ell.shape
    th_full = np.zeros((Th.shape[0], E, m)); th_full[:, ent[:, 0], ent[:, 1]] = Th
    lp = sampler.log_softmax(sampler.primal_field(dec, th_full))
    N = model.n_vars
    mine_x = lp[:, np.arange(N)[None, :], X].sum(-1).T
    np.testing.assert_allclose(mine_x, cond_x, atol=1e-11)


@pytest.mark.parametrize("model", _tiny_models(), ids=lambda m: m.name)
def test_sweep_kernel_is_stationary(model):
    """p K = p for the exact transition matrix of one sweep."""
    dec = dc.decompose(model)
    X, p, _ = brute.exact_distribution(model)
    K = brute.sweep_kernel(dec, X)
    np.testing.assert_allclose(K.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(p @ K, p, atol=1e-12)


def test_stationarity_fails_for_a_planted_mistake():
    """Control: swapping beta1/beta2 (a plausible routing error) breaks p K = p."""
    model = wl.tiny_random(3, 3, 3, seed=2)
    dec = dc.decompose(model)
    X, p, _ = brute.exact_distribution(model)
    dec.beta1, dec.beta2 = dec.beta2.copy(), dec.beta1.copy()
    K = brute.sweep_kernel(dec, X)
    assert np.abs(p @ K - p).max() > 1e-4


def test_sampled_marginals_within_3_sigma():
    model = wl.tiny_random(5, 3, 6, seed=12, w_std=0.8)
    dec = dc.decompose(model)
    exact, _ = brute.exact_marginals(model)
    C, T, burn = 512, 120, 20
    runs = []
    for seed in (78, 79):                                   # two independent runs, 1024 chains
        x = ph.init_labels(model.n_vars, model.n_labels, C, seed=seed)
        acc = np.zeros((C, model.n_vars, model.n_labels))
        for t in range(T):
            x = sampler.sweep(dec, x, t, seed)["x"]
            if t >= burn:
                acc[np.arange(C)[:, None], np.arange(model.n_vars)[None, :], x] += 1
        runs.append(acc / (T - burn))
    chain_means = np.concatenate(runs)
    C = chain_means.shape[0]
    est = chain_means.mean(0)
    sigma = chain_means.std(0, ddof=1) / np.sqrt(C)
    z = np.abs(est - exact) / np.maximum(sigma, 1e-12)
    assert z.max() < 4.0 and np.mean(z < 3.0) > 0.95, (z.max(), est, exact)


def test_theta_frequency_matches_probability():
    """Bernoulli draws theta = [u < p] follow p: empirical frequency over many
    (edge, chain) draws matches the mean of p within 4 sigma."""
    model = wl.potts_grid3d(4, 4, 4, L=3, seed=3)
    dec = dc.decompose(model)
    x = ph.init_labels(model.n_vars, 3, 32, seed=5)
    theta, p, u = sampler.dual_step(dec, x, 0, 5)
    act = dec.active[None] & np.ones_like(theta, bool)
    f, pm = theta[act].mean(), p[act].mean()
    n = act.sum()
    assert abs(f - pm) < 4 * np.sqrt(pm * (1 - pm) / n)


def test_inverse_cdf_rule():
    logp = np.log(np.array([[0.2, 0.3, 0.5]]))
    for u, want in [(0.0, 0), (0.199999, 0), (0.2000001, 1), (0.4999999, 1), (0.5, 2), (0.50001, 2), (0.999999, 2)]:
        x, _ = sampler.inverse_cdf(logp, np.array([u]))
        assert x[0] == want
    # rounding leaves none: pick the largest label with p > 0
    x, _ = sampler.inverse_cdf(np.log(np.array([[0.5, 0.5 - 1e-9, 0.0]])), np.array([0.9999999999]))
    assert x[0] == 1


def test_sub_model_sweep_equals_full_sweep_at_sampled_sites():
    """A sweep of the sampled sites' incident edges (with the full model's edge
    slots and site ids as RNG indices) draws exactly the full sweep's labels at
    those sites: a site's conditional involves only its incident edges."""
    model = wl.potts_grid3d(7, 6, 5, L=4, seed=3)
    dec = dc.decompose(model)
    C, seed, t = 3, 11, 4
    x0 = np.random.default_rng(2).integers(0, 4, size=(C, model.n_vars))
    full = sampler.sweep(dec, x0, t, seed)
    sites = np.sort(np.random.default_rng(4).choice(model.n_vars, size=25, replace=False))
    eids = np.nonzero(np.isin(model.src, sites) | np.isin(model.dst, sites))[0]
    local = np.unique(np.concatenate([sites, model.src[eids], model.dst[eids]]))
    sub = wl.Model(n_vars=len(local), n_labels=4, unary=model.unary[local],
                   src=np.searchsorted(local, model.src[eids]).astype(np.int32),
                   dst=np.searchsorted(local, model.dst[eids]).astype(np.int32), pair=model.pair[eids])
    ref = sampler.sweep(dc.decompose(sub), x0[:, local], t, seed, edge_ids=eids, site_ids=local)
    pos = np.searchsorted(local, sites)
    assert np.array_equal(ref["x"][:, pos], full["x"][:, sites])
    np.testing.assert_allclose(ref["logp"][:, pos], full["logp"][:, sites], rtol=0, atol=1e-12)
    assert np.array_equal(ref["theta"], full["theta"][:, eids])
