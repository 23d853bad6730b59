"""Pins of the sequential Gibbs sampler (the comparator of Section 6)."""
import numpy as np
import pytest

from oracle import brute, gibbs
from oracle.sampler import log_softmax
from paper_1611_06684_gb300 import workloads as wl


def _enumerated_conditional(model, X, v, x_row):
    lp = brute.log_ptilde(model, X)
    match = np.all(np.delete(X, v, axis=1) == np.delete(x_row, v)[None, :], axis=1)
    sub = lp[match]
    labs = X[match, v]
    out = np.full(model.n_labels, -np.inf)
    out[labs] = sub
    return out - np.logaddexp.reduce(out)


@pytest.mark.parametrize("model", [wl.tiny_random(4, 3, 5, seed=1, w_std=0.9), wl.tiny_potts(5, 3, 6, seed=2, beta_max=1.5)])
def test_site_conditional_is_the_enumerated_conditional(model):
    X = brute.all_labelings(model.n_vars, model.n_labels)
    rng = np.random.default_rng(0)
    x = rng.integers(0, model.n_labels, size=(6, model.n_vars))
    for v in range(model.n_vars):
        lp = log_softmax(gibbs.site_field(model, x, v))
        for c in range(6):
            np.testing.assert_allclose(lp[c], _enumerated_conditional(model, X, v, x[c]), rtol=0, atol=1e-12)


def _sweep_kernel(model, X):
    K = np.eye(X.shape[0])
    for v in range(model.n_vars):
        K = K @ gibbs.site_kernel(model, X, v)
    return K


@pytest.mark.parametrize("model", [wl.tiny_random(4, 3, 5, seed=3, w_std=1.0), wl.ising_grid(2, 3, seed=4)])
def test_sweep_kernel_leaves_p_invariant(model):
    X, p, _ = brute.exact_distribution(model)
    K = _sweep_kernel(model, X)
    np.testing.assert_allclose(K.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(p @ K, p, rtol=0, atol=1e-12)


def test_planted_transposed_table_breaks_invariance():
    """A site field that reads a destination site's table transposed (a
    plausible slip for asymmetric tables) is no longer stationary."""
    model = wl.tiny_random(4, 3, 5, seed=3, w_std=1.0)
    X, p, _ = brute.exact_distribution(model)
    bad = wl.Model(model.n_vars, model.n_labels, model.unary, model.src, model.dst,
                   np.ascontiguousarray(np.transpose(model.pair, (0, 2, 1))), name="transposed")
    K = np.eye(X.shape[0])
    index = {tuple(r): i for i, r in enumerate(X)}
    for v in range(model.n_vars):
        # the kernel of the slipped sampler: destinations see w_e^T, sources see w_e
        lp_ok = log_softmax(gibbs.site_field(model, X, v))
        lp_bad = log_softmax(gibbs.site_field(bad, X, v))
        is_dst = np.isin(v, model.dst)
        lp = lp_bad if is_dst else lp_ok
        Kv = np.zeros_like(K)
        for i in range(X.shape[0]):
            y = X[i].copy()
            for a in range(model.n_labels):
                y[v] = a
                Kv[i, index[tuple(y)]] += np.exp(lp[i, a])
        K = K @ Kv
    assert np.abs(p @ K - p).max() > 1e-4


def test_independent_set_update_equals_single_site_updates():
    """Redrawing the sites of a colour class together has the exact kernel of
    redrawing them one after another (they are conditionally independent)."""
    model = wl.ising_grid(2, 3, seed=5)
    X, p, _ = brute.exact_distribution(model)
    classes = gibbs.grid_colour_classes((3, 2, 1))
    index = {tuple(r): i for i, r in enumerate(X)}
    for sites in classes:
        K_seq = np.eye(X.shape[0])
        for v in sites:
            K_seq = K_seq @ gibbs.site_kernel(model, X, v)
        lp = log_softmax(gibbs.class_fields(model, X, np.asarray(sites)))     # [S][n][L]
        K_cls = np.zeros_like(K_seq)
        import itertools
        for i in range(X.shape[0]):
            for labs in itertools.product(range(model.n_labels), repeat=len(sites)):
                y = X[i].copy()
                y[sites] = labs
                K_cls[i, index[tuple(y)]] += np.exp(sum(lp[i, k, a] for k, a in enumerate(labs)))
        np.testing.assert_allclose(K_cls, K_seq, rtol=0, atol=1e-12)


def test_class_sweep_marginals_within_3_sigma():
    model = wl.ising_grid(3, 3, seed=6)
    marg, _ = brute.exact_marginals(model)
    rng = np.random.default_rng(7)
    C, T, burn = 256, 300, 50
    x = rng.integers(0, 2, size=(C, model.n_vars))
    classes = gibbs.grid_colour_classes((3, 3, 1))
    acc = np.zeros((C, model.n_vars))
    for t in range(T):
        gibbs.sweep_classes(model, x, rng, classes)
        if t >= burn:
            acc += x
    est = acc / (T - burn)                                  # per-chain estimates of P(x_v = 1)
    mean = est.mean(axis=0)
    sd = est.std(axis=0, ddof=1) / np.sqrt(C)
    assert (np.abs(mean - marg[:, 1]) <= 3 * sd + 1e-12).all()
