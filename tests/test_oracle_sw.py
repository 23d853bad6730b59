"""Pins of the Swendsen-Wang duality (Section 4.3) by enumeration."""
import itertools

import numpy as np
import pytest

from oracle import brute, philox as ph, swendsen_wang as sw
from oracle.sampler import log_softmax
from paper_1611_06684_gb300 import workloads as wl


def _model(seed, N=5, L=3, E=6):
    """Generalised ferromagnetic Potts tables w_e(a, b) = beta_{e,a} [a = b] with a
    different beta per label, so that a label-independent slip in the bond weight
    log(e^l - 1) would not cancel out of the cluster label distribution."""
    m = wl.tiny_potts(N, L, E, seed=seed, beta_max=1.0)
    rng = np.random.default_rng(100 + seed)
    beta = rng.uniform(0.05, 1.5, (m.src.size, L)).astype(np.float32)
    pair = np.zeros((m.src.size, L, L), np.float32)
    pair[:, np.arange(L), np.arange(L)] = beta
    return wl.Model(m.n_vars, L, m.unary, m.src, m.dst, pair, name="tinypotts_gen")


def _model_two_labels(seed, N=5, E=7):
    """Two labels, arbitrary ferromagnetic tables (w00 + w11 >= w01 + w10) with
    nonzero off-diagonal entries, so that the folded offsets matter."""
    m = wl.tiny_random(N, 2, E, seed=seed)
    w = m.pair.astype(np.float64)
    k = 0.5 * (w[:, 0, 0] + w[:, 1, 1] - w[:, 0, 1] - w[:, 1, 0])
    w[:, 0, 0] += np.where(k < 0, -2 * k + 0.1, 0.0)                # make every coupling positive
    return wl.Model(m.n_vars, 2, m.unary, m.src, m.dst, w.astype(np.float32), name="tiny_two_labels")


MODELS = {"potts_L3_s1": lambda: _model(1), "potts_L3_s2": lambda: _model(2),
          "two_labels_s3": lambda: _model_two_labels(3), "two_labels_s4": lambda: _model_two_labels(4)}


def _joint_log(model, X, B):
    """log p~(x, theta) [S_x][S_theta] = sum u + sum over bonded edges of log(e^{l} - 1)
    (-inf where a bond joins unequal labels or has l = 0), from the SW tables."""
    ell, u = sw.sw_tables(model)
    lu = u[np.arange(model.n_vars)[None, :], X].sum(axis=1)
    xs, xt = X[:, model.src], X[:, model.dst]
    l_at = ell[np.arange(model.src.size)[None, :], xs]
    with np.errstate(divide="ignore"):
        lb = np.where(xs == xt, np.log(np.expm1(l_at)), -np.inf)          # [S_x][E]
    out = lu[:, None] + (B[None, :, :] * np.where(np.isfinite(lb), lb, -1e300)[:, None, :]).sum(axis=2)
    ok = ~((B[None, :, :] == 1) & ~np.isfinite(lb)[:, None, :]).any(axis=2)
    return np.where(ok, out, -np.inf)


def _normalised(lp):
    return lp - np.logaddexp.reduce(lp)


def test_decomposition_reproduces_the_factor():
    """sum_theta g(theta) exp(-theta I(a = b)) = exp(w(a, b)) with g(0) = 1,
    g(1) = e^l - 1 (the paper's g(0) = e^{-w}, g(1) = 1 - e^{-w} after scaling by e^{-l})."""
    for l in (0.1, 0.7, 2.5):
        for a, b in itertools.product(range(3), repeat=2):
            I0 = 0.0 if a == b else np.inf
            val = 1.0 + (np.expm1(l) * np.exp(-I0))
            assert abs(val - np.exp(l * (a == b))) < 1e-12
            # paper's normalisation
            assert abs(np.exp(-l) + (1 - np.exp(-l)) * np.exp(-I0) - np.exp(l * (a == b) - l)) < 1e-12


@pytest.mark.parametrize("name", list(MODELS))
def test_joint_marginalises_and_cluster_rule_is_the_conditional(name):
    model = MODELS[name]()
    X = brute.all_labelings(model.n_vars, model.n_labels)
    B = brute.all_dual_configs(model.src.size)
    J = _joint_log(model, X, B)
    # p~(x) up to the dropped constants c_e
    np.testing.assert_allclose(_normalised(np.logaddexp.reduce(J, axis=1)), _normalised(brute.log_ptilde(model, X)),
                               atol=1e-10)
    ell, u = sw.sw_tables(model)
    rng = np.random.default_rng(len(name))
    for bi in rng.choice(B.shape[0], size=6, replace=False):
        col = J[:, bi]
        if not np.isfinite(col).any():
            continue
        p_exact = np.exp(col - np.logaddexp.reduce(col))
        root = sw.clusters(model.n_vars, model.src, model.dst, B[bi].astype(bool))
        lw = sw.cluster_log_weights(u, ell, model.src, root, B[bi].astype(bool))
        rs = np.unique(root)
        lp = log_softmax(lw[rs])
        pos = {r: i for i, r in enumerate(rs)}
        p_rule = np.zeros(X.shape[0])
        for xi, x in enumerate(X):
            if all(x[v] == x[root[v]] for v in range(model.n_vars)):
                p_rule[xi] = np.exp(sum(lp[pos[r], x[r]] for r in rs))
        np.testing.assert_allclose(p_rule, p_exact, atol=1e-12)


@pytest.mark.parametrize("name", ["potts_L3_s1", "two_labels_s3"])
def test_sw_kernel_is_stationary(name):
    model = MODELS[name]()
    X = brute.all_labelings(model.n_vars, model.n_labels)
    B = brute.all_dual_configs(model.src.size)
    J = _joint_log(model, X, B)
    lp_b_x = J - np.logaddexp.reduce(J, axis=1)[:, None]                # p(theta | x)
    lp_x_b = J - np.logaddexp.reduce(J, axis=0)[None, :]                # p(x | theta)
    with np.errstate(invalid="ignore"):
        K = np.nan_to_num(np.exp(lp_b_x)) @ np.nan_to_num(np.exp(lp_x_b)).T
    _, p, _ = brute.exact_distribution(model)
    np.testing.assert_allclose(K.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(p @ K, p, atol=1e-12)


@pytest.mark.parametrize("name", ["potts_L3", "two_labels"])
def test_sw_chain_marginals_within_3_sigma(name):
    model = _model(4, N=6, L=3, E=8) if name == "potts_L3" else _model_two_labels(5, N=7, E=10)
    L = model.n_labels
    exact, _ = brute.exact_marginals(model)
    C, T, burn, seed = 512, 60, 10, 5
    x = ph.init_labels(model.n_vars, L, C, seed)
    tables = sw.sw_tables(model)
    acc = np.zeros((C, model.n_vars, L))
    for t in range(T):
        x = sw.sw_sweep(model, x, t, seed, tables=tables)["x"]
        if t >= burn:
            acc[np.arange(C)[:, None], np.arange(model.n_vars)[None, :], x] += 1
    cm = acc / (T - burn)
    z = np.abs(cm.mean(0) - exact) / np.maximum(cm.std(0, ddof=1) / np.sqrt(C), 1e-12)
    assert z.max() < 4.5 and np.mean(z < 3.0) > 0.9, z


def test_sw_tables_reject_other_models():
    with pytest.raises(ValueError):
        sw.sw_tables(wl.tiny_random(5, 3, 6, seed=1))                      # full L = 3 tables
    m = _model(1)
    m.pair[2, 1, 1] = -0.3
    with pytest.raises(ValueError):
        sw.sw_tables(m)                                                  # antiferromagnetic entry
    m = _model_two_labels(3)
    m.pair[0, 0, 1] += 10.0
    with pytest.raises(ValueError):
        sw.sw_tables(m)                                                  # w00 + w11 < w01 + w10


@pytest.mark.parametrize("name", ["potts_L3_s1", "two_labels_s3"])
def test_log_v_mean_is_log_z_minus_mutual_information(name):
    """Section 5.2 on the SW duality, by enumeration of (x, theta) under the joint.
    log V = log Z + log p(x) p(theta) / p(x, theta), so E[log V] = log Z - I(x; theta)
    exactly.  The joint is zero wherever a bond joins unequal labels, so
    E[V] = Z (p(x) x p(theta))(support) < Z: V is not unbiased on this
    degenerate duality, but E[log V] <= log E[V] < log Z keeps the lower bound."""
    model = MODELS[name]()
    X = brute.all_labelings(model.n_vars, model.n_labels)
    B = brute.all_dual_configs(model.src.size).astype(bool)
    J = _joint_log(model, X, B)                                         # up to the dropped constants
    logZ = np.logaddexp.reduce(brute.log_ptilde(model, X))
    P = np.exp(J - np.logaddexp.reduce(J.ravel()))
    tables = sw.sw_tables(model)
    lv = np.full(J.shape, np.nan)
    for bi in range(B.shape[0]):
        ok = np.isfinite(J[:, bi])
        if ok.any():
            lv[ok, bi] = sw.log_v(model, X[ok], np.repeat(B[bi][None], ok.sum(), 0), tables)
    m = P > 0
    assert np.all(np.isfinite(lv[m]))
    px, pt = P.sum(axis=1), P.sum(axis=0)
    # E[V] = Z times the product measure of the support
    mass = np.outer(px, pt)[m].sum()
    np.testing.assert_allclose(np.logaddexp.reduce(np.log(P[m]) + lv[m]), logZ + np.log(mass), atol=1e-10)
    assert mass < 1.0
    # log Z - E[log V] = I(x; theta) = sum p log p(x,theta) / (p(x) p(theta))
    mi = (P[m] * (np.log(P[m]) - np.log(np.outer(px, pt)[m]))).sum()
    np.testing.assert_allclose(logZ - (P[m] * lv[m]).sum(), mi, atol=1e-10)
    assert mi > 0


def test_log_v_of_the_ising_model_without_fields_counts_clusters():
    """Example of Section 5.2: log V = C(theta) log 2 + log p~(x)."""
    m = wl.ising_grid(4, 5, h_std=0.0, j_lo=0.2, j_hi=0.9, seed=7)
    C, seed = 64, 3
    x = ph.init_labels(m.n_vars, 2, C, seed)
    for t in range(4):
        res = sw.sw_sweep(m, x, t, seed)
        x = res["x"]
        n_clusters = np.array([np.unique(r).size for r in res["roots"]])
        np.testing.assert_allclose(sw.log_v(m, x, res["bonds"]), n_clusters * np.log(2.0) + sw.log_ptilde(m, x),
                                   rtol=0, atol=1e-10)


def test_exact_moments_match_the_enumerated_joint():
    model = MODELS["potts_L3_s2"]()
    e_logv, logZ, mi = sw.exact_moments(model)
    X = brute.all_labelings(model.n_vars, model.n_labels)
    np.testing.assert_allclose(logZ, np.logaddexp.reduce(brute.log_ptilde(model, X)), atol=1e-10)
    assert mi > 0
    np.testing.assert_allclose(e_logv, logZ - mi, atol=1e-10)
