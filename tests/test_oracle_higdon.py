"""Pins of Higdon's partial Swendsen-Wang duality (Section 4.3) by enumeration."""
import itertools

import numpy as np
import pytest

from oracle import brute, higdon as hg, philox as ph, swendsen_wang as sw
from oracle.sampler import log_softmax, primal_field
from paper_1611_06684_gb300 import workloads as wl
from tests.test_oracle_sw import _model as _potts_model, _model_two_labels


def _joint_log(model, rho, X, states):
    """log p~(x, theta) [S_x][S_theta] from the split written out: per edge either
    a bond (log alpha_{x_s} if x_s = x_t, else impossible) or A's bits theta'
    with the Theorem-2 form of each entry k,
    alpha1 y_k + alpha2 z_k + theta'_k (q_k + beta1 y_k + beta2 z_k) - log(1 + e^{q_k})."""
    ell, u = sw.sw_tables(model)
    alpha, dec = hg.higdon_split(model, rho)
    src, dst = np.asarray(model.src), np.asarray(model.dst)
    L = model.n_labels
    out = u[np.arange(model.n_vars)[None, :], X].sum(axis=1)[:, None].repeat(len(states), axis=1)
    k = np.arange(L)
    for si, st in enumerate(states):
        for e, (bond, bits) in enumerate(st):
            xs, xt = X[:, src[e]], X[:, dst[e]]
            if bond:
                with np.errstate(divide="ignore"):
                    out[:, si] += np.where(xs == xt, np.log(alpha[e, xs]), -np.inf)
            else:
                y = (xs[:, None] == k[None, :]).astype(float)
                z = (xt[:, None] == k[None, :]).astype(float)
                b = np.asarray(bits, float)[None, :]
                out[:, si] += (dec.alpha1[e] * y + dec.alpha2[e] * z
                               + b * (dec.q[e] + dec.beta1[e] * y + dec.beta2[e] * z)
                               - np.logaddexp(0.0, dec.q[e])).sum(axis=1)
    return out


def _states(E, L):
    per_edge = [(True, (0,) * L)] + [(False, bits) for bits in itertools.product((0, 1), repeat=L)]
    return list(itertools.product(per_edge, repeat=E))


def _tiny(kind):
    if kind == "potts":
        return _potts_model(6, N=4, L=3, E=3)
    return _model_two_labels(7, N=4, E=4)


def _norm(v):
    return v - np.logaddexp.reduce(v)


def test_split_reproduces_every_factor():
    L = 4
    for l in (0.05, 0.6, 2.0):
        for rho in (0.0, 0.3, 1.0):
            alpha = rho * np.expm1(l)
            lp = np.log1p((1 - rho) * np.expm1(l))
            for a, b in itertools.product(range(L), repeat=2):
                P = 1.0 + np.expm1(l) * (a == b)
                assert abs(alpha * (a == b) + np.exp(lp * (a == b)) - P) < 1e-12


@pytest.mark.parametrize("kind,rho", [("potts", 0.4), ("two", 0.7)])
def test_joint_marginal_and_conditionals_by_enumeration(kind, rho):
    model = _tiny(kind)
    L, E = model.n_labels, model.src.size
    X = brute.all_labelings(model.n_vars, L)
    states = _states(E, L)
    J = _joint_log(model, rho, X, states)
    np.testing.assert_allclose(_norm(np.logaddexp.reduce(J, axis=1)), _norm(brute.log_ptilde(model, X)), atol=1e-10)
    alpha, dec = hg.higdon_split(model, rho)
    # the duals given x, as the oracle's sweep draws them: per edge the bond
    # probability, and A's bit probabilities given no bond (the joint factorises over edges)
    sel = np.arange(0, X.shape[0], max(1, X.shape[0] // 7))
    res = hg.higdon_sweep(model, X[sel], rho, 0, 0)
    for i, xi in enumerate(sel):
        P = np.exp(J[xi] - np.logaddexp.reduce(J[xi]))
        for e in range(E):
            p_bond = sum(P[si] for si, st in enumerate(states) if st[e][0])
            assert abs(p_bond - res["p_bond"][i, e]) < 1e-12
            for k in range(L):
                p1 = sum(P[si] for si, st in enumerate(states) if not st[e][0] and st[e][1][k] == 1)
                assert abs(p1 / (1 - p_bond) - res["p_dual"][i, e, k]) < 1e-12
    # the cluster rule given the duals
    rng = np.random.default_rng(3)
    for si in rng.choice(len(states), size=8, replace=False):
        col = J[:, si]
        if not np.isfinite(col).any():
            continue
        p_exact = np.exp(col - np.logaddexp.reduce(col))
        bonds = np.array([st[0] for st in states[si]])
        theta = np.array([st[1] for st in states[si]], bool)[None]
        F = primal_field(dec, theta)[0]
        root, lw = hg.cluster_log_weights(model, (alpha, dec), bonds, F)
        rs = np.unique(root)
        lp = log_softmax(lw[rs])
        pos = {r: i for i, r in enumerate(rs)}
        p_rule = np.array([np.exp(sum(lp[pos[r], x[r]] for r in rs)) if all(x[v] == x[root[v]] for v in range(model.n_vars))
                           else 0.0 for x in X])
        np.testing.assert_allclose(p_rule, p_exact, atol=1e-12)


def test_kernel_is_stationary():
    model, rho = _tiny("two"), 0.5
    L, E = model.n_labels, model.src.size
    X = brute.all_labelings(model.n_vars, L)
    J = _joint_log(model, rho, X, _states(E, L))
    with np.errstate(invalid="ignore"):
        K = np.nan_to_num(np.exp(J - np.logaddexp.reduce(J, axis=1)[:, None])) @ \
            np.nan_to_num(np.exp(J - np.logaddexp.reduce(J, axis=0)[None, :])).T
    _, p, _ = brute.exact_distribution(model)
    np.testing.assert_allclose(K.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(p @ K, p, atol=1e-12)


def test_rho_one_is_swendsen_wang_and_rho_zero_the_plain_sweep():
    model = _potts_model(8, N=6, L=3, E=8)
    C, t, seed = 16, 4, 9
    x = ph.init_labels(model.n_vars, 3, C, seed)
    h1 = hg.higdon_sweep(model, x, 1.0, t, seed)
    s1 = sw.sw_sweep(model, x, t, seed)
    np.testing.assert_array_equal(h1["bonds"], s1["bonds"])
    assert not h1["theta"].any()                                      # A = 1: no bits
    for c in range(C):                                                # same label distribution per cluster
        rs = np.unique(s1["roots"][c])
        np.testing.assert_allclose(h1["cdf_cluster"][c, rs], s1["cdf_cluster"][c, rs], atol=1e-12)
    h0 = hg.higdon_sweep(model, x, 0.0, t, seed)
    assert not h0["bonds"].any()
    from oracle import decompose as dc, sampler
    dec = dc.decompose(model)                                         # the model's own diagonal decomposition
    ref = sampler.sweep(dec, x, t, seed)
    np.testing.assert_array_equal(h0["theta"], ref["theta"])
    np.testing.assert_allclose(h0["field"], primal_field(dec, ref["theta"]), atol=1e-12)


@pytest.mark.parametrize("kind,rho", [("potts", 0.5), ("two", 0.8)])
def test_chain_marginals_within_3_sigma(kind, rho):
    model = _potts_model(4, N=6, L=3, E=8) if kind == "potts" else _model_two_labels(5, N=7, E=10)
    L = model.n_labels
    exact, _ = brute.exact_marginals(model)
    C, T, burn, seed = 512, 60, 10, 5
    x = ph.init_labels(model.n_vars, L, C, seed)
    split = hg.higdon_split(model, rho)
    acc = np.zeros((C, model.n_vars, L))
    for t in range(T):
        x = hg.higdon_sweep(model, x, rho, t, seed, split=split)["x"]
        if t >= burn:
            acc[np.arange(C)[:, None], np.arange(model.n_vars)[None, :], x] += 1
    cm = acc / (T - burn)
    z = np.abs(cm.mean(0) - exact) / np.maximum(cm.std(0, ddof=1) / np.sqrt(C), 1e-12)
    assert z.max() < 4.5 and np.mean(z < 3.0) > 0.9, z


def test_log_v_mean_is_log_z_minus_mutual_information():
    """Section 5.2 on the three-state duality, by enumerating (x, theta)."""
    model, rho = _tiny("two"), 0.6
    L, E = model.n_labels, model.src.size
    X = brute.all_labelings(model.n_vars, L)
    states = _states(E, L)
    J = _joint_log(model, rho, X, states)
    P = np.exp(J - np.logaddexp.reduce(J.ravel()))
    logZ = np.logaddexp.reduce(brute.log_ptilde(model, X))
    split = hg.higdon_split(model, rho)
    lv = np.zeros(J.shape)
    for si, st in enumerate(states):
        ok = P[:, si] > 0
        if not ok.any():
            continue
        bonds = np.array([b for b, _ in st], bool)
        theta = np.array([bits for _, bits in st], bool)
        n = int(ok.sum())
        lv[ok, si] = hg.log_v(model, X[ok], np.repeat(bonds[None], n, 0), np.repeat(theta[None], n, 0), split)
    m = P > 0
    assert np.all(np.isfinite(lv[m]))
    px, pt = P.sum(axis=1), P.sum(axis=0)
    mi = (P[m] * (np.log(P[m]) - np.log(np.outer(px, pt)[m]))).sum()
    np.testing.assert_allclose(logZ - (P[m] * lv[m]).sum(), mi, atol=1e-10)
    assert mi > 0
