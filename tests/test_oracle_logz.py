"""Pins of the log-partition estimator (Section 5.2) by exact enumeration."""
import numpy as np
import pytest

from oracle import brute, decompose as dc, logz, sampler
from paper_1611_06684_gb300 import workloads as wl

MODELS = {
    "ising": lambda: wl.ising_grid(2, 3, seed=1),
    "potts": lambda: wl.tiny_potts(4, 3, 4, seed=2, beta_max=1.2),
    "random": lambda: wl.tiny_random(4, 3, 4, seed=3, w_std=0.8),
}


@pytest.mark.parametrize("name", list(MODELS))
def test_expected_v_is_the_partition_function(name):
    model = MODELS[name]()
    dec = dc.decompose(model)
    log_ev, e_logv, mi = logz.exact_moments(model, dec)
    _, _, logZ = brute.exact_distribution(model)
    assert abs(log_ev - logZ) < 1e-10
    # Jensen gap of the log estimator = mutual information of x and theta
    assert mi > 0
    assert abs((logZ - e_logv) - mi) < 1e-10


@pytest.mark.parametrize("name", list(MODELS))
def test_log_v_matches_theorem1_joint(name):
    """log V from the sweep's conditionals equals log p~(x) + log p~(theta) -
    log p~(x, theta) with the joint of Theorem 1, for every (x, theta)."""
    model = MODELS[name]()
    dec = dc.decompose(model)
    X = brute.all_labelings(model.n_vars, model.n_labels)
    ent = brute.active_entries(dec)
    Th = brute.all_dual_configs(ent.shape[0])
    J = brute.joint_log(dec, X, Th)
    lv_ref = brute.log_ptilde(model, X)[:, None] + np.logaddexp.reduce(J, axis=0)[None, :] - J
    rng = np.random.default_rng(0)
    xi = rng.integers(0, X.shape[0], size=40)
    ti = rng.integers(0, Th.shape[0], size=40)
    theta = np.zeros((40,) + dec.ell.shape, bool)
    theta[:, ent[:, 0], ent[:, 1]] = Th[ti].astype(bool)
    got = logz.log_v(model, dec, X[xi], theta)
    np.testing.assert_allclose(got, lv_ref[xi, ti], rtol=0, atol=1e-10)


def test_chain_estimates_bracket_log_z():
    """Sweeps of the oracle chain: log-mean-exp of V within 4 sigma of log Z,
    the mean of log V below it (up to sampling error)."""
    model = wl.tiny_potts(5, 3, 6, seed=4, beta_max=0.8)
    dec = dc.decompose(model)
    _, _, logZ = brute.exact_distribution(model)
    C, seed = 256, 9
    x = np.random.default_rng(1).integers(0, 3, size=(C, model.n_vars))
    for t in range(20):                                               # burn-in
        x = sampler.sweep(dec, x, t, seed)["x"]
    lv = []
    for t in range(20, 60):
        v, r = logz.sweep_log_v(model, dec, x, t, seed)
        lv.append(v)
        x = r["x"]
    lv = np.concatenate(lv)
    w = np.exp(lv - lv.max())
    est = lv.max() + np.log(w.mean())
    se = w.std() / w.mean() / np.sqrt(len(w) / 10)                    # blocks of correlated sweeps
    assert abs(est - logZ) < 4 * se + 1e-3
    assert lv.mean() < logZ + 4 * lv.std() / np.sqrt(len(lv) / 10)


@pytest.mark.parametrize("name", list(MODELS))
def test_mutual_information_is_expected_kl(name):
    """Lemma 5: I(x; theta) = E_theta KL(p(x | theta), p(x)) >= min over theta of
    the same KL (by enumeration; p(x | theta) is of the form p(x | xi))."""
    model = MODELS[name]()
    dec = dc.decompose(model)
    _, _, mi = logz.exact_moments(model, dec)
    X = brute.all_labelings(model.n_vars, model.n_labels)
    Th = brute.all_dual_configs(brute.active_entries(dec).shape[0])
    J = brute.joint_log(dec, X, Th)
    lpj = J - np.logaddexp.reduce(J, axis=None)
    lpt = np.logaddexp.reduce(lpj, axis=0)                          # log p(theta)
    lpx = np.logaddexp.reduce(lpj, axis=1)                          # log p(x)
    lp_x_t = lpj - lpt[None, :]                                     # log p(x | theta)
    kl = (np.exp(lp_x_t) * (lp_x_t - lpx[:, None])).sum(axis=0)     # KL(p(x|theta), p(x)) per theta
    assert abs((np.exp(lpt) * kl).sum() - mi) < 1e-10
    assert mi >= kl.min() - 1e-12
