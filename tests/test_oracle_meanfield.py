"""Pins of the primal-dual EM and mean-field updates (Section 5.3)."""
import numpy as np
import pytest

from oracle import brute, decompose as dc, meanfield as mf
from paper_1611_06684_gb300 import workloads as wl


@pytest.mark.parametrize("model", [wl.potts_grid3d(6, 5, 4, L=4, seed=1), wl.random_graph(60, k=3, L=3, seed=2),
                                   wl.ising_grid(8, 8, seed=3)])
def test_em_never_decreases_log_ptilde(model):
    dec = dc.decompose(model)
    x = np.random.default_rng(0).integers(0, model.n_labels, size=(6, model.n_vars))
    prev = brute.log_ptilde(model, x)
    for _ in range(12):
        x, _, _ = mf.em_step(dec, x)
        cur = brute.log_ptilde(model, x)
        assert (cur >= prev - 1e-9).all()
        prev = cur


@pytest.mark.parametrize("model", [wl.tiny_potts(4, 3, 4, seed=2, beta_max=1.2), wl.tiny_random(4, 3, 4, seed=3, w_std=0.8)])
def test_mean_field_objective_decreases_and_bounds_primal_kl(model):
    dec = dc.decompose(model)
    rng = np.random.default_rng(1)
    q = rng.dirichlet(np.ones(model.n_labels), size=(1, model.n_vars))
    prev = None
    for _ in range(10):
        # theta-update alone (from q), then check the objective and Lemma 6 at (q, pi*)
        eta_y = q[:, dec.src][:, :, dec.i_pos]; eta_z = q[:, dec.dst][:, :, dec.j_pos]
        pi = mf.dual_mean(dec, eta_y, eta_z)
        kl_joint, kl_x = mf.mf_objective(model, dec, q[0], pi[0])
        assert kl_joint >= kl_x - 1e-10                        # Lemma 6
        if prev is not None:
            assert kl_joint <= prev + 1e-10                    # coordinate descent on the objective
        q, _, _ = mf.mf_step(dec, q)
        kl_after, _ = mf.mf_objective(model, dec, q[0], pi[0])
        assert kl_after <= kl_joint + 1e-10                    # the x-update does not increase it either
        prev = kl_after


def test_mf_step_uses_expected_indicators():
    """A mean-field step from one-hot marginals equals the EM step's field."""
    model = wl.random_graph(30, k=2, L=4, seed=5)
    dec = dc.decompose(model)
    x = np.random.default_rng(2).integers(0, 4, size=(3, model.n_vars))
    q = np.eye(4)[x]
    _, pi_m, F_m = mf.mf_step(dec, q)
    _, pi_e, F_e = mf.em_step(dec, x)
    np.testing.assert_allclose(pi_m, pi_e, rtol=0, atol=1e-15)
    np.testing.assert_allclose(F_m, F_e, rtol=0, atol=1e-12)


def test_tree_map_is_the_enumerated_argmax():
    """One 4x4x4-block lattice small enough to enumerate: the tree MAP equals
    the argmax of phi + exact tree factors over all labelings."""
    model = wl.potts_grid3d(3, 2, 2, L=3, seed=6)
    dec = dc.decompose(model)
    from oracle import blocked
    parent = blocked.comb_forest(model.grid, (0, 0, 0))
    tree = blocked.tree_edge_mask(dec.src, dec.dst, parent)
    rng = np.random.default_rng(3)
    phi = rng.normal(0, 1, size=(4, model.n_vars, 3))
    order, _ = blocked.bfs_order(parent)
    x = mf.tree_map(model, phi, parent, tree, order)
    X = brute.all_labelings(model.n_vars, 3)
    w = np.asarray(model.pair, np.float64)
    te = np.nonzero(tree)[0]
    for c in range(4):
        score = phi[c][np.arange(model.n_vars)[None, :], X].sum(axis=1)
        score += w[te[None, :], X[:, model.src[te]], X[:, model.dst[te]]].sum(axis=1)
        assert np.array_equal(x[c], X[np.argmax(score)])


def test_blocked_em_never_decreases_log_ptilde():
    model = wl.potts_grid3d(9, 7, 6, L=4, seed=7)
    dec = dc.decompose(model)
    x = np.random.default_rng(4).integers(0, 4, size=(3, model.n_vars))
    prev = brute.log_ptilde(model, x)
    for it in range(8):
        x = mf.blocked_em_step(model, dec, x, it, 11)
        cur = brute.log_ptilde(model, x)
        assert (cur >= prev - 1e-9).all()
        prev = cur


def _tree_setup(model, offset=(0, 0, 0)):
    from oracle import blocked
    dec = dc.decompose(model)
    parent = blocked.comb_forest(model.grid, offset)
    tree = blocked.tree_edge_mask(dec.src, dec.dst, parent)
    order, _ = blocked.bfs_order(parent)
    return dec, parent, tree, order


def _enumerated_tree_marginals(model, tree, phi_c):
    X = brute.all_labelings(model.n_vars, model.n_labels)
    w = np.asarray(model.pair, np.float64)
    te = np.nonzero(tree)[0]
    score = phi_c[np.arange(model.n_vars)[None, :], X].sum(axis=1)
    score += w[te[None, :], X[:, model.src[te]], X[:, model.dst[te]]].sum(axis=1)
    p = np.exp(score - np.logaddexp.reduce(score))
    marg = np.zeros((model.n_vars, model.n_labels))
    for v in range(model.n_vars):
        np.add.at(marg[v], X[:, v], p)
    return marg


@pytest.mark.parametrize("offset", [(0, 0, 0), (1, 2, 3)])
def test_tree_marginals_are_the_enumerated_tree_marginals(offset):
    """Sum-product marginals of the tree MRF (node potentials phi, exact
    forest factors) equal the marginals of the enumerated distribution; with
    offset (1, 2, 3) the clipped blocks give a forest of several trees."""
    model = wl.potts_grid3d(3, 2, 2, L=3, seed=6, w_half=1.0)
    dec, parent, tree, order = _tree_setup(model, offset)
    rng = np.random.default_rng(3)
    phi = rng.normal(0, 1, size=(2, model.n_vars, 3))
    q = mf.tree_marginals(model, phi, parent, tree, order)
    for c in range(2):
        np.testing.assert_allclose(q[c], _enumerated_tree_marginals(model, tree, phi[c]), rtol=0, atol=1e-12)


def test_tree_marginals_planted_mistake_fails():
    """A downward pass that does not remove the child's own upward message
    from its parent's belief (a plausible slip) misses the enumeration."""
    from oracle import blocked
    model = wl.potts_grid3d(3, 2, 2, L=3, seed=6, w_half=1.0)
    dec, parent, tree, order = _tree_setup(model)
    phi = np.random.default_rng(3).normal(0, 1, size=(1, model.n_vars, 3))
    inbox, psi = blocked.tree_messages(model, phi, parent, tree, order)
    down = np.zeros_like(phi)
    for v in order:
        p = parent[v]
        if p < 0:
            continue
        bp = phi[:, p, :] + inbox[:, p, :] + down[:, p, :]              # the child's message not removed
        down[:, v, :] = np.logaddexp.reduce(bp[:, :, None] + psi[v][None], axis=1)
    wrong = np.exp(phi + inbox + down - np.logaddexp.reduce(phi + inbox + down, axis=2)[..., None])
    assert np.abs(wrong[0] - _enumerated_tree_marginals(model, tree, phi[0])).max() > 1e-3


@pytest.mark.parametrize("model", [wl.potts_grid3d(2, 2, 2, L=2, seed=8, w_half=1.5),
                                   wl.potts_grid3d(3, 2, 1, L=3, seed=9, w_half=1.2)])
def test_blocked_mean_field_objective_decreases_and_bounds_primal_kl(model):
    """Tree mean field with a fixed forest: the theta-update (expected
    non-forest duals from the tree marginals) and the x-update (the tree MRF of
    their potentials) each never increase KL(q_x q_theta1 || p(x, theta_1)),
    which stays above KL(q_x || p(x)) (Lemma 6 with the forest's duals summed out)."""
    from oracle import blocked
    dec, parent, tree, order = _tree_setup(model)
    assert tree.any() and (~tree).any()
    rng = np.random.default_rng(4)
    phi = rng.normal(0, 1, size=(1, model.n_vars, model.n_labels))
    prev = None
    for _ in range(8):
        q = mf.tree_marginals(model, phi, parent, tree, order)
        eta_y = q[:, dec.src][:, :, dec.i_pos]; eta_z = q[:, dec.dst][:, :, dec.j_pos]
        pi = np.where(~tree[None, :, None], mf.dual_mean(dec, eta_y, eta_z), 0.0)
        kl_joint, kl_x = mf.blocked_mf_objective(model, dec, tree, phi[0], pi[0])
        assert kl_joint >= kl_x - 1e-10
        if prev is not None:
            assert kl_joint <= prev + 1e-10
        phi = blocked.node_potentials(model, dec, tree, pi)
        kl_after, _ = mf.blocked_mf_objective(model, dec, tree, phi[0], pi[0])
        assert kl_after <= kl_joint + 1e-10
        prev = kl_after


def test_blocked_mf_step_composes_the_two_updates():
    """blocked_mf_step from marginals q equals the tree marginals of the node
    potentials of the expected non-forest duals of q, with the forest of the
    iteration's block offset."""
    from oracle import blocked, philox as ph
    model = wl.potts_grid3d(7, 6, 5, L=4, seed=10)
    dec = dc.decompose(model)
    q = np.random.default_rng(5).dirichlet(np.ones(4), size=(2, model.n_vars))
    q1, pi, phi = mf.blocked_mf_step(model, dec, q, 3, 17)
    parent = blocked.comb_forest(model.grid, ph.splash_offset(3, 17))
    tree = blocked.tree_edge_mask(dec.src, dec.dst, parent)
    assert (pi[:, tree] == 0).all()
    np.testing.assert_allclose(q1.sum(axis=2), 1.0, atol=1e-12)
    order, _ = blocked.bfs_order(parent)
    np.testing.assert_allclose(q1, mf.tree_marginals(model, phi, parent, tree, order), rtol=0, atol=0)
