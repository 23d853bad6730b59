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
