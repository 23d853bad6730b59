"""Pins of the oracle's blocked sweep (Section 5.4): the comb forest is a
spanning forest of each block, the tree sampler draws from the exact
p(x | theta_1) (enumeration), and the blocked kernel leaves p invariant."""
import itertools

import numpy as np
import pytest

from oracle import blocked as bl, brute, decompose as dc, sampler, philox as ph
from paper_1611_06684_gb300 import workloads as wl


@pytest.mark.parametrize("grid", [(5, 6, 7), (4, 4, 4), (9, 3, 1)])
@pytest.mark.parametrize("offset", [(0, 0, 0), (1, 2, 3), (3, 3, 1)])
def test_comb_forest_spans_every_block(grid, offset):
    nx, ny, nz = grid
    parent = bl.comb_forest(grid, offset)
    src, dst = wl.grid3d_edges(nx, ny, nz)
    tree = bl.tree_edge_mask(src, dst, parent)
    x = np.arange(nx * ny * nz) % nx; y = (np.arange(nx * ny * nz) // nx) % ny; z = np.arange(nx * ny * nz) // (nx * ny)
    bid = ((x + offset[0]) // 4) + 100 * ((y + offset[1]) // 4) + 10000 * ((z + offset[2]) // 4)
    # every tree edge lies inside one block and every non-root's parent is a lattice neighbour
    assert np.all(bid[src[tree]] == bid[dst[tree]])
    # #roots == #blocks, #tree edges == N - #blocks  (spanning forest of the blocks)
    n_blocks = np.unique(bid).size
    assert int((parent < 0).sum()) == n_blocks
    assert int(tree.sum()) == nx * ny * nz - n_blocks
    # each root is the minimum corner of its block
    for b in np.unique(bid):
        members = np.nonzero(bid == b)[0]
        roots = members[parent[members] < 0]
        assert roots.size == 1 and roots[0] == members.min()


def _enumerate_tree_conditional(model, phi, tree):
    """p(x | theta_1) by enumeration: prod_v exp(phi_v) prod_{e in T} exp(w_e)."""
    X = brute.all_labelings(model.n_vars, model.n_labels)
    w = model.pair.astype(np.float64)
    te = np.nonzero(tree)[0]
    lp = phi[np.arange(model.n_vars)[None, :], X].sum(1)
    lp += w[te[None, :], X[:, model.src[te]], X[:, model.dst[te]]].sum(1)
    return X, lp - np.logaddexp.reduce(lp)


@pytest.mark.parametrize("dims,L", [((3, 2, 2), 2), ((3, 2, 1), 3)])
def test_tree_sampler_matches_enumeration(dims, L):
    model = wl.potts_grid3d(*dims, L=L, seed=4, w_half=0.6)
    dec = dc.decompose(model)
    parent = bl.comb_forest(model.grid, (1, 0, 1))
    tree = bl.tree_edge_mask(dec.src, dec.dst, parent)
    rng = np.random.default_rng(0)
    theta = (rng.random((1,) + dec.ell.shape) < 0.5) & dec.active[None] & ~tree[None, :, None]
    phi = bl.node_potentials(model, dec, tree, theta)
    order, _ = bl.bfs_order(parent)
    X, lp_exact = _enumerate_tree_conditional(model, phi[0], tree)
    lp_tree = bl.tree_conditional_logprob(model, phi, parent, tree, order, X)
    np.testing.assert_allclose(lp_tree, lp_exact, atol=1e-11)


def test_blocked_kernel_is_stationary():
    """p K_blocked = p, with K_blocked(x, x') = sum_theta1 p(theta1|x) p(x'|theta1)."""
    model = wl.potts_grid3d(3, 2, 1, L=2, seed=6, w_half=0.8)
    dec = dc.decompose(model)
    X, p, _ = brute.exact_distribution(model)
    for offset in [(0, 0, 0), (1, 1, 0), (2, 3, 0)]:
        parent = bl.comb_forest(model.grid, offset)
        tree = bl.tree_edge_mask(dec.src, dec.dst, parent)
        order, _ = bl.bfs_order(parent)
        ent = np.argwhere(dec.active & ~tree[:, None])
        Th = brute.all_dual_configs(ent.shape[0])
        pa = sampler.dual_probs(dec, X)[:, ent[:, 0], ent[:, 1]]
        log_pt = (np.log(pa)[:, None, :] * Th[None] + np.log1p(-pa)[:, None, :] * (1 - Th[None])).sum(-1)
        K = np.zeros((X.shape[0], X.shape[0]))
        for ti in range(Th.shape[0]):
            th = np.zeros((1,) + dec.ell.shape); th[0, ent[:, 0], ent[:, 1]] = Th[ti]
            phi = bl.node_potentials(model, dec, tree, th)
            lq = bl.tree_conditional_logprob(model, phi, parent, tree, order, X)
            K += np.exp(log_pt[:, ti])[:, None] * np.exp(lq)[None, :]
        np.testing.assert_allclose(K.sum(1), 1.0, atol=1e-12)
        np.testing.assert_allclose(p @ K, p, atol=1e-12)


def test_ffbs_draws_follow_their_conditionals():
    model = wl.potts_grid3d(4, 4, 4, L=4, seed=8)
    dec = dc.decompose(model)
    x = ph.init_labels(model.n_vars, 4, 3, seed=9)
    out = bl.blocked_sweep(model, dec, x, 2, 9)
    # each draw is the inverse-CDF draw of the conditional it reports
    xr, _ = sampler.inverse_cdf(out["logp"], out["u_site"])
    assert np.array_equal(xr, out["x"])
    assert not out["theta"][:, out["tree"], :].any()
