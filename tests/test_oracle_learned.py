"""Pins of the oracle's learned MH block step: MLP gradients against central
finite differences, and exact stationarity of the learned sweep (cut duals,
then one MH step per block with the MLP proposal) on enumerable models, for
arbitrary network weights."""
import itertools

import numpy as np
import pytest

from oracle import brute, decompose as dc, learned as ln, sampler
from oracle.blocked import node_potentials
from paper_1611_06684_gb300 import workloads as wl


def _rand_params(L, hidden, seed, scale=0.5):
    rng = np.random.default_rng(seed)
    d, dp = ln.feature_width(L)
    shapes = [(hidden, dp), (hidden,), (hidden, hidden), (hidden,), (ln.BLOCK * L, hidden), (ln.BLOCK * L,)]
    return [rng.normal(0, scale, s) for s in shapes]


def test_mlp_gradients_match_finite_differences():
    L, hidden, R = 3, 6, 5
    params = _rand_params(L, hidden, 1)
    rng = np.random.default_rng(2)
    d, dp = ln.feature_width(L)
    X = rng.normal(size=(R, dp))
    y = rng.integers(0, L, size=(R, ln.BLOCK))
    nmem = np.array([16, 3, 9, 1, 16])
    loss, grads = ln.loss_and_grads(params, X, y, nmem, L)
    h = 1e-6
    for pi, P in enumerate(params):
        flat = P.reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h; lp, _, _ = ln.ce_loss(ln.mlp_forward(params, X)[0], y, nmem, L)
            flat[idx] = old - h; lm, _, _ = ln.ce_loss(ln.mlp_forward(params, X)[0], y, nmem, L)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            g = grads[pi].reshape(-1)[idx]
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(fd)), (pi, idx, fd, g)


def test_pair_index_is_a_bijection():
    idx = [ln.pair_index(i, j) for i in range(16) for j in range(i + 1, 16)]
    assert sorted(idx) == list(range(120))


def test_bf16_rounding():
    v = np.array([1.0, 1.00390625, 1.005859375, -3.1415926, 65504.0, 1e-30])
    r = ln.to_bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0            # tie rounds to even
    assert r[2] == 1.0078125
    assert abs(r[3] + 3.140625) < 1e-12


def _learned_kernel(model, dec, block_of_site, params, drop_q_ratio=False):
    """Exact K(x, x') of one learned sweep over all labelings.  drop_q_ratio:
    plant the mistake of accepting with pi(x') / pi(x) alone."""
    L, N = model.n_labels, model.n_vars
    X_all = brute.all_labelings(N, L)
    members = ln.block_members(block_of_site)
    intra = ln.intra_mask(dec.src, dec.dst, block_of_site)
    cut_ent = np.argwhere(dec.active & ~intra[:, None])
    Th = brute.all_dual_configs(cut_ent.shape[0])
    cf = ln.coupling_features(model, block_of_site, members)
    lists = ln.intra_edge_lists(model, block_of_site, len(members))
    w = np.asarray(model.pair, np.float64)
    S = X_all.shape[0]
    index = {tuple(x): i for i, x in enumerate(X_all)}
    K = np.zeros((S, S))
    p1 = sampler.dual_probs(dec, X_all)[:, cut_ent[:, 0], cut_ent[:, 1]]           # [S][M]
    for ti in range(Th.shape[0]):
        th = np.zeros((1,) + dec.ell.shape); th[0, cut_ent[:, 0], cut_ent[:, 1]] = Th[ti]
        pth = np.prod(np.where(Th[ti][None, :] == 1, p1, 1 - p1), axis=1)          # p(theta_cut | x) [S]
        phi_f = sampler.primal_field(dec, th)
        phi = node_potentials(model, dec, intra, th)
        Xf = ln.features(phi_f, members, cf, L)
        z, _ = ln.mlp_forward(params, Xf)
        lz = sampler.log_softmax(z.reshape(len(members), ln.BLOCK, L))
        # per block MH kernel over its own labels; blocks are independent given theta_cut
        for xi in range(S):
            x = X_all[xi]
            trans = [(x.copy(), 1.0)]
            for b, m in enumerate(members):
                lq = lz[b][:len(m)]
                new = []
                for (xx, pr) in trans:
                    lp_cur = ln.block_log_target(phi, w, members, lists, xx[None], b)[0]
                    lq_cur = lq[np.arange(len(m)), xx[m]].sum()
                    stay = 1.0
                    for lab in itertools.product(range(L), repeat=len(m)):
                        lab = np.array(lab)
                        if np.array_equal(lab, xx[m]):
                            continue
                        xp = xx.copy(); xp[m] = lab
                        lq_new = lq[np.arange(len(m)), lab].sum()
                        lp_new = ln.block_log_target(phi, w, members, lists, xp[None], b)[0]
                        q_term = 0.0 if drop_q_ratio else lq_cur - lq_new
                        a = min(1.0, np.exp(lp_new - lp_cur + q_term))
                        pm = np.exp(lq_new) * a
                        stay -= pm
                        new.append((xp, pr * pm))
                    new.append((xx, pr * stay))
                trans = new
            for (xx, pr) in trans:
                K[xi, index[tuple(xx)]] += pth[xi] * pr
    return X_all, K


@pytest.mark.parametrize("case", ["potts", "random"])
def test_learned_sweep_kernel_is_stationary(case):
    if case == "potts":
        model = wl.tiny_potts(4, 3, 3, seed=2, beta_max=1.2)
        block_of_site = np.array([0, 0, 1, 1])
    else:
        model = wl.tiny_random(5, 2, 6, seed=3, w_std=0.9)
        block_of_site = np.array([0, 0, 1, 1, 1])
    dec = dc.decompose(model)
    params = _rand_params(model.n_labels, 5, seed=9)
    X_all, K = _learned_kernel(model, dec, block_of_site, params)
    _, p, _ = brute.exact_distribution(model)
    np.testing.assert_allclose(K.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(p @ K, p, atol=1e-12)


def test_learned_sweep_draws_follow_definition():
    model = wl.tiny_potts(40, 4, 80, seed=5)
    dec = dc.decompose(model)
    bos = wl.bfs_blocks(model, 16, seed=1)
    params = ln.init_params(4, hidden=16, seed=3)
    x = np.random.default_rng(0).integers(0, 4, size=(3, 40))
    out = ln.learned_sweep(model, dec, x, 4, 11, bos, params)
    # rejected blocks keep their labels; accepted blocks take the proposal
    for b, m in enumerate(out["members"]):
        for c in range(3):
            if not out["accepted"][b, c]:
                assert np.array_equal(out["x"][c, m], x[c, m])
    assert not out["theta"][:, ln.intra_mask(dec.src, dec.dst, bos), :].any()


def test_planted_acceptance_without_proposal_ratio_breaks_stationarity():
    model = wl.tiny_potts(4, 3, 3, seed=2, beta_max=1.2)
    block_of_site = np.array([0, 0, 1, 1])
    dec = dc.decompose(model)
    params = _rand_params(model.n_labels, 5, seed=9)
    _, K = _learned_kernel(model, dec, block_of_site, params, drop_q_ratio=True)
    _, p, _ = brute.exact_distribution(model)
    np.testing.assert_allclose(K.sum(axis=1), 1.0, atol=1e-12)
    assert np.abs(p @ K - p).max() > 1e-4


def test_sub_model_of_whole_blocks_reproduces_the_full_sweep():
    """The learned sweep of a few whole blocks on their sub-model (incident
    edges and far-end sites, full-model indices for the draws) equals the full
    model's sweep on those blocks: cut duals, logits and new labels."""
    from tests.learned_helpers import learned_sub_model
    model = wl.ba_potts(500, m=4, L=3, seed=9)
    dec = dc.decompose(model)
    bos = wl.bfs_blocks(model, 16, seed=2)
    C, seed, t = 3, 7, 5
    params = ln.init_params(3, hidden=64, seed=4)
    x0 = np.random.default_rng(1).integers(0, 3, size=(C, model.n_vars))
    full = ln.learned_sweep(model, dec, x0, t, seed, bos, params)
    blocks = np.array([0, 3, int(bos.max()), int(bos[np.argmax(np.bincount(np.concatenate([model.src, model.dst])))])])
    blocks = np.unique(blocks)
    sub, local, eids, sbos, bids, k = learned_sub_model(model, bos, blocks)
    ref = ln.learned_sweep(sub, dc.decompose(sub), x0[:, local], t, seed, sbos, params, edge_ids=eids,
                           site_ids=local, block_ids=bids, blocks=range(k))
    assert np.array_equal(ref["theta"], full["theta"][:, eids])
    for i, b in enumerate(blocks):
        rows_s, rows_f = i * C + np.arange(C), b * C + np.arange(C)
        assert np.allclose(ref["z"][rows_s], full["z"][rows_f], rtol=1e-12, atol=1e-12)
        m_full = full["members"][b]
        assert np.array_equal(local[ref["members"][i]], m_full)
        assert np.array_equal(ref["x"][:, ref["members"][i]], full["x"][:, m_full])
        assert np.array_equal(ref["accepted"][i], full["accepted"][b])
