"""Pins of the oracle's factor decomposition (Sections 4.1-4.2) against what
the paper and the mathematics fix, independent of the oracle's own code paths."""
import numpy as np
import pytest

from oracle import decompose as dc
from paper_1611_06684_gb300 import workloads as wl

ELLS = np.array([-3.0, -2.0, -1.0, -0.5, -0.1, -1e-3, 1e-3, 0.1, 0.5, 1.0, 2.0, 3.0, 4.0, 7.5, -9.0])


def _mix(params, y, z):
    a1, a2, q, b1, b2 = params
    # Theorem 2: sum_theta h(x) g(theta) exp(<x, r(theta)>)
    return np.exp(a1 * y + a2 * z) * (1.0 + np.exp(q + b1 * y + b2 * z))


def test_entry_factor_reconstructs_exp_l_yz():
    """Q(y,z) = exp(l*y*z) up to one constant, for every (y, z)."""
    params, _ = dc.entry_params_literal(ELLS)
    base = _mix(params, 0.0, 0.0)
    for y in (0.0, 1.0):
        for z in (0.0, 1.0):
            got = _mix(params, y, z) / base
            np.testing.assert_allclose(got, np.exp(ELLS * y * z), rtol=1e-12)


def test_literal_pipeline_matches_closed_form():
    lit, _ = dc.entry_params_literal(ELLS)
    cf = dc.closed_form(ELLS)
    for a, b in zip(lit, cf):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_factors_strictly_positive_and_multiply_back():
    """Lemmas 2-4: B, C > 0 entrywise and B C^T = P for random positive P."""
    rng = np.random.default_rng(1)
    P = np.exp(rng.normal(0, 1.5, size=(500, 2, 2)))
    B, C = dc.factor_2x2(P)
    assert np.all(B > 0) and np.all(C > 0)
    np.testing.assert_allclose(B @ np.swapaxes(C, -1, -2), P, rtol=1e-12)
    # Theorem 2 on a general positive P: the mixture is proportional to P
    a1, a2, q, b1, b2 = dc.theorem2_params(B, C)
    for y in (0, 1):
        for z in (0, 1):
            mix = np.exp(a1 * y + a2 * z) * (1 + np.exp(q + b1 * y + b2 * z))
            np.testing.assert_allclose(mix / (np.exp(0) * (1 + np.exp(q))),
                                       P[:, y, z] / P[:, 0, 0], rtol=1e-11)


def test_lemma2_symmetric_factor():
    rng = np.random.default_rng(2)
    d = np.exp(rng.normal(size=(200, 2)))
    c = rng.uniform(0.01, 0.99, 200) * np.sqrt(d[:, 0] * d[:, 1])
    S = np.stack([np.stack([d[:, 0], c], -1), np.stack([c, d[:, 1]], -1)], 1)
    B = dc.lemma2_factor(S)
    assert np.all(B > 0)
    np.testing.assert_allclose(B @ np.swapaxes(B, -1, -2), S, rtol=1e-12)


def test_lemma3_and_lemma4():
    rng = np.random.default_rng(3)
    P = np.exp(rng.normal(size=(100, 2, 2)))
    D = np.zeros_like(P); D[:, 0, 0] = 1 / P[:, 0, 1]; D[:, 1, 1] = 1 / P[:, 1, 0]
    S = D @ P
    np.testing.assert_allclose(S[:, 0, 1], S[:, 1, 0], rtol=1e-14)
    det = np.linalg.det(P)
    J = np.array([[0.0, 1.0], [1.0, 0.0]])
    assert np.all(np.linalg.det(J @ P[det < 0]) > 0)


def _edge_log_table(dec, E_idx, fold_s, fold_t, const):
    """Rebuild w_e(a,b) from the decomposition by enumerating theta of the edge."""
    L = dec.n_labels
    out = np.zeros((L, L))
    act = np.nonzero(dec.active[E_idx])[0]
    thetas = np.array(np.meshgrid(*[[0, 1]] * len(act), indexing="ij")).reshape(len(act), -1).T if len(act) else np.zeros((1, 0))
    for a in range(L):
        for b in range(L):
            y = (dec.i_pos[act] == a).astype(float); z = (dec.j_pos[act] == b).astype(float)
            logits = dec.q[E_idx, act] + dec.beta1[E_idx, act] * y + dec.beta2[E_idx, act] * z
            tot = np.logaddexp.reduce(thetas @ logits) if len(act) else 0.0
            out[a, b] = fold_s[a] + fold_t[b] + tot
    return out + const


@pytest.mark.parametrize("L,diag", [(2, False), (3, False), (4, False), (3, True), (4, True)])
def test_full_edge_table_enumeration(L, diag):
    """log sum_theta of the edge's mixture = w_e(a,b) for every (a,b), 1e-12."""
    m = wl.tiny_potts(4, L, 5, seed=L) if diag else wl.tiny_random(4, L, 5, seed=L)
    dec = dc.decompose(m)
    assert dec.layout == (dc.LAYOUT_DIAG if diag else dc.LAYOUT_PIVOT)
    fold_s, fold_t = dc.fold_vectors(m, dec)
    _, _, _, const = dc.normalise(m.pair, dec.layout)
    for e in range(m.n_edges):
        consts = -np.logaddexp(0.0, dec.q[e, dec.active[e]]).sum() + const[e]
        got = _edge_log_table(dec, e, fold_s[e], fold_t[e], consts)
        np.testing.assert_allclose(got, m.pair[e].astype(np.float64), rtol=0, atol=1e-12)


def test_full_edge_table_product_identity_L8():
    """L=8: prod_k c_k^{[a=i_k][b=j_k]} times offsets = exp(w(a,b)) for random tables."""
    m = wl.potts_grid3d(3, 2, 2, L=8, seed=5)
    dec = dc.decompose(m)
    ell, off_s, off_t, const = dc.normalise(m.pair, dec.layout)
    L = 8
    for e in range(m.n_edges):
        rec = np.zeros((L, L))
        for k in range(dec.n_entries):
            rec[dec.i_pos[k], dec.j_pos[k]] += ell[e, k]
        rec += off_s[e][:, None] + off_t[e][None, :] + const[e]
        np.testing.assert_allclose(rec, m.pair[e], atol=1e-12)


def test_binary_ising_single_dual_bit():
    """Theorem 2 special case: an Ising edge J s_s s_t has one dual bit with l = 4J."""
    m = wl.ising_grid(3, 3, seed=7)
    dec = dc.decompose(m)
    assert dec.layout == dc.LAYOUT_PIVOT and dec.n_entries == 1
    J = m.pair[:, 1, 1].astype(np.float64)
    np.testing.assert_allclose(dec.ell[:, 0], 4 * J, rtol=1e-7)


def test_potts_needs_L_dual_bits():
    """Section 4.2: a Potts factor of order n needs only n auxiliary variables."""
    m = wl.tiny_potts(6, 5, 8, seed=9)
    dec = dc.decompose(m)
    assert dec.layout == dc.LAYOUT_DIAG and dec.n_entries == 5


def test_zero_entries_get_no_dual_variable():
    m = wl.tiny_random(4, 3, 4, seed=11)
    m.pair[0] = 0.0
    # dyadic table whose pivot entry (1, 2) is exactly 0.75 - 0.5 - 0.25 + 0 = 0
    m.pair[1] = np.array([[0.0, 0.5, 0.25], [0.5, 1.0, 0.75], [0.125, 0.375, 1.5]], np.float32)
    dec = dc.decompose(m)
    assert not dec.active[0].any()
    k = (1 - 1) * 2 + (2 - 1)
    assert dec.ell[1, k] == 0 and not dec.active[1, k]
