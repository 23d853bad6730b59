"""Primal-dual EM (local MAP) and mean field of Section 5.3 (oracle side, float64).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
legs use this package.

With Theorem 1's joint p~(x, theta) = h(x) g(theta) exp(<s(x), r(theta)>),
s(x) = ([x_s = i_k], [x_t = j_k])_k, r(theta) = (beta1_k theta_k,
beta2_k theta_k)_k, log g(theta) = sum_k q_k theta_k and log h(x) = sum_v
u~_v(x_v), both conditionals factorise, so Section 5.3's updates are
parallel over entries and over sites:
  theta-update   pi_k = E[theta_k | eta] = sigmoid(q_k + beta1_k eta_y,k + beta2_k eta_z,k)
                 with eta = E[s(x)]: for EM the indicators of the current
                 labels, for mean field the current site marginals
                 (eta_y,k = q_s(i_k), eta_z,k = q_t(j_k));
  x-update       F_v(a) = u~_v(a) + sum of beta pi over the entries of v's
                 incident edges in row / column a (the primal field with theta
                 replaced by pi); EM: x_v = argmax_a F_v(a) (first maximum);
                 mean field: q_v = softmax(F_v).
One iteration is a theta-update followed by an x-update.

Blocked EM (Sections 5.3 and 5.4): the duals of a spanning forest T are not
introduced (their factors stay exact); the theta-update runs on the other
edges and the x-update is the exact MAP of the tree MRF with node potentials
phi (oracle.blocked.node_potentials of pi) and the exact edge factors on T,
by max-product from the leaves and argmax from the roots.  On lattices the
forest is the comb forest of the blocked sweep, its block-grid offset drawn
from the SPLASH phase with index = iteration number.

Blocked (tree) mean field (Sections 5.3 and 5.4, Figure 1 caption): the
same alternation with sum-product in place of max-product.  The x-update
sets q_x to the tree MRF p(x | xi) itself (node potentials phi of pi on the
non-forest edges, exact factors on the forest); the theta-update needs only
its site marginals eta, which sum-product gives exactly: upward messages from
the leaves (oracle.blocked.tree_messages), then downward messages from the
roots,
  m_{p->v}(a) = log sum_b exp(psi_v(b, a) + phi_p(b) + in_p(b) + m_{pp->p}(b) - m_{v->p}(b)),
and eta_v = softmax(phi_v + in_v + m_{p->v}).

Pins (tests/test_oracle_meanfield.py): EM and blocked EM never decrease
log p~(x) (EM on the latent theta); the tree MAP equals the enumerated argmax
of the tree MRF; the mean-field objective KL(q_x q_theta || p(x, theta)),
computed by enumeration, never increases; Lemma 6's inequality
KL(q_x q_theta* || p(x, theta)) >= KL(q_x || p(x)) at every iterate; tree
sum-product marginals equal the enumerated marginals of the tree MRF; the
blocked objective KL(q_x q_theta1 || p(x, theta_1)) (forest duals summed
out), by enumeration, never increases under either half-step of the tree
mean field and bounds KL(q_x || p(x)) from above.
"""
from __future__ import annotations

import numpy as np

from . import blocked, brute, philox as ph
from .decompose import Decomposition
from .sampler import dual_probs, primal_field, log_softmax, sigmoid


def dual_mean(dec: Decomposition, eta_y, eta_z):
    """pi [C][E][m] = sigmoid(q + beta1 eta_y + beta2 eta_z) on active entries (0 elsewhere)."""
    pi = sigmoid(dec.q[None] + dec.beta1[None] * eta_y + dec.beta2[None] * eta_z)
    return np.where(dec.active[None], pi, 0.0)


def em_step(dec: Decomposition, x):
    """One EM iteration from labels x [C][N]; returns new labels and pi."""
    x = np.asarray(x, np.int64)
    eta_y = (x[:, dec.src][:, :, None] == dec.i_pos[None, None, :]).astype(np.float64)
    eta_z = (x[:, dec.dst][:, :, None] == dec.j_pos[None, None, :]).astype(np.float64)
    pi = dual_mean(dec, eta_y, eta_z)
    F = primal_field(dec, pi)
    return np.argmax(F, axis=2), pi, F


def mf_step(dec: Decomposition, q):
    """One mean-field iteration from site marginals q [C][N][L]; returns new marginals and pi."""
    q = np.asarray(q, np.float64)
    C = q.shape[0]
    eta_y = q[:, dec.src][:, :, dec.i_pos] if dec.src.size else np.zeros((C, 0, dec.ell.shape[1]))
    eta_z = q[:, dec.dst][:, :, dec.j_pos] if dec.dst.size else np.zeros((C, 0, dec.ell.shape[1]))
    pi = dual_mean(dec, eta_y, eta_z)
    F = primal_field(dec, pi)
    return np.exp(log_softmax(F)), pi, F


def mf_objective(model, dec: Decomposition, q, pi):
    """KL(q_x q_theta || p(x, theta)) for one chain (q [N][L], pi [E][m]) and
    KL(q_x || p(x)), both by enumeration (tiny models)."""
    X = brute.all_labelings(model.n_vars, model.n_labels)
    ent = brute.active_entries(dec)
    Th = brute.all_dual_configs(ent.shape[0])
    J = brute.joint_log(dec, X, Th)
    lpj = J - np.logaddexp.reduce(J, axis=None)
    lqx = np.log(np.maximum(q[np.arange(model.n_vars)[None, :], X], 1e-300)).sum(axis=1)
    p1 = pi[ent[:, 0], ent[:, 1]]
    lqt = (Th * np.log(np.maximum(p1, 1e-300)) + (1 - Th) * np.log(np.maximum(1 - p1, 1e-300))).sum(axis=1)
    w = np.exp(lqx[:, None] + lqt[None, :])
    kl_joint = float((w * (lqx[:, None] + lqt[None, :] - lpj)).sum())
    lpx = np.logaddexp.reduce(lpj, axis=1)
    wx = np.exp(lqx)
    kl_x = float((wx * (lqx - lpx)).sum())
    return kl_joint, kl_x


def tree_map(model, phi, parent, tree, order):
    """MAP labels [C][N] of the tree MRF (node potentials phi [C][N][L], exact
    edge factors on the forest), by max-product messages and argmax (first
    maximum) from the roots down."""
    C, N, L = phi.shape
    pe, child_is_src = blocked._edge_to_parent(model.src, model.dst, parent, tree)
    w = np.asarray(model.pair, np.float64)
    inbox = np.zeros((C, N, L))
    psi = np.zeros((N, L, L))
    for v in order[::-1]:
        p = parent[v]
        if p < 0:
            continue
        psi[v] = w[pe[v]].T if child_is_src[v] else w[pe[v]]      # [parent label][child label]
        lv = phi[:, v, :] + inbox[:, v, :]
        inbox[:, p, :] += np.max(lv[:, None, :] + psi[v][None], axis=-1)
    x = np.zeros((C, N), np.int64)
    for v in order:
        lv = phi[:, v, :] + inbox[:, v, :]
        p = parent[v]
        if p >= 0:
            lv = lv + psi[v][x[:, p]]
        x[:, v] = np.argmax(lv, axis=1)
    return x


def blocked_em_step(model, dec: Decomposition, x, iteration: int, seed: int, parent=None):
    """One blocked EM iteration from labels x [C][N]; returns the new labels."""
    if parent is None:
        parent = blocked.comb_forest(model.grid, ph.splash_offset(iteration, seed))
    tree = blocked.tree_edge_mask(dec.src, dec.dst, parent)
    pi = np.where(dec.active[None] & ~tree[None, :, None], dual_probs(dec, x), 0.0)
    phi = blocked.node_potentials(model, dec, tree, pi)
    order, _ = blocked.bfs_order(parent)
    return tree_map(model, phi, parent, tree, order)


def tree_marginals(model, phi, parent, tree, order):
    """Site marginals [C][N][L] of the tree MRF with node potentials phi
    [C][N][L] and the exact edge factors on the forest, by sum-product: the
    upward messages of oracle.blocked.tree_messages, then downward messages
    from every root to its children (parents before children in `order`)."""
    C, N, L = phi.shape
    inbox, psi = blocked.tree_messages(model, phi, parent, tree, order)
    down = np.zeros((C, N, L))
    for v in order:
        p = parent[v]
        if p < 0:
            continue
        up = np.logaddexp.reduce((phi[:, v, :] + inbox[:, v, :])[:, None, :] + psi[v][None], axis=-1)   # m_{v->p}
        bp = phi[:, p, :] + inbox[:, p, :] + down[:, p, :] - up                                          # [C][L_parent]
        down[:, v, :] = np.logaddexp.reduce(bp[:, :, None] + psi[v][None], axis=1)                      # m_{p->v}
    return np.exp(log_softmax(phi + inbox + down))


def blocked_mf_step(model, dec: Decomposition, q, iteration: int, seed: int, parent=None):
    """One tree mean-field iteration from site marginals q [C][N][L]: expected
    duals pi of the non-forest entries given q (theta-update), node potentials
    phi of pi, exact forest marginals by sum-product (x-update).  On lattices
    the forest is the comb forest of the blocked sweep with the block-grid
    offset of the SPLASH draw indexed by the iteration.  Returns the new
    marginals, pi and phi."""
    if parent is None:
        parent = blocked.comb_forest(model.grid, ph.splash_offset(iteration, seed))
    tree = blocked.tree_edge_mask(dec.src, dec.dst, parent)
    q = np.asarray(q, np.float64)
    C = q.shape[0]
    m = dec.ell.shape[1]
    eta_y = q[:, dec.src][:, :, dec.i_pos] if dec.src.size else np.zeros((C, 0, m))
    eta_z = q[:, dec.dst][:, :, dec.j_pos] if dec.dst.size else np.zeros((C, 0, m))
    pi = np.where(~tree[None, :, None], dual_mean(dec, eta_y, eta_z), 0.0)
    phi = blocked.node_potentials(model, dec, tree, pi)
    order, _ = blocked.bfs_order(parent)
    return tree_marginals(model, phi, parent, tree, order), pi, phi


def blocked_mf_objective(model, dec: Decomposition, tree, phi, pi):
    """For one chain: KL(q_x q_theta1 || p(x, theta_1)) and KL(q_x || p(x)) by
    enumeration, where q_x is the tree MRF with node potentials phi [N][L] and
    the exact factors on the forest, q_theta1 = prod of Bernoulli(pi) over the
    active non-forest entries (pi [E][m]) and p(x, theta_1) is Theorem 1's
    joint with the forest's duals summed out (each contributes
    log(1 + e^{logit_k(x)}))."""
    X = brute.all_labelings(model.n_vars, model.n_labels)
    N = model.n_vars
    w = np.asarray(model.pair, np.float64)
    te = np.nonzero(tree)[0]
    lq = phi[np.arange(N)[None, :], X].sum(axis=1)
    if te.size:
        lq = lq + w[te[None, :], X[:, model.src[te]], X[:, model.dst[te]]].sum(axis=1)
    lq = lq - np.logaddexp.reduce(lq)
    ent = brute.active_entries(dec)
    on_tree = tree[ent[:, 0]]
    e, k = ent[:, 0], ent[:, 1]
    y = (X[:, dec.src[e]] == dec.i_pos[k][None, :]).astype(np.float64)
    z = (X[:, dec.dst[e]] == dec.j_pos[k][None, :]).astype(np.float64)
    logit = dec.q[e, k][None] + dec.beta1[e, k][None] * y + dec.beta2[e, k][None] * z     # [S_x][M]
    base = dec.utilde[np.arange(N)[None, :], X].sum(axis=1) + np.logaddexp(0.0, logit[:, on_tree]).sum(axis=1)
    Th = brute.all_dual_configs(int((~on_tree).sum()))
    J = base[:, None] + logit[:, ~on_tree] @ Th.T                                          # log p~(x, theta_1) + const
    lpj = J - np.logaddexp.reduce(J, axis=None)
    p1 = pi[e[~on_tree], k[~on_tree]]
    lqt = (Th * np.log(np.maximum(p1, 1e-300)) + (1 - Th) * np.log(np.maximum(1 - p1, 1e-300))).sum(axis=1)
    wq = np.exp(lq[:, None] + lqt[None, :])
    kl_joint = float((wq * (lq[:, None] + lqt[None, :] - lpj)).sum())
    lpx = np.logaddexp.reduce(lpj, axis=1)
    kl_x = float((np.exp(lq) * (lq - lpx)).sum())
    return kl_joint, kl_x
