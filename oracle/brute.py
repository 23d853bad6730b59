"""Brute-force enumeration for tiny models (oracle pins; float64).

Everything here is computed from the raw model (unary, pair) or from the
definitions of Theorem 1 and Lemma 1 by explicit enumeration over all
labelings (L^N <= ~2^20) and all dual configurations (2^M, M <= ~20):
  * p(x) from the raw log-potentials (Section 4, Hammersley-Clifford form),
  * p~(x, theta) = h(x) g(theta) exp(<s(x), r(theta)>) (Theorem 1),
  * the exact transition matrix of a sweep,
    K(x, x') = sum_theta p(theta | x) p(x' | theta).
"""
from __future__ import annotations

import itertools

import numpy as np

from .decompose import Decomposition
from .sampler import dual_probs, primal_field, log_softmax


def all_labelings(n_vars: int, n_labels: int):
    """[L^N][N] labelings, site 0 varying slowest."""
    return np.array(list(itertools.product(range(n_labels), repeat=n_vars)), np.int64).reshape(-1, n_vars)


def log_ptilde(model, X):
    """log p~(x) = sum_v u_v(x_v) + sum_e w_e(x_s, x_t) for labelings X [S][N]."""
    u = np.asarray(model.unary, np.float64)
    w = np.asarray(model.pair, np.float64)
    out = u[np.arange(model.n_vars)[None, :], X].sum(axis=1)
    if model.n_edges:
        out += w[np.arange(model.n_edges)[None, :], X[:, model.src], X[:, model.dst]].sum(axis=1)
    return out


def exact_distribution(model):
    X = all_labelings(model.n_vars, model.n_labels)
    lp = log_ptilde(model, X)
    logZ = np.logaddexp.reduce(lp)
    return X, np.exp(lp - logZ), logZ


def exact_marginals(model):
    X, p, logZ = exact_distribution(model)
    marg = np.zeros((model.n_vars, model.n_labels))
    for v in range(model.n_vars):
        np.add.at(marg[v], X[:, v], p)
    return marg, logZ


def active_entries(dec: Decomposition):
    """(edge, entry) index pairs of all dual variables."""
    return np.argwhere(dec.active)


def joint_log(dec: Decomposition, X, Theta):
    """log p~(x, theta) [S_x][S_theta] by Theorem 1 with Theorem 2's h, g, r.

    Theta [S_theta][M] lists the dual configurations over active_entries(dec)."""
    ent = active_entries(dec)
    e, k = ent[:, 0], ent[:, 1]
    N = dec.utilde.shape[0]
    log_h = dec.utilde[np.arange(N)[None, :], X].sum(axis=1)              # h(x), folded
    y = (X[:, dec.src[e]] == dec.i_pos[k][None, :]).astype(np.float64)     # s(x) components
    z = (X[:, dec.dst[e]] == dec.j_pos[k][None, :]).astype(np.float64)
    r1 = dec.beta1[e, k]; r2 = dec.beta2[e, k]; q = dec.q[e, k]
    Th = np.asarray(Theta, np.float64)
    inner = (y * r1[None]) @ Th.T + (z * r2[None]) @ Th.T                 # <s(x), r(theta)>
    log_g = Th @ q                                                        # g(theta)
    return log_h[:, None] + log_g[None, :] + inner + dec.log_const


def all_dual_configs(M: int):
    return np.array(list(itertools.product((0, 1), repeat=M)), np.int64).reshape(-1, M)


def sweep_kernel(dec: Decomposition, X):
    """Exact K(x, x') of one sweep (theta | x, then x' | theta) over labelings X."""
    ent = active_entries(dec)
    M = ent.shape[0]
    Th = all_dual_configs(M)                                              # [S_t][M]
    p1 = dual_probs(dec, X)                                               # [S_x][E][m]
    pa = p1[:, ent[:, 0], ent[:, 1]]                                      # [S_x][M]
    log_pt = (np.log(pa)[:, None, :] * Th[None] + np.log1p(-pa)[:, None, :] * (1 - Th[None])).sum(-1)
    E, m = dec.ell.shape
    theta_full = np.zeros((Th.shape[0], E, m))
    theta_full[:, ent[:, 0], ent[:, 1]] = Th
    logp = log_softmax(primal_field(dec, theta_full))                     # [S_t][N][L]
    N = X.shape[1]
    log_px = logp[:, np.arange(N)[None, :], X].sum(-1)                    # [S_t][S_x']
    return np.exp(log_pt) @ np.exp(log_px)
