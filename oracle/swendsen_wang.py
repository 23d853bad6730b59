"""Swendsen-Wang as a degenerate duality (Section 4.3), oracle side, float64.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
legs use this package.

Every table is first written as w_e(a, b) = c_e + f_e(a) + g_e(b) + l_{e,a} [a = b]
(sw_tables), with f and g folded into the unaries and c_e dropped:
  * L >= 3, diagonal tables (w(a, b) = 0 for a != b): l_{e,a} = w(a, a), f = g = 0;
  * L = 2, any table: one coupling l = (w00 + w11 - w01 - w10) / 2 for both
    labels, f(1) = w10 - w00 + l, g(1) = w01 - w00 + l, f(0) = g(0) = 0
    (the paper's Ising factor [[1, e^{-w}], [e^{-w}, 1]] is the case f = g = 0).
For a ferromagnetic factor (every l >= 0) the remaining table exp(l_a [a = b]) is
    sum_{theta in {0,1}} g(theta) exp(-theta I(a = b)),
    g(0) = 1, g(1) = e^{l_a} - 1 on the diagonal (the paper's form up to the
    factor e^{l}: g(0) = e^{-l}, g(1) = 1 - e^{-l}),
with I(a = b) = 0 if a = b and infinity otherwise.  Hence
    p(theta_e = 1 | x) = 1 - e^{-l_{x_s}} if x_s = x_t, else 0     (a bond),
    p(x | theta): the bonds' connected components ("clusters") take one
    label each, cluster K with probability proportional to
    exp(sum_{v in K} u_v(a) + sum_{bonded e in K} log(e^{l_{e,a}} - 1))
(u the unaries with the offsets folded in; a bonded edge with l_{e,a} = 0
excludes a).  One sweep draws the bonds given x, then the cluster labels.

Draws: bond of edge e, chain c, sweep t: u from word 0 of Philox(e, t, c,
BOND) (23-bit form), bond = [u < p]; label of cluster K: inverse CDF with u
from word 0 of Philox(r, t, c, CLUSTER), r = the smallest site of K.

log_v: Section 5.2's estimator log V = log p~(x) - log p(x | theta) on this
duality, for the labels a sweep draws given its bonds.

Pins (tests/test_oracle_sw.py): the decomposition reproduces every factor;
p~(x, theta) marginalises to p~(x) (enumeration, diagonal Potts and two-label
tables); the cluster label distribution equals p(x | theta) by enumeration;
the SW kernel leaves p invariant (enumeration); chain marginals within 3 sigma
of exact; log V: E[log V] = log Z - I(x; theta) under the joint and
E[V] = Z (p(x) x p(theta))(support) (enumeration; the joint is not strictly
positive here, so V is not unbiased, but E[log V] stays a lower bound on
log Z), and C(theta) log 2 + log p~(x) for the Ising model without fields.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

from . import philox as ph
from .sampler import log_softmax, inverse_cdf


def sw_tables(model):
    """(l [E][L], u [N][L]) of the Swendsen-Wang form of the model (float64).
    Raises ValueError for tables outside the form or with some l < 0."""
    L, N = model.n_labels, model.n_vars
    w = np.asarray(model.pair, np.float64)
    u = np.asarray(model.unary, np.float64).copy()
    E = w.shape[0]
    if E == 0:
        return np.zeros((0, L)), u
    if L == 2:
        kappa = 0.5 * (w[:, 0, 0] + w[:, 1, 1] - w[:, 0, 1] - w[:, 1, 0])
        ell = np.repeat(kappa[:, None], 2, axis=1)
        np.add.at(u[:, 1], np.asarray(model.src, np.int64), w[:, 1, 0] - w[:, 0, 0] + kappa)
        np.add.at(u[:, 1], np.asarray(model.dst, np.int64), w[:, 0, 1] - w[:, 0, 0] + kappa)
    else:
        if np.any(w[:, ~np.eye(L, dtype=bool)] != 0):
            raise ValueError("Swendsen-Wang needs diagonal (Potts-type) tables when L >= 3")
        ell = np.diagonal(w, axis1=1, axis2=2).copy()
    if np.any(ell < 0):
        raise ValueError("Swendsen-Wang needs ferromagnetic tables (l >= 0)")
    return ell, u


def bond_probs(ell, src, dst, x):
    """p(theta_e = 1 | x) [C][E]."""
    x = np.asarray(x, np.int64)
    xs, xt = x[:, src], x[:, dst]
    l_at = np.take_along_axis(np.broadcast_to(ell, (x.shape[0],) + ell.shape), xs[:, :, None], axis=2)[:, :, 0]
    return np.where(xs == xt, -np.expm1(-l_at), 0.0)


def clusters(n_vars, src, dst, bonds_c):
    """Root (smallest site) of every site's cluster for one chain's bonds [E]."""
    sel = np.nonzero(bonds_c)[0]
    g = coo_matrix((np.ones(sel.size), (src[sel], dst[sel])), shape=(n_vars, n_vars))
    _, comp = connected_components(g, directed=False)
    smallest = np.full(comp.max() + 1, n_vars, np.int64)
    np.minimum.at(smallest, comp, np.arange(n_vars))
    return smallest[comp]


def cluster_log_weights(u, ell, src, root, bonds_c):
    """log weight [N][L] of each cluster's label, indexed by its root (other rows 0)."""
    lw = np.zeros(u.shape)
    np.add.at(lw, root, u)
    with np.errstate(divide="ignore"):
        lb = np.log(np.expm1(ell))                                         # log(e^l - 1); -inf where l = 0
    sel = np.nonzero(bonds_c)[0]
    if sel.size:
        np.add.at(lw, root[src[sel]], lb[sel])
    return lw


def log_ptilde(model, x):
    """log p~(x) [C] of the model itself: sum u_v(x_v) + sum w_e(x_s, x_t) (Section 4)."""
    x = np.asarray(x, np.int64)
    u = np.asarray(model.unary, np.float64)
    w = np.asarray(model.pair, np.float64)
    lp = u[np.arange(model.n_vars)[None, :], x].sum(axis=1)
    if w.shape[0]:
        lp += w[np.arange(w.shape[0])[None, :], x[:, model.src], x[:, model.dst]].sum(axis=1)
    return lp


def log_v(model, x, bonds, tables=None):
    """Section 5.2's estimator on the Swendsen-Wang duality, per chain:
    log V = log p~(x) + log p~(theta) - log p~(x, theta) = log p~(x) - log p(x | theta),
    p(x | theta) the product over clusters of the probability of the cluster's
    label (zero where x is not constant on a cluster: log V = +inf).  For the
    Ising model without fields every cluster label has probability 1/2, so
    log V = C(theta) log 2 + log p~(x) (the example of Section 5.2)."""
    ell, u = sw_tables(model) if tables is None else tables
    src, dst = np.asarray(model.src, np.int64), np.asarray(model.dst, np.int64)
    x = np.asarray(x, np.int64)
    out = log_ptilde(model, x)
    for c in range(x.shape[0]):
        root = clusters(model.n_vars, src, dst, bonds[c])
        rs = np.unique(root)
        if np.any(x[c] != x[c][root]):
            out[c] = np.inf
            continue
        lw = cluster_log_weights(u, ell, src, root, bonds[c])
        out[c] -= log_softmax(lw[rs])[np.arange(rs.size), x[c][rs]].sum()
    return out


def exact_moments(model):
    """(E[log V], log Z, I(x; theta)) under the joint of the labels and the bonds,
    by enumerating every (x, theta) (tiny models): the joint is
    p~(x, theta) = exp(sum u_v(x_v) + sum over bonds log(e^{l_{x_s}} - 1)) where
    every bond joins equal labels, else 0 (the tables' split constants dropped)."""
    from .brute import all_labelings, all_dual_configs
    ell, u = sw_tables(model)
    src, dst = np.asarray(model.src, np.int64), np.asarray(model.dst, np.int64)
    X = all_labelings(model.n_vars, model.n_labels)
    B = all_dual_configs(src.size).astype(bool)
    lu = u[np.arange(model.n_vars)[None, :], X].sum(axis=1)
    xs, xt = X[:, src], X[:, dst]
    with np.errstate(divide="ignore"):
        lb = np.where(xs == xt, np.log(np.expm1(ell[np.arange(src.size)[None, :], xs])), -np.inf)   # [S_x][E]
    J = np.full((X.shape[0], B.shape[0]), -np.inf)
    for bi in range(B.shape[0]):
        sel = B[bi]
        J[:, bi] = lu + (lb[:, sel].sum(axis=1) if sel.any() else 0.0)
    logZ = np.logaddexp.reduce(log_ptilde(model, X))
    P = np.exp(J - np.logaddexp.reduce(J.ravel()))
    m = P > 0
    lv = np.zeros(J.shape)
    for bi in range(B.shape[0]):
        ok = m[:, bi]
        if ok.any():
            lv[ok, bi] = log_v(model, X[ok], np.repeat(B[bi][None], ok.sum(), 0), (ell, u))
    e_logv = float((P[m] * lv[m]).sum())
    px, pt = P.sum(axis=1), P.sum(axis=0)
    mi = float((P[m] * (np.log(P[m]) - np.log(np.outer(px, pt)[m]))).sum())
    return e_logv, float(logZ), mi


def sw_sweep(model, x, sweep_index: int, seed: int, edge_ids=None, chain_ids=None, tables=None):
    """One Swendsen-Wang sweep from labels x [C][N].  edge_ids are the RNG
    indices of the edges (default 0..E-1), chain_ids those of the rows of x
    (default 0..C-1); tables = sw_tables(model) if already computed."""
    ell, u = sw_tables(model) if tables is None else tables
    src, dst = np.asarray(model.src, np.int64), np.asarray(model.dst, np.int64)
    x = np.asarray(x, np.int64)
    C, N = x.shape
    ch = np.arange(C, dtype=np.int64) if chain_ids is None else np.asarray(chain_ids, np.int64)
    p = bond_probs(ell, src, dst, x)
    e = np.arange(src.shape[0], dtype=np.int64) if edge_ids is None else np.asarray(edge_ids, np.int64)
    ub = ph.site_uniform(e[None, :], ch[:, None], sweep_index, seed, ph.PH_BOND)
    bonds = ub < p
    x_new = np.zeros_like(x)
    roots = np.zeros_like(x)
    u_cl = np.zeros((C, N)); cdf_cl = np.zeros((C, N, model.n_labels))
    for c in range(C):
        root = clusters(N, src, dst, bonds[c])
        lw = cluster_log_weights(u, ell, src, root, bonds[c])
        rs = np.unique(root)
        uc = ph.site_uniform(rs, ch[c], sweep_index, seed, ph.PH_CLUSTER)
        lab, cdf = inverse_cdf(log_softmax(lw[rs]), uc)
        lab_of = np.zeros(N, np.int64); lab_of[rs] = lab
        x_new[c] = lab_of[root]
        roots[c] = root
        u_cl[c, rs] = uc; cdf_cl[c, rs] = cdf
    return dict(x=x_new, bonds=bonds, p_bond=p, u_bond=ub, roots=roots, u_cluster=u_cl, cdf_cluster=cdf_cl)
