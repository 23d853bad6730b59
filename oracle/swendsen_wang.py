"""Swendsen-Wang as a degenerate duality (Section 4.3), oracle side, float64.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
legs use this package.

For a ferromagnetic Potts factor P(a, b) = exp(l_a [a = b]) with l_a >= 0
(the diagonal layout of oracle.decompose, every active entry positive),
    P(a, b) = sum_{theta in {0,1}} g(theta) exp(-theta I(a = b)),
    g(0) = 1, g(1) = e^{l_a} - 1 on the diagonal (the paper's form up to the
    factor e^{l}: g(0) = e^{-l}, g(1) = 1 - e^{-l}),
with I(a = b) = 0 if a = b and infinity otherwise.  Hence
    p(theta_e = 1 | x) = 1 - e^{-l_{x_s}} if x_s = x_t, else 0     (a bond),
    p(x | theta): the bonds' connected components ("clusters") take one
    label each, cluster K with probability proportional to
    exp(sum_{v in K} u_v(a) + sum_{bonded e in K} log(e^{l_{e,a}} - 1)).
One sweep draws the bonds given x, then the cluster labels.

Draws: bond of edge e, chain c, sweep t: u from word 0 of Philox(e, t, c,
BOND) (23-bit form), bond = [u < p]; label of cluster K: inverse CDF with u
from word 0 of Philox(r, t, c, CLUSTER), r = the smallest site of K.

Pins (tests/test_oracle_sw.py): the decomposition reproduces every factor;
p~(x, theta) marginalises to p~(x); the cluster label distribution equals
p(x | theta) by enumeration; the SW kernel leaves p invariant (enumeration);
chain marginals within 3 sigma of exact.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

from . import philox as ph
from .decompose import Decomposition, LAYOUT_DIAG
from .sampler import log_softmax, inverse_cdf


def check_model(dec: Decomposition):
    """SW needs the diagonal layout with every active entry l > 0."""
    if dec.layout != LAYOUT_DIAG:
        raise ValueError("Swendsen-Wang needs Potts tables (diagonal layout)")
    if np.any(dec.ell[dec.active] <= 0):
        raise ValueError("Swendsen-Wang needs ferromagnetic tables (l >= 0)")


def bond_probs(dec: Decomposition, x):
    """p(theta_e = 1 | x) [C][E]."""
    x = np.asarray(x, np.int64)
    xs, xt = x[:, dec.src], x[:, dec.dst]
    ell = np.where(dec.active, dec.ell, 0.0)                              # [E][L]
    l_at = np.take_along_axis(np.broadcast_to(ell, (x.shape[0],) + ell.shape), xs[:, :, None], axis=2)[:, :, 0]
    return np.where(xs == xt, -np.expm1(-l_at), 0.0)


def bond_uniforms(dec: Decomposition, n_chains, sweep, seed, edge_ids=None):
    E = dec.src.shape[0]
    e = np.arange(E, dtype=np.int64) if edge_ids is None else np.asarray(edge_ids, np.int64)
    return ph.site_uniform(e[None, :], np.arange(n_chains)[:, None], sweep, seed, ph.PH_BOND)


def clusters(n_vars, src, dst, bonds_c):
    """Root (smallest site) of every site's cluster for one chain's bonds [E]."""
    sel = np.nonzero(bonds_c)[0]
    g = coo_matrix((np.ones(sel.size), (src[sel], dst[sel])), shape=(n_vars, n_vars))
    _, comp = connected_components(g, directed=False)
    smallest = np.full(comp.max() + 1, n_vars, np.int64)
    np.minimum.at(smallest, comp, np.arange(n_vars))
    return smallest[comp]


def cluster_log_weights(model, dec: Decomposition, root, bonds_c):
    """log weight [N][L] of each cluster's label, indexed by its root (other rows 0)."""
    N, L = model.n_vars, model.n_labels
    lw = np.zeros((N, L))
    np.add.at(lw, root, np.asarray(model.unary, np.float64))
    ell = np.where(dec.active, dec.ell, 0.0)
    with np.errstate(divide="ignore"):
        lb = np.log(np.expm1(ell))                                         # log(e^l - 1); -inf where l = 0
    sel = np.nonzero(bonds_c)[0]
    np.add.at(lw, root[dec.src[sel]], lb[sel])
    return lw


def sw_sweep(model, dec: Decomposition, x, sweep_index: int, seed: int):
    """One Swendsen-Wang sweep from labels x [C][N]."""
    check_model(dec)
    x = np.asarray(x, np.int64)
    C, N = x.shape
    p = bond_probs(dec, x)
    u = bond_uniforms(dec, C, sweep_index, seed)
    bonds = u < p
    x_new = np.zeros_like(x)
    roots = np.zeros_like(x)
    u_cl = np.zeros((C, N)); cdf_cl = np.zeros((C, N, model.n_labels))
    for c in range(C):
        root = clusters(N, dec.src, dec.dst, bonds[c])
        lw = cluster_log_weights(model, dec, root, bonds[c])
        rs = np.unique(root)
        uc = ph.site_uniform(rs, c, sweep_index, seed, ph.PH_CLUSTER)
        lab, cdf = inverse_cdf(log_softmax(lw[rs]), uc)
        lab_of = np.zeros(N, np.int64); lab_of[rs] = lab
        x_new[c] = lab_of[root]
        roots[c] = root
        u_cl[c, rs] = uc; cdf_cl[c, rs] = cdf
    return dict(x=x_new, bonds=bonds, p_bond=p, u_bond=u, roots=roots, u_cluster=u_cl, cdf_cluster=cdf_cl)
