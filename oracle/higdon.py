"""Higdon's partial Swendsen-Wang as a duality (Section 4.3), oracle side, float64.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
legs use this package.

Every table is first put in the Swendsen-Wang form of oracle.swendsen_wang
(sw_tables): exp(l_a [a = b]) up to folded unaries and a constant, l >= 0.
With a fraction rho in [0, 1] the factor splits as
    P(a, b) = 1 + (e^{l_a} - 1) [a = b] = A(a, b) + alpha_a [a = b],
    alpha_a = rho (e^{l_a} - 1),   A(a, b) = exp(l'_a [a = b]),
    l'_a = log(1 + (1 - rho)(e^{l_a} - 1)),
the bond part alpha [a = b] (Higdon's decomposition) and a remainder A that is
itself dualised as in Sections 4.1-4.2 (diagonal layout, one dual bit per
label with l' != 0), so that every cluster can be sampled on its own: the
dual variable of an edge has three kinds of state (a bond, or A with its
bits).  rho = 1 is Swendsen-Wang (A = 1), rho = 0 the plain dual sweep.

Given x: an edge with x_s = x_t = a is a bond with probability
alpha_a / P(a, a) = rho (1 - e^{-l_a}); every edge that is not a bond draws
A's dual bits from their conditionals (Lemma 1).  Given the duals: the bonds'
connected components (clusters) take one label each, cluster K label a with
weight exp(sum_{v in K} F_v(a) + sum_{bonds in K} (log alpha_a - alpha1_a -
alpha2_a)), F the primal field of A's decomposition (its folded unaries plus
the bits' fields; bonds carry no bits) and alpha1, alpha2 the Theorem-2 terms
of A's entry a, folded into the unaries for every edge and taken out again
for bonds.

Draws: bond of edge e, chain c, sweep t: 23-bit uniform of Philox(e, t, c,
BOND) against rho (1 - e^{-l}); A's bits by the dual-bit contract of the
plain sweep (phase DUAL); cluster labels by the inverse CDF with the 23-bit
uniform of Philox(smallest site of the cluster, t, c, CLUSTER).

log_v: Section 5.2's estimator log V = log p~(x) - log p(x | theta) on this
duality, for the labels a sweep draws given its duals.

Pins (tests/test_oracle_higdon.py): the split reproduces every factor; by
enumeration of the three-state duals, the joint marginalises to p~(x), the
bond and bit probabilities given x and the cluster rule given the duals are
the joint's conditionals, and the kernel leaves p invariant; rho = 1 gives
the Swendsen-Wang weights; chain marginals within 3 sigma of exact; log V:
E[log V] = log Z - I(x; theta) under the joint (enumeration).
"""
from __future__ import annotations

import numpy as np

from . import philox as ph
from .decompose import LAYOUT_DIAG, decompose
from .sampler import dual_step, inverse_cdf, log_softmax, primal_field
from .swendsen_wang import clusters, sw_tables


class _TableModel:
    """A model given by float64 unaries and pair tables (for oracle.decompose)."""

    def __init__(self, n_vars, n_labels, unary, src, dst, pair):
        self.n_vars, self.n_labels = n_vars, n_labels
        self.unary, self.src, self.dst, self.pair = unary, src, dst, pair


def higdon_split(model, rho: float, tables=None):
    """(alpha [E][L], A's decomposition) of the model's Swendsen-Wang form."""
    if not 0.0 <= rho <= 1.0:
        raise ValueError("rho must lie in [0, 1]")
    ell, u = sw_tables(model) if tables is None else tables
    E, L = ell.shape
    alpha = rho * np.expm1(ell)
    lp = np.log1p((1.0 - rho) * np.expm1(ell))
    pair = np.zeros((E, L, L))
    pair[:, np.arange(L), np.arange(L)] = lp
    A = _TableModel(model.n_vars, L, u, np.asarray(model.src, np.int64), np.asarray(model.dst, np.int64), pair)
    return alpha, decompose(A, layout=LAYOUT_DIAG)


def bond_log_weights(alpha, dec):
    """log alpha_a - alpha1_a - alpha2_a [E][L] of a bond at label a (-inf where alpha = 0)."""
    with np.errstate(divide="ignore"):
        return np.log(alpha) - dec.alpha1 - dec.alpha2


def cluster_log_weights(model, split, bonds_c, field_c):
    """(root [N], log weight [N][L] of each cluster's label at its root) of one
    chain, from its bonds [E] and the primal field [N][L] of A's bits."""
    alpha, dec = split
    src, dst = np.asarray(model.src, np.int64), np.asarray(model.dst, np.int64)
    root = clusters(model.n_vars, src, dst, bonds_c)
    lw = np.zeros(field_c.shape)
    np.add.at(lw, root, field_c)
    sel = np.nonzero(bonds_c)[0]
    if sel.size:
        np.add.at(lw, root[src[sel]], bond_log_weights(alpha, dec)[sel])
    return root, lw


def log_v(model, x, bonds, theta, split):
    """Section 5.2's estimator on this duality, per chain:
    log V = log p~(x) - log p(x | bonds, bits), p(x | .) the product over the
    clusters of the probability of the cluster's label (+inf where x is not
    constant on a cluster).  x [C][N], bonds [C][E], theta [C][E][L] (A's bits)."""
    from .swendsen_wang import log_ptilde
    alpha, dec = split
    x = np.asarray(x, np.int64)
    F = primal_field(dec, np.asarray(theta) & ~np.asarray(bonds)[:, :, None])
    out = log_ptilde(model, x)
    for c in range(x.shape[0]):
        root, lw = cluster_log_weights(model, split, bonds[c], F[c])
        if np.any(x[c] != x[c][root]):
            out[c] = np.inf
            continue
        rs = np.unique(root)
        out[c] -= log_softmax(lw[rs])[np.arange(rs.size), x[c][rs]].sum()
    return out


def higdon_sweep(model, x, rho: float, sweep_index: int, seed: int, edge_ids=None, chain_ids=None, split=None):
    """One partial Swendsen-Wang sweep from labels x [C][N]."""
    ell, _ = sw_tables(model)
    alpha, dec = higdon_split(model, rho) if split is None else split
    src, dst = np.asarray(model.src, np.int64), np.asarray(model.dst, np.int64)
    x = np.asarray(x, np.int64)
    C, N = x.shape
    L = model.n_labels
    ch = np.arange(C, dtype=np.int64) if chain_ids is None else np.asarray(chain_ids, np.int64)
    e_ids = np.arange(src.size, dtype=np.int64) if edge_ids is None else np.asarray(edge_ids, np.int64)
    # bonds given x
    xs, xt = x[:, src], x[:, dst]
    l_at = np.take_along_axis(np.broadcast_to(ell, (C,) + ell.shape), xs[:, :, None], axis=2)[:, :, 0]
    p_bond = np.where(xs == xt, rho * -np.expm1(-l_at), 0.0)
    u_bond = ph.site_uniform(e_ids[None, :], ch[:, None], sweep_index, seed, ph.PH_BOND)
    bonds = u_bond < p_bond
    # A's bits for the edges that are not bonds (the plain dual-bit contract)
    if chain_ids is None:
        theta, p_dual, u_dual = dual_step(dec, x, sweep_index, seed, edge_ids)
    else:
        theta = np.zeros((C, src.size, dec.n_entries), bool)
        p_dual = np.zeros(theta.shape); u_dual = np.zeros(theta.shape)
        for i, c in enumerate(ch):
            th, pd, ud = _dual_step_chain(dec, x[i], c, sweep_index, seed, edge_ids)
            theta[i], p_dual[i], u_dual[i] = th, pd, ud
    theta &= ~bonds[:, :, None]
    F = primal_field(dec, theta)                                         # [C][N][L]
    x_new = np.zeros_like(x)
    roots = np.zeros_like(x)
    u_cl = np.zeros((C, N)); cdf_cl = np.zeros((C, N, L))
    for i in range(C):
        root, lw = cluster_log_weights(model, (alpha, dec), bonds[i], F[i])
        rs = np.unique(root)
        uc = ph.site_uniform(rs, ch[i], sweep_index, seed, ph.PH_CLUSTER)
        lab, cdf = inverse_cdf(log_softmax(lw[rs]), uc)
        lab_of = np.zeros(N, np.int64); lab_of[rs] = lab
        x_new[i] = lab_of[root]
        roots[i] = root
        u_cl[i, rs] = uc; cdf_cl[i, rs] = cdf
    return dict(x=x_new, bonds=bonds, p_bond=p_bond, u_bond=u_bond, theta=theta, p_dual=p_dual, u_dual=u_dual,
                field=F, roots=roots, u_cluster=u_cl, cdf_cluster=cdf_cl)


def _dual_step_chain(dec, x_c, chain, sweep_index, seed, edge_ids):
    """The dual step of one chain with its own RNG chain index."""
    from .sampler import dual_probs
    E, m = dec.ell.shape
    e = np.arange(E, dtype=np.int64) if edge_ids is None else np.asarray(edge_ids, np.int64)
    p = dual_probs(dec, x_c[None])[0]
    u = ph.dual_uniform(e[:, None], np.arange(m)[None, :], np.int64(chain), sweep_index, seed, m)
    return (u < p) & dec.active, p, u
