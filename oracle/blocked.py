"""Blocked primal-dual sweep of Section 5.4 (Figure 1), float64 oracle side.

The dual variables are split into theta_0 (edges of a spanning forest T,
kept exact) and theta_1 (all other edges).  Because p(x | theta_1) is a
tree-structured MRF it is sampled exactly, by forward filtering (messages
from the leaves to each root) and backward sampling (root first, then every
child given its parent).  A sweep draws theta_1 | x (the plain dual step
restricted to non-tree edges), then x | theta_1.  The split may change every
sweep (Section 5.4, last paragraph).

With the folded unaries u~ of oracle.decompose, p(x | theta_1) has
  node potentials  phi_v(a) = u~_v(a) - sum_{e in T incident to v} fold_{e,v}(a)
                               + sum_{e not in T} (beta terms of theta_1)
  edge potentials  psi_e(a, b) = w_e(a, b)   for e in T (the exact factor).

Forest used for lattices ("comb" spanning tree of every block, reading of
"a tree or splash" for grids): the sites are cut into 4x4x4 blocks whose
grid is shifted by an offset o in [0,4)^3 drawn every sweep (boundary blocks
are clipped).  Inside a block with local coordinates (lx, ly, lz) the root is
(0,0,0) and
  parent(lx>0, ly, lz) = (lx-1, ly, lz)
  parent(0, ly>0, lz)  = (0, ly-1, lz)
  parent(0, 0, lz>0)   = (0, 0, lz-1).

Label draws inside blocks use phase FFBS of the draw contract (site-indexed,
so the order of the backward pass does not change which uniform a site uses).

Parity: pinned by enumeration on small blocks (the sampled tree conditional
equals the exact p(x | theta_1)) and by stationarity of the blocked kernel.
"""
from __future__ import annotations

import numpy as np

from . import philox as ph
from .decompose import Decomposition, fold_vectors
from .sampler import dual_probs, dual_uniforms, log_softmax, inverse_cdf


def comb_forest(grid, offset, block=4):
    """Parent of every site (-1 for roots) for the comb trees of the blocks."""
    nx, ny, nz = grid
    ox, oy, oz = offset
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    def lo(c, o):
        return np.maximum(0, ((c + o) // block) * block - o)
    lx, ly, lz = x - lo(x, ox), y - lo(y, oy), z - lo(z, oz)
    v = x + nx * (y + ny * z)
    parent = np.full(nx * ny * nz, -1, np.int64)
    px = lx > 0
    parent[v[px]] = v[px] - 1
    py = (lx == 0) & (ly > 0)
    parent[v[py]] = v[py] - nx
    pz = (lx == 0) & (ly == 0) & (lz > 0)
    parent[v[pz]] = v[pz] - nx * ny
    return parent


def tree_edge_mask(src, dst, parent):
    """Edge e is a tree edge when one endpoint is the other's parent."""
    return (parent[dst] == src) | (parent[src] == dst)


def bfs_order(parent):
    """Sites ordered so that every parent precedes its children."""
    N = parent.shape[0]
    depth = np.zeros(N, np.int64)
    # iterate pointer jumping: depth(v) = depth(parent)+1
    cur = parent.copy()
    active = cur >= 0
    while np.any(active):
        depth[active] += 1
        cur[active] = parent[cur[active]]
        active = cur >= 0
    return np.argsort(depth, kind="stable"), depth


def node_potentials(model, dec: Decomposition, tree, theta):
    """phi [C][N][L] for theta [C][E][m] (entries of tree edges are ignored)."""
    fold_s, fold_t = fold_vectors(model, dec)
    C = theta.shape[0]
    N, L = dec.utilde.shape
    base = dec.utilde.copy()
    te = np.nonzero(tree)[0]
    np.add.at(base, dec.src[te], -fold_s[te])
    np.add.at(base, dec.dst[te], -fold_t[te])
    phi = np.broadcast_to(base, (C, N, L)).copy()
    nt = np.nonzero(~tree)[0]
    if nt.size:
        m = dec.n_entries
        th = np.asarray(theta, np.float64)[:, nt, :]
        cc = np.broadcast_to(np.arange(C)[:, None, None], th.shape)
        ss = np.broadcast_to(dec.src[nt][None, :, None], th.shape)
        tt = np.broadcast_to(dec.dst[nt][None, :, None], th.shape)
        ii = np.broadcast_to(dec.i_pos[None, None, :], th.shape)
        jj = np.broadcast_to(dec.j_pos[None, None, :], th.shape)
        np.add.at(phi, (cc, ss, ii), dec.beta1[nt][None] * th)
        np.add.at(phi, (cc, tt, jj), dec.beta2[nt][None] * th)
    return phi


def _edge_to_parent(src, dst, parent, tree):
    """For every non-root site: (edge id, child-is-src flag) of its tree edge."""
    N = parent.shape[0]
    pe = np.full(N, -1, np.int64); child_is_src = np.zeros(N, bool)
    for e in np.nonzero(tree)[0]:
        s, t = int(src[e]), int(dst[e])
        if parent[t] == s:
            pe[t] = e; child_is_src[t] = False
        else:
            pe[s] = e; child_is_src[s] = True
    return pe, child_is_src


def tree_messages(model, phi, parent, tree, order):
    """Upward log-messages.  Returns inbox [C][N][L] (sum of children's messages)
    and the oriented edge potential of every child, psi_child[v] [L_parent][L_child]."""
    C, N, L = phi.shape
    pe, child_is_src = _edge_to_parent(model.src, model.dst, parent, tree)
    w = np.asarray(model.pair, np.float64)
    inbox = np.zeros((C, N, L))
    psi = np.zeros((N, L, L))
    for v in order[::-1]:
        p = parent[v]
        if p < 0:
            continue
        e = pe[v]
        psi[v] = w[e].T if child_is_src[v] else w[e]          # [parent label][child label]
        lv = phi[:, v, :] + inbox[:, v, :]                       # [C][L_child]
        msg = np.logaddexp.reduce(lv[:, None, :] + psi[v][None], axis=-1)   # [C][L_parent]
        inbox[:, p, :] += msg
    return inbox, psi


def ffbs(model, phi, parent, tree, order, sweep_index, seed):
    """Exact draw from the tree MRF; returns labels [C][N] and per-site
    sampling log-probabilities [C][N][L] (the conditional each draw used)."""
    C, N, L = phi.shape
    inbox, psi = tree_messages(model, phi, parent, tree, order)
    u = ph.site_uniform(np.arange(N)[None, :], np.arange(C)[:, None], sweep_index, seed, ph.PH_FFBS)
    x = np.zeros((C, N), np.int64)
    logp = np.zeros((C, N, L))
    cdf = np.zeros((C, N, L))
    for v in order:
        lv = phi[:, v, :] + inbox[:, v, :]
        p = parent[v]
        if p >= 0:
            lv = lv + psi[v][x[:, p], :]
        lp = log_softmax(lv)
        xv, cv = inverse_cdf(lp, u[:, v])
        x[:, v] = xv; logp[:, v] = lp; cdf[:, v] = cv
    return x, logp, u, cdf


def tree_conditional_logprob(model, phi, parent, tree, order, x):
    """log p(x | theta_1) of labels x [S][N] under the tree MRF (exact);
    phi is [S][N][L] or [1][N][L] (shared by all S labelings)."""
    _, N, L = phi.shape
    S = x.shape[0]
    inbox, psi = tree_messages(model, phi, parent, tree, order)
    out = np.zeros(S)
    for v in order:
        lv = np.broadcast_to(phi[:, v, :] + inbox[:, v, :], (S, L))
        p = parent[v]
        if p >= 0:
            lv = lv + psi[v][x[:, p], :]
        lp = log_softmax(lv)
        out += lp[np.arange(S), x[:, v]]
    return out


def blocked_sweep(model, dec: Decomposition, x, sweep_index, seed, parent=None, edge_ids=None):
    """One blocked sweep: theta_1 | x on non-tree edges, then x | theta_1 by FFBS.
    For lattice models the comb forest of this sweep's offset is used."""
    if parent is None:
        parent = comb_forest(model.grid, ph.splash_offset(sweep_index, seed))
    tree = tree_edge_mask(dec.src, dec.dst, parent)
    p = dual_probs(dec, x)
    u = dual_uniforms(dec, p.shape[0], sweep_index, seed, edge_ids)
    theta = (u < p) & dec.active[None] & ~tree[None, :, None]
    phi = node_potentials(model, dec, tree, theta)
    order, _ = bfs_order(parent)
    x_new, logp, u_site, cdf = ffbs(model, phi, parent, tree, order, sweep_index, seed)
    return dict(x=x_new, theta=theta, p_dual=p, u_dual=u, logp=logp, u_site=u_site, cdf=cdf,
                tree=tree, parent=parent)
