"""Learned block proposal with Metropolis-Hastings correction (float64, oracle side).

The paper has no learned component; this is the statement, in plain numpy,
of the MH-within-Gibbs step the library runs on top of Section 5.4's
blocking.  Sites are partitioned into blocks of at most B = 16 sites.  Each
sweep draws the dual variables of the cut edges (edges between blocks) given
x, exactly as the plain dual step; given those, p(x | theta_cut) factorises
over blocks with the intra-block factors kept exact:
    pi(x_B) ~ exp( sum_{v in B} phi_v(x_v) + sum_{e inside B} w_e(x_s, x_t) ),
    phi_v = u~_v - (folds of v's intra-block edges) + (beta terms of cut duals)
(oracle.blocked.node_potentials with the intra-block edges as the kept set).
The block's labels are updated by one independence Metropolis-Hastings step
with a factorised proposal q(x_B) = prod_i softmax(z_i)(x_i) whose logits z
come from an MLP of the block's features; acceptance
min(1, pi(x') q(x) / (pi(x) q(x'))) keeps p(x_B | theta_cut) invariant.

Features of block b, chain c (row b*C + c), width D = B*L + B(B-1)/2, padded
with zeros to a multiple of 32:
  * [i*L + a]: phi^f_{v_i}(a) - mean_a phi^f_{v_i}(a) for member i (sorted site
    ids), with phi^f_v = u~_v + (beta terms of the cut duals) -- the primal
    field of the plain sweep restricted to cut edges; zero for i >= n_b;
  * [B*L + pair(i, j)]: sum over edges between members i < j of
    kappa_e = mean_a w_e(a, a) - mean_{a != b} w_e(a, b), pair(i, j) the index
    of (i, j) in row-major order of the strict upper triangle.
MLP: h1 = relu(X W1^T + b1), h2 = relu(h1 W2^T + b2), z = h2 W3^T + b3,
z reshaped to [B][L].  Training minimises the mean over samples of
-sum_{i < n_b} log softmax(z_i)(y_i) (cross-entropy of the factorised proposal).

Draws: proposal label of member i uses the label-draw form of the contract
with phase PROPOSAL and index = its site id; the accept uniform uses phase
ACCEPT with index = block id, same 23-bit form; accept iff u < exp(min(0, log a)).

Parity: MLP forward/backward pinned by central finite differences; the MH
kernel pinned by exact stationarity on enumerable blocks (any weights).
"""
from __future__ import annotations

import numpy as np

from . import philox as ph
from .blocked import node_potentials
from .decompose import Decomposition
from .sampler import dual_probs, dual_uniforms, primal_field, log_softmax, inverse_cdf

BLOCK = 16


def pair_index(i, j, B=BLOCK):
    """Index of (i, j), i < j, in row-major order of the strict upper triangle."""
    return i * (2 * B - i - 1) // 2 + (j - i - 1)


def feature_width(L, B=BLOCK):
    d = B * L + B * (B - 1) // 2
    return d, (d + 31) // 32 * 32


def block_members(block_of_site):
    n_blocks = int(block_of_site.max()) + 1
    order = np.argsort(block_of_site, kind="stable")
    members = [[] for _ in range(n_blocks)]
    for v in order:
        members[block_of_site[v]].append(int(v))
    return [np.array(sorted(m), np.int64) for m in members]


def intra_mask(src, dst, block_of_site):
    return block_of_site[src] == block_of_site[dst]


def coupling_features(model, block_of_site, members, B=BLOCK):
    L = model.n_labels
    w = np.asarray(model.pair, np.float64)
    diag = np.diagonal(w, axis1=1, axis2=2).mean(axis=1)
    off = (w.sum(axis=(1, 2)) - np.diagonal(w, axis1=1, axis2=2).sum(axis=1)) / (L * (L - 1))
    kappa = diag - off
    pos = {}
    for b, m in enumerate(members):
        for i, v in enumerate(m):
            pos[int(v)] = i
    cf = np.zeros((len(members), B * (B - 1) // 2))
    for e in np.nonzero(intra_mask(model.src, model.dst, block_of_site))[0]:
        b = block_of_site[model.src[e]]
        i, j = pos[int(model.src[e])], pos[int(model.dst[e])]
        i, j = min(i, j), max(i, j)
        cf[b, pair_index(i, j, B)] += kappa[e]
    return cf


def features(phi_f, members, cf, L, B=BLOCK):
    """X [n_blocks * C][D_pad] from phi^f [C][N][L] (rows b*C + c)."""
    C = phi_f.shape[0]
    d, dp = feature_width(L, B)
    X = np.zeros((len(members) * C, dp))
    for b, m in enumerate(members):
        ph_b = phi_f[:, m, :]                                    # [C][n_b][L]
        ph_b = ph_b - ph_b.mean(axis=2, keepdims=True)
        X[b * C:(b + 1) * C, :len(m) * L] = ph_b.reshape(C, -1)
        X[b * C:(b + 1) * C, B * L:d] = cf[b][None, :]
    return X


# ----------------------------------------------------------------------------- MLP

def mlp_forward(params, X):
    W1, b1, W2, b2, W3, b3 = params
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ W3.T + b3
    return z, (X, a1, h1, a2, h2)


def mlp_forward_bf16(params, X):
    """Forward pass with the inputs and hidden activations rounded to bfloat16
    between layers (the precision in which the device stores them); the
    arithmetic itself stays float64."""
    W1, b1, W2, b2, W3, b3 = params
    Xb = to_bf16(X)
    h1 = to_bf16(np.maximum(Xb @ W1.T + b1, 0.0))
    h2 = to_bf16(np.maximum(h1 @ W2.T + b2, 0.0))
    return h2 @ W3.T + b3


def ce_loss(z, y, nmem, L, B=BLOCK):
    """Mean over rows of -sum_{i < n_b} log softmax(z_i)(y_i)."""
    R = z.shape[0]
    lz = log_softmax(z.reshape(R, B, L))
    mask = np.arange(B)[None, :] < nmem[:, None]
    lp = np.take_along_axis(lz, y[:, :, None].astype(np.int64), axis=2)[:, :, 0]
    return float(-(lp * mask).sum() / R), lz, mask


def loss_and_grads(params, X, y, nmem, L, B=BLOCK):
    """Loss and gradients (same order as params) by backpropagation."""
    W1, b1, W2, b2, W3, b3 = params
    z, (X, a1, h1, a2, h2) = mlp_forward(params, X)
    R = z.shape[0]
    loss, lz, mask = ce_loss(z, y, nmem, L, B)
    p = np.exp(lz)                                               # [R][B][L]
    onehot = np.zeros_like(p)
    np.put_along_axis(onehot, y[:, :, None].astype(np.int64), 1.0, axis=2)
    dz = ((p - onehot) * mask[:, :, None]).reshape(R, B * L) / R
    dW3 = dz.T @ h2; db3 = dz.sum(0)
    dh2 = dz @ W3
    da2 = dh2 * (a2 > 0)
    dW2 = da2.T @ h1; db2 = da2.sum(0)
    dh1 = da2 @ W2
    da1 = dh1 * (a1 > 0)
    dW1 = da1.T @ X; db1 = da1.sum(0)
    return loss, [dW1, db1, dW2, db2, dW3, db3]


def init_params(L, hidden=256, B=BLOCK, seed=0):
    """He-uniform weights, zero biases, rounded to bfloat16 values."""
    rng = np.random.default_rng(seed)
    d, dp = feature_width(L, B)
    shapes = [(hidden, dp), (hidden, hidden), (B * L, hidden)]
    out = []
    for (o, i) in shapes:
        lim = np.sqrt(6.0 / i)
        out += [to_bf16(rng.uniform(-lim, lim, size=(o, i))), np.zeros(o)]
    return out


def to_bf16(a):
    """Round float64 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# ----------------------------------------------------------------------------- MH sweep

def block_log_target(phi, w, members, intra_edges, x, b):
    """log pi(x_B) (unnormalised) for labels x [C][N] of block b."""
    m = members[b]
    C = x.shape[0]
    out = phi[np.arange(C)[:, None], m[None, :], x[:, m]].sum(axis=1)
    for e, s, t in intra_edges[b]:
        out = out + w[e, x[:, s], x[:, t]]
    return out


def intra_edge_lists(model, block_of_site, n_blocks):
    lists = [[] for _ in range(n_blocks)]
    for e in np.nonzero(intra_mask(model.src, model.dst, block_of_site))[0]:
        lists[block_of_site[model.src[e]]].append((int(e), int(model.src[e]), int(model.dst[e])))
    return lists


def learned_sweep(model, dec: Decomposition, x, sweep_index, seed, block_of_site, params, edge_ids=None,
                  bf16_activations=False, site_ids=None, block_ids=None, blocks=None):
    """One learned sweep from labels x [C][N]; returns a dict with the new labels.
    bf16_activations: evaluate the proposal with inputs and hidden activations
    rounded to bfloat16 (the device's storage precision).
    For a sub-model cut out of a larger one: edge_ids, site_ids and block_ids
    map its edges, sites and blocks to the larger model's (the indices of the
    draw contract), and blocks (default all) lists the blocks to update; the
    MLP then runs on those blocks' rows only (z has nb * C rows, zero
    elsewhere)."""
    C, N = x.shape
    L = model.n_labels
    members = block_members(block_of_site)
    nb = len(members)
    sid = np.arange(N) if site_ids is None else np.asarray(site_ids)
    bid = np.arange(nb) if block_ids is None else np.asarray(block_ids)
    todo = list(range(nb)) if blocks is None else [int(b) for b in blocks]
    intra = intra_mask(dec.src, dec.dst, block_of_site)
    # cut duals | x
    p = dual_probs(dec, x)
    u = dual_uniforms(dec, C, sweep_index, seed, edge_ids)
    theta = (u < p) & dec.active[None] & ~intra[None, :, None]
    phi_f = primal_field(dec, theta)                              # feature field u~ + cut terms
    phi = node_potentials(model, dec, intra, theta)               # target field
    cf = coupling_features(model, block_of_site, members)
    X = features(phi_f, members, cf, L)
    rows_todo = (np.asarray(todo, np.int64)[:, None] * C + np.arange(C)[None, :]).ravel()
    zt = mlp_forward_bf16(params, X[rows_todo]) if bf16_activations else mlp_forward(params, X[rows_todo])[0]
    z = np.zeros((nb * C, zt.shape[1]))
    z[rows_todo] = zt
    lz = log_softmax(z.reshape(nb * C, BLOCK, L))                 # rows b*C + c
    w = np.asarray(model.pair, np.float64)
    lists = intra_edge_lists(model, block_of_site, nb)
    x_new = x.copy()
    accepted = np.zeros((nb, C), bool)
    log_alpha = np.zeros((nb, C))
    u_acc_all = np.zeros((nb, C))
    prop_cdf = {}
    for b in todo:
        m = members[b]
        rows = b * C + np.arange(C)
        lzb = lz[rows][:, :len(m), :]                             # [C][n_b][L]
        u_prop = ph.site_uniform(sid[m][None, :], np.arange(C)[:, None], sweep_index, seed, ph.PH_PROPOSAL)
        xp, cdf = inverse_cdf(lzb, u_prop)                        # [C][n_b]
        prop_cdf[b] = (u_prop, cdf)
        cur = x[:, m]
        lq_cur = np.take_along_axis(lzb, cur[:, :, None], axis=2)[:, :, 0].sum(1)
        lq_new = np.take_along_axis(lzb, xp[:, :, None], axis=2)[:, :, 0].sum(1)
        xprop = x.copy(); xprop[:, m] = xp
        lp_cur = block_log_target(phi, w, members, lists, x, b)
        lp_new = block_log_target(phi, w, members, lists, xprop, b)
        la = (lp_new - lp_cur) + (lq_cur - lq_new)
        u_acc = ph.site_uniform(np.full((C, 1), bid[b]), np.arange(C)[:, None], sweep_index, seed, ph.PH_ACCEPT)[:, 0]
        acc = u_acc < np.exp(np.minimum(0.0, la))
        x_new[np.ix_(np.nonzero(acc)[0], m)] = xp[acc]
        accepted[b] = acc; log_alpha[b] = la; u_acc_all[b] = u_acc
    return dict(x=x_new, theta=theta, p_dual=p, u_dual=u, X=X, z=z, accepted=accepted, log_alpha=log_alpha,
                u_acc=u_acc_all, prop=prop_cdf, phi=phi, members=members)
