"""Sequential (single-site) Gibbs sampler on p(x) itself, float64 (oracle side).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
legs use this package.

The comparator of the paper's mixing experiments (Section 6): every step
redraws one site from its exact conditional given all others,
    p(x_v = a | x_-v) proportional to exp(u_v(a) + sum over incident edges of w_e),
computed from the raw log-potentials (Section 4's Hammersley-Clifford form),
with no duality involved.  A sweep visits every site once in a fixed order.
Sites of an independent set (no edge between any two of them) are
conditionally independent given the rest, so redrawing them together is the
same transition as redrawing them one after another; `sweep_classes` uses
this for a 2-colourable grid (all even sites, then all odd sites), a
systematic-scan sequential sampler with that visiting order.

Random numbers come from a numpy Generator: this sampler is compared with the
primal-dual sampler only through mixing statistics, never draw by draw.

Pins (tests/test_oracle_gibbs.py): the single-site conditional equals the
conditional of the enumerated p(x); the exact transition matrix of a sweep
leaves p invariant; the class-wise update of an independent set equals the
product of its single-site kernels; a planted mistake (a neighbour's table
read transposed) breaks the invariance.
"""
from __future__ import annotations

import numpy as np

from .sampler import log_softmax


def incidence(model):
    """Per site v: (edges where v is the source, their destinations, edges
    where v is the destination, their sources) as index arrays."""
    out = []
    for v in range(model.n_vars):
        es = np.nonzero(model.src == v)[0]
        et = np.nonzero(model.dst == v)[0]
        out.append((es, model.dst[es], et, model.src[et]))
    return out


def site_field(model, x, v, inc=None):
    """Unnormalised log conditional [C][L] of site v given the other sites of x [C][N]:
    u_v(a) + sum_{e: s(e) = v} w_e(a, x_t(e)) + sum_{e: t(e) = v} w_e(x_s(e), a)."""
    u = np.asarray(model.unary, np.float64)
    w = np.asarray(model.pair, np.float64)
    es, nt, et, ns = incidence(model)[v] if inc is None else inc[v]
    F = np.broadcast_to(u[v], (x.shape[0], model.n_labels)).copy()
    if es.size:
        F += w[es[None, :], :, x[:, nt]].sum(axis=1)          # [C][n][L] -> [C][L]
    if et.size:
        F += w[et[None, :], x[:, ns], :].sum(axis=1)
    return F


def draw_from_logp(logp, u):
    """Smallest a with u < cumsum(p)[a] (the last label when rounding leaves none)."""
    cdf = np.cumsum(np.exp(logp), axis=-1)
    hit = u[..., None] < cdf
    return np.where(hit.any(axis=-1), np.argmax(hit, axis=-1), logp.shape[-1] - 1)


def sweep(model, x, rng, order=None, inc=None):
    """One sequential sweep of x [C][N] (in place), sites in `order` (default 0..N-1)."""
    if inc is None:
        inc = incidence(model)
    order = range(model.n_vars) if order is None else order
    for v in order:
        lp = log_softmax(site_field(model, x, v, inc))
        x[:, v] = draw_from_logp(lp, rng.random(x.shape[0]))
    return x


def class_fields(model, x, sites):
    """Unnormalised log conditionals [C][S][L] of the sites of an independent
    set given the rest (vectorised over the set's incident edges)."""
    u = np.asarray(model.unary, np.float64)
    w = np.asarray(model.pair, np.float64)
    C = x.shape[0]
    pos = -np.ones(model.n_vars, np.int64)
    pos[sites] = np.arange(len(sites))
    F = np.broadcast_to(u[sites], (C, len(sites), model.n_labels)).copy()
    es = np.nonzero(pos[model.src] >= 0)[0]
    et = np.nonzero(pos[model.dst] >= 0)[0]
    for e_set, is_src in ((es, True), (et, False)):
        if not e_set.size:
            continue
        other = model.dst[e_set] if is_src else model.src[e_set]
        me = pos[model.src[e_set]] if is_src else pos[model.dst[e_set]]
        xo = x[:, other]                                                       # [C][n]
        if is_src:
            vals = w[e_set[None, :], :, xo]                                    # [C][n][L]: w_e(a, x_t)
        else:
            vals = w[e_set[None, :], xo, :]                                    # [C][n][L]: w_e(x_s, a)
        flat = (np.arange(C)[:, None] * len(sites) + me[None, :]).ravel()
        for a in range(model.n_labels):
            F[:, :, a] += np.bincount(flat, weights=vals[:, :, a].ravel(), minlength=C * len(sites)).reshape(C, -1)
    return F


def sweep_classes(model, x, rng, classes):
    """One sweep visiting the independent sets in `classes` in turn (in place)."""
    for sites in classes:
        sites = np.asarray(sites, np.int64)
        lp = log_softmax(class_fields(model, x, sites))
        x[:, sites] = draw_from_logp(lp, rng.random((x.shape[0], len(sites))))
    return x


def grid_colour_classes(grid):
    """The two colour classes (x + y + z even / odd) of a lattice."""
    nx, ny, nz = grid
    z, y, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v = (xx + nx * (y + ny * z)).ravel()
    par = ((xx + y + z) % 2).ravel()
    return [np.sort(v[par == 0]), np.sort(v[par == 1])]


def site_kernel(model, X, v):
    """Exact one-site kernel K_v(x, x') over the labelings X [S][N] (tiny models)."""
    S = X.shape[0]
    L = model.n_labels
    index = {tuple(r): i for i, r in enumerate(X)}
    lp = log_softmax(site_field(model, X, v))
    K = np.zeros((S, S))
    for i in range(S):
        y = X[i].copy()
        for a in range(L):
            y[v] = a
            K[i, index[tuple(y)]] += np.exp(lp[i, a])
    return K
