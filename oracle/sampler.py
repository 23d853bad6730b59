"""Two-block primal-dual Gibbs sweep of Section 5.1, in float64 (oracle side).

With the decomposition of Section 4 (oracle.decompose) the joint is
    p~(x, theta) = exp(sum_v u~_v(x_v)) * prod_{e,k} exp(theta_ek * logit_ek(x))
    logit_ek(x) = q_ek + beta1_ek [x_s = i_k] + beta2_ek [x_t = j_k]
(Theorem 1 with h, g, r from Theorem 2).  Lemma 1 / Corollary 1 give the two
conditionals, both fully factorised:
  * p(theta_ek = 1 | x) = sigmoid(logit_ek(x))                     (dual step)
  * p(x_v = a | theta) = softmax_a F_v(a),                          (primal step)
      F_v(a) = u~_v(a) + sum_{e: s=v} sum_{k: i_k=a} beta1_ek theta_ek
                       + sum_{e: t=v} sum_{k: j_k=a} beta2_ek theta_ek.
The state carried between sweeps is x; each sweep draws theta | x and then
x | theta (the paper lists x first; starting from x is the same chain shifted
by half a step).

Draws follow the contract in oracle.philox.  A Bernoulli draw is
theta = [u < p]; a label draw takes the smallest a with u < sum_{a' <= a} p(a'),
falling back to the largest a with p(a) > 0 when rounding leaves none.

Parity: pinned by brute-force enumeration on tiny models (conditionals equal
those of the enumerated joint; the exact sweep kernel leaves p invariant;
sampled marginals agree with exact ones within 3 sigma).
"""
from __future__ import annotations

import numpy as np

from . import philox as ph
from .decompose import Decomposition


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def dual_logits(dec: Decomposition, x):
    """logit_ek(x) for labels x [C][N] -> [C][E][m]."""
    x = np.asarray(x, np.int64)
    y = (x[:, dec.src][:, :, None] == dec.i_pos[None, None, :]).astype(np.float64)
    z = (x[:, dec.dst][:, :, None] == dec.j_pos[None, None, :]).astype(np.float64)
    return dec.q[None] + dec.beta1[None] * y + dec.beta2[None] * z


def dual_probs(dec: Decomposition, x):
    """p(theta_ek = 1 | x) [C][E][m]; exactly 0 for entries without a dual variable."""
    return np.where(dec.active[None], sigmoid(dual_logits(dec, x)), 0.0)


def dual_uniforms(dec: Decomposition, n_chains: int, sweep: int, seed: int, edge_ids=None):
    E, m = dec.ell.shape
    e = np.arange(E, dtype=np.int64) if edge_ids is None else np.asarray(edge_ids, np.int64)
    return ph.dual_uniform(e[None, :, None], np.arange(m)[None, None, :],
                           np.arange(n_chains)[:, None, None], sweep, seed, m)


def dual_step(dec: Decomposition, x, sweep: int, seed: int, edge_ids=None):
    """theta ~ p(theta | x): [C][E][m] bool.  edge_ids are the RNG slots of the edges."""
    p = dual_probs(dec, x)
    u = dual_uniforms(dec, p.shape[0], sweep, seed, edge_ids)
    return (u < p) & dec.active[None], p, u


def primal_field(dec: Decomposition, theta):
    """F [C][N][L] given theta [C][E][m]."""
    theta = np.asarray(theta, np.float64)
    C = theta.shape[0]
    N, L = dec.utilde.shape
    E, m = dec.ell.shape
    F = np.broadcast_to(dec.utilde, (C, N, L)).copy()
    cc = np.broadcast_to(np.arange(C)[:, None, None], (C, E, m))
    ss = np.broadcast_to(dec.src[None, :, None], (C, E, m))
    tt = np.broadcast_to(dec.dst[None, :, None], (C, E, m))
    ii = np.broadcast_to(dec.i_pos[None, None, :], (C, E, m))
    jj = np.broadcast_to(dec.j_pos[None, None, :], (C, E, m))
    np.add.at(F, (cc, ss, ii), dec.beta1[None] * theta)
    np.add.at(F, (cc, tt, jj), dec.beta2[None] * theta)
    return F


def log_softmax(F):
    mx = F.max(axis=-1, keepdims=True)
    return F - (mx + np.log(np.exp(F - mx).sum(axis=-1, keepdims=True)))


def inverse_cdf(logp, u):
    """Smallest a with u < cumsum(p)[a]; else the largest a with p(a) > 0."""
    p = np.exp(logp)
    cdf = np.cumsum(p, axis=-1)
    hit = u[..., None] < cdf
    first = np.argmax(hit, axis=-1)
    L = p.shape[-1]
    last_pos = L - 1 - np.argmax((p > 0)[..., ::-1], axis=-1)
    return np.where(hit.any(axis=-1), first, last_pos), cdf


def site_uniforms(n_vars: int, n_chains: int, sweep: int, seed: int, phase=ph.PH_PRIMAL, site_ids=None):
    v = np.arange(n_vars) if site_ids is None else np.asarray(site_ids, np.int64)
    return ph.site_uniform(v[None, :], np.arange(n_chains)[:, None], sweep, seed, phase)


def primal_step(dec: Decomposition, theta, sweep: int, seed: int, site_ids=None):
    """x ~ p(x | theta): returns labels [C][N], log p [C][N][L], uniforms, cdf.
    site_ids are the RNG indices of the sites (default 0..N-1)."""
    F = primal_field(dec, theta)
    logp = log_softmax(F)
    u = site_uniforms(F.shape[1], F.shape[0], sweep, seed, site_ids=site_ids)
    x, cdf = inverse_cdf(logp, u)
    return x, logp, u, cdf


def sweep(dec: Decomposition, x, sweep_index: int, seed: int, edge_ids=None, site_ids=None):
    """One sweep from labels x: theta | x, then x | theta.  Returns a dict.
    edge_ids / site_ids: RNG indices of the edges / sites (a sub-model of a
    larger one draws what the larger model draws for the same edges / sites)."""
    theta, p_dual, u_dual = dual_step(dec, x, sweep_index, seed, edge_ids)
    x_new, logp, u_site, cdf = primal_step(dec, theta, sweep_index, seed, site_ids)
    return dict(x=x_new, theta=theta, p_dual=p_dual, u_dual=u_dual, logp=logp, u_site=u_site, cdf=cdf)


def run(dec: Decomposition, n_chains: int, n_sweeps: int, seed: int, burn_in: int = 0, x0=None):
    """Run the chain from the contract's initial labels; returns final labels
    and label counts [N][L] summed over chains for sweeps >= burn_in."""
    N, L = dec.utilde.shape
    x = ph.init_labels(N, L, n_chains, seed) if x0 is None else np.asarray(x0, np.int64)
    counts = np.zeros((N, L), np.int64)
    for t in range(n_sweeps):
        x = sweep(dec, x, t, seed)["x"]
        if t >= burn_in:
            np.add.at(counts, (np.broadcast_to(np.arange(N), x.shape), x), 1)
    return x, counts


def boundary_draws(p_dual, u_dual, cdf, u_site, eps=1e-6):
    """Masks of draws whose uniform lies within eps of a decision boundary."""
    dual_b = np.abs(u_dual - p_dual) < eps
    site_b = np.any(np.abs(u_site[..., None] - cdf) < eps, axis=-1)
    return dual_b, site_b
