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

Pins (tests/test_oracle_meanfield.py): EM never decreases log p~(x) (EM on
the latent theta); the mean-field objective KL(q_x q_theta || p(x, theta)),
computed by enumeration, never increases; Lemma 6's inequality
KL(q_x q_theta* || p(x, theta)) >= KL(q_x || p(x)) at every iterate.
"""
from __future__ import annotations

import numpy as np

from . import brute
from .decompose import Decomposition
from .sampler import primal_field, log_softmax, sigmoid


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
