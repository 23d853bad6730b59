"""Estimator of the log-partition function of Section 5.2 (oracle side, float64).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
legs use this package.

Section 5.2 defines, for (x, theta) drawn from the joint p(x, theta),
    V(x, theta) = p~(x) p~(theta) / p~(x, theta),
an unbiased estimator of Z (E[V] = Z), whose logarithm has E[log V] <= log Z
with the gap equal to the mutual information I(x; theta).  Here p~(x) is the
model's unnormalised density exp(sum_v u_v + sum_e w_e) and p~(theta) =
sum_x p~(x, theta), so p~(x, theta) / p~(theta) = p(x | theta) and, with the
primal conditional factorised over sites (Corollary 1),
    log V = log p~(x) - sum_v log p(x_v | theta):
the model's log-potential at the drawn labels minus the log-probabilities of
the sweep's own label draws.  A sweep from a chain at stationarity draws
theta | x and then x' | theta, so (x', theta) is a draw from the joint.

Pins (tests/test_oracle_logz.py): by enumeration on tiny models, log E[V]
equals log Z and log Z - E[log V] equals I(x; theta); log_v agrees with V
computed from Theorem 1's joint (brute.joint_log) for every (x, theta).
"""
from __future__ import annotations

import numpy as np

from . import brute, sampler
from .decompose import Decomposition


def log_v(model, dec: Decomposition, x, theta):
    """log V per chain for labels x [C][N] drawn given duals theta [C][E][m]."""
    x = np.asarray(x, np.int64)
    C, N = x.shape
    logp = sampler.log_softmax(sampler.primal_field(dec, theta))          # [C][N][L]
    lp_cond = np.take_along_axis(logp, x[:, :, None], axis=2)[:, :, 0].sum(axis=1)
    return brute.log_ptilde(model, x) - lp_cond


def sweep_log_v(model, dec: Decomposition, x_old, sweep_index: int, seed: int, edge_ids=None, site_ids=None):
    """One sweep from x_old and log V of its (x', theta); returns (log V [C], sweep dict)."""
    r = sampler.sweep(dec, x_old, sweep_index, seed, edge_ids, site_ids)
    return log_v(model, dec, r["x"], r["theta"]), r


def exact_moments(model, dec: Decomposition):
    """log E[V], E[log V] and I(x; theta) under the exact joint (enumeration)."""
    X = brute.all_labelings(model.n_vars, model.n_labels)
    Th = brute.all_dual_configs(brute.active_entries(dec).shape[0])
    J = brute.joint_log(dec, X, Th)                                      # log p~(x, theta)
    logZj = np.logaddexp.reduce(J, axis=None)
    lp_joint = J - logZj                                                 # log p(x, theta)
    lp_x_given_t = J - np.logaddexp.reduce(J, axis=0)[None, :]           # log p(x | theta)
    lp_x = np.logaddexp.reduce(lp_joint, axis=1)                         # log p(x)
    lp_t = np.logaddexp.reduce(lp_joint, axis=0)                         # log p(theta)
    lv = brute.log_ptilde(model, X)[:, None] - lp_x_given_t              # log V(x, theta)
    pj = np.exp(lp_joint)
    log_ev = np.logaddexp.reduce((lp_joint + lv).ravel())
    e_logv = float((pj * lv).sum())
    mi = float((pj * (lp_joint - lp_x[:, None] - lp_t[None, :])).sum())
    return float(log_ev), e_logv, mi
