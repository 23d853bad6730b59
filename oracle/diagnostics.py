"""Mixing and accuracy diagnostics (float64, numpy).

* tv_mean: mean over sites of the total-variation distance
  1/2 sum_a |p^_v(a) - p_v(a)| between estimated and reference marginals.
* ess_geyer: effective sample size of one scalar trace by Geyer's
  initial-monotone-sequence estimator (Geyer 1992): autocovariances are
  summed in adjacent pairs Gamma_k = g(2k) + g(2k+1) while positive, with the
  pair sums forced to be non-increasing; tau = -1 + 2 sum_k Gamma_k.
* psrf: the Gelman-Rubin potential scale reduction factor over chains
  (Section 6 uses 10 chains and the first index after which PSRF < 1.01).

Parity: ESS pinned by an AR(1) trace whose integrated autocorrelation time
is known in closed form; PSRF by i.i.d. chains (-> 1) and shifted chains (> 1).
"""
from __future__ import annotations

import numpy as np


def tv_mean(p_hat, p_ref):
    return float(0.5 * np.abs(np.asarray(p_hat) - np.asarray(p_ref)).sum(axis=-1).mean())


def autocovariance(x):
    x = np.asarray(x, np.float64) - np.mean(x)
    n = x.shape[0]
    f = np.fft.rfft(x, n=2 * n)
    acov = np.fft.irfft(f * np.conj(f), n=2 * n)[:n] / n
    return acov


def ess_geyer(x):
    x = np.asarray(x, np.float64)
    n = x.shape[0]
    if n < 4:
        return float(n)
    g = autocovariance(x)
    if g[0] <= 0:
        return float(n)
    pairs = []
    for k in range(n // 2):
        s = g[2 * k] + g[2 * k + 1]
        if s <= 0:
            break
        pairs.append(s)
    if not pairs:
        return float(n)
    pairs = np.minimum.accumulate(np.array(pairs))
    tau = -1.0 + 2.0 * pairs.sum() / g[0]
    return float(n / max(tau, 1e-12))


def psrf(chains):
    """chains [M][n] of one scalar statistic."""
    c = np.asarray(chains, np.float64)
    M, n = c.shape
    means = c.mean(axis=1)
    W = c.var(axis=1, ddof=1).mean()
    B = n * means.var(ddof=1)
    if W <= 0:
        return 1.0 if B <= 0 else float("inf")
    var_hat = (n - 1) / n * W + B / n
    return float(np.sqrt(var_hat / W))


def mixing_time(psrf_trace, threshold=1.01):
    """First index after which the PSRF trace stays below threshold (len if never)."""
    t = np.asarray(psrf_trace)
    above = np.nonzero(t >= threshold)[0]
    return int(above[-1] + 1) if above.size else 0
