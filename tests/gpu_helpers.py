"""Shared helpers of the GPU parity tests: run the library through the C ABI
and compare with the oracle under the tolerances of the parity protocol:
  * dual bits and labels identical except draws whose uniform lies within
    1e-6 of the decision boundary (counted and reported);
  * conditional log-probabilities |lp_gpu - lp_oracle| <= 1e-5 max(1, |lp|).
"""
from __future__ import annotations

import numpy as np

from oracle import decompose as dc, sampler, philox as ph
from paper_1611_06684_gb300 import mrf as M

LOGP_RTOL = 1e-5
BOUNDARY_EPS = 1e-6


def make_handle(model, C, seed, **kw):
    h = M.MRF(model.n_vars, model.n_labels, C, seed=seed, **kw)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    return h


def affected_sites(dec, mismatch):
    """[C][N] mask of sites incident to an edge whose dual bits differ."""
    C = mismatch.shape[0]
    N = dec.utilde.shape[0]
    out = np.zeros((C, N), bool)
    c, e = np.nonzero(mismatch.any(axis=2))
    out[c, dec.src[e]] = True
    out[c, dec.dst[e]] = True
    return out


def compare_sweep(dec, ref, x_gpu, lp_gpu=None, theta_gpu=None, tree=None):
    """Check one sweep against the oracle; returns a dict of counts."""
    dual_b, site_b = sampler.boundary_draws(ref["p_dual"], ref["u_dual"], ref["cdf"], ref["u_site"], BOUNDARY_EPS)
    stats = dict(dual_boundary=int((dual_b & dec.active[None]).sum()), site_boundary=int(site_b.sum()))
    affected = np.zeros(x_gpu.shape, bool)
    if theta_gpu is None:
        # duals not compared: a boundary dual draw may flip a bit, so its endpoints are exempt
        affected = affected_sites(dec, dual_b & dec.active[None])
    else:
        mism = theta_gpu != ref["theta"]
        if tree is not None:
            mism &= ~tree[None, :, None]
        assert not (mism & ~dual_b).any(), f"{int((mism & ~dual_b).sum())} dual bits differ away from boundaries"
        stats["dual_mismatch"] = int(mism.sum())
        affected = affected_sites(dec, mism)
    if lp_gpu is not None:
        lr = ref["logp"]
        err = np.abs(lp_gpu - lr) / np.maximum(1.0, np.abs(lr))
        err[affected] = 0
        stats["logp_max_rel"] = float(err.max())
        assert err.max() <= LOGP_RTOL, f"log p differs: max rel {err.max():.3g}"
    bad = (x_gpu != ref["x"]) & ~site_b & ~affected
    if bad.any():
        c, v = np.nonzero(bad)
        detail = [(int(c[i]), int(v[i]), int(x_gpu[c[i], v[i]]), int(ref["x"][c[i], v[i]]),
                   float(ref["u_site"][c[i], v[i]]), ref["cdf"][c[i], v[i]].round(7).tolist()) for i in range(min(4, len(c)))]
        raise AssertionError(f"{int(bad.sum())} labels differ away from CDF boundaries: {detail}")
    stats["label_mismatch"] = int((x_gpu != ref["x"]).sum())
    return stats


def expected_threshold_words(dec):
    """Packed threshold words from the oracle's float64 decomposition: T+ from
    sigmoid(+tau), T- from sigmoid(-tau), d = T+ + T- - (2^24 - 1), sign bit."""
    tau = np.abs(dec.beta2)
    pp = 1.0 / (1.0 + np.exp(-tau))
    pm = 1.0 / (1.0 + np.exp(tau))
    tp = np.ceil(pp * 16777216.0 - 0.5).astype(np.int64)
    tm = np.ceil(pm * 16777216.0 - 0.5).astype(np.int64)
    d = tp + tm - ((1 << 24) - 1)
    word = (tp | (d << 25) | np.where(dec.ell < 0, 1 << 31, 0)).astype(np.uint64)
    word = np.where(dec.active, word, 0).astype(np.uint32)
    near = np.minimum(np.abs(pp * 16777216.0 - 0.5 - np.round(pp * 16777216.0 - 0.5)),
                      np.abs(pm * 16777216.0 - 0.5 - np.round(pm * 16777216.0 - 0.5))) < 1e-6
    return word, near & dec.active
