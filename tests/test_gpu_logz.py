"""GPU parity of the log-partition estimator (Section 5.2): log V of one sweep
per chain against the oracle, and the estimator's moments against exact
enumeration on a tiny model."""
import numpy as np
import pytest

from oracle import brute, decompose as dc, logz, sampler
from paper_1611_06684_gb300 import workloads as wl
from gpu_helpers import BOUNDARY_EPS, LOGP_RTOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_06684_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("C,schedule", [(16, 0), (32, 0), (32, 2)])
def test_log_v_of_one_sweep_matches_oracle(C, schedule):
    from paper_1611_06684_gb300 import mrf as M
    model = wl.potts_grid3d(7, 6, 5, L=4, seed=3)
    dec = dc.decompose(model)
    seed, t = 17, 11
    x0 = np.random.default_rng(4).integers(0, 4, size=(C, model.n_vars))
    h = M.MRF(model.n_vars, 4, C, seed=seed, grid=model.grid, schedule=schedule)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    h.set_labels(x0.astype(np.uint8))
    h.set_sweep_index(t)
    lv = h.estimate_log_partition(1)[0]
    x1 = h.get_labels()
    assert h.info().sweep_index == t + 1
    h.close()
    ref, r = logz.sweep_log_v(model, dec, x0, t, seed)
    dual_b, site_b = sampler.boundary_draws(r["p_dual"], r["u_dual"], r["cdf"], r["u_site"], BOUNDARY_EPS)
    clean = (x1 == r["x"]).all(axis=1) & ~(dual_b & dec.active[None]).any(axis=(1, 2)) & ~site_b.any(axis=1)
    assert clean.sum() >= C // 2
    lp = np.take_along_axis(r["logp"], r["x"][:, :, None], axis=2)[:, :, 0]
    tol = LOGP_RTOL * np.maximum(1.0, np.abs(lp)).sum(axis=1)        # the per-site tolerance, summed
    err = np.abs(lv - ref)
    assert (err[clean] <= tol[clean]).all(), (err[clean].max(), tol[clean].min())


def test_estimator_moments_match_enumeration():
    """Many chains of a tiny model at stationarity: the mean of log V matches
    the exact E[log V] and log mean V matches the exact log Z."""
    from paper_1611_06684_gb300 import mrf as M
    model = wl.tiny_potts(5, 3, 6, seed=4, beta_max=0.8)
    dec = dc.decompose(model)
    log_ev, e_logv, mi = logz.exact_moments(model, dec)
    _, _, logZ = brute.exact_distribution(model)
    C = 8192
    h = M.MRF(model.n_vars, 3, C, seed=5, exact_edges=True)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    h.sweep(30, M.MODE_PLAIN)
    lv = h.estimate_log_partition(16).ravel()
    h.close()
    n_eff = lv.size / 4                                               # consecutive sweeps are correlated
    se_mean = lv.std() / np.sqrt(n_eff)
    assert abs(lv.mean() - e_logv) < 4 * se_mean + 1e-6, (lv.mean(), e_logv, se_mean)
    w = np.exp(lv - lv.max())
    est = lv.max() + np.log(w.mean())
    se_log = w.std() / w.mean() / np.sqrt(n_eff)
    assert abs(est - logZ) < 4 * se_log + 1e-6, (est, logZ, se_log)
    assert e_logv < logZ and abs(logZ - e_logv - mi) < 1e-9
