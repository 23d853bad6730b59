"""Host-side statistics of bench.py (ESS, TV) against closed forms."""
import numpy as np

import bench


def _ar1(phi, T, C, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((T, C))
    x[0] = rng.normal(size=C) / np.sqrt(1 - phi ** 2)
    for t in range(1, T):
        x[t] = phi * x[t - 1] + rng.normal(size=C)
    return x


def test_ess_ar1_closed_form():
    # AR(1): integrated autocorrelation time (1 + phi) / (1 - phi)
    for phi in (0.0, 0.5, 0.9):
        T, C = 4000, 16
        ess = bench.ess_sum_over_chains(_ar1(phi, T, C, seed=1))
        exact = T * C * (1 - phi) / (1 + phi)
        assert abs(ess / exact - 1) < 0.2, (phi, ess, exact)


def test_ess_constant_and_short():
    assert bench.ess_sum_over_chains(np.ones((50, 3))) == 150.0


def test_tv_mean():
    p = np.array([[0.5, 0.5], [1.0, 0.0]])
    q = np.array([[0.25, 0.75], [0.0, 1.0]])
    assert bench.tv_mean(p, q) == 0.5 * (0.25 + 1.0)
