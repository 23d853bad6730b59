"""Pins of the oracle's Philox4x32-10 (statistical and structural; the bit-level
pin against CUDA's curand implementation runs on the GPU) and of the
diagnostics (ESS of an AR(1) process, PSRF)."""
import numpy as np

from oracle import philox as ph, diagnostics as dg


def test_philox_uniform_chi_square():
    n = 1 << 20
    c = np.arange(n // 4, dtype=np.uint64)
    w = np.concatenate(ph.philox4x32_10(c, 7, 3, 5 << 24, 0x12345678, 0x9ABCDEF0))
    bins = np.bincount((w >> np.uint32(24)).astype(np.int64), minlength=256)
    chi2 = ((bins - n / 256) ** 2 / (n / 256)).sum()
    assert 160 < chi2 < 360          # 255 dof: mean 255, sd 22.6
    bits = np.unpackbits(w.view(np.uint8)).mean()
    assert abs(bits - 0.5) < 5 * 0.5 / np.sqrt(32 * n)


def test_philox_counter_and_key_sensitivity():
    base = np.stack(ph.philox4x32_10(np.arange(4096), 0, 0, 0, 1, 2), -1)
    assert np.unique(base.view(np.uint8).reshape(4096, 16), axis=0).shape[0] == 4096
    for args in [(np.arange(4096), 1, 0, 0, 1, 2), (np.arange(4096), 0, 1, 0, 1, 2),
                 (np.arange(4096), 0, 0, 1, 1, 2), (np.arange(4096), 0, 0, 0, 2, 2),
                 (np.arange(4096), 0, 0, 0, 1, 3)]:
        other = np.stack(ph.philox4x32_10(*args), -1)
        flips = np.unpackbits((base ^ other).view(np.uint8)).mean()
        assert abs(flips - 0.5) < 0.01       # avalanche: half the output bits change


def test_uniform_mappings_are_exact():
    U = np.array([0, 1, 12345, (1 << 23) - 1, 1 << 23, (1 << 24) - 1])
    u = ph.u24_to_unit(U)
    assert np.all(u * 16777216.0 - 0.5 == U)        # exact in float64
    assert u[0] > 0 and u[-1] < 1
    V = np.array([0, 1, 777, (1 << 22), (1 << 23) - 1])
    v = ph.u23_to_unit(V)
    assert np.all(v.astype(np.float32).astype(np.float64) == v)   # exact in float32
    assert np.all(v * 8388608.0 - 0.5 == V)


def test_dual_prefix_planes_uniform_and_independent_of_position():
    pre = ph.dual_prefix(np.arange(4000)[:, None], np.arange(64)[None, :], 2, 9, 5)
    assert pre.min() >= 0 and pre.max() <= 255
    h = np.bincount(pre.ravel(), minlength=256)
    chi2 = ((h - pre.size / 256) ** 2 / (pre.size / 256)).sum()
    assert 160 < chi2 < 360
    # entries of the same group share Philox calls but use different bits
    c = np.corrcoef(pre[:, 0], pre[:, 1])[0, 1]
    assert abs(c) < 0.05


def test_packed_dual_prefix_for_small_tables():
    """m <= 16: the eight planes of all entries come from one Philox call, two
    planes per word (entry k at bit 16 (p div 4) + k of word p mod 4)."""
    for m in (1, 4, 9, 16):
        pre = ph.dual_prefix(np.arange(4000)[:, None], np.arange(m)[None, :], 1, 7, 3, m=m)
        assert pre.min() >= 0 and pre.max() <= 255
        h = np.bincount(pre.ravel(), minlength=256)
        chi2 = ((h - pre.size / 256) ** 2 / (pre.size / 256)).sum()
        assert 160 < chi2 < 360 + 2 * (16 - m)
        if m > 1:
            assert abs(np.corrcoef(pre[:, 0], pre[:, m - 1])[0, 1]) < 0.05
    # the words: prefix bit 7 - p of entry k is bit 16 (p div 4) + k of word p mod 4
    w = ph._words(np.array([5]), 2, np.array([1]), ph.PH_DUAL << 24, 9)[0]
    pre = ph.dual_prefix(5, np.arange(16), 1, 2, 9, m=16)
    for k in range(16):
        want = sum((((int(w[p % 4]) >> (16 * (p // 4) + k)) & 1) << (7 - p)) for p in range(8))
        assert pre[k] == want
    # tables with more entries keep the 32-entry groups
    assert np.array_equal(ph.dual_prefix(5, np.arange(17), 1, 2, 9, m=17), ph.dual_prefix(5, np.arange(17), 1, 2, 9))


def test_dual_uniform_prefix_and_low_bits_independent_streams():
    u = ph.dual_u24(np.arange(2000)[:, None], np.arange(49)[None, :], 0, 3, 11)
    pre = u >> 16; low = u & 0xFFFF
    assert abs(pre.mean() - 127.5) < 2 and abs(low.mean() - 32767.5) < 300
    assert abs(np.corrcoef(pre.ravel(), low.ravel())[0, 1]) < 0.01


def test_init_labels_uniform():
    x = ph.init_labels(10000, 3, 4, seed=1)
    f = np.bincount(x.ravel(), minlength=3) / x.size
    assert np.all(np.abs(f - 1 / 3) < 0.01) and x.max() == 2


def test_ess_ar1_closed_form():
    rng = np.random.default_rng(0)
    rho, n, reps = 0.9, 20000, 8
    tau = (1 + rho) / (1 - rho)               # integrated autocorrelation time of AR(1)
    ess = []
    for r in range(reps):
        e = rng.normal(size=n); x = np.zeros(n)
        for t in range(1, n):
            x[t] = rho * x[t - 1] + e[t]
        ess.append(dg.ess_geyer(x))
    assert abs(np.mean(ess) / (n / tau) - 1) < 0.15
    iid = dg.ess_geyer(rng.normal(size=n))
    assert 0.8 * n < iid < 1.25 * n


def test_psrf():
    rng = np.random.default_rng(1)
    assert abs(dg.psrf(rng.normal(size=(10, 5000))) - 1) < 0.01
    shifted = rng.normal(size=(10, 5000)) + np.arange(10)[:, None]
    assert dg.psrf(shifted) > 2
    assert dg.mixing_time([1.5, 1.2, 1.005, 1.02, 1.004, 1.003]) == 4


def test_tv():
    assert dg.tv_mean([[0.5, 0.5]], [[1.0, 0.0]]) == 0.5
