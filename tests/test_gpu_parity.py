"""GPU parity of the plain and fused sweeps (Sections 4.1-4.2 and 5.1) against
the CPU oracle, through the C ABI.  Sizes span many CTAs with ragged tails;
shapes follow the measured workloads (2-D Ising L=2, 3-D Potts L=8 with 64
chains, dense L=4 with 16 chains, Potts-diagonal L=4, random L=16)."""
import ctypes as ct
import os
import subprocess
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import brute, decompose as dc, sampler, philox as ph
from paper_1611_06684_gb300 import workloads as wl
from paper_1611_06684_gb300 import mrf as M
from tests.gpu_helpers import make_handle, compare_sweep, expected_threshold_words

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_06684_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _no_edges():
    rng = np.random.default_rng(21)
    return wl.Model(n_vars=37, n_labels=3, unary=rng.normal(size=(37, 3)).astype(np.float32),
                    src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32), pair=np.zeros((0, 3, 3), np.float32),
                    name="no_edges")


def _constant_tables():
    m = wl.random_graph(60, k=2, L=3, seed=22)
    m.pair[:] = 0.0                      # every entry l = 0: no dual variable at all
    return m


def _isolated_sites():
    return wl.tiny_random(80, 4, 30, seed=23)          # most sites have no edge


def _star(n_leaves=700, L=3, seed=24):
    rng = np.random.default_rng(seed)
    src = np.zeros(n_leaves, np.int32)
    dst = np.arange(1, n_leaves + 1, dtype=np.int32)
    return wl.Model(n_vars=n_leaves + 1, n_labels=L, unary=rng.normal(size=(n_leaves + 1, L)).astype(np.float32),
                    src=src, dst=dst, pair=rng.normal(0, 0.3, size=(n_leaves, L, L)).astype(np.float32), name="star")


CASES = {
    "ising32": (lambda: wl.ising_grid(32, 32, seed=0), 1),
    "potts3d_L8": (lambda: wl.potts_grid3d(13, 11, 9, L=8, seed=1), 64),
    "dense_L4": (lambda: wl.dense_potts(150, L=4, seed=2), 16),
    "pottsdiag_L4": (lambda: wl.tiny_potts(300, 4, 1500, seed=3), 32),
    "random_L16": (lambda: wl.random_graph(200, k=2, L=16, seed=4, w_std=0.3), 3),
    "random_L3_dup": (lambda: wl.tiny_random(40, 3, 120, seed=5, allow_duplicates=True), 5),
    # chains a multiple of 32 (warp-per-site primal): degree > 32 (two-sum flush), and L = 16
    "dense_L4_C32": (lambda: wl.dense_potts(120, L=4, seed=8), 32),
    "random_L16_C32": (lambda: wl.random_graph(60, k=2, L=16, seed=9, w_std=0.3), 32),
    # degenerate models
    "no_edges": (_no_edges, 4),
    "constant_tables": (_constant_tables, 32),
    "isolated_sites": (_isolated_sites, 7),
    "potts_L16_diag": (lambda: wl.tiny_potts(40, 16, 90, seed=25), 32),
    # few chains and more than 16 entries per edge (edge-partial plain sweep): degree > 32 too
    "random_L12_C1": (lambda: wl.random_graph(300, k=3, L=12, seed=31, w_std=0.3), 1),
    "random_L14_C4": (lambda: wl.random_graph(150, k=4, L=14, seed=32, w_std=0.3), 4),
    "star_degree700": (_star, 32),
}


@pytest.mark.parametrize("name", ["star_degree700", "dense_L4_C32", "random_L3_dup"])
def test_cta_schedule_matches_oracle(name):
    model, C = CASES[name][0](), CASES[name][1]
    seed, t = 77, 5
    dec = dc.decompose(model)
    x0 = np.random.default_rng(12).integers(0, model.n_labels, size=(C, model.n_vars))
    h = make_handle(model, C, seed, record_logp=True, schedule=2)
    h.set_labels(x0.astype(np.uint8))
    h.set_sweep_index(t)
    h.sweep(1, M.MODE_PLAIN)
    assert h.info().schedule == 2
    lp, _ = h.debug_logp()
    ref = sampler.sweep(dec, x0, t, seed)
    compare_sweep(dec, ref, h.get_labels(), lp, M.unpack_theta(h.debug_theta(), dec.n_entries))
    h.close()


def test_edges_times_chains_limit():
    # E x C must stay below 2^32 (item indices are 32-bit): 4096 edges x 2^20 chains is refused
    model = wl.tiny_random(10, 2, 4096, seed=26, allow_duplicates=True)
    h = M.MRF(10, 2, 1 << 20, seed=0)
    with pytest.raises(M.MrfError) as e:
        h.set_factors(model.unary, model.src, model.dst, model.pair)
    assert e.value.status == M.MRF_ERANGE
    h.close()


@pytest.mark.parametrize("name", list(CASES))
def test_decomposition_tables(name):
    model, C = CASES[name][0](), CASES[name][1]
    dec = dc.decompose(model)
    h = make_handle(model, C, seed=7)
    inf = h.info()
    assert inf.layout == dec.layout and inf.n_entries == dec.n_entries
    tau, thr, ut = h.debug_tables()
    np.testing.assert_allclose(tau, np.where(dec.active, dec.beta1, 0).astype(np.float32), rtol=2e-7, atol=0)
    want, near = expected_threshold_words(dec)
    assert np.array_equal(thr[~near], want[~near])
    np.testing.assert_allclose(ut, dec.utilde, rtol=1e-12, atol=1e-12)
    assert abs(inf.log_const - dec.log_const) <= 1e-9 * max(1.0, abs(dec.log_const))
    h.close()


def test_initial_labels_follow_contract():
    model = wl.potts_grid3d(7, 5, 3, L=5, seed=0)
    h = make_handle(model, 33, seed=99)
    assert np.array_equal(h.get_labels(), ph.init_labels(model.n_vars, 5, 33, 99))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("mode", [M.MODE_PLAIN, M.MODE_FUSED])
def test_one_sweep_matches_oracle(name, mode):
    model, C = CASES[name][0](), CASES[name][1]
    seed, t = 2024, 17
    dec = dc.decompose(model)
    rng = np.random.default_rng(11)
    x0 = rng.integers(0, model.n_labels, size=(C, model.n_vars))
    h = make_handle(model, C, seed, record_logp=True, use_graphs=(mode == M.MODE_FUSED))
    h.set_labels(x0.astype(np.uint8))
    h.set_sweep_index(t)
    h.sweep(1, mode)
    lp, _ = h.debug_logp()
    theta = M.unpack_theta(h.debug_theta(), dec.n_entries) if mode == M.MODE_PLAIN else None
    ref = sampler.sweep(dec, x0, t, seed)
    stats = compare_sweep(dec, ref, h.get_labels(), lp, theta)
    print(name, mode, stats)
    assert h.info().sweep_index == t + 1
    h.close()


def test_edge_partial_form_at_high_degree_matches_oracle():
    """The edge-partial plain sweep (few chains, > 16 entries per edge) on a
    fully connected model: 79 incidences per site, so the partial fields go
    through the two-sum flush; dual bits, log p and labels against the oracle.
    (The fused form keeps one running sum over ~4,000 weights per site here, so
    its float32 log p may drift past 1e-5: only the plain form is checked.)"""
    model, C = wl.dense_potts(80, L=12, seed=33), 2
    seed, t = 2024, 17
    dec = dc.decompose(model)
    x0 = np.random.default_rng(11).integers(0, model.n_labels, size=(C, model.n_vars))
    h = make_handle(model, C, seed, record_logp=True, kernel_timing=True)
    h.set_labels(x0.astype(np.uint8))
    h.set_sweep_index(t)
    h.sweep(1, M.MODE_PLAIN)
    lp, _ = h.debug_logp()
    ref = sampler.sweep(dec, x0, t, seed)
    print(compare_sweep(dec, ref, h.get_labels(), lp, M.unpack_theta(h.debug_theta(), dec.n_entries)))
    h.close()


def test_plain_and_fused_agree_exactly():
    model = wl.potts_grid3d(9, 8, 7, L=8, seed=6)
    outs = []
    for mode in (M.MODE_PLAIN, M.MODE_FUSED):
        h = make_handle(model, 64, seed=5)
        h.sweep(6, mode)
        outs.append(h.get_labels())
        h.close()
    assert np.array_equal(outs[0], outs[1])


def test_trajectory_until_first_boundary():
    model = wl.ising_grid(32, 32, seed=0)
    dec = dc.decompose(model)
    seed, C = 0, 1
    h = make_handle(model, C, seed)
    x = ph.init_labels(model.n_vars, 2, C, seed)
    steps = 0
    for t in range(200):
        ref = sampler.sweep(dec, x, t, seed)
        h.sweep(1, M.MODE_PLAIN)
        dual_b, site_b = sampler.boundary_draws(ref["p_dual"], ref["u_dual"], ref["cdf"], ref["u_site"])
        if dual_b.any() or site_b.any():
            break
        assert np.array_equal(h.get_labels(), ref["x"]), f"diverged at sweep {t}"
        x = ref["x"]
        steps += 1
    print("identical sweeps before first boundary draw:", steps)
    assert steps >= 50


def test_counts_and_marginals_accumulate():
    model = wl.tiny_random(6, 3, 8, seed=3)
    dec = dc.decompose(model)
    seed, C, T, burn = 3, 7, 12, 4
    h = make_handle(model, C, seed)
    h.reset_marginals(burn)
    h.sweep(T, M.MODE_PLAIN)
    x, counts = sampler.run(dec, C, T, seed, burn_in=burn)
    got = h.counts()
    # identical unless a boundary draw happened along the way (not expected at this size)
    assert np.array_equal(got, counts)
    m, ns = h.marginals()
    assert ns == (T - burn) * C
    np.testing.assert_allclose(m, counts / ns, rtol=1e-6)


def test_marginals_within_3_sigma_of_exact():
    model = wl.tiny_random(9, 3, 14, seed=21, w_std=0.7)
    exact, _ = brute.exact_marginals(model)
    C, T, burn = 4096, 150, 30
    h = make_handle(model, C, seed=8)
    acc = np.zeros((C, model.n_vars, 3))
    for t in range(T):
        h.sweep(1, M.MODE_PLAIN)
        if t >= burn:
            x = h.get_labels()
            acc[np.arange(C)[:, None], np.arange(model.n_vars)[None, :], x] += 1
    cm = acc / (T - burn)
    est, sig = cm.mean(0), cm.std(0, ddof=1) / np.sqrt(C)
    z = np.abs(est - exact) / np.maximum(sig, 1e-12)
    assert z.max() < 4.0 and np.mean(z < 3.0) > 0.95, z.max()


def test_resume_is_bit_exact():
    model = wl.potts_grid3d(8, 6, 5, L=4, seed=2)
    a = make_handle(model, 16, seed=4)
    a.sweep(10, M.MODE_PLAIN)
    b = make_handle(model, 16, seed=4)
    b.sweep(5, M.MODE_PLAIN)
    x_mid = b.get_labels()
    c = make_handle(model, 16, seed=4)
    c.set_labels(x_mid)
    c.set_sweep_index(5)
    c.sweep(5, M.MODE_FUSED)
    assert np.array_equal(a.get_labels(), c.get_labels())


def test_edits_follow_slot_rule_and_match_oracle():
    model = wl.er_graph(wl.ErGraphSpec(300, 4, 6.0, 17))
    C, seed = 4, 12
    h = make_handle(model, C, seed)
    rng = np.random.default_rng(0)
    rem, s, t, p = wl.er_edit(model, 0.05, rng)
    ids = h.edit_factors(rem, s, t, p)
    # rule: freed slots in increasing order, then fresh slots
    assert np.array_equal(ids[:len(rem)], np.sort(rem)[:len(ids)])
    E = model.n_edges
    keep = np.ones(E, bool); keep[rem] = False
    src = model.src.copy(); dst = model.dst.copy(); pair = model.pair.copy()
    src[ids] = s; dst[ids] = t; pair[ids] = p
    edited = wl.Model(model.n_vars, 4, model.unary, src, dst, pair)
    dec = dc.decompose(edited)
    assert h.info().n_edges == E
    x0 = h.get_labels().astype(np.int64)
    h.set_sweep_index(3)
    h.sweep(1, M.MODE_PLAIN)
    ref = sampler.sweep(dec, x0, 3, seed)
    compare_sweep(dec, ref, h.get_labels())


def test_error_statuses():
    model = wl.tiny_random(5, 3, 4, seed=1)
    h = M.MRF(5, 3, 2, seed=0)
    bad = model.pair.copy(); bad[1, 2, 0] = np.nan
    with pytest.raises(M.MrfError) as e:
        h.set_factors(model.unary, model.src, model.dst, bad)
    assert e.value.status == M.MRF_ENONFINITE
    loop = model.dst.copy(); loop[0] = model.src[0]
    with pytest.raises(M.MrfError) as e:
        h.set_factors(model.unary, model.src, loop, model.pair)
    assert e.value.status == M.MRF_ERANGE
    with pytest.raises(M.MrfError) as e:
        h.sweep(1, M.MODE_PLAIN)
    assert e.value.status == M.MRF_ESTATE
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    with pytest.raises(M.MrfError) as e:
        h.sweep(1, M.MODE_SPLASH)
    assert e.value.status == M.MRF_ESTATE
    with pytest.raises(M.MrfError) as e:
        h.edit_factors([99], [], [], np.zeros((0, 3, 3), np.float32))
    assert e.value.status == M.MRF_ERANGE


def test_device_pointer_inputs():
    torch = pytest.importorskip("torch")
    model = wl.potts_grid3d(6, 6, 6, L=4, seed=9)
    h1 = make_handle(model, 8, seed=1)
    h2 = M.MRF(model.n_vars, 4, 8, seed=1)
    h2.set_factors(*(torch.from_numpy(a).cuda() for a in (model.unary, model.src, model.dst, model.pair)))
    a, b = h1.debug_tables(), h2.debug_tables()
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_philox_matches_curand_and_oracle():
    """Bit-level pin of the Philox4x32-10 implementations against CUDA's
    curand_Philox4x32_10 (an independent implementation of the same
    definition): the oracle's, the device's with the key schedule, the one with
    precomputed round keys (the hot path's) and the dual step's four calls
    sharing their first rounds (draw_rk_subs)."""
    with tempfile.TemporaryDirectory() as d:
        so = os.path.join(d, "philox_check.so")
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                        "-cudart=shared", os.path.join(ROOT, "tests", "cuda", "philox_check.cu"), "-o", so], check=True)
        lib = ct.CDLL(so)
        rng = np.random.default_rng(5)
        n = 1 << 16
        ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
        ctr[:16] = 0; ctr[16:32, 0] = np.arange(16)
        for k0, k1 in [(0, 0), (0xDEADBEEF, 0x12345678), (2**32 - 1, 1)]:
            mine = np.zeros((n, 4), np.uint32); ref = np.zeros((n, 4), np.uint32)
            assert lib.philox_pair(ctr.ctypes.data_as(ct.c_void_p), ct.c_uint32(k0), ct.c_uint32(k1),
                                   mine.ctypes.data_as(ct.c_void_p), ref.ctypes.data_as(ct.c_void_p), n) == 0
            assert np.array_equal(mine, ref)
            orc = np.stack(ph.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], k0, k1), -1)
            assert np.array_equal(orc, ref)
            mine = np.zeros((n, 4), np.uint32); ref = np.zeros((n, 4), np.uint32)
            assert lib.philox_rk_pair(ctr.ctypes.data_as(ct.c_void_p), ct.c_uint32(k0), ct.c_uint32(k1),
                                      mine.ctypes.data_as(ct.c_void_p), ref.ctypes.data_as(ct.c_void_p), n) == 0
            assert np.array_equal(mine, ref)
            mine = np.zeros((n, 4, 4), np.uint32); ref = np.zeros((n, 4, 4), np.uint32)
            assert lib.philox_subs_pair(ctr.ctypes.data_as(ct.c_void_p), ct.c_uint32(k0), ct.c_uint32(k1),
                                        mine.ctypes.data_as(ct.c_void_p), ref.ctypes.data_as(ct.c_void_p), n) == 0
            assert np.array_equal(mine, ref)


@pytest.mark.parametrize("name", ["ising32", "random_L3_dup", "potts_L16_diag", "star_degree700", "random_L16_C32"])
def test_small_model_single_launch_equals_sweep_by_sweep(name):
    """Several sweeps of a small model run in one single-CTA launch; the chain
    (labels, counts, boundary count) is the same as one sweep at a time."""
    model, C = CASES[name][0](), CASES[name][1]
    out = []
    for one_at_a_time in (False, True):
        h = make_handle(model, C, seed=31, kernel_timing=True)
        h.reset_marginals(2)
        if one_at_a_time:
            for _ in range(9):
                h.sweep(1, M.MODE_PLAIN)
        else:
            h.sweep(9, M.MODE_PLAIN)
        kt = h.kernel_times()
        assert ("k_sweep_small" in kt) == (not one_at_a_time)
        out.append((h.get_labels(), h.counts(), h.info().sweep_index))
        h.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] == 9
