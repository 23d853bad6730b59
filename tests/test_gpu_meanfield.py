"""GPU parity of the primal-dual EM (local MAP) and mean field of Section 5.3."""
import numpy as np
import pytest

from oracle import brute, decompose as dc, meanfield as mf
from paper_1611_06684_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_06684_gb300 import build
    build.build()
    torch.cuda.set_device(0)


CASES = {
    "potts3d_L8": (lambda: wl.potts_grid3d(9, 8, 7, L=8, seed=1), 32),
    "potts_diag_L4": (lambda: wl.tiny_potts(300, 4, 1200, seed=2), 3),
    "random_L3": (lambda: wl.random_graph(200, k=3, L=3, seed=3), 5),
    "ising": (lambda: wl.ising_grid(20, 20, seed=4), 2),
    "dense_L4": (lambda: wl.dense_potts(90, L=4, seed=5), 32),
}


def _handle(model, C):
    from paper_1611_06684_gb300 import mrf as M
    h = M.MRF(model.n_vars, model.n_labels, C, seed=0)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    return h


def _near_tie(F, rel=1e-4):
    s = np.sort(F, axis=2)
    return (s[:, :, -1] - s[:, :, -2]) < rel * np.maximum(1.0, np.abs(s[:, :, -1]))


@pytest.mark.parametrize("name", list(CASES))
def test_em_iteration_matches_oracle(name):
    model, C = CASES[name][0](), CASES[name][1]
    dec = dc.decompose(model)
    x = np.random.default_rng(1).integers(0, model.n_labels, size=(C, model.n_vars))
    h = _handle(model, C)
    xg = h.map_em(x, 1)
    xr, _, F = mf.em_step(dec, x)
    bad = (xg != xr) & ~_near_tie(F)
    assert not bad.any(), int(bad.sum())
    # several iterations: log p~ never decreases along the GPU's own trajectory
    prev = brute.log_ptilde(model, x)
    xs = x
    for _ in range(6):
        xs = h.map_em(xs, 1)
        cur = brute.log_ptilde(model, xs)
        assert (cur >= prev - 1e-6 * np.maximum(1.0, np.abs(prev))).all()
        prev = cur
    h.close()


@pytest.mark.parametrize("name", list(CASES))
def test_mean_field_matches_oracle(name):
    model, C = CASES[name][0](), CASES[name][1]
    dec = dc.decompose(model)
    q0 = np.random.default_rng(2).dirichlet(np.ones(model.n_labels), size=(C, model.n_vars))
    h = _handle(model, C)
    q1 = h.mean_field(q0.astype(np.float32), 1)
    r1, _, _ = mf.mf_step(dec, q0.astype(np.float32).astype(np.float64))
    assert np.abs(q1 - r1).max() < 1e-5, np.abs(q1 - r1).max()
    # further iterations one at a time from the oracle's state (float32 round
    # trips amplify through an iteration of gain > 1, so trajectories are not
    # compared); the GPU's own 8-iteration result stays normalised
    r = r1
    for _ in range(4):
        qi = h.mean_field(r.astype(np.float32), 1)
        r, _, _ = mf.mf_step(dec, r.astype(np.float32).astype(np.float64))
        assert np.abs(qi - r).max() < 1e-5, np.abs(qi - r).max()
    qn = h.mean_field(q0.astype(np.float32), 8)
    np.testing.assert_allclose(qn.sum(axis=2), 1.0, atol=1e-5)
    assert (qn >= 0).all()
    h.close()


@pytest.mark.parametrize("dims,L,C", [((9, 8, 7), 8, 32), ((10, 9, 5), 4, 3), ((13, 5, 6), 3, 2)])
def test_blocked_em_matches_oracle(dims, L, C):
    from paper_1611_06684_gb300 import mrf as M
    model = wl.potts_grid3d(*dims, L=L, seed=8)
    dec = dc.decompose(model)
    x = np.random.default_rng(5).integers(0, L, size=(C, model.n_vars))
    h = M.MRF(model.n_vars, L, C, seed=13, grid=model.grid)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    prev = brute.log_ptilde(model, x)
    xr = x
    for it in range(3):
        xg = h.map_em_blocked(xr, 1) if it == 0 else None
        xr_next = mf.blocked_em_step(model, dec, xr, it, 13)
        if it == 0:
            # the GPU's first iteration (offset of iteration 0) equals the oracle's
            # away from near-ties of the max-product scores
            assert np.mean(xg != xr_next) < 1e-2, np.mean(xg != xr_next)   # a near-tie at a root flips its subtree
        xr = xr_next
    xg3 = h.map_em_blocked(x, 3)
    assert np.mean(xg3 != xr) < 3e-2
    cur = brute.log_ptilde(model, xg3)
    assert (cur >= prev - 1e-6 * np.abs(prev)).all()
    h.close()


# Tree mean-field marginals: float32 messages along a forest path of at most
# 9 edges (comb tree of a 4x4x4 block), each log-sum-exp off by a few units in
# the last place of log-beliefs of magnitude <= ~20, give log-marginal errors
# of order 9 x 4 x 2^-24 x 20 ~ 4e-5; the bound below leaves a factor 2.5.
MARGINAL_TOL = 1e-4


@pytest.mark.parametrize("dims,L,C", [((9, 8, 7), 8, 32), ((10, 9, 5), 4, 3), ((13, 5, 6), 3, 2), ((5, 4, 3), 16, 4)])
def test_blocked_mean_field_matches_oracle(dims, L, C):
    """Tree mean field (Sections 5.3-5.4): each GPU iteration from the
    oracle's state (float32-rounded) against the oracle's float64 iteration,
    with the forest of the iteration's block offset."""
    from paper_1611_06684_gb300 import mrf as M
    model = wl.potts_grid3d(*dims, L=L, seed=9)
    dec = dc.decompose(model)
    q0 = np.random.default_rng(6).dirichlet(np.ones(L), size=(C, model.n_vars))
    h = M.MRF(model.n_vars, L, C, seed=21, grid=model.grid)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    q1 = h.mean_field_blocked(q0.astype(np.float32), 1)
    r1, _, _ = mf.blocked_mf_step(model, dec, q0.astype(np.float32).astype(np.float64), 0, 21)
    err = np.abs(q1 - r1).max()
    print("iteration 0 max abs error", err)
    assert err < MARGINAL_TOL, err
    # three iterations (offsets of iterations 0, 1, 2) against the oracle's three
    r = q0.astype(np.float32).astype(np.float64)
    for it in range(3):
        r, _, _ = mf.blocked_mf_step(model, dec, r, it, 21)
    q3 = h.mean_field_blocked(q0.astype(np.float32), 3)
    err3 = np.abs(q3 - r).max()
    print("three iterations max abs error", err3)
    assert err3 < 3 * MARGINAL_TOL, err3
    qn = h.mean_field_blocked(q0.astype(np.float32), 6)
    np.testing.assert_allclose(qn.sum(axis=2), 1.0, atol=1e-5)
    assert (qn >= 0).all()
    h.close()


def test_blocked_mean_field_needs_a_lattice_handle():
    from paper_1611_06684_gb300 import mrf as M
    model = wl.random_graph(50, k=2, L=3, seed=3)
    h = M.MRF(model.n_vars, 3, 2, seed=0)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    with pytest.raises(M.MrfError):
        h.mean_field_blocked(np.full((2, 50, 3), 1 / 3, np.float32), 1)
    h.close()
