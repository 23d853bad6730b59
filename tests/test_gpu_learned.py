"""GPU parity of the learned block proposal: the tensor-core MLP forward and the
training gradients against the float64 oracle, one learned MH sweep against
oracle.learned, exactness of the MH-corrected chain (marginals within 3 sigma
for untrained weights), and the gain training gives (loss and acceptance)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import brute, decompose as dc, learned as ln, sampler
from paper_1611_06684_gb300 import workloads as wl
from paper_1611_06684_gb300 import mrf as M
from tests.gpu_helpers import compare_sweep


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_06684_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _flat(params):
    return np.concatenate([np.asarray(p, np.float64).ravel() for p in params]).astype(np.float32)


def _params(L, hidden, seed, bias_scale=0.1):
    p = ln.init_params(L, hidden=hidden, seed=seed)
    rng = np.random.default_rng(seed + 100)
    for k in (1, 3, 5):
        p[k] = rng.normal(0, bias_scale, p[k].shape).astype(np.float32).astype(np.float64)
    return p


def _setup(model, C, seed, hidden, bos, wseed=5, mlp_path=0):
    h = M.MRF(model.n_vars, model.n_labels, C, seed=seed, exact_edges=True, use_graphs=False, record_logp=False,
              mlp_path=mlp_path)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    h.learned_setup(bos, hidden=hidden, seed=1)
    params = _params(model.n_labels, hidden, wseed)
    h.learned_set_params(_flat(params))
    return h, params


def test_forward_matches_oracle():
    model = wl.ba_potts(2000, m=5, L=4, seed=1)
    bos = wl.bfs_blocks(model, 16, seed=2)
    h, params = _setup(model, 4, 3, 128, bos)
    d, dp = ln.feature_width(4)
    rng = np.random.default_rng(0)
    X = ln.to_bf16(rng.normal(0, 1.0, size=(300, dp)))
    X[:, d:] = 0
    zg = h.learned_forward(X, 64)
    zr = ln.mlp_forward_bf16(params, X)
    err = np.abs(zg - zr) / np.maximum(1.0, np.abs(zr))
    assert err.max() < 1e-2, err.max()
    assert np.median(err) < 1e-4


def test_training_gradients_match_oracle():
    model = wl.ba_potts(1500, m=5, L=4, seed=2)
    bos = wl.bfs_blocks(model, 16, seed=3)
    h, params = _setup(model, 2, 4, 64, bos)
    d, dp = ln.feature_width(4)
    rng = np.random.default_rng(1)
    R = 257
    X = ln.to_bf16(rng.normal(0, 1.0, size=(R, dp))); X[:, d:] = 0
    y = rng.integers(0, 4, size=(R, 16)).astype(np.uint8)
    nmem = rng.integers(1, 17, size=R).astype(np.uint8)
    loss_g, g = h.learned_grad(X, y, nmem)
    loss_r, grads = ln.loss_and_grads(params, X, y.astype(np.int64), nmem.astype(np.int64), 4)
    assert abs(loss_g - loss_r) <= 1e-3 * abs(loss_r)
    off = 0
    for gr in grads:
        n = gr.size
        gg = g[off:off + n].reshape(gr.shape)
        off += n
        assert np.abs(gg - gr).max() <= 1e-2 * max(np.abs(gr).max(), 1e-6)


def _tc_weight_bytes(L, hidden):
    """bf16 bytes of the tensor-core MLP's weight images (first layer padded to 64 columns)."""
    kx = (16 * L + 31) // 32 * 32
    return 2 * (hidden * ((kx + 63) // 64 * 64) + hidden * hidden + 16 * L * hidden)


@pytest.mark.parametrize("L,hidden", [(4, 256), (3, 64), (2, 128), (10, 256), (16, 256)])
def test_tensor_core_mlp_matches_gemm_path(L, hidden):
    """The fused tcgen05 MLP and the three mma.sync GEMMs give the same logits
    from the same features (several 128-row tiles, a partial last tile).  With
    L = 10 and 16 at hidden 256 the weights (311 KB, 393 KB) exceed the 200 KB
    the kernel keeps resident in shared memory, so the streaming tcgen05
    kernel (weights through a two-slot ring) is the one compared."""
    model = wl.ba_potts(1500, m=5, L=L, seed=11)
    bos = wl.bfs_blocks(model, 16, seed=3)
    C, seed, t = 24, 4, 9
    x0 = np.random.default_rng(8).integers(0, L, size=(C, model.n_vars)).astype(np.uint8)
    out = []
    for path in (0, 1):
        h, _ = _setup(model, C, seed, hidden, bos, mlp_path=path)
        h.set_labels(x0)
        h.set_sweep_index(t)
        h.sweep(1, M.MODE_LEARNED)
        nb = int(bos.max()) + 1
        d, dp = ln.feature_width(L)
        out.append(h.learned_debug(nb * C, dp, 16 * L))
        h.close()
    (X0, z0), (X1, z1) = out
    assert np.array_equal(X0, X1)
    assert nb * C > 256
    if L >= 10:
        assert _tc_weight_bytes(L, hidden) > 200 * 1024
    err = np.abs(z0 - z1) / np.maximum(1.0, np.abs(z1))
    assert err.max() < 2e-2, err.max()
    assert np.median(err) < 1e-5, np.median(err)


def test_streaming_tensor_core_mlp_matches_oracle():
    """The streaming tcgen05 MLP (L = 12, hidden 256: 352 KB of weights) against
    the float64 oracle with bf16 activations, from the GPU's own features."""
    L, hidden = 12, 256
    assert _tc_weight_bytes(L, hidden) > 200 * 1024
    model = wl.ba_potts(1200, m=5, L=L, seed=12)
    bos = wl.bfs_blocks(model, 16, seed=5)
    C, seed, t = 16, 7, 3
    h, params = _setup(model, C, seed, hidden, bos, mlp_path=0)
    x0 = np.random.default_rng(9).integers(0, L, size=(C, model.n_vars)).astype(np.uint8)
    h.set_labels(x0)
    h.set_sweep_index(t)
    h.sweep(1, M.MODE_LEARNED)
    nb = int(bos.max()) + 1
    d, dp = ln.feature_width(L)
    X, z = h.learned_debug(nb * C, dp, 16 * L)
    h.close()
    zr = ln.mlp_forward_bf16(params, X.astype(np.float64))
    err = np.abs(z - zr) / np.maximum(1.0, np.abs(zr))
    row_moved = err.max(axis=1) > 1e-4           # a hidden value on a bf16 rounding boundary
    assert err.max() < 5e-2 and row_moved.mean() < 0.02, (err.max(), row_moved.mean())
    assert np.median(err) < 1e-4


def test_learned_sweep_matches_oracle():
    model = wl.ba_potts(900, m=5, L=4, seed=3)
    dec = dc.decompose(model)
    bos = wl.bfs_blocks(model, 16, seed=4)
    C, seed, t = 4, 21, 6
    h, params = _setup(model, C, seed, 64, bos)
    rng = np.random.default_rng(2)
    x0 = rng.integers(0, 4, size=(C, model.n_vars))
    h.set_labels(x0.astype(np.uint8))
    h.set_sweep_index(t)
    h.sweep(1, M.MODE_LEARNED)
    ref = ln.learned_sweep(model, dec, x0, t, seed, bos, params, bf16_activations=True)
    # cut duals identical except boundary draws
    th = M.unpack_theta(h.debug_theta(), dec.n_entries)
    dual_b = np.abs(ref["u_dual"] - ref["p_dual"]) < 1e-6
    assert not ((th != ref["theta"]) & ~dual_b).any()
    nb = len(ref["members"])
    d, dp = ln.feature_width(4)
    Xg, zg = h.learned_debug(nb * C, dp, 64)
    Xr = ln.to_bf16(ref["X"])
    assert np.abs(Xg - Xr).max() <= 2.0 ** -7 * max(1.0, np.abs(Xr).max())
    # bf16 activations: float32 sums on the GPU and float64 sums in the oracle
    # round a hidden value that sits on a bf16 rounding boundary to neighbouring
    # bf16 values (a relative step of 2^-8), which moves the logits of that row
    # by up to a few 1e-2; everything else agrees to float32 accuracy
    errz = np.abs(zg - ref["z"]) / np.maximum(1.0, np.abs(ref["z"]))
    row_moved = errz.max(axis=1) > 1e-4                        # rows b * C + c with a flipped activation
    assert errz.max() < 5e-2 and row_moved.mean() < 0.02, (errz.max(), row_moved.mean())
    x_gpu = h.get_labels()
    compared = 0
    for b, m in enumerate(ref["members"]):
        u_prop, cdf = ref["prop"][b]
        for c in range(C):
            if row_moved[b * C + c]:
                continue
            near = np.any(np.abs(u_prop[c][:, None] - cdf[c]) < 1e-3)
            near |= abs(ref["u_acc"][b, c] - np.exp(min(0.0, ref["log_alpha"][b, c]))) < 1e-3
            if near:
                continue
            compared += 1
            assert np.array_equal(x_gpu[c, m], ref["x"][c, m]), (b, c)
    assert compared > 0.8 * nb * C
    p, a = h.learned_stats()
    assert p == nb * C and 0 <= a <= p


def test_learned_chain_marginals_within_3_sigma():
    model = wl.tiny_potts(10, 3, 16, seed=7, beta_max=1.0)
    exact, _ = brute.exact_marginals(model)
    bos = wl.bfs_blocks(model, 4, seed=1)
    C, T, burn = 4096, 150, 30
    h, _ = _setup(model, C, 8, 64, bos, wseed=11)         # untrained proposal
    acc = np.zeros((C, model.n_vars, 3))
    # learned and plain sweeps alternate: each leaves p invariant, the plain
    # sweep guarantees mixing, so any bias of the learned step would show
    for t in range(T):
        h.sweep(1, M.MODE_LEARNED if t % 2 == 0 else M.MODE_PLAIN)
        if t >= burn:
            x = h.get_labels()
            acc[np.arange(C)[:, None], np.arange(model.n_vars)[None, :], x] += 1
    cm = acc / (T - burn)
    est, sig = cm.mean(0), cm.std(0, ddof=1) / np.sqrt(C)
    z = np.abs(est - exact) / np.maximum(sig, 1e-12)
    assert z.max() < 4.0 and np.mean(z < 3.0) > 0.95, z.max()
    p, a = h.learned_stats()
    assert a > 0


def test_training_reduces_loss_and_raises_acceptance():
    model = wl.ba_potts(4000, m=5, L=4, seed=5)
    bos = wl.bfs_blocks(model, 16, seed=6)
    C = 8
    h, _ = _setup(model, C, 9, 128, bos)
    h.sweep(30, M.MODE_PLAIN)                         # towards stationarity
    def acceptance(n):
        p0, a0 = h.learned_stats()
        h.sweep(n, M.MODE_LEARNED)
        p1, a1 = h.learned_stats()
        return (a1 - a0) / (p1 - p0)
    before = acceptance(4)
    rows = h.learned_harvest(40, 4, 200000)
    assert rows > 10000
    trace = h.learned_train(400, 512, 2e-3, seed=3)
    assert trace[-40:].mean() < 0.8 * trace[:40].mean()
    after = acceptance(4)
    print("acceptance before", before, "after", after, "loss", trace[:5], trace[-5:])
    assert after > before + 0.05


def test_tensor_core_mlp_wait_timeout_is_reported_and_recoverable():
    """A completion that is never signalled (test hook) makes the MLP kernel's
    bounded waits run out: the sweep reports MRF_ETIMEOUT, and the handle and
    the CUDA context keep working (the next sweep matches a fresh handle's)."""
    model = wl.ba_potts(600, m=5, L=4, seed=13)
    bos = wl.bfs_blocks(model, 16, seed=2)
    C, seed = 8, 3
    h, params = _setup(model, C, seed, 128, bos)
    ref, _ = _setup(model, C, seed, 128, bos)
    x0 = np.random.default_rng(1).integers(0, 4, size=(C, model.n_vars)).astype(np.uint8)
    for hh in (h, ref):
        hh.set_labels(x0)
        hh.set_sweep_index(40)
    h.debug_mlp_timeout(True)
    with pytest.raises(M.MrfError) as e:
        h.sweep(1, M.MODE_LEARNED)
    assert e.value.status == M.MRF_ETIMEOUT
    h.set_labels(x0)
    h.set_sweep_index(40)
    h.sweep(1, M.MODE_LEARNED)
    ref.sweep(1, M.MODE_LEARNED)
    assert np.array_equal(h.get_labels(), ref.get_labels())
    h.close(); ref.close()
