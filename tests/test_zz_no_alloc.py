"""mrf_sweep_noalloc: the plain sweep for callers that cannot allocate device
memory when they sweep (for instance under a framework that forbids
allocation at that point, or when all device memory comes from the caller's
own fixed pool).  It keeps the dual bits in a fixed device array
inside the library and uses label buffers the caller owns; its result must
equal the handle's ordinary plain sweep from the same state.  This file is
collected last so that a run stopping at the first failure has already run
every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from paper_1611_06684_gb300 import workloads as wl
from paper_1611_06684_gb300 import mrf as M


@pytest.fixture(scope="module")
def torch_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_06684_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


@pytest.mark.parametrize("model_fn,C", [
    (lambda: wl.potts_grid3d(11, 9, 7, L=8, seed=3), 64),      # 3-D lattice, 49 dual bits per edge
    (lambda: wl.tiny_potts(400, 4, 1800, seed=4), 16),          # Potts tables, diagonal layout
    (lambda: wl.dense_potts(120, L=4, seed=5), 8),              # fully connected, high degree
])
def test_noalloc_matches_plain_sweep_twice(torch_gpu, model_fn, C):
    torch = torch_gpu
    model = model_fn()
    seed, t = 31, 7
    h = M.MRF(model.n_vars, model.n_labels, C, seed=seed, use_graphs=False)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    rng = np.random.default_rng(1)
    x0 = rng.integers(0, model.n_labels, size=(C, model.n_vars)).astype(np.uint8)
    # existing entry point: two plain sweeps from x0 at indices t, t+1
    h.set_labels(x0)
    h.set_sweep_index(t)
    h.sweep(1, M.MODE_PLAIN)
    ref1 = h.get_labels()
    h.sweep(1, M.MODE_PLAIN)
    ref2 = h.get_labels()
    # allocation-free entry point on caller-owned [N][C] device buffers
    xa = torch.from_numpy(np.ascontiguousarray(x0.T)).cuda()
    xb = torch.empty_like(xa)
    h.sweep_noalloc(xa, xb, t)
    h.sweep_noalloc(xb, xa, t + 1)
    torch.cuda.synchronize()
    got1 = xb.cpu().numpy().T
    got2 = xa.cpu().numpy().T
    assert np.array_equal(got1, ref1)
    assert np.array_equal(got2, ref2)
    # the handle's own state is untouched
    assert h.info().sweep_index == t + 2
    assert np.array_equal(h.get_labels(), ref2)
    h.close()


def test_noalloc_rejects_models_beyond_the_static_array(torch_gpu):
    torch = torch_gpu
    model = wl.potts_grid3d(40, 40, 40, L=8, seed=0)        # 187,200 edges x 16 chains x 2 words > 2^22
    C = 16
    h = M.MRF(model.n_vars, 8, C, seed=0)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    xa = torch.zeros((model.n_vars, C), dtype=torch.uint8, device="cuda")
    xb = torch.zeros_like(xa)
    with pytest.raises(M.MrfError) as e:
        h.sweep_noalloc(xa, xb, 0)
    assert e.value.status == M.MRF_ERANGE
    with pytest.raises(M.MrfError) as e:
        h.sweep_noalloc(xa, xa, 0)
    assert e.value.status == M.MRF_EINVAL
    h.close()
