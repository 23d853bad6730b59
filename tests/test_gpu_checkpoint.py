"""Checkpoint and resume (mrf_save / mrf_load): a chain resumed from a
checkpoint continues exactly as the uninterrupted one."""
import numpy as np
import pytest

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


def _state(h):
    marg, n = h.marginals()
    return h.get_labels(), h.counts(), n, h.info().sweep_index


@pytest.mark.parametrize("case", ["lattice", "edited_graph"])
def test_resume_from_checkpoint_is_bit_exact(case, tmp_path):
    from paper_1611_06684_gb300 import mrf as M
    if case == "lattice":
        model = wl.potts_grid3d(9, 8, 6, L=5, seed=1)
        h = M.MRF(model.n_vars, 5, 32, seed=3, grid=model.grid)
    else:
        model = wl.random_graph(300, k=3, L=4, seed=2)
        h = M.MRF(model.n_vars, 4, 6, seed=3)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    h.sweep(4, M.MODE_PLAIN)
    if case == "edited_graph":
        rng = np.random.default_rng(0)
        rem = rng.choice(model.n_edges, size=40, replace=False)
        s = rng.integers(0, model.n_vars, size=25).astype(np.int32)
        t = ((s + 1 + rng.integers(0, model.n_vars - 1, size=25)) % model.n_vars).astype(np.int32)
        h.edit_factors(rem, s, t, rng.normal(0, 0.5, size=(25, 4, 4)).astype(np.float32))   # leaves free slots
    h.reset_marginals(2)
    h.sweep(3, M.MODE_PLAIN)
    path = str(tmp_path / "ckpt.mrf")
    h.save(path)
    r = M.MRF.load(path)
    for hh in (h, r):
        hh.sweep(5, M.MODE_PLAIN)
        hh.sweep(1, M.MODE_PLAIN)
        if case == "lattice":
            hh.sweep(2, M.MODE_SPLASH)
    a, b = _state(h), _state(r)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    assert a[2] == b[2] and a[3] == b[3]
    ia, ib = h.info(), r.info()
    assert (ia.n_edge_slots, ia.n_edges, ia.layout, ia.n_entries) == (ib.n_edge_slots, ib.n_edges, ib.layout, ib.n_entries)
    h.close(); r.close()


def test_load_rejects_a_file_that_is_not_a_checkpoint(tmp_path):
    from paper_1611_06684_gb300 import mrf as M
    p = tmp_path / "junk.bin"
    p.write_bytes(b"not a checkpoint at all" * 10)
    with pytest.raises(M.MrfError) as e:
        M.MRF.load(str(p))
    assert e.value.status == M.MRF_EINVAL
