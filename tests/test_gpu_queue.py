"""GPU parity of the device edit queue of a batch (the dynamic networks of the
abstract and Section 6): a round {edit, sweeps} applied by kernels inside one
captured CUDA graph must give exactly what the host-side edit followed by the
same sweeps gives -- the same slots for the added edges, the same tables and
folded unaries, the same labels bit for bit -- and each of its sweeps must
match the oracle run on the edited class unions.  Rejected edits change
nothing and report their reasons."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import decompose as dc, sampler
from paper_1611_06684_gb300 import workloads as wl
from paper_1611_06684_gb300 import mrf as M
from tests.gpu_helpers import compare_sweep
from tests.test_gpu_batch import _union


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_06684_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _models(n=10, seed=3, diag_L=3):
    """ER graphs with L in {2, 3, 4, 8}; the L = diag_L graphs get Potts-type
    (diagonal) tables, so their class uses the diagonal layout."""
    specs = wl.er_batch_specs(n, n_min=40, n_max=400, labels=(2, 3, 4, 8), seed=seed)
    ms = [wl.er_graph(s) for s in specs]
    for m in ms:
        if m.n_labels == diag_L:
            m.pair = m.pair * np.eye(diag_L, dtype=np.float32)[None]
    return ms


def _batch(models, C, seed, stream, use_graphs=True):
    b = M.MRFBatch([m.n_vars for m in models], [m.n_labels for m in models], C, seed=seed,
                   stream=stream.cuda_stream, use_graphs=use_graphs)
    b.set_factors(models)
    return b


def _edit(models, frac, rng, diag_L=3):
    """One edit of every graph: (arrays for the batch, per-graph pending edits)."""
    rm_g, rm_s, add_g, add_s, add_t, add_p, pend = [], [], [], [], [], [], []
    for g, m in enumerate(models):
        rem, s_new, t_new, p_new = wl.er_edit(m, frac, rng)
        if m.n_labels == diag_L:
            p_new = p_new * np.eye(diag_L, dtype=np.float32)[None]
        rm_g += [g] * len(rem); rm_s += list(m.slots[rem])
        add_g += [g] * len(s_new); add_s += list(s_new); add_t += list(t_new); add_p.append(p_new.ravel())
        pend.append((rem, s_new, t_new, p_new))
    arrays = (np.array(rm_g, np.int32), np.array(rm_s, np.int64), np.array(add_g, np.int32),
              np.array(add_s, np.int32), np.array(add_t, np.int32), np.concatenate(add_p).astype(np.float32))
    return arrays, pend


def _apply(models, pend, new_slots):
    pos = 0
    for g, m in enumerate(models):
        rem, s_new, t_new, p_new = pend[g]
        k = len(s_new)
        keep = np.ones(m.n_edges, bool); keep[rem] = False
        m.src = np.concatenate([m.src[keep], s_new]).astype(np.int32)
        m.dst = np.concatenate([m.dst[keep], t_new]).astype(np.int32)
        m.pair = np.concatenate([m.pair[keep], p_new])
        m.slots = np.concatenate([m.slots[keep], new_slots[pos:pos + k]]); pos += k


def _labels(b, members):
    return np.concatenate([b.get_labels(g) for g in members], axis=1).astype(np.int64)


def test_queue_rounds_match_host_edits_and_oracle():
    torch = pytest.importorskip("torch")
    models = _models()
    C, seed = 2, 41
    stream = torch.cuda.Stream()
    bq = _batch(models, C, seed, stream)
    bh = _batch(models, C, seed, stream)
    for g, m in enumerate(models):
        m.slots = np.arange(m.n_edges) + bq.graph(g).first_edge_slot
    classes = sorted(set(m.n_labels for m in models))
    members = {L: [g for g, m in enumerate(models) if m.n_labels == L] for L in classes}
    assert any(bq.class_handle(k).info().layout == M.LAYOUT_DIAG for k in range(bq.n_classes()))
    rng = np.random.default_rng(5)
    bq.queue_create(4096, 4096, 4096 * 64, 512)
    bq.sweep(2); bh.sweep(2)
    t = 2
    for rnd in range(4):
        arrays, pend = _edit(models, 0.05, rng)
        before = {L: _labels(bq, members[L]) for L in classes}
        bq.queue_load(*arrays)
        bq.round(1)
        status, slots_q = bq.queue_result(len(arrays[3]))
        assert status == 0, status
        slots_h = bh.edit_factors(*arrays)
        bh.sweep(1)
        torch.cuda.synchronize()
        assert np.array_equal(slots_q, slots_h)
        _apply(models, pend, slots_q)
        for k in range(bq.n_classes()):
            hq, hh = bq.class_handle(k), bh.class_handle(k)
            assert hq.info().n_edges == hh.info().n_edges
            tq, thq, uq = hq.debug_tables()
            th, thh, uh = hh.debug_tables()
            n = min(tq.shape[0], th.shape[0])
            live = np.zeros(n, bool)
            L = hq.L
            for g in members[L]:
                live[models[g].slots[models[g].slots < n]] = True
            assert np.array_equal(tq[:n][live], th[:n][live]) and np.array_equal(thq[:n][live], thh[:n][live])
            assert np.array_equal(uq, uh)
        for L in classes:
            xq = _labels(bq, members[L])
            assert np.array_equal(xq, _labels(bh, members[L])), f"class L={L} round {rnd}"
            us = _union(models, members[L])
            slots = np.concatenate([models[g].slots for g in members[L]])
            order = np.argsort(slots)
            un = wl.Model(us.n_vars, L, us.unary, us.src[order], us.dst[order], us.pair[order])
            key = (seed + L * M.BATCH_KEY_STEP) & (2**64 - 1)
            ref = sampler.sweep(dc.decompose(un), before[L], t, key, edge_ids=slots[order])
            compare_sweep(dc.decompose(un), ref, xq)
        t += 1
        # a few plain sweeps between rounds (the round graph and the sweep graph share the classes)
        bq.sweep(2); bh.sweep(2)
        t += 2
    bq.close(); bh.close()


def test_queue_round_of_many_sweeps_and_host_edit_in_between():
    """Rounds of 5 sweeps with the graph replayed, a host-side edit between
    device rounds (the host mirror is read back first), and the direct
    (uncaptured) launch path: all equal to host edits + sweeps."""
    torch = pytest.importorskip("torch")
    models = _models(8, seed=11)
    stream = torch.cuda.Stream()
    bq = _batch(models, 1, 9, stream)
    bn = _batch(models, 1, 9, stream, use_graphs=False)
    bh = _batch(models, 1, 9, stream)
    for g, m in enumerate(models):
        m.slots = np.arange(m.n_edges) + bq.graph(g).first_edge_slot
    rng = np.random.default_rng(2)
    for b in (bq, bn):
        b.queue_create(2048, 2048, 2048 * 64, 256)
    for rnd in range(5):
        arrays, pend = _edit(models, 0.03, rng)
        if rnd == 2:                                   # host-side edit on the queue batches too
            outs = [b.edit_factors(*arrays) for b in (bq, bn, bh)]
            for b in (bq, bn, bh):
                b.sweep(5)
            assert all(np.array_equal(o, outs[2]) for o in outs)
            new = outs[2]
        else:
            for b in (bq, bn):
                b.queue_load(*arrays)
                b.round(5)
            sq, new = bq.queue_result(len(arrays[3]))
            sn, new_n = bn.queue_result(len(arrays[3]))
            assert sq == 0 and sn == 0
            assert np.array_equal(new, new_n)
            assert np.array_equal(bh.edit_factors(*arrays), new)
            bh.sweep(5)
        _apply(models, pend, new)
        for g in range(len(models)):
            x = bh.get_labels(g)
            assert np.array_equal(bq.get_labels(g), x) and np.array_equal(bn.get_labels(g), x), (rnd, g)
    # an empty round is plain sweeps
    for b in (bq, bh):
        if b is bq:
            b.round(5)
        else:
            b.sweep(5)
    st, _ = bq.queue_result(0)
    assert st == 0
    for g in range(len(models)):
        assert np.array_equal(bq.get_labels(g), bh.get_labels(g))
    # a new queue replaces the old one; the classes' edge counts stay right
    bq.queue_create(16, 16, 16 * 64, 8)
    for k in range(bq.n_classes()):
        assert bq.class_handle(k).info().n_edges == bh.class_handle(k).info().n_edges
    for b in (bq, bn, bh):
        b.close()


def _bad_cases(models, slots):
    g2 = next(g for g, m in enumerate(models) if m.n_labels == 2)
    g3 = next(g for g, m in enumerate(models) if m.n_labels == 3)
    m2 = models[g2]
    p2 = np.zeros((1, 2, 2), np.float32)
    live = int(slots[g2][0])
    ok_add = (np.array([g2], np.int32), np.array([0], np.int32), np.array([1], np.int32), p2.ravel())
    none_rm = (np.zeros(0, np.int32), np.zeros(0, np.int64))
    cases = {
        M.Q_SLOT: (np.array([g2], np.int32), np.array([10**9], np.int64)) + (np.zeros(0, np.int32),) * 3 + (np.zeros(0, np.float32),),
        M.Q_DUP: (np.array([g2, g2], np.int32), np.array([live, live], np.int64)) + (np.zeros(0, np.int32),) * 3 + (np.zeros(0, np.float32),),
        M.Q_GRAPH: (np.array([len(models)], np.int32), np.array([live], np.int64)) + (np.zeros(0, np.int32),) * 3 + (np.zeros(0, np.float32),),
        M.Q_VERTEX: none_rm + (np.array([g2], np.int32), np.array([0], np.int32), np.array([m2.n_vars], np.int32), p2.ravel()),
        M.Q_LOOP: none_rm + (np.array([g2], np.int32), np.array([1], np.int32), np.array([1], np.int32), p2.ravel()),
        M.Q_NONFINITE: none_rm + ok_add[:3] + (np.array([0, np.nan, 0, 0], np.float32),),
        M.Q_OFFDIAG: none_rm + (np.array([g3], np.int32), np.array([0], np.int32), np.array([1], np.int32),
                                np.arange(9, dtype=np.float32)),
    }
    return cases, ok_add, none_rm


def test_queue_rejects_bad_edits_without_changes():
    torch = pytest.importorskip("torch")
    models = _models(8, seed=4)
    stream = torch.cuda.Stream()
    bq = _batch(models, 2, 3, stream)
    bp = _batch(models, 2, 3, stream)
    slots = [np.arange(m.n_edges) + bq.graph(g).first_edge_slot for g, m in enumerate(models)]
    bq.queue_create(64, 64, 64 * 64, 0)
    cases, ok_add, none_rm = _bad_cases(models, slots)
    for bit, arrays in cases.items():
        bq.queue_load(*arrays)
        bq.round(1)
        st, out = bq.queue_result(len(arrays[2]))
        assert st & bit, (bit, st)
        assert (out == -1).all()
        bp.sweep(1)
        for g in range(len(models)):
            assert np.array_equal(bq.get_labels(g), bp.get_labels(g)), (bit, g)
        for k in range(bq.n_classes()):
            assert bq.class_handle(k).info().n_edges == bp.class_handle(k).info().n_edges
    # table floats that do not match the additions
    bq.queue_load(*(none_rm + ok_add[:3] + (np.zeros(8, np.float32),)))
    bq.round(1); bp.sweep(1)
    st, _ = bq.queue_result(1)
    assert st & M.Q_PAIR
    # no reserved slot (extra_slots = 0): an addition without a removal has nowhere to go
    bq.queue_load(*(none_rm + ok_add))
    bq.round(1); bp.sweep(1)
    st, _ = bq.queue_result(1)
    assert st & M.Q_SLOTS
    for g in range(len(models)):
        assert np.array_equal(bq.get_labels(g), bp.get_labels(g))
    # capacities are checked on the host
    with pytest.raises(M.MrfError):
        bq.queue_load(np.zeros(65, np.int32), np.zeros(65, np.int64), *(np.zeros(0, np.int32),) * 3, np.zeros(0, np.float32))
    bq.close(); bp.close()


def test_queue_sorts_long_incidence_lists_on_device():
    """A hub with more than 512 incidences: the host edit rebuilds its list on
    the host, the queue round sorts it on the device; both give the slot order,
    so the chains stay identical."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    N, L = 3000, 4
    hub_leaves = rng.choice(np.arange(1, N), size=900, replace=False)
    src = np.concatenate([np.zeros(900, np.int32), rng.integers(1, N, 4000).astype(np.int32)])
    dst = np.concatenate([hub_leaves.astype(np.int32), rng.integers(1, N, 4000).astype(np.int32)])
    keep = src != dst
    src, dst = src[keep], dst[keep]
    key = np.minimum(src, dst).astype(np.int64) * N + np.maximum(src, dst)
    _, first = np.unique(key, return_index=True)
    src, dst = src[np.sort(first)], dst[np.sort(first)]
    pair = rng.uniform(-0.5, 0.5, (len(src), L, L)).astype(np.float32)
    m = wl.Model(N, L, rng.normal(size=(N, L)).astype(np.float32), src, dst, pair)
    small = wl.er_graph(wl.er_batch_specs(1, n_min=50, n_max=60, labels=(2,), seed=1)[0])
    models = [m, small]
    stream = torch.cuda.Stream()
    bq = _batch(models, 2, 1, stream)
    bh = _batch(models, 2, 1, stream)
    for g, mm in enumerate(models):
        mm.slots = np.arange(mm.n_edges) + bq.graph(g).first_edge_slot
    bq.queue_create(256, 256, 256 * 16, 64)
    for rnd in range(3):
        rem = np.sort(rng.choice(m.n_edges, 40, replace=False))
        leaves = rng.choice(np.setdiff1d(np.arange(1, N), m.dst[m.src == 0]), 30, replace=False).astype(np.int32)
        p_new = rng.uniform(-0.5, 0.5, (30, L, L)).astype(np.float32)
        arrays = (np.zeros(40, np.int32), m.slots[rem].astype(np.int64), np.zeros(30, np.int32),
                  np.zeros(30, np.int32), leaves, p_new.ravel())
        bq.queue_load(*arrays)
        bq.round(2)
        st, new = bq.queue_result(30)
        assert st == 0
        assert np.array_equal(bh.edit_factors(*arrays), new)
        bh.sweep(2)
        _apply([m], [(rem, np.zeros(30, np.int32), leaves, p_new)], new)
        assert np.array_equal(bq.get_labels(0), bh.get_labels(0)), rnd
    assert int((m.src == 0).sum() + (m.dst == 0).sum()) > 512
    bq.close(); bh.close()


def test_queue_with_zero_capacity_and_edge_partial_classes():
    """A queue of capacity zero makes rounds plain sweeps; a batch whose
    classes take the edge-partial plain sweep (one chain, L = 12 and 16:
    121 and 225 entries per edge) gives the same chain with queue rounds as
    with host edits."""
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    specs = wl.er_batch_specs(6, n_min=60, n_max=500, labels=(12, 16), seed=21)
    models = [wl.er_graph(s) for s in specs]
    bz = _batch(models, 1, 4, stream)
    bp = _batch(models, 1, 4, stream)
    bz.queue_create(0, 0, 0, 0)
    bz.round(3); bp.sweep(3)
    st, _ = bz.queue_result(0)
    assert st == 0
    for g in range(len(models)):
        assert np.array_equal(bz.get_labels(g), bp.get_labels(g))
    bz.close(); bp.close()
    bq = _batch(models, 1, 4, stream)
    bh = _batch(models, 1, 4, stream)
    for g, m in enumerate(models):
        m.slots = np.arange(m.n_edges) + bq.graph(g).first_edge_slot
    bq.queue_create(1024, 1024, 1024 * 256, 64)
    rng = np.random.default_rng(8)
    for rnd in range(3):
        arrays, pend = _edit(models, 0.04, rng, diag_L=0)
        bq.queue_load(*arrays)
        bq.round(4)
        st, new = bq.queue_result(len(arrays[3]))
        assert st == 0
        assert np.array_equal(bh.edit_factors(*arrays), new)
        bh.sweep(4)
        _apply(models, pend, new)
        for g in range(len(models)):
            assert np.array_equal(bq.get_labels(g), bh.get_labels(g)), (rnd, g)
    bq.close(); bh.close()
