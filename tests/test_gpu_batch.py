"""GPU parity of batched uneven graphs with edits (the paper's dynamic-network
case, abstract and Section 6): a batch of graphs with mixed label counts is
swept per class of equal L as the disjoint union of its graphs; every graph's
labels and counts must equal the oracle run on that union with the class key,
before and after factor insertions and deletions."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import decompose as dc, sampler, philox as ph
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


def _union(models, ids):
    """Disjoint union of models[ids] (sites and edges appended in order)."""
    off = 0
    us, ss, ts, ps = [], [], [], []
    for g in ids:
        m = models[g]
        us.append(m.unary); ss.append(m.src + off); ts.append(m.dst + off); ps.append(m.pair)
        off += m.n_vars
    return wl.Model(off, models[ids[0]].n_labels, np.concatenate(us), np.concatenate(ss).astype(np.int32),
                    np.concatenate(ts).astype(np.int32), np.concatenate(ps))


def _batch_models(n=9, seed=3):
    specs = wl.er_batch_specs(n, n_min=40, n_max=300, labels=(2, 3, 4, 8), seed=seed)
    return [wl.er_graph(s) for s in specs]


def test_batch_sweeps_match_oracle_union_with_edits():
    torch = pytest.importorskip("torch")
    models = _batch_models()
    C, seed = 3, 77
    stream = torch.cuda.Stream()
    b = M.MRFBatch([m.n_vars for m in models], [m.n_labels for m in models], C, seed=seed,
                   stream=stream.cuda_stream, use_graphs=True)
    b.set_factors(models)
    classes = sorted(set(m.n_labels for m in models))
    assert b.n_classes() == len(classes)
    members = {L: [g for g, m in enumerate(models) if m.n_labels == L] for L in classes}
    rng = np.random.default_rng(4)
    # oracle state per class
    unions = {L: _union(models, members[L]) for L in classes}
    slots_u = {L: np.arange(unions[L].n_edges) for L in classes}
    xs = {L: ph.init_labels(unions[L].n_vars, L, C, seed + L * M.BATCH_KEY_STEP) for L in classes}
    t = 0
    def gpu_union_labels(L):
        return np.concatenate([b.get_labels(g) for g in members[L]], axis=1).astype(np.int64)
    for rnd in range(3):
        for s_ in range(3):                      # one sweep at a time from the common state
            before = {L: gpu_union_labels(L) for L in classes}
            b.sweep(1, M.MODE_PLAIN)
            torch.cuda.synchronize()
            for L in classes:
                dec = dc.decompose(unions[L])
                key = (seed + L * M.BATCH_KEY_STEP) & (2**64 - 1)
                if t == 0:
                    assert np.array_equal(before[L], ph.init_labels(unions[L].n_vars, L, C, key))
                ref = sampler.sweep(dec, before[L], t, key, edge_ids=slots_u[L])
                try:
                    compare_sweep(dec, ref, gpu_union_labels(L))
                except AssertionError as exc:
                    raise AssertionError(f"class L={L} sweep t={t} round {rnd}: {exc}")
            t += 1
        # edit: remove 5% of each graph's edges, add as many
        rm_g, rm_s, add_g, add_s, add_t, add_p = [], [], [], [], [], []
        for g, m in enumerate(models):
            info = b.graph(g)
            if not hasattr(m, "slots"):
                m.slots = np.arange(m.n_edges) + info.first_edge_slot
            rem, s_new, t_new, p_new = wl.er_edit(m, 0.05, rng)
            rm_g += [g] * len(rem); rm_s += list(m.slots[rem])
            add_g += [g] * len(s_new); add_s += list(s_new); add_t += list(t_new); add_p.append(p_new.ravel())
            m._pending = (rem, s_new, t_new, p_new)
        new_slots = b.edit_factors(rm_g, rm_s, add_g, add_s, add_t, np.concatenate(add_p))
        # apply the same edit to the oracle unions: removed slots replaced in slot order
        pos = 0
        for g, m in enumerate(models):
            rem, s_new, t_new, p_new = m._pending
            k = len(s_new)
            ids = new_slots[pos:pos + k]; pos += k
            keep = np.ones(m.n_edges, bool); keep[rem] = False
            m.src = np.concatenate([m.src[keep], s_new]).astype(np.int32)
            m.dst = np.concatenate([m.dst[keep], t_new]).astype(np.int32)
            m.pair = np.concatenate([m.pair[keep], p_new])
            m.slots = np.concatenate([m.slots[keep], ids])
        for L in classes:
            # the union's edges in slot order, with their slots as RNG indices
            us = _union(models, members[L])
            slots = np.concatenate([models[g].slots for g in members[L]])
            order = np.argsort(slots)
            unions[L] = wl.Model(us.n_vars, L, us.unary, us.src[order], us.dst[order], us.pair[order])
            slots_u[L] = slots[order]


def test_batch_counts_per_graph():
    models = _batch_models(5, seed=8)
    b = M.MRFBatch([m.n_vars for m in models], [m.n_labels for m in models], 2, seed=1, use_graphs=False)
    b.set_factors(models)
    b.reset_marginals(1)
    b.sweep(5, M.MODE_FUSED)
    for g, m in enumerate(models):
        c = b.counts(g)
        assert c.shape == (m.n_vars, m.n_labels)
        assert np.all(c.sum(1) == 4 * 2)


def _host_memory_gb():
    """Memory this process may use: MemAvailable, capped by a cgroup limit."""
    avail = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) / 2**20
    except OSError:
        pass
    for path in ("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory/memory.limit_in_bytes"):
        try:
            v = open(path).read().strip()
            if v.isdigit():
                avail = min(avail or 1e9, int(v) / 2**30)
        except OSError:
            pass
    return avail or 0.0


def test_full_batch_2000_graphs_sampled_graphs_match_oracle():
    """The batched workload at its stated size: 2000 Erdos-Renyi graphs
    (N ~ floor(exp U[ln 100, ln 50000]), mean degree U[3, 20], L in
    {2, 4, 8, 16}, tables exp(U[-0.5, 0.5]), one chain each), one sweep, one
    edit round (1 % of every graph's edges removed, as many added), one more
    sweep.  Per class of equal L the batch sweeps the disjoint union of its
    graphs; a graph interacts only with its own edges, so the oracle sweeps
    sampled graphs alone with their union site ids, edge slots and the class
    key as RNG indices (the smallest and a random graph of every class)."""
    torch = pytest.importorskip("torch")
    if _host_memory_gb() < 160:
        pytest.skip("the 2000-graph batch needs ~100 GB of host memory for its tables")
    specs = wl.er_batch_specs(2000, seed=0)
    models = [wl.er_graph(sp) for sp in specs]
    C, seed = 1, 5
    stream = torch.cuda.Stream()
    b = M.MRFBatch([m.n_vars for m in models], [m.n_labels for m in models], C, seed=seed,
                   stream=stream.cuda_stream, use_graphs=True)
    b.set_factors(models)
    rng = np.random.default_rng(11)
    sample = []
    for L in (2, 4, 8, 16):
        ids = [g for g, m in enumerate(models) if m.n_labels == L]
        sample += [min(ids, key=lambda g: models[g].n_vars), int(rng.choice(ids))]
    for g in range(len(models)):
        models[g].slots = np.arange(models[g].n_edges) + b.graph(g).first_edge_slot
    checked = 0
    for rnd in range(2):
        t = rnd
        before = {g: b.get_labels(g).astype(np.int64) for g in sample}
        b.sweep(1, M.MODE_PLAIN)
        torch.cuda.synchronize()
        for g in sample:
            m = models[g]
            info = b.graph(g)
            key = (seed + m.n_labels * M.BATCH_KEY_STEP) & (2**64 - 1)
            order = np.argsort(m.slots)
            sub = wl.Model(m.n_vars, m.n_labels, m.unary, m.src[order], m.dst[order], m.pair[order])
            dec = dc.decompose(sub)
            ref = sampler.sweep(dec, before[g], t, key, edge_ids=m.slots[order],
                                site_ids=info.site_offset + np.arange(m.n_vars))
            compare_sweep(dec, ref, b.get_labels(g))
            checked += 1
        if rnd == 0:
            # one edit round on every graph
            rm_g, rm_s, add_g, add_s, add_t, add_p, pend = [], [], [], [], [], [], []
            for g, m in enumerate(models):
                rem, s_new, t_new, p_new = wl.er_edit(m, 0.01, rng)
                rm_g.append(np.full(len(rem), g)); rm_s.append(m.slots[rem])
                add_g.append(np.full(len(s_new), g)); add_s.append(s_new); add_t.append(t_new)
                add_p.append(p_new.ravel()); pend.append((rem, s_new, t_new, p_new))
            ids = b.edit_factors(np.concatenate(rm_g), np.concatenate(rm_s), np.concatenate(add_g),
                                 np.concatenate(add_s), np.concatenate(add_t), np.concatenate(add_p))
            pos = 0
            for g, m in enumerate(models):
                rem, s_new, t_new, p_new = pend[g]
                keep = np.ones(m.n_edges, bool); keep[rem] = False
                m.src = np.concatenate([m.src[keep], s_new]).astype(np.int32)
                m.dst = np.concatenate([m.dst[keep], t_new]).astype(np.int32)
                m.pair = np.concatenate([m.pair[keep], p_new])
                m.slots = np.concatenate([m.slots[keep], ids[pos:pos + len(s_new)]])
                pos += len(s_new)
    assert checked == 2 * len(sample)
    b.close()


@pytest.mark.parametrize("mode", [M.MODE_SW, M.MODE_HIGDON])
def test_batch_cluster_sweeps_equal_one_handle_per_class(mode):
    """Swendsen-Wang and Higdon sweeps of a batch (ferromagnetic graphs, two
    label classes) equal the same sweeps of one handle on each class union
    with the class's key, bit for bit (the union handle is checked against
    the oracle in tests/test_gpu_sw.py and tests/test_gpu_higdon.py)."""
    torch = pytest.importorskip("torch")
    models = [wl.ferro_potts_graph(n, L, e, seed=s) for n, L, e, s in
              ((60, 2, 150, 1), (90, 3, 200, 2), (40, 2, 90, 3), (70, 3, 160, 4))]
    C, seed = 4, 19
    stream = torch.cuda.Stream()
    b = M.MRFBatch([m.n_vars for m in models], [m.n_labels for m in models], C, seed=seed,
                   stream=stream.cuda_stream)
    b.set_factors(models)
    b.sweep(2, M.MODE_PLAIN)
    b.sweep(3, mode)
    for L in (2, 3):
        ids = [g for g, m in enumerate(models) if m.n_labels == L]
        un = _union(models, ids)
        h = M.MRF(un.n_vars, L, C, seed=(seed + L * M.BATCH_KEY_STEP) & (2**64 - 1), use_graphs=False)
        h.set_factors(un.unary, un.src, un.dst, un.pair)
        h.sweep(2, M.MODE_PLAIN)
        h.sweep(3, mode)
        x = h.get_labels()
        h.close()
        xb = np.concatenate([b.get_labels(g) for g in ids], axis=1)
        assert np.array_equal(xb, x), (L, mode)
    b.close()
