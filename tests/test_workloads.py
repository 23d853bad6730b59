"""Host-side checks of the batched dynamic workload's edit generator: every
round keeps each graph's edge count, removes edges that exist, adds distinct
non-self-loop pairs absent from the graph, and draws one table per addition
with the stated distribution."""
import math

import numpy as np

from paper_1611_06684_gb300 import workloads as wl


def test_batch_edits_keep_graphs_simple_and_counts_fixed():
    specs = wl.er_batch_specs(30, n_min=20, n_max=2000, seed=4)
    models = [wl.er_graph(s) for s in specs]
    first = np.concatenate([[0], np.cumsum([m.n_edges for m in models])[:-1]])
    ed = wl.ErBatchEdits(models, first, seed=3)
    E0 = [m.n_edges for m in models]
    next_slot = 10**9
    for _ in range(4):
        before = [set(zip(np.minimum(ed.src[g], ed.dst[g]).tolist(), np.maximum(ed.src[g], ed.dst[g]).tolist()))
                  for g in range(ed.G)]
        slots_before = [set(ed.slot[g].tolist()) for g in range(ed.G)]
        rm_g, rm_s, add_g, s, t, tables = ed.edit(0.05)
        k = [math.ceil(0.05 * e) for e in E0]
        assert np.array_equal(np.bincount(rm_g, minlength=ed.G), k)
        assert np.array_equal(np.bincount(add_g, minlength=ed.G), k)
        assert np.all(np.diff(add_g) >= 0)                   # additions grouped by graph
        for g in range(ed.G):
            assert set(rm_s[rm_g == g].tolist()) <= slots_before[g]
            pairs = list(zip(np.minimum(s, t)[add_g == g].tolist(), np.maximum(s, t)[add_g == g].tolist()))
            assert len(set(pairs)) == len(pairs)
            assert not (set(pairs) & before[g])
            assert all(a != b and 0 <= a < models[g].n_vars and 0 <= b < models[g].n_vars for a, b in pairs)
        assert tables.shape[0] == int((ed.L[add_g] ** 2).sum())
        assert tables.dtype == np.float32 and tables.min() >= -0.5 and tables.max() <= 0.5
        new = np.arange(len(s)) + next_slot
        next_slot += len(s)
        ed.apply(new)
        for g in range(ed.G):
            assert len(ed.src[g]) == E0[g]
            assert not (set(rm_s[rm_g == g].tolist()) & set(ed.slot[g].tolist()))
        keys = np.sort(np.concatenate([ed.base[g] + ed.lo[g].astype(np.int64) * ed.n[g] + ed.hi[g]
                                       for g in range(ed.G)]))
        assert np.array_equal(keys, ed.keys) and np.all(np.diff(keys) > 0)
