"""Host-side parts of bench.py's other workloads: the algorithmic byte counts
behind the batched line's roofline (the edge-partial kernels), and the
embedding of the other workloads' lines in the default run (child processes
faked here, so no GPU is needed)."""
import json
import types

import bench


def test_edge_partial_byte_counts():
    # L = 16 pivot table: 225 entries, 8 words of dual bits, one chain
    info = dict(E=1000, N=200, L=16, m=225, partial=True)
    _, b_pass = bench.kernel_work("k_edge_partial", info, 1)
    assert b_pass == 1000 * (225 * 4 + 8 * 4 + 2 * 16 * 4 + 4)
    _, b_primal = bench.kernel_work("k_primal", info, 1)
    assert b_primal == 2 * 1000 * 16 * 4 + 2 * 1000 * 8 + 200 * 16 * 4 + 2 * 200 + 200 * 8
    # without the edge-partial form the primal step reads every incident weight row
    _, b_full = bench.kernel_work("k_primal", dict(info, partial=False), 1)
    assert b_full > 10 * b_primal


def test_other_configs_embeds_child_lines(monkeypatch):
    calls = []

    def fake_run(cmd, capture_output, text, timeout):
        calls.append(cmd)
        wl = cmd[cmd.index("--workload") + 1]
        if wl == "ba_learned":
            return types.SimpleNamespace(returncode=1, stdout="", stderr="no device\n")
        line = {"metric": bench.METRIC, "value": 1.0, "config": {"workload": wl}}
        return types.SimpleNamespace(returncode=0, stdout="noise\n" + json.dumps(line) + "\n", stderr="")

    monkeypatch.setattr(bench.subprocess, "run", fake_run)
    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(empty_cache=lambda: None))
    monkeypatch.setitem(__import__("sys").modules, "torch", fake_torch)
    args = types.SimpleNamespace(seed=3, no_cpu=True)
    out = bench.other_configs(args)
    assert set(out) == {"dense4096", "er_batch_2000", "ba_learned_1e6"}
    assert out["dense4096"]["config"]["workload"] == "dense4096"
    assert out["er_batch_2000"]["value"] == 1.0
    assert out["ba_learned_1e6"]["unavailable"].startswith("exit 1")
    for cmd in calls:
        assert "--no-configs" in cmd and "--no-cpu" in cmd and cmd[cmd.index("--seed") + 1] == "3"
