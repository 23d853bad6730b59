#!/usr/bin/env python
"""Throughput of the primal-dual Gibbs sweep on GB300.

One step = one full sweep of the sampler over the whole model for every chain:
the dual half-step (theta | x over all edges), the primal half-step (x | theta
over all sites) and the marginal-count accumulation.  Default workload: the
3-D 6-neighbour Potts grid 128^3 (2,097,152 sites, 6,242,304 edges), L = 8,
random positive tables exp(U[-0.3, 0.3]), unaries N(0, 1), 64 chains.

Metric: site-updates/s (= chains x sites x sweeps / device time).  Multi-GPU
runs (torchrun) give every rank its own independent chains (weak scaling, no
data-path collective); value = all ranks' site-updates / max time.

`--impl reference` times the CPU oracle (the float64 numpy statement of the
method) on a bounded sample of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "site-updates/s"
FERRO_BETA = (0.0, 1.0)
FERRO_U_STD = 0.5

WORKLOADS = {
    # name: (generator, chains, description)
    "potts3d": (lambda: __import__("paper_1611_06684_gb300.workloads", fromlist=["x"]).potts_grid3d(128, L=8, seed=0),
                64, "3-D 6-neighbour Potts grid 128^3, L=8, tables exp(U[-0.3,0.3]), unaries N(0,1), 64 chains"),
    "ising32": (lambda: __import__("paper_1611_06684_gb300.workloads", fromlist=["x"]).ising_grid(32, 32, seed=0),
                1, "2-D Ising grid 32x32, L=2, h~N(0,0.5^2), J~U[0,0.3], 1 chain"),
    "dense4096": (lambda: __import__("paper_1611_06684_gb300.workloads", fromlist=["x"]).dense_potts(4096, L=4, seed=0),
                  16, "fully connected N=4096 (8,386,560 edges), L=4, w~N(0,(0.2/64)^2), unaries N(0,1), 16 chains"),
    # ferromagnetic Potts lattice: the Swendsen-Wang sweep (Section 4.3) applies
    "ferro3d": (lambda: __import__("paper_1611_06684_gb300.workloads", fromlist=["x"]).ferro_potts_grid3d(
                    128, L=8, beta_lo=FERRO_BETA[0], beta_hi=FERRO_BETA[1], u_std=FERRO_U_STD, seed=0),
                64, "3-D 6-neighbour ferromagnetic Potts grid 128^3, L=8, w_e(a,b) = beta_e [a=b], "
                    "beta_e~U[%g,%g], unaries N(0,%g^2), 64 chains"),
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def clocks_start(path):
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                              "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"],
                             stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except Exception:
        return None, None


def clocks_stop(handle, path, gpu_index):
    p, f = handle
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    f.close()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or parts[0] != str(gpu_index):
            continue
        try:
            sm.append(float(parts[1])); mx.append(float(parts[2]))
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# Issue cost of one Philox4x32-10 call on GB300, from the ncu counters of the
# Philox-only kernel (mrf_philox_rate: 79.7 M calls, 146.3 us at 2068 MHz):
# 15.1 warp instructions per warp-wide call run on the fmaheavy pipe (integer
# multiplies), which is busy 83.2 % of the cycles, i.e. 61.5 pipe cycles per
# warp-wide call on each SM sub-partition; its 19.3 alu-pipe instructions
# (2 cycles each) and 38.6 issue slots per call fit inside that.
PHILOX_FMAHEAVY_CYCLES_PER_WARP_CALL = 61.5


def _describe(workload):
    if workload == "er_batch":
        return ("2000 Erdos-Renyi graphs, N ~ logU[100, 50000], mean degree U[3, 20], L in {2,4,8,16}, "
                "tables exp(U[-0.5,0.5]), 1 chain each; 1% edits every 10 sweeps")
    desc = WORKLOADS[workload][2]
    return desc % (FERRO_BETA[0], FERRO_BETA[1], FERRO_U_STD) if "%g" in desc else desc


def alu_peak_philox_calls(sm_mhz):
    """Philox4x32-10 calls/s roof of the fmaheavy pipe: 152 SMs x 4
    sub-partitions x 32 lanes x clock / 61.5 pipe cycles per warp-wide call."""
    return 152 * 4 * 32 / PHILOX_FMAHEAVY_CYCLES_PER_WARP_CALL * sm_mhz * 1e6


def kernel_work(name, model_info, C):
    """Algorithmic work of one launch: (philox calls, bytes) for the kernel."""
    E, N, L, m = model_info["E"], model_info["N"], model_info["L"], model_info["m"]
    W = (m + 31) // 32
    calls_dual = E * C * math.ceil(m / 16)
    if name == "k_dual":
        return calls_dual, E * m * 4 + E * C * W * 4 + N * C
    if name == "k_primal" and model_info.get("partial"):
        # edge-partial form: the partial fields of every incidence, incidence records, unaries, labels
        return N * C, 2 * E * C * L * 4 + 2 * E * 8 + N * L * 4 + 2 * N * C + N * 8
    if name == "k_edge_partial":
        return 0, E * m * 4 + E * C * W * 4 + 2 * E * C * L * 4 + E * 4
    if name == "k_primal":
        return N * C, 2 * E * C * W * 4 + 2 * E * m * 4 + N * L * 8 + 2 * E * 8 + 2 * N * C + N * 16
    if name == "k_primal<fused>":
        return 2 * calls_dual + N * C, 2 * E * m * 4 + N * L * 8 + 2 * E * 8 + 2 * N * C
    if name == "k_accumulate":
        return 0, N * C + 2 * N * L * 4
    # Swendsen-Wang: one pass over the arrays every item touches (labels of
    # both endpoints per (edge, chain), the per-edge tables; ban word, label
    # and the unaries per (site, chain)); union-find walks, bonded sites' rows
    # and list traffic depend on the clusters and are not counted
    if name == "k_sw_bond":
        return 0, E * 8 + E * L * 12 + 2 * E * C
    if name == "k_sw_draw":
        return 0, N * C * (4 + 1) + N * L * 4
    return 0, 0


# DRAM bytes of the dual step per (edge, chain) item, from ncu counters of a
# smaller case of the same workload; traffic grows with the items, so it is
# scaled to the bench's launch.  Keyed by (entries per edge, chains).
# (49, 64): k_dual at 64^3, L = 8, 64 chains: 327.7 MB read + 349.7 MB written
# for 774,144 x 64 items.
DUAL_DRAM_BYTES_PER_ITEM = {(49, 64): (327740928 + 349712896) / (774144 * 64)}

# DRAM bytes of the batched workload's partial-field pass per live edge, from
# ncu counters of a 30-graph L = 16 batch (1,691,481 edges: 1,604.7 MB read +
# 208.9 MB written per launch); keyed by (entries per edge, chains).
EDGE_PARTIAL_DRAM_BYTES_PER_EDGE = {(225, 1): (1604725000 + 208856832) / 1691481}

# kernels behind one kernel-timing record of the library
KERNELS_PER_RECORD = {"k_sw_draw": 2}


def rank_seed(seed: int, rank: int) -> int:
    """Independent chains per rank: the draw key of rank r is seed + 1000003 r."""
    return seed + 1000003 * rank


def aggregate(ms_local: float, units_local: int, ws: int, device=None):
    """Whole-job throughput over ranks: the slowest rank's time and the sum of
    all ranks' units (replicas; the only collective is this timing reduction)."""
    if ws == 1:
        return ms_local, units_local / (ms_local / 1e3)
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local, float(units_local)], dtype=torch.float64, device=device)
    mx = t[:1].clone(); tot = t[1:].clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return float(mx.item()), float(tot.item()) / (float(mx.item()) / 1e3)


def run_ours(args, ws, rank, local):
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_1611_06684_gb300 import build as B
    if rank == 0:
        B.build()
    if ws > 1:
        torch.distributed.barrier()
    from paper_1611_06684_gb300 import mrf as M
    gen, C, desc = WORKLOADS[args.workload]
    if args.scale and args.workload == "potts3d":
        from paper_1611_06684_gb300 import workloads as wl
        model = wl.potts_grid3d(args.scale, L=8, seed=0)
        desc = desc.replace("128^3", f"{args.scale}^3")
    elif args.scale and args.workload == "ferro3d":
        from paper_1611_06684_gb300 import workloads as wl
        model = wl.ferro_potts_grid3d(args.scale, L=8, beta_lo=FERRO_BETA[0], beta_hi=FERRO_BETA[1],
                                      u_std=FERRO_U_STD, seed=0)
        desc = desc.replace("128^3", f"{args.scale}^3")
    else:
        model = gen()
    if "%g" in desc:
        desc = desc % (FERRO_BETA[0], FERRO_BETA[1], FERRO_U_STD)
    mode = {"plain": M.MODE_PLAIN, "fused": M.MODE_FUSED, "sw": M.MODE_SW, "higdon": M.MODE_HIGDON}[args.mode]
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        h = M.MRF(model.n_vars, model.n_labels, C, seed=rank_seed(args.seed, rank), stream=stream.cuda_stream,
                  grid=model.grid if model.grid else None)
        h.set_factors(model.unary, model.src, model.dst, model.pair)
    h.set_higdon(args.higdon_rho)
    inf = h.info()
    minfo = dict(E=inf.n_edge_slots, N=inf.n_vars, L=inf.n_labels, m=inf.n_entries)
    # warm-up (the first plain sweep also runs the primal-schedule autotuner)
    h.sweep(args.warmup, mode)
    torch.cuda.synchronize()
    clk_path = os.path.join(tempfile.gettempdir(), f"bench_clocks_{rank}.csv")
    clk = clocks_start(clk_path)
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # timed region: the product path, every sweep one replay of its captured CUDA graph
    ev0.record(stream)
    h.sweep(args.steps, mode)
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ms_total = ev0.elapsed_time(ev1)
    clocks = clocks_stop(clk, clk_path, local)
    ms_total, value = aggregate(ms_total, C * model.n_vars * args.steps, ws, dev)
    ms_step = ms_total / args.steps
    # per-kernel split: the same sweeps again with CUDA events around every
    # launch on the handle's stream (graph replay off while timing kernels)
    h.set_kernel_timing(True)
    h.kernel_times()
    k_split = max(3, min(args.steps, 20))
    h.sweep(k_split, mode)
    ktimes = h.kernel_times()
    h.set_kernel_timing(False)
    # launches per sweep of the library's kernels (+ k_advance, which is not timed),
    # counted in the split run; the graph of a sweep replays the same launches
    if "k_sweep_small" in ktimes or "k_sw_small" in ktimes:
        launches = 1                              # a small model runs all sweeps of a call in one launch
    else:
        per_sweep = sum(n * KERNELS_PER_RECORD.get(k, 1) for k, (_, n) in ktimes.items()) / k_split + 1
        launches = int(round(per_sweep * args.steps))

    # roofline of the dominant kernel (device time from the per-kernel split run)
    peaks, peak_src = load_peaks()
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    dom_ms = ktimes[dom][0] / ktimes[dom][1]
    if dom == "k_sweep_small":                   # one launch = all sweeps of the call
        cd, bd = kernel_work("k_dual", minfo, C)
        cp, bp = kernel_work("k_primal", minfo, C)
        calls, nbytes = (cd + cp) * k_split, (bd + bp) * k_split
    elif dom == "k_sw_small":
        calls = 0
        nbytes = (kernel_work("k_sw_bond", minfo, C)[1] + kernel_work("k_sw_draw", minfo, C)[1]) * k_split
    else:
        calls, nbytes = kernel_work(dom, minfo, C)
    sm_mhz = clocks["sm_mhz"] if clocks else peaks.get("sm_max_mhz", 2070.0)
    hbm = {"bound": "hbm", "achieved": nbytes / (dom_ms / 1e3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    hbm["frac"] = hbm["achieved"] / hbm["peak"]
    try:
        philox_measured = M.philox_rate(stream=stream.cuda_stream)
    except Exception:
        philox_measured = None
    if calls and dom in ("k_dual", "k_primal<fused>", "k_sweep_small"):
        alu_peak = alu_peak_philox_calls(peaks.get("sm_max_mhz", 2070.0))
        per_item = DUAL_DRAM_BYTES_PER_ITEM.get((minfo["m"], C)) if dom == "k_dual" else None
        roof = {"bound": "alu", "achieved": calls / (dom_ms / 1e3) / 1e9, "peak": alu_peak / 1e9,
                "unit": "G Philox4x32-10 calls/s", "frac": calls / (dom_ms / 1e3) / alu_peak,
                "traffic": per_item * minfo["E"] * C if per_item else None,
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of k_dual at "
                                   "64^3, scaled by edge x chain items") if per_item else None,
                "kernel": dom, "peak_source": "derived: 152 SMs x 4 SMSPs x 32 lanes x 2070 MHz / 61.5 fmaheavy-pipe cycles per warp-wide call (ncu counters of the Philox-only kernel)",
                "hbm_view": {k: hbm[k] for k in ("achieved", "peak", "unit", "frac")},
                "philox_only_kernel": {"calls_per_s": philox_measured,
                                       "frac": (calls / (dom_ms / 1e3) / philox_measured) if philox_measured else None}}
    else:
        roof = dict(hbm, traffic=None, kernel=dom, peak_source=f"MEASURED_PEAKS.json hbm_gbs ({peak_src})")

    # other sweep forms on the same handle, timed separately (not part of the headline)
    variants = {}
    if not args.no_variants:
        # the Swendsen-Wang form exists for two labels and Potts-type tables with l >= 0
        try:
            h.sweep(1, M.MODE_SW)
            sw_ok = True
        except M.MrfError:
            sw_ok = False
        forms = [(n, md) for n, md in (("plain", M.MODE_PLAIN), ("fused", M.MODE_FUSED)) if n != args.mode] + \
            ([("splash", M.MODE_SPLASH)] if model.grid else []) + \
            ([("sw", M.MODE_SW)] if sw_ok and args.mode != "sw" else []) + \
            ([("higdon", M.MODE_HIGDON)] if sw_ok and args.mode != "higdon" else [])
        for name, md in forms:
            h.sweep(1, md)
            torch.cuda.synchronize()
            kv = 5
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.sweep(kv, md)
            e1.record(stream)
            torch.cuda.synchronize()
            msv = e0.elapsed_time(e1) / kv
            h.set_kernel_timing(True)
            h.kernel_times()
            h.sweep(kv, md)
            kt = h.kernel_times()
            h.set_kernel_timing(False)
            variants[name] = {"ms_per_step": msv, "value": C * model.n_vars / (msv / 1e3), "unit": METRIC,
                              "kernels": {k: v[0] / v[1] for k, v in kt.items()}}
        if model.grid:
            # log-partition estimator of Section 5.2 (plain sweeps recording log p of the drawn labels)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lv = h.estimate_log_partition(5)
            dt = (time.perf_counter() - t0) / 5
            w = np.exp(lv - lv.max())
            variants["log_partition"] = {
                "sweeps": 5, "chains": C, "ms_per_sweep_wall": dt * 1e3,
                "mean_log_v": float(lv.mean()), "log_mean_exp_v": float(lv.max() + np.log(w.mean())),
                "lower_bound_per_site": float(lv.mean() / model.n_vars),
                "note": "mean of log V is a lower bound on log Z (Section 5.2); chains after the timed sweeps"}
        if args.ess_sweeps > 0:
            ms_of = {args.mode: ms_step}
            ms_of.update({k: v["ms_per_step"] for k, v in variants.items() if "ms_per_step" in v})
            variants["ess_fixed_sweeps"] = ess_comparison(
                h, model, C, stream, args.ess_sweeps, ms_of,
                [("plain", M.MODE_PLAIN)] + ([("splash", M.MODE_SPLASH)] if model.grid else [])
                + ([("sw", M.MODE_SW), ("higdon", M.MODE_HIGDON)] if sw_ok else []))
        if args.tv_ref_sweeps > 0 and args.workload in ("potts3d", "ferro3d"):
            from paper_1611_06684_gb300 import workloads as wl
            n = args.tv_scale
            if args.workload == "potts3d":
                tvm = wl.potts_grid3d(n, L=8, seed=0)
            else:
                tvm = wl.ferro_potts_grid3d(n, L=8, beta_lo=FERRO_BETA[0], beta_hi=FERRO_BETA[1],
                                            u_std=FERRO_U_STD, seed=0)
            tv_forms = [("plain", [M.MODE_PLAIN]), ("fused", [M.MODE_FUSED]), ("splash", [M.MODE_SPLASH])] + \
                ([("sw", [M.MODE_SW]), ("higdon", [M.MODE_HIGDON])] if sw_ok else [])
            variants["ess"] = tv_protocol(tvm, C, stream, tv_forms, args.seed + 17, args.tv_ref_sweeps,
                                          workload=_describe(args.workload).replace("128^3", f"{n}^3"))
            if args.workload == "potts3d":
                # the target comparisons: the learned proposal and the batched launch
                # against the plain dual sweep, each in ESS/s at marginal TV <= 0.01
                variants["ess"]["learned"] = learned_tv_comparison(stream, args.tv_ba_sites, 512, args.seed + 23,
                                                                   args.tv_ba_ref_sweeps)
                variants["ess"]["batched"] = small_batch_tv_comparison(stream, args.tv_batch_graphs, C, args.seed + 29)
                variants["ess"]["batched_er"] = batch_tv_comparison(stream, 20, C, args.seed + 31, 50000,
                                                                    tv_target=0.0)
                variants["ess"]["targets"] = {
                    "learned_vs_plain": variants["ess"]["learned"]["versus_plain"]["learned"],
                    "learned+plain_vs_plain": variants["ess"]["learned"]["versus_plain"]["learned+plain"],
                    "batched_vs_plain_at_tv": variants["ess"]["batched"]["versus_plain"]["batched"],
                    "batched_vs_plain_er_family": variants["ess"]["batched_er"]["versus_plain"]["batched"]}
            variants["ess"]["versus_plain"] = versus_plain(variants["ess"], [n for n, _ in tv_forms if n != "plain"])

    # end to end through the C ABI with pinned host buffers: labels in, sweep, labels out
    e2e = None
    if not args.no_e2e:
        x_host = torch.empty((C, model.n_vars), dtype=torch.uint8).pin_memory()
        h.get_labels_into(x_host)
        h2 = M.MRF(model.n_vars, model.n_labels, C, seed=args.seed + 1000003 * rank, stream=stream.cuda_stream)
        with torch.cuda.stream(stream):
            h2.set_factors(model.unary, model.src, model.dst, model.pair)
        k_e2e = max(3, min(args.steps, 20))
        h2.set_labels(x_host); h2.sweep(1, mode); h2.get_labels_into(x_host)     # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            h2.set_labels(x_host)
            h2.sweep(1, mode)
            h2.get_labels_into(x_host)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if ws > 1:
            t = torch.tensor([dt], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": ws * C * model.n_vars * k_e2e / dt, "unit": METRIC,
               "h2d_bytes_per_step": C * model.n_vars, "d2h_bytes_per_step": C * model.n_vars,
               "steps": k_e2e, "api": "mrf_set_labels(host) + mrf_sweep(1) + mrf_get_labels(host), pinned buffers"}
        h2.close()

    out = None
    if rank == 0:
        cpu = None if (ws > 1 or args.no_cpu) else cpu_baseline(args, args.cpu_seconds)
        out = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32+f32 (dual step: u32 Philox and threshold compare; primal step: f32 with two-sum accumulation)",
            "data": "synthetic (seeded generators)",
            "config": {"workload": args.workload, "description": desc, "n_vars": model.n_vars,
                       "n_edges": model.n_edges, "n_labels": model.n_labels, "chains": C, "mode": args.mode,
                       "dual_bits_per_edge": inf.n_entries, "layout": ["pivot", "diag"][inf.layout],
                       "l2": "inputs larger than L2 (tables and theta are GBs); no flush needed",
                       "parallelism": f"replicas x{ws} (independent chains per GPU)"},
            "roofline": roof,
            "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches": v[1]} for k, v in ktimes.items()},
            "gpu_launches": launches,
            "variants": variants,
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
    h.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return out


class OracleSample:
    """The oracle, as it stands, on a bounded sample of the workload."""

    def __init__(self, args):
        from paper_1611_06684_gb300 import workloads as wl
        from oracle import decompose as dc, philox as ph
        if args.workload == "potts3d":
            self.C = 2
            model = wl.potts_grid3d(24, L=8, seed=0)
            self.sample = "{C} chains x {S} sweeps of a 24^3 sub-lattice with the same L=8 table and unary distributions"
        elif args.workload == "ferro3d":
            self.C = 2
            model = wl.ferro_potts_grid3d(24, L=8, beta_lo=FERRO_BETA[0], beta_hi=FERRO_BETA[1], u_std=FERRO_U_STD,
                                          seed=0)
            self.sample = "{C} chains x {S} sweeps of a 24^3 sub-lattice with the same L=8 coupling and unary distributions"
        elif args.workload == "dense4096":
            self.C = 1
            model = wl.dense_potts(256, L=4, w_std=0.2 / 64, seed=0)
            self.sample = "{C} chain x {S} sweeps of a N=256 fully connected model with the same L=4 distributions"
        elif args.workload == "er_batch":
            self.C = 1
            ms = [wl.er_graph(sp) for sp in wl.er_batch_specs(args.scale or 2000, seed=0)[:4]]
            self.parts = [(dc.decompose(m), ph.init_labels(m.n_vars, m.n_labels, 1, args.seed)) for m in ms]
            self.n_sites = sum(m.n_vars for m in ms)
            self.sample = "{C} chain x {S} sweeps of the first 4 of the batch's graphs (%d sites)" % self.n_sites
            self.mode, self.seed, self.t = "batch", args.seed, 0
            return
        else:
            self.C = 1
            model = WORKLOADS[args.workload][0]()
            self.sample = "{C} chain x {S} sweeps of the full workload"
        self.model = model
        self.dec = dc.decompose(model)
        self.mode = args.mode
        self.higdon_rho = args.higdon_rho
        self.sw_tables = None
        self.seed = args.seed
        self.x = ph.init_labels(model.n_vars, model.n_labels, self.C, args.seed)
        self.t = 0

    def sweep(self):
        """One oracle sweep; returns its wall time in seconds."""
        from oracle import sampler, swendsen_wang
        t0 = time.perf_counter()
        if self.mode == "batch":
            self.parts = [(d, sampler.sweep(d, x, self.t, self.seed)["x"]) for d, x in self.parts]
        elif self.mode == "sw":
            if self.sw_tables is None:
                self.sw_tables = swendsen_wang.sw_tables(self.model)
            self.x = swendsen_wang.sw_sweep(self.model, self.x, self.t, self.seed, tables=self.sw_tables)["x"]
        elif self.mode == "higdon":
            from oracle import higdon
            if self.sw_tables is None:
                self.sw_tables = higdon.higdon_split(self.model, self.higdon_rho)
            self.x = higdon.higdon_sweep(self.model, self.x, self.higdon_rho, self.t, self.seed,
                                         split=self.sw_tables)["x"]
        else:
            self.x = sampler.sweep(self.dec, self.x, self.t, self.seed)["x"]
        self.t += 1
        return time.perf_counter() - t0

    @property
    def units_per_sweep(self):
        return self.C * (self.n_sites if self.mode == "batch" else self.model.n_vars)


def openmp_baseline(args, budget_s=10.0):
    """The float32 OpenMP statement of the sweep (oracle/cpu_sweep.c) on every
    core this process may run on, on a bounded sample of the workload."""
    from paper_1611_06684_gb300 import workloads as wl
    from oracle import cpu_sweep, decompose as dc, philox as ph
    cores = len(os.sched_getaffinity(0))
    if args.workload == "potts3d":
        n, C = 40, 64
        model = wl.potts_grid3d(n, L=8, seed=0)
        sample = f"{C} chains x {{S}} sweeps of a {n}^3 sub-lattice with the same L=8 table and unary distributions"
    elif args.workload == "ferro3d":
        n, C = 40, 64
        model = wl.ferro_potts_grid3d(n, L=8, beta_lo=FERRO_BETA[0], beta_hi=FERRO_BETA[1], u_std=FERRO_U_STD, seed=0)
        sample = f"{C} chains x {{S}} sweeps of a {n}^3 sub-lattice with the same L=8 coupling and unary distributions"
    elif args.workload == "dense4096":
        C = 16
        model = wl.dense_potts(1024, L=4, w_std=0.2 / 64, seed=0)
        sample = f"{C} chains x {{S}} sweeps of a N=1024 fully connected model with the same L=4 distributions"
    else:
        C = WORKLOADS[args.workload][1]
        model = WORKLOADS[args.workload][0]()
        sample = f"{C} chain(s) x {{S}} sweeps of the full workload"
    dec = dc.decompose(model)
    cs = cpu_sweep.CpuSweep(dec, C, args.seed, threads=cores)
    x = ph.init_labels(model.n_vars, model.n_labels, C, args.seed).astype(np.uint8)
    x = cs.sweep(x, 0)                                   # warm-up (first touch of the workspace)
    el, S = 0.0, 0
    while el < budget_s:
        t0 = time.perf_counter()
        x = cs.sweep(x, S + 1)
        el += time.perf_counter() - t0
        S += 1
    return {"value": C * model.n_vars * S / el, "unit": METRIC, "cores": cores,
            "kind": "oracle (float32 OpenMP statement of the sweep, oracle/cpu_sweep.c)",
            "sample": sample.format(S=S), "seconds": el}


def cpu_baseline(args, budget_s=10.0):
    """CPU baselines: the float32 OpenMP sweep on every available core (the
    line's value) and the float64 numpy oracle on one core beside it."""
    o = OracleSample(args)
    el, S = 0.0, 0
    while el < budget_s:
        el += o.sweep(); S += 1
    single = {"value": o.units_per_sweep * S / el, "unit": METRIC, "cores": 1, "kind": "oracle (float64 numpy)",
              "sample": o.sample.format(C=o.C, S=S), "seconds": el}
    try:
        multi = openmp_baseline(args, budget_s)
    except Exception as exc:                 # no gcc / OpenMP on the host
        multi = None
        single["openmp_unavailable"] = f"{type(exc).__name__}: {exc}"
    out = dict(multi) if multi else dict(single)
    out["host_cores_available"] = len(os.sched_getaffinity(0))
    out["single_core_oracle"] = single
    return out


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    o = OracleSample(args)
    for _ in range(args.warmup):
        o.sweep()
    secs = [o.sweep() for _ in range(args.steps)]
    mean_s = statistics.mean(secs)
    value = o.units_per_sweep / mean_s
    sample = o.sample.format(C=o.C, S=1) + " per step"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generators)",
            "config": {"workload": args.workload, "description": _describe(args.workload), "mode": args.mode,
                       "reference": "CPU float64 oracle (oracle/), one bounded-sample sweep per step"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": value, "unit": METRIC},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _timed(stream, fn):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def batch_cpu_baseline(models, seed, budget_s=10.0):
    """CPU baselines of the batched workload on a bounded sample: the float32
    OpenMP sweep (all cores) over the class unions of the sample's graphs, and
    the float64 numpy oracle (one core) beside it."""
    from oracle import cpu_sweep, decompose as dc, philox as ph, sampler
    cores = len(os.sched_getaffinity(0))
    sample = models[:40]
    unions = []
    for L in sorted(set(m.n_labels for m in sample)):
        ms = [m for m in sample if m.n_labels == L]
        off = np.cumsum([0] + [m.n_vars for m in ms])[:-1]
        from paper_1611_06684_gb300 import workloads as wl
        unions.append(wl.Model(int(sum(m.n_vars for m in ms)), L, np.concatenate([m.unary for m in ms]),
                               np.concatenate([m.src + o for m, o in zip(ms, off)]).astype(np.int32),
                               np.concatenate([m.dst + o for m, o in zip(ms, off)]).astype(np.int32),
                               np.concatenate([m.pair for m in ms])))
    n_sites = sum(u.n_vars for u in unions)
    decs = [dc.decompose(u) for u in unions]
    sweeps = [cpu_sweep.CpuSweep(d, 1, seed, threads=cores) for d in decs]
    xs = [ph.init_labels(u.n_vars, u.n_labels, 1, seed).astype(np.uint8) for u in unions]
    xs = [cs.sweep(x, 0) for cs, x in zip(sweeps, xs)]
    el, S = 0.0, 0
    while el < budget_s:
        t0 = time.perf_counter()
        xs = [cs.sweep(x, S + 1) for cs, x in zip(sweeps, xs)]
        el += time.perf_counter() - t0
        S += 1
    multi = {"value": n_sites * S / el, "unit": METRIC, "cores": cores,
             "kind": "oracle (float32 OpenMP statement of the sweep, oracle/cpu_sweep.c)",
             "sample": f"{len(sample)} of the graphs ({n_sites} sites, their class unions), 1 chain x {S} sweeps",
             "seconds": el}
    small = models[:4]
    xo = [ph.init_labels(m.n_vars, m.n_labels, 1, seed) for m in small]
    do = [dc.decompose(m) for m in small]
    el1, S1 = 0.0, 0
    while el1 < budget_s:
        t0 = time.perf_counter()
        xo = [sampler.sweep(d, x, S1, seed)["x"] for d, x in zip(do, xo)]
        el1 += time.perf_counter() - t0
        S1 += 1
    multi["single_core_oracle"] = {"value": sum(m.n_vars for m in small) * S1 / el1, "unit": METRIC, "cores": 1,
                                   "kind": "oracle (float64 numpy)",
                                   "sample": f"{len(small)} of the graphs, 1 chain x {S1} sweeps", "seconds": el1}
    multi["host_cores_available"] = cores
    return multi


def run_batch_workload(args):
    """Batched dynamic workload: many Erdos-Renyi graphs (sizes logU[100, 50000],
    mean degree U[3, 20], L in {2,4,8,16}, tables exp(U[-0.5, 0.5])), one chain
    each.  A step is one round: an edit (remove ceil(1%) of every graph's edges,
    add as many with fresh tables) applied by the device edit queue, then 10
    sweeps, replayed as one CUDA graph.  The edit's inputs are resident in
    device memory when the timed region starts (the end-to-end figure copies
    them from pinned host memory and reads the added edges' slots back)."""
    import torch
    from paper_1611_06684_gb300 import build as B, mrf as M, workloads as wl
    B.build()
    n_graphs = args.scale or 2000
    labels = tuple(int(v) for v in args.er_labels.split(","))
    specs = wl.er_batch_specs(n_graphs, labels=labels, seed=0)
    t0 = time.time()
    models = [wl.er_graph(sp) for sp in specs]
    gen_s = time.time() - t0
    stream = torch.cuda.Stream()
    C = 1
    b = M.MRFBatch([m.n_vars for m in models], [m.n_labels for m in models], C, seed=args.seed,
                   stream=stream.cuda_stream, use_graphs=True)
    b.set_factors(models)
    N = sum(m.n_vars for m in models)
    E = sum(m.n_edges for m in models)
    ed = wl.ErBatchEdits(models, [b.graph(g).first_edge_slot for g in range(n_graphs)], seed=1)
    k = ed.counts(0.01)
    n_edit = int(k.sum())
    L_g = np.array([m.n_labels for m in models], np.int64)
    pair_max = int((k * L_g * L_g).sum())
    b.queue_create(n_edit, n_edit, pair_max, extra_slots=1024)
    sweeps_per_round = 10
    dev = torch.device("cuda", torch.cuda.current_device())

    def staged(arrays, where):
        if where == "device":
            return [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in arrays]
        return [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in arrays]

    def one_round(where, timed_list, e2e_list=None):
        arrays = ed.edit(0.01)                                   # untimed: draw the edit on the host
        st = staged(arrays, where)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        e0.record(stream)
        b.queue_load(*st)
        b.round(sweeps_per_round)
        e1.record(stream)
        status, slots = b.queue_result(len(arrays[3]))           # device -> host: status and the new slots
        w1 = time.perf_counter()
        if status != 0:
            raise RuntimeError(f"queue round rejected its edit: status {status}")
        timed_list.append(e0.elapsed_time(e1))
        if e2e_list is not None:
            e2e_list.append((w1 - w0, sum(a.nbytes for a in arrays), 8 * len(slots) + 4))
        ed.apply(slots)

    warm = []
    for _ in range(args.warmup):
        one_round("device", warm)
    clk_path = os.path.join(tempfile.gettempdir(), "bench_clocks_batch.csv")
    clk = clocks_start(clk_path)
    time.sleep(0.3)
    times = []
    for _ in range(args.steps):
        one_round("device", times)
    clocks = clocks_stop(clk, clk_path, torch.cuda.current_device())
    ms_round = float(np.mean(times))
    value = N * C * sweeps_per_round / (ms_round / 1e3)
    # end to end: the edit's arrays from pinned host memory, the slots read back
    e2e_rounds, e2e_ms = [], []
    for _ in range(max(3, min(args.steps, 5))):
        one_round("host", e2e_ms, e2e_rounds)
    e2e = {"value": N * C * sweeps_per_round * len(e2e_rounds) / sum(r[0] for r in e2e_rounds), "unit": METRIC,
           "h2d_bytes_per_step": int(np.mean([r[1] for r in e2e_rounds])),
           "d2h_bytes_per_step": int(np.mean([r[2] for r in e2e_rounds])), "steps": len(e2e_rounds),
           "api": "mrf_batch_queue_load(pinned host arrays) + mrf_batch_round(10) + mrf_batch_queue_result"}
    # sweeps alone, and the per-kernel split of one sweep of every class (CUDA events)
    ms_sweep = _timed(stream, lambda: b.sweep(sweeps_per_round, M.MODE_PLAIN)) / sweeps_per_round
    b.set_kernel_timing(True)
    for kk in range(b.n_classes()):
        b.class_handle(kk).kernel_times()
    b.sweep(3, M.MODE_PLAIN)
    torch.cuda.synchronize()
    per_class, dom = [], None
    for kk in range(b.n_classes()):
        hk = b.class_handle(kk)
        inf = hk.info()
        raw = hk.kernel_times()
        kt = {n: v[0] / v[1] for n, v in raw.items()}
        row = {"L": hk.L, "sites": hk.N, "edges": int(inf.n_edges), "edge_slots": int(inf.n_edge_slots),
               "dual_bits_per_edge": int(inf.n_entries), "kernels_ms": kt,
               "launches_per_sweep": sum(v[1] for v in raw.values()) / 3 + 1,          # + k_advance (not timed)
               "two_label_unaries": hk.L == 2}
        per_class.append(row)
        for name, ms in kt.items():
            if dom is None or ms > dom[2]:
                dom = (row, name, ms)
    b.set_kernel_timing(False)
    # the host-side edit of the same size, for comparison (one round)
    arrays = ed.edit(0.01)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    slots = b.edit_factors(*arrays)
    torch.cuda.synchronize()
    host_edit_s = time.perf_counter() - t1
    ed.apply(slots)
    peaks, peak_src = load_peaks()
    row, name, dom_ms = dom
    minfo = dict(E=row["edges"], N=row["sites"], L=row["L"], m=row["dual_bits_per_edge"],
                 partial=C <= 4 and row["dual_bits_per_edge"] >= 100)
    _, nbytes = kernel_work(name, minfo, C)
    per_edge = EDGE_PARTIAL_DRAM_BYTES_PER_EDGE.get((row["dual_bits_per_edge"], C)) if name == "k_edge_partial" else None
    roof = {"bound": "hbm", "achieved": nbytes / (dom_ms / 1e3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "traffic": per_edge * row["edges"] if per_edge else None,
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of k_edge_partial on a 30-graph "
                               "L = 16 batch, scaled by live edges") if per_edge else None,
            "kernel": f"{name} (class L={row['L']})", "bytes_per_launch": nbytes,
            "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # the whole sweep against the method's own minimum (each class's tables read once, labels, incidence lists)
    sweep_bytes = sum(r["edges"] * r["dual_bits_per_edge"] * 4 + r["edges"] * 24 + r["sites"] * (r["L"] * 4 + 2 * C)
                      for r in per_class)
    roof["sweep_view"] = {"bytes_per_sweep": sweep_bytes, "ms_per_sweep": ms_sweep,
                          "achieved": sweep_bytes / (ms_sweep / 1e3) / 1e9,
                          "frac": sweep_bytes / (ms_sweep / 1e3) / 1e9 / peaks["hbm_gbs"],
                          "counted": "tables once (4 B per dual entry), endpoints (8 B) and two incidence records "
                                     "(16 B) per edge, unaries (4 B per label) and labels in and out per site"}
    K = b.n_classes()
    # the edit: route (4 kernels), per class 15 (remove, slot rule 3, place, decomposition, planes, incidence
    # lists 6, long lists, refold) and one more where Swendsen-Wang unaries exist, finish (1); then the sweeps
    launches_per_round = int(round(4 + sum(15 + r["two_label_unaries"] for r in per_class) + 1
                                   + sweeps_per_round * sum(r["launches_per_sweep"] for r in per_class)))
    cpu = None if args.no_cpu else batch_cpu_baseline(models, args.seed, args.cpu_seconds)
    return {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_round, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "u32+f32 (dual step: u32 Philox and threshold compare; primal step: f32 with two-sum accumulation)",
            "data": "synthetic (seeded generators)",
            "config": {"workload": f"er_batch_{n_graphs}" + ("" if labels == (2, 4, 8, 16) else f"_L{args.er_labels}"),
                       "description": f"{n_graphs} Erdos-Renyi graphs, N ~ logU[100, 50000], mean degree U[3, 20], "
                                      f"L in {set(labels)}, tables exp(U[-0.5,0.5]), unaries N(0,1), 1 chain each",
                       "n_vars": N, "n_edges": E, "graphs": n_graphs, "chains": C,
                       "step": "one round: edit (remove ceil(1%) of every graph's edges, add as many) + 10 sweeps, "
                               "one CUDA graph replay",
                       "edges_edited_per_round": n_edit,
                       "l2": "inputs larger than L2 (tables are tens of GB); no flush needed",
                       "parallelism": "one GPU"},
            "roofline": roof, "gpu_launches": launches_per_round * args.steps,
            "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
            "sweep_only": {"ms_per_sweep": ms_sweep, "value": N * C / (ms_sweep / 1e3)},
            "edit_in_round_ms": ms_round - sweeps_per_round * ms_sweep,
            "host_edit_ms": host_edit_s * 1e3,
            "classes": per_class, "generation_s": gen_s}


def ess_sum_over_chains(trace):
    """Sum over chains of the effective sample size of a [T][C] trace, each
    chain by Geyer's initial monotone sequence estimator (Geyer 1992): pairs of
    consecutive autocovariances (by FFT) up to the first non-positive pair,
    made non-increasing; ESS = T / (-1 + 2 sum(pairs) / gamma_0)."""
    y = np.asarray(trace, np.float64)
    y = y - y.mean(axis=0)
    T = y.shape[0]
    f = np.fft.rfft(y, n=2 * T, axis=0)
    acov = np.fft.irfft(f * np.conj(f), n=2 * T, axis=0)[:T] / T
    total = 0.0
    for c in range(y.shape[1]):
        g = acov[:, c]
        m = T // 2
        pairs = g[0:2 * m:2] + g[1:2 * m:2]
        nonpos = np.nonzero(pairs <= 0)[0]
        k = int(nonpos[0]) if nonpos.size else m
        if g[0] <= 0 or k == 0:
            total += T
            continue
        tau = -1.0 + 2.0 * np.minimum.accumulate(pairs[:k]).sum() / g[0]
        total += T / max(tau, 1e-12)
    return float(total)


def ess_comparison(h, model, C, stream, T, ms_of, forms, n_sites=4096, n_edges=50000):
    """ESS/s of sweep forms on one handle from a common start: per chain, the
    fraction of label 0 over n_sites fixed sites, their unary energy, and the
    pairwise energy of n_edges fixed edges, traced every sweep on the device
    (labels copied device to device, statistics reduced by torch).  ESS/s =
    min over statistics of the ESS summed over chains / (T x ms per sweep)."""
    import torch
    from paper_1611_06684_gb300 import mrf as M
    dev = torch.device("cuda", torch.cuda.current_device())
    rng = np.random.default_rng(12345)
    sites = torch.as_tensor(np.sort(rng.choice(model.n_vars, size=min(n_sites, model.n_vars), replace=False)),
                            device=dev)
    esel = np.sort(rng.choice(model.n_edges, size=min(n_edges, model.n_edges), replace=False))
    es = torch.as_tensor(model.src[esel].astype(np.int64), device=dev)
    et = torch.as_tensor(model.dst[esel].astype(np.int64), device=dev)
    w = torch.as_tensor(model.pair[esel], device=dev)
    u = torch.as_tensor(model.unary, device=dev)
    ar = torch.arange(len(esel), device=dev)
    x = torch.empty((C, model.n_vars), dtype=torch.uint8, device=dev)
    h.get_labels_into(x)
    torch.cuda.synchronize()
    x_start = x.clone()
    t_start = h.info().sweep_index
    out = {}
    for name, md in forms:
        if ms_of.get(name) is None:
            continue
        h.set_labels(x_start)
        h.set_sweep_index(t_start + 7919)
        stats = torch.empty((3, T, C), dtype=torch.float64, device=dev)
        for t in range(T):
            h.sweep(1, md)
            with torch.cuda.stream(stream):
                h.get_labels_into(x)
                xl = x.long()
                xs = xl[:, sites]
                stats[0, t] = (xs == 0).double().mean(dim=1)
                stats[1, t] = u[sites[None, :], xs].double().sum(dim=1)
                stats[2, t] = w[ar[None, :], xl[:, es], xl[:, et]].double().sum(dim=1)
        torch.cuda.synchronize()
        tr = stats.cpu().numpy()
        ess = {k: ess_sum_over_chains(tr[i]) for i, k in enumerate(("label0_fraction", "unary_energy", "pair_energy"))}
        ms = ms_of[name]
        out[name] = {"ess": ess, "ess_min": min(ess.values()), "ms_per_sweep": ms,
                     "ess_per_s": min(ess.values()) / (T * ms / 1e3)}
    out["sweeps"] = T
    out["statistics"] = (f"per chain: label-0 fraction and unary energy of {len(sites)} fixed sites, pairwise "
                         f"energy of {len(esel)} fixed edges; ESS summed over chains, min over statistics")
    return out


def _stat_recorder(model, C, dev, n_sites=4096, n_edges=50000, seed=12345):
    """Per-chain statistics of a labelling on the device: the fraction of label
    0 over fixed sites, their unary energy and the pairwise energy of fixed
    edges.  Returns (labels buffer [C][N] uint8 on the device, fn(out[3][C]))."""
    import torch
    rng = np.random.default_rng(seed)
    sites = torch.as_tensor(np.sort(rng.choice(model.n_vars, size=min(n_sites, model.n_vars), replace=False)),
                            device=dev)
    esel = np.sort(rng.choice(model.n_edges, size=min(n_edges, model.n_edges), replace=False))
    es = torch.as_tensor(model.src[esel].astype(np.int64), device=dev)
    et = torch.as_tensor(model.dst[esel].astype(np.int64), device=dev)
    w = torch.as_tensor(model.pair[esel], device=dev)
    u = torch.as_tensor(model.unary, device=dev)
    ar = torch.arange(len(esel), device=dev)
    x = torch.empty((C, model.n_vars), dtype=torch.uint8, device=dev)

    def record(out):
        xl = x.long()
        xs = xl[:, sites]
        out[0] = (xs == 0).double().mean(dim=1)
        out[1] = u[sites[None, :], xs].double().sum(dim=1)
        out[2] = w[ar[None, :], xl[:, es], xl[:, et]].double().sum(dim=1)
    desc = (f"per chain: label-0 fraction and unary energy of {len(sites)} fixed sites, pairwise energy of "
            f"{len(esel)} fixed edges; ESS summed over chains, min over statistics")
    return x, record, desc


def tv_protocol(model, C, stream, forms, seed, ref_sweeps, tv_target=0.01, chunk=25, burn=300, workload="",
                handle=None, ref_chains=None, budget=None):
    """ESS/s at equal marginal accuracy.  From a common state after `burn`
    plain sweeps: a reference run of `ref_sweeps` plain sweeps gives reference
    marginals (label counts of every chain and sweep); then every form runs
    from the same state with fresh counts until the mean-site total-variation
    distance of its marginals to the reference is <= tv_target (checked every
    `chunk` sweeps, at most ref_sweeps / 100 sweeps, so the reference always
    has at least 100 times the samples).  A form is (name, [modes]); its
    sweeps cycle through the modes.  Reported per form: sweeps and seconds to
    the target (seconds = sweeps x the form's per-sweep time by CUDA events
    over graph replays), the ESS of the run up to there (minimum over the
    statistics of _stat_recorder, summed over chains) and ESS/s.  `handle`:
    an MRF handle of `model` already set up (else one is created).  With
    `ref_chains` the reference runs on a separate handle with that many
    chains (each sweep then gives ref_chains / C times the samples), and
    `budget` caps the sweeps per form at (reference samples) / (100 C)."""
    import torch
    from paper_1611_06684_gb300 import mrf as M
    dev = torch.device("cuda", torch.cuda.current_device())
    h = handle
    if h is None:
        with torch.cuda.stream(stream):
            h = M.MRF(model.n_vars, model.n_labels, C, seed=seed, stream=stream.cuda_stream,
                      grid=model.grid if model.grid else None)
            h.set_factors(model.unary, model.src, model.dst, model.pair)
    h.sweep(burn, M.MODE_PLAIN)
    x_start = h.get_labels()
    t_start = h.info().sweep_index
    ms_of = {}
    for name, modes in forms:
        for md in modes:
            h.sweep(2, md)
        per = {md: _timed(stream, lambda: h.sweep(20, md)) / 20 for md in set(modes)}
        ms_of[name] = sum(per[md] for md in modes) / len(modes)
    if ref_chains is None or ref_chains == C:
        hr, rc = h, C
        hr.set_labels(x_start)
        hr.set_sweep_index(t_start + 7)
    else:
        rc = ref_chains
        with torch.cuda.stream(stream):
            hr = M.MRF(model.n_vars, model.n_labels, rc, seed=seed + 99991, stream=stream.cuda_stream,
                       grid=model.grid if model.grid else None)
            hr.set_factors(model.unary, model.src, model.dst, model.pair)
        hr.sweep(burn, M.MODE_PLAIN)
    hr.reset_marginals(0)
    t0 = time.perf_counter()
    hr.sweep(ref_sweeps, M.MODE_PLAIN)
    torch.cuda.synchronize()
    ref_s = time.perf_counter() - t0
    ref, n_ref = hr.marginals()
    if hr is not h:
        hr.close()
    cap = (ref_sweeps * rc) // (100 * C)
    budget = cap if budget is None else min(budget, cap)
    xbuf, record, stat_desc = _stat_recorder(model, C, dev)
    out = {}
    for k, (name, modes) in enumerate(forms):
        h.set_labels(x_start)
        h.set_sweep_index(t_start + 1000003 * (k + 1))
        h.reset_marginals(0)
        stats = torch.empty((3, budget, C), dtype=torch.float64, device=dev)
        swept, reached, tv = 0, None, None
        while swept < budget:
            for t in range(min(chunk, budget - swept)):
                h.sweep(1, modes[(swept + t) % len(modes)])
                with torch.cuda.stream(stream):
                    h.get_labels_into(xbuf)
                    record(stats[:, swept + t])
            swept += min(chunk, budget - swept)
            est, _ = h.marginals()
            tv = tv_mean(est, ref)
            if tv <= tv_target:
                reached = swept
                break
        torch.cuda.synchronize()
        tr = stats[:, :swept].cpu().numpy()
        ess = {kk: ess_sum_over_chains(tr[i]) for i, kk in enumerate(("label0_fraction", "unary_energy", "pair_energy"))}
        secs = swept * ms_of[name] / 1e3
        out[name] = {"tv_reached": reached is not None, "sweeps_to_tv": reached, "tv_at_stop": tv,
                     "sweeps_run": swept, "ms_per_sweep": ms_of[name],
                     "seconds_to_tv": secs if reached else None, "ess": ess, "ess_min": min(ess.values()),
                     "ess_per_s": min(ess.values()) / secs,
                     "ess_per_s_at_tv": min(ess.values()) / secs if reached else None}
    if handle is None:
        h.close()
    out["protocol"] = {
        "workload": workload, "chains": C, "tv_target": tv_target, "burn_in_sweeps": burn,
        "reference": {"sweeps": ref_sweeps, "chains": rc, "form": "plain", "samples_per_site": int(n_ref),
                      "seconds": ref_s},
        "max_sweeps_per_form": budget, "check_every": chunk, "statistics": stat_desc,
        "tv": "mean over sites of 1/2 sum_a |p^_v(a) - p_ref,v(a)|, marginals from label counts of every chain and sweep"}
    return out


def versus_plain(res, names, key="ess_per_s_at_tv", basis="at the TV target"):
    """'win' / 'loss' of each form against the plain sweep in ESS/s (`key`)."""
    base = res.get("plain", {}).get(key)
    out = {}
    for n in names:
        v = res.get(n, {}).get(key)
        if v is None or base is None:
            out[n] = "no comparison (target not reached within the budget)"
        else:
            out[n] = f"{'win' if v > base else 'loss'}: {v / base:.2f}x the plain sweep's ESS/s {basis}"
    return out


def learned_tv_comparison(stream, N, C, seed, ref_sweeps, train_steps=2000, budget=1000, ref_chains=2048):
    """The learned MH block proposal (trained on ~1e5 harvested plain-chain
    samples) against the plain dual sweep, and their alternation, on a
    Barabasi-Albert Potts graph (m = 5, L = 4, beta_e ~ U[0, 0.8], unaries
    N(0, 1)) with BFS blocks of 16 sites: ESS/s over `budget` sweeps from a
    common state, and the mean-site TV of each run's marginals against a
    reference run (2048 chains).  On this family independent long runs do not
    agree to TV 0.01: the TV of 512-chain runs stays near 0.027 from 25 to
    1,600 sweeps (runs settle in different metastable states around the hubs),
    so the forms are compared at equal sweeps, with their TVs reported."""
    import torch
    from paper_1611_06684_gb300 import mrf as M, workloads as wl
    model = wl.ba_potts(N, m=5, L=4, seed=0)
    bos = wl.bfs_blocks(model, 16, seed=0)
    with torch.cuda.stream(stream):
        h = M.MRF(N, 4, C, seed=seed, stream=stream.cuda_stream, exact_edges=True, use_graphs=True)
        h.set_factors(model.unary, model.src, model.dst, model.pair)
    h.learned_setup(bos, hidden=256, seed=1)
    nb = int(bos.max()) + 1
    h.sweep(200, M.MODE_PLAIN)
    t0 = time.perf_counter()
    rows = h.learned_harvest(5, max(1, (nb * C * 5) // 100000), 100000)
    trace = h.learned_train(train_steps, 1024, 1e-3, seed=0)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    p0, a0 = h.learned_stats()
    h.sweep(4, M.MODE_LEARNED)
    p1, a1 = h.learned_stats()
    res = tv_protocol(model, C, stream, [("plain", [M.MODE_PLAIN]), ("learned", [M.MODE_LEARNED]),
                                         ("learned+plain", [M.MODE_LEARNED, M.MODE_PLAIN])],
                      seed, ref_sweeps, tv_target=0.0, burn=500, handle=h, ref_chains=ref_chains, budget=budget,
                      workload=f"Barabasi-Albert Potts graph N={N}, m=5, L=4, beta_e~U[0,0.8], unaries N(0,1), "
                               f"{C} chains, {nb} BFS blocks of <=16 sites")
    h.close()
    res["training"] = {"rows": rows, "steps": train_steps, "seconds": train_s,
                       "loss_first": float(np.mean(trace[:20])), "loss_last": float(np.mean(trace[-20:])),
                       "acceptance": (a1 - a0) / max(1, p1 - p0)}
    res["versus_plain"] = versus_plain(res, ["learned", "learned+plain"], key="ess_per_s",
                                       basis=f"at equal sweeps ({budget})")
    return res


def batch_tv_comparison(stream, n_graphs, C, seed, ref_sweeps, tv_target=0.01, chunk=25, burn=300):
    """The batched launch (all graphs of a batch swept by one set of class-union
    kernels) against one handle per graph (the plain dual sweep launched graph
    by graph), both run until the mean-site TV over all graphs' sites against
    a reference (a long run of the batch, >= 100 x the samples) is <= tv_target.
    Graphs: Erdos-Renyi, N ~ floor(exp U[ln 100, ln 2000]), mean degree U[3, 20],
    L in {2, 4, 8, 16}, tables exp(U[-0.5, 0.5]), unaries N(0, 1); C chains per
    graph.  ESS from the per-chain fraction of label 0 over all sites.  These
    graphs mix slowly (mean-site TV ~0.09 after 1,000 sweeps of 64 chains), so
    with tv_target = 0 both forms run the same number of sweeps and are
    compared at equal sweeps (their TVs then agree to within the noise)."""
    import torch
    from paper_1611_06684_gb300 import mrf as M, workloads as wl
    specs = wl.er_batch_specs(n_graphs, n_min=100, n_max=2000, seed=0)
    models = [wl.er_graph(sp) for sp in specs]
    Ns = [m.n_vars for m in models]
    Ls = [m.n_labels for m in models]
    Ntot = sum(Ns)

    def make_batch(sd):
        b = M.MRFBatch(Ns, Ls, C, seed=sd, stream=stream.cuda_stream, use_graphs=True)
        b.set_factors(models)
        return b

    def batch_marg(b, n):
        return [b.counts(g) / float(n * C) for g in range(n_graphs)]

    def tv_of(marg, ref):
        num = sum(0.5 * np.abs(m - r).sum() for m, r in zip(marg, ref))
        return float(num / Ntot)

    ref_b = make_batch(seed)
    ref_b.sweep(burn)
    ref_b.reset_marginals(0)
    t0 = time.perf_counter()
    ref_b.sweep(ref_sweeps)
    torch.cuda.synchronize()
    ref_s = time.perf_counter() - t0
    ref = batch_marg(ref_b, ref_sweeps)
    ref_b.close()
    budget = ref_sweeps // 100

    b = make_batch(seed + 1)
    hs = []
    for g, m in enumerate(models):
        with torch.cuda.stream(stream):
            hh = M.MRF(m.n_vars, m.n_labels, C, seed=seed + 2 + g, stream=stream.cuda_stream, use_graphs=True)
            hh.set_factors(m.unary, m.src, m.dst, m.pair)
        hs.append(hh)
    b.sweep(burn)
    for hh in hs:
        hh.sweep(burn)
    ms_batch = _timed(stream, lambda: b.sweep(20)) / 20
    ms_handles = _timed(stream, lambda: [hh.sweep(1) for _ in range(20) for hh in hs]) / 20
    out = {}
    for name in ("batched", "one_handle_per_graph"):
        if name == "batched":
            b.reset_marginals(0)
        else:
            for hh in hs:
                hh.reset_marginals(0)
        trace = []
        swept, reached, tv = 0, None, None
        while swept < budget:
            for _ in range(min(chunk, budget - swept)):
                if name == "batched":
                    b.sweep(1)
                    xs = [b.get_labels(g) for g in range(n_graphs)]
                else:
                    for hh in hs:
                        hh.sweep(1)
                    xs = [hh.get_labels() for hh in hs]
                trace.append(sum((x == 0).sum(axis=1) for x in xs) / Ntot)
            swept += min(chunk, budget - swept)
            if name == "batched":
                marg = batch_marg(b, swept)
            else:
                marg = [hh.counts() / float(swept * C) for hh in hs]
            tv = tv_of(marg, ref)
            if tv <= tv_target:
                reached = swept
                break
        ms = ms_batch if name == "batched" else ms_handles
        ess = ess_sum_over_chains(np.array(trace))
        secs = swept * ms / 1e3
        out[name] = {"tv_reached": reached is not None, "sweeps_to_tv": reached, "tv_at_stop": tv,
                     "sweeps_run": swept, "ms_per_sweep": ms, "seconds_to_tv": secs if reached else None,
                     "ess_min": ess, "ess_per_s": ess / secs, "ess_per_s_at_tv": ess / secs if reached else None}
    b.close()
    for hh in hs:
        hh.close()
    key = "ess_per_s_at_tv" if tv_target > 0 else "ess_per_s"
    base = out["one_handle_per_graph"][key]
    v = out["batched"][key]
    basis = "at the TV target" if tv_target > 0 else f"at equal sweeps ({budget})"
    out["versus_plain"] = {"batched": (f"{'win' if v > base else 'loss'}: {v / base:.2f}x the ESS/s of one plain "
                                       f"handle per graph {basis}") if (v and base) else
                           "no comparison (target not reached within the budget)"}
    out["protocol"] = {"graphs": n_graphs, "sites": Ntot, "edges": sum(m.n_edges for m in models),
                       "labels": sorted(set(Ls)), "chains_per_graph": C, "tv_target": tv_target,
                       "burn_in_sweeps": burn, "reference": {"sweeps": ref_sweeps, "form": "batched plain sweeps",
                                                            "seconds": ref_s},
                       "max_sweeps_per_form": budget, "check_every": chunk,
                       "statistics": "per chain: fraction of label 0 over all sites of all graphs; ESS summed over chains"}
    return out


def _enumerated_marginals(model):
    """Exact site marginals [N][L] of a small model by enumerating every labelling."""
    import itertools
    X = np.array(list(itertools.product(range(model.n_labels), repeat=model.n_vars)), np.int64)
    lp = np.asarray(model.unary, np.float64)[np.arange(model.n_vars)[None, :], X].sum(axis=1)
    if model.n_edges:
        w = np.asarray(model.pair, np.float64)
        lp += w[np.arange(model.n_edges)[None, :], X[:, model.src], X[:, model.dst]].sum(axis=1)
    p = np.exp(lp - lp.max())
    p /= p.sum()
    out = np.zeros((model.n_vars, model.n_labels))
    for v in range(model.n_vars):
        out[v] = np.bincount(X[:, v], weights=p, minlength=model.n_labels)
    return out


def small_batch_tv_comparison(stream, n_graphs, C, seed, tv_target=0.01, chunk=25, budget=4000, burn=200):
    """The batched launch against one handle per graph at marginal TV <= 0.01
    with exact reference marginals: many small uneven graphs (Erdos-Renyi,
    N in 4..14 with L^N <= 2^14, mean degree U[2, 5], L in {2, 3, 4}, tables
    exp(U[-0.5, 0.5]), unaries N(0, 1); the batched workload's families with
    sizes small enough to enumerate), C chains per graph.  Both forms run until
    the mean-site TV over all graphs' sites against the enumerated marginals is
    <= tv_target; ESS from the per-chain fraction of label 0 over all sites."""
    import torch
    from paper_1611_06684_gb300 import mrf as M, workloads as wl
    rng = np.random.default_rng(seed)
    models = []
    for g in range(n_graphs):
        L = int(rng.choice([2, 3, 4]))
        nmax = int(14 * np.log(2) / np.log(L))
        N = int(rng.integers(4, nmax + 1))
        spec = wl.ErGraphSpec(N, L, float(rng.uniform(2.0, 5.0)), int(rng.integers(0, 2**62)))
        models.append(wl.er_graph(spec))
    t0 = time.perf_counter()
    ref = [_enumerated_marginals(m) for m in models]
    enum_s = time.perf_counter() - t0
    Ns = [m.n_vars for m in models]
    Ntot = sum(Ns)
    b = M.MRFBatch(Ns, [m.n_labels for m in models], C, seed=seed, stream=stream.cuda_stream, use_graphs=True)
    b.set_factors(models)
    hs = []
    for g, m in enumerate(models):
        with torch.cuda.stream(stream):
            hh = M.MRF(m.n_vars, m.n_labels, C, seed=seed + 1 + g, stream=stream.cuda_stream, use_graphs=True)
            hh.set_factors(m.unary, m.src, m.dst, m.pair)
        hs.append(hh)
    b.sweep(burn)
    for hh in hs:
        hh.sweep(burn)
    ms_batch = _timed(stream, lambda: b.sweep(20)) / 20
    ms_handles = _timed(stream, lambda: [hh.sweep(1) for _ in range(5) for hh in hs]) / 5
    out = {}
    for name in ("batched", "one_handle_per_graph"):
        if name == "batched":
            b.reset_marginals(0)
        else:
            for hh in hs:
                hh.reset_marginals(0)
        trace = []
        swept, reached, tv = 0, None, None
        while swept < budget:
            for _ in range(chunk):
                if name == "batched":
                    b.sweep(1)
                    xs = [b.get_labels(g) for g in range(n_graphs)]
                else:
                    for hh in hs:
                        hh.sweep(1)
                    xs = [hh.get_labels() for hh in hs]
                trace.append(sum((x == 0).sum(axis=1) for x in xs) / Ntot)
            swept += chunk
            cnt = [b.counts(g) for g in range(n_graphs)] if name == "batched" else [hh.counts() for hh in hs]
            tv = float(sum(0.5 * np.abs(c / float(swept * C) - r).sum() for c, r in zip(cnt, ref)) / Ntot)
            if tv <= tv_target:
                reached = swept
                break
        ms = ms_batch if name == "batched" else ms_handles
        ess = ess_sum_over_chains(np.array(trace))
        secs = swept * ms / 1e3
        out[name] = {"tv_reached": reached is not None, "sweeps_to_tv": reached, "tv_at_stop": tv,
                     "sweeps_run": swept, "ms_per_sweep": ms, "seconds_to_tv": secs if reached else None,
                     "ess_min": ess, "ess_per_s": ess / secs, "ess_per_s_at_tv": ess / secs if reached else None}
    b.close()
    for hh in hs:
        hh.close()
    base = out["one_handle_per_graph"]["ess_per_s_at_tv"]
    v = out["batched"]["ess_per_s_at_tv"]
    out["versus_plain"] = {"batched": (f"{'win' if v > base else 'loss'}: {v / base:.2f}x the ESS/s of one plain "
                                       f"handle per graph") if (v and base) else
                           "no comparison (target not reached within the budget)"}
    out["protocol"] = {"graphs": n_graphs, "sites": Ntot, "edges": sum(m.n_edges for m in models),
                       "chains_per_graph": C, "tv_target": tv_target, "burn_in_sweeps": burn,
                       "reference": {"form": "exact marginals by enumeration", "seconds": enum_s},
                       "note": "mean-site TV over all sites of all graphs against the enumerated marginals",
                       "max_sweeps_per_form": budget, "check_every": chunk,
                       "statistics": "per chain: fraction of label 0 over all sites of all graphs; ESS summed over chains"}
    return out


def tv_mean(p, q):
    """Mean over sites of the total-variation distance of two [N][L] marginal tables."""
    return float(0.5 * np.abs(np.asarray(p, np.float64) - np.asarray(q, np.float64)).sum(axis=1).mean())


def run_learned_workload(args):
    """Barabasi-Albert Potts graph (m = 5, L = 4, beta_e ~ U[0, 0.8]), 32 chains,
    BFS blocks of 16 sites: plain sweeps, harvest of ~1e5 (block, chain) samples,
    training, learned sweeps; ESS/s and marginal TV of plain-only and of
    learned+plain alternation against a long plain reference run."""
    import torch
    from paper_1611_06684_gb300 import build as B, mrf as M, workloads as wl
    B.build()
    N = args.scale or 1_000_000
    C = 32
    t0 = time.time()
    model = wl.ba_potts(N, m=5, L=4, seed=0)
    bos = wl.bfs_blocks(model, 16, seed=0)
    gen_s = time.time() - t0
    stream = torch.cuda.Stream()
    h = M.MRF(N, 4, C, seed=args.seed, stream=stream.cuda_stream, exact_edges=True, use_graphs=True)
    h.set_factors(model.unary, model.src, model.dst, model.pair)
    h.learned_setup(bos, hidden=256, seed=1)
    nb = int(bos.max()) + 1
    h.sweep(200, M.MODE_PLAIN)                                   # burn-in
    ms_plain = _timed(stream, lambda: h.sweep(20, M.MODE_PLAIN)) / 20
    t1 = time.time()
    stride = max(1, (nb * C * 5) // 100000)
    rows = h.learned_harvest(5, stride, 100000)
    harvest_s = time.time() - t1
    p0, a0 = h.learned_stats()
    h.sweep(2, M.MODE_LEARNED)
    p1, a1 = h.learned_stats()
    acc_untrained = (a1 - a0) / max(1, p1 - p0)
    t1 = time.time()
    trace = h.learned_train(2000, 1024, 1e-3, seed=0)
    torch.cuda.synchronize()
    train_s = time.time() - t1
    h.sweep(3, M.MODE_LEARNED)                                   # warm-up (graph capture)
    torch.cuda.synchronize()
    clk_path = os.path.join(tempfile.gettempdir(), "bench_clocks_learned.csv")
    clk = clocks_start(clk_path)
    time.sleep(0.3)
    n_timed = max(10, args.steps)
    ms_learned = _timed(stream, lambda: h.sweep(n_timed, M.MODE_LEARNED)) / n_timed
    clocks = clocks_stop(clk, clk_path, torch.cuda.current_device())
    h.set_kernel_timing(True)
    h.kernel_times()
    h.sweep(5, M.MODE_LEARNED)
    kt_raw = h.kernel_times()
    kt_learned = {k: v[0] / v[1] for k, v in kt_raw.items()}
    launches_per_sweep = sum(v[1] for v in kt_raw.values()) / 5 + 1          # + k_advance (not timed)
    h.sweep(5, M.MODE_PLAIN)
    kt_plain = {k: v[0] / v[1] for k, v in h.kernel_times().items()}
    h.set_kernel_timing(False)
    R = nb * C
    Kx = (16 * 4 + 31) // 32 * 32                                 # per-chain first-layer width (couplings folded)
    mlp_flop = 2.0 * R * (256 * Kx + 256 * 256 + 64 * 256)
    ms_mlp = next((v for k, v in kt_learned.items() if k.startswith("k_gemm_nt") or "mlp" in k), float("nan"))
    peaks, peak_src = load_peaks()
    p0, a0 = h.learned_stats()
    h.sweep(4, M.MODE_LEARNED)
    p1, a1 = h.learned_stats()
    acc_trained = (a1 - a0) / max(1, p1 - p0)
    if args.ess_sweeps <= 0:
        args.ref_sweeps = 0
    # reference marginals: long plain run
    x_start = h.get_labels()
    t_start = h.info().sweep_index
    h.reset_marginals(0)
    h.sweep(args.ref_sweeps, M.MODE_PLAIN)
    ref = h.marginals()[0] if args.ref_sweeps > 0 else None
    rng = np.random.default_rng(0)
    subset = np.sort(rng.choice(N, size=4096, replace=False))
    esub = np.sort(rng.choice(model.n_edges, size=50000, replace=False))
    es, et, ew = model.src[esub], model.dst[esub], model.pair[esub].astype(np.float64)
    T = args.ess_sweeps
    out = {}
    for name, pattern in ((("plain", [M.MODE_PLAIN]), ("learned", [M.MODE_LEARNED]),
                           ("learned+plain", [M.MODE_LEARNED, M.MODE_PLAIN])) if T > 0 else ()):
        h.set_labels(x_start)
        h.set_sweep_index(t_start + 1000003)
        h.reset_marginals(0)
        stat_a = np.zeros((T, C)); stat_b = np.zeros((T, C))
        for t in range(T):
            h.sweep(1, pattern[t % len(pattern)])
            x = h.get_labels()
            stat_a[t] = (x[:, subset] == 0).mean(axis=1)
            stat_b[t] = ew[np.arange(len(esub))[None, :], x[:, es], x[:, et]].sum(axis=1)
        est, _ = h.marginals()
        ess_a = ess_sum_over_chains(stat_a)
        ess_b = ess_sum_over_chains(stat_b)
        ms = sum(ms_plain if md == M.MODE_PLAIN else ms_learned for md in pattern) / len(pattern)
        out[name] = {"ms_per_sweep": ms, "ess_label0_fraction": ess_a, "ess_pair_energy": ess_b,
                     "ess_per_s_label0": ess_a / (T * ms / 1e3), "ess_per_s_pair_energy": ess_b / (T * ms / 1e3),
                     "tv_vs_reference": tv_mean(est, ref), "sweeps": T}
    # end to end through the C ABI: labels from pinned host memory, one learned sweep, labels back
    x_host = torch.empty((C, N), dtype=torch.uint8).pin_memory()
    h.get_labels_into(x_host)
    k_e2e = 10
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        h.set_labels(x_host)
        h.sweep(1, M.MODE_LEARNED)
        h.get_labels_into(x_host)
    torch.cuda.synchronize()
    e2e = {"value": N * C * k_e2e / (time.perf_counter() - t0), "unit": METRIC, "h2d_bytes_per_step": N * C,
           "d2h_bytes_per_step": N * C, "steps": k_e2e,
           "api": "mrf_set_labels(host) + mrf_sweep(1, MRF_MODE_LEARNED) + mrf_get_labels(host), pinned buffers"}
    dom = max(kt_learned, key=kt_learned.get)
    roof = None
    if ms_mlp == ms_mlp:
        roof = {"bound": "tensor", "achieved": mlp_flop / (ms_mlp / 1e3) / 1e12, "peak": peaks["bf16_tflops"],
                "unit": "TFLOP/s", "frac": mlp_flop / (ms_mlp / 1e3) / 1e12 / peaks["bf16_tflops"], "traffic": None,
                "kernel": "k_mlp (fused tcgen05 MLP of the proposal)", "dominant_kernel_of_the_sweep": dom,
                "flop_per_launch": mlp_flop, "peak_source": f"MEASURED_PEAKS.json bf16_tflops ({peak_src})"}
    cpu = None
    if not args.no_cpu:
        from oracle import cpu_sweep, decompose as dc, philox as ph, sampler
        cores = len(os.sched_getaffinity(0))
        sm = wl.ba_potts(50000, m=5, L=4, seed=0)
        cs = cpu_sweep.CpuSweep(dc.decompose(sm), C, args.seed, threads=cores)
        xs = cs.sweep(ph.init_labels(sm.n_vars, 4, C, args.seed).astype(np.uint8), 0)
        el, S = 0.0, 0
        while el < args.cpu_seconds:
            t0 = time.perf_counter(); xs = cs.sweep(xs, S + 1); el += time.perf_counter() - t0; S += 1
        tiny = wl.ba_potts(2000, m=5, L=4, seed=0)
        dt_ = dc.decompose(tiny)
        xo = ph.init_labels(tiny.n_vars, 4, 2, args.seed)
        el1, S1 = 0.0, 0
        while el1 < args.cpu_seconds:
            t0 = time.perf_counter(); xo = sampler.sweep(dt_, xo, S1, args.seed)["x"]; el1 += time.perf_counter() - t0; S1 += 1
        cpu = {"value": sm.n_vars * C * S / el, "unit": METRIC, "cores": cores,
               "kind": "oracle (float32 OpenMP statement of the plain sweep, oracle/cpu_sweep.c)",
               "sample": f"{C} chains x {S} plain sweeps of a BA graph with N = 50,000 (same m, L and distributions)",
               "seconds": el, "host_cores_available": cores,
               "single_core_oracle": {"value": tiny.n_vars * 2 * S1 / el1, "unit": METRIC, "cores": 1,
                                      "kind": "oracle (float64 numpy)",
                                      "sample": f"2 chains x {S1} plain sweeps of a BA graph with N = 2,000",
                                      "seconds": el1},
               "note": "the learned proposal has no CPU statement; the baseline is the plain sweep"}
    contract = {"metric": METRIC, "value": N * C / (ms_learned / 1e3), "unit": METRIC, "n_gpus": 1,
                "steps": n_timed, "warmup": 3, "ms_per_step": ms_learned, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16 MLP (fp32 accumulation) + u32/f32 sweep", "data": "synthetic (seeded generators)",
                "config": {"workload": f"ba_potts_N{N}_L4_C32_blocks16",
                           "description": "Barabasi-Albert m=5, L=4, w_e(a,b) = beta_e [a=b], beta_e ~ U[0, 0.8], "
                                          "unaries N(0,1), 32 chains; learned MH proposal over 16-site BFS blocks "
                                          "(hidden 256 x 2, bf16 weights, trained on 1e5 harvested samples)",
                           "step": "one learned sweep (dual bits of the other edges, block potentials, features, "
                                   "fused MLP, MH accept) replayed as a CUDA graph",
                           "l2": "inputs larger than L2; no flush needed", "parallelism": "one GPU"},
                "roofline": roof, "gpu_launches": int(round(launches_per_sweep * n_timed)), "clocks": clocks,
                "e2e": e2e, "cpu_baseline": cpu}
    return {**contract, "ess_metric": "ESS/s", "workload": f"ba_potts_N{N}_L4_C32_blocks16", "blocks": nb,
            "generation_s": gen_s, "plain": {"ms_per_sweep": ms_plain, "site_updates_per_s": N * C / (ms_plain / 1e3)},
            "learned": {"ms_per_sweep": ms_learned, "site_updates_per_s": N * C / (ms_learned / 1e3),
                        "acceptance_untrained": acc_untrained, "acceptance_trained": acc_trained,
                        "train_rows": rows, "harvest_s": harvest_s, "train_s": train_s, "train_steps": 2000,
                        "loss_first": float(trace[:20].mean()), "loss_last": float(trace[-20:].mean())},
            "kernels_learned_ms": kt_learned, "kernels_plain_ms": kt_plain,
            "mlp_tflops": mlp_flop / (ms_mlp / 1e3) / 1e12 if ms_mlp == ms_mlp else None, "mlp_rows": R,
            "mlp_path": "fused tcgen05 (tensor memory accumulators, bulk-copied swizzled weights)",
            "mlp_roofline": {"bound": "tensor", "achieved": mlp_flop / (ms_mlp / 1e3) / 1e12,
                             "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                             "frac": mlp_flop / (ms_mlp / 1e3) / 1e12 / peaks["bf16_tflops"],
                             "flop_per_launch": mlp_flop,
                             "peak_source": f"MEASURED_PEAKS.json bf16_tflops ({peak_src})"} if ms_mlp == ms_mlp else None,
            "reference_sweeps": args.ref_sweeps,
            "statistics": "per chain: fraction of label 0 over 4096 fixed sites; pairwise energy of 50,000 fixed edges",
            "comparison": out}


def main():
    global FERRO_BETA, FERRO_U_STD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="potts3d", choices=list(WORKLOADS) + ["er_batch", "ba_learned"])
    ap.add_argument("--ref-sweeps", type=int, default=2000)
    ap.add_argument("--ess-sweeps", type=int, default=200)
    ap.add_argument("--tv-scale", type=int, default=32, help="lattice edge of the ESS/s-at-TV instance")
    ap.add_argument("--tv-ba-sites", type=int, default=1000, help="sites of the learned-proposal ESS/s-at-TV graph")
    ap.add_argument("--tv-ba-ref-sweeps", type=int, default=40000, help="reference sweeps (2048 chains) of that graph")
    ap.add_argument("--tv-batch-graphs", type=int, default=200, help="small graphs of the batched ESS/s-at-TV comparison")
    ap.add_argument("--tv-ref-sweeps", type=int, default=300000,
                    help="plain sweeps of the TV reference run (0: skip the ESS/s-at-TV protocol)")
    ap.add_argument("--mode", default="plain", choices=["plain", "fused", "sw", "higdon"])
    ap.add_argument("--higdon-rho", type=float, default=0.5, help="bond fraction of the Higdon sweep")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--scale", type=int, default=0, help="lattice edge for potts3d and ferro3d (default 128)")
    ap.add_argument("--ferro-beta", default=None, help="lo,hi of the ferro3d couplings (default %g,%g)" % FERRO_BETA)
    ap.add_argument("--ferro-u-std", type=float, default=None, help="unary std of ferro3d (default %g)" % FERRO_U_STD)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--er-labels", default="2,4,8,16", help="label counts of the batched workload's graphs")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="time budget of each CPU baseline sample")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads' lines (fully connected, batched, learned) of the default run")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.ferro_beta:
        FERRO_BETA = tuple(float(v) for v in args.ferro_beta.split(","))
    if args.ferro_u_std is not None:
        FERRO_U_STD = args.ferro_u_std
    ws, rank, local = dist_env()
    if args.workload in ("er_batch", "ba_learned") and args.impl == "ours":
        out = run_batch_workload(args) if args.workload == "er_batch" else run_learned_workload(args)
        print(json.dumps(out))
        return
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
    else:
        out = run_ours(args, ws, rank, local)
    if (args.impl == "ours" and ws == 1 and rank == 0 and out is not None and not args.no_configs
            and args.workload == "potts3d" and not args.scale):
        out["other_configs"] = other_configs(args)
    if rank == 0 and out is not None:
        print(json.dumps(out))


def other_configs(args):
    """The other workloads at their stated sizes, each as its own standard line
    from a child process (its own device memory): fully connected N = 4096,
    the 2,000-graph batched dynamic workload, the learned proposal on BA 10^6."""
    import torch
    torch.cuda.empty_cache()
    runs = {"dense4096": ["--workload", "dense4096", "--steps", "50", "--warmup", "3", "--no-variants"],
            "er_batch_2000": ["--workload", "er_batch", "--steps", "3", "--warmup", "3"],
            "ba_learned_1e6": ["--workload", "ba_learned", "--steps", "20", "--warmup", "3", "--ess-sweeps", "0"]}
    out = {}
    for name, extra in runs.items():
        cmd = [sys.executable, os.path.abspath(__file__)] + extra + ["--no-configs", "--seed", str(args.seed),
                                                                     "--cpu-seconds", "5"]
        if args.no_cpu:
            cmd.append("--no-cpu")
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=480)
            lines = [l for l in r.stdout.strip().splitlines() if l.startswith("{")]
            out[name] = json.loads(lines[-1]) if r.returncode == 0 and lines else \
                {"unavailable": f"exit {r.returncode}: {r.stderr.strip()[-300:]}"}
        except subprocess.TimeoutExpired:
            out[name] = {"unavailable": "timed out after 480 s"}
    return out


if __name__ == "__main__":
    main()
