"""Benchmark: KSG CMI estimates/s of one greedy multivariate-TE selection step.

Workload (the step the metric is quoted on): one target of a 10-node sparse
linear VAR(5) network, T = 10000, candidate sources = every (node, lag) with
lag 1..5 except the target's own lags 1..3 (47 candidates), target history 3
(so N = 9995 samples, joint dimension 5), k = 4, 200 permutation surrogates
per candidate: 47 x 201 = 9447 KSG estimates per step, plus the max-statistic
gate.  Synthetic seeded data (the paper reports no datasets).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs the same step for its own target (weak scaling).
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "KSG CMI estimates/s incl. surrogates (N=1e4,k=4); batched/screened vs plain"
# DRAM bytes (read + write) per launch of the 200-surrogate step, from ncu
# captures (profiles/), per kernel; None until the current kernel is captured.
# Tile kernel: profiles/ksg_fused_kernel_greedy_step_small.md (15-surrogate case,
# 31.68 MB, scaled by job groups 296/24).  List kernel: captured directly on the
# full-size launch (profiles/ksg_list_kernel_greedy_step_small.md).
TRAFFIC_BYTES = {"tile": 390.7e6, "list": 3288.1e6 + 744.7e6}
# Pipe utilisation of the list kernel from its committed full ncu capture
# (small case of the same step; profiles/ksg_list_kernel_greedy_step_small.md).
PIPES_FROM_PROFILE = {"alu_pct": 49.5, "fma_pct": 28.9, "lsu_pct": 30.7, "issue_active_pct": 71.5,
                      "l1_hit_pct": 68.6, "unit": "% of each pipe's peak, sustained active",
                      "source": "profiles/ksg_list_kernel_greedy_step_small.md"}

WORKLOAD = dict(n_proc=10, order=5, T=10000, n_past=3, min_lag=1, max_lag=5, k=4, n_surr=200,
                alpha=0.05, seed=20181029)


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        loaded = [v for v in sm if v > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def _timed(fn, min_s=1.0, sampler_gpu=0):
    """Call fn() once untimed, then repeatedly for at least min_s with CUDA
    events around the loop and nvidia-smi clocks sampled meanwhile; returns
    (ms per call, calls, clocks)."""
    import torch
    fn()
    torch.cuda.synchronize()
    sampler = ClockSampler(sampler_gpu)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    calls, t0 = 0, time.perf_counter()
    e0.record()
    while True:
        fn()
        calls += 1
        if calls >= 3 and time.perf_counter() - t0 >= min_s:
            torch.cuda.synchronize()
            if time.perf_counter() - t0 >= min_s:
                break
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    return e0.elapsed_time(e1) / calls, calls, clocks


def _dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_oracle_sample(series, target, budget_s=15.0, threads=None):
    """Time the oracle on a bounded sample of the step's estimates."""
    import oracle
    if threads:
        oracle.set_num_threads(threads)
    w = WORKLOAD
    L = max(w["max_lag"], w["n_past"])
    T = series.shape[1]
    y = series[target, L:]
    z = np.stack([series[target, L - lag:T - lag] for lag in range(1, w["n_past"] + 1)])
    cands = [(p, lag) for p in range(series.shape[0]) for lag in range(1, w["max_lag"] + 1)
             if not (p == target and lag <= w["n_past"])]
    done = 0
    t0 = time.perf_counter()
    for (p, lag) in cands:
        xc = series[p, L - lag:T - lag][None, :]
        for s in range(1 + w["n_surr"]):
            c = p * 5 + lag - 1
            xs = xc if s == 0 else xc[:, oracle.perm(w["seed"], (c << 24) | (s - 1), T - L)]
            oracle.cmi_ksg(xs, y, z, w["k"])
            done += 1
            if time.perf_counter() - t0 > budget_s:
                break
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "estimates/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{done} of the step's {len(cands) * (1 + w['n_surr'])} estimates "
                      f"(N={T - L}, d=5, k=4), brute-force C oracle, {dt:.1f} s wall"}


def run_reference(args):
    world, rank, _ = _dist_setup()
    if rank != 0:
        return
    from paper_1807_10459_gb300 import synth
    net = synth.var_network(n_nodes=WORKLOAD["n_proc"], order=WORKLOAD["order"],
                            T=WORKLOAD["T"])
    per_step = []
    cb = None
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_sample(net.series, 0, budget_s=8.0)
        if i >= args.warmup:
            per_step.append(r["value"])
            cb = r
    v = float(np.mean(per_step))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "estimates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": _config(),
            "cpu_baseline": {"value": v, "unit": "estimates/s", "cores": cb["cores"],
                             "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "estimates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config():
    w = WORKLOAD
    return {"workload": "greedy mTE step: 10-node sparse VAR(5), T=10000, target 0, "
                        f"lags 1..5, history 3, k=4, {w['n_surr']} surrogates",
            "n_proc": w["n_proc"], "T": w["T"], "N": w["T"] - max(w["max_lag"], w["n_past"]),
            "candidates": 47, "n_surr": w["n_surr"], "k": w["k"], "joint_dim": 5,
            "estimates_per_step": 47 * (1 + w["n_surr"]),
            "l2": "flushed by a 256 MiB device write before every step"}


def workloads_result(device: int) -> dict:
    """The other configurations, each timed for about a second with its own
    clock record (device time, inputs resident, every call synchronised):
    the Gaussian CMI problem (dx = dy = 1, dz = 2, k = 4, 100 surrogates) at
    N = 1e3 and 1e4; the logistic-map chain (50 replications x 1997 samples,
    joint dimension 12, 200 surrogates) with sample-level surrogates under
    the library's kernel choice and with each kernel forced, and with
    replication-level surrogates; and full greedy inference on the 50-node
    network in exact, screened and network-free mode."""
    import torch
    import paper_1807_10459_gb300 as idtx
    from paper_1807_10459_gb300 import synth
    dev = torch.device("cuda", device)
    out = {}

    def kernel_of(ctx):
        return "list" if ctx.stats()["list_launches"] > 0 else "tile"

    for n in (1000, 10000):
        g = synth.gaussian_problem(n, 1, 1, 2, seed=synth.BASE_SEED + 1)
        x, y, z = (torch.from_numpy(a).to(dev) for a in (g.x, g.y, g.z))
        ctx = idtx.Context(device)
        ms, calls, clocks = _timed(lambda: idtx.cmi_ksg(x, y, z, k=4, n_surr=100, seed=1,
                                                        ctx=ctx), 1.0, device)
        out[f"gaussian_n{n}"] = {
            "config": f"Gaussian CMI, N={n}, dx=dy=1, dz=2, k=4, 100 surrogates",
            "estimates_per_s": 101 / (ms / 1e3), "ms_per_call": ms, "calls": calls,
            "kernel": kernel_of(ctx), "clocks": clocks}

    lx, ly, lz = synth.logistic_problem(dx=1, dy=1, dz=10)
    n = lx.shape[1]
    x, y, z = (torch.from_numpy(a).to(dev) for a in (lx, ly, lz))
    logi = {"config": f"logistic-map chain, 50 replications x {n // 50} samples (N={n}), "
                      "dx=dy=1, dz=10, k=4, 200 surrogates"}
    for name, kern, reps in (("auto", idtx.KERNEL_AUTO, 0), ("list", idtx.KERNEL_LIST, 0),
                             ("tile", idtx.KERNEL_TILE, 0), ("replications", idtx.KERNEL_AUTO, 50)):
        ctx = idtx.Context(device)
        ctx.set_kernel(kern)
        ms, calls, clocks = _timed(lambda: idtx.cmi_ksg(x, y, z, k=4, n_surr=200, seed=3,
                                                        n_reps=reps, ctx=ctx), 1.0, device)
        logi[name] = {"estimates_per_s": 201 / (ms / 1e3), "ms_per_call": ms, "calls": calls,
                      "kernel": kernel_of(ctx), "clocks": clocks}
    out["logistic_n1e5"] = logi
    out["var50_greedy"] = var50_result(device)
    return out


def run_ours(args):
    import torch
    import paper_1807_10459_gb300 as idtx
    from paper_1807_10459_gb300 import synth

    world, rank, local = _dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = WORKLOAD
    net = synth.var_network(n_nodes=w["n_proc"], order=w["order"], T=w["T"])
    target = rank % w["n_proc"]
    series_d = torch.from_numpy(net.series).to(dev)
    ctx = idtx.Context(local)
    ctx.set_kernel({"auto": idtx.KERNEL_AUTO, "tile": idtx.KERNEL_TILE,
                    "list": idtx.KERNEL_LIST}[args.kernel])
    ctx.set_list_caps(*args.list_caps)
    rates = idtx.probe_issue_rates(local)  # the roofline's denominator, measured here
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    est_per_step = 47 * (1 + w["n_surr"])

    def step(series):
        return idtx.mte_step(series, target, w["n_past"], w["min_lag"], w["max_lag"], (), 0,
                             k=w["k"], n_surr=w["n_surr"], alpha=w["alpha"], seed=w["seed"],
                             ctx=ctx)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step(series_d)
    torch.cuda.synchronize()
    ctx.reset_stats()
    ctx.set_profiling(True)
    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        flush.fill_(1.0)
        step(series_d)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    st = ctx.stats()
    ctx.set_profiling(False)
    t_max = ms
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    value = est_per_step * args.steps * world / (t_max / 1e3)

    # the same step with each kernel forced (both give identical estimates)
    kernels = {}
    if rank == 0:
        for name, kern in (("tile", idtx.KERNEL_TILE), ("list", idtx.KERNEL_LIST)):
            kctx = idtx.Context(local)
            kctx.set_kernel(kern)
            step_k = lambda: idtx.mte_step(series_d, target, w["n_past"], w["min_lag"],
                                           w["max_lag"], (), 0, k=w["k"], n_surr=w["n_surr"],
                                           alpha=w["alpha"], seed=w["seed"], ctx=kctx)
            step_k()
            torch.cuda.synchronize()
            k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k0.record(stream)
            for _ in range(2):
                flush.fill_(1.0)
                step_k()
            k1.record(stream)
            torch.cuda.synchronize()
            kernels[name] = est_per_step * 2 / (k0.elapsed_time(k1) / 1e3)
            del kctx

    # plain schedule (one launch per estimate, no sharing) on a subset of the
    # step: the same 47 candidates with 4 surrogates each (its cost per estimate
    # does not depend on the number of surrogates)
    plain = None
    if rank == 0:
        def plain_step():
            return idtx.mte_step(series_d, target, w["n_past"], w["min_lag"], w["max_lag"], (),
                                 0, k=w["k"], n_surr=4, alpha=w["alpha"], seed=w["seed"],
                                 mode=idtx.MODE_PLAIN, ctx=ctx)
        plain_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plain_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        n = w["T"] - 5
        w_plain = n * (n - 1) * (4 * 5 + 9)  # brute-force lane-ops per estimate, d = 5
        plain = {"value": 47 * 5 / dt, "unit": "estimates/s",
                 "sample": "the step's 47 candidates with 4 surrogates each, one launch each",
                 "w_plain_lane_ops_per_estimate": w_plain, "w_plain_tops": 47 * 5 / dt * w_plain / 1e12}

    # screened schedule with the shipped screen, on the same step
    screened = None
    weights = os.path.join(ROOT, "paper_1807_10459_gb300", "screen_weights.npz")
    if rank == 0 and os.path.exists(weights):
        idtx.screen_set(idtx.Screen.load(weights), ctx=ctx)
        ex = step(series_d)

        def scr_step():
            return idtx.mte_step(series_d, target, w["n_past"], w["min_lag"], w["max_lag"], (),
                                 0, k=w["k"], n_surr=w["n_surr"], alpha=w["alpha"],
                                 seed=w["seed"], mode=idtx.MODE_SCREENED, ctx=ctx)
        scr_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)
            r = scr_step()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        screened = {"value": est_per_step / dt, "unit": "exact-equivalent estimates/s",
                    "candidates_with_full_surrogates": r.n_full, "candidates": r.n_cand,
                    "same_decision_as_exact": (r[0], r[1], r[3]) == (ex[0], ex[1], ex[3])}

    # end to end through the public API with host (pinned) inputs and outputs
    series_h = torch.from_numpy(net.series).pin_memory()
    step(series_h)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(series_h)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": est_per_step * args.steps * world / e2e_s, "unit": "estimates/s",
           "h2d_bytes_per_step": int(net.series.nbytes), "d2h_bytes_per_step": 24}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    sm_mhz = (clocks or {}).get("sm_mhz") or rates["sm_clock_mhz"]
    # Peak: the fastest lane-operation rate the probes measured (per SM per
    # clock), times the SMs and the median SM clock of the timed region.
    rate_keys = ("fadd_per_sm_clk", "fmnmx_per_sm_clk", "fsetp_add_per_sm_clk",
                 "iadd_per_sm_clk", "count_mix_per_sm_clk")
    best = max(rate_keys, key=lambda k2: rates[k2])
    peak = rates[best] * rates["n_sms"] * sm_mhz * 1e6 / 1e12
    sec = st["fused_ms"] / 1e3 if st["fused_ms"] else None
    achieved = st["fused_lane_ops"] / sec / 1e12 if sec else None
    used = "list" if st["list_launches"] > 0 else "tile"
    useful = st["useful_lane_ops"] / sec / 1e12 if (sec and used == "list") else None
    traffic = TRAFFIC_BYTES[used] if w["n_surr"] == 200 else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                "frac": (achieved / peak) if achieved else None,
                "useful_achieved": useful, "useful_frac": (useful / peak) if useful else None,
                "traffic": traffic,
                "traffic_unit": "DRAM bytes read + written per launch (ncu)",
                "kernel": ("ksg_list_kernel" if used == "list" else "ksg_fused_kernel") +
                          "<DX=1,DY=1,DZ=3,K1=5,exact,QC=64,NW=8>",
                "peak_basis": f"{best} measured by idtx_probe_issue_rates "
                              f"({rates[best]:.1f} lane-ops/SM/clk) x {rates['n_sms']} SMs x "
                              f"median SM clock {sm_mhz:.0f} MHz of the timed region",
                "issue_rates_per_sm_clk": {k2: rates[k2] for k2 in rate_keys},
                "probe_sm_clock_mhz": rates["sm_clock_mhz"],
                "pipes_from_profile": PIPES_FROM_PROFILE,
                "estimator_share_of_step": st["fused_ms"] / ms if ms else None,
                "list_caps": [st["list_cap_a"], st["list_cap_b"]] if used == "list" else None,
                "scanned_fraction_of_exhaustive":
                    ((st["scanned_a"] + st["scanned_b"]) / st["exhaustive_pairs"])
                    if st["exhaustive_pairs"] and used == "tile" else None,
                "work_per_step": {k2: st[k2] / args.steps for k2 in
                                  (("list_walk_a", "list_walk_b", "list_tail_a", "list_tail_b",
                                    "brute_samples", "fallbacks", "list_sum_nz", "list_sum_nyz",
                                    "fused_lane_ops", "useful_lane_ops")
                                   if used == "list" else
                                   ("scanned_a", "passed_a", "scanned_b", "passed_b",
                                    "fused_lane_ops"))},
                "ops_basis": ("achieved: lane-operations the kernel executes -- 2dx+2 per "
                              "(job, list A entry) and 2dx+4 per (job, list B entry) for every "
                              "lane of a shared walk, the same per (job, entry) pair of the "
                              "repacked count phases and neighbour tails, 2(dx+dy+dz')+2/+6 per "
                              "sample of a full-scan fallback; useful_achieved: only the "
                              "(2dx+2) n_yz + (2dx+4) n_z per (query, job) that a walk visiting "
                              "exactly the entries each job needs would do (counted in-kernel)")
                             if used == "list" else
                             ("lane-ops the kernel's algorithm needs for the tiles it scans: "
                              "shared scan per (query, reference, job group) plus per-job work "
                              "for pairs passing the shared bound (counted in-kernel)")}
    workloads = workloads_result(local) if (world == 1 and not args.no_workloads) else None
    cpu = cpu_oracle_sample(net.series, target, budget_s=12.0) if world == 1 else None
    line = {"metric": METRIC, "value": value, "unit": "estimates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": _config(), "mode": "batched (one fused launch "
            "per step over all candidates and surrogates)",
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(st["kernel_launches"]), "clocks": clocks,
            "kernels": {"chosen": used, "tile": kernels.get("tile"), "list": kernels.get("list"),
                        "unit": "estimates/s, the same step with the kernel forced"},
            "modes": {"batched": value, "plain": plain["value"] if plain else None,
                      "plain_frac_of_peak_by_w_plain": (plain["w_plain_tops"] / peak)
                      if plain else None,
                      "batched_over_plain": value / plain["value"] if plain else None,
                      "plain_sample": plain["sample"] if plain else None,
                      "screened": screened},
            "workloads": workloads}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_var50(args):
    print(json.dumps(var50_result(0)), flush=True)


def var50_result(device: int) -> dict:
    """Full greedy inference on a 50-node in-degree-3 VAR(3) network (T=5000,
    lags 1..3, history 3, k=4, 200 surrogates): every target in exact
    (batched) and screened mode; parent-set agreement and wall-time speedup,
    with the SM clocks sampled during each mode."""
    import torch
    import paper_1807_10459_gb300 as idtx
    from paper_1807_10459_gb300 import synth
    net = synth.var_network_indegree(n_nodes=50, order=3, indegree=3, T=5000)
    s = torch.from_numpy(net.series).to(torch.device("cuda", device))
    ctx = idtx.Context(device)
    trained = idtx.Screen.load(os.path.join(ROOT, "paper_1807_10459_gb300",
                                            "screen_weights.npz"))
    # the network-free rule the trained network improves on: cheap maximum plus
    # a constant margin calibrated the same way (an all-zero network)
    free = idtx.Screen(params=np.zeros(idtx.SCREEN_NPARAMS, np.float32), s0=trained.s0,
                       delta=float(trained.meta["network_free_margin"]))
    ctx_free = idtx.Context(device)
    idtx.screen_set(trained, ctx=ctx)
    idtx.screen_set(free, ctx=ctx_free)
    kw = dict(k=4, n_surr=200, alpha=0.05, seed=20181031, max_parents=10, ctx=ctx)
    idtx.mte_select_target(s, 0, 3, 1, 3, **kw)      # warm-up
    idtx.mte_select_target(s, 0, 3, 1, 3, mode=idtx.MODE_SCREENED, **kw)
    torch.cuda.synchronize()
    res, clocks = {}, {}
    for mode_name, mode, c in (("exact", idtx.MODE_BATCHED, ctx),
                               ("screened", idtx.MODE_SCREENED, ctx),
                               ("network_free", idtx.MODE_SCREENED, ctx_free)):
        kw["ctx"] = c
        sampler = ClockSampler(device)
        sampler.start()
        out, t0 = [], time.perf_counter()
        for t in range(50):
            out.append(idtx.mte_select_target(s, t, 3, 1, 3, mode=mode, **kw))
        torch.cuda.synchronize()
        res[mode_name] = (out, time.perf_counter() - t0)
        clocks[mode_name] = sampler.stop()
    nf = res["network_free"][0]
    ex, sc = res["exact"][0], res["screened"][0]
    same = [a["parents"] == b["parents"] for a, b in zip(ex, sc)]
    steps_same = sum(1 for a, b in zip(ex, sc) for u, v in zip(a["steps"], b["steps"])
                     if (u[0], u[1]) == (v[0], v[1]))
    n_steps = sum(len(a["steps"]) for a in ex)
    full = sum(st.n_full for b in sc for st in b["steps"])
    cands = sum(st.n_cand for b in sc for st in b["steps"])
    truth = {(p, q, lag) for (p, q, lag) in net.edges}
    found = {(c // 3, t, 1 + c % 3) for t, a in enumerate(ex) for c in a["parents"]}
    line = {"metric": "greedy mTE inference, 50-node VAR(3) (T=5000, k=4, 200 surrogates): "
                      "screened vs exact", "n_gpus": 1,
            "exact_seconds": res["exact"][1], "screened_seconds": res["screened"][1],
            "speedup": res["exact"][1] / res["screened"][1],
            "parent_set_agreement": sum(same) / len(same),
            "step_decision_agreement": steps_same / n_steps,
            "candidates_with_full_surrogates": full, "candidates_evaluated": cands,
            "network_free": {
                "seconds": res["network_free"][1],
                "speedup": res["exact"][1] / res["network_free"][1],
                "parent_set_agreement": sum(a["parents"] == b["parents"]
                                            for a, b in zip(ex, nf)) / len(ex),
                "candidates_with_full_surrogates": sum(st.n_full for b in nf
                                                       for st in b["steps"]),
                "margin": free.delta},
            "screen": {"delta": trained.delta, "s0": trained.s0,
                       "quantile": trained.meta.get("quantile")},
            "exact_true_positive_edges": len(found & truth), "true_edges": len(truth),
            "exact_false_positive_edges": len(found - truth), "clocks": clocks,
            "data": "synthetic"}
    return line


def run_post(args):
    """The tests after selection on the benchmarked network (10-node VAR(5),
    T=10000, target 0, lags 1..5, history 3, k=4, 200 surrogates): the greedy
    selection, then pruning, the omnibus test and the sequential maximum
    statistic of the selected parents, each timed; the oracle timed on a
    bounded sample of the same leave-one-out estimates."""
    import torch
    import paper_1807_10459_gb300 as idtx
    from paper_1807_10459_gb300 import synth
    w = WORKLOAD
    net = synth.var_network(n_nodes=w["n_proc"], order=w["order"], T=w["T"])
    s = torch.from_numpy(net.series).cuda()
    ctx = idtx.Context(0)
    kw = dict(k=w["k"], n_surr=w["n_surr"], alpha=w["alpha"], seed=w["seed"], ctx=ctx)
    geo = (0, w["n_past"], w["min_lag"], w["max_lag"])
    sel = idtx.mte_select_target(s, *geo, max_parents=10, **kw)
    par = sel["parents"]
    out = {"metric": "tests after selection: KSG CMI estimates/s (N=9995, k=4, 200 surrogates)",
           "unit": "estimates/s", "n_gpus": 1, "parents": par, "data": "synthetic",
           "config": {"workload": "10-node sparse VAR(5), T=10000, target 0, lags 1..5, "
                                  "history 3, parents from the greedy selection"}}
    if not par:
        print(json.dumps(out), flush=True)
        return
    for _ in range(max(args.warmup, 1)):   # also settles the kernel choice of every shape
        idtx.mte_prune(s, *geo, par, **kw)
        idtx.mte_seqmax(s, *geo, par, **kw)
        if len(par) <= 4:
            idtx.mte_omnibus(s, *geo, par, **kw)
    torch.cuda.synchronize()
    runs = {}
    t0 = time.perf_counter()
    pr = idtx.mte_prune(s, *geo, par, **kw)
    torch.cuda.synchronize()
    runs["prune"] = (time.perf_counter() - t0, sum(r_m for r_m in
                     [len(par) - i for i in range(len(pr["rounds"]))]) * (1 + w["n_surr"]))
    t0 = time.perf_counter()
    sq = idtx.mte_seqmax(s, *geo, par, **kw)
    torch.cuda.synchronize()
    runs["seqmax"] = (time.perf_counter() - t0, len(par) * (1 + w["n_surr"]))
    om = None
    if len(par) <= 4:
        t0 = time.perf_counter()
        om = idtx.mte_omnibus(s, *geo, par, **kw)
        torch.cuda.synchronize()
        runs["omnibus"] = (time.perf_counter() - t0, 1 + w["n_surr"])
    tot_s = sum(v[0] for v in runs.values())
    tot_e = sum(v[1] for v in runs.values())
    # the oracle on two leave-one-out estimates of the first parent
    import oracle
    L = max(w["max_lag"], w["n_past"])
    T = net.series.shape[1]
    n_lags = w["max_lag"] - w["min_lag"] + 1
    colv = lambda c: net.series[c // n_lags, L - (w["min_lag"] + c % n_lags):T - (w["min_lag"] + c % n_lags)]
    y = net.series[0, L:]
    z = np.stack([net.series[0, L - lag:T - lag] for lag in range(1, w["n_past"] + 1)] +
                 [colv(c) for c in par[1:]])
    t0 = time.perf_counter()
    ref = oracle.cmi_ksg(colv(par[0])[None, :], y, z, w["k"])
    cpu_dt = time.perf_counter() - t0
    out.update({"value": tot_e / tot_s, "seconds": {k2: v[0] for k2, v in runs.items()},
                "estimates": {k2: v[1] for k2, v in runs.items()},
                "kept": pr["kept"], "prune_rounds": pr["rounds"],
                "seqmax": {"stats": sq[0].tolist(), "pvals": sq[1].tolist(),
                           "significant": sq[2].tolist()},
                "omnibus": om,
                "first_loo_stat_vs_oracle": abs(float(sq[0][0]) - ref),
                "cpu_baseline": {"value": 1.0 / cpu_dt, "unit": "estimates/s",
                                 "cores": oracle.num_threads(), "kind": "oracle",
                                 "sample": "one leave-one-out estimate of the first parent"}})
    print(json.dumps(out), flush=True)


def run_batch64(args):
    """The uneven batch: 64 problems, N log-uniform in [2000, 50000], dx, dy in
    {1, 2}, dz in 1..8, 500 surrogates each (32 064 estimates) through
    idtx_cmi_batch (one persistent fused launch per kernel variant).  Plain
    mode (one launch per estimate) is timed on two estimates of every problem
    and scaled to the batch's 501 per problem."""
    import torch
    import paper_1807_10459_gb300 as idtx
    from paper_1807_10459_gb300 import synth
    probs = synth.batch_problems()
    dev = [dict(x=torch.from_numpy(p.x).cuda(), y=torch.from_numpy(p.y).cuda(),
                z=torch.from_numpy(p.z).cuda(), n_surr=p.n_surr, seed=p.seed) for p in probs]
    n_est = sum(1 + p.n_surr for p in probs)
    ctx = idtx.Context(0)
    for _ in range(max(args.warmup, 1)):
        idtx.cmi_batch(dev, k=4, ctx=ctx)
    torch.cuda.synchronize()
    ctx.set_profiling(True)
    ctx.reset_stats()
    sampler = ClockSampler(0)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        idtx.cmi_batch(dev, k=4, ctx=ctx)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    st = ctx.stats()
    ctx.set_profiling(False)
    # the same estimates as 64 separate calls (one fused launch per problem)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    for p, d in zip(probs, dev):
        idtx.cmi_ksg(d["x"], d["y"], d["z"], k=4, n_surr=p.n_surr, seed=p.seed, ctx=ctx)
    s1.record()
    torch.cuda.synchronize()
    ms_sep = s0.elapsed_time(s1)
    # CUDA-graph replay of the same call (captured once, then replayed)
    gctx = idtx.Context(0)
    gctx.set_graphs(True)
    idtx.cmi_batch(dev, k=4, ctx=gctx)
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record()
    for _ in range(args.steps):
        idtx.cmi_batch(dev, k=4, ctx=gctx)
    g1.record()
    torch.cuda.synchronize()
    ms_graph = g0.elapsed_time(g1) / args.steps
    replays = gctx.stats()["graph_launches"] - 1
    del gctx
    # plain mode: two estimates per problem, one launch each
    t_plain = 0.0
    for p, d in zip(probs, dev):
        for _ in range(2):   # the second pass is timed (the first builds buffers)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            idtx.cmi_ksg(d["x"], d["y"], d["z"], k=4, n_surr=1, seed=p.seed,
                         mode=idtx.MODE_PLAIN, ctx=ctx)
            b.record()
            torch.cuda.synchronize()
        t_plain += a.elapsed_time(b) / 2.0 * (1 + p.n_surr) / 1e3
    line = {"metric": "KSG CMI estimates/s, 64-problem uneven batch (N 2e3-5e4, k=4, "
                      "500 surrogates)", "value": n_est / (ms / 1e3), "unit": "estimates/s",
            "n_gpus": 1, "steps": args.steps, "ms_per_call": ms, "estimates_per_call": n_est,
            "fused_launches_per_call": st["fused_launches"] / args.steps,
            "fused_share_of_call": st["fused_ms"] / (ms * args.steps) if ms else None,
            "modes": {"batched": n_est / (ms / 1e3),
                      "separate_calls": n_est / (ms_sep / 1e3),
                      "graph_replay": n_est / (ms_graph / 1e3),
                      "graph_replays_timed": replays,
                      "plain_estimated": n_est / t_plain,
                      "batched_over_plain": t_plain / (ms / 1e3),
                      "plain_sample": "2 estimates of every problem, one launch each, "
                                      "scaled to 501 per problem"},
            "clocks": clocks, "dtype": "f32", "data": "synthetic"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="var10-step",
                    choices=["var10-step", "var50-greedy", "batch64", "post"],
                    help="var10-step: the benchmarked greedy step (default); var50-greedy: "
                         "full inference on a 50-node VAR(3), exact vs screened; batch64: "
                         "the 64-problem uneven batch; post: pruning, omnibus and sequential "
                         "maximum statistic after the greedy selection")
    ap.add_argument("--kernel", default="auto", choices=["auto", "tile", "list"],
                    help="estimator kernel of the timed step (auto: the library's timed choice)")
    ap.add_argument("--list-caps", type=int, nargs=2, default=(0, 0), metavar=("A", "B"),
                    help="list capacities of the list kernel (0 0: the library's choice)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the other configurations (Gaussian, logistic, 50-node network)")
    ap.add_argument("--n-surr", type=int, default=WORKLOAD["n_surr"],
                    help="surrogates per candidate (200 is the benchmarked workload; smaller "
                         "values give a small case for profiling)")
    args = ap.parse_args()
    WORKLOAD["n_surr"] = args.n_surr
    if args.workload == "var50-greedy":
        run_var50(args)
        return
    if args.workload == "batch64":
        run_batch64(args)
        return
    if args.workload == "post":
        run_post(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
