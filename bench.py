"""Benchmark of the GB300 Louvain+ hot path (local-move passes + contraction).

One step = one full Louvain+ clustering (Algorithm 1: every coarsening and
uncoarsening level, all local-move passes, every contraction) of one seeded
synthetic graph whose CSR is resident in HBM when the timed region starts.

Default workload: R-MAT scale 22 (4,194,304 vertices, edge factor 16,
a,b,c,d = .57/.19/.19/.05), symmetrised, deduplicated, loops removed, int32
weights uniform in [1,8], modularity (w(v) = weighted degree,
lambda = 1/sum of edge weights).  value = stored edges (nnz = 2m, the
paper's 2m/t rate) per second of device time, summed over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload rmat22|grid256|sbm10k|batched|served] [--no-cpu-baseline]

Multi-GPU: one process per GPU under torchrun; a single graph does not
shard, so each rank clusters its own replica (weak scaling, no collective on
the data path); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "local-move+contraction edges/s, e2e time; batched/served graphs/s, p99 vs plain"

WORKLOADS = {
    "rmat22": dict(desc="R-MAT scale 22, edge factor 16, (a,b,c,d)=(.57,.19,.19,.05), symmetrised, "
                        "dedup, no loops, int32 weights U[1,8], modularity, int32 indices", ),
    "grid256": dict(desc="3-D 7-point grid 256^3, 1% of edges rewired, int32 weights U[1,16], unit vertex "
                         "weights, CPM lambda=1/100"),
    "sbm10k": dict(desc="planted-partition SBM, 10,000 vertices in 100 blocks, p_in .05, p_out .0005, "
                        "unit weights, modularity, seed 0"),
    "batched": dict(desc="4,096 independent SBMs, vertices log-uniform in [100, 100,000], blocks "
                         "log-uniform in [2, 500], mean degree uniform in [4, 32], half of each vertex's "
                         "degree leaving its block, unit weights, modularity; packed in one CSR and "
                         "clustered together (lc_cluster_batch), versus one lc_cluster call per graph"),
    "served": dict(desc="Poisson stream of clustering requests on host buffers: 70% SBM (vertices "
                        "log-uniform in [1e3, 1e6], blocks and degree as in the batched recipe), 30% "
                        "R-MAT (scale uniform in 10..20, edge factor 16), weights U[1,8], modularity or "
                        "CPM lambda=1/50 with probability 1/2; served by lc_server (admission by device "
                        "footprint, batched runs on concurrent slots) versus plain FIFO, one "
                        "lc_cluster_host call at a time"),
}


# DRAM bytes per step of a kernel class, from one ncu capture (dram__bytes_read
# + dram__bytes_write over every launch of the class in one clustering) of the
# same kernels on the same workload with the same launch settings ("tuned":
# the cached lc_autotune choice); a class whose kernels changed since has none
# (null).
TRAFFIC_PER_STEP = {("rmat22", "move", "tuned"): 46_775_339_264}


def make_graph(name: str, scale_override: int | None = None):
    import graphgen as gg

    if name == "rmat22":
        return gg.rmat(scale_override or 22, 16, seed=1, wmax=8)
    if name == "grid256":
        return gg.grid_cpm(side=scale_override or 256)
    if name == "sbm10k":
        return gg.sbm_planted()
    raise ValueError(name)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    """The host CPU's model name (lscpu), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform

    return platform.processor() or platform.machine()


def _oracle_run(g, method):
    import oracle

    if method == "louvain+":
        return oracle.louvain_plus(g)
    return oracle.pleiden(g, oracle.Params(uncoarsen=method == "leiden+"))


def cpu_baseline(workload: str, g_full=None, method: str = "louvain+"):
    """The CPU oracle as it stands, timed on this host: its OpenMP build
    (the same source, every pass and contraction loop on all cores) once on
    the benchmarked graph itself, and the sequential build on a bounded
    sample of the same recipe.  Both in the metric's unit."""
    import graphgen as gg
    import oracle

    name = {"louvain+": "Louvain+", "leiden": "pLeiden", "leiden+": "pLeiden+"}[method]
    cores = host_cores()
    g = g_full if g_full is not None else make_graph(workload)
    with oracle.all_cores():
        t0 = time.perf_counter()
        _oracle_run(g, method)
        t_all = time.perf_counter() - t0
    if workload == "rmat22":
        g1, s1 = gg.rmat(20, 16, seed=1, wmax=8), "R-MAT scale 20 of the same recipe"
    elif workload == "grid256":
        g1, s1 = gg.grid_cpm(side=128), "the 128^3 grid of the same recipe (CPM 1/100)"
    else:
        g1, s1 = g, "the same graph"
    t0 = time.perf_counter()
    _oracle_run(g1, method)
    t_one = time.perf_counter() - t0
    return {"value": g.nnz / t_all, "unit": "edges/s", "cores": cores, "kind": "oracle",
            "sample": f"full {name} on the benchmarked graph itself (nnz={g.nnz}), OpenMP build of "
                      f"the oracle on all {cores} host cores, one run, {t_all:.1f} s",
            "cpu_model": cpu_model(),
            "one_thread": {"value": g1.nnz / t_one, "unit": "edges/s", "cores": 1,
                           "sample": f"full {name} on {s1} (nnz={g1.nnz}), sequential build, "
                                     f"one run, {t_one:.1f} s"}}


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle timed as it stands on the host's
    cores, one bounded sample of the workload per step, in the metric's
    unit.  Single graphs use the oracle's OpenMP build (every pass and
    contraction loop on all cores); the batched and served samples spread
    their graphs over the cores instead (one sequential oracle call each)."""
    if rank != 0:
        return
    import graphgen as gg
    import oracle

    unit = "edges/s"
    cores = host_cores()
    if args.workload == "batched":
        graphs = gg.batched_sbms(args.count, seed=3, indices=list(range(0, args.count, 16)))
        sample = f"every 16th graph of the batched workload ({len(graphs)} graphs) on {cores} host threads"
        unit = "graphs/s"
    elif args.workload == "served":
        graphs = gg.served_requests(8, seed=4)
        sample = f"the first 8 requests of the served stream on {cores} host threads"
        unit = "graphs/s"
    elif args.workload == "rmat22":
        graphs = [make_graph("rmat22", args.scale)]  # the benchmarked graph itself
        sample = (f"the benchmarked R-MAT graph itself (scale {args.scale or 22}), "
                  f"OpenMP oracle on {cores} host cores")
    elif args.workload == "grid256":
        graphs = [gg.grid_cpm(side=200)]
        sample = f"the 200^3 grid of the same recipe, OpenMP oracle on {cores} host cores"
    else:
        graphs = [gg.sbm_planted()]
        sample = f"the SBM graph itself, OpenMP oracle on {cores} host cores"
    method = getattr(args, "method", "louvain+")
    if method != "louvain+":
        sample += f"; {'pLeiden+' if method == 'leiden+' else 'pLeiden'}"
    many = unit == "graphs/s"

    def one_step():
        if many:
            oracle.louvain_plus_many(graphs)
        else:
            with oracle.all_cores():
                for g in graphs:
                    _oracle_run(g, method)

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_step()
    dt = time.perf_counter() - t0
    per_step = len(graphs) if many else sum(g.nnz for g in graphs)
    value = per_step * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload]["desc"],
                       "sample": sample, "nnz": sum(g.nnz for g in graphs),
                       "same_config": args.workload in ("rmat22", "sbm10k")},
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _dist_init(world, local):
    """NCCL process group for N > 1 (barriers and the max over ranks only)."""
    if world == 1:
        return None
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    return dist


def _max_over_ranks(dist, x, dev):
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _gpu_key(workload: str) -> str:
    import torch

    return f"{workload}/{torch.cuda.get_device_name()}"


def run_batched(args, rank, world):
    """Batched form: all graphs in one lc_cluster_batch call per step;
    the plain path clusters a stratified sample one lc_cluster call at a time.
    Timed three ways: the hand-picked default launch settings, the settings
    lc_autotune chose for this workload (tuning.json, or a fresh tune with
    --tune), and the tuned bins with CUDA-graph replay switched the other way.
    With N ranks each clusters its share of the graphs (longest-processing-
    time by expected stored edges); no collective touches the data."""
    import torch

    import graphgen as gg
    import paper_2608_01503_gb300 as lc
    from paper_2608_01503_gb300 import shard

    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = _dist_init(world, local)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    count = args.count
    mine = shard.local([gg.expected_nnz(p) for p in gg.batched_sbm_params(count, seed=3)], rank, world)
    graphs = gg.batched_sbms(count, seed=3, indices=mine)
    b = gg.pack(graphs)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    rp, col, ew, vw = t(b["row_ptr"]), t(b["col"]), t(b["ew"]), t(b["vw"])
    labels = torch.empty(rp.numel() - 1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    call = lambda o: lc.lc_cluster_batch(rp, col, ew, vw, b["graph_ptr"], b["lam_num"], b["lam_den"], opts=o,
                                         labels_out=labels)
    key = _gpu_key("batched" if count == 4096 else f"batched{count}")
    tuning = None if args.no_tuning else lc.load_tuning(key)
    if args.tune:
        tuning = lc.lc_autotune(rp, col, ew, vw, b["lam_num"], b["lam_den"], graph_ptr=b["graph_ptr"], repeats=2)
        if rank == 0:
            lc.save_tuning(key, tuning)
    arms = {"default": lc.Options()}
    if tuning:
        arms["tuned"] = lc.tuned_options(tuning)
        arms["tuned_graphs_" + ("off" if tuning["graphs"] else "on")] = lc.tuned_options(
            tuning, graphs=not tuning["graphs"])
    else:
        arms["default_graphs_on"] = lc.Options(graphs=True)
    main = "tuned" if tuning else "default"
    if args.main_only:  # one arm (profiling captures)
        arms = {main: arms[main]}
    # per-class breakdown from one profiled run of the main setting (not timed)
    opts_prof = lc.tuned_options(tuning, profile=True) if tuning else lc.Options(profile=True)
    for _ in range(args.warmup):
        for o in arms.values():
            call(o)
    _, pres = call(opts_prof)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    arm_ms, klaunch = {}, 0
    for name, o in arms.items():
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            _, res = call(o)
            if name == main:
                klaunch += sum(res[0]["kernel_launches"].values())
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        arm_ms[name] = _max_over_ranks(dist, ev0.elapsed_time(ev1) / args.steps, dev)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms_step = arm_ms[main]
    # plain: one lc_cluster call per graph, every 16th graph (device-resident)
    sample = graphs[::16] if not args.no_plain else []
    dg = [(t(g.row_ptr), t(g.col), t(g.ew), t(g.vw), g.lam_num, g.lam_den) for g in sample]
    for x in dg[:4]:
        lc.lc_cluster(*x)
    torch.cuda.synchronize(dev)
    p0 = time.perf_counter()
    plain_labels = []
    for x in dg:
        lab, _ = lc.lc_cluster(*x)
        plain_labels.append(lab)
    torch.cuda.synchronize(dev)
    plain_s = time.perf_counter() - p0
    # identical results in both forms
    call(arms[main])
    torch.cuda.synchronize(dev)
    gp = b["graph_ptr"]
    same = all(torch.equal(labels[gp[16 * i]:gp[16 * i + 1]], plain_labels[i]) for i in range(len(sample)))
    plain_gps = len(sample) / plain_s if sample else None
    nnz = int(b["col"].shape[0])
    if dist:  # stored edges of all ranks' graphs
        t_nnz = torch.tensor([nnz], dtype=torch.int64, device=dev)
        dist.all_reduce(t_nnz)
        nnz = int(t_nnz.item())
    value = count / (ms_step / 1000.0)
    line = {"metric": METRIC, "value": value, "unit": "graphs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "batched", "description": WORKLOADS["batched"]["desc"], "graphs": count,
                       "n_rank0": int(rp.numel() - 1), "nnz": nnz,
                       "sharding": "graphs split over ranks by expected edges (LPT); no data collective",
                       "l2": "inputs larger than L2; no flush", "settings": main,
                       "tuning": tuning},
            "edges_per_s": nnz / (ms_step / 1000.0),
            "arms_ms_per_step": arm_ms,
            "arms_graphs_per_s": {k: count / (v / 1000.0) for k, v in arm_ms.items()},
            "plain": {"graphs_per_s": plain_gps, "sample": f"every 16th graph ({len(sample)})",
                      "identical_labels": bool(same) if sample else None},
            "speedup_vs_plain": value / plain_gps if plain_gps else None,
            "breakdown_ms_per_step": pres[0]["kernel_ms"],
            "clocks": clocks, "gpu_launches": int(klaunch)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(q * len(xs)))] if xs else None


def _served_arm(lc, reqs, arrivals, slots, max_batch, graphs=False):
    """Submits reqs[i] at arrivals[i] seconds; returns (latencies, makespan, launches)."""
    lat, done, launches = [], [], 0
    opts = lc.Options(allocator="library", graphs=graphs)
    with lc.Server(slots=slots, max_batch=max_batch, opts=opts) as srv:
        ids, t_call = [], []
        t0 = time.perf_counter()
        for g, ta in zip(reqs, arrivals):
            d = ta - (time.perf_counter() - t0)
            if d > 0:
                time.sleep(d)
            t_call.append(time.perf_counter() - t0)
            ids.append(srv.submit(g.row_ptr, g.col, g.ew, g.vw, g.lam_num, g.lam_den))
        for j, tc in zip(ids, t_call):
            _, res, l = srv.wait(j)
            lat.append(l)
            done.append(tc + l)
            launches += sum(res["kernel_launches"].values())
    return lat, max(done) - arrivals[0], launches


def _plain_arm(lc, reqs, arrivals):
    """FIFO, one lc_cluster_host call at a time, starting each request when
    it has arrived and the previous one is done."""
    lat, launches = [], 0
    t0 = time.perf_counter()
    last = 0.0
    for g, ta in zip(reqs, arrivals):
        d = ta - (time.perf_counter() - t0)
        if d > 0:
            time.sleep(d)
        _, res = lc.lc_cluster_host(g.row_ptr, g.col, g.ew, g.vw, g.lam_num, g.lam_den)
        last = time.perf_counter() - t0
        lat.append(last - ta)
        launches += sum(res["kernel_launches"].values())
    return lat, last - arrivals[0], launches


def run_served(args, rank, world):
    """Served form: a saturated burst (all requests at once) gives graphs/s;
    Poisson streams at rates swept around the plain path's saturated
    throughput give p50/p99 latency for both arms.  With N ranks, request i
    goes to rank i mod N (each rank runs its own server on its GPU); the
    latencies are gathered on the host after each arm."""
    import torch

    import graphgen as gg
    import paper_2608_01503_gb300 as lc

    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = _dist_init(world, local)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    pool = gg.served_requests(args.pool, seed=4)
    R = args.requests
    reqs_all = [pool[i % len(pool)] for i in range(R)]
    reqs = reqs_all[rank::world]
    in_bytes = sum(16 * g.n + 8 + 8 * g.nnz for g in reqs_all) / R
    out_bytes = sum(4 * g.n for g in reqs_all) / R

    def all_lat(x):
        if dist is None:
            return x
        parts = [None] * world
        dist.all_gather_object(parts, x)
        return [v for p in parts for v in p]

    # warm-up: both paths, a few requests
    for g in pool[:max(args.warmup, 3)]:
        lc.lc_cluster_host(g.row_ptr, g.col, g.ew, g.vw, g.lam_num, g.lam_den)
    _served_arm(lc, pool[:max(args.warmup, 3)], [0.0] * max(args.warmup, 3), args.slots, args.max_batch)
    torch.cuda.synchronize()
    # plain saturated throughput (closed loop over the pool), all ranks together
    if dist:
        dist.barrier()
    p0 = time.perf_counter()
    for g in pool[rank::world]:
        lc.lc_cluster_host(g.row_ptr, g.col, g.ew, g.vw, g.lam_num, g.lam_den)
    x_plain = len(pool) / _max_over_ranks(dist, time.perf_counter() - p0, dev)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    sat = {}
    for gmode in (False, True):  # CUDA-graph replay of repeated passes off / on
        if dist:
            dist.barrier()
        lat_g, span_g, launches_g = _served_arm(lc, reqs, [0.0] * len(reqs), args.slots, args.max_batch, gmode)
        sat[gmode] = (all_lat(lat_g), _max_over_ranks(dist, span_g, dev), launches_g)
    clocks = sampler.stop()
    graphs_main = sat[True][1] < sat[False][1]
    lat, span, launches = sat[graphs_main]
    value = R / span
    rates = []
    for k, f in enumerate(float(x) for x in args.rates.split(",") if x):
        rate = f * x_plain
        rng = np.random.default_rng(4 + k)
        arr = np.cumsum(rng.exponential(1.0 / rate, size=R))
        arr = [float(a - arr[0]) for a in arr][rank::world]
        t0 = arr[0] if arr else 0.0
        arr = [a - t0 for a in arr]
        row = {"rate_vs_plain": f, "offered_per_s": rate}
        for gmode in (graphs_main, not graphs_main):
            if dist:
                dist.barrier()
            s_lat, s_span, _ = _served_arm(lc, reqs, arr, args.slots, args.max_batch, gmode)
            s_span = _max_over_ranks(dist, s_span, dev)
            s_lat = all_lat(s_lat)
            row["served" if gmode == graphs_main else "served_graphs_" + ("on" if gmode else "off")] = {
                "p50_s": _pct(s_lat, 0.5), "p99_s": _pct(s_lat, 0.99), "graphs_per_s": R / s_span}
        if dist:
            dist.barrier()
        p_lat, p_span, _ = _plain_arm(lc, reqs, arr)
        p_span = _max_over_ranks(dist, p_span, dev)
        p_lat = all_lat(p_lat)
        row["plain"] = {"p50_s": _pct(p_lat, 0.5), "p99_s": _pct(p_lat, 0.99), "graphs_per_s": R / p_span}
        rates.append(row)
    line = {"metric": METRIC, "value": value, "unit": "graphs/s", "n_gpus": world, "steps": R,
            "warmup": args.warmup, "ms_per_step": span * 1000.0 / R, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "served", "description": WORKLOADS["served"]["desc"], "requests": R,
                       "distinct_graphs": len(pool), "slots": args.slots, "max_batch": args.max_batch,
                       "mean_nnz": sum(g.nnz for g in reqs_all) / R,
                       "sharding": "request i served by rank i mod N; no data collective",
                       "l2": "each request's arrays are new to the device; no flush"},
            "saturated": {"graphs_per_s": value, "p50_s": _pct(lat, 0.5), "p99_s": _pct(lat, 0.99),
                          "plain_graphs_per_s": x_plain, "speedup_vs_plain": value / x_plain,
                          "graphs_replay": graphs_main,
                          "by_graphs_replay": {("on" if gm else "off"): {
                              "graphs_per_s": R / sat[gm][1], "p50_s": _pct(sat[gm][0], 0.5),
                              "p99_s": _pct(sat[gm][0], 0.99)} for gm in (False, True)}},
            "rates": rates,
            "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": int(in_bytes),
                    "d2h_bytes_per_step": int(out_bytes)},
            "clocks": clocks, "gpu_launches": int(launches)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


ABLATIONS = {  # the settings of Section VI's ablation study (Table 2), by name
    "default": {},
    "louvain": dict(uncoarsen=False),
    "louvain_2x_passes": dict(uncoarsen=False, pass_limit=12, phi=[(3, 4)] * 8 + [(1, 4)] * 4),
    "no_symmetry_phi0": dict(symmetry=1, phi=[(0, 1)] * 6),
    "phi0": dict(phi=[(0, 1)] * 6),
    "mlh_phi0": dict(symmetry=2, phi=[(0, 1)] * 6),
}


def run_ablations(args, rank, world):
    """Each ablation setting timed like the main line on the same graph;
    slowdown and modularity difference against the default, as in Table 2."""
    import torch

    import paper_2608_01503_gb300 as lc

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    g = make_graph(args.workload, args.scale)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    rp, col, ew, vw = t(g.row_ptr), t(g.col), t(g.ew), t(g.vw)
    labels = torch.empty(g.n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    rows, launches = {}, 0
    for name, kw in ABLATIONS.items():
        opts = lc.Options(**kw)
        for _ in range(args.warmup):
            lc.lc_cluster(rp, col, ew, vw, g.lam_num, g.lam_den, opts=opts, labels_out=labels)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            _, res = lc.lc_cluster(rp, col, ew, vw, g.lam_num, g.lam_den, opts=opts, labels_out=labels)
            launches += sum(res["kernel_launches"].values())
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / args.steps
        rows[name] = {"ms_per_step": ms, "modularity": res["modularity"], "passes": res["passes_total"],
                      "levels": res["levels"]}
    clocks = sampler.stop()
    base = rows["default"]
    for r in rows.values():
        r["slowdown"] = r["ms_per_step"] / base["ms_per_step"]
        r["modularity_delta"] = r["modularity"] - base["modularity"]
    line = {"metric": METRIC, "value": g.nnz / (base["ms_per_step"] / 1000.0), "unit": "edges/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": base["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload]["desc"],
                       "n": g.n, "nnz": g.nnz, "mode": "ablations (Section VI, Table 2 settings)"},
            "ablations": rows, "clocks": clocks, "gpu_launches": int(launches)}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat22", choices=sorted(WORKLOADS))
    ap.add_argument("--scale", type=int, default=None, help="override the size (R-MAT scale / grid side)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--count", type=int, default=4096, help="graphs of the batched workload")
    ap.add_argument("--ablations", action="store_true",
                    help="time the ablation settings of Section VI on the workload's graph")
    ap.add_argument("--method", default="louvain+", choices=["louvain+", "leiden", "leiden+"],
                    help="single-graph workloads: Louvain+ (default), pLeiden or pLeiden+")
    ap.add_argument("--iterations", type=int, default=1,
                    help="iterated Louvain+ runs per step (single-graph workloads)")
    ap.add_argument("--requests", type=int, default=2000, help="requests per rate (served)")
    ap.add_argument("--pool", type=int, default=256, help="distinct request graphs (served)")
    ap.add_argument("--rates", default="0.25,0.5,0.75,0.9,1.1",
                    help="arrival rates as fractions of the plain path's throughput (served)")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--tables", type=int, default=0, choices=[0, 1],
                    help="1: high-degree tables kept across passes and updated in place")
    ap.add_argument("--max-batch", type=int, default=64)
    ap.add_argument("--tune", action="store_true",
                    help="run lc_autotune on the workload first and cache its choice (tuning.json)")
    ap.add_argument("--no-tuning", action="store_true", help="ignore cached tunings")
    ap.add_argument("--no-plain", action="store_true",
                    help="batched: skip the one-call-per-graph comparison (profiling captures)")
    ap.add_argument("--main-only", action="store_true",
                    help="batched: time only the main launch settings (profiling captures)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batched":
        run_batched(args, rank, world)
        return
    if args.workload == "served":
        run_served(args, rank, world)
        return
    if args.ablations:
        run_ablations(args, rank, world)
        return

    import torch

    import paper_2608_01503_gb300 as lc

    dist = None
    if world > 1:
        import torch.distributed as dist_

        dist = dist_
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    g = make_graph(args.workload, args.scale)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    rp, col, ew, vw = t(g.row_ptr), t(g.col), t(g.ew), t(g.vw)
    labels = torch.empty(g.n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # launch settings: lc_autotune's choice for this workload and GPU when
    # cached (--tune makes one), else the defaults; results are identical
    key = _gpu_key(args.workload if args.scale is None else f"{args.workload}_s{args.scale}")
    tuning = None
    if args.tables == 0 and not args.no_tuning:
        tuning = lc.load_tuning(key)
        if args.tune:
            tuning = lc.lc_autotune(rp, col, ew, vw, g.lam_num, g.lam_den, repeats=3)
            if rank == 0:
                lc.save_tuning(key, tuning)
    K = max(1, args.iterations)
    extra = {"uncoarsen": args.method == "leiden+"} if args.method != "louvain+" else {}
    # the timed steps run as a user runs them; a second timed region of the
    # same steps records CUDA events around each kernel class inside the
    # library (opts.profile) for the breakdown and the roofline (the events
    # cost host time per pass and keep the passes out of graph replay, so
    # they are not in the first region)
    opts_run = lc.tuned_options(tuning, tables=args.tables, **extra)
    opts_prof = lc.tuned_options(tuning, profile=True, tables=args.tables, **extra)

    def call(opts):
        if args.method != "louvain+":
            return lc.lc_cluster_leiden(rp, col, ew, vw, g.lam_num, g.lam_den, None, opts=opts,
                                        labels_out=labels)
        if K > 1:  # iterated Louvain+ (Section V-B): K runs, each constrained by the last
            return lc.lc_cluster_iterated(rp, col, ew, vw, g.lam_num, g.lam_den, K, opts=opts,
                                          labels_out=labels)
        return lc.lc_cluster(rp, col, ew, vw, g.lam_num, g.lam_den, opts=opts, labels_out=labels)

    res = None
    for _ in range(args.warmup):
        _, res = call(opts_run)
    call(opts_prof)
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kms = {k: 0.0 for k in lc.LC_K_NAMES}
    kbytes = {k: 0.0 for k in lc.LC_K_NAMES}
    klaunch = {k: 0 for k in lc.LC_K_NAMES}
    launches = 0
    ev0.record(stream)
    for _ in range(args.steps):
        _, res = call(opts_run)
        launches += sum(res["kernel_launches"].values())
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    # second region: the same steps with per-class events
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(args.steps):
        _, pres = call(opts_prof)
        for k in lc.LC_K_NAMES:
            kms[k] += pres["kernel_ms"][k]
            kbytes[k] += pres["kernel_bytes"][k]
            klaunch[k] += pres["kernel_launches"][k]
    ev3.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    ms_prof_step = ev2.elapsed_time(ev3) / args.steps
    if dist:
        tt = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    ms_step = ms / args.steps
    value = g.nnz * K * world / (ms_step / 1000.0)

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e and K == 1 and args.method == "louvain+":
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        h_rp, h_col, h_ew, h_vw = pin(g.row_ptr), pin(g.col), pin(g.ew), pin(g.vw)
        h_lab = torch.empty(g.n, dtype=torch.int32).pin_memory().numpy()
        opts_e2e = lc.tuned_options(tuning, tables=args.tables)
        lc.lc_cluster_host(h_rp, h_col, h_ew, h_vw, g.lam_num, g.lam_den, labels_out=h_lab, opts=opts_e2e)
        k2 = max(1, min(args.steps, 5))
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(k2):
            lc.lc_cluster_host(h_rp, h_col, h_ew, h_vw, g.lam_num, g.lam_den, labels_out=h_lab, opts=opts_e2e)
        torch.cuda.synchronize(dev)
        e2e_s = (time.perf_counter() - t0) / k2
        if dist:
            tt = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e2e_s = float(tt.item())
        e2e = {"value": g.nnz * world / e2e_s, "unit": "edges/s", "seconds_per_step": e2e_s,
               "h2d_bytes_per_step": int(h_rp.nbytes + h_col.nbytes + h_ew.nbytes + h_vw.nbytes),
               "d2h_bytes_per_step": int(4 * g.n)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peak, peak_kind = load_peaks()
    dom = max(lc.LC_K_NAMES, key=lambda k: kms[k])
    achieved = kbytes[dom] / (kms[dom] / 1000.0) / 1e9 if kms[dom] > 0 else 0.0
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} copy bandwidth (hbm_gbs)",
                "traffic": (TRAFFIC_PER_STEP.get((args.workload, dom, "tuned" if tuning else "default"))
                            if args.scale is None and K == 1 and args.method == "louvain+" and args.tables == 0
                            else None),
                "traffic_unit": "DRAM bytes per step, all launches of the class (ncu)",
                "launches": klaunch[dom],
                "algorithmic_bytes_per_step": kbytes[dom] / args.steps,
                "measured": ("CUDA events the library records around each kernel class on its "
                             "stream, over a second timed region of the same steps"),
                "profiled_ms_per_step": ms_prof_step}
    breakdown = {k: {"ms_per_step": kms[k] / args.steps, "launches_per_step": klaunch[k] / args.steps,
                     "algorithmic_GBps": (kbytes[k] / (kms[k] / 1000.0) / 1e9) if kms[k] > 0 else None}
                 for k in lc.LC_K_NAMES}
    lm_ms = (kms["first_pass"] + kms["move"] + kms["table"] + kms["afterburner"] + kms["apply"]
             + kms["objective"]) / args.steps
    ct_ms = kms["contract"] / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload]["desc"],
                   "n": g.n, "nnz": g.nnz, "edges_counted": "nnz = 2m (both directions), the paper's 2m/t",
                   "l2": "inputs larger than L2 (CSR > 129 MB); no flush",
                   "parallelism": "replicas" if world > 1 else "single GPU", "method": args.method,
                   "settings": "tuned" if tuning else "default", "tuning": tuning,
                   **({"iterations": K, "edges_counted_iterated": "nnz once per iteration"}
                      if K > 1 else {})},
        "result": {"n_clusters": res["n_clusters"], "levels": res["levels"],
                   "passes": res["passes_total"], "modularity": res["modularity"], "phi": res["phi"]},
        "local_move_edges_per_s": res["edges_local_move"] / (lm_ms / 1000.0) if lm_ms > 0 else None,
        "contraction_edges_per_s": res["edges_contract"] / (ct_ms / 1000.0) if ct_ms > 0 else None,
        "breakdown": breakdown,
        "roofline": roofline,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": int(launches),
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, g, method=args.method)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
