"""Benchmark: decoupled closeness centrality on a HoMLN, one GPU per rank.

One step = one pass of the whole hot path over one HoMLN:
  CSR build of every layer -> all-sources BFS closeness of every layer (Psi) ->
  AND aggregation + all-sources BFS closeness of the AND graph (ground truth) ->
  top-10% CC nodes -> naive, CC1 and CC2 composition (Theta) -> accuracy of each.

Workload (default, the largest single-GPU configuration): 4 Barabasi-Albert layers
(m = 4) on 200,000 shared nodes, half of one base BA graph shared by every layer
(seeded synthetic stand-in for the paper's RMAT/PaRMAT HoMLNs). The 4-layer
Chung-Lu n = 50,000 workload is measured beside it (``configs``), as are the
batched 64-network workload and the serving stream.

Metric: GTEPS = sum over the analysed graphs of sum_s |E(component(s))| / time
(Graph500 convention for all-sources BFS), whole job over all ranks.

Prints one JSON line (rank 0); its last key, ``summary``, repeats the headline
figures, the batched-vs-plain speedup and the serving latencies in a few fields.
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

METRIC = "GTEPS and % HBM roofline of all-sources closeness; batched vs plain speedup"
L2_FLUSH_BYTES = 512 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="ba200k", choices=["powerlaw50k", "ba200k", "er1k"])
    p.add_argument("--secondary", default="powerlaw50k", choices=["powerlaw50k", "ba200k", "er1k", "none"],
                   help="another configuration measured beside the headline (none: skip)")
    p.add_argument("--no-autotune", action="store_true", help="library defaults instead of the autotuner's pick")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-sources", type=int, default=2000)
    p.add_argument("--words", type=int, default=0, help="BFS words per node (0 = auto)")
    p.add_argument("--alpha", type=int, default=0)
    p.add_argument("--teams", type=int, default=0, help="BFS teams (0 = auto)")
    p.add_argument("--team-mix", type=int, default=0, help="1: blocks on one SM join different teams")
    p.add_argument("--threads", type=int, default=0, help="threads per BFS block (0 = 512)")
    p.add_argument("--no-batch", action="store_true", help="skip the batched-vs-plain measurement")
    p.add_argument("--batch-count", type=int, default=64)
    p.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    p.add_argument("--no-paper-like", action="store_true", help="skip the paper-shaped accuracy/timing runs")
    p.add_argument("--no-widened", action="store_true",
                   help="skip the OR-aggregation, subset-sweep and directed-layer measurements")
    p.add_argument("--serve-seconds", type=float, default=15.0)
    p.add_argument("--serve-rate", type=float, default=50.0)
    p.add_argument("--single-bfs", action="store_true",
                   help="profiling aid: build the workload, run one layer's all-sources BFS once, exit")
    p.add_argument("--launch-list", action="store_true",
                   help="profiling aid: run exactly one plain step (no warm-up, no instrumented pass), exit")
    return p.parse_args()


def replica_seed(base: int, rank: int) -> int:
    """Each rank analyses its own HoMLN (replicas, weak scaling): same shape, its own seed."""
    return base + 7919 * rank


def job_aggregate(units: float, seconds: float, dist=None, device=None):
    """Whole-job throughput inputs: units summed over ranks, time = the slowest rank's."""
    if dist is None:
        return units, seconds
    import torch
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def make_workload(name: str, rank: int):
    from paper_2207_11662_gb300 import synth
    if name == "powerlaw50k":
        net = synth.homln_powerlaw(n=50000, avg_deg=10.0, n_layers=4, gamma=2.5, seed=replica_seed(2001, rank))
        desc = (f"4 Chung-Lu layers (gamma 2.5, avg deg 10), n=50000, shared pool rho={net.meta['rho']:.3f}; "
                "per-layer + AND all-sources closeness, top-10%, naive/CC1/CC2, accuracy")
    elif name == "ba200k":
        net = synth.homln_ba_large(n=200000, m_attach=4, n_layers=4, seed=replica_seed(4001, rank))
        desc = "4 BA layers (m=4), n=200000, ~50% shared edges; full hot path"
    else:
        net = synth.homln_small_er(seeds=(101 + rank, 102 + rank, 103 + rank))
        desc = "3 ER layers (avg deg 8), n=1000; full hot path"
    return net, desc


def teps_work(n: int, layers, want_per_graph: bool = False):
    """sum over analysed graphs of sum_s |E(comp(s))| = sum over components of n_c * m_c (and, with
    want_per_graph, the same per graph: every layer, then the AND graph)."""
    import scipy.sparse as sps
    from scipy.sparse.csgraph import connected_components

    def canon(s, d):
        s = s.astype(np.int64)
        d = d.astype(np.int64)
        k = s != d
        lo, hi = np.minimum(s[k], d[k]), np.maximum(s[k], d[k])
        return np.unique(lo * n + hi)

    keys = [canon(s, d) for s, d in layers]
    inter = keys[0]
    for k in keys[1:]:
        inter = np.intersect1d(inter, k, assume_unique=True)
    per_graph = []
    for k in keys + [inter]:
        lo, hi = k // n, k % n
        A = sps.coo_matrix((np.ones(lo.shape[0]), (lo, hi)), shape=(n, n)).tocsr()
        nc, lab = connected_components(A, directed=False)
        nodes = np.bincount(lab, minlength=nc).astype(np.int64)
        edges = np.bincount(lab[lo], minlength=nc).astype(np.int64)
        per_graph.append(int(np.sum(nodes * edges)))
    if want_per_graph:
        return sum(per_graph), [int(k.shape[0]) for k in keys + [inter]], per_graph
    return sum(per_graph), [int(k.shape[0]) for k in keys + [inter]]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


PROFILE_FILES = {"powerlaw50k": "k_msbfs_powerlaw50k_launch.md", "ba200k": "k_msbfs_ba200k_launch.md"}


def measured_traffic(workload: str, tiles: int, words: int, teams: int, alpha: int, mix: int = 0):
    """DRAM bytes (read + write) per BFS launch from the committed ncu summary under profiles/: the
    capture of the same (words per node, teams, alpha, team mix) setting, scaled from its tiles to
    this launch's (equal for the same workload). None when the kernel source changed since, or no
    capture has this setting."""
    import hashlib
    if workload not in PROFILE_FILES:
        return None
    path = os.path.join(ROOT, "profiles", PROFILE_FILES[workload])
    src = os.path.join(ROOT, "paper_2207_11662_gb300", "csrc", "msbfs.cu")
    try:
        with open(src, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
        ok_sha = False
        with open(path) as f:
            for line in f:
                if line.startswith("kernel_source_sha256_16:"):
                    ok_sha = line.split(":", 1)[1].strip() == sha
                if ok_sha and line.startswith("capture:"):
                    kv = dict(x.split("=") for x in line.split(":", 1)[1].split())
                    key = (int(kv["words_per_node"]), int(kv["teams"]), int(kv["push_alpha"]), int(kv.get("team_mix", 0)))
                    if key == (words, teams, alpha, mix):
                        return int(int(kv["dram_bytes_launch"]) * tiles / int(kv["tiles"]))
    except (OSError, KeyError, ValueError):
        return None
    return None


def bfs_bytes(prof: dict) -> float:
    """Algorithmic bytes of the BFS launches: the bytes the kernel's loads and stores request,
    counted by its instrumented variant -- per gathered frontier word 8 B, per scanned or pushed
    column index 4 B, per atomic OR 8 B, and per visited vertex its seen/next words, row bounds,
    F/R and per-vertex bytes (a load shared by the lanes of one vertex counted once)."""
    return float(prof["bytes"])


def tuning_from_args(args) -> dict:
    t = {}
    if args.words:
        t["words_per_node"] = args.words
    if args.alpha:
        t["push_alpha"] = args.alpha
    if args.teams:
        t["teams"] = args.teams
    if args.team_mix:
        t["team_mix"] = 1
    if args.threads:
        t["threads"] = args.threads
    return t


class HotPath:
    """One step of the hot path on one HoMLN through the binding: create (CSR builds), Psi of every
    layer and the AND graph in one persistent launch, closeness read-back, AND edge count, top-10%
    ground truth, naive/CC1/CC2 and the accuracy of each."""

    def __init__(self, H, net, dev, stream, tuning):
        self.H, self.net, self.dev, self.stream, self.tuning = H, net, dev, stream, dict(tuning)
        self.sel = H.make_select(H.HOMLN_TOPK_PERCENT, 10.0, cc1_overlap=0.5)

    def step(self, layers, host_out=False, profile=None):
        import torch
        H, n, L = self.H, self.net.n, self.net.n_layers
        full = (1 << L) - 1
        h = H.homln_create(n, layers, stream=self.stream.cuda_stream)
        try:
            if self.tuning:
                H.homln_set_tuning(h, **self.tuning)
            if profile is not None:
                H.homln_set_profiling(h, profile == "time", profile == "count")
            if host_out:
                F = np.empty(n, np.uint64)
                R = np.empty(n, np.uint32)
                cc = np.empty(n, np.float64)
                ids = [np.empty(n, np.int32) for _ in range(4)]
            else:
                F = torch.empty(n, dtype=torch.int64, device=self.dev)
                R = torch.empty(n, dtype=torch.int32, device=self.dev)
                cc = torch.empty(n, dtype=torch.float64, device=self.dev)
                ids = [torch.empty(n, dtype=torch.int32, device=self.dev) for _ in range(4)]
            H.homln_analyse(h, full, True)  # Psi of every layer and the AND graph in one launch
            for i in range(L):
                H.homln_layer_closeness(h, i, F, R, cc)
            m_and = H.homln_and_aggregate(h, full)
            H.homln_and_closeness(h, full, F, R, cc)
            cg = H.homln_topk(h, -1, full, self.sel, ids[0])
            accs = []
            for j, heur in enumerate((H.HOMLN_NAIVE, H.HOMLN_CC1, H.HOMLN_CC2)):
                c = H.homln_compose(h, full, heur, self.sel, ids[j + 1])
                accs.append(H.homln_accuracy(h, ids[j + 1], c, ids[0], cg))
            prof = H.homln_get_profile(h) if profile is not None else None
            return accs, prof, m_and
        finally:
            H.homln_destroy(h)


def autotune_workload(H, net, dev, stream, reps=3):
    """The autotuner's pick (W, teams, alpha) for this network's analysis (every layer + AND)."""
    import torch
    from paper_2207_11662_gb300 import autotune
    n, L = net.n, net.n_layers
    layers = [(torch.from_numpy(s).to(dev), torch.from_numpy(d).to(dev)) for s, d in net.layers]
    h = H.homln_create(n, layers, stream=stream.cuda_stream)
    try:
        edges = [int(s.shape[0]) for s, _ in net.layers]
        best, log = autotune.tune([h], [(1 << L) - 1], [n], edges, True, stream.cuda_stream, use_cache=False,
                                  reps=reps, skew=autotune.degree_skew(n, net.layers))
    finally:
        H.homln_destroy(h)
    return best, log


def measure(H, hp: HotPath, dev, steps, warmup, flush, dist=None, sample_clocks=False):
    """Warm-up, one untimed instrumented pass (the BFS kernel's algorithmic bytes), then `steps` timed
    steps on device-resident inputs with L2 flushed before each; CUDA events on the launch stream."""
    import torch
    net, stream = hp.net, hp.stream
    dlayers = [(torch.from_numpy(s).to(dev), torch.from_numpy(d).to(dev)) for s, d in net.layers]
    for _ in range(warmup):
        hp.step(dlayers)
    torch.cuda.synchronize()
    _, prof_count, m_and = hp.step(dlayers, profile="count")
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches0 = H.homln_kernel_launches()
    bfs_ms, bfs_launches = 0.0, 0
    accs = None
    clk = ClockSampler(dev.index) if sample_clocks else None
    if clk:
        clk.__enter__()
    try:
        for k in range(steps):
            flush.fill_(k)  # evict L2 between steps (512 MB > 129 MB)
            ev[k][0].record(stream)
            accs, prof, _ = hp.step(dlayers, profile="time")
            ev[k][1].record(stream)
            bfs_ms += prof["bfs_ms"]
            bfs_launches += prof["bfs_timed_launches"]
        torch.cuda.synchronize()
    finally:
        if clk:
            clk.__exit__(None, None, None)
    return {"step_ms": [a.elapsed_time(b) for a, b in ev], "bfs_ms": bfs_ms, "bfs_launches": bfs_launches,
            "prof_count": prof_count, "accs": accs, "m_and": m_and,
            "launches": H.homln_kernel_launches() - launches0, "clocks": clk.summary() if clk else None}


def roofline(workload, m, hp_tuning):
    prof = m["prof_count"]
    alg_bytes_per_launch = bfs_bytes(prof) / max(prof["bfs_launches"], 1)
    launch_ms = m["bfs_ms"] / max(m["bfs_launches"], 1)
    achieved = alg_bytes_per_launch / (launch_ms / 1000.0) / 1e9
    hbm, peak_kind = peaks()
    traffic = measured_traffic(workload, prof["batches"], prof["words_per_node"], prof["teams"],
                               hp_tuning.get("push_alpha", 16), hp_tuning.get("team_mix", 0))
    out = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
           "frac": round(achieved / hbm, 4), "traffic": traffic, "peak_kind": peak_kind,
           "kernel": "k_msbfs (persistent all-sources BFS: every layer and the AND graph in one launch)",
           "algorithmic_bytes_per_launch": round(alg_bytes_per_launch), "launch_ms": round(launch_ms, 4),
           "bfs_share_of_step": round(m["bfs_ms"] / sum(m["step_ms"]), 4)}
    if traffic:
        out["dram_gbs"] = round(traffic / (launch_ms / 1000.0) / 1e9, 1)
        out["dram_frac"] = round(out["dram_gbs"] / hbm, 4)
    return out


def per_graph_teps(H, net, dev, stream, tuning, per_graph_work, reps=3):
    """Each layer's and the AND graph's all-sources BFS in a launch of its own (a fresh handle each,
    best of reps), CUDA-event timed around the launch: GTEPS per graph; and the ground truth as one
    call (AND aggregation, relabelling, BFS and closeness of the AND graph), timed around the call."""
    import torch
    n, L = net.n, net.n_layers
    layers = [(torch.from_numpy(s).to(dev), torch.from_numpy(d).to(dev)) for s, d in net.layers]
    F = torch.empty(n, dtype=torch.int64, device=dev)
    out = []
    for g in range(L + 1):
        best = float("inf")
        for _ in range(reps):
            h = H.homln_create(n, layers, stream=stream.cuda_stream)
            try:
                if tuning:
                    H.homln_set_tuning(h, **tuning)
                H.homln_set_profiling(h, True, False)
                if g < L:
                    H.homln_layer_closeness(h, g, F, None, None)
                else:
                    H.homln_and_closeness(h, (1 << L) - 1, F, None, None)
                torch.cuda.synchronize()
                best = min(best, H.homln_get_profile(h)["bfs_ms"])
            finally:
                H.homln_destroy(h)
        out.append({"graph": f"layer {g}" if g < L else "AND", "bfs_ms": round(best, 3),
                    "gteps": round(per_graph_work[g] / best / 1e6, 1)})
    # the ground truth as one call: AND aggregation of the layers' CSRs, relabelling, BFS, closeness
    best = float("inf")
    for _ in range(reps):
        h = H.homln_create(n, layers, stream=stream.cuda_stream)
        try:
            if tuning:
                H.homln_set_tuning(h, **tuning)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            H.homln_and_closeness(h, (1 << L) - 1, F, None, None)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        finally:
            H.homln_destroy(h)
    out[-1]["ground_truth_call_ms"] = round(best, 3)
    out[-1]["ground_truth_gteps"] = round(per_graph_work[L] / best / 1e6, 1)
    return out


def run_ours(args, rank, world, dist):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_11662_gb300 import homln as H

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    net, desc = make_workload(args.workload, rank)
    n, L = net.n, net.n_layers
    stream = torch.cuda.current_stream(dev)
    tuning = tuning_from_args(args)
    tune_log = None
    if not tuning and not args.no_autotune and not (args.single_bfs or args.launch_list):
        tuning, tune_log = autotune_workload(H, net, dev, stream)
    hp = HotPath(H, net, dev, stream, tuning)
    dlayers = [(torch.from_numpy(s).to(dev), torch.from_numpy(d).to(dev)) for s, d in net.layers]

    if args.single_bfs:
        h = H.homln_create(n, dlayers, stream=stream.cuda_stream)
        if tuning:
            H.homln_set_tuning(h, **tuning)
        F = torch.empty(n, dtype=torch.int64, device=dev)
        H.homln_layer_closeness(h, 0, F, None, None)
        H.homln_destroy(h)
        torch.cuda.synchronize()
        return None, net
    if args.launch_list:
        hp.step(dlayers)
        torch.cuda.synchronize()
        return None, net
    work, edge_counts, work_per_graph = teps_work(n, net.layers, want_per_graph=True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    m = measure(H, hp, dev, args.steps, args.warmup, flush, dist, sample_clocks=True)
    t_local = sum(m["step_ms"]) / 1000.0
    units, t_max = job_aggregate(work * args.steps, t_local, dist, dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    # end to end through the C-ABI with host buffers: pinned inputs, H2D + D2H inside the timed region,
    # over as many steps as the device-timed value
    pinned = [(torch.from_numpy(s).pin_memory(), torch.from_numpy(d).pin_memory()) for s, d in net.layers]
    h2d = sum(int(s.numel() + d.numel()) * 4 for s, d in pinned)
    torch.cuda.synchronize()
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hp.step([(s.numpy(), d.numpy()) for s, d in pinned], host_out=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1000.0)
    d2h = (L + 1) * n * (8 + 4 + 8) + 4 * n * 4
    e2e_units, e2e_t = job_aggregate(work * args.steps, sum(e2e_ms) / 1000.0, dist, dev)
    per_graph = per_graph_teps(H, net, dev, stream, tuning, work_per_graph) if rank == 0 else None

    prof_count = m["prof_count"]
    result = {
        "metric": METRIC,
        "value": round(units / t_max / 1e9, 3),
        "unit": "GTEPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_max * 1000.0 / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic (seeded Chung-Lu/ER/BA HoMLN, shapes of the paper's workloads)",
        "config": {"workload": desc, "n": n, "layers": L, "undirected_edges": edge_counts,
                   "teps_edges_per_step": work, "l2": "flushed between steps (512 MB write)",
                   "parallelism": f"replicas x{world} (one HoMLN per GPU)"},
        "roofline": roofline(args.workload, m, tuning),
        "e2e": {"value": round(e2e_units / e2e_t / 1e9, 3), "unit": "GTEPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_t * 1000.0 / args.steps, 3)},
        "gpu_launches": int(m["launches"]),
        "clocks": m["clocks"],
        "tuning": {"chosen": {"words_per_node": prof_count["words_per_node"], "teams": prof_count["teams"],
                              "push_alpha": tuning.get("push_alpha", 16), "team_mix": tuning.get("team_mix", 0)},
                   "source": "autotuner" if tune_log else ("flags" if tuning else "library defaults"),
                   "candidates_timed": len(tune_log["candidates"]) if tune_log else 0,
                   "reps": tune_log["reps"] if tune_log else 0,
                   "top": tune_log["candidates"][:4] if tune_log else []},
        "per_graph": per_graph,
        "accuracy_vs_ground_truth": {nm: {k: round(a[k], 4) for k in ("jaccard", "precision", "recall", "f1")}
                                     for nm, a in zip(("naive", "cc1", "cc2"), m["accs"])},
        "bfs_profile": {k: prof_count[k] for k in ("levels", "pull_levels", "push_levels", "batches",
                                                   "edges_scanned", "words_gathered", "edges_pushed",
                                                   "words_pushed", "bytes", "visits", "words_per_node",
                                                   "teams")},
    }
    return result, net


def secondary_config(args, name, dev, steps=10, warmup=3):
    """Another single-GPU configuration measured the same way (device-resident inputs, L2 flushed,
    CUDA events), autotuned like the headline: GTEPS, ms per step and the BFS kernel's roofline."""
    import torch
    from paper_2207_11662_gb300 import homln as H
    net, desc = make_workload(name, 0)
    stream = torch.cuda.current_stream(dev)
    tuning, log = ({}, None) if args.no_autotune else autotune_workload(H, net, dev, stream)
    hp = HotPath(H, net, dev, stream, tuning)
    work, _ = teps_work(net.n, net.layers)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    m = measure(H, hp, dev, steps, warmup, flush)
    t = sum(m["step_ms"]) / 1000.0
    pc = m["prof_count"]
    return {"workload": desc, "gteps": round(work * steps / t / 1e9, 3), "ms_per_step": round(t * 1000.0 / steps, 3),
            "steps": steps, "roofline": roofline(name, m, tuning),
            "tuning": {"words_per_node": pc["words_per_node"], "teams": pc["teams"],
                       "push_alpha": tuning.get("push_alpha", 16), "team_mix": tuning.get("team_mix", 0)}}


def batch_vs_plain(args, dev):
    """64 HoMLNs (2-8 layers, 500-20,000 nodes, ER or BA layers): all their layers and AND graphs
    analysed (a) in one persistent launch over every (graph, batch) tile, autotuned, (b) one
    persistent launch per HoMLN, (c) plain -- one ordinary launch per BFS phase with the host driving
    the levels, layer by layer. Outputs must be bit-identical across the three."""
    import torch
    from paper_2207_11662_gb300 import autotune
    from paper_2207_11662_gb300 import homln as H
    from paper_2207_11662_gb300 import synth

    nets = synth.homln_batch(args.batch_count, 3001)
    stream = torch.cuda.current_stream(dev)
    hs = [H.homln_create(net.n, [(torch.from_numpy(s).to(dev), torch.from_numpy(d).to(dev)) for s, d in net.layers],
                         stream=stream.cuda_stream) for net in nets]
    masks = [(1 << net.n_layers) - 1 for net in nets]
    work = 0
    edges = []
    for net in nets:
        w, ec = teps_work(net.n, net.layers)
        work += w
        edges += ec
    ns = [net.n for net in nets]
    outs = [[torch.empty(net.n, dtype=torch.int64, device=dev) for _ in range(net.n_layers + 1)] for net in nets]

    def collect():
        snap = []
        for h, net, mask, o in zip(hs, nets, masks, outs):
            for i in range(net.n_layers):
                H.homln_layer_closeness(h, i, o[i], None, None)
            H.homln_and_closeness(h, mask, o[-1], None, None)
            snap.append([t.clone() for t in o])
        return snap

    def timed(fn, reps=3):
        best = []
        for _ in range(reps):
            for h in hs:
                H.homln_invalidate(h)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            best.append(e0.elapsed_time(e1))
        return statistics.mean(best)

    skew = max(autotune.degree_skew(net.n, net.layers) for net in nets)
    tuning, tune_log = autotune.tune(hs, masks, ns, edges, True, stream.cuda_stream, use_cache=False, skew=skew)
    H.homln_set_tuning(hs[0], **tuning)
    timed(lambda: H.homln_batch_analyse(hs, masks, True), reps=1)  # warm-up
    t_batch = timed(lambda: H.homln_batch_analyse(hs, masks, True))
    ref = collect()
    # the same analysis captured once in a CUDA graph and replayed
    graph = H.homln_graph_capture(hs, masks, True)
    t_graph = timed(lambda: H.homln_graph_launch(graph))
    same_graph = all(torch.equal(a, b) for x, y in zip(ref, collect()) for a, b in zip(x, y))
    H.homln_graph_destroy(graph)
    for h in hs:
        H.homln_set_tuning(h)
    t_per = timed(lambda: [H.homln_analyse(h, m, True) for h, m in zip(hs, masks)])
    same = all(torch.equal(a, b) for x, y in zip(ref, collect()) for a, b in zip(x, y))
    for h in hs:
        H.homln_set_tuning(h, schedule=1)
    t_plain = timed(lambda: [H.homln_analyse(h, m, True) for h, m in zip(hs, masks)], reps=1)
    same = same and same_graph and all(torch.equal(a, b) for x, y in zip(ref, collect()) for a, b in zip(x, y))
    for h in hs:
        H.homln_destroy(h)
    return {"workload": f"{len(nets)} HoMLNs, {sum(n.n_layers for n in nets)} layers + {len(nets)} AND graphs, "
                        f"n in [{min(ns)}, {max(ns)}], ER/BA layers",
            "batched_ms": round(t_batch, 3), "graph_replay_ms": round(t_graph, 3),
            "per_homln_persistent_ms": round(t_per, 3),
            "plain_ms": round(t_plain, 3), "speedup_vs_plain": round(t_plain / t_batch, 2),
            "graph_speedup_vs_plain": round(t_plain / t_graph, 2),
            "speedup_vs_per_homln": round(t_per / t_batch, 2), "batched_gteps": round(work / t_batch / 1e6, 1),
            "identical_outputs": bool(same), "autotuned": tuning,
            "autotune_candidates_timed": len(tune_log["candidates"]), "autotune_reps": tune_log["reps"]}


def paper_like(args, dev):
    """Two-layer HoMLNs shaped like the paper's synthetic sets (Section 6, Table 1; seeded R-MAT
    layers over a shared |V|-edge backbone): mean accuracy of naive, CC1 and CC2 against the AND
    ground truth with above-average CC nodes (Tables 2-5), CC1 at several overlap thresholds theta
    (Section 5.1 leaves theta undefined), and the timing comparison of Section 6.1 (largest
    composition time vs smallest layer-analysis time)."""
    import torch
    from paper_2207_11662_gb300 import homln as H
    from paper_2207_11662_gb300 import synth
    stream = torch.cuda.current_stream(dev)
    sets = {"S-1": (("powerlaw", "normal"), [(50000, 250000), (100000, 1000000)]),
            "S-2": (("powerlaw", "powerlaw"), [(50000, 250000)]),
            "S-3": (("normal", "normal"), [(50000, 250000)])}
    thetas = (0.1, 0.25, 0.5)
    sel = H.make_select(H.HOMLN_GE_MEAN, cc1_overlap=0.5)
    names = {"naive": H.HOMLN_NAIVE, "cc1": H.HOMLN_CC1, "cc2": H.HOMLN_CC2}
    out = {}
    psi_min, theta_max = float("inf"), {k: 0.0 for k in names}
    seed = 6001
    for sname, (kinds, bases) in sets.items():
        accs = {k: [] for k in names}
        sweep = {t: [] for t in thetas}
        for n, m in bases:
            for split in ((0.7, 0.3), (0.6, 0.4), (0.5, 0.5)):
                seed += 1
                net = synth.homln_parmat_like(n, m, split, kinds, seed)
                h = H.homln_create(n, [(torch.from_numpy(s).to(dev), torch.from_numpy(d).to(dev))
                                       for s, d in net.layers], stream=stream.cuda_stream)
                F = torch.empty(n, dtype=torch.int64, device=dev)
                for i in range(2):  # Psi of each layer, timed alone
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    H.homln_layer_closeness(h, i, F, None, None)
                    e1.record(stream)
                    e1.synchronize()
                    psi_min = min(psi_min, e0.elapsed_time(e1))
                gt = np.empty(n, np.int32)
                cg = H.homln_topk(h, -1, 3, sel, gt)
                est = np.empty(n, np.int32)
                for k, heur in names.items():
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    c = H.homln_compose(h, 3, heur, sel, est)
                    theta_max[k] = max(theta_max[k], (time.perf_counter() - t0) * 1000.0)
                    accs[k].append(H.homln_accuracy(h, est, c, gt, cg))
                for t in thetas:
                    c = H.homln_compose(h, 3, H.HOMLN_CC1, H.make_select(H.HOMLN_GE_MEAN, cc1_overlap=t), est)
                    sweep[t].append((H.homln_accuracy(h, est, c, gt, cg), c))
                H.homln_destroy(h)
        out[sname] = {k: {m_: round(100.0 * statistics.mean(a[m_] for a in v), 2)
                          for m_ in ("jaccard", "precision", "recall", "f1")} for k, v in accs.items()}
        out[sname]["cc1_theta_sweep"] = {
            str(t): {"jaccard": round(100.0 * statistics.mean(a["jaccard"] for a, _ in v), 2),
                     "recall": round(100.0 * statistics.mean(a["recall"] for a, _ in v), 2),
                     "mean_selected": round(statistics.mean(c for _, c in v), 1)} for t, v in sweep.items()}
    out["min_psi_ms"] = round(psi_min, 3)
    out["max_theta_ms"] = {k: round(v, 3) for k, v in theta_max.items()}
    out["max_theta_over_min_psi"] = {k: round(v / psi_min, 3) for k, v in theta_max.items()}
    out["note"] = ("accuracy in percent (Jaccard is what the paper calls accuracy); CC1's overlap threshold theta is "
                   "not given by the paper (0.5 above, swept in cc1_theta_sweep); paper (Table 2) S-1/S-2/S-3 mean "
                   "Jaccard CC1 43.56/55.95/48.87, CC2 46.77/55.20/50.90 on PaRMAT data, context only")
    return out


def _components_teps(n: int, lo, hi) -> int:
    """sum over the components of an undirected graph of n_c * m_c (edges as pairs lo < hi)."""
    import scipy.sparse as sps
    from scipy.sparse.csgraph import connected_components
    A = sps.coo_matrix((np.ones(lo.shape[0]), (lo, hi)), shape=(n, n)).tocsr()
    nc, lab = connected_components(A, directed=False)
    nodes = np.bincount(lab, minlength=nc).astype(np.int64)
    edges = np.bincount(lab[lo], minlength=nc).astype(np.int64)
    return int(np.sum(nodes * edges))


def widened(args, dev, reps: int = 3):
    """The follow-on rows on the power-law n=50,000 workload: the OR-aggregated ground truth, the
    layer-subset sweep, and the same network with directed layers."""
    import torch
    from paper_2207_11662_gb300 import homln as H
    from paper_2207_11662_gb300 import synth
    net, _ = make_workload("powerlaw50k", 0)
    n, L = net.n, net.n_layers
    full = (1 << L) - 1
    stream = torch.cuda.current_stream(dev)
    sel = H.make_select(H.HOMLN_TOPK_PERCENT, 10.0)

    def timed(fn):
        best = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    dl = [(torch.from_numpy(s).to(dev), torch.from_numpy(d).to(dev)) for s, d in net.layers]
    F = torch.empty(n, dtype=torch.int64, device=dev)
    out = {}
    # OR aggregation: build the OR graph and run its all-sources BFS (a fresh handle each time)
    def or_step():
        h = H.homln_create(n, dl, stream=stream.cuda_stream)
        H.homln_or_closeness(h, full, F, None, None)
        H.homln_destroy(h)
    h = H.homln_create(n, dl, stream=stream.cuda_stream)
    m_or = H.homln_or_aggregate(h, full)
    s_or = np.empty(m_or, np.int32)
    d_or = np.empty(m_or, np.int32)
    H.homln_or_aggregate(h, full, m_or, s_or, d_or)
    H.homln_destroy(h)
    ms = timed(or_step)
    work = _components_teps(n, s_or.astype(np.int64), d_or.astype(np.int64))
    out["or_aggregation"] = {"ms": round(ms, 3), "edges": int(m_or), "gteps": round(work / ms / 1e6, 1),
                             "includes": "CSR builds of 4 layers, OR union, relabelling, all-sources BFS"}
    # layer-subset sweep: ground truth, CC2 estimate and accuracy of all 11 subsets of >= 2 layers
    def sweep():
        h = H.homln_create(n, dl, stream=stream.cuda_stream)
        res = H.homln_subset_sweep(h, H.HOMLN_CC2, sel, 2)
        H.homln_destroy(h)
        return res
    res = sweep()
    ms = timed(sweep)
    out["subset_sweep"] = {"ms": round(ms, 3), "subsets": len(res),
                           "mean_jaccard_cc2": round(float(np.mean([r["jaccard"] for r in res])), 4),
                           "includes": "CSR builds, BFS of 4 layers + 11 AND graphs in one launch, "
                                       "11 x (ground truth, CC2, accuracy)"}
    # directed layers: each edge a random-direction arc, plus the reverse of 25% of them
    arcs = [synth.with_reciprocal(e, 0.25, 7001 + i) for i, e in enumerate(net.layers)]
    da = [(torch.from_numpy(s).to(dev), torch.from_numpy(d).to(dev)) for s, d in arcs]
    def directed_step():
        h = H.homln_create(n, da, stream=stream.cuda_stream, directed=True)
        H.homln_analyse(h, full, True)
        H.homln_destroy(h)
    ms = timed(directed_step)
    h = H.homln_create(n, da, stream=stream.cuda_stream, directed=True)
    m_and = H.homln_and_aggregate(h, full)
    H.homln_destroy(h)
    n_arcs = [int(np.unique(s.astype(np.int64)[s != d] * n + d[s != d]).shape[0]) for s, d in arcs]
    bound = n * (sum(n_arcs) + m_and)
    out["directed"] = {"ms": round(ms, 3), "arcs_per_layer": n_arcs, "and_arcs": int(m_and),
                       "gteps_bound": round(bound / ms / 1e6, 1),
                       "includes": "CSR builds (out- and in-edges) of 4 layers, AND, relabelling, in-closeness "
                                   "BFS of 4 layers + AND",
                       "teps_convention": "n x arcs per graph: an upper bound on the arcs the BFS traverses"}
    return out


def _serving_item(arg):
    """Spawn-pool worker: one request's HoMLN (raw edge lists) and its TEPS work."""
    i, spec, arrival = arg
    from paper_2207_11662_gb300 import synth
    net = synth.build_request(spec, raw=True)
    work, _ = teps_work(net.n, net.layers)
    return i, net.n, net.layers, arrival, work


def serving(args, dev):
    """Poisson stream (mean 50 req/s) of closeness/top-k queries on HoMLNs of 2-6 layers and
    1,000-100,000 nodes (log-uniform), ER or power-law layers of average degree 6-12, served by the
    continuous-batching server; latency = completion - arrival. The server's default (two workers:
    small requests on a high-priority stream, preempting the persistent BFS of a big request at a
    tile boundary while their wave runs) and, on the same stream, one worker whose waves take the
    whole GPU in arrival order."""
    import multiprocessing as mp
    from paper_2207_11662_gb300 import serve
    from paper_2207_11662_gb300 import synth
    specs = synth.serving_requests(duration_s=args.serve_seconds, rate=args.serve_rate, seed=5001)
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        items = pool.map(_serving_item, [(i, r["spec"], r["t"]) for i, r in enumerate(specs)], chunksize=4)

    def run(**kw):
        reqs = [serve.Request(i, n, layers, arrival=t, teps_work=w) for i, n, layers, t, w in items]
        srv = serve.Server(device=dev.index or 0, max_wave=16, mem_budget_bytes=32 << 30, **kw)
        t0 = time.perf_counter()
        done = srv.run(reqs, realtime=True)
        wall = time.perf_counter() - t0
        out = serve.latency_stats(done, wall, srv.big_work)
        out.update({"duration_s": round(wall, 2), "workers": srv.workers, "waves": srv.waves,
                    "errors": srv.errors[:3]})
        if srv.workers >= 2:
            out["preemptions"] = srv.preemptions
            if srv.small_sms:
                out["small_sms"] = srv.small_sms
        return out

    out = run()
    out["one_worker_whole_gpu"] = run(workers=1)
    out.update({"rate_req_per_s": args.serve_rate, "max_wave": 16,
                "workload": "Poisson arrivals, HoMLNs of 2-6 layers, n log-uniform in [1e3, 1e5], ER or "
                            "Chung-Lu layers (avg deg 6-12); per request: Psi of all layers + AND, top-10% ground "
                            "truth, CC2 estimate and its accuracy; big = nodes x edges > 2e10"})
    return out


class OracleSample:
    """The oracle as it stands: queue BFS from a seeded sample of sources on every analysed graph
    (the layers and their AND graph, built once), OpenMP over the host's cores."""

    def __init__(self, net):
        from oracle import oracle as O
        import scipy.sparse as sps
        from scipy.sparse.csgraph import connected_components
        self.O = O
        self.n = n = net.n
        keys = [O.edge_keys(n, s, d) for s, d in net.layers]
        self.graphs = [O.csr_from_keys(n, k) for k in keys] + [O.csr_from_keys(n, O.and_keys(n, keys))]
        self.comp = []
        for rp, col in self.graphs:
            A = sps.csr_matrix((np.ones(col.shape[0]), col, rp), shape=(n, n))
            nc, lab = connected_components(A, directed=False)
            self.comp.append((lab, np.bincount(lab, weights=np.diff(rp), minlength=nc) / 2))

    def run(self, count, nthreads, rng):
        """GTEPS of the sample (edges of the sources' components / BFS wall time) and the seconds."""
        work, t = 0, 0.0
        for (rp, col), (lab, m_comp) in zip(self.graphs, self.comp):
            src = np.sort(rng.choice(self.n, min(count, self.n), replace=False)).astype(np.int32)
            work += int(np.sum(m_comp[lab[src]]))
            t0 = time.perf_counter()
            self.O.farness_reach(self.n, rp, col, sources=src, threads=nthreads)
            t += time.perf_counter() - t0
        return work / t / 1e9, t


def cpu_baseline(net, sources_per_graph: int, seed: int = 2001, one_core_sources: int = 0, sampler=None):
    """The oracle timed on the host cores on a seeded sample of sources per graph (and, with
    one_core_sources, a smaller sample on one core)."""
    sampler = sampler or OracleSample(net)
    threads = os.cpu_count() or 1
    value, t = sampler.run(sources_per_graph, threads, np.random.default_rng(seed))
    out = {"value": round(value, 4), "unit": "GTEPS", "cores": threads, "kind": "oracle",
           "sample": f"queue BFS from {sources_per_graph} seeded sources on each of the {len(sampler.graphs)} graphs "
                     f"(4 layers + AND), {t:.1f} s wall on {threads} threads ({t * threads:.0f} core-seconds), "
                     f"OpenMP over sources"}
    if one_core_sources:
        v1, t1 = sampler.run(one_core_sources, 1, np.random.default_rng(seed + 1))
        out["one_core_value"] = round(v1, 4)
        out["one_core_sample"] = f"{one_core_sources} seeded sources per graph on 1 thread, {t1:.1f} s"
    return out


def summary(result: dict) -> dict:
    """The few figures a reader wants first, kept at the end of the line."""
    r = result.get("roofline", {})
    out = {"headline": f"{result['value']} GTEPS, {result['ms_per_step']} ms/step (200k BA)"
                       if "200000" in result["config"]["workload"] else f"{result['value']} GTEPS",
           "bfs_alg_frac": r.get("frac"), "bfs_dram_frac": r.get("dram_frac"),
           "e2e_gteps": result["e2e"]["value"]}
    for name, c in result.get("configs", {}).items():
        out[f"{name}_gteps"] = c["gteps"]
        out[f"{name}_bfs_alg_frac"] = c["roofline"]["frac"]
    b = result.get("batched_vs_plain")
    if b:
        out["batched"] = {"batched_ms": b["batched_ms"], "graph_replay_ms": b["graph_replay_ms"],
                          "plain_ms": b["plain_ms"], "speedup_vs_plain": b["speedup_vs_plain"],
                          "graph_speedup_vs_plain": b["graph_speedup_vs_plain"],
                          "identical_outputs": b["identical_outputs"]}
    v = result.get("serving")
    if v:
        out["serving"] = {k: v[k] for k in ("p50_ms", "p90_ms", "p99_ms", "req_per_s") if k in v}
        out["serving"]["small_p99_ms"] = v["small"]["p99_ms"]
        out["serving"]["big_p99_ms"] = v["big"]["p99_ms"]
        one = v.get("one_worker_whole_gpu")
        if one:
            out["serving"]["one_worker"] = {k: one[k] for k in ("p50_ms", "p90_ms", "p99_ms")}
            out["serving"]["one_worker"]["small_p99_ms"] = one["small"]["p99_ms"]
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    dist = None
    if args.impl == "reference":
        if rank != 0:
            return
        net, desc = make_workload(args.workload, 0)
        sampler = OracleSample(net)  # the graphs are built once; a step is one bounded BFS sample
        per_step = max(1, args.cpu_sample_sources // 2)
        for _ in range(args.warmup):
            cpu_baseline(net, max(50, per_step // 10), sampler=sampler)
        vals, secs = [], []
        for k in range(args.steps):
            t0 = time.perf_counter()
            vals.append(cpu_baseline(net, per_step, seed=2001 + k, sampler=sampler))
            secs.append(time.perf_counter() - t0)
        v = statistics.mean(x["value"] for x in vals)
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GTEPS",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": round(1000.0 * statistics.mean(secs), 3), "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                          "config": {"workload": desc},
                          "cpu_baseline": dict(vals[-1], value=round(v, 4)),
                          "e2e": {"value": round(v, 4), "unit": "GTEPS", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", init_method="env://")
        dist = tdist
    result, net = run_ours(args, rank, world, dist)
    if result is None:
        return
    if rank == 0:
        import torch
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
        extra = {}
        if args.secondary != "none" and args.secondary != args.workload and world == 1:
            extra["configs"] = {args.secondary: secondary_config(args, args.secondary, dev)}
        if not args.no_batch and world == 1:
            extra["batched_vs_plain"] = batch_vs_plain(args, dev)
        if not args.no_serve and world == 1:
            extra["serving"] = serving(args, dev)
        if not args.no_paper_like and world == 1:
            extra["paper_like"] = paper_like(args, dev)
        if not args.no_widened and world == 1:
            extra["widened"] = widened(args, dev)
        if not args.no_cpu_baseline and world == 1:
            result["cpu_baseline"] = cpu_baseline(net, args.cpu_sample_sources, one_core_sources=150)
        # headline keys first, the long detail next, the summary last
        head = {k: result.pop(k) for k in list(result)
                if k not in ("per_graph", "accuracy_vs_ground_truth", "bfs_profile")}
        out = dict(head)
        out.update(result)
        out.update(extra)
        out["summary"] = summary(out)
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
