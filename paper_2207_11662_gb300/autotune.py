"""Autotuner for the persistent multi-source BFS.

Picks the words per node W (64*W sources per tile), the team count and the
top-down threshold alpha for a set of graphs by timing real launches of
homln_batch_analyse on the GPU. The search is coordinate-wise: W first (at two
values of alpha, teams at the library's default), then the team count at the best W, then
alpha at the best (W, teams), then whether the blocks that share an SM join the same team or
different ones (team_mix). Every candidate is timed ``reps`` times (at
least 3) and scored by its median. Results are cached per workload class
(graph count, largest node count, total edges and degree skew, each bucketed
to a power of two) in a JSON file under the build directory, so a serving
process or a benchmark tunes once.
"""
from __future__ import annotations

import json
import math
import os
import statistics

from . import homln as H

_CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build", "autotune.json")

WORDS = (4, 8, 16, 32)           # 256 .. 2048 sources per tile
TEAMS = (0, 4, 8, 16, 32, 76, 152)  # 0: the library's default for the chosen W
ALPHAS = (4, 16, 64)             # top-down while alpha * frontier edges < unfinished edges
STATE_LIMIT = 2.0e9              # bytes of BFS state a candidate may take (2 snapshots of n x W words per team)


def workload_key(ns, edges, skew: float = 1.0) -> str:
    """Bucket a workload: graph count, largest n, total edges and degree skew (max / mean degree),
    each to a power of two."""
    b = lambda x: int(math.log2(max(int(x), 1)))
    return f"g{b(len(ns))}-n{b(max(ns))}-e{b(sum(edges))}-s{b(skew)}"


def degree_skew(n: int, layers) -> float:
    """Largest max-degree / mean-degree ratio over the layers of one network (edge lists as given)."""
    import numpy as np
    worst = 1.0
    for s, d in layers:
        s = np.asarray(s)
        d = np.asarray(d)
        if s.size == 0:
            continue
        deg = np.bincount(np.concatenate([s, d]), minlength=n)
        worst = max(worst, float(deg.max()) / max(float(deg.mean()), 1e-9))
    return worst


def _load():
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache):
    os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
    tmp = _CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, _CACHE)


def time_batch(handles, masks, with_and, stream_ptr: int, tuning: dict, reps: int = 3) -> float:
    """Median milliseconds of homln_batch_analyse over reps runs, CUDA events on the launch stream."""
    import torch
    stream = torch.cuda.ExternalStream(stream_ptr) if stream_ptr else torch.cuda.current_stream()
    H.homln_set_tuning(handles[0], **tuning)
    times = []
    for _ in range(reps):
        for h in handles:
            H.homln_invalidate(h)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        H.homln_batch_analyse(handles, masks, with_and)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def tune(handles, masks, ns, edges, with_and=True, stream_ptr: int = 0, use_cache=True, reps: int = 3,
         skew: float = 1.0, words=WORDS, teams=TEAMS, alphas=ALPHAS):
    """Best tuning dict for this set of graphs, and a log of every candidate timed."""
    reps = max(3, int(reps))
    key = workload_key(ns, edges, skew)
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key]["tuning"], cache[key]
    maxn = max(ns)
    time_batch(handles, masks, with_and, stream_ptr, {}, 1)  # untimed: builds the BFS graphs once
    results = []
    seen = {}

    def run(t):
        k = tuple(sorted(t.items()))
        if k not in seen:
            try:
                seen[k] = time_batch(handles, masks, with_and, stream_ptr, t, reps)
            except H.HomlnError:
                seen[k] = float("inf")
            results.append((seen[k], dict(t)))
        return seen[k]

    # W: no wider than the node count needs, one team's state within the limit
    ws = [w for w in words if 64 * (w // 2) < maxn and 2.0 * maxn * 8.0 * w <= STATE_LIMIT] or [1]
    # W together with two direction thresholds: a wide tile can win only with more top-down levels
    best = min(({"words_per_node": w, "teams": 0, "push_alpha": a} for w in ws for a in (4, 16)), key=run)
    tiles = sum(-(-n // (64 * best["words_per_node"])) for n in ns)
    per_team = 2.0 * maxn * 8.0 * best["words_per_node"]
    tcands = [t for t in teams if t == 0 or (t <= tiles and t * per_team <= STATE_LIMIT)]
    best = min((dict(best, teams=t) for t in tcands), key=run)
    best = min((dict(best, push_alpha=a) for a in alphas), key=run)
    best = min((dict(best, team_mix=m) for m in (0, 1)), key=run)
    results.sort(key=lambda x: x[0])
    entry = {"tuning": best, "key": key, "reps": reps,
             "candidates": [{"ms": round(ms, 3), **t} for ms, t in results]}
    if use_cache:
        cache[key] = entry
        _store(cache)
    for h in handles:
        H.homln_invalidate(h)
    return best, entry
