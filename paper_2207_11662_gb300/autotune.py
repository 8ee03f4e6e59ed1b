"""Autotuner for the persistent multi-source BFS.

Picks the team count, the words per node W (64*W sources per tile) and the
top-down threshold alpha for a set of graphs by timing real launches of
homln_batch_analyse on the GPU. Results are cached per workload class (graph
count, largest node count and edge count, bucketed) in a JSON file under the
build directory, so a serving process or a benchmark tunes once.
"""
from __future__ import annotations

import json
import math
import os

from . import homln as H

_CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build", "autotune.json")

# (teams, words per node, alpha); W = 0 lets the library size W to its state budget
DEFAULT_CANDIDATES = [
    (8, 0, 16), (4, 0, 16), (16, 0, 16), (32, 0, 16), (76, 0, 16), (152, 0, 16),
    (8, 0, 32), (16, 0, 4), (32, 0, 4),
]


def workload_key(ns, edges) -> str:
    """Bucket a workload: graph count, largest n and total edges, each to a power of two."""
    b = lambda x: int(math.log2(max(int(x), 1)))
    return f"g{b(len(ns))}-n{b(max(ns))}-e{b(sum(edges))}"


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


def time_batch(handles, masks, with_and, stream_ptr: int, tuning: dict, reps: int = 1) -> float:
    """Milliseconds of one homln_batch_analyse (best of reps), CUDA events on the launch stream."""
    import torch
    stream = torch.cuda.ExternalStream(stream_ptr) if stream_ptr else torch.cuda.current_stream()
    H.homln_set_tuning(handles[0], **tuning)
    best = float("inf")
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
        best = min(best, e0.elapsed_time(e1))
    return best


def tune(handles, masks, ns, edges, with_and=True, stream_ptr: int = 0, candidates=None, use_cache=True,
         reps: int = 1):
    """Best tuning dict for this set of graphs (and the timings of every candidate)."""
    key = workload_key(ns, edges)
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key]["tuning"], cache[key]
    results = []
    time_batch(handles, masks, with_and, stream_ptr, {}, 1)  # untimed: builds the BFS graphs once
    for teams, words, alpha in candidates or DEFAULT_CANDIDATES:
        t = dict(teams=teams, words_per_node=words, push_alpha=alpha)
        try:
            ms = time_batch(handles, masks, with_and, stream_ptr, t, reps)
        except H.HomlnError:
            continue
        results.append((ms, t))
    results.sort(key=lambda x: x[0])
    best = results[0][1]
    entry = {"tuning": best, "candidates": [{"ms": round(ms, 3), **t} for ms, t in results]}
    if use_cache:
        cache[key] = entry
        _store(cache)
    for h in handles:
        H.homln_invalidate(h)
    return best, entry
