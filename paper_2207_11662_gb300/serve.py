"""Serving loop: closeness queries on HoMLNs arriving over time, batched continuously.

Each request carries a HoMLN (n shared nodes, 2-6 layers as host edge lists) and
asks for the paper's decoupled pipeline on all its layers: closeness of every
layer and of the AND aggregate, the ground-truth top-k CC nodes, the CC2 estimate
(Section 5.2, Algorithm 1) and its accuracy against the ground truth.

Scheduling:
  * admission by device memory: a request is admitted only while the sum of the
    estimated device footprints of the requests in flight stays under the budget;
    a request that can never fit is rejected (HOMLN_ENOMEM) at once;
  * continuous batching: worker threads, each with its own CUDA stream, repeatedly
    take admitted requests that are waiting (up to ``max_wave``) and run them as one
    wave: CSR builds, then one persistent BFS launch over all (graph, source batch)
    tiles of the wave (homln_batch_analyse), then selection, composition and
    accuracy. Requests that arrive while a wave is on the GPU join the next wave of
    a free worker;
  * size classes and preemption: a request is "big" when its BFS work (nodes x edges)
    exceeds ``big_work``. With two or more workers (the default is two), worker 0 serves
    only small requests, on a high-priority stream; the other workers take big requests
    first (then small ones). The big waves' persistent BFS watches a yield flag
    (homln_set_yield) that worker 0 raises while one of its waves runs: the big BFS then
    finishes the tiles it has started, gives the GPU to the small wave and resumes its
    remaining tiles when the flag is lowered. So a small request that arrives while a big
    one is on the GPU waits about one BFS tile, not the whole big request. (``small_sms``
    instead splits the GPU by SMs between the two kinds of waves, without preemption;
    measured slower.) With one worker every wave takes the whole GPU, in arrival order;
  * no collector pauses: Python's full (oldest-generation) cyclic garbage collection
    walks every tracked object of the process while holding the interpreter lock; with
    torch loaded that is ~10^5 objects and tens of ms, during which no worker thread can
    launch or collect a wave. ``freeze_gc`` (default on) moves the objects that exist
    when ``run`` starts out of the collector's view for the run (``gc.freeze``) and
    gives them back afterwards (``gc.unfreeze``, which also undoes a freeze the process
    made before), so a collection during the run only walks what the run itself created.

Every GPU step runs in libhomln.so; this module only schedules.
"""
from __future__ import annotations

import collections
import contextlib
import gc
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import homln as H

ENOMEM_REJECT = "request can never fit the device memory budget"


@dataclass
class Request:
    rid: int
    n: int
    layers: list  # host (src, dst) int32 arrays
    arrival: float = 0.0  # seconds, relative to the start of the run
    teps_work: int = 0
    # filled in by the server
    t_submit: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0
    wave: int = -1
    status: int = H.HOMLN_OK
    error: str = ""
    gt: np.ndarray | None = None
    cc2: np.ndarray | None = None
    accuracy: dict = field(default_factory=dict)
    farness: list | None = None  # per layer + AND (kept only when requested)


def footprint_bytes(n: int, edge_counts) -> int:
    """Estimated peak device bytes of one request: the layer CSRs and their relabelled copies,
    the AND graph, the construction scratch, the per-graph outputs and the BFS state (per team
    2 snapshots of n x 8 words and 3 bytes per node; the library's default team count: at least
    16, up to about 240 MB of state in all, and no more teams than tiles of 512 sources)."""
    m = int(sum(edge_counts))
    L = len(edge_counts)
    csr = 2 * (8 * (n + 1) * (L + 1) + 8 * m)  # rowptr + col (symmetric), original and relabelled
    build = 8 * 2 * max(edge_counts, default=0) * 3  # sort keys, alternate keys, flags of one layer
    outputs = (L + 1) * n * (8 + 4 + 8 + 8 + 4)
    tiles = (L + 1) * -(-n // 512)
    teams = max(1, min(tiles, max(16, int(2.4e8 // (2 * 8 * 8 * max(n, 1))))))
    bfs_state = teams * (2 * 8 * 8 + 3) * n
    return int(csr + build + outputs + bfs_state + (1 << 20))


SMALL, BIG = 0, 1


class Admission:
    """FIFO admission per size class under one device-memory budget (host logic only)."""

    def __init__(self, budget_bytes: int):
        self.budget = int(budget_bytes)
        self.in_use = 0
        self.queues = (collections.deque(), collections.deque())  # SMALL, BIG
        self.lock = threading.Lock()
        self.cv = threading.Condition(self.lock)
        self.closed = False

    @property
    def waiting(self):
        return list(self.queues[SMALL]) + list(self.queues[BIG])

    def submit(self, req: Request, need: int, cls: int = SMALL) -> bool:
        """Queue a request; False (and no queueing) if it can never fit."""
        with self.cv:
            if need > self.budget:
                return False
            self.queues[cls].append((req, need))
            self.cv.notify_all()
            return True

    def _prefix(self, q, max_items):
        out = []
        while q and len(out) < max_items:
            req, need = q[0]
            if self.in_use + need > self.budget:
                break
            q.popleft()
            self.in_use += need
            out.append((req, need))
        return out

    def take(self, max_items: int, timeout: float, classes=None):
        """Admit the longest FIFO prefix that fits (at least one item when it fits) of the first
        class in `classes` that has one -- or, with classes=None, of the class whose oldest request
        was submitted first (FIFO across classes); blocks up to timeout. None once closed and
        drained."""
        deadline = time.monotonic() + timeout
        with self.cv:
            while True:
                order = classes
                if order is None:
                    heads = [(q[0][0].t_submit, c) for c, q in enumerate(self.queues) if q]
                    order = [c for _, c in sorted(heads)]
                for cls in order:
                    out = self._prefix(self.queues[cls], max_items)
                    if out:
                        return out
                if self.closed and not any(self.queues[c] for c in (classes or (SMALL, BIG))):
                    return None
                left = deadline - time.monotonic()
                if left <= 0:
                    return []
                self.cv.wait(left)

    def release(self, need: int):
        with self.cv:
            self.in_use -= need
            self.cv.notify_all()

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()


@contextlib.contextmanager
def gc_frozen(enabled: bool = True):
    """Keep the objects that exist on entry out of the cyclic collector until exit (gc.freeze);
    on exit every frozen object goes back to the oldest generation (gc.unfreeze), including any
    the process had frozen before entry."""
    if not enabled:
        yield
        return
    gc.freeze()
    try:
        yield
    finally:
        gc.unfreeze()


def work_estimate(n: int, edge_counts) -> int:
    """BFS work of a request, nodes x edges over its layers (a bound on its edge visits / 2)."""
    return int(n) * int(sum(edge_counts))


class Server:
    def __init__(self, device: int = 0, workers: int = 2, max_wave: int = 16, mem_budget_bytes: int = 16 << 30,
                 percent: float = 10.0, keep_farness: bool = False, tuning: dict | None = None,
                 big_work: float = 2e10, preempt: bool = True, small_sms: int = 0, big_max_tiles: int = 0,
                 freeze_gc: bool = True):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.workers = workers
        self.max_wave = max_wave
        self.big_work = big_work
        self.nsm = torch.cuda.get_device_properties(self.device).multi_processor_count
        self.small_sms = max(0, min(int(small_sms), self.nsm - 1))
        self.preempt = bool(preempt) and workers >= 2 and self.small_sms == 0
        self.big_max_tiles = big_max_tiles
        self.freeze_gc = bool(freeze_gc)
        self._yield = None          # the yield flag big waves watch (preempt)
        self._small_active = 0      # small waves running; the flag is raised while > 0
        self._ylock = threading.Lock()
        self.preemptions = 0
        self.adm = Admission(mem_budget_bytes)
        self.sel = H.make_select(H.HOMLN_TOPK_PERCENT, percent)
        self.keep_farness = keep_farness
        self.tuning = dict(tuning or {})
        self.done = []
        self.done_lock = threading.Lock()
        self.t0 = 0.0
        self.waves = 0
        self.errors = []

    # ---------------------------------------------------------------- workers
    def _small_wave(self, start: bool):
        """Raise the yield flag while at least one small wave runs."""
        with self._ylock:
            self._small_active += 1 if start else -1
            H.homln_yield_set(self._yield, self._small_active > 0)

    def _run_wave(self, items, stream, wave_id, tuning, small_only=False):
        reqs = [r for r, _ in items]
        t_admit = time.perf_counter() - self.t0
        handles = []
        preempting = self._yield is not None and small_only
        if preempting:
            self._small_wave(True)
        try:
            for r in reqs:
                r.t_admit = t_admit
                r.wave = wave_id
                handles.append(H.homln_create(r.n, r.layers, stream=stream.cuda_stream))
            H.homln_set_tuning(handles[0], **tuning)
            if self._yield is not None and not small_only:
                H.homln_set_yield(handles[0], self._yield)
            masks = [(1 << len(r.layers)) - 1 for r in reqs]
            H.homln_batch_analyse(handles, masks, True)
            for r, h, mask in zip(reqs, handles, masks):
                gt = np.empty(r.n, np.int32)
                est = np.empty(r.n, np.int32)
                cg = H.homln_topk(h, -1, mask, self.sel, gt)
                ce = H.homln_compose(h, mask, H.HOMLN_CC2, self.sel, est)
                r.gt, r.cc2 = gt[:cg].copy(), est[:ce].copy()
                r.accuracy = H.homln_accuracy(h, r.cc2, ce, r.gt, cg)
                if self.keep_farness:
                    fs = []
                    for i in range(len(r.layers)):
                        F = np.empty(r.n, np.uint64)
                        H.homln_layer_closeness(h, i, F, None, None)
                        fs.append(F)
                    F = np.empty(r.n, np.uint64)
                    H.homln_and_closeness(h, mask, F, None, None)
                    fs.append(F)
                    r.farness = fs
        except H.HomlnError as e:
            for r in reqs:
                r.status, r.error = e.code, str(e)
        finally:
            for h in handles:
                H.homln_destroy(h)
            if preempting:
                self._small_wave(False)
            t_done = time.perf_counter() - self.t0
            for r, need in items:
                r.t_done = t_done
                self.adm.release(need)
            with self.done_lock:
                self.done.extend(reqs)

    def _worker(self, idx):
        torch = self.torch
        torch.cuda.set_device(self.device)
        # worker 0 of two or more serves small requests only, at high priority (preempting the big
        # waves, or on small_sms SMs' worth of BFS blocks); the others take big requests first
        small_only = self.workers >= 2 and idx == 0
        classes = (SMALL,) if small_only else (BIG, SMALL) if self.workers >= 2 else None
        stream = torch.cuda.Stream(self.device, priority=-1 if small_only else 0)
        tuning = dict(self.tuning)
        if self.workers >= 2 and self.small_sms:
            tuning.setdefault("sm_count", self.small_sms if small_only else self.nsm - self.small_sms)
        if not small_only and self.big_max_tiles:
            tuning.setdefault("max_tiles_per_launch", self.big_max_tiles)
        while True:
            items = self.adm.take(self.max_wave, timeout=0.05, classes=classes)
            if items is None:
                return
            if not items:
                continue
            with self.done_lock:
                wave_id = self.waves
                self.waves += 1
            try:
                self._run_wave(items, stream, wave_id, tuning, small_only)
            except Exception as e:  # keep serving; record the failure
                self.errors.append(repr(e))

    # ---------------------------------------------------------------- driver
    def submit(self, req: Request):
        req.t_submit = time.perf_counter() - self.t0
        counts = [s.shape[0] for s, _ in req.layers]
        cls = BIG if work_estimate(req.n, counts) > self.big_work else SMALL
        if not self.adm.submit(req, footprint_bytes(req.n, counts), cls):
            req.status, req.error = H.HOMLN_ENOMEM, ENOMEM_REJECT
            req.t_admit = req.t_done = req.t_submit
            with self.done_lock:
                self.done.append(req)

    def run(self, requests, realtime: bool = True):
        """Replay the requests at their arrival times (or all at once) and serve them; returns them done."""
        with gc_frozen(self.freeze_gc):
            return self._run(requests, realtime)

    def _run(self, requests, realtime: bool):
        self.t0 = time.perf_counter()
        self.done = []
        if self.preempt:
            self.torch.cuda.set_device(self.device)
            self._yield = H.homln_yield_create()
            self._small_active = 0
        threads = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(self.workers)]
        for t in threads:
            t.start()
        for r in sorted(requests, key=lambda r: r.arrival):
            if realtime:
                delay = r.arrival - (time.perf_counter() - self.t0)
                if delay > 0:
                    time.sleep(delay)
            self.submit(r)
        self.adm.close()
        for t in threads:
            t.join()
        self.torch.cuda.synchronize(self.device)
        if self._yield is not None:
            self.preemptions = H.homln_yield_count(self._yield)
            H.homln_yield_destroy(self._yield)
            self._yield = None
        return sorted(self.done, key=lambda r: r.rid)


def latency_stats(done, wall_s: float, big_work: float = 2e10) -> dict:
    """Latency (completion - arrival) percentiles over the completed requests, overall and per size
    class (BFS work nodes x edges above or below big_work)."""
    ok = [r for r in done if r.status == H.HOMLN_OK]

    def pct(rs):
        lat = np.array([(r.t_done - r.arrival) * 1000.0 for r in rs]) if rs else np.zeros(1)
        return lat

    lat = pct(ok)
    big = [r for r in ok if work_estimate(r.n, [s.shape[0] for s, _ in r.layers]) > big_work]
    small = [r for r in ok if r not in big]
    out = {"requests": len(done), "completed": len(ok), "rejected": len(done) - len(ok),
           "p50_ms": round(float(np.percentile(lat, 50)), 3), "p90_ms": round(float(np.percentile(lat, 90)), 3),
           "p99_ms": round(float(np.percentile(lat, 99)), 3),
           "mean_ms": round(float(lat.mean()), 3), "req_per_s": round(len(ok) / wall_s, 2),
           "gteps": round(sum(r.teps_work for r in ok) / wall_s / 1e9, 2)}
    for name, rs in (("small", small), ("big", big)):
        la = pct(rs)
        out[name] = {"count": len(rs), "p50_ms": round(float(np.percentile(la, 50)), 3),
                     "p99_ms": round(float(np.percentile(la, 99)), 3)}
    return out
