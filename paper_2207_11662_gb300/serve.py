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
    take every admitted request that is waiting (up to ``max_wave``) and run them as
    one wave: CSR builds, then one persistent BFS launch over all (graph, source
    batch) tiles of the wave (homln_batch_analyse) on the whole GPU, then selection,
    composition and accuracy. Requests that arrive while a wave is on the GPU join
    the next wave of any free worker; a second worker prepares its wave (CSR builds,
    selections) while the other's BFS runs. Measured on GB300 at 50 requests/s:
    whole-GPU waves with two workers gave p50 9 ms / p99 127 ms, against 26 ms /
    326 ms for three workers whose waves took one block per SM each.

Every GPU step runs in libhomln.so; this module only schedules.
"""
from __future__ import annotations

import collections
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
    the AND graph, the construction scratch, the per-graph outputs and the BFS state (16 teams
    of 3 arrays of n x 8 words and 3 bytes per node at most)."""
    m = int(sum(edge_counts))
    L = len(edge_counts)
    csr = 2 * (8 * (n + 1) * (L + 1) + 8 * m)  # rowptr + col (symmetric), original and relabelled
    build = 8 * 2 * max(edge_counts, default=0) * 3  # sort keys, alternate keys, flags of one layer
    outputs = (L + 1) * n * (8 + 4 + 8 + 8 + 4)
    bfs_state = 16 * (3 * 8 * 8 + 3) * n
    return int(csr + build + outputs + bfs_state + (1 << 20))


class Admission:
    """FIFO admission under a device-memory budget (host logic only)."""

    def __init__(self, budget_bytes: int):
        self.budget = int(budget_bytes)
        self.in_use = 0
        self.waiting = collections.deque()
        self.lock = threading.Lock()
        self.cv = threading.Condition(self.lock)
        self.closed = False

    def submit(self, req: Request, need: int) -> bool:
        """Queue a request; False (and no queueing) if it can never fit."""
        with self.cv:
            if need > self.budget:
                return False
            self.waiting.append((req, need))
            self.cv.notify_all()
            return True

    def take(self, max_items: int, timeout: float):
        """Admit the longest FIFO prefix that fits (at least one item when it fits); blocks up to timeout."""
        deadline = time.monotonic() + timeout
        with self.cv:
            while True:
                out = []
                while self.waiting and len(out) < max_items:
                    req, need = self.waiting[0]
                    if self.in_use + need > self.budget:
                        break
                    self.waiting.popleft()
                    self.in_use += need
                    out.append((req, need))
                if out:
                    return out
                if self.closed and not self.waiting:
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


class Server:
    def __init__(self, device: int = 0, workers: int = 2, max_wave: int = 16, mem_budget_bytes: int = 16 << 30,
                 percent: float = 10.0, keep_farness: bool = False, tuning: dict | None = None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.workers = workers
        self.max_wave = max_wave
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
    def _run_wave(self, items, stream, wave_id):
        reqs = [r for r, _ in items]
        t_admit = time.perf_counter() - self.t0
        handles = []
        try:
            for r in reqs:
                r.t_admit = t_admit
                r.wave = wave_id
                handles.append(H.homln_create(r.n, r.layers, stream=stream.cuda_stream))
            H.homln_set_tuning(handles[0], **self.tuning)
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
            t_done = time.perf_counter() - self.t0
            for r, need in items:
                r.t_done = t_done
                self.adm.release(need)
            with self.done_lock:
                self.done.extend(reqs)

    def _worker(self, idx):
        torch = self.torch
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(self.device)
        while True:
            items = self.adm.take(self.max_wave, timeout=0.05)
            if items is None:
                return
            if not items:
                continue
            with self.done_lock:
                wave_id = self.waves
                self.waves += 1
            try:
                self._run_wave(items, stream, wave_id)
            except Exception as e:  # keep serving; record the failure
                self.errors.append(repr(e))

    # ---------------------------------------------------------------- driver
    def submit(self, req: Request):
        req.t_submit = time.perf_counter() - self.t0
        if not self.adm.submit(req, footprint_bytes(req.n, [s.shape[0] for s, _ in req.layers])):
            req.status, req.error = H.HOMLN_ENOMEM, ENOMEM_REJECT
            req.t_admit = req.t_done = req.t_submit
            with self.done_lock:
                self.done.append(req)

    def run(self, requests, realtime: bool = True):
        """Replay the requests at their arrival times (or all at once) and serve them; returns them done."""
        self.t0 = time.perf_counter()
        self.done = []
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
        return sorted(self.done, key=lambda r: r.rid)


def latency_stats(done, wall_s: float) -> dict:
    ok = [r for r in done if r.status == H.HOMLN_OK]
    lat = np.array([(r.t_done - r.arrival) * 1000.0 for r in ok]) if ok else np.zeros(1)
    return {"requests": len(done), "completed": len(ok), "rejected": len(done) - len(ok),
            "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3), "req_per_s": round(len(ok) / wall_s, 2),
            "gteps": round(sum(r.teps_work for r in ok) / wall_s / 1e9, 2)}
