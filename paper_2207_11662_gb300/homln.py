"""Python binding of the homln C-ABI (``include/homln.h``).

Argument marshalling only: every computation runs in ``libhomln.so``'s CUDA
kernels. The functions below carry the C names and take torch tensors (CUDA or
CPU), numpy arrays or raw integer pointers. ``Network`` wraps a handle and
returns torch CUDA tensors.

If ``libhomln.so`` has not been built, importing this module raises: there is
no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_size_t, c_uint32, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhomln.so")

HOMLN_OK, HOMLN_EINVAL, HOMLN_ENOMEM, HOMLN_ECUDA, HOMLN_ERANGE, HOMLN_ETIMEOUT, HOMLN_EBUSY = range(7)
HOMLN_PTR_HOST, HOMLN_PTR_DEVICE, HOMLN_DIRECTED = 0, 1, 2
HOMLN_NAIVE, HOMLN_CC1, HOMLN_CC2 = 0, 1, 2
HOMLN_TOPK_PERCENT, HOMLN_TOPK_COUNT, HOMLN_GE_MEAN, HOMLN_GT_MEAN = 0, 1, 2, 3
MAX_NODES = 1 << 20
MAX_LAYERS = 64
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ERANGE", 5: "ETIMEOUT", 6: "EBUSY"}

# Every symbol the header declares (checked by the CPU tests).
EXPORTS = [
    "homln_create", "homln_destroy", "homln_set_tuning", "homln_layer_closeness", "homln_and_aggregate",
    "homln_and_closeness", "homln_topk", "homln_compose", "homln_accuracy", "homln_set_profiling",
    "homln_get_profile", "homln_reset_profile", "homln_kernel_launches", "homln_sync", "homln_last_error",
    "homln_version", "homln_accuracy_noalloc", "homln_analyse", "homln_batch_analyse", "homln_invalidate",
    "homln_subset_sweep", "homln_or_aggregate", "homln_or_closeness", "homln_export_partials",
    "homln_import_partials", "homln_graph_capture", "homln_graph_launch", "homln_graph_destroy",
    "homln_shard_partials", "homln_batch_closeness", "homln_yield_create", "homln_yield_destroy",
    "homln_yield_set", "homln_yield_count", "homln_set_yield",
]


class homln_select(ctypes.Structure):
    _fields_ = [("mode", c_int32), ("reserved", c_int32), ("percent", c_double), ("k", c_int64),
                ("cc1_overlap", c_double)]


class homln_accuracy_t(ctypes.Structure):
    _fields_ = [("tp", c_int64), ("fp", c_int64), ("fn", c_int64), ("jaccard", c_double),
                ("precision", c_double), ("recall", c_double), ("f1", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class homln_subset_result(ctypes.Structure):
    _fields_ = [("mask", c_uint64), ("truth_count", c_int32), ("estimate_count", c_int32),
                ("acc", homln_accuracy_t)]


class homln_tuning(ctypes.Structure):
    _fields_ = [("words_per_node", c_int32), ("push_alpha", c_int32), ("threads", c_int32),
                ("blocks_per_sm", c_int32), ("relabel", c_int32), ("teams", c_int32), ("team_mix", c_int32),
                ("schedule", c_int32), ("wait_limit_ms", c_int32), ("test_phantom_blocks", c_int32),
                ("max_tiles_per_launch", c_int32), ("sm_count", c_int32)]


class homln_profile_t(ctypes.Structure):
    _fields_ = [("bfs_launches", c_int64), ("bfs_timed_launches", c_int64), ("bfs_ms", c_double),
                ("levels", c_int64), ("pull_levels", c_int64), ("push_levels", c_int64), ("batches", c_int64),
                ("edges_scanned", c_int64), ("words_gathered", c_int64), ("edges_pushed", c_int64),
                ("words_pushed", c_int64), ("bytes", c_int64), ("visits", c_int64), ("words_per_node", c_int32),
                ("teams", c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_void_p, c_size_t, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p, c_size_t, c_void_p)


class homln_allocator(ctypes.Structure):
    _fields_ = [("ctx", c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


class HomlnError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() (no fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    S = c_int32  # homln_status
    sig = {
        "homln_create": (S, [c_int32, c_int32, POINTER(c_int64), POINTER(c_void_p), POINTER(c_void_p), c_uint32,
                             POINTER(homln_allocator), c_void_p, POINTER(c_void_p)]),
        "homln_destroy": (S, [c_void_p]),
        "homln_set_tuning": (S, [c_void_p, POINTER(homln_tuning)]),
        "homln_layer_closeness": (S, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
        "homln_analyse": (S, [c_void_p, c_uint64, c_int32]),
        "homln_batch_analyse": (S, [POINTER(c_void_p), c_int32, POINTER(c_uint64), c_int32]),
        "homln_and_aggregate": (S, [c_void_p, c_uint64, c_int64, c_void_p, c_void_p, POINTER(c_int64)]),
        "homln_and_closeness": (S, [c_void_p, c_uint64, c_void_p, c_void_p, c_void_p]),
        "homln_or_aggregate": (S, [c_void_p, c_uint64, c_int64, c_void_p, c_void_p, POINTER(c_int64)]),
        "homln_or_closeness": (S, [c_void_p, c_uint64, c_void_p, c_void_p, c_void_p]),
        "homln_topk": (S, [c_void_p, c_int32, c_uint64, POINTER(homln_select), c_void_p, POINTER(c_int32)]),
        "homln_compose": (S, [c_void_p, c_uint64, c_int32, POINTER(homln_select), c_void_p, POINTER(c_int32)]),
        "homln_accuracy": (S, [c_void_p, c_void_p, c_int32, c_void_p, c_int32, POINTER(homln_accuracy_t)]),
        "homln_set_profiling": (S, [c_void_p, c_int32, c_int32]),
        "homln_get_profile": (S, [c_void_p, POINTER(homln_profile_t)]),
        "homln_reset_profile": (S, [c_void_p]),
        "homln_kernel_launches": (c_int64, []),
        "homln_sync": (S, [c_void_p]),
        "homln_invalidate": (S, [c_void_p]),
        "homln_subset_sweep": (S, [c_void_p, c_int32, POINTER(homln_select), c_int32, POINTER(homln_subset_result),
                                   c_int32, POINTER(c_int32)]),
        "homln_export_partials": (S, [c_void_p, c_int32, c_uint64, c_void_p, c_void_p, c_void_p]),
        "homln_graph_capture": (S, [POINTER(c_void_p), c_int32, POINTER(c_uint64), c_int32, POINTER(c_void_p)]),
        "homln_graph_launch": (S, [c_void_p]),
        "homln_shard_partials": (S, [c_void_p, c_int32, c_uint64, c_int32, c_int32, c_void_p, c_void_p]),
        "homln_batch_closeness": (S, [POINTER(c_void_p), c_int32, c_void_p]),
        "homln_graph_destroy": (S, [c_void_p]),
        "homln_import_partials": (S, [c_void_p, c_int32, c_uint64, c_void_p, c_void_p]),
        "homln_last_error": (c_char_p, []),
        "homln_version": (c_char_p, []),
        "homln_accuracy_noalloc": (S, [c_int32, c_void_p, c_int32, c_void_p, c_int32, c_void_p,
                                       POINTER(homln_accuracy_t)]),
        "homln_yield_create": (S, [POINTER(c_void_p)]),
        "homln_yield_destroy": (S, [c_void_p]),
        "homln_yield_set": (S, [c_void_p, c_int32]),
        "homln_yield_count": (S, [c_void_p, POINTER(c_int64)]),
        "homln_set_yield": (S, [c_void_p, c_void_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _check(rc: int, where: str):
    if rc != HOMLN_OK:
        raise HomlnError(rc, where, lib.homln_last_error().decode())


def ptr(x) -> int | None:
    """Address of a torch tensor, numpy array or integer (None stays NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def make_select(mode: int = HOMLN_TOPK_PERCENT, percent: float = 10.0, k: int = 0, cc1_overlap: float = 0.5):
    return homln_select(int(mode), 0, float(percent), int(k), float(cc1_overlap))


def torch_allocator():
    """An allocator struct backed by torch's caching allocator (keep the returned object alive)."""
    import torch

    @ALLOC_FN
    def _alloc(ctx, nbytes, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except RuntimeError:
            return None

    @FREE_FN
    def _free(ctx, p, nbytes, stream):
        torch.cuda.caching_allocator_delete(int(p))

    a = homln_allocator(None, _alloc, _free)
    a._keep = (_alloc, _free)
    return a


# ---------------------------------------------------------------------------
# C-named functions (raw handles)
# ---------------------------------------------------------------------------

def homln_create(n_nodes: int, layers, flags: int | None = None, allocator=None, stream=None,
                 directed: bool = False) -> int:
    """layers: list of (src, dst) int32 arrays/tensors. flags defaults to DEVICE if they are CUDA tensors."""
    L = len(layers)
    counts = (c_int64 * max(L, 1))(*[int(s.shape[0]) for s, _ in layers])
    srcs = (c_void_p * max(L, 1))(*[ptr(s) for s, _ in layers])
    dsts = (c_void_p * max(L, 1))(*[ptr(d) for _, d in layers])
    if flags is None:
        flags = HOMLN_PTR_DEVICE if L and getattr(layers[0][0], "is_cuda", False) else HOMLN_PTR_HOST
    if directed:
        flags |= HOMLN_DIRECTED
    out = c_void_p()
    rc = lib.homln_create(int(n_nodes), L, counts, srcs, dsts, int(flags),
                          ctypes.byref(allocator) if allocator is not None else None,
                          c_void_p(stream) if stream else None, ctypes.byref(out))
    _check(rc, "homln_create")
    return out.value


def homln_destroy(h) -> None:
    _check(lib.homln_destroy(h), "homln_destroy")


def homln_set_tuning(h, words_per_node=0, push_alpha=0, threads=0, blocks_per_sm=0, relabel=-1, teams=0,
                     team_mix=0, schedule=0, wait_limit_ms=0, test_phantom_blocks=0,
                     max_tiles_per_launch=0, sm_count=0) -> None:
    t = homln_tuning(words_per_node, push_alpha, threads, blocks_per_sm, relabel, teams, team_mix, schedule,
                     wait_limit_ms, test_phantom_blocks, max_tiles_per_launch, sm_count)
    _check(lib.homln_set_tuning(h, ctypes.byref(t)), "homln_set_tuning")


def homln_analyse(h, layer_mask: int, with_and: bool = True) -> None:
    _check(lib.homln_analyse(h, int(layer_mask), int(bool(with_and))), "homln_analyse")


def homln_batch_analyse(handles, masks, with_and: bool = True) -> None:
    n = len(handles)
    hs = (c_void_p * n)(*handles)
    ms = (c_uint64 * n)(*[int(m) for m in masks])
    _check(lib.homln_batch_analyse(hs, n, ms, int(bool(with_and))), "homln_batch_analyse")


def homln_layer_closeness(h, layer: int, farness=None, reach=None, cc=None) -> None:
    _check(lib.homln_layer_closeness(h, int(layer), ptr(farness), ptr(reach), ptr(cc)), "homln_layer_closeness")


def homln_and_aggregate(h, layer_mask: int, capacity: int = 0, and_src=None, and_dst=None) -> int:
    cnt = c_int64()
    _check(lib.homln_and_aggregate(h, int(layer_mask), int(capacity), ptr(and_src), ptr(and_dst),
                                   ctypes.byref(cnt)), "homln_and_aggregate")
    return cnt.value


def homln_and_closeness(h, layer_mask: int, farness=None, reach=None, cc=None) -> None:
    _check(lib.homln_and_closeness(h, int(layer_mask), ptr(farness), ptr(reach), ptr(cc)), "homln_and_closeness")


def homln_or_aggregate(h, layer_mask: int, capacity: int = 0, or_src=None, or_dst=None) -> int:
    cnt = c_int64()
    _check(lib.homln_or_aggregate(h, int(layer_mask), int(capacity), ptr(or_src), ptr(or_dst), ctypes.byref(cnt)),
           "homln_or_aggregate")
    return cnt.value


def homln_or_closeness(h, layer_mask: int, farness=None, reach=None, cc=None) -> None:
    _check(lib.homln_or_closeness(h, int(layer_mask), ptr(farness), ptr(reach), ptr(cc)), "homln_or_closeness")


def homln_graph_capture(handles, masks, with_and: bool = True) -> int:
    """Capture the batched analysis of `handles` into a replayable CUDA graph (opaque handle)."""
    n = len(handles)
    hs = (c_void_p * n)(*handles)
    ms = (c_uint64 * n)(*[int(m) for m in masks])
    out = c_void_p()
    _check(lib.homln_graph_capture(hs, n, ms, int(bool(with_and)), ctypes.byref(out)), "homln_graph_capture")
    return out.value


def homln_shard_partials(h, which: int, layer_mask: int, rank: int, world: int, farness, reach) -> None:
    _check(lib.homln_shard_partials(h, int(which), int(layer_mask), int(rank), int(world), ptr(farness), ptr(reach)),
           "homln_shard_partials")


def homln_batch_closeness(handles, stream=None) -> None:
    n = len(handles)
    hs = (c_void_p * n)(*handles)
    _check(lib.homln_batch_closeness(hs, n, c_void_p(stream) if stream else None), "homln_batch_closeness")


def homln_graph_launch(g) -> None:
    _check(lib.homln_graph_launch(g), "homln_graph_launch")


def homln_graph_destroy(g) -> None:
    _check(lib.homln_graph_destroy(g), "homln_graph_destroy")


def homln_export_partials(h, which: int, layer_mask: int, farness, reach, degree=None) -> None:
    _check(lib.homln_export_partials(h, int(which), int(layer_mask), ptr(farness), ptr(reach), ptr(degree)),
           "homln_export_partials")


def homln_import_partials(h, which: int, layer_mask: int, farness, reach) -> None:
    _check(lib.homln_import_partials(h, int(which), int(layer_mask), ptr(farness), ptr(reach)),
           "homln_import_partials")


def homln_topk(h, which: int, layer_mask: int, sel, nodes_out) -> int:
    cnt = c_int32()
    _check(lib.homln_topk(h, int(which), int(layer_mask), ctypes.byref(sel), ptr(nodes_out), ctypes.byref(cnt)),
           "homln_topk")
    return cnt.value


def homln_compose(h, layer_mask: int, heuristic: int, sel, nodes_out) -> int:
    cnt = c_int32()
    _check(lib.homln_compose(h, int(layer_mask), int(heuristic), ctypes.byref(sel), ptr(nodes_out),
                             ctypes.byref(cnt)), "homln_compose")
    return cnt.value


def homln_accuracy(h, pred, n_pred: int, truth, n_truth: int) -> dict:
    out = homln_accuracy_t()
    _check(lib.homln_accuracy(h, ptr(pred), int(n_pred), ptr(truth), int(n_truth), ctypes.byref(out)),
           "homln_accuracy")
    return out.as_dict()


def homln_accuracy_noalloc(n_nodes: int, pred, n_pred: int, truth, n_truth: int, stream=None) -> dict:
    """Accuracy for callers that cannot allocate device memory: pred/truth must be device memory of
    the current device. stream=None runs on torch's current stream (so inputs written there are ready)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    out = homln_accuracy_t()
    _check(lib.homln_accuracy_noalloc(int(n_nodes), ptr(pred), int(n_pred), ptr(truth), int(n_truth),
                                      c_void_p(stream) if stream else None, ctypes.byref(out)),
           "homln_accuracy_noalloc")
    return out.as_dict()


def homln_yield_create():
    """A lowered yield flag (pinned host memory the GPU reads): see homln_set_yield."""
    y = c_void_p()
    _check(lib.homln_yield_create(ctypes.byref(y)), "homln_yield_create")
    return y.value


def homln_yield_destroy(y) -> None:
    _check(lib.homln_yield_destroy(y), "homln_yield_destroy")


def homln_yield_set(y, raised: bool) -> None:
    _check(lib.homln_yield_set(y, int(bool(raised))), "homln_yield_set")


def homln_yield_count(y) -> int:
    out = c_int64()
    _check(lib.homln_yield_count(y, ctypes.byref(out)), "homln_yield_count")
    return int(out.value)


def homln_set_yield(h, y) -> None:
    """The persistent BFS of calls led by h stops handing out tiles while y is raised and resumes
    once it is lowered (identical results; the call waits for each launch to end)."""
    _check(lib.homln_set_yield(h, y), "homln_set_yield")


def homln_set_profiling(h, timing: bool, instrument: bool = False) -> None:
    _check(lib.homln_set_profiling(h, int(bool(timing)), int(bool(instrument))), "homln_set_profiling")


def homln_get_profile(h) -> dict:
    out = homln_profile_t()
    _check(lib.homln_get_profile(h, ctypes.byref(out)), "homln_get_profile")
    return out.as_dict()


def homln_reset_profile(h) -> None:
    _check(lib.homln_reset_profile(h), "homln_reset_profile")


def homln_kernel_launches() -> int:
    return int(lib.homln_kernel_launches())


def homln_subset_sweep(h, heuristic: int, sel, min_layers: int = 2) -> list:
    cnt = c_int32()
    _check(lib.homln_subset_sweep(h, int(heuristic), ctypes.byref(sel), int(min_layers), None, 0, ctypes.byref(cnt)),
           "homln_subset_sweep")
    out = (homln_subset_result * max(cnt.value, 1))()
    _check(lib.homln_subset_sweep(h, int(heuristic), ctypes.byref(sel), int(min_layers), out, cnt.value,
                                  ctypes.byref(cnt)), "homln_subset_sweep")
    return [{"mask": r.mask, "truth_count": r.truth_count, "estimate_count": r.estimate_count, **r.acc.as_dict()}
            for r in out[:cnt.value]]


def homln_invalidate(h) -> None:
    _check(lib.homln_invalidate(h), "homln_invalidate")


def homln_sync(h) -> None:
    _check(lib.homln_sync(h), "homln_sync")


def homln_version() -> str:
    return lib.homln_version().decode()


# ---------------------------------------------------------------------------
# Convenience wrapper over torch CUDA tensors
# ---------------------------------------------------------------------------

class Network:
    """One HoMLN resident on a GPU. Outputs are torch CUDA tensors (farness int64, reach int32)."""

    def __init__(self, n: int, layers, device=None, stream=None, allocator=None, tuning: dict | None = None,
                 directed: bool = False):
        import torch
        self.torch = torch
        self.n = int(n)
        self.device = torch.device(device if device is not None else "cuda")
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self.stream = stream
        self._alloc = allocator
        with torch.cuda.device(self.device):
            self.h = homln_create(self.n, layers, allocator=allocator, stream=stream, directed=directed)
        self.n_layers = len(layers)
        if tuning:
            homln_set_tuning(self.h, **tuning)

    def _empty(self, count, dtype):
        return self.torch.empty(max(int(count), 1), dtype=dtype, device=self.device)

    def analyse(self, mask: int, with_and: bool = True):
        homln_analyse(self.h, mask, with_and)

    def layer_closeness(self, layer: int):
        F, R, cc = self._empty(self.n, self.torch.int64), self._empty(self.n, self.torch.int32), \
            self._empty(self.n, self.torch.float64)
        homln_layer_closeness(self.h, layer, F, R, cc)
        return F[:self.n], R[:self.n], cc[:self.n]

    def and_closeness(self, mask: int):
        F, R, cc = self._empty(self.n, self.torch.int64), self._empty(self.n, self.torch.int32), \
            self._empty(self.n, self.torch.float64)
        homln_and_closeness(self.h, mask, F, R, cc)
        return F[:self.n], R[:self.n], cc[:self.n]

    def or_closeness(self, mask: int):
        F, R, cc = self._empty(self.n, self.torch.int64), self._empty(self.n, self.torch.int32), \
            self._empty(self.n, self.torch.float64)
        homln_or_closeness(self.h, mask, F, R, cc)
        return F[:self.n], R[:self.n], cc[:self.n]

    def or_aggregate(self, mask: int):
        m = homln_or_aggregate(self.h, mask)
        s, d = self._empty(m, self.torch.int32), self._empty(m, self.torch.int32)
        homln_or_aggregate(self.h, mask, m, s, d)
        return s[:m], d[:m]

    def and_aggregate(self, mask: int):
        m = homln_and_aggregate(self.h, mask)
        s, d = self._empty(m, self.torch.int32), self._empty(m, self.torch.int32)
        homln_and_aggregate(self.h, mask, m, s, d)
        return s[:m], d[:m]

    def topk(self, which: int, mask: int, sel):
        out = self._empty(self.n, self.torch.int32)
        c = homln_topk(self.h, which, mask, sel, out)
        return out[:c]

    def compose(self, mask: int, heuristic: int, sel):
        out = self._empty(self.n, self.torch.int32)
        c = homln_compose(self.h, mask, heuristic, sel, out)
        return out[:c]

    def accuracy(self, pred, truth) -> dict:
        return homln_accuracy(self.h, pred, int(pred.shape[0]), truth, int(truth.shape[0]))

    def shard_partials(self, which: int, mask: int, rank: int, world: int):
        """Partial farness/reach of graph `which` from the source batches of shard rank/world."""
        F, R = self._empty(self.n, self.torch.int64), self._empty(self.n, self.torch.int32)
        homln_shard_partials(self.h, which, mask, rank, world, F, R)
        return F[:self.n], R[:self.n]

    def save_partials(self, path: str, masks=()) -> None:
        """Checkpoint the Psi results of every layer and of the AND graphs of `masks` (host .npz)."""
        out = {"n": np.array([self.n]), "layers": np.array([self.n_layers])}
        items = [(i, 0) for i in range(self.n_layers)] + [(-1, int(m)) for m in masks]
        for which, mask in items:
            F, R, d = np.empty(self.n, np.uint64), np.empty(self.n, np.uint32), np.empty(self.n, np.int32)
            homln_export_partials(self.h, which, mask, F, R, d)
            key = f"layer{which}" if which >= 0 else f"and{mask}"
            out[key + "_F"], out[key + "_R"], out[key + "_deg"] = F, R, d
        np.savez(path, **out)

    def load_partials(self, path: str) -> None:
        """Resume from save_partials: later queries on those graphs run no BFS."""
        z = np.load(path)
        if int(z["n"][0]) != self.n or int(z["layers"][0]) != self.n_layers:
            raise ValueError("checkpoint was taken on a different network")
        for key in z.files:
            if not key.endswith("_F"):
                continue
            base = key[:-2]
            which, mask = (int(base[5:]), 0) if base.startswith("layer") else (-1, int(base[3:]))
            homln_import_partials(self.h, which, mask, np.ascontiguousarray(z[base + "_F"]),
                                  np.ascontiguousarray(z[base + "_R"]))

    def close(self):
        if getattr(self, "h", None):
            homln_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
