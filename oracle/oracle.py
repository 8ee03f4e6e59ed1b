"""Oracle for decoupled closeness centrality on HoMLNs. TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module. The product path (the CUDA library and its
Python binding) never imports it, and it imports nothing from the product.

Everything here is the plain definition of what the method computes, written
to be read against the paper:

* simple-graph semantics of each layer (undirected, unweighted, no self loops,
  no multi-edges; Section 4 uses NetworkX ``Graph``),
* Boolean AND aggregation: an edge is kept iff it is present in every selected
  layer (Section 3.1; ground truth, Section 4),
* all-sources BFS distance sums (``oracle/bfs.c``; Section 4),
* Wasserman-Faust normalised closeness, which reduces to Eq. 1 on a connected
  graph (Section 4),
* sumDist with the "unreachable costs n" convention (Section 5.1),
* CC-node selection: top-k, or at or above the average (Section 4, Section 5.2),
* composition heuristics naive (Section 4), CC1 (Section 5.1, Eqs. 2-3) and
  CC2 (Section 5.2, Algorithm 1),
* Jaccard / precision / recall / F1 of an estimated set against ground truth
  (Section 5, Section 6.1).

Floating point: closeness values are float64, as in the paper's NetworkX runs.
Each is one correctly rounded division of exact integers. Decisions that
depend on an average (at or above the average) are taken exactly on those
float64 values with ``fractions.Fraction`` (no summation-order dependence).

Parity status: everything is pinned by tests in ``tests/test_oracle_*.py``
except the CC1 overlap threshold, which the paper leaves undefined (Section 5.1 asks
for a large overlap without a number): parity unpinned for the value of theta (the
steps around it are pinned by a hand-worked example).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle_bfs.so")
_lib = None

# selection modes (same numbering as the C-ABI so tests can pass one struct to both)
TOPK_PERCENT, TOPK_COUNT, GE_MEAN, GT_MEAN = 0, 1, 2, 3
NAIVE, CC1, CC2 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ``bfs.c`` into ``liboracle_bfs.so`` next to it (gcc, OpenMP)."""
    src = os.path.join(_HERE, "bfs.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.oracle_bfs_farness.restype = ctypes.c_int
        lib.oracle_bfs_farness.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
        lib.oracle_bfs_dist.restype = ctypes.c_int
        lib.oracle_bfs_dist.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.c_void_p]
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


# ---------------------------------------------------------------------------
# Graphs (Section 4: simple undirected graphs; Section 3.1: AND aggregation)
# ---------------------------------------------------------------------------

def edge_keys(n: int, src, dst) -> np.ndarray:
    """The layer's undirected edge set as sorted unique keys lo*n+hi (self loops and repeats dropped)."""
    s = np.asarray(src, np.int64)
    d = np.asarray(dst, np.int64)
    if s.size and (s.min() < 0 or d.min() < 0 or s.max() >= n or d.max() >= n):
        raise ValueError("node id out of range")
    keep = s != d
    lo = np.minimum(s[keep], d[keep])
    hi = np.maximum(s[keep], d[keep])
    return np.unique(lo * n + hi)


def arc_keys(n: int, src, dst) -> np.ndarray:
    """A directed layer's arc set as sorted unique keys u*n+v for arcs u -> v (self loops and repeats dropped)."""
    s = np.asarray(src, np.int64)
    d = np.asarray(dst, np.int64)
    if s.size and (s.min() < 0 or d.min() < 0 or s.max() >= n or d.max() >= n):
        raise ValueError("node id out of range")
    keep = s != d
    return np.unique(s[keep] * n + d[keep])


def arc_csr(n: int, keys: np.ndarray, reverse: bool = False):
    """CSR of arcs: rows are tails (out-edges), or heads with reverse=True (in-edges); rows sorted."""
    u, v = (np.asarray(keys, np.int64) // n, np.asarray(keys, np.int64) % n)
    rows, cols = (v, u) if reverse else (u, v)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return rowptr, cols.astype(np.int32)


def keys_to_edges(n: int, keys: np.ndarray):
    keys = np.asarray(keys, np.int64)
    return (keys // n).astype(np.int32), (keys % n).astype(np.int32)


def csr_from_keys(n: int, keys: np.ndarray):
    """Symmetric CSR (rowptr int64[n+1], col int32) with each row sorted ascending."""
    lo, hi = keys_to_edges(n, keys)
    rows = np.concatenate([lo, hi]).astype(np.int64)
    cols = np.concatenate([hi, lo]).astype(np.int64)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return rowptr, cols.astype(np.int32)


def simple_csr(n: int, src, dst):
    return csr_from_keys(n, edge_keys(n, src, dst))


def and_keys(n: int, layer_keys) -> np.ndarray:
    """Edges present in every given layer (Boolean AND aggregation)."""
    out = layer_keys[0]
    for k in layer_keys[1:]:
        out = np.intersect1d(out, k, assume_unique=True)
    return out


def or_keys(n: int, layer_keys) -> np.ndarray:
    """Edges present in at least one given layer (Boolean OR aggregation, Section 3.1)."""
    out = layer_keys[0]
    for k in layer_keys[1:]:
        out = np.union1d(out, k)
    return out


# ---------------------------------------------------------------------------
# Distances (Section 4: BFS from every vertex, unreachable contributes 0)
# ---------------------------------------------------------------------------

def farness_reach(n: int, rowptr, col, sources=None, threads: int = 1):
    """F(s) = sum of hop distances from s over reached vertices, R(s) = reached vertices other than s."""
    lib = _load()
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    if sources is None:
        ns = n
        sp = None
    else:
        sources = np.ascontiguousarray(sources, np.int32)
        ns = sources.shape[0]
        sp = sources.ctypes.data
    F = np.zeros(ns, np.uint64)
    R = np.zeros(ns, np.uint32)
    if n == 0 or ns == 0:
        return F, R
    rc = lib.oracle_bfs_farness(n, rowptr.ctypes.data, col.ctypes.data if col.size else 0, ns, sp,
                                F.ctypes.data, R.ctypes.data, int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle_bfs_farness failed ({rc})")
    return F, R


def bfs_dist(n: int, rowptr, col, s: int) -> np.ndarray:
    lib = _load()
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    dist = np.empty(n, np.int32)
    rc = lib.oracle_bfs_dist(n, rowptr.ctypes.data, col.ctypes.data if col.size else 0, int(s), dist.ctypes.data)
    if rc != 0:
        raise RuntimeError("oracle_bfs_dist failed")
    return dist


# ---------------------------------------------------------------------------
# Closeness (Eq. 1; Wasserman-Faust normalisation for disconnected graphs)
# ---------------------------------------------------------------------------

def wf_closeness(n: int, F, R) -> np.ndarray:
    """cc(v) = (R/(n-1)) * (R/F) written as one division R^2 / ((n-1) F); 0 when F = 0.

    For a connected graph R = n-1 and this is exactly Eq. 1, (n-1)/F.
    Numerator and denominator are exact integers converted to float64 once.
    """
    F = np.asarray(F, np.uint64)
    R = np.asarray(R, np.uint64)
    out = np.zeros(F.shape[0], np.float64)
    nz = F > 0
    num = (R[nz] * R[nz]).astype(np.float64)
    den = (np.uint64(max(n - 1, 0)) * F[nz]).astype(np.float64)
    out[nz] = num / den
    return out


def sum_dist_n(n: int, F, R) -> np.ndarray:
    """sumDist(v) with distance n charged for each unreachable vertex (Section 5.1)."""
    F = np.asarray(F, np.uint64)
    R = np.asarray(R, np.uint64)
    return F + np.uint64(n) * (np.uint64(max(n - 1, 0)) - R)


def degrees(rowptr) -> np.ndarray:
    rowptr = np.asarray(rowptr, np.int64)
    return (rowptr[1:] - rowptr[:-1]).astype(np.int32)


# ---------------------------------------------------------------------------
# CC-node selection (top-k, or at or above the average)
# ---------------------------------------------------------------------------

@dataclass
class Select:
    mode: int = TOPK_PERCENT
    percent: float = 10.0
    k: int = 0
    cc1_overlap: float = 0.5


def topk_count(sel: Select, n: int) -> int:
    if sel.mode == TOPK_PERCENT:
        k = math.ceil((sel.percent * float(n)) / 100.0)
    else:
        k = sel.k
    return int(min(max(k, 0), n))


def rank_order(scores) -> np.ndarray:
    """Node ids by score descending, equal scores by ascending id."""
    scores = np.asarray(scores, np.float64)
    ids = np.arange(scores.shape[0])
    return np.lexsort((ids, -scores)).astype(np.int32)


def exact_sum(values) -> Fraction:
    return sum((Fraction(float(x)) for x in values), Fraction(0))


def select(scores, sel: Select) -> np.ndarray:
    """Selected node ids in rank order."""
    scores = np.asarray(scores, np.float64)
    n = scores.shape[0]
    order = rank_order(scores)
    if sel.mode in (TOPK_PERCENT, TOPK_COUNT):
        return order[:topk_count(sel, n)]
    if n == 0:
        return order
    total = exact_sum(scores)
    if sel.mode == GE_MEAN:
        keep = [u for u in order if Fraction(float(scores[u])) * n >= total]
    elif sel.mode == GT_MEAN:
        keep = [u for u in order if Fraction(float(scores[u])) * n > total]
    else:
        raise ValueError("unknown selection mode")
    return np.asarray(keep, np.int32)


# ---------------------------------------------------------------------------
# Composition heuristics (Section 4 naive, Section 5.1 CC1, Section 5.2 CC2)
# ---------------------------------------------------------------------------

def compose_naive(ch_sets) -> np.ndarray:
    """Intersection of the layers' CC-node sets, ascending id."""
    out = set(int(x) for x in ch_sets[0])
    for s in ch_sets[1:]:
        out &= set(int(x) for x in s)
    return np.asarray(sorted(out), np.int32)


def cc2_estimate(sumdists) -> np.ndarray:
    """Algorithm 1: estSumDist(u) = max over the layers of sumDist(u)."""
    est = np.asarray(sumdists[0], np.uint64).copy()
    for s in sumdists[1:]:
        est = np.maximum(est, np.asarray(s, np.uint64))
    return est


def cc2_scores(n: int, est) -> np.ndarray:
    """Eq. 1 on the estimate: (n-1)/estSumDist(u); 0 when the estimate is 0."""
    est = np.asarray(est, np.uint64)
    out = np.zeros(est.shape[0], np.float64)
    nz = est > 0
    out[nz] = np.float64(max(n - 1, 0)) / est[nz].astype(np.float64)
    return out


def compose_cc2(n: int, sumdists, sel: Select) -> np.ndarray:
    est = cc2_estimate(sumdists)
    return np.sort(select(cc2_scores(n, est), sel)).astype(np.int32)


def cc1_ratios(sumdists, degs):
    """Eq. 2 per layer: sumDist_i(u) / min over the layers of deg(u); +inf when that minimum is 0."""
    mind = np.asarray(degs[0], np.int64).copy()
    for d in degs[1:]:
        mind = np.minimum(mind, np.asarray(d, np.int64))
    ratios = []
    for s in sumdists:
        r = np.full(mind.shape[0], np.inf)
        ok = mind > 0
        r[ok] = np.asarray(s, np.uint64)[ok].astype(np.float64) / mind[ok].astype(np.float64)
        ratios.append(r)
    return ratios, mind


def cc1_average(ratios) -> Fraction:
    """Eq. 3: the largest of the layers' exact mean ratios (finite ratios only; 0 if none)."""
    best = None
    for r in ratios:
        fin = r[np.isfinite(r)]
        avg = exact_sum(fin) / len(fin) if len(fin) else Fraction(0)
        best = avg if best is None or avg > best else best
    return best if best is not None else Fraction(0)


def compose_cc1(n: int, csrs, sumdists, degs, ch_sets, theta: float) -> np.ndarray:
    """CC1: common CC nodes whose central one-hop neighbourhoods overlap enough across the layers.

    ``csrs`` holds each layer's (rowptr, col). A neighbour v of u is central in
    layer i when ratio_i(v) < avg (exact comparison). u is selected iff
    |intersection of C_i(u)| >= theta * |union of C_i(u)| with a non-empty union,
    where theta * |union| is one float64 product.
    """
    ratios, _ = cc1_ratios(sumdists, degs)
    avg = cc1_average(ratios)
    common = set(int(x) for x in ch_sets[0])
    for s in ch_sets[1:]:
        common &= set(int(x) for x in s)
    out = []
    for u in sorted(common):
        cs = []
        for (rowptr, col), r in zip(csrs, ratios):
            nb = col[rowptr[u]:rowptr[u + 1]]
            cs.append(set(int(v) for v in nb if np.isfinite(r[v]) and Fraction(float(r[v])) < avg))
        inter = set.intersection(*cs)
        union = set.union(*cs)
        if len(union) > 0 and float(len(inter)) >= float(theta) * float(len(union)):
            out.append(u)
    return np.asarray(out, np.int32)


# ---------------------------------------------------------------------------
# Accuracy (Jaccard as "accuracy", precision, recall, F1)
# ---------------------------------------------------------------------------

def accuracy(pred, truth) -> dict:
    P = set(int(x) for x in pred)
    T = set(int(x) for x in truth)
    tp = len(P & T)
    fp = len(P - T)
    fn = len(T - P)
    jac = tp / (tp + fp + fn) if (tp + fp + fn) > 0 else 1.0
    prec = tp / (tp + fp) if (tp + fp) > 0 else 0.0
    rec = tp / (tp + fn) if (tp + fn) > 0 else 0.0
    f1 = (2 * tp) / (2 * tp + fp + fn) if tp > 0 else 0.0
    return {"tp": tp, "fp": fp, "fn": fn, "jaccard": jac, "precision": prec, "recall": rec, "f1": f1}


# ---------------------------------------------------------------------------
# The whole path on one HoMLN, cached like the library (each layer analysed once)
# ---------------------------------------------------------------------------

class OracleHoMLN:
    """directed=True: layers are arc lists; closeness is in-closeness (distances d(v, u) of the
    vertices v that reach u, the NetworkX convention for directed graphs), i.e. BFS from u along
    in-edges; degrees are in-degrees and CC1's neighbourhoods are in-neighbourhoods."""

    def __init__(self, n: int, layers, threads: int = 1, directed: bool = False):
        self.n = int(n)
        self.threads = threads
        self.directed = directed
        self.keys = [arc_keys(n, s, d) if directed else edge_keys(n, s, d) for s, d in layers]
        self._layer = {}
        self._and = {}
        self._or = {}

    def _analyse(self, keys):
        n = self.n
        rowptr, col = arc_csr(n, keys, reverse=True) if self.directed else csr_from_keys(n, keys)
        F, R = farness_reach(n, rowptr, col, threads=self.threads)
        return {"rowptr": rowptr, "col": col, "F": F, "R": R, "cc": wf_closeness(n, F, R),
                "sumdist": sum_dist_n(n, F, R), "deg": degrees(rowptr), "keys": keys}

    def layer(self, i: int) -> dict:
        if i not in self._layer:
            self._layer[i] = self._analyse(self.keys[i])
        return self._layer[i]

    def mask_layers(self, mask: int):
        return [i for i in range(len(self.keys)) if (mask >> i) & 1]

    def and_graph(self, mask: int) -> dict:
        if mask not in self._and:
            ids = self.mask_layers(mask)
            self._and[mask] = self._analyse(and_keys(self.n, [self.keys[i] for i in ids]))
        return self._and[mask]

    def or_graph(self, mask: int) -> dict:
        if mask not in self._or:
            ids = self.mask_layers(mask)
            self._or[mask] = self._analyse(or_keys(self.n, [self.keys[i] for i in ids]))
        return self._or[mask]

    def or_edges(self, mask: int):
        return keys_to_edges(self.n, self.or_graph(mask)["keys"])

    def and_edges(self, mask: int):
        return keys_to_edges(self.n, self.and_graph(mask)["keys"])

    def topk(self, which: int, mask: int, sel: Select) -> np.ndarray:
        g = self.layer(which) if which >= 0 else self.and_graph(mask) if which == -1 else self.or_graph(mask)
        return select(g["cc"], sel)

    def compose(self, mask: int, heur: int, sel: Select) -> np.ndarray:
        ids = self.mask_layers(mask)
        L = [self.layer(i) for i in ids]
        if heur == CC2:
            return compose_cc2(self.n, [g["sumdist"] for g in L], sel)
        chs = [select(g["cc"], sel) for g in L]
        if heur == NAIVE:
            return compose_naive(chs)
        if heur == CC1:
            return compose_cc1(self.n, [(g["rowptr"], g["col"]) for g in L], [g["sumdist"] for g in L],
                               [g["deg"] for g in L], chs, sel.cc1_overlap)
        raise ValueError("unknown heuristic")
