"""Seeded synthetic HoMLN generators.

The paper evaluates on PaRMAT/RMAT two-layer HoMLNs (Section 6, Table 1):
power-law and normal degree layers over one shared vertex set, with layers that
share a backbone of edges. Those data sets are not available here, so the
workloads are regenerated from seeds with the same structure: Erdos-Renyi
(normal-like degrees), Chung-Lu (power law, exponent 2.5) and Barabasi-Albert
layers, overlapped through a shared edge pool.

This module only produces edge lists. It holds none of the method's arithmetic
(no BFS, no closeness, no selection), so both the oracle and the CUDA path can
consume its output. Every function is a pure function of its seed.

Edge lists are returned as int32 numpy arrays ``(src, dst)`` of undirected
edges. Lists may contain both orientations of a pair only where stated; self
loops are never produced except by ``noisy_copy`` (which adds them on purpose
to exercise normalisation).
"""
from __future__ import annotations

import math
import random
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "HoMLN", "er_edges", "chung_lu_edges", "ba_edges", "overlay",
    "homln_small_er", "homln_small_overlap", "homln_powerlaw", "homln_ba_large",
    "homln_batch", "serving_requests", "noisy_copy", "relabel", "rmat_edges", "homln_parmat_like",
]


@dataclass
class HoMLN:
    """A homogeneous multilayer network: ``n`` shared nodes, one edge list per layer."""
    n: int
    layers: list  # list of (src, dst) int32 arrays
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_layers(self) -> int:
        return len(self.layers)

    def edge_counts(self):
        return [int(s.shape[0]) for s, _ in self.layers]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _canon_unique(u: np.ndarray, v: np.ndarray, n: int):
    """Drop self loops and duplicate pairs; return canonical (min, max) pairs in first-seen order."""
    u = u.astype(np.int64)
    v = v.astype(np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    key = lo * n + hi
    _, first = np.unique(key, return_index=True)
    first.sort()
    return lo[first], hi[first]


def er_edges(n: int, m: int, seed: int):
    """G(n, m): ``m`` distinct undirected pairs drawn uniformly (fewer if the graph would be complete)."""
    rng = _rng(seed)
    m = int(min(m, n * (n - 1) // 2))
    lo = np.empty(0, np.int64)
    hi = np.empty(0, np.int64)
    while lo.shape[0] < m:
        need = m - lo.shape[0]
        k = int(need * 1.1) + 16
        a = rng.integers(0, n, size=k)
        b = rng.integers(0, n, size=k)
        lo = np.concatenate([lo, a])
        hi = np.concatenate([hi, b])
        lo, hi = _canon_unique(lo, hi, n)
    lo, hi = lo[:m], hi[:m]
    flip = rng.random(m) < 0.5  # random orientation so the CSR builder must symmetrise
    s = np.where(flip, hi, lo).astype(np.int32)
    d = np.where(flip, lo, hi).astype(np.int32)
    return s, d


def chung_lu_weights(n: int, avg_deg: float, gamma: float = 2.5, i0: float | None = None):
    """Expected-degree sequence w_i proportional to (i + i0)^(-1/(gamma-1)), scaled to mean ``avg_deg``.

    ``i0`` caps the largest expected degree near sqrt(avg_deg * n) (the structural
    cut-off), which keeps the sampled graph simple without a large loss of edges.
    """
    a = 1.0 / (gamma - 1.0)
    if i0 is None:
        # choose i0 so that w_0 is about sqrt(sum w)
        target = math.sqrt(avg_deg * n)
        i0 = 1.0
        for _ in range(60):
            w = (np.arange(n) + i0) ** (-a)
            w *= avg_deg * n / w.sum()
            if w[0] <= target:
                break
            i0 *= 1.5
    w = (np.arange(n, dtype=np.float64) + i0) ** (-a)
    w *= avg_deg * n / w.sum()
    return w


def chung_lu_edges(n: int, m: int, seed: int, gamma: float = 2.5, weights=None):
    """Chung-Lu graph with ``m`` distinct edges; endpoints drawn independently in proportion to the weights."""
    rng = _rng(seed)
    if weights is None:
        weights = chung_lu_weights(n, 2.0 * m / n, gamma)
    cdf = np.cumsum(weights)
    cdf /= cdf[-1]
    m = int(min(m, n * (n - 1) // 2))
    lo = np.empty(0, np.int64)
    hi = np.empty(0, np.int64)
    for _ in range(64):
        if lo.shape[0] >= m:
            break
        need = m - lo.shape[0]
        k = int(need * 1.25) + 16
        a = np.searchsorted(cdf, rng.random(k), side="right").clip(0, n - 1)
        b = np.searchsorted(cdf, rng.random(k), side="right").clip(0, n - 1)
        lo = np.concatenate([lo, a])
        hi = np.concatenate([hi, b])
        lo, hi = _canon_unique(lo, hi, n)
    lo, hi = lo[:m], hi[:m]
    return lo.astype(np.int32), hi.astype(np.int32)


def ba_edges(n: int, m_attach: int, seed: int):
    """Barabasi-Albert preferential attachment: each new node links to ``m_attach`` distinct earlier nodes."""
    rnd = random.Random(seed)
    m_attach = max(1, min(m_attach, n - 1))
    src = []
    dst = []
    repeated = list(range(m_attach))  # the seed nodes start with one ticket each
    for t in range(m_attach, n):
        targets = set()
        while len(targets) < m_attach:
            targets.add(repeated[rnd.randrange(len(repeated))])
        for x in targets:
            src.append(t)
            dst.append(x)
        repeated.extend(targets)
        repeated.extend([t] * m_attach)
    return np.asarray(src, np.int32), np.asarray(dst, np.int32)


def overlay(n: int, shared, own):
    """Union of a shared edge pool and a layer's own edges, deduplicated (canonical pairs)."""
    s = np.concatenate([shared[0], own[0]]).astype(np.int64)
    d = np.concatenate([shared[1], own[1]]).astype(np.int64)
    lo, hi = _canon_unique(s, d, n)
    return lo.astype(np.int32), hi.astype(np.int32)


def _take_fraction(edges, frac: float, seed: int):
    rng = _rng(seed)
    k = int(round(edges[0].shape[0] * frac))
    idx = np.sort(rng.permutation(edges[0].shape[0])[:k])
    return edges[0][idx], edges[1][idx]


def relabel(n: int, layers, seed: int):
    """Apply one random node permutation to every layer (hubs then sit at random ids)."""
    perm = _rng(seed).permutation(n).astype(np.int32)
    return [(perm[s], perm[d]) for s, d in layers]


def noisy_copy(n: int, edges, seed: int, self_loops: int = 8, duplicates: int = 8):
    """The same edge set, shuffled, with reversed duplicates and self loops mixed in."""
    rng = _rng(seed)
    s, d = edges
    k = s.shape[0]
    dup = rng.integers(0, max(k, 1), size=min(duplicates, k)) if k else np.empty(0, np.int64)
    loops = rng.integers(0, n, size=self_loops)
    ss = np.concatenate([s, d[dup], loops]).astype(np.int32)
    dd = np.concatenate([d, s[dup], loops]).astype(np.int32)
    order = rng.permutation(ss.shape[0])
    return ss[order], dd[order]


# ---------------------------------------------------------------------------
# Workloads shaped like the paper's (Section 6) and the benchmark configurations
# ---------------------------------------------------------------------------

RMAT_POWERLAW = (0.45, 0.15, 0.15)  # a, b, c (d = 0.25): skewed, power-law degrees
RMAT_NORMAL = (0.25, 0.25, 0.25)    # uniform quadrants: binomial (normal-like) degrees


def with_reciprocal(edges, frac: float, seed: int):
    """Arc list plus the reverse of a random ``frac`` of its arcs (directed layers with some 2-cycles)."""
    s, d = edges
    pick = _rng(seed).random(s.shape[0]) < frac
    return np.concatenate([s, d[pick]]).astype(np.int32), np.concatenate([d, s[pick]]).astype(np.int32)


def rmat_edges(n: int, m: int, seed: int, abc=RMAT_POWERLAW):
    """R-MAT: each edge picks one quadrant of the adjacency matrix per bit of the node id with
    probabilities (a, b, c, d); ids >= n are folded back with a modulus. Repeats and self loops
    are kept (the library normalises its input)."""
    a, b, c = abc
    rng = _rng(seed)
    scale = max(1, int(math.ceil(math.log2(max(n, 2)))))
    u = np.zeros(m, np.int64)
    v = np.zeros(m, np.int64)
    for _ in range(scale):
        r = rng.random(m)
        ubit = r >= a + b
        vbit = ((r >= a) & (r < a + b)) | (r >= a + b + c)
        u = (u << 1) | ubit
        v = (v << 1) | vbit
    perm = rng.permutation(n)  # random node labels, so high-degree nodes are not the small ids
    return perm[u % n].astype(np.int32), perm[v % n].astype(np.int32)


def homln_parmat_like(n: int = 50000, m: int = 250000, split=(0.7, 0.3), kinds=("powerlaw", "normal"),
                      seed: int = 6001) -> HoMLN:
    """A two-layer HoMLN shaped like the paper's synthetic sets (Section 6, Table 1): layer i holds
    split[i] of the base graph's m edges from its own R-MAT generator (power-law or normal) plus
    a shared backbone of n edges (a random Hamiltonian cycle), which Table 1's counts imply
    (|L_i| ~ split_i * m + |V|, |L1 AND L2| ~ |V|)."""
    rng = _rng(seed)
    order = rng.permutation(n)
    backbone = (order.astype(np.int32), np.roll(order, 1).astype(np.int32))
    layers = []
    for i, (frac, kind) in enumerate(zip(split, kinds)):
        own = rmat_edges(n, int(round(frac * m)), seed * 10 + i, RMAT_POWERLAW if kind == "powerlaw" else RMAT_NORMAL)
        layers.append((np.concatenate([backbone[0], own[0]]), np.concatenate([backbone[1], own[1]])))
    return HoMLN(n, layers, name=f"parmat{n}-{m}-{split[0]:.1f}", meta={"kinds": kinds, "split": split})


def homln_small_er(n: int = 1000, avg_deg: float = 8.0, n_layers: int = 3, seeds=(101, 102, 103)) -> HoMLN:
    """Independent ER layers on a shared node set (3 x ER(1000, m=4000))."""
    m = int(avg_deg * n / 2)
    layers = [er_edges(n, m, seeds[i]) for i in range(n_layers)]
    return HoMLN(n, layers, name=f"er{n}x{n_layers}", meta={"kind": "er", "avg_deg": avg_deg})


def homln_small_overlap(n: int = 1000, avg_deg: float = 8.0, n_layers: int = 3, rho: float = 0.5,
                        seed: int = 111) -> HoMLN:
    """ER layers sharing a pool of rho*m edges, so the AND graph keeps a backbone (as in Table 1)."""
    m = int(avg_deg * n / 2)
    pool = er_edges(n, int(rho * m), seed)
    layers = [overlay(n, pool, er_edges(n, m - int(rho * m), seed + 1 + i)) for i in range(n_layers)]
    return HoMLN(n, layers, name=f"erov{n}x{n_layers}", meta={"kind": "er-overlap", "rho": rho})


def homln_powerlaw(n: int = 50000, avg_deg: float = 10.0, n_layers: int = 4, gamma: float = 2.5,
                   seed: int = 2001, rho_range=(0.3, 0.7)) -> HoMLN:
    """Chung-Lu power-law layers with a shared pool of rho*m edges, rho ~ U[0.3, 0.7]."""
    rng = _rng(seed)
    rho = float(rng.uniform(*rho_range))
    m = int(avg_deg * n / 2)
    w = chung_lu_weights(n, avg_deg, gamma)
    m_pool = int(rho * m)
    pool = chung_lu_edges(n, m_pool, seed * 7 + 1, gamma, weights=w)
    layers = []
    for i in range(n_layers):
        own = chung_lu_edges(n, m - m_pool, seed * 7 + 2 + i, gamma, weights=w)
        layers.append(overlay(n, pool, own))
    layers = relabel(n, layers, seed * 7 + 99)
    return HoMLN(n, layers, name=f"cl{n}x{n_layers}",
                 meta={"kind": "chung-lu", "gamma": gamma, "avg_deg": avg_deg, "rho": rho})


def homln_ba_large(n: int = 200000, m_attach: int = 4, n_layers: int = 4, seed: int = 4001,
                   shared_frac: float = 0.5) -> HoMLN:
    """BA layers: a seeded half of one base BA graph shared by all, plus half of each layer's own BA graph."""
    base = ba_edges(n, m_attach, seed)
    pool = _take_fraction(base, shared_frac, seed + 1)
    layers = []
    for i in range(n_layers):
        own = _take_fraction(ba_edges(n, m_attach, seed + 10 + i), 1.0 - shared_frac, seed + 20 + i)
        layers.append(overlay(n, pool, own))
    layers = relabel(n, layers, seed + 99)
    return HoMLN(n, layers, name=f"ba{n}x{n_layers}", meta={"kind": "ba-overlap", "m": m_attach})


def homln_batch(count: int = 64, seed: int = 3001, n_range=(500, 20000), layer_range=(2, 8)):
    """Many small HoMLNs of uneven size: layers U{2..8}, n ~ U[500, 20000], ER (deg U[4,16]) or BA (m U{2..6})."""
    rnd = random.Random(seed)
    nets = []
    for k in range(count):
        n = rnd.randint(*n_range)
        L = rnd.randint(*layer_range)
        layers = []
        kinds = []
        for i in range(L):
            s = seed * 1000 + k * 16 + i
            if rnd.random() < 0.5:
                deg = rnd.uniform(4.0, 16.0)
                layers.append(er_edges(n, int(deg * n / 2), s))
                kinds.append(f"er{deg:.1f}")
            else:
                ma = rnd.randint(2, 6)
                layers.append(ba_edges(n, ma, s))
                kinds.append(f"ba{ma}")
        layers = relabel(n, layers, seed * 1000 + k * 16 + 15)
        nets.append(HoMLN(n, layers, name=f"batch{k}", meta={"kinds": kinds}))
    return nets


def serving_requests(duration_s: float = 60.0, rate: float = 50.0, seed: int = 5001,
                     n_range=(1000, 100000), layer_range=(2, 6)):
    """Poisson arrivals of closeness queries on HoMLNs with log-uniform node counts.

    Returns a list of dicts ``{"t": arrival_seconds, "spec": (kind, n, L, deg, seed)}``;
    ``build_request`` turns a spec into a HoMLN lazily.
    """
    rnd = random.Random(seed)
    t = 0.0
    reqs = []
    i = 0
    while True:
        t += rnd.expovariate(rate)
        if t > duration_s:
            break
        n = int(round(math.exp(rnd.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        L = rnd.randint(*layer_range)
        kind = "er" if rnd.random() < 0.5 else "cl"
        deg = rnd.uniform(6.0, 12.0)
        reqs.append({"t": t, "spec": (kind, n, L, deg, seed * 100000 + i)})
        i += 1
    return reqs


def _raw_er(n: int, m: int, rng):
    return rng.integers(0, n, size=m).astype(np.int32), rng.integers(0, n, size=m).astype(np.int32)


def _raw_cl(n: int, m: int, cdf, rng):
    a = np.searchsorted(cdf, rng.random(m), side="right").clip(0, n - 1).astype(np.int32)
    b = np.searchsorted(cdf, rng.random(m), side="right").clip(0, n - 1).astype(np.int32)
    return a, b


def build_request(spec, raw: bool = False) -> HoMLN:
    """The HoMLN of one serving request. raw=True samples endpoints without removing self loops
    or repeated pairs (the library normalises its input), which is much faster to generate."""
    kind, n, L, deg, s = spec
    m = int(deg * n / 2)
    if raw:
        rng = _rng(s)
        if kind == "er":
            layers = [_raw_er(n, m, rng) for _ in range(L)]
        else:
            w = chung_lu_weights(n, deg, 2.5)
            cdf = np.cumsum(w)
            cdf /= cdf[-1]
            pool = _raw_cl(n, m // 2, cdf, rng)
            layers = []
            for _ in range(L):
                own = _raw_cl(n, m - m // 2, cdf, rng)
                layers.append((np.concatenate([pool[0], own[0]]), np.concatenate([pool[1], own[1]])))
        return HoMLN(n, layers, name=f"req{s}", meta={"kind": kind, "deg": deg, "raw": True})
    if kind == "er":
        layers = [er_edges(n, m, s * 8 + i) for i in range(L)]
    else:
        w = chung_lu_weights(n, deg, 2.5)
        pool = chung_lu_edges(n, m // 2, s * 8 + 7, 2.5, weights=w)
        layers = [overlay(n, pool, chung_lu_edges(n, m - m // 2, s * 8 + i, 2.5, weights=w)) for i in range(L)]
    return HoMLN(n, layers, name=f"req{s}", meta={"kind": kind, "deg": deg})
