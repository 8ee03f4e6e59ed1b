"""The identity behind folding degree-1 vertices out of the BFS, checked by brute force (no GPU).

A vertex v whose only neighbour p has other neighbours is one hop further than p from every other
vertex, so the farness and reach of v follow from p's. The BFS kernel leaves such vertices out and
fills them in afterwards, also for a shard that holds partial sums over its own sources (every
world-th batch of spb sources): F_S(v) = F_S(p) + R_S(p) + [p in S] - 2 [v in S] and
R_S(v) = R_S(p) + [p in S] - [v in S]. Here the partial sums come from plain BFS distances and the
formula is evaluated in the kernel's unsigned 64/32-bit arithmetic."""
import collections

import numpy as np


def distances(n, adj, s):
    d = np.full(n, -1, np.int64)
    d[s] = 0
    q = collections.deque([s])
    while q:
        u = q.popleft()
        for w in adj[u]:
            if d[w] < 0:
                d[w] = d[u] + 1
                q.append(w)
    return d


def random_graph_with_leaves(n, seed):
    rng = np.random.default_rng(seed)
    core = n // 2
    edges = set()
    for u in range(1, core):  # a random tree over the core, plus chords
        edges.add((int(rng.integers(0, u)), u))
    for _ in range(core):
        a, b = (int(x) for x in rng.integers(0, core, 2))
        if a != b:
            edges.add((min(a, b), max(a, b)))
    for v in range(core, n - 4):  # leaves hung on core vertices
        edges.add((int(rng.integers(0, core)), v))
    edges.add((n - 4, n - 3))  # a two-vertex component: both ends have degree 1, neither is folded
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    return adj


def test_folded_leaf_identity_over_shards():
    n = 64
    for seed in range(20):
        adj = random_graph_with_leaves(n, seed)
        deg = [len(a) for a in adj]
        D = np.stack([distances(n, adj, s) for s in range(n)])  # D[s, v]
        leaves = [v for v in range(n) if deg[v] == 1 and deg[adj[v][0]] >= 2]
        assert leaves
        for spb, world in ((64, 1), (4, 3), (8, 2), (1, 5)):
            for rank in range(world):
                S = np.array([(s // spb) % world == rank for s in range(n)])

                def partial(v):  # F_S(v), R_S(v): over the shard's sources that reach v, other than v
                    m = S & (D[:, v] > 0)
                    return int(D[m, v].sum()), int(m.sum())

                for v in leaves:
                    p = adj[v][0]
                    Fp, Rp = partial(p)
                    ip, iv = int(S[p]), int(S[v])
                    F = (Fp + Rp + ip - 2 * iv) % (1 << 64)
                    R = (Rp + ip - iv) % (1 << 32)
                    assert (F, R) == partial(v), (seed, spb, world, rank, v)
        # one shard of everything: F(v) = F(p) + R(p) - 1, R(v) = R(p)
        for v in leaves:
            p = adj[v][0]
            Fv = int(D[D[:, v] > 0, v].sum())
            Fp, Rp = int(D[D[:, p] > 0, p].sum()), int((D[:, p] > 0).sum())
            assert Fv == Fp + Rp - 1 and int((D[:, v] > 0).sum()) == Rp
