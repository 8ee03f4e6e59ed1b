"""Pins for the oracle: closed forms, brute force, library routines, invariants and
hand-worked examples. None of these compares the oracle with itself.

Cited passages: Section 4 (BFS closeness, Eq. 1, Wasserman-Faust normalisation,
AND ground truth, naive composition), Section 5.1 (CC1, Eqs. 2-3),
Section 5.2 (CC2, Algorithm 1), Section 6.1 (Jaccard/precision/recall/F1).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2207_11662_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def edges_of(pairs):
    s = np.array([a for a, _ in pairs], np.int32)
    d = np.array([b for _, b in pairs], np.int32)
    return s, d


def path(n):
    return edges_of([(i, i + 1) for i in range(n - 1)])


def cycle(n):
    return edges_of([(i, (i + 1) % n) for i in range(n)])


def star(n):
    return edges_of([(0, i) for i in range(1, n)])


def complete(n):
    return edges_of([(i, j) for i in range(n) for j in range(i + 1, n)])


def fr(n, e):
    rp, c = O.simple_csr(n, *e)
    return O.farness_reach(n, rp, c)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 17, 40])
def test_path_closed_form(n):
    F, R = fr(n, path(n))
    for i in range(n):
        assert F[i] == i * (i + 1) // 2 + (n - 1 - i) * (n - i) // 2
        assert R[i] == n - 1


@pytest.mark.parametrize("n", [3, 4, 7, 10, 33])
def test_cycle_closed_form(n):
    F, R = fr(n, cycle(n))
    assert np.all(F == n * n // 4)
    assert np.all(R == n - 1)


@pytest.mark.parametrize("n", [2, 3, 6, 25])
def test_star_closed_form(n):
    F, R = fr(n, star(n))
    assert F[0] == n - 1
    assert np.all(F[1:] == 2 * n - 3)


@pytest.mark.parametrize("n", [2, 3, 9])
def test_complete_closed_form(n):
    F, R = fr(n, complete(n))
    assert np.all(F == n - 1) and np.all(R == n - 1)


def test_empty_graph():
    n = 7
    F, R = fr(n, (np.zeros(0, np.int32), np.zeros(0, np.int32)))
    assert np.all(F == 0) and np.all(R == 0)
    assert np.all(O.wf_closeness(n, F, R) == 0.0)
    # every other vertex unreachable: sumDist = n * (n - 1)
    assert np.all(O.sum_dist_n(n, F, R) == n * (n - 1))


def test_disjoint_components_wf_and_sumdist():
    # K_4 on {0..3}, K_3 on {4,5,6}, isolated 7 and 8: n = 9
    n = 9
    pairs = [(i, j) for i in range(4) for j in range(i + 1, 4)] + [(4, 5), (4, 6), (5, 6)]
    F, R = fr(n, edges_of(pairs))
    sizes = [4, 4, 4, 4, 3, 3, 3, 1, 1]
    cc = O.wf_closeness(n, F, R)
    sd = O.sum_dist_n(n, F, R)
    for v, c in enumerate(sizes):
        assert F[v] == c - 1 and R[v] == c - 1
        # Wasserman-Faust: (c-1)/(n-1) for a clique component, 0 for an isolated vertex
        assert cc[v] == ((c - 1) / (n - 1) if c > 1 else 0.0)
        # Section 5.1: unreachable vertices cost n each
        assert sd[v] == (c - 1) + n * (n - c)


def test_eq1_on_connected_graphs():
    # Eq. 1, CC(u) = (n-1) / sum of distances, is what the WF form gives on a connected graph
    for seed in range(20):
        n = 30
        s, d = synth.er_edges(n, 60, seed)
        s = np.concatenate([s, path(n)[0]]).astype(np.int32)
        d = np.concatenate([d, path(n)[1]]).astype(np.int32)
        F, R = fr(n, (s, d))
        assert np.all(R == n - 1)
        cc = O.wf_closeness(n, F, R)
        assert np.array_equal(cc, (n - 1) / F.astype(np.float64))


# ---------------------------------------------------------------- brute force

def floyd_warshall(n, pairs):
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0)
    for a, b in pairs:
        if a != b:
            D[a, b] = D[b, a] = 1
    for k in range(n):
        D = np.minimum(D, D[:, [k]] + D[[k], :])
    return D


@pytest.mark.parametrize("seed", range(60))
def test_floyd_warshall_random(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 41))
    m = int(rng.integers(0, 2 * n + 1))
    pairs = [(int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(m)]
    D = floyd_warshall(n, pairs)
    F, R = fr(n, edges_of(pairs) if pairs else (np.zeros(0, np.int32), np.zeros(0, np.int32)))
    fin = np.isfinite(D)
    assert np.array_equal(F, np.where(fin, D, 0).sum(axis=1).astype(np.uint64))
    assert np.array_equal(R, (fin.sum(axis=1) - 1).astype(np.uint32))


def test_scipy_shortest_path_and_threads():
    sp = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sps
    n = 400
    s, d = synth.er_edges(n, 500, 7)  # sparse: several components
    rp, c = O.simple_csr(n, s, d)
    A = sps.csr_matrix((np.ones(c.shape[0]), c, rp), shape=(n, n))
    D = sp.shortest_path(A, unweighted=True, directed=False)
    fin = np.isfinite(D)
    F1, R1 = O.farness_reach(n, rp, c, threads=1)
    F4, R4 = O.farness_reach(n, rp, c, threads=4)
    assert np.array_equal(F1, np.where(fin, D, 0).sum(axis=1).astype(np.uint64))
    assert np.array_equal(R1, (fin.sum(axis=1) - 1).astype(np.uint32))
    assert np.array_equal(F1, F4) and np.array_equal(R1, R4)
    sub = np.array([5, 0, 399, 17], np.int32)
    Fs, Rs = O.farness_reach(n, rp, c, sources=sub)
    assert np.array_equal(Fs, F1[sub]) and np.array_equal(Rs, R1[sub])


# ---------------------------------------------------------------- graphs

def brute_edge_set(pairs):
    return {(min(a, b), max(a, b)) for a, b in pairs if a != b}


def test_simple_graph_normalisation():
    n = 50
    e = synth.er_edges(n, 120, 3)
    noisy = synth.noisy_copy(n, e, 4)
    k1 = O.edge_keys(n, *e)
    k2 = O.edge_keys(n, *noisy)
    assert np.array_equal(k1, k2)
    want = sorted(brute_edge_set(zip(noisy[0].tolist(), noisy[1].tolist())))
    got = list(zip(*O.keys_to_edges(n, k2)))
    assert [tuple(map(int, x)) for x in got] == want
    rp, c = O.csr_from_keys(n, k2)
    for u in range(n):
        row = c[rp[u]:rp[u + 1]].tolist()
        assert row == sorted({b for a, b in want if a == u} | {a for a, b in want if b == u})


def test_and_aggregation_invariants():
    n = 200
    net = synth.homln_small_overlap(n, 6.0, 3, 0.5, 9)
    keys = [O.edge_keys(n, s, d) for s, d in net.layers]
    a = O.and_keys(n, keys)
    brute = brute_edge_set(zip(net.layers[0][0].tolist(), net.layers[0][1].tolist()))
    for s, d in net.layers[1:]:
        brute &= brute_edge_set(zip(s.tolist(), d.tolist()))
    assert [tuple(map(int, x)) for x in zip(*O.keys_to_edges(n, a))] == sorted(brute)
    for k in keys:
        assert np.all(np.isin(a, k))  # AND graph never has more edges than a layer
    assert np.array_equal(O.and_keys(n, [keys[2], keys[0], keys[1]]), a)  # order of the layers is irrelevant
    assert np.array_equal(O.and_keys(n, [keys[1], keys[1]]), keys[1])  # identical layers
    assert O.and_keys(n, [keys[0], np.zeros(0, np.int64)]).size == 0  # with an empty layer
    assert a.size > 0
    # OR aggregation: brute-force union; every layer is a subset of it; AND is a subset of OR
    o = O.or_keys(n, keys)
    union = set()
    for s, d in net.layers:
        union |= brute_edge_set(zip(s.tolist(), d.tolist()))
    assert [tuple(map(int, x)) for x in zip(*O.keys_to_edges(n, o))] == sorted(union)
    assert all(np.all(np.isin(k, o)) for k in keys) and np.all(np.isin(a, o))


# ---------------------------------------------------------------- selection

def test_selection_special_cases():
    ge = O.Select(O.GE_MEAN)
    gt = O.Select(O.GT_MEAN)
    for n, e in [(9, cycle(9)), (6, complete(6))]:
        F, R = fr(n, e)
        cc = O.wf_closeness(n, F, R)
        assert sorted(O.select(cc, ge).tolist()) == list(range(n))  # vertex-transitive: all equal the mean
        assert O.select(cc, gt).size == 0
    n = 8
    F, R = fr(n, star(n))
    assert O.select(O.wf_closeness(n, F, R), ge).tolist() == [0]
    assert O.select(np.full(10, 0.5), O.Select(O.TOPK_COUNT, k=4)).tolist() == [0, 1, 2, 3]
    assert O.topk_count(O.Select(O.TOPK_PERCENT, percent=10.0), 1000) == 100
    assert O.topk_count(O.Select(O.TOPK_PERCENT, percent=10.0), 1001) == 101
    assert O.topk_count(O.Select(O.TOPK_COUNT, k=50), 7) == 7


def test_exact_mean_boundary():
    s = np.array([0.5, 0.25, 0.75])  # mean is exactly 0.5
    assert O.select(s, O.Select(O.GE_MEAN)).tolist() == [2, 0]
    assert O.select(s, O.Select(O.GT_MEAN)).tolist() == [2]
    # 0.1 + 0.2 + 0.3 is not 0.6 in float64 arithmetic; the exact mean of the three doubles decides
    v = np.array([0.1, 0.2, 0.3])
    exact = Fraction(0.1) + Fraction(0.2) + Fraction(0.3)
    want = [i for i in (2, 1, 0) if Fraction(float(v[i])) * 3 >= exact]
    assert O.select(v, O.Select(O.GE_MEAN)).tolist() == want


# ---------------------------------------------------------------- golden examples

def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *rest = line.split()
            out[k] = rest
    return out


def pairs_of(tokens):
    return [tuple(int(x) for x in t.split("-")) for t in tokens]


def test_fig5_cc2_example():
    g = read_golden("fig5_cc2_example.txt")
    est = O.cc2_estimate([np.array([int(g["sumdist_layer1"][0])], np.uint64),
                          np.array([int(g["sumdist_layer2"][0])], np.uint64)])
    assert int(est[0]) == int(g["est"][0])


def test_hand_two_layer_example():
    g = read_golden("hand_two_layer_example.txt")
    n = int(g["n"][0])
    ex, ey = edges_of(pairs_of(g["layer_x"])), edges_of(pairs_of(g["layer_y"]))
    net = O.OracleHoMLN(n, [ex, ey])
    Lx, Ly = net.layer(0), net.layer(1)
    ints = lambda k: [int(x) for x in g[k]]
    fracs = lambda k: [Fraction(x) for x in g[k]]
    assert Lx["F"].tolist() == ints("F_x") and Ly["F"].tolist() == ints("F_y")
    assert Lx["deg"].tolist() == ints("deg_x") and Ly["deg"].tolist() == ints("deg_y")
    for got, want in [(Lx["cc"], fracs("cc_x")), (Ly["cc"], fracs("cc_y"))]:
        assert got.tolist() == [float(w) for w in want]
    top3 = O.Select(O.TOPK_COUNT, k=3, cc1_overlap=0.5)
    assert net.topk(0, 3, top3).tolist() == ints("CH_x")
    assert net.topk(1, 3, top3).tolist() == ints("CH_y")
    assert net.compose(3, O.NAIVE, top3).tolist() == ints("naive")
    ratios, _ = O.cc1_ratios([Lx["sumdist"], Ly["sumdist"]], [Lx["deg"], Ly["deg"]])
    assert O.cc1_average(ratios) == Fraction(g["cc1_avg"][0])
    assert net.compose(3, O.CC1, top3).tolist() == ints("cc1_theta_0.5")
    assert net.compose(3, O.CC1, O.Select(O.TOPK_COUNT, k=3, cc1_overlap=0.75)).tolist() == ints("cc1_theta_0.75")
    assert O.cc2_estimate([Lx["sumdist"], Ly["sumdist"]]).tolist() == ints("cc2_est")
    assert net.compose(3, O.CC2, top3).tolist() == ints("cc2")
    ae = list(zip(*[x.tolist() for x in net.and_edges(3)]))
    assert ae == pairs_of(g["and_edges"])
    A = net.and_graph(3)
    assert A["F"].tolist() == ints("F_and") and A["R"].tolist() == ints("R_and")
    assert A["cc"].tolist() == [float(x) for x in fracs("cc_and")]
    assert A["sumdist"].tolist() == ints("sumdist_and")
    assert net.topk(-1, 3, top3).tolist() == ints("gt_top3")
    assert net.topk(-1, 3, O.Select(O.GE_MEAN)).tolist() == ints("gt_ge_mean")
    gt = net.topk(-1, 3, top3)
    for key, pred in [("acc_naive", net.compose(3, O.NAIVE, top3)), ("acc_cc2", net.compose(3, O.CC2, top3))]:
        want = dict(t.split("=") for t in g[key])
        got = O.accuracy(pred, gt)
        for k in ("tp", "fp", "fn"):
            assert got[k] == int(want[k])
        for k in ("jaccard", "precision", "recall", "f1"):
            assert got[k] == float(Fraction(want[k]))


# ---------------------------------------------------------------- stated special cases of the method

def test_identical_layers_naive_equals_ground_truth():
    # Section 4: naive composition coincides with the ground truth when the layers are identical
    n = 300
    e = synth.er_edges(n, 900, 12)
    net = O.OracleHoMLN(n, [e, synth.noisy_copy(n, e, 1), e])
    for sel in [O.Select(O.TOPK_PERCENT, 10.0), O.Select(O.GE_MEAN)]:
        assert net.compose(7, O.NAIVE, sel).tolist() == sorted(net.topk(-1, 7, sel).tolist())


def test_cc2_subset_layers_equals_ground_truth():
    # Section 5.2: with E_x a subset of E_y the AND graph is G_x and the max rule returns sumDist_x;
    # for a connected G_x the CC2 estimate is exact, so its CC-node set is the ground truth's
    for seed in range(5):
        n = 200
        base = synth.er_edges(n, 500, 40 + seed)
        s = np.concatenate([base[0], path(n)[0]]).astype(np.int32)
        d = np.concatenate([base[1], path(n)[1]]).astype(np.int32)
        extra = synth.er_edges(n, 300, 80 + seed)
        ey = (np.concatenate([s, extra[0]]).astype(np.int32), np.concatenate([d, extra[1]]).astype(np.int32))
        net = O.OracleHoMLN(n, [(s, d), ey])
        est = O.cc2_estimate([net.layer(0)["sumdist"], net.layer(1)["sumdist"]])
        assert np.array_equal(est, net.and_graph(3)["F"])
        for sel in [O.Select(O.TOPK_PERCENT, 10.0), O.Select(O.GE_MEAN)]:
            assert net.compose(3, O.CC2, sel).tolist() == sorted(net.topk(-1, 3, sel).tolist())


def test_cc2_single_layer_is_sumdist_ranking():
    n = 150
    e = synth.er_edges(n, 200, 5)  # disconnected: exercises the unreachable = n convention
    net = O.OracleHoMLN(n, [e])
    sd = net.layer(0)["sumdist"]
    order = sorted(range(n), key=lambda u: (int(sd[u]), u))[:O.topk_count(O.Select(), n)]
    assert net.compose(1, O.CC2, O.Select()).tolist() == sorted(order)


# ---------------------------------------------------------------- metrics

def test_accuracy_metrics():
    a = O.accuracy([1, 2, 3, 4], [3, 4, 5])
    assert (a["tp"], a["fp"], a["fn"]) == (2, 2, 1)
    assert a["jaccard"] == 2 / 5 and a["precision"] == 2 / 4 and a["recall"] == 2 / 3
    assert math.isclose(a["f1"], 2 * 0.5 * (2 / 3) / (0.5 + 2 / 3), rel_tol=1e-15)
    e = O.accuracy([], [])
    assert (e["jaccard"], e["precision"], e["recall"], e["f1"]) == (1.0, 0.0, 0.0, 0.0)
    z = O.accuracy([1], [2])
    assert (z["tp"], z["fp"], z["fn"], z["jaccard"], z["f1"]) == (0, 1, 1, 0.0, 0.0)


# ---------------------------------------------------------------- directed layers (Section 4: closeness
# is defined for directed graphs too; in-closeness, the NetworkX convention)

def directed_fr(n, pairs):
    net = O.OracleHoMLN(n, [edges_of(pairs)], directed=True)
    L = net.layer(0)
    return L["F"], L["R"], L["deg"]


def test_directed_path_and_cycle_closed_forms():
    n = 12
    F, R, deg = directed_fr(n, [(i, i + 1) for i in range(n - 1)])  # 0 -> 1 -> ... -> n-1
    for i in range(n):
        assert F[i] == i * (i + 1) // 2 and R[i] == i  # reached from 0..i-1 at distances i..1
        assert deg[i] == (1 if i > 0 else 0)  # in-degree
    F, R, _ = directed_fr(n, [(i, (i + 1) % n) for i in range(n)])
    assert np.all(F == n * (n - 1) // 2) and np.all(R == n - 1)


@pytest.mark.parametrize("seed", range(20))
def test_directed_floyd_warshall(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 30))
    pairs = [(int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(int(rng.integers(1, 3 * n)))]
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0)
    for a, b in pairs:
        if a != b:
            D[a, b] = 1
    for k in range(n):
        D = np.minimum(D, D[:, [k]] + D[[k], :])
    F, R, _ = directed_fr(n, pairs)
    fin = np.isfinite(D)
    # in-closeness of u: distances d(v, u) over the v that reach u (column u)
    assert np.array_equal(F, np.where(fin, D, 0).sum(axis=0).astype(np.uint64))
    assert np.array_equal(R, (fin.sum(axis=0) - 1).astype(np.uint32))


def test_directed_symmetric_arcs_reduce_to_undirected():
    """Every arc together with its reverse: in-closeness equals undirected closeness."""
    net = synth.homln_small_overlap(300, 5.0, 2, 0.4, 17)
    und = O.OracleHoMLN(net.n, net.layers)
    both = [(np.concatenate([s, d]), np.concatenate([d, s])) for s, d in net.layers]
    dire = O.OracleHoMLN(net.n, both, directed=True)
    for i in range(2):
        for k in ("F", "R", "cc", "deg"):
            assert np.array_equal(dire.layer(i)[k], und.layer(i)[k]), k
    for k in ("F", "R", "cc"):
        assert np.array_equal(dire.and_graph(3)[k], und.and_graph(3)[k])
        assert np.array_equal(dire.or_graph(3)[k], und.or_graph(3)[k])


def test_directed_aggregates_are_arc_sets():
    """An arc and its reverse are different arcs: AND keeps only arcs present with the same direction."""
    n = 4
    x = edges_of([(0, 1), (1, 2), (2, 3)])
    y = edges_of([(1, 0), (1, 2), (3, 2)])
    net = O.OracleHoMLN(n, [x, y], directed=True)
    s, d = net.and_edges(3)
    assert list(zip(s.tolist(), d.tolist())) == [(1, 2)]
    s, d = net.or_edges(3)
    assert list(zip(s.tolist(), d.tolist())) == [(0, 1), (1, 0), (1, 2), (2, 3), (3, 2)]
    assert net.and_graph(3)["deg"].tolist() == [0, 0, 1, 0]  # in-degrees
