"""GPU-vs-oracle parity through the C-ABI.

Integer outputs (farness, reach, AND edge sets, CC-node lists, accuracy counts)
must match bit for bit. Closeness values are one correctly rounded division of
the same exact integers on both sides, so they are compared bit for bit too
(stricter than the 1e-12 relative tolerance the path allows; the tolerance is
used only where stated).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2207_11662_gb300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12


@pytest.fixture(scope="module")
def H():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    torch.cuda.set_device(0)
    from paper_2207_11662_gb300 import homln
    return homln


def to_dev(layers):
    import torch
    return [(torch.from_numpy(np.ascontiguousarray(s)).cuda(), torch.from_numpy(np.ascontiguousarray(d)).cuda())
            for s, d in layers]


def u64(t):
    return t.cpu().numpy().astype(np.uint64)


def check_graph(gF, gR, gcc, ref):
    assert np.array_equal(u64(gF), ref["F"])
    assert np.array_equal(gR.cpu().numpy().astype(np.uint32), ref["R"])
    cc = gcc.cpu().numpy()
    assert np.array_equal(cc, ref["cc"]), np.max(np.abs(cc - ref["cc"]))


def full_parity(H, net, sels, tuning=None, heuristics=(0, 1, 2), directed=False):
    g = H.Network(net.n, to_dev(net.layers), tuning=tuning, directed=directed)
    ref = O.OracleHoMLN(net.n, net.layers, threads=8, directed=directed)
    L = net.n_layers
    for i in range(L):
        check_graph(*g.layer_closeness(i), ref.layer(i))
    masks = sorted({(1 << L) - 1, 1, 3 if L >= 2 else 1})
    for mask in masks:
        s, d = g.and_aggregate(mask)
        rs, rd = ref.and_edges(mask)
        assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(d.cpu().numpy(), rd)
        check_graph(*g.and_closeness(mask), ref.and_graph(mask))
        for sel, osel in sels:
            gt = g.topk(-1, mask, sel)
            assert gt.cpu().numpy().tolist() == ref.topk(-1, mask, osel).tolist()
            for i in range(L):
                assert g.topk(i, mask, sel).cpu().numpy().tolist() == ref.topk(i, mask, osel).tolist()
            for heur in heuristics:
                est = g.compose(mask, heur, sel)
                want = ref.compose(mask, heur, osel)
                assert est.cpu().numpy().tolist() == want.tolist(), (mask, heur)
                acc = g.accuracy(est, gt)
                wa = O.accuracy(want, ref.topk(-1, mask, osel))
                for k in ("tp", "fp", "fn"):
                    assert acc[k] == wa[k]
                for k in ("jaccard", "precision", "recall", "f1"):
                    assert acc[k] == pytest.approx(wa[k], rel=REL_TOL, abs=0)
    g.close()


def sels_all(H):
    return [(H.make_select(H.HOMLN_TOPK_PERCENT, 10.0, cc1_overlap=0.5), O.Select(O.TOPK_PERCENT, 10.0, cc1_overlap=0.5)),
            (H.make_select(H.HOMLN_GE_MEAN, cc1_overlap=0.3), O.Select(O.GE_MEAN, cc1_overlap=0.3)),
            (H.make_select(H.HOMLN_GT_MEAN), O.Select(O.GT_MEAN)),
            (H.make_select(H.HOMLN_TOPK_COUNT, k=37, cc1_overlap=0.75), O.Select(O.TOPK_COUNT, k=37, cc1_overlap=0.75))]


def test_small_er_config(H):
    """3 independent ER layers, n = 1000, average degree 8 (the AND graph is almost empty)."""
    full_parity(H, synth.homln_small_er(), sels_all(H))


def test_small_overlap_config(H):
    """The same shape with a shared edge pool, so the AND graph and the heuristics are non-trivial."""
    full_parity(H, synth.homln_small_overlap(1000, 8.0, 3, 0.5, 111), sels_all(H))


def test_hand_example(H):
    import tests.test_oracle_pins as P
    g = P.read_golden("hand_two_layer_example.txt")
    n = int(g["n"][0])
    net = synth.HoMLN(n, [P.edges_of(P.pairs_of(g["layer_x"])), P.edges_of(P.pairs_of(g["layer_y"]))])
    full_parity(H, net, sels_all(H) + [(H.make_select(H.HOMLN_TOPK_COUNT, k=3), O.Select(O.TOPK_COUNT, k=3))])


@pytest.mark.parametrize("W", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("relabel", [0, 1])
def test_words_per_node_and_relabel(H, W, relabel):
    """Every batch width and both vertex orders give identical results (ragged last batch included)."""
    net = synth.homln_small_overlap(1537, 6.0, 2, 0.4, 5)
    sel = [(H.make_select(H.HOMLN_TOPK_PERCENT, 10.0), O.Select(O.TOPK_PERCENT, 10.0))]
    full_parity(H, net, sel, tuning=dict(words_per_node=W, relabel=relabel), heuristics=(2,))


@pytest.mark.parametrize("alpha", [1, 1000000])
def test_push_pull_extremes(H, alpha):
    """alpha = 1: almost always bottom-up; alpha = 1e6: almost always top-down. Same answers."""
    net = synth.HoMLN(3000, [synth.chung_lu_edges(3000, 12000, 9), synth.ba_edges(3000, 3, 10)])
    sel = [(H.make_select(H.HOMLN_TOPK_PERCENT, 10.0), O.Select(O.TOPK_PERCENT, 10.0))]
    full_parity(H, net, sel, tuning=dict(push_alpha=alpha, words_per_node=4), heuristics=(2,))


@pytest.mark.parametrize("teams,mix", [(1, 0), (2, 1), (7, 0), (7, 1), (100000, 0)])
def test_batched_analyse_and_teams(H, teams, mix):
    """All layers and the AND graph in one persistent launch, split over 1, 2, 7 or one-block teams."""
    net = synth.homln_small_overlap(2500, 7.0, 4, 0.5, 31)
    g = H.Network(net.n, to_dev(net.layers), tuning=dict(teams=teams, words_per_node=4, team_mix=mix))
    g.analyse(15, True)
    ref = O.OracleHoMLN(net.n, net.layers, threads=8)
    for i in range(4):
        check_graph(*g.layer_closeness(i), ref.layer(i))
    check_graph(*g.and_closeness(15), ref.and_graph(15))
    g.close()


def test_plain_schedule(H):
    """The plain schedule (one launch per phase, host-driven levels) gives the same answers."""
    net = synth.homln_small_overlap(3000, 8.0, 3, 0.5, 41)
    ref = O.OracleHoMLN(net.n, net.layers, threads=8)
    for W in (2, 8):
        g = H.Network(net.n, to_dev(net.layers), tuning=dict(schedule=1, words_per_node=W))
        for i in range(3):
            check_graph(*g.layer_closeness(i), ref.layer(i))
        check_graph(*g.and_closeness(7), ref.and_graph(7))
        g.close()


def test_batch_analyse_across_handles(H):
    """Many HoMLNs of uneven sizes (and streams) in one persistent launch; then invalidate and redo."""
    import torch
    nets = synth.homln_batch(count=6, seed=77, n_range=(300, 4000), layer_range=(2, 4))
    streams = [torch.cuda.Stream() for _ in range(2)]
    gs = [H.Network(net.n, to_dev(net.layers), stream=streams[i % 2].cuda_stream) for i, net in enumerate(nets)]
    masks = [(1 << net.n_layers) - 1 for net in nets]
    for rep in range(2):
        H.homln_batch_analyse([g.h for g in gs], masks, True)
        for g, net, mask in zip(gs, nets, masks):
            ref = O.OracleHoMLN(net.n, net.layers, threads=8)
            with torch.cuda.stream(torch.cuda.ExternalStream(g.stream)):
                for i in range(net.n_layers):
                    check_graph(*g.layer_closeness(i), ref.layer(i))
                check_graph(*g.and_closeness(mask), ref.and_graph(mask))
        for g in gs:
            H.homln_invalidate(g.h)
    for g in gs:
        g.close()


def test_subset_sweep(H):
    """Every subset of at least two of four layers: ground truth, estimate and accuracy vs the oracle."""
    net = synth.homln_small_overlap(900, 9.0, 4, 0.5, 61)
    ref = O.OracleHoMLN(net.n, net.layers, threads=8)
    g = H.Network(net.n, to_dev(net.layers))
    for heur in (H.HOMLN_NAIVE, H.HOMLN_CC1, H.HOMLN_CC2):
        sel, osel = H.make_select(H.HOMLN_TOPK_PERCENT, 10.0), O.Select(O.TOPK_PERCENT, 10.0)
        res = H.homln_subset_sweep(g.h, heur, sel, 2)
        assert [r["mask"] for r in res] == [m for m in range(1, 16) if bin(m).count("1") >= 2]
        for r in res:
            gt = ref.topk(-1, r["mask"], osel)
            est = ref.compose(r["mask"], heur, osel)
            want = O.accuracy(est, gt)
            assert (r["truth_count"], r["estimate_count"]) == (len(gt), len(est))
            assert (r["tp"], r["fp"], r["fn"]) == (want["tp"], want["fp"], want["fn"])
            assert r["jaccard"] == pytest.approx(want["jaccard"], rel=REL_TOL, abs=0)
    g.close()


def test_or_aggregation(H):
    """OR graphs (edges in at least one selected layer): edge lists, closeness and top-k vs the oracle."""
    net = synth.homln_small_overlap(1200, 6.0, 3, 0.3, 71)
    ref = O.OracleHoMLN(net.n, net.layers, threads=8)
    g = H.Network(net.n, to_dev(net.layers))
    sel, osel = H.make_select(H.HOMLN_TOPK_PERCENT, 10.0), O.Select(O.TOPK_PERCENT, 10.0)
    for mask in (7, 5, 2):
        s, d = g.or_aggregate(mask)
        rs, rd = ref.or_edges(mask)
        assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(d.cpu().numpy(), rd)
        check_graph(*g.or_closeness(mask), ref.or_graph(mask))
        out = g.topk(-2, mask, sel)
        assert out.cpu().numpy().tolist() == ref.topk(-2, mask, osel).tolist()
    g.close()


def directed_net(n=1500, avg=6.0, L=3, rho=0.4, seed=91, recip=0.25):
    net = synth.homln_small_overlap(n, avg, L, rho, seed)
    return synth.HoMLN(n, [synth.with_reciprocal(e, recip, seed + i) for i, e in enumerate(net.layers)])


@pytest.mark.parametrize("W,alpha,relabel", [(8, 16, 1), (2, 1, 0), (1, 1000000, 1), (32, 16, 0)])
def test_directed_layers(H, W, alpha, relabel):
    """Directed layers (in-closeness): pull along in-edges, push along out-edges, in-degree CC1."""
    full_parity(H, directed_net(), sels_all(H)[:2], directed=True,
                tuning=dict(words_per_node=W, push_alpha=alpha, relabel=relabel))


def test_batch_analyse_mixes_directed_and_undirected(H):
    """One persistent launch over the tiles of a directed and an undirected HoMLN."""
    nets = [directed_net(900, 5.0, 2, 0.3, 81), synth.homln_small_overlap(700, 6.0, 3, 0.4, 82)]
    kinds = [True, False]
    gs = [H.Network(net.n, to_dev(net.layers), directed=dr) for net, dr in zip(nets, kinds)]
    masks = [(1 << net.n_layers) - 1 for net in nets]
    H.homln_batch_analyse([g.h for g in gs], masks, True)
    for g, net, mask, dr in zip(gs, nets, masks, kinds):
        ref = O.OracleHoMLN(net.n, net.layers, threads=8, directed=dr)
        for i in range(net.n_layers):
            check_graph(*g.layer_closeness(i), ref.layer(i))
        check_graph(*g.and_closeness(mask), ref.and_graph(mask))
        g.close()


def test_directed_sinks_reached_after_the_core_is_full(H):
    """A strongly connected core (0..199) with sinks (200..299, out-degree 0) hanging off it, every
    level top-down, 64 sources per batch and no relabelling: in the batches whose sources all lie
    in the core, the core vertices become full while the sinks still wait for their last bits one
    level later. The BFS must run that level (nothing may end a directed batch early because the
    vertices that are not full have no out-edges)."""
    rng = np.random.default_rng(17)
    core = 200
    s = list(range(core)) + list(rng.integers(0, core, 400))
    d = [(i + 1) % core for i in range(core)] + list(rng.integers(0, core, 400))
    for k in range(100):  # sink 200 + k, fed by one or two core vertices
        for _ in range(1 + k % 2):
            s.append(int(rng.integers(0, core)))
            d.append(core + k)
    net = synth.HoMLN(300, [(np.array(s, np.int32), np.array(d, np.int32))])
    sel = [(H.make_select(H.HOMLN_TOPK_PERCENT, 10.0), O.Select(O.TOPK_PERCENT, 10.0))]
    for alpha in (1000000, 16):
        full_parity(H, net, sel, tuning=dict(words_per_node=1, push_alpha=alpha, relabel=0), heuristics=(2,),
                    directed=True)


def test_directed_or_hubs_and_closed_forms(H):
    """Directed OR graphs, an in-star and an out-star (hub tiers on the in-CSR), a directed path and cycle."""
    n = 3000
    path = (np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32))
    cyc = (np.arange(n, dtype=np.int32), ((np.arange(n) + 1) % n).astype(np.int32))
    g = H.Network(n, to_dev([path, cyc]), directed=True)
    F, R, _ = g.layer_closeness(0)
    i = np.arange(n, dtype=np.int64)
    assert np.array_equal(F.cpu().numpy(), i * (i + 1) // 2) and np.array_equal(R.cpu().numpy(), i)
    F, R, _ = g.layer_closeness(1)
    assert np.all(F.cpu().numpy() == n * (n - 1) // 2) and np.all(R.cpu().numpy() == n - 1)
    g.close()
    n = 5000
    into = (np.arange(1, n, dtype=np.int32), np.zeros(n - 1, np.int32))
    outof = (np.zeros(n - 1, np.int32), np.arange(1, n, dtype=np.int32))
    cl = synth.chung_lu_edges(n, 25000, 78)
    net = synth.HoMLN(n, [synth.overlay(n, into, cl), synth.overlay(n, outof, cl), cl])
    sel = [(H.make_select(H.HOMLN_TOPK_PERCENT, 10.0), O.Select(O.TOPK_PERCENT, 10.0))]
    for W in (2, 16):
        full_parity(H, net, sel, directed=True, tuning=dict(words_per_node=W, threads=256))
    dn = directed_net(1200, 5.0, 3, 0.3, 72)
    ref = O.OracleHoMLN(dn.n, dn.layers, threads=8, directed=True)
    g = H.Network(dn.n, to_dev(dn.layers), directed=True)
    for mask in (7, 5):
        s, d = g.or_aggregate(mask)
        rs, rd = ref.or_edges(mask)
        assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(d.cpu().numpy(), rd)
        check_graph(*g.or_closeness(mask), ref.or_graph(mask))
    g.close()


def test_hubs_use_block_and_warp_tiers(H):
    """A star plus a power-law layer: the centre's row exceeds the block threshold."""
    n = 5000
    star = (np.zeros(n - 1, np.int32), np.arange(1, n, dtype=np.int32))
    cl = synth.chung_lu_edges(n, 25000, 77)
    net = synth.HoMLN(n, [star, cl, synth.overlay(n, star, cl)])
    sel = [(H.make_select(H.HOMLN_TOPK_PERCENT, 10.0), O.Select(O.TOPK_PERCENT, 10.0)),
           (H.make_select(H.HOMLN_GE_MEAN), O.Select(O.GE_MEAN))]
    for W in (2, 16):
        full_parity(H, net, sel, tuning=dict(words_per_node=W, threads=256))


def test_rows_longer_than_the_shared_memory_sort(H):
    """A star whose centre row (19,999 entries) is longer than the block sort's 8,192: the CSR build
    and the relabelling sort it with the radix-sort fallback; plus duplicates in every row."""
    n = 20000
    star = (np.zeros(n - 1, np.int32), np.arange(1, n, dtype=np.int32))
    noisy = synth.noisy_copy(n, star, 5, self_loops=50, duplicates=3000)
    sel = [(H.make_select(H.HOMLN_TOPK_PERCENT, 10.0), O.Select(O.TOPK_PERCENT, 10.0))]
    full_parity(H, synth.HoMLN(n, [noisy, synth.overlay(n, star, synth.er_edges(n, 30000, 6))]), sel,
                heuristics=(0, 2))


def test_degenerate_graphs(H):
    sel = [(H.make_select(H.HOMLN_TOPK_PERCENT, 10.0), O.Select(O.TOPK_PERCENT, 10.0)),
           (H.make_select(H.HOMLN_GE_MEAN), O.Select(O.GE_MEAN))]
    empty = (np.zeros(0, np.int32), np.zeros(0, np.int32))
    # a single node, no edges
    full_parity(H, synth.HoMLN(1, [empty, empty]), sel)
    # two nodes joined in one layer only
    full_parity(H, synth.HoMLN(2, [(np.array([0], np.int32), np.array([1], np.int32)), empty]), sel)
    # self loops and duplicates only
    loops = (np.array([3, 3, 5, 5], np.int32), np.array([3, 3, 5, 5], np.int32))
    full_parity(H, synth.HoMLN(7, [loops, loops]), sel)
    # many small components with a ragged batch
    n = 4099
    e = synth.er_edges(n, 1500, 3)
    full_parity(H, synth.HoMLN(n, [e, synth.noisy_copy(n, e, 4)]), sel)


def test_many_nodes_small_components(H):
    """300,000 nodes in small components (average degree 0.8): the relabelling and selection
    sorts take the multi-block radix path with a separate scan (more than 64 tiles of 4,096)."""
    n = 300000
    a = synth.er_edges(n, 90000, 31)
    net = synth.HoMLN(n, [synth.overlay(n, a, synth.er_edges(n, 30000, 32)), synth.overlay(n, a, synth.er_edges(n, 30000, 33))])
    sel = [(H.make_select(H.HOMLN_TOPK_PERCENT, 10.0), O.Select(O.TOPK_PERCENT, 10.0)),
           (H.make_select(H.HOMLN_GE_MEAN), O.Select(O.GE_MEAN))]
    full_parity(H, net, sel, heuristics=(0, 2))


def _scattered_components(n, seed, equal_giants=False):
    """Edges of one graph whose components sit on random ids: a BA component (or two cycles of
    equal size), a path, components right at the BFS's small-component bound (a path and a cycle
    of 8 vertices, a star of 9), disjoint pairs, isolated vertices."""
    rng = np.random.default_rng(seed)
    ids = rng.permutation(n).astype(np.int32)
    parts = []
    if equal_giants:
        k = n // 4
        for off in (0, k):
            c = np.arange(k)
            parts.append((ids[off + c], ids[off + (c + 1) % k]))
        used = 2 * k
    else:
        k = n // 2
        s, d = synth.ba_edges(k, 3, seed)
        parts.append((ids[s], ids[d]))
        used = k
    p = n // 6  # a path: the second largest component
    parts.append((ids[used:used + p - 1], ids[used + 1:used + p]))
    used += p
    c = np.arange(8)
    parts.append((ids[used + c[:-1]], ids[used + c[1:]]))  # path of 8
    parts.append((ids[used + 8 + c], ids[used + 8 + (c + 1) % 8]))  # cycle of 8
    parts.append((np.full(8, ids[used + 16]), ids[used + 17 + c]))  # star of 9
    used += 25
    q = n // 20  # disjoint pairs; the rest stays isolated
    parts.append((ids[used:used + 2 * q:2], ids[used + 1:used + 2 * q:2]))
    s = np.concatenate([a for a, _ in parts]).astype(np.int32)
    d = np.concatenate([b for _, b in parts]).astype(np.int32)
    return s, d


@pytest.mark.parametrize("relabel", [1, 0])
def test_component_split_of_the_batches(H, relabel):
    """The BFS places the vertices of small components (at most 8 vertices) last and treats a
    batch's sources on the other side of that split as unreachable: graphs whose components sit
    on scattered ids, components at the bound, isolated vertices and pairs, each with and
    without the relabelling, and the AND graph of such layers (components of its own)."""
    n = 3001
    layers = [_scattered_components(n, 41), _scattered_components(n, 42, equal_giants=True)]
    shared = _scattered_components(n, 43)
    layers.append((np.concatenate([shared[0], layers[0][0][: len(layers[0][0]) // 2]]),
                   np.concatenate([shared[1], layers[0][1][: len(layers[0][1]) // 2]])))
    net = synth.HoMLN(n, layers)
    g = H.Network(n, to_dev(net.layers), tuning=dict(relabel=relabel, words_per_node=4))
    ref = O.OracleHoMLN(n, net.layers, threads=8)
    for i in range(len(layers)):
        check_graph(*g.layer_closeness(i), ref.layer(i))
    for mask in (0b101, 0b111):
        check_graph(*g.and_closeness(mask), ref.and_graph(mask))
    g.close()


def test_component_split_directed(H):
    """Directed layers: weak components, and vertices without in-arcs (never reached)."""
    n = 2500
    rng = np.random.default_rng(44)
    layers = []
    for seed in (45, 46):
        s, d = _scattered_components(n, seed)
        flip = rng.random(s.size) < 0.5
        s2, d2 = np.where(flip, d, s), np.where(flip, s, d)
        src_only = rng.choice(n, 40, replace=False).astype(np.int32)  # arcs out of them only
        tgt = rng.choice(n, 40).astype(np.int32)
        keep = ~np.isin(d2, src_only)
        layers.append((np.concatenate([s2[keep], src_only]).astype(np.int32),
                       np.concatenate([d2[keep], tgt]).astype(np.int32)))
    net = synth.HoMLN(n, layers)
    g = H.Network(n, to_dev(net.layers), directed=True)
    ref = O.OracleHoMLN(n, net.layers, threads=8, directed=True)
    for i in range(len(layers)):
        check_graph(*g.layer_closeness(i), ref.layer(i))
    check_graph(*g.and_closeness(0b11), ref.and_graph(0b11))
    g.close()


def _maximum_size_layer(n, seed):
    """Edges over the library's largest node count whose components sit on ids spread over the
    whole range: a 12,000-node BA component, a path of 600 (more levels than the level marks
    count before wrapping), components at the small-component bound (a path and a cycle of 8, a
    star of 9), 300 cycles of 12 just above it, 100,000 disjoint pairs; the rest is isolated."""
    rng = np.random.default_rng(seed)
    ids = rng.permutation(n).astype(np.int32)
    parts = []
    k = 12000
    s, d = synth.ba_edges(k, 3, seed)
    parts.append((ids[s], ids[d]))
    used = k
    p = 600
    parts.append((ids[used:used + p - 1], ids[used + 1:used + p]))
    used += p
    c = np.arange(8)
    parts.append((ids[used + c[:-1]], ids[used + c[1:]]))
    parts.append((ids[used + 8 + c], ids[used + 8 + (c + 1) % 8]))
    parts.append((np.full(8, ids[used + 16]), ids[used + 17 + c]))
    used += 25
    c = np.arange(12)
    for _ in range(300):
        parts.append((ids[used + c], ids[used + (c + 1) % 12]))
        used += 12
    q = 100000
    parts.append((ids[used:used + 2 * q:2], ids[used + 1:used + 2 * q:2]))
    s = np.concatenate([a for a, _ in parts]).astype(np.int32)
    d = np.concatenate([b for _, b in parts]).astype(np.int32)
    return s, d


def test_maximum_node_count_matches_oracle(H):
    """n = HOMLN_MAX_NODES (2^20): two layers (the second keeps a seeded 70% of the first's edges
    and adds 50,000 random ones), so the AND graph has components of its own. Every graph's
    farness, reach and closeness and the AND edge list against the oracle's full run; the top-10%
    ground truth, per-layer CC nodes, naive, CC1 and CC2 with their accuracy counts; the exact
    at-or-above-mean selection with CC2; farness and reach again at 32 words per node."""
    n = H.MAX_NODES
    s, d = _maximum_size_layer(n, 71)
    keep = np.random.default_rng(72).random(s.size) < 0.7
    extra = np.random.default_rng(73).integers(0, n, size=(2, 50000)).astype(np.int32)
    layers = [(s, d), (np.concatenate([s[keep], extra[0]]), np.concatenate([d[keep], extra[1]]))]
    ref = O.OracleHoMLN(n, layers, threads=os.cpu_count() or 1)
    g = H.Network(n, to_dev(layers))
    for i in range(2):
        check_graph(*g.layer_closeness(i), ref.layer(i))
    gs, gd = g.and_aggregate(3)
    rs, rd = ref.and_edges(3)
    assert np.array_equal(gs.cpu().numpy(), rs) and np.array_equal(gd.cpu().numpy(), rd)
    check_graph(*g.and_closeness(3), ref.and_graph(3))
    cases = [(H.make_select(H.HOMLN_TOPK_PERCENT, 10.0, cc1_overlap=0.5), O.Select(O.TOPK_PERCENT, 10.0, cc1_overlap=0.5),
              (0, 1, 2)),
             (H.make_select(H.HOMLN_GE_MEAN), O.Select(O.GE_MEAN), (2,))]
    for sel, osel, heuristics in cases:
        gt = g.topk(-1, 3, sel)
        want_gt = ref.topk(-1, 3, osel)
        assert gt.cpu().numpy().tolist() == want_gt.tolist()
        for i in range(2):
            assert g.topk(i, 3, sel).cpu().numpy().tolist() == ref.topk(i, 3, osel).tolist()
        for heur in heuristics:
            est = g.compose(3, heur, sel)
            want = ref.compose(3, heur, osel)
            assert est.cpu().numpy().tolist() == want.tolist(), heur
            acc = g.accuracy(est, gt)
            wa = O.accuracy(want, want_gt)
            assert (acc["tp"], acc["fp"], acc["fn"]) == (wa["tp"], wa["fp"], wa["fn"])
    g.close()
    g = H.Network(n, to_dev(layers), tuning=dict(words_per_node=32))
    for i in range(2):
        F, R, _ = g.layer_closeness(i)
        assert np.array_equal(u64(F), ref.layer(i)["F"])
        assert np.array_equal(R.cpu().numpy().astype(np.uint32), ref.layer(i)["R"])
    g.close()


def test_path_and_cycle_closed_forms(H):
    """Long diameters (thousands of levels) against the closed forms directly."""
    n = 3000
    path = (np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32))
    cyc = (np.arange(n, dtype=np.int32), ((np.arange(n) + 1) % n).astype(np.int32))
    g = H.Network(n, to_dev([path, cyc]))
    F, R, _ = g.layer_closeness(0)
    i = np.arange(n, dtype=np.uint64)
    want = i * (i + 1) // 2 + (n - 1 - i) * (n - i) // 2
    assert np.array_equal(u64(F), want)
    F, R, _ = g.layer_closeness(1)
    assert np.all(u64(F) == n * n // 4)
    g.close()


def test_host_buffers_match_device_buffers(H):
    net = synth.homln_small_overlap(800, 8.0, 2, 0.5, 21)
    ref = O.OracleHoMLN(net.n, net.layers)
    h = H.homln_create(net.n, net.layers)  # host edge lists
    F = np.zeros(net.n, np.uint64)
    R = np.zeros(net.n, np.uint32)
    cc = np.zeros(net.n, np.float64)
    H.homln_layer_closeness(h, 1, F, R, cc)
    assert np.array_equal(F, ref.layer(1)["F"]) and np.array_equal(R, ref.layer(1)["R"])
    assert np.array_equal(cc, ref.layer(1)["cc"])
    m = H.homln_and_aggregate(h, 3)
    s = np.zeros(m, np.int32)
    d = np.zeros(m, np.int32)
    assert H.homln_and_aggregate(h, 3, m, s, d) == m
    rs, rd = ref.and_edges(3)
    assert np.array_equal(s, rs) and np.array_equal(d, rd)
    out = np.zeros(net.n, np.int32)
    sel = H.make_select()
    c = H.homln_compose(h, 3, H.HOMLN_CC2, sel, out)
    assert out[:c].tolist() == ref.compose(3, O.CC2, O.Select()).tolist()
    gt = np.zeros(net.n, np.int32)
    cg = H.homln_topk(h, -1, 3, sel, gt)
    acc = H.homln_accuracy(h, out, c, gt, cg)
    want = O.accuracy(out[:c], gt[:cg])
    assert (acc["tp"], acc["fp"], acc["fn"]) == (want["tp"], want["fp"], want["fn"])
    H.homln_destroy(h)


def test_accuracy_edge_cases_match_the_oracle(H):
    """Accuracy of id lists against the oracle, exactly: empty lists on either or both sides,
    repeated ids, a node count that is not a multiple of 32, and lists long enough that the
    counts come from many blocks (the last of which forms the ratios)."""
    rng = np.random.default_rng(5)
    for n in (2, 33, 1000, 1_000_003):  # the largest: near the node limit of a handle, 2^20
        h = H.homln_create(n, [(np.array([0], np.int32), np.array([1], np.int32))])
        try:
            k = min(n, 5000 if n < 10**6 else 300_000)
            cases = [(np.zeros(0, np.int32), np.zeros(0, np.int32)),
                     (rng.choice(n, k, replace=False), np.zeros(0, np.int32)),
                     (np.zeros(0, np.int32), rng.choice(n, k, replace=False)),
                     (rng.choice(n, k, replace=True), rng.choice(n, k, replace=True)),
                     (rng.choice(n, k, replace=False), rng.choice(n, max(1, k // 3), replace=False)),
                     (np.full(7, n - 1), np.array([n - 1]))]
            for pred, truth in cases:
                pred = pred.astype(np.int32)
                truth = truth.astype(np.int32)
                got = H.homln_accuracy(h, pred, pred.size, truth, truth.size)
                want = O.accuracy(pred, truth)
                assert got == want, (n, pred.size, truth.size)
        finally:
            H.homln_destroy(h)


def test_error_statuses(H):
    n = 50
    bad = (np.array([0, 50], np.int32), np.array([1, 2], np.int32))
    with pytest.raises(H.HomlnError) as e:
        H.homln_create(n, [bad])
    assert e.value.code == H.HOMLN_EINVAL
    neg = (np.array([-1], np.int32), np.array([1], np.int32))
    with pytest.raises(H.HomlnError) as e:
        H.homln_create(n, [neg])
    assert e.value.code == H.HOMLN_EINVAL
    good = synth.er_edges(n, 100, 1)
    h = H.homln_create(n, [good, good])
    for mask in (0, 4, 1 << 63):
        with pytest.raises(H.HomlnError) as e:
            H.homln_and_aggregate(h, mask)
        assert e.value.code == H.HOMLN_EINVAL
    m = H.homln_and_aggregate(h, 3)
    with pytest.raises(H.HomlnError) as e:
        H.homln_and_aggregate(h, 3, m - 1, np.zeros(m, np.int32), np.zeros(m, np.int32))
    assert e.value.code == H.HOMLN_ERANGE
    with pytest.raises(H.HomlnError) as e:
        H.homln_layer_closeness(h, 2, None, None, None)
    assert e.value.code == H.HOMLN_EINVAL
    out = np.zeros(n, np.int32)
    for sel in (H.make_select(7), H.make_select(H.HOMLN_TOPK_PERCENT, 101.0), H.make_select(H.HOMLN_TOPK_COUNT, k=-1),
                H.make_select(cc1_overlap=1.5)):
        with pytest.raises(H.HomlnError) as e:
            H.homln_compose(h, 3, H.HOMLN_CC1, sel, out)
        assert e.value.code == H.HOMLN_EINVAL
    with pytest.raises(H.HomlnError) as e:
        H.homln_compose(h, 3, 9, H.make_select(), out)
    assert e.value.code == H.HOMLN_EINVAL
    with pytest.raises(H.HomlnError) as e:
        H.homln_accuracy(h, np.array([0, 60], np.int32), 2, np.array([1], np.int32), 1)
    assert e.value.code == H.HOMLN_EINVAL
    # the handle still works after every rejected call
    F = np.zeros(n, np.uint64)
    H.homln_layer_closeness(h, 0, F, None, None)
    assert np.array_equal(F, O.OracleHoMLN(n, [good]).layer(0)["F"])
    H.homln_destroy(h)


def test_allocator_failure_and_torch_allocator(H):
    """A caller allocator that fails on its k-th call gives ENOMEM and leaks nothing it handed out."""
    import ctypes
    import torch
    net = synth.homln_small_overlap(700, 6.0, 2, 0.5, 3)
    live = {}
    calls = [0]
    fail_at = [10 ** 9]

    @H.ALLOC_FN
    def alloc(ctx, nbytes, stream):
        calls[0] += 1
        if calls[0] == fail_at[0]:
            return None
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    @H.FREE_FN
    def free(ctx, p, nbytes, stream):
        live.pop(int(p))

    a = H.homln_allocator(None, alloc, free)
    h = H.homln_create(net.n, to_dev(net.layers), allocator=a)
    F = torch.empty(net.n, dtype=torch.int64, device="cuda")
    H.homln_layer_closeness(h, 0, F, None, None)
    H.homln_destroy(h)
    torch.cuda.synchronize()
    assert not live
    total = calls[0]
    assert total > 5
    for k in (1, 2, total // 2, total - 1):
        calls[0] = 0
        fail_at[0] = k
        try:
            h = H.homln_create(net.n, to_dev(net.layers), allocator=a)
            try:
                H.homln_layer_closeness(h, 0, F, None, None)
            except H.HomlnError as e:
                assert e.value.code == H.HOMLN_ENOMEM if hasattr(e, "value") else e.code == H.HOMLN_ENOMEM
            H.homln_destroy(h)
        except H.HomlnError as e:
            assert e.code == H.HOMLN_ENOMEM
        torch.cuda.synchronize()
        assert not live, f"leak after failing allocation {k}"
    # torch's caching allocator as the backend
    ta = H.torch_allocator()
    g = H.Network(net.n, to_dev(net.layers), allocator=ta)
    Fg, _, _ = g.layer_closeness(1)
    assert np.array_equal(u64(Fg), O.OracleHoMLN(net.n, net.layers).layer(1)["F"])
    g.close()


def test_bounded_wait_runs_out_and_the_handle_recovers(H):
    """Failure detection: team barriers that wait for blocks that do not exist give up after the
    wait limit; the call reports HOMLN_ETIMEOUT, the handle drops its results and stays usable."""
    import time
    net = synth.homln_small_overlap(700, 6.0, 2, 0.4, 44)
    ref = O.OracleHoMLN(net.n, net.layers, threads=8)
    g = H.Network(net.n, to_dev(net.layers))
    H.homln_set_tuning(g.h, wait_limit_ms=100, test_phantom_blocks=1)
    t0 = time.perf_counter()
    with pytest.raises(H.HomlnError) as e:
        g.layer_closeness(0)
        H.homln_sync(g.h)
    assert e.value.code == H.HOMLN_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    H.homln_set_tuning(g.h)
    for i in range(2):
        check_graph(*g.layer_closeness(i), ref.layer(i))
    check_graph(*g.and_closeness(3), ref.and_graph(3))
    g.close()


def test_checkpoint_and_resume_of_partials(H, tmp_path):
    """Export the Psi results of every layer and the AND graph, import them into a fresh handle:
    compositions and the ground truth match without running a BFS; impossible values are refused."""
    net = synth.homln_small_overlap(900, 7.0, 3, 0.5, 66)
    ref = O.OracleHoMLN(net.n, net.layers, threads=8)
    sel, osel = H.make_select(H.HOMLN_TOPK_PERCENT, 10.0), O.Select(O.TOPK_PERCENT, 10.0)
    a = H.Network(net.n, to_dev(net.layers))
    path = str(tmp_path / "partials.npz")
    a.save_partials(path, masks=(7, 3))
    a.close()
    b = H.Network(net.n, to_dev(net.layers))
    H.homln_set_profiling(b.h, True, False)
    b.load_partials(path)
    for i in range(3):
        check_graph(*b.layer_closeness(i), ref.layer(i))
    check_graph(*b.and_closeness(7), ref.and_graph(7))
    assert b.topk(-1, 7, sel).cpu().numpy().tolist() == ref.topk(-1, 7, osel).tolist()
    for heur in (0, 1, 2):
        assert b.compose(7, heur, sel).cpu().numpy().tolist() == ref.compose(7, heur, osel).tolist()
    assert H.homln_get_profile(b.h)["bfs_launches"] == 0
    # a reach larger than n - 1 cannot come from a BFS: refused, the imported results stay
    z = np.load(path)
    bad = np.ascontiguousarray(z["layer0_R"]).copy()
    bad[5] = net.n
    with pytest.raises(H.HomlnError) as e:
        H.homln_import_partials(b.h, 0, 0, np.ascontiguousarray(z["layer0_F"]), bad)
    assert e.value.code == H.HOMLN_ERANGE
    check_graph(*b.layer_closeness(0), ref.layer(0))
    assert H.homln_get_profile(b.h)["bfs_launches"] == 0
    b.close()


def test_relabel_setting_changed_between_analyses(H):
    """The BFS graphs are rebuilt when the relabelling setting changes on a live handle."""
    net = synth.homln_small_overlap(1100, 6.0, 3, 0.4, 87)
    ref = O.OracleHoMLN(net.n, net.layers, threads=8)
    g = H.Network(net.n, to_dev(net.layers))
    for relabel in (1, 0, 1):
        H.homln_set_tuning(g.h, relabel=relabel)
        H.homln_invalidate(g.h)
        H.homln_analyse(g.h, 7, True)
        for i in range(3):
            check_graph(*g.layer_closeness(i), ref.layer(i))
        check_graph(*g.and_closeness(7), ref.and_graph(7))
    g.close()


def test_batch_of_many_small_handles(H):
    """40 handles (each with its own side streams) analysed in one launch, then per handle."""
    nets = synth.homln_batch(count=40, seed=97, n_range=(150, 700), layer_range=(2, 5))
    gs = [H.Network(net.n, to_dev(net.layers)) for net in nets]
    masks = [(1 << net.n_layers) - 1 for net in nets]
    sel, osel = H.make_select(H.HOMLN_TOPK_PERCENT, 10.0), O.Select(O.TOPK_PERCENT, 10.0)
    H.homln_batch_analyse([g.h for g in gs], masks, True)
    for g, net, mask in zip(gs, nets, masks):
        ref = O.OracleHoMLN(net.n, net.layers)
        for i in range(net.n_layers):
            check_graph(*g.layer_closeness(i), ref.layer(i))
        check_graph(*g.and_closeness(mask), ref.and_graph(mask))
        assert g.compose(mask, 2, sel).cpu().numpy().tolist() == ref.compose(mask, 2, osel).tolist()
    for g in gs:
        g.close()


@pytest.mark.parametrize("max_tiles", [1, 3, 7])
def test_tiles_split_over_several_launches(H, max_tiles):
    """max_tiles_per_launch: the persistent BFS runs in several launches; results are identical."""
    net = synth.homln_small_overlap(2100, 6.0, 3, 0.4, 93)
    sel = [(H.make_select(H.HOMLN_TOPK_PERCENT, 10.0), O.Select(O.TOPK_PERCENT, 10.0))]
    full_parity(H, net, sel, tuning=dict(max_tiles_per_launch=max_tiles, words_per_node=2), heuristics=(2,))


def test_captured_graph_replays_the_batched_analysis(H):
    """homln_graph_capture: replays recompute every captured graph exactly; handles in use by a
    graph cannot be destroyed; after the graph is gone they can."""
    import torch
    nets = synth.homln_batch(count=5, seed=101, n_range=(300, 2500), layer_range=(2, 4))
    gs = [H.Network(net.n, to_dev(net.layers)) for net in nets]
    masks = [(1 << net.n_layers) - 1 for net in nets]
    graph = H.homln_graph_capture([g.h for g in gs], masks, True)
    refs = [O.OracleHoMLN(net.n, net.layers, threads=8) for net in nets]
    for rep in range(2):
        for g in gs:
            H.homln_invalidate(g.h)
        H.homln_graph_launch(graph)
        for g, net, mask, ref in zip(gs, nets, masks, refs):
            for i in range(net.n_layers):
                check_graph(*g.layer_closeness(i), ref.layer(i))
            check_graph(*g.and_closeness(mask), ref.and_graph(mask))
    with pytest.raises(H.HomlnError) as e:
        H.homln_destroy(gs[1].h)
    assert e.value.code == H.HOMLN_EBUSY
    H.homln_graph_destroy(graph)
    for g in gs:
        g.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("world", [1, 3, 5])
def test_sharded_partials_sum_to_the_analysis(H, world):
    """homln_shard_partials: the ranks' partial sums add up to the exact farness/reach (ranks run
    one after another on this GPU); imported into a fresh handle they give identical results."""
    import torch
    net = synth.homln_small_overlap(2700, 6.0, 3, 0.4, 57)
    ref = O.OracleHoMLN(net.n, net.layers, threads=8)
    sel, osel = H.make_select(H.HOMLN_TOPK_PERCENT, 10.0), O.Select(O.TOPK_PERCENT, 10.0)
    a = H.Network(net.n, to_dev(net.layers), tuning=dict(words_per_node=2))
    b = H.Network(net.n, to_dev(net.layers))
    for which, mask, want in [(0, 0, ref.layer(0)), (1, 0, ref.layer(1)), (2, 0, ref.layer(2)),
                              (-1, 7, ref.and_graph(7))]:
        F = torch.zeros(net.n, dtype=torch.int64, device="cuda")
        R = torch.zeros(net.n, dtype=torch.int32, device="cuda")
        for rank in range(world):
            f, r = a.shard_partials(which, mask, rank, world)
            F += f
            R += r
        assert np.array_equal(u64(F), want["F"]) and np.array_equal(R.cpu().numpy().astype(np.uint32), want["R"])
        H.homln_import_partials(b.h, which, mask, F, R)
    for i in range(3):
        check_graph(*b.layer_closeness(i), ref.layer(i))
    assert b.compose(7, 2, sel).cpu().numpy().tolist() == ref.compose(7, 2, osel).tolist()
    assert b.topk(-1, 7, sel).cpu().numpy().tolist() == ref.topk(-1, 7, osel).tolist()
    a.close()
    b.close()


def test_batch_closeness_on_an_explicit_stream(H):
    """homln_batch_closeness: every layer and the all-layer AND graph of each handle, ordered
    with the given stream."""
    import torch
    nets = synth.homln_batch(count=4, seed=131, n_range=(300, 1500), layer_range=(2, 4))
    gs = [H.Network(net.n, to_dev(net.layers)) for net in nets]
    side = torch.cuda.Stream()
    H.homln_batch_closeness([g.h for g in gs], side.cuda_stream)
    side.synchronize()
    for g, net in zip(gs, nets):
        ref = O.OracleHoMLN(net.n, net.layers)
        full = (1 << net.n_layers) - 1
        for i in range(net.n_layers):
            check_graph(*g.layer_closeness(i), ref.layer(i))
        check_graph(*g.and_closeness(full), ref.and_graph(full))
        g.close()
