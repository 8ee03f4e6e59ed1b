"""Full-size parity: every output of the CUDA path at the benchmark's sizes against the oracle.

The oracle's full runs (every source of every graph; minutes of CPU time) are stored as sha256
digests in ``tests/golden/full_size_goldens.json``, written by
``tests/golden/make_full_size_goldens.py``, which calls only ``oracle/`` and the seeded input
generators. These tests rebuild the same inputs (their digest is checked first, so a change of the
generators is reported as such), run the CUDA path through the C-ABI at full size and compare,
bit for bit: farness, reach and closeness of every layer and of the AND graph (Section 4), the
ranked ground-truth and per-layer CC-node lists, the naive, CC1 and CC2 estimates (Sections 4,
5.1, 5.2) and their accuracy counts. Where it is cheap, a live oracle BFS from a seeded sample of
sources is checked as well.
"""
import json
import os
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_2207_11662_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN_DIR = os.path.join(os.path.dirname(__file__), "golden")
sys.path.insert(0, GOLDEN_DIR)
import make_full_size_goldens as G  # noqa: E402  (test infrastructure: input specs and digest format)

REL_TOL = 1e-12


@pytest.fixture(scope="module")
def H():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    torch.cuda.set_device(0)
    from paper_2207_11662_gb300 import homln
    return homln


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(GOLDEN_DIR, "full_size_goldens.json")) as f:
        return json.load(f)


def to_dev(layers):
    import torch
    return [(torch.from_numpy(np.ascontiguousarray(s)).cuda(), torch.from_numpy(np.ascontiguousarray(d)).cuda())
            for s, d in layers]


def sha(t, dtype) -> str:
    return G.digest(t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t), dtype)


def check_inputs(net, ent):
    assert G.inputs_digest(net.layers) == ent["inputs"], \
        "the seeded generators produced other inputs than the goldens were written for"


def check_graph(F, R, cc, want, what):
    got_F = F.cpu().numpy().astype(np.uint64)
    assert int(got_F.sum(dtype=np.uint64)) == want["sum_F"], f"{what}: sum of farness"
    assert [int(x) for x in got_F[:4]] == want["F_head"], f"{what}: first farness values"
    assert sha(got_F, np.uint64) == want["F"], f"{what}: farness"
    assert sha(R.cpu().numpy().astype(np.uint32), np.uint32) == want["R"], f"{what}: reach"
    assert sha(cc, np.float64) == want["cc"], f"{what}: closeness"


def check_list(ids, want, what):
    a = ids.cpu().numpy().astype(np.int32)
    assert a.shape[0] == want["n"], f"{what}: length {a.shape[0]} != {want['n']}"
    assert [int(x) for x in a[:4]] == want["head"], f"{what}: first ids"
    assert sha(a, np.int32) == want["sha"], f"{what}: ids"


def check_network(H, g, L, ent, sels, heuristics=("naive", "cc1", "cc2"), tag=""):
    mask = (1 << L) - 1
    for i in range(L):
        check_graph(*g.layer_closeness(i), ent["graphs"][i], f"{tag} layer {i}")
    check_graph(*g.and_closeness(mask), ent["graphs"][L], f"{tag} AND graph")
    hmap = {"naive": H.HOMLN_NAIVE, "cc1": H.HOMLN_CC1, "cc2": H.HOMLN_CC2}
    for name, sel in sels.items():
        want = ent["select"][name]
        gt = g.topk(-1, mask, sel)
        check_list(gt, want["gt"], f"{tag} {name} ground truth")
        for i in range(L):
            check_list(g.topk(i, mask, sel), want["layers"][i], f"{tag} {name} layer {i} CC nodes")
        for heur in heuristics:
            est = g.compose(mask, hmap[heur], sel)
            check_list(est, want[heur], f"{tag} {name} {heur}")
            acc = g.accuracy(est, gt)
            assert (acc["tp"], acc["fp"], acc["fn"]) == (want[heur]["tp"], want[heur]["fp"], want[heur]["fn"])
            tp, fp, fn = acc["tp"], acc["fp"], acc["fn"]
            jac = tp / (tp + fp + fn) if tp + fp + fn else 1.0
            assert acc["jaccard"] == pytest.approx(jac, rel=REL_TOL, abs=0)


def live_sample(g, net, count, seed):
    """Oracle BFS from a seeded sample of sources on every graph, against the CUDA path's values there."""
    n, L = net.n, net.n_layers
    keys = [O.edge_keys(n, s, d) for s, d in net.layers]
    graphs = [O.csr_from_keys(n, k) for k in keys] + [O.csr_from_keys(n, O.and_keys(n, keys))]
    outs = [g.layer_closeness(i) for i in range(L)] + [g.and_closeness((1 << L) - 1)]
    sample = np.sort(np.random.default_rng(seed).choice(n, min(count, n), replace=False)).astype(np.int32)
    for (rp, col), (F, R, cc) in zip(graphs, outs):
        Fs, Rs = O.farness_reach(n, rp, col, sources=sample, threads=os.cpu_count() or 1)
        assert np.array_equal(F.cpu().numpy().astype(np.uint64)[sample], Fs)
        assert np.array_equal(R.cpu().numpy().astype(np.uint32)[sample], Rs)
        assert np.array_equal(cc.cpu().numpy()[sample], O.wf_closeness(n, Fs, Rs))


def sels_of(H):
    return {"top10": H.make_select(H.HOMLN_TOPK_PERCENT, 10.0, cc1_overlap=0.5),
            "ge_mean": H.make_select(H.HOMLN_GE_MEAN, cc1_overlap=0.5)}


@pytest.mark.parametrize("tuning", [None, dict(words_per_node=16, teams=8, push_alpha=4),
                                    dict(words_per_node=8, teams=32, push_alpha=16, team_mix=1)])
def test_powerlaw_full_size_matches_oracle(H, golden, tuning):
    """4 Chung-Lu layers on 50,000 nodes: every output against the oracle's full run, in the library's
    default launch configuration, in the setting the benchmark's autotuner picks (32 teams, blocks of an
    SM in different teams) and in another (wider tiles, fewer teams, another direction switch);
    F/R/closeness also against a live oracle BFS from 2,000 seeded sources."""
    net = synth.homln_powerlaw()
    ent = golden["powerlaw50k"]
    check_inputs(net, ent)
    g = H.Network(net.n, to_dev(net.layers), tuning=tuning)
    g.analyse((1 << net.n_layers) - 1, True)
    check_network(H, g, net.n_layers, ent, sels_of(H), tag="powerlaw50k")
    if tuning is None:
        live_sample(g, net, 2000, 2001)
    g.close()


@pytest.mark.parametrize("tuning", [None, dict(words_per_node=16, teams=16, push_alpha=4, team_mix=1),
                                    dict(words_per_node=4, teams=32, push_alpha=64)])
def test_large_ba_full_size_matches_oracle(H, golden, tuning):
    """4 Barabasi-Albert layers on 200,000 nodes (~50% shared edges): every output against the oracle's
    full run (all 200,000 sources of all 5 graphs), in the library's defaults, in the setting the
    benchmark's autotuner picks (1,024 sources per tile, alpha 4, blocks of an SM in different teams)
    and in a third; F/R/closeness also against a live oracle BFS from 2,000 seeded sources."""
    net = synth.homln_ba_large()
    ent = golden["ba200k"]
    check_inputs(net, ent)
    g = H.Network(net.n, to_dev(net.layers), tuning=tuning)
    g.analyse((1 << net.n_layers) - 1, True)
    check_network(H, g, net.n_layers, ent, sels_of(H), tag="ba200k")
    if tuning is None:
        live_sample(g, net, 2000, 4001)
    g.close()


def sampled_oracle(n, graphs, outs, count, seed):
    """Live oracle BFS from a seeded sample of vertices on each (rowptr, col) graph: farness, reach
    and closeness there against the CUDA path's (F, R, cc)."""
    sample = np.sort(np.random.default_rng(seed).choice(n, count, replace=False)).astype(np.int32)
    for (rp, col), (F, R, cc) in zip(graphs, outs):
        Fs, Rs = O.farness_reach(n, rp, col, sources=sample, threads=os.cpu_count() or 1)
        assert np.array_equal(F.cpu().numpy().astype(np.uint64)[sample], Fs)
        assert np.array_equal(R.cpu().numpy().astype(np.uint32)[sample], Rs)
        assert np.array_equal(cc.cpu().numpy()[sample], O.wf_closeness(n, Fs, Rs))


def test_widened_paths_at_full_size_match_sampled_oracle(H, golden):
    """The benchmark's largest network (4 BA layers, n = 200,000; the benchmark times these paths on
    the 50,000-node power-law network) through the paths beyond the AND ground truth:
    - OR graphs (edges in at least one layer) of layers {0,1,2,3} and {0,1,2};
    - the layer-subset sweep (all 11 subsets of two or more layers in one launch): two of its AND
      graphs against the oracle, and every subset's counts equal to the individual selection,
      composition and accuracy calls on the sweep's results;
    - the directed variant (each edge a random-direction arc, plus the reverse of 25% of them):
      in-closeness of the 4 layers and of their AND graph.
    Farness, reach and closeness at 1,000 seeded vertices per graph against live oracle BFS."""
    net = synth.homln_ba_large()
    check_inputs(net, golden["ba200k"])
    n, L = net.n, net.n_layers
    keys = [O.edge_keys(n, a, b) for a, b in net.layers]
    g = H.Network(n, to_dev(net.layers))
    sel = H.make_select(H.HOMLN_TOPK_PERCENT, 10.0)
    res = H.homln_subset_sweep(g.h, H.HOMLN_CC2, sel, 2)
    assert [r["mask"] for r in res] == [m for m in range(1, 16) if bin(m).count("1") >= 2]
    masks = (3, 10)
    sampled_oracle(n, [O.csr_from_keys(n, O.and_keys(n, [keys[i] for i in range(L) if m >> i & 1])) for m in masks],
                   [g.and_closeness(m) for m in masks], 1000, 5101)
    for r in res:
        gt = g.topk(-1, r["mask"], sel)
        est = g.compose(r["mask"], H.HOMLN_CC2, sel)
        acc = g.accuracy(est, gt)
        assert (r["truth_count"], r["estimate_count"]) == (gt.shape[0], est.shape[0])
        assert (r["tp"], r["fp"], r["fn"]) == (acc["tp"], acc["fp"], acc["fn"])
    or_masks = (15, 7)
    sampled_oracle(n, [O.csr_from_keys(n, O.or_keys(n, [keys[i] for i in range(L) if m >> i & 1])) for m in or_masks],
                   [g.or_closeness(m) for m in or_masks], 1000, 5102)
    g.close()
    arcs = [synth.with_reciprocal(e, 0.25, 7001 + i) for i, e in enumerate(net.layers)]
    gd = H.Network(n, to_dev(arcs), directed=True)
    akeys = [O.arc_keys(n, a, b) for a, b in arcs]
    graphs = [O.arc_csr(n, k, reverse=True) for k in akeys] + [O.arc_csr(n, O.and_keys(n, akeys), reverse=True)]
    sampled_oracle(n, graphs, [gd.layer_closeness(i) for i in range(L)] + [gd.and_closeness((1 << L) - 1)], 1000, 5103)
    gd.close()


def test_batch_config_full_size_matches_oracle(H, golden):
    """64 HoMLNs (2-8 ER/BA layers, 500-20,000 nodes) in one persistent launch with several teams: every
    graph's farness/reach/closeness and every network's top-10% ground truth, per-layer CC nodes,
    naive/CC1/CC2 estimates and accuracy counts against the oracle's full runs."""
    nets = synth.homln_batch(64, 3001)
    ents = golden["batch64"]["networks"]
    assert len(ents) == len(nets)
    gs = [H.Network(net.n, to_dev(net.layers)) for net in nets]
    H.homln_set_tuning(gs[0].h, teams=16)
    masks = [(1 << net.n_layers) - 1 for net in nets]
    H.homln_batch_analyse([g.h for g in gs], masks, True)
    sel = {"top10": H.make_select(H.HOMLN_TOPK_PERCENT, 10.0, cc1_overlap=0.5)}
    for k, (g, net, ent) in enumerate(zip(gs, nets, ents)):
        check_inputs(net, ent)
        check_network(H, g, net.n_layers, ent, sel, tag=f"network {k}")
        g.close()


def test_paper_shaped_network_matches_oracle(H, golden):
    """A two-layer network shaped like the paper's synthetic sets (Section 6, Table 1: R-MAT power-law
    and normal layers splitting 250,000 edges 70/30 over a shared 50,000-edge backbone), CC nodes at
    or above the average closeness (Section 4): ground truth, naive, CC1 at overlap thresholds 0.1,
    0.25 and 0.5, CC2 and the accuracy counts against the oracle's full run."""
    net = G.parmat_net()
    ent = golden["parmat50k"]
    check_inputs(net, ent)
    g = H.Network(net.n, to_dev(net.layers))
    sels = {f"ge_mean_theta{t}": H.make_select(H.HOMLN_GE_MEAN, cc1_overlap=t) for t in G.PARMAT_THETAS}
    check_network(H, g, net.n_layers, ent, sels, tag="parmat50k")
    g.close()


def test_yield_flag_stops_and_resumes_the_bfs(H, golden):
    """Preemption for serving: with the yield flag raised the persistent BFS hands out no tile and its
    launch ends; once lowered, the remaining tiles run in a new launch. Raised before the analysis and
    toggled every few milliseconds during it, the flag must cost nothing in correctness: every output
    equals the oracle's full run, and the stops are counted."""
    import threading
    import time
    net = synth.homln_powerlaw()
    ent = golden["powerlaw50k"]
    check_inputs(net, ent)
    y = H.homln_yield_create()
    g = H.Network(net.n, to_dev(net.layers), tuning=dict(words_per_node=4))  # 4 x 196 + 196 tiles
    try:
        H.homln_set_yield(g.h, y)
        H.homln_yield_set(y, True)  # raised before the analysis starts: the first launch stops at once
        done = threading.Event()

        def toggle():
            time.sleep(0.2)
            H.homln_yield_set(y, False)
            while not done.is_set():
                time.sleep(0.003)
                H.homln_yield_set(y, True)
                time.sleep(0.001)
                H.homln_yield_set(y, False)

        t = threading.Thread(target=toggle)
        t.start()
        try:
            g.analyse((1 << net.n_layers) - 1, True)
        finally:
            done.set()
            t.join()
        H.homln_yield_set(y, False)
        assert H.homln_yield_count(y) >= 1
        check_network(H, g, net.n_layers, ent, {"top10": sels_of(H)["top10"]}, heuristics=("cc2",), tag="yield")
        with pytest.raises(H.HomlnError) as err:  # a watching handle cannot be captured
            H.homln_graph_capture([g.h], [(1 << net.n_layers) - 1], True)
        assert err.value.code == H.HOMLN_EINVAL
        with pytest.raises(H.HomlnError) as err:  # nor can the flag be freed while watched
            H.homln_yield_destroy(y)
        assert err.value.code == H.HOMLN_EBUSY
        H.homln_set_yield(g.h, None)
        h2 = H.homln_create(net.n, to_dev(net.layers[:1]))  # destroying a watching handle ends its watch
        H.homln_set_yield(h2, y)
        H.homln_destroy(h2)
    finally:
        g.close()
        H.homln_yield_destroy(y)
