"""Serving: every request's result is the same alone and in the mix (continuous batching with
overlapping waves), and matches the oracle."""
import json
import os
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_2207_11662_gb300 import synth

pytestmark = pytest.mark.gpu


GOLDEN_DIR = os.path.join(os.path.dirname(__file__), "golden")


def make_requests(serve, count=14, seed=5005, n_range=(400, 6000)):
    specs = synth.serving_requests(duration_s=1.0, rate=float(count), seed=seed, n_range=n_range)[:count]
    reqs = []
    for i, sp in enumerate(specs):
        net = synth.build_request(sp["spec"], raw=True)
        reqs.append(serve.Request(i, net.n, net.layers, arrival=0.0))
    return reqs


def golden_requests(serve):
    """The first 18 requests of the seeded serving stream (n log-uniform in [1e3, 1e5], 2-6 layers; the
    largest has 98,311 nodes), with the oracle's full results written by
    tests/golden/make_full_size_goldens.py."""
    sys.path.insert(0, GOLDEN_DIR)
    import make_full_size_goldens as G
    with open(os.path.join(GOLDEN_DIR, "full_size_goldens.json")) as f:
        ents = json.load(f)["serving"]["requests"]
    nets = G.serving_nets()
    assert len(nets) == len(ents)
    for net, ent in zip(nets, ents):
        assert G.inputs_digest(net.layers) == ent["inputs"], "generator drift: other inputs than the goldens'"
    return G, ents, lambda: [serve.Request(i, net.n, net.layers, arrival=0.0) for i, net in enumerate(nets)]


def test_alone_equals_mix_and_oracle():
    """Each request served alone (one at a time) and in a mix with overlapping work on the device gives
    the same farness of every graph, ground truth, CC2 estimate and accuracy, equal to the oracle's."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_11662_gb300 import serve
    torch.cuda.set_device(0)
    G, ents, make = golden_requests(serve)
    alone = serve.Server(workers=1, max_wave=1, keep_farness=True).run(make(), realtime=False)
    srv = serve.Server(keep_farness=True, max_wave=5)  # the default: small waves preempt big ones
    mix = srv.run(make(), realtime=False)
    assert srv.waves >= 3 and not srv.errors
    for a, b, ent in zip(alone, mix, ents):
        assert a.status == b.status == 0, (a.error, b.error)
        assert np.array_equal(a.gt, b.gt) and np.array_equal(a.cc2, b.cc2)
        assert a.accuracy == b.accuracy
        for fa, fb in zip(a.farness, b.farness):
            assert np.array_equal(fa, fb)
        # against the oracle's full run of this request
        for f, want in zip(b.farness, ent["graphs"]):
            assert G.digest(f, np.uint64) == want["F"]
        sel = ent["select"]["top10"]
        assert G.digest(b.gt, np.int32) == sel["gt"]["sha"] and b.gt.shape[0] == sel["gt"]["n"]
        assert G.digest(b.cc2, np.int32) == sel["cc2"]["sha"] and b.cc2.shape[0] == sel["cc2"]["n"]
        assert (b.accuracy["tp"], b.accuracy["fp"], b.accuracy["fn"]) == \
            (sel["cc2"]["tp"], sel["cc2"]["fp"], sel["cc2"]["fn"])


def test_small_requests_in_a_mix_match_the_oracle():
    """Many small requests (400-6,000 nodes) through several overlapping waves, against the live oracle."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_11662_gb300 import serve
    torch.cuda.set_device(0)
    srv = serve.Server(workers=3, max_wave=5, keep_farness=True)
    mix = srv.run(make_requests(serve), realtime=False)
    assert srv.waves >= 3 and not srv.errors
    sel = O.Select(O.TOPK_PERCENT, 10.0)
    for r in mix:
        ref = O.OracleHoMLN(r.n, r.layers, threads=8)
        mask = (1 << len(r.layers)) - 1
        for i in range(len(r.layers)):
            assert np.array_equal(r.farness[i], ref.layer(i)["F"])
        assert np.array_equal(r.farness[-1], ref.and_graph(mask)["F"])
        assert r.gt.tolist() == ref.topk(-1, mask, sel).tolist()
        assert r.cc2.tolist() == ref.compose(mask, O.CC2, sel).tolist()


def test_memory_budget_rejects_and_serializes():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_11662_gb300 import serve
    reqs = make_requests(serve, count=6, seed=5006)
    need = max(serve.footprint_bytes(r.n, [s.shape[0] for s, _ in r.layers]) for r in reqs)
    srv = serve.Server(workers=2, max_wave=4, mem_budget_bytes=need)  # room for about one request at a time
    done = srv.run(reqs, realtime=False)
    assert all(r.status == 0 for r in done)
    tiny = serve.Server(workers=1, mem_budget_bytes=1024)
    done = tiny.run(make_requests(serve, count=2, seed=5007), realtime=False)
    assert all(r.status == tiny_status for r, tiny_status in zip(done, [2, 2]))
