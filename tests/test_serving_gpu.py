"""Serving: every request's result is the same alone and in the mix (continuous batching with
overlapping waves), and matches the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2207_11662_gb300 import synth

pytestmark = pytest.mark.gpu


def make_requests(serve, count=14, seed=5005):
    specs = synth.serving_requests(duration_s=1.0, rate=float(count), seed=seed, n_range=(400, 6000))[:count]
    reqs = []
    for i, sp in enumerate(specs):
        net = synth.build_request(sp["spec"], raw=True)
        reqs.append(serve.Request(i, net.n, net.layers, arrival=0.0))
    return reqs


def test_alone_equals_mix_and_oracle():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_11662_gb300 import serve
    torch.cuda.set_device(0)
    alone = serve.Server(workers=1, max_wave=1, keep_farness=True).run(make_requests(serve), realtime=False)
    srv = serve.Server(workers=3, max_wave=5, keep_farness=True)
    mix = srv.run(make_requests(serve), realtime=False)
    assert srv.waves >= 3 and not srv.errors
    for a, b in zip(alone, mix):
        assert a.status == b.status == 0, (a.error, b.error)
        assert np.array_equal(a.gt, b.gt) and np.array_equal(a.cc2, b.cc2)
        assert a.accuracy == b.accuracy
        for fa, fb in zip(a.farness, b.farness):
            assert np.array_equal(fa, fb)
    # a few requests against the oracle
    sel = O.Select(O.TOPK_PERCENT, 10.0)
    for r in mix[:4]:
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
