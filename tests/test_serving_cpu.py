"""Admission control of the serving loop (host logic, no GPU)."""
import threading

import pytest


def _mods():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_11662_gb300 import serve
    return serve


def test_fifo_admission_under_budget():
    serve = _mods()
    a = serve.Admission(100)
    reqs = [serve.Request(i, 10, []) for i in range(5)]
    for r, need in zip(reqs, [40, 40, 40, 10, 10]):
        assert a.submit(r, need)
    got = a.take(8, timeout=0.01)
    assert [r.rid for r, _ in got] == [0, 1]  # the third would exceed the budget; FIFO order is kept
    assert a.take(8, timeout=0.01) == []
    a.release(40)  # in use: 40; requests 2, 3 and 4 (40 + 10 + 10) now fit exactly
    assert [r.rid for r, _ in a.take(1, timeout=0.01)] == [2]  # max_items respected
    assert [r.rid for r, _ in a.take(8, timeout=0.01)] == [3, 4]
    assert a.in_use == 100
    a.close()
    assert a.take(8, timeout=0.01) is None


def test_never_fitting_request_is_rejected():
    serve = _mods()
    a = serve.Admission(100)
    assert not a.submit(serve.Request(0, 10, []), 101)
    assert len(a.waiting) == 0


def test_waiters_wake_on_release():
    serve = _mods()
    a = serve.Admission(50)
    a.submit(serve.Request(0, 10, []), 50)
    a.submit(serve.Request(1, 10, []), 50)
    first = a.take(4, timeout=0.01)
    out = []
    t = threading.Thread(target=lambda: out.append(a.take(4, timeout=5.0)))
    t.start()
    a.release(first[0][1])
    t.join(timeout=5.0)
    assert [r.rid for r, _ in out[0]] == [1]


def test_footprint_grows_with_size():
    serve = _mods()
    assert serve.footprint_bytes(1000, [4000, 4000]) < serve.footprint_bytes(100000, [400000, 400000, 400000])


def test_footprint_covers_the_bfs_state_of_the_default_teams():
    """The estimate holds the BFS state the library allocates by default: per team 2 snapshots of
    n x 8 words and 3 bytes per node, with at least 16 teams (no more than tiles), up to about
    240 MB of state in all."""
    serve = _mods()
    per_node = 2 * 8 * 8 + 3
    for n, layers in ((50000, 4), (200000, 2), (20000, 3), (3000, 2)):
        tiles = (layers + 1) * -(-n // 512)
        teams = min(tiles, max(16, int(2.4e8 // (2 * 8 * 8 * n))))
        assert serve.footprint_bytes(n, [5 * n] * layers) >= teams * per_node * n
    # 37 teams at n = 50,000 (the power-law workload), 16 at n = 200,000
    assert serve.footprint_bytes(50000, [250000] * 4) >= 37 * per_node * 50000
    assert serve.footprint_bytes(200000, [800000] * 4) >= 16 * per_node * 200000


def test_size_classes_keep_fifo_order_within_a_class():
    serve = _mods()
    a = serve.Admission(1000)
    small = [serve.Request(i, 10, []) for i in range(3)]
    big = [serve.Request(10 + i, 10, []) for i in range(2)]
    for r in (small[0], big[0], small[1], big[1], small[2]):
        a.submit(r, 10, serve.BIG if r.rid >= 10 else serve.SMALL)
    assert [r.rid for r, _ in a.take(8, 0.01, classes=(serve.SMALL,))] == [0, 1, 2]
    assert a.take(8, 0.01, classes=(serve.SMALL,)) == []
    assert [r.rid for r, _ in a.take(8, 0.01, classes=(serve.BIG, serve.SMALL))] == [10, 11]
    a.close()
    assert a.take(8, 0.01, classes=(serve.SMALL,)) is None


def test_work_estimate_splits_the_classes():
    serve = _mods()
    assert serve.work_estimate(1000, [4000, 4000]) < 2e10 < serve.work_estimate(100000, [500000] * 4)


def test_single_worker_takes_the_oldest_class_first():
    serve = _mods()
    a = serve.Admission(1000)
    reqs = [serve.Request(i, 10, []) for i in range(3)]
    for r, t, cls in zip(reqs, (0.3, 0.1, 0.2), (serve.SMALL, serve.BIG, serve.SMALL)):
        r.t_submit = t
        a.submit(r, 10, cls)
    assert [r.rid for r, _ in a.take(8, 0.01)] == [1]  # the big request arrived first
    assert [r.rid for r, _ in a.take(8, 0.01)] == [0, 2]


def test_gc_frozen_hides_old_objects_from_the_collector_and_restores():
    """Inside the block a full collection walks only what the block created, and cyclic garbage
    made inside is still collected; on exit every frozen object is back in the collector's view."""
    import gc
    serve = _mods()
    before = len(gc.get_objects())
    with serve.gc_frozen():
        assert gc.get_freeze_count() >= before * 0.9
        assert len(gc.get_objects()) < before * 0.1
        cycle = []
        cycle.append(cycle)
        del cycle
        assert gc.collect() >= 1
    assert gc.get_freeze_count() == 0
    assert len(gc.get_objects()) >= before * 0.9
    gc.freeze()
    try:
        with serve.gc_frozen(False):
            assert gc.get_freeze_count() > 0  # disabled: the collector's state is left alone
    finally:
        gc.unfreeze()
