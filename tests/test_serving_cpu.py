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
