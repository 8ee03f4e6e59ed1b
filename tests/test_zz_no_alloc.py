"""homln_accuracy_noalloc: the accuracy entry point for callers that cannot allocate
device memory (another allocator owns the GPU, or the caller's loop must not enter an
allocator). It keeps its scratch in a static device array, so it must give the oracle's
answers call after call, with the array reused, and must not change the device's free
memory or torch's allocated bytes.

This file is collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test. It passes alone in a fresh process too.
"""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12


def check(got, want):
    for k in ("tp", "fp", "fn"):
        assert got[k] == want[k], k
    for k in ("jaccard", "precision", "recall", "f1"):
        assert got[k] == pytest.approx(want[k], rel=REL_TOL, abs=0), k


def test_noalloc_accuracy_matches_oracle_and_allocates_nothing():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_11662_gb300 import homln as H

    torch.cuda.set_device(0)
    n = 100003
    rng = np.random.default_rng(11)
    # a handle over the same node set, for the allocating entry point
    e = (np.array([0], np.int32), np.array([1], np.int32))
    h = H.homln_create(n, [e])
    try:
        cases = [(rng.choice(n, 9000, replace=False), rng.choice(n, 10000, replace=False)),
                 (rng.choice(n, 300, replace=True), rng.choice(n, 7, replace=False)),  # fewer bits than before
                 (np.zeros(0, np.int64), rng.choice(n, 50, replace=False)),
                 (np.arange(n - 5, n), np.arange(n - 5, n))]  # the last ids of the node set
        dev_cases = [(torch.from_numpy(p.astype(np.int32)).cuda(), torch.from_numpy(t.astype(np.int32)).cuda())
                     for p, t in cases]
        torch.cuda.synchronize()
        p, t = dev_cases[0]
        H.homln_accuracy_noalloc(n, p, p.numel(), t, t.numel())  # first call on the device: symbol lookup
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        alloc0 = torch.cuda.memory_allocated()
        for rep in range(2):  # two calls in a row on every case: the shared array keeps no stale bits
            for (pred, truth), (p, t) in zip(cases, dev_cases):
                want = O.accuracy(pred, truth)
                got = H.homln_accuracy_noalloc(n, p, p.numel(), t, t.numel(),
                                               stream=torch.cuda.current_stream().cuda_stream)
                check(got, want)
                if rep == 0:  # the allocating entry point gives the same
                    check(H.homln_accuracy(h, p, p.numel(), t, t.numel()), want)
                # the default stream argument is torch's current stream
                check(H.homln_accuracy_noalloc(n, p, p.numel(), t, t.numel()), want)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == alloc0
        # homln_accuracy allocates from the library's own pool, which stays mapped; repeat only the
        # allocation-free calls for the free-memory check
        free1 = torch.cuda.mem_get_info()[0]
        for (pred, truth), (p, t) in zip(cases, dev_cases):
            H.homln_accuracy_noalloc(n, p, p.numel(), t, t.numel())
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free1
        assert free1 <= free0
        # sizes beyond the static array and host pointers are rejected, and the array still works after
        p = torch.zeros(3, dtype=torch.int32, device="cuda")
        with pytest.raises(H.HomlnError) as err:
            H.homln_accuracy_noalloc((1 << 20) + 1, p, 3, p, 3)
        assert err.value.code == H.HOMLN_EINVAL
        with pytest.raises(H.HomlnError) as err:
            H.homln_accuracy_noalloc(n, np.zeros(3, np.int32), 3, p, 3)
        assert err.value.code == H.HOMLN_EINVAL
        bad = torch.tensor([0, n], dtype=torch.int32, device="cuda")
        with pytest.raises(H.HomlnError) as err:
            H.homln_accuracy_noalloc(n, bad, 2, p, 3)
        assert err.value.code == H.HOMLN_EINVAL
        q = torch.tensor([1, 2, 3], dtype=torch.int32, device="cuda")
        got = H.homln_accuracy_noalloc(n, q, 3, q, 3)
        assert (got["tp"], got["fp"], got["fn"], got["jaccard"]) == (3, 0, 0, 1.0)
    finally:
        H.homln_destroy(h)
