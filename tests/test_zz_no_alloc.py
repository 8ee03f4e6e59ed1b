"""homln_accuracy_noalloc: the accuracy entry point for callers that cannot allocate
device memory (another allocator owns the GPU, or the caller's loop must not enter an
allocator). It keeps its scratch in a static device array, so it must give the same
answers as the allocating homln_accuracy, call after call, with the array reused.

This file is collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test. It passes alone in a fresh process too.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12


def test_noalloc_accuracy_matches_allocating_entry_point():
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
                 (np.zeros(0, np.int64), rng.choice(n, 50, replace=False))]
        for pred, truth in cases:
            p = torch.from_numpy(pred.astype(np.int32)).cuda()
            t = torch.from_numpy(truth.astype(np.int32)).cuda()
            want = H.homln_accuracy(h, p, p.numel(), t, t.numel())
            got = H.homln_accuracy_noalloc(n, p, p.numel(), t, t.numel(),
                                           stream=torch.cuda.current_stream().cuda_stream)
            for k in ("tp", "fp", "fn"):
                assert got[k] == want[k]
            for k in ("jaccard", "precision", "recall", "f1"):
                assert got[k] == pytest.approx(want[k], rel=REL_TOL, abs=0)
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
