"""CPU-side checks of the C-ABI: the library loads, exports every declared symbol,
and rejects bad arguments on the host before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_11662_gb300 import homln
    return homln


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "homln.h")).read()
    return sorted(set(re.findall(r"HOMLN_API\s+[\w\s\*]*?\b(homln_\w+)\s*\(", text)))


def test_header_symbols_exported(H):
    syms = declared_symbols()
    assert len(syms) >= 16
    lib = ctypes.CDLL(H.LIB_PATH)
    for s in syms:
        assert hasattr(lib, s), f"{s} declared in include/homln.h but not exported"
    assert sorted(H.EXPORTS) == syms


def test_version_and_errors_without_gpu(H):
    assert "sm_103a" in H.homln_version()
    n = 10
    s = np.array([0, 1], np.int32)
    d = np.array([1, 2], np.int32)
    with pytest.raises(H.HomlnError) as e:
        H.homln_create(0, [(s, d)])
    assert e.value.code == H.HOMLN_EINVAL
    with pytest.raises(H.HomlnError) as e:
        H.homln_create(H.MAX_NODES + 1, [(s, d)])
    assert e.value.code == H.HOMLN_EINVAL
    with pytest.raises(H.HomlnError) as e:
        H.homln_create(n, [])
    assert e.value.code == H.HOMLN_EINVAL
    with pytest.raises(H.HomlnError) as e:
        H.homln_create(n, [(s, d)] * 65)
    assert e.value.code == H.HOMLN_EINVAL
    # NULL handle everywhere
    sel = H.make_select()
    for fn, args in [(H.lib.homln_layer_closeness, (None, 0, None, None, None)),
                     (H.lib.homln_sync, (None,)),
                     (H.lib.homln_set_profiling, (None, 1, 0)),
                     (H.lib.homln_topk, (None, 0, 1, ctypes.byref(sel), None, ctypes.byref(ctypes.c_int32())))]:
        assert fn(*args) == H.HOMLN_EINVAL
    assert H.lib.homln_destroy(None) == H.HOMLN_OK


def test_create_without_device_reports_cuda_error(H):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    s = np.array([0, 1], np.int32)
    d = np.array([1, 2], np.int32)
    with pytest.raises(H.HomlnError) as e:
        H.homln_create(3, [(s, d)])
    assert e.value.code in (H.HOMLN_ECUDA, H.HOMLN_ENOMEM)
