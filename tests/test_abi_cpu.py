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


def test_noalloc_pointer_rule_without_gpu(tmp_path):
    """homln_accuracy_noalloc reads its id lists in kernels on the current device, so it accepts only
    managed memory and device memory of that device; another GPU's memory (no peer access) and host
    memory are refused with EINVAL. The rule is plain C++ over cudaPointerAttributes, checked here
    with faked attributes."""
    import shutil
    import subprocess
    gxx = shutil.which("g++")
    inc = "/usr/local/cuda/include"
    if not gxx or not os.path.exists(os.path.join(inc, "cuda_runtime_api.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    src = tmp_path / "rule.cpp"
    src.write_text(r'''
#include "devptr.h"
#include <cstdio>
static cudaPointerAttributes attr(cudaMemoryType t, int dev) {
    cudaPointerAttributes a{};
    a.type = t;
    a.device = dev;
    return a;
}
int main() {
    using homln::device_pointer_usable;
    int bad = 0;
    bad += !device_pointer_usable(attr(cudaMemoryTypeDevice, 0), 0);   // this GPU
    bad += !device_pointer_usable(attr(cudaMemoryTypeDevice, 3), 3);
    bad += device_pointer_usable(attr(cudaMemoryTypeDevice, 1), 0);    // another GPU
    bad += device_pointer_usable(attr(cudaMemoryTypeDevice, 0), 2);
    bad += !device_pointer_usable(attr(cudaMemoryTypeManaged, 1), 0);  // managed: any device
    bad += device_pointer_usable(attr(cudaMemoryTypeHost, 0), 0);      // pinned host
    bad += device_pointer_usable(attr(cudaMemoryTypeUnregistered, 0), 0);
    std::printf("%d\n", bad);
    return bad;
}
''')
    exe = tmp_path / "rule"
    subprocess.check_call([gxx, "-std=c++17", "-I", inc, "-I", os.path.join(ROOT, "paper_2207_11662_gb300", "csrc"),
                           str(src), "-o", str(exe)])
    assert subprocess.run([str(exe)], capture_output=True, text=True).stdout.strip() == "0"


def test_yield_flag_arguments_without_gpu(H):
    """The yield-flag calls reject NULL arguments on the host, before touching a GPU."""
    import ctypes
    assert H.lib.homln_yield_set(None, 1) == H.HOMLN_EINVAL
    assert H.lib.homln_yield_count(None, ctypes.byref(ctypes.c_int64())) == H.HOMLN_EINVAL
    assert H.lib.homln_set_yield(None, None) == H.HOMLN_EINVAL
    assert H.lib.homln_yield_create(None) == H.HOMLN_EINVAL
    assert H.lib.homln_yield_destroy(None) == H.HOMLN_OK


def test_concurrent_builds_take_turns(H):
    """A second process that builds while the build lock is held waits for it, then finds the
    library up to date; per-process temporary names keep two compilers off one file."""
    import fcntl
    import subprocess
    import sys
    import time
    from paper_2207_11662_gb300 import build_ext
    before = os.path.getmtime(build_ext.LIB)
    code = "import sys; sys.path.insert(0, %r); from paper_2207_11662_gb300 import build_ext; build_ext.build()" % ROOT
    with open(os.path.join(build_ext.BUILD, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        child = subprocess.Popen([sys.executable, "-c", code])
        time.sleep(2.0)
        assert child.poll() is None, "the second build did not wait for the lock"
    assert child.wait(timeout=300) == 0
    assert os.path.getmtime(build_ext.LIB) == before  # nothing was stale: no relink
    assert not [f for f in os.listdir(build_ext.BUILD) if ".tmp" in f]
