"""The oracle's C part under the undefined-behaviour sanitizer (host only): a build of
oracle/bfs.c with -fsanitize=undefined (no recovery) runs the BFS on random, disconnected and
degenerate graphs in a child process and must match the regular build."""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_bfs_under_ubsan(tmp_path):
    lib = str(tmp_path / "liboracle_bfs_ubsan.so")
    cmd = ["gcc", "-O1", "-g", "-fopenmp", "-fPIC", "-shared", "-fsanitize=undefined",
           "-fno-sanitize-recover=undefined", "-o", lib, os.path.join(ROOT, "oracle", "bfs.c")]
    if subprocess.run(cmd, capture_output=True).returncode != 0:
        pytest.skip("gcc without the undefined-behaviour sanitizer")
    code = textwrap.dedent(f"""
        import ctypes, sys
        import numpy as np
        sys.path.insert(0, {ROOT!r})
        from oracle import oracle as O
        from paper_2207_11662_gb300 import synth
        lib = ctypes.CDLL({lib!r})
        lib.oracle_bfs_farness.restype = ctypes.c_int
        lib.oracle_bfs_farness.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
        cases = [(1, synth.er_edges(1, 0, 1)), (2, synth.er_edges(2, 1, 2)), (50, synth.er_edges(50, 20, 3)),
                 (300, synth.er_edges(300, 900, 4)), (500, synth.chung_lu_edges(500, 2000, 5))]
        for n, (s, d) in cases:
            rp, col = O.simple_csr(n, s, d)
            F = np.zeros(n, np.uint64); R = np.zeros(n, np.uint32)
            rc = lib.oracle_bfs_farness(n, rp.ctypes.data, col.ctypes.data if col.size else None, 0, None,
                                        F.ctypes.data, R.ctypes.data, 4)
            assert rc == 0
            F2, R2 = O.farness_reach(n, rp, col)
            assert np.array_equal(F, F2) and np.array_equal(R, R2), n
        print("ok")
    """)
    env = dict(os.environ, UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
