"""Shape checks of the synthetic workload generators (no GPU)."""
import numpy as np

from oracle import oracle as O
from paper_2207_11662_gb300 import synth


def test_parmat_like_matches_table1_proportions():
    # Table 1, row 1: 50KV / 250KE split 70/30 -> 224,976 / 124,988 edges, AND 50,319
    net = synth.homln_parmat_like(50000, 250000, (0.7, 0.3), ("powerlaw", "normal"), seed=6001)
    keys = [O.edge_keys(net.n, s, d) for s, d in net.layers]
    sizes = [k.shape[0] for k in keys]
    inter = O.and_keys(net.n, keys).shape[0]
    assert abs(sizes[0] - 224976) / 224976 < 0.05
    assert abs(sizes[1] - 124988) / 124988 < 0.05
    assert 50000 <= inter < 52000
    # the power-law layer is much more skewed than the normal one
    deg = [np.diff(O.csr_from_keys(net.n, k)[0]) for k in keys]
    assert deg[0].max() > 3 * deg[1].max()


def test_generators_are_seeded():
    a = synth.homln_powerlaw(n=3000, seed=5)
    b = synth.homln_powerlaw(n=3000, seed=5)
    c = synth.homln_powerlaw(n=3000, seed=6)
    assert all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) for x, y in zip(a.layers, b.layers))
    assert not np.array_equal(a.layers[0][0], c.layers[0][0])
