"""Write ``full_size_goldens.json``: the oracle's results on the full-size workloads.

TEST INFRASTRUCTURE. This script calls only ``oracle/`` (the plain CPU
implementation of the paper's definitions) and the seeded input generators of
``paper_2207_11662_gb300.synth`` (edge lists only, none of the method's
arithmetic). No value in the output comes from the CUDA path.

Workloads (all exact, every source, no sampling):

* ``powerlaw50k``: 4 Chung-Lu layers, n = 50,000, average degree 10, shared
  edge pool (seed 2001);
* ``ba200k``: 4 Barabasi-Albert layers (m = 4), n = 200,000, half of one base
  graph shared (seed 4001);
* ``batch64``: 64 HoMLNs with 2-8 ER/BA layers on 500-20,000 nodes (seed 3001);
* ``serving``: the first 18 requests of a seeded Poisson stream with n
  log-uniform in [1e3, 1e5] and 2-6 ER or Chung-Lu layers (seed 5005);
* ``parmat50k``: a two-layer network shaped like the paper's synthetic sets
  (Section 6, Table 1: an R-MAT power-law layer and an R-MAT normal layer
  splitting 250,000 edges 70/30 over a shared n-edge backbone), selected with
  the at-or-above-average rule (Section 4), CC1 at several overlap thresholds.

For every analysed graph (each layer and the AND aggregate of all layers;
Section 4) the file keeps sha256 digests of farness F (uint64), reach R
(uint32) and closeness (float64, one correctly rounded division per vertex),
all little-endian, plus their sums and the first values for diagnosis. For the
selections it keeps digests and lengths of the ranked ground-truth list, each
layer's ranked list, the naive, CC1 and CC2 estimates (Sections 4, 5.1, 5.2)
and their accuracy counts against the ground truth. The digest of the input
edge lists is stored too, so a change of the generators shows up as such.

Run: ``python tests/golden/make_full_size_goldens.py [workload ...]`` (all by
default; about 40 minutes on 8 cores). Existing entries of workloads not named
are kept.
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2207_11662_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "full_size_goldens.json")
THREADS = os.cpu_count() or 1

# one fixed description of each workload; the GPU test rebuilds the inputs from the same calls
SERVING_SPEC = dict(duration_s=60.0, rate=50.0, seed=5005, n_range=(1000, 100000), count=18)
PARMAT_SPEC = dict(n=50000, m=250000, split=(0.7, 0.3), kinds=("powerlaw", "normal"), seed=6002)
PARMAT_THETAS = (0.1, 0.25, 0.5)


def digest(a, dtype) -> str:
    return hashlib.sha256(np.ascontiguousarray(np.asarray(a).astype(np.dtype(dtype).newbyteorder("<"))).tobytes()).hexdigest()


def inputs_digest(layers) -> str:
    h = hashlib.sha256()
    for s, d in layers:
        h.update(np.ascontiguousarray(s, "<i4").tobytes())
        h.update(np.ascontiguousarray(d, "<i4").tobytes())
    return h.hexdigest()


def graph_entry(g: dict) -> dict:
    return {"F": digest(g["F"], np.uint64), "R": digest(g["R"], np.uint32), "cc": digest(g["cc"], np.float64),
            "sum_F": int(np.sum(g["F"].astype(np.uint64), dtype=np.uint64)), "sum_R": int(np.sum(g["R"], dtype=np.uint64)),
            "F_head": [int(x) for x in g["F"][:4]], "edges": int(g["keys"].shape[0])}


def list_entry(ids) -> dict:
    ids = np.asarray(ids, np.int32)
    return {"n": int(ids.shape[0]), "sha": digest(ids, np.int32), "head": [int(x) for x in ids[:4]]}


def selection_entry(ref: O.OracleHoMLN, L: int, sel: O.Select, heuristics=(O.NAIVE, O.CC1, O.CC2)) -> dict:
    mask = (1 << L) - 1
    gt = ref.topk(-1, mask, sel)
    out = {"gt": list_entry(gt), "layers": [list_entry(ref.topk(i, mask, sel)) for i in range(L)]}
    names = {O.NAIVE: "naive", O.CC1: "cc1", O.CC2: "cc2"}
    for heur in heuristics:
        est = ref.compose(mask, heur, sel)
        acc = O.accuracy(est, gt)
        out[names[heur]] = dict(list_entry(est), tp=acc["tp"], fp=acc["fp"], fn=acc["fn"])
    return out


def network_entry(net, sels: dict, heuristics=(O.NAIVE, O.CC1, O.CC2)) -> dict:
    L = net.n_layers
    ref = O.OracleHoMLN(net.n, net.layers, threads=THREADS)
    ent = {"n": net.n, "layers": L, "inputs": inputs_digest(net.layers),
           "graphs": [graph_entry(ref.layer(i)) for i in range(L)] + [graph_entry(ref.and_graph((1 << L) - 1))]}
    ent["select"] = {name: selection_entry(ref, L, sel, heuristics) for name, sel in sels.items()}
    return ent


TOP10 = O.Select(O.TOPK_PERCENT, 10.0, cc1_overlap=0.5)
GEMEAN = O.Select(O.GE_MEAN, cc1_overlap=0.5)


def serving_nets():
    sp = dict(SERVING_SPEC)
    count = sp.pop("count")
    specs = synth.serving_requests(**sp)[:count]
    return [synth.build_request(r["spec"], raw=True) for r in specs]


def parmat_net():
    p = PARMAT_SPEC
    return synth.homln_parmat_like(p["n"], p["m"], p["split"], p["kinds"], p["seed"])


def make(name: str) -> dict:
    if name == "powerlaw50k":
        return network_entry(synth.homln_powerlaw(), {"top10": TOP10, "ge_mean": GEMEAN})
    if name == "ba200k":
        return network_entry(synth.homln_ba_large(), {"top10": TOP10, "ge_mean": GEMEAN})
    if name == "batch64":
        return {"networks": [network_entry(net, {"top10": TOP10}) for net in synth.homln_batch(64, 3001)]}
    if name == "serving":
        return {"spec": SERVING_SPEC,
                "requests": [network_entry(net, {"top10": TOP10}, (O.CC2,)) for net in serving_nets()]}
    if name == "parmat50k":
        net = parmat_net()
        sels = {f"ge_mean_theta{t}": O.Select(O.GE_MEAN, cc1_overlap=t) for t in PARMAT_THETAS}
        return dict(network_entry(net, sels), spec=PARMAT_SPEC)
    raise ValueError(name)


ALL = ("powerlaw50k", "parmat50k", "serving", "batch64", "ba200k")


def main(argv):
    names = argv or list(ALL)
    try:
        with open(OUT) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data["_about"] = ("Oracle results (oracle/ only) on the full-size workloads; written by "
                      "tests/golden/make_full_size_goldens.py. Digests are sha256 of little-endian arrays.")
    for name in names:
        t0 = time.time()
        data[name] = make(name)
        data[name]["_oracle_seconds"] = round(time.time() - t0, 1)
        data[name]["_threads"] = THREADS
        with open(OUT + ".tmp", "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)
        print(f"{name}: {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
