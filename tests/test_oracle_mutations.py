"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each.

Each mutant replaces one oracle function with a subtly wrong variant: a dropped
term, a wrong index or bound, a swapped operator. The pins in
``test_oracle_pins.py`` must fail for every one of them.
"""
import numpy as np
import pytest

from oracle import oracle as O
import tests.test_oracle_pins as P


def _sumdist_n_minus_1(n, F, R):  # unreachable charged n-1 instead of n
    F = np.asarray(F, np.uint64)
    return F + np.uint64(n - 1) * (np.uint64(n - 1) - np.asarray(R, np.uint64))


def _wf_without_normalisation(n, F, R):  # Eq. 1 applied to the component only: R / F
    F = np.asarray(F, np.float64)
    R = np.asarray(R, np.float64)
    return np.where(F > 0, R / np.where(F > 0, F, 1), 0.0)


def _cc2_min(sumdists):  # min instead of max in Algorithm 1
    est = np.asarray(sumdists[0], np.uint64).copy()
    for s in sumdists[1:]:
        est = np.minimum(est, np.asarray(s, np.uint64))
    return est


_orig_avg = O.cc1_average


def _cc1_avg_min(ratios):  # min instead of max in Eq. 3
    from fractions import Fraction
    vals = []
    for r in ratios:
        fin = r[np.isfinite(r)]
        vals.append(O.exact_sum(fin) / len(fin) if len(fin) else Fraction(0))
    return min(vals)


def _rank_high_id(scores):  # ties broken by the higher id
    scores = np.asarray(scores, np.float64)
    ids = np.arange(scores.shape[0])
    return np.lexsort((-ids, -scores)).astype(np.int32)


def _degrees_plus_one(rowptr):  # off-by-one degree
    rowptr = np.asarray(rowptr, np.int64)
    return (rowptr[1:] - rowptr[:-1] + 1).astype(np.int32)


def _accuracy_swapped(pred, truth):  # precision and recall swapped
    a = _orig_accuracy(pred, truth)
    a["precision"], a["recall"] = a["recall"], a["precision"]
    return a


_orig_accuracy = O.accuracy


def _and_union(n, layer_keys):  # OR instead of AND
    out = layer_keys[0]
    for k in layer_keys[1:]:
        out = np.union1d(out, k)
    return out


def _or_intersection(n, layer_keys):  # AND instead of OR
    out = layer_keys[0]
    for k in layer_keys[1:]:
        out = np.intersect1d(out, k)
    return out


_orig_arc_csr = O.arc_csr


def _arc_csr_out_edges(n, keys, reverse=False):  # out-closeness: the in-edge CSR is never built
    return _orig_arc_csr(n, keys, reverse=False)


_orig_arc_keys = O.arc_keys


def _arc_keys_symmetrised(n, src, dst):  # arcs made undirected (reverse arc added)
    return np.union1d(_orig_arc_keys(n, src, dst), _orig_arc_keys(n, dst, src))


def _directed_fw():
    for seed in range(5):
        P.test_directed_floyd_warshall(seed)


PINS = [P.test_empty_graph, P.test_disjoint_components_wf_and_sumdist, P.test_hand_two_layer_example,
        P.test_fig5_cc2_example, P.test_cc2_subset_layers_equals_ground_truth, P.test_selection_special_cases,
        P.test_accuracy_metrics, P.test_and_aggregation_invariants, P.test_cc2_single_layer_is_sumdist_ranking,
        P.test_directed_path_and_cycle_closed_forms, _directed_fw, P.test_directed_aggregates_are_arc_sets]


@pytest.mark.parametrize("name,fn", [
    ("sum_dist_n", _sumdist_n_minus_1),
    ("wf_closeness", _wf_without_normalisation),
    ("cc2_estimate", _cc2_min),
    ("cc1_average", _cc1_avg_min),
    ("rank_order", _rank_high_id),
    ("degrees", _degrees_plus_one),
    ("accuracy", _accuracy_swapped),
    ("and_keys", _and_union),
    ("or_keys", _or_intersection),
    ("arc_csr", _arc_csr_out_edges),
    ("arc_keys", _arc_keys_symmetrised),
])
def test_mutant_is_caught(monkeypatch, name, fn):
    monkeypatch.setattr(O, name, fn)
    caught = 0
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError, IndexError):
            caught += 1
    assert caught > 0, f"no pin catches the mutant of {name}"
