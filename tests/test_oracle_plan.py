"""Pins for the planner oracle (oracle/plan.py) and the literal PartialSorts
(oracle/partial_sort.py): Fig. 4, the worked values of Sections 3.3-3.4, an
exhaustive search over call sequences, and execution of the planned calls
as real stable sorts on data."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from oracle import plan as P
from oracle import partial_sort as PS

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_fig4_pass_histograms():
    fig4 = json.load(open(os.path.join(GOLDEN, "fig4_pass_histogram.json")))
    for r in (3, 4, 5):
        hist = P.pass_histogram(r)
        want = fig4[str(r)]
        assert hist == want[:r + 1] and all(x == 0 for x in want[r + 1:]), r


def test_section_3_4_worked_values():
    ex = json.load(open(os.path.join(GOLDEN, "planner_examples_sec3_4.json")))
    for e in ex["f_examples"]:
        tau = [m - 1 for m in e["tau"]]
        assert P.f(tau, e["p"] - 1) == frozenset(m - 1 for m in e["f"])
    for e in ex["b_examples"]:
        assert P.b([m - 1 for m in e["tau"]], [m - 1 for m in e["sigma"]]) == e["b"]
    for e in ex["min_calls"]:
        sigma = [m - 1 for m in e["sigma"]]
        calls = P.quesadilla_calls(sigma)
        assert len(calls) == e["calls"]
        (cost, _) = P.bfs_min_calls(range(4), sigma)
        assert cost[0] == e["calls"]
        if "bucketed" in e:
            assert sum(1 for pre, _ in calls if pre) == e["bucketed"] == cost[1]
        if "sequence" in e:
            want = [(tuple(m - 1 for m in pre), mode - 1) for pre, mode in e["sequence"]]
            assert calls == want
    # "(4,1,2,3) can be accomplished with the single call PartialSort(A, (), 4)"
    assert P.quesadilla_calls([3, 0, 1, 2]) == [((), 3)]


def test_partial_sort_order_eqs_1_and_2():
    # Eq. 1: (tau_k, tau_1..tau_{k-1}, tau_{k+1}..tau_r)
    assert P.partial_sort_order((0, 1, 2, 3), 0, 3) == (2, 0, 1, 3)
    # Eq. 2: (tau_1..tau_l, tau_k, tau_{l+1}..tau_{k-1}, tau_{k+1}..tau_r)
    assert P.partial_sort_order((0, 1, 2, 3), 2, 4) == (0, 1, 3, 2)
    assert P.partial_sort_order((5, 4, 3, 2, 1, 0), 1, 5) == (5, 1, 4, 3, 2, 0)


def _iddfs_min_calls(tau, sigma, max_depth):
    """Independent search: iterative deepening over every call sequence."""
    r = len(tau)
    best = None
    for depth in range(max_depth + 1):
        def rec(psi, d, nb):
            nonlocal best
            if d == depth:
                if psi == tuple(sigma) and (best is None or nb < best[1]):
                    best = (depth, nb)
                return
            for l in range(r):
                for k in range(l + 1, r + 1):
                    rec(P.partial_sort_order(psi, l, k), d + 1, nb + (l > 0))
        rec(tuple(tau), 0, 0)
        if best is not None:
            return best
    return None


def test_bfs_matches_iterative_deepening_r3_r4():
    for r in (3, 4):
        for tau in itertools.permutations(range(r)):
            for sigma in itertools.permutations(range(r)):
                (cost, _) = P.bfs_min_calls(tau, sigma)
                assert cost == _iddfs_min_calls(tau, sigma, r), (tau, sigma)
            if r == 4:
                break  # one tau for r = 4 keeps the search fast


@pytest.mark.parametrize("r", [2, 3, 4, 5])
def test_quesadilla_is_minimal_and_correct(r):
    rng = np.random.default_rng(r)
    taus = [tuple(range(r))] + [tuple(int(x) for x in rng.permutation(r)) for _ in range(3)]
    for tau in taus:
        for sigma in itertools.permutations(range(r)):
            calls = P.quesadilla_calls(sigma, tau)
            # Theorem 1: the calls reach sigma (Eqs. 1-2 track the ordering)
            assert P.apply_calls(tau, calls) == tuple(sigma)
            # Lemma 2 + Theorem 2: exactly b(tau, sigma) calls, the minimum
            (cost, path) = P.bfs_min_calls(tau, sigma)
            assert len(calls) == P.b(tau, sigma) == cost[0]
            # Theorem 3: fewest bucketed calls among minimum-length sequences
            assert sum(1 for pre, _ in calls if pre) == cost[1]
            assert P.apply_calls(tau, path) == tuple(sigma)


def test_r6_sampled_minimality():
    rng = np.random.default_rng(6)
    for _ in range(12):
        tau = tuple(int(x) for x in rng.permutation(6))
        sigma = tuple(int(x) for x in rng.permutation(6))
        calls = P.quesadilla_calls(sigma, tau)
        (cost, _) = P.bfs_min_calls(tau, sigma)
        assert (len(calls), sum(1 for pre, _ in calls if pre)) == cost


def _stable_by_mode_seq(coords, calls):
    """Executes PartialSort calls as numpy stable sorts (Eqs. 1-2 semantics):
    a call (prefix, mode) is a stable sort by (prefix..., mode)."""
    perm = np.arange(coords.shape[1])
    for prefix, mode in calls:
        keys = [coords[mode][perm]] + [coords[m][perm] for m in reversed(prefix)]
        perm = perm[np.lexsort(keys)]
    return perm


def test_bfs_and_quesadilla_sequences_sort_real_data():
    rng = np.random.default_rng(5)
    for r in (3, 4, 5):
        dims = [int(x) for x in rng.integers(2, 7, size=r)]
        coords = np.stack([rng.integers(0, d, size=4000) for d in dims]).astype(np.int32)
        order = np.lexsort([coords[m] for m in reversed(range(r))])
        coords = coords[:, order]  # simply ordered, with duplicates
        for sigma in list(itertools.permutations(range(r)))[::7]:
            want = oracle.permutation(coords, sigma)
            for calls in (P.quesadilla_calls(sigma), P.bfs_min_calls(range(r), sigma)[1]):
                got = _stable_by_mode_seq(coords, calls)
                assert np.array_equal(got, want), (sigma, calls)


def test_worked_example_arrays_section_3_3():
    ex = json.load(open(os.path.join(GOLDEN, "bucketed_example_sec3_3.json")))
    crd = [tuple(int(ch) - 1 for ch in str(x)) for x in ex["A_crd"]]  # 0-based digits
    prefix = [m - 1 for m in ex["prefix_1based"]]
    mode = ex["mode_1based"] - 1
    out, bucket, pos, perm = PS.partial_sort_bucketed(crd, prefix, mode, 9)
    assert bucket == ex["bucket"]
    assert pos == ex["pos"]
    assert perm == ex["perm"]
    assert [int("".join(str(d + 1) for d in crd[p - 1])) for p in perm] == ex["A_crd_perm"]
    assert [int("".join(str(d + 1) for d in c)) for c in out] == ex["B_crd"]
    # the same transposition is one bucketed call of Algorithm 3
    assert P.quesadilla_calls([m - 1 for m in ex["sigma_1based"]]) == [((0, 1), 3)]


def test_algorithm_1_is_stable_counting_sort():
    rng = np.random.default_rng(3)
    crd = [tuple(int(x) for x in rng.integers(0, 5, size=3)) for _ in range(300)]
    crd_tagged = [c + (j,) for j, c in enumerate(crd)]
    out, perm = PS.partial_sort_nonbucketed(crd_tagged, 1, 5)
    want = sorted(range(len(crd)), key=lambda j: crd[j][1])  # Python sort is stable
    assert perm == want and [c[3] for c in out] == want


@pytest.mark.parametrize("r", [3, 4])
def test_literal_quesadilla_equals_stable_sort(r):
    rng = np.random.default_rng(40 + r)
    dims = [int(x) for x in rng.integers(2, 6, size=r)]
    for tau in [tuple(range(r)), tuple(int(x) for x in rng.permutation(r))]:
        coords = np.stack([rng.integers(0, d, size=400) for d in dims]).astype(np.int32)
        order = np.lexsort([coords[m] for m in reversed(tau)])
        coords = coords[:, order]  # sorted under tau, with duplicates
        crd = [tuple(int(x) for x in coords[:, j]) for j in range(coords.shape[1])]
        vals = list(range(len(crd)))
        for sigma in itertools.permutations(range(r)):
            out_crd, out_vals, ordr = PS.quesadilla_sort(crd, dims, sigma, tau, vals)
            want = oracle.permutation(coords, sigma)
            assert ordr == [int(x) for x in want], (tau, sigma)
            assert out_vals == [int(x) for x in want]


def _sorted_under(coords, sigma):
    return [int(x) for x in np.lexsort([coords[m] for m in reversed(tuple(sigma))])]


@pytest.mark.parametrize("r", [3, 4])
def test_topk_sadilla_equals_stable_sort(r):
    # Section 3.6: for every K the two stages end in sigma order; ties
    # (duplicate coordinates) keep their input order
    rng = np.random.default_rng(70 + r)
    dims = [int(x) for x in rng.integers(2, 6, size=r)]
    for tau in [tuple(range(r)), tuple(int(x) for x in rng.permutation(r))]:
        coords = np.stack([rng.integers(0, d, size=300) for d in dims]).astype(np.int32)
        coords = coords[:, _sorted_under(coords, tau)]
        crd = [tuple(int(x) for x in coords[:, j]) for j in range(coords.shape[1])]
        vals = list(range(len(crd)))
        for sigma in itertools.permutations(range(r)):
            want = [int(x) for x in oracle.permutation(coords, sigma)]
            for K in range(r + 1):
                _, out_vals, ordr = PS.topk_sadilla_sort(crd, dims, sigma, K, tau, vals)
                assert ordr == want, (tau, sigma, K)
                assert out_vals == want


@pytest.mark.parametrize("r", [3, 4, 5])
def test_topk_first_stage_is_the_stable_sort_by_k_modes(r):
    # the calls of the first stage, run as real stable sorts, leave the data
    # exactly as one stable sort by (sigma_1..sigma_K) does, and they are never
    # more than Quesadilla's own
    rng = np.random.default_rng(80 + r)
    dims = [3] * r
    coords = np.stack([rng.integers(0, 3, size=200) for _ in range(r)]).astype(np.int32)
    tau = tuple(int(x) for x in rng.permutation(r))
    coords = coords[:, _sorted_under(coords, tau)]
    crd = [tuple(int(x) for x in coords[:, j]) for j in range(coords.shape[1])]
    for sigma in itertools.permutations(range(r)):
        for K in range(r + 1):
            calls, final = P.topk_steps(sigma, tau, K)
            target = P.topk_target(sigma, tau, K)
            assert target[:K] == tuple(sigma[:K])
            assert P.apply_calls(tau, calls) == target
            assert len(calls) == P.b(tau, target) <= P.b(tau, sigma)
            assert not any(P.needs_sort(target, tau, m) for m in target[K:])
            tagged = [c + (j,) for j, c in enumerate(crd)]
            for prefix, mode in calls:
                if prefix:
                    tagged, *_ = PS.partial_sort_bucketed(tagged, prefix, mode, dims[mode])
                else:
                    tagged, _ = PS.partial_sort_nonbucketed(tagged, mode, dims[mode])
            head = np.stack([coords[m] for m in sigma[:K]]) if K else np.zeros((0, coords.shape[1]))
            want = [int(x) for x in np.lexsort(head[::-1])] if K else list(range(coords.shape[1]))
            assert [t[r] for t in tagged] == want, (tau, sigma, K)
            if K >= r - 1:
                assert (calls, final) == (P.quesadilla_calls(sigma, tau), None)
            if K == 0:
                assert calls == [] and final == (None if tuple(sigma) == tau else ((), tuple(sigma)))
            if final is not None:
                assert final == (tuple(sigma[:K]), tuple(sigma[K:]))
