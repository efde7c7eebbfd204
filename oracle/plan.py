"""Reference oracle for the Quesadilla pass planner.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
bench's CPU-baseline leg; never by the product path. Shares no code with the
C++ planner in the library.

Everything here follows Section 3.4 (minimizing the number of partial sorts)
and Section 3.5 (Algorithm 3, QuesadillaSort) in the paper's notation, with
orderings written as tuples of 0-based mode labels (the paper writes 1-based
labels):

* ``f(tau, p)``: the set of modes that follow ``p`` in the complete ordering
  ``tau`` (Section 3.4.1, definition of f).
* ``b(tau, sigma)``: the number of modes ``sigma_i`` with
  ``f(sigma, sigma_i)`` not a subset of ``f(tau, sigma_i)`` -- the lower bound
  of Lemma 2 on the number of PartialSort calls.
* ``partial_sort_order(psi, l, k)``: the ordering produced by
  PartialSort(A, (psi_1..psi_l), psi_k), Eq. 1 when l = 0 and Eq. 2
  otherwise: (psi_1..psi_l, psi_k, psi_{l+1}..psi_{k-1}, psi_{k+1}..psi_r).
* ``quesadilla_calls(sigma, tau)``: the sequence of PartialSort calls that
  Algorithm 3 makes, as (prefix, mode) pairs. Algorithm 3 is stated for a
  simply ordered input; for an input sorted under another complete ordering
  ``tau`` its scan test compares against ``f(tau, .)`` instead of
  ``f((1..r), .)``, which is the paper's "without loss of generality"
  relabelling (Section 2.2) written without relabelling.
* ``topk_target(sigma, tau, K)`` and ``topk_steps(sigma, tau, K)``:
  Top-K-sadilla (Section 3.6): Algorithm 3's calls that sort the tensor to
  the order of its first K target modes, then one complete sort of every
  bucket of equal (sigma_1..sigma_K) by the remaining target modes.
* ``bfs_min_calls(tau, sigma)``: exhaustive search over every sequence of
  PartialSort calls (all l < k at every intermediate ordering) for the
  lexicographically smallest (#calls, #bucketed calls) that reaches sigma --
  the quantity Theorems 2 and 3 say Algorithm 3 attains.

Pins (tests/test_oracle_plan.py): Fig. 4's pass-count histograms, the worked
values of Section 3.4 (f((1,3,2,4),3) = {2,4}, b((1,3,2),(3,1,2)) = 1, the
(4,1,2,3) / (4,3,2,1) / (2,4,1,3) examples), and the BFS; the BFS itself is
pinned by executing its call sequences as real stable sorts on data.
"""
from __future__ import annotations

import heapq
from itertools import permutations
from typing import Iterable, List, Sequence, Tuple

Call = Tuple[Tuple[int, ...], int]  # (prefix modes, sorted mode)


def f(tau: Sequence[int], p: int) -> frozenset:
    """Modes that follow p in tau (Section 3.4.1)."""
    tau = tuple(tau)
    return frozenset(tau[tau.index(p) + 1:])


def needs_sort(sigma: Sequence[int], tau: Sequence[int], m: int) -> bool:
    """True when f(sigma, m) is not a subset of f(tau, m) (Lemma 2)."""
    return not f(sigma, m) <= f(tau, m)


def b(tau: Sequence[int], sigma: Sequence[int]) -> int:
    """Lower bound on PartialSort calls (definition after Lemma 2)."""
    return sum(1 for m in sigma if needs_sort(sigma, tau, m))


def partial_sort_order(psi: Sequence[int], l: int, k: int) -> Tuple[int, ...]:
    """Ordering after PartialSort(A, (psi_1..psi_l), psi_k), 1-based k > l.

    Eq. 1 (l = 0) and Eq. 2 (l > 0): psi_k moves to just after the prefix,
    every other mode keeps its relative position.
    """
    psi = tuple(psi)
    if not (0 <= l < k <= len(psi)):
        raise ValueError("PartialSort requires 0 <= l < k <= r")
    return psi[:l] + (psi[k - 1],) + psi[l:k - 1] + psi[k:]


def quesadilla_calls(sigma: Sequence[int],
                     tau: Sequence[int] | None = None) -> List[Call]:
    """The PartialSort calls Algorithm 3 makes, in execution order.

    Variables follow Algorithm 3 with its 1-based positions: ``s(i)`` is
    sigma_i. The scan loop grows k while sigma_{k+1} needs sorting (and
    k + 1 < r), the sort loop then sorts sigma_k, sigma_{k-1}, ...,
    sigma_{l+1}, each with prefix (sigma_1..sigma_l), and l jumps to l'.
    """
    sigma = tuple(sigma)
    r = len(sigma)
    if tau is None:
        tau = tuple(range(r))
    tau = tuple(tau)
    if sorted(sigma) != list(range(r)) or sorted(tau) != list(range(r)):
        raise ValueError("sigma and tau must be permutations of 0..r-1")

    def s(i: int) -> int:  # sigma_i, 1-based
        return sigma[i - 1]

    calls: List[Call] = []
    l = 0
    while l < r:
        k = l
        while k + 1 < r and needs_sort(sigma, tau, s(k + 1)):
            k += 1
        l_next = k + 1
        while k > l:
            calls.append((tuple(s(i) for i in range(1, l + 1)), s(k)))
            k -= 1
        l = l_next
    return calls


def topk_target(sigma: Sequence[int], tau: Sequence[int] | None, K: int) -> Tuple[int, ...]:
    """The complete ordering Top-K-sadilla's first stage sorts to.

    Section 3.6 fixes only its leading modes, sigma_1..sigma_K. The other
    modes follow here in their tau order: that is where a stable sort by the
    K leading modes leaves them, and none of them then needs a PartialSort
    call (each is followed only by modes that also follow it in tau).
    """
    sigma = tuple(sigma)
    tau = tuple(range(len(sigma))) if tau is None else tuple(tau)
    head = sigma[:max(0, K)]
    return head + tuple(m for m in tau if m not in head)


def topk_steps(sigma: Sequence[int], tau: Sequence[int] | None, K: int):
    """Top-K-sadilla (Section 3.6) as (calls, final).

    calls: the PartialSort calls Algorithm 3 makes from tau to
    topk_target(sigma, tau, K). final: (prefix modes, key modes) of the
    complete sort of every bucket of equal (sigma_1..sigma_K) by
    (sigma_{K+1}, ..., sigma_r), or None when the first stage already ends
    in sigma (always for K >= r - 1).
    """
    sigma = tuple(sigma)
    target = topk_target(sigma, tau, K)
    calls = quesadilla_calls(target, tau)
    final = None if target == sigma else (sigma[:K], sigma[K:])
    return calls, final


def apply_calls(tau: Sequence[int], calls: Iterable[Call]) -> Tuple[int, ...]:
    """Tracks the ordering through a sequence of calls (Eqs. 1 and 2).

    Each call's prefix must be the current ordering's leading modes, as in
    Lemma 2's statement of the allowed calls; otherwise ValueError.
    """
    psi = tuple(tau)
    for prefix, mode in calls:
        l = len(prefix)
        if psi[:l] != tuple(prefix):
            raise ValueError(f"prefix {prefix} is not the head of {psi}")
        k = psi.index(mode) + 1
        if k <= l:
            raise ValueError(f"mode {mode} lies inside the prefix {prefix}")
        psi = partial_sort_order(psi, l, k)
    return psi


def bfs_min_calls(tau: Sequence[int], sigma: Sequence[int]):
    """Smallest (#calls, #bucketed) over all call sequences from tau to sigma.

    Dijkstra over the r! complete orderings; an edge is one
    PartialSort(A, (psi_1..psi_l), psi_k) with 0 <= l < k <= r, of cost
    (1, 1 if l > 0 else 0). Returns (cost, one optimal call list).
    """
    tau, sigma = tuple(tau), tuple(sigma)
    r = len(tau)
    start = (0, 0)
    best = {tau: start}
    heap = [(start, tau, ())]
    while heap:
        cost, psi, path = heapq.heappop(heap)
        if psi == sigma:
            return cost, list(path)
        if best.get(psi, None) != cost:
            continue
        for l in range(r):
            for k in range(l + 1, r + 1):
                nxt = partial_sort_order(psi, l, k)
                c = (cost[0] + 1, cost[1] + (1 if l > 0 else 0))
                if nxt not in best or c < best[nxt]:
                    best[nxt] = c
                    heapq.heappush(heap, (c, nxt, path + ((psi[:l], psi[k - 1]),)))
    raise AssertionError("sigma is unreachable")  # every ordering is reachable


def pass_histogram(r: int) -> List[int]:
    """Fig. 4: number of target orderings per pass count, simple input."""
    hist = [0] * (r + 1)
    for sigma in permutations(range(r)):
        hist[len(quesadilla_calls(sigma))] += 1
    return hist
