"""Reference oracle: the paper's two PartialSort primitives, step by step.

TEST INFRASTRUCTURE ONLY (tests, smoke check, bench CPU-baseline leg).

``partial_sort_nonbucketed`` is Algorithm 1 (histogram / counting sort on
one mode) and ``partial_sort_bucketed`` is Algorithm 2 (discover the buckets
of equal prefix, counting-sort on the mode into ``perm``, then stably
re-bucket with ``pos``). Both keep the paper's 1-based positions internally
(``count[1] <- 1``, ``bucket[1] <- 1``, ``pos[1] <- 1``) so that the
intermediate arrays can be compared with the worked example of Section 3.3;
coordinates themselves are 0-based here, so index value ``c`` of a mode is
the paper's ``i = c + 1``.

These are plain Python loops meant for small inputs; ``quesadilla_sort``
runs the calls Algorithm 3 plans (``oracle.plan.quesadilla_calls``) with
them, which must agree with the stable-sort oracle.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

from .plan import quesadilla_calls, topk_steps

Coord = Tuple[int, ...]


def partial_sort_nonbucketed(crd: Sequence[Coord], mode: int, n_mode: int):
    """Algorithm 1: stable counting sort of ``crd`` on ``mode``.

    Returns (B.crd, perm) where perm[j'] (0-based) is the input position of
    output entry j'.
    """
    N = len(crd)
    count = [0] * (n_mode + 2)  # entries 1..n+1 used
    count[1] = 1
    for j in range(1, N + 1):  # compute the count array
        i = crd[j - 1][mode] + 1
        count[i + 1] += 1
    for v in range(2, n_mode + 2):  # prefix sum
        count[v] += count[v - 1]
    out: List[Coord] = [None] * N  # type: ignore[list-item]
    perm = [0] * N
    for j in range(1, N + 1):  # move to the output position
        i = crd[j - 1][mode] + 1
        jp = count[i]
        out[jp - 1] = crd[j - 1]
        perm[jp - 1] = j - 1
        count[i] += 1
    return out, perm


def partial_sort_bucketed(crd: Sequence[Coord], prefix: Sequence[int],
                          mode: int, n_mode: int):
    """Algorithm 2: sort on ``mode`` while keeping the order of ``prefix``.

    The input must be sorted under an ordering that starts with ``prefix``.
    Returns (B.crd, bucket, pos, perm) with the paper's 1-based ``bucket``,
    ``pos`` (bucket start positions, before the final loop advances them)
    and ``perm`` arrays, for comparison with Section 3.3.
    """
    N = len(crd)
    if N == 0:
        return [], [], [], []
    count = [0] * (n_mode + 2)
    count[1] = 1
    bucket = [0] * (N + 1)
    bucket[1] = 1
    pos = [0] * (N + 1)
    pos[1] = 1
    perm = [0] * (N + 1)
    n_b = 1

    def key(c: Coord):
        return tuple(c[m] for m in prefix)

    # count array, equivalence classes under the prefix, bucket starts
    i = crd[0]
    count[i[mode] + 1 + 1] += 1
    for j in range(2, N + 1):
        i, ip = crd[j - 1], crd[j - 2]
        if key(i) != key(ip):
            n_b += 1
            pos[n_b] = j
        bucket[j] = n_b
        count[i[mode] + 1 + 1] += 1
    for v in range(2, n_mode + 2):  # prefix sum
        count[v] += count[v - 1]
    for j in range(1, N + 1):  # permutation ordered on the mode
        i = crd[j - 1]
        perm[count[i[mode] + 1]] = j
        count[i[mode] + 1] += 1
    pos_start = list(pos[1:n_b + 1])
    out: List[Coord] = [None] * (N + 1)  # type: ignore[list-item]
    for j in range(1, N + 1):  # reintroduce the prefix order
        bk = bucket[perm[j]]
        out[pos[bk]] = crd[perm[j] - 1]
        pos[bk] += 1
    return out[1:], bucket[1:], pos_start, perm[1:]


def quesadilla_sort(crd: Sequence[Coord], dims: Sequence[int],
                    sigma: Sequence[int], tau: Sequence[int] | None = None,
                    vals: Sequence | None = None):
    """Runs Algorithm 3's calls with Algorithms 1 and 2 on (crd, vals).

    Values ride along with their coordinates; entries are tagged with their
    input position so ties stay distinguishable.
    """
    r = len(sigma)
    tagged = [tuple(c) + (j,) for j, c in enumerate(crd)]
    for prefix, mode in quesadilla_calls(sigma, tau):
        if len(prefix) == 0:
            tagged, _ = partial_sort_nonbucketed(tagged, mode, dims[mode])
        else:
            tagged, *_ = partial_sort_bucketed(tagged, prefix, mode, dims[mode])
    out_crd = [t[:r] for t in tagged]
    order = [t[r] for t in tagged]
    out_vals = None if vals is None else [vals[j] for j in order]
    return out_crd, out_vals, order


def topk_sadilla_sort(crd: Sequence[Coord], dims: Sequence[int], sigma: Sequence[int],
                      K: int, tau: Sequence[int] | None = None, vals: Sequence | None = None):
    """Top-K-sadilla (Section 3.6) on (crd, vals): Algorithm 3's calls, run
    with Algorithms 1 and 2, sort the tensor to the order of sigma_1..sigma_K
    (oracle.plan.topk_target); then every bucket of equal (sigma_1..sigma_K)
    is sorted completely by (sigma_{K+1}, ..., sigma_r) with a comparison
    sort. The section's quicksort is not stable; Python's sort, which is,
    stands in for it, so that duplicate coordinates keep their values in
    input order as every other path here does."""
    r = len(sigma)
    tagged = [tuple(c) + (j,) for j, c in enumerate(crd)]
    calls, final = topk_steps(sigma, tau, K)
    for prefix, mode in calls:
        if len(prefix) == 0:
            tagged, _ = partial_sort_nonbucketed(tagged, mode, dims[mode])
        else:
            tagged, *_ = partial_sort_bucketed(tagged, prefix, mode, dims[mode])
    if final is not None:
        prefix, keys = final
        out: List[Coord] = []
        j, N = 0, len(tagged)
        while j < N:  # one bucket of equal prefix at a time
            e = j + 1
            while e < N and all(tagged[e][m] == tagged[j][m] for m in prefix):
                e += 1
            out.extend(sorted(tagged[j:e], key=lambda t: tuple(t[m] for m in keys)))
            j = e
        tagged = out
    out_crd = [t[:r] for t in tagged]
    order = [t[r] for t in tagged]
    out_vals = None if vals is None else [vals[j] for j in order]
    return out_crd, out_vals, order
