"""Pins for the stable-sort transposition oracle (oracle/qsd_oracle.cpp).

Each check ties the oracle to something other than itself: a dense
brute-force enumeration of the coordinate space in sigma-lexicographic order
(Section 2's definition of the ordering, written as nested loops), numpy's
lexsort, the worked example of Section 3.3, and the invariants a
transposition must satisfy.
"""
import itertools
import json
import os

import numpy as np
import pytest

import cpu_method
import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_distinct(rng, dims, nnz):
    cap = int(np.prod(dims))
    flat = np.sort(rng.choice(cap, size=min(nnz, cap), replace=False))
    coords = np.stack(np.unravel_index(flat, dims)).astype(np.int32)
    return coords  # sorted in identity order, distinct


def _brute_force(coords, vals, dims, sigma):
    """Enumerate every coordinate in sigma-lex order; keep the stored ones."""
    r, nnz = coords.shape
    where = {}
    for j in range(nnz):
        where[tuple(int(x) for x in coords[:, j])] = j
    out_c, out_v = [], []
    for sub in itertools.product(*[range(dims[m]) for m in sigma]):
        c = [0] * r
        for p, m in enumerate(sigma):
            c[m] = sub[p]
        j = where.get(tuple(c))
        if j is not None:
            out_c.append(c)
            out_v.append(vals[j])
    return np.array(out_c, dtype=np.int32).T.reshape(r, -1), np.array(out_v, dtype=vals.dtype)


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5])
def test_dense_brute_force(r):
    rng = np.random.default_rng(100 + r)
    for trial in range(4):
        dims = [int(x) for x in rng.integers(1, 6, size=r)]
        cap = int(np.prod(dims))
        nnz = int(rng.integers(0, cap + 1))
        coords = _rand_distinct(rng, dims, nnz)
        vals = rng.standard_normal(coords.shape[1])
        perms = list(itertools.permutations(range(r)))
        if len(perms) > 24:
            perms = [perms[i] for i in rng.choice(len(perms), 24, replace=False)]
        for sigma in perms:
            oc, ov = oracle.transpose(coords, vals, sigma)
            bc, bv = _brute_force(coords, vals, dims, sigma)
            assert np.array_equal(oc, bc), (dims, sigma)
            assert np.array_equal(ov.view(np.uint64), bv.view(np.uint64))


@pytest.mark.parametrize("r", [2, 3, 4, 6, 8])
def test_matches_numpy_lexsort_with_duplicates(r):
    rng = np.random.default_rng(7 + r)
    nnz = 3000
    dims = [int(x) for x in rng.integers(1, 9, size=r)]
    coords = np.stack([rng.integers(0, d, size=nnz) for d in dims]).astype(np.int32)
    vals = np.arange(nnz, dtype=np.float32)
    for _ in range(6):
        sigma = [int(x) for x in rng.permutation(r)]
        # np.lexsort sorts by the LAST key first and is stable.
        ref = np.lexsort([coords[m] for m in reversed(sigma)])
        perm = oracle.permutation(coords, sigma)
        assert np.array_equal(perm, ref)
        oc, ov = oracle.transpose(coords, vals, sigma)
        assert np.array_equal(oc, coords[:, ref])
        assert np.array_equal(ov, vals[ref])


def test_invariants_random():
    rng = np.random.default_rng(11)
    for r in (3, 4, 5):
        nnz = 5000
        dims = [int(x) for x in rng.integers(2, 40, size=r)]
        coords = np.stack([rng.integers(0, d, size=nnz) for d in dims]).astype(np.int32)
        vals = rng.standard_normal(nnz).astype(np.float64)
        sigma = [int(x) for x in rng.permutation(r)]
        perm = oracle.permutation(coords, sigma)
        oc, ov = oracle.transpose(coords, vals, sigma)
        # nnz preserved and the output is a permutation of the input entries
        assert oc.shape == coords.shape and np.array_equal(np.sort(perm), np.arange(nnz))
        assert np.array_equal(oc, coords[:, perm]) and np.array_equal(ov, vals[perm])
        # sorted under sigma: each adjacent pair is non-decreasing lexicographically
        a = oc[:, :-1][sigma]
        b = oc[:, 1:][sigma]
        lt = np.zeros(nnz - 1, bool)
        eq = np.ones(nnz - 1, bool)
        for p in range(r):
            lt |= eq & (a[p] < b[p])
            eq &= a[p] == b[p]
        assert np.all(lt | eq)
        # stability: equal coordinates keep increasing input index
        assert np.all(perm[1:][eq] > perm[:-1][eq])


def test_values_move_bitwise():
    coords = np.array([[2, 1, 0, 1], [0, 0, 0, 1]], dtype=np.int32)
    raw = np.array([0x7FF8000000000123, 0x8000000000000000, 0x7FF0000000000001,
                    0x3FF0000000000000], dtype=np.uint64)
    vals = raw.view(np.float64)
    oc, ov = oracle.transpose(coords, vals, [0, 1])
    assert np.array_equal(ov.view(np.uint64), raw[[2, 1, 3, 0]])
    raw32 = np.array([0x7FC00001, 0x80000000, 0xFF800000, 1], dtype=np.uint32)
    oc, ov = oracle.transpose(coords, raw32.view(np.float32), [1, 0])
    assert np.array_equal(ov.view(np.uint32), raw32[[2, 1, 0, 3]])


def test_worked_example_section_3_3():
    ex = json.load(open(os.path.join(GOLDEN, "bucketed_example_sec3_3.json")))
    digits = [[int(ch) for ch in str(x)] for x in ex["A_crd"]]
    coords = np.array(digits, dtype=np.int32).T  # mode m = digit m
    sigma = [m - 1 for m in ex["sigma_1based"]]
    perm = oracle.permutation(coords, sigma)
    # the final permutation: input position (1-based) of each printed B.crd entry
    assert [int(p) + 1 for p in perm] == [ex["A_crd"].index(x) + 1 for x in ex["B_crd"]]
    oc, _ = oracle.transpose(coords, np.zeros(coords.shape[1]), sigma)
    got = [int("".join(str(d) for d in oc[:, j])) for j in range(oc.shape[1])]
    assert got == ex["B_crd"]
    got_sigma = [int("".join(str(oc[m, j]) for m in sigma)) for j in range(oc.shape[1])]
    assert got_sigma == ex["B_crd_sigma"]


def test_empty_and_single():
    c = np.zeros((3, 0), np.int32)
    oc, ov = oracle.transpose(c, np.zeros(0, np.float32), [2, 1, 0])
    assert oc.shape == (3, 0) and ov.shape == (0,)
    c = np.array([[4], [5], [6]], np.int32)
    oc, ov = oracle.transpose(c, np.array([1.5], np.float32), [1, 2, 0])
    assert np.array_equal(oc, c) and ov[0] == np.float32(1.5)


def test_rejects_bad_permutation():
    c = np.zeros((3, 4), np.int32)
    with pytest.raises(ValueError):
        oracle.transpose(c, None, [0, 0, 1])
    with pytest.raises(ValueError):
        oracle.transpose(c, None, [0, 1, 3])


def test_rank_under_matches_the_stable_sort():
    rng = np.random.default_rng(17)
    for r in (2, 3, 4):
        dims = [int(x) for x in rng.integers(2, 9, size=r)]
        coords = np.stack([rng.integers(0, d, size=2000) for d in dims]).astype(np.int32)
        sigma = [int(x) for x in rng.permutation(r)]
        perm = oracle.permutation(coords, sigma)
        out = coords[:, perm]
        for p in rng.choice(coords.shape[1], 40, replace=False):
            less, equal = oracle.rank_under(coords, sigma, out[:, p])
            assert less <= p < less + equal
        # the first entry of each run of equal coordinates sits exactly at `less`
        less, equal = oracle.rank_under(coords, sigma, out[:, 0])
        assert less == 0 and equal >= 1


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5])
def test_cpu_method_equals_oracle(r):
    # the paper's method restated on the host (Algorithms 1-3 as parallel
    # counting sorts) gives the definition's result for every order
    dims = [13, 7, 29, 5, 3][:r]
    t = synth.random_coo(dims, 2500, seed=90 + r, dup_frac=0.2, zipf=1.1)
    c, v = t.coords.numpy(), t.vals.numpy()
    for sigma in itertools.permutations(range(r)):
        a = oracle.transpose(c, v, sigma)
        for threads in (1, 3):
            b = cpu_method.transpose(c, v, dims, sigma, threads=threads)
            assert np.array_equal(a[0], b[0]), (sigma, threads)
            assert np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))


def test_cpu_method_non_identity_input_order():
    dims = [20, 30, 10, 6]
    tau = (2, 0, 3, 1)
    t = synth.random_coo(dims, 4000, seed=99, dup_frac=0.1, input_order=tau)
    c, v = t.coords.numpy(), t.vals.numpy()
    for sigma in itertools.permutations(range(4)):
        a = oracle.transpose(c, v, sigma)
        b = cpu_method.transpose(c, v, dims, sigma, tau=tau)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), sigma


@pytest.mark.parametrize("r", [3, 4, 5])
def test_cpu_method_topk_sadilla_equals_oracle(r):
    # Top-K-sadilla on the host (Section 3.6): Algorithm 3's calls to the
    # first K target modes, then a comparison sort of every bucket; the same
    # result for every K, with duplicates, on one and on several threads
    dims = [13, 7, 29, 5, 3][:r]
    t = synth.random_coo(dims, 2500, seed=120 + r, dup_frac=0.2, zipf=1.1)
    c, v = t.coords.numpy(), t.vals.numpy()
    rng = np.random.default_rng(r)
    for sigma in [tuple(int(x) for x in rng.permutation(r)) for _ in range(6)]:
        a = oracle.transpose(c, v, sigma)
        for K in range(r + 1):
            for threads in (1, 3):
                b = cpu_method.transpose(c, v, dims, sigma, threads=threads, top_k=K)
                assert np.array_equal(a[0], b[0]), (sigma, K, threads)
                assert np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))

