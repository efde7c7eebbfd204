"""Pins of the CSF-levels oracle (oracle/csf.py) against things other than
itself: a hand-worked tree, an independent nested-dictionary construction of
the tree, the round trip back to the coordinate list, and the matrix case,
which is compressed sparse row storage with the empty rows dropped (checked
against scipy.sparse)."""
import itertools

import numpy as np
import pytest

from oracle import csf as C


def test_hand_worked_tree():
    # sorted under (0,1,2); the last coordinate is duplicated
    coords = np.array([[0, 0, 0, 1, 1],
                       [0, 0, 2, 1, 1],
                       [1, 3, 0, 1, 1]])
    ids, ptr = C.csf_levels(coords, (0, 1, 2))
    assert [list(x) for x in ids] == [[0, 1], [0, 2, 1], [1, 3, 0, 1]]
    assert [list(x) for x in ptr] == [[0, 2], [0, 2, 3], [0, 2, 3, 4], [0, 1, 2, 3, 5]]


def nested_tree(tuples):
    """Levels of the tree built by inserting each coordinate tuple into
    nested dictionaries and walking them in key order."""
    root = {}
    leaf_count = {}
    for t in tuples:
        d = root
        for x in t:
            d = d.setdefault(x, {})
        leaf_count[t] = leaf_count.get(t, 0) + 1
    r = len(tuples[0]) if tuples else 0
    ids = [[] for _ in range(r)]
    ptr = [[0] for _ in range(r + 1)]
    frontier = [((), root)]
    for l in range(r):
        nxt = []
        for prefix, d in frontier:
            for key in sorted(d):
                ids[l].append(key)
                nxt.append((prefix + (key,), d[key]))
            ptr[l].append(len(ids[l]))
        frontier = nxt
    total = 0
    for prefix, _ in frontier:
        total += leaf_count[prefix]
        ptr[r].append(total)
    return ids, ptr


@pytest.mark.parametrize("r,seed", [(2, 1), (3, 2), (4, 3), (5, 4)])
def test_against_nested_dictionaries_and_round_trip(r, seed):
    rng = np.random.default_rng(seed)
    dims = [int(x) for x in rng.integers(1, 6, size=r)]
    n = 300
    coords = np.stack([rng.integers(0, d, size=n) for d in dims])
    for sigma in list(itertools.permutations(range(r)))[:6]:
        order = np.lexsort([coords[m] for m in reversed(sigma)])
        sc = coords[:, order]
        tuples = [tuple(int(sc[m, j]) for m in sigma) for j in range(n)]
        ids, ptr = C.csf_levels(sc, sigma)
        eids, eptr = nested_tree(tuples)
        assert [list(x) for x in ids] == eids
        assert [list(x) for x in ptr] == eptr
        assert C.expand(ids, ptr) == tuples


def test_matrix_case_is_csr_without_empty_rows():
    sp = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(5)
    rows, cols = 40, 30
    flat = rng.choice(rows * cols, size=200, replace=False)
    r_, c_ = np.divmod(np.sort(flat), cols)
    m = sp.csr_matrix((np.ones(len(r_)), (r_, c_)), shape=(rows, cols))
    m.sort_indices()
    ids, ptr = C.csf_levels(np.stack([r_, c_]), (0, 1))
    nonempty = np.nonzero(np.diff(m.indptr))[0]
    assert np.array_equal(ids[0], nonempty)
    assert np.array_equal(ptr[0], [0, len(nonempty)])
    assert np.array_equal(ids[1], m.indices)
    assert np.array_equal(ptr[1], np.concatenate([m.indptr[nonempty], [m.nnz]]))
    assert np.array_equal(ptr[2], np.arange(m.nnz + 1))


def test_empty_and_single_entry():
    ids, ptr = C.csf_levels(np.zeros((3, 0), dtype=np.int64), (2, 0, 1))
    assert all(len(x) == 0 for x in ids)
    assert [list(x) for x in ptr] == [[0, 0], [0], [0], [0]]
    ids, ptr = C.csf_levels(np.array([[4], [7], [9]]), (1, 2, 0))
    assert [list(x) for x in ids] == [[7], [9], [4]]
    assert [list(x) for x in ptr] == [[0, 1], [0, 1], [0, 1], [0, 1]]
