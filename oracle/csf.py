"""Oracle for the compressed sparse fiber (CSF) levels of a sorted tensor
(test infrastructure, plain numpy; shares nothing with the CUDA library).

Section 2.1 describes CSF as a tree over the lexicographically sorted
coordinates: the order sigma assigns modes to levels, a node of level l is
an index of mode sigma_l under its parent, the children of a node are ordered
by index, and the paths from the root to the leaves are the coordinates.
Written out for a coordinate list already sorted under sigma (0-based levels
1..r, entry j, coordinate rows coords[m]):

* the nodes of level l are the maximal runs of entries with equal prefix
  (sigma_0, ..., sigma_{l-1}), in order; a node starts at entry j when j == 0
  or some of those modes differ between entries j-1 and j;
* ids[l-1][k] is the coordinate of mode sigma_{l-1} of node k of level l;
* ptr[l][k] .. ptr[l][k+1]-1 are the children (level l+1 nodes) of node k of
  level l, for l = 0 (the root, one node) .. r-1;
* ptr[r][k] .. ptr[r][k+1]-1 are the entries of leaf k (more than one only
  for duplicate coordinates; the values array is indexed by entry).
"""
from __future__ import annotations

import numpy as np


def csf_levels(coords, sigma):
    """(ids, ptr) of a coordinate list sorted under sigma.

    coords: int array (r, nnz) sorted under sigma. Returns ids (r arrays,
    level 1..r) and ptr (r + 1 arrays, levels 0..r), all int64.
    """
    coords = np.asarray(coords)
    r, nnz = coords.shape
    sigma = [int(m) for m in sigma]
    starts = []  # starts[l]: entry indices where a level-(l+1) node begins
    new = np.zeros(nnz, dtype=bool)
    if nnz:
        new[0] = True
    for l in range(r):
        m = sigma[l]
        if nnz > 1:
            new[1:] |= coords[m, 1:] != coords[m, :-1]
        starts.append(np.nonzero(new)[0])
    ids = [coords[sigma[l], starts[l]].astype(np.int64) for l in range(r)]
    ptr = []
    root = np.array([0], dtype=np.int64)
    parents = [root] + starts  # node starts of levels 0..r (the root starts at entry 0)
    children = starts + [np.arange(nnz, dtype=np.int64)]  # level l+1 nodes; entries below leaves
    for l in range(r + 1):
        if nnz == 0:
            ptr.append(np.zeros(len(parents[l]) + 1 if l else 2, dtype=np.int64))
            continue
        p = np.searchsorted(children[l], parents[l]).astype(np.int64)
        ptr.append(np.concatenate([p, [len(children[l])]]))
    return ids, ptr


def expand(ids, ptr):
    """The coordinate tuples (one per entry, in order) a CSF tree stands for:
    every root-to-leaf path, repeated once per entry under the leaf."""
    r = len(ids)
    out = []

    def walk(level, node, prefix):
        if level == r:
            for _ in range(int(ptr[r][node + 1] - ptr[r][node])):
                out.append(tuple(prefix))
            return
        for child in range(int(ptr[level][node]), int(ptr[level][node + 1])):
            walk(level + 1, child, prefix + [int(ids[level][child])])

    walk(0, 0, [])
    return out
