"""GPU parity of the CSF levels (qsd_csf_build) with the oracle's
(oracle/csf.py), on transposition results: node ids and pointers must be
equal element by element (integer work: bit-exact)."""
import itertools

import numpy as np
import pytest
import torch

import oracle
from oracle import csf as OC
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qsd():
    import paper_2005_10427_gb300 as q
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    q.lib()
    return q


def check(qsd, coords_np, sigma):
    rc, _ = oracle.transpose(coords_np, None, sigma)  # the sorted tensor
    ids, ptr = qsd.csf_levels(torch.from_numpy(np.ascontiguousarray(rc)).cuda(), sigma)
    eids, eptr = OC.csf_levels(rc, sigma)
    assert len(ids) == len(eids) and len(ptr) == len(eptr)
    for l, (a, b) in enumerate(zip(ids, eids)):
        assert np.array_equal(a.cpu().numpy(), b), f"ids level {l + 1}, sigma={sigma}"
    for l, (a, b) in enumerate(zip(ptr, eptr)):
        assert np.array_equal(a.cpu().numpy(), b), f"ptr level {l}, sigma={sigma}"


@pytest.mark.parametrize("nnz", [0, 1, 2, 31, 33, 4095, 4096, 4097, 12289, 50000])
def test_sizes(qsd, nnz):
    dims = [30, 20, 40]
    if nnz:
        t = synth.random_coo(dims, nnz, seed=nnz + 1, zipf=1.1)
        c = t.coords.numpy()
    else:
        c = np.zeros((3, 0), np.int32)
    for sigma in [(0, 1, 2), (2, 0, 1)]:
        check(qsd, c, sigma)


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5])
def test_orders_and_duplicates(qsd, r):
    dims = [9, 5, 7, 3, 11][:r]
    t = synth.random_coo(dims, 3000, seed=40 + r, dup_frac=0.3)
    c = t.coords.numpy()
    for sigma in list(itertools.permutations(range(r)))[:8]:
        check(qsd, c, sigma)


def test_transpose_then_csf_full_pipeline(qsd):
    # the library's own transposition feeding the CSF build, at a few tiles' size
    dims = [300, 2000, 50]
    t = synth.random_coo(dims, 200_000, seed=9, zipf=1.1)
    c = t.coords.numpy()
    sigma = (1, 2, 0)
    plan = qsd.Plan(dims, sigma)
    oc, _ = qsd.transpose(torch.from_numpy(c).cuda(), None, plan)
    ids, ptr = qsd.csf_levels(oc, sigma)
    rc, _ = oracle.transpose(c, None, sigma)
    eids, eptr = OC.csf_levels(rc, sigma)
    for a, b in zip(ids + ptr, eids + eptr):
        assert np.array_equal(a.cpu().numpy(), b)
