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


def fused(qsd, coords_np, vals_np, dims, sigma, tau=None, **opts):
    """qsd_transpose_csf_from_ws: the transposition and the CSF levels of its
    result, the levels' neighbour comparisons made by the last movement."""
    plan = qsd.Plan(dims, sigma, input_mode_order=tau, **opts)
    r, n = coords_np.shape
    cin = torch.from_numpy(np.ascontiguousarray(coords_np)).cuda()
    vin = None if vals_np is None else torch.from_numpy(np.ascontiguousarray(vals_np)).cuda()
    cb = [torch.empty((r, max(n, 1)), dtype=torch.int32, device="cuda") for _ in range(2)]
    vb = None if vin is None else [torch.empty(max(n, 1), dtype=vin.dtype, device="cuda")
                                   for _ in range(2)]
    cap = max(n, 1)
    ids = [torch.full((cap,), -9, dtype=torch.int32, device="cuda") for _ in range(r)]
    ptr = [torch.full((2 if l == 0 else cap + 1,), -9, dtype=torch.int32, device="cuda")
           for l in range(r + 1)]
    nodes = torch.empty(r + 1, dtype=torch.int32, device="cuda")
    ws = torch.empty(qsd.transpose_csf_workspace_bytes(plan, n), dtype=torch.uint8, device="cuda")
    sel = qsd.transpose_csf_from(cin, vin, cb, vb, n, plan, ids, ptr, nodes, ws)
    assert qsd.workspace_status(ws) == 0
    nn = [int(x) for x in nodes.cpu()]
    oc = cb[sel][:, :n].cpu().numpy()
    ov = None if vb is None else vb[sel][:n].cpu().numpy()
    return (oc, ov, [ids[l][:nn[l + 1]].cpu().numpy() for l in range(r)],
            [ptr[l][:nn[l] + 1].cpu().numpy() for l in range(r + 1)])


def check_fused(qsd, coords, vals, dims, sigma, tau=None, **opts):
    oc, ov, ids, ptr = fused(qsd, coords, vals, dims, sigma, tau, **opts)
    rc, rv = oracle.transpose(coords, vals, sigma)
    assert np.array_equal(oc, rc), sigma
    if vals is not None:
        u = np.uint64 if vals.dtype.itemsize == 8 else np.uint32
        assert np.array_equal(ov.view(u), rv.view(u)), sigma
    eids, eptr = OC.csf_levels(rc, sigma)
    assert len(ids) == len(eids) and len(ptr) == len(eptr)
    for l, (a, b) in enumerate(zip(ids, eids)):
        assert np.array_equal(a, b), f"ids level {l + 1}, sigma={sigma}"
    for l, (a, b) in enumerate(zip(ptr, eptr)):
        assert np.array_equal(a, b), f"ptr level {l}, sigma={sigma}"


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5])
def test_fused_every_permutation(qsd, r):
    # global and bucketed groups, multi-group plans, the block-local sort of
    # small buckets and the digit passes of large ones all write the levels
    dims = [60, 300, 2000, 40, 9][:r]
    t = synth.random_coo(dims, 30_000, seed=60 + r, zipf=1.1, dup_frac=0.1)
    c, v = t.coords.numpy(), t.vals.numpy()
    for sigma in itertools.permutations(range(r)):
        check_fused(qsd, c, v, dims, sigma, local_capacity=1024)


@pytest.mark.parametrize("nnz", [0, 1, 2, 17, 1025, 4097, 70001])
def test_fused_sizes(qsd, nnz):
    dims = [50, 70, 90]
    if nnz:
        t = synth.random_coo(dims, nnz, seed=nnz + 2, zipf=1.1)
        c, v = t.coords.numpy(), t.vals.numpy()
    else:
        c, v = np.zeros((3, 0), np.int32), np.zeros(0, np.float32)
    for sigma in [(0, 1, 2), (0, 2, 1), (2, 1, 0), (1, 0, 2)]:
        check_fused(qsd, c, v, dims, sigma)


def test_fused_plan_variants(qsd):
    # the identity (no movement: every level from the rows), global groups,
    # Top-K-sadilla, the (key, index) form (gathered: levels from the rows)
    # and a non-identity input order, with duplicates
    dims = [40, 300, 200, 7]
    for tau in [None, (3, 1, 0, 2)]:
        t = synth.random_coo(dims, 120_000, seed=81, val_kind="f64_uniform", zipf=1.2,
                             dup_frac=0.2, input_order=tau)
        c, v = t.coords.numpy(), t.vals.numpy()
        base = tuple(range(4)) if tau is None else tau
        for sigma, opts in [(base, {}), ((1, 0, 3, 2), {"global_groups": True}),
                            ((0, 3, 2, 1), {"top_k": 1}), ((3, 2, 1, 0), {"key_index": True}),
                            ((2, 3, 0, 1), {})]:
            check_fused(qsd, c, v, dims, sigma, tau=tau, **opts)


def test_fused_equals_separate_build_at_size(qsd):
    # the same tree as transposing, then qsd_csf_build, on a Zipf tensor with
    # large and small buckets
    dims = [12000, 9000, 28000]
    t = synth.random_coo(dims, 2_000_000, seed=5, zipf=1.1)
    c, v = t.coords.numpy(), t.vals.numpy()
    for sigma in [(0, 2, 1), (1, 2, 0), (2, 0, 1)]:
        oc, _, ids, ptr = fused(qsd, c, v, dims, sigma)
        sids, sptr = qsd.csf_levels(torch.from_numpy(oc).cuda(), sigma)
        for a, b in zip(ids + ptr, sids + sptr):
            assert np.array_equal(a, b.cpu().numpy()), sigma
