"""Parity at the benchmark workloads' full sizes, in the launch configuration
bench.py times (out-of-place calls on resident inputs).

The 1M-entry uniform workload is compared with the oracle entry by entry.
The 76M- and 140M-entry workloads are too large for the oracle in a test, so
they are checked by properties that hold at any size -- the output is sorted
under sigma with strictly increasing keys (coordinates are distinct), and is
a permutation of the input (an order-independent hash over every entry's
coordinates and value bits) -- and at sampled output positions, whose exact
rank the oracle computes by counting the entries that precede them.
"""
import numpy as np
import pytest
import torch

import oracle
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


def _transpose_resident(qsd, t, sigma):
    r, n = t.coords.shape
    plan = qsd.Plan(t.dims, sigma)
    cb = [torch.empty((r, n), dtype=torch.int32, device="cuda") for _ in range(2)]
    vb = [torch.empty(n, dtype=t.vals.dtype, device="cuda") for _ in range(2)]
    ws = torch.empty(plan.workspace_bytes(n), dtype=torch.uint8, device="cuda")
    sel = qsd.transpose_from(t.coords, t.vals, cb, vb, n, plan, ws)
    assert qsd.workspace_status(ws) == 0
    return cb[sel], vb[sel]


def _hash(coords, vals):
    x = vals.view(torch.int32).long() if vals.element_size() == 4 else vals.view(torch.int64)
    acc = x * 0x9E3779B1
    for m in range(coords.shape[0]):
        acc = acc ^ (coords[m].long() * (0x85EBCA77 + 2 * m + 1))
        acc = acc * 0x27D4EB2F + 0x165667B1
    return int(acc.sum()), int((acc ^ (acc >> 29)).sum())


def _strictly_sorted(oc, sigma):
    n = oc.shape[1]
    lt = torch.zeros(n - 1, dtype=torch.bool, device=oc.device)
    eq = torch.ones(n - 1, dtype=torch.bool, device=oc.device)
    for m in sigma:
        k = oc[m]
        lt |= eq & (k[:-1] < k[1:])
        eq &= k[:-1] == k[1:]
    return bool(lt.all())


def _check_large(t, sigma, oc, ov, samples=6, seed=0):
    assert _strictly_sorted(oc, sigma), sigma
    assert _hash(t.coords, t.vals) == _hash(oc, ov), sigma
    host_in = t.coords.cpu().numpy()
    out_c = oc.cpu().numpy()
    rng = np.random.default_rng(seed)
    n = out_c.shape[1]
    for p in [0, n - 1] + [int(x) for x in rng.integers(0, n, samples)]:
        less, equal = oracle.rank_under(host_in, sigma, out_c[:, p])
        assert equal == 1 and less == p, (sigma, p, less, equal)


def test_uniform_1m_full_oracle(qsd):
    w = synth.WORKLOAD_3D_UNIFORM
    t = synth.make(w, device="cuda")
    coords, vals = t.coords.cpu().numpy(), t.vals.cpu().numpy()
    for sigma in w["perms"]:
        oc, ov = _transpose_resident(qsd, t, sigma)
        rc, rv = oracle.transpose(coords, vals, sigma)
        assert np.array_equal(oc.cpu().numpy(), rc)
        assert np.array_equal(ov.cpu().numpy().view(np.uint64), rv.view(np.uint64))


def test_nell2_like_76m_all_orders(qsd):
    w = synth.WORKLOAD_NELL2_LIKE
    t = synth.make(w, device="cuda")
    for i, sigma in enumerate(w["perms"]):
        oc, ov = _transpose_resident(qsd, t, sigma)
        _check_large(t, sigma, oc, ov, seed=i)
        del oc, ov


def test_delicious_like_140m_sampled_orders(qsd):
    w = synth.WORKLOAD_DELICIOUS_LIKE
    t = synth.make(w, device="cuda")
    for i, sigma in enumerate([(0, 1, 3, 2), (1, 0, 3, 2), (3, 2, 1, 0), (2, 0, 1, 3),
                               (0, 3, 2, 1)]):
        oc, ov = _transpose_resident(qsd, t, sigma)
        _check_large(t, sigma, oc, ov, samples=3, seed=10 + i)
        del oc, ov
