"""The allocation-free entry point, qsd_transpose_noalloc.

Some callers cannot allocate device memory: a host framework or serving
engine that owns all device memory through its own allocator and budget, or
a latency-critical path where an allocation could synchronise the device.
For them the library runs a transposition with a fixed device-global
scratch array instead of a workspace. This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

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


def _buffers(coords, vals):
    cb = [torch.from_numpy(coords).cuda(), torch.empty_like(torch.from_numpy(coords)).cuda()]
    if vals is None:
        return cb, None
    vb = [torch.from_numpy(vals).cuda(), torch.empty_like(torch.from_numpy(vals)).cuda()]
    return cb, vb


def _host(cb, vb, sel):
    return cb[sel].cpu().numpy(), (None if vb is None else vb[sel].cpu().numpy())


def _run_ws(qsd, coords, vals, plan, n):
    cb, vb = _buffers(coords, vals)
    ws = torch.empty(plan.workspace_bytes(n), dtype=torch.uint8, device="cuda")
    sel = qsd.transpose_buffers(cb, vb, 0, n, plan, ws)
    torch.cuda.synchronize()
    assert qsd.workspace_status(ws) == 0
    return _host(cb, vb, sel)


def _run_noalloc(qsd, coords, vals, plan, n):
    cb, vb = _buffers(coords, vals)
    sel = qsd.transpose_noalloc(cb, vb, 0, n, plan)
    torch.cuda.synchronize()
    assert qsd.get_async_status() == 0
    return _host(cb, vb, sel)


def _same(got, want):
    (gc, gv), (wc, wv) = got, want
    if not np.array_equal(gc, wc):
        return False
    if wv is None:
        return gv is None
    bits = np.uint64 if wv.dtype.itemsize == 8 else np.uint32
    return np.array_equal(gv.view(bits), wv.view(bits))


def test_noalloc_matches_workspace_entry_point_twice(qsd):
    t = synth.gen_coo([3000, 500, 700], 400_000, [("zipf", 1.1)] * 3, "f32_normal", seed=12)
    coords, vals = t.coords.numpy(), t.vals.numpy()
    n = coords.shape[1]
    for sigma in [(0, 2, 1), (2, 1, 0), (1, 0, 2)]:
        plan = qsd.Plan(t.dims, sigma)
        assert plan.workspace_bytes(n) <= 64 << 20
        want = _run_ws(qsd, coords, vals, plan, n)
        for _ in range(2):  # the shared scratch keeps the last call's contents
            assert _same(_run_noalloc(qsd, coords, vals, plan, n), want), sigma


@pytest.mark.parametrize("case", ["f64", "coords_only", "order4"])
def test_noalloc_value_widths_and_orders(qsd, case):
    if case == "order4":
        t = synth.gen_coo([900, 300, 400, 50], 300_000, [("zipf", 1.2)] * 3 + [("uniform",)],
                          "f64_normal", seed=13)
        sigmas = [(0, 1, 3, 2), (3, 2, 1, 0), (1, 0, 2, 3)]
    else:
        t = synth.gen_coo([2000, 800, 600], 300_000, [("zipf", 1.1)] * 3,
                          "f64_uniform" if case == "f64" else "f32_normal", seed=14)
        sigmas = [(0, 2, 1), (2, 0, 1), (1, 2, 0)]
    coords = t.coords.numpy()
    vals = None if case == "coords_only" else t.vals.numpy()
    n = coords.shape[1]
    for sigma in sigmas:
        plan = qsd.Plan(t.dims, sigma)
        want = _run_ws(qsd, coords, vals, plan, n)
        for _ in range(2):
            assert _same(_run_noalloc(qsd, coords, vals, plan, n), want), (case, sigma)


def test_noalloc_near_its_scratch_limit(qsd):
    # the largest bucketed request whose workspace still fits the 64 MiB array
    dims = [20000, 9000, 28000]
    plan = qsd.Plan(dims, (0, 2, 1))
    lo, hi = 1_000_000, 40_000_000
    while hi - lo > 1000:
        mid = (lo + hi) // 2
        if plan.workspace_bytes(mid) <= 64 << 20:
            lo = mid
        else:
            hi = mid
    n = lo
    assert plan.workspace_bytes(n) <= 64 << 20 < plan.workspace_bytes(n + 2000)
    t = synth.gen_coo(dims, n, [("zipf", 1.1)] * 3, "f32_normal", seed=15, device="cuda")
    coords, vals = t.coords.cpu().numpy(), t.vals.cpu().numpy()
    want = _run_ws(qsd, coords, vals, plan, n)
    for _ in range(2):
        assert _same(_run_noalloc(qsd, coords, vals, plan, n), want)


def test_noalloc_rejects_requests_beyond_its_scratch(qsd):
    plan = qsd.Plan([1 << 20, 1 << 20, 1 << 20], (0, 2, 1))
    n = 100_000_000  # needs far more than 64 MiB of scratch
    assert plan.workspace_bytes(n) > 64 << 20
    from paper_2005_10427_gb300 import _capi
    c = _capi.Coords()
    c.buf[0] = c.buf[1] = 256  # never dereferenced: rejected before any launch
    c.stride = n
    v = _capi.Values()
    st = qsd.lib().qsd_transpose_noalloc(ctypes.byref(c), ctypes.byref(v), n, plan.handle, None)
    assert st == 9  # QSD_ERR_WORKSPACE_TOO_SMALL
