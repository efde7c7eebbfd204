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


def _run_ws(qsd, coords, vals, plan, n):
    cb = [torch.from_numpy(coords).cuda(), torch.empty_like(torch.from_numpy(coords)).cuda()]
    vb = [torch.from_numpy(vals).cuda(), torch.empty(n, dtype=torch.float32, device="cuda")]
    ws = torch.empty(plan.workspace_bytes(n), dtype=torch.uint8, device="cuda")
    sel = qsd.transpose_buffers(cb, vb, 0, n, plan, ws)
    return cb[sel].cpu().numpy(), vb[sel].cpu().numpy()


def _run_noalloc(qsd, coords, vals, plan, n):
    cb = [torch.from_numpy(coords).cuda(), torch.empty_like(torch.from_numpy(coords)).cuda()]
    vb = [torch.from_numpy(vals).cuda(), torch.empty(n, dtype=torch.float32, device="cuda")]
    sel = qsd.transpose_noalloc(cb, vb, 0, n, plan)
    torch.cuda.synchronize()
    assert qsd.get_async_status() == 0
    return cb[sel].cpu().numpy(), vb[sel].cpu().numpy()


def test_noalloc_matches_workspace_entry_point_twice(qsd):
    t = synth.gen_coo([3000, 500, 700], 400_000, [("zipf", 1.1)] * 3, "f32_normal", seed=12)
    coords, vals = t.coords.numpy(), t.vals.numpy()
    n = coords.shape[1]
    for sigma in [(0, 2, 1), (2, 1, 0), (1, 0, 2)]:
        plan = qsd.Plan(t.dims, sigma)
        assert plan.workspace_bytes(n) <= 64 << 20
        want_c, want_v = _run_ws(qsd, coords, vals, plan, n)
        for _ in range(2):  # the shared scratch keeps the last call's contents
            got_c, got_v = _run_noalloc(qsd, coords, vals, plan, n)
            assert np.array_equal(got_c, want_c), sigma
            assert np.array_equal(got_v.view(np.uint32), want_v.view(np.uint32)), sigma


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
