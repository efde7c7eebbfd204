"""The bounded waits' abort path, on the GPU.

Every wait in the library's kernels gives up after a limit, records
QSD_ERR_TIMEOUT in the device status word and returns instead of trapping.
This test shortens the limit to 50 ms and makes one wait run out on purpose:
block 0 of the digit-pass move kernel arms its first staging slot but never
issues that slot's bulk copies, so the ranking warps' wait on the slot
expires, all warps of the block leave through their abort path, and the
producer's final drain gives up on the copies that were never issued. The
call must come back with QSD_ERR_TIMEOUT in its status word, the sticky
device status must report it, and the next call (limits restored) must run
clean and match the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TIMEOUT = 7


@pytest.fixture(scope="module")
def qsd():
    import paper_2005_10427_gb300 as q
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    q.lib()
    return q


def test_stalled_copy_times_out_and_the_next_call_is_clean(qsd):
    # a global group with two digit passes over ~560 chunks: every block of
    # the move kernel, block 0 included, claims chunks
    t = synth.gen_coo([3000, 500, 700], 4_000_000, [("zipf", 1.1)] * 3, "f32_normal", seed=21,
                      device="cuda")
    sigma = (1, 0, 2)
    plan = qsd.Plan(t.dims, sigma)
    assert plan.info()["groups"][0]["prefix"] == () and plan.info()["groups"][0]["passes"] >= 1
    r, n = t.coords.shape
    cb = [torch.empty((r, n), dtype=torch.int32, device="cuda") for _ in range(2)]
    vb = [torch.empty(n, dtype=t.vals.dtype, device="cuda") for _ in range(2)]
    ws = torch.empty(plan.workspace_bytes(n), dtype=torch.uint8, device="cuda")
    assert qsd.get_async_status() == 0
    qsd.debug_set_spin_limit_ns(50_000_000)
    try:
        qsd.debug_set_stall(1)
        try:
            qsd.transpose_from(t.coords, t.vals, cb, vb, n, plan, ws)
            assert qsd.workspace_status(ws) == TIMEOUT
        finally:
            qsd.debug_set_stall(0)
        assert qsd.get_async_status() == TIMEOUT  # sticky, then cleared
        assert qsd.get_async_status() == 0
    finally:
        qsd.debug_set_spin_limit_ns(0)
    sel = qsd.transpose_from(t.coords, t.vals, cb, vb, n, plan, ws)
    assert qsd.workspace_status(ws) == 0
    assert qsd.get_async_status() == 0
    rc, rv = oracle.transpose(t.coords.cpu().numpy(), t.vals.cpu().numpy(), sigma)
    assert np.array_equal(cb[sel].cpu().numpy(), rc)
    assert np.array_equal(vb[sel].cpu().numpy().view(np.uint32), rv.view(np.uint32))
