"""Graph-captured calls (qsd_exec_*): one out-of-place transposition captured
into a CUDA graph and replayed. Every launch must equal the oracle, bit for
bit, whatever the plan; launches repeat, run on other streams, and pick up
new input written in place."""
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


def make_exec(qsd, t, sigma, vals=True, **opts):
    r, n = t.coords.shape
    plan = qsd.Plan(t.dims, sigma, **opts)
    cin = t.coords.cuda()
    vin = t.vals.cuda() if vals else None
    cb = [torch.full((r, max(n, 1)), -3, dtype=torch.int32, device="cuda") for _ in range(2)]
    vb = [torch.zeros(max(n, 1), dtype=t.vals.dtype, device="cuda") for _ in range(2)] \
        if vals else None
    ws = torch.empty(max(plan.workspace_bytes(n), 256), dtype=torch.uint8, device="cuda")
    ex = qsd.Exec(cin, vin, cb, vb, n, plan, ws)
    return ex, cin, vin, cb, vb, ws


def check(qsd, ex, cin, vin, cb, vb, ws, sigma, stream=None):
    n = cin.shape[1]
    sel = ex.launch(stream)
    torch.cuda.synchronize()
    assert qsd.workspace_status(ws) == 0
    rc, rv = oracle.transpose(cin.cpu().numpy(), None if vin is None else vin.cpu().numpy(),
                              sigma)
    assert np.array_equal(cb[sel][:, :n].cpu().numpy(), rc), sigma
    if vin is not None:
        u = np.uint64 if vin.element_size() == 8 else np.uint32
        assert np.array_equal(vb[sel][:n].cpu().numpy().view(u), rv.view(u)), sigma


@pytest.mark.parametrize("sigma,opts", [((2, 1, 0), {}), ((0, 2, 1), {}), ((1, 0, 2), {}),
                                        ((1, 2, 0), {"key_index": True}),
                                        ((0, 2, 1), {"global_groups": True}),
                                        ((0, 1, 2), {})])
def test_exec_matches_oracle_twice(qsd, sigma, opts):
    t = synth.gen_coo([400, 3000, 500], 300_000, [("zipf", 1.1)] * 3, "f32_normal", seed=3)
    ex, cin, vin, cb, vb, ws = make_exec(qsd, t, sigma, **opts)
    for _ in range(2):
        check(qsd, ex, cin, vin, cb, vb, ws, sigma)


@pytest.mark.parametrize("nnz", [0, 1, 4097, 70000])
def test_exec_sizes_f64_and_no_values(qsd, nnz):
    dims = [60, 90, 40, 30]
    t = synth.random_coo(dims, nnz, seed=nnz + 9, val_kind="f64_uniform", zipf=1.1) if nnz \
        else synth.CooTensor(torch.zeros((4, 0), dtype=torch.int32),
                             torch.zeros(0, dtype=torch.float64), dims, [0, 1, 2, 3])
    for vals in (True, False):
        ex, cin, vin, cb, vb, ws = make_exec(qsd, t, (3, 1, 0, 2), vals=vals)
        check(qsd, ex, cin, vin, cb, vb, ws, (3, 1, 0, 2))


def test_exec_other_stream_and_new_input_in_place(qsd):
    dims = [700, 800, 900]
    t = synth.gen_coo(dims, 200_000, [("zipf", 1.2)] * 3, "f64_normal", seed=4)
    sigma = (2, 0, 1)
    ex, cin, vin, cb, vb, ws = make_exec(qsd, t, sigma)
    s = torch.cuda.Stream()
    check(qsd, ex, cin, vin, cb, vb, ws, sigma, stream=s)
    # another tensor of the same size and dims written into the bound input
    t2 = synth.gen_coo(dims, 200_000, [("zipf", 1.2)] * 3, "f64_normal", seed=5)
    cin.copy_(t2.coords.cuda())
    vin.copy_(t2.vals.cuda())
    torch.cuda.synchronize()
    check(qsd, ex, cin, vin, cb, vb, ws, sigma)
