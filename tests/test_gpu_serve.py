"""GPU tests of the serving engine (qsd_server_*): every served result equals
the standalone transposition of the same request bit for bit (alone vs in
the mix), admission respects the memory budget, steps overlap on the device,
and a server with queued work shuts down cleanly."""
import time

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

BUDGET_ERR = 8


@pytest.fixture(scope="module")
def qsd():
    import paper_2005_10427_gb300 as q
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    q.lib()
    return q


def pool(n, seed, nnz_hi=300_000, val_kind="f64_normal"):
    """Resident tensors: orders 3-4, log-uniform sizes, Zipf 1.2, f64 values."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        r = int(rng.integers(3, 5))
        nnz = int(np.exp(rng.uniform(np.log(1e3), np.log(nnz_hi))))
        while True:
            dims = [int(np.exp(rng.uniform(np.log(20), np.log(50_000)))) for _ in range(r)]
            if np.prod([float(d) for d in dims]) >= 8 * nnz:
                break
        t = synth.gen_coo(dims, nnz, [("zipf", 1.2)] * r, val_kind, seed * 100 + i, "cuda")
        out.append(t)
    return out


def standalone(qsd, t, sigma):
    # transpose() may use its input as scratch: give it copies, the pool stays intact
    plan = qsd.Plan(t.dims, sigma)
    c, v = qsd.transpose(t.coords.clone(), t.vals.clone(), plan)
    return c, v


def collect(srv, want, timeout_s=60):
    got = {}
    t0 = time.time()
    while len(got) < want and time.time() - t0 < timeout_s:
        for r in srv.poll(64, wait_ms=50):
            got[r["request"]] = r
    assert len(got) == want, f"{len(got)} of {want} requests completed"
    return got


def check_result(qsd, srv, t, sigma, rid):
    oc = torch.empty_like(t.coords)
    ov = torch.empty_like(t.vals)
    srv.copy_result(rid, oc, ov)
    sc, sv = standalone(qsd, t, sigma)
    torch.cuda.synchronize()
    assert torch.equal(oc, sc), f"request {rid}: coordinates differ from the standalone call"
    assert torch.equal(ov.view(torch.int64), sv.view(torch.int64)), f"request {rid}: values"


def test_served_results_equal_standalone(qsd):
    tens = pool(6, seed=1)
    srv = qsd.Server(1 << 30, val_bytes=8, max_batch=8, streams=2)
    ids = [srv.add_tensor(t.coords, t.vals, t.dims) for t in tens]
    rng = np.random.default_rng(7)
    reqs = {}
    for k in range(48):
        i = int(rng.integers(0, len(tens)))
        sigma = [int(x) for x in rng.permutation(tens[i].order)]
        reqs[srv.submit(ids[i], sigma)] = (i, sigma)
        if k % 8 == 7:
            time.sleep(0.002)  # arrivals while earlier steps run
    got = collect(srv, len(reqs))
    for rid, (i, sigma) in reqs.items():
        assert got[rid]["status"] == 0
        assert got[rid]["arrival_s"] <= got[rid]["admit_s"] <= got[rid]["done_s"]
        check_result(qsd, srv, tens[i], sigma, rid)
        srv.release(rid)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["released"] == len(reqs)
    assert st["bytes_in_use"] == 0
    srv.close()


def test_served_result_matches_oracle(qsd):
    t = synth.gen_coo([300, 40, 900], 50_000, [("zipf", 1.2)] * 3, "f64_normal", 5, "cuda")
    srv = qsd.Server(256 << 20, val_bytes=8)
    tid = srv.add_tensor(t.coords, t.vals, t.dims)
    sigma = (2, 0, 1)
    rid = srv.submit(tid, sigma)
    got = collect(srv, 1)
    assert got[rid]["status"] == 0
    oc = torch.empty_like(t.coords)
    ov = torch.empty_like(t.vals)
    srv.copy_result(rid, oc, ov)
    torch.cuda.synchronize()
    rc, rv = oracle.transpose(t.coords.cpu().numpy(), t.vals.cpu().numpy(), sigma)
    assert np.array_equal(oc.cpu().numpy(), rc)
    assert np.array_equal(ov.cpu().numpy().view(np.uint64), rv.view(np.uint64))
    srv.close()


def test_request_larger_than_budget_is_rejected(qsd):
    t = synth.gen_coo([100, 200, 300], 200_000, [("zipf", 1.2)] * 3, "f64_normal", 6, "cuda")
    srv = qsd.Server(1 << 20, val_bytes=8)  # 1 MiB: less than one result
    tid = srv.add_tensor(t.coords, t.vals, t.dims)
    rid = srv.submit(tid, (2, 1, 0))
    got = collect(srv, 1)
    assert got[rid]["status"] == BUDGET_ERR
    assert srv.stats()["rejected"] == 1
    srv.close()


def test_admission_under_a_tight_budget(qsd):
    tens = pool(3, seed=2, nnz_hi=200_000)
    one = max(t.nnz * (4 * t.order + 8) * 2 for t in tens)
    budget = int(2.5 * one) + (16 << 20)  # about two requests (plus scratch) at a time
    srv = qsd.Server(budget, val_bytes=8, streams=2, max_batch=4)
    ids = [srv.add_tensor(t.coords, t.vals, t.dims) for t in tens]
    reqs = {}
    for k in range(18):
        i = k % len(tens)
        sigma = list(reversed(range(tens[i].order))) if k % 2 else [1, 0] + list(
            range(2, tens[i].order))
        reqs[srv.submit(ids[i], sigma)] = (i, sigma)
    done = 0
    t0 = time.time()
    while done < len(reqs) and time.time() - t0 < 60:
        for r in srv.poll(16, wait_ms=50):
            assert r["status"] == 0
            i, sigma = reqs[r["request"]]
            check_result(qsd, srv, tens[i], sigma, r["request"])
            srv.release(r["request"])  # frees memory for the queued ones
            done += 1
    assert done == len(reqs)
    st = srv.stats()
    assert st["peak_bytes"] <= budget
    assert st["steps"] >= 3
    srv.close()


def test_steps_overlap_on_the_device(qsd):
    tens = pool(4, seed=3, nnz_hi=400_000)
    srv = qsd.Server(2 << 30, val_bytes=8, streams=2, max_batch=2)
    ids = [srv.add_tensor(t.coords, t.vals, t.dims) for t in tens]
    reqs = {}
    for k in range(24):
        i = k % len(tens)
        sigma = list(reversed(range(tens[i].order)))
        reqs[srv.submit(ids[i], sigma)] = (i, sigma)
    got = collect(srv, len(reqs))
    steps = sorted({(r["admit_s"], r["done_s"]) for r in got.values()})
    # some step was launched while an earlier one was still running
    assert any(b[0] < a[1] for a, b in zip(steps, steps[1:])), steps[:6]
    for rid, (i, sigma) in list(reqs.items())[:6]:
        check_result(qsd, srv, tens[i], sigma, rid)
    srv.close()


def test_destroy_with_queued_requests(qsd):
    tens = pool(2, seed=4, nnz_hi=300_000)
    srv = qsd.Server(1 << 30, val_bytes=8, streams=1, max_batch=1)
    ids = [srv.add_tensor(t.coords, t.vals, t.dims) for t in tens]
    for k in range(40):
        srv.submit(ids[k % 2], list(reversed(range(tens[k % 2].order))))
    srv.close()  # queued requests are dropped, the step in flight is waited for
    torch.cuda.synchronize()


def test_empty_tensor_and_f32_values(qsd):
    t = synth.gen_coo([50, 60, 70], 20_000, [("zipf", 1.2)] * 3, "f32_normal", 9, "cuda")
    e = torch.zeros((3, 0), dtype=torch.int32, device="cuda")
    ev = torch.zeros(0, dtype=torch.float32, device="cuda")
    srv = qsd.Server(256 << 20, val_bytes=4)
    a = srv.add_tensor(t.coords, t.vals, t.dims)
    b = srv.add_tensor(e, ev, [5, 5, 5])
    r0 = srv.submit(b, (2, 1, 0))
    r1 = srv.submit(a, (1, 2, 0))
    got = collect(srv, 2)
    assert got[r0]["status"] == 0 and got[r0]["nnz"] == 0
    oc = torch.empty_like(t.coords)
    ov = torch.empty_like(t.vals)
    srv.copy_result(r1, oc, ov)
    sc, sv = standalone(qsd, t, (1, 2, 0))
    torch.cuda.synchronize()
    assert torch.equal(oc, sc) and torch.equal(ov.view(torch.int32), sv.view(torch.int32))
    srv.close()


@pytest.mark.parametrize("val_kind,vb", [("f64_normal", 8), ("f32_normal", 4)])
def test_served_mix_each_result_matches_oracle(qsd, val_kind, vb):
    # every result of a mix served on two streams in continuous batches (arrivals
    # while earlier steps run, orders 3 and 4, every target order) against the
    # oracle's transposition of the same tensor
    tens = pool(5, seed=11 + vb, nnz_hi=250_000, val_kind=val_kind)
    srv = qsd.Server(1 << 30, val_bytes=vb, max_batch=6, streams=2)
    ids = [srv.add_tensor(t.coords, t.vals, t.dims) for t in tens]
    host = [(t.coords.cpu().numpy(), t.vals.cpu().numpy()) for t in tens]
    rng = np.random.default_rng(31 + vb)
    reqs = {}
    for k in range(36):
        i = int(rng.integers(0, len(tens)))
        sigma = tuple(int(x) for x in rng.permutation(tens[i].order))
        reqs[srv.submit(ids[i], sigma)] = (i, sigma)
        if k % 6 == 5:
            time.sleep(0.002)
    got = collect(srv, len(reqs))
    bits = np.uint64 if vb == 8 else np.uint32
    for rid, (i, sigma) in reqs.items():
        assert got[rid]["status"] == 0
        oc = torch.empty_like(tens[i].coords)
        ov = torch.empty_like(tens[i].vals)
        srv.copy_result(rid, oc, ov)
        torch.cuda.synchronize()
        rc, rv = oracle.transpose(host[i][0], host[i][1], sigma)
        assert np.array_equal(oc.cpu().numpy(), rc), (rid, sigma)
        assert np.array_equal(ov.cpu().numpy().view(bits), rv.view(bits)), (rid, sigma)
        srv.release(rid)
    srv.close()
