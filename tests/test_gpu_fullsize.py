"""Parity at the benchmark workloads' full sizes, in the launch configuration
bench.py times (out-of-place calls on resident inputs; one graph launch for
the batch), element by element against the oracle.

Every target order of the 1M-, 76M- and 140M-entry workloads and every one
of the 256 tensors of the batched workload is compared with the oracle's
transposition of the same input: coordinates exactly, values bit for bit.
The oracle (std::stable_sort on one host core per call) runs on several host
cores at once -- each call releases the interpreter lock -- while the GPU
computes the next order; the number of calls in flight is bounded by the
host's cores and free memory. Each GPU output is also checked on the device
for being strictly sorted under sigma (coordinates are distinct), a property
that holds at any size.
"""
import os
from concurrent.futures import FIRST_COMPLETED, ThreadPoolExecutor, wait

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
    oracle.lib()
    return q


def _mem_available() -> int:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 16 << 30


def _host_jobs(bytes_per_job: int) -> int:
    """Oracle calls that may run at once: one per host core (leaving one for
    this thread), as many as ~60% of the free host memory holds."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return max(1, min((cores or 2) - 1, int(0.6 * _mem_available()) // bytes_per_job))


def _bits(v: np.ndarray) -> np.ndarray:
    return v.view(np.uint64 if v.dtype.itemsize == 8 else np.uint32)


def _transpose_resident(qsd, t, sigma, cb, vb, ws):
    n = t.coords.shape[1]
    plan = qsd.Plan(t.dims, sigma)
    need = plan.workspace_bytes(n)
    w = ws if need <= ws.numel() else torch.empty(need, dtype=torch.uint8, device="cuda")
    sel = qsd.transpose_from(t.coords, t.vals, cb, vb, n, plan, w)
    assert qsd.workspace_status(w) == 0
    return cb[sel], vb[sel]


def _strictly_sorted(oc, sigma):
    n = oc.shape[1]
    lt = torch.zeros(n - 1, dtype=torch.bool, device=oc.device)
    eq = torch.ones(n - 1, dtype=torch.bool, device=oc.device)
    for m in sigma:
        k = oc[m]
        lt |= eq & (k[:-1] < k[1:])
        eq &= k[:-1] == k[1:]
    return bool(lt.all())


def _all_orders_against_oracle(qsd, wl):
    """GPU transposition of every target order of workload wl, each compared
    with the oracle element by element on the host."""
    t = synth.make(wl, device="cuda")
    r, n = t.coords.shape
    coords, vals = t.coords.cpu().numpy(), t.vals.cpu().numpy()
    cb = [torch.empty((r, n), dtype=torch.int32, device="cuda") for _ in range(2)]
    vb = [torch.empty(n, dtype=t.vals.dtype, device="cuda") for _ in range(2)]
    ws = torch.empty(max(qsd.Plan(wl["dims"], s).workspace_bytes(n) for s in wl["perms"]),
                     dtype=torch.uint8, device="cuda")
    rec = 4 * r + vals.dtype.itemsize
    # per job: the GPU result's host copy, the oracle's output, its index
    # array and std::stable_sort's merge buffer
    jobs = _host_jobs(n * (2 * rec + 16))

    def check(sigma, gc, gv):
        rc, rv = oracle.transpose(coords, vals, sigma)
        ok_c = np.array_equal(gc, rc)
        ok_v = np.array_equal(_bits(gv), _bits(rv))
        return sigma, ok_c, ok_v

    bad = []
    with ThreadPoolExecutor(jobs) as ex:
        pending = set()
        for sigma in wl["perms"]:
            oc, ov = _transpose_resident(qsd, t, sigma, cb, vb, ws)
            assert _strictly_sorted(oc, sigma), sigma
            gc, gv = oc.cpu().numpy(), ov.cpu().numpy()
            del oc, ov
            while len(pending) >= jobs:
                done, pending = wait(pending, return_when=FIRST_COMPLETED)
                bad += [f.result() for f in done if not all(f.result()[1:])]
            pending.add(ex.submit(check, sigma, gc, gv))
            del gc, gv
        for f in pending:
            if not all(f.result()[1:]):
                bad.append(f.result())
    assert not bad, bad


def test_uniform_1m_all_orders(qsd):
    _all_orders_against_oracle(qsd, synth.WORKLOAD_3D_UNIFORM)


def test_nell2_like_76m_all_orders(qsd):
    _all_orders_against_oracle(qsd, synth.WORKLOAD_NELL2_LIKE)


def test_delicious_like_140m_all_23_orders(qsd):
    _all_orders_against_oracle(qsd, synth.WORKLOAD_DELICIOUS_LIKE)


def test_batched_256_tensors_each_against_oracle(qsd):
    descs = synth.batch_workload()
    tens = [synth.gen_coo(d["dims"], d["nnz"], d["dists"], d["val_kind"], d["seed"], "cuda")
            for d in descs]
    plans = [qsd.Plan(d["dims"], d["perm"]) for d in descs]
    outs = [([torch.empty_like(t.coords) for _ in range(2)],
             [torch.empty_like(t.vals) for _ in range(2)]) for t in tens]
    batch = qsd.Batch([(p, t.coords, t.vals, o[0], o[1]) for p, t, o in zip(plans, tens, outs)])
    ws = torch.empty(batch.workspace_bytes(), dtype=torch.uint8, device="cuda")
    batch.run(ws)
    torch.cuda.synchronize()
    assert qsd.workspace_status(ws) == 0

    def check(i):
        t, d = tens[i], descs[i]
        sel = batch.result(i)
        gc = outs[i][0][sel].cpu().numpy()
        gv = outs[i][1][sel].cpu().numpy()
        rc, rv = oracle.transpose(t.coords.cpu().numpy(), t.vals.cpu().numpy(), d["perm"])
        return i, np.array_equal(gc, rc) and np.array_equal(_bits(gv), _bits(rv))

    with ThreadPoolExecutor(_host_jobs(4_000_000 * 64)) as ex:
        bad = [i for i, ok in ex.map(check, range(len(tens))) if not ok]
    assert not bad, bad
