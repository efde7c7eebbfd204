"""Host-side checks of the batch and tuning-cache entry points (no GPU
needed): every argument error is reported synchronously, before the library
touches the device, and the tuning cache round-trips through its text file."""
import ctypes
import os

import pytest

import paper_2005_10427_gb300 as qsd
from paper_2005_10427_gb300 import _capi

INVALID, UNSUPPORTED = 1, 2


@pytest.fixture(scope="module")
def L():
    qsd.build()
    return qsd.lib()


def items(plan, specs):
    arr = (_capi.BatchItem * len(specs))()
    for e, (nnz, stride, base) in zip(arr, specs):
        e.plan = plan.handle.value
        e.nnz = nnz
        e.in_ = base
        e.in_stride = stride
        e.out[0] = base + (1 << 36)
        e.out[1] = base + (2 << 36)
        e.out_stride = stride
    return arr


def create(L, arr, n, vb=0, opts=None):
    h = ctypes.c_void_p()
    o = opts if opts is not None else _capi.BatchOptions()
    return L.qsd_batch_create(arr, n, vb, ctypes.byref(o), ctypes.byref(h))


def test_batch_argument_errors(L):
    plan = qsd.Plan([10, 20, 30], [2, 1, 0])
    base = 1 << 40  # never dereferenced: every call below fails its checks first
    ok = items(plan, [(100, 100, base)])
    assert create(L, ok, 0) == INVALID
    assert create(L, None, 1) == INVALID
    assert create(L, ok, 1, vb=3) == INVALID
    assert create(L, ok, 1, vb=4) == INVALID  # values announced, no value buffers
    assert create(L, items(plan, [(100, 99, base)]), 1) == INVALID  # stride < nnz
    assert create(L, items(plan, [(-1, 100, base)]), 1) == INVALID
    null_plan = items(plan, [(100, 100, base)])
    null_plan[0].plan = None
    assert create(L, null_plan, 1) == INVALID
    overlap = items(plan, [(100, 100, base)])
    overlap[0].out[1] = base + 4 * 50  # inside the input rows
    assert create(L, overlap, 1) == INVALID
    huge = items(plan, [(1 << 29, 1 << 29, base), (1 << 29, 1 << 29, base + (1 << 38))])
    assert create(L, huge, 2) == UNSUPPORTED  # 2^30 entries in total
    for bad in [dict(tile=3000), dict(digit_bits=9), dict(local_capacity=5000),
                dict(chunk_tiles=300), dict(chunk_tiles=-1)]:
        o = _capi.BatchOptions()
        for k, v in bad.items():
            setattr(o, k, v)
        assert create(L, ok, 1, opts=o) == INVALID, bad
    out = ctypes.c_size_t()
    assert L.qsd_batch_workspace_bytes(None, ctypes.byref(out)) == INVALID
    assert L.qsd_batch_run(None, None, 0, None) == INVALID
    sel = ctypes.c_int()
    assert L.qsd_batch_result(None, 0, ctypes.byref(sel)) == INVALID
    L.qsd_batch_destroy(None)


def test_plan_tile_options(L):
    with pytest.raises(qsd.QsdError):
        qsd.Plan([4, 4], [1, 0], tile=3000)
    with pytest.raises(qsd.QsdError):
        qsd.Plan([4, 4], [1, 0], chunk_tiles=257)
    p = qsd.Plan([4, 4], [1, 0], tile=2048, chunk_tiles=4)
    assert p.options["tile"] == 2048


def test_tune_cache_file(L, tmp_path):
    good = os.path.join(tmp_path, "cache.txt")
    with open(good, "w") as f:
        f.write("n=3,vb=4,r=3,lgN4=80,P=6 7 2048 2048 16\n")
    qsd.tune_cache_load(good)
    saved = os.path.join(tmp_path, "saved.txt")
    qsd.tune_cache_save(saved)
    lines = open(saved).read().split("\n")
    assert "n=3,vb=4,r=3,lgN4=80,P=6 7 2048 2048 16" in lines
    bad = os.path.join(tmp_path, "bad.txt")
    with open(bad, "w") as f:
        f.write("n=3 7 2048 3000 16\n")  # tile 3000 is not a tile size
    with pytest.raises(qsd.QsdError):
        qsd.tune_cache_load(bad)
    with pytest.raises(qsd.QsdError):
        qsd.tune_cache_load(os.path.join(tmp_path, "missing.txt"))


def test_server_argument_errors(L):
    h = ctypes.c_void_p()
    assert L.qsd_server_create(None, ctypes.byref(h)) == INVALID
    for bad in [dict(memory_budget=0, val_bytes=8), dict(memory_budget=1 << 20, val_bytes=3),
                dict(memory_budget=1 << 20, val_bytes=8, max_batch=-1)]:
        o = _capi.ServerOptions()
        for k, v in bad.items():
            setattr(o, k, v)
        assert L.qsd_server_create(ctypes.byref(o), ctypes.byref(h)) == INVALID, bad
    o = _capi.ServerOptions()
    o.memory_budget, o.val_bytes, o.streams = 1 << 20, 8, 17
    assert L.qsd_server_create(ctypes.byref(o), ctypes.byref(h)) == UNSUPPORTED
    tid = ctypes.c_int()
    dims = (ctypes.c_int64 * 3)(4, 4, 4)
    assert L.qsd_server_add_tensor(None, 3, dims, None, None, 0, None, 0,
                                   ctypes.byref(tid)) == INVALID
    rid = ctypes.c_int64()
    assert L.qsd_server_submit(None, 0, None, 0.0, ctypes.byref(rid)) == INVALID
    n = ctypes.c_int()
    assert L.qsd_server_poll(None, None, 0, 0, ctypes.byref(n)) == INVALID
    assert L.qsd_server_release(None, 0) == INVALID
    L.qsd_server_destroy(None)
    t0 = L.qsd_server_clock()
    assert L.qsd_server_clock() >= t0 > 0
