"""GPU parity: the CUDA path, called through the C ABI, must equal the CPU
oracle (a stable sort under the target-order lexicographic comparator) bit
for bit in coordinates and values. Values are moved, never computed, so the
tolerance is zero."""
import itertools

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


def run_gpu(qsd, coords, vals, dims, sigma, tau=None, **opts):
    plan = qsd.Plan(dims, sigma, input_mode_order=tau, **opts)
    c = torch.from_numpy(np.ascontiguousarray(coords)).cuda()
    v = None if vals is None else torch.from_numpy(np.ascontiguousarray(vals)).cuda()
    oc, ov = qsd.transpose(c, v, plan)
    torch.cuda.synchronize()
    assert qsd.get_async_status() == 0
    return oc.cpu().numpy(), (None if ov is None else ov.cpu().numpy())


def check(qsd, coords, vals, dims, sigma, tau=None, **opts):
    gc, gv = run_gpu(qsd, coords, vals, dims, sigma, tau, **opts)
    rc, rv = oracle.transpose(coords, vals, sigma)
    assert gc.shape == rc.shape
    bad = np.nonzero(np.any(gc != rc, axis=0))[0]
    assert bad.size == 0, f"sigma={sigma} first mismatch at {bad[:5]} of {rc.shape[1]}"
    if vals is not None:
        u = np.uint64 if vals.dtype.itemsize == 8 else np.uint32
        assert np.array_equal(gv.view(u), rv.view(u)), f"values differ for sigma={sigma}"


def tensor(dims, nnz, seed, val_kind="f32_normal", zipf=0.0, dup=0.0, tau=None):
    t = synth.random_coo(dims, nnz, seed, val_kind, zipf=zipf, dup_frac=dup, input_order=tau)
    return t.coords.numpy(), t.vals.numpy()


@pytest.mark.parametrize("r", [2, 3, 4])
def test_small_all_permutations(qsd, r):
    dims = [13, 7, 29, 5][:r]
    coords, vals = tensor(dims, 900, seed=r, dup=0.2)
    for sigma in itertools.permutations(range(r)):
        check(qsd, coords, vals, dims, sigma)


@pytest.mark.parametrize("nnz", [0, 1, 2, 31, 32, 33, 1023, 1024, 1025, 4095, 4096, 4097,
                                 8191, 8192, 8193, 20000])
def test_sizes_and_ragged_tails(qsd, nnz):
    dims = [60, 50, 70]
    coords, vals = tensor(dims, nnz, seed=nnz + 3, zipf=1.1) if nnz else \
        (np.zeros((3, 0), np.int32), np.zeros(0, np.float32))
    for sigma in [(0, 2, 1), (2, 1, 0), (1, 0, 2)]:
        check(qsd, coords, vals, dims, sigma)


def test_global_multi_tile_and_large_buckets(qsd):
    # Zipf heads give buckets far above the shared-memory capacity, so both the
    # block-local sort and the segmented digit passes run in one group.
    dims = [300, 2000, 3000]
    coords, vals = tensor(dims, 400_000, seed=11, zipf=1.1)
    for sigma in itertools.permutations(range(3)):
        check(qsd, coords, vals, dims, sigma)


@pytest.mark.parametrize("val_kind", ["f32_normal", "f64_uniform", None])
def test_value_widths(qsd, val_kind):
    dims = [100, 80, 90]
    coords, vals = tensor(dims, 50_000, seed=5, val_kind=val_kind or "f32_normal", zipf=1.2)
    if val_kind is None:
        vals = None
    for sigma in [(0, 2, 1), (1, 2, 0)]:
        check(qsd, coords, vals, dims, sigma)


def test_payload_bits_preserved(qsd):
    dims = [50, 40, 30]
    coords, _ = tensor(dims, 30_000, seed=8, zipf=1.0)
    rng = np.random.default_rng(0)
    raw = rng.integers(0, 2**63, size=coords.shape[1], dtype=np.uint64)
    raw[::7] = 0x7FF8000000000001  # NaN payload
    raw[1::7] = 0x8000000000000000  # -0.0
    check(qsd, coords, raw.view(np.float64), dims, (2, 0, 1))
    raw32 = (raw & 0xFFFFFFFF).astype(np.uint32)
    check(qsd, coords, raw32.view(np.float32), dims, (1, 0, 2))


def test_duplicates_are_stable(qsd):
    dims = [6, 5, 7, 4]
    coords, vals = tensor(dims, 600, seed=21, dup=3.0)
    assert coords.shape[1] > 600
    for sigma in itertools.permutations(range(4)):
        check(qsd, coords, vals, dims, sigma)
    # many duplicates across several tiles and buckets
    coords, vals = tensor([40, 30, 20], 20_000, seed=22, zipf=1.3, dup=1.5)
    for sigma in [(0, 2, 1), (2, 1, 0)]:
        check(qsd, coords, vals, [40, 30, 20], sigma)


def test_non_identity_input_order(qsd):
    dims = [70, 40, 90, 11]
    for tau in [(2, 0, 3, 1), (3, 2, 1, 0)]:
        coords, vals = tensor(dims, 30_000, seed=31, zipf=1.1, tau=tau)
        rng = np.random.default_rng(1)
        for sigma in [tuple(int(x) for x in rng.permutation(4)) for _ in range(6)]:
            check(qsd, coords, vals, dims, sigma, tau=tau)


def test_wide_keys_over_32_and_64_bits(qsd):
    dims = [1 << 20, 1 << 21, 1 << 22, 1 << 20, 1 << 19]  # 102 packed bits
    coords, vals = tensor(dims, 60_000, seed=41, val_kind="f64_normal", zipf=1.05)
    for sigma in [(4, 3, 2, 1, 0), (2, 4, 0, 1, 3), (0, 4, 3, 2, 1), (1, 0, 4, 3, 2)]:
        check(qsd, coords, vals, dims, sigma)


def test_unit_modes_and_degenerate_keys(qsd):
    dims = [1, 9, 1, 7]
    coords, vals = tensor(dims, 50, seed=3)
    for sigma in itertools.permutations(range(4)):
        check(qsd, coords, vals, dims, sigma)
    # one giant bucket: every entry shares the prefix coordinate
    dims = [1, 500, 400]
    coords, vals = tensor(dims, 60_000, seed=4, zipf=0.8)
    check(qsd, coords, vals, dims, (0, 2, 1))
    # every bucket has one entry
    dims = [70_000, 3, 3]
    c = np.stack([np.arange(70_000), np.arange(70_000) % 3, np.arange(70_000) % 2]).astype(np.int32)
    check(qsd, c, np.arange(70_000, dtype=np.float32), dims, (0, 2, 1))


@pytest.mark.parametrize("digit_bits", [1, 3, 5, 7, 8])
def test_digit_widths(qsd, digit_bits):
    dims = [200, 300, 400]
    coords, vals = tensor(dims, 100_000, seed=50 + digit_bits, zipf=1.1)
    for sigma in [(0, 2, 1), (2, 0, 1)]:
        check(qsd, coords, vals, dims, sigma, digit_bits=digit_bits)


@pytest.mark.parametrize("tile,chunk_tiles", [(1024, 8), (2048, 3), (3584, 8), (3584, 1),
                                              (4096, 8), (4096, 16)])
def test_tile_sizes_and_chunk_lengths(qsd, tile, chunk_tiles):
    # ragged tiles and chunks inside large Zipf buckets and a global group
    dims = [40, 3000, 700]
    coords, vals = tensor(dims, 150_000, seed=tile + chunk_tiles, zipf=1.1)
    for sigma in [(0, 2, 1), (2, 1, 0)]:
        check(qsd, coords, vals, dims, sigma, tile=tile, chunk_tiles=chunk_tiles)


@pytest.mark.parametrize("extra", [0, 1, 21, 40])
def test_many_chunk_groups_with_ragged_parts(qsd, extra):
    # a whole tensor of more than 16 chunk groups takes the group prefix and
    # the four-part offset scan: 17 full groups of 64 one-tile chunks, then
    # `extra` chunks and a ragged last one (last group ending inside part 0,
    # 1 or 2 of its four 16-chunk parts)
    dims = [5000, 60000, 9]
    nnz = (17 * 64 + extra) * 1024 + 77
    coords, vals = tensor(dims, nnz, seed=extra + 5, zipf=1.1)
    for sigma in [(1, 0, 2), (2, 1, 0)]:
        check(qsd, coords, vals, dims, sigma, tile=1024, chunk_tiles=1)


@pytest.mark.parametrize("r", [3, 4])
def test_global_groups_give_the_same_result(qsd, r):
    # groups with a prefix run as global sorts by (prefix, key)
    dims = [30, 200, 50, 7][:r]
    coords, vals = tensor(dims, 60_000, seed=70 + r, zipf=1.2, dup=0.05)
    for sigma in itertools.permutations(range(r)):
        check(qsd, coords, vals, dims, sigma, global_groups=True)


@pytest.mark.parametrize("r", [3, 4, 5])
def test_topk_sadilla_plans(qsd, r):
    # Section 3.6: Quesadilla to the first K target modes, then a complete
    # sort of every bucket by the rest; the same result for every K
    rng = np.random.default_rng(100 + r)
    dims = [int(x) for x in rng.integers(20, 3000, size=r)]
    coords, vals = tensor(dims, 120_000, seed=100 + r, zipf=1.0, dup=0.1)
    sigmas = [tuple(int(x) for x in rng.permutation(r)) for _ in range(5)]
    for sigma in sigmas:
        for K in range(1, r - 1):
            check(qsd, coords, vals, dims, sigma, top_k=K)
    check(qsd, coords, vals, dims, sigmas[0], top_k=1, global_groups=True)
    check(qsd, coords, vals, dims, sigmas[1], top_k=1, local_capacity=1024)


def test_plan_tuner_result_and_options(qsd):
    dims = [300, 2000, 3000]
    coords, vals = tensor(dims, 300_000, seed=81, zipf=1.1)
    sigma = (0, 2, 1)
    plan = qsd.Plan(dims, sigma)
    c = torch.from_numpy(coords).cuda()
    v = torch.from_numpy(vals).cuda()
    tuned, ms, opts = qsd.tune_plan(plan, c, v, reps=1)
    assert ms > 0
    assert opts["digit_bits"] in (5, 6, 7, 8) and opts["tile"] in (0, 2048, 3584, 4096)
    assert opts["global_groups"] in (0, 1) and opts["chunk_tiles"] in (1, 2, 4)
    assert opts["top_k"] in (0, 1)
    assert torch.equal(c.cpu(), torch.from_numpy(coords))  # the input is left alone
    gc, gv = qsd.transpose(c.clone(), v.clone(), tuned)
    rc, rv = oracle.transpose(coords, vals, sigma)
    assert np.array_equal(gc.cpu().numpy(), rc)
    assert np.array_equal(gv.cpu().numpy().view(np.uint32), rv.view(np.uint32))


@pytest.mark.parametrize("cap", [1024, 2048, 4096, 8192])
def test_local_capacities(qsd, cap):
    dims = [3000, 500, 700]
    coords, vals = tensor(dims, 200_000, seed=60, zipf=1.1)
    for sigma in [(0, 2, 1), (0, 1, 2), (1, 0, 2)]:
        check(qsd, coords, vals, dims, sigma, local_capacity=cap)


@pytest.mark.parametrize("cap", [1024, 2048, 4096])
def test_tiny_buckets_ranked_by_counting(qsd, cap):
    # Zipf prefix coordinates: a few large buckets (the radix passes or the
    # digit passes), then thousands of buckets of a few entries, whose batches
    # are ranked by counting; packed keys of 36 bits (64-bit counting keys up
    # to capacity 2048, the radix passes above), of 4 bits with many equal
    # keys inside a bucket, and of 24 bits; duplicate coordinates keep their
    # input order.
    cases = [([20000, 4, 1 << 18, 1 << 18], (0, 3, 2, 1)),
             ([20000, 50, 3, 3], (0, 3, 2, 1)),
             ([30000, 1 << 12, 1 << 12, 7], (0, 2, 1, 3))]
    for i, (dims, sigma) in enumerate(cases):
        coords, vals = tensor(dims, 150_000, seed=90 + i, zipf=0.9, dup=0.2)
        check(qsd, coords, vals, dims, sigma, local_capacity=cap)


def test_no_skip_plan(qsd):
    dims = [50, 60, 70]
    coords, vals = tensor(dims, 40_000, seed=70, zipf=1.1)
    for sigma in [(0, 1, 2), (0, 2, 1), (2, 1, 0)]:
        check(qsd, coords, vals, dims, sigma, no_skip=True)


def test_validate_reports_bad_input(qsd):
    dims = [10, 10, 10]
    coords, vals = tensor(dims, 500, seed=1)
    plan = qsd.Plan(dims, (2, 1, 0), validate=True)
    c = torch.from_numpy(coords).cuda()
    qsd.transpose(c, torch.from_numpy(vals).cuda(), plan)
    assert qsd.get_async_status() == 0
    bad = coords.copy()
    bad[:, [10, 400]] = bad[:, [400, 10]]  # breaks the input order
    qsd.transpose(torch.from_numpy(bad).cuda(), torch.from_numpy(vals).cuda(), plan)
    assert qsd.get_async_status() == 5
    oob = coords.copy()
    oob[1, 7] = 10
    qsd.transpose(torch.from_numpy(oob).cuda(), torch.from_numpy(vals).cuda(), plan)
    assert qsd.get_async_status() == 6
    assert qsd.get_async_status() == 0  # read clears


def test_transpose_host_end_to_end(qsd):
    dims = [300, 200, 100]
    coords, vals = tensor(dims, 120_000, seed=80, zipf=1.1)
    plan = qsd.Plan(dims, (2, 0, 1))
    n = coords.shape[1]
    hc = torch.from_numpy(coords).pin_memory()
    hv = torch.from_numpy(vals).pin_memory()
    oc = torch.empty_like(hc).pin_memory()
    ov = torch.empty_like(hv).pin_memory()
    cb = [torch.empty((3, n), dtype=torch.int32, device="cuda") for _ in range(2)]
    vb = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(2)]
    ws = torch.empty(plan.workspace_bytes(n), dtype=torch.uint8, device="cuda")
    qsd.transpose_host(hc, hv, plan, cb, vb, ws, oc, ov)
    rc, rv = oracle.transpose(coords, vals, (2, 0, 1))
    assert np.array_equal(oc.numpy(), rc) and np.array_equal(ov.numpy(), rv)


def test_transpose_host_async_on_two_streams(qsd):
    # consecutive asynchronous calls alternate between two streams, each with
    # its own device buffers and workspace; every result equals the oracle's
    dims = [300, 200, 100]
    coords, vals = tensor(dims, 90_000, seed=81, zipf=1.1)
    n = coords.shape[1]
    hc = torch.from_numpy(coords).pin_memory()
    hv = torch.from_numpy(vals).pin_memory()
    sigmas = [(2, 0, 1), (0, 2, 1), (1, 2, 0), (2, 1, 0), (1, 0, 2), (0, 2, 1)]
    plans = [qsd.Plan(dims, sg) for sg in sigmas]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    cbs = [[torch.empty((3, n), dtype=torch.int32, device="cuda") for _ in range(2)] for _ in range(2)]
    vbs = [[torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(2)] for _ in range(2)]
    wss = [torch.empty(max(p.workspace_bytes(n) for p in plans), dtype=torch.uint8, device="cuda")
           for _ in range(2)]
    outs = [(torch.empty_like(hc).pin_memory(), torch.empty_like(hv).pin_memory()) for _ in sigmas]
    for k, (p, (oc, ov)) in enumerate(zip(plans, outs)):
        i = k % 2  # a stream's calls reuse its buffers in stream order
        qsd.transpose_host_async(hc, hv, p, cbs[i], vbs[i], wss[i], oc, ov, streams[i])
    for i in range(2):
        assert qsd.workspace_status(wss[i], streams[i]) == 0
    for sg, (oc, ov) in zip(sigmas, outs):
        rc, rv = oracle.transpose(coords, vals, sg)
        assert np.array_equal(oc.numpy(), rc) and np.array_equal(ov.numpy(), rv), sg


def test_repeated_calls_reuse_workspace(qsd):
    dims = [500, 400, 300]
    coords, vals = tensor(dims, 150_000, seed=90, zipf=1.1)
    plan = qsd.Plan(dims, (0, 2, 1))
    n = coords.shape[1]
    ws = torch.empty(plan.workspace_bytes(n), dtype=torch.uint8, device="cuda")
    rc, rv = oracle.transpose(coords, vals, (0, 2, 1))
    for _ in range(3):
        cb = [torch.from_numpy(coords).cuda(), torch.empty((3, n), dtype=torch.int32, device="cuda")]
        vb = [torch.from_numpy(vals).cuda(), torch.empty(n, dtype=torch.float32, device="cuda")]
        sel = qsd.transpose_buffers(cb, vb, 0, n, plan, ws)
        assert qsd.workspace_status(ws) == 0
        assert np.array_equal(cb[sel].cpu().numpy(), rc)
        assert np.array_equal(vb[sel].cpu().numpy(), rv)


def test_out_of_place_keeps_input(qsd):
    dims = [400, 300, 200]
    coords, vals = tensor(dims, 100_000, seed=95, zipf=1.1)
    n = coords.shape[1]
    ic = torch.from_numpy(coords).cuda()
    iv = torch.from_numpy(vals).cuda()
    cb = [torch.empty((3, n), dtype=torch.int32, device="cuda") for _ in range(2)]
    vb = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(2)]
    for sigma in [(0, 1, 2), (0, 2, 1), (1, 0, 2), (2, 1, 0), (1, 2, 0)]:
        plan = qsd.Plan(dims, sigma)
        ws = torch.empty(plan.workspace_bytes(n), dtype=torch.uint8, device="cuda")
        sel = qsd.transpose_from(ic, iv, cb, vb, n, plan, ws)
        assert qsd.workspace_status(ws) == 0
        rc, rv = oracle.transpose(coords, vals, sigma)
        assert np.array_equal(cb[sel].cpu().numpy(), rc), sigma
        assert np.array_equal(vb[sel].cpu().numpy(), rv), sigma
        assert np.array_equal(ic.cpu().numpy(), coords) and np.array_equal(iv.cpu().numpy(), vals)


def _key_index_groups(qsd, dims, sigma, tau=None):
    return [g["key_index"] for g in qsd.Plan(dims, sigma, input_mode_order=tau,
                                              key_index=True).info()["groups"]]


@pytest.mark.parametrize("r", [2, 3, 4, 5])
def test_key_index_every_permutation(qsd, r):
    # groups without a prefix sort (packed key, entry index) rows and gather
    # the entries once at the end; a small capacity keeps the digit passes in
    # play at this size
    dims = [300, 2000, 3000, 40, 9][:r]
    coords, vals = tensor(dims, 60_000, seed=40 + r, zipf=1.1, dup=0.05)
    used = 0
    for sigma in itertools.permutations(range(r)):
        used += sum(_key_index_groups(qsd, dims, sigma))
        check(qsd, coords, vals, dims, sigma, key_index=True, local_capacity=1024)
    assert used > 0


@pytest.mark.parametrize("nnz", [1, 3, 4, 5, 4097, 8193, 70001])
def test_key_index_sizes_and_tails(qsd, nnz):
    dims = [70, 90, 60]
    coords, vals = tensor(dims, nnz, seed=nnz + 5, zipf=1.1)
    for sigma in [(2, 1, 0), (1, 2, 0), (1, 0, 2)]:
        check(qsd, coords, vals, dims, sigma, key_index=True, local_capacity=1024)


@pytest.mark.parametrize("val_kind", ["f32_normal", "f64_uniform", None])
def test_key_index_value_widths_and_key_words(qsd, val_kind):
    # 20-, 40- and 60-bit keys: one and two key words; an 80-bit key stays in
    # whole-entry form
    for dims, sigma in [([1000, 1000, 1000], (2, 1, 0)),
                        ([1 << 20, 1 << 20, 1 << 20], (2, 1, 0)),
                        ([1 << 20] * 4, (3, 2, 1, 0)),
                        ([1 << 20] * 5, (4, 3, 2, 1, 0))]:
        coords, vals = tensor(dims, 50_000, seed=sum(dims) % 1000, val_kind=val_kind or
                              "f32_normal", zipf=1.2)
        if val_kind is None:
            vals = None
        check(qsd, coords, vals, dims, sigma, key_index=True, local_capacity=1024)


def test_key_index_duplicates_and_input_orders(qsd):
    dims = [40, 30, 50, 20]
    for tau in [None, (2, 0, 3, 1)]:
        coords, vals = tensor(dims, 40_000, seed=77, zipf=1.0, dup=0.3, tau=tau)
        for sigma in [(3, 2, 1, 0), (1, 3, 0, 2), (2, 0, 3, 1), (0, 3, 2, 1)]:
            check(qsd, coords, vals, dims, sigma, tau=tau, key_index=True, local_capacity=1024)


def test_key_index_multi_group_plans(qsd):
    # a global group in (key, index) form followed by bucketed groups
    dims = [4800, 1700, 1800, 110]
    coords, vals = tensor(dims, 300_000, seed=91, val_kind="f64_uniform", zipf=1.3)
    for sigma in [(1, 0, 3, 2), (2, 0, 3, 1), (3, 0, 2, 1), (1, 2, 3, 0), (3, 2, 1, 0)]:
        check(qsd, coords, vals, dims, sigma, key_index=True)


@pytest.mark.parametrize("first", [1, 3, 5, 6, 7])
def test_first_digit_widths(qsd, first):
    # a narrower least significant digit, the rest of the key split evenly
    dims = [300, 2000, 3000, 1100]
    coords, vals = tensor(dims, 120_000, seed=50 + first, val_kind="f64_uniform", zipf=1.2,
                          dup=0.05)
    for sigma in [(1, 2, 3, 0), (3, 0, 1, 2), (0, 3, 2, 1), (2, 1, 0, 3), (1, 3, 0, 2)]:
        check(qsd, coords, vals, dims, sigma, first_digit_bits=first, local_capacity=1024)
        check(qsd, coords, vals, dims, sigma, first_digit_bits=first, key_index=True,
              local_capacity=1024)


@pytest.mark.parametrize("opts", [{}, {"key_index": True}, {"global_groups": True}])
def test_unaligned_rows_and_odd_strides(qsd, opts):
    # rows that are not 16-byte aligned (odd row strides, buffers starting one
    # element into an allocation) take the scalar paths of the vectorised
    # kernels (boundary count, histograms, pack, gather, copies)
    dims = [300, 2000, 500, 40]
    coords, vals = tensor(dims, 90_001, seed=71, val_kind="f64_uniform", zipf=1.1)
    r, n = coords.shape
    stride = n + 3
    for sigma in [(0, 2, 1, 3), (3, 2, 1, 0), (1, 0, 3, 2), (0, 1, 2, 3)]:
        plan = qsd.Plan(dims, sigma, local_capacity=1024, **opts)
        big_in = torch.zeros(r * stride + 1, dtype=torch.int32, device="cuda")
        cin = big_in[1:].view(r, stride)[:, :n]
        cin.copy_(torch.from_numpy(coords).cuda())
        vin = torch.zeros(n + 1, dtype=torch.float64, device="cuda")[1:]
        vin.copy_(torch.from_numpy(vals).cuda())
        outs = [torch.zeros(r * stride + 1, dtype=torch.int32, device="cuda")[1:].view(r, stride)
                for _ in range(2)]
        vouts = [torch.zeros(n + 1, dtype=torch.float64, device="cuda")[1:] for _ in range(2)]
        ws = torch.empty(plan.workspace_bytes(n), dtype=torch.uint8, device="cuda")
        sel = qsd.transpose_from(cin, vin, outs, vouts, n, plan, ws)
        assert qsd.workspace_status(ws) == 0
        rc, rv = oracle.transpose(coords, vals, sigma)
        assert np.array_equal(outs[sel][:, :n].cpu().numpy(), rc), (sigma, opts)
        assert np.array_equal(vouts[sel].cpu().numpy().view(np.uint64), rv.view(np.uint64))
