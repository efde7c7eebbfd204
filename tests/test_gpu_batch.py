"""GPU parity of batches (qsd_batch_*): every tensor of a batch must come out
bit for bit equal to the oracle's transposition of it, and to what a single
qsd_transpose call gives, whatever the mix of orders, sizes, permutations,
value widths and execution options in the batch."""
import itertools
import os

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


class Item:
    """One tensor of a batch: host arrays, device input, device double buffers."""

    def __init__(self, qsd, dims, nnz, seed, sigma, val_kind="f32_normal", zipf=1.1,
                 tau=None, dup=0.0, pad=0, top_k=0):
        if nnz:
            t = synth.random_coo(dims, nnz, seed, val_kind or "f32_normal", zipf=zipf,
                                 dup_frac=dup, input_order=tau)
            self.coords = t.coords.numpy()
            self.vals = None if val_kind is None else t.vals.numpy()
        else:
            self.coords = np.zeros((len(dims), 0), np.int32)
            self.vals = None if val_kind is None else np.zeros(
                0, np.float64 if val_kind == "f64_uniform" else np.float32)
        nnz = self.coords.shape[1]  # duplicates add entries
        self.dims, self.sigma, self.nnz = list(dims), tuple(sigma), nnz
        self.plan = qsd.Plan(dims, sigma, input_mode_order=tau, top_k=top_k)
        r = len(dims)
        width = nnz + pad  # pad > 0: row stride above nnz
        cin = torch.zeros((r, max(width, 1)), dtype=torch.int32, device="cuda")
        cin[:, :nnz] = torch.from_numpy(self.coords)
        self.cin = cin
        self.cout = [torch.full((r, max(width, 1)), -7, dtype=torch.int32, device="cuda")
                     for _ in range(2)]
        if self.vals is not None:
            vt = torch.from_numpy(self.vals)
            vin = torch.zeros(max(width, 1), dtype=vt.dtype, device="cuda")
            vin[:nnz] = vt
            self.vin = vin
            self.vout = [torch.zeros_like(vin) for _ in range(2)]
        else:
            self.vin, self.vout = None, None

    def entry(self):
        return (self.plan, self.cin, self.vin, self.cout, self.vout, self.nnz)

    def result(self, sel):
        c = self.cout[sel][:, :self.nnz].cpu().numpy()
        v = None if self.vout is None else self.vout[sel][:self.nnz].cpu().numpy()
        return c, v


def run_batch(qsd, items, **opts):
    b = qsd.Batch([it.entry() for it in items], **opts)
    ws = torch.empty(max(b.workspace_bytes(), 256), dtype=torch.uint8, device="cuda")
    b.run(ws)
    torch.cuda.synchronize()
    assert qsd.workspace_status(ws) == 0
    return b, ws


def check_against_oracle(items, b):
    for i, it in enumerate(items):
        gc, gv = it.result(b.result(i))
        rc, rv = oracle.transpose(it.coords, it.vals, it.sigma)
        bad = np.nonzero(np.any(gc != rc, axis=0))[0]
        assert bad.size == 0, f"item {i} sigma={it.sigma} nnz={it.nnz}: mismatch at {bad[:5]}"
        if it.vals is not None:
            u = np.uint64 if it.vals.dtype.itemsize == 8 else np.uint32
            assert np.array_equal(gv.view(u), rv.view(u)), f"item {i}: values differ"


def mixed_items(qsd, n, seed, val_kind="f32_normal", max_nnz=120_000):
    rng = np.random.default_rng(seed)
    sizes = [0, 1, 2, 33, 1000, 4095, 4096, 4097, 9000, 70_000]
    items = []
    for i in range(n):
        r = int(rng.integers(3, 6))
        nnz = sizes[i] if i < len(sizes) else int(np.exp(rng.uniform(np.log(200),
                                                                      np.log(max_nnz))))
        while True:
            dims = [int(np.exp(rng.uniform(np.log(8), np.log(3000)))) for _ in range(r)]
            if np.prod([float(d) for d in dims]) >= 8 * max(nnz, 1):
                break
        sigma = tuple(int(x) for x in rng.permutation(r))
        items.append(Item(qsd, dims, nnz, seed * 1000 + i, sigma, val_kind=val_kind))
    return items


def test_batch_matches_oracle_mixed(qsd):
    items = mixed_items(qsd, 40, seed=1)
    b, _ = run_batch(qsd, items)
    check_against_oracle(items, b)


@pytest.mark.parametrize("val_kind", ["f64_uniform", None])
def test_batch_value_widths(qsd, val_kind):
    items = mixed_items(qsd, 16, seed=2, val_kind=val_kind, max_nnz=50_000)
    b, _ = run_batch(qsd, items)
    check_against_oracle(items, b)


def test_batch_every_permutation_of_one_shape(qsd):
    # all 24 orderings of a 4-order tensor, including the identity (a copy),
    # in one batch: rounds of different lengths and pass counts mix
    dims = [40, 300, 25, 900]
    items = [Item(qsd, dims, 30_000, 7, s, zipf=1.2) for s in itertools.permutations(range(4))]
    b, _ = run_batch(qsd, items)
    check_against_oracle(items, b)


def test_batch_equals_single_calls(qsd):
    items = mixed_items(qsd, 24, seed=3)
    b, _ = run_batch(qsd, items)
    for i, it in enumerate(items):
        if it.nnz == 0:
            continue
        gc, gv = it.result(b.result(i))
        sc, sv = qsd.transpose(it.cin[:, :it.nnz].clone(),
                               None if it.vin is None else it.vin[:it.nnz].clone(), it.plan)
        assert np.array_equal(gc, sc.cpu().numpy())
        assert np.array_equal(gv.view(np.uint32), sv.cpu().numpy().view(np.uint32))


def test_batch_graph_replay_and_direct_launch(qsd):
    items = mixed_items(qsd, 12, seed=4)
    b, ws = run_batch(qsd, items)
    for _ in range(3):  # replays recompute the same results
        b.run(ws)
    torch.cuda.synchronize()
    check_against_oracle(items, b)
    d, _ = run_batch(qsd, items, graph=False)
    check_against_oracle(items, d)


def test_batch_strided_rows_and_duplicates(qsd):
    items = [Item(qsd, [30, 20, 10], 5000, 11, (2, 0, 1), dup=0.3, pad=37),
             Item(qsd, [64, 64, 64, 4], 20000, 12, (3, 1, 0, 2), dup=0.2, pad=5),
             Item(qsd, [9, 2000, 50], 60000, 13, (0, 2, 1), zipf=1.3, pad=1)]
    b, _ = run_batch(qsd, items)
    check_against_oracle(items, b)


def test_batch_non_identity_input_orders(qsd):
    items = [Item(qsd, [50, 60, 70], 40000, 21, (1, 2, 0), tau=(2, 0, 1)),
             Item(qsd, [50, 60, 70, 8], 30000, 22, (0, 3, 2, 1), tau=(3, 1, 0, 2))]
    b, _ = run_batch(qsd, items)
    check_against_oracle(items, b)


def test_batch_of_topk_plans(qsd):
    # Top-K-sadilla plans (Section 3.6) beside Quesadilla plans in one batch;
    # digit width 6 re-plans every tensor and keeps top_k
    items = [Item(qsd, [300, 40, 500, 60], 50000, 31, (2, 0, 3, 1), top_k=1),
             Item(qsd, [300, 40, 500, 60], 50000, 31, (2, 0, 3, 1)),
             Item(qsd, [80, 90, 70, 60, 5], 40000, 32, (4, 1, 0, 3, 2), top_k=2),
             Item(qsd, [2000, 3000, 100], 60000, 33, (0, 2, 1), top_k=1, dup=0.1)]
    for opts in ({}, dict(digit_bits=6)):
        b, _ = run_batch(qsd, items, **opts)
        check_against_oracle(items, b)


@pytest.mark.parametrize("opts", [dict(tile=2048), dict(tile=1024, chunk_tiles=3),
                                  dict(digit_bits=5, local_capacity=2048),
                                  dict(local_capacity=8192, chunk_tiles=1),
                                  dict(digit_bits=8, local_capacity=1024, chunk_tiles=16)])
def test_batch_execution_options(qsd, opts):
    items = mixed_items(qsd, 14, seed=5)
    b, _ = run_batch(qsd, items, **opts)
    check_against_oracle(items, b)


def test_batch_tuner_keeps_results(qsd, tmp_path):
    items = mixed_items(qsd, 10, seed=6, max_nnz=200_000)
    b, _ = run_batch(qsd, items)
    big = torch.empty(4 * b.workspace_bytes() + (64 << 20), dtype=torch.uint8, device="cuda")
    best = b.tune(big, reps=1)
    assert best["tile"] in (1024, 2048, 3584, 4096)
    assert best["digit_bits"] in (6, 7, 8)
    assert best["local_capacity"] in (1024, 2048, 4096, 8192)
    assert best["chunk_tiles"] in (1, 2, 4, 8)
    assert b.options()["tile"] == best["tile"]
    b.run(big)
    torch.cuda.synchronize()
    check_against_oracle(items, b)
    path = os.path.join(tmp_path, "tune.txt")
    qsd.tune_cache_save(path)
    qsd.tune_cache_load(path)
    # a new batch of the same shape picks the tuned options from the cache
    b2 = qsd.Batch([it.entry() for it in items], use_tuned=True)
    o = b2.options()
    assert (o["tile"], o["digit_bits"], o["local_capacity"], o["chunk_tiles"]) == \
        (best["tile"], best["digit_bits"], best["local_capacity"], best["chunk_tiles"])


def test_batch_workload_shape_scaled(qsd):
    # the batched workload's recipe (orders 3-5, log-uniform sizes and dims,
    # Zipf 1.1, identity input order, random non-identity target), 64
    # tensors of up to 200K entries, every result checked in full
    descs = synth.batch_workload(n_tensors=64, seed=4, nnz_hi=2e5)
    items = []
    for d in descs:
        items.append(Item(qsd, d["dims"], d["nnz"], d["seed"], d["perm"]))
    b, _ = run_batch(qsd, items)
    check_against_oracle(items, b)
