"""Seeded synthetic COO tensors with the shapes of the benchmark workloads.

This module generates inputs only: it draws coordinates and values, removes
duplicate coordinates and sorts the result into the requested INPUT order.
It holds none of the transposition's own arithmetic and is shared by the
tests, the smoke check and the bench, which feed its output both to the CUDA
library and to the CPU oracle.

Recipe (the same for every workload; seeds are part of the workload name):

* per-mode index distributions: truncated Zipf(s) over ranks 1..n with
  P(rank k) proportional to k^-s, index = k - 1 (rank 1 is index 0), drawn by
  inverse CDF; or uniform over 0..n-1;
* draw about 1.5x the target count, drop duplicate coordinate tuples, top up
  with further draws until at least the target remains, then keep a seeded
  random subset of exactly the target size (so the result is "Zipf
  conditioned on distinctness": heavy heads saturate);
* sort lexicographically in the input mode order (identity by default);
* values: float32 N(0, 1), float64 U[0, 1) or float64 N(0, 1).

All arithmetic runs in torch on the given device (CPU for the tests' small
cases, CUDA for full-size bench inputs); a torch.Generator seeded with the
workload's seed makes each (device, seed) pair reproducible.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import torch


@dataclass
class CooTensor:
    coords: torch.Tensor          # int32, shape (r, nnz), sorted in input_order
    vals: torch.Tensor            # 1-D, float32 or float64
    dims: List[int]
    input_order: List[int] = field(default_factory=list)

    @property
    def order(self) -> int:
        return self.coords.shape[0]

    @property
    def nnz(self) -> int:
        return self.coords.shape[1]


def _bits(n: int) -> int:
    return 0 if n <= 1 else int(math.ceil(math.log2(n)))


_CDF_CACHE: dict = {}


def _zipf_cdf(n: int, s: float, device) -> torch.Tensor:
    key = (n, s, str(device))
    if key not in _CDF_CACHE:
        k = torch.arange(1, n + 1, dtype=torch.float64)
        w = k.pow(-s)
        cdf = torch.cumsum(w, 0)
        cdf = cdf / cdf[-1]
        _CDF_CACHE[key] = cdf.to(device)
        if len(_CDF_CACHE) > 64:
            _CDF_CACHE.pop(next(iter(_CDF_CACHE)))
    return _CDF_CACHE[key]


def _draw_mode(gen, count: int, n: int, dist, device) -> torch.Tensor:
    """count indices in [0, n) from dist: ('zipf', s) or ('uniform',)."""
    if dist[0] == "uniform":
        return torch.randint(0, n, (count,), generator=gen, device=device,
                             dtype=torch.int64)
    cdf = _zipf_cdf(n, float(dist[1]), device)
    u = torch.rand(count, generator=gen, device=device, dtype=torch.float64)
    idx = torch.searchsorted(cdf, u, right=True)
    return idx.clamp_(max=n - 1)


def _pack_words(cols: Sequence[torch.Tensor], widths: Sequence[int]):
    """Packs columns (MSD first) into a list of int64 words (<= 62 bits each)."""
    words, cur, used = [], None, 0
    for c, w in zip(cols, widths):
        if cur is not None and used + w > 62:
            words.append(cur)
            cur, used = None, 0
        cur = c.clone() if cur is None else (cur << w) | c
        used += w
    if cur is not None:
        words.append(cur)
    return words


def _sorted_unique_rows(words: List[torch.Tensor]) -> torch.Tensor:
    """Indices of the distinct rows of (words...), in lexicographic order."""
    n = words[0].numel()
    order = torch.arange(n, device=words[0].device)
    for w in reversed(words):  # LSD-first stable sorts
        _, o = torch.sort(w[order], stable=True)
        order = order[o]
    keep = torch.ones(n, dtype=torch.bool, device=order.device)
    if n > 1:
        same = torch.ones(n - 1, dtype=torch.bool, device=order.device)
        for w in words:
            ws = w[order]
            same &= ws[1:] == ws[:-1]
        keep[1:] = ~same
    return order[keep]


def gen_coo(dims: Sequence[int], nnz: int, dists, val_kind: str, seed: int,
            device="cpu", input_order: Optional[Sequence[int]] = None,
            oversample: float = 1.5) -> CooTensor:
    """Distinct random coordinates sorted in ``input_order``, with values.

    dists: one entry per mode, ('zipf', s) or ('uniform',). val_kind:
    'f32_normal', 'f64_uniform' or 'f64_normal'.
    """
    r = len(dims)
    dims = [int(d) for d in dims]
    if input_order is None:
        input_order = list(range(r))
    input_order = [int(m) for m in input_order]
    cap = 1
    for d in dims:
        cap *= d
    if nnz > cap:
        raise ValueError("more nonzeros than coordinates")
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    widths = [max(_bits(dims[m]), 1) for m in input_order]
    cols: List[torch.Tensor] = [torch.empty(0, dtype=torch.int64, device=device)
                                for _ in range(r)]
    want = int(math.ceil(nnz * oversample)) + 16
    while True:
        for m in range(r):
            cols[m] = torch.cat([cols[m], _draw_mode(gen, want, dims[m],
                                                     dists[m], device)])
        words = _pack_words([cols[m] for m in input_order], widths)
        keep = _sorted_unique_rows(words)
        cols = [c[keep] for c in cols]
        have = cols[0].numel()
        if have >= nnz:
            break
        want = max(int((nnz - have) * 2), 1024)
    if have > nnz:
        pick = torch.randperm(have, generator=gen, device=device)[:nnz]
        pick, _ = torch.sort(pick)
        cols = [c[pick] for c in cols]
    coords = torch.stack(cols).to(torch.int32)
    if val_kind == "f32_normal":
        vals = torch.randn(nnz, generator=gen, device=device, dtype=torch.float32)
    elif val_kind == "f64_uniform":
        vals = torch.rand(nnz, generator=gen, device=device, dtype=torch.float64)
    elif val_kind == "f64_normal":
        vals = torch.randn(nnz, generator=gen, device=device, dtype=torch.float64)
    else:
        raise ValueError(val_kind)
    return CooTensor(coords.contiguous(), vals, dims, input_order)


def random_coo(dims, nnz, seed, val_kind="f32_normal", device="cpu",
               dup_frac: float = 0.0, input_order=None, zipf: float = 0.0):
    """Small test tensor; with dup_frac > 0 some coordinates repeat.

    Duplicates are copies of existing tuples inserted next to them, so the
    result stays sorted in the input order; they exercise stability.
    """
    r = len(dims)
    dist = [("zipf", zipf) if zipf > 0 else ("uniform",)] * r
    cap = 1
    for d in dims:
        cap *= d
    base = min(nnz, cap)
    t = gen_coo(dims, base, dist, val_kind, seed, device, input_order)
    if dup_frac > 0 and t.nnz > 0:
        g = torch.Generator(device=device)
        g.manual_seed(int(seed) + 7919)
        extra = max(1, int(t.nnz * dup_frac))
        src = torch.randint(0, t.nnz, (extra,), generator=g, device=device)
        idx, _ = torch.sort(torch.cat([torch.arange(t.nnz, device=device), src]),
                            stable=True)
        coords = t.coords[:, idx].contiguous()
        if t.vals.dtype == torch.float32:
            vals = torch.randn(idx.numel(), generator=g, device=device)
        else:
            vals = torch.randn(idx.numel(), generator=g, device=device,
                               dtype=torch.float64)
        t = CooTensor(coords, vals, t.dims, t.input_order)
    return t


# ----------------------------------------------------------------------------
# Benchmark workloads (sizes and distributions as the configurations state).

WORKLOAD_3D_UNIFORM = dict(
    name="coo3d_1000^3_1M_uniform_f64", dims=[1000, 1000, 1000], nnz=1_000_000,
    dists=[("uniform",)] * 3, val_kind="f64_uniform", seed=1,
    perms=[(2, 1, 0)])

WORKLOAD_NELL2_LIKE = dict(
    name="coo3d_12000x9000x28000_76M_zipf1.1_f32",
    dims=[12000, 9000, 28000], nnz=76_000_000,
    dists=[("zipf", 1.1)] * 3, val_kind="f32_normal", seed=2,
    perms=[(0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)])

WORKLOAD_DELICIOUS_LIKE = dict(
    name="coo4d_4.8Mx1.7Mx1.8Mx1100_140M_zipf1.3_f64",
    dims=[4_800_000, 1_700_000, 1_800_000, 1100], nnz=140_000_000,
    dists=[("zipf", 1.3)] * 3 + [("uniform",)], val_kind="f64_normal", seed=3,
    perms=[p for p in __import__("itertools").permutations(range(4))
           if p != (0, 1, 2, 3)])


def scaled(workload: dict, nnz: int, seed_offset: int = 0) -> dict:
    """The same workload at a smaller nonzero count (dims unchanged)."""
    w = dict(workload)
    w["nnz"] = int(nnz)
    w["seed"] = workload["seed"] + seed_offset
    w["name"] = f"{workload['name']}@{nnz}"
    return w


def make(workload: dict, device="cpu") -> CooTensor:
    return gen_coo(workload["dims"], workload["nnz"], workload["dists"],
                   workload["val_kind"], workload["seed"], device)


def batch_workload(n_tensors: int = 256, seed: int = 4, nnz_lo: float = 1e3,
                   nnz_hi: float = 4e6, dim_lo: float = 100, dim_hi: float = 1e6,
                   zipf: float = 1.1):
    """Descriptions of the batched workload's tensors (no data yet).

    Order uniform in {3,4,5}; nnz log-uniform in [nnz_lo, nnz_hi]; each dim
    log-uniform in [dim_lo, dim_hi], redrawn until prod(dims) >= 8 * nnz;
    Zipf(zipf) coordinates, float32 values, identity input order, a random
    non-identity target permutation.
    """
    g = torch.Generator()
    g.manual_seed(seed)
    out = []
    for i in range(n_tensors):
        r = int(torch.randint(3, 6, (1,), generator=g))
        u = float(torch.rand(1, generator=g, dtype=torch.float64))
        nnz = int(round(math.exp(math.log(nnz_lo) + u * (math.log(nnz_hi) - math.log(nnz_lo)))))
        while True:
            us = torch.rand(r, generator=g, dtype=torch.float64)
            dims = [int(round(math.exp(math.log(dim_lo) + float(x) * (math.log(dim_hi) - math.log(dim_lo)))))
                    for x in us]
            if math.prod(dims) >= 8 * nnz:
                break
        while True:
            perm = tuple(int(x) for x in torch.randperm(r, generator=g))
            if perm != tuple(range(r)):
                break
        out.append(dict(name=f"batch{i}", dims=dims, nnz=nnz,
                        dists=[("zipf", zipf)] * r, val_kind="f32_normal",
                        seed=seed * 100003 + i, perm=perm))
    return out


def serving_workload(n_tensors: int = 64, n_requests: int = 10_000, rate: float = 2000.0,
                     seed: int = 5, nnz_lo: float = 1e4, nnz_hi: float = 5e7,
                     dim_lo: float = 100, dim_hi: float = 1e6, zipf: float = 1.2):
    """The serving workload: a resident pool and a Poisson request stream.

    Pool: n_tensors tensors, order uniform in {3,4}, nnz log-uniform in
    [nnz_lo, nnz_hi], each dim log-uniform in [dim_lo, dim_hi] (redrawn until
    prod(dims) >= 8 * nnz), Zipf(zipf) coordinates, float64 N(0,1) values,
    identity input order. Requests: exponential inter-arrival times at `rate`
    per second; each picks a pool tensor uniformly and a uniformly random
    non-identity target order. Returns (pool descriptions, [(arrival offset
    in seconds, tensor index, target order)]).
    """
    g = torch.Generator()
    g.manual_seed(seed)
    pool = []
    for i in range(n_tensors):
        r = int(torch.randint(3, 5, (1,), generator=g))
        u = float(torch.rand(1, generator=g, dtype=torch.float64))
        nnz = int(round(math.exp(math.log(nnz_lo) + u * (math.log(nnz_hi) - math.log(nnz_lo)))))
        while True:
            us = torch.rand(r, generator=g, dtype=torch.float64)
            dims = [int(round(math.exp(math.log(dim_lo) + float(x) * (math.log(dim_hi) -
                                                                       math.log(dim_lo)))))
                    for x in us]
            if math.prod(dims) >= 8 * nnz:
                break
        pool.append(dict(name=f"serve{i}", dims=dims, nnz=nnz, dists=[("zipf", zipf)] * r,
                         val_kind="f64_normal", seed=seed * 100003 + i))
    gaps = -torch.log1p(-torch.rand(n_requests, generator=g, dtype=torch.float64)) / rate
    times = torch.cumsum(gaps, 0)
    reqs = []
    for k in range(n_requests):
        i = int(torch.randint(0, n_tensors, (1,), generator=g))
        r = len(pool[i]["dims"])
        while True:
            perm = tuple(int(x) for x in torch.randperm(r, generator=g))
            if perm != tuple(range(r)):
                break
        reqs.append((float(times[k]), i, perm))
    return pool, reqs
