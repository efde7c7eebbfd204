"""The seeded generator: distinct coordinates, sorted in the input order,
reproducible per seed, in range, with the requested value types."""
import numpy as np
import torch

import synth


def _lex_sorted_strict(coords, order):
    c = coords.numpy()[list(order)]
    keys = np.lexsort(c[::-1])
    return np.array_equal(keys, np.arange(c.shape[1])) and (
        c.shape[1] < 2 or np.all(np.any(c[:, 1:] != c[:, :-1], axis=0)))


def test_distinct_sorted_reproducible():
    w = synth.scaled(synth.WORKLOAD_NELL2_LIKE, 20000)
    a = synth.make(w)
    b = synth.make(w)
    assert a.nnz == 20000 and a.coords.dtype == torch.int32
    assert torch.equal(a.coords, b.coords) and torch.equal(a.vals, b.vals)
    assert a.vals.dtype == torch.float32
    assert _lex_sorted_strict(a.coords, range(3))
    for m, d in enumerate(w["dims"]):
        assert int(a.coords[m].min()) >= 0 and int(a.coords[m].max()) < d
    # Zipf: index 0 is the most frequent value of each mode
    for m in range(3):
        cnt = torch.bincount(a.coords[m].long())
        assert int(cnt.argmax()) == 0


def test_wide_keys_and_input_order():
    w = synth.scaled(synth.WORKLOAD_DELICIOUS_LIKE, 5000)
    t = synth.make(w)
    assert t.vals.dtype == torch.float64 and _lex_sorted_strict(t.coords, range(4))
    t2 = synth.gen_coo([50, 60, 70], 3000, [("uniform",)] * 3, "f64_uniform", 9,
                       input_order=[2, 0, 1])
    assert _lex_sorted_strict(t2.coords, [2, 0, 1])


def test_duplicates_helper():
    t = synth.random_coo([5, 5, 5], 60, seed=1, dup_frac=0.5)
    c = t.coords.numpy()
    assert t.nnz == 60 + 30
    assert np.all(np.lexsort(c[::-1]) == np.arange(t.nnz))


def test_batch_workload_shapes():
    ws = synth.batch_workload(16)
    assert len(ws) == 16
    for w in ws:
        assert len(w["dims"]) in (3, 4, 5) and 1000 <= w["nnz"] <= 4_000_000
        assert np.prod([float(d) for d in w["dims"]]) >= 8 * w["nnz"]
        assert sorted(w["perm"]) == list(range(len(w["dims"])))
        assert tuple(w["perm"]) != tuple(range(len(w["dims"])))
