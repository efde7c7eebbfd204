"""Host-side tests of the C library (no GPU needed): every symbol declared in
include/qsd.h is exported, argument errors are reported synchronously, and
the planner behind qsd_plan matches the oracle planner call for call."""
import ctypes
import itertools
import os
import re

import numpy as np
import pytest

import paper_2005_10427_gb300 as qsd
from paper_2005_10427_gb300 import _capi
from oracle import plan as OP

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    qsd.build()
    return qsd.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "qsd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qsd_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    syms = declared_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(L, s), s
    assert {n for n, _, _ in _capi.SIGNATURES} == set(syms)
    assert L.qsd_version().decode().startswith("qsd")


def test_status_strings(L):
    for code, name in _capi.STATUS_NAMES.items():
        assert L.qsd_status_string(code).decode() == name


def test_plan_argument_errors(L):
    with pytest.raises(qsd.QsdError) as e:
        qsd.Plan([4, 4, 4], [0, 0, 1])
    assert e.value.status == 1
    with pytest.raises(qsd.QsdError):
        qsd.Plan([4, 0, 4], [2, 1, 0])
    with pytest.raises(qsd.QsdError):
        qsd.Plan([4, 4, 4], [2, 1, 0], input_mode_order=[0, 1, 1])
    with pytest.raises(qsd.QsdError) as e:
        qsd.Plan([2] * 9, list(range(9)))
    assert e.value.status == 2
    with pytest.raises(qsd.QsdError):
        qsd.Plan([4, 4], [1, 0], digit_bits=9)
    with pytest.raises(qsd.QsdError):
        qsd.Plan([4, 4], [1, 0], local_capacity=3000)


def test_transpose_argument_errors_without_gpu(L):
    p = qsd.Plan([4, 4], [1, 0])
    c = _capi.Coords()
    c.stride = 10
    c.selector = 0
    # null buffers with nnz > 0
    st = L.qsd_transpose_ws(ctypes.byref(c), None, 10, p.handle, None, 0, None)
    assert st == 1
    c.selector = 2
    assert L.qsd_transpose_ws(ctypes.byref(c), None, 0, p.handle, None, 0, None) == 1
    c.selector = 0
    assert L.qsd_transpose_ws(ctypes.byref(c), None, -1, p.handle, None, 0, None) == 1
    assert L.qsd_transpose_ws(ctypes.byref(c), None, 1 << 30, p.handle, None, 0, None) == 2
    out = ctypes.c_size_t()
    assert L.qsd_workspace_bytes(p.handle, -5, ctypes.byref(out)) == 1


def test_host_buffer_calls_check_arguments_before_device_work(L):
    # both host-buffer calls report argument errors before any copy or kernel
    # (device pointers here are never dereferenced)
    p = qsd.Plan([4, 4], [1, 0])
    c = _capi.Coords()
    c.stride = 10
    c.selector = 0
    host = (ctypes.c_int32 * 20)()
    for fn in (L.qsd_transpose_host, L.qsd_transpose_host_async):
        # null device buffers
        assert fn(host, 10, None, host, 10, None, 10, p.handle, ctypes.byref(c), None,
                  None, 0, None) == 1
        c.buf[0], c.buf[1] = 1 << 36, 2 << 36
        # null host arrays, host strides shorter than nnz
        assert fn(None, 10, None, host, 10, None, 10, p.handle, ctypes.byref(c), None,
                  None, 0, None) == 1
        assert fn(host, 10, None, None, 10, None, 10, p.handle, ctypes.byref(c), None,
                  None, 0, None) == 1
        assert fn(host, 9, None, host, 10, None, 10, p.handle, ctypes.byref(c), None,
                  None, 0, None) == 1
        assert fn(host, 10, None, host, 9, None, 10, p.handle, ctypes.byref(c), None,
                  None, 0, None) == 1
        # values declared but no host value arrays
        v = _capi.Values()
        v.buf[0], v.buf[1] = 3 << 36, 4 << 36
        v.elem_bytes = 4
        assert fn(host, 10, None, host, 10, None, 10, p.handle, ctypes.byref(c), ctypes.byref(v),
                  None, 0, None) == 1
        c.buf[0] = c.buf[1] = None


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5])
def test_planner_matches_oracle_planner(L, r):
    rng = np.random.default_rng(r)
    taus = [tuple(range(r))] + [tuple(int(x) for x in rng.permutation(r)) for _ in range(2)]
    for tau in taus:
        for sigma in itertools.permutations(range(r)):
            p = qsd.Plan([7] * r, sigma, input_mode_order=tau)
            inf = p.info()
            want = OP.quesadilla_calls(sigma, tau)
            assert inf["calls"] == want, (tau, sigma)
            assert inf["num_calls"] == OP.b(tau, sigma)
            assert inf["num_bucketed_calls"] == sum(1 for pre, _ in want if pre)
            # groups: consecutive calls sharing a prefix, keys most significant first
            groups = []
            for pre, mode in want:
                if groups and groups[-1][0] == pre:
                    groups[-1][1].insert(0, mode)
                else:
                    groups.append((pre, [mode]))
            assert [(g["prefix"], g["keys"]) for g in inf["groups"]] == \
                [(pre, tuple(k)) for pre, k in groups]


def _groups_of(calls):
    # consecutive calls sharing a prefix, keys most significant first
    groups = []
    for pre, mode in calls:
        if groups and groups[-1][0] == pre:
            groups[-1][1].insert(0, mode)
        else:
            groups.append((pre, [mode]))
    return [(pre, tuple(k)) for pre, k in groups]


@pytest.mark.parametrize("r", [3, 4, 5])
def test_topk_planner_matches_oracle_steps(L, r):
    rng = np.random.default_rng(10 + r)
    taus = [tuple(range(r)), tuple(int(x) for x in rng.permutation(r))]
    for tau in taus:
        for sigma in itertools.permutations(range(r)):
            for K in range(r + 2):
                inf = qsd.Plan([7] * r, sigma, input_mode_order=tau, top_k=K).info()
                calls, final = OP.topk_steps(sigma, tau, K if 0 < K < r - 1 else r)
                assert inf["calls"] == calls, (tau, sigma, K)
                want = _groups_of(calls) + ([final] if final else [])
                assert [(g["prefix"], g["keys"]) for g in inf["groups"]] == want, (tau, sigma, K)


def test_topk_and_digit_limits(L):
    with pytest.raises(qsd.QsdError) as e:
        qsd.Plan([4, 4, 4], (2, 1, 0), top_k=-1)
    assert e.value.status == 1
    with pytest.raises(qsd.QsdError) as e:
        qsd.Plan([4, 4, 4], (2, 1, 0), top_k=9)
    assert e.value.status == 1
    # 8 modes of 31 bits in one group: 248 bits, 31 passes of 8 bits, but
    # more passes than a group holds at 7 bits
    qsd.Plan([2**31 - 1] * 8, tuple(range(8)), no_skip=True)
    with pytest.raises(qsd.QsdError) as e:
        qsd.Plan([2**31 - 1] * 8, tuple(range(8)), no_skip=True, digit_bits=7)
    assert e.value.status == 2
    # no_skip (the full radix sort) takes precedence over top_k
    inf = qsd.Plan([9] * 4, (2, 0, 3, 1), top_k=1, no_skip=True).info()
    assert inf["num_calls"] == 4 and [(g["prefix"], g["keys"]) for g in inf["groups"]] == \
        [((), (2, 0, 3, 1))]
    # Top-1 of (2, 0, 3, 1) from the identity: Quesadilla's calls to
    # (2, 0, 1, 3), then every bucket of mode 2 sorted by (0, 3, 1)
    inf = qsd.Plan([9] * 4, (2, 0, 3, 1), top_k=1).info()
    assert inf["calls"] == [((), 2)]
    assert [(g["prefix"], g["keys"]) for g in inf["groups"]] == [((), (2,)), ((2,), (0, 3, 1))]


def test_planner_high_order_sampled(L):
    rng = np.random.default_rng(99)
    for r in (6, 7, 8):
        for _ in range(40):
            tau = tuple(int(x) for x in rng.permutation(r))
            sigma = tuple(int(x) for x in rng.permutation(r))
            assert qsd.Plan([3] * r, sigma, input_mode_order=tau).calls == \
                OP.quesadilla_calls(sigma, tau)


def test_fig4_through_the_c_abi(L):
    for r, want in ((3, [1, 3, 2]), (4, [1, 6, 11, 6]), (5, [1, 10, 35, 50, 24])):
        hist = [0] * r
        for sigma in itertools.permutations(range(r)):
            hist[qsd.Plan([5] * r, sigma).info()["num_calls"]] += 1
        assert hist == want


def test_key_bits_and_digit_passes(L):
    # 12000 x 9000 x 28000: widths 14, 14, 15
    cases = {(0, 2, 1): [((0,), (2,), 15)], (1, 0, 2): [((), (1,), 14)],
             (1, 2, 0): [((), (1, 2), 29)], (2, 1, 0): [((), (2, 1), 29)],
             (2, 0, 1): [((), (2,), 15)]}
    for sigma, want in cases.items():
        inf = qsd.Plan([12000, 9000, 28000], sigma).info()
        got = [(g["prefix"], g["keys"], g["key_bits"]) for g in inf["groups"]]
        assert got == want
        for g in inf["groups"]:
            assert g["passes"] == -(-g["key_bits"] // 8)
    inf = qsd.Plan([4_800_000, 1_700_000, 1_800_000, 1100], (1, 0, 3, 2)).info()
    assert [(g["prefix"], g["keys"], g["key_bits"]) for g in inf["groups"]] == \
        [((), (1,), 21), ((1, 0), (3,), 11)]
    inf = qsd.Plan([4_800_000, 1_700_000, 1_800_000, 1100], (3, 2, 1, 0)).info()
    assert inf["groups"][0]["key_bits"] == 11 + 21 + 21 and inf["groups"][0]["passes"] == 7
    # modes of size 1 contribute no bits; a key of only such modes needs no pass
    inf = qsd.Plan([1, 5, 1], (2, 0, 1)).info()
    assert inf["groups"][0]["key_bits"] == 0 and inf["groups"][0]["passes"] == 0
    inf = qsd.Plan([5, 5], (1, 0), digit_bits=1).info()
    assert inf["groups"][0]["passes"] == 3


def test_no_skip_plan_is_full_radix(L):
    inf = qsd.Plan([10, 10, 10, 10], (0, 1, 2, 3), no_skip=True).info()
    assert inf["num_calls"] == 4 and inf["groups"][0]["keys"] == (0, 1, 2, 3)
    assert qsd.Plan([10, 10, 10, 10], (0, 1, 2, 3)).info()["num_calls"] == 0


def test_workspace_bytes(L):
    p = qsd.Plan([12000, 9000, 28000], (0, 2, 1))
    small, big = p.workspace_bytes(1000), p.workspace_bytes(76_000_000)
    assert 0 < small < big < 76_000_000 * 16
    assert p.workspace_bytes(0) > 0


def test_tuner_workspace_bound_covers_every_candidate(L):
    # qsd_plan_tune skips candidates that do not fit the workspace it is
    # given; the bound it publishes must cover each single change of options
    # it can try, for every structure (Top-K and global groups included)
    import itertools as it
    for dims, sigma in [([12000, 9000, 28000], (0, 2, 1)), ([300, 40, 500, 60], (2, 0, 3, 1)),
                        ([80, 90, 70, 60, 5], (4, 1, 0, 3, 2))]:
        r = len(dims)
        base = qsd.Plan(dims, sigma)
        for nnz in (5_000, 3_000_000):
            need = ctypes.c_size_t()
            assert L.qsd_plan_tune_workspace_bytes(base.handle, nnz, ctypes.byref(need)) == 0
            for k, gg in it.product(range(max(r - 1, 1)), (False, True)):
                for opts in [dict(), dict(digit_bits=5), dict(digit_bits=6), dict(tile=2048),
                             dict(tile=4096), dict(local_capacity=1024 * 8), dict(chunk_tiles=1),
                             dict(local_capacity=4096, chunk_tiles=4)]:
                    p = qsd.Plan(dims, sigma, top_k=k, global_groups=gg, **opts)
                    assert p.workspace_bytes(nnz) <= need.value, (sigma, k, gg, opts, nnz)


def test_noalloc_refuses_while_the_profiler_is_on(L):
    # the launch profiler allocates pinned memory and events of its own, so
    # the allocation-free call refuses to run under it, before any device
    # work (the device pointers here are never dereferenced)
    p = qsd.Plan([4, 4, 4], [2, 1, 0])
    c = _capi.Coords()
    c.buf[0], c.buf[1] = 1 << 36, 2 << 36
    c.stride = 100
    assert L.qsd_profile_enable(1) == 0
    try:
        assert L.qsd_transpose_noalloc(ctypes.byref(c), None, 100, p.handle, None) == 2
    finally:
        assert L.qsd_profile_enable(0) == 0


def test_debug_controls_check_arguments_before_device_work(L):
    assert L.qsd_debug_set_stall(2) == 1
    assert L.qsd_debug_set_stall(-1) == 1
    assert L.qsd_debug_set_spin_limit_ns(61 * 10**9) == 1


def test_key_index_form_of_groups(L):
    # only groups without a prefix, keys of at most 64 bits and two or more
    # digit passes take the (key, index) form; the calls and passes are the
    # plain plan's
    cases = [([1000, 1000, 1000], (2, 1, 0), [True]),            # 20-bit key, 3 passes
             ([12000, 9000, 28000], (0, 2, 1), [False]),          # bucketed
             ([4800000, 1700000, 1800000, 1100], (1, 2, 3, 0), [True]),   # 53 bits
             ([4800000, 1700000, 1800000, 1100], (1, 0, 3, 2), [True, False]),
             ([1 << 20] * 5, (4, 3, 2, 1, 0), [False]),           # 80 bits
             ([300, 200, 100], (2, 0, 1), [True])]                 # 7-bit key: 1 pass
    for dims, sigma, want in cases:
        plain = qsd.Plan(dims, sigma).info()
        ki = qsd.Plan(dims, sigma, key_index=True).info()
        assert plain["calls"] == ki["calls"]
        assert [g["passes"] for g in plain["groups"]] == [g["passes"] for g in ki["groups"]]
        got = [g["key_index"] for g in ki["groups"]]
        want = [w and g["passes"] >= 2 for w, g in zip(want, plain["groups"])]
        assert got == want, (dims, sigma, got)
        assert not any(g["key_index"] for g in plain["groups"])
    # two sets of (key, index) rows in the workspace: 8 (<= 32-bit key) or
    # 12 bytes per entry and set
    n = 1 << 20
    p0 = qsd.Plan([1000, 1000, 1000], (2, 1, 0))
    p1 = qsd.Plan([1000, 1000, 1000], (2, 1, 0), key_index=True)
    assert p1.workspace_bytes(n) - p0.workspace_bytes(n) >= 2 * 8 * n
    d3 = [1 << 20] * 3
    p2 = qsd.Plan(d3, (2, 1, 0), key_index=True)  # 40-bit key: two words
    assert p2.workspace_bytes(n) - qsd.Plan(d3, (2, 1, 0)).workspace_bytes(n) >= 2 * 12 * n


def test_first_digit_bits_never_adds_passes(L):
    dims = [4800000, 1700000, 1800000, 1100]
    for sigma in itertools.permutations(range(4)):
        if sigma == (0, 1, 2, 3):
            continue
        plain = [g["passes"] for g in qsd.Plan(dims, sigma).info()["groups"]]
        for b in range(1, 9):
            got = [g["passes"] for g in qsd.Plan(dims, sigma, first_digit_bits=b).info()["groups"]]
            assert got == plain, (sigma, b)
    with pytest.raises(qsd.QsdError):
        qsd.Plan(dims, (3, 2, 1, 0), first_digit_bits=9)


def test_exec_create_checks_arguments_before_device_work(L):
    p = qsd.Plan([4, 4], [1, 0])
    c = _capi.Coords()
    c.buf[0], c.buf[1] = 1 << 36, 2 << 36
    c.stride = 10
    h = ctypes.c_void_p()
    src = ctypes.c_void_p(3 << 36)
    assert L.qsd_exec_create(src, 10, None, ctypes.byref(c), None, 10, p.handle,
                             ctypes.c_void_p(4 << 36), 1 << 20, None) == 1       # no out
    assert L.qsd_exec_create(src, 10, None, ctypes.byref(c), None, 10, p.handle,
                             ctypes.c_void_p((4 << 36) + 8), 1 << 20, ctypes.byref(h)) == 1  # alignment
    assert L.qsd_exec_create(src, 9, None, ctypes.byref(c), None, 10, p.handle,
                             ctypes.c_void_p(4 << 36), 1 << 20, ctypes.byref(h)) == 1   # stride < nnz
    assert L.qsd_exec_create(src, 10, None, ctypes.byref(c), None, 10, p.handle,
                             ctypes.c_void_p(4 << 36), 16, ctypes.byref(h)) == 9        # workspace
    assert L.qsd_exec_launch(None, None, None, None) == 1
    L.qsd_exec_destroy(None)
