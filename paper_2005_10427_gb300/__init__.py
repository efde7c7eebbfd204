"""GB300 sparse COO tensor transposition (the Quesadilla method, sm_103a).

Thin Python binding over the C ABI in include/qsd.h: it only marshals
arguments (torch tensors provide device memory and streams); every step of
the transposition runs in the CUDA library libqsd.so. There is no CPU
fallback: if the library is missing, calls raise.

    plan = Plan(dims, target_perm)                 # Algorithm 3 on the host
    coords_t, vals_t = transpose(coords, vals, plan)
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

from . import _capi

__all__ = ["Plan", "QsdError", "Batch", "Server", "server_clock", "csf_levels", "csf_build",
           "tune_plan",
           "csf_workspace_bytes", "transpose", "transpose_buffers", "transpose_from",
           "transpose_host", "transpose_noalloc", "tune_cache_save", "tune_cache_load",
           "get_async_status", "workspace_status", "build", "lib", "LIB_PATH"]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libqsd.so")


class QsdError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        name = _capi.STATUS_NAMES.get(self.status, f"status {status}")
        super().__init__(f"{where}: {name}" if where else name)


def build(force: bool = False) -> str:
    from .buildlib import build as _build
    return _build(force=force)


def lib() -> ctypes.CDLL:
    return _capi.load(LIB_PATH)


def _check(status: int, where: str):
    if status != 0:
        raise QsdError(status, where)


def _i32(seq: Sequence[int]):
    return (ctypes.c_int * len(seq))(*[int(x) for x in seq])


class Plan:
    """A transposition plan: input order tau -> target order sigma.

    dims: mode sizes; target_perm: sigma; input_mode_order: tau (identity by
    default). Options map to qsd_plan_options.
    """

    def __init__(self, dims: Sequence[int], target_perm: Sequence[int],
                 input_mode_order: Optional[Sequence[int]] = None, *,
                 validate: bool = False, digit_bits: int = 0,
                 local_capacity: int = 0, no_skip: bool = False, tile: int = 0,
                 chunk_tiles: int = 0, global_groups: bool = False, top_k: int = 0,
                 key_index: bool = False, first_digit_bits: int = 0):
        L = lib()
        r = len(dims)
        self.dims = [int(d) for d in dims]
        self.order = r
        self.target_perm = [int(x) for x in target_perm]
        self.input_mode_order = list(range(r)) if input_mode_order is None else \
            [int(x) for x in input_mode_order]
        opts = _capi.PlanOptions(int(bool(validate)), int(digit_bits), int(local_capacity),
                                 int(bool(no_skip)), int(tile), int(chunk_tiles),
                                 int(bool(global_groups)), int(top_k), int(bool(key_index)),
                                 int(first_digit_bits))
        self.options = dict(validate=bool(validate), digit_bits=int(digit_bits),
                            local_capacity=int(local_capacity), no_skip=bool(no_skip),
                            tile=int(tile), chunk_tiles=int(chunk_tiles),
                            global_groups=bool(global_groups), top_k=int(top_k),
                            key_index=bool(key_index), first_digit_bits=int(first_digit_bits))
        handle = ctypes.c_void_p()
        dims_arr = (ctypes.c_int64 * max(r, 1))(*self.dims)
        st = L.qsd_plan_ex(r, dims_arr, _i32(self.input_mode_order) if r else None,
                           _i32(self.target_perm) if r else None, ctypes.byref(opts),
                           ctypes.byref(handle))
        _check(st, "qsd_plan")
        self._h = handle
        self._lib = L

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.qsd_plan_destroy(h)
            self._h = None

    def info(self) -> dict:
        inf = _capi.PlanInfo()
        _check(self._lib.qsd_plan_get_info(self._h, ctypes.byref(inf)), "qsd_plan_get_info")
        r = inf.order
        sig = list(inf.target_perm[:r])
        calls = [(tuple(sig[:inf.call_prefix_len[i]]), int(inf.call_mode[i]))
                 for i in range(inf.num_calls)]
        groups = []
        for g in range(inf.num_groups):
            pl, nk = inf.group_prefix_len[g], inf.group_num_keys[g]
            groups.append(dict(prefix=tuple(sig[:pl]), keys=tuple(sig[pl:pl + nk]),
                               key_bits=int(inf.group_key_bits[g]),
                               passes=int(inf.group_digit_passes[g]),
                               key_index=bool(inf.group_key_index[g])))
        return dict(order=r, input_mode_order=list(inf.input_mode_order[:r]),
                    target_perm=sig, calls=calls, num_calls=inf.num_calls,
                    num_bucketed_calls=inf.num_bucketed_calls, groups=groups,
                    local_capacity=inf.local_capacity)

    @property
    def calls(self) -> List[Tuple[Tuple[int, ...], int]]:
        return self.info()["calls"]

    def workspace_bytes(self, nnz: int) -> int:
        out = ctypes.c_size_t()
        _check(self._lib.qsd_workspace_bytes(self._h, int(nnz), ctypes.byref(out)),
               "qsd_workspace_bytes")
        return int(out.value)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _val_bytes(vals) -> int:
    return 0 if vals is None else int(vals.element_size())


def transpose_buffers(cbuf: Sequence, vbuf: Optional[Sequence], selector: int, nnz: int,
                      plan: Plan, workspace, stream=None) -> int:
    """Runs qsd_transpose_ws on explicit double buffers.

    cbuf: two int32 CUDA tensors (r, stride); vbuf: two value tensors or None;
    selector: which buffer holds the input. workspace: a CUDA uint8 tensor of
    at least plan.workspace_bytes(nnz). Returns the selector of the result.
    """
    c = _capi.Coords()
    c.buf[0] = cbuf[0].data_ptr()
    c.buf[1] = cbuf[1].data_ptr()
    c.stride = int(cbuf[0].stride(0)) if cbuf[0].dim() == 2 else int(nnz)
    c.selector = int(selector)
    v = _capi.Values()
    if vbuf is not None:
        v.buf[0] = vbuf[0].data_ptr()
        v.buf[1] = vbuf[1].data_ptr()
        v.elem_bytes = _val_bytes(vbuf[0])
        v.selector = int(selector)
    st = lib().qsd_transpose_ws(ctypes.byref(c), ctypes.byref(v), int(nnz), plan.handle,
                                ctypes.c_void_p(workspace.data_ptr()),
                                int(workspace.numel()), _stream_handle(stream))
    _check(st, "qsd_transpose_ws")
    return int(c.selector)


def transpose_from(in_coords, in_vals, cbuf: Sequence, vbuf: Optional[Sequence], nnz: int,
                   plan: Plan, workspace, stream=None) -> int:
    """Out-of-place: qsd_transpose_from_ws. The input tensors stay unchanged;
    the result lands in cbuf[sel] / vbuf[sel]; returns sel."""
    c = _capi.Coords()
    c.buf[0] = cbuf[0].data_ptr()
    c.buf[1] = cbuf[1].data_ptr()
    c.stride = int(cbuf[0].stride(0))
    v = _capi.Values()
    if vbuf is not None:
        v.buf[0] = vbuf[0].data_ptr()
        v.buf[1] = vbuf[1].data_ptr()
        v.elem_bytes = _val_bytes(vbuf[0])
    st = lib().qsd_transpose_from_ws(
        ctypes.c_void_p(in_coords.data_ptr()), int(in_coords.stride(0)),
        ctypes.c_void_p(in_vals.data_ptr()) if in_vals is not None else None,
        ctypes.byref(c), ctypes.byref(v), int(nnz), plan.handle,
        ctypes.c_void_p(workspace.data_ptr()), int(workspace.numel()),
        _stream_handle(stream))
    _check(st, "qsd_transpose_from_ws")
    return int(c.selector)


def transpose_noalloc(cbuf: Sequence, vbuf: Optional[Sequence], selector: int, nnz: int,
                      plan: Plan, stream=None) -> int:
    """qsd_transpose_noalloc on explicit double buffers: like transpose_buffers
    but with the library's fixed 64 MiB device scratch instead of a workspace,
    for callers that cannot allocate device memory. Returns the result's
    selector."""
    c = _capi.Coords()
    c.buf[0] = cbuf[0].data_ptr()
    c.buf[1] = cbuf[1].data_ptr()
    c.stride = int(cbuf[0].stride(0)) if cbuf[0].dim() == 2 else int(nnz)
    c.selector = int(selector)
    v = _capi.Values()
    if vbuf is not None:
        v.buf[0] = vbuf[0].data_ptr()
        v.buf[1] = vbuf[1].data_ptr()
        v.elem_bytes = _val_bytes(vbuf[0])
        v.selector = int(selector)
    st = lib().qsd_transpose_noalloc(ctypes.byref(c), ctypes.byref(v), int(nnz), plan.handle,
                                     _stream_handle(stream))
    _check(st, "qsd_transpose_noalloc")
    return int(c.selector)


class Exec:
    """One out-of-place transposition captured into a CUDA graph
    (qsd_exec_*): launch() replays it. The tensors given here stay bound to
    it (keep them alive and in place); launch() returns the selector of the
    result buffer."""

    def __init__(self, in_coords, in_vals, cbuf: Sequence, vbuf: Optional[Sequence], nnz: int,
                 plan: Plan, workspace):
        L = lib()
        c = _capi.Coords()
        c.buf[0] = cbuf[0].data_ptr()
        c.buf[1] = cbuf[1].data_ptr()
        c.stride = int(cbuf[0].stride(0))
        v = _capi.Values()
        if vbuf is not None:
            v.buf[0] = vbuf[0].data_ptr()
            v.buf[1] = vbuf[1].data_ptr()
            v.elem_bytes = _val_bytes(vbuf[0])
        h = ctypes.c_void_p()
        st = L.qsd_exec_create(
            ctypes.c_void_p(in_coords.data_ptr()), int(in_coords.stride(0)),
            ctypes.c_void_p(in_vals.data_ptr()) if in_vals is not None else None,
            ctypes.byref(c), ctypes.byref(v), int(nnz), plan.handle,
            ctypes.c_void_p(workspace.data_ptr()), int(workspace.numel()), ctypes.byref(h))
        _check(st, "qsd_exec_create")
        self._h = h
        self._lib = L
        self._keep = (in_coords, in_vals, cbuf, vbuf, plan, workspace)

    def launch(self, stream=None) -> int:
        sel = ctypes.c_int()
        _check(self._lib.qsd_exec_launch(self._h, _stream_handle(stream), ctypes.byref(sel),
                                         None), "qsd_exec_launch")
        return int(sel.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.qsd_exec_destroy(h)
            self._h = None


_OPTION_KEYS = ("digit_bits", "local_capacity", "tile", "chunk_tiles", "no_graph",
                "use_tuned")


def _options_dict(o) -> dict:
    return {k: int(getattr(o, k)) for k in _OPTION_KEYS}


class Batch:
    """Many tensors transposed by one graph launch (qsd_batch_*).

    items: sequence of (plan, in_coords, in_vals, out_cbuf, out_vbuf) where
    in_coords is an int32 CUDA tensor (r, >= nnz) sorted under the plan's
    input order, in_vals a value tensor or None, out_cbuf two int32 CUDA
    tensors (r, >= nnz) and out_vbuf two value tensors or None; nnz is
    in_coords.shape[1] unless given as a sixth element. The buffers stay bound
    to the batch (keep them alive). run() recomputes every result; result(i)
    gives the buffer index holding tensor i's result.
    """

    def __init__(self, items, *, val_bytes: Optional[int] = None, digit_bits: int = 0,
                 local_capacity: int = 0, tile: int = 0, chunk_tiles: int = 0,
                 graph: bool = True, use_tuned: bool = False):
        L = lib()
        n = len(items)
        arr = (_capi.BatchItem * max(n, 1))()
        vb = val_bytes
        self._keep = []
        for i, it in enumerate(items):
            plan, cin, vin, cout, vout = it[:5]
            nnz = int(it[5]) if len(it) > 5 else int(cin.shape[1])
            e = arr[i]
            e.plan = plan.handle.value
            e.nnz = nnz
            e.in_ = cin.data_ptr()
            e.in_stride = int(cin.stride(0)) if cin.dim() == 2 else nnz
            e.in_vals = vin.data_ptr() if vin is not None else None
            e.out[0] = cout[0].data_ptr()
            e.out[1] = cout[1].data_ptr()
            e.out_stride = int(cout[0].stride(0)) if cout[0].dim() == 2 else nnz
            if vout is not None:
                e.out_vals[0] = vout[0].data_ptr()
                e.out_vals[1] = vout[1].data_ptr()
            if vb is None:
                vb = _val_bytes(vin)
            self._keep.append(it)
        opts = _capi.BatchOptions(int(digit_bits), int(local_capacity), int(tile),
                                  int(chunk_tiles), int(not graph), int(bool(use_tuned)))
        h = ctypes.c_void_p()
        _check(L.qsd_batch_create(arr, n, int(vb or 0), ctypes.byref(opts), ctypes.byref(h)),
               "qsd_batch_create")
        self._h = h
        self._lib = L
        self.n = n

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.qsd_batch_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def workspace_bytes(self) -> int:
        out = ctypes.c_size_t()
        _check(self._lib.qsd_batch_workspace_bytes(self._h, ctypes.byref(out)),
               "qsd_batch_workspace_bytes")
        return int(out.value)

    def run(self, workspace, stream=None) -> None:
        _check(self._lib.qsd_batch_run(self._h, ctypes.c_void_p(workspace.data_ptr()),
                                       int(workspace.numel()), _stream_handle(stream)),
               "qsd_batch_run")

    def result(self, i: int) -> int:
        out = ctypes.c_int()
        _check(self._lib.qsd_batch_result(self._h, int(i), ctypes.byref(out)),
               "qsd_batch_result")
        return int(out.value)

    def options(self) -> dict:
        o = _capi.BatchOptions()
        _check(self._lib.qsd_batch_get_options(self._h, ctypes.byref(o)),
               "qsd_batch_get_options")
        return _options_dict(o)

    def tune(self, workspace, reps: int = 3, stream=None) -> dict:
        """Autotunes the execution options (qsd_batch_tune); returns the choice."""
        o = _capi.BatchOptions()
        _check(self._lib.qsd_batch_tune(self._h, ctypes.c_void_p(workspace.data_ptr()),
                                        int(workspace.numel()), _stream_handle(stream),
                                        int(reps), ctypes.byref(o)), "qsd_batch_tune")
        return _options_dict(o)


def tune_plan(plan: "Plan", in_coords, in_vals, reps: int = 3, stream=None):
    """qsd_plan_tune: times the plan's equivalent variants on this tensor
    (out of place; the input is not modified) and returns (tuned Plan, ms per
    transposition, options dict)."""
    import torch
    nnz = int(in_coords.shape[1])
    need = ctypes.c_size_t()
    _check(lib().qsd_plan_tune_workspace_bytes(plan.handle, nnz, ctypes.byref(need)),
           "qsd_plan_tune_workspace_bytes")
    dev = in_coords.device
    ws = torch.empty(max(int(need.value), 256), dtype=torch.uint8, device=dev)
    cb = [torch.empty_like(in_coords) for _ in range(2)]
    c = _capi.Coords()
    c.buf[0], c.buf[1] = cb[0].data_ptr(), cb[1].data_ptr()
    c.stride = int(in_coords.stride(0))
    v = _capi.Values()
    vb = None
    if in_vals is not None:
        vb = [torch.empty_like(in_vals) for _ in range(2)]
        v.buf[0], v.buf[1] = vb[0].data_ptr(), vb[1].data_ptr()
        v.elem_bytes = _val_bytes(in_vals)
    best = _capi.PlanOptions()
    ms = ctypes.c_float()
    _check(lib().qsd_plan_tune(plan.handle, ctypes.c_void_p(in_coords.data_ptr()),
                               int(in_coords.stride(0)),
                               ctypes.c_void_p(in_vals.data_ptr()) if in_vals is not None else None,
                               ctypes.byref(c), ctypes.byref(v), nnz,
                               ctypes.c_void_p(ws.data_ptr()), int(ws.numel()),
                               _stream_handle(stream), int(reps), ctypes.byref(best),
                               ctypes.byref(ms)), "qsd_plan_tune")
    opts = {k: int(getattr(best, k)) for k, _ in _capi.PlanOptions._fields_}
    tuned = Plan(plan.dims, plan.target_perm, plan.input_mode_order,
                 validate=bool(opts["validate"]), digit_bits=opts["digit_bits"],
                 local_capacity=opts["local_capacity"], no_skip=bool(opts["no_skip"]),
                 tile=opts["tile"], chunk_tiles=opts["chunk_tiles"],
                 global_groups=bool(opts["global_groups"]), top_k=opts["top_k"],
                 key_index=bool(opts["key_index"]), first_digit_bits=opts["first_digit_bits"])
    return tuned, float(ms.value), opts


def csf_workspace_bytes(order: int, nnz: int) -> int:
    need = ctypes.c_size_t()
    _check(lib().qsd_csf_workspace_bytes(int(order), int(nnz), ctypes.byref(need)),
           "qsd_csf_workspace_bytes")
    return max(int(need.value), 256)


def csf_build(coords, sigma: Sequence[int], ids, ptr, nodes, workspace, stream=None) -> None:
    """qsd_csf_build into preallocated int32 CUDA tensors: ids[l] (capacity
    >= nnz), ptr[0] (2), ptr[l] (nnz + 1), nodes (r + 1)."""
    r, nnz = int(coords.shape[0]), int(coords.shape[1])
    out = _capi.Csf()
    for l in range(r):
        out.ids[l] = ids[l].data_ptr()
    for l in range(r + 1):
        out.ptr[l] = ptr[l].data_ptr()
    stride = int(coords.stride(0)) if nnz else 0
    _check(lib().qsd_csf_build(ctypes.c_void_p(coords.data_ptr()) if nnz else None, stride, nnz,
                               r, _i32(sigma), ctypes.byref(out),
                               ctypes.c_void_p(nodes.data_ptr()),
                               ctypes.c_void_p(workspace.data_ptr()), int(workspace.numel()),
                               _stream_handle(stream)), "qsd_csf_build")


def csf_levels(coords, sigma: Sequence[int], stream=None):
    """CSF levels (qsd_csf_build) of a tensor sorted under sigma.

    coords: int32 CUDA tensor (r, nnz) sorted under sigma (for example
    transpose()'s result for target order sigma). Returns (ids, ptr): ids[l]
    holds level l+1's node ids, ptr[l] the first child of each level-l node
    (l < r) or the first entry of each leaf (l == r), plus an end marker; all
    int32 CUDA tensors sized to the node counts (read back with one sync).
    """
    import torch
    r, nnz = int(coords.shape[0]), int(coords.shape[1])
    dev = coords.device
    cap = max(nnz, 1)
    ids = [torch.empty(cap, dtype=torch.int32, device=dev) for _ in range(r)]
    ptr = [torch.empty(2 if l == 0 else cap + 1, dtype=torch.int32, device=dev)
           for l in range(r + 1)]
    nodes = torch.empty(r + 1, dtype=torch.int32, device=dev)
    ws = torch.empty(csf_workspace_bytes(r, nnz), dtype=torch.uint8, device=dev)
    csf_build(coords, sigma, ids, ptr, nodes, ws, stream)
    n = [int(x) for x in nodes.cpu()]  # synchronises with the stream's work
    return ([ids[l][:n[l + 1]] for l in range(r)],
            [ptr[l][:n[l] + 1] for l in range(r + 1)])


def transpose_csf_workspace_bytes(plan: "Plan", nnz: int) -> int:
    need = ctypes.c_size_t()
    _check(lib().qsd_transpose_csf_workspace_bytes(plan.handle, int(nnz), ctypes.byref(need)),
           "qsd_transpose_csf_workspace_bytes")
    return max(int(need.value), 256)


def transpose_csf_from(in_coords, in_vals, cbuf: Sequence, vbuf: Optional[Sequence], nnz: int,
                       plan: "Plan", ids, ptr, nodes, workspace, stream=None) -> int:
    """qsd_transpose_csf_from_ws: out-of-place transposition into cbuf/vbuf
    (returns the result's selector) and the CSF levels of the result into
    preallocated int32 CUDA tensors ids[l] (capacity >= nnz), ptr[0] (2),
    ptr[l] (nnz + 1) and nodes (r + 1), as csf_build gives them."""
    r = plan.order
    c = _capi.Coords()
    c.buf[0] = cbuf[0].data_ptr()
    c.buf[1] = cbuf[1].data_ptr()
    c.stride = int(cbuf[0].stride(0))
    v = _capi.Values()
    if vbuf is not None:
        v.buf[0] = vbuf[0].data_ptr()
        v.buf[1] = vbuf[1].data_ptr()
        v.elem_bytes = _val_bytes(vbuf[0])
    out = _capi.Csf()
    for l in range(r):
        out.ids[l] = ids[l].data_ptr()
    for l in range(r + 1):
        out.ptr[l] = ptr[l].data_ptr()
    st = lib().qsd_transpose_csf_from_ws(
        ctypes.c_void_p(in_coords.data_ptr()), int(in_coords.stride(0)),
        ctypes.c_void_p(in_vals.data_ptr()) if in_vals is not None else None,
        ctypes.byref(c), ctypes.byref(v), int(nnz), plan.handle, ctypes.byref(out),
        ctypes.c_void_p(nodes.data_ptr()), ctypes.c_void_p(workspace.data_ptr()),
        int(workspace.numel()), _stream_handle(stream))
    _check(st, "qsd_transpose_csf_from_ws")
    return int(c.selector)


def server_clock() -> float:
    """Seconds of the monotonic clock the server stamps times with."""
    return float(lib().qsd_server_clock())


class Server:
    """Continuous-batching transposition server (qsd_server_*).

    Resident tensors are registered once (add_tensor; keep the tensors
    alive); submit() queues a request and returns its id; poll() returns
    completed requests as dicts (status, times, result pointers); copy_result()
    copies a result into caller tensors; release() returns its memory to the
    budget.
    """

    def __init__(self, memory_budget: int, *, val_bytes: int, max_inflight: int = 0,
                 streams: int = 0, max_batch: int = 0, digit_bits: int = 0,
                 local_capacity: int = 0, tile: int = 0, chunk_tiles: int = 0):
        L = lib()
        bo = _capi.BatchOptions(int(digit_bits), int(local_capacity), int(tile),
                                int(chunk_tiles), 1, 0)
        o = _capi.ServerOptions(int(memory_budget), int(max_inflight), int(streams),
                                int(max_batch), int(val_bytes), bo)
        h = ctypes.c_void_p()
        _check(L.qsd_server_create(ctypes.byref(o), ctypes.byref(h)), "qsd_server_create")
        self._h = h
        self._lib = L
        self._tensors = []
        self.val_bytes = int(val_bytes)

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.qsd_server_destroy(h)
            self._h = None

    def __del__(self):
        self.close()

    def add_tensor(self, coords, vals, dims: Sequence[int],
                   input_mode_order: Optional[Sequence[int]] = None) -> int:
        r = coords.shape[0]
        nnz = int(coords.shape[1])
        dims_arr = (ctypes.c_int64 * r)(*[int(d) for d in dims])
        tau = _i32(input_mode_order) if input_mode_order is not None else None
        out = ctypes.c_int()
        _check(self._lib.qsd_server_add_tensor(
            self._h, r, dims_arr, tau, ctypes.c_void_p(coords.data_ptr()),
            int(coords.stride(0)) if nnz else 0,
            ctypes.c_void_p(vals.data_ptr()) if vals is not None else None, nnz,
            ctypes.byref(out)), "qsd_server_add_tensor")
        self._tensors.append((coords, vals))
        return int(out.value)

    def submit(self, tensor: int, target_perm: Sequence[int], arrival_s: float = 0.0) -> int:
        rid = ctypes.c_int64()
        _check(self._lib.qsd_server_submit(self._h, int(tensor), _i32(target_perm),
                                           float(arrival_s), ctypes.byref(rid)),
               "qsd_server_submit")
        return int(rid.value)

    def poll(self, max_results: int = 256, wait_ms: int = 0) -> List[dict]:
        arr = (_capi.ServerResult * max(int(max_results), 1))()
        n = ctypes.c_int()
        _check(self._lib.qsd_server_poll(self._h, arr, int(max_results), int(wait_ms),
                                         ctypes.byref(n)), "qsd_server_poll")
        return [{"request": int(r.request), "tensor": int(r.tensor), "status": int(r.status),
                 "nnz": int(r.nnz), "coords": r.coords, "vals": r.vals,
                 "arrival_s": r.arrival_s, "admit_s": r.admit_s, "done_s": r.done_s}
                for r in arr[:n.value]]

    def copy_result(self, request: int, coords_out, vals_out=None, stream=None) -> None:
        _check(self._lib.qsd_server_copy_result(
            self._h, int(request), ctypes.c_void_p(coords_out.data_ptr()),
            int(coords_out.stride(0)),
            ctypes.c_void_p(vals_out.data_ptr()) if vals_out is not None else None,
            _stream_handle(stream)), "qsd_server_copy_result")

    def release(self, request: int) -> None:
        _check(self._lib.qsd_server_release(self._h, int(request)), "qsd_server_release")

    def stats(self) -> dict:
        st = _capi.ServerStats()
        _check(self._lib.qsd_server_get_stats(self._h, ctypes.byref(st)), "qsd_server_get_stats")
        return {k: int(getattr(st, k)) for k, _ in _capi.ServerStats._fields_}


def tune_cache_save(path: str) -> None:
    _check(lib().qsd_tune_cache_save(os.fsencode(path)), "qsd_tune_cache_save")


def tune_cache_load(path: str) -> None:
    _check(lib().qsd_tune_cache_load(os.fsencode(path)), "qsd_tune_cache_load")


def transpose(coords, vals, plan: Plan, *, workspace=None, stream=None):
    """Transposes a COO tensor on the GPU.

    coords: int32 CUDA tensor (r, nnz), rows contiguous; vals: 1-D CUDA tensor
    of 4- or 8-byte elements, or None. Returns (coords_out, vals_out); the
    result may live in the input tensors' storage (the library ping-pongs
    between the input and a second buffer it is given here).
    """
    import torch
    if coords.dim() != 2 or coords.dtype != torch.int32 or (
            coords.shape[1] > 1 and coords.stride(1) != 1):
        raise ValueError("coords must be an int32 tensor of shape (order, nnz) with unit "
                         "stride along entries")
    if not coords.is_cuda:
        raise ValueError("coords must be on a CUDA device (no CPU path exists)")
    nnz = coords.shape[1]
    alt_c = torch.empty_like(coords)
    vbuf = None
    if vals is not None:
        if vals.dim() != 1 or vals.numel() != nnz or vals.element_size() not in (4, 8):
            raise ValueError("vals must be 1-D with nnz elements of 4 or 8 bytes")
        vbuf = [vals, torch.empty_like(vals)]
    if workspace is None:
        workspace = torch.empty(plan.workspace_bytes(nnz), dtype=torch.uint8,
                                device=coords.device)
    sel = transpose_buffers([coords, alt_c], vbuf, 0, nnz, plan, workspace, stream)
    out_c = [coords, alt_c][sel]
    out_v = None if vbuf is None else vbuf[sel]
    return out_c, out_v


def transpose_host(coords_host, vals_host, plan: Plan, dev_cbuf, dev_vbuf, workspace,
                   out_coords_host, out_vals_host, stream=None) -> None:
    """End-to-end call on host tensors through qsd_transpose_host.

    coords_host (r, nnz) int32 / vals_host on the CPU (pinned for full
    bandwidth); dev_cbuf / dev_vbuf: two device buffers each; results are
    written into out_coords_host / out_vals_host. Waits for the stream.
    """
    _transpose_host_call(lib().qsd_transpose_host, "qsd_transpose_host", coords_host, vals_host,
                         plan, dev_cbuf, dev_vbuf, workspace, out_coords_host, out_vals_host,
                         stream)


def transpose_host_async(coords_host, vals_host, plan: Plan, dev_cbuf, dev_vbuf, workspace,
                         out_coords_host, out_vals_host, stream=None) -> None:
    """qsd_transpose_host_async: as transpose_host, but returns once the copies
    and kernels are enqueued on `stream`. Every tensor passed must stay
    untouched until the stream has passed the call; workspace_status(workspace,
    stream) then gives the device status."""
    _transpose_host_call(lib().qsd_transpose_host_async, "qsd_transpose_host_async", coords_host,
                         vals_host, plan, dev_cbuf, dev_vbuf, workspace, out_coords_host,
                         out_vals_host, stream)


def _transpose_host_call(fn, name, coords_host, vals_host, plan, dev_cbuf, dev_vbuf, workspace,
                         out_coords_host, out_vals_host, stream):
    nnz = coords_host.shape[1]
    c = _capi.Coords()
    c.buf[0] = dev_cbuf[0].data_ptr()
    c.buf[1] = dev_cbuf[1].data_ptr()
    c.stride = int(dev_cbuf[0].stride(0))
    c.selector = 0
    v = _capi.Values()
    if dev_vbuf is not None:
        v.buf[0] = dev_vbuf[0].data_ptr()
        v.buf[1] = dev_vbuf[1].data_ptr()
        v.elem_bytes = _val_bytes(dev_vbuf[0])
    st = fn(
        ctypes.c_void_p(coords_host.data_ptr()), int(coords_host.stride(0)),
        ctypes.c_void_p(vals_host.data_ptr()) if vals_host is not None else None,
        ctypes.c_void_p(out_coords_host.data_ptr()), int(out_coords_host.stride(0)),
        ctypes.c_void_p(out_vals_host.data_ptr()) if out_vals_host is not None else None,
        int(nnz), plan.handle, ctypes.byref(c), ctypes.byref(v),
        ctypes.c_void_p(workspace.data_ptr()), int(workspace.numel()),
        _stream_handle(stream))
    _check(st, name)


def workspace_status(workspace, stream=None) -> int:
    out = ctypes.c_int()
    _check(lib().qsd_workspace_status(ctypes.c_void_p(workspace.data_ptr()),
                                      _stream_handle(stream), ctypes.byref(out)),
           "qsd_workspace_status")
    return int(out.value)


def get_async_status(stream=None) -> int:
    out = ctypes.c_int()
    _check(lib().qsd_get_async_status(_stream_handle(stream), ctypes.byref(out)),
           "qsd_get_async_status")
    return int(out.value)


def debug_set_spin_limit_ns(limit_ns: int) -> None:
    """Test-only: the limit of every bounded device wait (0 = default 2 s)."""
    _check(lib().qsd_debug_set_spin_limit_ns(int(limit_ns)), "qsd_debug_set_spin_limit_ns")


def debug_set_stall(stall: int) -> None:
    """Test-only: 1 = the move kernel's block 0 never fills its first staging
    slot, so its waits expire (QSD_ERR_TIMEOUT); 0 = off."""
    _check(lib().qsd_debug_set_stall(int(stall)), "qsd_debug_set_stall")


def profile_enable(on: bool = True) -> None:
    """Records CUDA-event timings of every library kernel launch (qsd_profile_*)."""
    _check(lib().qsd_profile_enable(int(bool(on))), "qsd_profile_enable")


def profile_reset() -> None:
    _check(lib().qsd_profile_reset(), "qsd_profile_reset")


def profile_read() -> List[dict]:
    """The recorded launches since the last reset (waits for them)."""
    n = ctypes.c_int()
    _check(lib().qsd_profile_read(None, 0, ctypes.byref(n)), "qsd_profile_read")
    if n.value == 0:
        return []
    recs = (_capi.ProfileRecord * n.value)()
    _check(lib().qsd_profile_read(recs, n.value, ctypes.byref(n)), "qsd_profile_read")
    return [dict(kernel=r.kernel.decode(), group=r.group, pass_=r.pass_, entries=r.entries,
                 algo_bytes=r.algo_bytes, ms=r.ms) for r in recs]
