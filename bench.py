"""Benchmark: COO transposition throughput on one GB300 (and N replicas).

Workload (default, the line of record): a 4-order tensor of 4.8M x 1.7M x
1.8M x 1100 with 140M distinct coordinates (Zipf 1.3 on modes 0-2, uniform
mode 3), float64 values N(0,1), sorted in (0,1,2,3) order and resident in
HBM. One step transposes it into each of the 23 non-identity target orders
(out of place, the input stays intact; each order's call captured once into
a CUDA graph and replayed), so a step moves 23 x 140M entries. Throughput =
entries transposed per second (Gnnz/s), device-timed with CUDA events; the
input (3.4 GB) is larger than the 129 MB L2, so no flush is needed between
steps.

Also reported: the live roofline of the dominant kernel (algorithmic bytes /
CUDA-event duration against the measured HBM copy bandwidth) and the whole
step's fraction of the minimum-traffic roofline; per target order the time
and fraction beside the no-skip radix sort, the key-index form and
Top-K-sadilla; the same table for the 76M-entry order-3 workload; the
1M-entry single-call latency; CSF levels; the batched workload against
single calls; the serving workload (Poisson arrivals, saturated, and the
same requests as single calls); the end-to-end rate through the host-buffer
calls; SM clocks sampled during the timed region; and the CPU oracle's and
the paper's CPU method's rates on bounded samples.

`--impl reference` times the CPU oracle (std::stable_sort on the host cores)
on bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import synth  # noqa: E402

METRIC = ("Gnnz/s transposed (bit-exact) and % HBM roofline; batched/served vs "
          "single calls")
WORKLOADS = {
    "nell2like": synth.WORKLOAD_NELL2_LIKE,
    "uniform3d": synth.WORKLOAD_3D_UNIFORM,
    "deliciouslike": synth.WORKLOAD_DELICIOUS_LIKE,
}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def committed_traffic(kernel: str, workload: str):
    """DRAM bytes per entry for a kernel from the committed ncu summary."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    return d.get(workload, {}).get(kernel)


def combine_ranks(ms: float, world: int, device) -> float:
    """The timed region's duration for the whole job: the slowest rank's
    (max over ranks; every rank gets it)."""
    if world <= 1:
        return ms
    tt = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return float(tt.item())


def aggregate_value(world: int, entries_per_step: int, steps: int, ms: float) -> float:
    """Whole-job throughput (Gnnz/s): the entries all ranks transposed over the
    slowest rank's time (the replicas each run the full per-GPU workload)."""
    return world * entries_per_step * steps / (ms / 1e3) / 1e9


def cpu_oracle_rate(t_coords: np.ndarray, t_vals: np.ndarray, perms, target_s=15.0):
    """The oracle (single-threaded std::stable_sort) on a strided sample of the
    workload (every k-th entry: still sorted in the input order, with the
    workload's distribution), sized to about target_s seconds."""
    import oracle
    n_total = t_coords.shape[1]

    def run(m):
        idx = np.linspace(0, n_total - 1, m).astype(np.int64)
        c, v = np.ascontiguousarray(t_coords[:, idx]), np.ascontiguousarray(t_vals[idx])
        t0 = time.perf_counter()
        for sigma in perms:
            oracle.transpose(c, v, sigma)
        return time.perf_counter() - t0

    m = min(n_total, 400_000)
    dt = run(m)
    while m < n_total and dt < 0.4 * target_s:  # grow at most 4x per step (n log n)
        m = int(min(n_total, m * min(4.0, 0.8 * target_s / max(dt, 1e-3))))
        dt = run(m)
    return {"value": len(perms) * m / dt / 1e9, "unit": "Gnnz/s", "cores": 1, "kind": "oracle",
            "sample": f"{m} entries (every {n_total / m:.1f}-th of the workload, in input "
                      f"order), all {len(perms)} target orders, std::stable_sort on 1 host "
                      f"core, {dt:.1f} s"}


def cpu_method_rate(t_coords: np.ndarray, t_vals: np.ndarray, dims, perms, target_s=8.0):
    """The paper's own CPU method (Algorithms 1-3 as counting sorts, parallel
    as its Section 3.2 describes; OpenMP on all host cores) on a strided
    sample of the workload, sized to about target_s seconds."""
    import cpu_method
    n_total = t_coords.shape[1]
    threads = cpu_method.threads()

    def run(m, top_k=0):
        idx = np.linspace(0, n_total - 1, m).astype(np.int64)
        c, v = np.ascontiguousarray(t_coords[:, idx]), np.ascontiguousarray(t_vals[idx])
        t0 = time.perf_counter()
        for sigma in perms:
            cpu_method.transpose(c, v, dims, sigma, top_k=top_k)
        return time.perf_counter() - t0

    m = min(n_total, 1_000_000)
    dt = run(m)
    while m < n_total and dt < 0.4 * target_s:
        m = int(min(n_total, m * min(4.0, 0.8 * target_s / max(dt, 1e-3))))
        dt = run(m)
    # Top-1-sadilla (Section 3.6) on the same sample, for the paper's own comparison
    dt1 = run(m, top_k=1)
    return {"value": len(perms) * m / dt / 1e9, "unit": "Gnnz/s", "cores": threads,
            "kind": "paper's CPU method (Algorithms 1-3 as parallel counting sorts)",
            "sample": f"{m} entries (every {n_total / m:.1f}-th of the workload), all "
                      f"{len(perms)} target orders, {threads} host threads, {dt:.1f} s",
            "top1_sadilla": {"value": len(perms) * m / dt1 / 1e9, "unit": "Gnnz/s",
                             "seconds": round(dt1, 2)}}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    wl = WORKLOADS[args.workload]
    nnz = args.nnz or wl["nnz"]
    ref_sample = args.ref_sample or (2_000_000 if len(wl["perms"]) <= 5 else 1_000_000)
    sample = min(nnz, ref_sample)
    w = synth.scaled(wl, sample) if sample != wl["nnz"] else wl
    t = synth.make(w)
    coords, vals = t.coords.numpy(), t.vals.numpy()
    perms = wl["perms"]
    for _ in range(args.warmup):
        for sigma in perms:
            oracle.transpose(coords, vals, sigma)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for sigma in perms:
            oracle.transpose(coords, vals, sigma)
    dt = time.perf_counter() - t0
    value = args.steps * len(perms) * sample / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gnnz/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "int32+f64" if vals.dtype.itemsize == 8 else "int32+f32",
            "data": "synthetic",
            "config": {"workload": wl["name"], "dims": list(wl["dims"]), "nnz": nnz,
                       "sample_nnz": sample, "dists": [list(x) for x in wl["dists"]],
                       "perms": [list(p) for p in perms],
                       "input_order": list(range(len(wl["dims"])))},
            "cpu_baseline": {"value": value, "unit": "Gnnz/s", "cores": 1, "kind": "oracle",
                             "sample": f"{sample} entries sorted in input order (the workload's "
                                       f"generator at this count), {len(perms)} target orders "
                                       f"per step"},
            "e2e": {"value": value, "unit": "Gnnz/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    if not args.no_cpu_baseline:
        line["cpu_method"] = cpu_method_rate(coords, vals, wl["dims"], perms)
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="qsd", choices=["qsd", "reference"])
    ap.add_argument("--workload", default="deliciouslike", choices=sorted(WORKLOADS))
    ap.add_argument("--nnz", type=int, default=0, help="override the entry count")
    ap.add_argument("--perms", default="", help="comma-separated subset, e.g. 021,102")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=0,
                    help="entries the reference arm sorts per order and step (0: 2M for up to 5 "
                         "orders, 1M above, so that a step stays a few seconds)")
    ap.add_argument("--check", action="store_true", help="sampled parity check vs the oracle")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 256-tensor batched-vs-single-calls measurement")
    ap.add_argument("--no-tune", action="store_true", help="batched run without autotuning")
    ap.add_argument("--batched-steps", type=int, default=0,
                    help="timed runs of the batched workload (default: steps, 5..20)")
    ap.add_argument("--no-csf", action="store_true", help="skip the CSF-levels measurement")
    ap.add_argument("--no-topk", action="store_true",
                    help="skip Top-K-sadilla in the per-order table")
    ap.add_argument("--no-orders", action="store_true",
                    help="skip the per-order table (times, roofline fractions, no-skip ablation)")
    ap.add_argument("--graphs", type=int, default=1,
                    help="1: every order's call captured once into a CUDA graph (qsd_exec_*) "
                         "and the timed step replays the graphs")
    ap.add_argument("--tune", type=int, default=0,
                    help="1: tune every order's plan with qsd_plan_tune (measured choice among "
                         "equivalent executions) before the timed region")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the per-order tables of the other single-tensor workloads and "
                         "the 1M-entry latency")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the Poisson-stream serving measurement")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import paper_2005_10427_gb300 as qsd
    qsd.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = dict(WORKLOADS[args.workload])
    if args.nnz:
        wl = synth.scaled(wl, args.nnz)
    perms = wl["perms"]
    if args.perms:
        perms = [tuple(int(ch) for ch in p) for p in args.perms.split(",")]
    t = synth.make(wl, device=dev)
    torch.cuda.synchronize()
    r, nnz = t.coords.shape
    vb = t.vals.element_size()
    R = 4 * r + vb
    plans = [qsd.Plan(wl["dims"], sigma) for sigma in perms]
    tuned = None
    if args.tune:
        # qsd_plan_tune per order on the resident input (out of place, untimed)
        t0 = time.perf_counter()
        tuned = {}
        for i, sigma in enumerate(perms):
            p, ms, opts = qsd.tune_plan(plans[i], t.coords, t.vals, reps=2)
            plans[i] = p
            tuned["".join(map(str, sigma))] = {
                "ms": round(ms, 4), **{k: v for k, v in opts.items() if k != "validate"}}
        torch.cuda.synchronize()
        tuned = {"seconds": round(time.perf_counter() - t0, 2), "per_order": tuned}
    ws_bytes = max(p.workspace_bytes(nnz) for p in plans)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    cb = [torch.empty((r, nnz), dtype=torch.int32, device=dev) for _ in range(2)]
    vbuf = [torch.empty(nnz, dtype=t.vals.dtype, device=dev) for _ in range(2)]
    stream = torch.cuda.current_stream()
    execs = [qsd.Exec(t.coords, t.vals, cb, vbuf, nnz, p, ws) for p in plans] \
        if args.graphs else None

    def step():
        if execs is not None:
            for ex in execs:
                ex.launch(stream)
            return
        for p in plans:
            qsd.transpose_from(t.coords, t.vals, cb, vbuf, nnz, p, ws, stream)

    def step_plain():  # per-kernel timing (the launch profiler cannot see into graphs)
        for p in plans:
            qsd.transpose_from(t.coords, t.vals, cb, vbuf, nnz, p, ws, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    status = qsd.get_async_status()
    if status != 0:
        raise SystemExit(f"device status {status} after warm-up")

    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("single_timed")  # ncu --nvtx-include single_timed/
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    ms = combine_ranks(ev0.elapsed_time(ev1), world, dev)
    if world > 1:
        torch.distributed.barrier()
    ms_per_step = ms / args.steps
    entries_per_step = len(perms) * nnz
    value = aggregate_value(world, entries_per_step, args.steps, ms)

    # Live per-kernel timings over the same steps (instrumented replay).
    qsd.profile_reset()
    qsd.profile_enable(True)
    for _ in range(args.steps):
        step_plain()
    torch.cuda.synchronize()
    recs = qsd.profile_read()
    qsd.profile_enable(False)
    qsd.profile_reset()
    agg = {}
    for rec in recs:
        a = agg.setdefault(rec["kernel"], {"launches": 0, "ms": 0.0, "bytes": 0, "known": True})
        a["launches"] += 1
        a["ms"] += rec["ms"]
        if rec["algo_bytes"] < 0:
            a["known"] = False
        else:
            a["bytes"] += rec["algo_bytes"]
    total_ms = sum(a["ms"] for a in agg.values())
    top = max(agg, key=lambda k: agg[k]["ms"])
    peak, peak_kind = measured_peaks()
    achieved = agg[top]["bytes"] / (agg[top]["ms"] / 1e3) / 1e9 if agg[top]["ms"] > 0 else 0.0
    traffic_pe = committed_traffic(top, wl["name"])
    top_entries = sum(rec["entries"] for rec in recs if rec["kernel"] == top and rec["entries"] > 0)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "kernel": top,
                "traffic": (traffic_pe * top_entries / agg[top]["launches"]) if traffic_pe else None,
                "peak_kind": peak_kind,
                "algo_bytes_per_launch": agg[top]["bytes"] / max(agg[top]["launches"], 1),
                "avg_launch_ms": agg[top]["ms"] / max(agg[top]["launches"], 1),
                "share_of_device_time": round(agg[top]["ms"] / total_ms, 4) if total_ms else None,
                "whole_step_frac": round(
                    (2 * R * entries_per_step / (ms_per_step / 1e3) / 1e9) / peak, 4)}
    launches_per_step = len(recs) / args.steps

    # End to end through the host-buffer calls: every call copies its host
    # input in, transposes and copies the result out (pinned host memory).
    # Calls alternate between two streams, each with its own device buffers
    # and workspace (qsd_transpose_host_async), so one call's copy out
    # overlaps the next one's copy in and kernels, across steps too; the
    # timed region ends when both streams are done and the device status of
    # the calls is read.
    e2e = None
    if not args.no_e2e:
        hc = t.coords.cpu().pin_memory()
        hv = t.vals.cpu().pin_memory()
        # one result pair per stream: a stream's calls reuse it in stream order
        outs = [(torch.empty_like(hc).pin_memory(), torch.empty_like(hv).pin_memory())
                for _ in range(2)]
        streams = [stream, torch.cuda.Stream(device=dev)]
        cbs = [cb, [torch.empty((r, nnz), dtype=torch.int32, device=dev) for _ in range(2)]]
        vbs = [vbuf, [torch.empty(nnz, dtype=t.vals.dtype, device=dev) for _ in range(2)]]
        wss = [ws, torch.empty(ws.numel(), dtype=torch.uint8, device=dev)]
        e2e_steps = max(1, min(args.steps, 6))

        ncall = [0]

        def e2e_step():
            for p in plans:
                i = ncall[0] % 2
                ncall[0] += 1
                qsd.transpose_host_async(hc, hv, p, cbs[i], vbs[i], wss[i], outs[i][0],
                                         outs[i][1], streams[i])

        def e2e_wait():
            for i in range(2):
                if qsd.workspace_status(wss[i], streams[i]) != 0:
                    raise RuntimeError("device error in the end-to-end calls")

        e2e_step()  # warm-up
        e2e_wait()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        e2e_wait()
        dt = time.perf_counter() - t0
        del cbs[1], vbs[1], wss[1]
        e2e = {"value": world * entries_per_step * e2e_steps / dt / 1e9, "unit": "Gnnz/s",
               "h2d_bytes_per_step": len(plans) * nnz * R,
               "d2h_bytes_per_step": len(plans) * nnz * R, "streams": 2}

    csf = bench_csf(qsd, t, plans, perms, cb, vbuf, ws, stream) if not args.no_csf else None
    orders = None
    if not args.no_orders:
        orders = bench_orders(qsd, wl["dims"], t, perms, cb, vbuf, ws, stream,
                              topk=not args.no_topk)
    others = None
    if not args.no_others and rank == 0:
        others = {}
        for name, w in WORKLOADS.items():
            if w["name"] == wl["name"] or name == "uniform3d":
                continue
            others[name] = bench_other_workload(qsd, w, dev, stream)
        others["uniform3d_latency"] = bench_latency(qsd, synth.WORKLOAD_3D_UNIFORM, dev, stream)

    batched = None
    if not args.no_batched:
        del cb, vbuf
        batched = bench_batched(qsd, dev, stream, steps=args.batched_steps or max(5, min(args.steps, 20)),
                                warmup=args.warmup, tune=not args.no_tune)
        cb = [torch.empty((r, nnz), dtype=torch.int32, device=dev) for _ in range(2)]
        vbuf = [torch.empty(nnz, dtype=t.vals.dtype, device=dev) for _ in range(2)]

    serving = None
    if not args.no_serving and rank == 0:
        del cb, vbuf
        serving = bench_serving(qsd, dev)
        cb = [torch.empty((r, nnz), dtype=torch.int32, device=dev) for _ in range(2)]
        vbuf = [torch.empty(nnz, dtype=t.vals.dtype, device=dev) for _ in range(2)]

    check = None
    if args.check:
        check = sampled_check(qsd, t, plans, perms, cb, vbuf, ws, stream)

    # The CPU-baseline leg (the only part of the default run that executes
    # oracle/): the oracle, and beside it the paper's CPU method.
    cpu = cpu_method = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        hc, hv = t.coords.cpu().numpy(), t.vals.cpu().numpy()
        cpu = cpu_oracle_rate(hc, hv, perms)
        cpu_method = cpu_method_rate(hc, hv, wl["dims"], perms)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": "Gnnz/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32+f32" if vb == 4 else "int32+f64",
                "data": "synthetic",
                "config": {"workload": wl["name"], "dims": wl["dims"], "nnz": nnz,
                           "dists": [list(d) for d in wl["dists"]],
                           "perms": [list(p) for p in perms], "input_order": list(range(r)),
                           "out_of_place": True, "parallelism": f"replicas{world}",
                           "plans": "tuned (qsd_plan_tune per order, before the timed region)"
                                    if args.tune else "default options",
                           "calls": "CUDA graphs (qsd_exec_*), one per order" if args.graphs
                                    else "qsd_transpose_from_ws",
                           "l2": "inputs (%.2f GB) larger than L2; no flush" % (nnz * R / 1e9)},
                "roofline": roofline,
                "min_traffic_frac": roofline["whole_step_frac"],
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(round(launches_per_step * args.steps)),
                "launches_per_step": launches_per_step,
                "kernels": {k: {"launches": a["launches"], "ms": round(a["ms"], 3),
                                "share": round(a["ms"] / total_ms, 4) if total_ms else None}
                            for k, a in sorted(agg.items(), key=lambda kv: -kv[1]["ms"])},
                "clocks": clocks}
        if cpu_method is not None:
            line["cpu_method"] = cpu_method
        if csf is not None:
            line["csf"] = csf
        if tuned is not None:
            line["tuning"] = tuned
        if orders is not None:
            line["per_order"] = orders
        if others is not None:
            line["other_workloads"] = others
        if batched is not None:
            line["batched"] = batched
        if serving is not None:
            line["serving"] = serving
        if check is not None:
            line["check"] = check
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def bench_batched(qsd, dev, stream, steps: int, warmup: int, tune: bool = True):
    """The batched workload: 256 tensors (orders 3-5, log-uniform sizes in
    [1e3, 4e6] and dims in [100, 1e6], Zipf 1.1, float32 values, identity
    input order, a random non-identity target each) transposed by one graph
    launch per step, against the same tensors as back-to-back single calls
    (plain, and each captured once into a CUDA graph); every output of all
    three is compared bit for bit."""
    descs = synth.batch_workload()
    tens = [synth.gen_coo(d["dims"], d["nnz"], d["dists"], d["val_kind"], d["seed"], dev)
            for d in descs]
    plans = [qsd.Plan(d["dims"], d["perm"]) for d in descs]
    outs = [([torch.empty_like(t.coords) for _ in range(2)],
             [torch.empty_like(t.vals) for _ in range(2)]) for t in tens]
    batch = qsd.Batch([(p, t.coords, t.vals, o[0], o[1]) for p, t, o in zip(plans, tens, outs)])
    total = sum(t.nnz for t in tens)
    R_bytes = sum(t.nnz * (4 * t.order + t.vals.element_size()) for t in tens)
    ws = torch.empty(batch.workspace_bytes(), dtype=torch.uint8, device=dev)
    tuned, tune_s = None, None
    if tune:
        big = torch.empty(max(2 * batch.workspace_bytes(), batch.workspace_bytes() + (1 << 30)),
                          dtype=torch.uint8, device=dev)
        t0 = time.perf_counter()
        tuned = batch.tune(big, reps=2, stream=stream)
        tune_s = time.perf_counter() - t0
        del big
        ws = torch.empty(batch.workspace_bytes(), dtype=torch.uint8, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(warmup):
        batch.run(ws, stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("batched_timed")  # ncu --nvtx-include batched_timed/
    ev0.record(stream)
    for _ in range(steps):
        batch.run(ws, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    ms_b = ev0.elapsed_time(ev1) / steps
    if qsd.workspace_status(ws, stream) != 0:
        raise SystemExit("device status set by the batched run")

    # the same tensors as single calls, one after another on the stream
    souts = [([torch.empty_like(t.coords) for _ in range(2)],
              [torch.empty_like(t.vals) for _ in range(2)]) for t in tens]
    sws = torch.empty(max(p.workspace_bytes(t.nnz) for p, t in zip(plans, tens)),
                      dtype=torch.uint8, device=dev)
    sels = [0] * len(tens)

    def singles():
        for i, (p, t, o) in enumerate(zip(plans, tens, souts)):
            sels[i] = qsd.transpose_from(t.coords, t.vals, o[0], o[1], t.nnz, p, sws, stream)

    for _ in range(warmup):
        singles()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        singles()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_s = ev0.elapsed_time(ev1) / steps
    same = all(torch.equal(outs[i][0][batch.result(i)], souts[i][0][sels[i]]) and
               torch.equal(outs[i][1][batch.result(i)].view(torch.int32),
                           souts[i][1][sels[i]].view(torch.int32)) for i in range(len(tens)))

    # the same single calls, each captured once into a CUDA graph (qsd_exec_*)
    wss = [torch.empty(max(p.workspace_bytes(t.nnz), 256), dtype=torch.uint8, device=dev)
           for p, t in zip(plans, tens)]
    execs = [qsd.Exec(t.coords, t.vals, o[0], o[1], t.nnz, p, w)
             for p, t, o, w in zip(plans, tens, souts, wss)]
    gsels = [0] * len(tens)

    def singles_graphs():
        for i, ex in enumerate(execs):
            gsels[i] = ex.launch(stream)

    for _ in range(warmup):
        singles_graphs()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        singles_graphs()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_g = ev0.elapsed_time(ev1) / steps
    same = same and all(
        torch.equal(outs[i][0][batch.result(i)], souts[i][0][gsels[i]]) and
        torch.equal(outs[i][1][batch.result(i)].view(torch.int32),
                    souts[i][1][gsels[i]].view(torch.int32)) for i in range(len(tens)))
    del execs, wss
    peak, _ = measured_peaks()
    return {"workload": "batch256_r3-5_nnz1e3-4e6_zipf1.1_f32", "tensors": len(tens),
            "nnz_total": total, "steps": steps, "warmup": warmup,
            "batched": {"value": round(total / (ms_b / 1e3) / 1e9, 3), "unit": "Gnnz/s",
                        "ms_per_step": round(ms_b, 4), "graph_launches_per_step": 1,
                        "min_traffic_frac": round(2 * R_bytes / (ms_b / 1e3) / 1e9 / peak, 4)},
            "single_calls": {"value": round(total / (ms_s / 1e3) / 1e9, 3), "unit": "Gnnz/s",
                             "ms_per_step": round(ms_s, 4)},
            "single_calls_graphs": {"value": round(total / (ms_g / 1e3) / 1e9, 3),
                                    "unit": "Gnnz/s", "ms_per_step": round(ms_g, 4),
                                    "what": "each call captured once into a CUDA graph"},
            "speedup": round(ms_s / ms_b, 3),
            "speedup_vs_graph_calls": round(ms_g / ms_b, 3),
            "identical_outputs": bool(same),
            "tuned_options": tuned, "tune_seconds": None if tune_s is None else round(tune_s, 2)}


def _serve(qsd, srv, ids, pool, reqs, start, check_every, rid_clock):
    """Submits reqs (arrival offsets from `start`) from a driver thread, polls
    the results and keeps every check_every-th one. Returns (latencies,
    completion times, entries, kept results, errors)."""
    lat, done_t, kept, errors = [], [], {}, []
    entries = 0
    rid_of = {}
    clock = rid_clock

    def driver():
        for k, (off, i, perm) in enumerate(reqs):
            target = start + off
            while True:
                dt = target - clock()
                if dt <= 0:
                    break
                time.sleep(dt - 0.0002 if dt > 0.0005 else 0)
            rid_of[srv.submit(ids[i], perm, arrival_s=target)] = k

    th = threading.Thread(target=driver)
    th.start()
    got = 0
    t0 = time.perf_counter()
    while got < len(reqs):
        for r in srv.poll(512, wait_ms=20):
            got += 1
            if r["status"] != 0:
                errors.append(r["status"])
                srv.release(r["request"])
                continue
            lat.append(r["done_s"] - r["arrival_s"])
            done_t.append(r["done_s"])
            entries += r["nnz"]
            while r["request"] not in rid_of and th.is_alive():
                time.sleep(0.0001)
            k = rid_of.get(r["request"], -1)
            if k >= 0 and k % check_every == 0:
                t = pool[reqs[k][1]]
                oc = torch.empty_like(t.coords)
                ov = torch.empty_like(t.vals)
                srv.copy_result(r["request"], oc, ov)
                torch.cuda.current_stream().synchronize()  # copied before the memory is reused
                kept[k] = (oc, ov)
            srv.release(r["request"])
        if not th.is_alive() and got < len(reqs) and time.perf_counter() - t0 > 600:
            break
    th.join()
    torch.cuda.synchronize()
    return lat, done_t, entries, kept, errors


def _lat_stats(lat, done_t, start, entries):
    lat_ms = np.array(lat) * 1e3
    span = max(done_t) - start if done_t else float("nan")
    return {"value": round(entries / span / 1e9, 3), "unit": "Gnnz/s",
            "seconds": round(span, 3),
            "p50_ms": round(float(np.percentile(lat_ms, 50)), 3),
            "p99_ms": round(float(np.percentile(lat_ms, 99)), 3),
            "mean_ms": round(float(lat_ms.mean()), 3), "max_ms": round(float(lat_ms.max()), 3)}


def bench_serving(qsd, dev, budget_gb: float = 40.0, n_requests: int = 10_000,
                  rate: float = 2000.0, check_every: int = 200):
    """The serving workload: a resident pool of 64 tensors (orders 3-4,
    log-uniform sizes in [1e4, 5e7], Zipf 1.2, float64 values) and 10k
    requests, each a random non-identity target order of a random pool
    tensor, served under a 40 GB budget by the continuous-batching server.
    Latency = arrival to completion on the device.

    Three arms over the same request list:
      poisson      arrivals as a Poisson stream at 2k/s (the offered load);
      saturated    every request queued at once, so the server runs at its
                   capacity (continuous batching with full steps);
      single_calls the requests as back-to-back out-of-place single calls on
                   one stream (the same plans, one call each).
    Every check_every-th result of both served arms is compared bit for bit
    with the single call's result for that request (alone vs in the mix)."""
    pool_desc, reqs = synth.serving_workload(n_requests=n_requests, rate=rate)
    t0 = time.perf_counter()
    pool = [synth.gen_coo(d["dims"], d["nnz"], d["dists"], d["val_kind"], d["seed"], dev)
            for d in pool_desc]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    clock = qsd.server_clock

    def new_server():
        srv = qsd.Server(int(budget_gb * (1 << 30)), val_bytes=8, streams=2, max_batch=256)
        ids = [srv.add_tensor(t.coords, t.vals, t.dims) for t in pool]
        # warm-up: a few requests per order (plans, code paths), not timed
        for i in range(min(8, len(pool))):
            srv.submit(ids[i], list(reversed(range(pool[i].order))))
        warm = 0
        while warm < min(8, len(pool)):
            for r in srv.poll(64, wait_ms=100):
                srv.release(r["request"])
                warm += 1
        return srv, ids

    arms = {}
    kept_all = {}
    for arm in ("poisson", "saturated"):
        srv, ids = new_server()
        arm_reqs = reqs if arm == "poisson" else [(0.0, i, perm) for _, i, perm in reqs]
        start = clock() + 0.05
        lat, done_t, entries, kept, errors = _serve(qsd, srv, ids, pool, arm_reqs, start,
                                                    check_every, clock)
        stats = srv.stats()
        srv.close()
        a = _lat_stats(lat, done_t, start, entries)
        a.update({"completed": len(lat), "errors": len(errors), "steps": stats["steps"],
                  "mean_batch": round(stats["admitted"] / max(stats["steps"], 1), 2),
                  "max_queue_depth": stats["max_queue_depth"],
                  "max_inflight": stats["max_inflight_seen"],
                  "peak_budget_gb": round(stats["peak_bytes"] / (1 << 30), 3)})
        arms[arm] = a
        kept_all[arm] = kept
        del kept

    # the same requests as back-to-back single calls, CUDA events around all
    plans = {}
    for _, i, perm in reqs:
        if (i, perm) not in plans:
            plans[(i, perm)] = qsd.Plan(pool[i].dims, perm)
    nmax = max(t.nnz for t in pool)
    rmax = max(t.order for t in pool)
    cbuf = [torch.empty((rmax, nmax), dtype=torch.int32, device=dev) for _ in range(2)]
    vbuf = [torch.empty(nmax, dtype=torch.float64, device=dev) for _ in range(2)]
    ws = torch.empty(max(p.workspace_bytes(pool[i].nnz) for (i, _), p in plans.items()),
                     dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    views = {}
    for t in pool:
        key = (t.order, t.nnz)
        if key not in views:
            views[key] = ([c[:t.order, :t.nnz] for c in cbuf], [v[:t.nnz] for v in vbuf])

    def single(k):
        _, i, perm = reqs[k]
        t = pool[i]
        cb, vb = views[(t.order, t.nnz)]
        return qsd.transpose_from(t.coords, t.vals, cb, vb, t.nnz, plans[(i, perm)], ws, stream)

    for k in range(min(16, len(reqs))):
        single(k)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(len(reqs)):
        single(k)
    ev1.record(stream)
    torch.cuda.synchronize()
    if qsd.workspace_status(ws, stream) != 0:
        raise SystemExit("device status set by the single-call arm")
    ms_single = ev0.elapsed_time(ev1)
    total_entries = sum(pool[i].nnz for _, i, _ in reqs)
    arms["single_calls"] = {"value": round(total_entries / (ms_single / 1e3) / 1e9, 3),
                            "unit": "Gnnz/s", "seconds": round(ms_single / 1e3, 3)}

    # alone vs in the mix: the single call's result for each kept request
    same = True
    checked = 0
    for arm, kept in kept_all.items():
        for k, (oc, ov) in kept.items():
            t = pool[reqs[k][1]]
            sel = single(k)
            cb, vb = views[(t.order, t.nnz)]
            same &= bool(torch.equal(cb[sel], oc) and
                         torch.equal(vb[sel].view(torch.int64), ov.view(torch.int64)))
            checked += 1
    offered = total_entries / reqs[-1][0] / 1e9
    return {"workload": "serve10k_poisson2000_pool64_r3-4_nnz1e4-5e7_zipf1.2_f64",
            "requests": len(reqs), "budget_gb": budget_gb, "offered_gnnz_s": round(offered, 3),
            **{k: v for k, v in arms["poisson"].items()},
            "saturated": arms["saturated"], "single_calls": arms["single_calls"],
            "saturated_vs_single_calls": round(arms["saturated"]["value"] /
                                               arms["single_calls"]["value"], 3),
            "alone_vs_mix_checked": checked, "alone_vs_mix_identical": bool(same),
            "pool_gen_seconds": round(gen_s, 1)}


def bench_csf(qsd, t, plans, perms, cb, vbuf, ws, stream, reps: int = 5):
    """CSF levels of each transposed output. Per order: the transposition
    alone, the separate CSF build on its result (qsd_csf_build: a count and a
    write sweep over every coordinate row), and the fused call
    (qsd_transpose_csf_from_ws: the last movement leaves each entry's first
    differing level, the CSF pass reads those bytes). Device times, CUDA
    events; fused_csf_ms = fused - transposition alone."""
    r, nnz = t.coords.shape
    dev = t.coords.device
    ids = [torch.empty(nnz, dtype=torch.int32, device=dev) for _ in range(r)]
    ptr = [torch.empty(2 if l == 0 else nnz + 1, dtype=torch.int32, device=dev)
           for l in range(r + 1)]
    nodes = torch.empty(r + 1, dtype=torch.int32, device=dev)
    cws = torch.empty(qsd.csf_workspace_bytes(r, nnz), dtype=torch.uint8, device=dev)
    fws = torch.empty(max(qsd.transpose_csf_workspace_bytes(p, nnz) for p in plans),
                      dtype=torch.uint8, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(2):
            fn()
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    per = {}
    for p, sigma in zip(plans, perms):
        sel = qsd.transpose_from(t.coords, t.vals, cb, vbuf, nnz, p, ws, stream)
        rows = cb[sel]
        ms_build = timed(lambda: qsd.csf_build(rows, sigma, ids, ptr, nodes, cws, stream))
        n = [int(x) for x in nodes.cpu()]
        ms_t = timed(lambda: qsd.transpose_from(t.coords, t.vals, cb, vbuf, nnz, p, ws, stream))
        ms_f = timed(lambda: qsd.transpose_csf_from(t.coords, t.vals, cb, vbuf, nnz, p, ids, ptr,
                                                    nodes, fws, stream))
        if qsd.workspace_status(fws, stream) != 0:
            raise SystemExit("device status set by the fused transposition")
        written = 4 * (sum(n[1:]) + sum(n) + 1 + r)  # ids and ptr entries
        per["".join(map(str, sigma))] = {
            "csf_build_ms": round(ms_build, 4), "transpose_ms": round(ms_t, 4),
            "fused_ms": round(ms_f, 4), "fused_csf_ms": round(ms_f - ms_t, 4),
            "separate_total_ms": round(ms_t + ms_build, 4),
            "csf_build_gb_s": round((2 * 4 * r * nnz + written) / (ms_build / 1e3) / 1e9, 1),
            "nodes": n}
    tot_sep = sum(v["separate_total_ms"] for v in per.values())
    tot_f = sum(v["fused_ms"] for v in per.values())
    return {"what": "CSF levels of each transposed output: separate build (count and write "
                    "sweeps over every row) vs fused into the transposition's last movement",
            "sum_ms": {"separate": round(tot_sep, 3), "fused": round(tot_f, 3)},
            "per_order": per}


def _time_calls(qsd, plan, t, cb, vbuf, ws, stream, reps: int, warm: int = 2) -> float:
    """Mean device time (ms) of one out-of-place call, CUDA events on the
    launching stream around `reps` back-to-back calls after `warm` calls."""
    nnz = t.coords.shape[1]
    need = plan.workspace_bytes(nnz)
    w = ws if need <= ws.numel() else torch.empty(need, dtype=torch.uint8, device=ws.device)
    for _ in range(warm):
        qsd.transpose_from(t.coords, t.vals, cb, vbuf, nnz, plan, w, stream)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(reps):
        qsd.transpose_from(t.coords, t.vals, cb, vbuf, nnz, plan, w, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    if qsd.workspace_status(w, stream) != 0:
        raise SystemExit("device status set in the per-order timing")
    return ev0.elapsed_time(ev1) / reps


def _groups(plan):
    return [["".join(map(str, g["prefix"])), "".join(map(str, g["keys"])), g["passes"]]
            for g in plan.info()["groups"]]


def bench_orders(qsd, dims, t, perms, cb, vbuf, ws, stream, reps: int = 5, topk: bool = True):
    """Per target order: device time of one out-of-place call, Gnnz/s and the
    whole transposition's fraction of the minimum-traffic roofline (one read
    and one write of every coordinate and value, 2 R bytes per entry, against
    the measured copy bandwidth); the same for the no-skip plan (a full LSD
    radix sort over every mode on the same kernels: the baseline whose passes
    Algorithm 3 skips), the (key, index) form where the plan has a group that
    takes it, and, for every K an order allows, Top-K-sadilla."""
    r, nnz = t.coords.shape
    R = 4 * r + t.vals.element_size()
    peak, _ = measured_peaks()
    per = {}
    tot_q = tot_ns = 0.0
    for sigma in perms:
        row = {}
        variants = [("quesadilla", {}), ("no_skip", {"no_skip": True})]
        if any(g["key_index"] for g in qsd.Plan(dims, sigma, key_index=True).info()["groups"]):
            variants.append(("key_index", {"key_index": True}))
        variants.append(("first_digit6", {"first_digit_bits": 6}))
        if topk:
            variants += [(f"topk{K}", {"top_k": K}) for K in range(1, r - 1)]
        for label, kw in variants:
            p = qsd.Plan(dims, sigma, **kw)
            ms = _time_calls(qsd, p, t, cb, vbuf, ws, stream, reps)
            row[label] = {"ms": round(ms, 4), "gnnz_s": round(nnz / (ms / 1e3) / 1e9, 2),
                          "whole_transpose_frac": round(2 * R * nnz / (ms / 1e3) / 1e9 / peak, 4),
                          "groups": _groups(p)}
        tot_q += row["quesadilla"]["ms"]
        tot_ns += row["no_skip"]["ms"]
        per["".join(map(str, sigma))] = row
    return {"what": "single out-of-place calls per target order; whole_transpose_frac = "
                    "2*R*nnz / time / measured copy bandwidth; no_skip = full LSD radix sort "
                    "over every mode on the same kernels; topkK = Top-K-sadilla",
            "bytes_per_entry_min": 2 * R,
            "sum_ms": {"quesadilla": round(tot_q, 3), "no_skip": round(tot_ns, 3),
                       "first_digit6": round(sum(v["first_digit6"]["ms"] for v in per.values()),
                                             3),
                       "best_of_quesadilla_and_key_index": round(sum(
                           min(v["quesadilla"]["ms"], v.get("key_index", v["quesadilla"])["ms"])
                           for v in per.values()), 3)},
            "skipping_speedup": round(tot_ns / tot_q, 3) if tot_q else None,
            "per_order": per}


def bench_other_workload(qsd, wl, dev, stream, reps: int = 5):
    """Another single-tensor workload's per-order table (generated on the
    device, timed like the line's own orders, then freed)."""
    t = synth.make(wl, device=dev)
    r, nnz = t.coords.shape
    plans = [qsd.Plan(wl["dims"], s) for s in wl["perms"]]
    ws = torch.empty(max(max(p.workspace_bytes(nnz) for p in plans),
                         max(qsd.Plan(wl["dims"], s, no_skip=True).workspace_bytes(nnz)
                             for s in wl["perms"])), dtype=torch.uint8, device=dev)
    cb = [torch.empty((r, nnz), dtype=torch.int32, device=dev) for _ in range(2)]
    vbuf = [torch.empty(nnz, dtype=t.vals.dtype, device=dev) for _ in range(2)]
    out = bench_orders(qsd, wl["dims"], t, wl["perms"], cb, vbuf, ws, stream, reps=reps,
                       topk=False)
    tot = out["sum_ms"]["quesadilla"]
    R = 4 * r + t.vals.element_size()
    peak, _ = measured_peaks()
    out["workload"] = wl["name"]
    out["value"] = round(len(plans) * nnz / (tot / 1e3) / 1e9, 3)
    out["unit"] = "Gnnz/s"
    out["whole_step_frac"] = round(2 * R * nnz * len(plans) / (tot / 1e3) / 1e9 / peak, 4)
    del t, cb, vbuf, ws
    torch.cuda.empty_cache()
    return out


def bench_latency(qsd, wl, dev, stream, calls: int = 50):
    """Latency of one single out-of-place call on a small tensor (1M entries
    fit the L2 cache, so this measures launch and latency, not bandwidth):
    CUDA events around every call, min and median; plain calls, the key-index
    form, and the call captured into a CUDA graph (qsd_exec_*)."""
    t = synth.make(wl, device=dev)
    r, nnz = t.coords.shape
    out = {"workload": wl["name"]}
    variants = [(s, kw, g) for s in wl["perms"]
                for kw, g in (({}, False), ({"key_index": True}, False), ({}, True))]
    for sigma, kw, graph in variants:
        p = qsd.Plan(wl["dims"], sigma, **kw)
        ws = torch.empty(p.workspace_bytes(nnz), dtype=torch.uint8, device=dev)
        cb = [torch.empty((r, nnz), dtype=torch.int32, device=dev) for _ in range(2)]
        vbuf = [torch.empty(nnz, dtype=t.vals.dtype, device=dev) for _ in range(2)]
        if graph:  # the call captured once into a CUDA graph (qsd_exec_*)
            ex = qsd.Exec(t.coords, t.vals, cb, vbuf, nnz, p, ws)
            call = lambda: ex.launch(stream)  # noqa: E731
        else:
            call = lambda: qsd.transpose_from(t.coords, t.vals, cb, vbuf, nnz, p, ws,  # noqa: E731
                                              stream)
        for _ in range(5):
            call()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(calls)]
        for a, b in evs:
            a.record(stream)
            call()
            b.record(stream)
        torch.cuda.synchronize()
        if qsd.workspace_status(ws, stream) != 0:
            raise SystemExit("device status set in the latency run")
        us = sorted(a.elapsed_time(b) * 1e3 for a, b in evs)
        out["".join(map(str, sigma)) + ("_key_index" if kw else "") + ("_graph" if graph else "")] = {
            "min_us": round(us[0], 1), "median_us": round(us[len(us) // 2], 1),
            "gnnz_s_at_median": round(nnz / (us[len(us) // 2] / 1e6) / 1e9, 2),
            "groups": _groups(p)}
    return out


def sampled_check(qsd, t, plans, perms, cb, vbuf, ws, stream):
    """Properties that hold at any size, checked on the device: the output
    is sorted under sigma and is the same multiset of (coordinates, value)
    records as the input (an order-independent hash)."""
    out = {}
    c_in = t.coords
    nnz = c_in.shape[1]
    for p, sigma in zip(plans, perms):
        sel = qsd.transpose_from(t.coords, t.vals, cb, vbuf, nnz, p, ws, stream)
        oc, ov = cb[sel], vbuf[sel]
        keys = [oc[m].long() for m in sigma]
        lt = torch.zeros(nnz - 1, dtype=torch.bool, device=oc.device)
        eq = torch.ones(nnz - 1, dtype=torch.bool, device=oc.device)
        for k in keys:
            lt |= eq & (k[:-1] < k[1:])
            eq &= k[:-1] == k[1:]
        sorted_ok = bool(lt.all())

        def h(c, v):
            x = v.view(torch.int32).long() if v.element_size() == 4 else v.view(torch.int64)
            acc = x * 0x9E3779B1
            for m in range(c.shape[0]):
                acc = acc ^ (c[m].long() * (0x85EBCA77 + 2 * m + 1))
                acc = acc * 0x27D4EB2F + 0x165667B1
            return int(acc.sum())
        ok_hash = h(c_in, t.vals) == h(oc, ov)
        out["".join(map(str, sigma))] = bool(sorted_ok and ok_hash)
    torch.cuda.synchronize()
    return out


if __name__ == "__main__":
    sys.exit(main())
