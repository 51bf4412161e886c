#!/usr/bin/env python3
"""Benchmark: time-to-discord and pair-distances/s on one GB300.

Workload: a float32 random walk of m = 2^20 points with five injected
anomalies (seed 0), subsequence length n = 256 -- the size of the paper's
SCD-1M experiments (Section 4), synthetic because the SCD series are not
available.  One step = one full discord search (Algorithm 2: preparation,
PotentialDiscord, RefineDiscord, argmax) through the C ABI with the series
resident on the device.

value  = brute-force-equivalent unordered non-self pairs per second,
         P_u / time-to-discord with P_u = (N-n)(N-n+1)/2;
e2e    = the same metric through dd_find_discord_host (pinned host series,
         H2D copy and result D2H inside the timed region);
roofline = the distance-tile kernel, algorithmic work / its CUDA-event time
         against the GB300 peak of the pipe that bounds it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--precision all|best|fp32|tc_fp16|tc_bf16]
By default every form is timed (the metric compares the tensor-core forms with the
plain FP32 form); the headline value is the fastest exact (tensor-core) form.
Under torchrun each rank runs an independent replica (the search does not
exchange data between GPUs); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair-distances/s & time-to-discord (m=2^20,n=256), TC vs FP32; serve p99 ms"
UNIT = "pair-distances/s"
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM (Blackwell)


def _alu_peak(sms: int, peaks) -> float:
    """FP32 lane instructions per second: SMs x 128 lanes x the maximum SM clock (T/s)."""
    return sms * FP32_LANES_PER_SM * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


def _probe_peaks(dd, dev) -> dict:
    """The FP16 and FP32 / FP64 peaks the driver does not measure: cuBLAS FP16 (and BF16, for
    the ratio) dense 8192^3 GEMMs, best of 10 after warm-up, and the library's own FMA-rate
    probes of the CUDA cores."""
    import torch
    out = {}
    for name, dt in (("fp16", torch.float16), ("bf16", torch.bfloat16)):
        a = torch.randn(8192, 8192, device=dev, dtype=dt)
        b = torch.randn(8192, 8192, device=dev, dtype=dt)
        for _ in range(3):
            torch.matmul(a, b)
        ts = []
        for _ in range(10):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        out[f"{name}_tflops_cublas"] = 2.0 * 8192 ** 3 / (min(ts) * 1e-3) / 1e12
        del a, b
    out["fp32_fma_per_s"] = dd.probe_fma_rate(False)
    out["fp64_fma_per_s"] = dd.probe_fma_rate(True)
    out["fp32_tflops"] = 2.0 * out["fp32_fma_per_s"] / 1e12
    out["fp64_tflops"] = 2.0 * out["fp64_fma_per_s"] / 1e12
    out["how"] = ("torch.matmul 8192^3 fp16 / bf16, best of 10 (CUDA events); dd_probe_fma_rate: independent "
                  "FFMA / DFMA chains on every SM for ~20 ms")
    torch.cuda.empty_cache()
    return out


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def _pairs_unordered(N: int, n: int) -> int:
    k = N - n
    return k * (k + 1) // 2 if k > 0 else 0


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index: int):
        self.dev = dev_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self, busy_floor_mhz: float = 0.0):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, fl in rows for k, v in enumerate(fl) if v.lower() == "active"})
        loaded = [r[0] for r in rows if r[0] >= busy_floor_mhz] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def _kernel_traffic(precision: str):
    """dram bytes per launch of the distance kernel from the committed ncu
    summary, or None if a source it depends on changed since it was taken: the
    kernel itself and the search that schedules its waves (the sha-256 of the
    files' bytes concatenated in the listed order, first 16 hex digits)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    ent = d.get(precision)
    if not ent:
        return None
    try:
        blob = b"".join(open(os.path.join(ROOT, "paper_1901_00155_gb300", "csrc", f), "rb").read()
                        for f in ent["sources"])
    except Exception:
        return None
    h = hashlib.sha256(blob).hexdigest()[:16]
    return ent["dram_bytes_per_launch"] if h == ent.get("sources_sha256_16") else None


def _exhaustive(dd, Td, m: int, n: int, forms, peaks, sms: int, rows: int = 8192, reps: int = 3) -> dict:
    """Exhaustive mode (no abandon, metric (i)): dd_nn_rows over `rows` evenly spaced
    rows against all N columns, CUDA events around each call on its stream."""
    import torch
    N = m - n + 1
    stride = max(1, N // rows)
    R = torch.arange(0, stride * rows, stride, dtype=torch.int32, device=Td.device)
    R = R[R < N].contiguous()
    out = {}
    for prec in forms:
        with dd.Plan(m, n, prec) as p:
            y = p.nn_rows(Td, R)
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                p.nn_rows(Td, R, out=y)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        pairs = R.numel() * N
        if prec == "fp32":
            work = 2.0 * n * pairs / (ms * 1e-3) / 1e12
            peak = _alu_peak(sms, peaks)
            unit = "Tinstr/s"
        else:
            work = 2.0 * plan_nkpad(n) * pairs / (ms * 1e-3) / 1e12
            peak = float(peaks.get("bf16_tflops", 1900.0))
            unit = "TFLOP/s"
        out[prec] = {"pairs_per_s": pairs / (ms * 1e-3), "ms": ms, "rows": int(R.numel()), "columns": N,
                     "achieved": work, "unit": unit, "peak": peak, "frac": work / peak}
    return out


def _window(dd, Td, m: int, n: int, peaks, sms: int, reps: int = 3) -> dict:
    """Per-window z-normalised discords and the diagonal-recurrence profile (exhaustive, every
    pair once): time to the exact per-window discord, and the global-form profile rate next to
    the direct FP32 exhaustive rate.  The recurrence kernel is bound by the FP32/ALU issue rate;
    its algorithmic work is 6 lane instructions per pair (2 FMA of the recurrence, 2 for the
    score, the row and the column minimum)."""
    import torch
    N = m - n + 1
    pairs = _pairs_unordered(N, n)
    peak = _alu_peak(sms, peaks)
    out = {}
    with dd.Plan(m, n, znorm="window") as p:
        p.set_profiling(True)
        r = p.find_discord(Td)
        ts, kms = [], []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            r = p.find_discord(Td)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            kms.append(p.profile()["dist_ms"])
        ms, kd = statistics.median(ts), statistics.median(kms)
        ach = 6.0 * pairs / (kd * 1e-3) / 1e12
        out["window_discord"] = {"time_to_discord_ms": ms, "index": r.index, "nn_distance": r.nn_distance,
                                 "exact": r.exact, "candidates_rescored": r.candidates,
                                 "pairs_per_s": pairs / (ms * 1e-3), "k_diag_ms": kd,
                                 "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Tinstr/s",
                                              "frac": ach / peak, "kernel": "k_diag<window>",
                                              "work": "6 lane instructions per pair"}}
    with dd.Plan(m, n, diag=True) as p:
        p.set_profiling(True)
        y = p.nn_profile_diag(Td)
        ts, kms = [], []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            p.nn_profile_diag(Td, out=y)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        out["global_diag_profile"] = {"ms": ms, "pairs": pairs, "pairs_per_s": pairs / (ms * 1e-3)}
    return out


def _batch(dd, precision: str, count: int = 512, reps: int = 5) -> dict:
    """Many uneven series (m log-uniform in [2048, 65536], n in {64, 128, 256}) resident on
    the device.  Fused: one dd_batch_search per call (every step of the search one launch over
    all series, the call's launches a CUDA graph that later calls with the same shapes replay);
    median of `reps` calls after one warm-up call that captures the graph.  Engine: one
    dd_find_discord_batched call (32 workers, per-series searches side by side)."""
    import torch
    from paper_1901_00155_gb300 import synth
    specs = synth.workload_batch(0, count)
    series = [torch.from_numpy(synth.make_series(s)[0]).cuda() for s in specs]
    ns = [s.n for s in specs]
    pairs = sum(_pairs_unordered(s.m - s.n + 1, s.n) for s in specs)
    out = {"workload": f"{count} series, m log-uniform [2048, 65536], n in {{64,128,256}}, rw/sine, seed 0",
           "precision": precision, "unit": "pair-distances/s (brute-force equivalent)"}
    with dd.Batch(count, sum(int(t.numel()) for t in series), max(ns), precision) as b:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fused = b.search(series, ns)  # captures the graph
        first = time.perf_counter() - t0
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fused = b.search(series, ns)
            ts.append(time.perf_counter() - t0)
        dt = statistics.median(ts)
        out["fused"] = {"ms": dt * 1e3, "first_call_ms": first * 1e3, "series_per_s": count / dt,
                        "value": pairs / dt, "graph_replays": b.graph_replays(),
                        "failed": sum(1 for r in fused if isinstance(r, Exception))}
    dd.find_discord_batched(series[:16], ns[:16], precision)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = dd.find_discord_batched(series, ns, precision)
    dt_e = time.perf_counter() - t0
    out["engine"] = {"ms": dt_e * 1e3, "series_per_s": count / dt_e, "value": pairs / dt_e, "workers": 32,
                     "failed": sum(1 for r in res if isinstance(r, Exception))}
    out["index_mismatches"] = sum(1 for a, c in zip(fused, res)
                                  if isinstance(a, Exception) or isinstance(c, Exception) or a.index != c.index)
    out.update(ms=out["fused"]["ms"], series_per_s=out["fused"]["series_per_s"], value=out["fused"]["value"])
    return out


SIZE_CLASSES = (("m<2^15", 0, 1 << 15), ("2^15<=m<2^18", 1 << 15, 1 << 18), ("m>=2^18", 1 << 18, 1 << 62))


def _serve(dd, precision: str, duration_s: float = 20.0, workers: int = 8, rate: float = 200.0) -> dict:
    """Poisson arrivals (rate per s) of host series (m log-uniform in [4096, 2^20], n in
    {64, ..., 1024}) into an engine of `workers` admitting by device memory; latency =
    submission -> result on the host (queue + host->device copy + plan + search + result copy),
    overall and per size class of m."""
    import torch
    from paper_1901_00155_gb300 import synth
    trace = synth.serving_requests(0, rate, duration_s)
    series = [torch.from_numpy(synth.make_series(s)[0]).pin_memory() for _, s in trace]
    lat = []
    with dd.Engine(workers, 1 << 20, 1024, precision) as E:
        for k in range(min(workers, len(trace))):  # warm-up: every worker once
            E.submit(series[k], trace[k][1].n, id=-1 - k)
        E.drain()
        t_start = time.perf_counter()
        done = []
        for k, (t, s) in enumerate(trace):
            while True:
                now = time.perf_counter() - t_start
                if now >= t:
                    break
                done += E.poll(256, 0)
                time.sleep(min(0.0005, t - now))
            E.submit(series[k], s.n, id=k)
        done += E.drain()
        t_end = time.perf_counter()
    failed = sum(1 for c in done if isinstance(c.result, Exception))

    def stats(cs):
        lat = sorted(c.queue_ms + c.service_ms for c in cs)
        if not lat:
            return {"requests": 0}
        q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))]  # noqa: E731
        return {"requests": len(lat), "p50_ms": q(0.50), "p99_ms": q(0.99), "max_ms": lat[-1],
                "mean_ms": sum(lat) / len(lat), "mean_queue_ms": sum(c.queue_ms for c in cs) / len(cs)}

    measured = [c for c in done if c.id >= 0]
    by_class = {name: stats([c for c in measured if lo <= trace[c.id][1].m < hi]) for name, lo, hi in SIZE_CLASSES}
    out = {"workload": f"Poisson {rate:g}/s for {duration_s:g} s ({len(trace)} requests), m log-uniform "
                       f"[4096, 2^20], n in {{64..1024}}, host series, seed 0",
           "precision": precision, "workers": workers, "admission": "device-memory budget (default), bypass <= 32",
           "failed": failed, "throughput_rps": len(measured) / (t_end - t_start)}
    out.update(stats(measured))
    out["by_size_class"] = by_class
    return out


def _reference_arm(args, rank: int):
    """The FP64 oracle (CPU HOTSAX, Algorithms 2-4) on the host cores, each step a
    bounded prefix sample of the benchmark workload."""
    if rank != 0:
        return
    import oracle
    from paper_1901_00155_gb300 import synth
    spec = synth.workload_large(0)
    T, _ = synth.make_series(spec)
    m_s = 1 << 16
    Ts = T[:m_s].copy()
    N_s = m_s - spec.n + 1
    oracle.build()
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.hotsax(Ts, spec.n)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    t = statistics.mean(times)
    value = _pairs_unordered(N_s, spec.n) / t
    sample = f"first {m_s} points of the m=2^20 n=256 random walk (CPU HOTSAX, FP64), per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"rw m={m_s} n={spec.n} (prefix of the m=2^20 benchmark series)",
                       "m": m_s, "n": spec.n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _cpu_baseline():
    """The FP64 oracle's CPU HOTSAX on a bounded prefix of the benchmark series (about 10-30 s on
    the host's cores), as it stands."""
    import oracle
    from paper_1901_00155_gb300 import synth
    spec = synth.workload_large(0)
    T, _ = synth.make_series(spec)
    m_s = 1 << 18
    Ts = T[:m_s].copy()
    oracle.build()
    t0 = time.perf_counter()
    oracle.hotsax(Ts, spec.n)
    dt = time.perf_counter() - t0
    N_s = m_s - spec.n + 1
    return {"value": _pairs_unordered(N_s, spec.n) / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"CPU HOTSAX (FP64 oracle) on the first {m_s} points of the workload series, n={spec.n}: "
                      f"{dt:.2f} s"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="all", choices=["all", "best", "fp32", "tc_fp16", "tc_bf16"],
                    help="all (default): every form, headline on the fastest exact one; best: the first "
                         "supported tensor-core form only")
    ap.add_argument("--no-probe", action="store_true", help="skip the FP16 / FP32 / FP64 peak probes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-series batched search")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the 512-series batch (fused and engine) and print its JSON object")
    ap.add_argument("--batch-reps", type=int, default=5, help="timed fused-batch calls (median)")
    ap.add_argument("--eager", action="store_true",
                    help="enqueue each search's kernels directly instead of replaying its CUDA graph "
                         "(per-kernel profilers cannot profile kernels of graphs with conditional nodes)")
    ap.add_argument("--no-serve", action="store_true", help="skip the Poisson serving run (p50/p99)")
    ap.add_argument("--no-window", action="store_true",
                    help="skip the per-window discord and diagonal-recurrence profile")
    ap.add_argument("--no-exhaustive", action="store_true",
                    help="skip the exhaustive-mode (no abandon) pair-distances/s of each form")
    ap.add_argument("--workload", default="large", choices=["large", "medium"],
                    help="large: m=2^20 n=256 (the benchmark); medium: m=262144 n=256 (profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        _reference_arm(args, rank)
        return

    import torch
    import torch.distributed as dist

    import paper_1901_00155_gb300 as dd
    from paper_1901_00155_gb300 import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.batch_only:
        print(json.dumps(_batch(dd, "tc_fp16" if args.precision in ("all", "best") else args.precision,
                                reps=max(1, args.batch_reps))))
        return
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    spec = synth.workload_large(0) if args.workload == "large" else synth.workloads_medium()[2]
    T, _ = synth.make_series(spec)
    m, n = spec.m, spec.n
    N = m - n + 1
    P_u = _pairs_unordered(N, n)
    Td = torch.from_numpy(T).to(dev)
    Th = torch.from_numpy(T).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 126 MB L2
    peaks, peak_src = _peaks()

    supported = []
    for prec in ("tc_fp16", "tc_bf16", "fp32"):
        try:
            dd.Plan(m, n, prec).close()
            supported.append(prec)
        except dd.DDError:
            pass
    if args.precision == "best":
        forms = [supported[0]]
    elif args.precision == "all":
        forms = supported
    else:
        forms = [args.precision]

    results = {}
    clocks_all = None
    for prec in forms:
        plan = dd.Plan(m, n, prec)
        plan.set_profiling(True)
        if args.eager:
            plan.set_graph(False)
        for _ in range(args.warmup):
            plan.find_discord(Td)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        step_ms, dist_ms, pairs, launches, dlaunch = [], 0.0, 0, 0, 0
        res = None
        barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as cs:
            for _ in range(args.steps):
                flush.fill_(1)  # evict the series and workspace from L2 (not timed)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                res = plan.find_discord(Td)
                e1.record(stream)
                e1.synchronize()
                step_ms.append(e0.elapsed_time(e1))
                pr = plan.profile()
                dist_ms += pr["dist_ms"]
                pairs += pr["computed_pairs"]
                dlaunch += pr["dist_launches"]
                launches += plan.last_launches()
        torch.cuda.synchronize()
        barrier()
        clocks = cs.summary(busy_floor_mhz=600.0)
        if clocks_all is None:
            clocks_all = clocks
        ms = max_over_ranks(sum(step_ms) / len(step_ms))
        # end to end: pinned host series -> H2D -> search -> result D2H (synchronous API)
        e2e_ms = []
        for _ in range(max(3, args.steps // 2)):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.find_discord_host(Th)
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e = max_over_ranks(statistics.mean(e2e_ms))
        # roofline of the distance-tile kernel
        if prec == "fp32":
            work = 2.0 * n * pairs  # one FP32 subtract + one FFMA per element of each pair
            achieved = work / (dist_ms * 1e-3) / 1e12 if dist_ms > 0 else 0.0
            peak = _alu_peak(sms, peaks)
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinstr/s",
                    "frac": achieved / peak if peak else None, "traffic": _kernel_traffic(prec),
                    "kernel": "k_scan_fp32",
                    "peak_source": f"derived: {sms} SMs (device query) x 128 FP32 lanes x max SM clock",
                    "launches_per_step": dlaunch / args.steps}
        else:
            work = 2.0 * plan_nkpad(n) * pairs
            achieved = work / (dist_ms * 1e-3) / 1e12 if dist_ms > 0 else 0.0
            peak = float(peaks.get("bf16_tflops", 1900.0))
            roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak if peak else None, "traffic": _kernel_traffic(prec),
                    "kernel": "k_scan_tc", "peak_source": f"{peak_src} bf16 dense burst (fp16 rate equal)",
                    "launches_per_step": dlaunch / args.steps}
        results[prec] = {"time_to_discord_ms": ms, "value": P_u / (ms * 1e-3) * world,
                         "e2e_ms": e2e, "e2e_value": P_u / (e2e * 1e-3) * world, "index": res.index,
                         "nn_distance": res.nn_distance, "computed_pairs_per_step": pairs // args.steps,
                         "kernel_launches_per_step": launches / args.steps, "roofline": roof,
                         "dist_kernel_ms_per_step": dist_ms / args.steps}
        plan.close()

    exact = [f for f in forms if f != "fp32"]
    head_form = min(exact or forms, key=lambda f: results[f]["time_to_discord_ms"])
    head = results[head_form]
    # Batches and serving run the FP16 Gram form when it is measured: its error bound is 8x tighter
    # than BF16's, and with the BF16 bound noisy periodic requests with long subsequences cannot
    # abandon rows and fall back to near-exhaustive scans (the serving trace then backs up).
    side_form = "tc_fp16" if "tc_fp16" in results else head_form
    batch = serve = None
    if not args.no_batch:
        batch = _batch(dd, side_form, reps=max(1, args.batch_reps))
    if not args.no_serve:
        serve = _serve(dd, side_form)
    exh = None
    if not args.no_exhaustive:
        exh = _exhaustive(dd, Td, m, n, [f for f in ("tc_fp16", "tc_bf16", "fp32") if f in supported], peaks, sms)
    win = None
    if not args.no_window:
        try:
            win = _window(dd, Td, m, n, peaks, sms)
        except Exception as e:  # an optional object: report it, keep the headline line
            win = {"error": f"{type(e).__name__}: {e}"}
        if exh and "fp32" in exh and "global_diag_profile" in win:
            win["global_diag_profile"]["vs_direct_fp32_exhaustive"] = \
                win["global_diag_profile"]["pairs_per_s"] / exh["fp32"]["pairs_per_s"]
    probed = None
    if not args.no_probe:
        try:
            probed = _probe_peaks(dd, dev)
            probed["alu_peak_derived_tinstr"] = _alu_peak(sms, peaks)
            probed["sms"] = sms
        except Exception as e:
            probed = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        cpu = None if args.no_cpu_baseline else _cpu_baseline()
        line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["time_to_discord_ms"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "tc_fp16": "f16xf16->f32+f64", "tc_bf16": "bf16xbf16->f32+f64"}[head_form],
                "data": "synthetic",
                "config": {"workload": f"{spec.kind} m={m} n={n}, {len(spec.anomalies)} anomalies, seed {spec.seed} "
                                       f"(synthetic stand-in for SCD-1M)",
                           "m": m, "n": n, "precision": head_form, "parallelism": f"replicas x{world}",
                           "l2": "flushed between steps (256 MiB write)"},
                "time_to_discord_ms": head["time_to_discord_ms"],
                "roofline": head["roofline"], "cpu_baseline": cpu,
                "e2e": {"value": head["e2e_value"], "unit": UNIT, "h2d_bytes_per_step": 4 * m,
                        "d2h_bytes_per_step": 40, "ms_per_step": head["e2e_ms"]},
                "clocks": clocks_all, "gpu_launches": int(round(head["kernel_launches_per_step"] * args.steps)),
                "forms": {k: {kk: vv for kk, vv in v.items() if kk != "roofline"} | {"roofline_frac": v["roofline"]["frac"]}
                          for k, v in results.items()},
                "discord": {"index": head["index"], "nn_distance": head["nn_distance"]},
                "tc_vs_fp32_time_to_discord": (results["fp32"]["time_to_discord_ms"] / head["time_to_discord_ms"]
                                               if "fp32" in results and head_form != "fp32" else None),
                "exhaustive": exh, "window": win, "batch": batch, "serve": serve, "peaks_probed": probed}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def plan_nkpad(n: int) -> int:
    return ((n + 63) // 64) * 64


if __name__ == "__main__":
    main()
