#!/usr/bin/env python
"""Benchmark of the exact NN-DTW search with LB_Enhanced^V pruning.

One step = one full pass of the hot path over one batch: envelopes of the
training set, LB_Enhanced^V of every query x train pair, compaction, DTW with
early abandoning, FP64 recheck of near ties, argmin and labels (a single
``nn_dtw_search`` call).  Default workload: train 500 x test 500 series,
L=256, W=26 (0.1 L), V=5, seeded synthetic random-walk-plus-class-shape data.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
(the paper's search protocol: Euclidean ordering, LB_Enhanced^V, early-
abandoning DTW) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact NN-DTW queries/s + DTW GCUPS on 1 GB300: batched FP32 vs plain FP64 form"
UNIT = "queries/s"
L2_FLUSH_BYTES = 256 << 20
KERNELS_PER_STEP = 10   # envelopes, lb, dtw(seed), compact, dtw, filter, collect, dtw64, ties, final
INSTR_PER_CELL = 3      # FADD + 3-input FMNMX + FFMA
INSTR_PER_LB_ELEM = 4   # FMNMX + FMNMX + FADD + FFMA (Keogh bridge term)
FP32_LANES_PER_SM = 128
FALLBACK_HBM_GBS = 6800.0


def workload(name: str):
    from paper_1808_09617_gb300 import synth
    if name == "pairs":
        ds = synth.make_pairs(5)
        desc = "pairs: train 500 x test 500, L=256, W=26 (0.1 L), V=5, float32"
    elif name == "tiny":
        ds = synth.make_tiny()
        ds.train = ds.train.astype(np.float32)
        ds.test = ds.test.astype(np.float32)
        desc = "tiny: train 64 x test 32, L=128, W=13, V=5"
    elif name.startswith("precision-"):
        r = float(name.split("-")[1])
        ds = synth.make_precision(r)
        desc = f"precision: train 10000 x test 2000, L=1024, W={ds.W}, V=5, float32"
    else:
        raise SystemExit(f"unknown workload {name}")
    return ds, desc


def band_cells(L, W):
    w = min(W, L - 1)
    return L * (2 * w + 1) - w * (w + 1)


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_sel: str):
        self.sel = device_sel
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.sel, f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def source_sha(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


STAGE_SOURCES = {
    "dtw": ["paper_1808_09617_gb300/csrc/dtw32.cuh", "paper_1808_09617_gb300/csrc/dtw32_launch.cu"],
    "seed": ["paper_1808_09617_gb300/csrc/dtw32.cuh", "paper_1808_09617_gb300/csrc/dtw32_launch.cu"],
    "lb": ["paper_1808_09617_gb300/csrc/lb.cu"],
    "envelopes": ["paper_1808_09617_gb300/csrc/envelope.cu"],
}


def traffic_for(stage, workload_name):
    """DRAM bytes per launch from a committed ncu summary, if taken on the
    current source of that kernel; otherwise None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
    except Exception:
        return None
    e = t.get(f"{workload_name}:{stage}")
    if not e or e.get("source_sha") != source_sha(STAGE_SOURCES[stage]):
        return None
    return e.get("dram_bytes_per_launch")


def cpu_baseline(ds, budget_s=10.0):
    import oracle
    orc = oracle.get()
    threads = oracle.default_threads()
    n = min(ds.Q, max(8, threads))
    env = orc.envelopes(ds.train, ds.W)
    t0 = time.perf_counter()
    orc.nn_pruned(ds.train, ds.train_labels, ds.test[:n], ds.W, ds.V, env=env, threads=threads)
    dt = time.perf_counter() - t0
    n2 = min(ds.Q, max(n, int(n * budget_s / max(dt, 1e-3))))
    if n2 > n:
        t0 = time.perf_counter()
        orc.nn_pruned(ds.train, ds.train_labels, ds.test[:n2], ds.W, ds.V, env=env,
                      threads=threads)
        dt = time.perf_counter() - t0
        n = n2
    return {"value": n / dt, "unit": UNIT, "cores": min(threads, n), "kind": "oracle",
            "sample": f"first {n} of {ds.Q} queries against all {ds.N} training series "
                      f"(paper's search protocol, FP64, envelopes precomputed), {dt:.1f} s"}


# ------------------------------------------------------------------ reference arm

def run_reference(args, ds, desc):
    import oracle
    orc = oracle.get()
    threads = oracle.default_threads()
    env = orc.envelopes(ds.train, ds.W)
    n = min(ds.Q, max(threads, 16))
    t0 = time.perf_counter()
    orc.nn_pruned(ds.train, ds.train_labels, ds.test[:n], ds.W, ds.V, env=env, threads=threads)
    probe = time.perf_counter() - t0
    # size each step so the whole run stays within a few minutes
    per_q = probe / n
    total_steps = args.steps + args.warmup
    n = int(min(ds.Q, max(threads, (150.0 / total_steps) / max(per_q, 1e-6))))
    times = []
    for k in range(total_steps):
        lo = (k * n) % ds.Q
        idx = np.arange(lo, lo + n) % ds.Q
        t0 = time.perf_counter()
        orc.nn_pruned(ds.train, ds.train_labels, ds.test[idx], ds.W, ds.V, env=env,
                      threads=threads)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1000.0 * sum(times) / len(times)
    value = n / (ms / 1000.0)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": desc, "sample_queries_per_step": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": min(threads, n),
                             "kind": "oracle",
                             "sample": f"{n} queries per step against all {ds.N} training "
                                       f"series, paper's search protocol in FP64"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving

def run_serving(args):
    """Serving form: 16 resident training sets, Poisson query streams at
    several rates, continuous batching across sets; p50/p99 latency and
    sustained queries/s per rate.  Queries cycle through a pool of 1,024
    pre-drawn series per set (drawing them at 50k/s would dominate)."""
    import threading
    import torch
    from paper_1808_09617_gb300 import serving, synth
    specs = synth.serving_specs(16)
    sets = {}
    for d, sp in enumerate(specs):
        ds = synth.make_serving_set(d, sp)
        sets[d] = (ds.train, ds.train_labels, sp["W"], sp["V"])
    pools = {d: synth.serving_queries(d, specs[d], 1024)[0] for d in sets}
    srv = serving.Server(sets, n_slots=args.serve_slots, max_batch=args.serve_batch)
    rng = np.random.default_rng(7)
    results = []
    try:
        # warm-up: one batch per set
        fs = [srv.submit(pools[d][0], d) for d in sets]
        [f.result() for f in fs]
        for rate in args.serve_rates:
            srv.latencies.clear()
            srv.completed = 0
            srv.t_first = srv.t_last = None
            srv.batches = 0
            times = synth.arrival_times(rate, args.serve_seconds, seed_index=int(rate))
            which = rng.integers(0, len(sets), size=times.size)
            t0 = time.perf_counter() + 0.05
            futs = []
            for k, (t, d) in enumerate(zip(times, which)):
                target = t0 + t
                while True:
                    now = time.perf_counter()
                    if now >= target:
                        break
                    if target - now > 2e-4:
                        time.sleep(target - now - 1e-4)
                futs.append(srv.submit(pools[int(d)][k % 1024], int(d), t_arrival=target))
            for f in futs:
                f.result()
            st = srv.latency_stats()
            st.update({"offered_qps": rate, "queries": int(times.size)})
            results.append(st)
    finally:
        srv.close()
    line = {"metric": "serving: p50/p99 latency and sustained queries/s, continuous batching",
            "unit": "queries/s", "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "impl": "ours",
            "config": {"workload": "16 resident sets, L in {128, 512, 1500}, N log-uniform "
                                   "[1000, 20000], W=0.1 L, V=5; Poisson arrivals, set "
                                   "uniform per query", "slots": args.serve_slots,
                       "max_batch": args.serve_batch, "seconds_per_rate": args.serve_seconds},
            "rates": results}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batched

def run_batched(args):
    """Batching form: the 64 heterogeneous datasets searched by one CUDA-graph
    launch (FP32 with FP64 recheck), against the plain FP64 form run one
    dataset per call."""
    import torch
    from paper_1808_09617_gb300 import nndtw, synth
    nndtw.load()
    dsets = synth.make_batched(64)
    dev = torch.device("cuda")
    sets = [dict(train=torch.from_numpy(d.train).to(dev), labels=torch.from_numpy(d.train_labels).to(dev),
                 test=torch.from_numpy(d.test).to(dev), W=d.W, V=d.V) for d in dsets]
    Qtot = sum(d.Q for d in dsets)
    cells = sum(d.Q * d.N * band_cells(d.L, d.W) for d in dsets)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    bs = nndtw.BatchedSearch(sets, graph=True)
    for _ in range(args.warmup):
        flush.zero_()
        bs.run()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for a, b in evs:
        flush.zero_()
        a.record()
        bs.run()
        b.record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
    # plain FP64 form, one dataset per call, same data promoted
    t64 = [(s["train"].double(), s["test"].double()) for s in sets]
    torch.cuda.synchronize()
    e1, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    e1.record()
    for (tr, te), s in zip(t64, sets):
        nndtw.nn_dtw_search(tr, s["labels"], te, s["W"], s["V"])
    e2.record()
    torch.cuda.synchronize()
    ms64 = e1.elapsed_time(e2)
    line = {"metric": "batched: exact NN-DTW queries/s, 64 heterogeneous datasets, one CUDA-graph "
                      "launch (FP32 + FP64 recheck) vs plain FP64 form one dataset per call",
            "value": Qtot / (ms / 1e3), "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "impl": "ours",
            "config": {"workload": "64 datasets: L log-uniform [24, 2048], N log-uniform "
                                   "[16, 8000], Q = N/2, W in {0,.05,.1,.2,.5,1} L, V in 1..8",
                       "queries": Qtot, "l2": "flushed before every step"},
            "gcups_effective": cells / (ms * 1e-3) / 1e9,
            "fp64_plain": {"ms_per_batch": ms64, "value": Qtot / (ms64 / 1e3),
                           "fp32_batched_over_fp64_plain": ms64 / ms}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pairs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--serve-rates", type=float, nargs="*",
                    default=[1000, 5000, 10000, 20000, 50000])
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-batch", type=int, default=512)
    ap.add_argument("--dtw-group", type=int, default=-1,
                    help="lanes per pair in the FP32 DTW kernel (-1: autotune, 0: library "
                         "default, else G)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be at least 3")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.workload == "serving":
        if rank == 0:
            run_serving(args)
        return
    if args.workload == "batched":
        if rank == 0:
            run_batched(args)
        return
    ds, desc = workload(args.workload)
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, ds, desc)
        return

    import torch
    from paper_1808_09617_gb300 import nndtw

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    nndtw.load()

    stream = torch.cuda.current_stream()
    train = torch.from_numpy(ds.train).to(dev)
    test = torch.from_numpy(ds.test).to(dev)
    labels = torch.from_numpy(ds.train_labels).to(dev)
    N, L = ds.train.shape
    Q = ds.Q
    W, V = ds.W, ds.V
    ws = torch.empty(nndtw.nn_dtw_workspace_size(N, Q, L, W, V), dtype=torch.uint8, device=dev)
    out = (torch.empty(Q, dtype=torch.int32, device=dev), torch.empty(Q, dtype=torch.int32, device=dev),
           torch.empty(Q, dtype=torch.float64, device=dev))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    group = args.dtw_group
    if group < 0:
        from paper_1808_09617_gb300 import autotune
        group = autotune.tune_search(train, labels, test, W, V, workspace=ws, out=out)
    gflag = nndtw.DTW_GROUP(group) if group else 0

    def step(flags=0):
        return nndtw.nn_dtw_search(train, labels, test, W, V, flags=flags | gflag, workspace=ws,
                                   out=out)

    # counting pass (untimed): pruning and cells
    counts = nndtw.nn_dtw_search(train, labels, test, W, V, flags=gflag, workspace=ws, out=out,
                                 stats=True).stats
    for _ in range(args.warmup):
        flush.zero_()
        step(nndtw.TIME_STAGES)
        nndtw.nn_dtw_stage_times()
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(dev)
    try:
        sel = f"GPU-{props.uuid}" if not str(props.uuid).startswith("GPU-") else str(props.uuid)
    except Exception:
        sel = str(local)
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stages = []
    with ClockSampler(sel) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()                      # L2 flush, outside the step's events
            ev_s[k].record(stream)
            step(nndtw.TIME_STAGES)
            ev_e[k].record(stream)
            stages.append(nndtw.nn_dtw_stage_times())
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    step_ms = [ev_s[k].elapsed_time(ev_e[k]) for k in range(args.steps)]
    ms = sum(step_ms) / len(step_ms)
    if dist:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * Q / (ms / 1000.0)
    clocks = clk.summary()

    # per-stage means and the dominant kernel
    names = [s for s in nndtw.STAGES if s != "total"]
    stage_ms = {s: sum(d[s] for d in stages) / len(stages) for s in nndtw.STAGES}
    dominant = max(names, key=lambda s: stage_ms[s])
    peaks, peak_src = read_peaks()
    n_sm = props.multi_processor_count
    sm_max = float(clocks["sm_max_mhz"] or peaks.get("sm_max_mhz", 2070.0))
    cells_main = counts["dtw_cells"] - counts["seed_cells"]
    dtw_cells_total = counts["dtw_cells"]
    probe = nndtw.nn_dtw_probe_cell_rate(20000)
    if dominant in ("dtw", "seed"):
        units = cells_main if dominant == "dtw" else counts["seed_cells"]
        achieved = units / (stage_ms[dominant] * 1e-3) / 1e9
        peak = n_sm * FP32_LANES_PER_SM * sm_max * 1e6 / INSTR_PER_CELL / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gcell/s",
                "frac": achieved / peak,
                "peak_basis": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_max:.0f} MHz / "
                              f"{INSTR_PER_CELL} instructions per cell (derived)",
                "probe_measured": probe / 1e9, "frac_of_probe": achieved / (probe / 1e9)}
    elif dominant == "lb":
        units = N * Q * L
        achieved = units / (stage_ms["lb"] * 1e-3) / 1e9
        peak = n_sm * FP32_LANES_PER_SM * sm_max * 1e6 / INSTR_PER_LB_ELEM / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair-element/s",
                "frac": achieved / peak,
                "peak_basis": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_max:.0f} MHz / "
                              f"{INSTR_PER_LB_ELEM} instructions per pair-element (derived)"}
    else:
        byts = 12 * N * L if dominant == "envelopes" else 0
        achieved = byts / (stage_ms[dominant] * 1e-3) / 1e9
        peak = float(peaks["hbm_gbs"])
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if peak else None}
    roof["kernel"] = dominant
    roof["share_of_step"] = stage_ms[dominant] / stage_ms["total"] if stage_ms["total"] else None
    roof["traffic"] = traffic_for(dominant, args.workload) if dominant in STAGE_SOURCES else None
    if roof["bound"] == "hbm":
        roof["peak_source"] = f"{peak_src} copy bandwidth"

    # plain FP64 form on the same data
    fp64_ms = None
    if args.fp64_steps > 0:
        train64, test64 = train.double(), test.double()
        ws64 = torch.empty(nndtw.nn_dtw_workspace_size(N, Q, L, W, V, fp64=True),
                           dtype=torch.uint8, device=dev)
        nndtw.nn_dtw_search(train64, labels, test64, W, V, workspace=ws64, out=out)
        e1, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(args.fp64_steps):
            flush.zero_()
            e1.record(stream)
            nndtw.nn_dtw_search(train64, labels, test64, W, V, workspace=ws64, out=out)
            e2.record(stream)
            torch.cuda.synchronize()
            tot += e1.elapsed_time(e2)
        fp64_ms = tot / args.fp64_steps
        del ws64

    # end to end through the host-buffer C call, pinned host memory
    h_train = torch.from_numpy(ds.train).pin_memory().numpy()
    h_test = torch.from_numpy(ds.test).pin_memory().numpy()
    h_lab = torch.from_numpy(ds.train_labels).pin_memory().numpy()
    h_out = (torch.empty(Q, dtype=torch.int32).pin_memory().numpy(),
             torch.empty(Q, dtype=torch.int32).pin_memory().numpy(),
             torch.empty(Q, dtype=torch.float64).pin_memory().numpy())
    hbuf = torch.empty(nndtw.nn_dtw_host_buffer_size(N, Q, L, W, V), dtype=torch.uint8, device=dev)
    for _ in range(2):
        nndtw.nn_dtw_search_host(h_train, h_lab, h_test, W, V, buffer=hbuf, out=h_out)
    e2e_t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        nndtw.nn_dtw_search_host(h_train, h_lab, h_test, W, V, buffer=hbuf, out=h_out)
        e2e_t.append(time.perf_counter() - t0)
    e2e_ms = 1000.0 * sum(e2e_t) / len(e2e_t)
    if dist:
        t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(ds)

    if rank == 0:
        eff_cells = Q * N * band_cells(L, W)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": desc, "l2": "flushed before every step (256 MiB write, "
                                               "outside the step's events)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "dtw_group": group or "library default",
                       "dtw_group_source": "autotune" if args.dtw_group < 0 else "fixed",
                       "step": "one nn_dtw_search call: envelopes, LB, seed DTW, compaction, "
                               "DTW, FP64 recheck, argmin"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": world * Q / (e2e_ms / 1000.0), "unit": UNIT,
                    "h2d_bytes_per_step": int(ds.train.nbytes + ds.test.nbytes +
                                              ds.train_labels.nbytes),
                    "d2h_bytes_per_step": int(Q * (4 + 4 + 8)),
                    "ms_per_step": e2e_ms},
            "gpu_launches": KERNELS_PER_STEP * args.steps,
            "clocks": clocks,
            "gcups_effective": eff_cells / (ms * 1e-3) / 1e9,
            "gcups_dtw_kernel": (cells_main / (stage_ms["dtw"] * 1e-3) / 1e9
                                 if stage_ms["dtw"] > 0 else None),
            "stage_ms": stage_ms,
            "pruning": {"pairs": counts["pairs"], "lb_pruned": counts["lb_pruned"],
                        "lb_pruned_frac": counts["lb_pruned"] / counts["pairs"],
                        "dtw_started": counts["dtw_started"],
                        "dtw_abandoned": counts["dtw_abandoned"],
                        "dtw_cells": dtw_cells_total,
                        "rechecked": counts["rechecked"],
                        "recheck_queries": counts["recheck_queries"]},
            "fp64_plain": ({"ms_per_step": fp64_ms, "value": world * Q / (fp64_ms / 1000.0),
                            "unit": UNIT, "fp32_over_fp64": fp64_ms / ms}
                           if fp64_ms else None),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
