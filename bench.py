#!/usr/bin/env python
"""Benchmark of the exact NN-DTW search with LB_Enhanced^V pruning.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload batched|pairs|tiny|precision-R|serving|window|vsweep|varlen]

Default workload ("batched"): 64 seeded synthetic datasets of uneven shape
(L log-uniform in [24, 2048], train size log-uniform in [16, 8000], test size
half of it, W in {0, .05, .1, .2, .5, 1} L, V in 1..8), searched by ONE CUDA
graph launch of ``nn_dtw_search_batched`` (FP32 bulk with FP64 recheck).  One
step = one such launch over all 64 datasets (envelopes, bounds, compaction,
DTW, recheck, argmin for every query).  It is compared with the plain FP64
form run one dataset per call.  ``--workload pairs`` is the single-dataset
bound-comparison workload (500 x 500, L=256, W=26, V=5), one
``nn_dtw_search`` per step.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
(the paper's search protocol) on a bounded sample of the same workload on the
host cores.  ``--workload serving`` prints the serving (continuous batching)
line instead.
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
def stage_bytes(shapes, flags_of, nndtw) -> dict:
    """Algorithmic DRAM bytes per step of the two HBM-facing stages, from the
    datasets' shapes (dicts with N, Q, L) and search flags.  Envelopes: each
    training series read once (4 B/element) and its envelope pair written
    (8 B); with the cascade's second stage the queries' envelopes too; with
    the LB_Improved bridge the second envelopes (read 8, write 8) and their
    packing (read 4 + 8, write 8).  Bounds: the squared norms read every
    series once, the bound pass reads the queries, the training series and
    their envelopes once (the compulsory traffic of a tiled pass) and writes
    one FP32 bound per pair (and, with the reverse bound, one FP32 ends-and-
    bands sum)."""
    env = lb = 0
    for d, f in zip(shapes, flags_of):
        N, Q, L = d["N"], d["Q"], d["L"]
        rev = bool(f & nndtw.REVERSE) and not f & (nndtw.NO_PRUNE | nndtw.NO_REVERSE |
                                                     nndtw.KEOGH_BOUND)
        imp = bool(f & nndtw.IMPROVED) and not f & (nndtw.NO_PRUNE | nndtw.KEOGH_BOUND)
        env += 12 * N * L
        if rev or imp:
            env += 12 * Q * L
        if imp:
            env += (16 + 20) * N * L
        lb += 4 * (Q + N) * L + 4 * (Q * L + 3 * N * L) + 4 * Q * N * (2 if rev else 1)
    return {"envelopes": env, "lb": lb}


INSTR_PER_CELL = 3       # FADD + 3-input FMNMX + FFMA
INSTR_PER_LB_ELEM = 5    # bridge: FMNMX + FMNMX + FADD + FFMA; fused ED: FFMA (dot product)
FP32_LANES_PER_SM = 128
FALLBACK_HBM_GBS = 6800.0
STAGES = ("envelopes", "lb", "seed", "compact", "dtw", "recheck", "final", "total")


# ------------------------------------------------------------------ ranks

def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time (every rank gets it); ``dist`` is
    torch.distributed or None for a single process."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: int, ms: float) -> float:
    """Units per second of the whole job: every rank (an independent replica)
    processes units_per_rank units in the slowest rank's ms."""
    return world * units_per_rank / (ms / 1000.0)


# ------------------------------------------------------------------ workloads

def single_workload(name: str):
    from paper_1808_09617_gb300 import synth
    if name == "pairs":
        ds = synth.make_pairs(5)
        desc = "pairs: train 500 x test 500, L=256, W=26 (0.1 L), V=5, float32"
    elif name == "tiny":
        ds = synth.make_tiny()
        ds.train = ds.train.astype(np.float32)
        ds.test = ds.test.astype(np.float32)
        desc = "tiny: train 64 x test 32, L=128, W=13, V=5"
    elif name.startswith("batched-"):
        i = int(name.split("-")[1])
        spec = synth.batched_specs(64)[i]
        ds = synth.make_batched_dataset(i, spec)
        desc = (f"batched dataset {i} alone: train {ds.N} x test {ds.Q}, L={ds.L}, W={ds.W}, "
                f"V={ds.V}, float32")
    elif name.startswith("precision-"):
        r = float(name.split("-")[1])
        ds = synth.make_precision(r)
        desc = f"precision: train 10000 x test 2000, L=1024, W={ds.W}, V=5, float32"
    else:
        raise SystemExit(f"unknown workload {name}")
    return [ds], desc


def batched_workload():
    from paper_1808_09617_gb300 import synth
    dsets = synth.make_batched(64)
    desc = ("batched: 64 datasets in one CUDA-graph launch; L log-uniform [24, 2048], train "
            "log-uniform [16, 8000], test = train/2, W in {0,.05,.1,.2,.5,1} L, V in 1..8; "
            f"{sum(d.Q for d in dsets)} queries, float32")
    return dsets, desc


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
        self.lines = []

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


def device_selector(torch, dev, local):
    props = torch.cuda.get_device_properties(dev)
    try:
        u = str(props.uuid)
        return u if u.startswith("GPU-") else f"GPU-{u}"
    except Exception:
        return str(local)


# ------------------------------------------------------------------ roofline

def source_sha(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


_DTW_SOURCES = ["paper_1808_09617_gb300/csrc/dtw32.cuh", "paper_1808_09617_gb300/csrc/dtw32_launch.cu",
                "paper_1808_09617_gb300/csrc/dtw32_rows.cu", "paper_1808_09617_gb300/csrc/dtw32_rowsg.cu",
                "paper_1808_09617_gb300/csrc/dtw32_wide.cu"]
STAGE_SOURCES = {
    "dtw": _DTW_SOURCES,
    "seed": _DTW_SOURCES,
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
    if not e or stage not in STAGE_SOURCES or e.get("source_sha") != source_sha(STAGE_SOURCES[stage]):
        return None
    return e.get("dram_bytes_per_launch")


def roofline(stage_ms, launches, work, n_sm, sm_max, peaks, peak_src, probe, workload_name):
    """Roofline of the stage with the largest time.  ``work`` maps stage ->
    algorithmic units per step; ``launches`` maps stage -> launches per step."""
    names = [s for s in STAGES if s != "total"]
    dom = max(names, key=lambda s: stage_ms[s])
    per_launch_ms = stage_ms[dom] / max(1, launches.get(dom, 1))
    units = work.get(dom, 0) / max(1, launches.get(dom, 1))
    if dom in ("dtw", "seed"):
        achieved = units / (per_launch_ms * 1e-3) / 1e9
        peak = n_sm * FP32_LANES_PER_SM * sm_max * 1e6 / INSTR_PER_CELL / 1e9
        r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gcell/s",
             "frac": achieved / peak,
             "peak_basis": f"derived: {n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                           f"{sm_max:.0f} MHz / {INSTR_PER_CELL} instructions per cell",
             "probe_measured": probe / 1e9, "frac_of_probe": achieved / (probe / 1e9)}
    elif dom == "lb":
        achieved = units / (per_launch_ms * 1e-3) / 1e9
        peak = n_sm * FP32_LANES_PER_SM * sm_max * 1e6 / INSTR_PER_LB_ELEM / 1e9
        r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair-element/s",
             "frac": achieved / peak,
             "peak_basis": f"derived: {n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                           f"{sm_max:.0f} MHz / {INSTR_PER_LB_ELEM} instructions per element"}
    else:
        achieved = units / (per_launch_ms * 1e-3) / 1e9
        peak = float(peaks["hbm_gbs"])
        r = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
             "frac": achieved / peak, "peak_source": f"{peak_src} copy bandwidth"}
    r["kernel"] = dom
    r["launches_per_step"] = launches.get(dom, 1)
    r["mean_launch_ms"] = per_launch_ms
    r["share_of_step"] = stage_ms[dom] / stage_ms["total"] if stage_ms["total"] else None
    r["traffic"] = traffic_for(dom, workload_name)
    return r


# ------------------------------------------------------------------ tightness

def tightness_pairs(dev):
    """Mean tightness LB/DTW over all 250,000 pairs of the 500 x 500 pairs
    workload (L=256, W=26) for LB_Enhanced^V, V in {1, 2, 5}, with and
    without the LB_Improved bridge, and for the comparison bounds LB_Keogh,
    LB_Improved and LB_New (pairs with DTW = 0 excluded), with the search's
    pruning per V."""
    import torch
    from paper_1808_09617_gb300 import nndtw, synth
    ds = synth.make_pairs(5)
    train = torch.from_numpy(ds.train).to(dev)
    test = torch.from_numpy(ds.test).to(dev)
    labels = torch.from_numpy(ds.train_labels).to(dev)
    Q, N = test.shape[0], train.shape[0]
    q = torch.arange(Q, device=dev, dtype=torch.int32).repeat_interleave(N)
    t = torch.arange(N, device=dev, dtype=torch.int32).repeat(Q)
    pairs = torch.stack([q, t], 1).contiguous()
    dtw = nndtw.dtw_windowed(test, train, pairs, ds.W).double()
    env = nndtw.nn_dtw_build_envelopes(train, ds.W)
    keep = dtw > 0
    out = {"pairs": Q * N, "pairs_dtw_zero": int((~keep).sum().item()), "W": ds.W, "L": ds.L}
    lbk = nndtw.lb_enhanced(test, train, env, ds.W, 1, keogh=True).double().reshape(-1)
    out["LB_Keogh"] = float((lbk[keep] / dtw[keep]).mean().item())
    tenv = nndtw.nn_dtw_build_envelopes(test, ds.W)
    env2 = nndtw.nn_dtw_build_second_envelopes(env, ds.W)
    # the paper's comparison bounds (Sec. 2.2.4, 2.2.5)
    lbim = nndtw.lb_improved(test, tenv, train, env, env2, ds.W).double().reshape(-1)
    out["LB_Improved"] = float((lbim[keep] / dtw[keep]).mean().item())
    lbn = nndtw.lb_new(test, train, ds.W).double().reshape(-1)
    out["LB_New"] = float((lbn[keep] / dtw[keep]).mean().item())
    for V in (1, 2, 5):
        lb = nndtw.lb_enhanced(test, train, env, ds.W, V).double().reshape(-1)
        st = nndtw.nn_dtw_search(train, labels, test, ds.W, V, stats=True).stats
        lbi = nndtw.lb_enhanced_improved(test, tenv, train, env, env2, ds.W, V).double().reshape(-1)
        sti = nndtw.nn_dtw_search(train, labels, test, ds.W, V, flags=nndtw.IMPROVED,
                                  stats=True).stats
        out[f"LB_Enhanced^{V}"] = {
            "tightness": float((lb[keep] / dtw[keep]).mean().item()),
            "lb_pruned_frac": st["lb_pruned"] / st["pairs"],
            "dtw_abandoned_frac_of_started": st["dtw_abandoned"] / max(1, st["dtw_started"]),
            # the same bound with the LB_Improved bridge (Sec. 5), and the
            # search with it as the cascade's second stage
            "with_improved_bridge": {
                "tightness": float((lbi[keep] / dtw[keep]).mean().item()),
                "pruned_frac": (sti["lb_pruned"] + sti["lb_pruned_improved"]) / sti["pairs"],
                "dtw_started": sti["dtw_started"], "dtw_started_without": st["dtw_started"]}}
    return out


# ------------------------------------------------------------------ CPU oracle

def _sample_plan(dsets, per_ds):
    return [(d, np.arange(min(per_ds, d.Q))) for d in dsets]


def oracle_sample(dsets, budget_s):
    """Time the oracle's pruned search on a sample sized to about budget_s."""
    import oracle
    orc = oracle.get()
    threads = oracle.default_threads()
    envs = [orc.envelopes(d.train, d.W) for d in dsets]

    def run(per_ds):
        n = 0
        t0 = time.perf_counter()
        for (d, idx), env in zip(_sample_plan(dsets, per_ds), envs):
            if idx.size:
                orc.nn_pruned(d.train, d.train_labels, d.test[idx], d.W, d.V, env=env,
                              threads=threads)
                n += idx.size
        return n, time.perf_counter() - t0

    per = max(8, threads)   # the oracle threads over the queries of one dataset
    n, dt = run(per)
    maxq = max(d.Q for d in dsets)
    per2 = min(maxq, max(per, int(per * budget_s / max(dt, 1e-3))))
    if per2 > per:
        per = per2
        n, dt = run(per)
    return n, dt, per, threads


def cpu_baseline(dsets, budget_s=10.0):
    n, dt, per, threads = oracle_sample(dsets, budget_s)
    return {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {per} queries of each of {len(dsets)} dataset(s) ({n} queries) "
                      f"against all training series, paper's search protocol in FP64 "
                      f"(envelopes precomputed), {dt:.1f} s"}


def run_reference(args, dsets, desc):
    total_steps = args.steps + args.warmup
    n, dt, per, threads = oracle_sample(dsets, min(8.0, 150.0 / total_steps))
    import oracle
    orc = oracle.get()
    envs = [orc.envelopes(d.train, d.W) for d in dsets]
    times = []
    for k in range(total_steps):
        t0 = time.perf_counter()
        cnt = 0
        for (d, idx), env in zip(_sample_plan(dsets, per), envs):
            if idx.size:
                idx = (idx + k * per) % d.Q
                orc.nn_pruned(d.train, d.train_labels, d.test[idx], d.W, d.V, env=env,
                              threads=threads)
                cnt += idx.size
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1000.0 * sum(times) / len(times)
    value = cnt / (ms / 1000.0)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": desc, "sample_queries_per_step": cnt},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{per} queries per dataset per step ({cnt} queries) "
                                       "against all training series, paper's search protocol "
                                       "in FP64"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ window learning

VSWEEP_V = (1, 2, 3, 4, 5, 6, 8, 10, 12, 15, 20)
VSWEEP_W_ABS = (1, 3, 5, 7, 9)
VSWEEP_W_REL = (0.1, 0.2, 0.3, 0.5, 1.0)


def run_vsweep(args):
    """The paper's study of the tightness parameter V (Sec. 4.1) on synthetic
    data: for each window, the search time with LB_Enhanced^V as the bound,
    V = 1..20, divided by the search time with LB_Keogh as the bound on the
    same dataset, and the geometric mean of that ratio over the datasets.
    Envelopes are built beforehand and passed in, so that, as in the paper,
    their time is not counted; no cascade second stage; each time is the
    median of `--steps` searches timed by the library's stage events."""
    import torch
    from paper_1808_09617_gb300 import nndtw, synth
    dev = torch.device("cuda", 0)
    nndtw.load()
    # twelve mid-sized datasets of the batched generator (its W and V ignored)
    specs = [sp for sp in synth.batched_specs(64)]
    picked = [i for i, sp in enumerate(specs)
              if 20_000 <= sp["N"] * sp["Q"] <= 3_000_000 and sp["L"] <= 1024][:12]
    dsets = [synth.make_batched_dataset(i, specs[i]) for i in picked]
    reps = max(3, args.steps)

    def timed(tr, lb, te, env, W, V, flags):
        for _ in range(2):
            nndtw.nn_dtw_search(tr, lb, te, W, V, env=env, flags=flags)
        ts = []
        for _ in range(reps):
            nndtw.nn_dtw_search(tr, lb, te, W, V, env=env, flags=flags | nndtw.TIME_STAGES)
            ts.append(nndtw.nn_dtw_stage_times()["total"])
        return statistics.median(ts)

    windows = [("W=%d" % w, lambda L, w=w: w) for w in VSWEEP_W_ABS] + \
              [("W=%gL" % r, lambda L, r=r: int(np.floor(r * L + 0.5))) for r in VSWEEP_W_REL]
    logs = {name: {V: [] for V in VSWEEP_V} for name, _ in windows}
    base_flags = nndtw.NO_REVERSE
    t0 = time.perf_counter()
    for d in dsets:
        tr = torch.from_numpy(d.train).to(dev)
        te = torch.from_numpy(d.test).to(dev)
        lb = torch.from_numpy(d.train_labels).to(dev)
        for name, wf in windows:
            W = min(wf(d.L), d.L - 1)
            env = nndtw.nn_dtw_build_envelopes(tr, W)
            tk = timed(tr, lb, te, env, W, 1, base_flags | nndtw.KEOGH_BOUND)
            for V in VSWEEP_V:
                logs[name][V].append(np.log(timed(tr, lb, te, env, W, V, base_flags) / tk))
    wall = time.perf_counter() - t0
    table = {name: {str(V): float(np.exp(np.mean(v))) for V, v in row.items()}
             for name, row in logs.items()}
    best = {name: int(min(row, key=lambda V: row[V])) for name, row in
            ((n, {int(k): x for k, x in r.items()}) for n, r in table.items())}
    line = {"metric": "search time with LB_Enhanced^V / with LB_Keogh (geometric mean over datasets)",
            "value": table["W=0.1L"]["5"], "unit": "ratio at W=0.1L, V=5", "n_gpus": 1,
            "steps": reps, "warmup": 2, "higher_is_better": False, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"V sweep: {len(dsets)} datasets of the batched generator "
                                   f"(L {min(d.L for d in dsets)}..{max(d.L for d in dsets)}, "
                                   f"train {min(d.N for d in dsets)}..{max(d.N for d in dsets)}), "
                                   f"W in {[n for n, _ in windows]}, V in {list(VSWEEP_V)}",
                       "timing": "median of the searches' stage events (envelopes supplied, "
                                 "not counted), no cascade second stage"},
            "ratio": table, "best_V": best, "wall_s": wall}
    print(json.dumps(line), flush=True)


def run_window(args):
    """Window learning on the 500-series training set of the pairs workload
    (L=256): leave-one-out 1-NN accuracy for W = 0, 1 %, ..., 100 % of L (the
    paper's protocol), all windows in one batched call per step."""
    import torch
    from paper_1808_09617_gb300 import nndtw, synth
    ds = synth.make_pairs(5)
    L, N, V = ds.L, ds.N, ds.V
    windows = sorted({int(np.floor(r / 100.0 * L + 0.5)) for r in range(101)})
    windows = [min(w, L - 1) for w in windows]
    windows = sorted(set(windows))
    dev = torch.device("cuda", 0)
    nndtw.load()
    train = torch.from_numpy(ds.train).to(dev)
    labels = torch.from_numpy(ds.train_labels).to(dev)
    ws = torch.empty(nndtw.nn_dtw_learn_window_workspace_size(N, L, windows, V),
                     dtype=torch.uint8, device=dev)
    correct = torch.empty(len(windows), dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    run = lambda: nndtw.nn_dtw_learn_window(train, labels, windows, V, workspace=ws,
                                            correct=correct)
    for _ in range(args.warmup):
        flush.zero_()
        run()
    torch.cuda.synchronize()
    launches = nndtw.nn_dtw_last_call_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sel = device_selector(torch, dev, 0)
    with ClockSampler(sel) as clk:
        for a, b in ev:
            flush.zero_()
            a.record()
            run()
            b.record()
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
    acc = correct.cpu().numpy() / float(N)
    best = max(range(len(windows)), key=lambda k: (acc[k], -windows[k]))
    # the oracle on the host cores, a bounded sample: three of the windows
    from oracle import get as oracle_get, default_threads
    orc = oracle_get()
    sample_w = [windows[0], windows[len(windows) // 10], windows[len(windows) // 5]]
    t0 = time.perf_counter()
    ref = orc.loo_correct(ds.train, ds.train_labels, sample_w)
    cpu_s = time.perf_counter() - t0
    got = {w: int(correct[windows.index(w)].item()) for w in sample_w}
    queries = N * len(windows)
    line = {"metric": "window learning: leave-one-out 1-NN queries/s over candidate windows",
            "value": queries / (ms / 1e3), "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"window learning: train {N}, L={L}, V={V}, "
                                   f"{len(windows)} windows (0..100 % of L in 1 % steps)",
                       "l2": "flushed before every step (256 MiB write, outside the events)"},
            "learned_window": windows[best], "learned_accuracy": float(acc[best]),
            "accuracy_by_window": {str(w): float(a) for w, a in zip(windows, acc)},
            "oracle_check": {"windows": sample_w, "gpu_correct": [got[w] for w in sample_w],
                             "oracle_correct": [int(c) for c in ref]},
            "cpu_baseline": {"value": N * len(sample_w) / cpu_s, "unit": "queries/s",
                             "cores": default_threads(), "kind": "oracle",
                             "sample": f"leave-one-out brute force for W in {sample_w}, "
                                       f"{cpu_s:.1f} s"},
            # the batched search's launches (library count) and the tally kernel
            "gpu_launches": (launches + 1) * args.steps,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ unequal lengths

def run_varlen(args):
    """Series of unequal lengths (Sec. 2 generalised): one
    ``nn_dtw_search_varlen`` per step over the ragged workload (train 8,000 x
    test 2,000, lengths 448..576, W = 102, V = 5), stage events inside every
    timed step; e2e through the host-buffer entry point."""
    import torch
    from paper_1808_09617_gb300 import nndtw, synth
    ds = synth.make_varlen()
    dev = torch.device("cuda", 0)
    nndtw.load()
    tv, to = ds.pack(ds.train)
    qv, qo = ds.pack(ds.test)
    train = nndtw.Ragged(torch.from_numpy(tv).to(dev), torch.from_numpy(to).to(dev), ds.max_len)
    test = nndtw.Ragged(torch.from_numpy(qv).to(dev), torch.from_numpy(qo).to(dev), ds.max_len)
    labels = torch.from_numpy(ds.train_labels).to(dev)
    N, Q, ml = ds.N, ds.Q, ds.max_len
    ws = torch.empty(nndtw.nn_dtw_varlen_workspace_size(N, Q, ml, ds.W, ds.V), dtype=torch.uint8,
                     device=dev)
    outs = (torch.empty(Q, dtype=torch.int32, device=dev),
            torch.empty(Q, dtype=torch.int32, device=dev),
            torch.empty(Q, dtype=torch.float64, device=dev))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    tuned = nndtw.DTW_GROUP(args.dtw_group) if args.dtw_group else 0
    if not args.no_tune and not args.dtw_group:
        from paper_1808_09617_gb300 import autotune
        tuned = autotune.tune_search_varlen(train, labels, test, ds.W, ds.V, workspace=ws,
                                            out=outs)
    run = lambda flags=nndtw.TIME_STAGES, stats=False: nndtw.nn_dtw_search_varlen(
        train, labels, test, ds.W, ds.V, flags=flags | tuned, workspace=ws, out=outs,
        stats=stats)
    counted = run(flags=0, stats=True).stats          # work counters (slower: not timed)
    for _ in range(args.warmup):
        flush.zero_()
        run()
    torch.cuda.synchronize()
    launches = nndtw.nn_dtw_last_call_launches()
    stage_launches = nndtw.nn_dtw_last_call_stage_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stages = []
    sel = device_selector(torch, dev, 0)
    with ClockSampler(sel) as clk:
        torch.cuda.synchronize()
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            run()
            b.record(stream)
            stages.append(nndtw.nn_dtw_stage_times())
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
    clocks = clk.summary()
    stage_ms = {k: sum(d[k] for d in stages) / len(stages) for k in STAGES}
    idx = outs[0].cpu().numpy()
    # e2e: the host-buffer C-ABI call, copies of the ragged sets in and the
    # results out inside the timed region (pinned host arrays)
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    hs = nndtw.VarlenHostSearch(pin(tv), pin(to), pin(ds.train_labels), pin(qv), pin(qo), ds.W,
                                ds.V, ml, flags=tuned, device=dev)
    for _ in range(2):
        hs()
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hidx, _, _ = hs()
        e2e_t.append(time.perf_counter() - t0)
    e2e_ms = 1000.0 * sum(e2e_t) / len(e2e_t)
    h2d, d2h = hs.bytes_per_call()
    # roofline of the DTW stage against the derived FP32 cell peak
    peaks, peak_src = read_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(clocks["sm_max_mhz"] or peaks.get("sm_max_mhz", 2070.0))
    probe = nndtw.nn_dtw_probe_cell_rate(20000)
    cells = counted["dtw_cells"]
    dtw_ms = stage_ms["seed"] + stage_ms["dtw"]
    achieved = cells / (dtw_ms * 1e-3) / 1e9
    peak = n_sm * FP32_LANES_PER_SM * sm_max * 1e6 / INSTR_PER_CELL / 1e9
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gcell/s",
            "frac": achieved / peak, "kernel": "dtw (first candidates and survivors)",
            "peak_basis": f"derived: {n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                          f"{sm_max:.0f} MHz / {INSTR_PER_CELL} instructions per cell",
            "probe_measured": probe / 1e9, "frac_of_probe": achieved / (probe / 1e9),
            "launches_per_step": stage_launches["seed"] + stage_launches["dtw"],
            "share_of_step": dtw_ms / stage_ms["total"] if stage_ms["total"] else None,
            "traffic": None,
            "stage_timing": "CUDA events between the search's stages in every timed step"}
    line = {"metric": "unequal lengths: exact NN-DTW queries/s on 1 GB300 (FP32 with FP64 "
                      "recheck)",
            "value": Q / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"unequal lengths: train {N} x test {Q}, lengths "
                                   f"{ds.extra['L0'] - ds.extra['dL']}..{ds.extra['L0'] + ds.extra['dL']}, "
                                   f"W={ds.W}, V={ds.V}, float32",
                       "l2": "flushed before every step (256 MiB write, outside the events)",
                       "autotuned_dtw_group": (tuned >> 8) and 1 << (((tuned >> 8) & 7) - 1)},
            "roofline": roof, "stage_ms": stage_ms,
            "pruning": {k: counted[k] for k in ("pairs", "lb_pruned", "lb_pruned_live",
                                                "dtw_started", "dtw_abandoned", "dtw_cells",
                                                "rechecked")},
            "no_neighbour_queries": int((idx < 0).sum()),
            "e2e": {"value": Q / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms,
                    "results_equal_device_step": bool(np.array_equal(hidx, idx))},
            "gpu_launches": launches * args.steps, "gpu_launches_per_step_by_stage": stage_launches,
            "clocks": clocks}
    if not args.no_cpu_baseline:
        import oracle
        orc = oracle.get()
        env = orc.envelopes_var(tv, to, ds.W)
        n = 256
        t0 = time.perf_counter()
        sv, so = ds.pack(ds.test[:n])
        orc.nn_pruned_var(tv, to, ds.train_labels, sv, so, ds.W, ds.V, env=env)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": n / dt, "unit": UNIT, "cores": oracle.default_threads(),
                                "kind": "oracle",
                                "sample": f"first {n} queries against all {N} training series, "
                                          f"lower-bound search in FP64 (envelopes precomputed), "
                                          f"{dt:.1f} s"}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving

def run_serving(args):
    """Serving form: 16 resident training sets, Poisson query streams at
    several rates, continuous batching across sets; p50/p99 latency and
    sustained queries/s per rate.  Queries cycle through a pool of 1,024
    pre-drawn series per set (drawing them at 50k/s would dominate)."""
    from paper_1808_09617_gb300 import serving, synth
    specs = synth.serving_specs(16)
    sets = {}
    for d, sp in enumerate(specs):
        ds = synth.make_serving_set(d, sp)
        sets[d] = (ds.train, ds.train_labels, sp["W"], sp["V"])
    pools = {d: synth.serving_queries(d, specs[d], 1024)[0] for d in sets}
    srv = serving.Server(sets, n_slots=args.serve_slots, max_batch=args.serve_batch,
                         mix_ratio=args.serve_mix)
    rng = np.random.default_rng(7)
    results = []
    try:
        fs = [srv.submit(pools[d][0], d) for d in sets]
        [f.result() for f in fs]
        for rate in args.serve_rates:
            srv.latencies.clear()
            srv.completed = 0
            srv.t_first = srv.t_last = None
            srv.batches = 0
            srv.batch_sets = 0
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
                       "max_batch": args.serve_batch, "seconds_per_rate": args.serve_seconds,
                       "mix_ratio": args.serve_mix if args.serve_mix != float("inf") else None},
            "rates": results}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-graph", action="store_true",
                    help="launch each step's kernels directly instead of replaying a CUDA graph")
    ap.add_argument("--no-tune", action="store_true", help="skip the lanes-per-pair autotuner")
    ap.add_argument("--reverse", action="store_true",
                    help="test the cascade's reverse bound in every dataset (with --dtw-group "
                         "or --no-tune; the tuner decides otherwise)")
    ap.add_argument("--improved", action="store_true",
                    help="test the bound with the LB_Improved bridge in every dataset (with "
                         "--dtw-group or --no-tune; the tuner decides otherwise)")
    ap.add_argument("--tuned-flags", default=None,
                    help="JSON file of per-dataset search flags: read if it exists (no tuning), "
                         "else written after tuning, so that a profiled run repeats the choices "
                         "of a plain one")
    ap.add_argument("--lb-tile", type=int, default=0, choices=[0, 1, 2, 3],
                    help="tile shape of the bound pass for every dataset (1: 32 x 32, "
                         "2: 64 x 64, 3: 128 x 64); 0: the library's or the tuner's choice")
    ap.add_argument("--dtw-group", type=int, default=0,
                    help="lanes per pair for every dataset (1..32, or 64 for the row layout); "
                         "implies --no-tune")
    ap.add_argument("--serve-rates", type=float, nargs="*",
                    default=[1000, 5000, 10000, 20000, 50000])
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-batch", type=int, default=512)
    ap.add_argument("--serve-mix", type=float, default=float("inf"),
                    help="sets share a serving batch only within this factor of cost per query")
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
    if args.workload == "window":
        if rank == 0:
            run_window(args)
        return
    if args.workload == "vsweep":
        if rank == 0:
            run_vsweep(args)
        return
    if args.workload == "varlen":
        if rank == 0:
            run_varlen(args)
        return
    if args.workload == "batched":
        dsets, desc = batched_workload()
    else:
        dsets, desc = single_workload(args.workload)
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, dsets, desc)
        return

    import torch
    from paper_1808_09617_gb300 import autotune, nndtw

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    nndtw.load()
    stream = torch.cuda.current_stream()
    batched = args.workload == "batched"

    sets = [dict(train=torch.from_numpy(d.train).to(dev),
                 labels=torch.from_numpy(d.train_labels).to(dev),
                 test=torch.from_numpy(d.test).to(dev), W=d.W, V=d.V, flags=0) for d in dsets]
    Qtot = sum(d.Q for d in dsets)
    # lanes-per-pair per dataset (datasets with enough pairs to matter)
    tuned = {}
    cascade = (nndtw.REVERSE if args.reverse else 0) | (nndtw.IMPROVED if args.improved else 0)

    def record(g, flags):
        return {"group": g, "reverse": bool(flags & nndtw.REVERSE),
                "improved": bool(flags & nndtw.IMPROVED),
                "lb_tile": (flags & nndtw.LB_TILE_MASK) >> 19}
    if args.dtw_group:
        for i, s in enumerate(sets):
            s["flags"] = nndtw.DTW_GROUP(args.dtw_group) | cascade
            tuned[i] = record(args.dtw_group, cascade)
    elif args.no_tune and cascade:
        for i, s in enumerate(sets):
            s["flags"] = cascade
            tuned[i] = record(0, cascade)
    elif args.tuned_flags and os.path.exists(args.tuned_flags):
        with open(args.tuned_flags) as f:
            saved = json.load(f)
        if len(saved["flags"]) != len(sets):
            raise SystemExit(f"{args.tuned_flags}: {len(saved['flags'])} datasets, expected {len(sets)}")
        for i, s in enumerate(sets):
            s["flags"] = int(saved["flags"][i])
        tuned = {int(k): v for k, v in saved["tuned"].items()}
    elif not args.no_tune:
        for i, (d, s) in enumerate(zip(dsets, sets)):
            if d.N * d.Q >= 50_000:
                s["flags"] = autotune.tune_search_flags(s["train"], s["labels"], s["test"], d.W,
                                                        d.V, reps=2)
                g = autotune.tune_search(s["train"], s["labels"], s["test"], d.W, d.V, reps=2)
                if g or s["flags"] & (nndtw.REVERSE | nndtw.IMPROVED | nndtw.LB_TILE_MASK):
                    tuned[i] = record(g, s["flags"])
        if args.tuned_flags and rank == 0:
            with open(args.tuned_flags, "w") as f:
                json.dump({"flags": [s["flags"] for s in sets], "tuned": tuned}, f)
    if args.lb_tile:
        for s in sets:
            s["flags"] = (s["flags"] & ~nndtw.LB_TILE_MASK) | nndtw.LB_TILE(args.lb_tile)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # counting pass (untimed): pruning and cells per dataset
    counts = []
    for s in sets:
        counts.append(nndtw.nn_dtw_search(s["train"], s["labels"], s["test"], s["W"], s["V"],
                                          flags=s["flags"], stats=True).stats)

    # the timed step
    if batched:
        # stage events on the search's stream inside every timed step
        bs = nndtw.BatchedSearch(sets, flags=nndtw.TIME_STAGES, graph=not args.no_graph)
        run = bs.run
        outs = bs.outs
    else:
        s = sets[0]
        d0 = dsets[0]
        ws = torch.empty(nndtw.nn_dtw_workspace_size(d0.N, d0.Q, d0.L, d0.W, d0.V),
                         dtype=torch.uint8, device=dev)
        out = (torch.empty(d0.Q, dtype=torch.int32, device=dev),
               torch.empty(d0.Q, dtype=torch.int32, device=dev),
               torch.empty(d0.Q, dtype=torch.float64, device=dev))
        outs = [out]

        def one(flags=0):
            nndtw.nn_dtw_search(s["train"], s["labels"], s["test"], s["W"], s["V"],
                                flags=flags | s["flags"], workspace=ws, out=out)
        run = lambda: one(nndtw.TIME_STAGES)
        if not args.no_graph:
            one(nndtw.TIME_STAGES)
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            cs = torch.cuda.Stream(dev)
            cs.wait_stream(stream)
            with torch.cuda.stream(cs):
                with torch.cuda.graph(graph, stream=cs):
                    one(nndtw.TIME_STAGES)
            stream.wait_stream(cs)
            torch.cuda.synchronize()
            run = graph.replay

    for _ in range(args.warmup):
        flush.zero_()
        run()
        nndtw.nn_dtw_stage_times()
    torch.cuda.synchronize()
    # kernel launches of one step, in all and per stage (library counts of the
    # last search call this thread issued: the captured one when the step is a
    # graph replay, which launches the same kernels)
    launches_step = nndtw.nn_dtw_last_call_launches()
    stage_launches = nndtw.nn_dtw_last_call_stage_launches()

    sel = device_selector(torch, dev, local)
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
            run()
            ev_e[k].record(stream)
            # the step's own stage events (waits for this step to finish)
            stages.append(nndtw.nn_dtw_stage_times())
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    step_ms = [ev_s[k].elapsed_time(ev_e[k]) for k in range(args.steps)]
    ms = max_over_ranks(sum(step_ms) / len(step_ms), dist, dev)
    value = whole_job_rate(world, Qtot, ms)
    clocks = clk.summary()

    stage_ms = {k: sum(d[k] for d in stages) / len(stages) for k in STAGES}
    peaks, peak_src = read_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(clocks["sm_max_mhz"] or peaks.get("sm_max_mhz", 2070.0))
    probe = nndtw.nn_dtw_probe_cell_rate(20000)
    seed_cells = sum(c["seed_cells"] for c in counts)
    main_cells = sum(c["dtw_cells"] for c in counts) - seed_cells
    nds = len(dsets)
    work = {"dtw": main_cells, "seed": seed_cells,
            "lb": sum(d.N * d.Q * d.L for d in dsets),
            "envelopes": sum(12 * d.N * d.L for d in dsets)}
    launches = {k: max(1, stage_launches.get(k, 1)) for k in STAGES[:7]}
    roof = roofline(stage_ms, launches, work, n_sm, sm_max, peaks, peak_src, probe, args.workload)
    roof["stage_timing"] = ("CUDA events on the search's stream between its stages, in every "
                            "timed step; each stage is one launch per kernel variant over all "
                            "datasets, so a stage's time covers exactly its launches")
    # achieved HBM bandwidth of the envelope and bound stages (algorithmic bytes)
    sb = stage_bytes([dict(N=d.N, Q=d.Q, L=d.L) for d in dsets], [s["flags"] for s in sets],
                     nndtw)
    hbm_peak = float(peaks["hbm_gbs"])
    hbm = {}
    for key in ("envelopes", "lb"):
        if stage_ms[key] > 0:
            gbs = sb[key] / (stage_ms[key] * 1e-3) / 1e9
            hbm[key] = {"algorithmic_bytes_per_step": sb[key], "ms_per_step": stage_ms[key],
                        "launches_per_step": stage_launches.get(key, 0), "achieved_gbs": gbs,
                        "peak_gbs": hbm_peak, "frac": gbs / hbm_peak,
                        "peak_source": f"{peak_src} copy bandwidth"}
    roof["hbm_stages"] = hbm

    # plain FP64 form, one dataset per call, same data promoted
    fp64 = None
    if args.fp64_steps > 0:
        t64 = [(s["train"].double(), s["test"].double()) for s in sets]
        e1, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(args.fp64_steps):
            flush.zero_()
            e1.record()
            for (tr, te), s in zip(t64, sets):
                nndtw.nn_dtw_search(tr, s["labels"], te, s["W"], s["V"])
            e2.record()
            torch.cuda.synchronize()
            tot += e1.elapsed_time(e2)
        ms64 = tot / args.fp64_steps
        fp64 = {"ms_per_step": ms64, "value": world * Qtot / (ms64 / 1e3), "unit": UNIT,
                "fp32_over_fp64": ms64 / ms, "form": "plain FP64, one dataset per call"}
        del t64

    # end to end through the C ABI on host buffers: nn_dtw_search_batched_host
    # copies every dataset's series and labels in from pinned memory, searches
    # the batch and copies every result back, every step
    pinned = []

    def pin(x):
        t = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        pinned.append(t)
        return t.numpy()
    hsets = [dict(train=pin(d.train), labels=pin(d.train_labels), test=pin(d.test), W=d.W,
                  V=d.V, flags=s["flags"]) for d, s in zip(dsets, sets)]
    houts = [(pin(np.empty(d.Q, np.int32)), pin(np.empty(d.Q, np.int32)),
              pin(np.empty(d.Q, np.float64))) for d in dsets]
    hb = nndtw.BatchedHostSearch(hsets, outs=houts, device=dev)
    e2e_t = []
    for k in range(args.steps + 2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hb.run()
        if k >= 2:
            e2e_t.append(time.perf_counter() - t0)
    e2e_launches = nndtw.nn_dtw_last_call_launches()
    e2e_ms = max_over_ranks(1000.0 * sum(e2e_t) / len(e2e_t), dist, dev)
    e2e_same = all(np.array_equal(h, o.cpu().numpy()) for ho, out in zip(houts, outs)
                   for h, o in zip(ho, out))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(dsets)

    if rank == 0:
        eff_cells = sum(d.Q * d.N * band_cells(d.L, d.W) for d in dsets)
        pairs = sum(c["pairs"] for c in counts)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": desc, "queries_per_step": Qtot,
                       "l2": "flushed before every step (256 MiB write, outside the step's events)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "launch": "CUDA graph replay" if not args.no_graph else "direct launches",
                       "autotuned": {str(k): v for k, v in tuned.items()}},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": whole_job_rate(world, Qtot, e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": int(sum(d.train.nbytes + d.test.nbytes +
                                                  d.train_labels.nbytes for d in dsets)),
                    "d2h_bytes_per_step": int(Qtot * (4 + 4 + 8)), "ms_per_step": e2e_ms,
                    "call": "nn_dtw_search_batched_host (C ABI, pinned host buffers, direct "
                            "launches)",
                    "gpu_launches_per_step": e2e_launches,
                    "results_equal_device_step": bool(e2e_same)},
            "gpu_launches": launches_step * args.steps,
            "gpu_launches_per_step_by_stage": stage_launches,
            "clocks": clocks,
            "gcups_effective": eff_cells / (ms * 1e-3) / 1e9,
            "gcups_dtw_kernel": (main_cells / (stage_ms["dtw"] * 1e-3) / 1e9
                                 if stage_ms["dtw"] > 0 else None),
            "stage_ms": stage_ms,
            "pruning": {"pairs": pairs,
                        "lb_pruned": sum(c["lb_pruned"] for c in counts),
                        "lb_pruned_frac": sum(c["lb_pruned"] for c in counts) / pairs,
                        "lb_pruned_reverse": sum(c["lb_pruned_reverse"] for c in counts),
                        "lb_pruned_improved": sum(c["lb_pruned_improved"] for c in counts),
                        "lb_pruned_live": sum(c["lb_pruned_live"] for c in counts),
                        "dtw_started": sum(c["dtw_started"] for c in counts),
                        "dtw_abandoned": sum(c["dtw_abandoned"] for c in counts),
                        "dtw_cells": main_cells + seed_cells,
                        "rechecked": sum(c["rechecked"] for c in counts),
                        "recheck_queries": sum(c["recheck_queries"] for c in counts)},
            "fp64_plain": fp64,
            "tightness_pairs_workload": tightness_pairs(dev),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
