#!/usr/bin/env python3
"""Benchmark of batched leftmost-argmin RMQ (block-based sparse table) on GB300.

Workload (default): the paper-shaped single array, A int32 n = 1e8 uniform in
[0, 2^31), q = 1e7 queries with l, r uniform over [0, n) and l <= r.  One step
answers the batch once with each form of the method -- plain BbST (block
minima, sparse table, queries) and BbST_CON (endpoint sort, remap,
contraction, table over A_Q, queries) -- so a step covers every stage of the
hot path and answers 2q queries.  Inputs are resident in HBM before timing;
L2 is flushed before each form, outside the timed events: a 256 MiB write, then a
256 MiB read of another buffer so that the flush's dirty lines are written back
before the form starts.  Each form is one rmq_batch_ex call between two
events; the per-stage times (and the block-minima kernel time of the
roofline) come from rmq_batch_timed calls on the same batch right after the
timed region, since events between the kernels of a call cost it the overlap
of programmatic launches.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With --impl reference the CPU oracle (naive
per-query scan, all host cores) answers a bounded sample of the same batch.
Under torchrun every rank answers its own batch (weak scaling, no collective
on the data path); the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "queries/s incl. preprocessing and achieved HBM GB/s; served p50/p99 latency vs plain"
UNIT = "queries/s"
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["single", "multi", "served"], default="single",
                   help="single: one n=1e8 array (default); multi: 512 uneven arrays in one launch; "
                        "served: 64 resident arrays, Poisson request stream")
    p.add_argument("--duration", type=float, default=2.0, help="served: seconds of arrivals")
    p.add_argument("--rate", type=float, default=1e4, help="served: requests per second")
    p.add_argument("--arrays", type=int, default=512)
    p.add_argument("--n", "--array-size", dest="n", type=float, default=1e8)
    p.add_argument("--q", "--num-queries", dest="q", type=float, default=1e7)
    p.add_argument("--seed", type=int, default=1002)
    p.add_argument("--array", choices=["uniform", "permutation"], default="uniform",
                   help="single: A uniform int32 (default) or the paper's permutation with n/2 swaps")
    p.add_argument("--variant", choices=["both", "plain", "contracted"], default="both")
    p.add_argument("--k", type=int, default=0, help="plain-form block size (0 = tuned)")
    p.add_argument("--k-con", type=int, default=0, help="contracted-form block size (0 = tuned)")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--cpu-seconds", type=float, default=20.0, help="budget of the oracle baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


# ----------------------------------------------------------------- helpers

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


class Dist:
    """Barrier and max-reduction over ranks (gloo, host tensors)."""

    def __init__(self):
        self.rank, self.world, self.local = dist_env()
        self.pg = None
        if self.world > 1:
            import torch.distributed as td
            td.init_process_group("gloo")
            self.pg = td

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def workload(n, q, seed, rank, array="uniform"):
    from paper_1706_06940_gb300 import workloads as W
    if array == "permutation":
        A = W.paper_permutation(n, seed + 7919 * rank)
    else:
        A = W.uniform_array(n, seed + 7919 * rank)
    l, r = W.uniform_queries(n, q, seed + 7919 * rank + 1)
    return A, l, r


def workload_name(n, q, array="uniform"):
    what = ("the paper's array (1..n after n/2 random pair swaps)" if array == "permutation"
            else "uniform in [0,2^31)")
    return ("paper-shaped single array: A int32 n=%g %s, q=%g queries with l,r uniform "
            "over [0,n) swapped so l<=r; one step = the batch answered by plain BbST and by BbST_CON"
            % (n, what, q))


class ClockSampler:
    """nvidia-smi SM clock / throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, t0=None, t1=None):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        window = [ln for ts, ln in self.lines if t0 is None or t0 - 0.15 <= ts <= t1 + 0.15]
        for ln in window or [ln for _, ln in self.lines]:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def coarse_lc(nb, cap=4096):
    """Levels 0 .. lc of a plain block table of nb blocks are kept in memory:
    lc is the smallest shift whose coarse summary (nbc = ceil(nb / 2^lc)
    coarse blocks, level t holding its nbc - 2^t + 1 defined entries) has at
    most cap entries."""
    lc = 0
    while True:
        nbc = -(-nb // (1 << lc))
        lvc = nbc.bit_length()
        if lvc * (nbc + 1) - ((1 << lvc) - 1) <= cap:
            return lc
        lc += 1


def profiled_traffic(kernel_src_rel, summary_rel, n, k):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current source of the kernel (its sha256 is recorded there) and on
    this workload's n and k (recorded as workload_n, workload_k)."""
    try:
        text = open(os.path.join(ROOT, summary_rel)).read()
        src = open(os.path.join(ROOT, kernel_src_rel), "rb").read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", text)
    h = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    wn = re.search(r"workload_n:\s*([0-9]+)", text)
    wk = re.search(r"workload_k:\s*([0-9]+)", text)
    if not m or not h or h.group(1) != hashlib.sha256(src).hexdigest():
        return None
    if not wn or not wk or int(wn.group(1)) != n or int(wk.group(1)) != k:
        return None
    return int(m.group(1))


def cpu_baseline(A, l, r, budget_s):
    """The oracle (naive leftmost scan per query, OpenMP over all host cores)
    on the first queries of the same batch, sized to about budget_s."""
    import numpy as np

    import oracle
    threads = oracle.max_threads()
    # grow the sample until one run takes at least half the budget (a small
    # sample is dominated by its longest query on one thread)
    s2 = min(len(l), max(threads, 8))
    while True:
        t0 = time.perf_counter()
        oracle.rmq_naive(A, l[:s2], r[:s2])
        dt2 = time.perf_counter() - t0
        if dt2 >= 0.5 * budget_s or s2 == len(l):
            break
        s2 = int(min(len(l), max(2 * s2, 0.8 * budget_s * s2 / max(dt2, 1e-6))))
    width = float(np.sum(r[:s2].astype(np.int64) - l[:s2] + 1))
    return {"value": s2 / dt2, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "naive oracle on the first %d of the %d queries (%.3g cells scanned), %.1f s"
                      % (s2, len(l), width, dt2)}


# ----------------------------------------------------------------- reference arm

def run_reference(args, dist):
    """The CPU oracle on bounded samples of the same batch, rank 0 only."""
    if dist.rank != 0:
        return
    import numpy as np

    import oracle
    oracle.build()
    n, q = int(args.n), int(args.q)
    A, l, r = workload(n, q, args.seed, 0, args.array)
    threads = oracle.max_threads()
    per_step = max(0.2, min(2.0, 90.0 / max(args.steps + args.warmup, 1)))
    s = max(threads, 8)
    t0 = time.perf_counter()
    oracle.rmq_naive(A, l[:s], r[:s])
    rate = s / max(time.perf_counter() - t0, 1e-6)
    per = int(min(q, max(threads, per_step * rate)))
    cursor = 0
    times, answered = [], 0
    for i in range(args.warmup + args.steps):
        idx = (np.arange(cursor, cursor + per) % q)
        cursor += per
        t0 = time.perf_counter()
        oracle.rmq_naive(A, l[idx], r[idx])
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            answered += per
    total = sum(times)
    value = answered / total
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / max(len(times), 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": workload_name(n, q, args.array), "n": n, "q": q, "seed": args.seed,
                   "sample_queries_per_step": per},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "naive oracle, %d queries of the batch per step, %d timed steps"
                                   % (per, len(times))},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- our arm

def run_ours(args, dist):
    import numpy as np
    import torch

    import __graft_entry__
    if dist.rank == 0:
        __graft_entry__.build()
    dist.barrier()
    from paper_1706_06940_gb300 import rmq

    rmq.load()
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    n, q = int(args.n), int(args.q)
    A, l, r = workload(n, q, args.seed, dist.rank, args.array)
    dA = torch.from_numpy(A).to(dev)
    dl, dr = torch.from_numpy(l).to(dev), torch.from_numpy(r).to(dev)
    outs = {"plain": torch.empty(q, dtype=torch.int32, device=dev),
            "contracted": torch.empty(q, dtype=torch.int32, device=dev)}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    flush_rd = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    # block sizes: measured on this batch over 32..4096 (the autotuner), unless given
    tune_ms = {}
    k, k_con = args.k, args.k_con
    run_forms = ["plain", "contracted"] if args.variant == "both" else [args.variant]
    if not k:
        k = rmq.rmq_tune(n, q)["k"]
        if "plain" in run_forms:
            best, tune_ms["plain"] = rmq.rmq_autotune(dA, dl, dr, outs["plain"], variant=1, k_min=32, k_max=4096)
            k = best["k"]
    if not k_con:
        k_con = rmq.rmq_tune(n, q)["k_con"]
        if "contracted" in run_forms:
            best, tune_ms["contracted"] = rmq.rmq_autotune(dA, dl, dr, outs["contracted"], variant=2, k_min=32,
                                                           k_max=4096)
            k_con = best["k_con"]
    forms = ["plain", "contracted"] if args.variant == "both" else [args.variant]
    nev = {"plain": 4, "contracted": 6}
    vcode = {"plain": rmq.Variant.PLAIN, "contracted": rmq.Variant.CONTRACTED}
    stream = torch.cuda.current_stream(dev)

    # a step is one rmq_batch_ex call per form (the public entry point),
    # bracketed by two events; the per-stage breakdown comes from separate
    # rmq_batch_timed calls after the timed region (events between the
    # kernels of a call cost it the overlap of programmatic launches)
    def one_step(it):
        evs = {}
        for f in forms:
            flush.fill_(it & 0xFF)
            flush_rd.max()
            evs[f] = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            evs[f][0].record(stream)
            rmq.rmq_batch_ex(dA, dl, dr, outs[f], variant=vcode[f], k=k, k_con=k_con)
            evs[f][1].record(stream)
        return evs

    def staged_step(it):
        evs = {}
        for f in forms:
            flush.fill_(it & 0xFF)
            flush_rd.max()
            evs[f] = [torch.cuda.Event(enable_timing=True) for _ in range(nev[f])]
            rmq.rmq_batch_timed(dA, dl, dr, outs[f], evs[f], variant=vcode[f], k=k, k_con=k_con)
        return evs

    for i in range(args.warmup):
        one_step(i)
    torch.cuda.synchronize()
    st = rmq.rmq_stream_status()
    if st != rmq.Status.OK:
        raise RuntimeError("device status after warm-up: %s" % st.name)
    # spot check of the answers against the oracle on a sample (outside timing)
    import oracle
    idx = np.random.default_rng(5).choice(q, size=min(q, 48), replace=False)
    want = oracle.rmq_naive(A, l[idx], r[idx])
    for f in forms:
        got = outs[f].cpu().numpy()[idx]
        if not np.array_equal(got, want):
            raise RuntimeError("%s form: answers differ from the oracle on the spot check" % f)

    clocks = ClockSampler(dist.local)
    clocks.start()
    time.sleep(0.3)
    launches0 = rmq.rmq_launch_count()
    dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    all_evs = [one_step(args.warmup + i) for i in range(args.steps)]
    torch.cuda.synchronize()
    t_wall1 = time.perf_counter()
    t_wall = t_wall1 - t_wall0
    dist.barrier()
    launches = rmq.rmq_launch_count() - launches0
    clk = clocks.stop(t_wall0, t_wall1)

    form_ms = {f: 0.0 for f in forms}
    for evs in all_evs:
        for f in forms:
            form_ms[f] += evs[f][0].elapsed_time(evs[f][1]) / args.steps
    # per-stage device times (ms) from calls with events at the stage
    # boundaries, outside the timed region
    stage_names = {"plain": ["block_minima", "sparse_table", "queries"],
                   "contracted": ["mark", "rank", "contract", "table_AQ", "queries"]}
    stages = {f: {s: 0.0 for s in stage_names[f]} for f in forms}
    staged_ms = {f: 0.0 for f in forms}
    n_staged = max(3, min(args.steps, 20))
    staged = [staged_step(i) for i in range(n_staged)]
    torch.cuda.synchronize()
    for evs in staged:
        for f in forms:
            e = evs[f]
            for j, s in enumerate(stage_names[f]):
                stages[f][s] += e[j].elapsed_time(e[j + 1]) / n_staged
            staged_ms[f] += e[0].elapsed_time(e[-1]) / n_staged
    ms_step = sum(form_ms.values())
    ms_step_max = dist.max(ms_step)
    units = 2 * q if len(forms) == 2 else q
    value = dist.world * units / (ms_step_max * 1e-3)

    # roofline of the dominant single kernel: block minima over A (plain a1)
    peak, peak_kind = measured_peak_hbm()
    nb = -(-n // k)
    # the block table keeps levels 0 .. lc (the coarse level above lives in
    # shared memory); with k >= 128 the block-minima pass also writes the
    # minima of every 128 cells (Sec. 3.3's small blocks)
    lc = coarse_lc(nb)
    m1 = -(-n // 128) if k >= 128 else 0
    bytes_a1 = 4 * n + 8 * nb + 8 * m1
    ms_a1 = stages["plain"]["block_minima"] if "plain" in stages else None
    roof = None
    if ms_a1:
        ach = bytes_a1 / (ms_a1 * 1e-3) / 1e9
        roof = {"kernel": "k_block_min_warp (block minima over A, plain step a1)", "bound": "hbm",
                "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "peak_kind": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind if peak_kind == "measured"
                else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": bytes_a1,
                "kernel_time": "CUDA events around the block-minima stage of %d rmq_batch_timed calls on "
                               "the same batch, same stream, right after the timed region" % n_staged,
                "traffic": profiled_traffic("paper_1706_06940_gb300/csrc/block_min.cu",
                                            "profiles/block_minima_n1e8.md", n, k)}
    # device workspace of each form (the extra memory of Table 2)
    ws_bytes = {f: rmq.rmq_batch_workspace_bytes(n, q, vcode[f], k=k, k_con=k_con) for f in forms}
    # whole-form HBM accounting (algorithmic bytes of the plain form)
    hbm_plain = None
    if "plain" in form_ms:
        b = 4 * n + 8 * (nb * (lc + 1) + m1) + 12 * q
        hbm_plain = {"algorithmic_bytes": b, "gbs": b / (form_ms["plain"] * 1e-3) / 1e9,
                     "frac_of_measured": b / (form_ms["plain"] * 1e-3) / 1e9 / peak,
                     "frac_of_8tbs_nominal": b / (form_ms["plain"] * 1e-3) / 1e9 / 8000.0}

    # end to end: host buffers through rmq_batch_host, copies inside the timing
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        pA = torch.from_numpy(A).pin_memory()
        pl, pr = torch.from_numpy(l).pin_memory(), torch.from_numpy(r).pin_memory()
        pout = torch.empty(q, dtype=torch.int32).pin_memory()
        hA, hl, hr, ho = pA.numpy(), pl.numpy(), pr.numpy(), pout.numpy()
        for f in forms:                                          # warm the pool
            rmq.rmq_batch_host(hA, hl, hr, ho, variant=vcode[f], k=k, k_con=k_con)
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for f in forms:
                rmq.rmq_batch_host(hA, hl, hr, ho, variant=vcode[f], k=k, k_con=k_con)
        dt = dist.max(time.perf_counter() - t0)
        e2e = {"value": dist.world * units * args.e2e_steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": len(forms) * (4 * n + 8 * q),
               "d2h_bytes_per_step": len(forms) * 4 * q,
               "ms_per_step": 1e3 * dt / args.e2e_steps, "buffers": "pinned host"}

    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(A, l, r, args.cpu_seconds)

    if dist.rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": workload_name(n, q, args.array), "n": n, "q": q, "seed": args.seed,
                       "forms": forms, "k": k, "k_con": k_con, "k_autotuned": {"range": [32, 4096],
                                                                           "best_ms": tune_ms},
                       "l2": "flushed before each form (outside the timed events) by a 256 MiB write, then a 256 MiB "
                             "read of another buffer (the write's dirty lines leave L2 before the form); "
                             "A alone (%.0f MB) exceeds L2" % (4 * n / 1e6),
                       "parallelism": "replicas" if dist.world > 1 else "single GPU"},
            "forms": {f: {"ms": form_ms[f], "queries_per_s": q / (form_ms[f] * 1e-3),
                          "stages_ms": stages[f], "staged_call_ms": staged_ms[f]} for f in forms},
            "hbm_plain": hbm_plain,
            "memory": {f: {"workspace_bytes": ws_bytes[f], "pct_of_4n": 100.0 * ws_bytes[f] / (4 * n)}
                       for f in forms},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "wall_s_timed_region": t_wall,
        }
        print(json.dumps(line), flush=True)


def run_multi(args, dist):
    """512 arrays, n log-uniform in [1e4, 1e7] (uniform int32 values), q
    log-uniform in [10, 1e5] uniform queries each: one persistent launch
    (rmq_batch_multi, replayed from a CUDA graph) against one rmq_batch call
    per array on the same stream."""
    import numpy as np
    import torch

    import __graft_entry__
    if dist.rank == 0:
        __graft_entry__.build()
    dist.barrier()
    from paper_1706_06940_gb300 import rmq, workloads as W

    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    ns, qs = W.uneven_batch(args.arrays, args.seed + 7919 * dist.rank)
    dA, ls, rs = [], [], []
    for h, (n, q) in enumerate(zip(ns, qs)):
        dA.append(torch.from_numpy(W.uniform_array(int(n), args.seed + 17 * h)).to(dev))
        l, r = W.uniform_queries(int(n), int(q), args.seed + 17 * h + 1)
        ls.append(l)
        rs.append(r)
    L = torch.from_numpy(np.concatenate(ls)).to(dev)
    R = torch.from_numpy(np.concatenate(rs)).to(dev)
    qtot = int(qs.sum())
    out = torch.empty(qtot, dtype=torch.int32, device=dev)
    out_seq = torch.empty(qtot, dtype=torch.int32, device=dev)
    s = torch.cuda.Stream(dev)
    qlist = [int(q) for q in qs]
    with torch.cuda.stream(s):
        rmq.rmq_batch_multi(dA, qlist, L, R, out, stream=s.cuda_stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    c0 = rmq.rmq_launch_count()
    with torch.cuda.graph(g, stream=s):
        rmq.rmq_batch_multi(dA, qlist, L, R, out, stream=s.cuda_stream)
    kernels_per_replay = rmq.rmq_launch_count() - c0
    offs = np.concatenate([[0], np.cumsum(qs)])

    def seq_calls():
        for h in range(len(dA)):
            a, b = int(offs[h]), int(offs[h + 1])
            rmq.rmq_batch(dA[h], L[a:b], R[a:b], out_seq[a:b], stream=s.cuda_stream)

    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            g.replay()
            seq_calls()
    torch.cuda.synchronize()
    if rmq.rmq_stream_status() != rmq.Status.OK:
        raise RuntimeError("device status after warm-up")
    if not torch.equal(out, out_seq):
        raise RuntimeError("multi-array launch and per-array calls disagree")
    import oracle
    for h in np.random.default_rng(3).choice(len(dA), 8, replace=False):
        a, b = int(offs[h]), int(offs[h + 1])
        if b > a:
            idx = np.random.default_rng(int(h)).choice(b - a, min(32, b - a), replace=False)
            want = oracle.rmq_naive(dA[h].cpu().numpy(), ls[h][idx], rs[h][idx])
            if not np.array_equal(out[a:b].cpu().numpy()[idx], want):
                raise RuntimeError("multi-array answers differ from the oracle on array %d" % h)
    clocks = ClockSampler(dist.local)
    clocks.start()
    time.sleep(0.3)
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(s):
        for e0, e1 in ev:
            e0.record(s)
            g.replay()
            e1.record(s)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    launches_graph = kernels_per_replay * args.steps   # graph replays launch the captured kernels
    ms_multi = sum(e0.elapsed_time(e1) for e0, e1 in ev) / args.steps
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(max(3, args.steps // 10))]
    with torch.cuda.stream(s):
        for e0, e1 in ev2:
            e0.record(s)
            seq_calls()
            e1.record(s)
    torch.cuda.synchronize()
    clk = clocks.stop(t0, t1)
    ms_seq = sum(e0.elapsed_time(e1) for e0, e1 in ev2) / len(ev2)
    ms_max = dist.max(ms_multi)
    peak, peak_kind = measured_peak_hbm()
    nbytes = 0
    for n, q in zip(ns, qs):
        if q > 0:
            nbytes += 4 * int(n)
    nbytes += 12 * qtot
    if dist.rank == 0:
        line = {
            "metric": METRIC, "value": dist.world * qtot / (ms_max * 1e-3), "unit": UNIT, "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "batched uneven: %d int32 arrays, n log-uniform in [1e4,1e7] (sum %d), q "
                                   "log-uniform in [10,1e5] (sum %d), uniform values and queries; one persistent "
                                   "launch replayed from a CUDA graph" % (len(dA), int(ns.sum()), qtot),
                       "arrays": len(dA), "sum_n": int(ns.sum()), "sum_q": qtot,
                       "l2": "inputs (%.1f GB) exceed L2" % (4e-9 * ns.sum())},
            "per_array_calls": {"ms": ms_seq, "queries_per_s": qtot / (ms_seq * 1e-3),
                                "speedup_of_one_launch": ms_seq / ms_multi},
            "hbm": {"algorithmic_bytes": nbytes, "gbs": nbytes / (ms_multi * 1e-3) / 1e9,
                    "frac_of_measured": nbytes / (ms_multi * 1e-3) / 1e9 / peak, "peak": peak,
                    "peak_kind": peak_kind},
            "gpu_launches": launches_graph, "clocks": clk,
        }
        print(json.dumps(line), flush=True)


def run_served(args, dist):
    """64 resident arrays totalling 4e9 cells (n log-uniform in [1e6, 2e8],
    rescaled), requests arriving as a Poisson stream, each on a random array
    with a log-uniform batch of [1, 1e5] uniform queries.  The library's
    server (continuous batching over several streams) against one rmq_query
    per request in arrival order on one stream, on the same arrival trace."""
    import numpy as np
    import torch

    import __graft_entry__
    if dist.rank == 0:
        __graft_entry__.build()
    dist.barrier()
    from paper_1706_06940_gb300 import rmq, workloads as W

    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    sizes = W.served_array_sizes(64, 4_000_000_000, args.seed + 7919 * dist.rank)
    gen = torch.Generator(device=dev)
    dA = []
    for h, n in enumerate(sizes):
        gen.manual_seed(args.seed + 31 * h)
        dA.append(torch.randint(0, 2**31 - 1, (int(n),), dtype=torch.int32, device=dev, generator=gen))
    torch.cuda.synchronize()                    # the arrays are written before the server reads them
    free0, _ = torch.cuda.mem_get_info(dev)
    srv = rmq.Server(budget_bytes=int(free0 * 0.8), inflight=4)
    t_adm = time.perf_counter()
    ids = [srv.admit(A) for A in dA]
    t_adm = time.perf_counter() - t_adm
    g = np.random.default_rng(args.seed + 1)
    nreq = int(args.rate * args.duration)
    arrive = np.cumsum(g.exponential(1.0 / args.rate, nreq))
    arr = g.integers(0, len(dA), nreq)
    qs = W.log_uniform_ints(g, nreq, 1, 1e5)
    reqs = []
    for i in range(nreq):
        n = int(sizes[arr[i]])
        a = g.integers(0, n, int(qs[i]), dtype=np.int64)
        b = g.integers(0, n, int(qs[i]), dtype=np.int64)
        reqs.append((int(arr[i]), np.minimum(a, b).astype(np.int32), np.maximum(a, b).astype(np.int32)))
    qtot = int(qs.sum())

    def served_run():
        outs = [np.empty(len(l), np.int32) for _, l, _ in reqs]
        tickets = [None] * nreq
        lat = np.zeros(nreq)
        done_t = [0.0]

        def waiter():
            for i in range(nreq):
                while tickets[i] is None:
                    time.sleep(20e-6)
                lat[i] = srv.wait(tickets[i])
            done_t[0] = time.perf_counter()

        th = threading.Thread(target=waiter)
        th.start()
        t0 = time.perf_counter()
        for i, (h, l, r) in enumerate(reqs):
            while time.perf_counter() - t0 < arrive[i]:
                pass
            tickets[i] = srv.submit(ids[h], l, r, outs[i])
        th.join()
        return lat, done_t[0] - t0, outs

    handles = [rmq.rmq_build(A) for A in dA]
    torch.cuda.synchronize()
    s = torch.cuda.Stream(dev)

    def fifo_run():
        lat = np.zeros(nreq)
        outs = []
        t0 = time.perf_counter()
        with torch.cuda.stream(s):
            for i, (h, l, r) in enumerate(reqs):
                while time.perf_counter() - t0 < arrive[i]:
                    pass
                dl = torch.from_numpy(l).to(dev, non_blocking=False)
                dr = torch.from_numpy(r).to(dev, non_blocking=False)
                out = torch.empty(len(l), dtype=torch.int32, device=dev)
                rmq.rmq_query(handles[h], dl, dr, out, stream=s.cuda_stream)
                o = out.cpu()
                lat[i] = time.perf_counter() - t0 - arrive[i]
                outs.append(o.numpy())
        return lat, time.perf_counter() - t0, outs

    clocks = ClockSampler(dist.local)
    clocks.start()
    lat_s, wall_s, outs_s = served_run()
    clk = clocks.stop()
    lat_f, wall_f, outs_f = fifo_run()
    st = srv.stats()
    for i in range(0, nreq, max(1, nreq // 200)):
        if not np.array_equal(outs_s[i], outs_f[i]):
            raise RuntimeError("served and per-request answers differ on request %d" % i)
    import oracle
    for i in g.choice(nreq, 16, replace=False):
        h, l, r = reqs[i]
        idx = g.choice(len(l), min(len(l), 16), replace=False)
        if not np.array_equal(outs_s[i][idx], oracle.rmq_naive(dA[h].cpu().numpy(), l[idx], r[idx])):
            raise RuntimeError("served answers differ from the oracle on request %d" % i)
    srv.close()
    for hd in handles:
        hd.free()
    if dist.rank == 0:
        pct = lambda a, p: float(np.percentile(a, p) * 1e3)
        line = {
            "metric": METRIC, "value": qtot / wall_s, "unit": UNIT, "n_gpus": dist.world, "steps": nreq,
            "warmup": 0, "ms_per_step": 1e3 * wall_s / nreq, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "served: 64 resident int32 arrays totalling %d cells (n log-uniform in "
                                   "[1e6,2e8], rescaled), Poisson arrivals at %g req/s for %g s, batch log-uniform "
                                   "in [1,1e5] uniform queries on a random array" % (int(sizes.sum()), args.rate,
                                                                                      args.duration),
                       "requests": nreq, "queries": qtot, "admit_s": t_adm},
            "served": {"queries_per_s": qtot / wall_s, "p50_ms": pct(lat_s, 50), "p99_ms": pct(lat_s, 99),
                       "max_ms": float(lat_s.max() * 1e3), "batches": st["batches"], "wall_s": wall_s},
            "one_request_per_call": {"queries_per_s": qtot / wall_f, "p50_ms": pct(lat_f, 50),
                                     "p99_ms": pct(lat_f, 99), "max_ms": float(lat_f.max() * 1e3),
                                     "wall_s": wall_f},
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    dist = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        elif args.workload == "multi":
            run_multi(args, dist)
        elif args.workload == "served":
            run_served(args, dist)
        else:
            run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
