#!/usr/bin/env python3
"""Benchmark of batched leftmost-argmin RMQ (block-based sparse table) on GB300.

Default run (what `python bench.py` measures):

* The headline workload, the paper-shaped single array: A int32 n = 1e8
  uniform in [0, 2^31), q = 1e7 queries with l, r uniform over [0, n) and
  l <= r.  One step answers the batch once with each form of the method --
  plain BbST (block minima, sparse table, queries) and BbST_CON (endpoint
  marks, ranks, contraction, table over A_Q, queries) -- so a step covers
  every stage of the hot path and answers 2q queries.  Inputs are resident in
  HBM before timing; L2 is flushed before each form, outside the timed
  events: a 256 MiB write, then a 256 MiB read of another buffer so that the
  flush's dirty lines are written back before the form starts.  Each form is
  one rmq_batch_ex call between two events.  The per-stage times (one
  kernel, or a kernel and its memset, per stage) come from rmq_batch_timed
  calls on the same batch right after the timed region, since events between
  the kernels of a call cost it the overlap of programmatic launches.  The
  edge-scan work S comes from rmq_batch_counted (an instrumented query kernel)
  on the same batch, outside the timed region.
* Then the other workloads, each as an object of the same JSON line:
  config1 (n = 1e6, q = 1e3: per-call latency), config3 (tie-heavy, short
  ranges), config4 (512 uneven arrays in one persistent launch replayed from
  a CUDA graph) and config5 (64 resident arrays served by the library's
  continuous-batching server against one call per request).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload all|single|c1|c3|multi|served]

Prints one JSON line (rank 0).  With --impl reference the CPU oracle (naive
per-query scan, all host cores) answers a bounded sample of the headline
batch.  Under torchrun every rank answers its own batch (weak scaling, no
collective on the data path); the slowest rank's time is reported, and the
other workloads run at N = 1 only.
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
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["all", "single", "c1", "c3", "multi", "served", "hlevel", "qsweep"], default="all",
                   help="all: the headline workload plus configs 1, 3, 4 and 5 and the multi-level leg in one line (default); "
                        "single: the headline workload only; c1, c3, multi, served: one other workload; "
                        "hlevel: the multi-level layout of Sec. 3.3 beside the plain form; qsweep: config 2 at q = 1e2 .. 1e6")
    p.add_argument("--served-requests", type=int, default=8000, help="served: requests in the pool")
    p.add_argument("--served-clients", type=int, default=16, help="served: closed-loop client threads")
    p.add_argument("--served-window", type=float, default=0.8, help="served: seconds of each open-loop arm")
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


def plain_workspace(n, k):
    """Device bytes of a plain batch call (the library's rmq_batch_workspace_bytes):
    levels 0..lc of the block table and one key per 128 cells for k >= 128."""
    nb = -(-n // k)
    m1 = -(-n // 128) if k >= 128 else 0
    return 8 * (nb * (coarse_lc(nb) + 1) + m1)


def profiled_traffic(kernel, kernel_src_rel, want):
    """DRAM bytes per launch of `kernel` from a committed ncu summary under
    profiles/ that names it (a line "kernel: <name>"), if it was taken on the
    current source of the file that holds the kernel (its sha256 is recorded
    there) and on this workload (every "workload_<key>: <value>" line of the
    summary must equal want[key])."""
    import glob
    try:
        src = open(os.path.join(ROOT, kernel_src_rel), "rb").read()
    except OSError:
        return None
    sha = hashlib.sha256(src).hexdigest()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read()
        if not re.search(r"^kernel:\s*%s\s*$" % re.escape(kernel), text, re.M):
            continue
        m = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", text)
        h = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
        if not m or not h or h.group(1) != sha:
            continue
        wl = dict(re.findall(r"^workload_(\w+):\s*([0-9]+)\s*$", text, re.M))
        if any(str(int(want.get(key, -1))) != v for key, v in wl.items()) or not wl:
            continue
        return int(m.group(1))
    return None


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




def flush_l2(flush, flush_rd, it):
    """Evict the batch from L2: a write of 256 MiB, then a read of another
    256 MiB buffer, so that the write's dirty lines are written back first."""
    flush.fill_(it & 0xFF)
    flush_rd.max()


def distinct_endpoints(n, l, r):
    """m: the number of distinct endpoint positions of a batch (host)."""
    import numpy as np
    mark = np.zeros(n, dtype=bool)
    mark[l] = True
    mark[r] = True
    return int(np.count_nonzero(mark))


def coarse_lc_con(nbq):
    return coarse_lc(nbq, cap=6656)


def small_block(k, k1):
    """Cells per small block of the plain form's two-level layout (None: none)."""
    if k1 is None or k1 == 0:
        return 128 if k >= 128 else None
    return None if k1 < 0 else k1


def form_bytes(n, q, k, k_con, m, counts, k1=0):
    """Algorithmic bytes of each stage of each form (per call), the kernels
    that run it, and the whole forms' HBM terms (n cells, q queries, block
    sizes k and k_con, m distinct endpoints, counts from rmq_batch_counted).

    Plain (Sec. 3.2): A read once (4n), levels 0..lc of the block table
    written (8 nb (lc + 1)), the minima of every small block of k1 cells
    (Sec. 3.3; by default 128 when k >= 128), l, r read and out written (12q),
    and the edge scans: S cells of A (4S) and the small-block minima they read.
    Contracted (Sec. 3.1): l, r read by the marking (8q) and W bit words
    written (4W, W = ceil(n/32) + 1); the ranks read the words and write their
    counts (8W); the contraction reads A, the words and counts, and writes
    A_Q (4n + 8W + 8(m - 1)); the table over A_Q reads A_Q and writes its
    levels; the queries read l, r, write out (12q), and read S keys of A_Q
    and the ranks of their open queries.
    """
    nb = -(-n // k)
    lc = coarse_lc(nb)
    sb1 = small_block(k, k1)
    m1 = -(-n // sb1) if sb1 else 0
    W = -(-n // 32) + 1
    mq = max(m - 1, 1)
    nbq = -(-mq // k_con)
    lcq = coarse_lc_con(nbq)
    cp, cc = counts.get("plain", {}), counts.get("contracted", {})
    S_p = cp.get("scan_elems", 0)
    S_c = cc.get("scan_elems", 0)
    stages = {
        "plain": {
            "block_minima": ("k_block_min_warp" if k >= 128 else "k_block_min_group",
                             "block_min.cu", 4 * n + 8 * nb + 8 * m1),
            "sparse_table": ("k_st_first", "sparse_table.cu", 8 * nb * (lc + 1)),
            "queries": ("k_query_two<SrcI32>", "query.cuh",
                        12 * q + 4 * S_p + 8 * cp.get("m1_reads", 0)),
        },
        "contracted": {
            "mark": ("k_mark_endpoints", "contract.cu", 8 * q + 4 * W),   # after a memset of the W words
            "rank": ("k_bits_partial + k_bits_final", "contract.cu", 8 * W),
            "contract": ("k_contract_pf", "contract.cu", 4 * n + 8 * W + 8 * mq),   # k_contract only where A is not 16-B aligned
            "table_AQ": ("k_block_min_warp<SrcU64> + k_st_first", "block_min.cu", 8 * mq + 8 * nbq * (lcq + 1)),
            "queries": ("k_query_two<SrcU64, CON>", "query.cuh",
                        12 * q + 8 * S_c + 4 * cc.get("rank_reads", 0)),
        },
    }
    hbm_plain = 4 * n + 8 * nb * (lc + 1) + 8 * m1 + 12 * q + 4 * S_p
    # the contracted form's algorithmic minimum as the measurement model
    # states it (one pass over A between the extreme endpoints, l and r read,
    # 2q sorted 8-byte pairs written and read once, A_Q, its table, out)
    con_min = 4 * n + 8 * q + 32 * q + 8 * m + 8 * nbq * (lcq + 1) + 4 * q
    return stages, hbm_plain, con_min, {"nb": nb, "lc": lc, "m1": m1, "W": W, "m": m, "nbq": nbq, "lcq": lcq}


# ----------------------------------------------------------------- headline workload

def run_main(args, dist, rmq, torch, np):
    dev = torch.device("cuda", dist.local)
    n, q = int(args.n), int(args.q)
    A, l, r = workload(n, q, args.seed, dist.rank, args.array)
    dA = torch.from_numpy(A).to(dev)
    dl, dr = torch.from_numpy(l).to(dev), torch.from_numpy(r).to(dev)
    outs = {"plain": torch.empty(q, dtype=torch.int32, device=dev),
            "contracted": torch.empty(q, dtype=torch.int32, device=dev)}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    flush_rd = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    forms = ["plain", "contracted"] if args.variant == "both" else [args.variant]
    # block sizes: measured on this batch over 32..4096 (the autotuner), unless given
    tune_ms = {}
    k, k_con = args.k, args.k_con
    # the autotuner's other choices per form: lanes per partial-block scan and
    # (plain form) the small blocks of the two-level layout
    xo = {"plain": {}, "contracted": {}}
    if not k:
        k = rmq.rmq_tune(n, q)["k"]
        if "plain" in forms:
            best, tune_ms["plain"] = rmq.rmq_autotune(dA, dl, dr, outs["plain"], variant=1, k_min=32, k_max=4096)
            k = best["k"]
            xo["plain"] = {"threads_per_query": best["threads_per_query"], "k1": best["k1"]}
    if not k_con:
        k_con = rmq.rmq_tune(n, q)["k_con"]
        if "contracted" in forms:
            best, tune_ms["contracted"] = rmq.rmq_autotune(dA, dl, dr, outs["contracted"], variant=2, k_min=32,
                                                           k_max=4096)
            k_con = best["k_con"]
            xo["contracted"] = {"threads_per_query": best["threads_per_query"]}
    nev = {"plain": 4, "contracted": 7}   # the contracted form's 7th event: after the bitmap clear
    vcode = {"plain": rmq.Variant.PLAIN, "contracted": rmq.Variant.CONTRACTED}
    stream = torch.cuda.current_stream(dev)

    # a step is one rmq_batch_ex call per form (the public entry point),
    # bracketed by two events
    def one_step(it):
        evs = {}
        for f in forms:
            flush_l2(flush, flush_rd, it)
            evs[f] = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            evs[f][0].record(stream)
            rmq.rmq_batch_ex(dA, dl, dr, outs[f], variant=vcode[f], k=k, k_con=k_con, **xo[f])
            evs[f][1].record(stream)
        return evs

    def staged_step(it):
        evs = {}
        for f in forms:
            flush_l2(flush, flush_rd, it)
            evs[f] = [torch.cuda.Event(enable_timing=True) for _ in range(nev[f])]
            rmq.rmq_batch_timed(dA, dl, dr, outs[f], evs[f], variant=vcode[f], k=k, k_con=k_con, **xo[f])
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
    # per-stage device times (ms) from calls with events at the stage boundaries
    stage_names = {"plain": ["block_minima", "sparse_table", "queries"],
                   "contracted": ["mark", "rank", "contract", "table_AQ", "queries"]}
    stages = {f: {s: 0.0 for s in stage_names[f]} for f in forms}
    staged_ms = {f: 0.0 for f in forms}
    clear_ms = 0.0   # contracted: the memset of the bit words at the start of the mark stage
    n_staged = max(3, min(args.steps, 20))
    staged = [staged_step(i) for i in range(n_staged)]
    torch.cuda.synchronize()
    for evs in staged:
        for f in forms:
            e = evs[f]
            for j, s in enumerate(stage_names[f]):
                stages[f][s] += e[j].elapsed_time(e[j + 1]) / n_staged
            staged_ms[f] += e[0].elapsed_time(e[len(stage_names[f])]) / n_staged
            if f == "contracted":
                clear_ms += e[0].elapsed_time(e[6]) / n_staged
    # the work of the open queries (edge scans S, table gathers), counted by
    # the instrumented query kernel on the same batch
    counts = {}
    for f in forms:
        cnt_out = torch.empty(q, dtype=torch.int32, device=dev)
        counts[f] = rmq.rmq_batch_counted(dA, dl, dr, cnt_out, variant=vcode[f], k=k, k_con=k_con, **xo[f])
        if not torch.equal(cnt_out, outs[f]):
            raise RuntimeError("%s form: the instrumented kernel's answers differ" % f)
    ms_step = sum(form_ms.values())
    ms_step_max = dist.max(ms_step)
    units = 2 * q if len(forms) == 2 else q
    value = dist.world * units / (ms_step_max * 1e-3)

    # per-kernel roofline of every stage, and the dominant kernel
    peak, peak_kind = measured_peak_hbm()
    m = distinct_endpoints(n, l, r)
    sb, hbm_b, con_min_b, geo = form_bytes(n, q, k, k_con, m, counts, xo["plain"].get("k1", 0))
    per_kernel = []
    for f in forms:
        for s in stage_names[f]:
            kern, src, b = sb[f][s]
            ms = stages[f][s]
            if f == "contracted" and s == "mark":
                # the stage is the clear of the W bit words (a memset), then the
                # marking kernel: each is listed with its own time
                W = geo["W"]
                gbs = 4 * W / (clear_ms * 1e-3) / 1e9 if clear_ms > 0 else None
                per_kernel.append({"form": f, "stage": "mark (clear)", "kernel": "memset of the bit words",
                                   "source": "contract.cu", "ms": clear_ms, "algorithmic_bytes": 4 * W, "gbs": gbs,
                                   "frac": gbs / peak if gbs else None})
                ms = max(ms - clear_ms, 0.0)
            gbs = b / (ms * 1e-3) / 1e9 if ms > 0 else None
            per_kernel.append({"form": f, "stage": s, "kernel": kern, "source": src, "ms": ms,
                               "algorithmic_bytes": b, "gbs": gbs, "frac": gbs / peak if gbs else None})
    dom = max(per_kernel, key=lambda e: e["ms"])
    dom_src = "paper_1706_06940_gb300/csrc/" + dom["source"]
    roof = {"kernel": "%s (%s form, stage %s)" % (dom["kernel"], dom["form"], dom["stage"]),
            "bound": "hbm", "achieved": dom["gbs"], "peak": peak, "unit": "GB/s", "frac": dom["frac"],
            "peak_kind": ("measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                          else "fallback 6.8 TB/s"),
            "algorithmic_bytes_per_launch": dom["algorithmic_bytes"],
            "kernel_time": "CUDA events around the %s stage of %d rmq_batch_timed calls on the same batch, same "
                           "stream, right after the timed region; the dominant kernel is the one with the largest "
                           "time of the step (the contracted mark stage is split at its event after the memset of "
                           "the bit words)" % (dom["stage"], n_staged),
            "traffic": profiled_traffic(dom["kernel"], dom_src, {"n": n, "q": q, "k": k, "k_con": k_con}),
            "per_kernel": per_kernel}
    if dom["kernel"] == "k_mark_endpoints":
        # its DRAM traffic is its algorithmic bytes, but its time is set by the
        # L2's rate of reductions (one red.global.or per endpoint)
        rate = 2 * q / (dom["ms"] * 1e-3)
        roof["bound_note"] = ("the kernel (one L2 reduction per endpoint) is bound by the L2 reduction rate, not "
                              "DRAM: %.3g reductions/s against about 1.9e11/s measured for bare reductions" % rate)
    ws_bytes = {f: rmq.rmq_batch_workspace_bytes(n, q, vcode[f], k=k, k_con=k_con, **xo[f]) for f in forms}
    hbm_plain = None
    if "plain" in form_ms:
        gbs = hbm_b / (form_ms["plain"] * 1e-3) / 1e9
        hbm_plain = {"algorithmic_bytes": hbm_b, "S_cells": counts["plain"]["scan_elems"], "gbs": gbs,
                     "frac_of_measured": gbs / peak, "frac_of_8tbs_nominal": gbs / 8000.0,
                     "terms": "4n + 8 nb (lc+1) + 8 ceil(n/k1) + 12q + 4S (k1: small blocks, 128 by default)"}
    hbm_con = None
    if "contracted" in form_ms:
        gbs = con_min_b / (form_ms["contracted"] * 1e-3) / 1e9
        hbm_con = {"algorithmic_bytes_min": con_min_b, "m": m, "S_keys": counts["contracted"]["scan_elems"],
                   "gbs": gbs, "frac_of_measured": gbs / peak,
                   "terms": "4n + 8q + 32q + 8m + 8 nbq (lcq+1) + 4q (the measurement model's B_min)"}

    # end to end: host buffers through rmq_batch_host, copies inside the timing
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        pA = torch.from_numpy(A).pin_memory()
        pl, pr = torch.from_numpy(l).pin_memory(), torch.from_numpy(r).pin_memory()
        pout = torch.empty(q, dtype=torch.int32).pin_memory()
        hA, hl, hr, ho = pA.numpy(), pl.numpy(), pr.numpy(), pout.numpy()
        for f in forms:                                          # warm the pool
            rmq.rmq_batch_host(hA, hl, hr, ho, variant=vcode[f], k=k, k_con=k_con, **xo[f])
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for f in forms:
                rmq.rmq_batch_host(hA, hl, hr, ho, variant=vcode[f], k=k, k_con=k_con, **xo[f])
        dt = dist.max(time.perf_counter() - t0)
        e2e = {"value": dist.world * units * args.e2e_steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": len(forms) * (4 * n + 8 * q),
               "d2h_bytes_per_step": len(forms) * 4 * q,
               "ms_per_step": 1e3 * dt / args.e2e_steps, "buffers": "pinned host"}
        del pA, pl, pr, pout

    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(A, l, r, args.cpu_seconds)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": workload_name(n, q, args.array), "n": n, "q": q, "seed": args.seed,
                   "forms": forms, "k": k, "k_con": k_con, "tuned_options": xo,
                   "k_autotuned": {"range": [32, 4096], "best_ms": tune_ms},
                   "l2": "flushed before each form (outside the timed events) by a 256 MiB write, then a 256 MiB "
                         "read of another buffer (the write's dirty lines leave L2 before the form); "
                         "A alone (%.0f MB) exceeds L2" % (4 * n / 1e6),
                   "parallelism": "replicas" if dist.world > 1 else "single GPU"},
        "forms": {f: {"ms": form_ms[f], "queries_per_s": q / (form_ms[f] * 1e-3),
                      "stages_ms": stages[f], "staged_call_ms": staged_ms[f],
                      **({"mark_clear_ms": clear_ms} if f == "contracted" else {}),
                      "open_query_work": counts[f]} for f in forms},
        "hbm_plain": hbm_plain,
        "hbm_contracted": hbm_con,
        "memory": {f: {"workspace_bytes": ws_bytes[f], "pct_of_4n": 100.0 * ws_bytes[f] / (4 * n)}
                   for f in forms},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "wall_s_timed_region": t_wall,
    }
    del dA, dl, dr, outs, flush, flush_rd
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return line


# ----------------------------------------------------------------- config 1

def run_config1(args, rmq, torch, np, dev):
    """A int32 n = 1e6 uniform in [0, 2^31), q = 1e3 uniform queries: a
    launch-latency-bound call.  Both forms autotuned; the best one is timed
    per call (events around one rmq_batch_ex, L2 flushed before each) and as
    one call replayed from a CUDA graph."""
    import oracle
    n, q = 1_000_000, 1000
    A = W().uniform_array(n, 1001)
    l, r = W().uniform_queries(n, q, 1002)
    dA = torch.from_numpy(A).to(dev)
    dl, dr = torch.from_numpy(l).to(dev), torch.from_numpy(r).to(dev)
    out = torch.empty(q, dtype=torch.int32, device=dev)
    best, tune_ms = rmq.rmq_autotune(dA, dl, dr, out, variant=0, k_min=32, k_max=4096)
    opts = dict(variant=int(best["variant"]), k=best["k"], k_con=best["k_con"],
                threads_per_query=best["threads_per_query"], k1=best["k1"])
    rmq.rmq_batch_ex(dA, dl, dr, out, **opts)
    torch.cuda.synchronize()
    if rmq.rmq_stream_status() != rmq.Status.OK or not np.array_equal(out.cpu().numpy(), oracle.rmq_naive(A, l, r)):
        raise RuntimeError("config 1: answers differ from the oracle")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    flush_rd = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    s = torch.cuda.current_stream(dev)
    reps = 100
    direct = []
    for i in range(reps):
        flush_l2(flush, flush_rd, i)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        rmq.rmq_batch_ex(dA, dl, dr, out, **opts)
        e1.record(s)
        direct.append((e0, e1))
    # the same call captured once and replayed
    gs = torch.cuda.Stream(dev)
    with torch.cuda.stream(gs):
        rmq.rmq_batch_ex(dA, dl, dr, out, stream=gs.cuda_stream, **opts)    # pool warm on this stream
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=gs):
        rmq.rmq_batch_ex(dA, dl, dr, out, stream=gs.cuda_stream, **opts)
    replay = []
    with torch.cuda.stream(gs):
        for i in range(reps):
            flush_l2(flush, flush_rd, i)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(gs)
            g.replay()
            e1.record(gs)
            replay.append((e0, e1))
    # host-side latency of one synchronous call (enqueue, run, wait)
    host = []
    for i in range(reps):
        t0 = time.perf_counter()
        rmq.rmq_batch_ex(dA, dl, dr, out, **opts)
        torch.cuda.current_stream(dev).synchronize()
        host.append(time.perf_counter() - t0)
    torch.cuda.synchronize()
    d_ms = statistics.median(a.elapsed_time(b) for a, b in direct)
    g_ms = statistics.median(a.elapsed_time(b) for a, b in replay)
    if not np.array_equal(out.cpu().numpy(), oracle.rmq_naive(A, l, r)):
        raise RuntimeError("config 1: graph replay answers differ from the oracle")
    return {"workload": "plain RMQ: A int32 n=1e6 uniform in [0,2^31), q=1000 uniform queries (l<=r)",
            "choice": {"variant": best["variant"].name, "k": best["k"], "k_con": best["k_con"],
                       "threads_per_query": best["threads_per_query"], "k1": best["k1"],
                       "autotune_best_ms": tune_ms},
            "call_ms_median": d_ms, "queries_per_s": q / (d_ms * 1e-3),
            "graph_replay_ms_median": g_ms, "graph_queries_per_s": q / (g_ms * 1e-3),
            "host_sync_call_ms_median": 1e3 * statistics.median(host),
            "l2": "flushed before every timed call", "calls": reps,
            "oracle": "naive oracle on all 1000 queries: identical"}


# ----------------------------------------------------------------- config 3

def run_config3(args, rmq, torch, np, dev, peak):
    """A int32 n = 1e8 values uniform in [0, 1000) (many ties), q = 1e7
    queries of width log-uniform in [1, 1e4], l uniform: edge scans and the
    leftmost tie-break dominate.  Both forms autotuned over 32..4096; each
    form's best is timed (L2 flushed before each call) and its open-query work
    counted, so that the edge-scan bytes enter its HBM fraction."""
    import oracle
    n, q = 100_000_000, 10_000_000
    A = W().uniform_array(n, 1003, 0, 1000)
    l, r = W().log_width_queries(n, q, 1004, 1, 10_000)
    dA = torch.from_numpy(A).to(dev)
    dl, dr = torch.from_numpy(l).to(dev), torch.from_numpy(r).to(dev)
    out = torch.empty(q, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    flush_rd = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    s = torch.cuda.current_stream(dev)
    res = {}
    idx = np.random.default_rng(6).choice(q, size=4000, replace=False)
    want = oracle.rmq_naive(A, l[idx], r[idx])
    m = distinct_endpoints(n, l, r)
    for form, v in (("plain", 1), ("contracted", 2)):
        best, tms = rmq.rmq_autotune(dA, dl, dr, out, variant=v, k_min=32, k_max=4096)
        opts = dict(variant=v, k=best["k"], k_con=best["k_con"], threads_per_query=best["threads_per_query"],
                    k1=best["k1"])
        times = []
        for i in range(max(5, min(args.steps, 10))):
            flush_l2(flush, flush_rd, i)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            rmq.rmq_batch_ex(dA, dl, dr, out, **opts)
            e1.record(s)
            times.append((e0, e1))
        torch.cuda.synchronize()
        ms = statistics.median(a.elapsed_time(b) for a, b in times)
        if not np.array_equal(out.cpu().numpy()[idx], want):
            raise RuntimeError("config 3, %s form: answers differ from the oracle" % form)
        cnt = rmq.rmq_batch_counted(dA, dl, dr, out, **opts)
        k = best["k"] if form == "plain" else 1024
        k_con = best["k_con"] if form == "contracted" else 256
        sb, hbm_b, con_min_b, geo = form_bytes(n, q, k, k_con, m, {form: cnt}, best["k1"] if form == "plain" else 0)
        b = hbm_b + 8 * cnt["m1_reads"] if form == "plain" else con_min_b + 8 * cnt["scan_elems"] + 4 * cnt["rank_reads"]
        gbs = b / (ms * 1e-3) / 1e9
        res[form] = {"k": best["k"] if form == "plain" else best["k_con"], "ms": ms,
                     "threads_per_query": best["threads_per_query"], "k1": best["k1"] if form == "plain" else None,
                     "queries_per_s": q / (ms * 1e-3), "open_query_work": cnt,
                     "algorithmic_bytes": b, "gbs": gbs, "frac_of_measured": gbs / peak}
    bestf = min(res, key=lambda f: res[f]["ms"])
    return {"workload": "tie-heavy and short ranges: A int32 n=1e8 values uniform in [0,1000), q=1e7 queries "
                        "of width log-uniform in [1,1e4], l uniform",
            "best_form": bestf, "queries_per_s": res[bestf]["queries_per_s"], "forms": res,
            "bytes": "plain: 4n + 8 nb (lc+1) + 8 ceil(n/k1) + 12q + 4S + 8 M (S cells scanned, M small-block minima "
                     "read); contracted: the "
                     "measurement model's B_min + 8S (S keys of A_Q scanned) + the rank reads of open queries",
            "l2": "flushed before every timed call", "oracle": "naive oracle on 4000 sampled queries: identical"}


def W():
    from paper_1706_06940_gb300 import workloads
    return workloads


# ----------------------------------------------------------------- config 2, the other batch sizes

def run_qsweep(args, rmq, torch, np, dev, peak):
    """Config 2 at the batch sizes below the headline's (n = 1e8 uniform,
    q = 1e2 .. 1e6, the scan-bound cases): both forms autotuned over
    32..4096 for each q, each call timed with L2 flushed before it, the plain
    form's HBM fraction on its algorithmic bytes 4n + 8 nb (lc+1) + 8 ceil(n/k1)
    + 12q + 4S (S counted by the instrumented query kernel)."""
    import oracle
    n = 100_000_000
    A = W().uniform_array(n, 1009)
    dA = torch.from_numpy(A).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    flush_rd = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    s = torch.cuda.current_stream(dev)
    steps = max(5, min(args.steps, 10))
    rows = []
    for q in (100, 1_000, 10_000, 100_000, 1_000_000):
        l, r = W().uniform_queries(n, q, 1010 + q)
        dl, dr = torch.from_numpy(l).to(dev), torch.from_numpy(r).to(dev)
        out = torch.empty(q, dtype=torch.int32, device=dev)
        idx = np.random.default_rng(7).choice(q, size=min(q, 48), replace=False)
        want = oracle.rmq_naive(A, l[idx], r[idx])
        row = {"q": q}
        m = distinct_endpoints(n, l, r)
        for form, v in (("plain", 1), ("contracted", 2)):
            best, _ = rmq.rmq_autotune(dA, dl, dr, out, variant=v, k_min=32, k_max=4096)
            opts = dict(variant=v, k=best["k"], k_con=best["k_con"], threads_per_query=best["threads_per_query"])
            if form == "plain":
                opts["k1"] = best["k1"]
            ms = time_calls(torch, s, flush, flush_rd, steps, lambda: rmq.rmq_batch_ex(dA, dl, dr, out, **opts))
            if rmq.rmq_stream_status() != rmq.Status.OK or not np.array_equal(out.cpu().numpy()[idx], want):
                raise RuntimeError("config 2 sweep, q=%d, %s form: answers differ from the oracle" % (q, form))
            entry = {"ms": ms, "k": best["k"] if form == "plain" else best["k_con"]}
            if form == "plain":
                cnt = rmq.rmq_batch_counted(dA, dl, dr, out, **opts)
                _, hbm_b, _, _ = form_bytes(n, q, best["k"], 256, m, {"plain": cnt}, best["k1"])
                entry.update({"k1": best["k1"], "algorithmic_bytes": hbm_b, "S_cells": cnt["scan_elems"],
                              "frac_of_measured": hbm_b / (ms * 1e-3) / 1e9 / peak})
            row[form] = entry
        row["queries_per_s_both_forms"] = 2 * q / ((row["plain"]["ms"] + row["contracted"]["ms"]) * 1e-3)
        rows.append(row)
        del dl, dr, out
    return {"workload": "config 2 at q = 1e2 .. 1e6: A int32 n=1e8 uniform in [0,2^31), l,r uniform",
            "rows": rows, "l2": "flushed before every timed call",
            "oracle": "naive oracle on 48 sampled queries per q and form: identical"}


# ----------------------------------------------------------------- multi-level layout (Sec. 3.3)

def time_calls(torch, s, flush, flush_rd, steps, fn):
    """Median CUDA-event time (ms) of fn() over steps calls, L2 flushed before each."""
    times = []
    for i in range(steps):
        flush_l2(flush, flush_rd, i)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        fn()
        e1.record(s)
        times.append((e0, e1))
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in times)


def run_hlevel(args, rmq, torch, np, dev, peak):
    """The multi-level layout of Sec. 3.3 beside the one-level plain form on the
    n = 1e8, q = 1e7 workloads (uniform ranges over uniform values, and short
    ranges over tie-heavy values): per call time with L2 flushed, queries/s,
    the structure's bytes next to the one-level table's, and the fraction of
    measured HBM of the lower bound 4n + 8E + 12q (A read once, E structure
    entries written, l, r read and out written; end-part reads not counted).
    Block sizes: Sec. 3.3's choice for h = 2 and h = 3, and two smaller
    first levels.  Every answer equals the plain form's, and a sample the
    naive oracle's."""
    import oracle
    n, q = 100_000_000, 10_000_000
    ks_list = [rmq.rmq_hlevel_paper_ks(n, 2), rmq.rmq_hlevel_paper_ks(n, 3), (128, 1024), (128, 1024, 16384)]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    flush_rd = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    s = torch.cuda.current_stream(dev)
    steps = max(5, min(args.steps, 10))
    res = {}
    for name in ("uniform", "tie_heavy_short"):
        if name == "uniform":
            A = W().uniform_array(n, 1005)
            l, r = W().uniform_queries(n, q, 1006)
        else:
            A = W().uniform_array(n, 1007, 0, 1000)
            l, r = W().log_width_queries(n, q, 1008, 1, 10_000)
        dA = torch.from_numpy(A).to(dev)
        dl, dr = torch.from_numpy(l).to(dev), torch.from_numpy(r).to(dev)
        ref = torch.empty(q, dtype=torch.int32, device=dev)
        out = torch.empty(q, dtype=torch.int32, device=dev)
        idx = np.random.default_rng(9).choice(q, size=2000, replace=False)
        want = oracle.rmq_naive(A, l[idx], r[idx])
        best, _ = rmq.rmq_autotune(dA, dl, dr, ref, variant=1, k_min=32, k_max=4096)
        popts = dict(variant=1, k=best["k"], threads_per_query=best["threads_per_query"], k1=best["k1"])
        ms_p = time_calls(torch, s, flush, flush_rd, steps, lambda: rmq.rmq_batch_ex(dA, dl, dr, ref, **popts))
        if not np.array_equal(ref.cpu().numpy()[idx], want):
            raise RuntimeError("multi-level leg, %s: plain answers differ from the oracle" % name)
        row = {"plain": {"k": best["k"], "k1": best["k1"], "ms": ms_p, "queries_per_s": q / (ms_p * 1e-3),
                         "one_level_table_bytes": rmq.rmq_table_bytes(n, best["k"]),
                         "workspace_bytes": rmq.rmq_batch_workspace_bytes(n, q, **popts)}, "hlevel": []}
        for ks in ks_list:
            ms = time_calls(torch, s, flush, flush_rd, steps, lambda: rmq.rmq_batch_hlevel(dA, dl, dr, out, ks))
            if rmq.rmq_stream_status() != rmq.Status.OK or not torch.equal(out, ref):
                raise RuntimeError("multi-level leg, %s, ks=%s: answers differ from the plain form" % (name, ks))
            nbytes = rmq.rmq_hlevel_bytes(n, ks)
            lb = 4 * n + nbytes + 12 * q
            gbs = lb / (ms * 1e-3) / 1e9
            row["hlevel"].append({"ks": list(ks), "h": len(ks), "ms": ms, "queries_per_s": q / (ms * 1e-3),
                                  "structure_bytes": nbytes,
                                  "structure_vs_one_level_table": nbytes / rmq.rmq_table_bytes(n, best["k"]),
                                  "lower_bound_bytes": lb, "gbs": gbs, "frac_of_measured": gbs / peak})
        res[name] = row
        del dA, dl, dr, ref, out
        torch.cuda.empty_cache()
    return {"workload": "n=1e8 int32, q=1e7: uniform values with l,r uniform; and values uniform in [0,1000) with "
                        "width log-uniform in [1,1e4]",
            "paper_ks": {"h2": list(ks_list[0]), "h3": list(ks_list[1])}, "cases": res,
            "l2": "flushed before every timed call",
            "checks": "every answer equal to the plain form's; 2000 sampled answers equal to the naive oracle's"}


# ----------------------------------------------------------------- config 4

def run_config4(args, rmq, torch, np, dev, peak, seed):
    """512 arrays, n log-uniform in [1e4, 1e7] (uniform int32 values), q
    log-uniform in [10, 1e5] uniform queries each: one persistent launch
    (rmq_batch_multi, replayed from a CUDA graph) against one rmq_batch call
    per array on the same stream."""
    import oracle
    ns, qs = W().uneven_batch(args.arrays, seed)
    # the arrays are views of one device buffer (each starting on a 16-byte
    # boundary), as a ragged batch is usually held
    starts = np.concatenate([[0], np.cumsum((ns.astype(np.int64) + 3) // 4 * 4)])
    big = torch.empty(int(starts[-1]), dtype=torch.int32, device=dev)
    dA, ls, rs = [], [], []
    for h, (n, q) in enumerate(zip(ns, qs)):
        a = big[int(starts[h]):int(starts[h]) + int(n)]
        a.copy_(torch.from_numpy(W().uniform_array(int(n), seed + 17 * h)))
        dA.append(a)
        l, r = W().uniform_queries(int(n), int(q), seed + 17 * h + 1)
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
        for _ in range(3):
            g.replay()
            seq_calls()
    torch.cuda.synchronize()
    if rmq.rmq_stream_status(s.cuda_stream) != rmq.Status.OK:
        raise RuntimeError("config 4: device status after warm-up")
    if not torch.equal(out, out_seq):
        raise RuntimeError("config 4: the multi-array launch and the per-array calls disagree")
    for h in np.random.default_rng(3).choice(len(dA), 8, replace=False):
        a, b = int(offs[h]), int(offs[h + 1])
        if b > a:
            idx = np.random.default_rng(int(h)).choice(b - a, min(32, b - a), replace=False)
            want = oracle.rmq_naive(dA[h].cpu().numpy(), ls[h][idx], rs[h][idx])
            if not np.array_equal(out[a:b].cpu().numpy()[idx], want):
                raise RuntimeError("config 4: multi-array answers differ from the oracle on array %d" % h)
    steps = max(5, min(args.steps, 20))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(s):
        for e0, e1 in ev:
            e0.record(s)
            g.replay()
            e1.record(s)
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
    with torch.cuda.stream(s):
        for e0, e1 in ev2:
            e0.record(s)
            seq_calls()
            e1.record(s)
    torch.cuda.synchronize()
    ms_multi = statistics.median(e0.elapsed_time(e1) for e0, e1 in ev)
    ms_seq = statistics.median(e0.elapsed_time(e1) for e0, e1 in ev2)
    nbytes = sum(4 * int(n) for n, q in zip(ns, qs) if q > 0) + 12 * qtot
    gbs = nbytes / (ms_multi * 1e-3) / 1e9
    return {"workload": "batched uneven: %d int32 arrays, n log-uniform in [1e4,1e7] (sum %d), q log-uniform in "
                        "[10,1e5] (sum %d), uniform values and queries; one persistent launch replayed from a CUDA "
                        "graph" % (len(dA), int(ns.sum()), qtot),
            "layout": "the arrays are views of one device buffer, each 16-byte aligned",
            "ms": ms_multi, "queries_per_s": qtot / (ms_multi * 1e-3), "kernels_per_replay": kernels_per_replay,
            "per_array_calls": {"ms": ms_seq, "queries_per_s": qtot / (ms_seq * 1e-3),
                                "speedup_of_one_launch": ms_seq / ms_multi},
            "hbm": {"algorithmic_bytes": nbytes, "terms": "4 sum(n) + 12 sum(q)", "gbs": gbs,
                    "frac_of_measured": gbs / peak},
            "l2": "inputs (%.1f GB) exceed L2; graph replays back to back" % (4e-9 * ns.sum()),
            "oracle": "naive oracle on 32 queries of 8 sampled arrays: identical; all answers equal the "
                      "per-array calls'"}


# ----------------------------------------------------------------- config 5

def run_config5(args, rmq, torch, np, dev, seed):
    """64 resident arrays totalling 4e9 cells (n log-uniform in [1e6, 2e8],
    rescaled), admitted into the library's server by a memory budget.
    Requests: a random array, a batch log-uniform in [1, 1e5] of uniform
    queries, in pinned host buffers shared by both arms.

    * capacity (closed loop): client threads each submit a request and wait
      for it before the next, over the whole request pool; the server
      (continuous batching over several streams) against the plain path, one
      rmq_query_host call per request on one stream, one request at a time.
    * open loop: Poisson arrivals at the configuration's 1e4 requests/s and
      at higher rates; latency is arrival to answers in the host buffer.
    """
    import oracle
    sizes = W().served_array_sizes(64, 4_000_000_000, seed)
    gen = torch.Generator(device=dev)
    dA = []
    for h, n in enumerate(sizes):
        gen.manual_seed(seed + 31 * h)
        dA.append(torch.randint(0, 2**31 - 1, (int(n),), dtype=torch.int32, device=dev, generator=gen))
    torch.cuda.synchronize()                    # the arrays are written before the server reads them
    free0, _ = torch.cuda.mem_get_info(dev)
    budget = int(free0 * 0.8)
    srv = rmq.Server(budget_bytes=budget, inflight=4)
    t_adm = time.perf_counter()
    ids = [srv.admit(A) for A in dA]
    t_adm = time.perf_counter() - t_adm
    adm = srv.stats()
    handles = [rmq.rmq_build(A) for A in dA]
    torch.cuda.synchronize()
    g = np.random.default_rng(seed + 1)
    R = args.served_requests
    arr = g.integers(0, len(dA), R)
    qs = W().log_uniform_ints(g, R, 1, 1e5)
    offs = np.concatenate([[0], np.cumsum(qs)])
    qtot = int(offs[-1])
    pin = lambda: torch.empty(qtot, dtype=torch.int32).pin_memory().numpy()
    Lp, Rp, Os, Op = pin(), pin(), pin(), pin()
    for i in range(R):
        n = int(sizes[arr[i]])
        a = g.integers(0, n, int(qs[i]), dtype=np.int64)
        b = g.integers(0, n, int(qs[i]), dtype=np.int64)
        Lp[offs[i]:offs[i + 1]] = np.minimum(a, b)
        Rp[offs[i]:offs[i + 1]] = np.maximum(a, b)
    req = [(int(arr[i]), slice(int(offs[i]), int(offs[i + 1]))) for i in range(R)]

    def served_closed(nreq, clients):
        lat = np.zeros(nreq)

        def client(c):
            for i in range(c, nreq, clients):
                h, sl = req[i]
                t = srv.submit(ids[h], Lp[sl], Rp[sl], Os[sl])
                lat[i] = srv.wait(t)

        th = [threading.Thread(target=client, args=(c,)) for c in range(clients)]
        t0 = time.perf_counter()
        for t in th:
            t.start()
        for t in th:
            t.join()
        return time.perf_counter() - t0, lat

    def percall_closed(nreq):
        lat = np.zeros(nreq)
        t0 = time.perf_counter()
        for i in range(nreq):
            h, sl = req[i]
            t1 = time.perf_counter()
            rmq.rmq_query_host(handles[h], Lp[sl], Rp[sl], Op[sl])
            lat[i] = time.perf_counter() - t1
        return time.perf_counter() - t0, lat

    def served_open(rate, window):
        nreq = min(R, int(rate * window))
        arrive = np.cumsum(np.random.default_rng(seed + 2).exponential(1.0 / rate, nreq))
        tickets = [None] * nreq
        lag = np.zeros(nreq)
        lat = np.zeros(nreq)

        def waiter():
            for i in range(nreq):
                while tickets[i] is None:
                    time.sleep(20e-6)
                lat[i] = srv.wait(tickets[i]) + lag[i]

        th = threading.Thread(target=waiter)
        th.start()
        t0 = time.perf_counter()
        for i in range(nreq):
            while time.perf_counter() - t0 < arrive[i]:
                pass
            h, sl = req[i]
            lag[i] = time.perf_counter() - t0 - arrive[i]
            tickets[i] = srv.submit(ids[h], Lp[sl], Rp[sl], Os[sl])
        th.join()
        wall = time.perf_counter() - t0
        return nreq, int(offs[nreq]), wall, lat

    def percall_open(rate, window):
        nreq = min(R, int(rate * window))
        arrive = np.cumsum(np.random.default_rng(seed + 2).exponential(1.0 / rate, nreq))
        lat = np.zeros(nreq)
        t0 = time.perf_counter()
        for i in range(nreq):
            while time.perf_counter() - t0 < arrive[i]:
                pass
            h, sl = req[i]
            rmq.rmq_query_host(handles[h], Lp[sl], Rp[sl], Op[sl])
            lat[i] = time.perf_counter() - t0 - arrive[i]
        return nreq, int(offs[nreq]), time.perf_counter() - t0, lat

    pct = lambda a, p: float(np.percentile(a, p) * 1e3)
    # warm both paths (pools, staging), then the capacity arms over the whole pool
    served_closed(min(R, 200), args.served_clients)
    percall_closed(min(R, 50))
    wall_s, lat_s = served_closed(R, args.served_clients)
    wall_p, lat_p = percall_closed(R)
    if not np.array_equal(Os, Op):
        raise RuntimeError("config 5: served and per-call answers differ")
    for i in np.random.default_rng(seed + 3).choice(R, 16, replace=False):
        h, sl = req[i]
        idx = np.random.default_rng(int(i)).choice(sl.stop - sl.start, min(16, sl.stop - sl.start), replace=False)
        want = oracle.rmq_naive(dA[h].cpu().numpy(), Lp[sl][idx], Rp[sl][idx])
        if not np.array_equal(Os[sl][idx], want):
            raise RuntimeError("config 5: served answers differ from the oracle on request %d" % i)
    cap_s, cap_p = qtot / wall_s, qtot / wall_p
    open_arms = []
    for rate in (1e4, 3e4, 1e5):
        nr, nq, wall, lat = served_open(rate, args.served_window)
        nr2, nq2, wall2, lat2 = percall_open(rate, args.served_window)
        open_arms.append({"rate_req_per_s": rate, "requests": nr,
                          "served": {"queries_per_s": nq / wall, "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99)},
                          "one_request_per_call": {"queries_per_s": nq2 / wall2, "p50_ms": pct(lat2, 50),
                                                   "p99_ms": pct(lat2, 99)}})
    st = srv.stats()
    srv.close()
    for hd in handles:
        hd.free()
    del dA
    torch.cuda.empty_cache()
    return {"workload": "served: 64 resident int32 arrays totalling %d cells (n log-uniform in [1e6,2e8], "
                        "rescaled), requests on a random array with a batch log-uniform in [1,1e5] of uniform "
                        "queries (l<=r)" % int(sizes.sum()),
            "admission": {"budget_bytes": budget, "reserved_bytes": adm["table_bytes_in_use"],
                          "resident_arrays": adm["resident_arrays"], "admit_s": t_adm},
            "capacity": {"requests": R, "queries": qtot,
                         "served": {"clients": args.served_clients, "queries_per_s": cap_s,
                                    "requests_per_s": R / wall_s, "p50_ms": pct(lat_s, 50), "p99_ms": pct(lat_s, 99)},
                         "one_request_per_call": {"queries_per_s": cap_p, "requests_per_s": R / wall_p,
                                                  "p50_ms": pct(lat_p, 50), "p99_ms": pct(lat_p, 99)},
                         "served_over_per_call": cap_s / cap_p},
            "open_loop": open_arms, "batches": st["batches"],
            "oracle": "all answers of both arms identical; naive oracle on 16 queries of 16 sampled requests"}


# ----------------------------------------------------------------- reference arm

def run_reference(args, dist):
    """The CPU oracle on bounded samples of the headline batch, rank 0 only.
    Each step answers at least 16 queries per host thread, so that every
    thread has work (the oracle hands out one query at a time)."""
    if dist.rank != 0:
        return
    import numpy as np

    import oracle
    oracle.build()
    n, q = int(args.n), int(args.q)
    A, l, r = workload(n, q, args.seed, 0, args.array)
    threads = oracle.max_threads()
    per_step = max(0.2, min(2.0, 90.0 / max(args.steps + args.warmup, 1)))
    s = 4 * threads
    t0 = time.perf_counter()
    oracle.rmq_naive(A, l[:s], r[:s])
    rate = s / max(time.perf_counter() - t0, 1e-6)
    per = int(min(q, max(16 * threads, per_step * rate)))
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
                         "sample": "naive oracle, %d queries of the batch per step (at least 16 per thread), "
                                   "%d timed steps" % (per, len(times))},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- driver

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
    peak, _ = measured_peak_hbm()

    def guarded(name, fn, *a):
        t0 = time.perf_counter()
        try:
            res = fn(*a)
        except Exception as e:          # recorded in the line, which still prints
            res = {"error": "%s: %s" % (type(e).__name__, e)}
        res["bench_wall_s"] = time.perf_counter() - t0
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        return res

    if args.workload in ("all", "single"):
        line = run_main(args, dist, rmq, torch, np)
        if args.workload == "all":
            if dist.world == 1:
                line["config1"] = guarded("config1", run_config1, args, rmq, torch, np, dev)
                line["config3"] = guarded("config3", run_config3, args, rmq, torch, np, dev, peak)
                line["config4"] = guarded("config4", run_config4, args, rmq, torch, np, dev, peak, args.seed + 2)
                line["config5"] = guarded("config5", run_config5, args, rmq, torch, np, dev, args.seed + 3)
                line["config2_q_sweep"] = guarded("config2_q_sweep", run_qsweep, args, rmq, torch, np, dev, peak)
                line["hlevel"] = guarded("hlevel", run_hlevel, args, rmq, torch, np, dev, peak)
            else:
                line["other_configs"] = "configs 1, 3, 4 and 5 run at N = 1 only"
        if dist.rank == 0:
            print(json.dumps(line), flush=True)
        return
    fn = {"c1": lambda: run_config1(args, rmq, torch, np, dev),
          "c3": lambda: run_config3(args, rmq, torch, np, dev, peak),
          "multi": lambda: run_config4(args, rmq, torch, np, dev, peak, args.seed + 2),
          "served": lambda: run_config5(args, rmq, torch, np, dev, args.seed + 3),
          "hlevel": lambda: run_hlevel(args, rmq, torch, np, dev, peak),
          "qsweep": lambda: run_qsweep(args, rmq, torch, np, dev, peak)}[args.workload]
    res = fn()
    if dist.rank == 0:
        print(json.dumps({"workload_only": args.workload, **res}), flush=True)


def main():
    args = parse_args()
    dist = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        else:
            run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
