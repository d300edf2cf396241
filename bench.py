#!/usr/bin/env python3
"""Throughput of Slim Graph Triangle p-1-Reduction + CSR rebuild on GB300.

Workload (default): R-MAT scale 22, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05),
seed 1, symmetrised uint32 CSR with int64 offsets; one step = one
compress(G, edge-once TR, p = 0.5) -> H: degree-ordered orientation, triangle
enumeration with the edge-once reservation rounds, mask resolution and the
stream-compacted CSR rebuild.  Metric: input (undirected) edges per second.

The JSON line also carries: the roofline of the dominant kernel (measured live
with CUDA events on the library's stream), the end-to-end number through the
C-ABI with host buffers, the oracle timed on the host cores, SM clocks sampled
during the timed region, and per-row timings of the other kernels.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "rmat22": dict(scale=22, ef=16, desc="R-MAT scale 22, edge factor 16, (a,b,c)=(.57,.19,.19), seed 1"),
    "rmat26": dict(scale=26, ef=16, desc="R-MAT scale 26, edge factor 16, (a,b,c)=(.57,.19,.19), seed 1"),
    "rmat19": dict(scale=19, ef=16, desc="R-MAT scale 19, edge factor 16, (a,b,c)=(.57,.19,.19), seed 1"),
    "rmat20": dict(scale=20, ef=16, desc="R-MAT scale 20, edge factor 16, (a,b,c)=(.57,.19,.19), seed 1"),
    "rmat23": dict(scale=23, ef=16, desc="R-MAT scale 23, edge factor 16, (a,b,c)=(.57,.19,.19), seed 1"),
    "rmat24": dict(scale=24, ef=16, desc="R-MAT scale 24, edge factor 16, (a,b,c)=(.57,.19,.19), seed 1"),
    "rmat14": dict(scale=14, ef=16, desc="R-MAT scale 14, edge factor 16, (a,b,c)=(.57,.19,.19), seed 1"),
}
METRIC = "input edges/s compressed (TR + CSR rebuild)"
CPU_SAMPLE_SCALE = 16  # oracle sample: same generator, 64x fewer edges than scale 22


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the dominant kernel, from one ncu capture of this benchmark's own command
# (the summaries under profiles/ give the command).  Each entry records the
# digest of the enumeration sources it was taken on; once they change, the
# figure no longer describes the kernel and the JSON line reports null.
MEASURED_TRAFFIC = {
    # (workload, kernel): (bytes per launch, sha256 of the enumeration sources)
    # profiles/tri_enum_rmat22_tr_eo.md: 37.92 GB read + 18.83 GB written
    ("rmat22", "tr_eo"): (56742775000, "94d004d8e9f7af0cd065222fa68884b845cbe2e00ca03967c9c33ca361122db6"),
    # profiles/tri_enum_rmat26_tr_random.md: hub launch 1417.64 + 144.65 GB, main launch
    # 513.55 + 12.06 GB (read + written) per union pass
    ("rmat26", "tr_random"): (2087900042000, "94d004d8e9f7af0cd065222fa68884b845cbe2e00ca03967c9c33ca361122db6"),
}
TRAFFIC_SOURCES = ("paper_1912_08950_gb300/csrc/sg_triangles.cu", "paper_1912_08950_gb300/csrc/sg_internal.cuh")


def sources_digest() -> str:
    import hashlib

    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(workload: str, kernel: str):
    entry = MEASURED_TRAFFIC.get((workload, kernel))
    if entry is None or entry[1] != sources_digest():
        return None
    return entry[0]


# ------------------------------------------------------------ replicas
# N > 1: one independent replica per GPU (the path has no exchange step).
# Rank r compresses its own graph (seed 1 + r; rank 0 is the named
# workload), the step time is the maximum over ranks, and the whole-job
# throughput counts every rank's edges.
def replica_seed(rank: int) -> int:
    return 1 + rank


def max_over_ranks(x: float, dist=None, device: str = "cpu") -> float:
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, m_per_rank: int, seconds: float) -> float:
    return world * m_per_rank / seconds


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in self.rows if num(r[1])]
        mx = [num(r[2]) for r in self.rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def step_stats(samples):
    """Median, extremes and a 95% percentile-bootstrap interval of the mean of
    per-step times (fixed resampling seed)."""
    import numpy as np

    x = np.asarray(samples, dtype=np.float64)
    rng = np.random.default_rng(12345)
    means = x[rng.integers(0, x.size, size=(2000, x.size))].mean(axis=1)
    return {"median": float(np.median(x)), "min": float(x.min()), "max": float(x.max()),
            "ci95_mean": [float(np.percentile(means, 2.5)), float(np.percentile(means, 97.5))], "n": int(x.size)}


def byte_model(n, m, A_out, probes_total, launches, kernel, head_arcs=0, listed_total=0):
    """Algorithmic bytes of one launch of a named kernel."""
    A = 2 * m
    if kernel == "tri_enum":
        # off+ and the in-list length of every vertex (8 + 4 B), N+(x) staged in
        # the tables (4 B/arc), the off+ pair of every streamed list (8 B/arc),
        # the in-list records (8 B per arc streamed from the head's side), one
        # 4-byte read per probe (W = sum over arcs of min(d+(u), d+(v))) and,
        # for edge-once, the 16-byte record of every listed triangle
        per = max(launches, 1)
        return (8 * (n + 1) + 4 * n + 4 * m + 8 * m + 8 * head_arcs) + (4.0 * probes_total + 16.0 * listed_total) / per
    if kernel == "tri_enum_forward":
        # the enumeration's terms of the listing's byte model: E+ read once
        # (off+ and N+), one 4-byte read per probe of the plain forward algorithm
        # (W+ = sum over arcs u->v of d+(v); probes_total holds W+ scaled to the
        # arcs the passes actually streamed) and, for edge-once, the 16-byte
        # record of every listed triangle
        per = max(launches, 1)
        return (8 * (n + 1) + 4 * m) + (4.0 * probes_total + 16.0 * listed_total) / per
    if kernel == "tri_inarcs":
        # off+ and N+(u) of every vertex, the off+ pair and symmetric offsets of
        # every head, one 8-byte record written per gathered arc
        return 8 * (n + 1) + 4 * m + 8 * m + 16 * head_arcs + 8 * head_arcs
    if kernel == "compact_orient":
        return 8 * (n + 1) + 4 * A + 4 * A + 8 * (n + 1) + 4 * m + A / 8
    if kernel == "compact_trmask":
        return 8 * (n + 1) + 4 * A + A / 8 + 4 * m + A + 8 * (n + 1) + 4 * A_out
    return None


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import graphgen as gg
    import paper_1912_08950_gb300 as sg

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = WORKLOADS[args.workload]
    seed = replica_seed(rank)
    g = gg.rmat(wl["scale"], wl["ef"], seed=seed, device="cuda")
    torch.cuda.synchronize()
    # the library runs on this stream; every timing event is recorded on it
    stream = torch.cuda.Stream(local)
    ctx = sg.Context(local, stream=stream)
    G = sg.Graph.from_csr(ctx, g, copy=True)
    torch.cuda.empty_cache()  # hand the generator's scratch back before the library sizes its lists
    ctx.set_eo_list_capacity(args.eo_list_cap)
    n, m = G.n, G.m
    work = sg.tr_work(G)

    def step():
        H = sg.compress(G, args.kernel, args.p, 1)
        a = H.nnz
        H.free()
        return a

    for _ in range(args.warmup):
        A_out = step()
    ctx.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    ctx.stats(reset=True)
    ctx.reset_profile()
    ctx.set_profiling(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    time.sleep(0.3)
    barrier()
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev0.record(stream)
    marks[0].record(stream)
    for i in range(args.steps):
        A_out = step()
        marks[i + 1].record(stream)
    ev1.record(stream)
    barrier()
    clocks.stop()
    ctx.set_profiling(False)
    ms = ev0.elapsed_time(ev1) / args.steps
    step_ms = step_stats([marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps)])
    st = ctx.stats()
    kt = {}
    for name in ("tri_enum", "tri_hubs", "tri_inarcs", "tri_eo_fresh_reserve", "tri_eo_list_reserve", "tri_eo_list_accept",
                 "tri_eo_accept", "tri_eo_list_reset", "tri_classify", "compact_orient", "compact_trmask", "row_maps"):
        kt[name] = ctx.kernel_time(name)
    # one enumeration pass = the hub launch (vertices with long out-lists, when
    # there are any) + the main launch; the pass is the roofline's unit
    enum_ms = kt["tri_enum"][0] + kt["tri_hubs"][0]
    enum_launches = max(kt["tri_enum"][1], 1)
    ms = max_over_ranks(ms, dist, "cuda")

    hbm, peak_src = peaks()
    cand = {
        "tri_enum": (enum_ms, enum_launches, byte_model(n, m, A_out, st["probes"], enum_launches, "tri_enum",
                                                        work["head_arcs"], st["eo_listed"])),
        "compact_orient": (kt["compact_orient"][0], kt["compact_orient"][1],
                           byte_model(n, m, A_out, 0, 1, "compact_orient")),
        "compact_trmask": (kt["compact_trmask"][0], kt["compact_trmask"][1],
                           byte_model(n, m, A_out, 0, 1, "compact_trmask")),
    }
    # the listing's byte model counts the plain forward algorithm's probes W+;
    # the passes stream the shorter list of each arc instead (W probes), so W+
    # is scaled by the share of W they streamed (later edge-once passes skip
    # considered arcs)
    fwd_total = work["forward_probes"] * st["probes"] / max(work["probes"], 1)
    enum_fwd_bytes = byte_model(n, m, A_out, fwd_total, enum_launches, "tri_enum_forward", 0, st["eo_listed"])
    dom = max(cand, key=lambda k: cand[k][0])
    d_ms, d_launch, d_bytes = cand[dom]
    per_launch_s = d_ms / max(d_launch, 1) / 1e3
    streamed = None
    if dom == "tri_enum":
        streamed = {"algorithmic_bytes_per_launch": d_bytes,
                    "achieved": d_bytes / per_launch_s / 1e9 if per_launch_s > 0 else None}
        d_bytes = enum_fwd_bytes
    achieved = d_bytes / per_launch_s / 1e9 if per_launch_s > 0 else None

    # other rows of the hot path, timed once each (not part of the metric)
    rows = {}
    row_kernels = (("uniform", 0.5), ("spectral_avgdeg", 0.5), ("tr_random", 0.5), ("tr_p2", 0.5),
                   ("tr_mincount", 0.5), ("tr_eo_mincount", 0.5))
    if args.no_rows:
        row_kernels = ()
    for kern, p in row_kernels:
        for _ in range(2):
            sg.compress(G, kern, p, 1).free()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            sg.compress(G, kern, p, 1).free()
        e1.record(stream)
        torch.cuda.synchronize()
        rows[kern] = {"ms": e0.elapsed_time(e1) / 3, "edges_per_s": m / (e0.elapsed_time(e1) / 3e3)}
    if not args.no_rows:
        # the enumeration alone (triangle counting, no decisions) for comparison
        ctx.reset_profile()
        ctx.set_profiling(True)
        sg.tr_work(G)
        ctx.set_profiling(False)
        rows["enum_count_only"] = {"ms": ctx.kernel_time("tri_enum")[0] + ctx.kernel_time("tri_hubs")[0],
                                   "probes": work["probes"],
                                   "triangles": work["triangles"]}
        H = sg.compress(G, args.kernel, args.p, 1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        div = sg.divergence(G, H)
        e1.record(stream)
        torch.cuda.synchronize()
        rows["divergence"] = {"ms": e0.elapsed_time(e1), "kl_bits": div["kl_bits"], "cc_g": div["cc_g"],
                              "cc_h": div["cc_h"]}
        e0.record(stream)
        acc = sg.accuracy(G, H)
        e1.record(stream)
        torch.cuda.synchronize()
        rows["accuracy"] = {"ms": e0.elapsed_time(e1), "pr_aren": acc["pr_aren"], "tc_aren": acc["tc_aren"],
                            "critical_fraction": acc["critical_fraction"], "root": acc["root"]}
        H.free()
        for _ in range(2):
            sg.low_degree(G).free()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            L0 = sg.low_degree(G)
            kept_n = L0.n
            L0.free()
        e1.record(stream)
        torch.cuda.synchronize()
        rows["low_degree"] = {"ms": e0.elapsed_time(e1) / 3, "kept_vertices": kept_n,
                              "edges_per_s": m / (e0.elapsed_time(e1) / 3e3)}

    # end to end through the C-ABI with pinned host buffers
    off_h = g.off.cpu().pin_memory()
    col_h = g.col.cpu().pin_memory()
    out_off = torch.empty(n + 1, dtype=torch.int64).pin_memory()
    out_col = torch.empty(max(2 * m, 1), dtype=torch.int32).pin_memory()
    L = sg.lib()
    import ctypes

    def e2e_step():
        h = ctypes.c_void_p()
        sg._check(L.sg_graph_from_host(ctx.handle, n, 2 * m, off_h.data_ptr(), col_h.data_ptr(), None,
                                       ctypes.byref(h)))
        gi = sg.Graph(ctx, h)
        H = sg.compress(gi, args.kernel, args.p, 1)
        sg._check(L.sg_graph_download(ctx.handle, H.handle, out_off.data_ptr(), out_col.data_ptr(), None))
        nnz_out = H.nnz
        H.free()
        gi.free()
        return nnz_out

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(2, min(args.steps, 5))
    for _ in range(e2e_steps):
        nnz_out = e2e_step()
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")

    cpu_leg = rank == 0 and world == 1 and not args.no_cpu
    cpu = cpu_baseline(args) if cpu_leg else None
    cpu_cores = cpu_all_cores(args) if cpu_leg else None
    clk = clocks.summary()
    res = {
        "metric": METRIC,
        "value": replica_throughput(world, m, ms / 1e3),
        "unit": "edges/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "step_ms": step_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "kernel": args.kernel, "p": args.p, "n": n, "m": m,
                   "eo_list_capacity": args.eo_list_cap,
                   "arcs": 2 * m, "triangles": work["triangles"], "probes_per_pass": work["probes"],
                   "forward_probes": work["forward_probes"],
                   "head_arcs": work["head_arcs"],
                   "max_out_degree": work["max_out_degree"], "kept_arcs": int(A_out),
                   "l2": "inputs larger than L2 (CSR %.0f MB > 129 MB)" % ((8 * (n + 1) + 8 * m) / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if achieved else None,
                     "traffic": measured_traffic(args.workload, args.kernel) if dom == "tri_enum" else None,
                     "peak_source": peak_src, "algorithmic_bytes_per_launch": d_bytes,
                     "launch_ms": d_ms / max(d_launch, 1), "launches": d_launch,
                     "byte_model": ("forward listing: 8(n+1) + 4m + 4 W+ (+16 B per listed triangle)"
                                    if dom == "tri_enum" else dom),
                     "streamed": None if streamed is None else dict(
                         streamed, frac=(streamed["achieved"] / hbm) if streamed["achieved"] else None,
                         byte_model="probes made: 8(n+1) + 4n + 12m + 8H + 4 W (+16 B per listed triangle)")},
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in kt.items()},
        "eo_rounds_per_step": st["eo_rounds"] / args.steps,
        "eo_passes_per_step": st["eo_passes"] / args.steps,
        "eo_list_passes_per_step": st["eo_list_passes"] / args.steps,
        "gpu_launches": st["kernel_launches"],
        "clocks": clk,
        "e2e": {"value": replica_throughput(world, m, e2e_s), "unit": "edges/s",
                "h2d_bytes_per_step": 8 * (n + 1) + 8 * m,
                "d2h_bytes_per_step": 8 * (n + 1) + 4 * int(nnz_out)},
        "rows": rows,
        "cpu_baseline": cpu,
        "cpu_all_cores": cpu_cores,
    }
    if rank == 0:
        print(json.dumps(res), flush=True)
    G.free()
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def _digest(graphs, sync_stream):
    """Order-sensitive digest of many device CSRs, computed on the GPU."""
    import torch

    torch.cuda.current_stream().wait_stream(sync_stream)
    acc = torch.zeros((), dtype=torch.int64, device="cuda")
    for i, g in enumerate(graphs):
        off, col, _ = g.tensors()
        c = col.to(torch.int64)
        idx = torch.arange(c.numel(), device="cuda", dtype=torch.int64)
        acc = acc * 1000003 + (c * (idx * 2654435761 % 1000000007 + 1)).sum() + off.sum() * 31 + i
        acc = acc % (1 << 61)
    return int(acc.item())


def run_batch(args):
    """Batched compression of many R-MAT graphs vs the plain one-call-per-graph loop."""
    import numpy as np
    import torch

    import graphgen as gg
    import paper_1912_08950_gb300 as sg

    torch.cuda.set_device(0)
    G = args.batch_graphs
    rng = np.random.default_rng(7)
    scales = [int(round(8 + 8 * u)) for u in rng.random(G)]
    efs = [int(e) for e in rng.integers(8, 33, size=G)]
    seeds = [i + 1 for i in range(G)]
    ps = [float(x) for x in rng.choice([0.2, 0.5, 0.8], size=G)]
    kernels = [("uniform", "spectral_avgdeg", "tr_random")[i % 3] for i in range(G)]
    t0 = time.perf_counter()
    u, vbase, _ = gg.rmat_batch(scales, efs, seeds, device="cuda")
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    ctx = sg.Context(0, stream=stream)
    graphs = [sg.Graph.from_csr(ctx, gg.batch_member(u, vbase, i, 1 << scales[i]), copy=True) for i in range(G)]
    del u
    m_total = sum(g.m for g in graphs)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def plain():
        return [sg.compress(graphs[i], kernels[i], ps[i], seeds[i]) for i in range(G)]

    for _ in range(max(1, args.warmup // 2)):
        for h in plain():
            h.free()
    torch.cuda.synchronize()
    ctx.stats(reset=True)
    ev[0].record(stream)
    reps = max(1, args.steps // 2)
    for _ in range(reps):
        outs = plain()
        if _ < reps - 1:
            for h in outs:
                h.free()
    ev[1].record(stream)
    torch.cuda.synchronize()
    plain_ms = ev[0].elapsed_time(ev[1]) / reps
    plain_launches = ctx.stats(reset=True)["kernel_launches"] / reps
    d_plain = _digest(outs, stream)
    for h in outs:
        h.free()
    B = sg.Batch(ctx, graphs)
    t0 = time.perf_counter()
    outs_b = B.compress(kernels, ps, seeds)  # first call: autotune + capture
    tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        outs_b = B.compress(kernels, ps, seeds)
    torch.cuda.synchronize()
    ctx.stats(reset=True)
    ev[2].record(stream)
    for _ in range(args.steps):
        outs_b = B.compress(kernels, ps, seeds)
    ev[3].record(stream)
    torch.cuda.synchronize()
    batch_ms = ev[2].elapsed_time(ev[3]) / args.steps
    batch_launches = ctx.stats(reset=True)["kernel_launches"] / args.steps
    d_batch = _digest(outs_b, stream)
    info = B.info()
    print(json.dumps({
        "mode": "batch", "metric": METRIC + ", batched vs plain", "unit": "edges/s",
        "value": m_total / (batch_ms / 1e3), "plain_value": m_total / (plain_ms / 1e3),
        "speedup": plain_ms / batch_ms, "batch_ms": batch_ms, "plain_ms": plain_ms,
        "identical_outputs": d_plain == d_batch, "graphs": G, "m_total": m_total,
        "gpu_launches_per_call": {"batch": batch_launches, "plain": plain_launches},
        "autotune": info, "autotune_s": tune_s, "generation_s": gen_s, "steps": args.steps,
        "config": {"workload": f"{G} R-MAT graphs, scale round(8+8u) u~U[0,1), ef~U{{8..32}}, seed i+1, "
                               "p~U{0.2,0.5,0.8}, kernel round-robin uniform/spectral_avgdeg/tr_random"},
    }), flush=True)
    B.free()
    ctx.close()


def run_serve(args):
    """Continuous-batching serving of compress + divergence jobs with Poisson arrivals."""
    import numpy as np
    import torch

    import graphgen as gg
    from paper_1912_08950_gb300.serve import GpuExecutor, Job, Server, poisson_arrivals, replay

    rng = np.random.default_rng(5)
    pool = {}
    for s in range(args.serve_min_scale, args.serve_max_scale + 1):
        g = gg.rmat(s, 16, seed=s, device="cuda")
        off, col, _ = g.numpy()
        pool[s] = (g.n, np.ascontiguousarray(off), np.ascontiguousarray(col))
    kern = ["uniform", "spectral_avgdeg", "tr_random", "tr_eo"]

    def make_jobs(count, seed):
        r = np.random.default_rng(seed)
        jobs = []
        for i in range(count):
            s = int(r.integers(args.serve_min_scale, args.serve_max_scale + 1))
            n, off, col = pool[s]
            jobs.append(Job(n=n, off=off, col=col, kernel=kern[int(r.integers(0, 4))],
                            p=float(r.choice([0.2, 0.5, 0.8])), seed=i + 1))
        return jobs

    free, _ = torch.cuda.mem_get_info()
    budget = int(free * 0.6)
    slots = args.serve_slots
    res = {}
    for label, rate in (("offered", args.serve_rate), ("capacity70", None)):
        if rate is None:
            rate = 0.7 * res["offered"]["jobs_per_s"]
        srv = Server(lambda i: GpuExecutor(0), slots=slots, memory_budget=budget)
        jobs = make_jobs(args.serve_jobs, 11)
        out = replay(srv, jobs, poisson_arrivals(rate, len(jobs), seed=3))
        srv.close()
        out.pop("results")
        out["rate"] = rate
        res[label] = out
    print(json.dumps({"mode": "serve", "slots": slots, "memory_budget": budget, **res,
                      "config": {"workload": f"Poisson arrivals; jobs = compress + KL/CC on R-MAT scale "
                                             f"U{{{args.serve_min_scale}..{args.serve_max_scale}}} ef 16; "
                                             "kernels uniform/spectral_avgdeg/tr_random/tr_eo, p~U{0.2,0.5,0.8}"}}),
          flush=True)


def _oracle_sample(kernel, p):
    """One bounded oracle run: the same generator at scale 16 (a 64x smaller sample)."""
    import graphgen as gg
    import oracle

    g = gg.rmat(CPU_SAMPLE_SCALE, 16, seed=1)
    t0 = time.perf_counter()
    oracle.compress(g, kernel, p, 1)
    dt = time.perf_counter() - t0
    return g.m, dt


def cpu_baseline(args):
    m, dt = _oracle_sample(args.kernel, args.p)
    return {"value": m / dt, "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": f"R-MAT scale {CPU_SAMPLE_SCALE}, edge factor 16, seed 1 ({m} edges), "
                      f"{args.kernel} p={args.p}; single-threaded C oracle, {dt:.1f} s"}


def _oracle_job(job):
    """One oracle compress of a sample handed over as arrays (in a spawned worker)."""
    import oracle

    n, off, col, kernel, p, seed = job
    t0 = time.perf_counter()
    oracle.compress((n, off, col, None), kernel, p, seed)
    return time.perf_counter() - t0


def cpu_all_cores(args):
    """The same single-threaded oracle on every host core at once: one sample run
    per core, in spawned worker processes (the oracle itself is not changed)."""
    import multiprocessing as mp

    import numpy as np

    import graphgen as gg
    import oracle

    oracle.build()
    g = gg.rmat(CPU_SAMPLE_SCALE, 16, seed=1)
    off, col, _ = g.numpy()
    cores = os.cpu_count() or 1
    tiny = (2, np.array([0, 1, 2], dtype=np.int64), np.array([1, 0], dtype=np.uint32), args.kernel, args.p, 1)
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_job, [tiny] * cores, chunksize=1)  # workers up and the library loaded
        t0 = time.perf_counter()
        pool.map(_oracle_job, [(g.n, off, col, args.kernel, args.p, 1 + i) for i in range(cores)], chunksize=1)
        dt = time.perf_counter() - t0
    return {"value": cores * g.m / dt, "unit": "edges/s", "cores": cores, "kind": "oracle, one sample per core",
            "sample": f"{cores} runs of the R-MAT scale {CPU_SAMPLE_SCALE} sample ({g.m} edges each), "
                      f"{args.kernel} p={args.p}, seeds 1..{cores}, in {dt:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    for _ in range(args.warmup):
        _oracle_sample(args.kernel, args.p)
    tot_m, tot_s = 0, 0.0
    for _ in range(args.steps):
        m, dt = _oracle_sample(args.kernel, args.p)
        tot_m += m
        tot_s += dt
    v = tot_m / tot_s
    wl = WORKLOADS[args.workload]
    sample = (f"R-MAT scale {CPU_SAMPLE_SCALE}, edge factor 16, seed 1 per step, {args.kernel} p={args.p}; "
              "single-threaded C oracle")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": wl["desc"], "kernel": args.kernel, "p": args.p, "sample": sample},
        "cpu_baseline": {"value": v, "unit": "edges/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rmat22")
    ap.add_argument("--kernel", default="tr_eo")
    ap.add_argument("--p", type=float, default=0.5)
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-rows", action="store_true", help="skip the extra per-kernel rows and analytics")
    ap.add_argument("--eo-list-cap", type=int, default=0,
                    help="edge-once triangle list capacity in records (0: automatic, -1: none)")
    ap.add_argument("--mode", choices=["compress", "batch", "serve"], default="compress")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-jobs", type=int, default=300)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-min-scale", type=int, default=10)
    ap.add_argument("--serve-max-scale", type=int, default=22)
    args = ap.parse_args()
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
