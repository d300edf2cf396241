#!/usr/bin/env python3
"""Throughput of Slim Graph Triangle p-1-Reduction + CSR rebuild on GB300.

Headline workload (default): R-MAT scale 26, edge factor 16,
(a,b,c,d) = (.57,.19,.19,.05), seed 1, symmetrised uint32 CSR with int64
offsets; one step = one compress(G, Triangle p-1-Reduction with a random edge
per selected triangle, p = 0.5) -> H: degree-ordered orientation, triangle
enumeration with the decisions fused in, mask resolution and the
stream-compacted CSR rebuild.  Metric: input (undirected) edges per second.
The headline is timed with per-launch events off; a second, shorter timed
region with per-launch events on gives the per-kernel split and the roofline.

The JSON line also carries: the roofline of the dominant kernel (the triangle
enumeration pass, measured with CUDA events on the library's stream) and of
the whole step, both on the TR byte model (8(n+1) + 4m + 4 W+ for the
enumeration, W+ = sum over oriented arcs u->v of d+(v)); the end-to-end number
through the C-ABI with host buffers; the oracle timed on the host cores; SM
clocks sampled during the timed region; and rows for the other kernels and
workloads: Edge-Once TR on the same graph, the R-MAT scale-22 kernels and
analytics, a batch of 4096 graphs against the plain per-graph loop, and a
Poisson-arrival serving run.

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


def _rmat_desc(s):
    return f"R-MAT scale {s}, edge factor 16, (a,b,c)=(.57,.19,.19), seed 1"


WORKLOADS = {f"rmat{s}": dict(scale=s, ef=16, desc=_rmat_desc(s)) for s in (14, 19, 20, 22, 23, 24, 26)}
METRIC = "input edges/s compressed (TR + CSR rebuild)"
CPU_SAMPLE_SCALE = 16  # oracle sample: same generator, 1024x fewer edges than scale 26


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one enumeration
# pass, from an ncu capture.  Each entry records the digest of the enumeration
# sources it was taken on; once they change, the figure no longer describes
# the kernel and the JSON line reports null.
# (workload, kernel): (DRAM bytes per enumeration pass from one ncu capture,
# sha256 of the enumeration sources it was taken with).  An entry only counts
# while the sources are unchanged; otherwise the line reports traffic null.
# Counters beyond the launch duration are captured on small cases only, and
# the enumeration's traffic does not scale from them (small graphs re-read
# their lists from L2), so the scale-26 pass has no current entry.
MEASURED_TRAFFIC = {}
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


# ------------------------------------------------------------ byte models
def tr_step_bytes(n, m, A_out, fwd_probes):
    """Algorithmic bytes of one TR compression (the method's whole step):
    read the symmetric CSR (8n + 4A), the degree of every arc's head (4A),
    write and read E+ (2 x (8n + 4m)), one 4-byte read per probe of the
    forward algorithm (4 W+), the deletion flags (2m: write + read), re-read
    the symmetric CSR for the mask (4A) and write the output CSR
    (8n + 4A_out)."""
    A = 2 * m
    return ((8 * n + 4 * A) + 4 * A + 2 * (8 * n + 4 * m) + 4 * fwd_probes + 2 * m + 4 * A
            + (8 * n + 4 * A_out))


def enum_pass_bytes(n, m, fwd_probes):
    """Algorithmic bytes of one enumeration pass: E+ read once (off+ and N+)
    and one 4-byte read per probe of the forward algorithm (W+)."""
    return 8 * (n + 1) + 4 * m + 4 * fwd_probes


def enum_streamed_bytes(n, m, probes):
    """Bytes the enumeration actually reads per pass: off+ and the in-degree
    of every vertex (8 + 4 B), N+(x) staged in the tables (4 B/arc), the off+
    pair of every streamed list (8 B/arc), the in-list entry of every in-arc
    (8 B/arc: the entries of in-arcs streamed from the tail's side are read
    and skipped) and one 4-byte read per probe made (W = sum over arcs of
    min(d+(u), d+(v)))."""
    return 8 * (n + 1) + 4 * n + 4 * m + 8 * m + 8 * m + 4 * probes


def byte_model(n, m, A_out, kernel):
    """Algorithmic bytes of one launch of a streaming kernel."""
    A = 2 * m
    if kernel == "compact_orient":
        return 8 * (n + 1) + 4 * A + 4 * A + 8 * (n + 1) + 4 * m + A / 8
    if kernel == "compact_trmask":
        # offsets and columns, forward bits, the deletion flag of every arc's
        # oriented arc (the reverse arcs' through their 8-byte list entry), the
        # output CSR
        return 8 * (n + 1) + 4 * A + A / 8 + 2 * m + 8 * m + 8 * (n + 1) + 4 * A_out
    if kernel == "tri_reverse_list":
        # offsets and columns, forward bits, the orientation's chunk prefixes;
        # per reverse arc the E+ row bounds of its tail (16 B), the found column
        # (4 B) and its list entry written (8 B)
        return 8 * (n + 1) + 4 * A + A / 8 + 28 * m
    if kernel in ("compact_uniform",):
        return 8 * (n + 1) + 4 * A + 8 * (n + 1) + 4 * A_out
    if kernel in ("compact_spectral",):
        return 8 * (n + 1) + 4 * A + 4 * A + 8 * (n + 1) + 4 * A_out
    return None


def streaming_rows(kt, steps, n, m, A_out, hbm):
    """Per-call time and roofline of the step's streaming kernels.  kt maps a
    kernel name to (total ms, launches) over `steps` profiled steps; each step
    makes one call of each, and a compaction call is several launches (decide,
    chunk scan, scatter, offsets; the orientation's degree pass) timed together."""
    rows = {}
    for name in ("compact_orient", "tri_reverse_list", "compact_trmask"):
        t, launches = kt.get(name, (0.0, 0))
        if launches and t > 0:
            b = byte_model(n, m, A_out, name)
            per = t / steps
            rows[name] = {"ms": per, "launches": launches / steps, "algorithmic_bytes": b,
                          "achieved": b / per / 1e6, "frac": b / per / 1e6 / hbm}
    return rows


KERNEL_NAMES = ("tri_enum", "tri_hubs", "tri_reverse_list", "tri_eo_fresh_reserve", "tri_eo_list_reserve",
                "tri_eo_list_accept", "tri_eo_accept", "tri_eo_list_reset", "tri_classify", "compact_orient",
                "compact_trmask", "row_maps")


def _timed(stream, fn, reps):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _kernel_row(sg, ctx, stream, G, kern, p, reps, warm=1, names=()):
    """Time compress(G, kern, p) end of enqueue to done, plus per-kernel times."""
    for _ in range(warm):
        sg.compress(G, kern, p, 1).free()
    ms = _timed(stream, lambda: sg.compress(G, kern, p, 1).free(), reps)
    row = {"ms": ms, "edges_per_s": G.m / (ms / 1e3)}
    if names:
        ctx.reset_profile()
        ctx.set_profiling(True)
        H = sg.compress(G, kern, p, 1)
        ctx.synchronize()
        ctx.set_profiling(False)
        row["kept_arcs"] = H.nnz
        H.free()
        row["kernel_ms"] = {k: ctx.kernel_time(k)[0] for k in names}
    return row


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
    off_h = g.off.cpu().pin_memory()
    col_h = g.col.cpu().pin_memory()
    del g
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

    # ---- headline: K steps, per-launch events off
    clocks = ClockSampler(local)
    ctx.stats(reset=True)
    ctx.set_profiling(False)
    clocks.start()
    time.sleep(0.3)
    barrier()
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    marks[0].record(stream)
    for i in range(args.steps):
        A_out = step()
        marks[i + 1].record(stream)
    barrier()
    clocks.stop()
    ms = marks[0].elapsed_time(marks[-1]) / args.steps
    step_ms = step_stats([marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps)])
    st = ctx.stats()
    ms = max_over_ranks(ms, dist, "cuda")

    # ---- per-kernel split: a second timed region with per-launch events on
    psteps = max(1, min(args.steps, args.profile_steps))
    ctx.stats(reset=True)
    ctx.reset_profile()
    ctx.set_profiling(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(psteps):
        step()
    e1.record(stream)
    barrier()
    ctx.set_profiling(False)
    prof_ms = e0.elapsed_time(e1) / psteps
    pst = ctx.stats()
    kt = {name: ctx.kernel_time(name) for name in KERNEL_NAMES}

    hbm, peak_src = peaks()
    # one enumeration pass = the hub launch (vertices with long out-lists, when
    # there are any) + the main launch; the pass is the roofline's unit
    enum_ms = kt["tri_enum"][0] + kt["tri_hubs"][0]
    passes = max(kt["tri_enum"][1], 1)
    # the passes stream the shorter list of each arc (W probes in all); W+ is
    # scaled by the share of W they streamed (later edge-once passes skip
    # considered arcs)
    fwd_total = work["forward_probes"] * pst["probes"] / max(work["probes"], 1)
    enum_bytes = enum_pass_bytes(n, m, fwd_total / passes)
    pass_s = enum_ms / passes / 1e3
    enum_achieved = enum_bytes / pass_s / 1e9 if pass_s > 0 else None
    streamed_bytes = enum_streamed_bytes(n, m, pst["probes"] / passes)
    streams = streaming_rows(kt, psteps, n, m, A_out, hbm)
    step_bytes = tr_step_bytes(n, m, A_out, work["forward_probes"])

    # ---- other rows of the hot path (not part of the metric)
    rows = {}
    if not args.no_rows and world == 1:
        rows.update(rows_same_graph(args, sg, ctx, stream, G))
    # ---- end to end through the C-ABI with pinned host buffers.  Every step
    # uploads its graph from host memory (sg_graph_from_host), compresses it
    # and downloads the output CSR (sg_graph_download).  As a serving pipeline
    # would, a second context with its own stream moves the data: it uploads
    # step i+1 and downloads step i-1 while step i computes.
    import ctypes
    from concurrent.futures import ThreadPoolExecutor

    L = sg.lib()
    xctx = sg.Context(local)
    outs = [(torch.empty(n + 1, dtype=torch.int64).pin_memory(),
             torch.empty(max(2 * m, 1), dtype=torch.int32).pin_memory()) for _ in range(2)]

    def upload():
        h = ctypes.c_void_p()
        sg._check(L.sg_graph_from_host(xctx.handle, n, 2 * m, off_h.data_ptr(), col_h.data_ptr(), None,
                                       ctypes.byref(h)))
        xctx.synchronize()
        return sg.Graph(xctx, h)

    def download(H, k):
        o_off, o_col = outs[k & 1]
        sg._check(L.sg_graph_download(xctx.handle, H.handle, o_off.data_ptr(), o_col.data_ptr(), None))
        return H.nnz

    def e2e_run(k_steps):
        nnz = 0
        with ThreadPoolExecutor(1) as ex:
            g_next = upload()
            prev = None
            for i in range(k_steps):
                g_cur = g_next
                fut = ex.submit(lambda i=i, prev=prev: (upload() if i + 1 < k_steps else None,
                                                        download(prev, i - 1) if prev is not None else None))
                # compress on the compute context (sg.compress would use the graph's own, the transfer one)
                h = ctypes.c_void_p()
                sg._check(L.sg_compress(ctx.handle, g_cur.handle, sg.KERNELS[args.kernel], float(args.p), 1, 0,
                                        ctypes.byref(h)))
                H = sg.Graph(ctx, h)
                g_next, got = fut.result()
                if prev is not None:
                    nnz = got
                    prev.free()
                g_cur.free()
                prev = H
            nnz = download(prev, k_steps - 1)
            prev.free()
        return nnz

    e2e_run(2)
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(3, min(args.steps, 8))
    nnz_out = e2e_run(e2e_steps)
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    xctx.close()
    G.free()
    del off_h, col_h, outs
    torch.cuda.empty_cache()

    if not args.no_rows and world == 1:
        rows.update(rows_rmat22(args, sg, ctx, stream))
        ctx.release_workspace()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        rows["batch"] = batch_row(args, ctx, stream)
        torch.cuda.empty_cache()
        rows["serve"] = serve_row(args)

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
        "config": {"workload": wl["desc"], "kernel": args.kernel, "p": args.p, "seed": 1, "n": n, "m": m,
                   "eo_list_capacity": args.eo_list_cap,
                   "arcs": 2 * m, "triangles": work["triangles"], "probes_per_pass": work["probes"],
                   "forward_probes": work["forward_probes"],
                   "head_arcs": work["head_arcs"],
                   "max_out_degree": work["max_out_degree"], "kept_arcs": int(A_out),
                   "l2": "inputs larger than L2 (CSR %.0f MB > 129 MB)" % ((8 * (n + 1) + 8 * m) / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": "tri_enum pass (hub launch + main launch)",
                     "achieved": enum_achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (enum_achieved / hbm) if enum_achieved else None,
                     "traffic": measured_traffic(args.workload, args.kernel),
                     "peak_source": peak_src, "algorithmic_bytes_per_launch": enum_bytes,
                     "launch_ms": enum_ms / passes, "launches": passes / psteps,
                     "byte_model": "8(n+1) + 4m + 4 W+ per enumeration pass",
                     "launch_split_ms": {"tri_hubs": kt["tri_hubs"][0] / passes, "tri_enum": kt["tri_enum"][0] / passes},
                     "streamed": {"algorithmic_bytes_per_launch": streamed_bytes,
                                  "achieved": streamed_bytes / pass_s / 1e9 if pass_s > 0 else None,
                                  "frac": streamed_bytes / pass_s / 1e9 / hbm if pass_s > 0 else None,
                                  "byte_model": "probes made: 8(n+1) + 4n + 20m + 4 W"},
                     "eo_list_bytes_per_step": 16 * pst["eo_listed"] / psteps},
        "step_roofline": {"bytes_per_step": step_bytes, "achieved": step_bytes / (ms / 1e3) / 1e9,
                          "frac": step_bytes / (ms / 1e3) / 1e9 / hbm, "unit": "GB/s",
                          "byte_model": "TR step: (8n+4A) + 4A + 2(8n+4m) + 4 W+ + 2m + 4A + (8n+4A')"},
        "streaming_kernels": streams,
        "profiled_ms_per_step": prof_ms,
        "kernel_ms_per_step": {k: v[0] / psteps for k, v in kt.items()},
        "eo_rounds_per_step": pst["eo_rounds"] / psteps,
        "eo_passes_per_step": pst["eo_passes"] / psteps,
        "eo_list_passes_per_step": pst["eo_list_passes"] / psteps,
        "gpu_launches": st["kernel_launches"],
        "clocks": clk,
        "e2e": {"value": replica_throughput(world, m, e2e_s), "unit": "edges/s",
                "h2d_bytes_per_step": 8 * (n + 1) + 8 * m,
                "d2h_bytes_per_step": 8 * (n + 1) + 4 * int(nnz_out), "steps": e2e_steps,
                "pipeline": "a transfer context uploads step i+1 and downloads step i-1 while step i computes"},
        "rows": rows,
        "cpu_baseline": cpu,
        "cpu_all_cores": cpu_cores,
    }
    if rank == 0:
        print(json.dumps(res), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def rows_same_graph(args, sg, ctx, stream, G):
    """Other kernels on the headline graph: Edge-Once TR (p = 0.5) and the
    edge kernels, with kernel-only times."""
    rows = {}
    key = args.workload
    if args.kernel != "tr_eo":
        rows[f"{key}.tr_eo"] = _kernel_row(sg, ctx, stream, G, "tr_eo", 0.5, 2, 1,
                                           names=("tri_enum", "tri_hubs", "tri_eo", "compact_trmask"))
    for kern, name in (("uniform", "compact_uniform"), ("spectral_avgdeg", "compact_spectral")):
        r = _kernel_row(sg, ctx, stream, G, kern, 0.5, 3, 2, names=(name, "row_maps"))
        t = r["kernel_ms"][name]
        b = byte_model(G.n, G.m, r["kept_arcs"], name)
        r["kernel_roofline"] = {"kernel": name, "ms": t, "algorithmic_bytes": b, "achieved": b / t / 1e6,
                                "frac": b / t / 1e6 / peaks()[0]}
        rows[f"{key}.{kern}"] = r
    return rows


def rows_rmat22(args, sg, ctx, stream):
    """The R-MAT scale-22 kernels and analytics (edge-once TR at three p,
    spectral, uniform, the other TR variants, divergence, accuracy)."""
    import torch

    import graphgen as gg

    rows = {}
    g = gg.rmat(22, 16, seed=1, device="cuda")
    torch.cuda.synchronize()
    G = sg.Graph.from_csr(ctx, g, copy=True)
    del g
    torch.cuda.empty_cache()
    for kern, p in (("tr_eo", 0.2), ("tr_eo", 0.5), ("tr_eo", 0.8), ("tr_random", 0.5), ("uniform", 0.5),
                    ("spectral_avgdeg", 0.5), ("spectral_logn", 0.5), ("tr_p2", 0.5), ("tr_mincount", 0.5),
                    ("tr_eo_mincount", 0.5)):
        rows[f"rmat22.{kern}.p{p}"] = _kernel_row(sg, ctx, stream, G, kern, p, 3, 2)
    H = sg.compress(G, "tr_eo", 0.5, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    div = sg.divergence(G, H)
    ms = (time.perf_counter() - t0) * 1e3
    rows["rmat22.divergence"] = {"ms": ms, "kl_bits": div["kl_bits"], "cc_g": div["cc_g"], "cc_h": div["cc_h"],
                                 "pr_residual_g": div["pr_residual_g"], "pr_residual_h": div["pr_residual_h"]}
    t0 = time.perf_counter()
    acc = sg.accuracy(G, H)
    rows["rmat22.accuracy"] = {"ms": (time.perf_counter() - t0) * 1e3, "pr_aren": acc["pr_aren"],
                               "tc_aren": acc["tc_aren"], "critical_fraction": acc["critical_fraction"]}
    H.free()
    for _ in range(2):
        sg.low_degree(G).free()
    rows["rmat22.low_degree"] = {"ms": _timed(stream, lambda: sg.low_degree(G).free(), 3)}
    G.free()
    return rows


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


def batch_row(args, ctx, stream):
    """Batched compression of many R-MAT graphs (one captured CUDA-graph replay)
    against the plain loop of one compress call per graph, at identical outputs."""
    import numpy as np
    import torch

    import graphgen as gg
    import paper_1912_08950_gb300 as sg

    count = args.batch_graphs
    rng = np.random.default_rng(7)
    scales = [int(round(8 + 8 * u)) for u in rng.random(count)]
    efs = [int(e) for e in rng.integers(8, 33, size=count)]
    seeds = [i + 1 for i in range(count)]
    ps = [float(x) for x in rng.choice([0.2, 0.5, 0.8], size=count)]
    kernels = [("uniform", "spectral_avgdeg", "tr_random")[i % 3] for i in range(count)]
    t0 = time.perf_counter()
    u, vbase, _ = gg.rmat_batch(scales, efs, seeds, device="cuda")
    gen_s = time.perf_counter() - t0
    graphs = [sg.Graph.from_csr(ctx, gg.batch_member(u, vbase, i, 1 << scales[i]), copy=True) for i in range(count)]
    del u
    torch.cuda.empty_cache()
    m_total = sum(g.m for g in graphs)
    reps = max(1, min(args.steps, args.batch_steps))

    def plain():
        return [sg.compress(graphs[i], kernels[i], ps[i], seeds[i]) for i in range(count)]

    for h in plain():
        h.free()
    ctx.stats(reset=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for r in range(reps):
        outs = plain()
        if r < reps - 1:
            for h in outs:
                h.free()
    ev[1].record(stream)
    torch.cuda.synchronize()
    plain_ms = ev[0].elapsed_time(ev[1]) / reps
    plain_launches = ctx.stats(reset=True)["kernel_launches"] / reps
    d_plain = _digest(outs, stream)  # one compress call per graph: the solo outputs
    for h in outs:
        h.free()
    B = sg.Batch(ctx, graphs)
    t0 = time.perf_counter()
    B.compress(kernels, ps, seeds)  # first call: autotune + capture
    tune_s = time.perf_counter() - t0
    B.compress(kernels, ps, seeds)
    torch.cuda.synchronize()
    ctx.stats(reset=True)
    ev[2].record(stream)
    for _ in range(reps):
        outs_b = B.compress(kernels, ps, seeds)
    ev[3].record(stream)
    torch.cuda.synchronize()
    batch_ms = ev[2].elapsed_time(ev[3]) / reps
    batch_launches = ctx.stats(reset=True)["kernel_launches"] / reps
    d_batch = _digest(outs_b, stream)
    info = B.info()
    B.free()
    for g in graphs:
        g.free()
    return {"metric": METRIC + ", batched vs plain", "unit": "edges/s",
            "value": m_total / (batch_ms / 1e3), "plain_value": m_total / (plain_ms / 1e3),
            "speedup": plain_ms / batch_ms, "batch_ms": batch_ms, "plain_ms": plain_ms, "reps": reps,
            "identical_outputs": d_plain == d_batch, "graphs": count, "m_total": m_total,
            "gpu_launches_per_call": {"batch": batch_launches, "plain": plain_launches},
            "autotune": info, "autotune_s": tune_s, "generation_s": gen_s,
            "workload": f"{count} R-MAT graphs, scale round(8+8u) u~U[0,1), ef~U{{8..32}}, seed i+1, "
                        "p~U{0.2,0.5,0.8}, kernel round-robin uniform/spectral_avgdeg/tr_random"}


def serve_row(args):
    """Continuous-batching serving of compress + divergence jobs with Poisson
    arrivals: at the offered rate, then at 70% of the capacity that run showed."""
    import numpy as np
    import torch

    import graphgen as gg
    from paper_1912_08950_gb300.serve import GpuExecutor, Job, Server, poisson_arrivals, replay

    pool = {}
    for s in range(args.serve_min_scale, args.serve_max_scale + 1):
        g = gg.rmat(s, 16, seed=s, device="cuda")
        off, col, _ = g.numpy()
        pool[s] = (g.n, np.ascontiguousarray(off), np.ascontiguousarray(col))
    del g
    torch.cuda.empty_cache()
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

    res = {}
    for label, rate in (("offered", args.serve_rate), ("capacity70", None)):
        if rate is None:
            rate = 0.7 * res["offered"]["jobs_per_s"]
        srv = Server(lambda i: GpuExecutor(0), slots=args.serve_slots)
        jobs = make_jobs(args.serve_jobs, 11)
        out = replay(srv, jobs, poisson_arrivals(rate, len(jobs), seed=3))
        srv.close()
        out.pop("results")
        out["rate"] = rate
        res[label] = out
    return {"slots": args.serve_slots, **res,
            "workload": f"Poisson arrivals; jobs = compress + KL/CC on R-MAT scale "
                        f"U{{{args.serve_min_scale}..{args.serve_max_scale}}} ef 16; "
                        "kernels uniform/spectral_avgdeg/tr_random/tr_eo, p~U{0.2,0.5,0.8}; admitted by free HBM"}


def _oracle_sample(kernel, p):
    """One bounded oracle run: the same generator at scale 16."""
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
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rmat26")
    ap.add_argument("--kernel", default="tr_random")
    ap.add_argument("--p", type=float, default=0.5)
    ap.add_argument("--profile-steps", type=int, default=3, help="steps of the per-kernel timing region")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-rows", action="store_true", help="skip the extra rows (other kernels, batch, serve)")
    ap.add_argument("--eo-list-cap", type=int, default=0,
                    help="edge-once triangle list capacity in records (0: automatic, -1: none)")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--batch-steps", type=int, default=4)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-jobs", type=int, default=300)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-min-scale", type=int, default=10)
    ap.add_argument("--serve-max-scale", type=int, default=22)
    ap.add_argument("--mode", choices=["compress", "batch", "serve"], default="compress",
                    help="batch / serve: print only that row of the default line")
    args = ap.parse_args()
    if args.mode != "compress":
        import torch

        import paper_1912_08950_gb300 as sg

        torch.cuda.set_device(0)
        if args.mode == "serve":
            print(json.dumps({"mode": "serve", **serve_row(args)}), flush=True)
        else:
            stream = torch.cuda.Stream()
            ctx = sg.Context(0, stream=stream)
            print(json.dumps({"mode": "batch", **batch_row(args, ctx, stream)}), flush=True)
            ctx.close()
        return
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
