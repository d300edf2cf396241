"""Continuous-batching serving loop for compression + divergence jobs.

A job is one request of the form "compress this graph with (kernel, p, seed),
then judge the result with divergence(G, H)" -- the two calls of the library
(Listing 1 kernels; Sec. 5 metrics).  The server admits jobs while others are
still running on the GPU, as soon as an execution slot and enough device
memory are free, so their work overlaps on the device (every slot owns its own
context and CUDA stream).  Jobs keep their graphs device-resident from upload
to the last analytic.  Latency is measured from arrival to completion.

The scheduling logic is independent of the GPU: an executor object does the
work, so the admission policy can be tested with a fake executor on the CPU.
"""
from __future__ import annotations

import heapq
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field
from typing import Callable, List, Optional


@dataclass
class Job:
    """One request: a host CSR plus the compression parameters."""

    n: int
    off: object  # int64[n+1] (numpy or torch CPU tensor, ideally pinned)
    col: object  # int32/uint32[nnz]
    kernel: str
    p: float
    seed: int
    w: object = None
    arrival: float = 0.0
    job_id: int = 0

    @property
    def nnz(self) -> int:
        return int(len(self.col))

    def device_bytes(self) -> int:
        """Peak device memory the job needs: input and output CSR, the
        orientation, per-arc flags and reservations and, for the edge-once
        kernels, the triangle list (16 B per listed triangle) and its two
        active lists (32 B each), with the workspaces' quarter of headroom."""
        base = 8 * (self.n + 1) + 4 * self.nnz
        if self.w is not None:
            base += 4 * self.nnz
        per_arc = 4 + 1 + 1 + 8 + 4  # E+ column, del, considered, reservation, output
        total = 3 * base + per_arc * self.nnz + 64 * (self.n + 1) + (64 << 20)
        if self.kernel.startswith("tr_eo"):
            # the list never holds more than EO_LIST_CAP triangles (the executor's
            # cap), nor, in practice, more than 64 per arc
            total += int(min(EO_LIST_CAP, 64 * self.nnz) * (16 + 2 * 32) * 5 // 4)
        return total


# triangles an executor's edge-once list may hold (2 GB of list): enough for
# the largest served graphs to list a window of the schedule per enumeration
EO_LIST_CAP = 1 << 27


@dataclass(order=True)
class _Pending:
    arrival: float
    job_id: int
    job: Job = field(compare=False)
    fut: Future = field(compare=False)


class Server:
    """Admit jobs by free device memory and free slots; run them concurrently.

    executor_factory(slot) returns an object with run(job) -> dict and an
    optional close(); one executor per slot, each on its own stream.

    Admission reads the device's free memory at the moment it decides
    (free_memory(), by default the first executor's free_memory() method):
    the oldest waiting job starts once a slot is free and its estimate fits in
    that free memory less what the running jobs reserved and less
    `reserve_bytes` of headroom.  Running jobs' reservations are subtracted
    even where they have already allocated (and so no longer show as free),
    which errs on the safe side.  memory_budget, if given, additionally caps
    the total reserved at once.  A job that does not fit while nothing else
    runs fails with MemoryError instead of waiting forever.
    """

    def __init__(self, executor_factory: Callable[[int], object], slots: int, memory_budget: Optional[int] = None,
                 free_memory: Optional[Callable[[], int]] = None, reserve_bytes: int = 1 << 30):
        if slots < 1:
            raise ValueError("slots must be >= 1")
        self.slots = slots
        self.budget = None if memory_budget is None else int(memory_budget)
        self.reserve_bytes = int(reserve_bytes)
        self.reserved = 0
        self._cv = threading.Condition()
        self._pending: List[_Pending] = []
        self._free_slots = list(range(slots))
        self._stop = False
        self._executors = [executor_factory(i) for i in range(slots)]
        if free_memory is None and hasattr(self._executors[0], "free_memory"):
            free_memory = self._executors[0].free_memory
        self._free_memory = free_memory
        self._records = []
        self._active = 0
        self.max_active = 0
        self.admitted_room = []  # (room seen, job estimate) at every admission
        self._next_id = 0
        self._dispatcher = threading.Thread(target=self._dispatch, daemon=True)
        self._dispatcher.start()

    # ---------------------------------------------------------------- public
    def submit(self, job: Job) -> Future:
        fut: Future = Future()
        if self.budget is not None and job.device_bytes() > self.budget:
            fut.set_exception(MemoryError(f"job needs {job.device_bytes()} bytes, budget is {self.budget}"))
            return fut
        with self._cv:
            if self._stop:
                raise RuntimeError("server is closed")
            job.arrival = job.arrival or time.perf_counter()
            job.job_id = self._next_id
            self._next_id += 1
            heapq.heappush(self._pending, _Pending(job.arrival, job.job_id, job, fut))
            self._cv.notify_all()
        return fut

    def close(self, wait: bool = True):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        if wait:
            self._dispatcher.join()
        for ex in self._executors:
            if hasattr(ex, "close"):
                ex.close()

    def records(self):
        with self._cv:
            return list(self._records)

    # -------------------------------------------------------------- internal
    def room(self) -> Optional[int]:
        """Bytes a new job may reserve now (None: no limit known)."""
        limit = None
        if self.budget is not None:
            limit = self.budget - self.reserved
        if self._free_memory is not None:
            free = int(self._free_memory()) - self.reserved - self.reserve_bytes
            limit = free if limit is None else min(limit, free)
        return limit

    def _admissible(self) -> Optional[_Pending]:
        # first come, first served: the oldest job waits until it fits, which
        # keeps large jobs from starving behind a stream of small ones
        if not self._pending or not self._free_slots:
            return None
        head = self._pending[0]
        room = self.room()
        if room is not None and head.job.device_bytes() > room:
            if self._active == 0:
                # nothing will free memory for it: fail it rather than wait
                item = heapq.heappop(self._pending)
                item.fut.set_exception(MemoryError(
                    f"job needs {item.job.device_bytes()} bytes, {room} are free for it"))
                return self._admissible()
            return None
        self.admitted_room.append((room, head.job.device_bytes()))
        return heapq.heappop(self._pending)

    def _dispatch(self):
        while True:
            with self._cv:
                item = None
                while item is None:
                    if self._stop and not self._pending:
                        # wait for running jobs to finish
                        while self._active:
                            self._cv.wait()
                        return
                    item = self._admissible()
                    if item is None:
                        self._cv.wait()
                slot = self._free_slots.pop()
                self.reserved += item.job.device_bytes()
                self._active += 1
                self.max_active = max(self.max_active, self._active)
            t = threading.Thread(target=self._run, args=(slot, item), daemon=True)
            t.start()

    def _run(self, slot: int, item: _Pending):
        start = time.perf_counter()
        try:
            res = self._executors[slot].run(item.job)
            err = None
        except Exception as e:  # reported through the future
            res, err = None, e
        end = time.perf_counter()
        with self._cv:
            self.reserved -= item.job.device_bytes()
            self._free_slots.append(slot)
            self._active -= 1
            self._records.append({"job": item.job.job_id, "arrival": item.job.arrival, "start": start, "end": end,
                                  "latency": end - item.job.arrival, "m": item.job.nnz // 2, "ok": err is None})
            self._cv.notify_all()
        if err is None:
            item.fut.set_result(res)
        else:
            item.fut.set_exception(err)


class GpuExecutor:
    """Runs one job on its own context/stream: upload, compress, divergence.
    With keep_output, the result also holds H's CSR (host arrays)."""

    def __init__(self, device: int = 0, eo_list_cap: int = EO_LIST_CAP, keep_output: bool = False):
        import paper_1912_08950_gb300 as sg

        self.sg = sg
        self.device = device
        self.keep_output = keep_output
        self.ctx = sg.Context(device)
        # a bounded triangle list keeps each job's footprint predictable
        self.ctx.set_eo_list_capacity(eo_list_cap)

    def free_memory(self) -> int:
        """Device memory free for new work now: what the driver reports free,
        what the library's stream-ordered pool and torch's caching allocator
        hold but do not use."""
        import torch

        slack = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        return self.sg.device_free_memory(self.device) + max(0, slack)

    def run(self, job: Job) -> dict:
        sg = self.sg
        import numpy as np

        off = np.ascontiguousarray(job.off, dtype=np.int64)
        col = np.ascontiguousarray(job.col).view(np.uint32)
        G = sg.Graph.from_host(self.ctx, job.n, off, col, job.w)
        try:
            H = sg.compress(G, job.kernel, job.p, job.seed)
            try:
                d = sg.divergence(G, H)
                d["nnz_out"] = H.nnz
                if self.keep_output:
                    d["off"], d["col"], _ = H.download()
            finally:
                H.free()
        finally:
            G.free()
            # the job's memory estimate covers its list workspaces only while it runs
            self.ctx.release_workspace()
        return d

    def close(self):
        self.ctx.close()


def poisson_arrivals(rate: float, count: int, seed: int = 1):
    """Arrival times (seconds from 0) of a Poisson process with the given rate."""
    import numpy as np

    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def replay(server: Server, jobs: List[Job], arrivals) -> dict:
    """Submit jobs at their arrival times; return latency percentiles and throughput."""
    import numpy as np

    t0 = time.perf_counter()
    futs = []
    for job, at in zip(jobs, arrivals):
        now = time.perf_counter() - t0
        if at > now:
            time.sleep(at - now)
        job.arrival = time.perf_counter()
        futs.append(server.submit(job))
    results = [f.result() for f in futs]
    t1 = time.perf_counter()
    recs = server.records()
    lat = np.array([r["latency"] for r in recs])
    edges = sum(r["m"] for r in recs)
    return {"jobs": len(recs), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "wall_s": t1 - t0, "edges_per_s": edges / (t1 - t0),
            "jobs_per_s": len(recs) / (t1 - t0), "max_concurrent": server.max_active, "results": results}
