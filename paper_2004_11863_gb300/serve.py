"""Continuous-batching run server on one GPU.

Requests (simulation runs of any lattice, size and level count) arrive over
time.  The server admits an arrived request as soon as a slot and enough
device memory are free (memory counted with the library's own sizing,
lbm_bytes), keeps every admitted run resident on the device, and advances
all admitted runs in chunks of coarse steps, each run on its own CUDA stream
so that the work of different runs overlaps on the device.  When a run has
taken all its steps, its result (the macroscopic fields at probe nodes of
the finest level, and the per-level FP64 mass) is read back, its memory is
released and waiting requests are admitted: requests that arrive while
others are running join as slots and memory free up.

Runs never share memory or reductions, so a run's result does not depend
on what else is being served (the tests check it bit for bit).

Reported: runs/s, p50 and p99 time-to-result (arrival to result on the
host), and how many runs ended unstable (non-finite mass).
"""
from __future__ import annotations

import dataclasses
import time
from typing import Dict, List, Optional

import numpy as np

from . import mlbm, workloads


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    probes: np.ndarray    # [n_probes, 4] rho, u of the finest level at the end
    mass: np.ndarray      # per level
    stable: bool

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class _Active:
    def __init__(self, req, handle, stream, bytes_, now):
        self.req = req
        self.h = handle
        self.stream = stream
        self.bytes = bytes_
        self.admitted = now
        self.done_steps = 0
        self.issued_steps = 0
        self.event = None


def probe_nodes(case: workloads.Case) -> np.ndarray:
    """Four probe nodes on the finest level (fixed fractions of its extent)."""
    n = workloads.level_layout(case)[-1]["n"]
    pts = []
    for fx, fy in ((0.25, 0.5), (0.5, 0.5), (0.75, 0.5), (0.5, 0.25)):
        pts.append([int(fx * (n[0] - 1)), int(fy * (n[1] - 1)), int(0.5 * (n[2] - 1))])
    return np.asarray(pts, dtype=np.int32)


class Server:
    def __init__(self, hbm_budget: float = 32e9, max_active: int = 64, streams: int = 16,
                 chunk: int = 25, storage: str = "fp16", moving_reference: bool = True,
                 torch_allocator: bool = True, graph_min_steps: int = 0):
        """torch_allocator: take each run's device memory from PyTorch's
        caching allocator (no cudaMalloc / cudaFree, and their
        synchronisation, per run).  graph_min_steps: runs with fewer coarse
        steps than this launch their kernels directly instead of capturing a
        CUDA graph per step phase (capture costs more than it saves on short
        runs)."""
        import torch
        self.torch = torch
        self.budget = float(hbm_budget)
        self.max_active = max_active
        self.chunk = chunk
        self.storage = storage
        self.moving_reference = moving_reference
        self.torch_allocator = torch_allocator
        self.graph_min_steps = graph_min_steps
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self._next_stream = 0

    def bytes_of(self, case) -> int:
        return mlbm.lbm_bytes(case.lattice, case.collision, case.tau0, case.dims, case.boxes,
                              self.storage)

    def _open(self, req: workloads.Request):
        case = req.case
        stream = self.streams[self._next_stream % len(self.streams)]
        self._next_stream += 1
        u_ref = case.u_ref if self.moving_reference else (0.0, 0.0, 0.0)
        h = mlbm.Lbm(case.lattice, case.collision, case.tau0, case.dims, case.boxes,
                     storage=self.storage, stream=stream.cuda_stream, u_ref=u_ref,
                     torch_allocator=self.torch_allocator)
        if case.steps < self.graph_min_steps:
            h.set_graphs(False)
        h.init_analytic(case.ic)
        h.probe_add(case.nlevels - 1, probe_nodes(case))
        return h, stream

    def run(self, requests: List[workloads.Request], realtime: bool = True) -> Dict:
        """Serve a request stream; returns results and summary figures.
        realtime: honour the arrival times (else every request is there at 0)."""
        torch = self.torch
        pending = sorted(requests, key=lambda r: r.arrival)
        need = {r.rid: self.bytes_of(r.case) for r in pending}
        for r in pending:
            if need[r.rid] > self.budget:
                raise ValueError(f"request {r.rid} needs {need[r.rid]} B, above the budget")
        active: List[_Active] = []
        results: List[Result] = []
        used = 0.0
        peak_used = 0.0
        max_conc = 0
        t0 = time.perf_counter()
        while pending or active:
            now = time.perf_counter() - t0
            # admit arrived requests, first fit, while slots and memory allow
            i = 0
            while i < len(pending) and len(active) < self.max_active:
                r = pending[i]
                if realtime and r.arrival > now:
                    break
                if used + need[r.rid] <= self.budget:
                    h, st = self._open(r)
                    active.append(_Active(r, h, st, need[r.rid], time.perf_counter() - t0))
                    used += need[r.rid]
                    pending.pop(i)
                else:
                    i += 1
            peak_used = max(peak_used, used)
            max_conc = max(max_conc, len(active))
            # issue the next chunk of every run whose previous chunk is done
            progressed = False
            for a in list(active):
                if a.event is not None and not a.event.query():
                    continue
                a.done_steps = a.issued_steps
                if a.done_steps >= a.req.case.steps:
                    rec = a.h.probe(max_steps=1)
                    mass, _, stable = a.h.diag()
                    arrival = a.req.arrival if realtime else 0.0
                    results.append(Result(a.req.rid, arrival, a.admitted,
                                          time.perf_counter() - t0, rec[-1, 0], mass, stable))
                    a.h.close()
                    used -= a.bytes
                    active.remove(a)
                    progressed = True
                    continue
                n = min(self.chunk, a.req.case.steps - a.issued_steps)
                a.h.step(n)
                a.issued_steps += n
                a.event = torch.cuda.Event()
                a.event.record(a.stream)
                progressed = True
            if not progressed:
                if active:
                    time.sleep(50e-6)
                elif pending and realtime:
                    time.sleep(max(0.0, min(pending[0].arrival - now, 0.01)))
        wall = time.perf_counter() - t0
        lat = np.array([r.latency for r in results])
        return {"results": sorted(results, key=lambda r: r.rid), "wall_s": wall,
                "runs_per_s": len(results) / wall,
                "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
                "unstable": int(sum(not r.stable for r in results)),
                "peak_bytes": peak_used, "max_concurrent": max_conc}


def serve_sequential(requests: List[workloads.Request], storage: str = "fp32",
                     moving_reference: bool = True, realtime: bool = True) -> Dict:
    """Plain one-run-at-a-time stepping (the comparison for the server):
    each request waits for the previous one, runs alone with the library's
    defaults, then its result is read back.  realtime=False: every request
    is there at the start (the measured figure is then a capacity)."""
    s = Server(max_active=1, streams=1, chunk=1 << 30, storage=storage,
               moving_reference=moving_reference, torch_allocator=False)
    return s.run(requests, realtime=realtime)
