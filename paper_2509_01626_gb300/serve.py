"""Served form: a request loop over compressed fields resident on the device.

Region requests (box, level) arrive over time.  ``Server.run`` admits them
as slots free up -- the device-memory budget is carved into slots, each with
a workspace and an output buffer large enough for the largest request -- and
launches every admitted request at once, each on its slot's stream, through
``stz_decompress_region_async``: no host wait per request, so requests that
arrive while others are on the GPU join the next launches and their kernels
overlap with the running ones (continuous batching).  Each field's level-1
grid is decoded once when the field is loaded and reused by every request
(it is bitwise what each request would decode), and its header is parsed
from a host copy.  Completion is polled with events; latency = completion
time - arrival time, on the host clock.

``BatchServer`` batches the requests of each admission round into one
``stz_decode_requests`` call: a fixed number of kernel launches per round.

``serial`` is the plain path for comparison: one synchronous
``stz_decompress_region`` per request, in arrival order.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np
import torch

from . import stz


@dataclasses.dataclass
class Request:
    arrival: float            # seconds after the start of the run
    field: int
    lo: tuple
    hi: tuple
    level: int


@dataclasses.dataclass
class Result:
    request: Request
    latency: float            # seconds, arrival to completion seen by the host
    shape: tuple
    status: int
    out: torch.Tensor | None  # kept when the server was asked to


class _Field:
    def __init__(self, comp: torch.Tensor, cache_level1: bool):
        self.comp = comp
        self.meta = stz.info(comp)
        self.hdr = stz.header_bytes(comp)
        self.level1 = stz.decompress_progressive(comp, 1).clone() if cache_level1 else None


def poisson_requests(shapes, n: int, rate: float, seed: int, emin: int = 16, emax: int = 256,
                     levels=(1, 2, 3)) -> list[Request]:
    """n requests with exponential inter-arrival gaps (rate per second), a
    uniformly chosen field, per-axis box edge uniform in [emin, emax]
    (clipped to the field) with origin uniform inside, and a uniform level."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for i in range(n):
        f = int(rng.integers(0, len(shapes)))
        lo, hi = [], []
        for d in shapes[f]:
            e = int(min(d, rng.integers(emin, emax + 1)))
            o = int(rng.integers(0, d - e + 1))
            lo.append(o)
            hi.append(o + e)
        lv = int(levels[int(rng.integers(0, len(levels)))])
        out.append(Request(float(t[i]), f, tuple(lo), tuple(hi), lv))
    return out


class Server:
    def __init__(self, containers, budget_bytes: int, max_edge: int = 256, max_slots: int = 32,
                 cache_level1: bool = True, device=None):
        self.device = device or containers[0].device
        self.max_edge = int(max_edge)
        self.fields = [_Field(c, cache_level1) for c in containers]
        # the largest request: a max_edge box at full resolution.  Where a box
        # sits changes how many bricks (of at most 16 cells = 64 points at
        # level 2) it touches, so the workspace is sized for a box 128 points
        # wider, which covers every placement; the output for max_edge.
        slot_ws, slot_out = 0, 0
        for f in self.fields:
            shape = f.meta["shape"]
            lo = tuple(0 for _ in shape)
            hi = tuple(min(max_edge + 128, d) for d in shape)
            L = f.meta["levels"]
            ws = stz.region_workspace_size(f.hdr, f.comp.numel(), lo, hi, L,
                                           f.level1 is not None)
            if ws == 0:
                raise ValueError("cannot size the region workspace")
            npts = 1
            for d in shape:
                npts *= min(max_edge, d)
            slot_ws = max(slot_ws, ws)
            slot_out = max(slot_out, npts * (8 if f.meta["dtype"] == torch.float64 else 4))
        self.slot_bytes = slot_ws + slot_out
        self.nslots = int(max(1, min(max_slots, budget_bytes // self.slot_bytes)))
        self.ws = [torch.empty(slot_ws, dtype=torch.uint8, device=self.device)
                   for _ in range(self.nslots)]
        self.outs = [torch.empty(slot_out, dtype=torch.uint8, device=self.device)
                     for _ in range(self.nslots)]
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(self.nslots)]
        self.events = [torch.cuda.Event() for _ in range(self.nslots)]

    def _launch(self, slot: int, r: Request, status: torch.Tensor):
        f = self.fields[r.field]
        if any(b - a > self.max_edge for a, b in zip(r.lo, r.hi)):
            raise ValueError(f"box edge above the server's maximum {self.max_edge}: {r}")
        dt = f.meta["dtype"]
        out = self.outs[slot].view(dt)
        shape = stz.decompress_region_async(f.comp, f.hdr, r.lo, r.hi, r.level, out,
                                            self.ws[slot], status,
                                            level1=f.level1, stream=self.streams[slot])
        self.events[slot].record(self.streams[slot])
        return shape

    def run(self, requests, keep_outputs: bool = False, realtime: bool = True):
        """Serve the requests (sorted by arrival); returns the results in
        completion order and the wall time of the run."""
        order = sorted(range(len(requests)), key=lambda i: requests[i].arrival)
        pending = collections.deque((i, requests[i]) for i in order)
        # one status word per request: each decode writes its own, and the
        # words are read once, after the run
        status = torch.zeros(max(1, len(requests)), dtype=torch.int32, device=self.device)
        waiting = collections.deque()
        free = list(range(self.nslots - 1, -1, -1))
        inflight = {}
        results, index = [], []
        t0 = time.perf_counter()
        while pending or waiting or inflight:
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0][1].arrival <= now):
                waiting.append(pending.popleft())
            # admit every waiting request a slot is free for, and launch them
            while waiting and free:
                i, r = waiting.popleft()
                slot = free.pop()
                inflight[slot] = (i, r, self._launch(slot, r, status[i:i + 1]))
            # completions
            done = [s for s in inflight if self.events[s].query()]
            if done:
                now = time.perf_counter() - t0
                for s in done:
                    i, r, shape = inflight.pop(s)
                    out = None
                    if keep_outputs:
                        n = int(np.prod(shape)) if len(shape) else 0
                        with torch.cuda.stream(self.streams[s]):
                            out = self.outs[s].view(self.fields[r.field].meta["dtype"])[:n] \
                                .reshape(shape).clone()
                    results.append(Result(r, now - r.arrival, shape, 0, out))
                    index.append(i)
                    free.append(s)
        wall = time.perf_counter() - t0
        torch.cuda.synchronize(self.device)
        st = status.cpu().numpy()
        for res, i in zip(results, index):
            res.status = int(st[i])
        if st.any():
            raise RuntimeError(f"{int((st != 0).sum())} request decodes reported a corrupt "
                               "container")
        return results, wall


class BatchServer:
    """The served form with batched launches: every admission round takes up
    to ``max_batch`` waiting requests (in arrival order) and decodes them
    with one ``stz_decode_requests`` call -- a fixed number of kernel
    launches whatever the number of requests -- on one of ``nbatch`` streams;
    rounds that start while others run overlap with them on the GPU
    (continuous batching).  Each field's level-1 grid and decode tables are
    built once when the field is loaded."""

    def __init__(self, containers, budget_bytes: int, max_edge: int = 256, max_batch: int = 16,
                 max_inflight: int = 4, device=None):
        self.device = device or containers[0].device
        self.max_edge = int(max_edge)
        self.fields = [_Field(c, True) for c in containers]
        self.tables = [stz.decode_tables(f.comp, f.hdr) for f in self.fields]
        self.farr = stz.served_fields([(f.comp, f.hdr, f.level1, t)
                                       for f, t in zip(self.fields, self.tables)])
        # the largest request: a max_edge box at full resolution, sized for
        # any placement (128 points wider, as in Server); a batch of them
        # bounds every batch's workspace
        shape = self.fields[0].meta["shape"]
        itemsize = 8 if self.fields[0].meta["dtype"] == torch.float64 else 4
        npts = 1
        for d in shape:
            npts *= min(max_edge, d)
        self.slot_out = npts * itemsize
        probe_out = torch.empty(16, dtype=torch.uint8, device=self.device)
        mb = int(max_batch)
        while True:
            reqs = (stz.RegionRequest * mb)()
            for q in reqs:
                q.field = 0
                q.level = self.fields[0].meta["levels"]
                for a, d in enumerate(shape):
                    q.lo[a] = 0
                    q.hi[a] = min(max_edge + 128, d)
                q.out_dev = probe_out.data_ptr()
                q.out_cap = 1 << 62
            ws = stz.decode_requests_workspace(reqs, self.farr)
            if ws == 0:
                raise ValueError("cannot size the batch workspace")
            per = ws + mb * self.slot_out
            if per * 2 <= budget_bytes or mb == 1:
                break
            mb = max(1, mb // 2)
        self.max_batch = mb
        self.nbatch = int(max(1, min(max_inflight, budget_bytes // per)))
        self.ws = [torch.empty(ws, dtype=torch.uint8, device=self.device)
                   for _ in range(self.nbatch)]
        self.outs = [torch.empty(mb * self.slot_out, dtype=torch.uint8, device=self.device)
                     for _ in range(self.nbatch)]
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(self.nbatch)]
        self.events = [torch.cuda.Event() for _ in range(self.nbatch)]

    def _launch(self, b: int, batch, status: torch.Tensor):
        reqs = (stz.RegionRequest * len(batch))()
        base = self.outs[b].data_ptr()
        for k, (q, (_, r)) in enumerate(zip(reqs, batch)):
            if any(h - l > self.max_edge for l, h in zip(r.lo, r.hi)):
                raise ValueError(f"box edge above the server's maximum {self.max_edge}: {r}")
            q.field = r.field
            q.level = r.level
            for a in range(len(r.lo)):
                q.lo[a] = r.lo[a]
                q.hi[a] = r.hi[a]
            q.out_dev = base + k * self.slot_out
            q.out_cap = self.slot_out
        stz.decode_requests(reqs, self.farr, self.ws[b], status, stream=self.streams[b])
        self.events[b].record(self.streams[b])
        return [tuple(int(v) for v in q.out_dims[:len(self.fields[q.field].meta["shape"])])
                for q in reqs]

    def run(self, requests, keep_outputs: bool = False, realtime: bool = True):
        """Serve the requests; returns the results in completion order and the
        wall time of the run (as Server.run)."""
        order = sorted(range(len(requests)), key=lambda i: requests[i].arrival)
        pending = collections.deque(requests[i] for i in order)
        # one status word per request, in arrival order: a batch's requests are
        # consecutive in that order, so its words are one contiguous run
        status = torch.zeros(max(1, len(requests)), dtype=torch.int32, device=self.device)
        waiting = collections.deque()
        free = list(range(self.nbatch - 1, -1, -1))
        inflight = {}
        results, index = [], []
        moved = 0  # requests moved to `waiting` so far = arrival-order index of the next
        t0 = time.perf_counter()
        while pending or waiting or inflight:
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                waiting.append((moved, pending.popleft()))
                moved += 1
            while waiting and free:
                batch = [waiting.popleft() for _ in range(min(self.max_batch, len(waiting)))]
                b = free.pop()
                k0 = batch[0][0]
                shapes = self._launch(b, batch, status[k0:k0 + len(batch)])
                inflight[b] = (batch, shapes)
            done = [b for b in inflight if self.events[b].query()]
            if done:
                now = time.perf_counter() - t0
                for b in done:
                    batch, shapes = inflight.pop(b)
                    for k, ((i, r), shape) in enumerate(zip(batch, shapes)):
                        out = None
                        if keep_outputs:
                            n = int(np.prod(shape)) if len(shape) else 0
                            dt = self.fields[r.field].meta["dtype"]
                            with torch.cuda.stream(self.streams[b]):
                                off = k * self.slot_out
                                out = self.outs[b][off:off + self.slot_out].view(dt)[:n] \
                                    .reshape(shape).clone()
                        results.append(Result(r, now - r.arrival, shape, 0, out))
                        index.append(i)
                    free.append(b)
        wall = time.perf_counter() - t0
        torch.cuda.synchronize(self.device)
        st = status.cpu().numpy()
        for res, i in zip(results, index):
            res.status = int(st[i])
        if st.any():
            raise RuntimeError(f"{int((st != 0).sum())} request decodes reported a corrupt "
                               "container")
        return results, wall


def serial(containers, requests, workspace: torch.Tensor, out: torch.Tensor,
           realtime: bool = True, keep_outputs: bool = False):
    """Plain per-request path: one synchronous stz_decompress_region each, in
    arrival order.  Returns results and wall time."""
    metas = [stz.info(c) for c in containers]
    results = []
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda r: r.arrival):
        if realtime:
            while time.perf_counter() - t0 < r.arrival:
                pass
        m = metas[r.field]
        y = stz.decompress_region(containers[r.field], r.lo, r.hi, r.level,
                                  out=out.view(m["dtype"]), workspace=workspace, meta=m)
        now = time.perf_counter() - t0
        results.append(Result(r, now - r.arrival, tuple(y.shape), 0,
                              y.clone() if keep_outputs else None))
    return results, time.perf_counter() - t0


def latency_stats(results, wall: float) -> dict:
    lat = np.array([r.latency for r in results]) * 1e3
    return {"requests": len(results), "throughput_rps": round(len(results) / wall, 1),
            "p50_ms": round(float(np.percentile(lat, 50)), 4),
            "p99_ms": round(float(np.percentile(lat, 99)), 4),
            "mean_ms": round(float(lat.mean()), 4)}
