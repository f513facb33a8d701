"""Batched form of compression: many fields of uneven shapes in one call.

``BatchCompressor`` owns, per field, the output buffer and the workspace
(sized by the library), and the batch workspace of the work-queue
arrangement; it builds the job list of ``stz_compress_batch`` once, and runs
it with a launch arrangement (``BatchOpts``): concurrent lanes, SM share of
each field's persistent grids, one captured CUDA graph or plain launches,
and optionally the work queue -- the level stages of all 3D fields in one
persistent launch per dtype over (field, level, tile) items, with a level
schedule (every field's level 2 first, or field by field) and a tile
granularity (interior brick tiles per item).  ``autotune`` times each
candidate arrangement on the batch itself and keeps the fastest; the
containers are identical under every candidate, only the time changes.
``loop`` is the plain per-field path (one ``stz_compress`` per field, each
waiting for its size) for comparison.
"""
from __future__ import annotations

import itertools

import torch

from . import stz

# candidate arrangements: (lanes, sm_share_den, use_graph, queue), queue =
# None (per-field launches) or (schedule, tiles_per_item, blocks_per_sm)
DEFAULT_CANDIDATES = (
    [(l, d, g, None) for l, d, g in itertools.product((1, 2, 4, 8, 16), (1, 2, 4), (0, 1))
     if d <= l] +
    [(l, d, 1, (sch, gran, 0)) for l, d, sch, gran in
     itertools.product((4, 16), (1, 4), (0, 1), (1, 4)) if d <= l])


def make_opts(lanes: int, share_den: int, use_graph: int, queue=None, ws=None) -> stz.BatchOpts:
    o = stz.BatchOpts()
    o.lanes, o.sm_share_den, o.use_graph = int(lanes), int(share_den), int(use_graph)
    if queue is not None:
        if ws is None:
            raise ValueError("the work-queue arrangement needs the batch workspace")
        o.persistent = 1
        o.schedule, o.tiles_per_item, o.blocks_per_sm = (int(v) for v in queue)
        o.ws_dev, o.ws_bytes = ws.data_ptr(), ws.numel()
    return o


class BatchCompressor:
    def __init__(self, fields, ebs, modes, device=None):
        """fields: contiguous CUDA tensors (2D or 3D, float32/float64);
        ebs / modes: per-field error bound and "rel" / "abs"."""
        if not (len(fields) == len(ebs) == len(modes)) or not fields:
            raise ValueError("one bound and one mode per field")
        self.device = device or fields[0].device
        self.fields = list(fields)
        self.ebs = [float(e) for e in ebs]
        self.modes = list(modes)
        n = len(fields)
        self.outs, self.wss = [], []
        self.jobs = (stz.FieldJob * n)()
        for i, (f, eb, mode) in enumerate(zip(self.fields, self.ebs, self.modes)):
            if not f.is_cuda or not f.is_contiguous() or f.dim() not in (2, 3):
                raise ValueError("fields must be contiguous 2D/3D CUDA tensors")
            shape = tuple(f.shape)
            out = torch.empty(stz.compress_bound(shape, f.dtype), dtype=torch.uint8,
                              device=self.device)
            ws = stz.alloc_workspace(shape, f.dtype, self.device)
            self.outs.append(out)
            self.wss.append(ws)
            j = self.jobs[i]
            j.field_dev = f.data_ptr()
            for a, v in enumerate(list(shape) + [0] * (3 - len(shape))):
                j.dims[a] = int(v)
            j.ndim = len(shape)
            j.dtype = stz._dt(f.dtype)
            j.eb_mode = stz.EB_REL if mode == "rel" else stz.EB_ABS
            j.eb = eb
            j.out_dev = out.data_ptr()
            j.out_cap = out.numel()
            j.ws_dev = ws.data_ptr()
            j.ws_bytes = ws.numel()
        self.sizes_dev = torch.zeros(n, dtype=torch.int64, device=self.device)
        # the work queue's batch workspace (256-byte aligned, as torch's are)
        self.bws = torch.empty(max(1, stz.compress_batch_workspace_size(self.jobs)),
                               dtype=torch.uint8, device=self.device)
        self.opts = make_opts(4, 1, 1)
        self.tuning: list[dict] = []

    @property
    def input_bytes(self) -> int:
        return sum(f.numel() * f.element_size() for f in self.fields)

    def run(self, opts: stz.BatchOpts | None = None, stream=None) -> None:
        """Queue the whole batch (asynchronous)."""
        stz.compress_batch(self.jobs, self.sizes_dev, opts or self.opts, stream)

    def sizes(self) -> list[int]:
        """Container sizes (one copy; waits for the batch)."""
        v = self.sizes_dev.cpu().tolist()
        out = []
        for i, s in enumerate(v):
            if s < 0:  # bit 63: output buffer too small
                raise stz.StzError(stz.ERR_CAPACITY, f"stz_compress_batch field {i}")
            out.append(int(s))
        return out

    def containers(self) -> list[torch.Tensor]:
        return [o[:s] for o, s in zip(self.outs, self.sizes())]

    def loop(self, stream=None) -> list[int]:
        """The plain per-field path: one stz_compress per field."""
        sizes = []
        for f, eb, mode, out, ws in zip(self.fields, self.ebs, self.modes, self.outs, self.wss):
            c = stz.compress(f, eb, mode, out=out, workspace=ws, stream=stream)
            sizes.append(int(c.numel()))
        return sizes

    def time_ms(self, fn, reps: int = 3, warmup: int = 1) -> float:
        stream = torch.cuda.current_stream(self.device)
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(self.device)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps

    def opts_for(self, lanes: int, share_den: int, use_graph: int, queue=None) -> stz.BatchOpts:
        """The BatchOpts of an arrangement (queue: (schedule, tiles_per_item,
        blocks_per_sm) for the work queue, None for per-field launches)."""
        return make_opts(lanes, share_den, use_graph, queue, self.bws)

    def autotune(self, candidates=None, reps: int = 3) -> stz.BatchOpts:
        """Time every candidate (lanes, sm_share_den, use_graph, queue) on this
        batch and keep the fastest; returns it (also stored as self.opts)."""
        cands = candidates or [c for c in DEFAULT_CANDIDATES if c[0] <= len(self.fields)]
        self.tuning = []
        best, best_ms = None, float("inf")
        for cand in cands:
            lanes, den, graph = cand[:3]
            queue = cand[3] if len(cand) > 3 else None
            o = self.opts_for(lanes, den, graph, queue)
            ms = self.time_ms(lambda o=o: self.run(o), reps=reps)
            rec = {"lanes": lanes, "sm_share_den": den, "graph": graph, "ms": round(ms, 4)}
            if queue is not None:
                rec.update({"queue": 1, "schedule": queue[0], "tiles_per_item": queue[1],
                            "blocks_per_sm": queue[2]})
            self.tuning.append(rec)
            if ms < best_ms:
                best, best_ms = o, ms
        self.opts = best
        return best
