#!/usr/bin/env python3
"""Benchmark of the STZ hot path on GB300 (one JSON line on stdout).

Workload: one 512^3 float32 log-normal Gaussian random field (power spectrum
k^-3, exp(1.5 g); stand-in for the Nyx baryon density, Table 4), relative
error bound 1e-3, L = 3 levels.  One step is one pass of the whole hot path
over that field:

    compress  ->  full decompress  ->  progressive decompress to levels 1 and 2
              ->  random-access decompress of a 64^3 box and of a 512^2 slice

`value` = field bytes / step time (GB/s, 1e9 B), inputs resident in HBM;
per-operation rates and the region-decode latency distribution (p50/p99 over
random boxes, edges 16-256, random level) are reported beside it.  `e2e`
repeats the step through the same C-ABI calls with the field and the
container in pinned host memory, the copies inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank compresses its own field (weak scaling, no
collective on the data path); the step time is the maximum over ranks.
`--impl reference` times the CPU oracle (single thread) on a bounded sample
of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "compress/decompress GB/s vs HBM roofline at eb=1e-3; p99 region-decode latency"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--size", type=int, default=512, help="edge of the cubic field")
    p.add_argument("--eb", type=float, default=1e-3)
    p.add_argument("--region-requests", type=int, default=200)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-profile", action="store_true")
    p.add_argument("--no-batch", action="store_true", help="skip the batched-form section")
    p.add_argument("--no-serve", action="store_true", help="skip the served-form section")
    p.add_argument("--serve-fields", type=int, default=8)
    p.add_argument("--serve-size", type=int, default=1024)
    p.add_argument("--serve-requests", type=int, default=1000, help="requests per rate")
    p.add_argument("--serve-rates", default="1000,5000,10000,50000")
    p.add_argument("--no-bounds", action="store_true", help="skip the four-bound section")
    p.add_argument("--no-large", action="store_true",
                   help="skip the 1024^3 f32 / 768^3 f64 section")
    p.add_argument("--no-ablation", action="store_true", help="skip the predictor ablation")
    p.add_argument("--no-roi", action="store_true", help="skip the ROI workflow")
    p.add_argument("--write-traffic", nargs=4, metavar=("KERNEL", "NCU_RAW_CSV", "BENCH_JSON",
                                                        "CAPTURE"),
                   help="record KERNEL's DRAM traffic per algorithmic byte in "
                        "profiles/ncu_traffic.json from an ncu raw CSV (ncu -i REP --page raw "
                        "--csv) of one bench step and that step's bench line (same size, with "
                        "the kernel timer on); CAPTURE describes the ncu command; then exit")
    return p.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# --------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ workload
def make_field(size, rank, device):
    from paper_2509_01626_gb300 import synth

    return synth.grf((size, size, size), synth.seed_for(2, rank), slope=-3.0,
                     lognormal_sigma=1.5, dtype=np.float32, device=device)


def reduce_max(value: float, device) -> float:
    """Maximum of `value` over the ranks (the value itself with one rank)."""
    import torch
    import torch.distributed as tdist

    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def step_boxes(size):
    b = min(64, max(1, size // 2))
    o = (size - b) // 3
    box = ((o, o, o), (o + b, o + b, o + b))
    z = size // 2
    slab = ((z, 0, 0), (z + 1, size, size))
    return box, slab


def traffic_ratio(kernel):
    """DRAM bytes per algorithmic byte of `kernel` from the committed ncu
    capture summary, if that capture was taken of the current sources (else
    None).  profiles/ncu_traffic.json: kernel -> {"sources": [...],
    "sources_sha256": ..., "dram_bytes": D, "algo_bytes": A, "capture": ...}."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e:
        return None
    h = hashlib.sha256()
    for src in e["sources"]:
        full = os.path.join(ROOT, src)
        if not os.path.exists(full):
            return None
        with open(full, "rb") as f:
            h.update(f.read())
    if h.hexdigest() != e["sources_sha256"]:
        return None
    return float(e["dram_bytes"]) / float(e["algo_bytes"])


# sources whose hash keys a recorded traffic ratio (any change voids it), by
# kernel name prefix
TRAFFIC_SOURCES = {
    "k_decode_chunks": ["paper_2509_01626_gb300/csrc/stz_huffman.cu"],
    "k_chunk_words": ["paper_2509_01626_gb300/csrc/stz_huffman.cu"],
    "k_pack": ["paper_2509_01626_gb300/csrc/stz_huffman.cu"],
    "k_range": ["paper_2509_01626_gb300/csrc/stz_range.cu"],
    "k_level": ["paper_2509_01626_gb300/csrc/stz_level.cu",
                "paper_2509_01626_gb300/csrc/stz_predict.cuh"],
}
COMMON_SOURCES = ["paper_2509_01626_gb300/csrc/stz_common.cuh",
                  "paper_2509_01626_gb300/csrc/stz_kernels.cuh",
                  "paper_2509_01626_gb300/csrc/stz_prof.cuh", "include/stz.h"]


def write_traffic(kernel, ncu_csv, bench_json, capture):
    """DRAM bytes (read + written) of every captured launch of `kernel` over
    the algorithmic bytes the library counted for one bench step, into
    profiles/ncu_traffic.json.  The capture must hold exactly one step's
    launches of the kernel (ncu -c with the step's launch count)."""
    import csv

    rows = list(csv.reader(open(ncu_csv)))
    head = rows[0]
    ci = {n: i for i, n in enumerate(head)}
    dram = 0.0
    n = 0
    for r in rows[2:]:  # row 1 holds the units
        if len(r) < len(head):
            continue
        scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
        for m in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            dram += float(r[ci[m]].replace(",", "")) * scale.get(rows[1][ci[m]], 1.0)
        n += 1
    line = [ln for ln in open(bench_json) if ln.startswith("{")][0]
    d = json.loads(line)
    k = [e for e in d["kernels"] if e["kernel"] == kernel][0]
    algo = k["achieved_gbs"] * 1e9 * k["ms_per_step"] * 1e-3  # bytes of one step
    if abs(k["launches_per_step"] - n) > 1e-6:
        raise SystemExit(f"captured {n} launches, the step has {k['launches_per_step']}")
    key = [k for k in TRAFFIC_SOURCES if kernel.startswith(k)][0]
    srcs = TRAFFIC_SOURCES[key] + COMMON_SOURCES
    h = hashlib.sha256()
    for src in srcs:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    table = json.load(open(path)) if os.path.exists(path) else {}
    table[kernel] = {"sources": srcs, "sources_sha256": h.hexdigest(), "dram_bytes": dram,
                     "algo_bytes": algo, "launches": n, "capture": capture}
    with open(path, "w") as f:
        json.dump(table, f, indent=1)
    print(json.dumps({kernel: table[kernel]}))


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2509_01626_gb300 import stz

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    size = args.size
    shape = (size, size, size)
    x_host = make_field(size, rank, f"cuda:{local_rank}")
    field = torch.from_numpy(x_host).to(dev)
    field_bytes = field.numel() * 4
    ws = stz.alloc_workspace(shape, torch.float32, dev)
    out = torch.empty(stz.compress_bound(shape, torch.float32), dtype=torch.uint8, device=dev)
    full = torch.empty(shape, dtype=torch.float32, device=dev)
    p_out = {k: torch.empty(field.numel() // (8 ** (3 - k)) + 1, dtype=torch.float32, device=dev)
             for k in (1, 2)}
    (blo, bhi), (slo, shi) = step_boxes(size)
    box_out = torch.empty(max(1, (bhi[0] - blo[0])) ** 3, dtype=torch.float32, device=dev)
    slab_out = torch.empty(size * size, dtype=torch.float32, device=dev)

    meta = {"shape": shape, "dtype": torch.float32, "ndim": 3, "levels": 3}

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        comp = stz.compress(field, args.eb, "rel", out=out, workspace=ws)
        if ev:
            ev[1].record(stream)
        stz.decompress_full(comp, out=full, workspace=ws, meta=meta)
        if ev:
            ev[2].record(stream)
        for k in (1, 2):
            stz.decompress_progressive(comp, k, out=p_out[k], workspace=ws, meta=meta)
        if ev:
            ev[3].record(stream)
        stz.decompress_region(comp, blo, bhi, 3, out=box_out, workspace=ws, meta=meta)
        if ev:
            ev[4].record(stream)
        stz.decompress_region(comp, slo, shi, 3, out=slab_out, workspace=ws, meta=meta)
        if ev:
            ev[5].record(stream)
        return comp

    dist = world > 1
    if dist:
        import torch.distributed as tdist

    def barrier():
        if dist:
            tdist.barrier()

    for _ in range(max(args.warmup, 1)):
        comp = step()
    torch.cuda.synchronize()
    comp_bytes = int(comp.numel())

    clocks = ClockSampler(_gpu_uuid(local_rank))
    clocks.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    launches0 = stz.launch_count()
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        step(evs[i])
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = stz.launch_count() - launches0
    ms_step = t0.elapsed_time(t1) / args.steps
    clk = clocks.stop()
    # per-kernel device times and algorithmic bytes: the same steps once more
    # with an event pair around every launch, on the launching stream (kept
    # out of the timed region above)
    kernels = {}
    if not args.no_profile:
        stz.profile_reset()
        stz.profile_enable(True)
        for i in range(args.steps):
            step()
        torch.cuda.synchronize()
        stz.profile_enable(False)
        kernels = stz.profile_read()
    ms_step = reduce_max(ms_step, dev)
    ops = np.array([[e[j].elapsed_time(e[j + 1]) for j in range(5)] for e in evs])
    op_ms = ops.mean(axis=0)

    # region-decode latency distribution (synchronous calls, host clock)
    from paper_2509_01626_gb300 import synth

    boxes = synth.random_boxes(shape, args.region_requests, synth.seed_for(5, rank), 16, 256)
    rng = np.random.Generator(np.random.PCG64(synth.seed_for(5, 1000 + rank)))
    levels = rng.integers(1, 4, size=len(boxes))
    reg_out = torch.empty(256 ** 3, dtype=torch.float32, device=dev)
    lat = []
    # warm-up on other boxes: every measured request is a first sight
    for lo, hi in synth.random_boxes(shape, 5, synth.seed_for(5, 2000 + rank), 16, 256):
        stz.decompress_region(comp, lo, hi, 3, out=reg_out, workspace=ws, meta=meta)
    torch.cuda.synchronize()
    for (lo, hi), lv in zip(boxes, levels):
        a = time.perf_counter()
        stz.decompress_region(comp, lo, hi, int(lv), out=reg_out, workspace=ws, meta=meta)
        lat.append((time.perf_counter() - a) * 1e3)
    lat = np.array(lat)

    # the ROI workflow of Sec. 3.3: decode level 1 (the 1/64 coarse grid),
    # select the top 1% of its 4^3 blocks by value range, decode those regions
    # at full resolution
    roi = None
    if not args.no_roi:
        coarse = stz.decompress_progressive(comp, 1, workspace=ws, meta=meta).clone()
        for _ in range(3):
            stz.roi_select(coarse, (4, 4, 4), "range", "top", 0.01)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        roi_ms = []
        for _ in range(10):
            ev[0].record(stream)
            sel = stz.roi_select(coarse, (4, 4, 4), "range", "top", 0.01)
            ev[1].record(stream)
            torch.cuda.synchronize()
            roi_ms.append(ev[0].elapsed_time(ev[1]))
        boxes_roi = stz.roi_boxes(sel.cpu().numpy(), tuple(coarse.shape), (4, 4, 4), 4, shape)
        t = time.perf_counter()
        for lo, hi in boxes_roi:
            stz.decompress_region(comp, lo, hi, 3, out=reg_out, workspace=ws, meta=meta)
        torch.cuda.synchronize()
        serial_ms = (time.perf_counter() - t) * 1e3
        # all selected regions in one batched call (the level-1 grid just decoded
        # and the decode tables built once for the resident field)
        hdr = stz.header_bytes(comp)
        tables = stz.decode_tables(comp, hdr)
        for _ in range(2):
            stz.decode_regions(comp, boxes_roi, 3, level1=coarse, tables=tables, hdr=hdr, meta=meta)
        torch.cuda.synchronize()
        batched_ms = []
        for _ in range(5):
            t = time.perf_counter()
            stz.decode_regions(comp, boxes_roi, 3, level1=coarse, tables=tables, hdr=hdr, meta=meta)
            batched_ms.append((time.perf_counter() - t) * 1e3)
        roi = {"select_ms": round(float(np.median(roi_ms)), 4), "units": int(coarse.numel() // 64),
               "selected": len(boxes_roi),
               "regions_ms": round(float(np.median(batched_ms)), 3),
               "regions_serial_ms": round(serial_ms, 3),
               "workflow": "level-1 decode, top 1% of 4^3 blocks by range, 16^3 regions at level 3 "
                           "(regions_ms: one batched call, host wall time with its status "
                           "read-back; regions_serial_ms: one stz_decompress_region per region)"}

    # end to end through the same calls, host buffers, copies timed.  The
    # copies run on two copy streams (one per direction) beside the compute:
    # step i's outputs go to the host while step i+1 computes, and step i+2's
    # field is uploaded while step i decodes (three field buffers, two sets of
    # outputs).  Copies of one direction queue on one copy engine, so step
    # i's output copies are issued after step i+1's container round trip,
    # which the compute waits for.
    # Every copy of every timed step lies inside the timed region.
    e2e = None
    if not args.no_e2e:
        h_field = torch.from_numpy(x_host).pin_memory()
        h_comp = torch.empty(comp_bytes, dtype=torch.uint8).pin_memory()
        h_full = torch.empty(shape, dtype=torch.float32).pin_memory()
        h_p = {k: torch.empty(p_out[k].numel(), dtype=torch.float32).pin_memory() for k in (1, 2)}
        h_box = torch.empty(box_out.numel(), dtype=torch.float32).pin_memory()
        h_slab = torch.empty(slab_out.numel(), dtype=torch.float32).pin_memory()
        nf = 3  # field buffers: step i+2's field is uploaded while step i decodes
        d_field = [torch.empty_like(field) for _ in range(nf)]
        d_comp = torch.empty(comp_bytes, dtype=torch.uint8, device=dev)
        fulls = [full, torch.empty_like(full)]
        pouts = [p_out, {k: torch.empty_like(v) for k, v in p_out.items()}]
        boxes = [box_out, torch.empty_like(box_out)]
        slabs = [slab_out, torch.empty_like(slab_out)]
        # one stream per copy direction, and the compute on a stream of its
        # own: uploads, downloads and compute all overlap
        up = torch.cuda.Stream(device=dev)
        down = torch.cuda.Stream(device=dev)
        cstream = torch.cuda.Stream(device=dev)
        up_ev = [torch.cuda.Event() for _ in range(nf)]
        out_free = [torch.cuda.Event() for _ in range(2)]  # set b's host copies done
        for e in out_free:
            e.record(cstream)

        def upload(f):
            with torch.cuda.stream(up):
                d_field[f % nf].copy_(h_field, non_blocking=True)
                up_ev[f % nf].record(up)

        pending = []  # the previous step's output copies: (ready event, dst, src), set

        def done_on(st):
            ev = torch.cuda.Event()
            ev.record(st)
            return ev

        def flush():
            # issue the previous step's output copies on the download stream
            if not pending:
                return
            items, ob = pending.pop()
            for ev, dst, src in items:
                down.wait_event(ev)
                with torch.cuda.stream(down):
                    dst.copy_(src, non_blocking=True)
            out_free[ob].record(down)

        def e2e_step(i, n):
            b = i & 1
            cstream.wait_event(up_ev[i % nf])
            c = stz.compress(d_field[i % nf], args.eb, "rel", out=out, workspace=ws,
                             stream=cstream)
            with torch.cuda.stream(cstream):
                h_comp.copy_(c, non_blocking=True)
                d_comp.copy_(h_comp, non_blocking=True)
            flush()
            cstream.wait_event(out_free[b])
            items = []
            y = stz.decompress_full(d_comp, out=fulls[b], workspace=ws, meta=meta, stream=cstream)
            items.append((done_on(cstream), h_full, y))
            # the field two steps ahead: issued once this step's small upload
            # has gone (copies of one direction queue on one engine)
            if i + 2 < n:
                upload(i + 2)
            for k in (1, 2):
                pk = stz.decompress_progressive(d_comp, k, out=pouts[b][k], workspace=ws,
                                                meta=meta, stream=cstream)
                items.append((done_on(cstream), h_p[k][: pk.numel()], pk.reshape(-1)))
            bx = stz.decompress_region(d_comp, blo, bhi, 3, out=boxes[b], workspace=ws,
                                       meta=meta, stream=cstream)
            items.append((done_on(cstream), h_box[: bx.numel()], bx.reshape(-1)))
            sl = stz.decompress_region(d_comp, slo, shi, 3, out=slabs[b], workspace=ws,
                                       meta=meta, stream=cstream)
            items.append((done_on(cstream), h_slab[: sl.numel()], sl.reshape(-1)))
            pending.append((items, b))

        def run(n):
            for f in range(min(2, n)):
                upload(f)
            for i in range(n):
                e2e_step(i, n)
            flush()
            for cs in (up, down):
                done = torch.cuda.Event()
                done.record(cs)
                cstream.wait_event(done)

        run(max(args.warmup, 1))
        torch.cuda.synchronize()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b_ = torch.cuda.Event(enable_timing=True)
        a.record(cstream)
        run(args.steps)
        b_.record(cstream)
        torch.cuda.synchronize()
        e2e_ms = a.elapsed_time(b_) / args.steps
        e2e_ms = reduce_max(e2e_ms, dev)
        box_n = (bhi[0] - blo[0]) * (bhi[1] - blo[1]) * (bhi[2] - blo[2])
        d2h = comp_bytes + field_bytes + 4 * (p_out[1].numel() - 1) + 4 * (p_out[2].numel() - 1) \
            + 4 * box_n + 4 * size * size
        e2e = {"value": round(world * field_bytes / (e2e_ms * 1e-3) / 1e9, 3), "unit": "GB/s",
               "h2d_bytes_per_step": int(field_bytes + comp_bytes),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_ms, 4)}

    return dict(ms_step=ms_step, op_ms=op_ms, lat=lat, kernels=kernels, e2e=e2e, clk=clk, roi=roi,
                comp_bytes=comp_bytes, field_bytes=field_bytes, launches=launches,
                x_host=x_host)


def _gpu_uuid(local_rank):
    try:
        import torch

        u = torch.cuda.get_device_properties(local_rank).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:  # noqa: BLE001
        return str(local_rank)


# ------------------------------------------------------------ batched form
def run_batched(args, dev):
    """The mixed batch of 64 uneven fields: the plain per-field loop (one
    stz_compress each) against stz_compress_batch with the autotuned
    arrangement; containers checked identical."""
    import torch

    from paper_2509_01626_gb300 import batch, synth

    items = synth.batch_workload()
    fields = [synth.make_batch_field(it, device=str(dev)) for it in items]
    ebs = [it[4] for it in items]
    bc = batch.BatchCompressor(fields, ebs, ["rel"] * len(fields), device=dev)
    nbytes = bc.input_bytes
    loop_ms = bc.time_ms(bc.loop, reps=3)
    loop_sizes = bc.loop()
    loop_out = [o[:n].clone() for o, n in zip(bc.outs, loop_sizes)]
    best = bc.autotune(reps=2)
    batch_ms = bc.time_ms(bc.run, reps=5)
    bc.run()
    sizes = bc.sizes()
    identical = sizes == loop_sizes and all(
        torch.equal(o[:n], r) for o, n, r in zip(bc.outs, sizes, loop_out))
    del loop_out
    out = {"workload": "64 fields: 40 3D f32 dims U[64,512] (sinusoids + noise), 16 2D f32 "
                       "1800x3600 (banded), 8 3D f64 256^3 (smooth); rel eb from "
                       "{1e-2,1e-3,1e-4}",
           "input_gb": round(nbytes / 1e9, 3),
           "loop_ms": round(loop_ms, 3), "loop_gbs": round(nbytes / (loop_ms * 1e-3) / 1e9, 2),
           "batch_ms": round(batch_ms, 3),
           "batch_gbs": round(nbytes / (batch_ms * 1e-3) / 1e9, 2),
           "speedup": round(loop_ms / batch_ms, 3),
           "autotuned": {"lanes": best.lanes, "sm_share_den": best.sm_share_den,
                         "graph": best.use_graph, "work_queue": best.persistent,
                         "schedule": (("level-major", "field-major")[best.schedule]
                                      if best.persistent else None),
                         "tiles_per_item": best.tiles_per_item if best.persistent else None},
           "best_ms_by_arrangement": {
               "per_field_launches": min((t["ms"] for t in bc.tuning if not t.get("queue")),
                                         default=None),
               "work_queue": min((t["ms"] for t in bc.tuning if t.get("queue")), default=None)},
           "identical_to_loop": bool(identical),
           "compression_ratio": round(nbytes / sum(sizes), 3),
           "candidates": len(bc.tuning)}
    del bc, fields
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------- served form
def run_served(args, dev):
    """Resident compressed fields; Poisson request streams of random boxes at
    several rates, served by the continuous-batching loop and by the serial
    per-request path."""
    import torch

    from paper_2509_01626_gb300 import serve, stz, synth

    size = args.serve_size
    shape = (size, size, size)
    comps = []
    ws = stz.alloc_workspace(shape, torch.float32, dev)
    out = torch.empty(stz.compress_bound(shape, torch.float32), dtype=torch.uint8, device=dev)
    raw = 0
    for i in range(args.serve_fields):
        x = synth.grf(shape, synth.seed_for(5, i), slope=-5.0 / 3.0, lognormal_sigma=None,
                      dtype=np.float32, device=str(dev), white_source="torch", as_tensor=True)
        comps.append(stz.compress(x, 1e-3, "rel", out=out, workspace=ws).clone())
        raw += x.numel() * 4
        del x
        torch.cuda.empty_cache()
    del out
    resident = sum(c.numel() for c in comps)
    free, _ = torch.cuda.mem_get_info(dev)
    budget = int(min(16 << 30, free // 4))
    srv = serve.Server(comps, budget_bytes=budget, max_edge=256, max_slots=32)
    # the same loop with one slot: requests one after another, with the same
    # cached level-1 grids and parsed headers -- isolates what the overlap of
    # requests (continuous batching) adds beyond the caching
    srv1 = serve.Server(comps, budget_bytes=budget, max_edge=256, max_slots=1)
    # every admission round decoded by one stz_decode_requests call: a fixed
    # number of launches per round, rounds overlapping on their streams
    bsrv = serve.BatchServer(comps, budget_bytes=budget, max_edge=256, max_batch=16)
    reg_out = torch.empty(256 ** 3 * 4, dtype=torch.uint8, device=dev)
    rates = [float(r) for r in args.serve_rates.split(",") if r]
    # warm both paths
    warm = serve.poisson_requests([shape] * len(comps), 20, 1e5, synth.seed_for(5, 99))
    srv.run(warm)
    srv1.run(warm)
    bsrv.run(warm)
    serve.serial(comps, warm, ws, reg_out, realtime=False)
    per_rate = []
    for k, rate in enumerate(rates):
        reqs = serve.poisson_requests([shape] * len(comps), args.serve_requests, rate,
                                      synth.seed_for(5, 200 + k))
        res, wall = srv.run(reqs)
        bres, bwall = bsrv.run(reqs)
        cres, cwall = srv1.run(reqs)
        sres, swall = serve.serial(comps, reqs, ws, reg_out)
        per_rate.append({"rate_rps": rate, "served_batched": serve.latency_stats(bres, bwall),
                         "served": serve.latency_stats(res, wall),
                         "serial_cached": serve.latency_stats(cres, cwall),
                         "serial": serve.latency_stats(sres, swall)})
    out = {"workload": f"{len(comps)} resident {size}^3 f32 k^-5/3 GRFs (rel eb 1e-3); "
                       "Poisson requests, box edge U[16,256] per axis, level U{1,2,3}",
           "resident_gb": round(resident / 1e9, 3), "raw_gb": round(raw / 1e9, 3),
           "slots": srv.nslots, "batch": {"max_batch": bsrv.max_batch, "inflight": bsrv.nbatch},
           "budget_gb": round(budget / 1e9, 2), "per_rate": per_rate}
    del srv, srv1, bsrv, comps, ws, reg_out
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------- further timed workloads
def _time_ms(fn, reps=5, warm=2):
    """Median device time of fn() over `reps` calls (CUDA events on the
    current stream, after `warm` untimed calls)."""
    import torch

    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def _psnr(x, y) -> float:
    """20 log10(max - min) - 10 log10(MSE), in float64 (the paper uses PSNR
    without defining it)."""
    import torch

    xd = x.double()
    mse = float(((xd - y.double()) ** 2).mean())
    rng = float(xd.max() - xd.min())
    return float("inf") if mse == 0 else 20 * np.log10(rng) - 10 * np.log10(mse)


def run_bounds(args, dev, field, peak):
    """The 512^3 field at every relative bound of its workload: compress and
    full-decode rates, compression ratio, PSNR and the largest error."""
    import torch

    from paper_2509_01626_gb300 import stz

    shape = tuple(field.shape)
    ws = stz.alloc_workspace(shape, torch.float32, dev)
    out = torch.empty(stz.compress_bound(shape, torch.float32), dtype=torch.uint8, device=dev)
    full = torch.empty_like(field)
    fb = field.numel() * 4
    meta = {"shape": shape, "dtype": torch.float32, "ndim": 3, "levels": 3}
    rows = []
    for eb in (1e-2, 1e-3, 1e-4, 1e-5):
        comp = stz.compress(field, eb, "rel", out=out, workspace=ws)
        cms = _time_ms(lambda: stz.compress(field, eb, "rel", out=out, workspace=ws))
        dms = _time_ms(lambda: stz.decompress_full(comp, out=full, workspace=ws, meta=meta))
        y = stz.decompress_full(comp, out=full, workspace=ws, meta=meta)
        ea = stz.info(comp)["eb_abs"]
        err = float((y.double() - field.double()).abs().max())
        rows.append({"eb": eb, "compress_gbs": round(fb / cms / 1e6, 1),
                     "decompress_gbs": round(fb / dms / 1e6, 1),
                     "compress_frac": round(fb / cms / 1e6 / peak, 4),
                     "decompress_frac": round(fb / dms / 1e6 / peak, 4),
                     "cr": round(fb / comp.numel(), 3), "psnr_db": round(_psnr(field, y), 2),
                     "max_err_over_eb": round(err / ea, 4)})
    del ws, out, full
    torch.cuda.empty_cache()
    return rows


def run_large(args, dev, peak):
    """1024^3 f32 k^-5/3 turbulence-like field and 768^3 f64 smooth field at
    relative bound 1e-4: compress, full decode and decode to each progressive
    level; the f32 field also with four levels (Sec. 3.2)."""
    import torch

    from paper_2509_01626_gb300 import stz, synth

    out_rows = []
    cases = [("1024^3 f32 GRF k^-5/3", lambda: synth.grf(
                 (1024,) * 3, synth.seed_for(4, 0), slope=-5.0 / 3.0, lognormal_sigma=None,
                 dtype=np.float32, device=str(dev), white_source="torch", as_tensor=True), (3, 4)),
             ("768^3 f64 smooth", lambda: synth.sinusoids_device(
                 (768,) * 3, synth.seed_for(4, 1), n_terms=4, fmin=1.0, fmax=3.0, noise=0.0,
                 dtype=np.float64, device=str(dev)), (3,))]
    for name, gen, levels in cases:
        x = gen()
        shape = tuple(x.shape)
        fb = x.numel() * x.element_size()
        for L in levels:
            ws = stz.alloc_workspace(shape, x.dtype, dev, L)
            out = torch.empty(stz.compress_bound(shape, x.dtype, L), dtype=torch.uint8,
                              device=dev)
            full = torch.empty_like(x)
            comp = stz.compress(x, 1e-4, "rel", out=out, workspace=ws, levels=L)
            meta = {"shape": shape, "dtype": x.dtype, "ndim": 3, "levels": L}
            cms = _time_ms(lambda: stz.compress(x, 1e-4, "rel", out=out, workspace=ws, levels=L),
                           reps=3)
            dms = _time_ms(lambda: stz.decompress_full(comp, out=full, workspace=ws, meta=meta),
                           reps=3)
            prog = {}
            for k in range(1, L):
                pk = torch.empty(x.numel() // (8 ** (L - k)) + 8 ** L, dtype=x.dtype, device=dev)
                prog[str(k)] = round(_time_ms(lambda: stz.decompress_progressive(
                    comp, k, out=pk, workspace=ws, meta=meta), reps=3), 4)
                del pk
            out_rows.append({"field": name, "levels": L, "eb": 1e-4,
                             "compress_ms": round(cms, 3), "decompress_ms": round(dms, 3),
                             "compress_gbs": round(fb / cms / 1e6, 1),
                             "decompress_gbs": round(fb / dms / 1e6, 1),
                             "compress_frac": round(fb / cms / 1e6 / peak, 4),
                             "decompress_frac": round(fb / dms / 1e6 / peak, 4),
                             "progressive_ms": prog, "cr": round(fb / comp.numel(), 3)})
            del ws, out, full, comp
            torch.cuda.empty_cache()
        del x
        torch.cuda.empty_cache()
    return out_rows


# the rate-distortion ablation of Sec. 3.1 (Fig. 2), in the paper's order; the
# partition-only baseline (sub-blocks coded independently by SZ3) is not built
ABLATION = [("direct prediction (opt. 1)", "direct", 2, 1.0),
            ("multi-dim linear + quantize only (opts. 2-3)", "linear", 2, 1.0),
            ("cubic multi-dim (opt. 4)", "cubic", 2, 1.0),
            ("cubic + adaptive bound 2.5 (opt. 5)", "cubic", 2, 2.5),
            ("3 levels + all (Sec. 3.2)", "cubic", 3, 2.5)]


def run_ablation(args, dev, field512):
    """Compression ratio and PSNR of each step of the Sec. 3.1 ablation on the
    128^3 sinusoid field and the 512^3 log-normal GRF, at three bounds."""
    import torch

    from paper_2509_01626_gb300 import stz, synth

    fields = [("128^3 f32 sinusoids", torch.from_numpy(
                  synth.sinusoids((128,) * 3, synth.seed_for(1))).to(dev)),
              ("512^3 f32 log-normal GRF", field512)]
    rows = []
    for fname, x in fields:
        shape = tuple(x.shape)
        fb = x.numel() * 4
        for label, pred, L, ratio in ABLATION:
            ws = stz.alloc_workspace(shape, torch.float32, dev, L)
            out = torch.empty(stz.compress_bound(shape, torch.float32, L), dtype=torch.uint8,
                              device=dev)
            full = torch.empty_like(x)
            for eb in (1e-2, 1e-3, 1e-4):
                comp = stz.compress(x, eb, "rel", out=out, workspace=ws, levels=L,
                                    predictor=pred, eb_ratio=ratio)
                y = stz.decompress_full(comp, out=full, workspace=ws)
                rows.append({"field": fname, "step": label, "predictor": pred, "levels": L,
                             "eb_ratio": ratio, "eb": eb, "cr": round(fb / comp.numel(), 3),
                             "psnr_db": round(_psnr(x, y), 2)})
            del ws, out, full
            torch.cuda.empty_cache()
    return rows


# --------------------------------------------------------------- oracle arm
def oracle_step(ora, x, eb):
    """One pass of the hot path with the CPU oracle over field x."""
    size = x.shape[0]
    c = ora.compress(x, eb, "rel")
    ora.decompress(c)
    for k in (1, 2):
        ora.decompress(c, k)
    (blo, bhi), (slo, shi) = step_boxes(size)
    ora.decompress_region(c, blo, bhi, 3)
    ora.decompress_region(c, slo, shi, 3)
    return c


def oracle_sample(x, edge):
    s = min(edge, x.shape[0])
    return np.ascontiguousarray(x[:s, :s, :s])


def run_cpu_baseline(x, eb, edge=512):
    """One step of the oracle, single-threaded, on the bench's own field (the
    whole 512^3 field: about 20 s of CPU work)."""
    from oracle import oracle as ora

    ora.build()
    xs = oracle_sample(x, edge)
    t = time.perf_counter()
    oracle_step(ora, xs, eb)
    dt = time.perf_counter() - t
    whole = xs.shape[0] == x.shape[0]
    return {"value": round(xs.nbytes / dt / 1e9, 5), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "one step (compress, full, progressive 1-2, 64^3 box, slice) on "
                      + ("the whole field" if whole else f"the {xs.shape[0]}^3 corner of the field")
                      + ", single thread",
            "seconds": round(dt, 3)}


def run_reference(args):
    import platform

    from oracle import oracle as ora
    from paper_2509_01626_gb300 import synth

    ora.build()
    edge = min(256, args.size)
    x = synth.grf((args.size,) * 3, synth.seed_for(2, 0), device="cpu")
    xs = oracle_sample(x, edge)
    for _ in range(max(args.warmup, 0)):
        oracle_step(ora, xs, args.eb)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(ora, xs, args.eb)
    dt = (time.perf_counter() - t) / max(args.steps, 1)
    val = round(xs.nbytes / dt / 1e9, 5)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": val, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"{edge}^3 corner of the field per step, single thread",
                         "host": platform.machine()},
        "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args):
    s = args.size
    return {"workload": f"{s}^3 f32 log-normal Gaussian random field (k^-3 spectrum, "
                        f"sigma 1.5), rel eb {args.eb:g}, L=3",
            "field_shape": [s, s, s], "eb": args.eb, "eb_mode": "rel", "levels": 3,
            "step": "compress + full decompress + progressive(1,2) + 64^3 box + 512^2 slice",
            "l2_policy": "inputs larger than L2 (512 MiB field per step)",
            "parallelism": "independent fields per GPU"}


# ---------------------------------------------------------------------- main
def main():
    args = parse_args()
    if args.write_traffic:
        write_traffic(*args.write_traffic)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    import torch

    from paper_2509_01626_gb300 import build as libbuild

    if world > 1:
        import torch.distributed as tdist

        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
        if rank == 0:
            libbuild.build()
        tdist.barrier()
    else:
        libbuild.build()
    r = run_ours(args, rank, world, local_rank)
    peak, peak_kind = load_peaks()
    fb = r["field_bytes"]
    value = world * fb / (r["ms_step"] * 1e-3) / 1e9
    op = r["op_ms"]
    kern = r["kernels"]
    breakdown = []
    total_ms = sum(v[1] for v in kern.values()) or 1.0
    for name, (cnt, ms, nbytes) in sorted(kern.items(), key=lambda kv: -kv[1][1]):
        e = {"kernel": name, "launches_per_step": round(cnt / args.steps, 2),
             "ms_per_step": round(ms / args.steps, 4), "share": round(ms / total_ms, 4)}
        if nbytes > 0 and ms > 0:
            e["achieved_gbs"] = round(nbytes / (ms * 1e-3) / 1e9, 1)
        breakdown.append(e)
    # the dominant kernel with an algorithmic-byte figure: achieved = its
    # bytes over all timed launches / its summed launch time
    roofline = None
    cand = [b for b in breakdown if "achieved_gbs" in b]
    if cand:
        top = cand[0]
        cnt, ms, nbytes = kern[top["kernel"]]
        ach = nbytes / (ms * 1e-3) / 1e9
        ratio = traffic_ratio(top["kernel"])
        roofline = {"kernel": top["kernel"], "bound": "hbm", "achieved": round(ach, 1),
                    "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                    "peak_source": f"{peak_kind} HBM copy bandwidth",
                    "traffic": None if ratio is None else int(ratio * nbytes / cnt),
                    "algorithmic_bytes_per_launch": int(nbytes / cnt),
                    "launches_per_step": round(cnt / args.steps, 2)}
    # the metric's own figures: each operation's input GB/s against the peak
    op_rates = {}
    for name, ms in (("compress", op[0]), ("decompress_full", op[1])):
        gbs = fb / (ms * 1e-3) / 1e9
        op_rates[name] = {"gbs": round(gbs, 2), "ms": round(float(ms), 4),
                          "frac_of_hbm": round(gbs / peak, 4)}
    op_rates["progressive_levels_1_2_ms"] = round(float(op[2]), 4)
    op_rates["box_64cube_ms"] = round(float(op[3]), 4)
    op_rates["slice_512sq_ms"] = round(float(op[4]), 4)
    op_rates["region_p99_ms"] = round(float(np.percentile(r["lat"], 99)), 4)
    if roofline is not None:
        roofline["ops"] = op_rates
    dev = torch.device("cuda", local_rank)
    bounds = large = ablation = None
    if rank == 0 and not (args.no_bounds and args.no_ablation):
        field = torch.from_numpy(r["x_host"]).to(dev)
        bounds = None if args.no_bounds else run_bounds(args, dev, field, peak)
        ablation = None if args.no_ablation else run_ablation(args, dev, field)
        del field
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_large and args.size >= 512:
        large = run_large(args, dev, peak)
    batched = None if args.no_batch else run_batched(args, dev)
    served = None if args.no_serve else run_served(args, dev)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(r["x_host"], args.eb)
    if rank != 0:
        return
    lat = r["lat"]
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(r["ms_step"], 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": workload_config(args),
        "compress_gbs": round(fb / (op[0] * 1e-3) / 1e9, 2),
        "decompress_gbs": round(fb / (op[1] * 1e-3) / 1e9, 2),
        "compress_frac_of_hbm": round(fb / (op[0] * 1e-3) / 1e9 / peak, 4),
        "decompress_frac_of_hbm": round(fb / (op[1] * 1e-3) / 1e9 / peak, 4),
        "progressive_ms_levels_1_2": round(float(op[2]), 4),
        "box_ms": round(float(op[3]), 4),
        "slice_ms": round(float(op[4]), 4),
        "region_latency_ms": {"p50": round(float(np.percentile(lat, 50)), 4),
                              "p99": round(float(np.percentile(lat, 99)), 4),
                              "n": int(lat.size), "edges": "16-256", "levels": "1-3"},
        "compression_ratio": round(fb / r["comp_bytes"], 3),
        "roi": r["roi"],
        "roofline": roofline, "cpu_baseline": cpu, "e2e": r["e2e"],
        "gpu_launches": int(r["launches"]), "clocks": r["clk"], "kernels": breakdown[:24],
        "bounds": bounds, "large": large, "ablation": ablation,
        "batched": batched, "served": served,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
