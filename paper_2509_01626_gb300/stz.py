"""Python binding of the C ABI in include/stz.h (libstz.so).

Argument marshalling only: every step of compression and decompression runs
in the library's CUDA kernels.  torch supplies device memory and the current
CUDA stream.  If the library is not built, importing the functions raises
-- there is no CPU fallback.

Shapes are C order, slowest first: (nz, ny, nx) or (ny, nx).  Boxes are
half-open [lo, hi) in the same axis order.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libstz.so")

F32, F64 = 0, 1
EB_ABS, EB_REL = 0, 1
OK, ERR_ARG, ERR_CAPACITY, ERR_CORRUPT, ERR_CUDA, ERR_TIMEOUT, ERR_NOMEM = 0, -1, -2, -3, -4, -5, -6


class StzError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class _Info(ctypes.Structure):
    _fields_ = [
        ("dtype", ctypes.c_int),
        ("ndim", ctypes.c_int),
        ("dims", ctypes.c_int64 * 3),
        ("levels", ctypes.c_int),
        ("eb", ctypes.c_double),
        ("eb_mode", ctypes.c_int),
        ("eb_abs", ctypes.c_double),
        ("total_bytes", ctypes.c_uint64),
    ]


class FieldJob(ctypes.Structure):
    """stz_field_job: one field of a stz_compress_batch call."""
    _fields_ = [
        ("field_dev", ctypes.c_void_p),
        ("dims", ctypes.c_int64 * 3),
        ("ndim", ctypes.c_int),
        ("dtype", ctypes.c_int),
        ("eb_mode", ctypes.c_int),
        ("eb", ctypes.c_double),
        ("out_dev", ctypes.c_void_p),
        ("out_cap", ctypes.c_size_t),
        ("ws_dev", ctypes.c_void_p),
        ("ws_bytes", ctypes.c_size_t),
    ]


class CompressOpts(ctypes.Structure):
    """stz_compress_opts: level count, predictor, adaptive-bound ratio."""
    _fields_ = [("levels", ctypes.c_int), ("predictor", ctypes.c_int),
                ("eb_ratio", ctypes.c_double)]


# predictors of levels 2..L (Sec. 3.1 ablation): opt. 4 cubic (the method),
# opt. 2 multi-linear, opt. 1 direct
PREDICTORS = {"cubic": 0, "linear": 1, "direct": 2}


class BatchOpts(ctypes.Structure):
    """stz_batch_opts: launch arrangement of a batch (never changes bytes).
    persistent = 1 runs the level stages of the 3D fields in one work-queue
    launch per dtype (schedule, tiles_per_item, blocks_per_sm), with the
    batch workspace ws_dev / ws_bytes."""
    _fields_ = [("lanes", ctypes.c_int), ("sm_share_den", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("persistent", ctypes.c_int),
                ("schedule", ctypes.c_int), ("tiles_per_item", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("ws_dev", ctypes.c_void_p),
                ("ws_bytes", ctypes.c_size_t)]


class ServedField(ctypes.Structure):
    """stz_served_field: a resident container with its cached level-1 grid
    and decode tables."""
    _fields_ = [("comp_dev", ctypes.c_void_p), ("comp_bytes", ctypes.c_size_t),
                ("hdr_host", ctypes.c_void_p), ("hdr_bytes", ctypes.c_size_t),
                ("level1_dev", ctypes.c_void_p), ("tables_dev", ctypes.c_void_p)]


class RegionRequest(ctypes.Structure):
    """stz_region_request: one box of a batched decode."""
    _fields_ = [("field", ctypes.c_int), ("level", ctypes.c_int),
                ("lo", ctypes.c_int64 * 3), ("hi", ctypes.c_int64 * 3),
                ("out_dev", ctypes.c_void_p), ("out_cap", ctypes.c_size_t),
                ("out_dims", ctypes.c_int64 * 3)]


class _KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_ulonglong),
                ("total_ms", ctypes.c_double), ("algo_bytes", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libstz.so (build it with paper_2509_01626_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libstz.so is not built ({LIB_PATH}); run "
                              "`python -m paper_2509_01626_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, sz, i64p = ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int64)
        L.stz_strerror.restype = ctypes.c_char_p
        L.stz_strerror.argtypes = [ctypes.c_int]
        L.stz_version.restype = ctypes.c_char_p
        L.stz_compress_bound.restype = sz
        L.stz_compress_bound.argtypes = [i64p, ctypes.c_int, ctypes.c_int]
        L.stz_workspace_size.restype = sz
        L.stz_workspace_size.argtypes = [i64p, ctypes.c_int, ctypes.c_int]
        L.stz_compress.argtypes = [vp, i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double, vp, sz, ctypes.POINTER(sz), vp, sz, vp]
        L.stz_compress_ex.argtypes = [vp, i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.POINTER(CompressOpts), vp, sz,
                                      ctypes.POINTER(sz), vp, sz, vp]
        L.stz_compress_bound_ex.restype = sz
        L.stz_compress_bound_ex.argtypes = [i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.stz_workspace_size_ex.restype = sz
        L.stz_workspace_size_ex.argtypes = [i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.stz_info.argtypes = [vp, sz, ctypes.c_int, ctypes.POINTER(_Info)]
        L.stz_decompress_full.argtypes = [vp, sz, vp, sz, vp, sz, vp]
        L.stz_decompress_progressive.argtypes = [vp, sz, ctypes.c_int, vp, sz, i64p, vp, sz, vp]
        L.stz_decompress_region.argtypes = [vp, sz, i64p, i64p, ctypes.c_int, vp, sz, i64p, vp,
                                            sz, vp]
        L.stz_decompress_region_noalloc.argtypes = [vp, sz, i64p, i64p, ctypes.c_int, vp, sz,
                                                    i64p, vp]
        L.stz_compress_batch.argtypes = [ctypes.c_int, ctypes.POINTER(FieldJob), vp,
                                         ctypes.POINTER(BatchOpts), vp]
        L.stz_compress_batch_workspace_size.restype = sz
        L.stz_compress_batch_workspace_size.argtypes = [ctypes.c_int, ctypes.POINTER(FieldJob)]
        L.stz_region_workspace_size.restype = sz
        L.stz_region_workspace_size.argtypes = [vp, sz, sz, i64p, i64p, ctypes.c_int,
                                                ctypes.c_int]
        L.stz_region_chunks.argtypes = [vp, sz, sz, i64p, i64p, ctypes.c_int, ctypes.c_int,
                                         i64p, ctypes.c_int]
        L.stz_roi_units.restype = ctypes.c_int64
        L.stz_roi_units.argtypes = [i64p, ctypes.c_int, i64p]
        L.stz_roi_workspace_size.restype = sz
        L.stz_roi_workspace_size.argtypes = [i64p, ctypes.c_int, i64p]
        L.stz_roi_select.argtypes = [vp, i64p, ctypes.c_int, ctypes.c_int, i64p, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_double, vp, sz, vp, i64p, vp, sz, vp]
        L.stz_decompress_region_async.argtypes = [vp, sz, vp, sz, vp, i64p, i64p, ctypes.c_int,
                                                  vp, sz, i64p, vp, sz, vp, vp]
        L.stz_decode_tables_size.restype = sz
        L.stz_decode_tables_size.argtypes = [vp, sz, sz]
        L.stz_decode_tables.argtypes = [vp, sz, vp, sz, vp, sz, vp]
        L.stz_decode_requests_workspace.restype = sz
        L.stz_decode_requests_workspace.argtypes = [ctypes.c_int, ctypes.POINTER(RegionRequest),
                                                    ctypes.POINTER(ServedField), ctypes.c_int]
        L.stz_decode_requests.argtypes = [ctypes.c_int, ctypes.POINTER(RegionRequest),
                                          ctypes.POINTER(ServedField), ctypes.c_int, vp, sz, vp,
                                          vp]
        L.stz_launch_count.restype = ctypes.c_ulonglong
        L.stz_profile_enable.argtypes = [ctypes.c_int]
        L.stz_profile_read.argtypes = [ctypes.POINTER(_KernelTime), ctypes.c_int]
        _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().stz_strerror(int(code)).decode()
    except ImportError:
        return str(code)


def version() -> str:
    return lib().stz_version().decode()


def _i64(vals):
    vals = list(vals) + [0] * (3 - len(vals))
    return (ctypes.c_int64 * 3)(*[int(v) for v in vals])


def _dt(dtype) -> int:
    if dtype in (torch.float32, "float32"):
        return F32
    if dtype in (torch.float64, "float64"):
        return F64
    raise TypeError(f"unsupported dtype {dtype}")


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc: int, what: str):
    if rc != OK:
        raise StzError(rc, what)


def compress_bound(shape, dtype, levels: int = 3) -> int:
    return int(lib().stz_compress_bound_ex(_i64(shape), len(shape), _dt(dtype), int(levels)))


def workspace_size(shape, dtype, levels: int = 3) -> int:
    return int(lib().stz_workspace_size_ex(_i64(shape), len(shape), _dt(dtype), int(levels)))


def alloc_workspace(shape, dtype, device=None, levels: int = 3) -> torch.Tensor:
    return torch.empty(workspace_size(shape, dtype, levels), dtype=torch.uint8,
                       device=device or torch.device("cuda"))


def compress(field: torch.Tensor, eb: float, mode: str = "rel", out: torch.Tensor | None = None,
             workspace: torch.Tensor | None = None, stream=None, levels: int = 3,
             predictor: str = "cubic", eb_ratio: float = 2.5) -> torch.Tensor:
    """stz_compress (stz_compress_ex for other levels / predictors / bound
    ratios): returns the container as a uint8 view of `out`."""
    if not field.is_cuda or not field.is_contiguous():
        raise ValueError("field must be a contiguous CUDA tensor")
    shape = tuple(field.shape)
    dt = _dt(field.dtype)
    if out is None:
        out = torch.empty(compress_bound(shape, field.dtype, levels), dtype=torch.uint8,
                          device=field.device)
    if workspace is None:
        workspace = alloc_workspace(shape, field.dtype, field.device, levels)
    nbytes = ctypes.c_size_t(0)
    args = (ctypes.c_void_p(field.data_ptr()), _i64(shape), len(shape), dt,
            EB_REL if mode == "rel" else EB_ABS, float(eb))
    rest = (ctypes.c_void_p(out.data_ptr()), out.numel(), ctypes.byref(nbytes),
            ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), _stream(stream))
    if levels == 3 and predictor == "cubic" and eb_ratio == 2.5:
        rc = lib().stz_compress(*args, *rest)
        _check(rc, "stz_compress")
    else:
        opts = CompressOpts(int(levels), PREDICTORS[predictor], float(eb_ratio))
        rc = lib().stz_compress_ex(*args, ctypes.byref(opts), *rest)
        _check(rc, "stz_compress_ex")
    return out[: nbytes.value]


def compress_batch(jobs, sizes_dev: torch.Tensor, opts: BatchOpts | None = None,
                   stream=None) -> None:
    """stz_compress_batch over a ctypes array of FieldJob; asynchronous.
    sizes_dev: int64 CUDA tensor of len(jobs) entries receiving the sizes
    (bit 63 set: that field's out_cap was too small)."""
    if sizes_dev.dtype != torch.int64 or not sizes_dev.is_cuda or sizes_dev.numel() < len(jobs):
        raise ValueError("sizes_dev must be an int64 CUDA tensor with one entry per job")
    rc = lib().stz_compress_batch(len(jobs), jobs, ctypes.c_void_p(sizes_dev.data_ptr()),
                                  ctypes.byref(opts) if opts is not None else None,
                                  _stream(stream))
    _check(rc, "stz_compress_batch")


def compress_batch_workspace_size(jobs) -> int:
    """stz_compress_batch_workspace_size: bytes of the work-queue
    arrangement's batch workspace for these jobs."""
    return int(lib().stz_compress_batch_workspace_size(len(jobs), jobs))


def info(comp: torch.Tensor) -> dict:
    inf = _Info()
    on_dev = 1 if comp.is_cuda else 0
    rc = lib().stz_info(ctypes.c_void_p(comp.data_ptr()), comp.numel(), on_dev, ctypes.byref(inf))
    if rc not in (OK, ERR_ARG):
        _check(rc, "stz_info")
    shape = tuple(inf.dims[:3]) if inf.ndim == 3 else tuple(inf.dims[:2])
    return {
        "dtype": torch.float32 if inf.dtype == F32 else torch.float64,
        "ndim": inf.ndim,
        "shape": shape,
        "levels": inf.levels,
        "eb": inf.eb,
        "eb_mode": "rel" if inf.eb_mode == EB_REL else "abs",
        "eb_abs": inf.eb_abs,
        "total_bytes": int(inf.total_bytes),
        "supported": rc == OK,
    }


def _shape_out(od, ndim):
    return (int(od[0]), int(od[1]), int(od[2])) if ndim == 3 else (int(od[0]), int(od[1]))


def decompress_full(comp: torch.Tensor, out: torch.Tensor | None = None,
                    workspace: torch.Tensor | None = None, stream=None,
                    meta: dict | None = None) -> torch.Tensor:
    """stz_decompress_full; `meta` (from info()) skips reading the header here."""
    inf = meta or info(comp)
    if out is None:
        out = torch.empty(inf["shape"], dtype=inf["dtype"], device=comp.device)
    if workspace is None:
        workspace = alloc_workspace(inf["shape"], inf["dtype"], comp.device, inf["levels"])
    rc = lib().stz_decompress_full(ctypes.c_void_p(comp.data_ptr()), comp.numel(),
                                   ctypes.c_void_p(out.data_ptr()),
                                   out.numel() * out.element_size(),
                                   ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                   _stream(stream))
    _check(rc, "stz_decompress_full")
    return out.view(inf["shape"])


def decompress_progressive(comp: torch.Tensor, level: int, out: torch.Tensor | None = None,
                           workspace: torch.Tensor | None = None, stream=None,
                           meta: dict | None = None) -> torch.Tensor:
    inf = meta or info(comp)
    s = 1 << (inf["levels"] - level) if 1 <= level <= inf["levels"] else 1
    shape = tuple(-(-d // s) for d in inf["shape"])
    if out is None:
        out = torch.empty(shape, dtype=inf["dtype"], device=comp.device)
    if workspace is None:
        workspace = alloc_workspace(inf["shape"], inf["dtype"], comp.device, inf["levels"])
    od = (ctypes.c_int64 * 3)()
    rc = lib().stz_decompress_progressive(ctypes.c_void_p(comp.data_ptr()), comp.numel(),
                                          int(level), ctypes.c_void_p(out.data_ptr()),
                                          out.numel() * out.element_size(), od,
                                          ctypes.c_void_p(workspace.data_ptr()),
                                          workspace.numel(), _stream(stream))
    _check(rc, "stz_decompress_progressive")
    oshape = _shape_out(od, inf["ndim"])
    return out.reshape(-1)[: int(torch.tensor(oshape).prod())].view(oshape)


def decompress_region(comp: torch.Tensor, lo, hi, level: int | None = None,
                      out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                      stream=None, meta: dict | None = None) -> torch.Tensor:
    inf = meta or info(comp)
    if level is None:
        level = inf["levels"]
    if out is not None and (out.dtype != inf["dtype"] or out.device != comp.device
                            or not out.is_contiguous()):
        raise ValueError("out must be a contiguous tensor of the container's dtype on its device")
    if out is None:
        n = 1
        for a, b in zip(lo, hi):
            n *= max(1, b - a)
        out = torch.empty(n, dtype=inf["dtype"], device=comp.device)
    if workspace is None:
        workspace = alloc_workspace(inf["shape"], inf["dtype"], comp.device, inf["levels"])
    od = (ctypes.c_int64 * 3)()
    rc = lib().stz_decompress_region(ctypes.c_void_p(comp.data_ptr()), comp.numel(), _i64(lo),
                                     _i64(hi), int(level), ctypes.c_void_p(out.data_ptr()),
                                     out.numel() * out.element_size(), od,
                                     ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                     _stream(stream))
    _check(rc, "stz_decompress_region")
    oshape = _shape_out(od, inf["ndim"])
    n = 1
    for v in oshape:
        n *= v
    return out.reshape(-1)[:n].view(oshape)


# Scratch bytes of decompress_region_noalloc (STZ_NOALLOC_SCRATCH_BYTES).
NOALLOC_SCRATCH_BYTES = 32 << 20


def decompress_region_noalloc(comp: torch.Tensor, lo, hi, level: int, out: torch.Tensor,
                              stream=None, meta: dict | None = None) -> torch.Tensor:
    """stz_decompress_region_noalloc: like decompress_region, but the library
    allocates nothing and takes no workspace -- its scratch is a fixed array
    in the library's device memory.  For callers that cannot allocate device
    memory when they decode; `out` must be given.  Calls share that array,
    so issue them on one stream."""
    inf = meta or info(comp)
    if out.dtype != inf["dtype"] or out.device != comp.device or not out.is_contiguous():
        raise ValueError("out must be a contiguous tensor of the container's dtype on its device")
    od = (ctypes.c_int64 * 3)()
    # the library looks up its scratch array on the current device
    with torch.cuda.device(comp.device):
        rc = lib().stz_decompress_region_noalloc(ctypes.c_void_p(comp.data_ptr()), comp.numel(),
                                                 _i64(lo), _i64(hi), int(level),
                                                 ctypes.c_void_p(out.data_ptr()),
                                                 out.numel() * out.element_size(), od,
                                                 _stream(stream))
    _check(rc, "stz_decompress_region_noalloc")
    oshape = _shape_out(od, inf["ndim"])
    n = 1
    for v in oshape:
        n *= v
    return out.reshape(-1)[:n].view(oshape)


ROI_METRICS = {"range": 0, "max": 1}
ROI_MODES = {"threshold": 0, "top": 1}


def roi_select(field: torch.Tensor, block, metric: str = "range", mode: str = "top",
               value: float = 0.01, metric_out: bool = False, stream=None):
    """stz_roi_select (Sec. 3.3 ROI module): the selected unit indices
    (ascending, int64 CUDA tensor) and, with metric_out, every unit's
    metric (float64 CUDA tensor).  block: (bz, by, bx), or (by, bx) for 2D."""
    if not field.is_cuda or not field.is_contiguous():
        raise ValueError("field must be a contiguous CUDA tensor")
    shape = tuple(field.shape)
    nd = len(shape)
    nu = int(lib().stz_roi_units(_i64(shape), nd, _i64(block)))
    if nu < 1:
        raise StzError(ERR_ARG, "stz_roi_units")
    ws = torch.empty(lib().stz_roi_workspace_size(_i64(shape), nd, _i64(block)),
                     dtype=torch.uint8, device=field.device)
    sel = torch.empty(nu, dtype=torch.int64, device=field.device)
    met = torch.empty(nu, dtype=torch.float64, device=field.device) if metric_out else None
    ns = ctypes.c_int64(0)
    rc = lib().stz_roi_select(ctypes.c_void_p(field.data_ptr()), _i64(shape), nd,
                              _dt(field.dtype), _i64(block), ROI_METRICS[metric], ROI_MODES[mode],
                              float(value), ctypes.c_void_p(sel.data_ptr()), nu,
                              ctypes.c_void_p(met.data_ptr()) if met is not None else None,
                              ctypes.byref(ns), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                              _stream(stream))
    _check(rc, "stz_roi_select")
    return (sel[: ns.value], met) if metric_out else sel[: ns.value]


def roi_boxes(units, grid_shape, block, stride: int = 1, field_shape=None):
    """Boxes [lo, hi) in field coordinates of ROI units chosen on a grid of
    shape grid_shape that samples the field every `stride` points (the
    output of a progressive decode); each box covers its unit's grid points
    and the field points between them."""
    nb = [-(-g // b) for g, b in zip(grid_shape, block)]
    field_shape = field_shape or tuple(g * stride for g in grid_shape)
    boxes = []
    for u in (int(v) for v in units):
        idx = []
        for n in reversed(nb):
            idx.append(u % n)
            u //= n
        idx = idx[::-1]
        lo = tuple(i * b * stride for i, b in zip(idx, block))
        hi = tuple(min(min((i + 1) * b, g) * stride, f)
                   for i, b, g, f in zip(idx, block, grid_shape, field_shape))
        boxes.append((lo, hi))
    return boxes


HEADER_MAX_BYTES = 1984  # STZ_HEADER_MAX_BYTES


def header_bytes(comp: torch.Tensor) -> bytes:
    """Host copy of a container's header and directory (one read)."""
    n = min(comp.numel(), HEADER_MAX_BYTES)
    return bytes(comp[:n].cpu().numpy().tobytes())


def region_workspace_size(hdr: bytes, comp_bytes: int, lo, hi, level: int,
                          level1_given: bool) -> int:
    return int(lib().stz_region_workspace_size(hdr, len(hdr), int(comp_bytes), _i64(lo), _i64(hi),
                                               int(level), 1 if level1_given else 0))


def region_chunks(hdr: bytes, comp_bytes: int, lo, hi, level: int,
                  level1_given: bool = False) -> list[int]:
    """stz_region_chunks (host only): per stream, the chunks a region decode
    of [lo, hi) at `level` entropy-decodes."""
    buf = (ctypes.c_int64 * 64)()
    n = lib().stz_region_chunks(hdr, len(hdr), int(comp_bytes), _i64(lo), _i64(hi), int(level),
                                1 if level1_given else 0, buf, 64)
    if n < 0:
        _check(n, "stz_region_chunks")
    return [int(buf[i]) for i in range(n)]


def decompress_region_async(comp: torch.Tensor, hdr: bytes, lo, hi, level: int,
                            out: torch.Tensor, workspace: torch.Tensor, status: torch.Tensor,
                            level1: torch.Tensor | None = None, stream=None):
    """stz_decompress_region_async: queues the decode on `stream` and returns
    the output shape (slowest first) without waiting; `status` (int32 CUDA
    tensor, one entry) becomes nonzero if the container proved corrupt."""
    od = (ctypes.c_int64 * 3)()
    rc = lib().stz_decompress_region_async(
        ctypes.c_void_p(comp.data_ptr()), comp.numel(), hdr, len(hdr),
        ctypes.c_void_p(level1.data_ptr()) if level1 is not None else None,
        _i64(lo), _i64(hi), int(level), ctypes.c_void_p(out.data_ptr()),
        out.numel() * out.element_size(), od, ctypes.c_void_p(workspace.data_ptr()),
        workspace.numel(), ctypes.c_void_p(status.data_ptr()), _stream(stream))
    _check(rc, "stz_decompress_region_async")
    return tuple(int(v) for v in od[: len(lo)])


def decode_tables(comp: torch.Tensor, hdr: bytes, stream=None) -> torch.Tensor:
    """stz_decode_tables: the container's decode tables (uint8 CUDA tensor),
    built once per resident field for stz_decode_requests."""
    n = int(lib().stz_decode_tables_size(hdr, len(hdr), comp.numel()))
    if n == 0:
        raise StzError(ERR_CORRUPT, "stz_decode_tables_size")
    t = torch.empty(n, dtype=torch.uint8, device=comp.device)
    rc = lib().stz_decode_tables(ctypes.c_void_p(comp.data_ptr()), comp.numel(), hdr, len(hdr),
                                 ctypes.c_void_p(t.data_ptr()), n, _stream(stream))
    _check(rc, "stz_decode_tables")
    return t


def served_fields(entries):
    """ctypes array of ServedField from (comp, hdr bytes, level1, tables)
    tuples; the caller keeps the tensors and the bytes alive."""
    arr = (ServedField * len(entries))()
    for f, (comp, hdr, level1, tables) in zip(arr, entries):
        f.comp_dev = comp.data_ptr()
        f.comp_bytes = comp.numel()
        f.hdr_host = ctypes.cast(ctypes.c_char_p(hdr), ctypes.c_void_p).value
        f.hdr_bytes = len(hdr)
        f.level1_dev = level1.data_ptr()
        f.tables_dev = tables.data_ptr()
    return arr


def decode_requests_workspace(reqs, fields) -> int:
    return int(lib().stz_decode_requests_workspace(len(reqs), reqs, fields, len(fields)))


def decode_requests(reqs, fields, workspace: torch.Tensor, status: torch.Tensor,
                    stream=None) -> None:
    """stz_decode_requests: decode every request of the ctypes RegionRequest
    array `reqs` in a fixed number of launches, without waiting; `status`
    (int32 CUDA tensor, one entry per request) receives each request's
    status, and reqs[i].out_dims its output shape."""
    rc = lib().stz_decode_requests(len(reqs), reqs, fields, len(fields),
                                   ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                   ctypes.c_void_p(status.data_ptr()), _stream(stream))
    _check(rc, "stz_decode_requests")


def decode_regions(comp: torch.Tensor, boxes, level: int | None = None,
                   level1: torch.Tensor | None = None, tables: torch.Tensor | None = None,
                   hdr: bytes | None = None, stream=None, meta: dict | None = None,
                   check: bool = True):
    """Decode many boxes [lo, hi) of one container with a single
    stz_decode_requests call: a fixed number of kernel launches however many
    boxes there are.  Each returned tensor equals decompress_region of its
    box bit for bit.  `level1` (decompress_progressive at level 1) and
    `tables` (decode_tables) are built here unless given.  With check=True
    the call waits and raises StzError if any box's decode reported a
    corrupt container; with check=False it returns (outputs, status) without
    waiting, status an int32 CUDA tensor with one entry per box."""
    inf = meta or info(comp)
    level = inf["levels"] if level is None else int(level)
    boxes = [(tuple(int(v) for v in lo), tuple(int(v) for v in hi)) for lo, hi in boxes]
    status = torch.zeros(max(1, len(boxes)), dtype=torch.int32, device=comp.device)
    if not boxes:
        return [] if check else ([], status[:0])
    hdr = hdr or header_bytes(comp)
    if level1 is None:
        level1 = decompress_progressive(comp, 1, stream=stream, meta=inf)
    if tables is None:
        tables = decode_tables(comp, hdr, stream)
    fields = served_fields([(comp, hdr, level1, tables)])
    reqs = (RegionRequest * len(boxes))()
    offs, off = [], 0
    for lo, hi in boxes:
        offs.append(off)
        n = 1
        for a, b in zip(lo, hi):
            n *= max(1, b - a)
        off += -(-n // 64) * 64
    out = torch.empty(off, dtype=inf["dtype"], device=comp.device)
    es = out.element_size()
    for q, (lo, hi), o in zip(reqs, boxes, offs):
        q.field = 0
        q.level = level
        for a in range(len(lo)):
            q.lo[a] = lo[a]
            q.hi[a] = hi[a]
        q.out_dev = out.data_ptr() + o * es
        q.out_cap = (off - o) * es
    ws = torch.empty(max(1, decode_requests_workspace(reqs, fields)), dtype=torch.uint8,
                     device=comp.device)
    decode_requests(reqs, fields, ws, status, stream)
    outs = []
    for q, o in zip(reqs, offs):
        shape = _shape_out(q.out_dims, inf["ndim"])
        n = 1
        for v in shape:
            n *= v
        outs.append(out[o:o + n].view(shape))
    if not check:
        return outs, status
    bad = torch.nonzero(status.cpu()).reshape(-1)
    if len(bad):
        raise StzError(ERR_CORRUPT, f"stz_decode_requests: box {int(bad[0])}")
    return outs


def launch_count() -> int:
    """Kernel launches made by the library so far (all streams)."""
    return int(lib().stz_launch_count())


def profile_enable(on: bool = True) -> None:
    lib().stz_profile_enable(1 if on else 0)


def profile_reset() -> None:
    lib().stz_profile_reset()


def profile_read() -> dict:
    """{kernel name: (timed launches, total device ms, total algorithmic
    bytes)} since the last reset."""
    buf = (_KernelTime * 64)()
    n = lib().stz_profile_read(buf, 64)
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms),
                                   float(buf[i].algo_bytes))
            for i in range(min(n, 64))}
