"""The C-ABI library builds, loads and exports every function include/stz.h
declares; its host-side argument checks and header parser work without a
GPU (no compute call is made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module")
def stzmod():
    from paper_2509_01626_gb300 import build, stz

    build.build()
    stz.lib()
    return stz


def declared_functions():
    src = open(os.path.join(ROOT, "include", "stz.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(stz_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(stzmod):
    names = declared_functions()
    assert len(names) >= 9
    L = stzmod.lib()
    for n in names:
        assert hasattr(L, n), n
    out = os.popen(f"nm -D --defined-only {stzmod.LIB_PATH}").read()
    exported = set(re.findall(r" T (stz_\w+)", out))
    assert set(names) <= exported


def test_version_and_errors(stzmod):
    assert "sm_103a" in stzmod.version()
    for c in (0, -1, -2, -3, -4, -5, -6):
        assert stzmod.strerror(c) != "unknown error"


def test_sizes(stzmod):
    assert stzmod.compress_bound((512, 512, 512), "float32") > 512 ** 3 * 4
    assert stzmod.workspace_size((512, 512, 512), "float32") > 512 ** 3 // 8 * 4
    assert stzmod.compress_bound((1800, 3600), "float32") > 0
    L = stzmod.lib()
    bad = (ctypes.c_int64 * 3)(0, 5, 5)
    assert L.stz_compress_bound(bad, 3, 0) == 0
    assert L.stz_workspace_size((ctypes.c_int64 * 3)(5, 5, 5), 4, 0) == 0


def test_argument_errors_need_no_gpu(stzmod):
    L = stzmod.lib()
    dims = (ctypes.c_int64 * 3)(8, 8, 8)
    nb = ctypes.c_size_t(0)
    vp = ctypes.c_void_p
    # bad ndim, bad eb, null pointers: rejected before any CUDA call
    assert L.stz_compress(vp(256), dims, 4, 0, 1, 1e-3, vp(256), 1 << 20, ctypes.byref(nb),
                          vp(256), 1 << 20, None) == stzmod.ERR_ARG
    assert L.stz_compress(vp(256), dims, 3, 0, 1, -1.0, vp(256), 1 << 20, ctypes.byref(nb),
                          vp(256), 1 << 20, None) == stzmod.ERR_ARG
    assert L.stz_compress(vp(256), dims, 3, 0, 1, float("nan"), vp(256), 1 << 20,
                          ctypes.byref(nb), vp(256), 1 << 20, None) == stzmod.ERR_ARG
    assert L.stz_compress(None, dims, 3, 0, 1, 1e-3, vp(256), 1 << 20, ctypes.byref(nb),
                          vp(256), 1 << 20, None) == stzmod.ERR_ARG
    assert L.stz_decompress_full(None, 100, vp(256), 100, vp(256), 100, None) == stzmod.ERR_ARG


@pytest.mark.parametrize("name", ["sin3d_f32_22x19x27", "sin3d_f64_9x14x10", "sin2d_f32_37x50"])
def test_host_header_parser_reads_oracle_containers(stzmod, ora, name):
    comp = np.fromfile(os.path.join(GOLDEN, name + ".stz"), dtype=np.uint8)
    ref = ora.info(comp)
    inf = stzmod._Info()
    rc = stzmod.lib().stz_info(comp.ctypes.data, comp.size, 0, ctypes.byref(inf))
    assert rc == 0
    dims = tuple(ref["dims"]) if ref["ndim"] == 3 else (ref["dims"][1], ref["dims"][2], 1)
    assert tuple(inf.dims) == dims
    assert inf.levels == ref["levels"] and inf.ndim == ref["ndim"]
    assert inf.eb_abs == ref["eb_abs"] and inf.total_bytes == comp.size


def test_host_header_parser_rejects_corruption(stzmod):
    comp = np.fromfile(os.path.join(GOLDEN, "sin3d_f32_22x19x27.stz"), dtype=np.uint8)
    inf = stzmod._Info()
    L = stzmod.lib()
    for cut in (0, 100, 255, 300):
        b = comp[:cut].copy() if cut else np.zeros(1, np.uint8)
        assert L.stz_info(b.ctypes.data, cut, 0, ctypes.byref(inf)) == stzmod.ERR_CORRUPT
    rng = np.random.default_rng(0)
    hits = 0
    for _ in range(400):
        b = comp.copy()
        i = int(rng.integers(0, 256 + 15 * 48))
        b[i] ^= np.uint8(1 << int(rng.integers(0, 8)))
        rc = L.stz_info(b.ctypes.data, b.size, 0, ctypes.byref(inf))
        assert rc in (0, stzmod.ERR_CORRUPT, stzmod.ERR_ARG)
        hits += rc != 0
    assert hits > 100


def test_batch_argument_errors_need_no_gpu(stzmod):
    L = stzmod.lib()
    jobs = (stzmod.FieldJob * 2)()
    sizes = ctypes.c_void_p(256)
    assert L.stz_compress_batch(0, jobs, sizes, None, None) == stzmod.ERR_ARG
    assert L.stz_compress_batch(2, None, sizes, None, None) == stzmod.ERR_ARG
    assert L.stz_compress_batch(2, jobs, None, None, None) == stzmod.ERR_ARG
    o = stzmod.BatchOpts()
    o.lanes = 33
    assert L.stz_compress_batch(2, jobs, sizes, ctypes.byref(o), None) == stzmod.ERR_ARG
    # zeroed jobs (no dims, null pointers) are rejected before any CUDA call
    o.lanes = 2
    assert L.stz_compress_batch(2, jobs, sizes, ctypes.byref(o), None) == stzmod.ERR_ARG
    # the work queue: an unknown schedule or tile count is rejected up front
    o.persistent, o.schedule = 1, 5
    assert L.stz_compress_batch(2, jobs, sizes, ctypes.byref(o), None) == stzmod.ERR_ARG
    o.schedule, o.tiles_per_item = 0, 65
    assert L.stz_compress_batch(2, jobs, sizes, ctypes.byref(o), None) == stzmod.ERR_ARG
    assert L.stz_compress_batch_workspace_size(2, jobs) == 0  # invalid jobs


def test_batch_queue_workspace_needs_no_gpu(stzmod):
    """The work queue's batch workspace holds the level groups of the 3D
    fields only (sizing reads no device memory)."""
    L = stzmod.lib()

    def job(j, dims, dtype=0):
        j.field_dev, j.out_dev, j.ws_dev = 1 << 12, 1 << 13, 1 << 20
        for a, v in enumerate(dims + (0,) * (3 - len(dims))):
            j.dims[a] = v
        j.ndim, j.dtype, j.eb_mode, j.eb = len(dims), dtype, 1, 1e-3
        j.out_cap, j.ws_bytes = 1 << 40, 1 << 40

    jobs = (stzmod.FieldJob * 3)()
    job(jobs[0], (64, 64, 64))
    job(jobs[1], (180, 360))
    job(jobs[2], (40, 33, 27), 1)
    both = L.stz_compress_batch_workspace_size(3, jobs)
    first = L.stz_compress_batch_workspace_size(1, jobs)
    assert both > first > 0 and both % 256 == 0
    only2d = (stzmod.FieldJob * 1)()
    job(only2d[0], (180, 360))
    assert L.stz_compress_batch_workspace_size(1, only2d) == 0


def test_region_sizes_and_async_errors_need_no_gpu(stzmod):
    L = stzmod.lib()
    comp = np.fromfile(os.path.join(GOLDEN, "sin3d_f32_22x19x27.stz"), dtype=np.uint8)
    hdr = bytes(comp[:stzmod.HEADER_MAX_BYTES].tobytes())
    full = stzmod.region_workspace_size(hdr, comp.size, (0, 0, 0), (22, 19, 27), 3, False)
    cached = stzmod.region_workspace_size(hdr, comp.size, (0, 0, 0), (22, 19, 27), 3, True)
    small = stzmod.region_workspace_size(hdr, comp.size, (2, 3, 4), (6, 7, 8), 3, True)
    assert full > cached > small > 0
    assert stzmod.region_workspace_size(hdr, comp.size, (0, 0, 0), (23, 19, 27), 3, False) == 0
    assert stzmod.region_workspace_size(hdr, comp.size, (0, 0, 0), (2, 2, 2), 4, False) == 0
    assert stzmod.region_workspace_size(b"xxxx" + hdr[4:], comp.size, (0, 0, 0), (2, 2, 2), 3,
                                        False) == 0
    # header checks and box checks happen before any CUDA call
    lo = (ctypes.c_int64 * 3)(0, 0, 0)
    hi = (ctypes.c_int64 * 3)(2, 2, 2)
    od = (ctypes.c_int64 * 3)()
    dev = ctypes.c_void_p(1 << 20)
    bad = b"xxxx" + hdr[4:]
    assert L.stz_decompress_region_async(dev, comp.size, bad, len(bad), None, lo, hi, 3, dev,
                                         64, od, dev, 1 << 20, dev, None) == stzmod.ERR_CORRUPT
    assert L.stz_decompress_region_async(dev, comp.size, None, 0, None, lo, hi, 3, dev, 64, od,
                                         dev, 1 << 20, dev, None) == stzmod.ERR_ARG
    hi_bad = (ctypes.c_int64 * 3)(2, 2, 99)
    assert L.stz_decompress_region_async(dev, comp.size, hdr, len(hdr), None, lo, hi_bad, 3, dev,
                                         64, od, dev, 1 << 20, dev, None) == stzmod.ERR_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libstz.so every call raises: there is no CPU fallback."""
    import torch

    from paper_2509_01626_gb300 import stz

    monkeypatch.setattr(stz, "_lib", None)
    monkeypatch.setattr(stz, "LIB_PATH", str(tmp_path / "libstz.so"))
    with pytest.raises(ImportError):
        stz.lib()
    # a host tensor is refused outright (there is no CPU path to fall back to)
    with pytest.raises((ImportError, ValueError)):
        stz.compress(torch.zeros(8, 8, 8), 1e-3)
    with pytest.raises(ImportError):
        stz.compress_bound((8, 8, 8), torch.float32)


def test_product_code_never_reaches_the_oracle():
    """The package (the product path) neither imports nor runs anything under
    oracle/: only tests, the smoke check and the bench's CPU baseline may."""
    pkg = os.path.join(ROOT, "paper_2509_01626_gb300")
    pat = re.compile(r"^\s*(import|from)\s+oracle\b|stz_oracle|oracle[/\\]", re.M)
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not pat.search(src), os.path.join(dirpath, f)


def _golden(name="sin3d_f32_22x19x27"):
    return np.fromfile(os.path.join(GOLDEN, name + ".stz"), dtype=np.uint8)


def _i64(*v):
    return (ctypes.c_int64 * len(v))(*v)


def test_sizes_for_other_level_counts(stzmod):
    L = stzmod.lib()
    d = _i64(64, 64, 64)
    assert L.stz_compress_bound_ex(d, 3, 0, 0) == L.stz_compress_bound(d, 3, 0)
    assert L.stz_workspace_size_ex(d, 3, 0, 0) == L.stz_workspace_size(d, 3, 0)
    assert L.stz_compress_bound_ex(d, 3, 0, 3) == L.stz_compress_bound(d, 3, 0)
    for lv in (1, 2, 4, 5, 6):
        assert L.stz_compress_bound_ex(d, 3, 0, lv) > 64 ** 3 * 4
        assert L.stz_workspace_size_ex(d, 3, 1, lv) > 0
    for lv in (-1, 7):
        assert L.stz_compress_bound_ex(d, 3, 0, lv) == 0
        assert L.stz_workspace_size_ex(d, 3, 0, lv) == 0
    assert L.stz_compress_bound_ex(d, 3, 2, 3) == 0  # no such dtype


def test_compress_ex_rejects_bad_options_before_any_cuda_call(stzmod):
    L = stzmod.lib()
    d = _i64(8, 8, 8)
    nb = ctypes.c_size_t(0)
    vp = ctypes.c_void_p

    def call(opts, field=vp(256), out_bytes=ctypes.byref(nb)):
        o = ctypes.byref(opts) if opts is not None else None
        return L.stz_compress_ex(field, d, 3, 0, 1, 1e-3, o, vp(256), 1 << 20, out_bytes,
                                 vp(256), 1 << 30, None)

    for lv, pred, ratio in ((7, 0, 2.5), (-1, 0, 2.5), (3, 3, 2.5), (3, -1, 2.5),
                            (3, 0, 0.5), (3, 0, 65.0), (3, 0, float("nan"))):
        assert call(stzmod.CompressOpts(lv, pred, ratio)) == stzmod.ERR_ARG, (lv, pred, ratio)
    assert call(None, field=None) == stzmod.ERR_ARG
    assert call(None, field=vp(8)) == stzmod.ERR_ARG  # field not 16-byte aligned
    assert call(None, out_bytes=None) == stzmod.ERR_ARG


def test_decode_calls_reject_bad_pointers_before_any_cuda_call(stzmod):
    L = stzmod.lib()
    vp = ctypes.c_void_p
    od = _i64(0, 0, 0)
    assert L.stz_decompress_progressive(None, 1000, 1, vp(256), 100, od, vp(256), 100,
                                        None) == stzmod.ERR_ARG
    assert L.stz_decompress_progressive(vp(256), 1000, 0, vp(256), 100, od, vp(256), 100,
                                        None) == stzmod.ERR_ARG
    assert L.stz_decompress_progressive(vp(260), 1000, 1, vp(256), 100, od, vp(256), 100,
                                        None) == stzmod.ERR_ARG  # container not 8-byte aligned
    comp = _golden()
    hdr = comp[:1984].copy()
    assert L.stz_decode_tables(None, comp.size, hdr.ctypes.data, hdr.size, vp(256), 1 << 20,
                               None) == stzmod.ERR_ARG
    assert L.stz_decode_tables(vp(256), comp.size, hdr.ctypes.data, hdr.size, vp(264), 1 << 20,
                               None) == stzmod.ERR_ARG  # tables not 16-byte aligned
    assert L.stz_decode_tables(vp(256), comp.size, hdr.ctypes.data, hdr.size, vp(256), 16,
                               None) == stzmod.ERR_CAPACITY


@pytest.mark.parametrize("name", ["sin3d_f32_22x19x27", "sin3d_f64_9x14x10", "sin2d_f32_37x50"])
def test_sizes_read_from_a_host_header(stzmod, name):
    """Decode-table and region-workspace sizes come from the host copy of a
    container's first bytes alone."""
    L = stzmod.lib()
    comp = _golden(name)
    hdr = comp[:1984].copy()
    chunks = (ctypes.c_int64 * 64)()
    inf = stzmod._Info()
    assert L.stz_info(comp.ctypes.data, comp.size, 0, ctypes.byref(inf)) == 0
    nd, lv = inf.ndim, inf.levels
    dims = tuple(inf.dims)[:nd]
    full_lo, full_hi = _i64(*([0] * nd)), _i64(*dims)
    ns = L.stz_region_chunks(hdr.ctypes.data, hdr.size, comp.size, full_lo, full_hi, lv, 0,
                             chunks, 64)
    # 1 + 7 (L - 1) streams; a 2D field leaves 4 of each level's 7 empty
    assert ns == 1 + 7 * (lv - 1)
    if nd == 2:
        assert sum(1 for k in range(1, ns) if chunks[k] > 0) == 3 * (lv - 1)
    # one table of 4096 four-byte entries per stream
    assert L.stz_decode_tables_size(hdr.ctypes.data, hdr.size, comp.size) == 16384 * ns
    bad = hdr.copy()
    bad[:4] = 0
    assert L.stz_decode_tables_size(bad.ctypes.data, bad.size, comp.size) == 0
    ws_full = L.stz_region_workspace_size(hdr.ctypes.data, hdr.size, comp.size, full_lo, full_hi,
                                          lv, 0)
    assert ws_full > 0
    small_hi = _i64(*[min(2, n) for n in dims])
    ws_small = L.stz_region_workspace_size(hdr.ctypes.data, hdr.size, comp.size, full_lo,
                                           small_hi, lv, 0)
    assert 0 < ws_small <= ws_full
    # a supplied level-1 grid never needs more room
    assert L.stz_region_workspace_size(hdr.ctypes.data, hdr.size, comp.size, full_lo, small_hi,
                                       lv, 1) <= ws_small
    for level in (0, lv + 1):
        assert L.stz_region_workspace_size(hdr.ctypes.data, hdr.size, comp.size, full_lo,
                                           full_hi, level, 0) == 0
    empty_hi = _i64(*([0] * nd))
    assert L.stz_region_workspace_size(hdr.ctypes.data, hdr.size, comp.size, full_lo, empty_hi,
                                       lv, 0) == 0
    past_hi = _i64(*[n + 1 for n in dims])
    assert L.stz_region_workspace_size(hdr.ctypes.data, hdr.size, comp.size, full_lo, past_hi,
                                       lv, 0) == 0


def test_roi_geometry_and_argument_errors(stzmod):
    L = stzmod.lib()
    assert L.stz_roi_units(_i64(64, 64, 64), 3, _i64(4, 4, 4)) == 16 ** 3
    assert L.stz_roi_units(_i64(37, 50), 2, _i64(4, 8)) == 10 * 7
    assert L.stz_roi_units(_i64(30, 31, 33), 3, _i64(4, 8, 16)) == 8 * 4 * 3
    assert L.stz_roi_units(_i64(64, 64, 64), 3, _i64(0, 4, 4)) == -1
    assert L.stz_roi_units(_i64(64, 64, 64), 3, None) == -1
    assert L.stz_roi_workspace_size(_i64(64, 64, 64), 3, _i64(0, 4, 4)) == 0
    assert L.stz_roi_workspace_size(_i64(64, 64, 64), 3, _i64(4, 4, 4)) >= 3 * 8 * 16 ** 3
    vp = ctypes.c_void_p
    d, b = _i64(64, 64, 64), _i64(4, 4, 4)
    ns = ctypes.c_int64(0)
    ws = L.stz_roi_workspace_size(d, 3, b)

    def sel(metric=0, mode=1, value=0.01, field=vp(256), cap=4096, wsb=ws, dtype=0):
        return L.stz_roi_select(field, d, 3, dtype, b, metric, mode, value, vp(256), cap, None,
                                ctypes.byref(ns), vp(256), wsb, None)

    assert sel(metric=2) == stzmod.ERR_ARG
    assert sel(mode=2) == stzmod.ERR_ARG
    assert sel(value=0.0) == stzmod.ERR_ARG
    assert sel(value=1.5) == stzmod.ERR_ARG
    assert sel(dtype=2) == stzmod.ERR_ARG
    assert sel(field=None) == stzmod.ERR_ARG
    assert sel(field=vp(258)) == stzmod.ERR_ARG  # not aligned to the element
    assert sel(cap=4095) == stzmod.ERR_CAPACITY
    assert sel(wsb=ws - 1) == stzmod.ERR_CAPACITY


def test_batched_requests_are_planned_on_the_host(stzmod):
    """stz_decode_requests checks every request against its field's host
    header before queuing anything; the workspace size is a host plan."""
    L = stzmod.lib()
    comp = _golden()
    hdr = comp[:1984].copy()
    vp = ctypes.c_void_p
    f = (stzmod.ServedField * 1)()
    f[0].comp_dev, f[0].comp_bytes = 256, comp.size
    f[0].hdr_host, f[0].hdr_bytes = hdr.ctypes.data, hdr.size
    f[0].level1_dev, f[0].tables_dev = 256, 256
    r = (stzmod.RegionRequest * 2)()
    for i in range(2):
        r[i].field, r[i].level = 0, 3
        r[i].lo[:] = [0, 0, 0]
        r[i].hi[:] = [4 + i, 5, 6]
        r[i].out_dev, r[i].out_cap = 256, 1 << 20
    ws = L.stz_decode_requests_workspace(2, r, f, 1)
    assert ws > 0
    assert L.stz_decode_requests_workspace(1, r, f, 1) <= ws
    assert L.stz_decode_requests_workspace(0, r, f, 1) == 0
    assert L.stz_decode_requests_workspace(2, r, None, 0) == 0
    st = vp(256)
    assert L.stz_decode_requests(2, r, f, 1, None, ws, st, None) == stzmod.ERR_ARG
    assert L.stz_decode_requests(2, r, f, 1, vp(256), ws, None, None) == stzmod.ERR_ARG
    assert L.stz_decode_requests(2, r, f, 1, vp(256), ws - 1, st, None) == stzmod.ERR_CAPACITY
    r[1].field = 1  # no such field
    assert L.stz_decode_requests(2, r, f, 1, vp(256), ws, st, None) == stzmod.ERR_ARG
    r[1].field, r[1].level = 0, 4  # past the container's levels
    assert L.stz_decode_requests(2, r, f, 1, vp(256), ws, st, None) == stzmod.ERR_ARG
    r[1].level = 3
    f[0].tables_dev = None
    assert L.stz_decode_requests(2, r, f, 1, vp(256), ws, st, None) == stzmod.ERR_ARG


def test_launch_counter_and_timer_need_no_gpu(stzmod):
    L = stzmod.lib()
    c0 = L.stz_launch_count()
    nb = ctypes.c_size_t(0)
    # a rejected call launches nothing
    assert L.stz_compress(None, _i64(8, 8, 8), 3, 0, 1, 1e-3, ctypes.c_void_p(256), 1 << 20,
                          ctypes.byref(nb), ctypes.c_void_p(256), 1 << 20,
                          None) == stzmod.ERR_ARG
    assert L.stz_launch_count() == c0
    L.stz_profile_enable(1)
    L.stz_profile_reset()
    buf = (stzmod._KernelTime * 4)()
    assert L.stz_profile_read(buf, 4) == 0
    L.stz_profile_enable(0)
