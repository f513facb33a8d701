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
