"""ctypes wrapper of the CPU oracle (stz_oracle.c).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The product path never does.

Arrays are numpy, C order.  A 3D field has shape (nz, ny, nx); a 2D field has
shape (ny, nx) and is handled as nz = 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "stz_oracle.c"), os.path.join(_HERE, "stz_oracle_roi.c")]
_DEPS = _SRC + [os.path.join(_HERE, "stz_oracle_real.inc"), os.path.join(_HERE, "stz_oracle.h")]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")

# Default brick of one chunk, in sub-block cells (z, y, x): 2048 symbols.
BRICK_3D = (8, 16, 16)
BRICK_2D = (1, 32, 64)

OK, ERR_ARG, ERR_CAPACITY, ERR_CORRUPT, ERR_NOMEM = 0, -1, -2, -3, -6


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle error {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (single thread, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH):
        lib_m = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(d) <= lib_m for d in _DEPS):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp] + _SRC + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("dtype", ctypes.c_int),
        ("ndim", ctypes.c_int),
        ("dims", ctypes.c_int64 * 3),
        ("eb_mode", ctypes.c_int),
        ("eb", ctypes.c_double),
        ("levels", ctypes.c_int),
        ("radius", ctypes.c_int),
        ("max_code_len", ctypes.c_int),
        ("brick", ctypes.c_int * 3),
        ("nsub", ctypes.c_int),
        ("predictor", ctypes.c_int),
        ("eb_ratio", ctypes.c_double),
    ]


# predictors of levels 2..L (ablation of Sec. 3.1): opt. 4 cubic (the method),
# opt. 2 multi-linear, opt. 1 direct
PREDICTORS = {"cubic": 0, "linear": 1, "direct": 2}


class _Info(ctypes.Structure):
    _fields_ = [
        ("p", _Params),
        ("eb_abs", ctypes.c_double),
        ("eb_level", ctypes.c_double * 7),
        ("two_eb", ctypes.c_double * 7),
        ("nstreams", ctypes.c_int),
        ("total_bytes", ctypes.c_uint64),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
        L.ora_compress_bound.restype = ctypes.c_size_t
        L.ora_compress_bound.argtypes = [ctypes.POINTER(_Params)]
        L.ora_compress.argtypes = [vp, ctypes.POINTER(_Params), vp, ctypes.c_size_t,
                                   ctypes.POINTER(ctypes.c_size_t)]
        L.ora_quantize.argtypes = [vp, ctypes.POINTER(_Params), vp, i64p, vp,
                                   ctypes.POINTER(ctypes.c_double)]
        L.ora_decompress.argtypes = [vp, ctypes.c_size_t, ctypes.c_int, vp, ctypes.c_size_t, i64p]
        L.ora_decompress_region.argtypes = [vp, ctypes.c_size_t, i64p, i64p, ctypes.c_int, vp,
                                            ctypes.c_size_t, i64p]
        L.ora_decode_streams.argtypes = [vp, ctypes.c_size_t, vp, i64p]
        L.ora_parse_info.argtypes = [vp, ctypes.c_size_t, ctypes.POINTER(_Info)]
        L.ora_huffman_lengths.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
        L.ora_predict_f64.restype = ctypes.c_double
        L.ora_predict_f64.argtypes = [vp, i64p, ctypes.c_int, ctypes.c_int, i64p, ctypes.c_int,
                                      ctypes.c_int64]
        L.ora_predict_f32.restype = ctypes.c_float
        L.ora_predict_f32.argtypes = [vp, i64p, ctypes.c_int, ctypes.c_int, i64p, ctypes.c_int,
                                      ctypes.c_int64]
        L.ora_predict_mode_f64.restype = ctypes.c_double
        L.ora_predict_mode_f64.argtypes = [vp, i64p, ctypes.c_int, ctypes.c_int, i64p,
                                           ctypes.c_int]
        L.ora_roi_units.restype = ctypes.c_int64
        L.ora_roi_units.argtypes = [i64p, i64p]
        L.ora_roi_select.argtypes = [vp, ctypes.c_int, i64p, i64p, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, vp, vp, i64p]
        L.ora_stream_pos.restype = ctypes.c_int64
        L.ora_stream_pos.argtypes = [i64p, ctypes.POINTER(ctypes.c_int), i64p]
        _lib = L
    return _lib


def _i64(vals):
    return (ctypes.c_int64 * 3)(*[int(v) for v in vals])


def _dims3(shape):
    if len(shape) == 3:
        return 3, tuple(int(s) for s in shape)
    if len(shape) == 2:
        return 2, (1, int(shape[0]), int(shape[1]))
    raise ValueError("field must be 2D or 3D")


def make_params(shape, dtype, eb, mode="rel", levels=3, radius=1024, max_code_len=12,
                brick=None, nsub=8, predictor="cubic", eb_ratio=2.5) -> _Params:
    ndim, d3 = _dims3(shape)
    if brick is None:
        brick = BRICK_3D if ndim == 3 else BRICK_2D
    p = _Params()
    p.dtype = 0 if np.dtype(dtype) == np.float32 else 1
    p.ndim = ndim
    for a in range(3):
        p.dims[a] = d3[a]
        p.brick[a] = int(brick[a])
    p.eb_mode = 1 if mode == "rel" else 0
    p.eb = float(eb)
    p.levels = int(levels)
    p.radius = int(radius)
    p.max_code_len = int(max_code_len)
    p.nsub = int(nsub)
    p.predictor = PREDICTORS[predictor]
    p.eb_ratio = float(eb_ratio)
    return p


def nstreams(levels: int) -> int:
    return 1 + 7 * (levels - 1)


def compress(x: np.ndarray, eb: float, mode: str = "rel", **kw) -> np.ndarray:
    """Compress a float32/float64 array; returns the container as uint8."""
    x = np.ascontiguousarray(x)
    if x.dtype not in (np.float32, np.float64):
        raise TypeError("field must be float32 or float64")
    p = make_params(x.shape, x.dtype, eb, mode, **kw)
    L = lib()
    cap = L.ora_compress_bound(ctypes.byref(p))
    if cap == 0:
        raise OracleError(ERR_ARG, "compress_bound")
    out = np.zeros(cap, dtype=np.uint8)
    nb = ctypes.c_size_t(0)
    rc = L.ora_compress(x.ctypes.data, ctypes.byref(p), out.ctypes.data, cap, ctypes.byref(nb))
    if rc != OK:
        raise OracleError(rc, "compress")
    return out[: nb.value].copy()


def quantize(x: np.ndarray, eb: float, mode: str = "rel", **kw):
    """Codes of all streams (concatenated, stream order), stream offsets,
    reconstruction and [eb_abs, eb_1, ..., eb_L]."""
    x = np.ascontiguousarray(x)
    p = make_params(x.shape, x.dtype, eb, mode, **kw)
    ns = nstreams(p.levels)
    codes = np.zeros(x.size, dtype=np.uint16)
    soff = np.zeros(ns + 1, dtype=np.int64)
    recon = np.zeros_like(x)
    ebs = np.zeros(p.levels + 1, dtype=np.float64)
    rc = lib().ora_quantize(x.ctypes.data, ctypes.byref(p), codes.ctypes.data,
                            soff.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            recon.ctypes.data,
                            ebs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != OK:
        raise OracleError(rc, "quantize")
    return codes, soff, recon, ebs


def info(comp: np.ndarray) -> dict:
    comp = np.ascontiguousarray(comp, dtype=np.uint8)
    inf = _Info()
    rc = lib().ora_parse_info(comp.ctypes.data, comp.size, ctypes.byref(inf))
    if rc != OK:
        raise OracleError(rc, "info")
    p = inf.p
    L_ = p.levels
    return {
        "dtype": np.float32 if p.dtype == 0 else np.float64,
        "ndim": p.ndim,
        "dims": tuple(p.dims),
        "levels": L_,
        "radius": p.radius,
        "max_code_len": p.max_code_len,
        "brick": tuple(p.brick),
        "nsub": p.nsub,
        "predictor": {v: k for k, v in PREDICTORS.items()}[p.predictor],
        "eb_ratio": p.eb_ratio,
        "eb_mode": "rel" if p.eb_mode == 1 else "abs",
        "eb": p.eb,
        "eb_abs": inf.eb_abs,
        "eb_level": [inf.eb_level[l] for l in range(1, L_ + 1)],
        "two_eb": [inf.two_eb[l] for l in range(1, L_ + 1)],
        "nstreams": inf.nstreams,
        "total_bytes": int(inf.total_bytes),
    }


def _out_shape(ndim, od):
    return (int(od[1]), int(od[2])) if ndim == 2 else (int(od[0]), int(od[1]), int(od[2]))


def decompress(comp: np.ndarray, level: int | None = None) -> np.ndarray:
    """Decode to `level` (default: full resolution)."""
    comp = np.ascontiguousarray(comp, dtype=np.uint8)
    inf = info(comp)
    if level is None:
        level = inf["levels"]
    s = 1 << (inf["levels"] - level) if 1 <= level <= inf["levels"] else 1
    od = [-(-d // s) for d in inf["dims"]]
    out = np.zeros(max(1, od[0] * od[1] * od[2]), dtype=inf["dtype"])
    odims = (ctypes.c_int64 * 3)()
    rc = lib().ora_decompress(comp.ctypes.data, comp.size, int(level), out.ctypes.data,
                              out.nbytes, odims)
    if rc != OK:
        raise OracleError(rc, "decompress")
    n = odims[0] * odims[1] * odims[2]
    return out[:n].reshape(_out_shape(inf["ndim"], odims))


def decompress_region(comp: np.ndarray, lo, hi, level: int | None = None) -> np.ndarray:
    """Box [lo, hi) in field coordinates ((y, x) for 2D) at `level`."""
    comp = np.ascontiguousarray(comp, dtype=np.uint8)
    inf = info(comp)
    if level is None:
        level = inf["levels"]
    if inf["ndim"] == 2:
        lo, hi = (0,) + tuple(lo), (1,) + tuple(hi)
    cap = max(1, int(np.prod([max(0, h - l) for l, h in zip(lo, hi)])))
    out = np.zeros(cap, dtype=inf["dtype"])
    odims = (ctypes.c_int64 * 3)()
    rc = lib().ora_decompress_region(comp.ctypes.data, comp.size, _i64(lo), _i64(hi), int(level),
                                     out.ctypes.data, out.nbytes, odims)
    if rc != OK:
        raise OracleError(rc, "decompress_region")
    n = odims[0] * odims[1] * odims[2]
    return out[:n].reshape(_out_shape(inf["ndim"], odims))


def decode_streams(comp: np.ndarray):
    """Entropy-decoded symbols of every stream (concatenated) and offsets."""
    comp = np.ascontiguousarray(comp, dtype=np.uint8)
    inf = info(comp)
    n = int(np.prod(inf["dims"]))
    codes = np.zeros(n, dtype=np.uint16)
    soff = np.zeros(inf["nstreams"] + 1, dtype=np.int64)
    rc = lib().ora_decode_streams(comp.ctypes.data, comp.size, codes.ctypes.data,
                                  soff.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc != OK:
        raise OracleError(rc, "decode_streams")
    return codes, soff


def huffman_lengths(freq, max_len: int = 12) -> np.ndarray:
    f = np.ascontiguousarray(freq, dtype=np.uint64)
    out = np.zeros(f.size, dtype=np.uint8)
    rc = lib().ora_huffman_lengths(f.ctypes.data, f.size, int(max_len), out.ctypes.data)
    if rc != OK:
        raise OracleError(rc, "huffman_lengths")
    return out


def predict(grid: np.ndarray, levels: int, level: int, g, axis: int = 0, t: int = 1):
    """Prediction of field point g (z, y, x) from `grid` taken as the
    reconstruction; level 1 uses the base coder's rule along `axis` with pass
    stride `t` (in level-1 grid units)."""
    grid = np.ascontiguousarray(grid)
    n = grid.shape if grid.ndim == 3 else (1,) + grid.shape
    if grid.dtype == np.float64:
        return lib().ora_predict_f64(grid.ctypes.data, _i64(n), levels, level, _i64(g), axis, t)
    return np.float32(lib().ora_predict_f32(grid.ctypes.data, _i64(n), levels, level, _i64(g),
                                            axis, t))


def predict_mode(grid: np.ndarray, levels: int, level: int, g, predictor: str) -> float:
    """Level >= 2 prediction of field point g with the chosen predictor
    ("cubic", "linear", "direct"); float64 grids."""
    grid = np.ascontiguousarray(grid, dtype=np.float64)
    n = grid.shape if grid.ndim == 3 else (1,) + grid.shape
    return lib().ora_predict_mode_f64(grid.ctypes.data, _i64(n), levels, level, _i64(g),
                                      PREDICTORS[predictor])


ROI_METRICS = {"range": 0, "max": 1}
ROI_MODES = {"threshold": 0, "top": 1}


def roi_select(field: np.ndarray, block, metric: str = "range", mode: str = "top",
               value: float = 0.01):
    """ROI selection (Sec. 3.3): (selected unit indices ascending, metric of
    every unit).  block: (bz, by, bx) points ((by, bx) for 2D fields)."""
    x = np.ascontiguousarray(field)
    _, d3 = _dims3(x.shape)
    b3 = tuple(block) if x.ndim == 3 else (1,) + tuple(block)
    nu = int(lib().ora_roi_units(_i64(d3), _i64(b3)))
    if nu < 1:
        raise OracleError(ERR_ARG, "roi_select")
    met = np.zeros(nu, dtype=np.float64)
    sel = np.zeros(nu, dtype=np.int64)
    ns = ctypes.c_int64(0)
    rc = lib().ora_roi_select(x.ctypes.data, 0 if x.dtype == np.float32 else 1, _i64(d3), _i64(b3),
                              ROI_METRICS[metric], ROI_MODES[mode], float(value), met.ctypes.data,
                              sel.ctypes.data, ctypes.byref(ns))
    if rc != OK:
        raise OracleError(rc, "roi_select")
    return sel[: ns.value].copy(), met


def stream_pos(e, b, c) -> int:
    return lib().ora_stream_pos(_i64(e), (ctypes.c_int * 3)(*b), _i64(c))
