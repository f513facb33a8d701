"""Round trips, streaming equalities and container checks of the oracle.

* Brute force over every 3D shape in {1..12}^3 and 2D shape in {1..16}^2:
  decode(compress(x)) holds the bound at every point and equals the
  reconstruction the compressor computed.
* Progressive decompression (Sec. 3.3): decoding to level k equals the full
  decode sampled at stride 2^(L-k).  Random access: a region decode equals the
  slice of the full decode (bitwise).
* Level counts 1..5, f32 and f64, small bricks (many chunks).
* Corrupted or truncated containers are rejected without crashing.
"""
import itertools
import struct

import numpy as np
import pytest

from paper_2509_01626_gb300 import synth


def bound_ok(x, y, eb_abs):
    d = np.abs(x.astype(np.float64) - y.astype(np.float64))
    return bool((d <= eb_abs).all())


def test_every_small_3d_shape(ora):
    rng = np.random.default_rng(0)
    for shape in itertools.product(range(1, 13), repeat=3):
        x = rng.standard_normal(shape).astype(np.float32).cumsum(axis=-1)
        c = ora.compress(x, 1e-3)
        y = ora.decompress(c)
        codes, soff, recon, ebs = ora.quantize(x, 1e-3)
        assert np.array_equal(y.view(np.uint32), recon.view(np.uint32)), shape
        assert bound_ok(x, y, ebs[0]), shape


def test_every_small_2d_shape(ora):
    rng = np.random.default_rng(1)
    for shape in itertools.product(range(1, 17), repeat=2):
        x = rng.standard_normal(shape).cumsum(axis=0)
        c = ora.compress(x, 1e-2)
        y = ora.decompress(c)
        assert y.shape == shape
        assert bound_ok(x, y, ora.info(c)["eb_abs"]), shape


@pytest.mark.parametrize("levels", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_levels_and_progressive(ora, levels, dtype):
    shape = (37, 29, 41)
    x = synth.sinusoids(shape, levels, dtype=dtype)
    c = ora.compress(x, 1e-3, levels=levels, brick=(2, 4, 8))
    full = ora.decompress(c)
    assert bound_ok(x, full, ora.info(c)["eb_abs"])
    for k in range(1, levels + 1):
        s = 1 << (levels - k)
        p = ora.decompress(c, k)
        assert np.array_equal(p, full[::s, ::s, ::s]), k


@pytest.mark.parametrize("shape", [(64, 48, 80), (100, 70)])
def test_regions_equal_slices(ora, shape):
    x = synth.sinusoids(shape, 5)
    c = ora.compress(x, 1e-4, brick=(2, 8, 8) if len(shape) == 3 else (1, 8, 8))
    full = ora.decompress(c)
    L = 3
    for i, (lo, hi) in enumerate(synth.random_boxes(shape, 20, 42, 1, 40)):
        level = 1 + i % L
        s = 1 << (L - level)
        r = ora.decompress_region(c, lo, hi, level)
        sl = tuple(slice(-(-l // s) * s, h, s) for l, h in zip(lo, hi))
        assert np.array_equal(r, full[sl]), (lo, hi, level)


def test_region_rejects_bad_boxes(ora):
    x = synth.sinusoids((10, 10, 10), 1)
    c = ora.compress(x, 1e-3)
    for lo, hi in [((0, 0, 0), (11, 5, 5)), ((3, 3, 3), (3, 5, 5)), ((-1, 0, 0), (2, 2, 2))]:
        with pytest.raises(ora.OracleError) as e:
            ora.decompress_region(c, lo, hi)
        assert e.value.code == ora.ERR_ARG
    with pytest.raises(ora.OracleError):
        ora.decompress(c, 4)


def test_header_layout(ora):
    x = synth.sinusoids((9, 10, 11), 2)
    c = ora.compress(x, 1e-3)
    b = c.tobytes()
    assert b[:4] == b"STZ1"
    (version,) = struct.unpack_from("<H", b, 4)
    dtype, ndim, levels, mode, maxlen, nsub = b[6], b[7], b[8], b[9], b[10], b[11]
    (radius,) = struct.unpack_from("<I", b, 12)
    bricks = struct.unpack_from("<3I", b, 16)
    (ns,) = struct.unpack_from("<I", b, 28)
    dims = struct.unpack_from("<3q", b, 32)
    eb, eb_abs, vmin, vmax = struct.unpack_from("<4d", b, 56)
    (total,) = struct.unpack_from("<Q", b, 88)
    assert (version, dtype, ndim, levels, mode, maxlen, nsub) == (1, 0, 3, 3, 1, 12, 8)
    assert radius == 1024 and bricks == (8, 16, 16) and ns == 15 and dims == (9, 10, 11)
    assert total == len(b)
    assert vmin == float(x.min()) and vmax == float(x.max())
    assert eb_abs == 1e-3 * (float(x.max()) - float(x.min()))
    ebl = struct.unpack_from("<3d", b, 96)
    assert ebl == (eb_abs / 6.25, eb_abs / 2.5, eb_abs)
    two = struct.unpack_from("<3d", b, 144)
    assert two == tuple(float(np.float32(2 * e)) for e in ebl)
    # directory: sections are 8-aligned, consecutive, and end at total
    offs = [struct.unpack_from("<Q", b, 256 + 48 * s)[0] for s in range(ns)]
    assert offs[0] == 256 + 48 * ns and all(o % 8 == 0 for o in offs)
    assert offs == sorted(offs)


def test_corruption_is_detected_or_harmless(ora):
    x = synth.sinusoids((20, 21, 22), 3)
    c = ora.compress(x, 1e-3, brick=(4, 4, 4))
    for cut in (0, 10, 255, 300, c.size // 2, c.size - 1):
        with pytest.raises(ora.OracleError) as e:
            ora.decompress(c[:cut])
        assert e.value.code == ora.ERR_CORRUPT
    bad = c.copy()
    bad[0] ^= 0xFF
    with pytest.raises(ora.OracleError):
        ora.decompress(bad)
    rng = np.random.default_rng(5)
    outcomes = {"ok": 0, "corrupt": 0}
    for _ in range(300):
        b = c.copy()
        i = int(rng.integers(0, b.size))
        b[i] ^= np.uint8(1 << int(rng.integers(0, 8)))
        try:
            ora.decompress(b)
            outcomes["ok"] += 1
        except ora.OracleError as e:
            assert e.code in (ora.ERR_CORRUPT, ora.ERR_ARG)
            outcomes["corrupt"] += 1
    assert outcomes["corrupt"] > 0


@pytest.mark.parametrize("nsub", [1, 2, 4, 8])
def test_sub_chunk_counts(ora, nsub):
    """Any sub-chunk count round-trips; the stored sub-chunk offsets are
    checked against the decode (a shifted offset is rejected)."""
    x = synth.sinusoids((30, 26, 33), 21)
    c = ora.compress(x, 1e-3, nsub=nsub, brick=(4, 4, 8))
    assert ora.info(c)["nsub"] == nsub
    y = ora.decompress(c)
    codes, soff, recon, ebs = ora.quantize(x, 1e-3)
    assert np.array_equal(y.view(np.uint32), recon.view(np.uint32))
    if nsub > 1:
        # first sub-chunk offset of the level-3 x-odd stream (index 8)
        sect = int(struct.unpack_from("<Q", c.tobytes(), 256 + 48 * 8)[0])
        nlive = int(struct.unpack_from("<I", c.tobytes(), 256 + 48 * 8 + 20)[0])
        nch = int(struct.unpack_from("<I", c.tobytes(), 256 + 48 * 8 + 16)[0])
        off_subs = ((3 * nlive + 3) & ~3) + 4 * nch
        b = c.copy()
        v = struct.unpack_from("<H", b.tobytes(), sect + off_subs)[0]
        struct.pack_into("<H", b, sect + off_subs, v + 1)
        with pytest.raises(ora.OracleError) as e:
            ora.decompress(b)
        assert e.value.code == ora.ERR_CORRUPT
