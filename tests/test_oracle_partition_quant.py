"""Pins of the oracle's partition and quantizer.

* Partition (Sec. 3.1 Fig. 3, Sec. 3.2): with L = 3 and dims divisible by 4,
  level 1 holds 1/64 of the points ("1.6%"), level 2 7/64, level 3 56/64
  ("87.5% of the data"); in 2D 1/16, 3/16, 12/16.  Each stream holds exactly
  the points of its sub-block (brute-force enumeration from coordinates),
  and the brick-major stream order is a permutation with contiguous bricks.
* Quantizer: |x - x'| <= eb at every point, checked in exact rational
  arithmetic where double could round, with the per-level bounds of
  Sec. 3.1 opt. 5 (eb / 2.5 per level towards the coarsest); constant and
  exactly-interpolated fields give the zero code on every finer level.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from paper_2509_01626_gb300 import synth


def level_of_points(shape3, L):
    """Level of each field point from its coordinates (independent of the oracle)."""
    lv = np.full(shape3, L, dtype=np.int64)
    z, y, x = np.meshgrid(*[np.arange(n) for n in shape3], indexing="ij")
    for l in range(L - 1, 0, -1):
        s = 1 << (L - l)
        on = (z % s == 0) & (y % s == 0) & (x % s == 0)
        lv[on] = l
    return lv


@pytest.mark.parametrize("shape,frac", [((32, 32, 32), (1, 7, 56)), ((24, 16, 40), (1, 7, 56)),
                                        ((64, 64), (1, 3, 12))])
def test_level_fractions(ora, shape, frac):
    x = synth.sinusoids(shape, 3)
    codes, soff, recon, ebs = ora.quantize(x, 1e-3)
    n = x.size
    L = 3
    sizes = np.diff(soff)
    per_level = [sizes[0], sizes[1:8].sum(), sizes[8:15].sum()]
    tot = sum(frac)
    assert per_level == [n * f // tot for f in frac]
    if len(shape) == 2:
        # 2D: sub-blocks with an odd z are empty, 3 live per level
        assert all(sizes[1 + 7 * j + k - 1] == 0 for j in range(2) for k in (4, 5, 6, 7))


@pytest.mark.parametrize("e,b", [((5, 7, 9), (2, 3, 4)), ((8, 16, 16), (8, 16, 16)),
                                 ((1, 13, 6), (1, 4, 4)), ((9, 9, 9), (8, 16, 16))])
def test_stream_order_is_brick_major_permutation(ora, e, b):
    pos = {}
    for c in itertools.product(*[range(v) for v in e]):
        pos[c] = ora.stream_pos(e, b, c)
    vals = sorted(pos.values())
    assert vals == list(range(int(np.prod(e))))
    # each brick is one contiguous run, in raster order inside the brick
    bricks = {}
    for c, p in pos.items():
        bricks.setdefault(tuple(ci // bi for ci, bi in zip(c, b)), []).append((c, p))
    for key, items in bricks.items():
        ps = sorted(p for _, p in items)
        assert ps == list(range(ps[0], ps[0] + len(ps)))
        items.sort()
        assert [p for _, p in items] == ps
    order = sorted(bricks, key=lambda k: min(p for _, p in bricks[k]))
    assert order == sorted(bricks)


def test_streams_hold_their_subblocks(ora):
    """Codes land in the stream of their sub-block: a field whose value is the
    sub-block id times a large constant (plus a smooth part) gives, with a tiny
    quantization radius, outliers only where prediction fails; instead check
    the stream sizes against brute-force sub-block enumeration."""
    shape = (11, 6, 13)
    L = 3
    codes, soff, recon, ebs = ora.quantize(synth.sinusoids(shape, 1), 1e-3)
    sizes = np.diff(soff)
    lv = level_of_points(shape, L)
    assert sizes[0] == (lv == 1).sum()
    for l in (2, 3):
        s = 1 << (L - l)
        for k in range(1, 8):
            o = ((k >> 2) & 1, (k >> 1) & 1, k & 1)
            cnt = 0
            for p in itertools.product(*[range(n) for n in shape]):
                if lv[p] != l:
                    continue
                g = [v // s for v in p]
                if all(v % s == 0 for v in p) and tuple(v & 1 for v in g) == o:
                    cnt += 1
            assert sizes[1 + 7 * (l - 2) + k - 1] == cnt


def exact_max_violation(x, y, bound):
    """Largest |x - y| - bound over points, in exact arithmetic where needed."""
    xd = x.astype(np.float64)
    yd = y.astype(np.float64)
    diff = np.abs(xd - yd)
    worst = -1.0
    # double differences of float32 values are exact unless the exponents are far
    # apart; re-check every close call with rationals
    close = np.nonzero(diff >= 0.999 * bound)[0] if np.ndim(bound) == 0 else \
        np.nonzero(diff >= 0.999 * bound)[0]
    for i in close:
        b = bound if np.ndim(bound) == 0 else bound[i]
        d = abs(Fraction(float(xd[i])) - Fraction(float(yd[i])))
        if d > Fraction(float(b)):
            return float(d - Fraction(float(b)))
        worst = max(worst, float(d - Fraction(float(b))))
    return worst


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("eb", [1e-2, 1e-3, 1e-5])
@pytest.mark.parametrize("mode", ["rel", "abs"])
def test_error_bound_every_point(ora, dtype, eb, mode):
    shape = (33, 20, 27)
    x = synth.sinusoids(shape, 11, dtype=dtype)
    c = ora.compress(x, eb, mode)
    y = ora.decompress(c)
    fin = np.isfinite(x)
    rng = float(x[fin].max()) - float(x[fin].min())
    eb_abs = eb * rng if mode == "rel" else eb
    L = 3
    lv = level_of_points(shape, L)
    bound = eb_abs / 2.5 ** (L - lv.astype(np.float64))
    assert exact_max_violation(x.ravel(), y.ravel(), bound.ravel()) <= 0
    # the tighter bound of the coarse levels is used: its errors are smaller
    assert np.abs(x - y)[lv == 1].max() <= eb_abs / 2.5 ** 2


def test_constant_field_gives_zero_codes(ora):
    x = np.full((20, 20, 20), 3.25, dtype=np.float32)
    codes, soff, recon, ebs = ora.quantize(x, 1e-3)
    R = 1024
    # the value range is 0, so the bound is taken as absolute (1e-3)
    assert ebs[0] == 1e-3
    lvl1 = codes[soff[0]:soff[1]]
    assert (codes[soff[1]:] == R).all()
    # level 1: all but the origin (predicted as 0) are exact
    assert (lvl1 == R).sum() >= lvl1.size - 1
    assert np.array_equal(recon, x)


@pytest.mark.parametrize("shape", [(16, 16, 16), (13, 9, 21), (40, 33)])
def test_linear_field_gives_zero_codes_on_finer_levels(ora, shape):
    idx = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    f = 7.0 + sum((a + 2) * v for a, v in enumerate(idx))     # exactly representable
    for dtype in (np.float32, np.float64):
        x = f.astype(dtype)
        codes, soff, recon, ebs = ora.quantize(x, 1e-4)
        assert (codes[soff[1]:] == 1024).all()
        assert np.array_equal(recon, x)


def test_nonfinite_values_are_outliers_and_exact(ora):
    x = synth.sinusoids((17, 18, 19), 2)
    x[3, 4, 5] = np.nan
    x[0, 0, 0] = np.inf
    x[16, 17, 18] = -np.inf
    x[8, 8, 8] = np.float32(3e38)
    c = ora.compress(x, 1e-3)
    y = ora.decompress(c)
    bad = ~np.isfinite(x)
    assert np.array_equal(x[bad].view(np.uint32), y[bad].view(np.uint32))
    assert np.isnan(y[3, 4, 5]) and y[0, 0, 0] == np.inf and y[16, 17, 18] == -np.inf
    assert y[8, 8, 8] == x[8, 8, 8]
    fin = np.isfinite(x)
    # range of the finite values sets the bound (the inf values are excluded)
    rng = float(x[fin].max()) - float(x[fin].min())
    assert np.abs(x[fin].astype(np.float64) - y[fin]).max() <= 1e-3 * rng


def test_tiny_radius_forces_outliers(ora):
    x = synth.sinusoids((24, 24, 24), 4)
    c = ora.compress(x, 1e-4, radius=2, max_code_len=12)
    codes, soff = ora.decode_streams(c)
    assert (codes == 0).sum() > 1000
    y = ora.decompress(c)
    assert np.abs(x.astype(np.float64) - y).max() <= 1e-4 * float(x.max() - x.min())


def test_psnr_near_uniform_error_closed_form(ora):
    """With uniform quantization error the PSNR is 20 log10(range / eb) + 4.77 dB;
    the coarse levels' smaller bounds and exact zero codes only raise it."""
    x = synth.sinusoids((64, 64, 64), 7)
    c = ora.compress(x, 1e-3)
    y = ora.decompress(c)
    rng = float(x.max()) - float(x.min())
    mse = np.mean((x.astype(np.float64) - y) ** 2)
    psnr = 20 * np.log10(rng) - 10 * np.log10(mse)
    closed = 20 * np.log10(1 / 1e-3) + 10 * np.log10(3)
    assert closed - 0.5 <= psnr <= closed + 6
