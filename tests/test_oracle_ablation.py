"""Pins of the oracle's ablation modes (Sec. 3.1 optimisations 1, 2, 4, 5;
Fig. 2) and of level counts other than three (Sec. 3.2), against the paper's
equations and closed forms rather than against the oracle's own code.

* Multi-linear prediction (opt. 2): impulse responses are the weights of
  Eq. 3 (1/2, 1/2), Eq. 4 (1/4 each) and Eq. 5 (1/8 each), and no point at
  offset 3 contributes; it is exact on every multi-linear field but not on a
  quadratic, where the cubic stencils of opt. 4 are exact.
* Direct prediction (opt. 1, Eq. 1): the impulse response is a single 1 at
  the coarse point of the cell (offset -1 along each odd axis), so a field
  that is constant on the 2x2x2 blocks of the coarse grid's cells gives
  all-zero-error codes at the finest level.
* Adaptive bound (opt. 5): level l gets eb_abs / ratio^(L-l) (ratio 2.5 in
  the paper, 1 = no adaptive bound), and every point honours its level's
  bound.
* Four levels (Sec. 3.2: a 4-level partition leaves 511/512 of the data
  outside level 1): the level sizes are 1, 7, 56 and 448 parts of 512.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from paper_2509_01626_gb300 import synth


def impulse(ora, n, L, level, g, mode):
    s = 1 << (L - level)
    cs = 2 * s
    resp = {}
    r = range(-7, 8)
    for d in itertools.product(r, r, r):
        p = [g[i] + d[i] * s for i in range(3)]
        if any(q < 0 or q >= n[i] for i, q in enumerate(p)) or any(q % cs for q in p):
            continue
        grid = np.zeros(n)
        grid[tuple(p)] = 1.0
        v = ora.predict_mode(grid, L, level, g, mode)
        if v != 0.0:
            resp[d] = v
    return resp


@pytest.mark.parametrize("k", range(1, 8))
@pytest.mark.parametrize("level", [2, 3])
def test_linear_impulse_weights_eqs_3_to_5(ora, k, level):
    L, n = 3, (40, 40, 40)
    s = 1 << (L - level)
    o = ((k >> 2) & 1, (k >> 1) & 1, k & 1)
    g = tuple((8 + o[i]) * s for i in range(3))
    odd = [a for a in range(3) if o[a]]
    want = {}
    for signs in itertools.product((-1, 1), repeat=len(odd)):
        d = [0, 0, 0]
        for a, sg in zip(odd, signs):
            d[a] = sg
        want[tuple(d)] = 0.5 ** len(odd)     # Eq. 3: 1/2, Eq. 4: 1/4, Eq. 5: 1/8
    assert impulse(ora, n, L, level, g, "linear") == want


@pytest.mark.parametrize("k", range(1, 8))
def test_direct_impulse_is_the_cell_point_eq_1(ora, k):
    L, n = 3, (40, 40, 40)
    o = ((k >> 2) & 1, (k >> 1) & 1, k & 1)
    g = tuple(8 + o[i] for i in range(3))
    want = {tuple(-o[i] for i in range(3)): 1.0}
    assert impulse(ora, n, L, 3, g, "direct") == want


def test_linear_exact_on_multilinear_not_on_quadratic(ora):
    n = (24, 26, 28)
    z, y, x = np.meshgrid(*[np.arange(v, dtype=np.float64) for v in n], indexing="ij")
    tri = 3.0 + 2.0 * z - y + 0.5 * x + z * y - 2.0 * y * x + z * y * x / 8.0
    quad = z * z + 2.0 * y * x
    miss_lin = 0
    for g in itertools.product(range(n[0]), range(n[1]), range(n[2])):
        if all(v % 2 == 0 for v in g):
            continue
        assert ora.predict_mode(tri, 3, 3, g, "linear") == tri[g], g
        interior = all(3 <= g[a] < n[a] - 3 for a in range(3) if g[a] % 2)
        if interior:
            assert ora.predict_mode(quad, 3, 3, g, "cubic") == quad[g], g
            miss_lin += ora.predict_mode(quad, 3, 3, g, "linear") != quad[g]
    assert miss_lin > 0


def test_direct_zero_codes_on_blockwise_constant_field(ora):
    rng = np.random.default_rng(4)
    c = rng.normal(size=(10, 12, 9)).astype(np.float32)
    x = np.ascontiguousarray(c.repeat(2, 0).repeat(2, 1).repeat(2, 2))   # 20 x 24 x 18
    codes, soff, recon, ebs = ora.quantize(x, 1e-3, predictor="direct")
    R = 1024
    assert (codes[soff[8]:soff[15]] == R).all()       # level 3: every residual is zero
    cl, sl, _, _ = ora.quantize(x, 1e-3, predictor="linear")
    assert not (cl[sl[8]:sl[15]] == R).all()
    # the modes are stored in the container and decode to within the bound
    for mode in ("cubic", "linear", "direct"):
        comp = ora.compress(x, 1e-3, predictor=mode)
        assert ora.info(comp)["predictor"] == mode
        y = ora.decompress(comp)
        assert np.abs(y.astype(np.float64) - x).max() <= ora.info(comp)["eb_abs"]


@pytest.mark.parametrize("ratio", [1.0, 1.5, 2.0, 2.5, 4.0])
@pytest.mark.parametrize("L", [2, 3, 4])
def test_adaptive_bound_ratio(ora, ratio, L):
    x = synth.sinusoids((33, 30, 35), 6)
    comp = ora.compress(x, 1e-3, levels=L, eb_ratio=ratio)
    inf = ora.info(comp)
    assert inf["eb_ratio"] == ratio
    ea = Fraction(inf["eb_abs"])
    for l in range(1, L + 1):
        want = ea / Fraction(ratio) ** (L - l)
        # the stored double is the correctly rounded quotient of eb_abs by
        # ratio^(L-l) (itself exact in double for these ratios and L <= 4)
        assert Fraction(inf["eb_level"][l - 1]) == Fraction(float(want)), (l, ratio)
    y = ora.decompress(comp)
    n = x.shape
    lvl = np.full(n, L)
    zz, yy, xx = np.meshgrid(*[np.arange(v) for v in n], indexing="ij")
    for l in range(L - 1, 0, -1):
        s = 1 << (L - l)
        lvl[(zz % s == 0) & (yy % s == 0) & (xx % s == 0)] = l
    err = np.abs(y.astype(np.float64) - x)
    for l in range(1, L + 1):
        assert err[lvl == l].max() <= inf["eb_level"][l - 1], l


def test_four_levels_leave_511_of_512_outside_level_1(ora):
    x = synth.sinusoids((32, 40, 48), 8)
    codes, soff, recon, ebs = ora.quantize(x, 1e-3, levels=4)
    sizes = np.diff(soff)
    n = x.size
    per_level = [sizes[0], sizes[1:8].sum(), sizes[8:15].sum(), sizes[15:22].sum()]
    assert per_level == [n // 512, 7 * n // 512, 56 * n // 512, 448 * n // 512]
    comp = ora.compress(x, 1e-3, levels=4)
    y = ora.decompress(comp)
    assert np.abs(y.astype(np.float64) - x).max() <= ora.info(comp)["eb_abs"]
    for k in range(1, 5):
        s = 1 << (4 - k)
        assert np.array_equal(ora.decompress(comp, k), y[::s, ::s, ::s])


def test_bad_modes_rejected(ora):
    x = synth.sinusoids((8, 8, 8), 1)
    for kw in (dict(eb_ratio=0.5), dict(eb_ratio=float("nan")), dict(eb_ratio=100.0)):
        with pytest.raises(ora.OracleError):
            ora.compress(x, 1e-3, **kw)
