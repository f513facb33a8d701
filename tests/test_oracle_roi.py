"""Pins of the oracle's ROI selection module (Sec. 3.3, last paragraph:
range- or maximum-value thresholding per slice or block, by a threshold or
as the top x% of units).

* Closed forms: on f = a z + b y + c x the range of a z-slice is
  |b| (ny - 1) + |c| (nx - 1) and its maximum is known, so the top slices and
  the thresholded ones follow exactly.
* Brute force with numpy (a separate plain implementation: reductions over
  reshaped views, a lexicographic sort) on random fields with repeated
  values, non-finite values and ragged blocks.
"""
import math

import numpy as np
import pytest


def brute(x, block, metric, mode, value):
    x3 = x if x.ndim == 3 else x[None]
    b = tuple(block) if x.ndim == 3 else (1,) + tuple(block)
    nb = [-(-x3.shape[a] // b[a]) for a in range(3)]
    met = np.full(nb, -np.inf)
    for i in range(nb[0]):
        for j in range(nb[1]):
            for k in range(nb[2]):
                v = x3[i * b[0]:(i + 1) * b[0], j * b[1]:(j + 1) * b[1],
                       k * b[2]:(k + 1) * b[2]].astype(np.float64)
                v = v[np.isfinite(v)]
                if v.size:
                    met[i, j, k] = v.max() if metric == "max" else v.max() - v.min()
    met = met.reshape(-1)
    if mode == "threshold":
        sel = np.nonzero(met >= value)[0]
    else:
        kk = min(met.size, math.ceil(value * met.size))
        order = np.lexsort((np.arange(met.size), -met))
        sel = np.sort(order[:kk])
    return sel, met


def test_slices_of_a_linear_field(ora):
    n = (12, 10, 14)
    z, y, x = np.meshgrid(*[np.arange(v, dtype=np.float64) for v in n], indexing="ij")
    f = (3.0 * z - 2.0 * y + 0.5 * x).astype(np.float32)
    # z-slices: every slice has the same range, the maximum grows with z
    sel, met = ora.roi_select(f, (1, n[1], n[2]), "range", "threshold", 0.0)
    assert np.array_equal(met, np.full(n[0], 2.0 * 9 + 0.5 * 13))
    assert np.array_equal(sel, np.arange(n[0]))
    sel, met = ora.roi_select(f, (1, n[1], n[2]), "max", "top", 0.25)
    assert np.array_equal(met, 3.0 * np.arange(n[0]) + 0.5 * 13)
    assert np.array_equal(sel, np.arange(n[0] - 3, n[0]))        # ceil(0.25 * 12) = 3
    # y-slices: the maximum falls with y; range 3 * 11 + 0.5 * 13
    sel, met = ora.roi_select(f, (n[0], 1, n[2]), "max", "threshold", 3.0 * 11 + 0.5 * 13 - 2.0)
    assert np.array_equal(met, 3.0 * 11 + 0.5 * 13 - 2.0 * np.arange(n[1]))
    assert np.array_equal(sel, [0, 1])
    # x-slices by range: all equal, top 50% takes the lowest indices
    sel, met = ora.roi_select(f, (n[0], n[1], 1), "range", "top", 0.5)
    assert np.array_equal(met, np.full(n[2], 3.0 * 11 + 2.0 * 9))
    assert np.array_equal(sel, np.arange(7))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("block", [(4, 5, 6), (1, 13, 17), (13, 1, 1), (3, 3, 64), (7, 7, 7)])
def test_against_brute_force(ora, dtype, block):
    rng = np.random.default_rng(sum(block))
    x = np.round(rng.normal(size=(13, 17, 19)) * 4).astype(dtype)   # many ties
    x[2, 3, 4] = np.nan
    x[5, :, :] = np.inf          # a whole plane of non-finite values
    x[0, 0, 0] = -np.inf
    for metric in ("range", "max"):
        for mode, value in (("threshold", 3.0), ("threshold", -np.inf), ("top", 0.01),
                            ("top", 0.3), ("top", 1.0)):
            got, met = ora.roi_select(x, block, metric, mode, value)
            want, wmet = brute(x, block, metric, mode, value)
            assert np.array_equal(met, wmet), (metric, mode, value)
            assert np.array_equal(got, want), (metric, mode, value)


def test_2d_and_single_unit(ora):
    rng = np.random.default_rng(3)
    x = rng.normal(size=(30, 41)).astype(np.float32)
    got, met = ora.roi_select(x, (8, 8), "max", "top", 0.2)
    want, wmet = brute(x, (8, 8), "max", "top", 0.2)
    assert np.array_equal(got, want) and np.array_equal(met, wmet)
    got, met = ora.roi_select(x, (64, 64), "range", "top", 1.0)
    assert np.array_equal(got, [0]) and met[0] == float(x.max()) - float(x.min())


def test_bad_arguments(ora):
    x = np.zeros((4, 4, 4), dtype=np.float32)
    for kw in (dict(mode="top", value=0.0), dict(mode="top", value=1.5)):
        with pytest.raises(ora.OracleError):
            ora.roi_select(x, (2, 2, 2), "range", **kw)
    with pytest.raises(ora.OracleError):
        ora.roi_select(x, (0, 2, 2), "range", "top", 0.5)
