"""Pins of the oracle's predictors against the paper's equations and closed forms.

* Impulse responses reproduce the printed weights of Eq. 6 (1D cubic,
  -1/16, 9/16, 9/16, -1/16), Eq. 7 (approximate bicubic, 9/32 inner, -1/32
  diagonal corners) and Eq. 8 (approximate tricubic, 9/64 inner, -1/64 outer),
  and every other coarse point has weight 0.
* Eqs. 6-8 average cubic interpolants along lines, so they reproduce every
  polynomial of total degree <= 3 exactly and no quartic: checked on integer
  polynomials whose values are exact in floating point.
* The boundary rules (midpoint, Eqs. 3-5; one-sided extrapolation) are exact
  on multilinear fields wherever an axis has at least two coarse neighbours.
"""
import itertools

import numpy as np
import pytest

W6 = {-3: -1 / 16, -1: 9 / 16, 1: 9 / 16, 3: -1 / 16}          # Eq. 6
W7_INNER, W7_OUTER = 9 / 32, -1 / 32                             # Eq. 7
W8_INNER, W8_OUTER = 9 / 64, -1 / 64                             # Eq. 8


def expected_weights(odd_axes):
    """Offsets (fine-grid units) -> weight of the interior stencil."""
    w = {}
    if len(odd_axes) == 1:
        a = odd_axes[0]
        for o, v in W6.items():
            d = [0, 0, 0]
            d[a] = o
            w[tuple(d)] = v
    elif len(odd_axes) == 2:
        a, b = odd_axes
        for sa, sb in itertools.product((-1, 1), repeat=2):
            d = [0, 0, 0]
            d[a], d[b] = sa, sb
            w[tuple(d)] = W7_INNER
            d[a], d[b] = 3 * sa, 3 * sb
            w[tuple(d)] = W7_OUTER
    else:
        for s in itertools.product((-1, 1), repeat=3):
            w[tuple(s)] = W8_INNER
            w[tuple(3 * v for v in s)] = W8_OUTER
    return w


def impulse_response(ora, n, L, level, g, dtype=np.float64, axis=0, t=1):
    """Prediction at g with a unit impulse at each coarse point near g."""
    s = 1 << (L - level)
    cs = 2 * s if level >= 2 else None
    resp = {}
    rng = range(-7, 8)
    for d in itertools.product(rng, rng, rng):
        p = [g[i] + d[i] * s for i in range(3)]
        if any(q < 0 or q >= n[i] for i, q in enumerate(p)):
            continue
        if level >= 2 and any(q % cs for q in p):
            continue
        grid = np.zeros(n, dtype=dtype)
        grid[tuple(p)] = 1
        v = float(ora.predict(grid, L, level, g, axis, t))
        if v != 0.0:
            resp[d] = v
    return resp


@pytest.mark.parametrize("level", [2, 3])
@pytest.mark.parametrize("k", range(1, 8))
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_interior_impulse_weights(ora, level, k, dtype):
    L = 3
    n = (40, 40, 40)
    s = 1 << (L - level)
    o = ((k >> 2) & 1, (k >> 1) & 1, k & 1)
    g = tuple((8 + o[i]) * s for i in range(3))     # grid coordinate 8 + o: interior
    odd = [a for a in range(3) if o[a]]
    got = impulse_response(ora, n, L, level, g, dtype)
    want = expected_weights(odd)
    assert got == pytest.approx(want, abs=0, rel=0)
    assert sum(got.values()) == 1.0


def test_base_pass_interior_weights(ora):
    """Level-1 passes use Eq. 6 along the pass axis with the pass stride."""
    L, n = 3, (64, 64, 64)       # level-1 grid: stride 4, extent 16
    for axis in range(3):
        for t, c in ((1, 9), (2, 6)):   # c: odd multiple of t with c-3t >= 0, c+3t < 16
            g = [8 * 4, 8 * 4, 8 * 4]
            g[axis] = c * 4
            resp = impulse_response(ora, n, L, 1, tuple(g), np.float64, axis=axis, t=t)
            want = {}
            for off, w in W6.items():
                d = [0, 0, 0]
                d[axis] = off * t
                want[tuple(d)] = w
            assert resp == want, (axis, t)


def int_poly(n, coeffs):
    z, y, x = np.meshgrid(*[np.arange(v, dtype=np.int64) for v in n], indexing="ij")
    f = np.zeros(n, dtype=np.int64)
    for (i, j, k), c in coeffs.items():
        f += c * z ** i * y ** j * x ** k
    return f


def random_coeffs(rng, max_deg, cmax):
    return {(i, j, k): int(rng.integers(-cmax, cmax + 1))
            for i in range(4) for j in range(4) for k in range(4) if i + j + k <= max_deg}


@pytest.mark.parametrize("seed", range(4))
def test_cubic_exact_on_total_degree_3(ora, seed):
    rng = np.random.default_rng(seed)
    n = (22, 21, 20)
    f = int_poly(n, random_coeffs(rng, 3, 3))
    assert np.abs(f).max() < 2 ** 40
    grid = f.astype(np.float64)
    L = 3
    checked = 0
    for level in (2, 3):
        s = 1 << (L - level)
        m = [-(-v // s) for v in n]
        for gz, gy, gx in itertools.product(*[range(v) for v in m]):
            gg = (gz, gy, gx)
            odd = [a for a in range(3) if gg[a] & 1]
            if not odd:
                continue
            if not all(3 <= gg[a] <= m[a] - 4 for a in odd):
                continue
            p = tuple(v * s for v in gg)
            assert ora.predict(grid, L, level, p) == grid[p], (level, p)
            checked += 1
    assert checked > 500


@pytest.mark.parametrize("k", range(1, 8))
def test_cubic_not_exact_on_quartics(ora, k):
    """A quartic along the odd axes breaks the stencil: the test has teeth."""
    n = (24, 24, 24)
    odd = [a for a in range(3) if (k >> (2 - a)) & 1]
    coeffs = {}
    e = [0, 0, 0]
    if len(odd) == 1:
        e[odd[0]] = 4
    else:
        e[odd[0]] = 2
        e[odd[1]] = 2
    coeffs[tuple(e)] = 1
    grid = int_poly(n, coeffs).astype(np.float64)
    g = tuple(11 if a in odd else 10 for a in range(3))
    assert ora.predict(grid, 3, 3, g) != grid[g]


@pytest.mark.parametrize("n", [(13, 10, 11), (9, 7, 12), (16, 16, 16), (6, 17, 9)])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_boundary_rules_exact_on_multilinear(ora, n, dtype):
    rng = np.random.default_rng(sum(n))
    c = rng.integers(-4, 5, size=8)
    z, y, x = np.meshgrid(*[np.arange(v, dtype=np.int64) for v in n], indexing="ij")
    f = (c[0] + c[1] * z + c[2] * y + c[3] * x + c[4] * z * y + c[5] * z * x + c[6] * y * x
         + c[7] * z * y * x)
    grid = f.astype(dtype)
    L = 3
    checked = 0
    for level in (2, 3):
        s = 1 << (L - level)
        m = [-(-v // s) for v in n]
        if min(m) < 3:
            continue
        for gg in itertools.product(*[range(v) for v in m]):
            if not any(v & 1 for v in gg):
                continue
            p = tuple(v * s for v in gg)
            assert ora.predict(grid, L, level, p) == grid[p], (level, p)
            checked += 1
    assert checked > 0


def test_boundary_extrapolation_and_copy_weights(ora):
    """At the top edge (no +1 neighbour) the rule is 1.5 v(-1) - 0.5 v(-3); with
    only v(-1) available it is a copy (Sec. 3.1: predicted from available data)."""
    n = (1, 1, 12)
    # level 3, x = 11 is odd and the last point: -1 = 10, -3 = 8
    resp = impulse_response(ora, n, 3, 3, (0, 0, 11))
    assert resp == {(0, 0, -1): 1.5, (0, 0, -3): -0.5}
    n2 = (1, 1, 2)
    resp = impulse_response(ora, n2, 3, 3, (0, 0, 1))
    assert resp == {(0, 0, -1): 1.0}
    # midpoint (Eq. 3) near the lower edge: x = 1 has -1 = 0 and +1 = 2, no -3
    resp = impulse_response(ora, (1, 1, 12), 3, 3, (0, 0, 1))
    assert resp == {(0, 0, -1): 0.5, (0, 0, 1): 0.5}
    # bilinear (Eq. 4) at a 2D corner region
    resp = impulse_response(ora, (1, 12, 12), 3, 3, (0, 1, 1))
    assert resp == {(0, -1, -1): 0.25, (0, -1, 1): 0.25, (0, 1, -1): 0.25, (0, 1, 1): 0.25}
    # trilinear (Eq. 5)
    resp = impulse_response(ora, (12, 12, 12), 3, 3, (1, 1, 1))
    assert resp == {d: 0.125 for d in itertools.product((-1, 1), repeat=3)}
