"""Which chunks a region decode reads (Sec. 3.3, random access), checked on the
host with no GPU: stz_region_chunks reports, per stream, the chunks that
stz_decompress_region entropy-decodes.

The check is a brute-force dependency walk written here from the paper's
prediction rules: the box's lattice points at the requested level, then for
each level-l point its interpolation taps on the coarser grid (Eq. 6 along
one odd axis, Eq. 7 / Eq. 8 inner points and diagonal corners, the one-sided
rules at the field boundary), and the copies of the points the coarser grid
holds itself.  Each stream's needed bricks are those holding its needed
points.  The plan must cover every one of them, skip exactly the streams
with none, and on boxes away from the boundary read no more than their
bounding boxes.  An axis-aligned slice at an even coordinate holds no point
whose coordinate along that axis is odd, so it reads 3 of the 7 finest
streams (4 at an odd coordinate): the slice decoding saving of Sec. 3.3.
"""
import itertools

import numpy as np
import pytest

from paper_2509_01626_gb300 import synth

L = 3
BRICK3 = (8, 16, 16)


@pytest.fixture(scope="module")
def stzmod():
    from paper_2509_01626_gb300 import build, stz

    build.build()
    stz.lib()
    return stz


def _ext(n, j):
    s = 1 << (L - j)
    return tuple(-(-d // s) for d in n)


def _taps(g, m):
    """Coarse taps (points of G_{j-1}) of the level-j point g (G_j extent m)."""
    odd = [a for a in range(3) if g[a] % 2]
    c = [v // 2 for v in g]
    cubic = all(g[a] >= 3 and g[a] + 3 < m[a] for a in odd)
    if cubic:
        if len(odd) == 1:
            sets = [[c[a] + d for d in (-1, 0, 1, 2)] if a in odd else [c[a]] for a in range(3)]
            return set(itertools.product(*sets))
        inner = [[c[a], c[a] + 1] if a in odd else [c[a]] for a in range(3)]
        outer_pts = set()
        for corner in itertools.product((-1, 2), repeat=len(odd)):
            p = list(c)
            for a, d in zip(odd, corner):
                p[a] = c[a] + d
            outer_pts.add(tuple(p))
        return set(itertools.product(*inner)) | outer_pts
    sets = []
    for a in range(3):
        if a not in odd:
            sets.append([c[a]])
        elif g[a] + 1 < m[a]:
            sets.append([c[a], c[a] + 1])       # midpoint
        elif g[a] >= 3:
            sets.append([c[a], c[a] - 1])       # extrapolation from -1, -3
        else:
            sets.append([c[a]])                 # copy of -1
    return set(itertools.product(*sets))


def brute_bricks(n, lo, hi, k):
    """{stream: set of bricks} of levels 2..k that a box decode needs."""
    sk = 1 << (L - k)
    need = set(itertools.product(*[range(-(-lo[a] // sk), -(-hi[a] // sk)) for a in range(3)]))
    out = {}
    for j in range(k, 1, -1):
        m = _ext(n, j)
        coarse = set()
        for g in need:
            if all(v % 2 == 0 for v in g):
                coarse.add(tuple(v // 2 for v in g))
                continue
            K = 4 * (g[0] % 2) + 2 * (g[1] % 2) + (g[2] % 2)
            sid = 1 + 7 * (j - 2) + K - 1
            cell = tuple(v // 2 for v in g)
            out.setdefault(sid, set()).add(tuple(cell[a] // BRICK3[a] for a in range(3)))
            coarse |= _taps(g, m)
        need = coarse
    return out


def bbox_count(bricks):
    arr = np.array(sorted(bricks))
    return int(np.prod(arr.max(axis=0) - arr.min(axis=0) + 1))


@pytest.fixture(scope="module")
def hdr(ora):
    n = (70, 61, 83)
    x = synth.sinusoids(n, 5, n_terms=4)
    comp = ora.compress(x, 1e-3, "rel")
    return n, bytes(comp[:1984].tobytes()), comp.size


def plan(stzmod, hdr, lo, hi, k):
    n, h, nb = hdr
    return stzmod.region_chunks(h, nb, lo, hi, k)


def check_box(stzmod, hdr, lo, hi, k, exact):
    n = hdr[0]
    got = plan(stzmod, hdr, lo, hi, k)
    want = brute_bricks(n, lo, hi, k)
    for sid in range(1, 1 + 7 * (k - 1)):
        bricks = want.get(sid, set())
        if not bricks:
            assert got[sid] == 0, (lo, hi, k, sid)
            continue
        assert got[sid] >= bbox_count(bricks), (lo, hi, k, sid, got[sid])
        if exact:
            assert got[sid] == bbox_count(bricks), (lo, hi, k, sid, got[sid])
    for sid in range(1 + 7 * (k - 1), len(got)):
        assert got[sid] == 0


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_slice_reads_three_or_four_of_seven_finest_streams(stzmod, hdr, axis):
    n = hdr[0]
    for z in (20, 21, 36, 37):
        lo, hi = [0, 0, 0], list(n)
        lo[axis], hi[axis] = z, z + 1
        got = plan(stzmod, hdr, lo, hi, 3)
        level3 = got[8:15]
        live = [K for K in range(1, 8) if level3[K - 1] > 0]
        bit = 1 << (2 - axis)
        want = [K for K in range(1, 8) if bool(K & bit) == bool(z % 2)]
        assert live == want, (axis, z, level3)
        assert len(live) == (4 if z % 2 else 3)
        # at level 2 the same rule applies to the coarse plane of an even slice
        level2 = got[1:8]
        if z % 2 == 0:
            zz = z // 2
            live2 = [K for K in range(1, 8) if level2[K - 1] > 0]
            assert live2 == [K for K in range(1, 8) if bool(K & bit) == bool(zz % 2)]
        else:
            assert all(c > 0 for c in level2)
        check_box(stzmod, hdr, lo, hi, 3, exact=False)


def test_slices_and_boxes_against_dependency_walk(stzmod, hdr):
    n = hdr[0]
    rng = np.random.default_rng(7)
    # interior boxes: the plan equals the walk's bounding boxes
    for _ in range(12):
        e = rng.integers(1, 14, size=3)
        lo = [int(rng.integers(12, n[a] - 12 - e[a])) for a in range(3)]
        hi = [lo[a] + int(e[a]) for a in range(3)]
        for k in (2, 3):
            check_box(stzmod, hdr, lo, hi, k, exact=True)
    # boxes touching the boundary, single lines, points: covered, skipped where empty
    cases = [((0, 0, 0), (3, 5, 7)), ((69, 60, 82), (70, 61, 83)), ((0, 30, 40), (70, 31, 41)),
             ((33, 0, 0), (34, 61, 83)), ((5, 6, 7), (6, 7, 8)), ((64, 0, 70), (70, 61, 83))]
    for lo, hi in cases:
        for k in (1, 2, 3):
            check_box(stzmod, hdr, lo, hi, k, exact=False)


def test_full_box_reads_every_chunk(stzmod, hdr):
    n = hdr[0]
    got = plan(stzmod, hdr, (0, 0, 0), n, 3)
    m1 = _ext(n, 1)
    want = [int(np.prod([-(-m1[a] // BRICK3[a]) for a in range(3)]))]
    for j in (2, 3):
        m = _ext(n, j)
        for K in range(1, 8):
            o = ((K >> 2) & 1, (K >> 1) & 1, K & 1)
            e = [(m[a] - o[a] + 1) // 2 for a in range(3)]
            want.append(int(np.prod([-(-e[a] // BRICK3[a]) for a in range(3)])))
    assert got == want
