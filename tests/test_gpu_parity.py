"""GPU parity: the CUDA path reproduces the CPU oracle bit for bit.

Compression must give the identical container (codes, outliers, codebooks,
payload, header); every decode (full, progressive to each level, random
boxes) must give bitwise the oracle's values.  Inputs are the seeded
synthetic workloads (paper_2509_01626_gb300.synth) at sizes the oracle
finishes in seconds, ragged shapes that leave partial bricks, 2D and f64
fields, degenerate fields (constant, tiny, non-finite values), and the full
512^3 workload.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2509_01626_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module")
def stzg():
    from paper_2509_01626_gb300 import build, stz

    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    stz.lib()
    return stz


def _nonfinite():
    x = synth.sinusoids((23, 31, 17), 8)
    x[1, 2, 3] = np.nan
    x[0, 0, 0] = np.inf
    x[22, 30, 16] = -np.inf
    x[10, 10, 10] = np.float32(3e38)
    return x


CASES = {
    "sin128_rel1e-3": (lambda: synth.sinusoids((128, 128, 128), synth.seed_for(1)), 1e-3, "rel"),
    "grf128_rel1e-2": (lambda: synth.grf((128, 128, 128), synth.seed_for(2)), 1e-2, "rel"),
    "grf128_rel1e-3": (lambda: synth.grf((128, 128, 128), synth.seed_for(2)), 1e-3, "rel"),
    "grf128_rel1e-4": (lambda: synth.grf((128, 128, 128), synth.seed_for(2)), 1e-4, "rel"),
    "grf128_rel1e-5": (lambda: synth.grf((128, 128, 128), synth.seed_for(2)), 1e-5, "rel"),
    "ragged_37x29x41": (lambda: synth.sinusoids((37, 29, 41), 3), 1e-3, "rel"),
    "ragged_5x3x200": (lambda: synth.sinusoids((5, 3, 200), 4), 1e-4, "rel"),
    "tiny_1x1x1": (lambda: np.array([[[1.5]]], dtype=np.float32), 1e-3, "rel"),
    "tiny_2x3x1": (lambda: synth.sinusoids((2, 3, 1), 5), 1e-3, "abs"),
    "ones_axis_1x40x1": (lambda: synth.sinusoids((1, 40, 1), 6), 1e-3, "rel"),
    "2d_180x360": (lambda: synth.banded2d((180, 360), 7), 1e-3, "rel"),
    "2d_97x33": (lambda: synth.banded2d((97, 33), 8), 1e-2, "abs"),
    "f64_40x33x27": (lambda: synth.sinusoids((40, 33, 27), 9, dtype=np.float64), 1e-5, "rel"),
    "f64_2d_70x90": (lambda: synth.banded2d((70, 90), 10, dtype=np.float64), 1e-6, "rel"),
    "abs_64": (lambda: synth.sinusoids((64, 64, 64), 11), 5e-3, "abs"),
    "const_20": (lambda: np.full((20, 20, 20), 3.25, dtype=np.float32), 1e-3, "rel"),
    "nonfinite": (_nonfinite, 1e-3, "rel"),
    # interior-kernel variants: even rows (paired accesses) over coarse rows that are
    # not a multiple of 16 bytes (element-wise tile copies), and the reverse
    "pair_rows_24x20x108": (lambda: synth.sinusoids((24, 20, 108), 12), 1e-3, "rel"),
    "odd_rows_20x24x63": (lambda: synth.sinusoids((20, 24, 63), 13), 1e-3, "rel"),
}

_cache = {}


def case(name, ora):
    if name not in _cache:
        gen, eb, mode = CASES[name]
        x = np.ascontiguousarray(gen())
        _cache[name] = (x, eb, mode, ora.compress(x, eb, mode))
    return _cache[name]


def describe_mismatch(ora, got, ref):
    """Which stream differs (decode both with the oracle)."""
    msg = [f"sizes gpu={got.size} oracle={ref.size}"]
    n = min(got.size, ref.size)
    d = np.nonzero(got[:n] != ref[:n])[0]
    if d.size:
        msg.append(f"first differing byte {int(d[0])}")
    try:
        cg, sg = ora.decode_streams(got)
        cr, sr = ora.decode_streams(ref)
        for s in range(len(sr) - 1):
            a, b = cg[sg[s]:sg[s + 1]], cr[sr[s]:sr[s + 1]]
            if not np.array_equal(a, b):
                k = int(np.nonzero(a != b)[0][0])
                msg.append(f"stream {s} first code mismatch at {k}: gpu {a[k]} oracle {b[k]}")
                break
    except Exception as e:  # noqa: BLE001
        msg.append(f"gpu container not decodable by the oracle: {e}")
    return "; ".join(msg)


def gpu_compress(stzg, x, eb, mode):
    comp = stzg.compress(torch.from_numpy(x).cuda(), eb, mode)
    return comp


@pytest.mark.parametrize("name", sorted(CASES))
def test_compress_matches_oracle(stzg, ora, name):
    x, eb, mode, ref = case(name, ora)
    got = gpu_compress(stzg, x, eb, mode).cpu().numpy()
    assert got.size == ref.size and np.array_equal(got, ref), describe_mismatch(ora, got, ref)


def _bits(a):
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint64)


@pytest.mark.parametrize("name", sorted(CASES))
def test_decode_matches_oracle(stzg, ora, name):
    x, eb, mode, ref = case(name, ora)
    comp = torch.from_numpy(ref).cuda()
    full = stzg.decompress_full(comp).cpu().numpy()
    want = ora.decompress(ref)
    assert full.shape == want.shape
    assert np.array_equal(_bits(full), _bits(want))
    fin = np.isfinite(x)
    eb_abs = ora.info(ref)["eb_abs"]
    assert (np.abs(full[fin].astype(np.float64) - x[fin]) <= eb_abs).all()
    L = ora.info(ref)["levels"]
    for k in range(1, L + 1):
        p = stzg.decompress_progressive(comp, k).cpu().numpy()
        assert np.array_equal(_bits(p), _bits(ora.decompress(ref, k))), k


@pytest.mark.parametrize("name", ["sin128_rel1e-3", "ragged_37x29x41", "2d_180x360",
                                  "f64_40x33x27", "nonfinite", "ones_axis_1x40x1",
                                  "pair_rows_24x20x108"])
def test_regions_match_oracle(stzg, ora, name):
    x, eb, mode, ref = case(name, ora)
    comp = torch.from_numpy(ref).cuda()
    emax = min(64, max(x.shape))
    boxes = synth.random_boxes(x.shape, 20, 1234, min(8, emax), emax)
    full = ora.decompress(ref)
    for i, (lo, hi) in enumerate(boxes):
        level = 1 + i % 3
        r = stzg.decompress_region(comp, lo, hi, level).cpu().numpy()
        s = 1 << (3 - level)
        sl = tuple(slice(-(-a // s) * s, b, s) for a, b in zip(lo, hi))
        assert np.array_equal(_bits(r), _bits(np.ascontiguousarray(full[sl]))), (lo, hi, level)


@pytest.mark.parametrize("name", ["grf128_rel1e-3", "ragged_37x29x41", "2d_180x360",
                                  "f64_40x33x27", "ones_axis_1x40x1"])
def test_axis_slices_match_oracle(stzg, ora, name):
    """Axis-aligned slices, thin slabs and lines at even and odd coordinates,
    at every level: a slice decodes only the sub-block streams that hold its
    points (Sec. 3.3), and its values equal the oracle's region decode and
    the slice of the oracle's full decode."""
    x, eb, mode, ref = case(name, ora)
    comp = torch.from_numpy(ref).cuda()
    full = ora.decompress(ref)
    nd = x.ndim
    for axis in range(nd):
        n = x.shape[axis]
        for c in sorted({0, 1, n // 2 - n // 2 % 2, n // 2 - n // 2 % 2 + 1, n - 2, n - 1}):
            if not 0 <= c < n:
                continue
            for width in (1, 2, 3):
                if c + width > n:
                    continue
                lo = [0] * nd
                hi = list(x.shape)
                lo[axis], hi[axis] = c, c + width
                for level in (1, 2, 3):
                    s = 1 << (3 - level)
                    sl = tuple(slice(-(-a // s) * s, b, s) for a, b in zip(lo, hi))
                    want = np.ascontiguousarray(full[sl])
                    if want.size == 0:
                        continue
                    r = stzg.decompress_region(comp, lo, hi, level).cpu().numpy()
                    assert np.array_equal(_bits(r), _bits(want)), (axis, c, width, level)
                    o = ora.decompress_region(ref, lo, hi, level)
                    assert np.array_equal(_bits(r), _bits(o)), (axis, c, width, level)
    # lines along each axis (two coordinates fixed)
    if nd == 3:
        for axis in range(3):
            lo = [5 % x.shape[0], 6 % x.shape[1], 7 % x.shape[2]]
            hi = [v + 1 for v in lo]
            lo[axis], hi[axis] = 0, x.shape[axis]
            r = stzg.decompress_region(comp, lo, hi, 3).cpu().numpy()
            sl = tuple(slice(a, b) for a, b in zip(lo, hi))
            assert np.array_equal(_bits(r), _bits(np.ascontiguousarray(full[sl]))), axis


@pytest.mark.parametrize("nsub", [1, 2, 4, 8])
def test_sub_chunk_counts_decode(stzg, ora, nsub):
    """Containers with every sub-chunk count the format allows decode as the
    oracle decodes them, in full and in boxes."""
    x = synth.grf((48, 40, 72), synth.seed_for(2, 7))
    ref = ora.compress(x, 1e-4, nsub=nsub)
    assert ora.info(ref)["nsub"] == nsub
    comp = torch.from_numpy(ref).cuda()
    full = ora.decompress(ref)
    assert np.array_equal(_bits(stzg.decompress_full(comp).cpu().numpy()), _bits(full))
    for lo, hi in synth.random_boxes(x.shape, 4, 99, 8, 40):
        r = stzg.decompress_region(comp, lo, hi, 3).cpu().numpy()
        sl = tuple(slice(a, b) for a, b in zip(lo, hi))
        assert np.array_equal(_bits(r), _bits(np.ascontiguousarray(full[sl]))), (lo, hi)


@pytest.mark.parametrize("name", ["sin3d_f32_22x19x27", "sin3d_f64_9x14x10", "sin2d_f32_37x50"])
def test_golden_containers_decode(stzg, ora, name):
    ref = np.fromfile(os.path.join(GOLDEN, name + ".stz"), dtype=np.uint8)
    got = stzg.decompress_full(torch.from_numpy(ref).cuda()).cpu().numpy()
    assert np.array_equal(_bits(got), _bits(ora.decompress(ref)))


def test_capacity_error_reports_size(stzg, ora):
    x = synth.sinusoids((32, 32, 32), 3)
    xt = torch.from_numpy(x).cuda()
    ref = ora.compress(x, 1e-3)
    small = torch.empty(1000, dtype=torch.uint8, device="cuda")
    with pytest.raises(stzg.StzError) as e:
        stzg.compress(xt, 1e-3, out=small)
    assert e.value.code == stzg.ERR_CAPACITY
    ok = stzg.compress(xt, 1e-3).cpu().numpy()
    assert np.array_equal(ok, ref)


def test_corrupt_payload_is_harmless(stzg, ora):
    """Bit flips after the directory never fault the device: each decode
    returns ok or STZ_ERR_CORRUPT, and the context stays usable."""
    x = synth.sinusoids((48, 40, 36), 12)
    ref = ora.compress(x, 1e-3)
    rng = np.random.default_rng(3)
    start = 256 + 15 * 48
    for _ in range(40):
        b = ref.copy()
        for _ in range(4):
            i = int(rng.integers(start, b.size))
            b[i] ^= np.uint8(1 << int(rng.integers(0, 8)))
        try:
            stzg.decompress_full(torch.from_numpy(b).cuda())
        except stzg.StzError as e:
            assert e.code in (stzg.ERR_CORRUPT, stzg.ERR_ARG)
    torch.cuda.synchronize()
    got = stzg.decompress_full(torch.from_numpy(ref).cuda()).cpu().numpy()
    assert np.array_equal(got, ora.decompress(ref))


def test_full_size_512_grf(stzg, ora):
    """The 512^3 workload: the GPU container equals the oracle's, and the GPU
    decode equals the oracle's reconstruction, in full."""
    x = synth.grf((512, 512, 512), synth.seed_for(2), device="cuda")
    xt = torch.from_numpy(x).cuda()
    got = stzg.compress(xt, 1e-3, "rel").cpu().numpy()
    ref = ora.compress(x, 1e-3, "rel")
    assert got.size == ref.size and np.array_equal(got, ref), describe_mismatch(ora, got, ref)
    comp = torch.from_numpy(ref).cuda()
    full = stzg.decompress_full(comp).cpu().numpy()
    codes, soff, recon, ebs = ora.quantize(x, 1e-3, "rel")
    assert np.array_equal(_bits(full), _bits(recon))
    p2 = stzg.decompress_progressive(comp, 2).cpu().numpy()
    assert np.array_equal(_bits(p2), _bits(recon[::2, ::2, ::2]))
    for lo, hi in synth.random_boxes(x.shape, 5, 77, 16, 256):
        r = stzg.decompress_region(comp, lo, hi, 3).cpu().numpy()
        sl = tuple(slice(a, b) for a, b in zip(lo, hi))
        assert np.array_equal(_bits(r), _bits(np.ascontiguousarray(recon[sl])))
    # 512^2 slices on every axis, at even and odd coordinates (3 or 4 of the 7
    # finest streams decoded)
    for axis in range(3):
        for c in (256, 257, 0, 511):
            lo, hi = [0, 0, 0], [512, 512, 512]
            lo[axis], hi[axis] = c, c + 1
            r = stzg.decompress_region(comp, lo, hi, 3).cpu().numpy()
            sl = tuple(slice(a, b) for a, b in zip(lo, hi))
            assert np.array_equal(_bits(r), _bits(np.ascontiguousarray(recon[sl]))), (axis, c)


def test_region_dependencies_256_grf(stzg, ora):
    """A region decode runs only the level-1 passes the box depends on (cut
    backwards pass by pass, the box growing by the predictor's reach 3t);
    small remainders run in the single coarse block, large ones grid-wide.
    Corner, face, single-point, thin and almost-whole boxes at every level
    equal slices of the oracle's full decode."""
    shape = (256, 256, 256)
    x = synth.grf(shape, synth.seed_for(2, 1))
    ref = ora.compress(x, 1e-3, "rel")
    full = ora.decompress(ref)
    comp = torch.from_numpy(ref).cuda()
    boxes = [((0, 0, 0), (1, 1, 1)), ((255, 255, 255), (256, 256, 256)),
             ((0, 0, 0), (256, 256, 256)), ((1, 1, 1), (256, 256, 256)),
             ((0, 0, 0), (255, 255, 255)), ((100, 0, 37), (101, 256, 38)),
             ((0, 128, 0), (256, 129, 256)), ((3, 5, 7), (9, 250, 11)),
             ((120, 120, 120), (136, 136, 136)), ((0, 0, 200), (256, 256, 256)),
             ((250, 0, 0), (256, 6, 256))]
    boxes += synth.random_boxes(shape, 8, 4321, 1, 200)
    for level in (1, 2, 3):
        s = 1 << (3 - level)
        for lo, hi in boxes:
            sl = tuple(slice(-(-a // s) * s, b, s) for a, b in zip(lo, hi))
            want = np.ascontiguousarray(full[sl])
            if want.size == 0:
                continue
            r = stzg.decompress_region(comp, lo, hi, level).cpu().numpy()
            assert np.array_equal(_bits(r), _bits(want)), (lo, hi, level)


def test_header_cache_follows_new_container(stzg, ora):
    """Decodes of a device buffer reuse its parsed header; when another
    container is written to the same address (same size passed), the decode
    still returns the new container's values, also when its shape differs."""
    xa = synth.sinusoids((40, 36, 52), 31)
    xb = synth.sinusoids((40, 36, 52), 32) * 3.0
    xc = synth.sinusoids((24, 60, 33), 33)
    ca, cb, cc = (ora.compress(x, 1e-3) for x in (xa, xb, xc))
    cap = max(ca.size, cb.size, cc.size)
    buf = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    out = torch.empty(max(xa.size, xc.size), dtype=torch.float32, device="cuda")
    ws = stzg.alloc_workspace((40, 60, 52), torch.float32)
    for _ in range(2):
        for c, x in ((ca, xa), (cb, xb), (cc, xc), (ca, xa)):
            buf.zero_()
            buf[: c.size].copy_(torch.from_numpy(c))
            meta = {"shape": x.shape, "dtype": torch.float32, "ndim": 3, "levels": 3}
            y = stzg.decompress_full(buf, out=out[: x.size], workspace=ws,
                                     meta=meta).cpu().numpy()
            assert np.array_equal(_bits(y), _bits(ora.decompress(c)))
            r = stzg.decompress_region(buf, (2, 3, 4), (20, 30, 31), 2, out=out, workspace=ws,
                                       meta=meta).cpu().numpy()
            assert np.array_equal(_bits(r), _bits(ora.decompress_region(c, (2, 3, 4),
                                                                        (20, 30, 31), 2)))
