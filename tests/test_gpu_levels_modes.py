"""GPU parity for level counts other than three (Sec. 3.2: "4-level (or
higher)" for large fields) and for the predictor ablation of Sec. 3.1
(opt. 1 direct Eq. 1, opt. 2 multi-linear Eqs. 3-5, opt. 4 cubic Eqs. 6-8,
opt. 5 adaptive-bound ratio), through stz_compress_ex: every container is
byte-identical to the oracle's, and every decode of an oracle container --
full, each progressive level, boxes and slices -- equals the oracle's bit
for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2509_01626_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stzg():
    from paper_2509_01626_gb300 import build, stz

    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    stz.lib()
    return stz


def _bits(a):
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint64)


FIELDS = {
    "grf_96x80x112": lambda: synth.grf((96, 80, 112), synth.seed_for(2, 31)),
    "sin_70x61x83": lambda: synth.sinusoids((70, 61, 83), 32),
    "f64_50x41x66": lambda: synth.sinusoids((50, 41, 66), 33, dtype=np.float64),
    "2d_300x257": lambda: synth.banded2d((300, 257), 34),
}


def check_decodes(stzg, ora, ref, x, boxes=6, seed=5):
    comp = torch.from_numpy(ref).cuda()
    inf = ora.info(ref)
    L = inf["levels"]
    full = ora.decompress(ref)
    got = stzg.decompress_full(comp).cpu().numpy()
    assert np.array_equal(_bits(got), _bits(full))
    fin = np.isfinite(x)
    assert (np.abs(got[fin].astype(np.float64) - x[fin]) <= inf["eb_abs"]).all()
    for k in range(1, L + 1):
        p = stzg.decompress_progressive(comp, k).cpu().numpy()
        assert np.array_equal(_bits(p), _bits(ora.decompress(ref, k))), k
    rng = np.random.default_rng(seed)
    cases = synth.random_boxes(x.shape, boxes, seed, 1, max(2, min(x.shape) // 2))
    # slices at even and odd coordinates along every axis
    for axis in range(x.ndim):
        for c in (x.shape[axis] // 2 & ~1, x.shape[axis] // 2 | 1):
            lo, hi = [0] * x.ndim, list(x.shape)
            lo[axis], hi[axis] = c, c + 1
            cases.append((tuple(lo), tuple(hi)))
    for lo, hi in cases:
        level = int(rng.integers(1, L + 1))
        s = 1 << (L - level)
        sl = tuple(slice(-(-a // s) * s, b, s) for a, b in zip(lo, hi))
        want = np.ascontiguousarray(full[sl])
        if want.size == 0:
            continue
        r = stzg.decompress_region(comp, lo, hi, level).cpu().numpy()
        assert np.array_equal(_bits(r), _bits(want)), (lo, hi, level)


@pytest.mark.parametrize("levels", [1, 2, 4, 5])
@pytest.mark.parametrize("name", sorted(FIELDS))
def test_levels_compress_and_decode_match_oracle(stzg, ora, name, levels):
    x = np.ascontiguousarray(FIELDS[name]())
    ref = ora.compress(x, 1e-3, "rel", levels=levels)
    got = stzg.compress(torch.from_numpy(x).cuda(), 1e-3, "rel", levels=levels).cpu().numpy()
    assert got.size == ref.size and np.array_equal(got, ref), (name, levels)
    check_decodes(stzg, ora, ref, x)


@pytest.mark.parametrize("predictor", ["linear", "direct", "cubic"])
@pytest.mark.parametrize("ratio", [1.0, 2.5, 4.0])
@pytest.mark.parametrize("levels", [2, 3])
def test_ablation_modes_match_oracle(stzg, ora, predictor, ratio, levels):
    x = synth.grf((72, 64, 88), synth.seed_for(2, 40))
    kw = dict(levels=levels, predictor=predictor, eb_ratio=ratio)
    ref = ora.compress(x, 1e-3, "rel", **kw)
    got = stzg.compress(torch.from_numpy(x).cuda(), 1e-3, "rel", **kw).cpu().numpy()
    assert got.size == ref.size and np.array_equal(got, ref), kw
    info = ora.info(got)
    assert info["predictor"] == predictor and info["eb_ratio"] == ratio
    check_decodes(stzg, ora, ref, x, boxes=4)


@pytest.mark.parametrize("predictor", ["linear", "direct"])
def test_ablation_modes_2d_f64_and_ragged(stzg, ora, predictor):
    for x in (synth.banded2d((181, 95), 41, dtype=np.float64),
              synth.sinusoids((9, 30, 17), 42), synth.sinusoids((1, 40, 3), 43)):
        ref = ora.compress(x, 1e-4, "rel", predictor=predictor)
        got = stzg.compress(torch.from_numpy(x).cuda(), 1e-4, "rel",
                            predictor=predictor).cpu().numpy()
        assert np.array_equal(got, ref), (x.shape, predictor)
        check_decodes(stzg, ora, ref, x, boxes=3)


def test_four_levels_256_cube(stzg, ora):
    """L = 4 on a 256^3 field (level 1 = 32^3, 1/512 of the points)."""
    x = synth.grf((256, 256, 256), synth.seed_for(4, 5), slope=-5.0 / 3.0, lognormal_sigma=None)
    ref = ora.compress(x, 1e-4, "rel", levels=4)
    got = stzg.compress(torch.from_numpy(x).cuda(), 1e-4, "rel", levels=4).cpu().numpy()
    assert got.size == ref.size and np.array_equal(got, ref)
    comp = torch.from_numpy(ref).cuda()
    full = ora.decompress(ref)
    assert np.array_equal(_bits(stzg.decompress_full(comp).cpu().numpy()), _bits(full))
    for k in (1, 2, 3):
        s = 1 << (4 - k)
        p = stzg.decompress_progressive(comp, k).cpu().numpy()
        assert np.array_equal(_bits(p), _bits(full[::s, ::s, ::s])), k


def test_bad_options_rejected(stzg):
    x = torch.from_numpy(synth.sinusoids((16, 16, 16), 1)).cuda()
    for kw in (dict(levels=7), dict(eb_ratio=0.5), dict(eb_ratio=65.0)):
        with pytest.raises((stzg.StzError, ValueError)) as e:
            stzg.compress(x, 1e-3, **kw)
        if isinstance(e.value, stzg.StzError):
            assert e.value.code == stzg.ERR_ARG
