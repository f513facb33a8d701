"""GPU parity of the ROI selection module (Sec. 3.3, last paragraph): per
slice or block the value range or the maximum, threshold or top-x%
selection.  The selection and every unit's metric equal the oracle's bit for
bit, on fields with ties and non-finite values, on slices along each axis,
on ragged blocks, in 2D and f64.  The paper's workflow -- decode the coarse
level, pick the regions of interest on it, decode only those at full
resolution, one by one or all in one batched call -- gives regions equal to
the oracle's decodes of the same boxes.
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


def check(stzg, ora, x, block, metric, mode, value):
    sel, met = stzg.roi_select(torch.from_numpy(x).cuda(), block, metric, mode, value,
                               metric_out=True)
    wsel, wmet = ora.roi_select(x, block, metric, mode, value)
    assert np.array_equal(sel.cpu().numpy(), wsel), (block, metric, mode, value)
    assert np.array_equal(met.cpu().numpy().view(np.uint64), wmet.view(np.uint64)), \
        (block, metric, mode, value)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_roi_matches_oracle_with_ties_and_nonfinite(stzg, ora, dtype):
    rng = np.random.default_rng(11)
    x = np.round(rng.normal(size=(37, 45, 53)) * 3).astype(dtype)
    x[3, 4, 5] = np.nan
    x[10, :, :] = np.inf
    x[0, 0, 0] = -np.inf
    x[20, 20, 20] = -0.0
    blocks = [(1, 45, 53), (37, 1, 53), (37, 45, 1), (8, 8, 8), (5, 7, 11), (37, 45, 53),
              (1, 1, 64), (2, 3, 1)]
    for block in blocks:
        for metric in ("range", "max"):
            for mode, value in (("threshold", 4.0), ("top", 0.01), ("top", 0.25), ("top", 1.0)):
                check(stzg, ora, x, block, metric, mode, value)


def test_roi_2d_and_smooth_fields(stzg, ora):
    for x, block in ((synth.banded2d((180, 360), 3), (16, 16)),
                     (synth.banded2d((97, 33), 4, dtype=np.float64), (1, 33)),
                     (synth.grf((64, 64, 64), 5), (4, 4, 4)),
                     (synth.sinusoids((30, 40, 50), 6), (1, 40, 50))):
        for metric in ("range", "max"):
            check(stzg, ora, x, block, metric, "top", 0.05)
            check(stzg, ora, x, block, metric, "threshold", float(np.median(x)))


def test_roi_workflow_coarse_then_regions(stzg, ora):
    """Decode level 1 (the 1/64 coarse grid), select the top 2% of its 4^3
    blocks by value range, then decode those regions at full resolution,
    one by one and with one decode_regions call: each equals the oracle's
    region decode."""
    x = synth.grf((128, 128, 128), synth.seed_for(2, 9))
    ref = ora.compress(x, 1e-3, "rel")
    comp = torch.from_numpy(ref).cuda()
    coarse = stzg.decompress_progressive(comp, 1)
    sel = stzg.roi_select(coarse, (4, 4, 4), "range", "top", 0.02)
    wsel, _ = ora.roi_select(ora.decompress(ref, 1), (4, 4, 4), "range", "top", 0.02)
    assert np.array_equal(sel.cpu().numpy(), wsel)
    boxes = stzg.roi_boxes(sel.cpu().numpy(), tuple(coarse.shape), (4, 4, 4), 4, x.shape)
    assert len(boxes) == int(np.ceil(0.02 * 8 ** 3))
    batched = stzg.decode_regions(comp, boxes, 3, level1=coarse)
    assert len(batched) == len(boxes)
    for (lo, hi), b in zip(boxes, batched):
        want = ora.decompress_region(ref, lo, hi, 3).view(np.uint32)
        r = stzg.decompress_region(comp, lo, hi, 3).cpu().numpy()
        assert np.array_equal(r.view(np.uint32), want), (lo, hi)
        assert np.array_equal(b.cpu().numpy().view(np.uint32), want), (lo, hi)
    # the same boxes at level 2 (every other point), tables given, without waiting
    tables = stzg.decode_tables(comp, stzg.header_bytes(comp))
    outs, status = stzg.decode_regions(comp, boxes[:5], 2, level1=coarse, tables=tables,
                                       check=False)
    assert (status.cpu().numpy() == 0).all()
    for (lo, hi), b in zip(boxes[:5], outs):
        want = ora.decompress_region(ref, lo, hi, 2).view(np.uint32)
        assert np.array_equal(b.cpu().numpy().view(np.uint32), want), (lo, hi)


def test_roi_rejects_bad_arguments(stzg):
    x = torch.zeros((8, 8, 8), device="cuda")
    for kw in (dict(mode="top", value=0.0), dict(mode="top", value=2.0)):
        with pytest.raises(stzg.StzError):
            stzg.roi_select(x, (2, 2, 2), "range", **kw)
    with pytest.raises(stzg.StzError):
        stzg.roi_select(x, (0, 2, 2), "range", "top", 0.5)
