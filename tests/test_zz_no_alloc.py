"""Region decode through stz_decompress_region_noalloc, the entry point for
callers that cannot allocate device memory when they decode (a plug-in handed
only the input and output buffers by its host application, or a path that
must not pay cudaMalloc's device synchronisation).  Its scratch is a fixed
array in the library's device memory instead of a caller workspace.

Its output must equal stz_decompress_region's, bit for bit (the tolerance of
every decode test here), on calls made one after another -- they share that
array -- and a decode that needs more scratch than the array holds must be
refused.  This file is collected last so that a run stopping at the first
failure has run every other test before it.
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


def test_noalloc_region_matches_workspace_region(stzg):
    x = synth.sinusoids((128, 128, 128), synth.seed_for(1))
    xt = torch.from_numpy(x).cuda()
    comp = stzg.compress(xt, 1e-3, "rel").clone()
    meta = stzg.info(comp)
    ws = stzg.alloc_workspace(x.shape, torch.float32)
    out = torch.empty(64 ** 3, dtype=torch.float32, device="cuda")
    # two calls in a row, with different boxes and levels, then the first
    # again: each must equal the workspace path's result
    cases = [((3, 10, 17), (67, 50, 81), 3), ((0, 64, 5), (128, 128, 40), 2),
             ((3, 10, 17), (67, 50, 81), 3)]
    for lo, hi, level in cases:
        want = stzg.decompress_region(comp, lo, hi, level, workspace=ws, meta=meta).cpu().numpy()
        out.fill_(float("nan"))
        got = stzg.decompress_region_noalloc(comp, lo, hi, level, out, meta=meta).cpu().numpy()
        assert got.shape == want.shape, (lo, hi, level)
        assert np.array_equal(_bits(got), _bits(want)), (lo, hi, level)


def test_noalloc_region_f64_and_2d(stzg):
    for x, lo, hi in [(synth.sinusoids((40, 33, 27), 9, dtype=np.float64), (1, 2, 3), (39, 30, 20)),
                      (synth.banded2d((180, 360), 7), (5, 17), (150, 300))]:
        comp = stzg.compress(torch.from_numpy(x).cuda(), 1e-4, "rel").clone()
        out = torch.empty(x.size, dtype=torch.from_numpy(x).dtype, device="cuda")
        for level in (1, 3):
            want = stzg.decompress_region(comp, lo, hi, level).cpu().numpy()
            got = stzg.decompress_region_noalloc(comp, lo, hi, level, out).cpu().numpy()
            assert np.array_equal(_bits(got), _bits(want)), (x.shape, level)


def test_noalloc_refuses_oversized_decode(stzg):
    # a whole 256^3 field at full resolution needs far more than the array
    x = synth.sinusoids((256, 256, 256), 21, n_terms=4)
    comp = stzg.compress(torch.from_numpy(x).cuda(), 1e-3, "rel").clone()
    out = torch.empty(x.size, dtype=torch.float32, device="cuda")
    with pytest.raises(stzg.StzError) as e:
        stzg.decompress_region_noalloc(comp, (0, 0, 0), x.shape, 3, out)
    assert e.value.code == stzg.ERR_CAPACITY
    # a small box of the same field still decodes, and matches
    want = stzg.decompress_region(comp, (100, 90, 80), (140, 150, 120), 3).cpu().numpy()
    got = stzg.decompress_region_noalloc(comp, (100, 90, 80), (140, 150, 120), 3, out)
    assert np.array_equal(_bits(got.cpu().numpy()), _bits(want))
