"""Served form with batched launches: stz_decode_requests decodes many region
requests with a fixed number of kernel launches (one for all chunk decoding,
one interior and one boundary launch per level, one for all level-1 copies).
Every result must equal, bit for bit, the same request decoded alone by
stz_decompress_region -- and the oracle's decode of that box -- in bursts
and in the real-time continuous-batching loop, for 3D and 2D fields (2D
bricks take the per-request kernels inside the same call), f32 and f64, with
outlier-heavy streams, every level and boxes holding no lattice point.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2509_01626_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2509_01626_gb300 import build, serve, stz

    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return stz, serve


def _bits(a):
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint64)


def _fields_f32(stz):
    xs = [synth.sinusoids((96, 80, 112), synth.seed_for(5, 1)),
          synth.grf((70, 61, 83), synth.seed_for(4, 7), slope=-5.0 / 3.0, lognormal_sigma=None),
          synth.banded2d((180, 360), synth.seed_for(5, 2))]
    ebs = [1e-3, 1e-5, 1e-3]
    comps = [stz.compress(torch.from_numpy(x).cuda(), eb, "rel").clone()
             for x, eb in zip(xs, ebs)]
    return xs, comps


def _check(stz, comps, results, ora=None, hosts=None, n_oracle=0):
    for k, res in enumerate(results):
        r = res.request
        alone = stz.decompress_region(comps[r.field], r.lo, r.hi, r.level).cpu().numpy()
        got = res.out.cpu().numpy()
        assert res.status == 0
        assert got.shape == alone.shape and np.array_equal(_bits(got), _bits(alone)), r
        if k < n_oracle:
            want = ora.decompress_region(hosts[r.field], r.lo, r.hi, r.level)
            assert np.array_equal(_bits(got), _bits(want)), r


def test_batched_burst_and_realtime_f32(mods, ora):
    stz, serve = mods
    xs, comps = _fields_f32(stz)
    hosts = [c.cpu().numpy() for c in comps]
    reqs = serve.poisson_requests([x.shape for x in xs], 150, rate=1e6, seed=21, emin=1,
                                  emax=64)
    srv = serve.BatchServer(comps, budget_bytes=2 << 30, max_edge=64, max_batch=12)
    assert srv.max_batch == 12
    res, _ = srv.run(reqs, keep_outputs=True, realtime=False)
    assert len(res) == len(reqs)
    _check(stz, comps, res, ora, hosts, n_oracle=30)
    reqs = serve.poisson_requests([x.shape for x in xs], 80, rate=20000.0, seed=22, emin=4,
                                  emax=64)
    res, _ = srv.run(reqs, keep_outputs=True)
    assert len(res) == len(reqs)
    _check(stz, comps, res)


def test_batched_f64_fields(mods, ora):
    stz, serve = mods
    xs = [synth.sinusoids((40, 33, 27), 9, dtype=np.float64, noise=0.0),
          synth.sinusoids((64, 48, 56), 10, dtype=np.float64)]
    comps = [stz.compress(torch.from_numpy(x).cuda(), 1e-6, "rel").clone() for x in xs]
    reqs = serve.poisson_requests([x.shape for x in xs], 60, rate=1e6, seed=23, emin=1, emax=40)
    srv = serve.BatchServer(comps, budget_bytes=1 << 30, max_edge=40, max_batch=16)
    res, _ = srv.run(reqs, keep_outputs=True, realtime=False)
    _check(stz, comps, res, ora, [c.cpu().numpy() for c in comps], n_oracle=20)


def test_decode_requests_call_every_level_and_empty_boxes(mods):
    """One stz_decode_requests call over every level, single points, slices,
    and level-1 boxes holding no multiple of 4 (shape with a zero)."""
    stz, serve = mods
    xs, comps = _fields_f32(stz)
    srv = serve.BatchServer(comps, budget_bytes=1 << 30, max_edge=96, max_batch=4)
    boxes = [(0, (0, 0, 0), (96, 80, 112), 1), (0, (5, 6, 7), (6, 7, 8), 3),
             (0, (1, 1, 1), (3, 3, 3), 1), (0, (40, 0, 0), (41, 80, 112), 3),
             (0, (41, 0, 0), (42, 80, 112), 2), (1, (0, 0, 0), (70, 61, 83), 3),
             (1, (3, 10, 20), (60, 11, 83), 2), (2, (17, 0), (18, 360), 3),
             (2, (0, 100), (180, 101), 1), (1, (69, 60, 82), (70, 61, 83), 2)]
    reqs = (stz.RegionRequest * len(boxes))()
    outs = []
    for q, (f, lo, hi, lv) in zip(reqs, boxes):
        q.field = f
        q.level = lv
        for a in range(len(lo)):
            q.lo[a] = lo[a]
            q.hi[a] = hi[a]
        n = int(np.prod([h - l for l, h in zip(lo, hi)]))
        o = torch.full((n,), float("nan"), device="cuda")
        q.out_dev = o.data_ptr()
        q.out_cap = n * 4
        outs.append(o)
    ws = torch.empty(stz.decode_requests_workspace(reqs, srv.farr), dtype=torch.uint8,
                     device="cuda")
    status = torch.full((len(boxes),), 7, dtype=torch.int32, device="cuda")
    stz.decode_requests(reqs, srv.farr, ws, status)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    for q, o, (f, lo, hi, lv) in zip(reqs, outs, boxes):
        nd = len(lo)
        shape = tuple(int(v) for v in q.out_dims[:nd])
        alone = stz.decompress_region(comps[f], lo, hi, lv).cpu().numpy()
        assert shape == alone.shape, (f, lo, hi, lv)
        n = int(np.prod(shape))
        assert np.array_equal(_bits(o[:n].cpu().numpy()).reshape(shape), _bits(alone))
