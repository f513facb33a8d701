"""Served form: requests decoded in the continuous-batching loop (several in
flight on their own streams, level-1 grids cached per field, no host wait
per request) give, bit for bit, what the same request gives alone through
stz_decompress_region -- and what the oracle gives."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2509_01626_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2509_01626_gb300 import build, serve, stz

    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    xs = [synth.sinusoids((96, 80, 112), synth.seed_for(5, 1)),
          synth.sinusoids((40, 33, 27), 9, dtype=np.float64, noise=0.0),
          synth.banded2d((180, 360), synth.seed_for(5, 2))]
    ebs = [1e-3, 1e-5, 1e-3]
    comps = [stz.compress(torch.from_numpy(x).cuda(), eb, "rel").clone() for x, eb in zip(xs, ebs)]
    return stz, serve, xs, ebs, comps


def _bits(a):
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint64)


def _check(stz, comps, results, ora=None, xs=None, ebs=None):
    for res in results:
        r = res.request
        alone = stz.decompress_region(comps[r.field], r.lo, r.hi, r.level).cpu().numpy()
        got = res.out.cpu().numpy()
        assert res.status == 0
        assert got.shape == alone.shape and np.array_equal(_bits(got), _bits(alone)), r


def test_served_results_equal_alone_realtime(setup, ora):
    stz, serve, xs, ebs, comps = setup
    reqs = serve.poisson_requests([x.shape for x in xs], 120, rate=20000.0, seed=11, emin=4,
                                  emax=64)
    srv = serve.Server(comps, budget_bytes=1 << 30, max_edge=64, max_slots=6)
    assert srv.nslots == 6
    results, wall = srv.run(reqs, keep_outputs=True)
    assert len(results) == len(reqs)
    _check(stz, comps, results)
    # against the oracle on the host copies of the same containers
    hosts = [c.cpu().numpy() for c in comps]
    for res in results[:25]:
        r = res.request
        want = ora.decompress_region(hosts[r.field], r.lo, r.hi, r.level)
        assert np.array_equal(_bits(res.out.cpu().numpy()), _bits(want)), r


def test_served_burst_and_without_level1_cache(setup):
    stz, serve, xs, ebs, comps = setup
    reqs = serve.poisson_requests([x.shape for x in xs], 60, rate=1e6, seed=12, emin=1, emax=96)
    for cache in (True, False):
        srv = serve.Server(comps, budget_bytes=1 << 30, max_edge=96, max_slots=16,
                           cache_level1=cache)
        results, _ = srv.run(reqs, keep_outputs=True, realtime=False)
        assert len(results) == len(reqs)
        _check(stz, comps, results)


def test_serial_path_matches(setup):
    stz, serve, xs, ebs, comps = setup
    reqs = serve.poisson_requests([x.shape for x in xs], 30, rate=50000.0, seed=13, emin=4,
                                  emax=48)
    ws = stz.alloc_workspace((96, 80, 112), torch.float64)
    out = torch.empty(48 ** 3 * 8, dtype=torch.uint8, device="cuda")
    results, _ = serve.serial(comps, reqs, ws, out, keep_outputs=True)
    _check(stz, comps, results)
    st = serve.latency_stats(results, 1.0)
    assert st["requests"] == 30 and st["p99_ms"] >= st["p50_ms"]
