"""Batched form (stz_compress_batch): every field's container equals the
single-field path's and the oracle's, bit for bit, under every launch
arrangement the autotuner may pick (lanes, SM share, captured graph or plain
launches, the work queue with either level schedule and several tile
granularities and grid sizes); a replayed graph reads the fields' current
contents; a field whose output buffer is too small is reported without
disturbing the others."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2509_01626_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2509_01626_gb300 import batch, build, stz

    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    stz.lib()
    return stz, batch


def small_batch():
    xs = [synth.sinusoids((37, 29, 41), 3),
          synth.sinusoids((64, 64, 64), synth.seed_for(3, 1)),
          synth.sinusoids((5, 3, 200), 4),
          synth.banded2d((180, 360), synth.seed_for(3, 2)),
          synth.banded2d((97, 33), 8),
          synth.sinusoids((40, 33, 27), 9, dtype=np.float64, noise=0.0),
          np.full((20, 20, 20), 3.25, dtype=np.float32),
          synth.sinusoids((1, 1, 1), 5)]
    ebs = [1e-3, 1e-2, 1e-4, 1e-3, 1e-2, 1e-5, 1e-3, 1e-3]
    modes = ["rel", "rel", "abs", "rel", "abs", "rel", "rel", "rel"]
    return xs, ebs, modes


def test_batch_matches_single_and_oracle_under_every_arrangement(mods, ora):
    stz, batch = mods
    xs, ebs, modes = small_batch()
    fields = [torch.from_numpy(x).cuda() for x in xs]
    refs = [ora.compress(x, eb, m) for x, eb, m in zip(xs, ebs, modes)]
    singles = [stz.compress(f, eb, m).cpu().numpy() for f, eb, m in zip(fields, ebs, modes)]
    for r, s in zip(refs, singles):
        assert np.array_equal(r, s)
    bc = batch.BatchCompressor(fields, ebs, modes)
    for lanes, den, graph in [(1, 1, 0), (4, 1, 0), (8, 2, 0), (1, 1, 1), (4, 2, 1), (8, 4, 1),
                              (16, 1, 1)]:
        for o in bc.outs:
            o.fill_(0xA5)
        bc.sizes_dev.fill_(-1)
        bc.run(batch.make_opts(lanes, den, graph))
        got = [c.cpu().numpy() for c in bc.containers()]
        for i, (g, r) in enumerate(zip(got, refs)):
            assert g.size == r.size and np.array_equal(g, r), (lanes, den, graph, i)


def test_graph_replay_reads_current_fields(mods, ora):
    stz, batch = mods
    xs, ebs, modes = small_batch()
    fields = [torch.from_numpy(x).cuda() for x in xs]
    bc = batch.BatchCompressor(fields, ebs, modes)
    o = batch.make_opts(4, 2, 1)
    bc.run(o)
    first = [c.cpu().numpy() for c in bc.containers()]
    # new contents in the same buffers: the cached graph must compress them
    xs2 = [np.ascontiguousarray(x * 1.5 + 0.25).astype(x.dtype) for x in xs]
    for f, x2 in zip(fields, xs2):
        f.copy_(torch.from_numpy(x2))
    bc.run(o)
    second = [c.cpu().numpy() for c in bc.containers()]
    for x2, eb, m, s, f0 in zip(xs2, ebs, modes, second, first):
        assert np.array_equal(s, ora.compress(x2, eb, m))
    assert any(a.size != b.size or not np.array_equal(a, b) for a, b in zip(first, second))


def test_autotune_picks_an_arrangement_and_keeps_bytes(mods, ora):
    stz, batch = mods
    xs, ebs, modes = small_batch()
    fields = [torch.from_numpy(x).cuda() for x in xs]
    bc = batch.BatchCompressor(fields, ebs, modes)
    best = bc.autotune(candidates=[(1, 1, 0), (2, 1, 1), (4, 2, 1)], reps=2)
    assert len(bc.tuning) == 3 and best.lanes in (1, 2, 4)
    bc.run()
    for c, x, eb, m in zip(bc.containers(), xs, ebs, modes):
        assert np.array_equal(c.cpu().numpy(), ora.compress(x, eb, m))
    # the plain per-field loop gives the same sizes
    assert bc.loop() == bc.sizes()


def test_capacity_reported_per_field(mods, ora):
    stz, batch = mods
    xs, ebs, modes = small_batch()
    fields = [torch.from_numpy(x).cuda() for x in xs]
    bc = batch.BatchCompressor(fields, ebs, modes)
    bc.jobs[1].out_cap = 1000  # far below what field 1 needs
    bc.run(batch.make_opts(4, 1, 0))
    v = bc.sizes_dev.cpu().tolist()
    assert v[1] < 0  # bit 63
    need = v[1] & ((1 << 63) - 1)
    assert need == ora.compress(xs[1], ebs[1], modes[1]).size
    for i in (0, 2, 3, 4, 5, 6, 7):
        got = bc.outs[i][: v[i]].cpu().numpy()
        assert np.array_equal(got, ora.compress(xs[i], ebs[i], modes[i])), i


def test_work_queue_matches_oracle_under_every_schedule(mods, ora):
    """The level stages of the 3D fields in one persistent launch per dtype
    over (field, level, tile) items: containers equal the oracle's whatever
    the schedule, tiles per item, blocks per SM, lanes and graph; the 2D and
    tiny fields take the per-field path beside it."""
    stz, batch = mods
    xs, ebs, modes = small_batch()
    xs = xs + [synth.sinusoids((70, 90, 110), synth.seed_for(3, 5)),
               synth.sinusoids((48, 40, 64), 11, dtype=np.float64, noise=0.0)]
    ebs = ebs + [1e-3, 1e-4]
    modes = modes + ["rel", "rel"]
    fields = [torch.from_numpy(x).cuda() for x in xs]
    refs = [ora.compress(x, eb, m) for x, eb, m in zip(xs, ebs, modes)]
    bc = batch.BatchCompressor(fields, ebs, modes)
    assert bc.bws.numel() > 1  # some fields are queued
    for lanes, den, graph, queue in [(1, 1, 0, (0, 1, 0)), (4, 1, 0, (1, 1, 0)),
                                     (4, 2, 1, (0, 4, 0)), (8, 1, 1, (1, 2, 1)),
                                     (16, 4, 1, (0, 64, 2)), (2, 1, 0, (1, 3, 1))]:
        for o in bc.outs:
            o.fill_(0xA5)
        bc.sizes_dev.fill_(-1)
        bc.run(bc.opts_for(lanes, den, graph, queue))
        got = [c.cpu().numpy() for c in bc.containers()]
        for i, (g, r) in enumerate(zip(got, refs)):
            assert g.size == r.size and np.array_equal(g, r), (lanes, den, graph, queue, i)
    # a replayed work-queue graph compresses the fields' current contents
    o = bc.opts_for(4, 1, 1, (0, 2, 0))
    bc.run(o)
    xs2 = [np.ascontiguousarray(x * 0.75 - 1.0).astype(x.dtype) for x in xs]
    for f, x2 in zip(fields, xs2):
        f.copy_(torch.from_numpy(x2))
    bc.run(o)
    for c, x2, eb, m in zip(bc.containers(), xs2, ebs, modes):
        assert np.array_equal(c.cpu().numpy(), ora.compress(x2, eb, m))


def test_work_queue_rejects_missing_workspace(mods):
    stz, batch = mods
    xs, ebs, modes = small_batch()
    fields = [torch.from_numpy(x).cuda() for x in xs]
    bc = batch.BatchCompressor(fields, ebs, modes)
    o = bc.opts_for(4, 1, 0, (0, 1, 0))
    o.ws_bytes = 0
    with pytest.raises(stz.StzError):
        bc.run(o)
    o = bc.opts_for(4, 1, 0, (2, 1, 0))  # no such schedule
    with pytest.raises(stz.StzError):
        bc.run(o)
