"""Bit parity with the oracle on the larger workloads, at their stated sizes:

* the mixed batch: 64 uneven fields (40 3D f32 with dims in [64, 512], 16
  2D f32 1800 x 3600, 8 3D f64 256^3) compressed by one stz_compress_batch
  call -- every container equals the oracle's and every full decode equals
  the oracle's reconstruction;
* the large pair: a 1024^3 f32 k^-5/3 Gaussian random field and a 768^3 f64
  smooth field at relative bound 1e-4 -- the container, the full decode and
  the decode at every progressive level;
* the served form: a resident 1024^3 f32 field at relative bound 1e-3 --
  the container, and 50 requests (box edges 16-256, random level) served by
  the continuous-batching loop, each equal to the oracle's decode of that
  box.

The oracle runs on the host's cores in spawned processes (one field each,
single-threaded as always) while the GPU works; comparisons are by SHA-256
of the raw bytes.  Host memory is checked first so that the oracle runs
never exhaust it.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os
import sys
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)

import oracle_jobs  # noqa: E402

from paper_2509_01626_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

GB = 1 << 30


def mem_available() -> int:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


@pytest.fixture(scope="module")
def stzg():
    from paper_2509_01626_gb300 import build, stz

    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    stz.lib()
    return stz


@pytest.fixture(scope="module")
def workdir():
    with tempfile.TemporaryDirectory(prefix="stz_cfg_") as d:
        yield d


class Pool:
    """Spawned oracle processes.  A job's memory estimate is held while it
    runs: a job is submitted only when the estimates of the jobs in flight
    leave room for it, so the host's memory is never exhausted."""

    def __init__(self):
        self.budget = int(mem_available() * 0.6)
        self.ex = cf.ProcessPoolExecutor(max_workers=max(1, min(14, os.cpu_count() or 1)),
                                         mp_context=mp.get_context("spawn"))

    def submit_all(self, jobs):
        """jobs: list of (job dict, bytes estimate); largest first.  Returns
        the futures in the order of `jobs`."""
        futs = [None] * len(jobs)
        inflight = {}
        for i in sorted(range(len(jobs)), key=lambda k: -jobs[k][1]):
            need = jobs[i][1]
            if need > self.budget:
                self.ex.shutdown(cancel_futures=True)
                pytest.skip(f"host memory too small for an oracle job "
                            f"({need / GB:.1f} GiB > {self.budget / GB:.1f} GiB)")
            while inflight and sum(inflight.values()) + need > self.budget:
                done, _ = cf.wait([futs[k] for k in inflight], return_when=cf.FIRST_COMPLETED)
                for k in [k for k in inflight if futs[k] in done]:
                    del inflight[k]
            futs[i] = self.ex.submit(oracle_jobs.run_job, jobs[i][0])
            inflight[i] = need
        return futs

    def close(self):
        self.ex.shutdown(wait=True, cancel_futures=True)


def _estimate(shape, itemsize):
    n = int(np.prod(shape))
    # field + codes + reconstruction + container + decode (codes, reconstruction)
    return n * (3 * itemsize + 6) + (256 << 20)


def _dump(workdir, name, x: np.ndarray) -> str:
    path = os.path.join(workdir, name + ".raw")
    x.tofile(path)
    return path


def _sha_t(t) -> str:
    return oracle_jobs.sha(t.cpu().numpy())


def test_large_pair_1024_f32_and_768_f64(stzg, workdir):
    """1024^3 f32 k^-5/3 GRF and 768^3 f64 smooth field, rel eb 1e-4: the
    GPU container, full decode and every progressive level equal the
    oracle's (Sec. 3.3: progressive(k) is the full decode at stride
    2^(L-k))."""
    cases = []
    x32 = synth.grf((1024,) * 3, synth.seed_for(4, 0), slope=-5.0 / 3.0, lognormal_sigma=None,
                    dtype=np.float32, device="cuda", white_source="torch", as_tensor=True)
    cases.append(("grf1024_f32", x32))
    x64 = synth.sinusoids_device((768,) * 3, synth.seed_for(4, 1), n_terms=4, fmin=1.0, fmax=3.0,
                                 noise=0.0, dtype=np.float64, device="cuda")
    cases.append(("smooth768_f64", x64))
    jobs = []
    for name, x in cases:
        xh = x.cpu().numpy()
        path = _dump(workdir, name, xh)
        jobs.append(({"path": path, "shape": list(xh.shape), "dtype": str(xh.dtype),
                      "eb": 1e-4, "mode": "rel", "levels": 3, "strides": [2, 4], "boxes": []},
                     _estimate(xh.shape, xh.itemsize)))
        del xh
    pool = Pool()
    futs = pool.submit_all(jobs)
    got = []
    for name, x in cases:
        comp = stzg.compress(x, 1e-4, "rel").clone()
        full = stzg.decompress_full(comp)
        d = {"container": _sha_t(comp), "full": _sha_t(full),
             "strided": {"2": _sha_t(stzg.decompress_progressive(comp, 2)),
                         "4": _sha_t(stzg.decompress_progressive(comp, 1))}}
        del full, comp
        got.append(d)
        torch.cuda.empty_cache()
    names = [name for name, _ in cases]
    del x32, x64, cases
    wants = [f.result() for f in futs]
    pool.close()
    for name, d, want in zip(names, got, wants):
        assert d["container"] == want["container"], name
        assert d["full"] == want["full"], name
        assert d["strided"] == want["strided"], name


def test_mixed_batch_64_fields(stzg, workdir):
    """The 64-field batch in one stz_compress_batch call (graph, 8 lanes):
    every container and every full decode equals the oracle's."""
    from paper_2509_01626_gb300 import stz

    items = synth.batch_workload()
    jobs, gpu = [], []
    sizes_dev = torch.zeros(len(items), dtype=torch.int64, device="cuda")
    fjobs = (stz.FieldJob * len(items))()
    keep = []
    for i, it in enumerate(items):
        x = synth.make_batch_field(it, device="cuda")
        xh = x.cpu().numpy()
        path = _dump(workdir, f"batch{i}", xh)
        jobs.append(({"path": path, "shape": list(xh.shape), "dtype": str(xh.dtype),
                      "eb": it[4], "mode": "rel", "levels": 3, "strides": [], "boxes": []},
                     _estimate(xh.shape, xh.itemsize)))
        shape = tuple(x.shape)
        out = torch.empty(stz.compress_bound(shape, x.dtype), dtype=torch.uint8, device="cuda")
        ws = stz.alloc_workspace(shape, x.dtype, "cuda")
        j = fjobs[i]
        j.field_dev = x.data_ptr()
        for a in range(3):
            j.dims[a] = shape[a] if a < len(shape) else 0
        j.ndim = len(shape)
        j.dtype = stz.F32 if x.dtype == torch.float32 else stz.F64
        j.eb_mode = stz.EB_REL
        j.eb = it[4]
        j.out_dev = out.data_ptr()
        j.out_cap = out.numel()
        j.ws_dev = ws.data_ptr()
        j.ws_bytes = ws.numel()
        keep.append((x, out, ws))
    pool = Pool()
    futs = pool.submit_all(jobs)
    stz.compress_batch(fjobs, sizes_dev, stz.BatchOpts(8, 2, 1))
    torch.cuda.synchronize()
    sizes = sizes_dev.cpu().numpy()
    assert not (sizes < 0).any(), "a batch output was too small"
    for i, (x, out, ws) in enumerate(keep):
        comp = out[: int(sizes[i])]
        gpu.append((_sha_t(comp), _sha_t(stz.decompress_full(comp, workspace=ws))))
    del keep
    torch.cuda.empty_cache()
    wants = [f.result() for f in futs]
    pool.close()
    for i, (want, (c, y)) in enumerate(zip(wants, gpu)):
        assert c == want["container"], (i, items[i][:2])
        assert y == want["full"], (i, items[i][:2])


def test_served_1024_field_matches_oracle(stzg, workdir):
    """A resident 1024^3 f32 field (k^-5/3 GRF, rel eb 1e-3): the container
    equals the oracle's, and 50 requests served by the continuous-batching
    loop each equal the oracle's decode of that box at that level."""
    from paper_2509_01626_gb300 import serve

    shape = (1024,) * 3
    x = synth.grf(shape, synth.seed_for(5, 0), slope=-5.0 / 3.0, lognormal_sigma=None,
                  dtype=np.float32, device="cuda", white_source="torch", as_tensor=True)
    reqs = serve.poisson_requests([shape], 50, 1e4, synth.seed_for(5, 300))
    path = _dump(workdir, "served1024", x.cpu().numpy())
    job = {"path": path, "shape": list(shape), "dtype": "float32", "eb": 1e-3, "mode": "rel",
           "levels": 3, "strides": [],
           "boxes": [(list(r.lo), list(r.hi), r.level) for r in reqs]}
    pool = Pool()
    (fut,) = pool.submit_all([(job, _estimate(shape, 4))])
    comp = stzg.compress(x, 1e-3, "rel").clone()
    del x
    torch.cuda.empty_cache()
    csha = _sha_t(comp)
    srv = serve.Server([comp], budget_bytes=4 * GB, max_edge=256, max_slots=8)
    res, _ = srv.run(reqs, keep_outputs=True, realtime=False)
    by_req = {id(r.request): r for r in res}
    got = [_sha_t(by_req[id(r)].out) for r in reqs]
    want = fut.result()
    pool.close()
    assert csha == want["container"]
    for i, (g, w) in enumerate(zip(got, want["boxes"])):
        assert g == w, (i, reqs[i])
