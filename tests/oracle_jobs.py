"""Oracle runs on whole workloads, for the parity tests at full size.

Each job reads a field from a raw file, compresses it with the CPU oracle,
decodes the oracle's container in full, and reports SHA-256 digests: of the
container, of the full reconstruction, of strided views of it (progressive
levels: the oracle's pins show progressive(k) equals the full decode at
stride 2^(L-k)) and of requested boxes (region decodes: the oracle's pins
show a region equals the slice of the full decode, Sec. 3.3).  Digests keep
the exchange with the test process small.  Results are cached by the
input's SHA-256 and the job's parameters in ``STZ_ORACLE_CACHE`` when that
directory is set.

Only ``oracle/`` computes here; this module holds no step of the method.

    python tests/oracle_jobs.py FIELD.raw SHAPE DTYPE EB [LEVELS]   # one job, digests as JSON
"""
from __future__ import annotations

import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).view(np.uint8).reshape(-1).data).hexdigest()


def file_sha(path: str) -> str:
    h = hashlib.sha256()
    with open(path, "rb") as f:
        for chunk in iter(lambda: f.read(1 << 24), b""):
            h.update(chunk)
    return h.hexdigest()


def run_job(job: dict) -> dict:
    """job: path, shape, dtype ("float32" / "float64"), eb, mode, levels,
    strides (list of ints), boxes (list of (lo, hi, level)).  Returns the
    digests and the container size."""
    from oracle import oracle as ora

    key = None
    cache = os.environ.get("STZ_ORACLE_CACHE")
    if cache:
        params = {k: job[k] for k in ("shape", "dtype", "eb", "mode", "levels", "strides",
                                       "boxes")}
        key = hashlib.sha256((file_sha(job["path"]) + json.dumps(params, sort_keys=True))
                             .encode()).hexdigest()
        hit = os.path.join(cache, key + ".json")
        if os.path.exists(hit):
            with open(hit) as f:
                return json.load(f)
    ora.build()
    x = np.fromfile(job["path"], dtype=np.dtype(job["dtype"])).reshape(job["shape"])
    comp = ora.compress(x, job["eb"], job["mode"], levels=job["levels"])
    del x
    out = {"container": sha(comp), "container_bytes": int(comp.size)}
    y = ora.decompress(comp)
    out["full"] = sha(y)
    out["strided"] = {}
    for s in job["strides"]:
        sl = tuple(slice(None, None, s) for _ in y.shape)
        out["strided"][str(s)] = sha(y[sl])
    L = job["levels"]
    out["boxes"] = []
    for lo, hi, level in job["boxes"]:
        s = 1 << (L - level)
        sl = tuple(slice(-(-a // s) * s, b, s) for a, b in zip(lo, hi))
        out["boxes"].append(sha(y[sl]))
    if key:
        os.makedirs(cache, exist_ok=True)
        with open(os.path.join(cache, key + ".json"), "w") as f:
            json.dump(out, f)
    return out


if __name__ == "__main__":
    path, shape, dtype, eb = sys.argv[1], sys.argv[2], sys.argv[3], float(sys.argv[4])
    levels = int(sys.argv[5]) if len(sys.argv) > 5 else 3
    job = {"path": path, "shape": [int(v) for v in shape.split("x")], "dtype": dtype, "eb": eb,
           "mode": "rel", "levels": levels, "strides": [], "boxes": []}
    print(json.dumps(run_job(job)))
