"""Write the golden containers under tests/golden/ with the CPU oracle only.

Each fixture is a small seeded field (paper_2509_01626_gb300.synth), its
container as produced by oracle.compress, and the SHA-256 of both.  The
tests check that the oracle still writes these exact bytes (format
stability) and the GPU tests decode them.

    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle  # noqa: E402
from paper_2509_01626_gb300 import synth  # noqa: E402

# nsub = 4 sub-chunks per chunk (not the compressors' default of 8): the
# fixtures also check that a decoder reads any count the format allows
CASES = {
    "sin3d_f32_22x19x27": dict(shape=(22, 19, 27), seed=11, dtype="float32", eb=1e-3, mode="rel",
                               nsub=4),
    "sin3d_f64_9x14x10": dict(shape=(9, 14, 10), seed=12, dtype="float64", eb=1e-5, mode="rel",
                              nsub=4),
    "sin2d_f32_37x50": dict(shape=(37, 50), seed=13, dtype="float32", eb=2e-2, mode="abs",
                            nsub=4),
}


def main():
    manifest = {}
    for name, c in CASES.items():
        x = synth.sinusoids(c["shape"], c["seed"], dtype=np.dtype(c["dtype"]).type)
        comp = oracle.compress(x, c["eb"], c["mode"], nsub=c["nsub"])
        np.save(os.path.join(HERE, name + ".npy"), x)
        comp.tofile(os.path.join(HERE, name + ".stz"))
        manifest[name] = dict(c, shape=list(c["shape"]),
                              field_sha256=hashlib.sha256(x.tobytes()).hexdigest(),
                              stz_sha256=hashlib.sha256(comp.tobytes()).hexdigest(),
                              stz_bytes=int(comp.size))
    with open(os.path.join(HERE, "manifest.json"), "w") as f:
        json.dump(manifest, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
