"""The oracle still writes the committed golden containers byte for byte
(format stability; fixtures written by tests/golden/make_golden.py)."""
import hashlib
import json
import os

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
MANIFEST = json.load(open(os.path.join(HERE, "manifest.json")))


@pytest.mark.parametrize("name", sorted(MANIFEST))
def test_golden_bytes(ora, name):
    c = MANIFEST[name]
    x = np.load(os.path.join(HERE, name + ".npy"))
    assert hashlib.sha256(x.tobytes()).hexdigest() == c["field_sha256"]
    comp = ora.compress(x, c["eb"], c["mode"], nsub=c.get("nsub", 4))
    ref = np.fromfile(os.path.join(HERE, name + ".stz"), dtype=np.uint8)
    assert hashlib.sha256(ref.tobytes()).hexdigest() == c["stz_sha256"]
    assert np.array_equal(comp, ref)
    y = ora.decompress(ref)
    assert np.abs(x.astype(np.float64) - y).max() <= ora.info(ref)["eb_abs"]
