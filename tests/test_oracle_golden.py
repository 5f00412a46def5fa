"""Regression guard: the oracle still reproduces its recorded tiny-workload
sample (written by tests/golden/make_golden.py from oracle/ only)."""
import hashlib
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2609_19190_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_tiny_sample.json")


def test_oracle_matches_recorded_tiny_sample():
    rec = json.load(open(GOLDEN))
    img, mask = synth.tiny(seed=1)
    h = hashlib.sha256()
    h.update(img.tobytes())
    h.update(mask.tobytes())
    if h.hexdigest() != rec["sha256"]:
        pytest.skip("the generator draws different bytes on this platform")
    p = O.make_params(img.shape, disc_mode=O.FBN, bin_count=16, radius=1)
    levels, ng, xmin, xmax = O.discretise(p, img, mask)
    assert (ng, xmin, xmax) == (rec["ng"], rec["xmin"], rec["xmax"])
    maps = O.map_voxels(p, img, levels, ng, np.array(rec["voxels"]), nthreads=1)
    ref = np.array([[np.nan if v is None else v for v in row] for row in rec["values"]])
    assert O.feature_names() == rec["features"]
    np.testing.assert_allclose(maps, ref, rtol=1e-12, atol=1e-12, equal_nan=True)
