"""Write oracle_tiny_sample.json from the FP64 oracle (calls only oracle/ and
the seeded input generator).  Run from the repository root:

    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2609_19190_gb300 import synth  # noqa: E402


def digest(img, mask):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(img).tobytes())
    h.update(np.ascontiguousarray(mask).tobytes())
    return h.hexdigest()


def main():
    img, mask = synth.tiny(seed=1)
    p = O.make_params(img.shape, disc_mode=O.FBN, bin_count=16, radius=1)
    levels, ng, xmin, xmax = O.discretise(p, img, mask)
    vox = synth.sample_voxels(mask, 24, seed=7)
    maps = O.map_voxels(p, img, levels, ng, vox, nthreads=1)
    rec = {
        "workload": "tiny 32^3 uniform 0..255, ball r=10, FBN 16, r=1, delta=1",
        "sha256": digest(img, mask),
        "ng": ng, "xmin": xmin, "xmax": xmax,
        "voxels": vox.tolist(),
        "features": O.feature_names(),
        "values": [[None if np.isnan(v) else float(v) for v in row] for row in maps],
    }
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tiny_sample.json")
    with open(out, "w") as f:
        json.dump(rec, f, indent=0)
    print(out)


if __name__ == "__main__":
    main()
