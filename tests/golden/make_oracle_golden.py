"""Writes tests/golden/oracle_tiny.json: outputs of the FP64 oracle on a few
seeded inputs of the tiny workload (a bake of 12 texel rays, SHADE and
SHADOW queries of 6 points, FPS of 40 points). Calls only oracle/ and the
input generators. The values are a regression record of the oracle, not a
pin: the oracle's pins are the closed forms and brute-force checks of the
tests/test_oracle_*.py files. Rerun (python tests/golden/make_oracle_golden.py)
only with a change of the oracle's arithmetic that names its passage."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2510_07729_gb300 import inputs as I  # noqa: E402


def compute():
    c = I.make_tiny()
    probe_of = np.array([0, 0, 3, 7, 7, 12, 20, 33, 41, 50, 58, 63], np.int32)
    ti = np.array([0, 3, 7, 1, 5, 2, 6, 4, 0, 7, 3, 5], np.int32)
    tj = np.array([0, 4, 2, 7, 1, 6, 3, 5, 7, 0, 2, 4], np.int32)
    rgb, occ, dep, fl = oracle.bake_rays(c["gauss"], c["probe_pos"], c["R"], probe_of, ti, tj)
    maps = I.synthetic_maps(np.random.default_rng(5), 64, 8)
    pts = {k: c[k][:6] for k in ("x", "n", "wo", "albedo", "rough", "metal")}
    args = [pts[k] for k in ("x", "n", "wo", "albedo", "rough", "metal")] + [c["probe_pos"], maps["rgb"],
                                                                           maps["occ"], c["env"], 4, 32]
    shade, idx, _ = oracle.query_shade(*args, mode=oracle.MODE_SHADE)
    shadow, _, _ = oracle.query_shade(*args, mode=oracle.MODE_SHADOW)
    pc = np.random.default_rng(6).uniform(-1, 1, (40, 3)).astype(np.float32)
    fps, _ = oracle.fps(pc, 10)
    return {"bake": {"probe_of": probe_of.tolist(), "ti": ti.tolist(), "tj": tj.tolist(), "rgb": rgb.tolist(),
                     "occ": occ.tolist(), "depth": dep.tolist(), "flags": fl.tolist()},
            "query": {"idx": idx.tolist(), "shade": shade.tolist(), "shadow": shadow.tolist()},
            "fps": fps.tolist()}


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tiny.json")
    with open(out, "w") as f:
        json.dump(compute(), f, indent=1)
    print("wrote", out)
