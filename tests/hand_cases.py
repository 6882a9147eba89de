"""The hand-enumerated 4x4x4 cases of tests/golden/hand_4x4x4.json: their volumes, built from the
recipes stored beside them, and their expected joint histograms."""
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_4x4x4.json")
_AXIS = {"x": 2, "y": 1, "z": 0}


def load():
    d = json.load(open(GOLDEN))
    return d["volumes"], d["cases"]


def volume(spec):
    """A 4x4x4 uint8 volume ([z][y][x]) from its recipe."""
    idx = np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij")
    if "ramp" in spec:
        r = spec["ramp"]
        return (r["step"] * idx[_AXIS[r["axis"]]]).astype(np.uint8)
    if "alternate" in spec:
        r = spec["alternate"]
        return np.where(idx[_AXIS[r["axis"]]] % 2 == 1, r["odd"], r["even"]).astype(np.uint8)
    r = spec["points"]
    v = np.full((4, 4, 4), r["base"], dtype=np.uint8)
    for x, y, z, val in r["values"]:
        v[z, y, x] = val
    return v


def bins_of(case):
    return case.get("bins", 4)


def expected_hist(case, dtype=np.uint64):
    b = bins_of(case)
    want = np.zeros((b, b), dtype=dtype)
    for r, c, v in case["hist"]:
        want[r, c] = v
    return want
