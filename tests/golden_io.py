"""Reader for the hand-derived fixtures in tests/golden/hand_examples.txt."""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def hand_examples():
    """List of dicts {name, A, lam, vsq} parsed from hand_examples.txt."""
    out, cur = [], None
    with open(os.path.join(GOLDEN, "hand_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if line.startswith("# name:"):
                cur = {"name": line.split(":", 1)[1].strip(), "A": [], "vsq": []}
                out.append(cur)
                continue
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            nums = [float(v) for v in vals]
            if key == "n":
                cur["n"] = int(nums[0])
            elif key == "A":
                cur["A"].append(nums)
            elif key == "lam":
                cur["lam"] = np.array(nums)
            elif key == "vsq":
                cur["vsq"].append(nums)
    for ex in out:
        ex["A"] = np.array(ex["A"])
        ex["vsq"] = np.array(ex["vsq"])
        assert ex["A"].shape == (ex["n"], ex["n"]) and ex["vsq"].shape == (ex["n"], ex["n"])
    return out
