"""Reader of the stored expected values in tests/golden/ (written by
tests/golden/make_golden.py from the oracle alone)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read(name="c1_tiny.txt"):
    exc, elem, evals = [], [], []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tag, *rest = line.split()
            if tag == "x":
                exc.append([int(v) for v in rest])
            elif tag == "e":
                elem.append((int(rest[0]), int(rest[1]), float(rest[2])))
            elif tag == "w":
                evals.append(float(rest[1]))
    return np.array(exc, dtype=np.int64), elem, np.array(evals)
