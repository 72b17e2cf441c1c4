"""Reader of the stored equilibria under tests/golden/ (written by
tests/golden/make_golden.py from the FP64 oracle)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_equilibrium(name="c1_equilibrium.txt"):
    """Return {"p", "t", "x"} (float64 arrays) and the header lines."""
    out, header = {}, []
    with open(os.path.join(GOLDEN, name)) as f:
        lines = f.read().splitlines()
    i = 0
    while i < len(lines):
        line = lines[i]
        if line.startswith("#"):
            header.append(line)
            i += 1
            continue
        key, cnt = line.split()
        cnt = int(cnt)
        out[key] = np.array([float(v) for v in lines[i + 1:i + 1 + cnt]])
        i += 1 + cnt
    out["header"] = header
    return out
