"""Reader for the small text fixtures under tests/golden/ (values printed in
the paper, each file citing its example)."""
import os

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    out = {"shape": {}}
    with open(os.path.join(HERE, name)) as fh:
        lines = [ln.strip() for ln in fh if ln.strip() and not ln.lstrip().startswith("#")]
    i = 0
    while i < len(lines):
        head = lines[i].split()
        kind, key = head[0], head[1]
        dims = [int(v) for v in head[2:]]
        if kind == "shape":
            out["shape"][key] = tuple(dims)
            i += 1
        elif kind == "matrix":
            rows, cols = dims
            M = np.array([[float(v) for v in lines[i + 1 + r].split()] for r in range(rows)])
            assert M.shape == (rows, cols), (name, key, M.shape)
            out[key] = M
            i += 1 + rows
        elif kind == "vector":
            v = np.array([float(x) for x in lines[i + 1].split()])
            assert v.shape == (dims[0],)
            out[key] = v
            i += 2
        else:
            raise ValueError(f"{name}: unknown record {kind}")
    return out
