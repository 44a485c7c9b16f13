import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")


def read_token_matrix(name):
    """Parse a golden fixture of tokens 0 1 -1 i -i s -s (s = 1/sqrt 2)."""
    import numpy as np

    s = 2.0 ** -0.5
    table = {"0": 0.0, "1": 1.0, "-1": -1.0, "i": 1j, "-i": -1j, "s": s, "-s": -s}
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([table[t] for t in line.split()])
    return np.array(rows, dtype=np.complex128)


def read_named_matrices(name):
    import numpy as np

    s = 2.0 ** -0.5
    table = {"0": 0.0, "1": 1.0, "-1": -1.0, "i": 1j, "-i": -1j, "s": s, "-s": -s}
    out, cur, key = {}, [], None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            toks = line.split()
            if len(toks) == 1 and toks[0] not in table:
                if key is not None:
                    out[key] = np.array(cur, dtype=np.complex128)
                key, cur = toks[0], []
            else:
                cur.append([table[t] for t in toks])
    if key is not None:
        out[key] = np.array(cur, dtype=np.complex128)
    return out
