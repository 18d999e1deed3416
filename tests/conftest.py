import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running case")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def fig1():
    """Parsed tests/golden/fig1_3x3.txt (the paper's worked 3x3 example)."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", "fig1_3x3.txt")
    z, lst, order, w, A = [], {}, None, None, []
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        tag, *vals = line.split()
        if tag == "z":
            z.append([float(v) for v in vals])
        elif tag == "list":
            lst[int(vals[0])] = int(vals[1])
        elif tag == "order":
            order = [int(v) for v in vals]
        elif tag == "w":
            w = [float(v) for v in vals]
        elif tag == "A":
            row = {}
            for item in vals:
                c, v = item.split(":")
                row[int(c)] = float(v)
            A.append(row)
    Ad = np.zeros((9, 9))
    for i, row in enumerate(A):
        for c, v in row.items():
            Ad[i, c - 1] = v
    return {"z": np.array(z, np.float32), "list": lst, "order": order,
            "w": np.array(w), "A": Ad}
