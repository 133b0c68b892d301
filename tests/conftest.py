import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


def unit(v):
    import numpy as np
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def rand_cap(rng, c, r, n):
    """n random points within angle r of the unit vector c."""
    import numpy as np
    v = rng.normal(size=(n, 3))
    v -= (v @ c)[:, None] * c
    v /= np.linalg.norm(v, axis=1)[:, None]
    a = r * np.sqrt(rng.random(n))
    return np.cos(a)[:, None] * c + np.sin(a)[:, None] * v
