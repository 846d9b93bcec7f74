import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def rel_err(x, r):
    """Normwise relative error max|x - r| / max|r| over all points."""
    x = np.asarray(x, np.float64)
    r = np.asarray(r, np.float64)
    den = np.max(np.abs(r))
    return float(np.max(np.abs(x - r)) / (den if den > 0 else 1.0))


# tolerances on the normwise relative error against the FP64 oracle
TOL = {"f64": 1e-13, "f32": 1e-5}


@pytest.fixture(scope="session")
def liboec():
    """Build (if stale) and load the CUDA library; no GPU is needed to load it."""
    from paper_2005_13014_gb300 import build, _lib
    build.build()
    return _lib.lib()


def has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
