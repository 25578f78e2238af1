import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def tiny8():
    """8^3 model system (box 8 bohr, 4 wells, seed 0) with every eigenpair of the dense H0."""
    import sbse_inputs as si
    p = si.model_system.Preset("tiny8", N=8, box=8.0, n_wells=4, seed=0, n_occ=2, n_o=2, n_c=2)
    v, e, phi = si.dense_eigensystem(p)
    return p, v, e, phi


@pytest.fixture(scope="session")
def tiny16():
    import sbse_inputs as si
    return si.make_system(si.preset("tiny16"))


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
