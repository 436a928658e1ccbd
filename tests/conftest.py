import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_collection_finish(session):
    """Start the full-size tests' slow oracle solves in spawned processes as
    soon as collection ends, if those GPU tests are selected and a GPU is
    there, so that they run while the other GPU tests do."""
    mods = {item.module for item in session.items
            if item.get_closest_marker("gpu") and hasattr(item.module, "start_background")}
    if not mods:
        return
    import torch
    if not torch.cuda.is_available():
        return
    for m in mods:
        m.start_background()


def unit_links(volume):
    U = np.zeros((volume, 4, 3, 3), dtype=np.complex128)
    U[:] = np.eye(3)
    return U


@pytest.fixture
def rng():
    return np.random.default_rng(1234)
