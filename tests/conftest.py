import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def sg():
    """The GPU library (built in-tree); GPU tests only."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2607_08006_gb300.builder import build

    build()
    import paper_2607_08006_gb300 as pkg

    pkg.lib()
    return pkg


@pytest.fixture
def heapf(sg):
    """Factory of initialised heaps; finalises whatever it created."""
    made = []

    def make(npes, H, **kw):
        h = sg.Heap(npes, H, **kw)
        made.append(h)
        return h

    yield make
    for h in made:
        h.close()
