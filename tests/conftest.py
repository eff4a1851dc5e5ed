import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    # The binding loads liblqt_gb300.so when it is imported, which some test
    # modules do at collection: compile it first if it is missing or stale
    # (nvcc cross-compiles without a GPU; an up-to-date build returns at once).
    from paper_2104_03186_gb300 import build

    build.build()


@pytest.fixture(scope="session")
def orc():
    import oracle

    return oracle.default()


def rel_fro(a, b):
    """||a - b||_F / ||b||_F over the whole stacked array (0 when both are 0)."""
    from paper_2104_03186_gb300.accuracy import rel_fro as _rel_fro

    return _rel_fro(a, b)


@pytest.fixture
def single_tile():
    """Sets the single-tile threshold (lqt_set_single_tile_chunk, default 2)
    for one test and restores it afterwards; yields the setter."""
    from paper_2104_03186_gb300 import lqt

    prev = lqt.lqt_set_single_tile_chunk(2)
    yield lqt.lqt_set_single_tile_chunk
    lqt.lqt_set_single_tile_chunk(prev)
