import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(autouse=True)
def _lattice_guards_intact(request):
    """After every GPU test: no lattice closed during it had a guard byte
    (around its device allocation) overwritten."""
    yield
    if request.node.get_closest_marker("gpu") is None:
        return
    import gc

    import paper_1007_3726_gb300 as P

    gc.collect()  # close the lattices the test left to the garbage collector
    bad = list(P.guard_failures)
    P.guard_failures.clear()
    assert not bad, "guard bytes overwritten around lattices %r" % bad
