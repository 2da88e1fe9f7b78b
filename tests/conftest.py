import os
import sys
import weakref

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.lib()
    return oracle


@pytest.fixture(autouse=True)
def _debug_index_checks(request):
    """With GS_DEBUG=1 (the index-checking library), every Rasterizer a GPU test creates must
    end the test with no failed index check in its device error word."""
    if os.environ.get("GS_DEBUG") != "1" or "gpu" not in request.keywords:
        yield
        return
    from paper_2509_06433_gb300 import api
    made = []
    orig = api.Rasterizer._configure

    def configure(self, cap):
        orig(self, cap)
        made.append(weakref.ref(self))

    api.Rasterizer._configure = configure
    try:
        yield
    finally:
        api.Rasterizer._configure = orig
    for ref in made:
        r = ref()
        if r is not None:
            err = r.status()[1]
            assert not err & 0x8, f"a debug-build index check failed (device error word {err:#x})"
