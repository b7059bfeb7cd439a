import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libfcoo.so")
    # the C ABI tests load libfcoo.so: build it (nvcc cross-compiles without a GPU)
    lib = os.path.join(ROOT, "paper_1705_09905_gb300", "lib", "libfcoo.so")
    if not os.path.exists(lib):
        import __graft_entry__

        __graft_entry__.build()


@pytest.fixture(scope="session")
def oracle():
    import oracle as orc

    orc.build()
    return orc
