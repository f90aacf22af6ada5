import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer oracle runs (still CPU only)")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as o
    o.build()
    return o


@pytest.fixture
def errlog(request):
    """Append measured parity errors as JSON lines to $LBM_ERRLOG (if set)."""
    import json

    path = os.environ.get("LBM_ERRLOG")

    def log(**kw):
        if path:
            with open(path, "a") as fh:
                fh.write(json.dumps(dict(test=request.node.name, **kw), default=float) + "\n")
    return log
