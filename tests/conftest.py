import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libglcm.so")
    config.addinivalue_line("markers", "slow: full-size case, seconds to minutes")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def gctx():
    """A libglcm context on cuda:0 (private stream, synchronous calls)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_06189_gb300 import build as b
    b.build()
    import paper_1710_06189_gb300 as G
    c = G.Context(0, hbm_budget_bytes=8 << 30)
    yield c
    c.close()


def to_u32(t):
    import numpy as np
    return t.detach().cpu().numpy().view(np.uint32)
