import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libhq.so")
    config.addinivalue_line("markers", "slow: large sizes; still part of the default run")


@pytest.fixture(scope="session")
def n28_oracle():
    """The 28-qubit subset of the 33-qubit layout (942 gates) simulated by the
    oracle, gate by gate in complex128 (4 GiB, ~80 s on 16 host cores);
    computed once per test session."""
    import oracle
    from paper_2111_06868_gb300 import circuits as C

    circ = C.config_n33(seed=0, first=28)
    return circ, oracle.simulate(circ)
