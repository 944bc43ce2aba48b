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


def pytest_terminal_summary(terminalreporter):
    """The achieved agreement of X with the oracle in every FP64 parity check,
    beside the oracle's own spread under a half-ulp perturbation of A."""
    mod = sys.modules.get("test_gpu_parity")
    rec = getattr(mod, "X_RECORD", None) if mod is not None else None
    if not rec:
        return
    terminalreporter.write_sep("-", "X parity: ||X_gpu - X_oracle||_F / ||X_oracle||_F")
    for what, rel, spread, bar in rec:
        terminalreporter.write_line("%-44s achieved %.3e   oracle spread %.3e   bar %.1e" % (what, rel, spread, bar))
