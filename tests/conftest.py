import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: oracle runs that take tens of seconds")


@pytest.fixture(scope="session")
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")


_RECORDS = []


@pytest.fixture
def record(request):
    """Record a measured value (an error, a condition number) of the running test;
    every record is printed in the terminal summary, so the log states what each
    parity test measured, not only that it passed."""
    def _rec(name, **vals):
        _RECORDS.append((request.node.nodeid, name, vals))
    return _rec


def pytest_terminal_summary(terminalreporter):
    if not _RECORDS:
        return
    terminalreporter.section("measured values")
    for nodeid, name, vals in _RECORDS:
        items = ", ".join("%s=%s" % (k, ("%.3e" % v) if isinstance(v, float) else v) for k, v in vals.items())
        terminalreporter.write_line("%s  %s: %s" % (nodeid.split("::")[-1], name, items))
