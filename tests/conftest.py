import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size workloads")


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("SGKS_PARITY_LOG")
    if not path:
        return
    import parity_log
    if parity_log.RECORDS:
        with open(path, "w") as f:
            json.dump(parity_log.summary(), f, indent=1)
